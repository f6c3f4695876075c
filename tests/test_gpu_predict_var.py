"""Prediction (cokriging) variances on a kept factor against the oracle:
diag(C(0) - c0' Sigma^-1 c0).  Bound: 1e-10 absolute + 1e-8 relative for dense
factors; 1e-9 absolute + 1e-7 relative for tile-low-rank factors at tile
accuracy 1e-12."""
import numpy as np
import pytest

import oracle
import paper_2008_07437_gb300 as geo
from paper_2008_07437_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_07437_gb300 import build
    build.build()
    c = geo.geo_create(0)
    yield c
    c.close()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def o_theta(t):
    return oracle.Theta(list(t.sigma2), t.a, list(t.nu), t.beta_matrix())


def _var(ctx, th, locs, new, opts):
    p = len(th.sigma2)
    z = torch.zeros(p * len(locs), dtype=torch.float64, device="cuda")
    _, fac = geo.geo_loglik(ctx, dev(locs), z, th, opts, keep=True)
    out = torch.empty(p * len(new), dtype=torch.float64, device="cuda")
    geo.geo_predict_var(ctx, fac, dev(new), out)
    fac.free()
    return out.cpu().numpy()


@pytest.mark.parametrize("th,n,m,nb", [
    (geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5), 400, 30, 128),
    (geo.Theta((1.3, 0.7), 0.05, (0.35, 1.75), -0.4), 333, 17, 256),
    (geo.Theta((1.0, 1.0, 1.0), 0.1, (0.5, 1.0, 1.5), (0.5, 0.3, 0.4)), 150, 12, 128),
])
def test_predict_var_matches_oracle(ctx, th, n, m, nb):
    allp = inputs.jittered_grid(n + m, 81 + n)
    locs, new = allp[:n], allp[n:]
    got = _var(ctx, th, locs, new, geo.opts(nb=nb))
    ref = oracle.predict_var(o_theta(th), locs, new)
    assert np.all(np.abs(got - ref) <= 1e-10 + 1e-8 * np.abs(ref)), np.max(np.abs(got - ref))


def test_predict_var_zero_at_observed_locations(ctx):
    th = geo.Theta((1.0, 2.0), 0.1, (0.5, 1.0), 0.5)
    locs = inputs.jittered_grid(200, 90)
    got = _var(ctx, th, locs, locs[[0, 57, 123, 199]], geo.opts(nb=64))
    assert np.all(np.abs(got) < 1e-9)


@pytest.mark.parametrize("th,n,m,nb", [
    (geo.Theta((1.0, 1.0, 1.0), 0.1, (0.5, 1.0, 1.5), (0.5, 0.3, 0.4)), 200, 15, 120),
    (geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5), 384, 20, 128),
])
def test_predict_var_tile_low_rank_matches_oracle(ctx, th, n, m, nb):
    # tile accuracy 1e-12: a CPU model (tiles truncated by exact SVD at that threshold, solved
    # exactly) moves the variances by 2.4e-15 at the first case, well inside the bound
    allp = inputs.jittered_grid(n + m, 93 + n)
    locs, new = allp[:n], allp[n:]
    got = _var(ctx, th, locs, new, geo.opts(prec=geo.GEO_PREC_TLR, nb=nb, tlr_tol=1e-12, tlr_kmax=nb))
    ref = oracle.predict_var(o_theta(th), locs, new)
    assert np.all(np.abs(got - ref) <= 1e-9 + 1e-7 * np.abs(ref)), np.max(np.abs(got - ref))
    # prediction on the same kind of factor after the variances (the solve's arena is shared)
    z = torch.as_tensor(inputs.normals(95, len(th.sigma2) * n), dtype=torch.float64, device="cuda")
    _, fac = geo.geo_loglik(ctx, dev(locs), z, th, geo.opts(prec=geo.GEO_PREC_TLR, nb=nb, tlr_tol=1e-12,
                                                            tlr_kmax=nb), keep=True)
    out = torch.empty(len(th.sigma2) * m, dtype=torch.float64, device="cuda")
    geo.geo_predict_var(ctx, fac, dev(new), out)
    zhat = torch.empty_like(out)
    geo.geo_predict(ctx, fac, dev(new), zhat)
    fac.free()
    zref = oracle.predict(o_theta(th), locs, z.cpu().numpy(), new)
    assert np.linalg.norm(zhat.cpu().numpy() - zref) <= 1e-7 * np.linalg.norm(zref)
    assert np.all(np.abs(out.cpu().numpy() - ref) <= 1e-9 + 1e-7 * np.abs(ref))
