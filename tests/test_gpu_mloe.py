"""MLOE / MMOM (Eq. 5 - Eq. 8, Algorithm 1) on the device against the oracle.
Bound: per-location LOE and MOM within 1e-9 absolute + 1e-7 relative (they are
ratios of traces that differ in the fourth to eighth digit)."""
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


def _check(ctx, th_t, th_a, n, m, seed, nb=128):
    allp = inputs.jittered_grid(n + m, seed)
    locs, pred = allp[:n], allp[n:]
    ml, mm, loe, mom = geo.geo_mloe_mmom(ctx, dev(locs), dev(pred), th_t, th_a, geo.opts(nb=nb))
    rml, rmm, rloe, rmom = oracle.mloe_mmom(o_theta(th_t), o_theta(th_a), locs, pred)
    assert np.all(np.abs(loe - rloe) <= 1e-9 + 1e-7 * np.abs(rloe)), np.max(np.abs(loe - rloe))
    assert np.all(np.abs(mom - rmom) <= 1e-9 + 1e-7 * np.abs(rmom)), np.max(np.abs(mom - rmom))
    assert ml == pytest.approx(rml, rel=1e-7, abs=1e-9)
    assert mm == pytest.approx(rmm, rel=1e-7, abs=1e-9)
    return ml, mm


TH = geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5)


def test_mloe_mmom_bivariate_misspecified(ctx):
    th_a = geo.Theta((1.2, 0.9), 0.12, (0.45, 1.1), 0.3)
    ml, mm = _check(ctx, TH, th_a, 250, 15, 71)
    assert ml > 0.0   # a misspecified model predicts worse (Eq. 5)


def test_mloe_mmom_zero_at_the_true_parameters(ctx):
    allp = inputs.jittered_grid(230, 72)
    ml, mm, loe, mom = geo.geo_mloe_mmom(ctx, dev(allp[:200]), dev(allp[200:]), TH, TH, geo.opts(nb=64))
    assert abs(ml) < 1e-11 and abs(mm) < 1e-11
    assert np.all(np.abs(loe) < 1e-11) and np.all(np.abs(mom) < 1e-11)


def test_mloe_mmom_trivariate(ctx):
    th_t = geo.Theta((1.0, 1.0, 1.0), 0.1, (0.5, 1.0, 1.5), (0.5, 0.3, 0.4))
    th_a = geo.Theta((0.9, 1.1, 1.0), 0.08, (0.6, 1.0, 1.4), (0.4, 0.3, 0.2))
    _check(ctx, th_t, th_a, 150, 10, 73, nb=128)


@pytest.mark.parametrize("n,m,nb", [(97, 3, 64), (333, 41, 256)])
def test_mloe_mmom_ragged_sizes(ctx, n, m, nb):
    th_a = geo.Theta((1.0, 1.0), 0.07, (0.5, 1.2), 0.6)
    _check(ctx, TH, th_a, n, m, 74 + n, nb=nb)
