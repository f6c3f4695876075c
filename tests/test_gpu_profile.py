"""Profile likelihood (Sec. 4.2) on the device against the CPU FP64 oracle.

sigma^2_ii = n^-1 Z_i' R_ii^-1 Z_i from each variable's own correlation matrix,
then Eq. 1 at the estimate.  Tolerances:
* dense FP64: 1e-10 relative on sigma^2 and l (the stated FP64 bound);
* TLR at tile accuracy 1e-11: 1e-8 relative;
* mixed precision (FP16 x 2 beyond band 4, two refinement sweeps): sigma^2 to
  2e-6 relative (Z_i' R_ii^-1 Z_i comes from the refined solve) and
  |dl| <= 1e-6 N, the mixed form's c N bound with room for the sigma^2 error.
The Nelder-Mead run over (log a, log nu, beta) follows the oracle's simplex
exactly (same vertices after every iteration) and carries each vertex's
sigma^2 estimate."""
import numpy as np
import pytest

import oracle
import paper_2008_07437_gb300 as geo
from paper_2008_07437_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_07437_gb300 import build
    build.build()
    c = geo.geo_create(0)
    yield c
    c.close()


def o_theta(t):
    return oracle.Theta(list(t.sigma2), t.a, list(t.nu), t.beta_matrix())


TH2 = geo.Theta((1.4, 0.6), 0.07, (0.5, 1.3), 0.5)
TH3 = geo.Theta((1.0, 2.0, 0.5), 0.05, (0.5, 1.0, 1.5), (0.5, 0.3, 0.4))
TH_MIX = geo.Theta((1.0, 1.0), 0.1, (0.5, 1.0), 0.7)


def _problem(n, theta, seed):
    p = len(theta.sigma2)
    locs = inputs.jittered_grid(n, 700 + seed)
    Z = oracle.simulate(o_theta(theta), locs, inputs.normals(800 + seed, p * n))
    return locs, Z


@pytest.mark.parametrize("theta,n,nb", [(TH2, 333, 64), (TH3, 250, 96), (TH2, 1000, 128)])
def test_sigma2_hat_and_profile_loglik_match_oracle(ctx, theta, n, nb):
    locs, Z = _problem(n, theta, n)
    ll_ref, s2_ref = oracle.profile_loglik(o_theta(theta), locs, Z)
    o = geo.opts(nb=nb)
    s2 = geo.geo_sigma2_hat(ctx, dev(locs), dev(Z), theta, o)
    np.testing.assert_allclose(s2, s2_ref, rtol=1e-10)
    ll, s2b = geo.geo_loglik_profile(ctx, dev(locs), dev(Z), theta, o)
    np.testing.assert_array_equal(s2b, s2)
    assert ll == pytest.approx(ll_ref, rel=1e-10)


def test_profile_ignores_the_given_variances(ctx):
    locs, Z = _problem(300, TH2, 5)
    o = geo.opts(nb=64)
    other = geo.Theta((9.0, 0.01), TH2.a, TH2.nu, TH2.beta)
    a = geo.geo_loglik_profile(ctx, dev(locs), dev(Z), TH2, o)
    b = geo.geo_loglik_profile(ctx, dev(locs), dev(Z), other, o)
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1], b[1])


def test_profile_tlr_matches_oracle(ctx):
    locs, Z = _problem(1200, TH3, 7)
    ll_ref, s2_ref = oracle.profile_loglik(o_theta(TH3), locs, Z)
    o = geo.opts(prec=geo.GEO_PREC_TLR, nb=240, tlr_tol=1e-11, tlr_kmax=120)
    ll, s2 = geo.geo_loglik_profile(ctx, dev(locs), dev(Z), TH3, o)
    np.testing.assert_allclose(s2, s2_ref, rtol=1e-8)
    assert ll == pytest.approx(ll_ref, rel=1e-8)


def test_profile_mixed_matches_oracle(ctx):
    n = 1000
    locs, Z = _problem(n, TH_MIX, 9)
    ll_ref, s2_ref = oracle.profile_loglik(o_theta(TH_MIX), locs, Z)
    o = geo.opts(prec=geo.GEO_PREC_MIXED, nb=128, band=4, refine_iters=2)
    ll, s2 = geo.geo_loglik_profile(ctx, dev(locs), dev(Z), TH_MIX, o)
    np.testing.assert_allclose(s2, s2_ref, rtol=2e-6)
    assert abs(ll - ll_ref) <= 1e-6 * 2 * n


def test_profile_mle_matches_oracle_nelder_mead(ctx):
    n = 120
    locs, Z = _problem(n, TH2, 13)
    start = geo.Theta((1.0, 1.0), 0.12, (0.6, 0.9), 0.3)
    st = geo.geo_mle_init(start, 0.1, profile=True)
    assert st.q == 4 and st.profile == 1
    onm = oracle.NelderMead(oracle.profile_objective(locs, Z, 2),
                            oracle.profile_theta_to_x(o_theta(start)), step=0.1)
    o = geo.opts(nb=64)
    for it in range(8):
        geo.geo_mle_step(ctx, st, dev(locs), dev(Z), o)
        onm.step()
        gx = np.array([[st.x[v][d] for d in range(st.q)] for v in range(st.q + 1)])
        gf = np.array([st.f[v] for v in range(st.q + 1)])
        assert np.array_equal(gx, np.array(onm.X)), it
        np.testing.assert_allclose(gf, np.array(onm.F), rtol=1e-10)
    assert st.evals == onm.evals
    best, ll = geo.geo_mle_best(st)
    assert ll == pytest.approx(-onm.best[1], rel=1e-10)
    s2_ref = oracle.sigma2_hat(oracle.profile_x_to_theta(onm.best[0], 2), locs, Z)
    np.testing.assert_allclose(best.sigma2, s2_ref, rtol=1e-10)
    for v in range(st.q + 1):   # every vertex carries its own estimate
        th_v = oracle.profile_x_to_theta(np.array(onm.X[v]), 2)
        np.testing.assert_allclose([st.s2[v][i] for i in range(2)], oracle.sigma2_hat(th_v, locs, Z), rtol=1e-10)


def test_profile_rejects_bad_theta(ctx):
    locs, Z = _problem(100, TH2, 3)
    bad = geo.Theta((1.0, 1.0), -0.1, (0.5, 1.0), 0.5)
    with pytest.raises(geo.GeoError):
        geo.geo_loglik_profile(ctx, dev(locs), dev(Z), bad, geo.opts(nb=64))
