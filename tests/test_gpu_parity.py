"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances (all FP64; the arithmetic is the same up to rounding order):
* covariance entries: (5e-14 + 2e-15 x) relative, x = h / a -- both K_nu
  implementations are within 3e-15 of 25-digit mpmath values and Eq. 2's
  prefactor adds a few ulps; for large x the factor e^-x magnifies the
  rounding of its argument by x (x = 700 gives entries near 1e-300);
* l(theta): 1e-10 relative (the stated FP64 bound);
* Cholesky factor entries and y = L^-1 Z: 1e-9 absolute on O(1) entries for
  matrices of order <= 2,000 whose condition numbers stay below ~1e5;
* cokriging predictions, entry by entry: |dz| <= 1e-8 (max |z| + |z|)
  (Sigma^-1 amplifies rounding by the condition number).
"""
import ctypes
import math

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


def cov_rtol(theta, l1, l2=None):
    """Per-entry relative tolerance of Eq. 2 in Representation I: 5e-14 + 2e-15 h/a."""
    l2 = l1 if l2 is None else l2
    p = len(theta.sigma2)
    h = np.hypot(l1[:, None, 0] - l2[None, :, 0], l1[:, None, 1] - l2[None, :, 1])
    x = np.repeat(np.repeat(h / theta.a, p, axis=0), p, axis=1)
    return 5e-14 + 2e-15 * x


def assert_pred_close(got, ref, tol):
    """Every prediction within tol (max |ref| + |ref|)."""
    err = np.abs(got - ref)
    bound = tol * (np.abs(ref).max() + np.abs(ref))
    assert np.all(err <= bound), "%d of %d off; worst err / bound %.3g" % ((err > bound).sum(), err.size,
                                                                          (err / bound).max())


def assert_cov_close(got, ref, rtol):
    err = np.abs(got - ref)
    bad = err > rtol * np.abs(ref)
    assert not bad.any(), "%d entries off; worst rel %.3e" % (bad.sum(), (err / np.abs(ref))[bad].max())


def o_theta(t: geo.Theta) -> oracle.Theta:
    return oracle.Theta(list(t.sigma2), t.a, list(t.nu), t.beta_matrix())


TH2 = geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5)                 # Fig. 5 theta
TH2G = geo.Theta((1.3, 0.7), 0.05, (0.35, 1.75), -0.4)              # general orders everywhere
TH3 = geo.Theta((1.0, 1.0, 1.0), 0.05, (0.5, 1.0, 1.5), (0.5, 0.3, 0.4))
# p = 4 (the largest p): every K_nu table slot in use, and nu_44 = 3.6 above the tabulated range
TH4 = geo.Theta((1.0, 0.8, 1.2, 0.6), 0.08, (0.4, 0.9, 1.3, 3.6), (0.3, 0.2, 0.1, 0.25, 0.15, 0.35))


# ------------------------------------------------------------------ covgen --

@pytest.mark.parametrize("theta", [TH2, TH2G, TH3, TH4], ids=["fig5", "general", "trivariate", "p4"])
def test_covgen_symmetric_matches_oracle(ctx, theta):
    locs = inputs.jittered_grid(150, 3)
    p = len(theta.sigma2)
    N = p * 150
    out = torch.zeros((N, N), dtype=torch.float64, device="cuda")   # column-major view = out.T
    geo.geo_covgen(ctx, dev(locs), theta, out, ld=N)
    torch.cuda.synchronize()
    got = out.cpu().numpy().T
    ref = oracle.covgen(o_theta(theta), locs)
    assert_cov_close(got, ref, cov_rtol(theta, locs))


@pytest.mark.parametrize("a", [0.002, 0.03, 0.3, 5.0])
def test_covgen_rect_all_ranges(ctx, a):
    # x = h / a spans both K_nu branches (x <= 2 series, x > 2 recurrence)
    theta = geo.Theta((1.0, 2.0), a, (0.3, 2.2), 0.6)
    l1 = inputs.jittered_grid(70, 11)
    l2 = inputs.jittered_grid(45, 12)
    out = torch.zeros((90, 140), dtype=torch.float64, device="cuda")
    geo.geo_covgen(ctx, dev(l1), theta, out, locs2=dev(l2), ld=140)
    torch.cuda.synchronize()
    got = out.cpu().numpy().T
    ref = oracle.covgen(o_theta(theta), l1, l2)
    assert_cov_close(got, ref, cov_rtol(theta, l1, l2))


@pytest.mark.parametrize("nu", [(0.5, 1.0), (0.3, 0.8), (0.05, 0.15), (1.2, 2.7), (2.9, 3.3), (0.6, 3.4)])
def test_covgen_bessel_every_interval(ctx, nu):
    # x = h / a from 1e-4 to 1.1e3: the small-x series (x < 1/4), every
    # Chebyshev interval [2^k, 2^(k+1)), k = -2 .. 9, the cut-off at 1024, and
    # orders above 3 (reference evaluator)
    a = 0.01
    h = np.geomspace(1e-6, 11.0, 701)
    l1 = np.array([[0.25, 0.5]])
    l2 = np.stack([0.25 + h, np.full_like(h, 0.5)], axis=1)
    theta = geo.Theta((1.0, 2.0), a, nu, 0.3)
    out = torch.zeros((2 * len(h), 2), dtype=torch.float64, device="cuda")
    geo.geo_covgen(ctx, dev(l1), theta, out, locs2=dev(l2), ld=2)
    torch.cuda.synchronize()
    got = out.cpu().numpy().T
    ref = oracle.covgen(o_theta(theta), l1, l2)
    x = np.repeat(h / a, 2)[None, :]
    tiny = np.abs(ref) < 1e-280
    assert np.all(np.abs(got[tiny]) < 1e-280)
    rtol = 1e-14 + 1e-15 * x
    err = np.abs(got - ref)
    bad = (err > rtol * np.abs(ref)) & ~tiny
    assert not bad.any(), "%d entries off; worst rel %.3e at x = %s" % (
        bad.sum(), (err / np.abs(ref))[bad].max(), x[bad][:5])


# ------------------------------------------------------------------ loglik --

def _problem(n, theta, seed=1):
    locs = inputs.jittered_grid(n, 100 + seed)
    p = len(theta.sigma2)
    e = inputs.normals(200 + seed, p * n)
    Z = oracle.simulate(o_theta(theta), locs, e)
    return locs, Z


@pytest.mark.parametrize("nb", [64, 128, 960])
def test_loglik_bivariate_n400(ctx, nb):
    w = inputs.WORKLOADS["bivariate-n400"]
    theta = geo.Theta.from_spec(w.theta)
    locs, _ = w.locations()
    Z = oracle.simulate(o_theta(theta), locs, w.white_noise())
    ref = oracle.loglik(o_theta(theta), locs, Z)
    got, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), theta, geo.opts(nb=nb))
    assert got == pytest.approx(ref.loglik, rel=1e-10)


@pytest.mark.parametrize("n,theta", [(1, TH2), (31, TH2), (37, TH3), (100, TH3), (513, TH2G), (37, TH4),
                                     (150, TH4)],
                         ids=["n1", "n31", "n37p3", "n100p3", "n513", "n37p4", "n150p4"])
def test_loglik_ragged_sizes(ctx, n, theta):
    locs, Z = _problem(n, theta, seed=n)
    ref = oracle.loglik(o_theta(theta), locs, Z)
    for nb in (64, 192):
        got, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), theta, geo.opts(nb=nb))
        assert got == pytest.approx(ref.loglik, rel=1e-10), nb


def test_loglik_without_morton(ctx):
    locs, Z = _problem(300, TH2)
    ref = oracle.loglik(o_theta(TH2), locs, Z)
    got, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, geo.opts(nb=128, morton=0))
    assert got == pytest.approx(ref.loglik, rel=1e-10)


def test_factor_matches_oracle_entrywise(ctx):
    n = 600
    locs, Z = _problem(n, TH2, seed=5)
    perm = oracle.morton_order(locs)
    got, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, geo.opts(nb=256), keep=True)
    try:
        gperm = geo.geo_factor_read(fac, 2, 0, n).astype(np.int64)
        assert np.array_equal(gperm, perm)
        sl = locs[perm]
        sz = Z.reshape(n, 2)[perm].reshape(-1)
        r = oracle.loglik(o_theta(TH2), sl, sz, keep_factor=True)
        N = 2 * n
        L = geo.geo_factor_read(fac, 0, 0, N, 0, N)
        np.testing.assert_allclose(L, r.L, rtol=0, atol=1e-9)
        y = geo.geo_factor_read(fac, 1, 0, N)
        np.testing.assert_allclose(y, r.y, rtol=0, atol=1e-9)
        st = geo.geo_factor_stats_get(fac)
        assert st.logdet == pytest.approx(r.logdet, rel=1e-11)
        assert st.quad == pytest.approx(r.quad, rel=1e-10)
        assert st.loglik == got
    finally:
        fac.free()


def test_beta_zero_splits_on_gpu(ctx):
    # beta = 0: l is the sum of the univariate likelihoods (Sec. 4.2).
    theta = geo.Theta((1.0, 0.6), 0.07, (0.5, 1.3), 0.0)
    locs, _ = _problem(200, TH2)
    Z = inputs.normals(77, 400)
    full, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), theta, geo.opts(nb=128))
    parts = 0.0
    for i in range(2):
        th1 = geo.Theta((theta.sigma2[i],), theta.a, (theta.nu[i],), None)
        v, _ = geo.geo_loglik(ctx, dev(locs), dev(Z[i::2].copy()), th1, geo.opts(nb=128))
        parts += v
    assert full == pytest.approx(parts, rel=1e-12)


def test_not_positive_definite_reports_and_recovers(ctx):
    # very smooth, long-range field on a dense grid: numerically singular
    theta = geo.Theta((1.0,), 1.0, (5.0,), None)
    locs = inputs.jittered_grid(900, 9)
    _, info = oracle.cholesky(oracle.covgen(o_theta(theta), locs))
    assert info > 0   # the oracle fails too
    with pytest.raises(geo.GeoError) as ei:
        geo.geo_loglik(ctx, dev(locs), dev(np.zeros(900)), theta, geo.opts(nb=128))
    assert ei.value.code == geo.GEO_ENOTSPD and ei.value.info >= 1
    # the context is still usable
    locs2, Z2 = _problem(50, TH2)
    ref = oracle.loglik(o_theta(TH2), locs2, Z2)
    got, _ = geo.geo_loglik(ctx, dev(locs2), dev(Z2), TH2)
    assert got == pytest.approx(ref.loglik, rel=1e-10)


def test_invalid_theta_rejected(ctx):
    locs, Z = _problem(10, TH2)
    bad = geo.Theta((1.0, 1.0), 0.1, (0.5, 1.0), np.array([[1.0, 1.2], [1.2, 1.0]]))
    with pytest.raises(geo.GeoError) as ei:
        geo.geo_loglik(ctx, dev(locs), dev(Z), bad)
    assert ei.value.code == geo.GEO_EINVAL
    with pytest.raises(geo.GeoError):
        geo.geo_loglik(ctx, dev(locs), dev(Z), geo.Theta((1.0, -1.0), 0.1, (0.5, 1.0), 0.2))


# ----------------------------------------------------------------- predict --

@pytest.mark.parametrize("theta", [TH2, TH3], ids=["bivariate", "trivariate"])
def test_predict_matches_oracle(ctx, theta):
    n, m = 500, 77
    p = len(theta.sigma2)
    allp = inputs.jittered_grid(n + m, 31)
    locs, new = allp[:n], allp[n:]
    Zall = oracle.simulate(o_theta(theta), allp, inputs.normals(32, p * (n + m)))
    Z = Zall[: p * n]
    ref = oracle.predict(o_theta(theta), locs, Z, new)
    _, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), theta, geo.opts(nb=192), keep=True)
    try:
        zhat = torch.zeros(p * m, dtype=torch.float64, device="cuda")
        geo.geo_predict(ctx, fac, dev(new), zhat)
        got = zhat.cpu().numpy()
    finally:
        fac.free()
    assert_pred_close(got, ref, 1e-8)


def test_predict_at_observed_locations_returns_data(ctx):
    locs, Z = _problem(300, TH2, seed=8)
    _, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, geo.opts(nb=128), keep=True)
    try:
        zhat = torch.zeros(6, dtype=torch.float64, device="cuda")
        geo.geo_predict(ctx, fac, dev(locs[[0, 17, 299]]), zhat)
        got = zhat.cpu().numpy()
    finally:
        fac.free()
    np.testing.assert_allclose(got, np.concatenate([Z[0:2], Z[34:36], Z[598:600]]), atol=1e-8)


def test_predict_batch_equals_single_calls_across_forms(ctx):
    """geo_predict_batch over factors of different forms, orders and sizes gives,
    bit for bit, what one geo_predict per factor gives, and matches the oracle."""
    cases = [(TH2, 500, 61, geo.opts(nb=192), 1e-8),
             (TH3, 300, 40, geo.opts(nb=128), 1e-8),
             (TH2G, 700, 0, geo.opts(nb=128, fp64_gemm=1), 1e-8),          # no new locations
             (TH2, 640, 129, geo.opts(nb=128, fp64_gemm=1), 1e-8),
             (TH3, 600, 33, geo.opts(prec=geo.GEO_PREC_TLR, nb=120, tlr_tol=1e-9, tlr_kmax=120), 1e-6)]
    facs, entries, refs = [], [], []
    try:
        for k, (theta, n, m, o, _) in enumerate(cases):
            p = len(theta.sigma2)
            allp = inputs.jittered_grid(n + m, 70 + k)
            locs, new = allp[:n], allp[n:]
            Z = oracle.simulate(o_theta(theta), allp, inputs.normals(80 + k, p * (n + m)))[: p * n]
            refs.append(oracle.predict(o_theta(theta), locs, Z, new) if m else np.zeros(0))
            _, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), theta, o, keep=True)
            facs.append(fac)
            entries.append((fac, dev(new.reshape(m, 2)), torch.full((p * m,), float("nan"), dtype=torch.float64,
                                                                     device="cuda")))
        geo.geo_predict_batch(ctx, entries)
        got = [z.cpu().numpy() for _, _, z in entries]
        for k, (fac, new, z) in enumerate(entries):
            if new.shape[0] == 0:
                continue
            single = torch.full_like(z, float("nan"))
            geo.geo_predict(ctx, fac, new, single)
            assert np.array_equal(got[k], single.cpu().numpy()), "entry %d differs from geo_predict" % k
            assert_pred_close(got[k], refs[k], cases[k][4])
        # a NULL factor in entry 1 is refused by name, before anything runs
        lib, vp = ctx.lib, ctypes.c_void_p
        fa = (vp * 2)(entries[0][0].handle, None)
        la = (vp * 2)(entries[0][1].data_ptr(), entries[1][1].data_ptr())
        ma = (ctypes.c_int * 2)(entries[0][1].shape[0], entries[1][1].shape[0])
        za = (vp * 2)(entries[0][2].data_ptr(), entries[1][2].data_ptr())
        assert lib.geo_predict_batch(ctx.handle, 2, fa, la, ma, za, None) == geo.GEO_EINVAL
        assert b"batch entry 1" in lib.geo_last_error(ctx.handle)
    finally:
        for f in facs:
            f.free()


# ---------------------------------------------------------------- simulate --

def test_simulate_matches_oracle(ctx):
    locs = inputs.jittered_grid(400, 41)
    e = inputs.normals(42, 800)
    ref = oracle.simulate(o_theta(TH2), locs, e)
    out = torch.zeros(800, dtype=torch.float64, device="cuda")
    geo.geo_simulate(ctx, dev(locs), dev(e), TH2, out, geo.opts(nb=128, morton=0))
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-10)


# -------------------------------------------------------------------- MLE ---

def test_mle_steps_match_oracle_nelder_mead(ctx):
    n = 120
    locs, Z = _problem(n, TH2, seed=13)
    start = geo.Theta((0.8, 1.2), 0.12, (0.6, 0.9), 0.3)
    st = geo.geo_mle_init(start, 0.1)
    o = geo.opts(nb=64)
    onm = oracle.NelderMead(oracle.mle_objective(locs, Z, 2),
                            oracle.theta_to_x(o_theta(start)), step=0.1)
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
    assert ll >= -onm.F[-1]   # the simplex improved on its worst vertex


def test_mle_state_checkpoint_resumes_bit_identically(ctx):
    # geo_mle_state is a plain host struct: a copy taken after 4 steps and
    # resumed later follows the same simplex trajectory, bit for bit
    n = 120
    locs, Z = _problem(n, TH2, seed=17)
    start = geo.Theta((0.8, 1.2), 0.12, (0.6, 0.9), 0.3)
    o = geo.opts(nb=64)
    st = geo.geo_mle_init(start, 0.1)
    for _ in range(4):
        geo.geo_mle_step(ctx, st, dev(locs), dev(Z), o)
    saved = bytes(st)                                  # checkpoint (e.g. written to disk)
    for _ in range(5):
        geo.geo_mle_step(ctx, st, dev(locs), dev(Z), o)
    resumed = geo.geo_mle_state.from_buffer_copy(saved)
    for _ in range(5):
        geo.geo_mle_step(ctx, resumed, dev(locs), dev(Z), o)
    assert bytes(resumed) == bytes(st)
    assert resumed.iter == st.iter and resumed.evals == st.evals


def test_predict_and_variance_p4(ctx):
    n, m = 150, 20
    allp = inputs.jittered_grid(n + m, 35)
    locs, new = allp[:n], allp[n:]
    Zall = oracle.simulate(o_theta(TH4), allp, inputs.normals(36, 4 * (n + m)))
    Z = Zall[: 4 * n]
    ref = oracle.predict(o_theta(TH4), locs, Z, new)
    ref_var = oracle.predict_var(o_theta(TH4), locs, new)
    _, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), TH4, geo.opts(nb=128), keep=True)
    try:
        zhat = torch.zeros(4 * m, dtype=torch.float64, device="cuda")
        var = torch.zeros(4 * m, dtype=torch.float64, device="cuda")
        geo.geo_predict(ctx, fac, dev(new), zhat)
        geo.geo_predict_var(ctx, fac, dev(new), var)
        got, got_var = zhat.cpu().numpy(), var.cpu().numpy()
    finally:
        fac.free()
    assert_pred_close(got, ref, 1e-8)
    assert np.all(np.abs(got_var - ref_var) <= 1e-10 + 1e-8 * np.abs(ref_var))
