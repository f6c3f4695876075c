"""FP64 emulated on the BF16 tensor cores (the Ozaki scheme), through the C ABI.

``geo_gemm_f64e`` computes C -= A B' from 7-bit integer digit slices of the
rows of A and B; ``fp64_gemm = 1`` makes every trailing update of the dense
Cholesky factorisation (the GEMM / SYRK tile tasks of Sec. 5.1) use it.

Tolerances:
* integer-valued operands of at most 11 bits are represented exactly by any
  slice count >= 3, so the product must be bit-exact;
* random FP64 operands: |error| <= (k + 1) 2^(1 - 7 S) max|a_r| max|b_c|
  (digit truncation of both operands and the dropped levels) plus the
  rounding of the FP64 additions, 4 u (|C| + sum |a||b|);
* the likelihood of the FP64 form with 8 slices: the FP64 bounds of the
  native path (l 1e-10 relative, L and y entries 1e-9 absolute);
* fewer slices: the digits carry each entry to 2^(-7S) of its row's
  maximum, so the emulated updates act like floating point with unit
  roundoff 2^(-7S) in place of FP64's 2^(-53), up to the per-row (not
  per-entry) scaling, which costs entries at least 2^-6 of their row's
  maximum up to 6 bits.  The likelihood's sensitivity to the rounding of
  the updates is the same for both, so
      |dl_S| / |l| <= 2^(53 - 7 S) 2^6 max(e_64, 2^-53),
  e_64 = |dl| / |l| of the native FP64 path against the oracle on the same
  problem (measured in the test).  At the mixed workload's theta and the
  largest size the oracle finishes in seconds (N = 8,000), 5 slices must
  also meet the 1e-6 target of the reduced forms.  With 8 slices the digit
  error is below the FP64 rounding of the rest of the computation and the
  FP64 bound (1e-10) applies instead.
* the level cut (oz_cut = 1) drops, per output tile, only digit levels below
  the first level every tile drops, measured against the update's largest
  rows: each entry's error stays within the same absolute bound, so the
  same tolerances apply with and without it.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import paper_2008_07437_gb300 as geo
from paper_2008_07437_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def colmajor(a):
    """A float64 CUDA tensor of shape a.shape stored column-major."""
    return torch.as_tensor(np.ascontiguousarray(np.asarray(a).T), dtype=torch.float64, device="cuda").t()


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_07437_gb300 import build
    build.build()
    c = geo.geo_create(0)
    yield c
    c.close()


def o_theta(t: geo.Theta) -> oracle.Theta:
    return oracle.Theta(list(t.sigma2), t.a, list(t.nu), t.beta_matrix())


TH2 = geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5)
TH2G = geo.Theta((1.3, 0.7), 0.05, (0.35, 1.75), -0.4)
TH3 = geo.Theta((1.0, 1.0, 1.0), 0.05, (0.5, 1.0, 1.5), (0.5, 0.3, 0.4))
TH4 = geo.Theta((1.0, 0.8, 1.2, 0.6), 0.08, (0.4, 0.9, 1.3, 3.6), (0.3, 0.2, 0.1, 0.25, 0.15, 0.35))


def emu(nb=128, slices=8, **kw):
    return geo.opts(nb=nb, fp64_gemm=1, oz_slices=slices, **kw)


# ------------------------------------------------------------- the product --

@pytest.mark.parametrize("S", [3, 4, 5, 6, 7, 8])
def test_gemm_integer_operands_exact(ctx, S):
    # m, n, k ragged against the 128 x 64 tiles and the 32-deep chunks; k = 700
    # exceeds 4096 / S for S >= 6, so those runs also take two launches
    rng = np.random.default_rng(10 + S)
    m, n, k = 300, 201, 700
    A = rng.integers(-1000, 1001, size=(m, k)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(n, k)).astype(np.float64)
    A[7] = rng.integers(-5, 6, size=k)          # a row with a small exponent
    B[3] = 0.0                                   # a zero row
    C = rng.integers(-10 ** 6, 10 ** 6, size=(m, n)).astype(np.float64)
    ref = C.astype(np.int64) - A.astype(np.int64) @ B.astype(np.int64).T
    Ct = colmajor(C)
    geo.geo_gemm_f64e(ctx, colmajor(A), colmajor(B), Ct, slices=S)
    got = Ct.cpu().numpy()
    assert np.array_equal(got, ref.astype(np.float64))


@pytest.mark.parametrize("S", [4, 6, 8])
def test_gemm_random_fp64_within_bound(ctx, S):
    rng = np.random.default_rng(20 + S)
    m, n, k = 257, 130, 1000
    A = rng.standard_normal((m, k)) * np.exp(rng.uniform(-3, 3, size=(m, 1)))
    B = rng.standard_normal((n, k)) * np.exp(rng.uniform(-3, 3, size=(n, 1)))
    C = rng.standard_normal((m, n))
    ref = C - A @ B.T
    Ct = colmajor(C)
    geo.geo_gemm_f64e(ctx, colmajor(A), colmajor(B), Ct, slices=S)
    got = Ct.cpu().numpy()
    amax = np.abs(A).max(axis=1)[:, None]
    bmax = np.abs(B).max(axis=1)[None, :]
    bound = (k + 1) * 2.0 ** (1 - 7 * S) * amax * bmax + 4 * U * (np.abs(C) + np.abs(A) @ np.abs(B).T)
    err = np.abs(got - ref)
    assert np.all(err <= bound), "worst err / bound %.3g" % (err / bound).max()
    if S == 8:   # FP64-class: within a few roundings of the FP64 product
        assert np.all(err <= 8 * U * (np.abs(C) + np.abs(A) @ np.abs(B).T))


def _digits_model(x_digits, S, K, scale):
    """The kept levels t + u <= S + 1 of sum_k a_k b_k for rows whose digits are all x_digits:
    2^(2e) K sum_{t+u<=S+1} d_t d_u 2^(2 - 7(t + u)), exactly."""
    tot = Fraction(0)
    for t in range(1, S + 1):
        for u in range(1, S + 1):
            if t + u <= S + 1:
                tot += Fraction(x_digits[t - 1] * x_digits[u - 1]) * Fraction(2) ** (2 - 7 * (t + u))
    return tot * K * Fraction(scale) ** 2


def test_gemm_accumulation_near_the_exactness_bound(ctx):
    # every digit 63 and depth k = 4096 / S: level S + 1 sums S * 63^2 * k =
    # 16,003,008 (95 % of 2^24) in the FP32 tensor-memory accumulator; the
    # result must equal the exact sum of the kept levels
    S = 7
    k = (4096 // S) // 32 * 32          # 576, one launch
    digits = [63] * S
    xval = sum(Fraction(63) * Fraction(2) ** (1 - 7 * t) for t in range(1, S + 1))   # 48 bits: exact in FP64
    assert float(xval) == xval
    m, n = 130, 70
    scales = [2.0 ** e for e in (-3, 0, 5)]
    A = np.empty((m, k))
    B = np.empty((n, k))
    for r in range(m):
        A[r] = float(xval) * scales[r % 3]
    for c in range(n):
        B[c] = float(xval) * scales[c % 3]
    Ct = colmajor(np.zeros((m, n)))
    geo.geo_gemm_f64e(ctx, colmajor(A), colmajor(B), Ct, slices=S)
    got = Ct.cpu().numpy()
    for r in (0, 1, 2, 64, 129):
        for c in (0, 1, 2, 63, 69):
            exact = -_digits_model(digits, S, k, 1) * Fraction(scales[r % 3]) * Fraction(scales[c % 3])
            assert abs(Fraction(got[r, c]) - exact) <= abs(exact) * Fraction(2) ** -52, (r, c)


def test_gemm_rejects_bad_arguments(ctx):
    A = colmajor(np.ones((4, 3)))
    with pytest.raises(geo.GeoError) as ei:
        geo.geo_gemm_f64e(ctx, A, A, colmajor(np.zeros((4, 4))), slices=9)
    assert ei.value.code == geo.GEO_EINVAL
    with pytest.raises(ValueError):
        geo.geo_gemm_f64e(ctx, A, A, colmajor(np.zeros((4, 5))))


# ----------------------------------------------------- the FP64 likelihood --

def _problem(n, theta, seed=1):
    locs = inputs.jittered_grid(n, 100 + seed)
    p = len(theta.sigma2)
    Z = oracle.simulate(o_theta(theta), locs, inputs.normals(200 + seed, p * n))
    return locs, Z


@pytest.mark.parametrize("n,theta", [(1, TH2), (100, TH2), (37, TH3), (333, TH3), (513, TH2G), (150, TH4)],
                         ids=["n1", "n100", "n37p3", "n333p3", "n513", "n150p4"])
def test_loglik_emulated_matches_oracle(ctx, n, theta):
    locs, Z = _problem(n, theta, seed=n)
    ref = oracle.loglik(o_theta(theta), locs, Z)
    for nb in (64, 192):
        got, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), theta, emu(nb))
        assert got == pytest.approx(ref.loglik, rel=1e-10), nb


def test_loglik_emulated_workload_theta_n400(ctx):
    w = inputs.WORKLOADS["bivariate-n400"]
    theta = geo.Theta.from_spec(w.theta)
    locs, _ = w.locations()
    Z = oracle.simulate(o_theta(theta), locs, w.white_noise())
    ref = oracle.loglik(o_theta(theta), locs, Z)
    for nb in (128, 512):
        got, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), theta, emu(nb))
        assert got == pytest.approx(ref.loglik, rel=1e-10)


def test_factor_emulated_entrywise(ctx):
    n = 700
    locs, Z = _problem(n, TH2, seed=5)
    perm = oracle.morton_order(locs)
    got, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, emu(128), keep=True)
    try:
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
    finally:
        fac.free()


def _derived_bound(S, e64):
    if S >= 8:
        return 1e-10
    return 2.0 ** (53 - 7 * S) * 2.0 ** 6 * max(e64, 2.0 ** -53)


def test_loglik_fewer_slices_within_derived_bound(ctx):
    n = 1000
    locs, Z = _problem(n, TH2, seed=9)
    ref = oracle.loglik(o_theta(TH2), locs, Z).loglik
    nat, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, geo.opts(nb=128))
    e64 = abs(nat - ref) / abs(ref)
    for S in (4, 5, 6, 7, 8):
        got, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, emu(128, slices=S))
        rel = abs(got - ref) / abs(ref)
        print("N = %d, S = %d: |dl| / |l| = %.3e (bound %.3e, FP64 %.3e)" % (2 * n, S, rel, _derived_bound(S, e64), e64))
        assert rel <= _derived_bound(S, e64), S


def test_reduced_form_at_the_largest_oracle_size(ctx):
    # the mixed workload's theta (a = 0.1, nu = (0.5, 1), beta = 0.7) at N = 8,000
    th = geo.Theta((1.0, 1.0), 0.1, (0.5, 1.0), 0.7)
    n = 4000
    locs = inputs.jittered_grid(n, 1002)
    Z = oracle.simulate(o_theta(th), locs, inputs.normals(2002, 2 * n))
    ref = oracle.loglik(o_theta(th), locs, Z).loglik
    nat, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), th, geo.opts(nb=512))
    e64 = abs(nat - ref) / abs(ref)
    for S, nb, cut in ((4, 1024, 0), (5, 768, 0), (5, 768, 1), (8, 512, 0), (8, 512, 1)):
        got, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), th, emu(nb, slices=S, oz_cut=cut))
        rel = abs(got - ref) / abs(ref)
        print("N = %d, S = %d, cut %d: |dl| / |l| = %.3e (bound %.3e, FP64 %.3e)"
              % (2 * n, S, cut, rel, _derived_bound(S, e64), e64))
        assert rel <= _derived_bound(S, e64), (S, cut)
        if S >= 5:
            assert rel <= 1e-6


# ---------------------------------------------------------- the level cut --

@pytest.mark.parametrize("n,theta", [(1, TH2), (333, TH3), (513, TH2G), (150, TH4)],
                         ids=["n1", "n333p3", "n513", "n150p4"])
def test_level_cut_loglik_matches_oracle(ctx, n, theta):
    locs, Z = _problem(n, theta, seed=n)
    ref = oracle.loglik(o_theta(theta), locs, Z)
    for nb in (64, 192):
        got, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), theta, emu(nb, oz_cut=1))
        assert got == pytest.approx(ref.loglik, rel=1e-10), nb


def test_level_cut_factor_entrywise(ctx):
    # a short range: the far tiles' entries are small, so the cut drops levels and whole tiles
    th = geo.Theta((1.0, 1.0), 0.02, (0.5, 1.0), 0.5)
    n = 1500
    locs, Z = _problem(n, th, seed=15)
    perm = oracle.morton_order(locs)
    got, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), th, emu(128, oz_cut=1), keep=True)
    try:
        r = oracle.loglik(o_theta(th), locs[perm], Z.reshape(n, 2)[perm].reshape(-1), keep_factor=True)
        N = 2 * n
        L = geo.geo_factor_read(fac, 0, 0, N, 0, N)
        np.testing.assert_allclose(L, r.L, rtol=0, atol=1e-9)
        np.testing.assert_allclose(geo.geo_factor_read(fac, 1, 0, N), r.y, rtol=0, atol=1e-9)
        assert got == pytest.approx(r.loglik, rel=1e-10)
    finally:
        fac.free()


def _tensor_flops(ctx, locs, Z, theta, o):
    geo.geo_profile_enable(ctx, True)
    ll, _ = geo.geo_loglik(ctx, locs, Z, theta, o)
    prof = geo.geo_profile_read(ctx)
    geo.geo_profile_enable(ctx, False)
    return ll, prof["tcgemm"]["tensor_flops"]


def test_level_cut_saves_tensor_work_within_the_bounds(ctx):
    # N = 8,000 at a short range (a = 0.03): the cut must remove tensor-core work and keep the
    # FP64 bound with 8 slices and the derived bound with 5
    th = geo.Theta((1.0, 1.0), 0.03, (0.5, 1.5), 0.5)
    n = 4000
    locs = inputs.jittered_grid(n, 1001)
    Z = oracle.simulate(o_theta(th), locs, inputs.normals(2001, 2 * n))
    ref = oracle.loglik(o_theta(th), locs, Z).loglik
    dl, dz = dev(locs), dev(Z)
    nat, _ = geo.geo_loglik(ctx, dl, dz, th, geo.opts(nb=512))
    e64 = abs(nat - ref) / abs(ref)
    for S, nb in ((8, 512), (5, 768)):
        full, tf_full = _tensor_flops(ctx, dl, dz, th, emu(nb, slices=S))
        cut, tf_cut = _tensor_flops(ctx, dl, dz, th, emu(nb, slices=S, oz_cut=1))
        again, tf_again = _tensor_flops(ctx, dl, dz, th, emu(nb, slices=S, oz_cut=1))
        print("S = %d: tensor work with the cut %.3f of the full; |dl| / |l| %.2e (cut) %.2e (full)"
              % (S, tf_cut / tf_full, abs(cut - ref) / abs(ref), abs(full - ref) / abs(ref)))
        assert tf_full > 0 and tf_cut < 0.9 * tf_full
        assert again == cut and tf_again == tf_cut   # deterministic
        assert abs(cut - ref) / abs(ref) <= _derived_bound(S, e64), S


def test_level_cut_rejects_bad_values(ctx):
    locs, Z = _problem(100, TH2)
    with pytest.raises(geo.GeoError):
        geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, emu(128, oz_cut=2))


def test_predict_emulated_entrywise(ctx):
    n, m = 500, 77
    p = 2
    allp = inputs.jittered_grid(n + m, 31)
    locs, new = allp[:n], allp[n:]
    Z = oracle.simulate(o_theta(TH2), allp, inputs.normals(32, p * (n + m)))[: p * n]
    ref = oracle.predict(o_theta(TH2), locs, Z, new)
    _, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, emu(192), keep=True)
    try:
        zhat = torch.zeros(p * m, dtype=torch.float64, device="cuda")
        geo.geo_predict(ctx, fac, dev(new), zhat)
        got = zhat.cpu().numpy()
    finally:
        fac.free()
    assert np.all(np.abs(got - ref) <= 1e-9 + 1e-8 * np.abs(ref))


def test_simulate_emulated_matches_oracle(ctx):
    locs = inputs.jittered_grid(400, 41)
    e = inputs.normals(42, 800)
    ref = oracle.simulate(o_theta(TH2), locs, e)
    out = torch.zeros(800, dtype=torch.float64, device="cuda")
    geo.geo_simulate(ctx, dev(locs), dev(e), TH2, out, emu(128, morton=0))
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-10)


def test_emulated_updates_run_on_the_tensor_cores(ctx):
    locs, Z = _problem(600, TH2, seed=3)
    geo.geo_profile_enable(ctx, True)
    geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, emu(128))
    prof = geo.geo_profile_read(ctx)
    geo.geo_profile_enable(ctx, False)
    assert prof["tcgemm"]["launches"] > 0
    # native FP64 updates remain only inside the panels (rank-64 steps of the TRSM)
    assert prof["gemm"]["flops"] < 0.25 * prof["tcgemm"]["flops"]


def test_emulated_not_positive_definite_reports_and_recovers(ctx):
    theta = geo.Theta((1.0,), 1.0, (5.0,), None)
    locs = inputs.jittered_grid(900, 9)
    with pytest.raises(geo.GeoError) as ei:
        geo.geo_loglik(ctx, dev(locs), dev(np.zeros(900)), theta, emu(128))
    assert ei.value.code == geo.GEO_ENOTSPD and ei.value.info >= 1
    locs2, Z2 = _problem(300, TH2)
    ref = oracle.loglik(o_theta(TH2), locs2, Z2)
    got, _ = geo.geo_loglik(ctx, dev(locs2), dev(Z2), TH2, emu(128))
    assert got == pytest.approx(ref.loglik, rel=1e-10)


def test_mloe_mmom_level_cut_equals_native(ctx):
    # a short range at N = 4,000: the cut drops levels of the far tiles in both factorisations; the
    # m cross-covariance rows ride along as right-hand-side rows and keep every level
    n, m = 2000, 30
    allp = inputs.jittered_grid(n + m, 67)
    locs, pred = allp[:n], allp[n:]
    tht = geo.Theta((1.0, 1.0), 0.03, (0.5, 1.5), 0.5)
    tha = geo.Theta((1.1, 0.9), 0.036, (0.45, 1.35), 0.4)
    a = geo.geo_mloe_mmom(ctx, dev(locs), dev(pred), tht, tha, geo.opts(nb=256))
    b = geo.geo_mloe_mmom(ctx, dev(locs), dev(pred), tht, tha, emu(256, oz_cut=1))
    assert b[0] == pytest.approx(a[0], rel=1e-9, abs=1e-13)
    assert b[1] == pytest.approx(a[1], rel=1e-9, abs=1e-13)
    np.testing.assert_allclose(b[2], a[2], rtol=1e-8, atol=1e-12)


def test_mloe_mmom_emulated_equals_native(ctx):
    n, m = 300, 20
    allp = inputs.jittered_grid(n + m, 61)
    locs, pred = allp[:n], allp[n:]
    tha = geo.Theta((1.1, 0.9), 0.11, (0.45, 1.1), 0.4)
    a = geo.geo_mloe_mmom(ctx, dev(locs), dev(pred), TH2, tha, geo.opts(nb=128))
    b = geo.geo_mloe_mmom(ctx, dev(locs), dev(pred), TH2, tha, emu(128))
    assert b[0] == pytest.approx(a[0], rel=1e-9, abs=1e-13)
    assert b[1] == pytest.approx(a[1], rel=1e-9, abs=1e-13)
    np.testing.assert_allclose(b[2], a[2], rtol=1e-8, atol=1e-12)
