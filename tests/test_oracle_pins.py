"""Pins for the CPU oracle: each test ties the oracle to something other than
itself -- closed forms, numbers the paper prints, invariants the paper states,
library routines for special cases, or brute force on tiny inputs -- so that a
dropped term, a wrong sign or index, or a transposed operand fails here."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2008_07437_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.json")


# ---------------------------------------------------------------- K_nu -----

@pytest.mark.parametrize("x", [1e-3, 0.01, 0.1, 0.5, 1.0, 1.9, 2.0, 2.1, 5.0, 13.0, 40.0, 120.0, 600.0])
def test_besselk_half_integer_closed_forms(x):
    # K_{1/2}(x) = sqrt(pi/(2x)) e^-x, K_{3/2} = K_{1/2}(1 + 1/x), K_{5/2} = K_{1/2}(1 + 3/x + 3/x^2)
    base = math.sqrt(math.pi / (2 * x))
    exact = {0.5: base, 1.5: base * (1 + 1 / x), 2.5: base * (1 + 3 / x + 3 / x ** 2)}
    for nu, val in exact.items():
        got = oracle.besselk_scaled(nu, x)
        assert got == pytest.approx(val, rel=2e-15), (nu, x)


@pytest.mark.parametrize("nu", [0.1, 0.25, 0.75, 1.0, 1.25, 2.2])
@pytest.mark.parametrize("x", [0.002, 0.3, 1.0, 3.0, 17.0, 80.0])
def test_besselk_recurrence(nu, x):
    # K_{nu+1}(x) = K_{nu-1}(x) + (2 nu / x) K_nu(x)
    lhs = oracle.besselk_scaled(nu + 1, x)
    rhs = oracle.besselk_scaled(abs(nu - 1), x) + 2 * nu / x * oracle.besselk_scaled(nu, x)
    assert lhs == pytest.approx(rhs, rel=3e-15)


@pytest.mark.parametrize("nu", [0.0, 0.25, 0.75, 1.0, 1.25, 1.75, 2.2, 3.0])
def test_besselk_matches_scipy(nu):
    special = pytest.importorskip("scipy.special")
    for x in np.geomspace(1e-3, 500.0, 61):
        ref = special.kve(nu, x)
        # scipy's kve itself is only good to ~1e-13 near x = 2
        assert oracle.besselk_scaled(nu, float(x)) == pytest.approx(ref, rel=2e-13), (nu, x)


@pytest.mark.parametrize("nu", [0.05, 0.25, 0.6, 0.75, 1.0, 1.25, 2.2])
def test_besselk_matches_mpmath(nu):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 25
    for x in np.concatenate([np.geomspace(1e-4, 2, 15), np.geomspace(2.01, 600, 25)]):
        ref = float(mp.besselk(nu, float(x)) * mp.exp(float(x)))
        assert oracle.besselk_scaled(nu, float(x)) == pytest.approx(ref, rel=3e-15), (nu, x)


def test_besselk_small_x_limit():
    # K_nu(x) ~ Gamma(nu)/2 (2/x)^nu as x -> 0 (nu > 0)
    for nu in (0.5, 1.0, 1.5):
        x = 1e-7
        assert oracle.besselk(nu, x) == pytest.approx(0.5 * math.gamma(nu) * (2 / x) ** nu, rel=1e-5)


# ------------------------------------------------------------- Eq. 2 -------

def test_printed_effective_range():
    g = json.load(open(GOLDEN))["effective_range"]
    for case in g["cases"]:
        _, nuij = oracle.matern_params([case["nu"]], np.eye(1))
        c = oracle.matern(case["h"], g["a"], float(nuij[0, 0]), g["sigma2"])
        assert abs(c - case["cov"]) < g["printed_digits_tol"], (case, c)


def test_printed_effective_range_vs_a():
    # The printed ER lies between the nu = 0.5 and nu = 1 distances where the
    # marginal covariance reaches 0.05 (the two marginals of the paper's fields).
    g = json.load(open(GOLDEN))["effective_range_vs_a"]
    from scipy.optimize import brentq
    for a, er in zip(g["a"], g["er"]):
        lo = brentq(lambda h: oracle.matern(h, a, 0.5, 1.0) - 0.05, 1e-6, 10)
        hi = brentq(lambda h: oracle.matern(h, a, 1.0, 1.0) - 0.05, 1e-6, 10)
        assert lo < er < hi * 1.01, (a, er, lo, hi)


@pytest.mark.parametrize("h", [1e-4, 0.01, 0.07, 0.3, 1.2])
def test_matern_half_integer_closed_forms(h):
    a, s2 = 0.09, 1.7
    x = h / a
    assert oracle.matern(h, a, 0.5, s2) == pytest.approx(s2 * math.exp(-x), rel=1e-14)
    assert oracle.matern(h, a, 1.5, s2) == pytest.approx(s2 * (1 + x) * math.exp(-x), rel=1e-14)


def test_matern_zero_distance_limit():
    for nu in (0.5, 0.8, 1.0, 1.5):
        assert oracle.matern(0.0, 0.1, nu, 2.5) == 2.5
        assert oracle.matern(1e-9, 0.1, nu, 2.5) == pytest.approx(2.5, rel=1e-6)


def test_rho_closed_form_d2():
    # d = 2: Gamma(nu + 1) = nu Gamma(nu) turns rho_ij into beta_ij sqrt(nu_i nu_j) / nu_ij
    nu = [0.5, 1.0, 1.5]
    beta = np.array([[1, 0.5, 0.3], [0.5, 1, 0.4], [0.3, 0.4, 1.0]])
    rho, nuij = oracle.matern_params(nu, beta, d=2)
    for i in range(3):
        assert rho[i, i] == pytest.approx(1.0, rel=1e-15)
        for j in range(3):
            nij = 0.5 * (nu[i] + nu[j])
            assert nuij[i, j] == nij
            if i != j:
                assert rho[i, j] == pytest.approx(beta[i, j] * math.sqrt(nu[i] * nu[j]) / nij, rel=1e-14)
    # Fig. 5 theta: rho_12 = 0.5 sqrt(0.5) / 0.75
    rho, _ = oracle.matern_params([0.5, 1.0], np.array([[1, 0.5], [0.5, 1]]))
    assert rho[0, 1] == pytest.approx(0.5 * math.sqrt(0.5) / 0.75, rel=1e-14)


def test_rho_d1_closed_form():
    # d = 1, nu_i = nu_j = nu: rho = beta * Gamma(nu+1/2)/Gamma(nu) * Gamma(nu)/Gamma(nu+1/2) = beta
    rho, _ = oracle.matern_params([0.7, 0.7], np.array([[1, 0.3], [0.3, 1]]), d=1)
    assert rho[0, 1] == pytest.approx(0.3, rel=1e-14)


# ------------------------------------------------------------- Sigma -------

def _small_problem(n=40, seed=7, theta=None):
    th = theta or oracle.Theta([1.0, 1.3], 0.09, [0.5, 1.0], 0.5)
    locs = inputs.jittered_grid(n, seed)
    return th, locs


def test_sigma_structure():
    th, locs = _small_problem(30)
    S = oracle.covgen(th, locs)
    p = 2
    assert np.array_equal(S, S.T)
    rho, _ = oracle.matern_params(th.nu, th.beta)
    for l in range(30):
        blk = S[p * l:p * l + p, p * l:p * l + p]
        assert blk[0, 0] == pytest.approx(th.sigma2[0], rel=1e-15)
        assert blk[1, 1] == pytest.approx(th.sigma2[1], rel=1e-15)
        assert blk[0, 1] == pytest.approx(rho[0, 1] * math.sqrt(th.sigma2[0] * th.sigma2[1]), rel=1e-15)
    # off-diagonal block (l, r) = C(|s_l - s_r|) entry by entry, Rep. I ordering
    l, r = 3, 17
    h = float(np.hypot(*(locs[l] - locs[r])))
    for i in range(p):
        for j in range(p):
            rs = rho[i, j] * math.sqrt(th.sigma2[i] * th.sigma2[j])
            assert S[p * l + i, p * r + j] == pytest.approx(
                oracle.matern(h, th.a, 0.5 * (th.nu[i] + th.nu[j]), rs), rel=1e-14)
    assert np.linalg.eigvalsh(S).min() > 0


def test_cross_covariance_block_is_rep_i():
    th, locs = _small_problem(12)
    new = inputs.jittered_grid(5, 99)
    S21 = oracle.covgen(th, new, locs)
    assert S21.shape == (10, 24)
    full = oracle.covgen(th, np.vstack([new, locs]))
    assert np.array_equal(S21, full[:10, 10:])


# ---------------------------------------------------- Cholesky / solve -----

def _leibniz_det(A):
    n = A.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        sgn = 1
        p = list(perm)
        for i in range(n):
            while p[i] != i:
                j = p[i]
                p[i], p[j] = p[j], p[i]
                sgn = -sgn
        prod = 1.0
        for i in range(n):
            prod *= A[i, perm[i]]
        tot += sgn * prod
    return tot


def _cramer_solve(A, b):
    d = _leibniz_det(A)
    x = np.empty(len(b))
    for i in range(len(b)):
        Ai = A.copy()
        Ai[:, i] = b
        x[i] = _leibniz_det(Ai) / d
    return x


@pytest.mark.parametrize("n_loc,p", [(3, 2), (4, 2), (2, 3)])
def test_tiny_brute_force_det_and_solve(n_loc, p):
    if p == 2:
        th = oracle.Theta([1.0, 2.0], 0.3, [0.5, 1.0], 0.6)
    else:
        th = oracle.Theta([1.0, 2.0, 0.5], 0.3, [0.5, 1.0, 1.5], [0.5, 0.3, 0.4])
    locs = inputs.jittered_grid(n_loc, 5)
    S = oracle.covgen(th, locs)
    N = S.shape[0]
    Z = inputs.normals(11, N)
    r = oracle.loglik(th, locs, Z, keep_factor=True)
    det = _leibniz_det(S)
    assert r.logdet == pytest.approx(math.log(det), rel=1e-12, abs=1e-12)
    x = _cramer_solve(S, Z)
    assert r.quad == pytest.approx(float(Z @ x), rel=1e-11)
    expect = -0.5 * N * math.log(2 * math.pi) - 0.5 * math.log(det) - 0.5 * float(Z @ x)
    assert r.loglik == pytest.approx(expect, rel=1e-12)


def test_cholesky_reconstruction_and_library():
    th, locs = _small_problem(150)
    S = oracle.covgen(th, locs)
    L, info = oracle.cholesky(S)
    assert info == 0
    assert np.allclose(np.triu(L, 1), 0)
    assert np.linalg.norm(L @ L.T - S) / np.linalg.norm(S) < 1e-15 * S.shape[0]
    assert np.allclose(L, np.linalg.cholesky(S), rtol=0, atol=1e-12)


def test_cholesky_info_on_indefinite():
    A = np.diag([1.0, 2.0, -1.0, 4.0])
    _, info = oracle.cholesky(A)
    assert info == 3
    B = np.array([[1.0, 2.0], [2.0, 1.0]])  # eigenvalues 3, -1
    assert oracle.cholesky(B)[1] == 2


def test_forward_backward_solves():
    th, locs = _small_problem(60)
    S = oracle.covgen(th, locs)
    L, _ = oracle.cholesky(S)
    z = inputs.normals(3, S.shape[0])
    y = oracle.forward(L, z)
    assert np.allclose(L @ y, z, atol=1e-10)
    w = oracle.backward(L, y)
    assert np.allclose(S @ w, z, atol=1e-8)
    assert np.allclose(w, np.linalg.solve(S, z), rtol=1e-8, atol=1e-8)


# ------------------------------------------------------------- Eq. 1 -------

def test_loglik_zero_data():
    th, locs = _small_problem(50)
    N = 100
    r = oracle.loglik(th, locs, np.zeros(N))
    sign, logdet = np.linalg.slogdet(oracle.covgen(th, locs))
    assert sign > 0
    assert r.quad == 0.0
    assert r.loglik == pytest.approx(-0.5 * N * math.log(2 * math.pi) - 0.5 * logdet, rel=1e-13)


def test_loglik_beta_zero_splits_into_univariate():
    # beta = 0: the variables are independent (Sec. 4.2), so l is the sum of
    # the p univariate likelihoods of the per-variable sub-vectors.
    locs = inputs.jittered_grid(70, 21)
    th = oracle.Theta([1.0, 0.7], 0.09, [0.5, 1.0], 0.0)
    Z = inputs.normals(4, 140)
    full = oracle.loglik(th, locs, Z).loglik
    parts = 0.0
    for i in range(2):
        thi = oracle.Theta([th.sigma2[i]], th.a, [th.nu[i]], np.eye(1))
        parts += oracle.loglik(thi, locs, Z[i::2]).loglik
    assert full == pytest.approx(parts, rel=1e-12)


def test_loglik_permutation_invariance_rep_i_rep_ii():
    # Rep. I and Rep. II give the same likelihood (Sec. 5.2); any symmetric
    # permutation of Sigma and Z leaves Eq. 1 unchanged.
    th, locs = _small_problem(45)
    Z = inputs.normals(8, 90)
    base = oracle.loglik(th, locs, Z).loglik
    # Rep. II: variable-major order, evaluated with library routines
    S = oracle.covgen(th, locs)
    perm = np.concatenate([np.arange(0, 90, 2), np.arange(1, 90, 2)])
    S2 = S[np.ix_(perm, perm)]
    z2 = Z[perm]
    sign, logdet = np.linalg.slogdet(S2)
    ref = -45 * math.log(2 * math.pi) - 0.5 * logdet - 0.5 * float(z2 @ np.linalg.solve(S2, z2))
    assert base == pytest.approx(ref, rel=1e-11)
    # location reordering (Morton)
    order = oracle.morton_order(locs)
    zi = Z.reshape(-1, 2)[order].reshape(-1)
    assert oracle.loglik(th, locs[order], zi).loglik == pytest.approx(base, rel=1e-12)


def test_forward_solve_whitens_simulated_draw():
    # Z = L e  =>  y = L^-1 Z = e and Z' Sigma^-1 Z = e'e.
    th, locs = _small_problem(80)
    e = inputs.normals(17, 160)
    Z = oracle.simulate(th, locs, e)
    r = oracle.loglik(th, locs, Z)
    assert np.allclose(r.y, e, rtol=0, atol=1e-9)
    assert r.quad == pytest.approx(float(e @ e), rel=1e-10)


def test_quadratic_form_chi_square_mean():
    # E[Z' Sigma^-1 Z] = N over seeded draws (chi-square with N dof).
    th, locs = _small_problem(40)
    N = 80
    S = oracle.covgen(th, locs)
    L, _ = oracle.cholesky(S)
    qs = []
    for s in range(200):
        Z = oracle.lower_matvec(L, inputs.normals(5000 + s, N))
        qs.append(oracle.forward(L, Z) @ oracle.forward(L, Z))
    m = float(np.mean(qs))
    assert abs(m - N) < 4 * math.sqrt(2 * N / 200)


# ------------------------------------------------------- Eq. 3 / Eq. 4 -----

def test_predict_at_observed_location_returns_data():
    th, locs = _small_problem(50)
    Z = oracle.simulate(th, locs, inputs.normals(9, 100))
    zhat = oracle.predict(th, locs, Z, locs[[4, 31]])
    assert np.allclose(zhat, np.concatenate([Z[8:10], Z[62:64]]), atol=1e-8)


def test_predict_beta_zero_is_separate_kriging():
    locs = inputs.jittered_grid(60, 13)
    new = inputs.jittered_grid(7, 77)
    th = oracle.Theta([1.0, 2.0], 0.1, [0.5, 1.5], 0.0)
    Z = inputs.normals(12, 120)
    zhat = oracle.predict(th, locs, Z, new).reshape(-1, 2)
    for i in range(2):
        thi = oracle.Theta([th.sigma2[i]], th.a, [th.nu[i]], np.eye(1))
        zi = oracle.predict(thi, locs, Z[i::2], new)
        assert np.allclose(zhat[:, i], zi, rtol=1e-10, atol=1e-12)


def test_predict_matches_library_solve():
    th, locs = _small_problem(40)
    new = inputs.jittered_grid(6, 55)
    Z = inputs.normals(19, 80)
    S = oracle.covgen(th, locs)
    c0t = oracle.covgen(th, new, locs)
    ref = c0t @ np.linalg.solve(S, Z)
    assert np.allclose(oracle.predict(th, locs, Z, new), ref, rtol=1e-9, atol=1e-10)


def test_mspe_definition():
    zhat = np.array([1.0, 2.0, 3.0, 4.0])
    z = np.array([0.0, 2.0, 3.0, 2.0])
    assert oracle.mspe(zhat, z, 2) == pytest.approx((1.0 + 4.0) / 2)


# ------------------------------------------------------------- Morton ------

def test_morton_keys_bit_interleave():
    locs = np.array([[0.0, 0.0], [1.0, 1.0], [0.0, 1.0], [1.0, 0.0]])
    keys = oracle.morton_keys(locs)
    assert keys[0] == 0
    assert keys[3] == oracle._spread16(65535)          # x only: even bits
    assert keys[2] == oracle._spread16(65535) << 1     # y only: odd bits
    assert keys[1] == 0xFFFFFFFF


def test_morton_order_z_pattern():
    g = np.array([[(i + 0.5) / 4, (j + 0.5) / 4] for j in range(4) for i in range(4)])
    order = oracle.morton_order(g)
    # first quadrant (x < 1/2, y < 1/2) comes first, in Z order: (0,0),(1,0),(0,1),(1,1)
    first4 = [tuple(np.round(g[k] * 4 - 0.5).astype(int)) for k in order[:4]]
    assert first4 == [(0, 0), (1, 0), (0, 1), (1, 1)]


# -------------------------------------------------------------- MLE --------

def test_nelder_mead_quadratic_and_rosenbrock():
    c = np.array([0.3, -1.2, 2.0])
    nm = oracle.NelderMead(lambda x: float(np.sum((x - c) ** 2)), np.zeros(3), step=0.5)
    for _ in range(300):
        nm.step()
    assert np.allclose(nm.best[0], c, atol=1e-5)
    rb = oracle.NelderMead(lambda x: (1 - x[0]) ** 2 + 100 * (x[1] - x[0] ** 2) ** 2, np.array([-1.2, 1.0]), step=0.1)
    for _ in range(600):
        rb.step()
    assert np.allclose(rb.best[0], [1.0, 1.0], atol=1e-4)


def test_nelder_mead_first_iteration_by_hand():
    # f(x) = x0^2 + 2 x1^2 from x0 = (1, 1), step 0.5: the vertices are
    # (1,1) f=3, (1.5,1) f=4.25, (1,1.5) f=5.5.  Centroid of the two best is
    # (1.25, 1); reflection of (1, 1.5) gives (1.5, 0.5), f = 2.75 < 3, so an
    # expansion to (1.75, 0) follows, f = 3.0625 > 2.75: the reflection is kept.
    nm = oracle.NelderMead(lambda x: x[0] ** 2 + 2 * x[1] ** 2, np.array([1.0, 1.0]), step=0.5)
    nm.step()
    assert nm.F == [3.0, 4.25, 5.5]
    nm.step()
    assert np.allclose(nm.X[0], [1.5, 0.5]) and nm.F[0] == 2.75
    assert [tuple(v) for v in nm.X[1:]] == [(1.0, 1.0), (1.5, 1.0)]


def test_theta_transform_roundtrip():
    th = oracle.Theta([1.0, 2.0, 0.5], 0.05, [0.5, 1.0, 1.5], [0.5, 0.3, 0.4])
    x = oracle.theta_to_x(th)
    assert len(x) == 10
    back = oracle.x_to_theta(x, 3)
    assert np.allclose(back.sigma2, th.sigma2) and back.a == pytest.approx(0.05)
    assert np.allclose(back.beta, th.beta)
    assert oracle.beta_is_pd(th.beta)
    assert not oracle.beta_is_pd(np.array([[1, 0.9, -0.9], [0.9, 1, 0.9], [-0.9, 0.9, 1.0]]))


# -------------------------------------------------------------- TLR --------

def test_tlr_reference_ranks_decay_and_order():
    # Fig. 5: off-diagonal ranks grow towards the diagonal; a tighter accuracy
    # never lowers a rank.  Morton-ordered bivariate matrix, Fig. 5 theta.
    g = json.load(open(GOLDEN))["fig5_theta"]
    th = oracle.Theta(g["sigma2"], g["a"], g["nu"], g["beta"])
    locs = inputs.jittered_grid(400, 1)
    locs = locs[oracle.morton_order(locs)]
    S = oracle.covgen(th, locs)
    nb = 100
    r5 = oracle.tlr_reference_ranks(S, nb, 1e-5)
    r9 = oracle.tlr_reference_ranks(S, nb, 1e-9)
    T = r5.shape[0]
    assert np.all(r9[r9 >= 0] >= r5[r5 >= 0])
    near = np.mean([r9[i, i - 1] for i in range(1, T)])
    far = np.mean([r9[i, j] for i in range(T) for j in range(i) if i - j >= T - 2])
    assert near > far
    assert r9.max() < nb


# --------------------------------------------------------- MLOE / MMOM -----

def test_mloe_mmom_zero_at_true_parameters():
    th, locs = _small_problem(40)
    pred = inputs.jittered_grid(5, 123)
    mloe, mmom, loe, mom = oracle.mloe_mmom(th, th, locs, pred)
    assert abs(mloe) < 1e-10 and abs(mmom) < 1e-10


def test_mloe_mmom_one_observation_hand_computed():
    # p = 1, nu = 1/2 (C(h) = sigma^2 e^(-h/a)), one observed location and one
    # prediction location 0.1 apart.  S = sigma^2, c = C(h) and C(0) = sigma^2
    # are scalars, so Eq. 5 - Eq. 7 are scalar algebra:
    #   E_t = s_t - c_t^2 / s_t,  E_ta = s_t - 2 c_t c_a / s_a + c_a^2 s_t / s_a^2,
    #   E_a = s_a - c_a^2 / s_a  (C(0; theta_a) = s_a: Algorithm 1's E_a).
    # With s_t = 1, a_t = 0.1, s_a = 2, a_a = 0.2: c_t = e^-1, c_a = 2 e^-1/2, so
    #   E_t = 1 - e^-2, E_ta = 1 - 2 e^-3/2 + e^-1, E_a = 2 - 2 e^-1.
    th_t = oracle.Theta([1.0], 0.1, [0.5], np.eye(1))
    th_a = oracle.Theta([2.0], 0.2, [0.5], np.eye(1))
    locs = np.array([[0.3, 0.4]])
    pred = np.array([[0.3, 0.5]])
    Et = 1.0 - math.exp(-2.0)
    Eta = 1.0 - 2.0 * math.exp(-1.5) + math.exp(-1.0)
    Ea = 2.0 - 2.0 * math.exp(-1.0)
    mloe, mmom, loe, mom = oracle.mloe_mmom(th_t, th_a, locs, pred)
    assert loe[0] == pytest.approx(Eta / Et - 1.0, rel=1e-12)
    assert mom[0] == pytest.approx(Ea / Eta - 1.0, rel=1e-12)
    assert (mloe, mmom) == (loe[0], mom[0])
    # the three energies are distinct here, so E_a with C(0; theta_t) (= 1 - 2 e^-1) would not pass
    assert abs(Ea - (1.0 - 2.0 * math.exp(-1.0))) > 0.5 and abs(Ea - Eta) > 0.1 and abs(Eta - Et) > 0.01


def _matern_half_integer(h, a, nu):
    x = h / a
    if nu == 0.5:
        return math.exp(-x)
    if nu == 1.5:
        return (1.0 + x) * math.exp(-x)
    if nu == 2.5:
        return (1.0 + x + x * x / 3.0) * math.exp(-x)
    raise ValueError(nu)


def _block(theta_s2, a, nus, beta, h):
    """2 x 2 Eq. 2 block at distance h from the half-integer closed forms, rho_12 = beta sqrt(nu1 nu2) / nu12."""
    nu12 = 0.5 * (nus[0] + nus[1])
    rho = beta * math.sqrt(nus[0] * nus[1]) / nu12
    s1, s2 = math.sqrt(theta_s2[0]), math.sqrt(theta_s2[1])
    c11 = theta_s2[0] * _matern_half_integer(h, a, nus[0])
    c22 = theta_s2[1] * _matern_half_integer(h, a, nus[1])
    c12 = rho * s1 * s2 * _matern_half_integer(h, a, nu12)
    return np.array([[c11, c12], [c12, c22]])


def test_mloe_mmom_bivariate_one_observation_closed_forms():
    # p = 2 with nu = (1/2, 5/2), so nu_12 = 3/2: every entry of S (the colocated
    # block), c and C(0) has a closed form; E_t, E_ta and E_a are 2 x 2 algebra.
    nus = (0.5, 2.5)
    tt = ((1.0, 1.5), 0.12, 0.6)   # (sigma^2, a, beta)
    ta = ((0.7, 2.0), 0.2, -0.3)
    h = 0.15
    locs = np.array([[0.5, 0.5]])
    pred = np.array([[0.5 + h, 0.5]])
    St, Sa = _block(tt[0], tt[1], nus, tt[2], 0.0), _block(ta[0], ta[1], nus, ta[2], 0.0)
    ct, ca = _block(tt[0], tt[1], nus, tt[2], h), _block(ta[0], ta[1], nus, ta[2], h)
    Sai = np.linalg.inv(Sa)
    Et = np.trace(St - ct.T @ np.linalg.inv(St) @ ct)
    Eta = np.trace(St - 2.0 * ct.T @ Sai @ ca + ca.T @ Sai @ St @ Sai @ ca)
    Ea = np.trace(Sa - ca.T @ Sai @ ca)
    th_t = oracle.Theta(list(tt[0]), tt[1], list(nus), tt[2])
    th_a = oracle.Theta(list(ta[0]), ta[1], list(nus), ta[2])
    _, _, loe, mom = oracle.mloe_mmom(th_t, th_a, locs, pred)
    assert loe[0] == pytest.approx(Eta / Et - 1.0, rel=1e-11)
    assert mom[0] == pytest.approx(Ea / Eta - 1.0, rel=1e-11)
    assert abs(Ea - np.trace(St - ca.T @ Sai @ ca)) > 0.1   # C(0; theta_t) in E_a would differ


@pytest.mark.parametrize("p", [1, 2])
def test_mloe_mmom_variance_scale_only(p):
    # theta_a = theta_t except every sigma^2 times c: Sigma_a = c Sigma_t, c_a = c c_t,
    # so S_a^-1 c_a = S_t^-1 c_t, E_ta = E_t (LOE = 0) and E_a = c E_t (MOM = c - 1) exactly.
    cfac = 1.7
    if p == 1:
        th_t = oracle.Theta([0.8], 0.09, [1.0], np.eye(1))
        th_a = oracle.Theta([0.8 * cfac], 0.09, [1.0], np.eye(1))
    else:
        th_t = oracle.Theta([1.0, 1.3], 0.09, [0.5, 1.0], 0.5)
        th_a = oracle.Theta([1.0 * cfac, 1.3 * cfac], 0.09, [0.5, 1.0], 0.5)
    locs = inputs.jittered_grid(40, 7)
    pred = inputs.jittered_grid(5, 123)
    mloe, mmom, loe, mom = oracle.mloe_mmom(th_t, th_a, locs, pred)
    np.testing.assert_allclose(loe, 0.0, atol=1e-10)
    np.testing.assert_allclose(mom, cfac - 1.0, rtol=1e-10)
    assert mmom == pytest.approx(cfac - 1.0, rel=1e-10)


def test_mloe_nonnegative_for_misspecified():
    # E_ta >= E_t since the true-parameter cokriging predictor is the BLUP.
    th, locs = _small_problem(40)
    tha = oracle.Theta([1.2, 1.0], 0.12, [0.6, 1.0], 0.3)
    pred = inputs.jittered_grid(5, 123)
    mloe, mmom, loe, mom = oracle.mloe_mmom(th, tha, locs, pred)
    assert np.all(loe >= -1e-12)


# ---- prediction variance (diag of C(0) - c0' Sigma^-1 c0) --------------------

def test_predict_var_zero_at_observed_locations_and_bounded():
    th = oracle.Theta([1.0, 2.0], 0.1, [0.5, 1.0], np.array([[1.0, 0.5], [0.5, 1.0]]))
    locs = inputs.jittered_grid(60, 5)
    v_obs = oracle.predict_var(th, locs, locs[[3, 17, 42]])
    assert np.all(np.abs(v_obs) < 1e-10)   # no nugget: an observed location is known exactly
    new = inputs.jittered_grid(25, 6)
    v = oracle.predict_var(th, locs, new)
    s2 = np.tile([1.0, 2.0], 25)
    assert np.all(v >= -1e-12) and np.all(v <= s2 + 1e-12)


def test_predict_var_far_from_the_data_is_the_prior_variance():
    th = oracle.Theta([1.3, 0.7], 0.02, [0.5, 1.5], np.array([[1.0, -0.4], [-0.4, 1.0]]))
    locs = inputs.jittered_grid(40, 7) * 0.2          # all data in [0, 0.2]^2
    v = oracle.predict_var(th, locs, np.array([[0.95, 0.95]]))
    # the nearest datum is > 1 away, 50 a: every covariance with it is below e^-50
    assert v == pytest.approx([1.3, 0.7], abs=1e-15)


def test_predict_var_beta_zero_is_univariate_kriging():
    thb = oracle.Theta([1.0, 2.0], 0.1, [0.5, 1.5], np.eye(2))
    locs = inputs.jittered_grid(50, 8)
    new = inputs.jittered_grid(10, 9)
    v = oracle.predict_var(thb, locs, new)
    for i, (s2, nu) in enumerate([(1.0, 0.5), (2.0, 1.5)]):
        th1 = oracle.Theta([s2], 0.1, [nu], np.eye(1))
        assert v[i::2] == pytest.approx(oracle.predict_var(th1, locs, new), rel=1e-12, abs=1e-14)


def test_predict_var_matches_library_solve():
    th = oracle.Theta([1.0, 1.0], 0.09, [0.5, 1.0], np.array([[1.0, 0.5], [0.5, 1.0]]))
    locs = inputs.jittered_grid(70, 10)
    new = inputs.jittered_grid(8, 11)
    S = oracle.covgen(th, locs)
    c0 = oracle.covgen(th, locs, new)                     # (2 * 70) x (2 * 8)
    ref = np.diag(oracle.covgen(th, new)) - np.einsum("ij,ij->j", c0, np.linalg.solve(S, c0))
    assert oracle.predict_var(th, locs, new) == pytest.approx(ref, rel=1e-9, abs=1e-12)


# ---- Diagonal Super Tile (Sec. 3.4) -----------------------------------------

def _dst_problem():
    th = oracle.Theta([1.0, 1.5], 0.04, [0.5, 1.0], np.array([[1.0, 0.4], [0.4, 1.0]]))
    locs = inputs.jittered_grid(120, 21)
    Z = oracle.simulate(th, locs, inputs.normals(22, 240))
    return th, locs, Z


def test_dst_with_every_tile_kept_is_the_exact_likelihood():
    th, locs, Z = _dst_problem()
    full = oracle.loglik(th, locs, Z).loglik
    assert oracle.dst_loglik(th, locs, Z, 48, 5) == pytest.approx(full, rel=1e-12)   # 240 / 48 = 5 tiles


def test_dst_one_tile_diagonal_is_a_sum_of_block_likelihoods():
    th, locs, Z = _dst_problem()
    perm = oracle.morton_order(locs)
    ls, zs = locs[perm], Z.reshape(-1, 2)[perm]
    # nb = 48 rows = 24 locations per tile: independent blocks of consecutive Morton locations
    ref = sum(oracle.loglik(th, ls[b:b + 24], zs[b:b + 24].ravel()).loglik for b in range(0, 120, 24))
    assert oracle.dst_loglik(th, locs, Z, 48, 1) == pytest.approx(ref, rel=1e-12)


def test_dst_matches_a_direct_numpy_evaluation():
    th, locs, Z = _dst_problem()
    perm = oracle.morton_order(locs)
    S = oracle.covgen(th, locs[perm])
    idx = np.arange(240) // 40
    S[np.abs(idx[:, None] - idx[None, :]) >= 3] = 0.0
    zs = Z.reshape(-1, 2)[perm].ravel()
    sign, logdet = np.linalg.slogdet(S)
    ref = -0.5 * 240 * np.log(2 * np.pi) - 0.5 * logdet - 0.5 * zs @ np.linalg.solve(S, zs)
    assert sign > 0
    assert oracle.dst_loglik(th, locs, Z, 40, 3) == pytest.approx(ref, rel=1e-10)


# ------------------------------------------------ profile likelihood -------

def _profile_problem(p, beta, nu, seed):
    th = oracle.Theta([1.3, 0.7, 2.0][:p], 0.08, nu, beta)
    locs = inputs.jittered_grid(90, seed)
    Z = oracle.simulate(th, locs, inputs.normals(seed + 1, p * 90))
    return th, locs, Z


def test_profile_p1_is_the_maximum_over_sigma2():
    # p = 1: sigma2_hat is the exact maximiser of Eq. 1 over sigma^2 (Sec. 4.2),
    # found here by a bounded scalar search on the full likelihood
    optimize = pytest.importorskip("scipy.optimize")
    th, locs, Z = _profile_problem(1, np.eye(1), [0.8], 61)
    f = lambda ls: -oracle.loglik(oracle.Theta([math.exp(ls)], th.a, th.nu, th.beta), locs, Z).loglik
    r = optimize.minimize_scalar(f, bounds=(-5, 5), method="bounded", options={"xatol": 1e-10})
    ll, s2 = oracle.profile_loglik(th, locs, Z)
    assert s2[0] == pytest.approx(math.exp(r.x), rel=1e-7)
    assert ll == pytest.approx(-r.fun, rel=1e-12)


def test_profile_beta_zero_maximises_each_variance():
    # beta = 0: Sigma is block diagonal by variable, Eq. 1 splits into p
    # univariate likelihoods and the joint maximiser over sigma^2 is sigma2_hat
    optimize = pytest.importorskip("scipy.optimize")
    th, locs, Z = _profile_problem(2, np.eye(2), [0.5, 1.3], 63)

    def f(ls):
        return -oracle.loglik(oracle.Theta(np.exp(ls), th.a, th.nu, th.beta), locs, Z).loglik

    r = optimize.minimize(f, np.zeros(2), method="Nelder-Mead",
                          options={"xatol": 1e-10, "fatol": 1e-13, "maxiter": 4000})
    ll, s2 = oracle.profile_loglik(th, locs, Z)
    np.testing.assert_allclose(s2, np.exp(r.x), rtol=1e-6)
    assert ll == pytest.approx(-r.fun, rel=1e-11)


def test_sigma2_hat_closed_form_correlations():
    # nu = 1/2 and 3/2 have closed-form Matern correlations, exp(-t) and (1 + t) exp(-t),
    # t = h / a; sigma2_hat by a dense numpy solve with them (beta does not enter)
    th, locs, Z = _profile_problem(2, np.array([[1.0, 0.6], [0.6, 1.0]]), [0.5, 1.5], 65)
    t = np.linalg.norm(locs[:, None, :] - locs[None, :, :], axis=2) / th.a
    R = [np.exp(-t), (1 + t) * np.exp(-t)]
    ref = [Z[i::2] @ np.linalg.solve(R[i], Z[i::2]) / 90 for i in range(2)]
    np.testing.assert_allclose(oracle.sigma2_hat(th, locs, Z), ref, rtol=1e-12)


def test_profile_scale_equivariance_and_joint_bound():
    # Z -> c Z: sigma2_hat -> c^2 sigma2_hat and l_profile -> l_profile - N log c;
    # the plug-in value never exceeds the joint maximum of Eq. 1 over sigma^2
    optimize = pytest.importorskip("scipy.optimize")
    th, locs, Z = _profile_problem(3, np.array([[1.0, 0.5, 0.2], [0.5, 1.0, 0.3], [0.2, 0.3, 1.0]]),
                                   [0.5, 1.0, 1.5], 67)
    ll, s2 = oracle.profile_loglik(th, locs, Z)
    c = 3.0
    ll_c, s2_c = oracle.profile_loglik(th, locs, c * Z)
    np.testing.assert_allclose(s2_c, c * c * s2, rtol=1e-12)
    assert ll_c == pytest.approx(ll - 270 * math.log(c), rel=1e-12)
    f = lambda ls: -oracle.loglik(oracle.Theta(np.exp(ls), th.a, th.nu, th.beta), locs, Z).loglik
    r = optimize.minimize(f, np.log(s2), method="Nelder-Mead", options={"xatol": 1e-9, "fatol": 1e-12})
    assert ll <= -r.fun + 1e-9


def test_profile_coordinates_roundtrip():
    th = oracle.Theta([2.0, 3.0], 0.07, [0.4, 1.7], 0.35)
    x = oracle.profile_theta_to_x(th)
    assert x.shape == (4,)
    back = oracle.profile_x_to_theta(x, 2)
    assert back.a == pytest.approx(0.07, rel=1e-15)
    np.testing.assert_allclose(back.nu, [0.4, 1.7], rtol=1e-15)
    assert back.beta[0, 1] == 0.35 and back.beta[1, 0] == 0.35
    np.testing.assert_array_equal(back.sigma2, [1.0, 1.0])


def test_profile_mle_reaches_the_full_mle_at_p1():
    # p = 1: the profile likelihood is exact (Sec. 4.2), so Nelder-Mead over (log a, log nu)
    # on it and over (log sigma^2, log a, log nu) on Eq. 1 reach the same maximum
    th = oracle.Theta([1.5], 0.15, [0.9], np.eye(1))
    locs = inputs.jittered_grid(64, 71)
    Z = oracle.simulate(th, locs, inputs.normals(72, 64))

    def run(nm, iters):
        for _ in range(iters):
            nm.step()
        return nm.best

    full = oracle.NelderMead(oracle.mle_objective(locs, Z, 1), oracle.theta_to_x(th), step=0.2)
    prof = oracle.NelderMead(oracle.profile_objective(locs, Z, 1), oracle.profile_theta_to_x(th), step=0.2)
    xf, ff = run(full, 300)
    xp, fp = run(prof, 200)
    assert fp == pytest.approx(ff, abs=1e-6)
    np.testing.assert_allclose(xp, xf[1:], atol=2e-3)                 # log a, log nu
    s2 = oracle.sigma2_hat(oracle.profile_x_to_theta(xp, 1), locs, Z)
    assert math.log(s2[0]) == pytest.approx(xf[0], abs=2e-3)          # log sigma^2
