"""CPU FP64 oracle for the multivariate Matern likelihood and cokriging (arxiv 2008.07437).

TEST INFRASTRUCTURE ONLY.  This package is a slow, plain, obviously correct
restatement of what the paper computes.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_2008_07437_gb300``) never imports, links or runs it,
and the two share no code: this package does not import the product package
and the product package does not import this one.

Contents and the passage each part follows:

* ``oracle.c`` (built to ``liboracle.so`` with gcc + OpenMP):
  K_nu by trapezoid quadrature of an integral representation, Eq. 2 (Sec. 4.2),
  rho_ij and nu_ij (Sec. 4.2), Representation I covariance (Sec. 5.2),
  an unblocked Crout Cholesky, forward/back substitution, Eq. 1 and the
  cokriging predictor Eq. 3 / Eq. 4 (Sec. 4.3).
* ``morton_order``: Z-order location sorting (Sec. 5.3).
* ``NelderMead``: the textbook Nelder-Mead simplex method used as the MLE
  optimiser (the paper maximises Eq. 1 with NLopt, algorithm unnamed).
* ``tlr_reference_ranks``: exact truncated-SVD ranks of the off-diagonal tiles
  at an absolute accuracy threshold (Sec. 5.3, Fig. 5).
* ``mloe_mmom``: the multivariate MLOE/MMOM criteria, Eq. 5 - Eq. 8 and
  Algorithm 1 (Sec. 5.4).
* ``sigma2_hat`` / ``profile_loglik`` / ``profile_objective``: the profile
  likelihood of Sec. 4.2 (marginal variances from each variable's own
  correlation matrix, plugged into Eq. 1).

Pins that tie this oracle to the paper and to mathematics (not to itself) live
in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, OpenMP, no fast-math)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        d, i, P = ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
        lib.oracle_besselk_scaled.restype = d
        lib.oracle_besselk_scaled.argtypes = [d, d]
        lib.oracle_besselk.restype = d
        lib.oracle_besselk.argtypes = [d, d]
        lib.oracle_matern.restype = d
        lib.oracle_matern.argtypes = [d, d, d, d]
        lib.oracle_matern_params.restype = None
        lib.oracle_matern_params.argtypes = [i, i, P, P, P, P]
        lib.oracle_covgen.restype = None
        lib.oracle_covgen.argtypes = [i, P, P, P, d, P, i, P, i, P]
        lib.oracle_cholesky.restype = i
        lib.oracle_cholesky.argtypes = [P, i]
        lib.oracle_forward.restype = None
        lib.oracle_forward.argtypes = [P, i, P]
        lib.oracle_backward.restype = None
        lib.oracle_backward.argtypes = [P, i, P]
        lib.oracle_loglik_from_factor.restype = None
        lib.oracle_loglik_from_factor.argtypes = [P, i, P, P, P]
        lib.oracle_predict.restype = None
        lib.oracle_predict.argtypes = [i, P, P, P, d, P, P, i, P, P, i, P]
        lib.oracle_lower_matvec.restype = None
        lib.oracle_lower_matvec.argtypes = [P, i, P, P]
        lib.oracle_num_threads.restype = i
        lib.oracle_num_threads.argtypes = []
        lib.oracle_set_threads.restype = None
        lib.oracle_set_threads.argtypes = [i]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


# ----------------------------------------------------------------------------
# Special functions and Eq. 2
# ----------------------------------------------------------------------------

def besselk(nu: float, x: float) -> float:
    """K_nu(x), trapezoid quadrature of int_0^inf exp(-x cosh t) cosh(nu t) dt."""
    return _load().oracle_besselk(float(nu), float(x))


def besselk_scaled(nu: float, x: float) -> float:
    """e^x K_nu(x)."""
    return _load().oracle_besselk_scaled(float(nu), float(x))


def matern_params(nu, beta, d: int = 2):
    """Sec. 4.2: (rho_ij, nu_ij) as p x p arrays, rho_ii = 1."""
    nu = _f64(nu)
    p = nu.shape[0]
    beta = _f64(beta).reshape(p, p)
    rho = np.zeros((p, p))
    nuij = np.zeros((p, p))
    _load().oracle_matern_params(p, d, _ptr(nu), _ptr(beta), _ptr(rho), _ptr(nuij))
    return rho, nuij


def matern(h: float, a: float, nuij: float, rho_sig: float) -> float:
    """Eq. 2 for one (i, j): rho_sig = rho_ij sigma_i sigma_j."""
    return _load().oracle_matern(float(h), float(a), float(nuij), float(rho_sig))


class Theta:
    """theta = (sigma^2_1..p, a, nu_1..p, beta) (Sec. 4.2)."""

    def __init__(self, sigma2, a, nu, beta):
        self.sigma2 = _f64(sigma2)
        self.a = float(a)
        self.nu = _f64(nu)
        p = self.sigma2.shape[0]
        b = np.eye(p)
        beta = np.asarray(beta, dtype=np.float64)
        if beta.ndim == 0:
            b[0, 1] = b[1, 0] = float(beta)
        elif beta.ndim == 1:  # upper-triangle list b12, b13, ..., b23, ...
            k = 0
            for i in range(p):
                for j in range(i + 1, p):
                    b[i, j] = b[j, i] = beta[k]
                    k += 1
        else:
            b = beta.copy()
        self.beta = _f64(b)
        self.p = p

    def as_tuple(self):
        return (self.sigma2.copy(), self.a, self.nu.copy(), self.beta.copy())


def covgen(theta: Theta, locs1, locs2=None) -> np.ndarray:
    """Representation I cross-covariance (Sec. 5.2, Eq. 4): (p n1) x (p n2) dense."""
    locs1 = _f64(locs1).reshape(-1, 2)
    locs2 = locs1 if locs2 is None else _f64(locs2).reshape(-1, 2)
    p = theta.p
    out = np.empty((p * locs1.shape[0], p * locs2.shape[0]))
    _load().oracle_covgen(p, _ptr(theta.sigma2), _ptr(theta.nu), _ptr(theta.beta), theta.a,
                          _ptr(locs1), locs1.shape[0], _ptr(locs2), locs2.shape[0], _ptr(out))
    return out


# ----------------------------------------------------------------------------
# Cholesky, solves and Eq. 1
# ----------------------------------------------------------------------------

def cholesky(A) -> tuple[np.ndarray, int]:
    """Unblocked Crout Cholesky; returns (L, info) with info = 1-based failing column or 0."""
    L = _f64(A).copy()
    info = _load().oracle_cholesky(_ptr(L), L.shape[0])
    return L, info


def forward(L, z) -> np.ndarray:
    y = _f64(z).copy()
    _load().oracle_forward(_ptr(_f64(L)), y.shape[0], _ptr(y))
    return y


def backward(L, y) -> np.ndarray:
    w = _f64(y).copy()
    _load().oracle_backward(_ptr(_f64(L)), w.shape[0], _ptr(w))
    return w


def lower_matvec(L, e) -> np.ndarray:
    e = _f64(e)
    out = np.empty_like(e)
    _load().oracle_lower_matvec(_ptr(_f64(L)), e.shape[0], _ptr(e), _ptr(out))
    return out


class LoglikResult:
    def __init__(self, loglik, logdet, quad, L, y, info):
        self.loglik, self.logdet, self.quad = loglik, logdet, quad
        self.L, self.y, self.info = L, y, info


def loglik(theta: Theta, locs, Z, keep_factor: bool = False) -> LoglikResult:
    """Eq. 1: l = -(N/2) log 2pi - 1/2 log|Sigma| - 1/2 Z' Sigma^-1 Z, N = p n."""
    S = covgen(theta, locs)
    L, info = cholesky(S)
    if info:
        return LoglikResult(float("nan"), float("nan"), float("nan"), None, None, info)
    Z = _f64(Z)
    N = Z.shape[0]
    y = np.empty(N)
    out3 = np.empty(3)
    _load().oracle_loglik_from_factor(_ptr(L), N, _ptr(Z), _ptr(y), _ptr(out3))
    return LoglikResult(float(out3[0]), float(out3[1]), float(out3[2]), L if keep_factor else None, y, 0)


def predict(theta: Theta, locs, Z, new_locs, L=None) -> np.ndarray:
    """Eq. 3 / Eq. 4: Zhat(s0) = c0' Sigma^-1 Z for every new location (Rep. I, p m entries)."""
    locs = _f64(locs).reshape(-1, 2)
    new_locs = _f64(new_locs).reshape(-1, 2)
    if L is None:
        L, info = cholesky(covgen(theta, locs))
        if info:
            raise ValueError("Sigma not positive definite (info=%d)" % info)
    p = theta.p
    zhat = np.empty(p * new_locs.shape[0])
    _load().oracle_predict(p, _ptr(theta.sigma2), _ptr(theta.nu), _ptr(theta.beta), theta.a, _ptr(_f64(L)),
                           _ptr(locs), locs.shape[0], _ptr(_f64(Z)), _ptr(new_locs), new_locs.shape[0],
                           _ptr(zhat))
    return zhat


def predict_var(theta: Theta, locs, new_locs, L=None) -> np.ndarray:
    """Prediction (cokriging) variances, the diagonal of C(0) - c0' Sigma^-1 c0 at
    every new location (the mean square error of Eq. 3's predictor under the
    true model, the E_t term of Eq. 5 before the trace); p m entries, Rep. I."""
    locs = _f64(locs).reshape(-1, 2)
    new_locs = _f64(new_locs).reshape(-1, 2)
    if L is None:
        L, info = cholesky(covgen(theta, locs))
        if info:
            raise ValueError("Sigma not positive definite (info=%d)" % info)
    p = theta.p
    out = np.empty(p * new_locs.shape[0])
    for l in range(new_locs.shape[0]):
        s0 = new_locs[l:l + 1]
        c0 = covgen(theta, locs, s0)                 # (p n) x p
        C0 = covgen(theta, s0)                       # p x p
        for i in range(p):
            y = forward(L, c0[:, i])                 # L^-1 c0_i
            out[p * l + i] = C0[i, i] - float(y @ y)
    return out


def dst_loglik(theta: Theta, locs, Z, nb: int, dst: int) -> float:
    """Eq. 1 for the Diagonal Super Tile approximation (Sec. 3.4): Sigma in
    Morton order (Sec. 5.3), cut into nb x nb tiles; the tiles with
    |I - J| >= dst are set to zero and the rest kept exactly."""
    locs = _f64(locs).reshape(-1, 2)
    p = theta.p
    perm = morton_order(locs)
    ls = locs[perm]
    zs = _f64(Z).reshape(-1, p)[perm].ravel()
    S = covgen(theta, ls)
    N = S.shape[0]
    idx = np.arange(N) // nb
    S[np.abs(idx[:, None] - idx[None, :]) >= dst] = 0.0
    L, info = cholesky(S)
    if info:
        raise ValueError("the DST matrix is not positive definite (info=%d)" % info)
    y = forward(L, zs)
    logdet = 2.0 * float(np.sum(np.log(np.diag(L))))
    return -0.5 * N * math.log(2.0 * math.pi) - 0.5 * logdet - 0.5 * float(y @ y)


def simulate(theta: Theta, locs, e) -> np.ndarray:
    """Z = L e with L L' = Sigma(theta): a draw from N(0, Sigma) given standard normals e."""
    L, info = cholesky(covgen(theta, locs))
    if info:
        raise ValueError("Sigma not positive definite (info=%d)" % info)
    return lower_matvec(L, e)


def mspe(zhat, ztrue, p: int) -> float:
    """Sec. 4.5: MSPE = (1/n_pred) sum_l ||Zhat(s0_l) - Z(s0_l)||^2."""
    d = (np.asarray(zhat) - np.asarray(ztrue)).reshape(-1, p)
    return float(np.mean(np.sum(d * d, axis=1)))


# ----------------------------------------------------------------------------
# Morton (Z-order) ordering of locations (Sec. 5.3)
# ----------------------------------------------------------------------------

def _spread16(v: int) -> int:
    out = 0
    for b in range(16):
        out |= ((v >> b) & 1) << (2 * b)
    return out


def morton_keys(locs) -> list[int]:
    """32-bit Z-order keys: both coordinates quantised to 16 bits over the square
    bounding box [xmin, xmin + span] x [ymin, ymin + span], span = max extent;
    x bits take the even positions, y bits the odd ones."""
    locs = _f64(locs).reshape(-1, 2)
    xmin = float(np.min(locs[:, 0])) if len(locs) else 0.0
    ymin = float(np.min(locs[:, 1])) if len(locs) else 0.0
    span = max(float(np.max(locs[:, 0])) - xmin, float(np.max(locs[:, 1])) - ymin) if len(locs) else 0.0
    keys = []
    for x, y in locs:
        if span > 0.0:
            qx = math.floor((float(x) - xmin) / span * 65536.0)
            qy = math.floor((float(y) - ymin) / span * 65536.0)
        else:
            qx = qy = 0
        qx = min(max(qx, 0), 65535)
        qy = min(max(qy, 0), 65535)
        keys.append(_spread16(qx) | (_spread16(qy) << 1))
    return keys


def morton_order(locs) -> np.ndarray:
    """Permutation that sorts locations by (Morton key, original index)."""
    keys = morton_keys(locs)
    return np.array(sorted(range(len(keys)), key=lambda i: (keys[i], i)), dtype=np.int64)


# ----------------------------------------------------------------------------
# Nelder-Mead maximisation of Eq. 1 (the paper's MLE driver; NLopt algorithm
# unnamed, read as the textbook simplex method with coefficients 1, 2, 1/2, 1/2)
# ----------------------------------------------------------------------------

def theta_to_x(theta: Theta) -> np.ndarray:
    """Unconstrained coordinates: (log sigma^2_i, log a, log nu_i, beta_ij for i<j)."""
    p = theta.p
    xs = [math.log(s) for s in theta.sigma2] + [math.log(theta.a)] + [math.log(v) for v in theta.nu]
    for i in range(p):
        for j in range(i + 1, p):
            xs.append(float(theta.beta[i, j]))
    return np.array(xs, dtype=np.float64)


def x_to_theta(x, p: int) -> Theta:
    sigma2 = [math.exp(v) for v in x[:p]]
    a = math.exp(x[p])
    nu = [math.exp(v) for v in x[p + 1:2 * p + 1]]
    return Theta(sigma2, a, nu, np.array(x[2 * p + 1:], dtype=np.float64))


def beta_is_pd(beta: np.ndarray) -> bool:
    """Positive definiteness of the correlation matrix beta via an unpivoted
    Cholesky (every pivot > 0); |beta_ij| < 1 is implied."""
    p = beta.shape[0]
    L = np.zeros((p, p))
    for j in range(p):
        s = beta[j, j] - sum(L[j, k] * L[j, k] for k in range(j))
        if not s > 0.0:
            return False
        L[j, j] = math.sqrt(s)
        for i in range(j + 1, p):
            L[i, j] = (beta[i, j] - sum(L[i, k] * L[j, k] for k in range(j))) / L[j, j]
    return True


class NelderMead:
    """Textbook Nelder-Mead minimisation of f(x) = -l(theta(x)).

    * Initial simplex: x0 and x0 + step * e_k, k = 1..q.
    * Each iteration: order vertices by (f, index) ascending, centroid of the q
      best, reflection (1), expansion (2), outside / inside contraction (1/2),
      shrink towards the best (1/2).
    * Infeasible theta (beta not positive definite) gives f = +inf.
    One call of ``step`` = initialisation on the first call, one iteration after.
    """

    def __init__(self, f, x0, step: float = 0.1):
        self.f = f
        self.q = len(x0)
        x0 = np.array(x0, dtype=np.float64)
        self.X = [x0.copy()]
        for k in range(self.q):
            v = x0.copy()
            v[k] = v[k] + step
            self.X.append(v)
        self.F = None
        self.iters = 0
        self.evals = 0
        self.log = []  # (x, f) for every evaluation, in order

    def _eval(self, x):
        v = self.f(x)
        self.evals += 1
        self.log.append((np.array(x), v))
        return v

    def _order(self):
        idx = sorted(range(self.q + 1), key=lambda k: (self.F[k], k))
        self.X = [self.X[k] for k in idx]
        self.F = [self.F[k] for k in idx]

    def step(self):
        q = self.q
        if self.F is None:
            self.F = [self._eval(x) for x in self.X]
            self._order()
            return
        xbar = np.zeros(q)
        for k in range(q):
            xbar = xbar + self.X[k]
        xbar = xbar / q
        xw, fw = self.X[q], self.F[q]
        xr = xbar + 1.0 * (xbar - xw)
        fr = self._eval(xr)
        if self.F[0] <= fr < self.F[q - 1]:
            self.X[q], self.F[q] = xr, fr
        elif fr < self.F[0]:
            xe = xbar + 2.0 * (xr - xbar)
            fe = self._eval(xe)
            if fe < fr:
                self.X[q], self.F[q] = xe, fe
            else:
                self.X[q], self.F[q] = xr, fr
        else:
            shrink = False
            if fr < fw:
                xc = xbar + 0.5 * (xr - xbar)
                fc = self._eval(xc)
                if fc <= fr:
                    self.X[q], self.F[q] = xc, fc
                else:
                    shrink = True
            else:
                xc = xbar - 0.5 * (xbar - xw)
                fc = self._eval(xc)
                if fc < fw:
                    self.X[q], self.F[q] = xc, fc
                else:
                    shrink = True
            if shrink:
                for k in range(1, q + 1):
                    self.X[k] = self.X[0] + 0.5 * (self.X[k] - self.X[0])
                    self.F[k] = self._eval(self.X[k])
        self._order()
        self.iters += 1

    @property
    def best(self):
        return self.X[0], self.F[0]


def mle_objective(locs, Z, p: int):
    """f(x) = -l(theta(x)) with +inf outside the feasible set (beta not PD,
    Cholesky failure)."""
    def f(x):
        th = x_to_theta(x, p)
        if not beta_is_pd(th.beta):
            return math.inf
        r = loglik(th, locs, Z)
        if r.info:
            return math.inf
        return -r.loglik
    return f


# ----------------------------------------------------------------------------
# Profile likelihood (Sec. 4.2): the marginal variances leave the optimisation
# ----------------------------------------------------------------------------

def sigma2_hat(theta: Theta, locs, Z) -> np.ndarray:
    """Sec. 4.2: sigma^2_ii = n^-1 Z_i' R_ii^-1 Z_i for i = 1..p, where Z_i holds
    the n values of variable i (every p-th entry of Representation I, from i)
    and R_ii is the correlation matrix of variable i alone: the Matern of
    Eq. 2 with i = j, sigma^2_ii = 1, smoothness nu_ii and range a.  sigma^2 and
    beta of ``theta`` are not used."""
    locs = _f64(locs).reshape(-1, 2)
    Z = _f64(Z)
    p, n = theta.p, locs.shape[0]
    out = np.empty(p)
    for i in range(p):
        Rii = covgen(Theta([1.0], theta.a, [theta.nu[i]], np.eye(1)), locs)
        L, info = cholesky(Rii)
        if info:
            raise np.linalg.LinAlgError(f"R_{i + 1}{i + 1} is not positive definite (column {info})")
        y = forward(L, Z[i::p])
        out[i] = float(y @ y) / n
    return out


def profile_loglik(theta: Theta, locs, Z) -> tuple[float, np.ndarray]:
    """Profile log-likelihood (Sec. 4.2): Eq. 1 at theta with its marginal
    variances replaced by sigma2_hat(theta).  Returns (l, sigma2_hat)."""
    s2 = sigma2_hat(theta, locs, Z)
    r = loglik(Theta(s2, theta.a, theta.nu, theta.beta), locs, Z)
    return r.loglik, s2


def profile_theta_to_x(theta: Theta) -> np.ndarray:
    """Profile coordinates: (log a, log nu_i, beta_ij for i<j), the sigma^2 dropped."""
    return theta_to_x(theta)[theta.p:].copy()


def profile_x_to_theta(x, p: int) -> Theta:
    """Inverse of profile_theta_to_x with sigma^2 = 1 (replaced by sigma2_hat when evaluated)."""
    return x_to_theta(np.concatenate([np.zeros(p), np.asarray(x, dtype=np.float64)]), p)


def profile_objective(locs, Z, p: int):
    """f(x) = -l_profile(theta(x)) over the profile coordinates, +inf outside the
    feasible set (beta not PD, a Cholesky failure)."""
    def f(x):
        th = profile_x_to_theta(x, p)
        if not beta_is_pd(th.beta):
            return math.inf
        try:
            ll, _ = profile_loglik(th, locs, Z)
        except np.linalg.LinAlgError:
            return math.inf
        if not math.isfinite(ll):
            return math.inf
        return -ll
    return f


# ----------------------------------------------------------------------------
# TLR reference: exact truncated SVD ranks (Sec. 5.3, Fig. 5)
# ----------------------------------------------------------------------------

def tlr_reference_ranks(S: np.ndarray, nb: int, tol: float) -> np.ndarray:
    """Rank of every off-diagonal tile of the lower triangle: the number of
    singular values above the absolute threshold ``tol`` (exact SVD).  Entry
    (i, j), i > j; -1 elsewhere."""
    N = S.shape[0]
    T = (N + nb - 1) // nb
    R = -np.ones((T, T), dtype=np.int64)
    for i in range(T):
        for j in range(i):
            tile = S[i * nb:min(N, (i + 1) * nb), j * nb:min(N, (j + 1) * nb)]
            s = np.linalg.svd(tile, compute_uv=False)
            R[i, j] = int(np.sum(s > tol))
    return R


# ----------------------------------------------------------------------------
# Multivariate MLOE / MMOM (Eq. 5 - Eq. 8, Algorithm 1)
# ----------------------------------------------------------------------------

def mloe_mmom(theta_t: Theta, theta_a: Theta, locs, pred_locs):
    """Eq. 5 - Eq. 8 at every prediction location, following Algorithm 1:
    E_t  = tr{C(0; t) - c_t' S_t^-1 c_t}
    E_ta = tr{C(0; t) - 2 c_t' S_a^-1 c_a + c_a' S_a^-1 S_t S_a^-1 c_a}
    E_a  = tr{C(0; a) - c_a' S_a^-1 c_a}
    LOE = E_ta / E_t - 1,  MOM = E_a / E_ta - 1.
    Returns (MLOE, MMOM, per-location LOE, per-location MOM)."""
    locs = _f64(locs).reshape(-1, 2)
    pred_locs = _f64(pred_locs).reshape(-1, 2)
    St = covgen(theta_t, locs)
    Sa = covgen(theta_a, locs)
    Lt, it = cholesky(St)
    La, ia = cholesky(Sa)
    if it or ia:
        raise ValueError("Sigma not positive definite")
    loe, mom = [], []
    for l in range(pred_locs.shape[0]):
        s0 = pred_locs[l:l + 1]
        ct = covgen(theta_t, locs, s0)  # (pn) x p
        ca = covgen(theta_a, locs, s0)
        C0t = covgen(theta_t, s0)
        C0a = covgen(theta_a, s0)
        # S_a^-1 c_a and S_t^-1 c_t, column by column
        wa = np.column_stack([backward(La, forward(La, ca[:, k])) for k in range(ca.shape[1])])
        wt = np.column_stack([backward(Lt, forward(Lt, ct[:, k])) for k in range(ct.shape[1])])
        Et = float(np.trace(C0t - ct.T @ wt))
        Eta = float(np.trace(C0t - 2.0 * ct.T @ wa + wa.T @ (St @ wa)))
        Ea = float(np.trace(C0a - ca.T @ wa))
        loe.append(Eta / Et - 1.0)
        mom.append(Ea / Eta - 1.0)
    return float(np.mean(loe)), float(np.mean(mom)), np.array(loe), np.array(mom)
