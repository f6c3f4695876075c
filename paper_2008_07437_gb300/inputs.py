"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds none of the likelihood's arithmetic: it only draws random
numbers and lays out locations.  It imports nothing from the rest of the
package, so the oracle-side tests can use it without loading the CUDA library.

* ``splitmix64`` / ``uniforms`` / ``normals``: a counter-based generator
  (SplitMix64: Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014) mapped to 53-bit uniforms in [0, 1) and to
  standard normals by the Box-Muller transform.
* ``jittered_grid``: n locations on [0, 1]^2, one per cell of an m x m grid
  (m = ceil(sqrt(n))), each jittered uniformly by up to +-0.4 cell, cells chosen
  by a seeded Fisher-Yates shuffle.  This stands in for the paper's synthetic
  irregular locations (Sec. 6.4.1); the paper's real WRF dataset is not used.
* ``Workload``: the workloads the paper's experiments are shaped like.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of the SplitMix64 sequence started at ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """53-bit uniforms in [0, 1)."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normals(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on pairs of uniforms (u1 in (0, 1])."""
    npair = (count + 1) // 2
    u = uniforms(seed, 2 * npair)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npair)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


def jittered_grid(n: int, seed: int, jitter: float = 0.4) -> np.ndarray:
    """n x 2 locations on [0,1]^2: cell (i, j) of an m x m grid gives
    ((i + 1/2 + u)/m, (j + 1/2 + v)/m), u, v ~ U(-jitter, jitter); the first n
    cells of a seeded Fisher-Yates permutation are kept (all of them when n = m^2)."""
    if n <= 0:
        return np.zeros((0, 2))
    m = int(math.ceil(math.sqrt(n)))
    cells = np.arange(m * m, dtype=np.int64)
    u = uniforms(seed, m * m)
    for k in range(m * m - 1, 0, -1):  # Fisher-Yates, j uniform in [0, k]
        j = int(u[k] * (k + 1))
        cells[k], cells[j] = cells[j], cells[k]
    cells = cells[:n]
    jit = uniforms(seed ^ 0x5DEECE66D, 2 * n)
    ix = (cells % m).astype(np.float64)
    iy = (cells // m).astype(np.float64)
    x = (ix + 0.5 + (2.0 * jit[0::2] - 1.0) * jitter) / m
    y = (iy + 0.5 + (2.0 * jit[1::2] - 1.0) * jitter) / m
    return np.ascontiguousarray(np.stack([x, y], axis=1))


@dataclass
class ThetaSpec:
    """theta = (sigma^2_1..p, a, nu_1..p, beta_ij for i < j) (Sec. 4.2)."""
    sigma2: tuple
    a: float
    nu: tuple
    beta: tuple  # upper-triangle list b12, b13, ..., b23, ...

    @property
    def p(self) -> int:
        return len(self.sigma2)

    def beta_matrix(self) -> np.ndarray:
        p = self.p
        b = np.eye(p)
        k = 0
        for i in range(p):
            for j in range(i + 1, p):
                b[i, j] = b[j, i] = self.beta[k]
                k += 1
        return b


@dataclass
class Workload:
    name: str
    n: int
    theta: ThetaSpec
    n_pred: int = 0
    nb: int = 960
    loc_seed: int = 1000
    z_seed: int = 2000
    extra: dict = field(default_factory=dict)   # factorisation options (prec, band, lowp, refine_iters, ...)

    def locations(self) -> tuple[np.ndarray, np.ndarray]:
        """(observed n x 2, held-out n_pred x 2), drawn jointly then split."""
        allp = jittered_grid(self.n + self.n_pred, self.loc_seed)
        return allp[: self.n].copy(), allp[self.n:].copy()

    def white_noise(self) -> np.ndarray:
        """Standard normals e for the joint draw Z = L e (observed + held out)."""
        return normals(self.z_seed, self.theta.p * (self.n + self.n_pred))


# The paper's bivariate example (Fig. 5 / Sec. 5.3): theta = (1, 1, 0.09, 0.5, 1, 0.5).
THETA_FIG5 = ThetaSpec(sigma2=(1.0, 1.0), a=0.09, nu=(0.5, 1.0), beta=(0.5,))

WORKLOADS = {
    # 400 locations on a jittered 20 x 20 grid, N = 800, plain dense FP64.
    "bivariate-n400": Workload("bivariate-n400", 400, THETA_FIG5, nb=128, loc_seed=1000, z_seed=2000),
    # 20,000 locations (N = 40,000), dense FP64 tiled Cholesky, 2,000 held-out locations to
    # predict; the trailing updates and panel solves emulated on the tensor cores with 8 digit
    # slices (FP64-class accuracy), tile 512, with the magnitude-aware level cut.
    "bivariate-n20000": Workload("bivariate-n20000", 20000,
                                 ThetaSpec((1.0, 1.0), 0.03, (0.5, 1.5), (0.5,)),
                                 n_pred=2000, nb=512, loc_seed=1001, z_seed=2001,
                                 extra={"fp64_gemm": 1, "oz_slices": 8, "oz_cut": 1}),
    # The same with native FP64 FMA updates, tile 960.
    "bivariate-n20000-native": Workload("bivariate-n20000-native", 20000,
                                        ThetaSpec((1.0, 1.0), 0.03, (0.5, 1.5), (0.5,)),
                                        n_pred=2000, nb=960, loc_seed=1001, z_seed=2001),
    # 50,000 locations (N = 100,000), reduced precision: FP64 diagonal tiles, BF16 tensor cores
    # with a power-of-two scale per row and FP32 accumulation for every other tile, as 5 digit
    # slices (about 35 bits per operand), with the magnitude-aware level cut.
    "bivariate-n50000-mixed": Workload("bivariate-n50000-mixed", 50000,
                                       ThetaSpec((1.0, 1.0), 0.1, (0.5, 1.0), (0.7,)),
                                       nb=768, loc_seed=1002, z_seed=2002,
                                       extra={"fp64_gemm": 1, "oz_slices": 5, "oz_cut": 1}),
    # The FP32-class mixed form: FP64 diagonal tiles, FP32 band of 4 tiles, FP16 x 2 tensor cores
    # beyond, 2 refinement sweeps.
    "bivariate-n50000-fp16x2": Workload("bivariate-n50000-fp16x2", 50000,
                                        ThetaSpec((1.0, 1.0), 0.1, (0.5, 1.0), (0.7,)),
                                        nb=1024, loc_seed=1002, z_seed=2002,
                                        extra={"prec": 1, "band": 4, "lowp": 0, "refine_iters": 2}),
    # 60,000 locations, trivariate (N = 180,000), tile low-rank at accuracy 1e-9, rank <= 200.
    "trivariate-n60000-tlr": Workload("trivariate-n60000-tlr", 60000,
                                      ThetaSpec((1.0, 1.0, 1.0), 0.05, (0.5, 1.0, 1.5), (0.5, 0.3, 0.4)),
                                      nb=1800, loc_seed=1003, z_seed=2003,
                                      extra={"prec": 2, "tlr_tol": 1e-9, "tlr_kmax": 200}),
}


@dataclass
class ServingRequest:
    """One request of a serving stream.  kind: "loglik" or "predict"."""
    k: int
    t_arrival: float          # seconds after the stream starts
    kind: str
    n: int = 0                # loglik: locations (bivariate, N = 2 n)
    theta: ThetaSpec | None = None
    dataset: int = 0          # key of the factor a loglik keeps / a predict reuses
    keep: bool = False
    release: bool = False
    m: int = 0                # predict: new locations

    def locations(self) -> np.ndarray:
        return jittered_grid(self.n, 30000 + self.k)

    def observations(self) -> np.ndarray:
        """Z for a loglik request: seeded standard normals (the evaluation's
        cost does not depend on Z's values)."""
        return normals(40000 + self.k, 2 * self.n)

    def new_locations(self) -> np.ndarray:
        return jittered_grid(self.m, 50000 + self.k)


def serving_stream(count: int, rate: float = 200.0, seed: int = 3000, n_lo: int = 1000, n_hi: int = 20000,
                   m_lo: int = 100, m_hi: int = 2000, p_loglik: float = 0.7) -> list[ServingRequest]:
    """A seeded Poisson stream of bivariate requests: exponential gaps of mean
    1/rate; a fraction p_loglik of likelihood evaluations with n uniform in
    [n_lo, n_hi] at a random theta (a in [0.03, 0.2], nu_i in [0.5, 1.5],
    beta in [-0.7, 0.7], sigma^2_i in [0.5, 2]); the rest cokriging requests
    of m uniform in [m_lo, m_hi] new locations on the factor of the latest
    likelihood request, which then keeps its factor; the last request on a
    factor releases it.  A cokriging request with no likelihood before it
    becomes a likelihood request."""
    U = uniforms(seed, 10 * count).reshape(count, 10)
    out: list[ServingRequest] = []
    t = 0.0
    last_ll = None
    for k in range(count):
        u = U[k]
        t += -math.log1p(-u[0]) / rate
        if u[1] < p_loglik or last_ll is None:
            th = ThetaSpec(sigma2=(0.5 + 1.5 * u[3], 0.5 + 1.5 * u[4]), a=0.03 + 0.17 * u[5],
                           nu=(0.5 + u[6], 0.5 + u[7]), beta=(-0.7 + 1.4 * u[8],))
            r = ServingRequest(k, t, "loglik", n=n_lo + int(u[2] * (n_hi - n_lo + 1)), theta=th, dataset=k)
            last_ll = r
        else:
            last_ll.keep = True
            r = ServingRequest(k, t, "predict", dataset=last_ll.dataset, m=m_lo + int(u[9] * (m_hi - m_lo + 1)))
        out.append(r)
    last_use = {}
    for r in out:
        if r.kind == "predict":
            last_use[r.dataset] = r
    for r in last_use.values():
        r.release = True
    return out


def batch_problems(count: int, seed: int = 3100, n_lo: int = 50, n_hi: int = 1000) -> list[tuple]:
    """count bivariate likelihood problems of uneven size for the batched
    path: (n, theta, location seed, noise seed) with n uniform in [n_lo, n_hi]
    and theta drawn from the serving box (a in [0.03, 0.2], nu_i in [0.5, 1.5],
    beta in [-0.7, 0.7], sigma^2_i in [0.5, 2])."""
    U = uniforms(seed, 8 * count).reshape(count, 8)
    out = []
    for k in range(count):
        u = U[k]
        th = ThetaSpec(sigma2=(0.5 + 1.5 * u[1], 0.5 + 1.5 * u[2]), a=0.03 + 0.17 * u[3],
                       nu=(0.5 + u[4], 0.5 + u[5]), beta=(-0.7 + 1.4 * u[6],))
        out.append((n_lo + int(u[0] * (n_hi - n_lo + 1)), th, seed * 10 + 2 * k, seed * 10 + 2 * k + 1))
    return out
