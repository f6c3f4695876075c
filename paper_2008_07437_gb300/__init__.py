"""GB300 library for the multivariate Matern log-likelihood and cokriging of
arxiv 2008.07437 ("High Performance Multivariate Geospatial Statistics on
Manycore Systems").

The computation lives in ``libgeo.so`` (hand-written CUDA for sm_103a behind
the C ABI of ``include/geo.h``).  This module is the thin Python binding: the
functions carry the C names (``geo_loglik``, ``geo_predict``, ...) and only
marshal arguments -- torch tensors for device memory, torch streams for
ordering.  There is no CPU fallback: if the library is missing or no CUDA
device is present, every call raises.

``inputs`` (seeded synthetic workloads) does not load the library.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgeo.so")

GEO_OK, GEO_EINVAL, GEO_ENOTSPD, GEO_ENOMEM, GEO_ETIMEOUT, GEO_ECUDA, GEO_EUNSUPPORTED, GEO_ESCRATCH = range(8)
GEO_NOALLOC_MAX_N = 2048
GEO_PREC_FP64, GEO_PREC_MIXED, GEO_PREC_TLR = 0, 1, 2
GEO_PMAX = 4
GEO_MLE_QMAX = 16

_c_double_p = ctypes.POINTER(ctypes.c_double)


class geo_theta(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("sigma2", _c_double_p), ("nu", _c_double_p), ("beta", _c_double_p),
                ("a", ctypes.c_double)]


class geo_opts(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("prec", ctypes.c_int), ("band", ctypes.c_int), ("lowp", ctypes.c_int),
                ("refine_iters", ctypes.c_int), ("tlr_tol", ctypes.c_double), ("tlr_kmax", ctypes.c_int),
                ("morton", ctypes.c_int), ("fp64_gemm", ctypes.c_int), ("dst", ctypes.c_int),
                ("oz_slices", ctypes.c_int), ("oz_cut", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class geo_factor_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("p", ctypes.c_int), ("N", ctypes.c_int), ("nb", ctypes.c_int),
                ("prec", ctypes.c_int), ("loglik", ctypes.c_double), ("logdet", ctypes.c_double),
                ("quad", ctypes.c_double), ("device_bytes", ctypes.c_longlong),
                ("tlr_bytes_ratio", ctypes.c_double), ("tlr_max_rank", ctypes.c_int),
                ("tlr_dense_tiles", ctypes.c_int)]


class geo_mle_state(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("q", ctypes.c_int), ("iter", ctypes.c_int), ("evals", ctypes.c_int),
                ("initialized", ctypes.c_int), ("step", ctypes.c_double),
                ("x", (ctypes.c_double * GEO_MLE_QMAX) * (GEO_MLE_QMAX + 1)),
                ("f", ctypes.c_double * (GEO_MLE_QMAX + 1)), ("last_f", ctypes.c_double),
                ("profile", ctypes.c_int), ("s2", (ctypes.c_double * GEO_PMAX) * (GEO_MLE_QMAX + 1))]


GEO_K_NAMES = ["covgen", "potrf", "trsm", "gemm", "reduce", "solve", "predict", "aux", "tcgemm", "sgemm", "tlr"]
GEO_K_COUNT = len(GEO_K_NAMES)


class geo_batch_item(ctypes.Structure):
    _fields_ = [("locs_dev", ctypes.c_void_p), ("n", ctypes.c_int), ("z_dev", ctypes.c_void_p), ("theta", geo_theta)]


GEO_REQ_LOGLIK, GEO_REQ_PREDICT = 0, 1


class geo_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dataset", ctypes.c_longlong), ("keep", ctypes.c_int),
                ("release", ctypes.c_int), ("n", ctypes.c_int), ("locs_host", ctypes.c_void_p),
                ("z_host", ctypes.c_void_p), ("theta", geo_theta), ("opts", ctypes.c_void_p), ("m", ctypes.c_int),
                ("new_locs_host", ctypes.c_void_p), ("escalate", ctypes.c_int)]


class geo_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("dataset", ctypes.c_longlong), ("kind", ctypes.c_int),
                ("status", ctypes.c_int), ("loglik", ctypes.c_double), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_end", ctypes.c_double), ("prec", ctypes.c_int)]


class geo_kstat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double), ("timed", ctypes.c_longlong), ("tensor_flops", ctypes.c_double)]


# every symbol include/geo.h declares, with (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
_LL = ctypes.c_longlong
_D = ctypes.c_double
SIGNATURES = {
    "geo_opts_default": (None, [ctypes.POINTER(geo_opts)]),
    "geo_create": (_I, [ctypes.POINTER(_P), _I, ctypes.c_size_t]),
    "geo_destroy": (_I, [_P]),
    "geo_last_error": (ctypes.c_char_p, [_P]),
    "geo_covgen": (_I, [_P, _P, _I, _P, _I, ctypes.POINTER(geo_theta), _P, _LL, _P]),
    "geo_loglik": (_I, [_P, _P, _I, _P, ctypes.POINTER(geo_theta), ctypes.POINTER(geo_opts),
                        ctypes.POINTER(_D), ctypes.POINTER(_P), ctypes.POINTER(_I), _P]),
    "geo_predict": (_I, [_P, _P, _P, _I, _P, _P]),
    "geo_predict_batch": (_I, [_P, _I, _P, _P, _P, _P, _P]),
    "geo_simulate": (_I, [_P, _P, _I, _P, ctypes.POINTER(geo_theta), ctypes.POINTER(geo_opts), _P,
                          ctypes.POINTER(_I), _P]),
    "geo_factor_stats_get": (_I, [_P, ctypes.POINTER(geo_factor_stats)]),
    "geo_factor_read": (_I, [_P, _I, _LL, _LL, _LL, _LL, _P]),
    "geo_factor_free": (None, [_P]),
    "geo_morton_order": (_I, [_P, _I, _P]),
    "geo_abi_layout": (_I, [_P, _I]),
    "geo_mle_init": (_I, [ctypes.POINTER(geo_mle_state), ctypes.POINTER(geo_theta), _D]),
    "geo_mle_init_profile": (_I, [ctypes.POINTER(geo_mle_state), ctypes.POINTER(geo_theta), _D]),
    "geo_sigma2_hat": (_I, [_P, _P, _I, _P, ctypes.POINTER(geo_theta), ctypes.POINTER(geo_opts), _P,
                            ctypes.POINTER(_I), _P]),
    "geo_loglik_profile": (_I, [_P, _P, _I, _P, ctypes.POINTER(geo_theta), ctypes.POINTER(geo_opts), _P, _P,
                                ctypes.POINTER(_I), _P]),
    "geo_mle_step": (_I, [_P, ctypes.POINTER(geo_mle_state), _P, _I, _P, ctypes.POINTER(geo_opts), _P]),
    "geo_mle_best": (_I, [ctypes.POINTER(geo_mle_state), _P, _P, _P, _P, _P]),
    "geo_profile_enable": (_I, [_P, _I]),
    "geo_profile_read": (_I, [_P, ctypes.POINTER(geo_kstat)]),
    "geo_server_profile_read": (_I, [_P, ctypes.POINTER(geo_kstat)]),
    "geo_predict_var": (_I, [_P, _P, _P, _I, _P, _P]),
    "geo_mloe_mmom": (_I, [_P, _P, _I, _P, _I, ctypes.POINTER(geo_theta), ctypes.POINTER(geo_theta), _P, _P, _P, _P,
                           _P, _P]),
    "geo_loglik_noalloc": (_I, [_P, _I, _P, ctypes.POINTER(geo_theta), _I, _P, _P, _P]),
    "geo_loglik_batch": (_I, [_P, _I, _P, _P, _P, _P]),
    "geo_gemm_f64e": (_I, [_P, _I, _I, _I, _P, _LL, _P, _LL, _P, _LL, _I, _P]),
    "geo_selftest_bounded_wait": (_I, [_P, _I, _LL, ctypes.POINTER(_I), _P]),
    "geo_server_create": (_I, [ctypes.POINTER(_P), _I, ctypes.c_size_t, _I]),
    "geo_server_submit": (_I, [_P, _P, _P, ctypes.POINTER(_LL)]),
    "geo_server_poll": (_I, [_P, _P, _I, ctypes.POINTER(_I), _I]),
    "geo_server_pending": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_LL)]),
    "geo_server_destroy": (_I, [_P]),
    "geo_autotune_nb": (_I, [_P, _P, _I, _P, ctypes.POINTER(geo_theta), ctypes.POINTER(geo_opts), _P, _I,
                             ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
    "geo_autotune": (_I, [_P, _P, _I, _P, ctypes.POINTER(geo_theta), ctypes.POINTER(geo_opts), _P, _I, _P, _I, _I,
                          ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
}

_lib = None
_lib_lock = threading.Lock()


class GeoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("geo error %d: %s" % (code, msg))
        self.code = code


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libgeo.so (raises if it has not been built: there is no fallback)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("libgeo.so is not built (%s); run __graft_entry__.build() or "
                               "python -m paper_2008_07437_gb300.build" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


# ----------------------------------------------------------------------------
# argument marshalling
# ----------------------------------------------------------------------------

@dataclass
class Theta:
    """theta = (sigma^2_1..p, a, nu_1..p, beta) of Eq. 2 (Sec. 4.2)."""
    sigma2: tuple
    a: float
    nu: tuple
    beta: object = None  # p x p matrix, upper-triangle list, or scalar (p = 2)

    def beta_matrix(self) -> np.ndarray:
        p = len(self.sigma2)
        b = np.eye(p)
        if self.beta is None:
            return b
        arr = np.asarray(self.beta, dtype=np.float64)
        if arr.ndim == 0:
            b[0, 1] = b[1, 0] = float(arr)
        elif arr.ndim == 1:
            k = 0
            for i in range(p):
                for j in range(i + 1, p):
                    b[i, j] = b[j, i] = arr[k]
                    k += 1
        else:
            b = arr.copy()
        return b

    def to_c(self):
        p = len(self.sigma2)
        keep = (np.ascontiguousarray(self.sigma2, dtype=np.float64),
                np.ascontiguousarray(self.nu, dtype=np.float64),
                np.ascontiguousarray(self.beta_matrix(), dtype=np.float64).reshape(-1))
        th = geo_theta(p, keep[0].ctypes.data_as(_c_double_p), keep[1].ctypes.data_as(_c_double_p),
                       keep[2].ctypes.data_as(_c_double_p), float(self.a))
        return th, keep

    @staticmethod
    def from_spec(spec) -> "Theta":
        return Theta(tuple(spec.sigma2), spec.a, tuple(spec.nu), tuple(spec.beta))


def opts(**kw) -> geo_opts:
    o = geo_opts()
    load_library().geo_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _dev_ptr(t, name, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA torch tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """Owns a geo_ctx (device workspaces, kept factors)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.lib = load_library()
        h = ctypes.c_void_p()
        rc = self.lib.geo_create(ctypes.byref(h), int(device), int(hbm_budget_bytes))
        if rc != GEO_OK:
            raise GeoError(rc, "geo_create failed on device %d" % device)
        self.handle = h
        self.device = device

    def check(self, rc: int):
        if rc != GEO_OK:
            raise GeoError(rc, self.lib.geo_last_error(self.handle).decode())

    def close(self):
        if self.handle:
            self.lib.geo_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Factor:
    def __init__(self, ctx: Context, handle):
        self.ctx, self.handle = ctx, handle

    def free(self):
        if self.handle:
            self.ctx.lib.geo_factor_free(self.handle)
            self.handle = None


def geo_create(device: int = 0, hbm_budget_bytes: int = 0) -> Context:
    return Context(device, hbm_budget_bytes)


def geo_covgen(ctx: Context, locs1, theta: Theta, out, locs2=None, ld: int | None = None, stream=None):
    """Eq. 2 cross-covariance in Representation I, column-major into ``out``."""
    import torch
    th, _keep = theta.to_c()
    n1 = locs1.shape[0]
    n2 = locs2.shape[0] if locs2 is not None else n1
    p = len(theta.sigma2)
    ld = ld if ld is not None else p * n1
    l2 = _dev_ptr(locs2, "locs2", torch.float64) if locs2 is not None else None
    ctx.check(ctx.lib.geo_covgen(ctx.handle, _dev_ptr(locs1, "locs1", torch.float64), n1, l2, n2,
                                 ctypes.byref(th), _dev_ptr(out, "out", torch.float64), ld, _stream(stream)))
    return out


def geo_loglik(ctx: Context, locs, z, theta: Theta, options: geo_opts | None = None, keep: bool = False,
               stream=None):
    """Eq. 1 on the device.  Returns (loglik, Factor or None)."""
    import torch
    th, _keep = theta.to_c()
    val = ctypes.c_double()
    fac = ctypes.c_void_p()
    info = ctypes.c_int()
    rc = ctx.lib.geo_loglik(ctx.handle, _dev_ptr(locs, "locs", torch.float64), locs.shape[0],
                            _dev_ptr(z, "z", torch.float64), ctypes.byref(th),
                            ctypes.byref(options) if options is not None else None, ctypes.byref(val),
                            ctypes.byref(fac) if keep else None, ctypes.byref(info), _stream(stream))
    if rc == GEO_ENOTSPD:
        err = GeoError(rc, ctx.lib.geo_last_error(ctx.handle).decode())
        err.info = info.value
        raise err
    ctx.check(rc)
    return val.value, (Factor(ctx, fac) if keep else None)


def _raise_info(ctx: Context, rc: int, info: ctypes.c_int):
    if rc == GEO_ENOTSPD:
        err = GeoError(rc, ctx.lib.geo_last_error(ctx.handle).decode())
        err.info = info.value
        raise err
    ctx.check(rc)


def geo_sigma2_hat(ctx: Context, locs, z, theta: Theta, options: geo_opts | None = None, stream=None) -> np.ndarray:
    """Sec. 4.2 marginal variances n^-1 Z_i' R_ii^-1 Z_i (theta's sigma^2 and beta unused)."""
    import torch
    th, _keep = theta.to_c()
    out = np.zeros(len(theta.sigma2))
    info = ctypes.c_int()
    rc = ctx.lib.geo_sigma2_hat(ctx.handle, _dev_ptr(locs, "locs", torch.float64), locs.shape[0],
                                _dev_ptr(z, "z", torch.float64), ctypes.byref(th),
                                ctypes.byref(options) if options is not None else None,
                                out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info), _stream(stream))
    _raise_info(ctx, rc, info)
    return out


def geo_loglik_profile(ctx: Context, locs, z, theta: Theta, options: geo_opts | None = None, stream=None):
    """Profile log-likelihood (Sec. 4.2).  Returns (loglik, sigma2_hat)."""
    import torch
    th, _keep = theta.to_c()
    val = ctypes.c_double()
    s2 = np.zeros(len(theta.sigma2))
    info = ctypes.c_int()
    rc = ctx.lib.geo_loglik_profile(ctx.handle, _dev_ptr(locs, "locs", torch.float64), locs.shape[0],
                                    _dev_ptr(z, "z", torch.float64), ctypes.byref(th),
                                    ctypes.byref(options) if options is not None else None, ctypes.byref(val),
                                    s2.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info), _stream(stream))
    _raise_info(ctx, rc, info)
    return val.value, s2


def geo_predict(ctx: Context, factor: Factor, new_locs, zhat, stream=None):
    """Eq. 3 / Eq. 4 cokriging at ``new_locs`` into ``zhat`` (p*m, Rep. I)."""
    import torch
    ctx.check(ctx.lib.geo_predict(ctx.handle, factor.handle, _dev_ptr(new_locs, "new_locs", torch.float64),
                                  new_locs.shape[0], _dev_ptr(zhat, "zhat", torch.float64), _stream(stream)))
    return zhat


def geo_predict_batch(ctx: Context, entries, stream=None):
    """Cokriging on many kept factors in one launch: entries = [(factor, new_locs, zhat), ...]."""
    import torch
    count = len(entries)
    facs = (ctypes.c_void_p * count)(*[f.handle.value if isinstance(f.handle, ctypes.c_void_p) else f.handle
                                       for f, _, _ in entries])
    locs = (ctypes.c_void_p * count)(*[_dev_ptr(l, "new_locs", torch.float64).value for _, l, _ in entries])
    ms = (ctypes.c_int * count)(*[l.shape[0] for _, l, _ in entries])
    outs = (ctypes.c_void_p * count)(*[_dev_ptr(z, "zhat", torch.float64).value for _, _, z in entries])
    ctx.check(ctx.lib.geo_predict_batch(ctx.handle, count, facs, locs, ms, outs, _stream(stream)))
    return [z for _, _, z in entries]


def geo_simulate(ctx: Context, locs, e, theta: Theta, out, options: geo_opts | None = None, stream=None):
    """Z = L e (L L' = Sigma(theta)) into ``out``."""
    import torch
    th, _keep = theta.to_c()
    info = ctypes.c_int()
    ctx.check(ctx.lib.geo_simulate(ctx.handle, _dev_ptr(locs, "locs", torch.float64), locs.shape[0],
                                   _dev_ptr(e, "e", torch.float64), ctypes.byref(th),
                                   ctypes.byref(options) if options is not None else None,
                                   _dev_ptr(out, "out", torch.float64), ctypes.byref(info), _stream(stream)))
    return out


def geo_factor_stats_get(factor: Factor) -> geo_factor_stats:
    st = geo_factor_stats()
    factor.ctx.check(factor.ctx.lib.geo_factor_stats_get(factor.handle, ctypes.byref(st)))
    return st


def geo_factor_read(factor: Factor, what: int, r0: int, r1: int, c0: int = 0, c1: int = 0) -> np.ndarray:
    """Modes 0 (block of L), 1 (y = L^-1 Z), 2 (permutation), 3 (TLR ranks); see geo_tlr_tile for 4-6."""
    n = (r1 - r0) * (c1 - c0) if what == 0 else (r1 - r0)
    out = np.zeros(max(n, 1), dtype=np.float64)
    factor.ctx.check(factor.ctx.lib.geo_factor_read(factor.handle, what, r0, r1, c0, c1,
                                                    out.ctypes.data_as(ctypes.c_void_p)))
    out = out[:n]
    return out.reshape(r1 - r0, c1 - c0) if what == 0 else out


def geo_factor_free(factor: Factor):
    factor.free()


def geo_morton_order(locs) -> np.ndarray:
    """Host Morton permutation (internal position k holds caller location perm[k])."""
    locs = np.ascontiguousarray(locs, dtype=np.float64)
    n = locs.shape[0]
    perm = np.zeros(max(n, 1), dtype=np.int32)
    rc = load_library().geo_morton_order(locs.ctypes.data_as(ctypes.c_void_p), n, perm.ctypes.data_as(ctypes.c_void_p))
    if rc != GEO_OK:
        raise GeoError(rc, "geo_morton_order")
    return perm[:n].astype(np.int64)


def geo_mle_init(theta0: Theta, step: float = 0.1, profile: bool = False) -> geo_mle_state:
    """Nelder-Mead state at theta0; ``profile`` runs it over the profile likelihood (Sec. 4.2)."""
    st = geo_mle_state()
    th, _keep = theta0.to_c()
    name = "geo_mle_init_profile" if profile else "geo_mle_init"
    rc = getattr(load_library(), name)(ctypes.byref(st), ctypes.byref(th), float(step))
    if rc != GEO_OK:
        raise GeoError(rc, name)
    return st


def geo_mle_step(ctx: Context, state: geo_mle_state, locs, z, options: geo_opts | None = None, stream=None):
    import torch
    ctx.check(ctx.lib.geo_mle_step(ctx.handle, ctypes.byref(state), _dev_ptr(locs, "locs", torch.float64),
                                   locs.shape[0], _dev_ptr(z, "z", torch.float64),
                                   ctypes.byref(options) if options is not None else None, _stream(stream)))
    return state


def geo_mle_best(state: geo_mle_state):
    p = state.p
    s2 = np.zeros(p)
    nu = np.zeros(p)
    beta = np.zeros(p * p)
    a = ctypes.c_double()
    ll = ctypes.c_double()
    rc = load_library().geo_mle_best(ctypes.byref(state), s2.ctypes.data_as(ctypes.c_void_p), ctypes.byref(a),
                                     nu.ctypes.data_as(ctypes.c_void_p), beta.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(ll))
    if rc != GEO_OK:
        raise GeoError(rc, "geo_mle_best")
    return Theta(tuple(s2), a.value, tuple(nu), beta.reshape(p, p)), ll.value


def geo_profile_enable(ctx: Context, enable: bool = True):
    """Clear the per-kernel-class counters and (stop) recording CUDA events around launches."""
    ctx.check(ctx.lib.geo_profile_enable(ctx.handle, 1 if enable else 0))


def geo_profile_read(ctx: Context) -> dict:
    """{class: {launches, ms, flops, bytes, timed}} for every kernel class."""
    arr = (geo_kstat * GEO_K_COUNT)()
    ctx.check(ctx.lib.geo_profile_read(ctx.handle, arr))
    return {GEO_K_NAMES[k]: dict(launches=arr[k].launches, ms=arr[k].ms, flops=arr[k].flops,
                                 bytes=arr[k].bytes, timed=arr[k].timed, tensor_flops=arr[k].tensor_flops) for k in range(GEO_K_COUNT)}


def _check_noalloc_args(locs, z, theta: Theta, out, info) -> int:
    """Shapes, dtypes and placement of geo_loglik_noalloc's tensors (raises before anything runs)."""
    import torch
    p = len(theta.sigma2)
    named = [("locs", locs, torch.float64), ("z", z, torch.float64), ("out", out, torch.float64)]
    if info is not None:
        named.append(("info", info, torch.int32))
    for name, t, dt in named:
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s must be a torch tensor" % name)
        if t.dtype != dt:
            raise TypeError("%s must be %s" % (name, dt))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    if locs.dim() != 2 or locs.shape[1] != 2:
        raise ValueError("locs must be n x 2")
    n = locs.shape[0]
    if z.numel() != p * n:
        raise ValueError("z must hold p * n = %d values" % (p * n))
    if out.numel() < 3:
        raise ValueError("out must hold 3 doubles")
    if info is not None and info.numel() < 1:
        raise ValueError("info must hold one int")
    if len({t.device for _, t, _ in named}) != 1:
        raise ValueError("locs, z, out and info must be on one device")
    if not locs.is_cuda:
        raise TypeError("geo_loglik_noalloc needs CUDA tensors")
    return n


def geo_loglik_noalloc(locs, z, theta: Theta, out, info=None, nb: int = 960, stream=None) -> int:
    """Eq. 1 without any device allocation (fixed library-owned scratch, p*n <= GEO_NOALLOC_MAX_N).
    ``out`` (3 doubles) and ``info`` (1 int32, optional) are device tensors written asynchronously on
    the stream; returns the status code (GEO_OK, GEO_ESCRATCH, ...) without raising.  The tensors must
    share one device; the call runs with that device current."""
    import torch
    n = _check_noalloc_args(locs, z, theta, out, info)
    th, _keep = theta.to_c()
    with torch.cuda.device(locs.device):
        return load_library().geo_loglik_noalloc(
            ctypes.c_void_p(locs.data_ptr()), n, ctypes.c_void_p(z.data_ptr()), ctypes.byref(th), int(nb),
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(info.data_ptr()) if info is not None else None,
            _stream(stream))


def geo_gemm_f64e(ctx: Context, A, B, C, slices: int = 0, stream=None):
    """C -= A @ B.T on the tensor cores with FP64-class accuracy (``slices`` 7-bit digits per operand).
    A (m x k), B (n x k), C (m x n): float64 CUDA tensors in column-major storage, i.e. the
    transposes ``X.t()`` of contiguous row-major tensors are passed as ``X``."""
    import torch
    for name, t in (("A", A), ("B", B), ("C", C)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or t.dim() != 2:
            raise TypeError("%s must be a 2-D float64 CUDA tensor" % name)
        if t.stride(0) != 1 or t.stride(1) < max(1, t.shape[0]):
            raise ValueError("%s must be column-major (stride(0) == 1)" % name)
        if t.device != A.device:
            raise ValueError("A, B and C must be on one device")
    m, k = A.shape
    n = B.shape[0]
    if B.shape[1] != k or tuple(C.shape) != (m, n):
        raise ValueError("shapes: A (m, k), B (n, k), C (m, n)")
    with torch.cuda.device(A.device):
        ctx.check(ctx.lib.geo_gemm_f64e(ctx.handle, m, n, k, ctypes.c_void_p(A.data_ptr()), max(1, A.stride(1)),
                                        ctypes.c_void_p(B.data_ptr()), max(1, B.stride(1)),
                                        ctypes.c_void_p(C.data_ptr()), max(1, C.stride(1)), int(slices),
                                        _stream(stream)))
    return C


def geo_selftest_bounded_wait(ctx: Context, n_blocks: int = 8, wait_cycles: int = 2_000_000, stream=None):
    """Run the forward solve with a withheld dependency and a short wait budget.
    Returns (status code, wait site); GEO_ETIMEOUT with site 3 is the expected outcome."""
    site = ctypes.c_int()
    rc = ctx.lib.geo_selftest_bounded_wait(ctx.handle, int(n_blocks), int(wait_cycles), ctypes.byref(site),
                                           _stream(stream))
    return rc, site.value


def geo_tlr_tile(factor: Factor, i: int, j: int, which: str = "U") -> np.ndarray:
    """A tile of a TLR factor: "U" / "V" of the off-diagonal tile (i, j), i > j
    (columns = rank), or "D" for the diagonal tile i of L."""
    st = geo_factor_stats_get(factor)
    nb, N = st.nb, st.N
    mt = lambda t: min(nb, N - t * nb)
    if which == "D":
        m = mt(i)
        out = np.zeros(m * m)
        factor.ctx.check(factor.ctx.lib.geo_factor_read(factor.handle, 6, i, i + 1, 0, 0,
                                                        out.ctypes.data_as(ctypes.c_void_p)))
        return out.reshape(m, m, order="F")
    r = int(geo_factor_read(factor, 3, i, i + 1, j, j + 1)[0])
    m = mt(i) if which == "U" else mt(j)
    out = np.zeros(max(m * r, 1))
    factor.ctx.check(factor.ctx.lib.geo_factor_read(factor.handle, 4 if which == "U" else 5, i, i + 1, j, j + 1,
                                                    out.ctypes.data_as(ctypes.c_void_p)))
    return out[:m * r].reshape(m, r, order="F")


def geo_tlr_ranks(factor: Factor) -> np.ndarray:
    """T x T matrix of off-diagonal tile ranks (-1 on and above the diagonal)."""
    st = geo_factor_stats_get(factor)
    T = (st.N + st.nb - 1) // st.nb
    R = -np.ones((T, T), dtype=np.int64)
    for j in range(T):
        R[:, j] = geo_factor_read(factor, 3, 0, T, j, j + 1).astype(np.int64)
    return R


def geo_loglik_batch(ctx: Context, problems, stream=None):
    """Eq. 1 for a list of (locs, z, theta) small problems in one batched launch sequence.
    Returns (loglik array, info array)."""
    import torch
    count = len(problems)
    items = (geo_batch_item * count)()
    keep = []
    for k, (locs, z, theta) in enumerate(problems):
        th, kk = theta.to_c()
        keep.append(kk)
        items[k].locs_dev = _dev_ptr(locs, "locs", torch.float64).value
        items[k].n = locs.shape[0]
        items[k].z_dev = _dev_ptr(z, "z", torch.float64).value
        items[k].theta = th
    out = np.zeros(count)
    info = np.zeros(count, dtype=np.int32)
    ctx.check(ctx.lib.geo_loglik_batch(ctx.handle, count, items, out.ctypes.data_as(ctypes.c_void_p),
                                       info.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return out, info


class Server:
    """geo_server: continuous admission of likelihood / cokriging requests (host inputs, copied at submit)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, slots: int = 4):
        self.lib = load_library()
        h = ctypes.c_void_p()
        rc = self.lib.geo_server_create(ctypes.byref(h), device, int(hbm_budget_bytes), int(slots))
        if rc != GEO_OK:
            raise GeoError(rc, "geo_server_create")
        self.handle = h
        self._keep = {}   # request id -> host buffers kept alive until the result is polled

    def submit_loglik(self, locs, z, theta: Theta, options: geo_opts | None = None, dataset: int = 0,
                      keep: bool = False, escalate: bool = False) -> int:
        locs = np.ascontiguousarray(locs, dtype=np.float64)
        z = np.ascontiguousarray(z, dtype=np.float64)
        th, kk = theta.to_c()
        req = geo_request(GEO_REQ_LOGLIK, int(dataset), int(keep), 0, locs.shape[0], locs.ctypes.data, z.ctypes.data,
                          th, ctypes.addressof(options) if options is not None else None, 0, None, int(escalate))
        rid = ctypes.c_longlong()
        rc = self.lib.geo_server_submit(self.handle, ctypes.byref(req), None, ctypes.byref(rid))
        if rc != GEO_OK:
            raise GeoError(rc, "geo_server_submit")
        self._keep[rid.value] = (locs, z, kk, options)
        return rid.value

    def submit_predict(self, dataset: int, new_locs, p: int, release: bool = False):
        new_locs = np.ascontiguousarray(new_locs, dtype=np.float64)
        out = np.zeros(p * new_locs.shape[0])
        req = geo_request(GEO_REQ_PREDICT, int(dataset), 0, int(release), 0, None, None, geo_theta(), None,
                          new_locs.shape[0], new_locs.ctypes.data, 0)
        rid = ctypes.c_longlong()
        rc = self.lib.geo_server_submit(self.handle, ctypes.byref(req), out.ctypes.data_as(ctypes.c_void_p),
                                        ctypes.byref(rid))
        if rc != GEO_OK:
            raise GeoError(rc, "geo_server_submit")
        self._keep[rid.value] = (new_locs, out)
        return rid.value, out

    def poll(self, max_results: int = 256, wait_ms: int = 0):
        arr = (geo_result * max_results)()
        n = ctypes.c_int()
        rc = self.lib.geo_server_poll(self.handle, arr, max_results, ctypes.byref(n), int(wait_ms))
        if rc != GEO_OK:
            raise GeoError(rc, "geo_server_poll")
        out = []
        for k in range(n.value):
            r = arr[k]
            out.append(dict(id=r.id, dataset=r.dataset, kind=r.kind, status=r.status, loglik=r.loglik,
                            t_submit=r.t_submit, t_start=r.t_start, t_end=r.t_end, prec=r.prec))
            self._keep.pop(r.id, None)
        return out

    def pending(self):
        q, f, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        self.lib.geo_server_pending(self.handle, ctypes.byref(q), ctypes.byref(f), ctypes.byref(b))
        return q.value, f.value, b.value

    def profile(self) -> dict:
        """Kernel counters summed over the workers (call when nothing is queued or running)."""
        arr = (geo_kstat * GEO_K_COUNT)()
        rc = self.lib.geo_server_profile_read(self.handle, arr)
        if rc != GEO_OK:
            raise GeoError(rc, "geo_server_profile_read")
        return {GEO_K_NAMES[k]: dict(launches=arr[k].launches, ms=arr[k].ms, flops=arr[k].flops,
                                     bytes=arr[k].bytes) for k in range(GEO_K_COUNT)}

    def close(self):
        if self.handle:
            self.lib.geo_server_destroy(self.handle)
            self.handle = None


def geo_predict_var(ctx: Context, factor: "Factor", new_locs, out, stream=None):
    """Prediction variances diag(C(0) - c0' Sigma^-1 c0) at new_locs into out (p m doubles, device)."""
    import torch
    ctx.check(ctx.lib.geo_predict_var(ctx.handle, factor.handle, _dev_ptr(new_locs, "new_locs", torch.float64),
                                      new_locs.shape[0], _dev_ptr(out, "out", torch.float64), _stream(stream)))
    return out


def geo_mloe_mmom(ctx: Context, locs, pred, theta_t: Theta, theta_a: Theta, options: geo_opts | None = None,
                  stream=None):
    """MLOE, MMOM and the per-location LOE / MOM of Eq. 5 - Eq. 8 (Algorithm 1)."""
    import torch
    tt, _k1 = theta_t.to_c()
    ta, _k2 = theta_a.to_c()
    m = pred.shape[0]
    loe = np.zeros(m)
    mom = np.zeros(m)
    ml = ctypes.c_double()
    mm = ctypes.c_double()
    ctx.check(ctx.lib.geo_mloe_mmom(ctx.handle, _dev_ptr(locs, "locs", torch.float64), locs.shape[0],
                                    _dev_ptr(pred, "pred", torch.float64), m, ctypes.byref(tt), ctypes.byref(ta),
                                    ctypes.byref(options) if options is not None else None, ctypes.byref(ml),
                                    ctypes.byref(mm), loe.ctypes.data_as(ctypes.c_void_p),
                                    mom.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return ml.value, mm.value, loe, mom


def geo_autotune_nb(ctx: Context, locs, z, theta: Theta, candidates, options: geo_opts | None = None, stream=None):
    """Fastest tile size among ``candidates`` on this problem (cached in the context for nb = 0)."""
    import torch
    th, _keep = theta.to_c()
    cand = (ctypes.c_int * len(candidates))(*candidates)
    best = ctypes.c_int()
    ms = ctypes.c_double()
    ctx.check(ctx.lib.geo_autotune_nb(ctx.handle, _dev_ptr(locs, "locs", torch.float64), locs.shape[0],
                                      _dev_ptr(z, "z", torch.float64), ctypes.byref(th),
                                      ctypes.byref(options) if options is not None else None, cand, len(candidates),
                                      ctypes.byref(best), ctypes.byref(ms), _stream(stream)))
    return best.value, ms.value


def geo_autotune(ctx: Context, locs, z, theta: Theta, nb_candidates, band_candidates=(), samples: int = 3,
                 options: geo_opts | None = None, stream=None):
    """Fastest (nb, band) on this problem (band only in the mixed form, else -1); median of ``samples``
    timed evaluations per candidate.  Cached process-wide for nb = 0.  Returns (nb, band, ms)."""
    import torch
    th, _keep = theta.to_c()
    nbc = (ctypes.c_int * len(nb_candidates))(*nb_candidates)
    bc = (ctypes.c_int * max(1, len(band_candidates)))(*band_candidates) if band_candidates else None
    bnb, bband, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    ctx.check(ctx.lib.geo_autotune(ctx.handle, _dev_ptr(locs, "locs", torch.float64), locs.shape[0],
                                   _dev_ptr(z, "z", torch.float64), ctypes.byref(th),
                                   ctypes.byref(options) if options is not None else None, nbc, len(nb_candidates),
                                   bc, len(band_candidates), int(samples), ctypes.byref(bnb), ctypes.byref(bband),
                                   ctypes.byref(ms), _stream(stream)))
    return bnb.value, bband.value, ms.value
