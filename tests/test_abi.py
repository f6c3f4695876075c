"""The C ABI library loads without a GPU and exports every symbol that
include/geo.h declares; host-side logic (Morton order, options, simplex
set-up) runs without a device and agrees with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2008_07437_gb300 as geo
from paper_2008_07437_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "geo.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(geo_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_07437_gb300 import build
    build.build()
    return geo.load_library()


def test_header_declares_expected_entry_points():
    syms = _declared_symbols()
    for name in ("geo_covgen", "geo_loglik", "geo_predict", "geo_mle_step"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    syms = _declared_symbols()
    assert syms, "no declarations parsed"
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    # the binding covers every declared entry point
    assert sorted(geo.SIGNATURES) == syms


def test_opts_default(lib):
    o = geo.opts()
    assert o.nb == 960 and o.prec == geo.GEO_PREC_FP64 and o.morton == 1 and o.band == 4
    assert o.tlr_kmax == 200 and o.tlr_tol == 1e-9


@pytest.mark.parametrize("n,seed", [(1, 1), (7, 2), (400, 1000), (2000, 5)])
def test_morton_order_matches_oracle(lib, n, seed):
    locs = inputs.jittered_grid(n, seed)
    assert np.array_equal(geo.geo_morton_order(locs), oracle.morton_order(locs))


def test_morton_order_ties_and_degenerate(lib):
    locs = np.array([[0.5, 0.5]] * 5 + [[0.1, 0.9], [0.9, 0.1]])
    assert np.array_equal(geo.geo_morton_order(locs), oracle.morton_order(locs))
    same = np.zeros((4, 2))
    assert np.array_equal(geo.geo_morton_order(same), np.arange(4))


def test_mle_init_simplex(lib):
    th = geo.Theta((1.0, 2.0), 0.09, (0.5, 1.0), 0.5)
    st = geo.geo_mle_init(th, 0.1)
    assert st.p == 2 and st.q == 6 and st.initialized == 0
    x0 = oracle.theta_to_x(oracle.Theta([1.0, 2.0], 0.09, [0.5, 1.0], 0.5))
    for v in range(7):
        row = np.array([st.x[v][d] for d in range(6)])
        expect = x0.copy()
        if v:
            expect[v - 1] += 0.1
        assert np.array_equal(row, expect)


def test_mle_init_profile_simplex(lib):
    # profile coordinates (log a, log nu_i, beta_ij): the sigma^2 leave the simplex (Sec. 4.2)
    th = geo.Theta((1.0, 2.0, 3.0), 0.09, (0.5, 1.0, 1.5), (0.5, 0.2, 0.1))
    st = geo.geo_mle_init(th, 0.05, profile=True)
    assert st.p == 3 and st.q == 7 and st.profile == 1 and st.initialized == 0
    x0 = oracle.profile_theta_to_x(oracle.Theta([1.0, 2.0, 3.0], 0.09, [0.5, 1.0, 1.5], [0.5, 0.2, 0.1]))
    for v in range(8):
        row = np.array([st.x[v][d] for d in range(7)])
        expect = x0.copy()
        if v:
            expect[v - 1] += 0.05
        assert np.array_equal(row, expect)
    assert geo.geo_mle_init(th, 0.05).profile == 0


def test_mle_init_rejects_bad_theta_and_best_before_steps(lib):
    for bad in (geo.Theta((1.0, 1.0), -0.1, (0.5, 1.0), 0.5), geo.Theta((1.0, 1.0), 0.1, (0.0, 1.0), 0.5)):
        for profile in (False, True):
            with pytest.raises(geo.GeoError):
                geo.geo_mle_init(bad, 0.1, profile=profile)
    with pytest.raises(geo.GeoError):
        geo.geo_mle_init(geo.Theta((-1.0, 1.0), 0.1, (0.5, 1.0), 0.5), 0.1)     # sigma^2 <= 0 (full run)
    # the profile run does not read sigma^2
    geo.geo_mle_init(geo.Theta((-1.0, 1.0), 0.1, (0.5, 1.0), 0.5), 0.1, profile=True)
    th = geo.Theta((1.5, 2.5), 0.09, (0.5, 1.0), 0.4)
    best, ll = geo.geo_mle_best(geo.geo_mle_init(th, 0.1))
    assert np.isnan(ll) and best.sigma2 == pytest.approx((1.5, 2.5)) and best.a == pytest.approx(0.09)
    best, ll = geo.geo_mle_best(geo.geo_mle_init(th, 0.1, profile=True))
    assert np.isnan(ll) and all(np.isnan(best.sigma2))
    assert best.nu == pytest.approx((0.5, 1.0)) and best.beta[0][1] == pytest.approx(0.4)


def test_create_without_gpu_reports_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.geo_create(ctypes.byref(h), 0, 0) == geo.GEO_ECUDA


def test_noalloc_wrapper_checks_shapes_before_any_launch():
    # the binding refuses mismatched buffers before it touches the library or a device
    torch = pytest.importorskip("torch")
    th = geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5)
    locs = torch.zeros((10, 2), dtype=torch.float64)
    z = torch.zeros(20, dtype=torch.float64)
    out = torch.zeros(3, dtype=torch.float64)
    info = torch.zeros(1, dtype=torch.int32)
    with pytest.raises(ValueError, match="p \\* n"):
        geo.geo_loglik_noalloc(locs, torch.zeros(19, dtype=torch.float64), th, out, info)
    with pytest.raises(ValueError, match="n x 2"):
        geo.geo_loglik_noalloc(torch.zeros((10, 3), dtype=torch.float64), z, th, out, info)
    with pytest.raises(ValueError, match="3 doubles"):
        geo.geo_loglik_noalloc(locs, z, th, torch.zeros(2, dtype=torch.float64), info)
    with pytest.raises(ValueError, match="one int"):
        geo.geo_loglik_noalloc(locs, z, th, out, torch.zeros(0, dtype=torch.int32))
    with pytest.raises(TypeError):
        geo.geo_loglik_noalloc(locs, z, th, out, torch.zeros(1, dtype=torch.int64))
    with pytest.raises(TypeError, match="CUDA"):
        geo.geo_loglik_noalloc(locs, z, th, out, info)


def test_struct_layouts_match_the_library(lib):
    """The ctypes structures of the binding have the sizes and field offsets of the C ABI."""
    import ctypes
    out = (ctypes.c_longlong * 16)()
    count = lib.geo_abi_layout(out, 16)
    assert count == 11
    py = [ctypes.sizeof(geo.geo_theta), ctypes.sizeof(geo.geo_opts), ctypes.sizeof(geo.geo_factor_stats),
          ctypes.sizeof(geo.geo_mle_state), ctypes.sizeof(geo.geo_batch_item), ctypes.sizeof(geo.geo_request),
          ctypes.sizeof(geo.geo_result), ctypes.sizeof(geo.geo_kstat),
          geo.geo_opts.oz_slices.offset, geo.geo_opts.oz_cut.offset, geo.geo_kstat.tensor_flops.offset]
    assert list(out[:count]) == py
    assert lib.geo_abi_layout(None, 0) == 11
    assert lib.geo_abi_layout(None, 3) == geo.GEO_EINVAL
