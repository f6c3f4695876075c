"""geo_loglik_noalloc: the log-likelihood for callers that cannot allocate
device memory (a host whose memory pool belongs to another allocator, or a
latency-critical loop that cannot pay for cudaMalloc / cudaFree).  It works
in a fixed, library-owned scratch array instead of allocating.

The test calls it through the C ABI twice in a row -- a larger problem, then a
smaller one, so leftovers of the first call in the shared scratch must not
leak into the second -- and checks each result against geo_loglik within the
FP64 tolerance of the other parity tests (1e-10 relative on l, log|Sigma| and
the quadratic form).  It also checks that the second call leaves the device's
free memory unchanged, that oversized problems are refused, that a Sigma that
is not positive definite gives NaN outputs and a failing row while the next
good call reports info = 0 again (the status words live in the shared scratch
and are cleared per call), and that buffers which are not device memory of
the current device are refused before anything runs.
This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

import paper_2008_07437_gb300 as geo
from paper_2008_07437_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_07437_gb300 import build
    build.build()
    c = geo.geo_create(0)
    yield c
    c.close()


def _case(n, theta, seed):
    locs = torch.as_tensor(inputs.jittered_grid(n, seed), device="cuda")
    p = len(theta.sigma2)
    z = torch.as_tensor(inputs.normals(seed + 1, p * n), device="cuda")
    return locs, z


def _reference(ctx, locs, z, theta, nb):
    ll, fac = geo.geo_loglik(ctx, locs, z, theta, geo.opts(nb=nb), keep=True)
    st = geo.geo_factor_stats_get(fac)
    fac.free()
    return np.array([ll, st.logdet, st.quad])


def test_noalloc_matches_loglik_on_two_calls_in_a_row(ctx):
    th_a = geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5)
    th_b = geo.Theta((1.0, 0.8, 1.2), 0.05, (0.5, 1.0, 1.5), (0.5, 0.3, 0.4))
    cases = [(_case(1000, th_a, 7), th_a, 128),    # N = 2,000
             (_case(300, th_b, 11), th_b, 192)]    # N = 900, after the larger call
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for k, ((locs, z), theta, nb) in enumerate(cases):
        ref = _reference(ctx, locs, z, theta, nb)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = geo.geo_loglik_noalloc(locs, z, theta, out, info, nb=nb)
        assert rc == geo.GEO_OK
        torch.cuda.synchronize()
        if k == 1:   # the scratch array is resident after the first call: nothing new on the device
            assert torch.cuda.mem_get_info()[0] == free_before
        got = out.cpu().numpy()
        assert int(info.cpu()[0]) == 0
        np.testing.assert_allclose(got, ref, rtol=RTOL)


def test_noalloc_rejects_problems_beyond_the_scratch(ctx):
    th = geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5)
    n = geo.GEO_NOALLOC_MAX_N // 2 + 1          # p * n = GEO_NOALLOC_MAX_N + 2
    locs, z = _case(n, th, 3)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    assert geo.geo_loglik_noalloc(locs, z, th, out) == geo.GEO_ESCRATCH
    # the largest admissible size still runs and matches
    n = geo.GEO_NOALLOC_MAX_N // 2
    locs, z = _case(n, th, 5)
    ref = _reference(ctx, locs, z, th, 256)
    assert geo.geo_loglik_noalloc(locs, z, th, out, nb=256) == geo.GEO_OK
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=RTOL)


def test_noalloc_not_positive_definite_then_recovers(ctx):
    th = geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5)
    base = inputs.jittered_grid(200, 21)
    dup = np.concatenate([base, base[:1]])          # a repeated location: Sigma is singular
    locs = torch.as_tensor(dup, device="cuda")
    z = torch.as_tensor(inputs.normals(22, 2 * 201), device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert geo.geo_loglik_noalloc(locs, z, th, out, info, nb=128) == geo.GEO_OK
    torch.cuda.synchronize()
    assert np.all(np.isnan(out.cpu().numpy()))
    assert int(info.cpu()[0]) > 0
    locs2, z2 = _case(200, th, 23)
    ref = _reference(ctx, locs2, z2, th, 128)
    assert geo.geo_loglik_noalloc(locs2, z2, th, out, info, nb=128) == geo.GEO_OK
    torch.cuda.synchronize()
    assert int(info.cpu()[0]) == 0
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=RTOL)


def test_noalloc_refuses_host_buffers(ctx):
    # a host pointer in place of a device buffer is refused by the C entry point itself
    th = geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5)
    locs, z = _case(50, th, 31)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    host_z = np.asarray(inputs.normals(32, 100), dtype=np.float64)
    thc, _keep = th.to_c()
    lib = geo.load_library()
    rc = lib.geo_loglik_noalloc(ctypes.c_void_p(locs.data_ptr()), 50, host_z.ctypes.data_as(ctypes.c_void_p),
                                ctypes.byref(thc), 128, ctypes.c_void_p(out.data_ptr()), None, None)
    assert rc == geo.GEO_EINVAL
