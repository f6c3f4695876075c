"""Failure handling on the device without a GPU fault.

Every spin-wait of the library's kernels is bounded: a wait that runs out of
its clock budget records its site in the context's status word, makes the
other waiters give up and returns.  geo_selftest_bounded_wait withholds a
dependency from the host (the forward solve's first block is never taken, so
its completion is never published) with a short budget; the call must report
GEO_ETIMEOUT at the solve's wait, and the same context must then pass a
normal likelihood parity check (l within 1e-10 of the oracle)."""
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


def test_withheld_dependency_times_out_and_context_recovers(ctx):
    rc, site = geo.geo_selftest_bounded_wait(ctx, n_blocks=8, wait_cycles=2_000_000)   # ~1 ms budget
    assert rc == geo.GEO_ETIMEOUT and site == 3
    th = geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5)
    locs = inputs.jittered_grid(300, 77)
    o_th = oracle.Theta([1.0, 1.0], 0.09, [0.5, 1.0], 0.5)
    Z = oracle.simulate(o_th, locs, inputs.normals(78, 600))
    ref = oracle.loglik(o_th, locs, Z).loglik
    got, fac = geo.geo_loglik(ctx, torch.as_tensor(locs, device="cuda"), torch.as_tensor(Z, device="cuda"), th,
                              geo.opts(nb=128), keep=True)
    try:
        assert got == pytest.approx(ref, rel=1e-10)
        # the one-launch solves of the kept factor still complete (cokriging weights)
        zhat = torch.zeros(2, dtype=torch.float64, device="cuda")
        geo.geo_predict(ctx, fac, torch.as_tensor(locs[5:6], device="cuda"), zhat)
        np.testing.assert_allclose(zhat.cpu().numpy(), Z[10:12], atol=1e-8)
    finally:
        fac.free()


def test_selftest_rejects_bad_arguments(ctx):
    rc, _ = geo.geo_selftest_bounded_wait(ctx, n_blocks=1)
    assert rc == geo.GEO_EINVAL
    rc, _ = geo.geo_selftest_bounded_wait(ctx, n_blocks=8, wait_cycles=0)
    assert rc == geo.GEO_EINVAL
