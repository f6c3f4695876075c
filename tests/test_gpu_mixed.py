"""Mixed-precision form against the FP64 oracle.

FP64 diagonal tiles (storage and factorisation), FP32 band, tensor-core
updates beyond the band with FP16 operands split in two terms (hi + lo, per-row
power-of-two scale) or one BF16 term, FP64 iterative refinement of the solve.

The log-determinant comes from the reduced-precision factor and is not
refined, so the error of l is an absolute error that grows with N; when the
two terms of l nearly cancel (|l| << N) a relative bound says little.  Stated
bounds, |dl| <= c N (measured values at N = 2,000 / 4,000 in brackets):
  FP16 x 2, band >= 1, >= 2 refinement sweeps : c = 5e-7   (2.5e-8 / 5e-8)
  FP16 x 2, band 0                            : c = 5e-6   (2.5e-7 / 1.2e-6)
  BF16 x 1                                    : c = 2e-4   (7.8e-6 / 6.8e-5)
  no refinement (FP16 x 2, band 4)            : c = 5e-6   (5.4e-7 / 3.3e-8)
and |dl| / |l| <= 1e-6 for the mixed workload's theta at N = 2,000.
These c N bounds are fitted at N = 2,000 - 4,000 and hold only there: the
error of this FP32-class form grows faster than N (at N = 100,000 a run of
the FP16 x 2 form gave |dl| = 6.9, 6.9e-5 N, |dl| / |l| = 6e-5), so it does
not meet 1e-6 at the mixed workload's size; the tensor-core form with 5
digit slices (geo_opts.fp64_gemm = 1, tests/test_gpu_ozaki.py) does.
Predictions with refinement: 1e-6 (max |z| + |z|) entry by entry.
Tile size 128 keeps several tiles beyond the band at oracle-sized problems."""
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


TH_MIX = geo.Theta((1.0, 1.0), 0.1, (0.5, 1.0), 0.7)          # the mixed-precision workload's theta
TH3 = geo.Theta((1.0, 1.0, 1.0), 0.05, (0.5, 1.0, 1.5), (0.5, 0.3, 0.4))


def _problem(n, theta, seed):
    p = len(theta.sigma2)
    locs = inputs.jittered_grid(n, 500 + seed)
    Z = oracle.simulate(o_theta(theta), locs, inputs.normals(600 + seed, p * n))
    return locs, Z


@pytest.mark.parametrize("n", [1000, 2000])
@pytest.mark.parametrize("band,lowp,iters,c", [(4, 0, 2, 5e-7), (1, 0, 2, 5e-7), (0, 0, 2, 5e-6),
                                               (4, 1, 2, 2e-4), (4, 0, 0, 5e-6)],
                         ids=["band4-fp16x2-ir2", "band1-fp16x2-ir2", "band0-fp16x2-ir2", "band4-bf16-ir2",
                              "band4-fp16x2-noir"])
def test_mixed_loglik_within_bound(ctx, n, band, lowp, iters, c):
    locs, Z = _problem(n, TH_MIX, 1)        # N = 2,000 / 4,000: 16 / 32 tiles of 128
    ref = oracle.loglik(o_theta(TH_MIX), locs, Z)
    got, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), TH_MIX,
                            geo.opts(prec=geo.GEO_PREC_MIXED, nb=128, band=band, lowp=lowp, refine_iters=iters))
    N = 2 * n
    assert abs(got - ref.loglik) <= c * N, (got, ref.loglik)
    if n == 1000 and lowp == 0 and band >= 1 and iters >= 2:
        assert abs(got - ref.loglik) / abs(ref.loglik) <= 1e-6


def test_mixed_wide_band_is_fp32_everywhere(ctx):
    # band >= number of tiles: no tensor-core tile; still within the bound
    locs, Z = _problem(500, TH3, 2)          # N = 1,500
    ref = oracle.loglik(o_theta(TH3), locs, Z)
    got, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), TH3,
                            geo.opts(prec=geo.GEO_PREC_MIXED, nb=128, band=100, refine_iters=2))
    assert abs(got - ref.loglik) <= 5e-7 * 1500


def test_mixed_ragged_and_trivariate(ctx):
    locs, Z = _problem(700, TH3, 3)          # N = 2,100: ragged last tile of 52 rows
    ref = oracle.loglik(o_theta(TH3), locs, Z)
    got, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), TH3,
                            geo.opts(prec=geo.GEO_PREC_MIXED, nb=128, band=2, refine_iters=2))
    assert abs(got - ref.loglik) <= 5e-7 * 2100


def test_mixed_predictions_with_refinement(ctx):
    n, m = 900, 50
    allp = inputs.jittered_grid(n + m, 77)
    locs, new = allp[:n], allp[n:]
    Zall = oracle.simulate(o_theta(TH_MIX), allp, inputs.normals(78, 2 * (n + m)))
    Z = Zall[:2 * n]
    ref = oracle.predict(o_theta(TH_MIX), locs, Z, new)
    _, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), TH_MIX,
                            geo.opts(prec=geo.GEO_PREC_MIXED, nb=128, band=2, refine_iters=3), keep=True)
    try:
        zhat = torch.zeros(2 * m, dtype=torch.float64, device="cuda")
        geo.geo_predict(ctx, fac, dev(new), zhat)
        got = zhat.cpu().numpy()
    finally:
        fac.free()
    err = np.abs(got - ref)
    assert np.all(err <= 1e-6 * (np.abs(ref).max() + np.abs(ref))), (err / np.abs(ref).max()).max()


def test_mixed_rejects_bad_tile(ctx):
    locs, Z = _problem(50, TH_MIX, 4)
    with pytest.raises(geo.GeoError) as ei:
        geo.geo_loglik(ctx, dev(locs), dev(Z), TH_MIX, geo.opts(prec=geo.GEO_PREC_MIXED, nb=192))
    assert ei.value.code == geo.GEO_EINVAL
