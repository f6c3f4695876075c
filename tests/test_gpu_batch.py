"""Batched small likelihoods (one launch sequence per batch shape, replayed
as a CUDA graph) against the oracle.  Bounds: 1e-10 relative on l (FP64);
a problem's result is bit-identical alone and inside a batch."""
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


def _problems(sizes, seed=0):
    thetas = [geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5),
              geo.Theta((1.2,), 0.05, (0.8,), None),
              geo.Theta((1.0, 0.5, 2.0), 0.1, (0.5, 1.0, 1.5), (0.5, 0.3, 0.4))]
    out = []
    for k, n in enumerate(sizes):
        th = thetas[k % 3]
        p = len(th.sigma2)
        locs = inputs.jittered_grid(n, 3000 + seed + k)
        z = oracle.simulate(o_theta(th), locs, inputs.normals(4000 + seed + k, p * n))
        out.append((locs, z, th))
    return out


def test_batch_uneven_matches_oracle(ctx):
    probs = _problems([1, 7, 40, 130, 257, 600, 333, 64])
    got, info = geo.geo_loglik_batch(ctx, [(dev(l), dev(z), th) for l, z, th in probs])
    assert np.all(info == 0)
    for (locs, z, th), g in zip(probs, got):
        ref = oracle.loglik(o_theta(th), locs, z).loglik
        assert g == pytest.approx(ref, rel=1e-10)


def test_batch_result_is_identical_alone_and_in_the_mix(ctx):
    probs = _problems([200, 350, 90, 500], seed=10)
    dp = [(dev(l), dev(z), th) for l, z, th in probs]
    mix, _ = geo.geo_loglik_batch(ctx, dp)
    for k in range(len(dp)):
        alone, _ = geo.geo_loglik_batch(ctx, [dp[k]])
        assert alone[0] == mix[k]          # bitwise
    rev, _ = geo.geo_loglik_batch(ctx, dp[::-1])
    assert np.array_equal(rev[::-1], mix)


def test_batch_graph_replay_with_new_theta(ctx):
    probs = _problems([150, 220, 300], seed=20)
    dp = [(dev(l), dev(z), th) for l, z, th in probs]
    geo.geo_loglik_batch(ctx, dp)   # capture
    for a in (0.03, 0.2):
        dp2 = [(l, z, geo.Theta(th.sigma2, a, th.nu, th.beta)) for l, z, th in dp]
        got, info = geo.geo_loglik_batch(ctx, dp2)
        for (locs, z, th), g in zip(probs, got):
            ref = oracle.loglik(o_theta(geo.Theta(th.sigma2, a, th.nu, th.beta)), locs, z).loglik
            assert g == pytest.approx(ref, rel=1e-10)


def test_batch_matches_single_loglik(ctx):
    probs = _problems([400, 410], seed=30)
    got, _ = geo.geo_loglik_batch(ctx, [(dev(l), dev(z), th) for l, z, th in probs])
    for (locs, z, th), g in zip(probs, got):
        single, _ = geo.geo_loglik(ctx, dev(locs), dev(z), th, geo.opts(nb=128))
        assert g == pytest.approx(single, rel=1e-11)


def test_batch_reports_not_spd_per_problem(ctx):
    good = _problems([100], seed=40)[0]
    bad_th = geo.Theta((1.0,), 1.0, (5.0,), None)
    bad_locs = inputs.jittered_grid(900, 9)
    got, info = geo.geo_loglik_batch(ctx, [(dev(good[0]), dev(good[1]), good[2]),
                                           (dev(bad_locs), dev(np.zeros(900)), bad_th)])
    assert info[0] == 0 and info[1] > 0
    assert np.isfinite(got[0]) and np.isnan(got[1])


def test_batch_with_four_variables(ctx):
    th4 = geo.Theta((1.0, 0.8, 1.2, 0.6), 0.08, (0.4, 0.9, 1.3, 3.6), (0.3, 0.2, 0.1, 0.25, 0.15, 0.35))
    probs = _problems([60, 90], seed=50)
    locs4 = inputs.jittered_grid(70, 55)
    z4 = oracle.simulate(o_theta(th4), locs4, inputs.normals(56, 280))
    items = [(dev(l), dev(z), th) for l, z, th in probs] + [(dev(locs4), dev(z4), th4)]
    got, info = geo.geo_loglik_batch(ctx, items)
    assert np.all(info == 0)
    for (locs, z, th), g in zip(probs + [(locs4, z4, th4)], got):
        assert g == pytest.approx(oracle.loglik(o_theta(th), locs, z).loglik, rel=1e-10)
