"""Request server (continuous admission by device memory, overlapping
workers, device-resident factors reused by cokriging) and the tile-size
autotuner.  Bounds: l within 1e-10 relative of the oracle, predictions 1e-8
relative in the 2-norm; a request's result is bit-identical alone and in a
mix of concurrent requests."""
import time

import numpy as np
import pytest

import oracle
import paper_2008_07437_gb300 as geo
from paper_2008_07437_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_07437_gb300 import build
    build.build()


def o_theta(t):
    return oracle.Theta(list(t.sigma2), t.a, list(t.nu), t.beta_matrix())


TH = [geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5), geo.Theta((1.3, 0.8), 0.05, (0.7, 1.2), -0.3)]


def _dataset(n, m, k):
    th = TH[k % 2]
    allp = inputs.jittered_grid(n + m, 5000 + k)
    Z = oracle.simulate(o_theta(th), allp, inputs.normals(6000 + k, 2 * (n + m)))
    return allp[:n], Z[:2 * n], allp[n:], th


def _collect(srv, count, timeout=120.0):
    out, t0 = [], time.time()
    while len(out) < count and time.time() - t0 < timeout:
        out += srv.poll(64, wait_ms=50)
    return {r["id"]: r for r in out}


def test_server_mixed_requests_match_oracle(built):
    srv = geo.Server(0, 0, slots=3)
    try:
        data = [_dataset(n, 30, k) for k, n in enumerate([300, 520, 150, 700])]
        ids = {}
        for k, (locs, Z, new, th) in enumerate(data):
            ids[srv.submit_loglik(locs, Z, th, geo.opts(nb=128), dataset=100 + k, keep=True)] = ("ll", k)
        preds = {}
        for k, (locs, Z, new, th) in enumerate(data):
            rid, buf = srv.submit_predict(100 + k, new, 2, release=True)
            preds[rid] = (k, buf)
        res = _collect(srv, len(ids) + len(preds))
        assert len(res) == len(ids) + len(preds)
        for rid, (_, k) in ids.items():
            locs, Z, new, th = data[k]
            assert res[rid]["status"] == geo.GEO_OK
            assert res[rid]["loglik"] == pytest.approx(oracle.loglik(o_theta(th), locs, Z).loglik, rel=1e-10)
        for rid, (k, buf) in preds.items():
            locs, Z, new, th = data[k]
            assert res[rid]["status"] == geo.GEO_OK
            ref = oracle.predict(o_theta(th), locs, Z, new)
            assert np.all(np.abs(buf - ref) <= 1e-8 * (np.abs(ref).max() + np.abs(ref)))
            assert res[rid]["t_end"] >= res[rid]["t_start"] >= res[rid]["t_submit"]
    finally:
        srv.close()


def test_server_result_same_alone_and_in_the_mix(built):
    locs, Z, new, th = _dataset(600, 20, 7)
    srv = geo.Server(0, 0, slots=1)
    try:
        rid = srv.submit_loglik(locs, Z, th, geo.opts(nb=128))
        alone = _collect(srv, 1)[rid]["loglik"]
    finally:
        srv.close()
    srv = geo.Server(0, 0, slots=4)
    try:
        others = [_dataset(n, 10, 20 + k) for k, n in enumerate([900, 400, 800, 650, 1000])]
        for k, (l2, z2, _, t2) in enumerate(others[:3]):
            srv.submit_loglik(l2, z2, t2, geo.opts(nb=128))
        rid = srv.submit_loglik(locs, Z, th, geo.opts(nb=128))
        for k, (l2, z2, _, t2) in enumerate(others[3:]):
            srv.submit_loglik(l2, z2, t2, geo.opts(nb=128))
        res = _collect(srv, 6)
        assert res[rid]["loglik"] == alone   # bitwise
        _assert_some_overlap(res)
    finally:
        srv.close()


def _assert_some_overlap(res):
    """At least two requests ran at the same time: their [t_start, t_end] intersect."""
    spans = sorted((r["t_start"], r["t_end"]) for r in res.values())
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1)), spans


def test_server_emulated_reduced_form_same_alone_and_in_the_mix(built):
    # the served reduced form: tensor-core updates with 5 digit slices; the
    # result of a request does not depend on what runs beside it
    opt = geo.opts(nb=128, fp64_gemm=1, oz_slices=5)
    locs, Z, new, th = _dataset(700, 20, 9)
    srv = geo.Server(0, 0, slots=1)
    try:
        rid = srv.submit_loglik(locs, Z, th, opt)
        alone = _collect(srv, 1)[rid]["loglik"]
    finally:
        srv.close()
    ref = oracle.loglik(o_theta(th), locs, Z).loglik
    assert abs(alone - ref) <= 1e-8 * abs(ref)
    srv = geo.Server(0, 0, slots=4)
    try:
        others = [_dataset(n, 10, 40 + k) for k, n in enumerate([900, 400, 800, 650, 1000])]
        for l2, z2, _, t2 in others[:3]:
            srv.submit_loglik(l2, z2, t2, opt)
        rid = srv.submit_loglik(locs, Z, th, opt)
        for l2, z2, _, t2 in others[3:]:
            srv.submit_loglik(l2, z2, t2, opt)
        res = _collect(srv, 6)
        assert all(r["status"] == geo.GEO_OK for r in res.values())
        assert res[rid]["loglik"] == alone   # bitwise
        _assert_some_overlap(res)
    finally:
        srv.close()


def test_server_budget_admission_and_rejection(built):
    # a budget that admits one request of this size at a time: the matrix
    # (ld x N doubles, ld = N + 1 rounded up to 32) dominates the footprint
    n = 800
    N = 2 * n
    one = 8 * ((N + 1 + 31) // 32 * 32) * N
    srv = geo.Server(0, int(one * 1.5), slots=4)
    try:
        data = [_dataset(n, 5, 40 + k) for k in range(4)]
        ids = [srv.submit_loglik(l, z, th, geo.opts(nb=128)) for l, z, _, th in data]
        res = _collect(srv, 4)
        assert all(res[i]["status"] == geo.GEO_OK for i in ids)
        spans = sorted((res[i]["t_start"], res[i]["t_end"]) for i in ids)
        for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
            assert s1 >= e0 - 1e-6   # never two at once under this budget
        _, _, reserved = srv.pending()
        assert reserved <= int(one * 1.5)
        big = _dataset(3000, 5, 50)
        with pytest.raises(geo.GeoError) as ei:
            srv.submit_loglik(big[0], big[1], big[3], geo.opts(nb=128))
        assert ei.value.code == geo.GEO_ENOMEM
    finally:
        srv.close()


def test_server_failed_likelihood_fails_its_predictions(built):
    srv = geo.Server(0, 0, slots=2)
    try:
        bad_th = geo.Theta((1.0,), 1.0, (5.0,), None)
        locs = inputs.jittered_grid(900, 9)
        r1 = srv.submit_loglik(locs, np.zeros(900), bad_th, geo.opts(nb=128), dataset=9, keep=True)
        r2, _ = srv.submit_predict(9, inputs.jittered_grid(5, 1), 1, release=True)
        res = _collect(srv, 2)
        assert res[r1]["status"] == geo.GEO_ENOTSPD
        assert res[r2]["status"] != geo.GEO_OK
    finally:
        srv.close()


def test_autotuner_picks_a_candidate_and_nb0_uses_it(built):
    ctx = geo.geo_create(0)
    try:
        locs, Z, _, th = _dataset(1500, 0, 60)
        dl, dz = torch.as_tensor(locs, device="cuda"), torch.as_tensor(Z, device="cuda")
        best, ms = geo.geo_autotune_nb(ctx, dl, dz, th, [128, 256, 512])
        assert best in (128, 256, 512) and ms > 0
        v0, _ = geo.geo_loglik(ctx, dl, dz, th, geo.opts(nb=0))
        vb, _ = geo.geo_loglik(ctx, dl, dz, th, geo.opts(nb=best))
        assert v0 == vb
    finally:
        ctx.close()


def test_autotuner_tunes_nb_and_band_and_nb0_uses_both(built):
    # mixed form: the tuned (nb, band) pair is what nb = 0 runs -- the likelihood with nb = 0 is
    # bitwise the one of the explicit pair, and the band changes the arithmetic
    ctx = geo.geo_create(0)
    try:
        locs, Z, _, th = _dataset(1200, 0, 61)
        dl, dz = torch.as_tensor(locs, device="cuda"), torch.as_tensor(Z, device="cuda")
        base = geo.opts(prec=geo.GEO_PREC_MIXED, refine_iters=2)
        nb, band, ms = geo.geo_autotune(ctx, dl, dz, th, [128, 256], [0, 1, 3], samples=3, options=base)
        assert nb in (128, 256) and band in (0, 1, 3) and ms > 0
        v0, _ = geo.geo_loglik(ctx, dl, dz, th, geo.opts(nb=0, prec=geo.GEO_PREC_MIXED, refine_iters=2))
        vb, _ = geo.geo_loglik(ctx, dl, dz, th, geo.opts(nb=nb, band=band, prec=geo.GEO_PREC_MIXED, refine_iters=2))
        assert v0 == vb
        others = [geo.geo_loglik(ctx, dl, dz, th, geo.opts(nb=nb, band=b, prec=geo.GEO_PREC_MIXED,
                                                             refine_iters=2))[0] for b in (0, 1, 3) if b != band]
        assert any(v != v0 for v in others)   # the band is not a no-op at this size
    finally:
        ctx.close()


def test_server_escalates_a_reduced_form_that_is_not_spd(built):
    # a = 0.2, nu_2 = 1.5 at 5,000 locations: FP32 off-diagonal tiles lose
    # positive definiteness, FP64 does not
    th = geo.Theta((1.0, 1.0), 0.2, (0.5, 1.5), 0.7)
    locs = inputs.jittered_grid(5000, 77)
    z = inputs.normals(78, 10000)
    mixed = geo.opts(nb=0, prec=1, band=1 << 20, refine_iters=2)
    srv = geo.Server(0, 0, slots=2)
    try:
        r_plain = srv.submit_loglik(locs, z, th, mixed)
        r_esc = srv.submit_loglik(locs, z, th, mixed, escalate=True)
        res = _collect(srv, 2)
    finally:
        srv.close()
    assert res[r_plain]["status"] == geo.GEO_ENOTSPD and res[r_plain]["prec"] == 1
    assert res[r_esc]["status"] == geo.GEO_OK and res[r_esc]["prec"] == 0
    ctx = geo.geo_create(0)
    try:
        l64, _ = geo.geo_loglik(ctx, torch.as_tensor(locs, device="cuda"), torch.as_tensor(z, device="cuda"), th,
                                geo.opts(nb=0))
    finally:
        ctx.close()
    assert res[r_esc]["loglik"] == l64
