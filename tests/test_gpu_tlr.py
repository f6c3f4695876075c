"""Tile-low-rank form (Sec. 5.3) against the FP64 oracle.

Stated bounds (per-tile absolute accuracy tol, kmax = 200):
* tol = 1e-13 with kmax = nb: l within 1e-9 relative of the dense oracle;
* a tile whose rank would exceed kmax is stored dense (L_ij itself): with
  kmax = 8 and tol = 1e-12, |dl| <= 1e-6;
* tol = 1e-9: |dl| <= 1e-4, tol = 1e-7: |dl| <= 1e-2 (N <= 2,400; the error of
  log|Sigma| and of the quadratic form is of order N * tol * ||Sigma^-1||-weighted);
* ranks of the first tile column (compressed from Sigma itself, before any
  update) equal the oracle's exact-SVD ranks at the same threshold within 1;
* the 2-norm error of each first-column tile is <= 4 tol (the randomized SVD
  keeps every singular value above tol; the sketch error is below tol);
* ranks decay away from the diagonal (Fig. 5) and the factor takes less
  memory than dense tiles;
* cokriging with the TLR factor at tol = 1e-9: 1e-6 relative in the 2-norm.
"""
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


TH2 = geo.Theta((1.0, 1.0), 0.09, (0.5, 1.0), 0.5)                              # Fig. 5 theta
TH3 = geo.Theta((1.0, 1.0, 1.0), 0.05, (0.5, 1.0, 1.5), (0.5, 0.3, 0.4))       # trivariate workload theta


def _problem(n, theta, seed):
    p = len(theta.sigma2)
    locs = inputs.jittered_grid(n, 700 + seed)
    Z = oracle.simulate(o_theta(theta), locs, inputs.normals(800 + seed, p * n))
    return locs, Z


def tlr_opts(nb, tol, kmax=200):
    return geo.opts(prec=geo.GEO_PREC_TLR, nb=nb, tlr_tol=tol, tlr_kmax=kmax)


def test_tlr_tight_tolerance_equals_dense(ctx):
    locs, Z = _problem(600, TH2, 1)           # N = 1,200, 10 tiles of 120
    ref = oracle.loglik(o_theta(TH2), locs, Z)
    got, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, tlr_opts(120, 1e-13, kmax=120))
    assert got == pytest.approx(ref.loglik, rel=1e-9)


@pytest.mark.parametrize("theta,n,nb,tol,bound", [(TH2, 1200, 240, 1e-9, 1e-4), (TH3, 800, 240, 1e-9, 1e-4),
                                                  (TH3, 800, 240, 1e-7, 1e-2)],
                         ids=["bivariate-1e-9", "trivariate-1e-9", "trivariate-1e-7"])
def test_tlr_loglik_within_bound(ctx, theta, n, nb, tol, bound):
    locs, Z = _problem(n, theta, 2)
    ref = oracle.loglik(o_theta(theta), locs, Z)
    got, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), theta, tlr_opts(nb, tol), keep=True)
    try:
        st = geo.geo_factor_stats_get(fac)
        assert st.tlr_bytes_ratio < 1.0
        assert st.tlr_dense_tiles == 0
    finally:
        fac.free()
    assert abs(got - ref.loglik) <= bound, (got, ref.loglik)


def test_tlr_first_column_ranks_and_error(ctx):
    n, nb, tol = 900, 180, 1e-9
    locs, Z = _problem(n, TH2, 3)
    perm = oracle.morton_order(locs)
    sl = locs[perm]
    S = oracle.covgen(o_theta(TH2), sl)        # Sigma in the library's internal order
    ref_ranks = oracle.tlr_reference_ranks(S, nb, tol)
    _, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, tlr_opts(nb, tol), keep=True)
    try:
        R = geo.geo_tlr_ranks(fac)
        T = R.shape[0]
        D0 = geo.geo_tlr_tile(fac, 0, 0, "D")     # L_00
        for i in range(1, T):
            assert abs(R[i, 0] - ref_ranks[i, 0]) <= 1, (i, R[i, 0], ref_ranks[i, 0])
            U = geo.geo_tlr_tile(fac, i, 0, "U")
            V = geo.geo_tlr_tile(fac, i, 0, "V")   # stored as L_00^-1 V
            tile = S[i * nb:(i + 1) * nb, 0:nb]
            approx = U @ (D0 @ V).T
            err = np.linalg.norm(tile - approx, 2)
            assert err <= 4 * tol, (i, err)
        # Fig. 5: ranks grow towards the diagonal
        near = np.mean([R[i, i - 1] for i in range(1, T)])
        far = np.mean([R[i, j] for i in range(T) for j in range(i) if i - j >= T - 2])
        assert near >= far
    finally:
        fac.free()


def test_tlr_predictions(ctx):
    n, m = 700, 40
    allp = inputs.jittered_grid(n + m, 91)
    locs, new = allp[:n], allp[n:]
    Zall = oracle.simulate(o_theta(TH2), allp, inputs.normals(92, 2 * (n + m)))
    Z = Zall[:2 * n]
    ref = oracle.predict(o_theta(TH2), locs, Z, new)
    _, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, tlr_opts(140, 1e-9), keep=True)
    try:
        zhat = torch.zeros(2 * m, dtype=torch.float64, device="cuda")
        geo.geo_predict(ctx, fac, dev(new), zhat)
        got = zhat.cpu().numpy()
    finally:
        fac.free()
    err = np.abs(got - ref)
    assert np.all(err <= 1e-6 * (np.abs(ref).max() + np.abs(ref))), (err / np.abs(ref).max()).max()


def test_tlr_rank_above_kmax_stores_tile_dense(ctx):
    # tiles that need more than kmax columns are kept dense (exact), so l stays accurate
    locs, Z = _problem(600, TH2, 4)
    ref = oracle.loglik(o_theta(TH2), locs, Z)
    got, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, tlr_opts(120, 1e-12, kmax=8), keep=True)
    try:
        st = geo.geo_factor_stats_get(fac)
        assert st.tlr_dense_tiles > 0 and st.tlr_max_rank <= 8
    finally:
        fac.free()
    assert abs(got - ref.loglik) <= 1e-6


def test_tlr_rejects_tile_not_multiple_of_p(ctx):
    locs, Z = _problem(100, TH3, 5)
    with pytest.raises(geo.GeoError) as ei:
        geo.geo_loglik(ctx, dev(locs), dev(Z), TH3, tlr_opts(100, 1e-9))
    assert ei.value.code == geo.GEO_EINVAL


# ---- Diagonal Super Tile (Sec. 3.4): the tiles beyond a band dropped, the band exact ----

@pytest.mark.parametrize("dst", [1, 2, 3, 5])
def test_dst_matches_oracle(ctx, dst):
    th = geo.Theta((1.0, 1.5), 0.03, (0.5, 1.0), 0.4)
    locs, Z = _problem(600, th, seed=61)            # N = 1,200: 5 tiles of 240
    ref = oracle.dst_loglik(o_theta(th), locs, Z, 240, dst)
    got, fac = geo.geo_loglik(ctx, dev(locs), dev(Z), th, geo.opts(prec=2, nb=240, dst=dst), keep=True)
    st = geo.geo_factor_stats_get(fac)
    fac.free()
    assert got == pytest.approx(ref, rel=1e-10)
    assert st.tlr_dense_tiles == sum(5 - d for d in range(1, min(dst, 5)))   # the kept off-diagonal tiles
    if dst >= 5:
        dense, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), th, geo.opts(nb=240))
        assert got == pytest.approx(dense, rel=1e-12)


def test_tlr_long_k_products_split_k(ctx):
    # nb = 600: the cores V_ik' V_jk and the other K = nb products of a 6-tile column have few
    # output tiles, so the batched GEMM splits their K loops; the result must still equal dense
    # to the tolerance and be the same on every run
    locs, Z = _problem(1800, TH2, 6)          # N = 3,600
    ref = oracle.loglik(o_theta(TH2), locs, Z)
    o = tlr_opts(600, 1e-12, kmax=600)
    a, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, o)
    b, _ = geo.geo_loglik(ctx, dev(locs), dev(Z), TH2, o)
    assert a == b
    assert a == pytest.approx(ref.loglik, rel=1e-9)
