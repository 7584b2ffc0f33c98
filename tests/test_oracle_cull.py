"""Pins of the FP32 culling specification held by the oracle.

The specification (records + detector boxes in binary32, exact op order) is
what the GPU tile lists must reproduce bit for bit; here it is pinned to the
FP64 geometry: its covariances match FP64 to a few ulp, its exponential is
accurate, and every pair that the 3-sigma cut keeps (m <= 9, including the
FP32/FP64 ambiguity band) lies inside one of the tiles it emits.
"""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth


def test_records_fp32_close_to_fp64(oracle):
    G = synth.gaussians_uniform(2000, 5, log_sigma=math.log(0.05), log_sigma_std=0.8)
    s32 = oracle.records_fp32(G["ls"], G["q"]).astype(np.float64)
    sig, _ = oracle.cov(G["ls"], G["q"])
    packed = sig[:, [0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
    scale = np.abs(sig).reshape(-1, 9).max(axis=1, keepdims=True)
    err = np.abs(s32 - packed) / scale
    assert err.max() < 3e-6


def test_fp32_exponential_accuracy(oracle):
    """The Cody-Waite exponential used by the records: <= 2 ulp on [-20, 20]."""
    x = np.linspace(-10, 10, 20001).astype(np.float32)
    ls = np.stack([x, x, x], axis=1)
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (x.size, 1))
    s32 = oracle.records_fp32(ls, q)[:, 0]          # Sigma_00 = exp(2 l)
    ref = np.exp(2.0 * x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(s32 - ref) / ulp) <= 2.0


def _all_pairs_m(oracle, g, G):
    """m = C - B^2/A of every (view, Gaussian, pixel), via the oracle's pair()."""
    V, H, W = g["n_views"], g["n_rows"], g["n_cols"]
    n = G["mu"].shape[0]
    idx = np.arange(V * H * W)
    o, d, ta, tb = oracle.rays(g, idx)
    m = np.zeros((n, idx.size))
    for k in range(n):
        for r in range(idx.size):
            m[k, r] = oracle.pair(o[r], d[r], ta[r], tb[r], G["mu"][k], G["ls"][k], G["q"][k],
                                  G["rho"][k])[1]
    return m


@pytest.mark.parametrize("kind", ["parallel", "cone", "pet_arc", "pet_raw"])
def test_cull_is_conservative(oracle, kind):
    tw, th = 4, 4
    if kind == "parallel":
        g = synth.geom_parallel(3, 14, 13, 0.12, 0.12, -2.0, 2.0)
        G = synth.gaussians_uniform(25, 61, log_sigma=math.log(0.12))
    elif kind == "cone":
        g = synth.geom_cone(3, 13, 15, 0.2, 0.2, 3.0, 4.5)
        G = synth.gaussians_uniform(25, 62, log_sigma=math.log(0.12))
    else:
        g = synth.geom_pet(3, 31, 9, 400.0, 576, 2.0, arc_mode=0 if kind == "pet_arc" else 1)
        G = synth.gaussians_uniform(25, 63, half_box=30.0, log_sigma=math.log(3.0))
        G["mu"][:, 2] *= 0.2
    m = _all_pairs_m(oracle, g, G)
    box, rect, cnt = oracle.cull_fp32(g, G, tw, th)
    V, H, W = g["n_views"], g["n_rows"], g["n_cols"]
    kept = 0
    for k in range(G["mu"].shape[0]):
        mk = m[k].reshape(-1) if kind not in ("pet_arc", "pet_raw") else m[k]
        for r in np.nonzero(mk <= 9.0 + oracle.BAND)[0]:
            i = r % W
            if kind.startswith("pet"):
                v = (r // W) % V
                j = r // (W * V)
            else:
                j = (r // W) % H
                v = r // (W * H)
            tx0, tx1, ty0, ty1 = rect[v, k]
            assert cnt[v, k] > 0
            assert tx0 <= i // tw <= tx1 and ty0 <= j // th <= ty1, (k, v, j, i)
            kept += 1
    assert kept > 50


def test_cull_tiles_not_wider_than_needed(oracle):
    """Each emitted rectangle is the tile cover of the 3.0104-sigma box: its
    corner tiles hold a pixel within that box (checked in FP64, away from ties)."""
    g = synth.geom_cone(4, 64, 64, 0.04, 0.04, 3.0, 4.5)
    G = synth.gaussians_uniform(200, 64, half_box=0.9, log_sigma=math.log(0.08))
    box, rect, cnt = oracle.cull_fp32(g, G, 8, 8)
    assert (cnt > 0).mean() > 0.9
    # rectangle sizes bounded by the projected 3-sigma extent plus one tile
    sig, _ = oracle.cov(G["ls"], G["q"])
    smax = np.sqrt(np.linalg.eigvalsh(sig)[:, -1])
    mag = g["dsd"] / (g["dso"] - 1.8)
    width_tiles = (2 * 3.0104 * smax * mag / g["pitch_u"]) / 8 + 2
    w = rect[..., 1] - rect[..., 0] + 1
    assert np.all(w[cnt > 0] <= np.broadcast_to(width_tiles, w.shape)[cnt > 0] + 1e-9)


def _lor_pairs_m(oracle, g, G):
    """m of every (Gaussian, 3-D PET pixel) whose row holds a LOR, via pair()."""
    V = g["n_views"] * (2 * g["max_ring_diff"] + 1)
    H, W = g["n_rows"], g["n_cols"]
    idx = np.arange(V * H * W)
    o, d, ta, tb = oracle.rays(g, idx)
    live = ~((ta == 0.0) & (tb == 0.0))
    n = G["mu"].shape[0]
    m = np.full((n, idx.size), np.inf)
    for k in range(n):
        for r in np.nonzero(live)[0]:
            m[k, r] = oracle.pair(o[r], d[r], ta[r], tb[r], G["mu"][k], G["ls"][k], G["q"][k],
                                  G["rho"][k])[1]
    return m


@pytest.mark.parametrize("arc_mode,n_cryst", [(0, 72), (1, 72), (1, 24)])
def test_pet3d_cull_is_conservative(oracle, arc_mode, n_cryst):
    """Fully 3-D PET: every LOR pair with m <= 9 (+ the FP32/FP64 band) lies in
    a tile the FP32 cull emits.  A ring of 50 mm with 8 mm ring pitch makes
    the LOR slopes large (kappa up to 0.16 at the centre and more at the
    edge); with 24 crystals the raw radial bins reach the ring itself
    (R^2 - s^2 = 0 at the outermost column: every row of the segment)."""
    g = synth.geom_pet3d(5, 25, 6, 50.0, n_cryst, 8.0, 2, arc_mode=arc_mode)
    G = synth.gaussians_uniform(20, 70 + arc_mode, half_box=25.0, log_sigma=math.log(4.0))
    G["mu"][:, 2] *= 0.6
    tw, th = 4, 2
    m = _lor_pairs_m(oracle, g, G)
    box, rect, cnt = oracle.cull_fp32(g, G, tw, th)
    H, W = g["n_rows"], g["n_cols"]
    kept = 0
    for k in range(G["mu"].shape[0]):
        for r in np.nonzero(m[k] <= 9.0 + oracle.BAND)[0]:
            i, j, v = r % W, (r // W) % H, r // (W * H)
            tx0, tx1, ty0, ty1 = rect[v, k]
            assert cnt[v, k] > 0
            assert tx0 <= i // tw <= tx1 and ty0 <= j // th <= ty1, (k, v, j, i)
            kept += 1
    assert kept > 100
    # rows past a segment's last ring pair are never emitted
    D, V = g["max_ring_diff"], g["n_views"]
    for v in range(V * (2 * D + 1)):
        ad = abs(v // V - D)
        on = cnt[v] > 0
        assert np.all(box[v, on, 3] <= H - 1 - ad)


def test_tile_lists_expand_the_rectangles(oracle):
    """The CSR tile sets equal the cull's rectangles expanded tile by tile
    (a plain loop over views, Gaussians and tiles here)."""
    g = synth.geom_pet3d(4, 37, 7, 400.0, 576, 4.0, 2, arc_mode=0)
    G = synth.gaussians_uniform(80, 71, half_box=40.0, log_sigma=math.log(5.0))
    G["mu"][:, 2] *= 0.2
    tw, th = 8, 2
    box, rect, cnt = oracle.cull_fp32(g, G, tw, th)
    start, gid = oracle.tile_lists_fp32(g, G, tw, th)
    V, n = cnt.shape
    tx_n, ty_n = -(-g["n_cols"] // tw), -(-g["n_rows"] // th)
    sets = [[] for _ in range(V * tx_n * ty_n)]
    for v in range(V):
        for k in range(n):
            if cnt[v, k] == 0:
                continue
            tx0, tx1, ty0, ty1 = rect[v, k]
            for ty in range(ty0, ty1 + 1):
                for tx in range(tx0, tx1 + 1):
                    sets[v * tx_n * ty_n + ty * tx_n + tx].append(k)
    assert start[-1] == sum(len(s) for s in sets) > 0
    for t, s in enumerate(sets):
        assert list(gid[start[t]:start[t + 1]]) == sorted(s)
    # a view range gives the same tiles, renumbered from its first view
    s2, g2 = oracle.tile_lists_fp32(g, G, tw, th, views=(5, 9))
    T0, T1 = 5 * tx_n * ty_n, 9 * tx_n * ty_n
    assert np.array_equal(s2, start[T0:T1 + 1] - start[T0])
    assert np.array_equal(g2, gid[start[T0]:start[T1]])
