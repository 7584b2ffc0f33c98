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
