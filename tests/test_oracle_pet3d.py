"""Pins of the oracle's structured fully-3-D PET geometry (sinograms per ring
difference and angle, the oblique LORs of the paper's §3 geometric-flexibility
discussion): the LOR endpoints sit on the detector cylinder at the two rings'
heights, the ring-difference-0 segment is the 2-D ring sinogram of the direct
planes, every segment equals the same LORs traced as explicit rays (forward
and adjoint), the bounding box loses no pair, and rows past a segment's last
ring pair are empty."""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth

R_RING, N_CRYST = 400.0, 576


def _geom(n_ang=10, n_rad=37, n_rings=7, pitch=4.0, D=3, arc_mode=0):
    return synth.geom_pet3d(n_ang, n_rad, n_rings, R_RING, N_CRYST, pitch, D, arc_mode=arc_mode)


def _lors(g):
    """Each valid pixel's LOR from the ring geometry written out here: the
    chord at signed distance s from the axis, perpendicular to e_u = (cos
    phi, sin phi, 0), from ring min(j) at -h e_w to the other ring at +h e_w.
    Returns flat indices and endpoints (a, b) in FP64."""
    V, H, W, D = g["n_views"], g["n_rows"], g["n_cols"], g["max_ring_diff"]
    k = np.arange(W) - 0.5 * (W - 1)
    if g["arc_mode"] == 0:
        s = k * math.pi * g["radius"] / g["n_crystals"]
    else:
        s = g["radius"] * np.sin(k * math.pi / g["n_crystals"])
    h = np.sqrt(g["radius"] ** 2 - s ** 2)
    zr = (np.arange(H) - 0.5 * (H - 1)) * g["pitch_v"]
    idx, A, B = [], [], []
    for sg, delta in enumerate(range(-D, D + 1)):
        for a in range(V):
            phi = math.pi * a / V
            eu = np.array([math.cos(phi), math.sin(phi), 0.0])
            ew = np.array([math.sin(phi), -math.cos(phi), 0.0])
            for j in range(H - abs(delta)):
                r1, r2 = (j, j + delta) if delta >= 0 else (j - delta, j)
                for i in range(W):
                    idx.append(((sg * V + a) * H + j) * W + i)
                    A.append(s[i] * eu - h[i] * ew + np.array([0, 0, zr[r1]]))
                    B.append(s[i] * eu + h[i] * ew + np.array([0, 0, zr[r2]]))
    return np.array(idx), np.array(A), np.array(B)


def _phantom(seed, n=60):
    G = synth.gaussians_uniform(n, seed, half_box=150.0, log_sigma=math.log(6.0))
    G["mu"][:, 2] *= 0.08
    rng = np.random.default_rng(seed + 1)
    G["ls"] = (G["ls"] + rng.normal(0.0, 0.4, G["ls"].shape)).astype(np.float32)
    return G


@pytest.mark.parametrize("arc_mode", [0, 1])
def test_lor_endpoints_on_the_cylinder(oracle, arc_mode):
    g = _geom(arc_mode=arc_mode)
    idx, A, B = _lors(g)
    o, d, ta, tb = oracle.rays(g, idx)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(o + ta[:, None] * d, A, rtol=0, atol=1e-10)
    np.testing.assert_allclose(o + tb[:, None] * d, B, rtol=0, atol=1e-10)
    np.testing.assert_allclose(np.hypot(A[:, 0], A[:, 1]), R_RING, rtol=1e-14)
    assert oracle.Geometry(g).n_rays == 7 * 10 * 7 * 37


def test_segment_zero_is_the_direct_plane_sinogram(oracle):
    G = _phantom(3)
    g = _geom(D=0)
    got = oracle.forward(g, G)["I"].reshape(10, 7, 37)
    g2 = synth.geom_pet(10, 37, 7, R_RING, N_CRYST, 4.0)
    want = oracle.forward(g2, G)["I"].reshape(7, 10, 37).transpose(1, 0, 2)
    assert np.count_nonzero(want) > 200
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * np.abs(want).max())


@pytest.mark.parametrize("arc_mode", [0, 1])
def test_forward_equals_the_explicit_lors(oracle, arc_mode):
    G = _phantom(5)
    g = _geom(arc_mode=arc_mode)
    idx, A, B = _lors(g)
    I = oracle.forward(g, G)["I"]
    L = np.linalg.norm(B - A, axis=1)
    ref = oracle.forward_list(A, B - A, np.stack([np.zeros_like(L), L], 1), G)["I"]
    assert np.count_nonzero(ref) > 1000
    np.testing.assert_allclose(I[idx], ref, rtol=1e-11, atol=1e-14 * np.abs(ref).max())
    empty = np.ones(I.size, bool)
    empty[idx] = False
    assert empty.sum() == 10 * 37 * 2 * (1 + 2 + 3)
    assert not I[empty].any()


def test_oblique_lor_through_the_centre_closed_form(oracle):
    """An axis-aligned Gaussian at the centre and the LOR of each even ring
    difference that passes through it (s = 0, mid-height 0): the integral
    over a line of direction d is rho sqrt(2 pi / d^T P d) (the segment is
    hundreds of sigma long), d^T P d = cos^2(theta) / sigma_w^2 + sin^2(theta)
    / sigma_z^2 with tan(theta) = delta pitch / (2 R)."""
    ls = np.log(np.array([[4.0, 5.0, 30.0]], np.float32)).astype(np.float32)
    G = dict(mu=np.zeros((1, 3), np.float32), ls=ls, q=np.array([[1.0, 0.0, 0.0, 0.0]], np.float32),
             rho=np.array([1.0], np.float32))
    sx, sy, sz = np.exp(ls[0].astype(np.float64))
    n_rings, pitch, D = 41, 20.0, 20
    g = synth.geom_pet3d(4, 21, n_rings, R_RING, N_CRYST, pitch, D)
    I = oracle.forward(g, G)["I"].reshape(2 * D + 1, 4, n_rings, 21)
    for delta in range(-D, D + 1, 2):
        j = (n_rings - 1) // 2 - abs(delta) // 2
        th = math.atan2(delta * pitch, 2 * R_RING)
        for a, sw in ((0, sy), (2, sx)):   # angle 0: e_w = -e_y; angle pi/2: e_w = e_x
            A = math.cos(th) ** 2 / sw ** 2 + math.sin(th) ** 2 / sz ** 2
            assert I[delta + D, a, j, 10] == pytest.approx(math.sqrt(2 * math.pi / A), rel=1e-13), (delta, a)


def test_bounding_box_loses_no_pair(oracle):
    G = _phantom(7, n=80)
    # a few needles tilted in z and Gaussians near the ring's edge and the
    # axial ends, where the LOR slope and the row clamp matter
    G["q"][:10] = np.array([0.8, 0.5, 0.1, 0.3], np.float32)
    G["ls"][:10, 2] = math.log(25.0)
    G["mu"][10:20, 0] = np.linspace(-370.0, 370.0, 10, dtype=np.float32)
    G["mu"][20:30, 2] = np.linspace(-14.0, 14.0, 10, dtype=np.float32)
    g = _geom(n_ang=8, n_rad=65, n_rings=8, D=5)
    a = oracle.forward(g, G)
    b = oracle.forward(g, G, brute=True)
    assert a["pairs"] == b["pairs"] > 1000
    for k in ("I", "I_lo", "I_hi"):
        np.testing.assert_array_equal(a[k], b[k])
    w = synth.random_weights(a["I"].size, 9)
    ga = oracle.backward(g, G, w)
    gb = oracle.backward(g, G, w, brute=True)
    for k in ("mu", "ls", "q", "rho"):
        np.testing.assert_array_equal(ga[k], gb[k])


def test_adjoint_equals_the_explicit_lors(oracle):
    G = _phantom(11, n=40)
    g = _geom()
    idx, A, B = _lors(g)
    n_rays = oracle.Geometry(g).n_rays
    w = synth.random_weights(n_rays, 12)
    got = oracle.backward(g, G, w)
    L = np.linalg.norm(B - A, axis=1)
    ref = oracle.backward_list(A, B - A, np.stack([np.zeros_like(L), L], 1), G, w[idx])
    for k in ("mu", "ls", "q", "rho"):
        scale = np.abs(ref[k]).max()
        assert scale > 0
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-9, atol=1e-12 * scale)
