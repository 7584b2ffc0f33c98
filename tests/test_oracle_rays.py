"""Pins of the oracle's explicit-ray projector (any set of lines).

It must agree with the detector-geometry oracle on the same rays, follow the
isotropic closed form on random lines, be invariant to the length and the
sense of the direction, give half the full-line value on a half-line through
the centre, and its adjoint must match central finite differences.
"""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth


@pytest.mark.parametrize("kind", ["cone", "parallel", "pet"])
def test_list_equals_detector_geometry(oracle, kind):
    if kind == "pet":
        g = synth.geom_pet(6, 17, 5, 400.0, 576, 2.0)
        G = synth.gaussians_uniform(25, 3, half_box=40.0, log_sigma=math.log(6.0))
        G["mu"][:, 2] *= 0.1
    elif kind == "cone":
        g = synth.geom_cone(5, 9, 10, 0.2, 0.2, 3.0, 4.5)
        G = synth.gaussians_uniform(25, 4, log_sigma=math.log(0.2))
    else:
        g = synth.geom_parallel(5, 9, 10, 0.2, 0.2, -0.4, 0.6)
        G = synth.gaussians_uniform(25, 5, log_sigma=math.log(0.2))
    ref = oracle.forward(g, G)
    idx = np.arange(synth.num_rays(g))
    o, d, ta, tb = oracle.rays(g, idx)
    t = np.stack([ta, tb], 1)
    scale = np.random.default_rng(1).uniform(0.3, 3.0, (idx.size, 1))   # any direction length
    got = oracle.forward_list(o, d * scale, t, G)
    assert ref["pairs"] == got["pairs"]
    np.testing.assert_allclose(got["I"], ref["I"], rtol=1e-12, atol=1e-14 * np.abs(ref["I"]).max())
    w = np.random.default_rng(2).normal(size=idx.size)
    gb = oracle.backward(g, G, w)
    gl = oracle.backward_list(o, d, t, G, w)
    for k in ("mu", "ls", "q", "rho"):
        np.testing.assert_allclose(gl[k], gb[k], rtol=1e-10, atol=1e-12 * np.abs(gb[k]).max())


def test_isotropic_closed_form_on_random_lines(oracle):
    sigma, rho = 0.15, 0.7
    G = dict(mu=np.array([[0.1, -0.2, 0.05]], np.float32), ls=np.full((1, 3), math.log(sigma), np.float32),
             q=np.array([[1.0, 0, 0, 0]], np.float32), rho=np.array([rho], np.float32))
    R = synth.rays_random(400, 9, radius=0.5)
    got = oracle.forward_list(R["o"], R["d"], R["t"], G, cut2=1e30)["I"]
    o = R["o"].astype(np.float64)
    d = R["d"].astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    v = o - G["mu"].astype(np.float64)
    r2 = np.sum(np.cross(v, d) ** 2, axis=1)
    s = math.exp(float(np.float32(math.log(sigma))))    # the oracle reads float32 log-scales
    want = float(np.float32(rho)) * s * math.sqrt(2 * math.pi) * np.exp(-r2 / (2 * s * s))
    np.testing.assert_allclose(got, want, rtol=1e-12)


def test_direction_sense_and_length_do_not_matter(oracle):
    G = synth.gaussians_uniform(40, 11, half_box=0.6, log_sigma=math.log(0.12))
    R = synth.rays_random(300, 12, radius=0.7, seg=0.4)
    a = oracle.forward_list(R["o"], R["d"], R["t"], G)["I"]
    t_rev = np.stack([-R["t"][:, 1], -R["t"][:, 0]], 1)
    b = oracle.forward_list(R["o"], -2.5 * R["d"].astype(np.float64), t_rev, G)["I"]
    np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-15)
    assert np.count_nonzero(a) > 50


def test_half_line_through_the_centre_is_half(oracle):
    G = synth.gaussians_uniform(1, 13, half_box=0.0, log_sigma=math.log(0.2))
    G["mu"][:] = 0.0
    d = synth.rays_random(50, 14)["d"]
    o = np.zeros_like(d)
    full = oracle.forward_list(o, d, np.tile([-np.inf, np.inf], (50, 1)), G, cut2=1e30)["I"]
    half = oracle.forward_list(o, d, np.tile([0.0, np.inf], (50, 1)), G, cut2=1e30)["I"]
    np.testing.assert_allclose(half, 0.5 * full, rtol=1e-13)


def test_helical_without_pitch_is_the_circular_cone(oracle):
    g = synth.geom_cone(6, 7, 9, 0.25, 0.25, 3.0, 4.5)
    G = synth.gaussians_uniform(30, 15, log_sigma=math.log(0.2))
    R = synth.rays_helical(6, 7, 9, 0.25, 3.0, 4.5, z_per_turn=0.0)
    ref = oracle.forward(g, G)["I"]
    got = oracle.forward_list(R["o"], R["d"], R["t"], G)["I"]
    # the ray set is stored in binary32: agreement to its rounding
    np.testing.assert_allclose(got, ref, rtol=2e-5, atol=1e-6 * np.abs(ref).max())


def test_adjoint_matches_finite_differences(oracle):
    G = synth.gaussians_uniform(3, 16, half_box=0.3, log_sigma=math.log(0.25))
    R = synth.rays_random(200, 17, radius=0.5, seg=0.3)
    w = np.random.default_rng(18).normal(size=200)
    g = oracle.backward_list(R["o"], R["d"], R["t"], G, w, cut2=1e30)

    def loss(Gx):
        return float(w @ oracle.forward_list(R["o"], R["d"], R["t"], Gx, cut2=1e30)["I"])

    for key, shape in (("mu", 3), ("ls", 3), ("q", 4)):
        for c in range(shape):
            Gp = {k: v.astype(np.float64).copy() for k, v in G.items()}
            Gm = {k: v.astype(np.float64).copy() for k, v in G.items()}
            h = 1e-4
            Gp[key][1, c] += h
            Gm[key][1, c] -= h
            # the oracle takes float32 parameters: use the rounded step
            hp = float(np.float32(Gp[key][1, c]) - np.float32(G[key][1, c]))
            hm = float(np.float32(G[key][1, c]) - np.float32(Gm[key][1, c]))
            fd = (loss({k: v.astype(np.float32) for k, v in Gp.items()})
                  - loss({k: v.astype(np.float32) for k, v in Gm.items()})) / (hp + hm)
            assert fd == pytest.approx(g[key][1, c], rel=2e-3, abs=1e-6), (key, c)


def test_rays_missing_everything_are_zero(oracle):
    G = synth.gaussians_uniform(20, 19, half_box=0.5, log_sigma=math.log(0.05))
    o = np.tile([[5.0, 5.0, 5.0]], (10, 1))
    d = np.tile([[0.0, 0.0, 1.0]], (10, 1))
    t = np.tile([[-np.inf, np.inf]], (10, 1))
    out = oracle.forward_list(o, d, t, G)
    assert np.all(out["I"] == 0.0) and out["pairs"] == 0


def test_pet_3d_direct_planes_are_the_ring_sinogram(oracle):
    """The ring-difference-0 LORs of the 3-D PET generator are the direct
    planes (plane 2r) of the 2-D ring geometry with half the ring pitch."""
    n_rings, pitch, n_ang, n_rad = 6, 4.0, 12, 41
    R = synth.pet_rays_3d(n_rings, pitch, 400.0, 576, n_ang, n_rad, max_ring_diff=2)
    G = synth.gaussians_uniform(40, 33, half_box=60.0, log_sigma=math.log(5.0))
    G["mu"][:, 2] *= 0.15
    g2 = synth.geom_pet(n_ang, n_rad, 2 * n_rings - 1, 400.0, 576, pitch / 2)
    ref = oracle.forward(g2, G)["I"].reshape(2 * n_rings - 1, n_ang, n_rad)
    ix = R["index"]
    sel = ix[:, 0] == ix[:, 1]
    got = oracle.forward_list(R["o"][sel], R["d"][sel], R["t"][sel], G)["I"]
    want = ref[2 * ix[sel, 0], ix[sel, 2], ix[sel, 3]]
    assert np.count_nonzero(want) > 100
    np.testing.assert_allclose(got, want, rtol=2e-5, atol=1e-6 * np.abs(want).max())
    # every ring pair within the difference appears once per (angle, radial)
    n_pairs = sum(1 for a in range(n_rings) for b in range(n_rings) if abs(a - b) <= 2)
    assert R["o"].shape[0] == n_pairs * n_ang * n_rad
    assert len({tuple(r) for r in ix.tolist()}) == ix.shape[0]
