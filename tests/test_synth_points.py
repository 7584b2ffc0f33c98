"""The inputs of the arc vs raw sampling study: radial bin positions, the
point-source sinogram (chord lengths through small spheres), arc-correction
resampling, the blind grid of Gaussians and the FWHM measurement."""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth


def _ring(arc_mode, n_angles=36, n_radial=329, n_planes=3):
    return synth.geom_pet(n_angles, n_radial, n_planes, 400.0, 576, 2.0, arc_mode=arc_mode)


def test_radial_positions():
    k = np.arange(329) - 164
    np.testing.assert_allclose(synth.pet_radial_positions(_ring(0)), k * math.pi * 400.0 / 576, rtol=0, atol=1e-12)
    np.testing.assert_allclose(synth.pet_radial_positions(_ring(1)), 400.0 * np.sin(k * math.pi / 576),
                               rtol=0, atol=1e-12)


@pytest.mark.parametrize("arc_mode", [0, 1])
def test_sphere_projection_area_and_sinusoid(arc_mode):
    """A 20 mm sphere at (50, 30, 0): every projection of the central plane
    integrates over s to the great circle's area pi a^2, a plane 2 mm off
    centre to the area of its smaller circle pi (a^2 - 4), and the projection
    peaks at s = c . e_u (the sinogram's sinusoid)."""
    g = _ring(arc_mode)
    y = synth.point_source_sinogram(g, [(50.0, 30.0, 0.0)], radius=20.0, n_sub=9)
    s = synth.pet_radial_positions(g)
    ds = np.gradient(s)
    np.testing.assert_allclose((y[1] * ds).sum(axis=1), math.pi * 400.0, rtol=2e-3)
    np.testing.assert_allclose((y[0] * ds).sum(axis=1), math.pi * 396.0, rtol=2e-3)
    phi = math.pi * np.arange(36) / 36
    cu = 50.0 * np.cos(phi) + 30.0 * np.sin(phi)
    peak = s[np.argmax(y[1], axis=1)]
    assert np.abs(peak - cu).max() <= np.abs(np.diff(s)).max()


def test_point_source_density_scales():
    g = _ring(1)
    a = synth.point_source_sinogram(g, [(0.0, 100.0, 0.0)], radius=1.0)
    b = synth.point_source_sinogram(g, [(0.0, 100.0, 0.0)], radius=1.0, density=3.0)
    np.testing.assert_allclose(b, 3.0 * a)
    two = synth.point_source_sinogram(g, [(0.0, 100.0, 0.0), (0.0, 10.0, 0.0)], radius=1.0)
    np.testing.assert_allclose(two, a + synth.point_source_sinogram(g, [(0.0, 10.0, 0.0)], radius=1.0))


def test_arc_resample_interpolates_linearly():
    g = _ring(1, n_angles=4, n_planes=2)
    s_raw = synth.pet_radial_positions(g)
    s_arc = synth.pet_radial_positions(dict(g, arc_mode=0))
    y = np.broadcast_to(3.0 + 0.5 * s_raw, (2, 4, 329)).copy()
    out = synth.arc_resample(y, g)
    inside = np.abs(s_arc) <= s_raw.max()
    np.testing.assert_allclose(out[..., inside], np.broadcast_to(3.0 + 0.5 * s_arc[inside], out[..., inside].shape),
                               rtol=1e-12, atol=1e-12)
    assert not out[..., ~inside].any()
    assert (~inside).sum() > 0            # raw bins span less than the arc-corrected ones


def test_grid_gaussians():
    G = synth.grid_gaussians(30.0, 4.0, sigma=2.0, rho=0.5, z=1.5)
    r = np.hypot(G["mu"][:, 0], G["mu"][:, 1])
    assert r.max() <= 30.0 and G["mu"].shape[0] > 0.8 * math.pi * 900 / 16
    np.testing.assert_array_equal(G["mu"][:, 2], np.float32(1.5))
    np.testing.assert_allclose(np.exp(G["ls"]), 2.0, rtol=1e-6)
    np.testing.assert_array_equal(G["rho"], np.float32(0.5))


def test_fwhm():
    h = 0.01
    x = (np.arange(2001) - 1000) * h
    sigma = 1.3
    assert synth.fwhm(np.exp(-x * x / (2 * sigma * sigma)), h) == pytest.approx(
        2 * math.sqrt(2 * math.log(2)) * sigma, rel=1e-4)
    tri = np.maximum(1.0 - np.abs(x) / 2.0, 0.0)       # triangle of half-width 2: FWHM 2, exact
    assert synth.fwhm(tri, h) == pytest.approx(2.0, rel=1e-9)
    assert math.isnan(synth.fwhm(np.ones(10), 1.0))   # no half-maximum crossing


def test_pet_lors_are_the_oracle_lors(oracle):
    """The explicit-ray LORs of a PET ring sinogram (input generator) are the
    oracle's LORs of the same geometry, arc-corrected and raw, with a listed
    angle subset."""
    for arc in (0, 1):
        g = synth.geom_pet(5, 21, 3, 200.0, 288, 4.0, arc_mode=arc)
        g["angles"] = np.array([0.1, 0.7, 1.3, 2.0, 2.9])
        o, d, ta, tb = synth.pet_lors(g)
        n = synth.num_rays(g)
        ro, rd, rta, rtb = oracle.rays(g, np.arange(n))
        np.testing.assert_allclose(o, ro, atol=1e-9)
        np.testing.assert_allclose(d, rd, atol=1e-12)
        np.testing.assert_allclose(ta, rta, atol=1e-9)
        np.testing.assert_allclose(tb, rtb, atol=1e-9)
