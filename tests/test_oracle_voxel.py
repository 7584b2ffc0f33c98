"""Pins of the oracle's voxeliser (density field of the Gaussians on a grid):
the centre value, the separable closed form of an axis-aligned Gaussian, the
mass invariant of a rotated one, the 3-sigma cut, the box loop against brute
force, and the line sums of the grid against the projector's line integrals."""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth


def _one(mu, ls, q, rho):
    return dict(mu=np.array([mu], np.float32), ls=np.array([ls], np.float32),
                q=np.array([q], np.float32), rho=np.array([rho], np.float32))


def test_value_at_the_centre_is_rho(oracle):
    G = _one([0.125, -0.25, 0.5], [-2.0, -1.5, -1.8], [0.9, 0.1, -0.3, 0.2], 0.75)
    vol = dict(origin=(0.125, -0.25, 0.5), size=(0.1, 0.1, 0.1), dims=(3, 2, 2))
    V = oracle.voxelize(vol, G)["V"]
    assert V[0, 0, 0] == pytest.approx(0.75, rel=1e-15)


def test_axis_aligned_closed_form(oracle):
    s = np.array([0.07, 0.11, 0.05])
    mu = np.array([0.013, -0.021, 0.008])
    G = _one(mu, np.log(s), [1.0, 0.0, 0.0, 0.0], 1.3)
    vol = dict(origin=(-0.3, -0.4, -0.25), size=(0.02, 0.025, 0.02), dims=(31, 33, 26))
    V = oracle.voxelize(vol, G, cut2=1e30)["V"]
    s32 = np.exp(np.log(s).astype(np.float32).astype(np.float64))
    mu32 = mu.astype(np.float32).astype(np.float64)
    x = vol["origin"][0] + vol["size"][0] * np.arange(31) - mu32[0]
    y = vol["origin"][1] + vol["size"][1] * np.arange(33) - mu32[1]
    z = vol["origin"][2] + vol["size"][2] * np.arange(26) - mu32[2]
    want = (float(np.float32(1.3)) * np.exp(-z[:, None, None] ** 2 / (2 * s32[2] ** 2))
            * np.exp(-y[None, :, None] ** 2 / (2 * s32[1] ** 2)) * np.exp(-x[None, None, :] ** 2 / (2 * s32[0] ** 2)))
    np.testing.assert_allclose(V, want, rtol=1e-12, atol=1e-300)


def test_mass_of_a_rotated_gaussian(oracle):
    """sum V h^3 = rho (2 pi)^{3/2} s1 s2 s3 (Poisson summation: the grid error
    is ~exp(-2 pi^2 sigma^2 / h^2), negligible at sigma >= 2 h)."""
    ls = np.log([0.06, 0.09, 0.045])
    G = _one([0.01, 0.02, -0.015], ls, [0.7, 0.3, -0.5, 0.4], 0.9)
    h = 0.015
    vol = dict(origin=(-0.6, -0.6, -0.6), size=(h, h, h), dims=(81, 81, 81))
    V = oracle.voxelize(vol, G, cut2=1e30)["V"]
    s = np.exp(ls.astype(np.float32).astype(np.float64))
    mass = float(np.float32(0.9)) * (2 * math.pi) ** 1.5 * np.prod(s)
    assert V.sum() * h ** 3 == pytest.approx(mass, rel=1e-9)


def test_cut_at_three_sigma(oracle):
    G = _one([0.0, 0.0, 0.0], np.log([0.1, 0.1, 0.1]), [1.0, 0, 0, 0], 1.0)
    vol = dict(origin=(-0.5, -0.5, -0.5), size=(0.01, 0.01, 0.5), dims=(101, 101, 3))
    cut = oracle.voxelize(vol, G)
    full = oracle.voxelize(vol, G, cut2=1e30)["V"]
    x = -0.5 + 0.01 * np.arange(101)
    s = math.exp(float(np.float32(math.log(0.1))))
    r2 = (x[None, :] ** 2 + x[:, None] ** 2) / s ** 2          # z = 0 slice
    sl = cut["V"][1]
    assert np.all(sl[r2 > 9.0 + 1e-6] == 0.0)
    np.testing.assert_array_equal(sl[r2 < 9.0 - 1e-3], full[1][r2 < 9.0 - 1e-3])
    assert np.all(cut["V"][0] == 0.0)                           # z = -0.5 is 5 sigma away


def test_box_loop_equals_brute_force(oracle):
    G = synth.gaussians_uniform(60, 31, half_box=0.8, log_sigma=math.log(0.08))
    vol = dict(origin=(-1.0, -0.9, -1.1), size=(0.07, 0.06, 0.08), dims=(29, 31, 28))
    a = oracle.voxelize(vol, G)
    b = oracle.voxelize(vol, G, brute=True)
    for k in ("V", "V_lo", "V_hi"):
        np.testing.assert_array_equal(a[k], b[k])
    assert np.count_nonzero(a["V"]) > 1000


def test_line_sums_are_projections(oracle):
    """Summing the grid along x gives the line integrals of rays along x
    (parallel beam at angle 0: d = e_x, detector u = y, v = z), exactly up to
    the grid's Poisson-summation error."""
    G = synth.gaussians_uniform(5, 32, half_box=0.3, log_sigma=math.log(0.07))
    W, H, p = 24, 20, 0.03
    g = synth.geom_parallel(1, H, W, p, p, -math.inf, math.inf)
    I = oracle.forward(g, G, cut2=1e30)["I"].reshape(H, W)
    h = 0.012
    nx = 121
    vol = dict(origin=(-h * (nx - 1) / 2, -p * (W - 1) / 2, -p * (H - 1) / 2), size=(h, p, p), dims=(nx, W, H))
    V = oracle.voxelize(vol, G, cut2=1e30)["V"]                 # [z = row][y = col][x]
    np.testing.assert_allclose(V.sum(axis=2) * h, I, rtol=1e-9, atol=1e-12 * I.max())
