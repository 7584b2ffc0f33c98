"""Pins of the phantom ground truth used by the reconstruction demo: exact
chord integrals (sphere closed form, quadrature of the density along random
rays), detector rays against the oracle's, and the PSNR definition."""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth


def test_sphere_chord_closed_form():
    ph = dict(axes=np.array([[0.3, 0.3, 0.3]]), rot=np.eye(3)[None], centre=np.array([[0.1, 0.0, 0.0]]),
              density=np.array([2.0]))
    b = np.array([0.0, 0.05, 0.1, 0.15, 0.2, 0.25, 0.29, 0.35])   # not tangent: sqrt of a rounded 0
    o = np.stack([np.full_like(b, -5.0), b, np.zeros_like(b)], 1)
    d = np.tile([1.0, 0.0, 0.0], (b.size, 1))
    got = synth.phantom_projection(ph, o, d, np.full(b.size, -np.inf), np.full(b.size, np.inf))
    want = 2.0 * 2.0 * np.sqrt(np.maximum(0.09 - b ** 2, 0.0))
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)
    # a segment that ends at the centre sees half the chord
    half = synth.phantom_projection(ph, o, d, np.full(b.size, -np.inf), np.full(b.size, 5.1))
    np.testing.assert_allclose(half, want / 2, rtol=1e-12, atol=1e-15)


def test_chords_match_quadrature_of_the_density():
    ph = synth.ellipsoid_phantom(12, seed=1000, semi=(0.05, 0.6), dens=(0.1, 1.0))
    R = synth.rays_random(40, 5, radius=0.6, seg=1.5)
    d = R["d"].astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = R["o"].astype(np.float64)
    got = synth.phantom_projection(ph, o, d, R["t"][:, 0].astype(np.float64), R["t"][:, 1].astype(np.float64))
    m = 40000
    t = -1.5 + 3.0 * (np.arange(m) + 0.5) / m
    for r in range(40):
        pts = o[r] + t[:, None] * d[r]
        q = synth._phantom_density(ph, pts).sum() * 3.0 / m
        assert got[r] == pytest.approx(q, abs=2e-4)
    assert np.count_nonzero(got) > 20


@pytest.mark.parametrize("kind", ["cone", "parallel"])
def test_detector_rays_match_the_oracle(oracle, kind):
    g = synth.geom_cone(3, 5, 6, 0.2, 0.2, 3.0, 4.5) if kind == "cone" else \
        synth.geom_parallel(3, 5, 6, 0.2, 0.2, -1.0, 1.5)
    o, d, ta, tb = synth.detector_rays(g)
    idx = np.arange(synth.num_rays(g))
    ro, rd, rta, rtb = oracle.rays(g, idx)
    # the same lines and segments (the origins may differ along the line)
    for a in range(idx.size):
        pa = o[a] + ta[a] * d[a]
        pb = o[a] + tb[a] * d[a]
        qa = ro[a] + rta[a] * rd[a]
        qb = ro[a] + rtb[a] * rd[a]
        np.testing.assert_allclose(d[a], rd[a], atol=1e-14)
        np.testing.assert_allclose(pa, qa, atol=1e-12)
        np.testing.assert_allclose(pb, qb, atol=1e-12)


def test_psnr():
    ref = np.linspace(0.0, 2.0, 1000)
    assert synth.psnr(ref + 0.02, ref) == pytest.approx(10 * math.log10(4.0 / 4e-4))
