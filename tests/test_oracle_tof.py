"""Pins of the oracle's time-of-flight weighting on explicit rays: the
weighted line integral against adaptive quadrature, the sum over a dense set
of TOF centres against the plain projection, an infinite width as no TOF, and
the adjoint against central finite differences."""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth

quad = pytest.importorskip("scipy.integrate").quad


def _one(rng):
    mu = rng.uniform(-0.2, 0.2, 3).astype(np.float32)
    ls = np.log(rng.uniform(0.06, 0.2, 3)).astype(np.float32)
    q = rng.normal(size=4).astype(np.float32)
    rho = np.float32(rng.uniform(0.3, 1.2))
    return dict(mu=mu[None], ls=ls[None], q=q[None], rho=np.array([rho]))


def test_weighted_integral_matches_quadrature(oracle):
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(30):
        G = _one(rng)
        _, P = oracle.cov(G["ls"], G["q"])
        P = P[0]
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        o = rng.uniform(-0.3, 0.3, 3)
        ta, tb = sorted(rng.uniform(-0.8, 0.8, 2))
        if trial % 3 == 0:
            ta, tb = -np.inf, np.inf
        tc, sT = float(rng.uniform(-0.4, 0.4)), float(rng.uniform(0.03, 0.3))
        mu = G["mu"][0].astype(np.float64)
        rho = float(G["rho"][0])

        def f(t):
            x = o + t * d - mu
            return rho * math.exp(-0.5 * x @ P @ x) * math.exp(-0.5 * (t - tc) ** 2 / sT ** 2) / (
                math.sqrt(2 * math.pi) * sT)
        lo, hi = max(ta, tc - 12 * sT), min(tb, tc + 12 * sT)
        want = quad(f, lo, hi, points=[tc] if lo < tc < hi else None, limit=400, epsabs=1e-15,
                    epsrel=1e-12)[0] if lo < hi else 0.0
        got = oracle.forward_list(o[None], d[None], np.array([[ta, tb]]), G, cut2=1e30,
                                  tof=np.array([[tc, sT]]))["I"][0]
        assert got == pytest.approx(want, rel=1e-8, abs=1e-13)
        checked += got > 1e-6
    assert checked > 10


def test_dense_tof_centres_sum_to_the_plain_projection(oracle):
    G = synth.gaussians_uniform(20, 12, half_box=0.4, log_sigma=math.log(0.08))
    R = synth.rays_random(50, 13, radius=0.5)
    plain = oracle.forward_list(R["o"], R["d"], R["t"], G, cut2=1e30)["I"]
    sT, step = 0.05, 0.02
    centres = np.arange(-3.0, 3.0 + step / 2, step)
    n = R["o"].shape[0]
    total = np.zeros(n)
    for c in centres:
        tof = np.tile([c, sT], (n, 1))
        total += oracle.forward_list(R["o"], R["d"], R["t"], G, cut2=1e30, tof=tof)["I"] * step
    # o is within 0.5 of the origin and the Gaussians within ~0.7: every
    # contribution lies well inside [-3, 3] along the ray
    np.testing.assert_allclose(total, plain, rtol=1e-9, atol=1e-12)


def test_infinite_width_is_no_tof(oracle):
    G = synth.gaussians_uniform(30, 14, half_box=0.5, log_sigma=math.log(0.1))
    R = synth.rays_random(80, 15, radius=0.6, seg=0.4)
    a = oracle.forward_list(R["o"], R["d"], R["t"], G)["I"]
    b = oracle.forward_list(R["o"], R["d"], R["t"], G, tof=np.tile([0.0, np.inf], (80, 1)))["I"]
    np.testing.assert_array_equal(a, b)


def test_adjoint_matches_finite_differences(oracle):
    G = synth.gaussians_uniform(3, 16, half_box=0.3, log_sigma=math.log(0.2))
    R = synth.rays_random(150, 17, radius=0.5, seg=0.35)
    rng = np.random.default_rng(18)
    tof = np.stack([rng.uniform(-0.3, 0.3, 150), rng.uniform(0.05, 0.2, 150)], 1)
    w = rng.normal(size=150)
    g = oracle.backward_list(R["o"], R["d"], R["t"], G, w, cut2=1e30, tof=tof)

    def loss(Gx):
        return float(w @ oracle.forward_list(R["o"], R["d"], R["t"], Gx, cut2=1e30, tof=tof)["I"])

    for key, shape in (("mu", 3), ("ls", 3), ("q", 4), ("rho", 1)):
        for c in range(shape):
            Gp = {k: v.astype(np.float64).copy() for k, v in G.items()}
            Gm = {k: v.astype(np.float64).copy() for k, v in G.items()}
            h = 1e-4
            if key == "rho":
                Gp[key][1] += h; Gm[key][1] -= h
                hp = float(np.float32(Gp[key][1]) - np.float32(G[key][1]))
                hm = float(np.float32(G[key][1]) - np.float32(Gm[key][1]))
                want = g[key][1]
            else:
                Gp[key][1, c] += h; Gm[key][1, c] -= h
                hp = float(np.float32(Gp[key][1, c]) - np.float32(G[key][1, c]))
                hm = float(np.float32(G[key][1, c]) - np.float32(Gm[key][1, c]))
                want = g[key][1, c]
            fd = (loss({k: v.astype(np.float32) for k, v in Gp.items()})
                  - loss({k: v.astype(np.float32) for k, v in Gm.items()})) / (hp + hm)
            assert fd == pytest.approx(want, rel=2e-3, abs=1e-6), (key, c)
