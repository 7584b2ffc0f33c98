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


def _sinogram_lors(oracle, gd):
    """The LORs of a PET sinogram geometry without time of flight, as
    explicit rays (the oracle's own LOR definition)."""
    g0 = {k: v for k, v in gd.items() if k not in ("n_tof", "tof_spacing", "tof_sigma")}
    n = synth.num_rays(g0)
    o, d, ta, tb = oracle.rays(g0, np.arange(n))
    return g0, o, d, np.stack([ta, tb], 1)


@pytest.mark.parametrize("kind", ["pet", "pet3d"])
def test_tof_sinogram_is_the_explicit_tof_rays(oracle, kind):
    """Structured TOF sinograms (bin k of every LOR centred at (k - (n-1)/2)
    spacing from the LOR's midpoint) equal the same LORs traced as explicit
    rays with time of flight, forward and adjoint."""
    if kind == "pet":
        gd = synth.geom_pet(6, 41, 5, 200.0, 288, 4.0)
    else:
        gd = synth.geom_pet3d(5, 41, 4, 200.0, 288, 4.0, 1)
    gd = synth.with_tof_bins(gd, 5, 30.0, 25.0)
    G = synth.gaussians_uniform(40, 31, half_box=60.0, log_sigma=math.log(6.0))
    G["mu"][:, 2] *= 0.05
    g0, o, d, t = _sinogram_lors(oracle, gd)
    nl = o.shape[0]
    nb = gd["n_tof"]
    centres = ((np.arange(nb) - 0.5 * (nb - 1)) * gd["tof_spacing"])
    # explicit rays, TOF-bin major like the sinogram: the LOR midpoint is t = 0
    mid = 0.5 * (t[:, 0] + t[:, 1])
    assert np.allclose(mid, 0.0, atol=1e-9)
    O = np.tile(o, (nb, 1)); D = np.tile(d, (nb, 1)); T = np.tile(t, (nb, 1))
    tof = np.stack([np.repeat(centres, nl), np.full(nb * nl, gd["tof_sigma"])], 1)
    live = ~((T[:, 0] == 0.0) & (T[:, 1] == 0.0))     # 3-D PET rows without a ring pair
    ref = oracle.forward_list(O[live], D[live], T[live], G, tof=tof[live])
    got = oracle.forward(gd, G)
    assert got["I"].size == nb * nl
    want = np.zeros(nb * nl)
    want[live] = ref["I"]
    assert np.count_nonzero(want) > 100
    np.testing.assert_allclose(got["I"], want, rtol=1e-12, atol=1e-14 * np.abs(want).max())
    w = synth.random_weights(nb * nl, 4).astype(np.float64)
    gb = oracle.backward(gd, G, w)
    gl = oracle.backward_list(O[live], D[live], T[live], G, w[live], tof=tof[live])
    for k in ("mu", "ls", "q", "rho"):
        np.testing.assert_allclose(gb[k], gl[k], rtol=1e-9, atol=1e-12 * np.abs(gl[k]).max())


def test_tof_bins_sum_to_the_plain_sinogram(oracle):
    """Dense TOF bins (spacing small against the TOF width) over the whole
    LOR sum, times the spacing, to the sinogram without time of flight (the
    weights form a partition of unity up to the Riemann-sum error)."""
    g0 = synth.geom_pet(4, 31, 3, 200.0, 288, 4.0)
    G = synth.gaussians_uniform(25, 32, half_box=50.0, log_sigma=math.log(5.0))
    G["mu"][:, 2] *= 0.05
    plain = oracle.forward(g0, G)["I"]
    h = 4.0
    n = int(2 * 200.0 / h) + 41
    gd = synth.with_tof_bins(g0, n, h, 12.0)
    tof = oracle.forward(gd, G)["I"].reshape(n, -1)
    np.testing.assert_allclose(h * tof.sum(axis=0), plain, rtol=1e-9, atol=1e-12 * plain.max())
