"""Pins of the oracle's Epanechnikov kernel, rho (1 - m(x)/kappa^2)_+ with
kappa^2 = 7: the closed form of an isotropic kernel on a line, adaptive
quadrature along finite and half-infinite segments, the projected and the
voxelised mass rho (8 pi / 15) kappa^3 sqrt(det Sigma), and the analytic pair
gradient against central finite differences."""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth

quad = pytest.importorskip("scipy.integrate").quad

K2 = 7.0


def _kernel_along(o, d, mu, P, rho):
    def f(t):
        x = o + t * d - mu
        m = x @ P @ x
        return rho * max(0.0, 1.0 - m / K2)
    return f


def _cov(oracle, ls, q):
    sig, P = oracle.cov(np.asarray([ls], np.float32), np.asarray([q], np.float32))
    return sig[0], P[0]


def test_isotropic_line_closed_form(oracle):
    s, rho = 0.2, 0.8
    mu, ls, q = np.zeros(3), np.full(3, math.log(s)), np.array([1.0, 0, 0, 0])
    s32 = math.exp(float(np.float32(math.log(s))))
    for r in (0.0, 0.1, 0.3, 0.5, 0.52, 0.6):
        v = oracle.pair([-3.0, r, 0.0], [1.0, 0.0, 0.0], -np.inf, np.inf, mu, ls, q, rho, "epanechnikov")[0]
        m = r * r / (s32 * s32)
        want = 4.0 / 3.0 * float(np.float32(rho)) * s32 * max(K2 - m, 0.0) ** 1.5 / K2
        assert v == pytest.approx(want, rel=1e-13, abs=1e-300), r


def test_quadrature_on_finite_and_half_segments(oracle):
    rng = np.random.default_rng(3)
    n_checked = 0
    for _ in range(40):
        mu = rng.uniform(-0.2, 0.2, 3)
        ls = np.log(rng.uniform(0.08, 0.3, 3))
        q = rng.normal(size=4)
        rho = float(rng.uniform(0.2, 1.5))
        _, P = _cov(oracle, ls, q)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        o = rng.uniform(-0.4, 0.4, 3)
        ta, tb = sorted(rng.uniform(-0.6, 0.6, 2))
        if rng.uniform() < 0.3:
            ta = -np.inf
        mu32 = np.asarray(mu, np.float32).astype(np.float64)
        f = _kernel_along(o, d, mu32, P, float(np.float32(rho)))
        lo, hi = (max(ta, -5.0), tb)
        # break the quadrature where the line enters and leaves the support
        e = o - mu32
        A, B, C = d @ P @ d, d @ P @ e, e @ P @ e
        kinks = []
        if C - B * B / A < K2:
            a = math.sqrt((K2 - (C - B * B / A)) / A)
            kinks = [x for x in (-B / A - a, -B / A + a) if lo < x < hi]
        want = quad(f, lo, hi, points=kinks or None, limit=400, epsabs=1e-15, epsrel=1e-13)[0]
        got = oracle.pair(o, d, ta, tb, mu, ls, q, rho, "epanechnikov")[0]
        assert got == pytest.approx(want, rel=1e-9, abs=1e-12)
        n_checked += got > 0
    assert n_checked > 15


def test_projected_mass(oracle):
    """Parallel projection along x summed over a fine detector grid times the
    pixel area equals the kernel's integral rho (8 pi / 15) kappa^3 sqrt(det Sigma)."""
    ls = np.log([0.05, 0.08, 0.06])
    G = dict(mu=np.array([[0.01, -0.02, 0.015]], np.float32), ls=np.array([ls], np.float32),
             q=np.array([[0.8, 0.2, -0.4, 0.3]], np.float32), rho=np.array([0.9], np.float32),
             kernel="epanechnikov")
    W = 241
    p = 0.8 / W
    g = synth.geom_parallel(1, W, W, p, p, -math.inf, math.inf)
    I = oracle.forward(g, G)["I"]
    s = np.exp(ls.astype(np.float32).astype(np.float64))
    mass = float(np.float32(0.9)) * 8.0 * math.pi / 15.0 * K2 ** 1.5 * np.prod(s)
    assert I.sum() * p * p == pytest.approx(mass, rel=2e-4)


def test_voxelised_mass_and_centre(oracle):
    ls = np.log([0.05, 0.07, 0.06])
    G = dict(mu=np.array([[0.0, 0.0, 0.0]], np.float32), ls=np.array([ls], np.float32),
             q=np.array([[0.9, -0.1, 0.3, 0.2]], np.float32), rho=np.array([1.1], np.float32),
             kernel="epanechnikov")
    h = 0.004
    n = 151
    vol = dict(origin=(-h * (n - 1) / 2,) * 3, size=(h, h, h), dims=(n, n, n))
    V = oracle.voxelize(vol, G)["V"]
    assert V[n // 2, n // 2, n // 2] == pytest.approx(float(np.float32(1.1)), rel=1e-15)
    s = np.exp(ls.astype(np.float32).astype(np.float64))
    mass = float(np.float32(1.1)) * 8.0 * math.pi / 15.0 * K2 ** 1.5 * np.prod(s)
    assert V.sum() * h ** 3 == pytest.approx(mass, rel=1e-3)


def test_pair_gradient_matches_finite_differences(oracle):
    rng = np.random.default_rng(5)
    checked = 0
    for trial in range(25):
        mu = rng.uniform(-0.1, 0.1, 3).astype(np.float32)
        ls = np.log(rng.uniform(0.1, 0.3, 3)).astype(np.float32)
        q = rng.normal(size=4).astype(np.float32)
        rho = np.float32(rng.uniform(0.3, 1.2))
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        o = rng.uniform(-0.3, 0.3, 3)
        ta, tb = sorted(rng.uniform(-0.5, 0.5, 2))
        if trial % 3 == 0:
            tb = np.inf
        g = oracle.pair_grad(o, d, ta, tb, mu, ls, q, rho, "epanechnikov")
        if oracle.pair(o, d, ta, tb, mu, ls, q, rho, "epanechnikov")[0] <= 1e-6:
            continue
        checked += 1
        params = [mu, ls, q]
        k = 0
        for arr in params:
            for c in range(arr.size):
                h = 1e-3 * max(1.0, abs(float(arr[c])))
                ap = arr.astype(np.float64).copy(); am = ap.copy()
                ap[c] += h; am[c] -= h
                hp = float(np.float32(ap[c]) - arr[c]); hm = float(arr[c] - np.float32(am[c]))
                args_p = [x if x is not arr else ap.astype(np.float32) for x in params]
                args_m = [x if x is not arr else am.astype(np.float32) for x in params]
                fp = oracle.pair(o, d, ta, tb, *args_p, rho, "epanechnikov")[0]
                fm = oracle.pair(o, d, ta, tb, *args_m, rho, "epanechnikov")[0]
                fd = (fp - fm) / (hp + hm)
                assert fd == pytest.approx(g[k], rel=5e-3, abs=5e-5 * (1 + abs(g[k]))), (trial, k)
                k += 1
        assert g[10] == pytest.approx(oracle.pair(o, d, ta, tb, mu, ls, q, 1.0, "epanechnikov")[0], rel=1e-12)
    assert checked > 10
