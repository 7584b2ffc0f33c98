"""Pins of the FP64 oracle against things other than itself.

Each test fixes the oracle to a closed form, a library routine, quadrature,
finite differences or an invariant that a plausible mistake (a dropped term,
a wrong sign or index, a transposed operand) would break.  CPU only.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special
from scipy.spatial.transform import Rotation

from paper_2602_01057_gb300 import synth

INF = float("inf")


def _gauss_density(x, mu, P):
    d = x - mu
    return math.exp(-0.5 * d @ P @ d)


def _rand_pair(rng, finite=True):
    mu = rng.uniform(-1, 1, 3).astype(np.float32)
    ls = rng.normal(math.log(0.1), 0.4, 3).astype(np.float32)
    q = rng.normal(size=4).astype(np.float32)
    rho = np.float32(rng.uniform(0.2, 2.0))
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    # ray passing within ~2 sigma of mu, origin some distance back along d
    off = rng.normal(size=3) * 0.12
    o = mu.astype(np.float64) + off - d * rng.uniform(0.5, 3.0)
    if finite:
        ta, tb = sorted(rng.uniform(0.0, 4.0, 2))
    else:
        ta, tb = -INF, INF
    return o, d, ta, tb, mu, ls, q, rho


# --------------------------------------------------------------------------
# closed forms (Eqs. 9-12)
# --------------------------------------------------------------------------

def test_isotropic_closed_form(oracle):
    """Isotropic Gaussian, impact distance r: rho sigma sqrt(2 pi) exp(-r^2/2 sigma^2)."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        sigma = float(np.exp(rng.uniform(-4, 0)))
        ls = np.full(3, math.log(sigma), np.float32)
        sigma = float(np.exp(np.float64(ls[0])))
        q = rng.normal(size=4).astype(np.float32)
        mu = rng.uniform(-1, 1, 3).astype(np.float32)
        rho = float(np.float32(rng.uniform(0.1, 3)))
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        perp = np.cross(d, rng.normal(size=3)); perp /= np.linalg.norm(perp)
        r = rng.uniform(0, 3) * sigma
        o = mu.astype(np.float64) + r * perp - 5.0 * d
        val, m, A, B, C = oracle.pair(o, d, -INF, INF, mu, ls, q, rho)
        expect = rho * sigma * math.sqrt(2 * math.pi) * math.exp(-r * r / (2 * sigma * sigma))
        assert val == pytest.approx(expect, rel=1e-11, abs=1e-300)
        assert m == pytest.approx((r / sigma) ** 2, rel=1e-9, abs=1e-12)
        assert A == pytest.approx(1.0 / sigma ** 2, rel=1e-12)


def test_central_ray_principal_axis(oracle):
    """A ray through mu along principal axis k integrates to rho s_k sqrt(2 pi)."""
    rng = np.random.default_rng(2)
    for _ in range(30):
        mu = rng.uniform(-1, 1, 3).astype(np.float32)
        ls = rng.normal(math.log(0.1), 0.5, 3).astype(np.float32)
        qf = rng.normal(size=4).astype(np.float32)
        rho = float(np.float32(rng.uniform(0.1, 3)))
        w, x, y, z = (qf / np.linalg.norm(qf.astype(np.float64)))
        Rm = Rotation.from_quat([x, y, z, w]).as_matrix()
        for k in range(3):
            d = Rm[:, k]
            o = mu.astype(np.float64) - 3.0 * d
            val = oracle.pair(o, d, -INF, INF, mu, ls, qf, rho)[0]
            s_k = math.exp(float(ls[k]))
            assert val == pytest.approx(rho * s_k * math.sqrt(2 * math.pi), rel=1e-10)


def test_rotation_matches_library(oracle):
    """Sigma = R S S^T R^T with R from scipy's quaternion routine (scalar last)."""
    rng = np.random.default_rng(3)
    n = 64
    ls = rng.normal(-2, 0.5, (n, 3)).astype(np.float32)
    q = rng.normal(size=(n, 4)).astype(np.float32)
    sig, P = oracle.cov(ls, q)
    for k in range(n):
        w, x, y, z = q[k].astype(np.float64)
        Rm = Rotation.from_quat([x, y, z, w]).as_matrix()
        S2 = np.diag(np.exp(2 * ls[k].astype(np.float64)))
        np.testing.assert_allclose(sig[k], Rm @ S2 @ Rm.T, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(sig[k] @ P[k], np.eye(3), atol=1e-10)
        assert np.linalg.det(sig[k]) == pytest.approx(math.exp(2 * float(ls[k].astype(np.float64).sum())), rel=1e-10)


# --------------------------------------------------------------------------
# quadrature on tiny inputs (finite segments, the erf form)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("finite", [True, False])
def test_pair_matches_quadrature(oracle, finite):
    rng = np.random.default_rng(4 if finite else 5)
    for _ in range(40):
        o, d, ta, tb, mu, ls, q, rho = _rand_pair(rng, finite)
        sig, P = oracle.cov(ls, q)
        P = P[0]
        mu64 = mu.astype(np.float64)
        f = lambda t: float(rho) * _gauss_density(o + t * d, mu64, P)
        if finite:
            ref, err = integrate.quad(f, ta, tb, epsabs=0, epsrel=1e-13, limit=400,
                                      points=None)
        else:
            # integrate over a window that holds all mass around the minimum
            val, m, A, B, C = oracle.pair(o, d, ta, tb, mu, ls, q, rho)
            tc, w = -B / A, 40.0 / math.sqrt(A)
            ref, err = integrate.quad(f, tc - w, tc + w, epsabs=0, epsrel=1e-13, limit=400)
        got = oracle.pair(o, d, ta, tb, mu, ls, q, rho)[0]
        assert got == pytest.approx(ref, rel=1e-9, abs=1e-14 * max(1.0, abs(ref)))


def test_segment_beyond_gaussian_uses_stable_tail(oracle):
    """A Gaussian far beyond the segment end: tiny but accurate (erfc branch)."""
    mu = np.array([0.0, 0.0, 1.0], np.float32)
    ls = np.full(3, math.log(0.1), np.float32)
    q = np.array([1, 0, 0, 0], np.float32)
    d = np.array([0.0, 0.0, 1.0])
    o = np.array([0.0, 0.0, 0.0])
    for tb in (0.3, 0.5, 0.6):
        got = oracle.pair(o, d, 0.0, tb, mu, ls, q, 1.0)[0]
        s = float(np.exp(np.float64(ls[0])))
        expect = s * math.sqrt(math.pi / 2) * (special.erfc((1 - tb) / (s * math.sqrt(2)))
                                               - special.erfc(1 / (s * math.sqrt(2))))
        assert got == pytest.approx(expect, rel=1e-12)


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def _rotate_quat(Rm, q):
    w, x, y, z = q.astype(np.float64)
    r = Rotation.from_matrix(Rm) * Rotation.from_quat([x, y, z, w])
    x, y, z, w = r.as_quat()
    return np.array([w, x, y, z], np.float32)


def test_joint_rotation_translation_invariance(oracle):
    """Moving ray and Gaussian together leaves the integral unchanged."""
    rng = np.random.default_rng(6)
    for _ in range(30):
        o, d, ta, tb, mu, ls, q, rho = _rand_pair(rng, True)
        base = oracle.pair(o, d, ta, tb, mu, ls, q, rho)[0]
        Rm = Rotation.random(random_state=rng.integers(1 << 30)).as_matrix()
        t = rng.uniform(-2, 2, 3).astype(np.float32).astype(np.float64)
        q2 = _rotate_quat(Rm, q)
        # the Gaussian rotated by Rm about mu, on the ray (o, d), equals the
        # original Gaussian on the ray rotated by Rm^T about mu
        o_r = Rm.T @ (o - mu.astype(np.float64)) + mu.astype(np.float64)
        d_r = Rm.T @ d
        rotated_gauss = oracle.pair(o, d, ta, tb, mu, ls, q2, rho)[0]
        rotated_ray = oracle.pair(o_r, d_r, ta, tb, mu, ls, q, rho)[0]
        assert rotated_gauss == pytest.approx(rotated_ray, rel=1e-6)
        mu_t = (mu.astype(np.float64) + t).astype(np.float32)
        shift = mu_t.astype(np.float64) - mu.astype(np.float64)
        val_t = oracle.pair(o + shift, d, ta, tb, mu_t, ls, q, rho)[0]
        assert val_t == pytest.approx(base, rel=1e-9)


def test_scale_covariance(oracle):
    """x -> k x (positions, sizes and segment scaled): I -> k I."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        o, d, ta, tb, mu, ls, q, rho = _rand_pair(rng, True)
        k = 2.0 ** int(rng.integers(-3, 4))  # exact in binary
        base = oracle.pair(o, d, ta, tb, mu, ls, q, rho)[0]
        ls2 = (ls.astype(np.float64) + math.log(k)).astype(np.float32)
        # the log shift is not exact in float32: compare against the exact sizes
        ratio = float(np.exp(ls2.astype(np.float64) - ls.astype(np.float64)).mean())
        val = oracle.pair(o * k, d, ta * k, tb * k, (mu * k).astype(np.float32), ls2, q, rho)[0]
        assert val == pytest.approx(k * base, rel=2e-6)
        assert ratio == pytest.approx(k, rel=1e-6)


def test_permutation_linearity_additivity(oracle):
    g = synth.geom_parallel(3, 12, 10, 0.2, 0.2, -2.0, 2.0)
    G = synth.gaussians_uniform(40, 8, half_box=0.8, log_sigma=math.log(0.15))
    base = oracle.forward(g, G, cut2=1e30)["I"]
    perm = np.random.default_rng(0).permutation(40)
    Gp = {k: v[perm] for k, v in G.items()}
    np.testing.assert_allclose(oracle.forward(g, Gp, cut2=1e30)["I"], base, rtol=1e-13, atol=1e-15)
    G2 = dict(G, rho=(G["rho"] * 2).astype(np.float32))
    np.testing.assert_allclose(oracle.forward(g, G2, cut2=1e30)["I"], 2 * base, rtol=1e-13)
    Ga = {k: v[:17] for k, v in G.items()}
    Gb = {k: v[17:] for k, v in G.items()}
    s = oracle.forward(g, Ga, cut2=1e30)["I"] + oracle.forward(g, Gb, cut2=1e30)["I"]
    np.testing.assert_allclose(s, base, rtol=1e-12, atol=1e-15)


def test_mass_invariant_parallel_beam(oracle):
    """Pixel sum x h^2 = rho (2 pi)^{3/2} s1 s2 s3 in every view (Poisson
    summation error ~ exp(-2 pi^2 sigma^2/h^2) is far below 1e-12 here)."""
    h = 2.0 / 64
    g = synth.geom_parallel(16, 64, 64, h, h, -2.0, 2.0)
    G = dict(mu=np.array([[0.1, -0.2, 0.05]], np.float32),
             ls=np.array([[math.log(0.06), math.log(0.09), math.log(0.05)]], np.float32),
             q=np.array([[0.3, -0.5, 0.7, 0.2]], np.float32),
             rho=np.array([0.7], np.float32))
    I = oracle.forward(g, G, cut2=1e30)["I"].reshape(16, 64, 64)
    s = np.exp(G["ls"][0].astype(np.float64))
    mass = float(G["rho"][0]) * (2 * math.pi) ** 1.5 * s.prod()
    np.testing.assert_allclose(I.sum(axis=(1, 2)) * h * h, mass, rtol=1e-11)


def test_parallel_beam_is_exact_2d_gaussian(oracle):
    """Parallel beam: I(u, v) = rho sqrt(2 pi/A) exp(-1/2 du^T Sigma2^-1 du)
    with Sigma2 the projected 2x2 covariance."""
    g = synth.geom_parallel(4, 20, 24, 0.05, 0.05, -3.0, 3.0, span=2.0)
    G = synth.gaussians_uniform(1, 11, half_box=0.3, log_sigma=math.log(0.12))
    I = oracle.forward(g, G, cut2=1e30)["I"].reshape(4, 20, 24)
    sig, P = oracle.cov(G["ls"], G["q"])
    sig, P = sig[0], P[0]
    mu = G["mu"][0].astype(np.float64)
    u, v = oracle.tables(g)
    for vi, th in enumerate(g["angles"]):
        ew = np.array([math.cos(th), math.sin(th), 0.0])
        eu = np.array([-math.sin(th), math.cos(th), 0.0])
        ev = np.array([0.0, 0.0, 1.0])
        E = np.stack([eu, ev])
        S2 = E @ sig @ E.T
        A = ew @ P @ ew
        du = np.stack(np.meshgrid(v - mu @ ev, u - mu @ eu, indexing="ij"), axis=-1)[..., ::-1]
        m = np.einsum("...i,ij,...j->...", du, np.linalg.inv(S2), du)
        ref = float(G["rho"][0]) * np.sqrt(2 * math.pi / A) * np.exp(-0.5 * m)
        np.testing.assert_allclose(I[vi], ref, rtol=1e-9, atol=1e-14)


def test_cone_beam_tends_to_parallel(oracle):
    """Source distance -> infinity: cone-beam projection -> parallel-beam."""
    G = synth.gaussians_uniform(5, 12, half_box=0.08, log_sigma=math.log(0.05))
    par = synth.geom_parallel(3, 16, 16, 0.02, 0.02, -1.5, 1.5, span=2 * math.pi)
    dso = 1.0e4
    dsd = dso + 5.0
    mag = dsd / dso
    cone = synth.geom_cone(3, 16, 16, 0.02 * mag, 0.02 * mag, dso, dsd, span=2 * math.pi)
    a = oracle.forward(par, G, cut2=1e30)["I"]
    b = oracle.forward(cone, G, cut2=1e30)["I"]
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 2e-5


def test_pet_point_source_traces_sinusoid(oracle):
    """A point-like Gaussian at radius r, angle phi0 peaks at
    s(phi) = r cos(phi - phi0) (arc-corrected: uniform bins; raw: s = R sin)."""
    r, phi0 = 150.0, 0.7
    mu = np.array([[r * math.cos(phi0), r * math.sin(phi0), 0.0]], np.float32)
    G = dict(mu=mu, ls=np.full((1, 3), math.log(3.0), np.float32),
             q=np.array([[1, 0, 0, 0]], np.float32), rho=np.ones(1, np.float32))
    for arc in (0, 1):
        g = synth.geom_pet(36, 329, 3, 400.0, 576, 2.0, arc_mode=arc)
        I = oracle.forward(g, G, cut2=1e30)["I"].reshape(3, 36, 329)[1]
        u, _ = oracle.tables(g)
        du = np.gradient(u)   # local bin width (uniform when arc-corrected)
        for j in range(36):
            phi = math.pi * j / 36
            s_exp = r * math.cos(phi - phi0)
            w = I[j] * du
            s_est = float((w * u).sum() / w.sum())   # centroid of the radial profile
            assert s_est == pytest.approx(s_exp, abs=0.02)
        if arc == 1:
            c = (329 - 1) / 2
            k = np.arange(329)
            np.testing.assert_allclose(u, 400.0 * np.sin((k - c) * math.pi / 576), rtol=1e-14)
            kk = 576 / math.pi * np.arcsin(u / 400.0) + c
            np.testing.assert_allclose(kk, k, atol=1e-9)
        else:
            np.testing.assert_allclose(np.diff(u), math.pi * 400.0 / 576, rtol=1e-12)


def test_cone_geometry_fov():
    """c2: the magnified 256 mm field of view fills the 256-pixel panel."""
    g = synth.geom_c2()
    half = 0.5 * (g["n_cols"]) * g["pitch_u"] * g["dso"] / g["dsd"]
    assert half == pytest.approx(1.0, rel=1e-12)


# --------------------------------------------------------------------------
# the oracle's own bounding-box loop equals brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["parallel", "cone", "pet_arc", "pet_raw"])
def test_fast_equals_brute(oracle, kind):
    if kind == "parallel":
        g = synth.geom_parallel(5, 20, 23, 0.1, 0.1, -2.0, 2.0)
        G = synth.gaussians_uniform(60, 21, log_sigma=math.log(0.1))
    elif kind == "cone":
        g = synth.geom_cone(5, 21, 19, 0.15, 0.15, 3.0, 4.5)
        G = synth.gaussians_uniform(60, 22, log_sigma=math.log(0.1))
    else:
        g = synth.geom_pet(7, 41, 9, 400.0, 576, 2.0, arc_mode=0 if kind == "pet_arc" else 1)
        G = synth.gaussians_uniform(60, 23, half_box=40.0, log_sigma=math.log(3.0))
        G["mu"][:, 2] *= 0.2
    a = oracle.forward(g, G)
    b = oracle.forward(g, G, brute=True)
    for key in ("I", "I_lo", "I_hi"):
        np.testing.assert_array_equal(a[key], b[key])
    assert a["pairs"] == b["pairs"] and a["pairs"] > 0
    w = synth.random_weights(a["I"].size, 5)
    ga = oracle.backward(g, G, w)
    gb = oracle.backward(g, G, w, brute=True)
    for key in ("mu", "ls", "q", "rho"):
        np.testing.assert_array_equal(ga[key], gb[key])
        np.testing.assert_array_equal(ga["lo"][key], gb["lo"][key])
        np.testing.assert_array_equal(ga["hi"][key], gb["hi"][key])
        assert np.all(ga["lo"][key] <= ga[key]) and np.all(ga[key] <= ga["hi"][key])


def test_sampled_rays_equal_full(oracle):
    g = synth.geom_cone(4, 16, 16, 0.2, 0.2, 3.0, 4.5)
    G = synth.gaussians_uniform(50, 31, log_sigma=math.log(0.1))
    full = oracle.forward(g, G)
    idx = np.random.default_rng(0).choice(full["I"].size, 100, replace=False)
    part = oracle.forward_rays(g, G, idx)
    for key in ("I", "I_lo", "I_hi"):
        np.testing.assert_allclose(part[key], full[key][idx], rtol=1e-13, atol=1e-300)


# --------------------------------------------------------------------------
# gradients: analytic (O4) vs central finite differences of the oracle
# --------------------------------------------------------------------------

def _params_vec(mu, ls, q, rho):
    return np.concatenate([mu, ls, q, [rho]]).astype(np.float64)


def test_pair_gradient_finite_differences(oracle):
    rng = np.random.default_rng(41)
    for trial in range(30):
        o, d, ta, tb, mu, ls, q, rho = _rand_pair(rng, finite=trial % 2 == 0)
        g = oracle.pair_grad(o, d, ta, tb, mu, ls, q, rho)
        base = _params_vec(mu, ls, q, rho)
        # finite differences in float64 through a float64-exact re-parameterisation:
        # shift the ray instead of mu (d/dmu = -d/do), and differentiate l, q, rho
        # through the closed form evaluated on float32-representable steps.
        for k in range(11):
            h = 1e-3 * max(1e-2, abs(base[k]))
            vals = []
            for s in (+1, -1):
                p = base.copy()
                p[k] += s * h
                pf = p.astype(np.float32)
                hh = (pf.astype(np.float64) - base)[k]
                if k < 3:
                    # move the ray by -delta instead (exact in float64)
                    oo = o.copy(); oo[k] -= s * h
                    vals.append((oracle.pair(oo, d, ta, tb, mu, ls, q, rho)[0], s * h))
                else:
                    vals.append((oracle.pair(o, d, ta, tb, pf[:3], pf[3:6], pf[6:10], pf[10])[0], hh))
            (fp, hp), (fm, hm) = vals
            fd = (fp - fm) / (hp - hm)
            assert g[k] == pytest.approx(fd, rel=2e-4, abs=2e-7 * (abs(fp) + 1e-3)), (trial, k)


def test_backward_matches_finite_differences_of_forward(oracle):
    """Geometry-wide adjoint (no cut-off) vs FD of the projection: <w, dI/dp>."""
    g = synth.geom_cone(3, 12, 12, 0.2, 0.2, 3.0, 4.5)
    G = synth.gaussians_uniform(6, 42, half_box=0.5, log_sigma=math.log(0.2))
    w = synth.random_weights(synth.num_rays(g), 3).astype(np.float64)
    grad = oracle.backward(g, G, w, cut2=1e30)
    rng = np.random.default_rng(0)
    for _ in range(12):
        k = int(rng.integers(6))
        name, comp = [("mu", i) for i in range(3)] + [("ls", i) for i in range(3)] + \
            [("q", i) for i in range(4)] + [("rho", None)], None
        name, c = name[int(rng.integers(11))]
        vals = []
        for s in (+1, -1):
            Gp = {kk: vv.copy() for kk, vv in G.items()}
            arr = Gp[name]
            old = arr[k] if c is None else arr[k, c]
            step = np.float32(1e-3 * max(abs(float(old)), 0.05))
            if c is None:
                arr[k] = old + s * step
                hh = float(arr[k]) - float(old)
            else:
                arr[k, c] = old + s * step
                hh = float(arr[k, c]) - float(old)
            vals.append((float(w @ oracle.forward(g, Gp, cut2=1e30)["I"]), hh))
        (fp, hp), (fm, hm) = vals
        fd = (fp - fm) / (hp - hm)
        got = grad[name][k] if c is None else grad[name][k, c]
        assert got == pytest.approx(fd, rel=5e-4, abs=1e-6 * (abs(fp) + abs(fm) + 1e-3))


# --------------------------------------------------------------------------
# losses and Adam
# --------------------------------------------------------------------------

def test_losses_finite_differences(oracle):
    rng = np.random.default_rng(5)
    I = rng.uniform(0.5, 2.0, 50)
    y = rng.poisson(30.0, 50).astype(np.float64)
    L, g = oracle.loss_poisson(I, y, 20.0, 1e-9)
    L2, g2 = oracle.loss_l2(I, y / 20.0)
    for k in range(0, 50, 7):
        for lossf, grad in ((lambda v: oracle.loss_poisson(v, y, 20.0, 1e-9)[0], g),
                            (lambda v: oracle.loss_l2(v, y / 20.0)[0], g2)):
            e = np.zeros(50); e[k] = 1e-6
            fd = (lossf(I + e) - lossf(I - e)) / 2e-6
            assert grad[k] == pytest.approx(fd, rel=1e-5, abs=1e-6)


def test_losses_with_measurement_model(oracle):
    """Per-ray factor and background: finite differences, and a factor /
    background that reduce to the plain losses on rescaled data."""
    rng = np.random.default_rng(6)
    I = rng.uniform(0.5, 2.0, 40)
    y = rng.poisson(30.0, 40).astype(np.float64)
    m = rng.uniform(0.2, 0.9, 40)
    a = rng.uniform(0.5, 3.0, 40)
    for lossf in (lambda v: oracle.loss_poisson(v, y, 20.0, 1e-9, m, a),
                  lambda v: oracle.loss_l2(v, y / 20.0, m, a)):
        L, g = lossf(I)
        for k in range(0, 40, 5):
            e = np.zeros(40); e[k] = 1e-6
            fd = (lossf(I + e)[0] - lossf(I - e)[0]) / 2e-6
            assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-6)
    # m I + a with m = 1, a = 0 is the plain loss; Poisson with m and a equals the
    # plain Poisson loss of the predicted mean (m I + a / kappa)
    assert oracle.loss_l2(I, y, np.ones(40), np.zeros(40))[0] == oracle.loss_l2(I, y)[0]
    Lm, gm = oracle.loss_poisson(I, y, 20.0, 1e-9, m, a)
    Lp, gp = oracle.loss_poisson(m * I + a / 20.0, y, 20.0, 1e-9)
    assert Lm == pytest.approx(Lp, rel=1e-12)
    np.testing.assert_allclose(gm, m * gp, rtol=1e-12)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    from oracle import oracle as o
    rng = np.random.default_rng(9)
    p0 = rng.normal(size=20)
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    pn, m, v = p0.copy(), np.zeros(20), np.zeros(20)
    for t in range(1, 6):
        g = rng.normal(size=20)
        opt.zero_grad()
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        pn, m, v = o.adam(pn, g, m, v, t, 1e-2)
    np.testing.assert_allclose(pn, p.detach().numpy(), rtol=1e-12, atol=1e-14)
