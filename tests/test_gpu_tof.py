"""Time of flight on PET ring sinograms (geometry_set_tof) on the GPU against
the FP64 oracle: forward and adjoint (Gaussians well inside the ring, which
take the view-space form with the closed-form TOF weight, and Gaussians near
the ring, whose LOR ends fall inside them: the world-space form per bin),
the loss gradient, the same LORs as explicit TOF rays, and the rejections."""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5
GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01057_gb300 import build, rgrt
    build.build()
    ctx = rgrt.Context(0)
    yield torch, rgrt, ctx
    ctx.close()


def _dist(x, ref, lo, hi, nom):
    x = np.asarray(x, np.float64).reshape(-1)
    c = np.clip(x, np.asarray(lo).reshape(-1), np.asarray(hi).reshape(-1))
    den = np.linalg.norm(np.asarray(nom).reshape(-1))
    return np.linalg.norm(x - c) / (den if den > 0 else 1.0)


def _case(n_tof=7, near_ring=False, seed=3):
    gd = synth.with_tof_bins(synth.geom_pet(12, 129, 9, 200.0, 288, 4.0), n_tof, 45.0, 32.0)
    G = synth.gaussians_uniform(600, seed, half_box=120.0, log_sigma=math.log(5.0))
    G["mu"][:, 2] *= 0.12
    if near_ring:
        ang = np.random.default_rng(seed).uniform(0, 2 * np.pi, 150)
        G["mu"][:150, 0] = (190.0 * np.cos(ang)).astype(np.float32)
        G["mu"][:150, 1] = (190.0 * np.sin(ang)).astype(np.float32)
    return G, gd


def _gauss(torch, rg, ctx, G):
    return rg.Gaussians(ctx, *[torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")])


@pytest.mark.parametrize("near_ring", [False, True])
@pytest.mark.parametrize("n_tof", [1, 7, 16])
def test_tof_forward_and_adjoint(env, oracle, near_ring, n_tof):
    torch, rg, ctx = env
    G, gd = _case(n_tof, near_ring)
    geom = rg.Geometry(ctx, gd)
    assert geom.n_rays == synth.num_rays(gd) == n_tof * 12 * 129 * 9
    gs = _gauss(torch, rg, ctx, G)
    I = torch.full((geom.n_rays,), float("nan"), device="cuda")
    rg.project_forward(ctx, gs, geom, I)
    torch.cuda.synchronize()
    ref = oracle.forward(gd, G)
    assert np.count_nonzero(ref["I"]) > 1000
    assert _dist(I.cpu().numpy(), ref["I"], ref["I_lo"], ref["I_hi"], ref["I"]) < FWD_TOL
    w = synth.random_weights(geom.n_rays, 5)
    outs = [torch.empty(s, device="cuda") for s in ((gs.n, 3), (gs.n, 3), (gs.n, 4), (gs.n,))]
    rg.project_backward(ctx, gs, geom, torch.from_numpy(w).cuda(), *outs)
    torch.cuda.synchronize()
    gref = oracle.backward(gd, G, w)
    for k, o in zip(("mu", "ls", "q", "rho"), outs):
        e = _dist(o.cpu().numpy(), gref[k], gref["lo"][k], gref["hi"][k], gref[k])
        assert e < GRAD_TOL, (k, e)


def test_tof_loss_gradient(env, oracle):
    """loss_grad (Poisson) against the oracle's loss of the GPU projection
    and the oracle's adjoint of its dL/dI."""
    torch, rg, ctx = env
    G, gd = _case(9)
    true = synth.perturbed(G, 41, pos_std=1.0)
    geom = rg.Geometry(ctx, gd)
    gt = _gauss(torch, rg, ctx, true)
    y = torch.empty(geom.n_rays, device="cuda")
    rg.project_forward(ctx, gt, geom, y)
    kappa = 1e6 / float(y.sum())
    y = torch.poisson(kappa * y, generator=torch.Generator(device="cuda").manual_seed(3))
    hp = rg.adam_params(kappa=kappa, poisson_eps=1e-3)
    gs = _gauss(torch, rg, ctx, G)
    outs = [torch.empty(s, device="cuda") for s in ((gs.n, 3), (gs.n, 3), (gs.n, 4), (gs.n,))]
    lo = np.zeros(1, np.float32)
    rg.loss_grad(ctx, gs, geom, y, rg.RGRT_LOSS_POISSON, hp, lo, *outs)
    I = torch.empty(geom.n_rays, device="cuda")
    rg.project_forward(ctx, gs, geom, I)
    torch.cuda.synchronize()
    L, dLdI = oracle.loss_poisson(I.cpu().numpy(), y.cpu().numpy(), kappa, 1e-3)
    assert float(lo[0]) == pytest.approx(L, rel=1e-5)
    gref = oracle.backward(gd, G, dLdI)
    for k, o in zip(("mu", "ls", "q", "rho"), outs):
        e = _dist(o.cpu().numpy(), gref[k], gref["lo"][k], gref["hi"][k], gref[k])
        assert e < GRAD_TOL, (k, e)


def test_tof_sinogram_equals_explicit_tof_rays(env, oracle):
    """The structured TOF projection equals the same LORs traced as explicit
    rays with the same TOF kernels (geometry_set_rays_tof), bin-major."""
    torch, rg, ctx = env
    G, gd = _case(5)
    g0 = {k: v for k, v in gd.items() if k not in ("n_tof", "tof_spacing", "tof_sigma")}
    nl = synth.num_rays(g0)
    o, d, ta, tb = oracle.rays(g0, np.arange(nl))
    nb = gd["n_tof"]
    centres = (np.arange(nb) - 0.5 * (nb - 1)) * gd["tof_spacing"]
    mid = 0.5 * (ta + tb)
    R = dict(kind="rays", o=np.tile(o, (nb, 1)).astype(np.float32), d=np.tile(d, (nb, 1)).astype(np.float32),
             t=np.tile(np.stack([ta, tb], 1), (nb, 1)).astype(np.float32),
             tof=np.stack([np.repeat(centres, nl) + np.tile(mid, nb), np.full(nb * nl, gd["tof_sigma"])],
                          1).astype(np.float32))
    gs = _gauss(torch, rg, ctx, G)
    a = torch.empty(synth.num_rays(gd), device="cuda")
    rg.project_forward(ctx, gs, rg.Geometry(ctx, gd), a)
    b = torch.empty(nb * nl, device="cuda")
    rg.project_forward(ctx, gs, rg.Geometry(ctx, R), b)
    torch.cuda.synchronize()
    a, b = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
    assert np.count_nonzero(b) > 1000
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 2e-5


def test_tof_rejections(env):
    torch, rg, ctx = env
    G, gd = _case(4)
    gs = _gauss(torch, rg, ctx, G)
    with pytest.raises(rg.RgrtError):       # CT geometry
        rg.Geometry(ctx, dict(synth.geom_c2(n_views=4, side=32), n_tof=3, tof_spacing=1.0, tof_sigma=1.0))
    for bad in (dict(n_tof=17), dict(tof_spacing=0.0), dict(tof_sigma=float("nan"))):
        with pytest.raises(rg.RgrtError):
            rg.Geometry(ctx, dict(gd, **bad))
    geom = rg.Geometry(ctx, gd)
    gs.set_kernel("epanechnikov")
    with pytest.raises(rg.RgrtError):
        rg.project_forward(ctx, gs, geom, torch.empty(geom.n_rays, device="cuda"))
