"""The Epanechnikov kernel on the GPU (gaussians_set_kernel) against the FP64
oracle's: forward and adjoint on parallel, cone-beam and PET detectors
(including segments that end inside the support, which take the general
path), explicit rays, voxels, loss_step; batches reject the kernel."""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5
GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def rg(torch):
    from paper_2602_01057_gb300 import build, rgrt
    build.build()
    return rgrt


@pytest.fixture(scope="module")
def ctx(rg):
    c = rg.Context(0)
    yield c
    c.close()


def rel_err(got, ref):
    got = np.asarray(got, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


def epan(G):
    return dict(G, kernel="epanechnikov")


def gauss(rg, ctx, torch, G):
    g = rg.Gaussians(ctx, *[torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")])
    return g.set_kernel("epanechnikov")


def case(name):
    if name == "parallel":
        return synth.workload_c1(0)
    if name == "parallel_short_segment":
        return (synth.gaussians_uniform(300, 13, half_box=0.7, log_sigma=math.log(0.1)),
                synth.geom_parallel(4, 40, 48, 0.04, 0.04, -0.3, 0.4))
    if name == "cone":
        G, _ = synth.workload_c2(0, n=3000, n_views=12, side=64)
        return G, synth.geom_c2(n_views=12, side=64)
    if name == "cone_near_source":
        return (synth.gaussians_uniform(400, 14, log_sigma=math.log(0.08)),
                synth.geom_cone(6, 48, 40, 0.06, 0.06, 1.6, 2.4))
    if name == "pet":
        G, _ = synth.workload_c3(0, n=4000, n_angles=24, n_radial=329, n_planes=63)
        return G, synth.geom_c3(24, 329, 63, arc_mode=0)
    if name == "rays":
        return (synth.gaussians_uniform(500, 23, half_box=0.8, log_sigma=math.log(0.08)),
                synth.rays_random(3000, 24, radius=0.9, seg=0.25))
    raise KeyError(name)


@pytest.mark.parametrize("name", ["parallel", "parallel_short_segment", "cone", "cone_near_source", "pet", "rays"])
def test_forward_and_adjoint(rg, ctx, torch, oracle, name):
    G, gd = case(name)
    gs = gauss(rg, ctx, torch, G)
    geom = rg.Geometry(ctx, gd)
    I = torch.empty(geom.n_rays, device="cuda")
    rg.project_forward(ctx, gs, geom, I)
    w = synth.random_weights(geom.n_rays, 51).astype(np.float32)
    n = gs.n
    outs = [torch.empty(s, device="cuda") for s in ((n, 3), (n, 3), (n, 4), (n,))]
    rg.project_backward(ctx, gs, geom, torch.from_numpy(w).cuda(), *outs)
    torch.cuda.synchronize()
    if gd["kind"] == "rays":
        ref = oracle.forward_list(gd["o"], gd["d"], gd["t"], epan(G))
        gref = oracle.backward_list(gd["o"], gd["d"], gd["t"], epan(G), w.astype(np.float64))
    else:
        ref = oracle.forward(gd, epan(G))
        gref = oracle.backward(gd, epan(G), w.astype(np.float64))
    assert np.count_nonzero(ref["I"]) > 100
    assert rel_err(I.cpu().numpy(), ref["I"]) < FWD_TOL
    for k, o in zip(("mu", "ls", "q", "rho"), outs):
        assert rel_err(o.cpu().numpy(), gref[k]) < GRAD_TOL, k


def test_differs_from_the_gaussian(rg, ctx, torch):
    G, gd = case("cone")
    geom = rg.Geometry(ctx, gd)
    a = torch.empty(geom.n_rays, device="cuda")
    b = torch.empty(geom.n_rays, device="cuda")
    gs = rg.Gaussians(ctx, *[torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")])
    rg.project_forward(ctx, gs, geom, a)
    gs.set_kernel("epanechnikov")
    rg.project_forward(ctx, gs, geom, b)
    gs.set_kernel("gaussian")
    c = torch.empty(geom.n_rays, device="cuda")
    rg.project_forward(ctx, gs, geom, c)
    torch.cuda.synchronize()
    assert rel_err(b.cpu().numpy(), a.cpu().numpy()) > 1e-2
    np.testing.assert_array_equal(a.cpu().numpy(), c.cpu().numpy())


def test_voxels(rg, ctx, torch, oracle):
    G = synth.gaussians_uniform(800, 41, half_box=0.9, log_sigma=math.log(0.06))
    vol = dict(origin=(-0.93, -0.71, -1.02), size=(0.041, 0.037, 0.052), dims=(45, 37, 29))
    V = rg.gaussians_voxelize(ctx, gauss(rg, ctx, torch, G), vol)
    ref = oracle.voxelize(vol, epan(G))["V"]
    assert np.count_nonzero(ref) > 1000
    assert rel_err(V, ref) < FWD_TOL


def test_loss_step(rg, ctx, torch, oracle):
    G, gd = case("cone")
    T = synth.perturbed(G, 61, pos_std=0.01)
    y = oracle.forward(gd, epan(T))["I"].astype(np.float32)
    ref = oracle.forward(gd, epan(G))["I"]
    L_ref, _ = oracle.loss_l2(ref, y)
    gs = gauss(rg, ctx, torch, G)
    geom = rg.Geometry(ctx, gd)
    lo = np.zeros(1, np.float32)
    rg.loss_step(ctx, gs, geom, y, rg.RGRT_LOSS_L2, rg.adam_params(), 1, lo)
    tol = 2.0 * FWD_TOL * np.linalg.norm(ref) / np.linalg.norm(ref - y)
    assert float(lo[0]) == pytest.approx(L_ref, rel=max(tol, 1e-6))


def test_batch_rejects_the_kernel(rg, ctx, torch):
    G, gd = case("cone")
    gs = gauss(rg, ctx, torch, G)
    geom = rg.Geometry(ctx, gd)
    with pytest.raises(rg.RgrtError):
        rg.Batch(ctx, [gs], [geom])
