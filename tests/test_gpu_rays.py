"""Explicit-ray geometries on the GPU (geometry_set_rays) against the FP64
oracle's explicit-ray projector: coherent helical cone-beam rays, incoherent
random lines (infinite and finite segments, half-lines), the circular cone
beam given as rays (also against the detector-geometry kernels), loss_step,
host pointers, rays that miss everything, and invalid rays."""
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


def _dev(torch, G):
    return [torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")]


def fwd_err(I, ref):
    I = np.asarray(I, np.float64)
    clip = np.clip(I, ref["I_lo"], ref["I_hi"])
    den = np.linalg.norm(clip)
    return np.linalg.norm(I - clip) / (den if den > 0 else 1.0)


def grad_err(got, ref, k):
    g = np.asarray(got[k], np.float64)
    clip = np.clip(g, ref["lo"][k], ref["hi"][k])
    den = np.linalg.norm(ref[k])
    return np.linalg.norm(g - clip) / (den if den > 0 else 1.0)


def case(name):
    if name == "helical":
        G, _ = synth.workload_c2(3, n=2000, n_views=12, side=48)
        R = synth.rays_helical(12, 48, 48, 1.5 * 256 / 48 / 128, 7.8125, 11.71875, z_per_turn=0.4,
                               turns=1.5)
        return G, R
    if name == "random_lines":
        return (synth.gaussians_uniform(500, 21, half_box=0.8, log_sigma=math.log(0.08)),
                synth.rays_random(3000, 22, radius=0.9))
    if name == "random_segments":
        return (synth.gaussians_uniform(500, 23, half_box=0.8, log_sigma=math.log(0.08)),
                synth.rays_random(3000, 24, radius=0.9, seg=0.25))
    if name == "half_lines":
        R = synth.rays_random(2000, 25, radius=0.6)
        R["t"][:, 0] = 0.0
        return synth.gaussians_uniform(400, 26, half_box=0.7, log_sigma=math.log(0.1)), R
    raise KeyError(name)


def gpu_fwd(torch, rg, ctx, G, R):
    geom = rg.Geometry(ctx, R)
    gs = rg.Gaussians(ctx, *_dev(torch, G))
    out = torch.empty(geom.n_rays, device="cuda")
    rg.project_forward(ctx, gs, geom, out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), gs, geom


@pytest.mark.parametrize("name", ["helical", "random_lines", "random_segments", "half_lines"])
def test_forward_and_adjoint_parity(rg, ctx, torch, oracle, name):
    G, R = case(name)
    I, gs, geom = gpu_fwd(torch, rg, ctx, G, R)
    ref = oracle.forward_list(R["o"], R["d"], R["t"], G)
    assert ref["pairs"] > 1000
    assert fwd_err(I, ref) < FWD_TOL
    w = synth.random_weights(I.size, 31)
    n = gs.n
    outs = [torch.empty(s, device="cuda") for s in ((n, 3), (n, 3), (n, 4), (n,))]
    rg.project_backward(ctx, gs, geom, torch.from_numpy(w.astype(np.float32)).cuda(), *outs)
    torch.cuda.synchronize()
    got = dict(zip(("mu", "ls", "q", "rho"), (o.cpu().numpy() for o in outs)))
    gref = oracle.backward_list(R["o"], R["d"], R["t"], G, w.astype(np.float32).astype(np.float64))
    for k in ("mu", "ls", "q", "rho"):
        assert grad_err(got, gref, k) < GRAD_TOL, k


@pytest.mark.parametrize("n", [1, 7, 33, 100])
def test_partial_clusters(rg, ctx, torch, oracle, n):
    """Gaussian counts that leave the last cluster of 32 bounding balls
    partly filled (or a single ball): forward and adjoint against the oracle."""
    G = synth.gaussians_uniform(n, 70 + n, half_box=0.5, log_sigma=math.log(0.15))
    R = synth.rays_random(4000, 71 + n, radius=0.8, seg=0.5)
    I, gs, geom = gpu_fwd(torch, rg, ctx, G, R)
    ref = oracle.forward_list(R["o"], R["d"], R["t"], G)
    assert np.count_nonzero(ref["I"]) > 50
    assert fwd_err(I, ref) < FWD_TOL
    w = synth.random_weights(I.size, 72)
    outs = [torch.empty(sz, device="cuda") for sz in ((n, 3), (n, 3), (n, 4), (n,))]
    rg.project_backward(ctx, gs, geom, torch.from_numpy(w.astype(np.float32)).cuda(), *outs)
    torch.cuda.synchronize()
    got = dict(zip(("mu", "ls", "q", "rho"), (o.cpu().numpy() for o in outs)))
    gref = oracle.backward_list(R["o"], R["d"], R["t"], G, w.astype(np.float32).astype(np.float64))
    for k in ("mu", "ls", "q", "rho"):
        assert grad_err(got, gref, k) < GRAD_TOL, k


def test_circular_cone_as_rays_matches_detector_kernels(rg, ctx, torch):
    """The same cone-beam scan through the detector kernels and as explicit
    rays: two different FP32 evaluations of the same sums."""
    G, _ = synth.workload_c2(4, n=3000, n_views=8, side=64)
    gd = synth.geom_c2(n_views=8, side=64)
    R = synth.rays_helical(8, 64, 64, gd["pitch_u"], gd["dso"], gd["dsd"], z_per_turn=0.0)
    a, _, _ = gpu_fwd(torch, rg, ctx, G, gd)
    b, _, _ = gpu_fwd(torch, rg, ctx, G, R)
    assert np.linalg.norm(b - a) / np.linalg.norm(a) < 1e-5


def test_loss_step_on_rays(rg, ctx, torch, oracle):
    G, R = case("helical")
    T = synth.perturbed(G, 41, pos_std=0.01)
    y = oracle.forward_list(R["o"], R["d"], R["t"], T)["I"].astype(np.float32)
    ref = oracle.forward_list(R["o"], R["d"], R["t"], G)
    L_ref, _ = oracle.loss_l2(ref["I"], y)
    gs = rg.Gaussians(ctx, *_dev(torch, G))
    geom = rg.Geometry(ctx, R)
    lo = np.zeros(1, np.float32)
    rg.loss_step(ctx, gs, geom, y, rg.RGRT_LOSS_L2, rg.adam_params(), 1, lo)
    # L = |r|^2 / 2 with r = I - y: an error dI of the projection (|dI| <=
    # FWD_TOL |I|) moves L by at most |r| |dI|
    r = ref["I"] - y
    tol = 2.0 * FWD_TOL * np.linalg.norm(ref["I"]) / np.linalg.norm(r)
    assert float(lo[0]) == pytest.approx(L_ref, rel=max(tol, 1e-6))
    after = gs.numpy()
    assert not np.array_equal(after["mu"], G["mu"])       # the step moved the Gaussians


def test_host_and_device_ray_arrays_agree(rg, ctx, torch):
    G, R = case("random_segments")
    a, _, _ = gpu_fwd(torch, rg, ctx, G, R)
    Rd = dict(kind="rays", **{k: torch.from_numpy(np.ascontiguousarray(R[k])).cuda() for k in ("o", "d", "t")})
    b, _, _ = gpu_fwd(torch, rg, ctx, G, Rd)
    np.testing.assert_array_equal(a, b)


def test_rays_that_miss_everything(rg, ctx, torch):
    G = synth.gaussians_uniform(200, 27, half_box=0.5, log_sigma=math.log(0.05))
    R = synth.rays_random(500, 28, radius=0.1)
    R["o"] = R["o"] + np.float32(10.0)
    R["d"][:] = np.array([0.0, 0.0, 1.0], np.float32)
    I, _, _ = gpu_fwd(torch, rg, ctx, G, R)
    assert np.all(I == 0.0)


@pytest.mark.parametrize("bad", ["zero_direction", "reversed_segment", "nan_origin"])
def test_invalid_rays_rejected(rg, ctx, bad):
    R = synth.rays_random(300, 29, radius=0.5, seg=0.3)
    if bad == "zero_direction":
        R["d"][17] = 0.0
    elif bad == "reversed_segment":
        R["t"][5] = (1.0, -1.0)
    else:
        R["o"][200, 1] = np.nan
    with pytest.raises(rg.RgrtError):
        rg.Geometry(ctx, R)


def test_fully_3d_pet_lors(rg, ctx, torch, oracle):
    """Oblique PET segments (ring differences up to 3) as explicit rays."""
    R = synth.pet_rays_3d(8, 4.0, 400.0, 576, 24, 65, max_ring_diff=3)
    G, _ = synth.workload_c3(2, n=3000, n_angles=24, n_radial=65, n_planes=15)
    G["mu"][:, 2] *= 0.25            # keep the activity within the 8 rings' axial field
    I, gs, geom = gpu_fwd(torch, rg, ctx, G, R)
    ref = oracle.forward_list(R["o"], R["d"], R["t"], G)
    assert ref["pairs"] > 10000
    assert fwd_err(I, ref) < FWD_TOL
    w = synth.random_weights(I.size, 35).astype(np.float32)
    n = gs.n
    outs = [torch.empty(s, device="cuda") for s in ((n, 3), (n, 3), (n, 4), (n,))]
    rg.project_backward(ctx, gs, geom, torch.from_numpy(w).cuda(), *outs)
    torch.cuda.synchronize()
    got = dict(zip(("mu", "ls", "q", "rho"), (o.cpu().numpy() for o in outs)))
    gref = oracle.backward_list(R["o"], R["d"], R["t"], G, w.astype(np.float64))
    for k in ("mu", "ls", "q", "rho"):
        assert grad_err(got, gref, k) < GRAD_TOL, k


def test_time_of_flight(rg, ctx, torch, oracle):
    """TOF rays (3-D PET LORs, 9 TOF bins each) against the oracle, forward
    and adjoint; the TOF bins of a LOR sum to its plain projection."""
    R0 = synth.pet_rays_3d(6, 4.0, 400.0, 576, 12, 49, max_ring_diff=2)
    G, _ = synth.workload_c3(3, n=1500, n_angles=12, n_radial=49, n_planes=11)
    G["mu"][:, 2] *= 0.2
    R = synth.with_tof(R0, 9, 40.0, 30.0)            # 40 mm bins, 30 mm kernel width
    I, gs, geom = gpu_fwd(torch, rg, ctx, G, R)
    ref = oracle.forward_list(R["o"], R["d"], R["t"], G, tof=R["tof"])
    assert fwd_err(I, ref) < FWD_TOL
    w = synth.random_weights(I.size, 37).astype(np.float32)
    n = gs.n
    outs = [torch.empty(s, device="cuda") for s in ((n, 3), (n, 3), (n, 4), (n,))]
    rg.project_backward(ctx, gs, geom, torch.from_numpy(w).cuda(), *outs)
    torch.cuda.synchronize()
    got = dict(zip(("mu", "ls", "q", "rho"), (o.cpu().numpy() for o in outs)))
    gref = oracle.backward_list(R["o"], R["d"], R["t"], G, w.astype(np.float64), tof=R["tof"])
    for k in ("mu", "ls", "q", "rho"):
        assert grad_err(got, gref, k) < GRAD_TOL, k
    # dense TOF bins (spacing below the width) sum to the plain projection
    Rd = synth.with_tof(R0, 81, 10.0, 20.0)
    Id, _, _ = gpu_fwd(torch, rg, ctx, G, Rd)
    plain, _, _ = gpu_fwd(torch, rg, ctx, G, R0)
    summed = Id.reshape(-1, 81).sum(axis=1) * 10.0
    assert np.linalg.norm(summed - plain) / np.linalg.norm(plain) < 1e-5


def test_time_of_flight_takes_the_gaussian_kernel(rg, ctx, torch):
    R = synth.with_tof(synth.rays_random(200, 38, radius=0.5, seg=0.4), 3, 0.1, 0.1)
    G = synth.gaussians_uniform(50, 39, half_box=0.5, log_sigma=math.log(0.1))
    geom = rg.Geometry(ctx, R)
    gs = rg.Gaussians(ctx, *[torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")])
    gs.set_kernel("epanechnikov")
    out = torch.empty(geom.n_rays, device="cuda")
    with pytest.raises(rg.RgrtError):
        rg.project_forward(ctx, gs, geom, out)
