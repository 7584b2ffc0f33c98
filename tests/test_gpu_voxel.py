"""Voxelisation on the GPU (gaussians_voxelize) against the FP64 oracle's
voxeliser: every voxel of small ragged grids, sampled slabs of a 256^3 grid
of the cone-beam workload's Gaussians, an empty set, Gaussians off the grid,
host and device outputs, invalid grids."""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def err(V, ref):
    V = np.asarray(V, np.float64)
    clip = np.clip(V, ref["V_lo"], ref["V_hi"])
    den = np.linalg.norm(clip)
    return np.linalg.norm(V - clip) / (den if den > 0 else 1.0)


def gauss(rg, ctx, torch, G):
    return rg.Gaussians(ctx, *[torch.from_numpy(np.ascontiguousarray(G[k])).cuda()
                               for k in ("mu", "ls", "q", "rho")])


@pytest.mark.parametrize("case", ["cube64", "ragged", "anisotropic_voxels"])
def test_voxelize_parity(rg, ctx, torch, oracle, case):
    if case == "cube64":
        G, _ = synth.workload_c2(0, n=3000, n_views=1, side=16)
        vol = dict(origin=(-1 + 1 / 64, -1 + 1 / 64, -1 + 1 / 64), size=(2 / 64,) * 3, dims=(64, 64, 64))
    elif case == "ragged":
        G = synth.gaussians_uniform(800, 41, half_box=0.9, log_sigma=math.log(0.06))
        vol = dict(origin=(-0.93, -0.71, -1.02), size=(0.041, 0.037, 0.052), dims=(45, 37, 29))
    else:
        G = synth.gaussians_uniform(600, 42, half_box=0.8, log_sigma=math.log(0.07))
        vol = dict(origin=(-1.0, -1.0, -1.0), size=(0.02, 0.05, 0.1), dims=(101, 41, 21))
    V = rg.gaussians_voxelize(ctx, gauss(rg, ctx, torch, G), vol)
    ref = oracle.voxelize(vol, G)
    assert np.count_nonzero(ref["V"]) > 1000
    assert err(V, ref) < TOL


def test_full_size_sampled_slabs(rg, ctx, torch, oracle):
    """50,000 fitted Gaussians on a 256^3 grid of [-1, 1]^3; three 4-voxel
    slabs recomputed by the oracle."""
    G, _ = synth.workload_c2(0)
    n = 256
    h = 2.0 / n
    vol = dict(origin=(-1 + h / 2,) * 3, size=(h, h, h), dims=(n, n, n))
    out = torch.empty((n, n, n), device="cuda")
    rg.gaussians_voxelize(ctx, gauss(rg, ctx, torch, G), vol, out)
    torch.cuda.synchronize()
    V = out.cpu().numpy()
    for k0 in (0, 101, 252):
        sub = dict(origin=(vol["origin"][0], vol["origin"][1], vol["origin"][2] + k0 * h), size=vol["size"],
                   dims=(n, n, 4))
        ref = oracle.voxelize(sub, G)
        assert err(V[k0:k0 + 4], ref) < TOL, k0


def test_host_and_device_outputs_agree(rg, ctx, torch):
    G = synth.gaussians_uniform(500, 43, half_box=0.7, log_sigma=math.log(0.08))
    vol = dict(origin=(-1.0, -1.0, -1.0), size=(0.05, 0.05, 0.05), dims=(41, 41, 41))
    g = gauss(rg, ctx, torch, G)
    a = rg.gaussians_voxelize(ctx, g, vol)
    b = torch.empty((41, 41, 41), device="cuda")
    rg.gaussians_voxelize(ctx, g, vol, b)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a, b.cpu().numpy())


def test_empty_set_and_gaussians_off_the_grid(rg, ctx, torch):
    vol = dict(origin=(0.0, 0.0, 0.0), size=(0.1, 0.1, 0.1), dims=(10, 9, 8))
    z = {k: np.zeros((0, w), np.float32) for k, w in (("mu", 3), ("ls", 3), ("q", 4))}
    z["rho"] = np.zeros(0, np.float32)
    g0 = rg.Gaussians(ctx, z["mu"], z["ls"], z["q"], z["rho"])
    assert np.all(rg.gaussians_voxelize(ctx, g0, vol) == 0.0)
    G = synth.gaussians_uniform(100, 44, half_box=0.2, log_sigma=math.log(0.05))
    G["mu"] += np.float32(5.0)
    assert np.all(rg.gaussians_voxelize(ctx, gauss(rg, ctx, torch, G), vol) == 0.0)


@pytest.mark.parametrize("bad", ["zero_dim", "negative_size", "nan_origin"])
def test_invalid_grid_rejected(rg, ctx, torch, bad):
    G = synth.gaussians_uniform(10, 45)
    vol = dict(origin=(0.0, 0.0, 0.0), size=(0.1, 0.1, 0.1), dims=(4, 4, 4))
    if bad == "zero_dim":
        vol["dims"] = (4, 0, 4)
    elif bad == "negative_size":
        vol["size"] = (0.1, -0.1, 0.1)
    else:
        vol["origin"] = (0.0, float("nan"), 0.0)
    with pytest.raises(rg.RgrtError):
        rg.gaussians_voxelize(ctx, gauss(rg, ctx, torch, G), vol, np.zeros(64, np.float32))
