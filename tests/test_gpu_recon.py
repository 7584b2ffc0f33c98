"""Reconstruction on the GPU: Adam steps of loss_step on the exact line
integrals of an ellipsoid phantom raise the PSNR of the voxelised Gaussians
against the phantom's density and lower the loss."""
import numpy as np
import pytest

from paper_2602_01057_gb300 import synth

pytestmark = pytest.mark.gpu


def test_reconstruction_improves_psnr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01057_gb300 import build, rgrt
    build.build()
    ph = synth.ellipsoid_phantom(12, seed=1000, semi=(0.05, 0.6), dens=(0.1, 1.0))
    G, _ = synth.workload_c2(0, n=4000, n_views=36, side=64)
    gd = synth.geom_c2(n_views=36, side=64)
    y = synth.phantom_projection(ph, *synth.detector_rays(gd)).astype(np.float32)
    vol = synth.voxel_grid(48)
    ref = synth.phantom_volume(ph, vol)
    ctx = rgrt.Context(0)
    geom = rgrt.Geometry(ctx, gd)
    gs = rgrt.Gaussians(ctx, *[np.ascontiguousarray(G[k]) for k in ("mu", "ls", "q", "rho")])
    p0 = synth.psnr(rgrt.gaussians_voxelize(ctx, gs, vol), ref)
    hp = rgrt.adam_params()
    lo = np.zeros(1, np.float32)
    losses = []
    for it in range(150):
        rgrt.loss_step(ctx, gs, geom, y, rgrt.RGRT_LOSS_L2, hp, it + 1, lo)
        losses.append(float(lo[0]))
    p1 = synth.psnr(rgrt.gaussians_voxelize(ctx, gs, vol), ref)
    gs.close()
    geom.close()
    ctx.close()
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-10:]) < 0.5 * losses[0]
    assert p1 > p0 + 1.0, (p0, p1)
