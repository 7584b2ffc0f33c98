"""The allocation-free forward projection (project_forward_noalloc) against
the regular one.

project_forward_noalloc exists for callers that must not allocate device
memory where they project; it takes its scratch from a static device array.
This file runs last (its name sorts last) so that a failure here never hides
the other GPU tests; it also passes on its own in a fresh process.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5   # the projection tolerance of the parity tests


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01057_gb300 import build, rgrt
    build.build()
    return torch, rgrt


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("case", ["c1", "cone", "pet"])
def test_noalloc_matches_project_forward_twice(env, case):
    torch, rg = env
    if case == "c1":
        G, gd = synth.workload_c1(3)
    elif case == "cone":
        G, _ = synth.workload_c2(1, n=2000, n_views=8, side=64)
        gd = synth.geom_c2(n_views=8, side=64)
    else:
        G, _ = synth.workload_c3(2, n=2000, n_angles=12, n_radial=129, n_planes=31)
        gd = synth.geom_c3(12, 129, 31)
    t = {k: torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")}
    ctx = rg.Context(0)
    geom = rg.Geometry(ctx, gd)
    gs = rg.Gaussians(ctx, t["mu"], t["ls"], t["q"], t["rho"])
    ref = torch.empty(geom.n_rays, device="cuda")
    rg.project_forward(ctx, gs, geom, ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    assert np.abs(ref).max() > 0
    for _ in range(2):   # the scratch keeps the last call's contents
        out = torch.full((geom.n_rays,), float("nan"), device="cuda")
        rg.project_forward_noalloc(gd, t["mu"], t["ls"], t["q"], t["rho"], out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) < FWD_TOL


def test_noalloc_rejects_oversized_problems(env):
    torch, rg = env
    G = synth.gaussians_uniform(200_000, 5, log_sigma=math.log(0.05))
    gd = synth.geom_c2(n_views=180, side=256)
    t = {k: torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")}
    out = torch.empty(synth.num_rays(gd), device="cuda")
    with pytest.raises(rg.RgrtError) as e:
        rg.project_forward_noalloc(gd, t["mu"], t["ls"], t["q"], t["rho"], out)
    assert e.value.code == -3 and "static scratch" in str(e.value)
    with pytest.raises(rg.RgrtError):
        rg.project_forward_noalloc(gd, G["mu"], G["ls"], G["q"], G["rho"], out)   # host arrays
