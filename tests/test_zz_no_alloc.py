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


def _case(case):
    if case == "c1":
        return synth.workload_c1(3)
    if case == "cone":
        G, _ = synth.workload_c2(1, n=2000, n_views=8, side=64)
        return G, synth.geom_c2(n_views=8, side=64)
    if case == "pet":
        G, _ = synth.workload_c3(2, n=2000, n_angles=12, n_radial=129, n_planes=31)
        return G, synth.geom_c3(12, 129, 31)
    # fully 3-D PET: 12 angles x 5 ring differences of a 4-ring scanner
    G = synth.gaussians_uniform(1500, 4, half_box=120.0, log_sigma=math.log(4.0))
    G["mu"][:, 2] *= 0.05
    return G, synth.geom_pet3d(12, 129, 4, 200.0, 288, 4.0, 2)


@pytest.mark.parametrize("case", ["c1", "cone", "pet", "pet3d"])
def test_noalloc_matches_project_forward_twice(env, case):
    """Two calls in a row against project_forward: the same kernels on the
    same lists (per-ray sums in fixed point, independent of the order of
    the additions), so the projections agree bit for bit."""
    torch, rg = env
    G, gd = _case(case)
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
        assert np.array_equal(got, ref)


def test_noalloc_all_gaussians_culled(env):
    """Every Gaussian outside the field of view: no tile entries at all, and
    the output (NaN before the call) is all zeros."""
    torch, rg = env
    G, gd = synth.workload_c1(5)
    G = dict(G, mu=(G["mu"] + np.float32(50.0)).astype(np.float32))
    t = {k: torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")}
    for _ in range(2):
        out = torch.full((synth.num_rays(gd),), float("nan"), device="cuda")
        rg.project_forward_noalloc(gd, t["mu"], t["ls"], t["q"], t["rho"], out)
        torch.cuda.synchronize()
        assert torch.count_nonzero(out).item() == 0


def test_noalloc_refuses_non_finite_parameters(env):
    """A NaN parameter is refused with the error project_forward gives, and a
    following call with finite parameters succeeds (the flag is cleared)."""
    torch, rg = env
    G, gd = _case("cone")
    t = {k: torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")}
    bad = t["rho"].clone()
    bad[17] = float("nan")
    out = torch.empty(synth.num_rays(gd), device="cuda")
    ctx = rg.Context(0)
    geom = rg.Geometry(ctx, gd)
    gs = rg.Gaussians(ctx, t["mu"], t["ls"], t["q"], bad)
    with pytest.raises(rg.RgrtError) as e_ref:
        rg.project_forward(ctx, gs, geom, out)
    with pytest.raises(rg.RgrtError) as e:
        rg.project_forward_noalloc(gd, t["mu"], t["ls"], t["q"], bad, out)
    assert e.value.code == e_ref.value.code == -1
    rg.project_forward_noalloc(gd, t["mu"], t["ls"], t["q"], t["rho"], out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    gs.close()
    geom.close()
    ctx.close()


def test_noalloc_rejects_oversized_problems(env):
    torch, rg = env
    G = synth.gaussians_uniform(200_000, 5, log_sigma=math.log(0.05))
    gd = synth.geom_c2(n_views=180, side=256)
    t = {k: torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")}
    out = torch.empty(synth.num_rays(gd), device="cuda")
    with pytest.raises(rg.RgrtError) as e:
        rg.project_forward_noalloc(gd, t["mu"], t["ls"], t["q"], t["rho"], out)
    assert e.value.code == -3 and "static scratch" in str(e.value)
    with pytest.raises(ValueError):     # host arrays: refused by the binding
        rg.project_forward_noalloc(gd, G["mu"], G["ls"], G["q"], G["rho"], out)
    with pytest.raises(ValueError):     # a short output
        rg.project_forward_noalloc(gd, t["mu"], t["ls"], t["q"], t["rho"], out[:-1])
    # host arrays given to the C entry point directly: refused there too
    d, angles = rg.make_desc(gd)
    mu = np.ascontiguousarray(G["mu"])
    rc = rg.lib().project_forward_noalloc(ctypes.byref(d), mu.shape[0], mu.ctypes.data, mu.ctypes.data,
                                          mu.ctypes.data, mu.ctypes.data, out.data_ptr(), None)
    assert rc == -1
