"""GPU parity of the CUDA projector against the FP64 oracle, through the C ABI.

Tolerances (stated by the method's targets): projections within 1e-5
relative L2 of the oracle, gradients within 1e-4 relative L2, culling
records and tile lists bit-exact.  For projections the reference is the
oracle's admissible interval [I_lo, I_hi] (pairs whose m is within 1e-4*9 of
the 3-sigma cut may go either way in FP32), i.e. the error is the distance
of the GPU result from that interval.
"""
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
    c.stats_enable(True)
    yield c
    c.close()


def _dev(torch, G):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in G.items()}


def fwd_err(I_gpu, ref):
    I = np.asarray(I_gpu, np.float64)
    clip = np.clip(I, ref["I_lo"], ref["I_hi"])
    den = np.linalg.norm(clip)
    return np.linalg.norm(I - clip) / (den if den > 0 else 1.0)


def grad_err(got, ref, k, rows=None):
    """Distance of the GPU gradient from the oracle's admissible bracket
    [lo, hi] (pairs within the band of the 3-sigma cut may go either way),
    relative to the oracle's nominal gradient."""
    g = np.asarray(got[k], np.float64)
    lo, hi, nom = ref["lo"][k], ref["hi"][k], ref[k]
    if rows is not None:
        g, lo, hi, nom = g[rows], lo[rows], hi[rows], nom[rows]
    clip = np.clip(g, lo, hi)
    den = np.linalg.norm(nom)
    return np.linalg.norm(g - clip) / (den if den > 0 else 1.0)


def rel_l2(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def gpu_forward(torch, rg, ctx, G, gd):
    geom = rg.Geometry(ctx, gd)
    gs = rg.Gaussians(ctx, *[_dev(torch, G)[k] for k in ("mu", "ls", "q", "rho")])
    out = torch.empty(geom.n_rays, device="cuda", dtype=torch.float32)
    rg.project_forward(ctx, gs, geom, out)
    torch.cuda.synchronize()
    return out.cpu().numpy(), gs, geom


def gpu_backward(torch, rg, ctx, gs, geom, w):
    n = gs.n
    wd = torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda()
    outs = [torch.empty(s, device="cuda") for s in ((n, 3), (n, 3), (n, 4), (n,))]
    rg.project_backward(ctx, gs, geom, wd, *outs)
    torch.cuda.synchronize()
    return dict(zip(("mu", "ls", "q", "rho"), (o.cpu().numpy() for o in outs)))


# ------------------------------------------------------------------ cases

def case(name):
    if name == "c1":
        return synth.workload_c1(0)
    if name == "parallel_ragged":
        return (synth.gaussians_uniform(400, 11, log_sigma=math.log(0.08)),
                synth.geom_parallel(5, 37, 53, 0.04, 0.04, -2.0, 2.0))
    if name == "parallel_infinite":
        return (synth.gaussians_uniform(300, 12, half_box=0.7, log_sigma=math.log(0.08)),
                synth.geom_parallel(4, 40, 48, 0.04, 0.04, -math.inf, math.inf))
    if name == "parallel_short_segment":
        # segment [-0.3, 0.4] cuts through the Gaussians: erf terms matter
        return (synth.gaussians_uniform(300, 13, half_box=0.7, log_sigma=math.log(0.1)),
                synth.geom_parallel(4, 40, 48, 0.04, 0.04, -0.3, 0.4))
    if name == "cone_small":
        G, _ = synth.workload_c2(0, n=3000, n_views=12, side=64)
        return G, synth.geom_c2(n_views=12, side=64)
    if name == "cone_near_source":
        # detector close behind the volume: segments end inside Gaussians
        return (synth.gaussians_uniform(400, 14, log_sigma=math.log(0.08)),
                synth.geom_cone(6, 48, 40, 0.06, 0.06, 1.6, 2.4))
    if name == "cone_source_inside":
        # the sources of views 0 and 3 lie inside the 3-sigma ellipsoids of two
        # wide Gaussians: their detector box is the whole detector, and every
        # ray of those views starts inside them (finite-segment erf terms)
        G = synth.gaussians_uniform(300, 15, half_box=0.8, log_sigma=math.log(0.08))
        gd = synth.geom_cone(6, 32, 40, 0.08, 0.08, 1.6, 2.4)
        for k, th in ((0, 0.0), (1, math.pi)):
            G["mu"][k] = (-1.6 * math.cos(th) + 0.05, -1.6 * math.sin(th) - 0.04, 0.03)
            G["ls"][k] = (math.log(0.3), math.log(0.22), math.log(0.26))
        return G, gd
    if name == "pet_arc":
        G, _ = synth.workload_c3(0, n=4000, n_angles=24, n_radial=329, n_planes=63)
        return G, synth.geom_c3(24, 329, 63, arc_mode=0)
    if name == "pet_raw":
        G, _ = synth.workload_c3(1, n=4000, n_angles=24, n_radial=329, n_planes=63)
        return G, synth.geom_c3(24, 329, 63, arc_mode=1)
    if name == "tile8x4":
        G, gd = synth.workload_c1(1)
        gd = dict(gd, tile_w=8, tile_h=4)
        return G, gd
    if name == "tile32x8":
        G, gd = synth.workload_c1(2)
        gd = dict(gd, tile_w=32, tile_h=8)
        return G, gd
    raise KeyError(name)


FWD_CASES = ["c1", "parallel_ragged", "parallel_infinite", "parallel_short_segment", "cone_small",
             "cone_near_source", "cone_source_inside", "pet_arc", "pet_raw", "tile8x4", "tile32x8"]


def test_records_bit_exact(rg, ctx, torch, oracle):
    G = synth.gaussians_uniform(5000, 3, log_sigma=math.log(0.05), log_sigma_std=1.0)
    gs = rg.Gaussians(ctx, *[_dev(torch, G)[k] for k in ("mu", "ls", "q", "rho")])
    got = rg.debug_records(ctx, gs)
    ref = oracle.records_fp32(G["ls"], G["q"])
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def same_tile_sets(start, gid, rstart, rgid):
    """The GPU's per-tile lists hold exactly the oracle's sets: equal CSR
    offsets, and equal ids once each tile's entries are put in id order (the
    order within a tile is the kernel's own; the projection needs none)."""
    assert gid.size == rgid.size and gid.size > 0
    assert np.array_equal(start, rstart)
    tile = np.repeat(np.arange(start.size - 1), np.diff(start))
    canon = gid[np.lexsort((gid, tile))]
    assert np.array_equal(canon, rgid)


@pytest.mark.parametrize("name", ["c1", "parallel_ragged", "cone_small", "cone_near_source",
                                  "cone_source_inside", "pet_arc", "pet_raw", "tile8x4"])
def test_tile_lists_bit_exact(rg, ctx, torch, oracle, name):
    G, gd = case(name)
    geom = rg.Geometry(ctx, gd)
    gs = rg.Gaussians(ctx, *[_dev(torch, G)[k] for k in ("mu", "ls", "q", "rho")])
    start, gid = rg.debug_tile_lists(ctx, gs, geom)
    rstart, rgid = oracle.tile_lists_fp32(gd, G, gd["tile_w"], gd["tile_h"])
    same_tile_sets(start, gid, rstart, rgid)


@pytest.mark.parametrize("name,views", [("c2", (0, 2)), ("c2", (97, 99)), ("c3", (0, 2)),
                                        ("c3", (143, 145))])
def test_tile_lists_bit_exact_full_size(rg, ctx, torch, oracle, name, views):
    """The benchmark workloads at full size (cone beam: 50,000 Gaussians on
    256 x 256; PET: 200,000 Gaussians, 329 x 63), lists of two views each."""
    if name == "c2":
        G, gd = synth.workload_c2(0)
    else:
        G, gd = synth.workload_c3(0)
    geom = rg.Geometry(ctx, gd)
    gs = rg.Gaussians(ctx, *[_dev(torch, G)[k] for k in ("mu", "ls", "q", "rho")])
    start, gid = rg.debug_tile_lists(ctx, gs, geom, *views)
    rstart, rgid = oracle.tile_lists_fp32(gd, G, gd["tile_w"], gd["tile_h"], views=views)
    same_tile_sets(start, gid, rstart, rgid)


@pytest.mark.parametrize("name", FWD_CASES)
def test_forward_parity(rg, ctx, torch, oracle, name):
    G, gd = case(name)
    I, gs, geom = gpu_forward(torch, rg, ctx, G, gd)
    ref = oracle.forward(gd, G)
    assert ref["pairs"] > 1000
    err = fwd_err(I, ref)
    assert err < FWD_TOL, f"{name}: forward rel-L2 {err:.3e}"
    st = ctx.stats()
    assert st["pairs_kept"] >= 0.999 * ref["pairs"] - 10


@pytest.mark.parametrize("name", ["c1", "parallel_ragged", "parallel_short_segment", "cone_small",
                                  "cone_near_source", "cone_source_inside", "pet_arc", "tile8x4"])
def test_backward_parity(rg, ctx, torch, oracle, name):
    G, gd = case(name)
    I, gs, geom = gpu_forward(torch, rg, ctx, G, gd)
    w = synth.random_weights(geom.n_rays, 5)
    got = gpu_backward(torch, rg, ctx, gs, geom, w)
    ref = oracle.backward(gd, G, w)
    for k in ("mu", "ls", "q", "rho"):
        e = grad_err(got, ref, k)
        assert e < GRAD_TOL, f"{name}: grad {k} rel-L2 {e:.3e}"


def test_host_pointers_match_device(rg, ctx, torch):
    G, gd = case("parallel_ragged")
    I_dev, gs, geom = gpu_forward(torch, rg, ctx, G, gd)
    gh = rg.Gaussians(ctx, G["mu"], G["ls"], G["q"], G["rho"])    # host arrays, copied
    I_host = np.zeros(geom.n_rays, np.float32)
    rg.project_forward(ctx, gh, geom, I_host)
    assert np.array_equal(I_host, I_dev)
    w = synth.random_weights(geom.n_rays, 9)
    gd_dev = gpu_backward(torch, rg, ctx, gs, geom, w)
    outs = [np.zeros(s, np.float32) for s in ((gh.n, 3), (gh.n, 3), (gh.n, 4), (gh.n,))]
    rg.project_backward(ctx, gh, geom, w.astype(np.float32), *outs)
    for k, o in zip(("mu", "ls", "q", "rho"), outs):
        assert rel_l2(o, gd_dev[k]) < 1e-6


def test_autograd_function_matches_c_abi(rg, ctx, torch):
    G, gd = case("cone_small")
    geom = rg.Geometry(ctx, gd)
    t = _dev(torch, G)
    leaves = [t[k].clone().requires_grad_() for k in ("mu", "ls", "q", "rho")]
    I = rg.gaussian_project(*leaves, geom)
    w = torch.from_numpy(synth.random_weights(geom.n_rays, 2)).cuda()
    (I * w).sum().backward()
    gs = rg.Gaussians(ctx, t["mu"], t["ls"], t["q"], t["rho"])
    ref = gpu_backward(torch, rg, ctx, gs, geom, w.cpu().numpy())
    for leaf, k in zip(leaves, ("mu", "ls", "q", "rho")):
        assert rel_l2(leaf.grad.cpu().numpy(), ref[k]) < 1e-5


# ------------------------------------------------------------------ edge cases

def test_no_gaussians(rg, ctx, torch):
    gd = synth.geom_c1()
    geom = rg.Geometry(ctx, gd)
    z = np.zeros((0, 3), np.float32)
    gs = rg.Gaussians(ctx, z, z, np.zeros((0, 4), np.float32), np.zeros(0, np.float32))
    out = torch.full((geom.n_rays,), 7.0, device="cuda")
    rg.project_forward(ctx, gs, geom, out)
    assert float(out.abs().max()) == 0.0


def test_gaussians_outside_detector(rg, ctx, torch, oracle):
    G = synth.gaussians_uniform(200, 21, half_box=0.5, log_sigma=math.log(0.05))
    G["mu"][:, 2] += 5.0     # far above the detector rows
    gd = synth.geom_c1()
    I, gs, geom = gpu_forward(torch, rg, ctx, G, gd)
    assert float(np.abs(I).max()) == 0.0
    w = synth.random_weights(geom.n_rays, 1)
    g = gpu_backward(torch, rg, ctx, gs, geom, w)
    assert all(float(np.abs(v).max()) == 0.0 for v in g.values())


def test_huge_gaussian_covers_detector(rg, ctx, torch, oracle):
    G = synth.gaussians_uniform(3, 22, half_box=0.2, log_sigma=math.log(0.9), log_sigma_std=0.05)
    gd = synth.geom_parallel(3, 40, 40, 0.05, 0.05, -6.0, 6.0)
    I, gs, geom = gpu_forward(torch, rg, ctx, G, gd)
    ref = oracle.forward(gd, G)
    assert fwd_err(I, ref) < FWD_TOL


def test_degenerate_quaternion_and_flat_gaussian(rg, ctx, torch, oracle):
    G = synth.gaussians_uniform(50, 23, half_box=0.6, log_sigma=math.log(0.08))
    G["q"][:5] = 0.0                     # zero quaternion: identity rotation
    G["ls"][5:10, 2] = math.log(0.004)   # nearly flat pancakes
    gd = synth.geom_parallel(6, 48, 48, 0.04, 0.04, -2.0, 2.0)
    I, gs, geom = gpu_forward(torch, rg, ctx, G, gd)
    ref = oracle.forward(gd, G)
    assert fwd_err(I, ref) < FWD_TOL


def test_invalid_geometry_rejected(rg, ctx):
    bad = synth.geom_cone(4, 16, 16, 0.1, 0.1, 5.0, 4.0)   # detector before the origin
    with pytest.raises(rg.RgrtError):
        rg.Geometry(ctx, bad)
    bad = dict(synth.geom_c1(), tile_w=12)
    with pytest.raises(rg.RgrtError):
        rg.Geometry(ctx, bad)
    bad = synth.geom_pet(8, 400, 5, 100.0, 64, 2.0)       # bins beyond the ring
    with pytest.raises(rg.RgrtError):
        rg.Geometry(ctx, bad)


# ------------------------------------------------------------------ full sizes, sampled

@pytest.mark.parametrize("cfg", ["c2", "c3"])
def test_full_size_sampled_parity(rg, ctx, torch, oracle, cfg):
    """At the benchmark sizes: sampled rays against the oracle's brute force,
    sampled Gaussians' gradients against the oracle's adjoint."""
    G, gd = synth.workload_c2(0) if cfg == "c2" else synth.workload_c3(0)
    I, gs, geom = gpu_forward(torch, rg, ctx, G, gd)
    rng = np.random.default_rng(0)
    nz = np.nonzero(I)[0]
    idx = np.concatenate([rng.choice(nz, 300, replace=False), rng.choice(I.size, 100, replace=False)])
    ref = oracle.forward_rays(gd, G, idx)
    err = fwd_err(I[idx], ref)
    assert err < FWD_TOL, f"{cfg}: sampled forward rel-L2 {err:.3e}"
    w = synth.random_weights(geom.n_rays, 4)
    got = gpu_backward(torch, rg, ctx, gs, geom, w)
    sel = rng.choice(G["mu"].shape[0], 24, replace=False)
    gref = oracle.backward(gd, G, w, sel=sel)
    for k in ("mu", "ls", "q", "rho"):
        e = grad_err(got, gref, k, rows=sel)
        assert e < GRAD_TOL, f"{cfg}: sampled grad {k} rel-L2 {e:.3e}"


# ------------------------------------------------------------------ loss_step

@pytest.mark.parametrize("loss", ["l2", "poisson"])
def test_loss_step_matches_oracle(rg, ctx, torch, oracle, loss):
    G, gd = case("cone_small")
    ref_fwd = oracle.forward(gd, G)
    rng = np.random.default_rng(3)
    if loss == "l2":
        y = (ref_fwd["I"] * rng.uniform(0.8, 1.2, ref_fwd["I"].size)).astype(np.float32)
        kappa, eps = 1.0, 0.0
        L_ref, dLdI = oracle.loss_l2(ref_fwd["I"], y)
        kind = rg.RGRT_LOSS_L2
    else:
        kappa = 50.0
        eps = 1e-3
        y = rng.poisson(kappa * ref_fwd["I"] + eps).astype(np.float32)
        L_ref, dLdI = oracle.loss_poisson(ref_fwd["I"], y, kappa, eps)
        kind = rg.RGRT_LOSS_POISSON
    hp = rg.adam_params(kappa=kappa, poisson_eps=eps)
    gs = rg.Gaussians(ctx, *[_dev(torch, G)[k] for k in ("mu", "ls", "q", "rho")])
    geom = rg.Geometry(ctx, gd)
    loss_out = np.zeros(1, np.float32)
    rg.loss_step(ctx, gs, geom, y, kind, hp, 1, loss_out)
    assert float(loss_out[0]) == pytest.approx(L_ref, rel=1e-5)
    g = oracle.backward(gd, G, dLdI)
    new = gs.numpy()
    lrs = dict(mu=hp.lr_mu, ls=hp.lr_logscale, q=hp.lr_quat, rho=hp.lr_rho)
    for k in ("mu", "ls", "q", "rho"):
        p_ref, _, _ = oracle.adam(G[k].astype(np.float64), g[k], 0.0, 0.0, 1, lrs[k])
        strong = np.abs(g[k]) > 1e-2 * np.abs(g[k]).max()   # well-determined update signs
        d_got = (new[k].astype(np.float64) - G[k])[strong]
        d_ref = (p_ref - G[k])[strong]
        assert rel_l2(d_got, d_ref) < 1e-3, k


# ------------------------------------------------------------------ loss_grad

@pytest.mark.parametrize("loss", ["l2", "poisson"])
def test_loss_grad_matches_oracle(rg, ctx, torch, oracle, loss):
    """loss_grad: the loss and the gradient (no update) against the FP64
    oracle's loss, dL/dI and adjoint; the Gaussians stay unchanged.  The
    measurements come from a perturbed copy of the Gaussians, so the gradient
    is taken away from the optimum (at the optimum it is a sum of noise terms
    that cancel, and any FP32 rounding of I dominates it)."""
    G, gd = case("pet_arc" if loss == "poisson" else "cone_small")
    ref_fwd = oracle.forward(gd, G)
    rng = np.random.default_rng(4)
    T = synth.perturbed(G, 77, pos_std=2.0 if loss == "poisson" else 0.01)
    I_true = oracle.forward(gd, T)["I"]
    if loss == "l2":
        y = I_true.astype(np.float32)
        kappa, eps = 1.0, 0.0
        L_ref, dLdI = oracle.loss_l2(ref_fwd["I"], y)
        kind = rg.RGRT_LOSS_L2
    else:
        kappa, eps = 50.0, 1e-3
        y = rng.poisson(kappa * I_true + eps).astype(np.float32)
        L_ref, dLdI = oracle.loss_poisson(ref_fwd["I"], y, kappa, eps)
        kind = rg.RGRT_LOSS_POISSON
    hp = rg.adam_params(kappa=kappa, poisson_eps=eps)
    gs = rg.Gaussians(ctx, *[_dev(torch, G)[k] for k in ("mu", "ls", "q", "rho")])
    geom = rg.Geometry(ctx, gd)
    n = gs.n
    outs = [np.zeros(s, np.float32) for s in ((n, 3), (n, 3), (n, 4), (n,))]   # host outputs
    lo = np.zeros(1, np.float32)
    rg.loss_grad(ctx, gs, geom, y, kind, hp, lo, *outs)
    assert float(lo[0]) == pytest.approx(L_ref, rel=1e-5)
    ref = oracle.backward(gd, G, dLdI)
    got = dict(zip(("mu", "ls", "q", "rho"), outs))
    for k in ("mu", "ls", "q", "rho"):
        assert grad_err(got, ref, k) < GRAD_TOL, k
    after = gs.numpy()
    for k in ("mu", "ls", "q", "rho"):
        np.testing.assert_array_equal(after[k], G[k])


@pytest.mark.parametrize("loss", ["l2", "poisson"])
def test_loss_grad_in_view_chunks(rg, ctx, torch, oracle, loss):
    """A context whose HBM budget holds the tile lists of a few views only:
    the step bins, projects, takes the loss of and back-projects one view
    chunk at a time.  Loss and gradient against the FP64 oracle."""
    G, gd = case("cone_small")
    ref_fwd = oracle.forward(gd, G)
    T = synth.perturbed(G, 78, pos_std=0.01)
    I_true = oracle.forward(gd, T)["I"]
    if loss == "l2":
        y = I_true.astype(np.float32)
        kappa, eps = 1.0, 0.0
        L_ref, dLdI = oracle.loss_l2(ref_fwd["I"], y)
        kind = rg.RGRT_LOSS_L2
    else:
        kappa, eps = 50.0, 1e-3
        y = np.random.default_rng(5).poisson(kappa * I_true + eps).astype(np.float32)
        L_ref, dLdI = oracle.loss_poisson(ref_fwd["I"], y, kappa, eps)
        kind = rg.RGRT_LOSS_POISSON
    hp = rg.adam_params(kappa=kappa, poisson_eps=eps)
    ref = oracle.backward(gd, G, dLdI)
    chunked = 0
    budget = 64 << 20
    while budget >= 256 << 10 and not chunked:
        c = rg.Context(0, budget)
        try:
            gs = rg.Gaussians(c, *[_dev(torch, G)[k] for k in ("mu", "ls", "q", "rho")])
            geom = rg.Geometry(c, gd)
            n = gs.n
            outs = [np.zeros(sz, np.float32) for sz in ((n, 3), (n, 3), (n, 4), (n,))]
            lo = np.zeros(1, np.float32)
            c.prof_enable(True)
            rg.loss_grad(c, gs, geom, y, kind, hp, lo, *outs)
            launches, _ = c.prof_get("k_forward")
            if launches >= 2:
                chunked = launches
                assert float(lo[0]) == pytest.approx(L_ref, rel=1e-5)
                got = dict(zip(("mu", "ls", "q", "rho"), outs))
                for k in ("mu", "ls", "q", "rho"):
                    assert grad_err(got, ref, k) < GRAD_TOL, k
            gs.close()
            geom.close()
        except rg.RgrtError:
            break          # the budget no longer holds one view's lists
        finally:
            c.close()
        budget //= 2
    assert chunked >= 2


# ------------------------------------------------------------------ view subsets

@pytest.mark.parametrize("name", ["cone_small", "pet_arc"])
def test_view_subset_geometry_bit_exact(rg, ctx, torch, oracle, name):
    """A geometry holding a subset of a scan's views (explicit angles; for PET
    the sinogram angles pi j / n_views) projects to exactly those views of the
    full scan, and matches the oracle on its own."""
    G, gd = case(name)
    full, _, _ = gpu_forward(torch, rg, ctx, G, gd)
    V, H, W = gd["n_views"], gd["n_rows"], gd["n_cols"]
    idx = np.array([5, 0, V - 1, 7])
    sub = dict(gd)
    sub["n_views"] = idx.size
    base = (np.pi * np.arange(V, dtype=np.float64) / V) if gd["kind"] == "pet" else gd["angles"]
    sub["angles"] = np.asarray(base, np.float64)[idx].copy()
    part, _, _ = gpu_forward(torch, rg, ctx, G, sub)
    if gd["kind"] == "pet":
        want = full.reshape(H, V, W)[:, idx, :].reshape(-1)
    else:
        want = full.reshape(V, H, W)[idx].reshape(-1)
    np.testing.assert_array_equal(part, want)
    assert fwd_err(part, oracle.forward(sub, G)) < FWD_TOL


@pytest.mark.parametrize("loss", ["l2", "poisson"])
def test_loss_with_measurement_model(rg, ctx, torch, oracle, loss):
    """geometry_set_corrections: per-ray factor (attenuation) and background
    (scatter + randoms) in the loss; loss and gradient against the oracle."""
    G, gd = case("cone_small")
    R = synth.num_rays(gd)
    rng = np.random.default_rng(8)
    mult = rng.uniform(0.3, 1.0, R).astype(np.float32)
    add = rng.uniform(0.0, 0.2, R).astype(np.float32)
    ref_fwd = oracle.forward(gd, G)
    I_true = oracle.forward(gd, synth.perturbed(G, 78, pos_std=0.01))["I"]
    if loss == "l2":
        y = (mult * I_true + add).astype(np.float32)
        kappa, eps = 1.0, 0.0
        L_ref, dLdI = oracle.loss_l2(ref_fwd["I"], y, mult, add)
        kind = rg.RGRT_LOSS_L2
    else:
        kappa, eps = 50.0, 1e-3
        y = rng.poisson(kappa * mult * I_true + add + eps).astype(np.float32)
        L_ref, dLdI = oracle.loss_poisson(ref_fwd["I"], y, kappa, eps, mult, add)
        kind = rg.RGRT_LOSS_POISSON
    gs = rg.Gaussians(ctx, *[_dev(torch, G)[k] for k in ("mu", "ls", "q", "rho")])
    geom = rg.Geometry(ctx, gd).set_corrections(mult, add)
    n = gs.n
    outs = [np.zeros(s, np.float32) for s in ((n, 3), (n, 3), (n, 4), (n,))]
    lo = np.zeros(1, np.float32)
    rg.loss_grad(ctx, gs, geom, y, kind, rg.adam_params(kappa=kappa, poisson_eps=eps), lo, *outs)
    assert float(lo[0]) == pytest.approx(L_ref, rel=1e-5)
    ref = oracle.backward(gd, G, dLdI)
    got = dict(zip(("mu", "ls", "q", "rho"), outs))
    for k in ("mu", "ls", "q", "rho"):
        assert grad_err(got, ref, k) < GRAD_TOL, k
    # clearing the corrections restores the plain loss
    geom.set_corrections(None, None)
    rg.loss_grad(ctx, gs, geom, y, kind, rg.adam_params(kappa=kappa, poisson_eps=eps), lo)
    L_plain = (oracle.loss_l2(ref_fwd["I"], y) if loss == "l2"
               else oracle.loss_poisson(ref_fwd["I"], y, kappa, eps))[0]
    assert float(lo[0]) == pytest.approx(L_plain, rel=1e-5)


@pytest.mark.parametrize("field", ["mu", "ls", "q", "rho"])
def test_non_finite_parameters_are_refused(rg, ctx, torch, field):
    """A NaN or infinite parameter (a diverged optimisation) makes the
    projector return an error instead of a silently wrong projection; finite
    parameters set afterwards project again."""
    G, gd = case("cone_small")
    bad = {k: np.array(G[k], copy=True) for k in ("mu", "ls", "q", "rho")}
    if field == "rho":
        bad["rho"][17] = np.nan
    else:
        bad[field][17, 1] = np.inf if field == "ls" else np.nan
    gs = rg.Gaussians(ctx, *[_dev(torch, bad)[k] for k in ("mu", "ls", "q", "rho")])
    geom = rg.Geometry(ctx, gd)
    out = torch.empty(geom.n_rays, device="cuda")
    with pytest.raises(rg.RgrtError):
        rg.project_forward(ctx, gs, geom, out)
    with pytest.raises(rg.RgrtError):
        rg.loss_step(ctx, gs, geom, np.zeros(geom.n_rays, np.float32), rg.RGRT_LOSS_L2, rg.adam_params(), 1,
                     np.zeros(1, np.float32))
    gs.set(*[G[k] for k in ("mu", "ls", "q", "rho")])
    rg.project_forward(ctx, gs, geom, out)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(out.cpu().numpy()))
