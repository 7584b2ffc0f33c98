"""Structured fully-3-D PET sinograms (geometry kind PET_3D: one view per ring
difference and angle) on the GPU against the FP64 oracle: forward and
adjoint for arc-corrected and raw radial bins, several tile shapes, the
Epanechnikov kernel, loss_step, the ring-difference-0 segment against the
2-D ring geometry, rows without a ring pair, sampled rays at the full-size
workload, the allocation-free entry point, and the rejections."""
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


def fwd_err(I_gpu, ref):
    I = np.asarray(I_gpu, np.float64)
    clip = np.clip(I, ref["I_lo"], ref["I_hi"])
    den = np.linalg.norm(clip)
    return np.linalg.norm(I - clip) / (den if den > 0 else 1.0)


def grad_err(got, ref, k, rows=None):
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


def gaussians(rg, ctx, torch, G):
    g = rg.Gaussians(ctx, *[torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")])
    if G.get("kernel", "gaussian") != "gaussian":
        g.set_kernel(G["kernel"])
    return g


def forward(rg, ctx, torch, G, gd):
    gs = gaussians(rg, ctx, torch, G)
    geom = rg.Geometry(ctx, gd)
    I = torch.empty(geom.n_rays, device="cuda")
    rg.project_forward(ctx, gs, geom, I)
    torch.cuda.synchronize()
    return I.cpu().numpy(), gs, geom


def backward(rg, ctx, torch, gs, geom, w):
    n = gs.n
    outs = [torch.empty(s, device="cuda") for s in ((n, 3), (n, 3), (n, 4), (n,))]
    rg.project_backward(ctx, gs, geom, torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda(), *outs)
    torch.cuda.synchronize()
    return dict(zip(("mu", "ls", "q", "rho"), (o.cpu().numpy() for o in outs)))


def scanner(n_ang=24, n_rad=129, n_rings=16, D=5, arc_mode=0, tile=(16, 16)):
    """A small ring (radius 200 mm, 288 crystals) with a 4 mm ring pitch."""
    return synth.geom_pet3d(n_ang, n_rad, n_rings, 200.0, 288, 4.0, D, arc_mode=arc_mode, tile=tile)


def phantom(seed, n=1500):
    G = synth.gaussians_uniform(n, seed, half_box=120.0, log_sigma=math.log(4.0))
    G["mu"][:, 2] *= 0.26        # inside the 64 mm axial field of view
    rng = np.random.default_rng(seed + 1)
    G["ls"] = (G["ls"] + rng.normal(0.0, 0.3, G["ls"].shape)).astype(np.float32)
    return G


CASES = {
    "arc": dict(),
    "raw": dict(arc_mode=1),
    "tile8x8": dict(tile=(8, 8)),
    "tile32x8": dict(tile=(32, 8)),
    "all_ring_pairs": dict(n_rings=10, D=9),
    "ragged": dict(n_ang=7, n_rad=53, n_rings=13, D=3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_forward_and_adjoint(rg, ctx, torch, oracle, name):
    G = phantom(3)
    gd = scanner(**CASES[name])
    I, gs, geom = forward(rg, ctx, torch, G, gd)
    ref = oracle.forward(gd, G)
    assert geom.n_rays == ref["I"].size
    assert np.count_nonzero(ref["I"]) > 1000
    assert fwd_err(I, ref) < FWD_TOL
    w = synth.random_weights(geom.n_rays, 5)
    got = backward(rg, ctx, torch, gs, geom, w)
    gref = oracle.backward(gd, G, w)
    for k in ("mu", "ls", "q", "rho"):
        assert grad_err(got, gref, k) < GRAD_TOL, k


def same_tile_sets(start, gid, rstart, rgid):
    """Equal CSR offsets, and equal ids once each tile's entries are put in id
    order (a tile's list is a set; its order is the kernel's own)."""
    assert gid.size == rgid.size and gid.size > 0
    assert np.array_equal(start, rstart)
    tile = np.repeat(np.arange(start.size - 1), np.diff(start))
    assert np.array_equal(gid[np.lexsort((gid, tile))], rgid)


@pytest.mark.parametrize("name", ["arc", "raw", "tile8x8", "all_ring_pairs", "ragged"])
def test_tile_lists_bit_exact(rg, ctx, torch, oracle, name):
    """Candidate lists of the 3-D PET cull (the ring-pair rows and the LOR
    slopes' z bounds) against the oracle's FP32 specification, every view."""
    G = phantom(3)
    gd = scanner(**CASES[name])
    gs = gaussians(rg, ctx, torch, G)
    geom = rg.Geometry(ctx, gd)
    start, gid = rg.debug_tile_lists(ctx, gs, geom)
    rstart, rgid = oracle.tile_lists_fp32(gd, G, gd["tile_w"], gd["tile_h"])
    same_tile_sets(start, gid, rstart, rgid)


def test_tile_lists_bit_exact_steep_lors(rg, ctx, torch, oracle):
    """A small ring (50 mm) with 8 mm ring pitch: LOR slopes 0.24 at the
    centre and 1.9 at the outermost raw bin (s = 49.6 mm)."""
    gd = synth.geom_pet3d(6, 25, 8, 50.0, 26, 8.0, 3, arc_mode=1, tile=(8, 4))
    G = synth.gaussians_uniform(300, 21, half_box=25.0, log_sigma=math.log(4.0))
    G["mu"][:, 2] *= 0.8
    gs = gaussians(rg, ctx, torch, G)
    geom = rg.Geometry(ctx, gd)
    start, gid = rg.debug_tile_lists(ctx, gs, geom)
    rstart, rgid = oracle.tile_lists_fp32(gd, G, 8, 4)
    same_tile_sets(start, gid, rstart, rgid)


@pytest.mark.parametrize("seg", [-5, 0, 3, 5])
def test_tile_lists_bit_exact_full_size(rg, ctx, torch, oracle, seg):
    """The benchmark scanner at full size (200,000 Gaussians, 32 rings, ring
    differences up to 5, 288 angles x 329 radial bins): lists of two views
    (angles 100 and 101) of one segment."""
    G, _ = synth.workload_c3(0)
    gd = synth.geom_c3_3d()
    v0 = (seg + gd["max_ring_diff"]) * gd["n_views"] + 100
    gs = gaussians(rg, ctx, torch, G)
    geom = rg.Geometry(ctx, gd)
    start, gid = rg.debug_tile_lists(ctx, gs, geom, v0, v0 + 2)
    rstart, rgid = oracle.tile_lists_fp32(gd, G, gd["tile_w"], gd["tile_h"], views=(v0, v0 + 2))
    same_tile_sets(start, gid, rstart, rgid)
    gs.close()
    geom.close()


def test_segment_ends_inside_gaussians(rg, ctx, torch, oracle):
    """Gaussians near the ring: LOR ends (on the ring) fall inside their
    3-sigma ellipsoids, so the erf terms matter (the general path)."""
    G = phantom(7, n=400)
    ang = np.random.default_rng(8).uniform(0, 2 * np.pi, 400)
    G["mu"][:, 0] = (190.0 * np.cos(ang)).astype(np.float32)
    G["mu"][:, 1] = (190.0 * np.sin(ang)).astype(np.float32)
    gd = scanner()
    I, gs, geom = forward(rg, ctx, torch, G, gd)
    ref = oracle.forward(gd, G)
    assert fwd_err(I, ref) < FWD_TOL
    w = synth.random_weights(geom.n_rays, 9)
    got = backward(rg, ctx, torch, gs, geom, w)
    gref = oracle.backward(gd, G, w)
    for k in ("mu", "ls", "q", "rho"):
        assert grad_err(got, gref, k) < GRAD_TOL, k


def test_epanechnikov(rg, ctx, torch, oracle):
    G = dict(phantom(11), kernel="epanechnikov")
    gd = scanner()
    I, gs, geom = forward(rg, ctx, torch, G, gd)
    ref = oracle.forward(gd, G)
    assert rel_l2(I, ref["I"]) < FWD_TOL
    w = synth.random_weights(geom.n_rays, 12)
    got = backward(rg, ctx, torch, gs, geom, w)
    gref = oracle.backward(gd, G, w)
    for k in ("mu", "ls", "q", "rho"):
        assert rel_l2(got[k], gref[k]) < GRAD_TOL, k


def test_rows_without_a_ring_pair_are_zero(rg, ctx, torch):
    G = phantom(13)
    gd = scanner(D=6)
    I, gs, geom = forward(rg, ctx, torch, G, gd)
    I = I.reshape(13, 24, 16, 129)
    for sg, delta in enumerate(range(-6, 7)):
        assert not I[sg, :, 16 - abs(delta):].any()
        assert I[sg, :, :16 - abs(delta)].any()
    # their dL/dI is ignored (up to the order of the gradient atomics: a
    # weight of 1e3 on those rows would move the gradients by far more)
    w = synth.random_weights(geom.n_rays, 14).reshape(13, 24, 16, 129)
    a = backward(rg, ctx, torch, gs, geom, w)
    w2 = w.copy()
    for sg, delta in enumerate(range(-6, 7)):
        w2[sg, :, 16 - abs(delta):] = 1e3
    b = backward(rg, ctx, torch, gs, geom, w2)
    for k in a:
        assert rel_l2(b[k], a[k]) < 1e-5, k


def test_segment_zero_matches_the_ring_geometry(rg, ctx, torch):
    G = phantom(17)
    I3, _, _ = forward(rg, ctx, torch, G, scanner(D=0))
    g2 = synth.geom_pet(24, 129, 16, 200.0, 288, 4.0)
    I2, _, _ = forward(rg, ctx, torch, G, g2)
    want = I2.reshape(16, 24, 129).transpose(1, 0, 2)
    assert rel_l2(I3.reshape(24, 16, 129), want) < 2e-6


def test_loss_step_matches_oracle(rg, ctx, torch, oracle):
    G = phantom(19)
    gd = scanner()
    T = synth.perturbed(G, 20, pos_std=1.0)
    y = oracle.forward(gd, T)["I"].astype(np.float32)
    ref = oracle.forward(gd, G)["I"]
    L_ref, _ = oracle.loss_l2(ref, y)
    gs = gaussians(rg, ctx, torch, G)
    geom = rg.Geometry(ctx, gd)
    lo = np.zeros(1, np.float32)
    rg.loss_step(ctx, gs, geom, y, rg.RGRT_LOSS_L2, rg.adam_params(), 1, lo)
    tol = 2.0 * FWD_TOL * np.linalg.norm(ref) / np.linalg.norm(ref - y)
    assert float(lo[0]) == pytest.approx(L_ref, rel=max(tol, 1e-6))


def test_full_size_sampled(rg, ctx, torch, oracle):
    """The benchmark workload (288 angles x 329 radial bins, 32 rings at 4 mm,
    ring differences up to 5, the 2-D PET phantom): sampled rays against the
    oracle's brute force, sampled Gaussians' gradients."""
    G, _ = synth.workload_c3(0)
    gd = synth.geom_c3_3d()
    I, gs, geom = forward(rg, ctx, torch, G, gd)
    rng = np.random.default_rng(0)
    nz = np.nonzero(I)[0]
    idx = np.concatenate([rng.choice(nz, 300, replace=False), rng.choice(I.size, 100, replace=False)])
    ref = oracle.forward_rays(gd, G, idx)
    assert fwd_err(I[idx], ref) < FWD_TOL
    w = synth.random_weights(geom.n_rays, 4)
    got = backward(rg, ctx, torch, gs, geom, w)
    sel = rng.choice(G["mu"].shape[0], 16, replace=False)
    gref = oracle.backward(gd, G, w, sel=sel)
    for k in ("mu", "ls", "q", "rho"):
        assert grad_err(got, gref, k, rows=sel) < GRAD_TOL, k


def test_noalloc_matches_project_forward(rg, ctx, torch):
    G = phantom(23)
    gd = scanner(n_ang=12, D=3)
    I, _, _ = forward(rg, ctx, torch, G, gd)
    t = {k: torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")}
    out = torch.empty(I.size, device="cuda")
    rg.project_forward_noalloc(gd, t["mu"], t["ls"], t["q"], t["rho"], out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), I)


def test_rejections(rg, ctx, torch):
    with pytest.raises(rg.RgrtError):
        rg.Geometry(ctx, scanner(n_rings=8, D=8))     # ring difference beyond the rings
    with pytest.raises(rg.RgrtError):
        rg.Geometry(ctx, scanner(D=-1))
    G = phantom(29, n=100)
    gs = gaussians(rg, ctx, torch, G)
    geom = rg.Geometry(ctx, scanner())
    with pytest.raises(rg.RgrtError):
        rg.Batch(ctx, [gs], [geom])


def test_reconstruction_job_in_angle_minibatches(rg, torch, oracle):
    """A serving reconstruction job on a 3-D PET scanner: mini-batches of
    angles (every ring difference of each), Adam steps lower the loss."""
    from paper_2602_01057_gb300 import serve
    G = phantom(31, n=600)
    T = synth.perturbed(G, 32, pos_std=1.5)
    gd = scanner(n_ang=16, D=3)
    y = oracle.forward(gd, T)["I"].astype(np.float32)
    job = serve.Job(serve.RECON, G, gd, y=y, n_iter=24, views_per_iter=4, seed=5,
                    hp=dict(lr_mu=0.05, lr_rho=1e-3))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        res = serve.run_job(job, 0, serve.job_budget(job), s)
    assert res["iterations"] == 24
    L = res["losses"]
    assert np.all(np.isfinite(L)) and L[-4:].mean() < 0.8 * L[:4].mean()


def test_no_gaussians_and_gaussians_outside_the_rings(rg, ctx, torch, oracle):
    gd = scanner(D=4)
    empty = dict(mu=np.zeros((0, 3), np.float32), ls=np.zeros((0, 3), np.float32),
                 q=np.zeros((0, 4), np.float32), rho=np.zeros(0, np.float32))
    I, gs, geom = forward(rg, ctx, torch, empty, gd)
    assert I.size == geom.n_rays and not I.any()
    # beyond the axial field of view (the rings span +-30 mm): every LOR misses
    G = phantom(37, n=200)
    G["mu"][:, 2] = np.where(np.arange(200) % 2 == 0, 80.0, -90.0).astype(np.float32)
    I, gs, geom = forward(rg, ctx, torch, G, gd)
    ref = oracle.forward(gd, G)
    assert not ref["I"].any() and not I.any()
    w = synth.random_weights(geom.n_rays, 38)
    got = backward(rg, ctx, torch, gs, geom, w)
    for k in got:
        assert not np.asarray(got[k]).any(), k


def test_single_ring(rg, ctx, torch, oracle):
    """One ring, ring difference 0 only: a single row per view."""
    G = phantom(41, n=300)
    G["mu"][:, 2] = 0.0
    gd = scanner(n_rings=1, D=0)
    I, gs, geom = forward(rg, ctx, torch, G, gd)
    ref = oracle.forward(gd, G)
    assert np.count_nonzero(ref["I"]) > 100
    assert fwd_err(I, ref) < FWD_TOL
