"""The batched form (many scans per step, persistent launches, CUDA graph)
against one-scan-at-a-time calls of the same library and against the FP64
oracle, and the autotuner."""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01057_gb300 import build, rgrt
    build.build()
    ctx = rgrt.Context(0)
    return torch, rgrt, ctx


def _scans(seed, k, tile=(16, 16)):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        n = int(np.exp(rng.uniform(math.log(500), math.log(6000))))
        v = int(rng.integers(3, 12))
        side = int(rng.choice([32, 48, 64]))
        G, _ = synth.workload_c2(seed * 100 + i, n=n, n_views=v, side=side)
        gd = synth.geom_c2(n_views=v, side=side, tile=tile)
        out.append((G, gd))
    return out


def _dev(torch, G):
    return [torch.from_numpy(np.ascontiguousarray(G[k])).cuda() for k in ("mu", "ls", "q", "rho")]


def test_batch_forward_equals_single_scans(env):
    torch, rg, ctx = env
    scans = _scans(1, 7)
    gs = [rg.Gaussians(ctx, *_dev(torch, G)) for G, _ in scans]
    geoms = [rg.Geometry(ctx, gd) for _, gd in scans]
    b = rg.Batch(ctx, gs, geoms)
    outs = [torch.empty(g.n_rays, device="cuda") for g in geoms]
    for _ in range(2):            # the second call replays the captured graph
        b.forward(outs)
        for g, geom, o in zip(gs, geoms, outs):
            ref = torch.empty(geom.n_rays, device="cuda")
            rg.project_forward(ctx, g, geom, ref)
            torch.cuda.synchronize()
            assert torch.equal(o, ref)   # same tiles and pairs: fixed-point sums, identical


def test_batch_forward_matches_oracle(env, oracle):
    """The batched forward against the FP64 oracle: every ray of the first 4
    scans, a stratified 1/64 subsample (every 64th ray) of the others."""
    torch, rg, ctx = env
    scans = _scans(3, 8)
    gs = [rg.Gaussians(ctx, *_dev(torch, G)) for G, _ in scans]
    geoms = [rg.Geometry(ctx, gd) for _, gd in scans]
    b = rg.Batch(ctx, gs, geoms)
    outs = [torch.empty(g.n_rays, device="cuda") for g in geoms]
    b.forward(outs)
    torch.cuda.synchronize()
    for i, ((G, gd), o) in enumerate(zip(scans, outs)):
        I = o.cpu().numpy().astype(np.float64)
        if i < 4:
            ref = oracle.forward(gd, G)
        else:
            idx = np.arange(0, I.size, 64)
            ref = oracle.forward_rays(gd, G, idx)
            I = I[idx]
        clip = np.clip(I, ref["I_lo"], ref["I_hi"])
        err = np.linalg.norm(I - clip) / max(np.linalg.norm(clip), 1e-300)
        assert np.count_nonzero(ref["I"]) > 0
        assert err < 1e-5, (i, err)


def test_batch_loss_step_matches_single_scans(env):
    torch, rg, ctx = env
    scans = _scans(2, 5)
    hp = rg.adam_params()
    # measured data: projections of perturbed copies
    ys = []
    for G, gd in scans:
        geom = rg.Geometry(ctx, gd)
        gt = rg.Gaussians(ctx, *_dev(torch, synth.perturbed(G, 7, pos_std=0.01)))
        y = torch.empty(geom.n_rays, device="cuda")
        rg.project_forward(ctx, gt, geom, y)
        ys.append(y)
    gb = [rg.Gaussians(ctx, *_dev(torch, G)) for G, _ in scans]
    gsingle = [rg.Gaussians(ctx, *_dev(torch, G)) for G, _ in scans]
    geoms = [rg.Geometry(ctx, gd) for _, gd in scans]
    b = rg.Batch(ctx, gb, geoms)
    for t in (1, 2, 3):
        lb = b.loss_step(ys, rg.RGRT_LOSS_L2, hp, t)
        for i in range(len(scans)):
            ls = np.zeros(1, np.float32)
            rg.loss_step(ctx, gsingle[i], geoms[i], ys[i], rg.RGRT_LOSS_L2, hp, t, ls)
            assert lb[i] == pytest.approx(float(ls[0]), rel=1e-5, abs=1e-12)
    for i in range(len(scans)):
        a, c = gb[i].numpy(), gsingle[i].numpy()
        for k in ("mu", "ls", "q", "rho"):
            G0 = scans[i][0][k]
            da = a[k].astype(np.float64) - G0
            dc = c[k].astype(np.float64) - G0
            assert np.linalg.norm(da - dc) <= 1e-3 * np.linalg.norm(dc) + 1e-7, (i, k)


def test_batch_with_large_and_small_scans(env):
    """A scan large enough to fill the GPU for many waves (40 views of 256^2,
    10,240 tiles of 16 x 16) is projected with launches of its own inside the
    batch; the small ones share the persistent launches.  Forward and three
    optimisation steps against single-scan calls."""
    torch, rg, ctx = env
    G, _ = synth.workload_c2(31, n=5000, n_views=40, side=256)
    scans = [(G, synth.geom_c2(n_views=40, side=256))] + _scans(4, 3)
    gb = [rg.Gaussians(ctx, *_dev(torch, G)) for G, _ in scans]
    gsingle = [rg.Gaussians(ctx, *_dev(torch, G)) for G, _ in scans]
    geoms = [rg.Geometry(ctx, gd) for _, gd in scans]
    b = rg.Batch(ctx, gb, geoms)
    outs = [torch.empty(g.n_rays, device="cuda") for g in geoms]
    b.forward(outs)
    for g, geom, o in zip(gsingle, geoms, outs):
        ref = torch.empty(geom.n_rays, device="cuda")
        rg.project_forward(ctx, g, geom, ref)
        torch.cuda.synchronize()
        assert torch.equal(o, ref)
    hp = rg.adam_params()
    ys = []
    for (G, gd), geom in zip(scans, geoms):
        gt = rg.Gaussians(ctx, *_dev(torch, synth.perturbed(G, 9, pos_std=0.01)))
        y = torch.empty(geom.n_rays, device="cuda")
        rg.project_forward(ctx, gt, geom, y)
        ys.append(y)
    for t in (1, 2, 3):
        lb = b.loss_step(ys, rg.RGRT_LOSS_L2, hp, t)
        for i in range(len(scans)):
            ls = np.zeros(1, np.float32)
            rg.loss_step(ctx, gsingle[i], geoms[i], ys[i], rg.RGRT_LOSS_L2, hp, t, ls)
            assert lb[i] == pytest.approx(float(ls[0]), rel=1e-5, abs=1e-12)
    for i in range(len(scans)):
        a, c = gb[i].numpy(), gsingle[i].numpy()
        for k in ("mu", "ls", "q", "rho"):
            G0 = scans[i][0][k]
            da = a[k].astype(np.float64) - G0
            dc = c[k].astype(np.float64) - G0
            assert np.linalg.norm(da - dc) <= 1e-3 * np.linalg.norm(dc) + 1e-7, (i, k)
    assert b.info()["work_items"] == sum(g.n_rays // 256 for g in geoms[:1]) + sum(
        (gd["n_views"] * ((gd["n_cols"] + 15) // 16) * ((gd["n_rows"] + 15) // 16)) for _, gd in scans[1:])


def test_batch_replans_when_entries_outgrow_capacity(env):
    torch, rg, ctx = env
    scans = _scans(3, 3)
    gs = [rg.Gaussians(ctx, *_dev(torch, G)) for G, _ in scans]
    geoms = [rg.Geometry(ctx, gd) for _, gd in scans]
    b = rg.Batch(ctx, gs, geoms)
    cap0 = b.info()["key_capacity"]
    # grow every Gaussian 3x: far more (tile, Gaussian) entries than planned
    for (G, _), g in zip(scans, gs):
        ls = torch.from_numpy(np.ascontiguousarray(G["ls"] + math.log(3.0)).astype(np.float32)).cuda()
        g.set(ls=ls)
    outs = [torch.empty(g.n_rays, device="cuda") for g in geoms]
    b.forward(outs)
    info = b.info()
    assert info["replans"] >= 1 and info["key_capacity"] > cap0
    for g, geom, o in zip(gs, geoms, outs):
        ref = torch.empty(geom.n_rays, device="cuda")
        rg.project_forward(ctx, g, geom, ref)
        torch.cuda.synchronize()
        assert torch.equal(o, ref)


def test_batch_rejects_mixed_tiles(env):
    torch, rg, ctx = env
    (G1, gd1), (G2, gd2) = _scans(4, 2)
    gd2 = dict(gd2, tile_w=8, tile_h=8)
    gs = [rg.Gaussians(ctx, *_dev(torch, G)) for G in (G1, G2)]
    geoms = [rg.Geometry(ctx, gd) for gd in (gd1, gd2)]
    with pytest.raises(rg.RgrtError):
        rg.Batch(ctx, gs, geoms)


def test_autotune_returns_a_candidate(env):
    torch, rg, ctx = env
    G, _ = synth.workload_c2(5, n=4000, n_views=24, side=96)
    gd = synth.geom_c2(n_views=24, side=96)
    g = rg.Gaussians(ctx, *_dev(torch, G))
    tw, th, ms = rg.autotune_tile(ctx, g, gd, max_views=8)
    assert (tw, th) in {(16, 16), (16, 8), (8, 8), (32, 8)} and ms > 0


def test_batch_tile_lists_match_the_oracle(env, oracle):
    """The batch's own binning (device-side key count, padding keys past the
    step's entries, shared sort scratch) gives every scan the oracle's FP32
    tile sets -- scans small enough for the persistent launches and a scan
    large enough for launches of its own."""
    torch, rg, ctx = env
    scans = _scans(5, 5)
    G, _ = synth.workload_c2(77, n=20_000, n_views=90, side=256)
    scans.append((G, synth.geom_c2(n_views=90, side=256)))
    gs = [rg.Gaussians(ctx, *_dev(torch, G)) for G, _ in scans]
    geoms = [rg.Geometry(ctx, gd) for _, gd in scans]
    b = rg.Batch(ctx, gs, geoms)
    outs = [torch.empty(g.n_rays, device="cuda") for g in geoms]
    for rep in range(2):              # planning pass, then a graph replay
        b.forward(outs)
        for i, (G, gd) in enumerate(scans):
            start, gid = b.debug_tile_lists(i)
            rstart, rgid = oracle.tile_lists_fp32(gd, G, gd["tile_w"], gd["tile_h"])
            assert gid.size == rgid.size and gid.size > 0, (rep, i)
            assert np.array_equal(start, rstart), (rep, i)
            tile = np.repeat(np.arange(start.size - 1), np.diff(start))
            assert np.array_equal(gid[np.lexsort((gid, tile))], rgid), (rep, i)
