"""Serving on the GPU: every job's result is the same alone and in the mix.

The jobs (forward, loss + gradient and mini-batch reconstructions, CT and
PET) first run one at a time, then all together through a server with four
slots, so that their kernels overlap on the device.  Forward projections and
losses are deterministic (per-ray sums in fixed point, FP64 loss partials in
a fixed order) and must agree bit for bit; gradients are accumulated with
float atomics, so they agree to rounding: within the projector's gradient
tolerance (1e-4 relative L2).  Reconstructions feed those gradients back through Adam, so
their parameters agree within the same tolerance.  One forward job is also
checked against the FP64 oracle.
"""
import math

import numpy as np
import pytest

from paper_2602_01057_gb300 import synth

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4
FWD_TOL = 1e-5


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_01057_gb300 import build, rgrt, serve
    build.build()
    return torch, rgrt, serve


def rel_l2(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def _jobs(serve, rgrt, orc):
    jobs = []
    # CT cone: loss + gradient, and a reconstruction from perturbed Gaussians
    Gt, _ = synth.workload_c2(0, n=3000, n_views=24, side=64)
    gct = synth.geom_c2(n_views=24, side=64)
    y_ct = orc.forward(gct, Gt)["I"].astype(np.float32)
    G0 = synth.perturbed(Gt, 5, pos_std=0.01)
    jobs.append(serve.Job(kind=serve.GRAD, G=G0, geom=gct, y=y_ct, tag="ct_grad"))
    jobs.append(serve.Job(kind=serve.RECON, G=G0, geom=gct, y=y_ct, n_iter=15, views_per_iter=8,
                          seed=11, tag="ct_recon"))
    # PET (arc-corrected): Poisson loss + gradient, and a reconstruction
    Gp, _ = synth.workload_c3(0, n=3000, n_angles=24, n_radial=129, n_planes=15)
    gp = synth.geom_c3(24, 129, 15, arc_mode=0)
    lam = 50.0 * orc.forward(gp, Gp)["I"] + 1e-3
    y_pet = np.random.default_rng(2).poisson(lam).astype(np.float32)
    hp = dict(kappa=50.0, poisson_eps=1e-3)
    Gp0 = synth.perturbed(Gp, 6, pos_std=2.0)
    jobs.append(serve.Job(kind=serve.GRAD, G=Gp0, geom=gp, y=y_pet, loss=rgrt.RGRT_LOSS_POISSON, hp=hp,
                          tag="pet_grad"))
    jobs.append(serve.Job(kind=serve.RECON, G=Gp0, geom=gp, y=y_pet, loss=rgrt.RGRT_LOSS_POISSON, hp=hp,
                          n_iter=10, views_per_iter=8, seed=12, tag="pet_recon"))
    # parallel-beam forward
    G1, g1 = synth.workload_c1(0)
    jobs.append(serve.Job(kind=serve.FWD, G=G1, geom=g1, tag="c1_fwd"))
    return jobs


def _alone(torch, serve, jobs):
    out = {}
    s = torch.cuda.Stream()
    for j in jobs:
        with torch.cuda.stream(s):
            out[j.tag] = serve.run_job(j, 0, serve.job_budget(j), s)
    return out


def _compare(serve, a, b, kind):
    if kind == serve.FWD:
        np.testing.assert_array_equal(a["I"], b["I"])
    elif kind == serve.GRAD:
        assert a["loss"] == b["loss"]
        for k in ("mu", "ls", "q", "rho"):
            assert rel_l2(b["grad"][k], a["grad"][k]) < GRAD_TOL, k
    else:
        assert a["iterations"] == b["iterations"]
        assert a["losses"][0] == b["losses"][0]      # first forward: same parameters
        np.testing.assert_allclose(b["losses"], a["losses"], rtol=1e-4)
        for k in ("mu", "ls", "q", "rho"):
            d_a = a["params"][k].astype(np.float64)
            d_b = b["params"][k].astype(np.float64)
            assert rel_l2(d_b, d_a) < GRAD_TOL, k


def test_results_same_alone_and_in_the_mix(mods, oracle):
    torch, rgrt, serve = mods
    jobs = _jobs(serve, rgrt, oracle)
    alone = _alone(torch, serve, jobs)
    # the forward job against the FP64 oracle
    fj = [j for j in jobs if j.kind == serve.FWD][0]
    ref = oracle.forward(fj.geom, fj.G)
    I = alone[fj.tag]["I"].astype(np.float64)
    clip = np.clip(I, ref["I_lo"], ref["I_hi"])
    assert np.linalg.norm(I - clip) / np.linalg.norm(clip) < FWD_TOL
    # the reconstructions make progress
    for t in ("ct_recon", "pet_recon"):
        L = alone[t]["losses"]
        assert L[-8:].mean() < L[:8].mean()
    # every job twice in the mix, interleaved, four slots
    srv = serve.Server(n_slots=4, hbm_budget_bytes=24 << 30, device=0)
    mix = []
    for rep in range(2):
        for j in _jobs(serve, rgrt, oracle):
            j.tag = (j.tag, rep)
            mix.append((j, srv.submit(j)))
    res = [(j, f.result(timeout=600)) for j, f in mix]
    srv.close()
    assert srv.peak_running > 1                 # jobs were in flight together
    # and their work lay on the device together: the jobs' device intervals
    # (CUDA events on their streams) cover some time two or more at once
    ov = srv.device_overlap()
    assert ov["jobs"] == len(mix) and ov["max_concurrent"] >= 2 and ov["overlapped_ms"] > 0.0
    for j, r in res:
        _compare(serve, alone[j.tag[0]], r, j.kind)


def test_cancelled_reconstruction_stops(mods):
    torch, rgrt, serve = mods
    G, _ = synth.workload_c2(1, n=2000, n_views=16, side=48)
    g = synth.geom_c2(n_views=16, side=48)
    y = np.zeros(synth.num_rays(g), np.float32)
    srv = serve.Server(n_slots=1, hbm_budget_bytes=8 << 30, device=0)
    j = serve.Job(kind=serve.RECON, G=G, geom=g, y=y, n_iter=100000, tag="long")
    f = srv.submit(j)
    import time
    while j.t_start == 0.0:
        time.sleep(0.01)
    time.sleep(0.2)
    assert not srv.cancel(j, f)                 # already running: stops at an iteration boundary
    r = f.result(timeout=120)
    srv.close()
    assert 0 < r["iterations"] < 100000
    assert np.all(np.isfinite(r["params"]["mu"]))
