"""Host-side tests of the serving scheduler (no GPU): admission by slots and
HBM budget in arrival order, cancellation, failure isolation, and the
mini-batch view subsets of reconstruction jobs (pinned with the oracle)."""
import math
import threading
import time

import numpy as np
import pytest

from paper_2602_01057_gb300 import serve, synth


def _job(tag, n=1000, views=8, side=32, kind=serve.GRAD):
    G = synth.gaussians_uniform(n, 1)
    g = synth.geom_cone(views, side, side, 0.05, 0.05, 3.0, 4.5)
    return serve.Job(kind=kind, G=G, geom=g, y=np.zeros(synth.num_rays(g), np.float32), tag=tag)


class Recorder:
    """Host runner: sleeps, records how many jobs and bytes were in flight."""

    def __init__(self, server_ref, dt=0.02, fail_tags=()):
        self.ref = server_ref
        self.dt = dt
        self.fail_tags = set(fail_tags)
        self.lock = threading.Lock()
        self.live = 0
        self.max_live = 0
        self.ran = []

    def __call__(self, job, budget, stream):
        assert stream is None
        with self.lock:
            self.live += 1
            self.max_live = max(self.max_live, self.live)
            self.ran.append(job.tag)
            srv = self.ref[0]
            assert srv.used <= srv.budget
        time.sleep(self.dt)
        with self.lock:
            self.live -= 1
        if job.tag in self.fail_tags:
            raise RuntimeError(f"job {job.tag} failed")
        return job.tag


def _server(n_slots, budget, **kw):
    ref = [None]
    rec = Recorder(ref, **kw)
    srv = serve.Server(n_slots=n_slots, hbm_budget_bytes=budget, device=None, runner=rec)
    ref[0] = srv
    return srv, rec


def test_slots_bound_concurrency_and_results_return():
    big = 1 << 40
    srv, rec = _server(3, big)
    futs = [srv.submit(_job(i)) for i in range(12)]
    assert [f.result(timeout=30) for f in futs] == list(range(12))
    srv.close()
    assert rec.max_live <= 3 and srv.peak_running <= 3
    assert rec.max_live >= 2           # jobs do overlap
    assert srv.admit_order == list(range(12))
    assert len(srv.latencies()) == 12 and np.all(srv.latencies() > 0)


def test_budget_bounds_memory_and_keeps_arrival_order():
    small = _job("s")
    need = serve.job_budget(small)
    srv, rec = _server(8, int(2.5 * need))  # at most two small jobs fit
    jobs = [_job(i) for i in range(6)]
    futs = [srv.submit(j) for j in jobs]
    for f in futs:
        f.result(timeout=30)
    srv.close()
    assert srv.peak_used <= srv.budget
    assert rec.max_live <= 2
    assert srv.admit_order == list(range(6))


def test_large_job_is_not_overtaken():
    s = _job("s")
    need_s = serve.job_budget(s)
    L = _job("L", n=200000, views=64, side=64)
    need_L = serve.job_budget(L)
    assert need_L > 3 * need_s
    srv, rec = _server(4, need_L + need_s, dt=0.05)
    order = [_job("a"), L, _job("b"), _job("c")]
    futs = [srv.submit(j) for j in order]
    for f in futs:
        f.result(timeout=30)
    srv.close()
    # L waits for "a" to finish, and b, c wait for L to be admitted
    assert srv.admit_order == ["a", "L", "b", "c"]


def test_job_over_budget_rejected():
    srv, _ = _server(2, 1 << 20)
    f = srv.submit(_job("x"))
    with pytest.raises(ValueError):
        f.result(timeout=5)
    srv.close()


def test_cancel_before_admission_never_runs():
    srv, rec = _server(1, 1 << 40, dt=0.1)
    j0, j1, j2 = _job(0), _job(1), _job(2)
    f0 = srv.submit(j0)
    f1 = srv.submit(j1)
    f2 = srv.submit(j2)
    assert srv.cancel(j1, f1)
    assert f0.result(timeout=30) == 0 and f2.result(timeout=30) == 2
    srv.close()
    assert f1.cancelled()
    assert 1 not in rec.ran


def test_failed_job_does_not_stop_the_server():
    srv, rec = _server(2, 1 << 40, fail_tags={1})
    futs = [srv.submit(_job(i)) for i in range(4)]
    with pytest.raises(RuntimeError):
        futs[1].result(timeout=30)
    assert [futs[i].result(timeout=30) for i in (0, 2, 3)] == [0, 2, 3]
    srv.close()
    assert srv.used == 0 and srv.running == 0


def test_budget_grows_with_size():
    a = serve.job_budget(_job("a", n=1000))
    b = serve.job_budget(_job("b", n=100000))
    c = serve.job_budget(_job("c", n=1000, side=512))
    assert b > a and c > a
    # a 3-D PET job counts one view per (ring difference, angle)
    G = synth.gaussians_uniform(1000, 1)
    p0 = serve.job_budget(serve.Job(serve.FWD, G, synth.geom_pet3d(48, 65, 8, 400.0, 576, 4.0, 0)))
    p3 = serve.job_budget(serve.Job(serve.FWD, G, synth.geom_pet3d(48, 65, 8, 400.0, 576, 4.0, 3)))
    assert p3 > p0


@pytest.mark.parametrize("kind", ["cone", "parallel", "pet", "pet3d"])
def test_minibatch_subsets_reproduce_the_full_scan(oracle, kind):
    """The mini-batch geometries (explicit angles, PET included) project to
    exactly the matching views of the full scan (FP64 oracle)."""
    if kind == "pet3d":
        g = synth.geom_pet3d(12, 17, 5, 400.0, 576, 4.0, 2)
        G = synth.gaussians_uniform(30, 6, half_box=40.0, log_sigma=math.log(6.0))
        G["mu"][:, 2] *= 0.1
    elif kind == "pet":
        g = synth.geom_pet(12, 17, 5, 400.0, 576, 2.0)
        G = synth.gaussians_uniform(30, 7, half_box=40.0, log_sigma=math.log(6.0))
        G["mu"][:, 2] *= 0.1
    elif kind == "cone":
        g = synth.geom_cone(11, 9, 10, 0.2, 0.2, 3.0, 4.5)
        G = synth.gaussians_uniform(30, 8, log_sigma=math.log(0.2))
    else:
        g = synth.geom_parallel(11, 9, 10, 0.2, 0.2, -2.0, 2.0)
        G = synth.gaussians_uniform(30, 9, log_sigma=math.log(0.2))
    full = oracle.forward(g, G)["I"]
    geoms, order = serve.subset_geometries(g, 4, seed=3)
    assert sorted(order.tolist()) == list(range(g["n_views"]))
    assert [x["n_views"] for x in geoms] == [4] * (g["n_views"] // 4) + ([g["n_views"] % 4] if g["n_views"] % 4 else [])
    ys = serve.subset_measurements(g, full.astype(np.float32), order, 4)
    parts = np.concatenate([oracle.forward(x, G)["I"] for x in geoms])
    np.testing.assert_array_equal(parts.astype(np.float32), ys)
    assert np.abs(parts).max() > 0


def test_overlap_stats():
    """Sum, union, multiply covered time and peak concurrency of intervals."""
    from paper_2602_01057_gb300 import serve
    st = serve.overlap_stats([(0.0, 4.0), (1.0, 3.0), (2.0, 6.0), (10.0, 11.0)])
    assert st["busy_sum_ms"] == 4 + 2 + 4 + 1
    assert st["union_ms"] == 6 + 1
    assert st["overlapped_ms"] == 3          # [1, 4] has two or more
    assert st["max_concurrent"] == 3
    assert serve.overlap_stats([])["jobs"] == 0
