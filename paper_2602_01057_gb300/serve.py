"""Continuous-batching server for projection jobs.

Three kinds of job, all on one geometry and one set of Gaussians each:

* ``fwd``   forward projection (returns I);
* ``grad``  loss and gradient (forward, loss against the job's measurements,
  adjoint, parameter chain: returns the loss and dL/d(mu, logscale, quat, rho));
* ``recon`` reconstruction: ``n_iter`` Adam steps of ``loss_step``, each on a
  mini-batch of ``views_per_iter`` views (the views are split into mini-batches
  by a permutation seeded per job and visited in turn); returns the fitted
  parameters and the loss of every iteration.

The server keeps up to ``n_slots`` jobs on the device at once.  Each admitted
job gets its own library context (its binning scratch is bounded by the job's
memory budget), its own CUDA stream and its own host thread, so the kernels of
different jobs overlap on the GPU; a job's Gaussians, measurements and Adam
state stay on the device from admission to completion.  A job is admitted as
soon as a slot is free and its memory budget fits what the running jobs leave
of the server's HBM budget, in arrival order (a job that does not fit yet holds
back the ones behind it, so large jobs are not starved).  A job cancelled
before admission never runs; a reconstruction cancelled while running stops
after its current iteration.  Latency is measured from arrival (or submission)
to completion.

All projector arithmetic runs in the CUDA library; this module only schedules.
``n_slots = 1`` is the one-job-at-a-time (FIFO) server used as the baseline.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import threading
import time
from collections import deque

import numpy as np

from . import rgrt, synth

FWD, GRAD, RECON = "fwd", "grad", "recon"


@dataclasses.dataclass
class Job:
    kind: str                      # FWD, GRAD or RECON
    G: dict                        # mu[n,3], ls[n,3], q[n,4], rho[n] (host, float32)
    geom: dict                     # geometry description (synth format)
    y: np.ndarray | None = None    # measurements [num_rays] (GRAD, RECON)
    loss: int = rgrt.RGRT_LOSS_L2
    n_iter: int = 1                # RECON
    views_per_iter: int = 8        # RECON
    seed: int = 0                  # RECON mini-batch permutation
    hp: dict | None = None         # adam_params keyword arguments
    tag: object = None
    t_arrive: float | None = None  # arrival time (perf_counter); default: submission
    t_start: float = 0.0
    t_done: float = 0.0
    dev_ms: tuple | None = None    # (start, end) on the device, ms after the server's reference event
    rays: int = 0                  # rays projected (forward + adjoint counted once)
    cancelled: threading.Event = dataclasses.field(default_factory=threading.Event)


def num_rays(geom: dict) -> int:
    return synth.num_rays(geom)


def job_budget(job: Job) -> int:
    """Device bytes the job may use: resident state plus binning scratch.

    Resident, per Gaussian: parameters (11 floats), Adam moments (22), records
    (32), gradient accumulator (16), flat gradients and staged gradient
    outputs (22); per ray: measurements, projection, residual and a staging
    copy.  Binning: per (Gaussian, view) of a chunk 16 bytes of counts,
    offsets and boxes plus room for ~12 tile entries of 16 bytes (keys,
    values and their sort buffers); the library splits views into chunks
    that fit the context's budget, so the chunk is capped at 64 views.
    Plus 64 MiB of slack for tables and small buffers."""
    n = int(job.G["mu"].shape[0])
    r = num_rays(job.geom)
    v = int(job.geom.get("n_views", 1))
    if job.kind == RECON:
        v = min(v, int(job.views_per_iter))
    if job.geom.get("kind") == "pet3d":
        v *= 2 * int(job.geom["max_ring_diff"]) + 1      # one view per ring difference and angle
    v = min(v, 64)
    resident = 4 * n * (11 + 22 + 32 + 16 + 22) + 16 * r
    scratch = n * v * (16 + 12 * 16)
    return int(resident + scratch + (64 << 20))


def next_admissible(queue, free_bytes: int, free_slots: int):
    """Position in `queue` (jobs in arrival order) of the job to admit, or None.

    The head is admitted when a slot is free and its budget fits what is
    free; otherwise nothing is (no job overtakes an earlier one)."""
    if free_slots <= 0 or not queue:
        return None
    return 0 if job_budget(queue[0]) <= free_bytes else None


def subset_geometries(geom: dict, views_per_iter: int, seed: int):
    """Split the views of `geom` into mini-batch geometries.

    Returns (geoms, order): geoms[b] holds views order[b*k:(b+1)*k] with
    explicit angles (CT, or PET sinogram angles pi j / n_views; a 3-D PET
    mini-batch keeps every ring difference of its angles), order the seeded
    permutation of the views."""
    V = int(geom["n_views"])
    order = np.random.default_rng(seed).permutation(V)
    if geom["kind"] in ("pet", "pet3d"):
        all_angles = np.pi * np.arange(V, dtype=np.float64) / V
    else:
        all_angles = np.asarray(geom["angles"], dtype=np.float64)
    out = []
    for b in range(0, V, views_per_iter):
        idx = order[b:b + views_per_iter]
        g = dict(geom)
        g["n_views"] = int(idx.size)
        g["angles"] = all_angles[idx].copy()
        out.append(g)
    return out, order


def subset_measurements(geom: dict, y: np.ndarray, order: np.ndarray, views_per_iter: int):
    """y rearranged so that mini-batch b's measurements are one contiguous
    block in its geometry's layout (CT [view][row][col], PET
    [plane][angle][radial], 3-D PET [ring difference][angle][ring pair][radial])."""
    V, H, W = int(geom["n_views"]), int(geom["n_rows"]), int(geom["n_cols"])
    parts = []
    for b in range(0, V, views_per_iter):
        idx = order[b:b + views_per_iter]
        if geom["kind"] == "pet":
            parts.append(y.reshape(H, V, W)[:, idx, :].reshape(-1))
        elif geom["kind"] == "pet3d":
            parts.append(y.reshape(-1, V, H, W)[:, idx].reshape(-1))
        else:
            parts.append(y.reshape(V, H, W)[idx].reshape(-1))
    return np.concatenate(parts).astype(np.float32)


def run_job(job: Job, device: int, budget: int, stream) -> dict:
    """Run one job on `stream` with its own context (device `device`)."""
    import torch
    dev = torch.device("cuda", device)
    s = stream.cuda_stream if stream is not None else None
    ctx = rgrt.Context(device, budget)
    objs = []
    try:
        g = rgrt.Gaussians(ctx, *(np.ascontiguousarray(job.G[k], dtype=np.float32)
                                  for k in ("mu", "ls", "q", "rho")))
        objs.append(g)
        if job.G.get("kernel", "gaussian") != "gaussian":
            g.set_kernel(job.G["kernel"])
        hp = rgrt.adam_params(**(job.hp or {}))
        if job.kind == FWD:
            geom = rgrt.Geometry(ctx, job.geom)
            objs.append(geom)
            I = torch.empty(geom.n_rays, device=dev)
            rgrt.project_forward(ctx, g, geom, I, stream=s)
            job.rays = geom.n_rays
            return dict(I=I.cpu().numpy())
        if job.kind == GRAD:
            geom = rgrt.Geometry(ctx, job.geom)
            objs.append(geom)
            y = torch.from_numpy(np.ascontiguousarray(job.y, dtype=np.float32)).to(dev)
            n = g.n
            outs = [torch.empty(sz, device=dev) for sz in ((n, 3), (n, 3), (n, 4), (n,))]
            lo = np.zeros(1, np.float32)
            rgrt.loss_grad(ctx, g, geom, y, job.loss, hp, lo, *outs, stream=s)
            job.rays = geom.n_rays
            return dict(loss=float(lo[0]),
                        grad={k: o.cpu().numpy() for k, o in zip(("mu", "ls", "q", "rho"), outs)})
        if job.kind != RECON:
            raise ValueError(f"unknown job kind {job.kind!r}")
        if job.geom["kind"] == "rays":
            raise ValueError("reconstruction jobs take detector geometries (mini-batches are views)")
        geoms, order = subset_geometries(job.geom, job.views_per_iter, job.seed)
        ys = subset_measurements(job.geom, job.y, order, job.views_per_iter)
        yd = torch.from_numpy(ys).to(dev)
        hs, offs, off = [], [], 0
        for gd in geoms:
            h = rgrt.Geometry(ctx, gd)
            objs.append(h)
            hs.append(h)
            offs.append(off)
            off += h.n_rays
        losses = np.zeros(job.n_iter, np.float32)
        lo = np.zeros(1, np.float32)
        done = 0
        for it in range(job.n_iter):
            if job.cancelled.is_set():
                break
            b = it % len(hs)
            rgrt.loss_step(ctx, g, hs[b], yd[offs[b]:offs[b] + hs[b].n_rays], job.loss, hp, it + 1, lo,
                           stream=s)
            losses[it] = lo[0]
            job.rays += hs[b].n_rays
            done += 1
        return dict(losses=losses[:done], params=g.numpy(), iterations=done)
    finally:
        for o in reversed(objs):
            o.close()
        ctx.close()


def overlap_stats(iv):
    """Sum, union, time with two or more intervals, and peak concurrency of
    (start, end) intervals."""
    if not iv:
        return dict(jobs=0, busy_sum_ms=0.0, union_ms=0.0, overlapped_ms=0.0, max_concurrent=0)
    ev = sorted([(a, 1) for a, _ in iv] + [(b, -1) for _, b in iv], key=lambda x: (x[0], x[1]))
    cur = peak = 0
    last = ev[0][0]
    union = multi = 0.0
    for t, dlt in ev:
        if cur >= 1:
            union += t - last
        if cur >= 2:
            multi += t - last
        cur += dlt
        peak = max(peak, cur)
        last = t
    return dict(jobs=len(iv), busy_sum_ms=float(sum(b - a for a, b in iv)), union_ms=union,
                overlapped_ms=multi, max_concurrent=peak)


class Server:
    """Up to `n_slots` jobs in flight, admitted by HBM budget in arrival order.

    runner(job, budget, stream) -> result runs one job; the default runs it
    through the CUDA library on `device`.  With device=None no CUDA stream is
    made (host-only runners, for tests of the scheduling)."""

    def __init__(self, n_slots: int = 4, hbm_budget_bytes: int = 150 << 30, device: int | None = 0,
                 runner=None):
        if n_slots < 1:
            raise ValueError("n_slots must be >= 1")
        self.n_slots = n_slots
        self.budget = int(hbm_budget_bytes)
        self.device = device
        self.runner = runner or (lambda job, budget, stream: run_job(job, device, budget, stream))
        self.queue: deque = deque()
        self.used = 0
        self.running = 0
        self.peak_used = 0
        self.peak_running = 0
        self.cv = threading.Condition()
        self.stop = False
        self.done: list[Job] = []
        self.admit_order: list[object] = []
        # device time line: CUDA events on each job's stream at its start and
        # end, measured from a reference event recorded when the server starts
        self.ref = None
        if device is not None:
            import torch
            with torch.cuda.device(device):
                self.ref = torch.cuda.Event(enable_timing=True)
                self.ref.record()
                self.ref.synchronize()
        self.threads = [threading.Thread(target=self._worker, daemon=True) for _ in range(n_slots)]
        for t in self.threads:
            t.start()

    # -- client side ---------------------------------------------------------
    def submit(self, job: Job) -> cf.Future:
        fut: cf.Future = cf.Future()
        if job.t_arrive is None:
            job.t_arrive = time.perf_counter()
        if job_budget(job) > self.budget:
            fut.set_exception(ValueError(f"job needs {job_budget(job)} bytes, the server has {self.budget}"))
            return fut
        with self.cv:
            if self.stop:
                fut.set_exception(RuntimeError("server closed"))
                return fut
            self.queue.append((job, fut))
            self.cv.notify_all()
        return fut

    def cancel(self, job: Job, fut: cf.Future) -> bool:
        """Cancel a job: before admission it never runs (returns True); a
        running reconstruction stops after its current iteration."""
        job.cancelled.set()
        return fut.cancel()

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()

    def latencies(self):
        """Seconds from arrival to completion of every finished job."""
        return np.array([j.t_done - j.t_arrive for j in self.done])

    def device_overlap(self):
        """How the finished jobs' work lay on the device: from each job's
        device interval (first to last operation on its stream), the sum of
        the intervals, their union, the time covered by two jobs or more and
        the largest number at once (ms)."""
        iv = sorted(j.dev_ms for j in self.done if j.dev_ms is not None)
        return overlap_stats(iv)

    # -- worker side ---------------------------------------------------------

    def _take(self):
        """Block until a job can be admitted; returns (job, fut, need) or None."""
        with self.cv:
            while True:
                while self.queue and self.queue[0][1].cancelled():
                    self.queue.popleft()
                if self.stop and not self.queue:
                    return None
                jobs = [j for j, _ in self.queue]
                k = next_admissible(jobs, self.budget - self.used, self.n_slots - self.running)
                if k is not None:
                    job, fut = self.queue[k]
                    del self.queue[k]
                    if not fut.set_running_or_notify_cancel():
                        continue
                    need = job_budget(job)
                    self.used += need
                    self.running += 1
                    self.peak_used = max(self.peak_used, self.used)
                    self.peak_running = max(self.peak_running, self.running)
                    self.admit_order.append(job.tag)
                    return job, fut, need
                self.cv.wait()

    def _worker(self):
        stream = None
        if self.device is not None:
            import torch
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream(device=self.device)
        while True:
            got = self._take()
            if got is None:
                return
            job, fut, need = got
            job.t_start = time.perf_counter()
            try:
                if stream is not None:
                    import torch
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    with torch.cuda.stream(stream):
                        e0.record(stream)
                        res = self.runner(job, need, stream)
                        e1.record(stream)
                    e1.synchronize()
                    job.dev_ms = (self.ref.elapsed_time(e0), self.ref.elapsed_time(e1))
                else:
                    res = self.runner(job, need, stream)
                job.t_done = time.perf_counter()
                fut.set_result(res)
            except Exception as e:  # the job fails; the server keeps serving
                job.t_done = time.perf_counter()
                fut.set_exception(e)
            with self.cv:
                self.used -= need
                self.running -= 1
                self.done.append(job)
                self.cv.notify_all()
