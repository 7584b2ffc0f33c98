"""Benchmark: rays/s of one full optimisation step (forward projection, L2
loss, adjoint, parameter chain, Adam) of the analytic Gaussian ray-tracing
projector on the cone-beam CT workload (50,000 Gaussians fitted to a
12-ellipsoid phantom, 180 views x 256 x 256 detector).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  Under torchrun each rank runs its own independent
scan (weak scaling, no collective on the data path); the reported time is the
maximum over ranks.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload (its rays/s extrapolates linearly in the
number of rays).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2602_01057_gb300 import synth  # noqa: E402

METRIC = "rays/s fwd+bwd"
UNIT = "rays/s"
# Algorithmic work per kept (ray, Gaussian) pair (m <= 9) of the closed form
# (Eqs. 7-11) in its recentred form: 39 FP32 operations for the value
# (delta 3, recentring 6, P d 9, A and B 6, P delta and C 12, m 3, value and
# sum ~5) and 2.5 times that for the adjoint; 3 special-function operations
# (1/A, A^-1/2, exp) for either.  FP32 peak = SMs x 128 lanes x SM clock (one
# operation per lane per clock), MUFU peak = SMs x 16 x SM clock; the SM
# count is read from the device and the clock is the median sampled during
# the timed region.
OPS_PER_PAIR_FWD = 39.0
OPS_PER_PAIR_ADJ = 97.5
MUFU_PER_PAIR = 3.0
# With time of flight each kept pair adds, per bin, 4 operations and one
# exponential to the forward (the bin's offset, its square, the scale, the
# accumulation) and 8 operations and one exponential to the adjoint (the same
# weight, times dL/dI, and its three sums).
OPS_PER_BIN_FWD = 4.0
OPS_PER_BIN_ADJ = 8.0
MUFU_PER_BIN = 1.0
FP32_LANES_PER_SM = 128
MUFU_LANES_PER_SM = 16
# DRAM bytes (read + write) of one launch of an integration kernel, from an
# ncu capture of the workload at full size (dram__bytes.sum.per_second x
# gpu__time_duration.sum of one timed-step launch), valid only while the
# kernel sources hash to the recorded digest (otherwise the bench line
# reports null)
TRAFFIC = {
    ("c2", "k_forward"): (261.9e6, "7259bc5991d372fe"),
    ("c2", "k_adjoint"): (275.9e6, "7259bc5991d372fe"),
    ("c3", "k_forward"): (472.0e6, "7259bc5991d372fe"),
    ("c3", "k_adjoint"): (477.1e6, "7259bc5991d372fe"),
}
KERNEL_SOURCES = ("paper_2602_01057_gb300/csrc/project.cu", "paper_2602_01057_gb300/csrc/pair.cuh")
WORKLOADS = {
    "c2": "cone-beam CT fwd+bwd (L2 + Adam): 50,000 Gaussians fitted to a 12-ellipsoid phantom, "
          "180 views over 360 deg, 256x256 detector, source-origin 1000 mm, source-detector 1500 mm",
    "c3": "PET fwd+bwd (Poisson NLL + Adam): 200,000 Gaussians, ring radius 400 mm, 576 crystals, "
          "arc-corrected 288 angles x 329 radial x 63 planes",
    "c1": "parallel-beam CT fwd+bwd (L2 + Adam): 1,000 Gaussians, 16 views x 64x64",
    "c4": "batching: 64 cone-beam CT scans of uneven size (Gaussians log-uniform 5k-500k, views "
          "U{30..360}, detector side U{128,256,384,512}), fwd+bwd (L2 + Adam) as one graph-captured "
          "step with persistent launches, tile shape from the autotuner; against 64 plain steps",
    "c4-small": "batching, small scans: 64 cone-beam CT scans (Gaussians log-uniform 1k-20k, views "
                "U{16..64}, detector side U{64,96,128}), fwd+bwd (L2 + Adam) as one graph-captured step; "
                "against 64 plain steps",
    "recon": "reconstruction quality: the 50,000 Gaussians of the cone-beam CT workload fitted (L2 + Adam) "
             "to the exact line integrals of their 12-ellipsoid phantom over 180 views x 256^2; PSNR of the "
             "voxelised volume (128^3) against the phantom's density",
    "pet3d": "fully 3-D PET fwd+bwd (Poisson NLL + Adam) on structured sinograms: 200,000 Gaussians, 32 "
             "rings of 576 crystals (radius 400 mm, ring pitch 4 mm), ring differences up to 5 (11 segments), "
             "288 angles x 329 arc-corrected radial bins (30.5M LORs; 33.4M sinogram bins with the rows "
             "past each segment's last ring pair)",
    "c3-tof": "time-of-flight PET fwd+bwd (Poisson NLL + Adam): the C3 workload (200,000 Gaussians, 288 x 329 "
              "x 63 arc-corrected sinogram) with 13 TOF bins per LOR (47 mm apart, Gaussian TOF kernel of "
              "31.85 mm, 500 ps FWHM): 77.6M outputs",
    "pet3d-rays": "the LORs of pet3d as explicit rays (geometry_set_rays, no detector structure), fwd+bwd "
                  "(Poisson NLL + Adam)",
    "helical": "helical cone-beam CT as explicit rays (geometry_set_rays): the 50,000 Gaussians of the "
               "cone-beam workload, one turn of 180 views x 256x256 (source-origin 1000 mm, source-detector "
               "1500 mm, 128 mm feed per turn), fwd+bwd (L2 + Adam)",
    "points": "arc vs raw radial sampling (a synthetic analogue of the three-point-source study): 1 mm "
              "spheres at (0, 10), (0, 100), (0, 200) mm in the C3 ring (5 planes 2 mm apart), 5M Poisson "
              "counts sampled at raw crystal-pair positions; reconstructed (L2 + Adam, blind 4 mm grid of "
              "Gaussians) from the raw sinogram with the raw geometry and from its arc-corrected resampling "
              "with the arc-corrected geometry; FWHM of the voxelised sources",
    "vox": "voxelisation: the 50,000 Gaussians of the cone-beam CT workload on a 256^3 grid of "
           "[-1, 1]^3 (density field with the 3-sigma cut)",
    "c5": "serving: Poisson arrivals, 70% loss+gradient jobs / 30% 200-iteration Adam reconstructions "
          "(8 views per iteration); CT (cone, C2 geometry scaled to the side) and PET (288x329x63 "
          "arc-corrected) 50:50; admission by a 150 GB HBM budget; continuous batching vs a "
          "one-job-at-a-time server",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=list(WORKLOADS))
    ap.add_argument("--scans", type=int, default=64, help="c4: number of scans")
    ap.add_argument("--jobs", type=int, default=48, help="c5: jobs per run")
    ap.add_argument("--slots", type=int, default=4, help="c5: slots of the continuous server")
    ap.add_argument("--rate", type=float, default=200.0, help="c5: arrival rate (jobs/s)")
    ap.add_argument("--iters", type=int, default=300, help="recon: optimisation steps")
    ap.add_argument("--point-iters", type=int, default=1500, help="points: optimisation steps per reconstruction")
    ap.add_argument("--pet3d-angles", type=int, default=288,
                    help="pet3d: sinogram angles (fewer: a smaller case of the same scanner, for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="c2 default run: skip the PET, batching and serving measurements in the same line")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fitted", action="store_true", help="skip the fitted-state timing")
    ap.add_argument("--tile", default="auto", help="binning tile WxH, or auto (the autotuner)")
    ap.add_argument("--seed", type=int, default=0, help="c1-c3: workload seed (rank r uses seed + r)")
    ap.add_argument("--no-flush", action="store_true", help="skip the L2 flush between steps")
    ap.add_argument("--cpu-views", type=int, default=0, help="views in the CPU sample (0 = auto)")
    return ap.parse_args()


def _params(G):
    return {k: G[k] for k in ("mu", "ls", "q", "rho")}


def workload(name, seed, pet3d_angles=288):
    G, true, gd, loss = _workload(name, seed)
    if name == "pet3d" and pet3d_angles != gd["n_views"]:
        gd = dict(gd, n_views=int(pet3d_angles))
    return _params(G), _params(true), gd, loss


def _workload(name, seed):
    if name == "c2":
        G, gd = synth.workload_c2(seed)
        true = synth.perturbed(G, seed + 101, pos_std=0.01)
        return G, true, gd, "l2"
    if name == "c3":
        G, gd = synth.workload_c3(seed)
        true = synth.perturbed(G, seed + 101, pos_std=1.0)
        return G, true, gd, "poisson"
    if name == "pet3d":
        G, _ = synth.workload_c3(seed)
        true = synth.perturbed(G, seed + 101, pos_std=1.0)
        return G, true, synth.geom_c3_3d(), "poisson"
    if name == "c3-tof":
        G, gd = synth.workload_c3(seed)
        true = synth.perturbed(G, seed + 101, pos_std=1.0)
        return G, true, synth.with_tof_bins(gd, *TOF_BINS), "poisson"
    if name == "c1":
        G, gd = synth.workload_c1(seed)
        true = synth.perturbed(G, seed + 101, pos_std=0.01)
        return G, true, gd, "l2"
    raise ValueError(f"no single-scan step for workload {name!r}")


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device="cuda"):
    """Maximum of a per-rank scalar over all ranks (identity for one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(rays_per_step, steps, world, ms_max):
    """Whole-job rays/s: every rank projects its own scan of rays_per_step rays
    per step; the job takes as long as the slowest rank."""
    return rays_per_step * steps * world / (ms_max / 1e3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def sample_geometry(gd, n_views):
    """The first n_views views of a geometry."""
    sub = dict(gd)
    sub["n_views"] = n_views
    if gd["kind"] not in ("pet", "pet3d"):
        sub["angles"] = gd["angles"][:n_views]
    return sub


def oracle_sample(G, gd, loss, n_views, nthreads=0, keep=False):
    """Oracle fwd + loss + bwd on the first n_views views: (seconds, rays)
    (and, with keep, the projection, dL/dI and gradients)."""
    from oracle import oracle
    sub = sample_geometry(gd, n_views)
    rays = synth.num_rays(sub)
    y = np.zeros(rays)
    t0 = time.perf_counter()
    f = oracle.forward(sub, G, nthreads=nthreads)
    if loss == "l2":
        _, w = oracle.loss_l2(f["I"], y)
    else:
        _, w = oracle.loss_poisson(f["I"], y + 1.0, 1.0, 1e-9)
    g = oracle.backward(sub, G, w, nthreads=nthreads)
    sec = time.perf_counter() - t0
    return (sec, rays, f, w, g) if keep else (sec, rays)


def cpu_baseline(G, gd, loss, n_views, rgrt=None, ctx=None):
    """The oracle timed on the host cores on a sample of the workload (and on
    one core on one view); with the library at hand, also the FP32-vs-FP64
    error of the GPU projection and adjoint on that sample."""
    from oracle import oracle
    sec, rays, f, w, g = oracle_sample(G, gd, loss, n_views, keep=True)
    out = dict(value=rays / sec, unit=UNIT, cores=oracle.max_threads(), kind="oracle",
               sample=f"FP64 oracle fwd+loss+bwd on {n_views} of {gd['n_views']} views "
                      f"({rays} rays, all Gaussians); {sec:.1f} s")
    s1, r1 = oracle_sample(G, gd, loss, 1, nthreads=1)
    out["single_core"] = dict(value=r1 / s1, unit=UNIT, cores=1,
                              sample=f"1 view ({r1} rays, all Gaussians); {s1:.1f} s")
    if rgrt is not None:
        out["fp32_vs_fp64"] = gpu_error(rgrt, ctx, G, sample_geometry(gd, n_views), f, w, g)
    return out


def gpu_error(rgrt, ctx, G, sub, f, w, g):
    """Relative L2 distance of the GPU projection and gradients from the
    oracle's admissible bracket (pairs within the band of the 3-sigma cut may
    go either way), on the sample geometry, from the initial Gaussians."""
    import torch
    geom = rgrt.Geometry(ctx, sub)
    gs = rgrt.Gaussians(ctx, *[torch.from_numpy(np.ascontiguousarray(G[k])).cuda()
                              for k in ("mu", "ls", "q", "rho")])
    I = torch.empty(geom.n_rays, device="cuda")
    rgrt.project_forward(ctx, gs, geom, I)
    n = gs.n
    outs = [torch.empty(sz, device="cuda") for sz in ((n, 3), (n, 3), (n, 4), (n,))]
    rgrt.project_backward(ctx, gs, geom, torch.from_numpy(np.asarray(w, np.float32)).cuda(), *outs)
    torch.cuda.synchronize()

    def dist(x, lo, hi, nom):
        x = np.asarray(x, np.float64).reshape(-1)
        c = np.clip(x, np.asarray(lo).reshape(-1), np.asarray(hi).reshape(-1))
        return float(np.linalg.norm(x - c) / max(np.linalg.norm(np.asarray(nom).reshape(-1)), 1e-300))

    res = dict(forward_rel_l2=dist(I.cpu().numpy(), f["I_lo"], f["I_hi"], f["I"]))
    for k, o in zip(("mu", "ls", "q", "rho"), outs):
        res[f"grad_{k}_rel_l2"] = dist(o.cpu().numpy(), g["lo"][k], g["hi"][k], g[k])
    res["tolerance"] = dict(forward=1e-5, gradient=1e-4)
    gs.close()
    geom.close()
    return res


def auto_views(name):
    return {"c2": 4, "c3": 4, "c1": 16, "pet3d": 1}[name]


REFERENCE_WORKLOADS = ("c1", "c2", "c3", "pet3d")


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    if args.workload not in REFERENCE_WORKLOADS:
        print(json.dumps(dict(impl="reference", unavailable=(
            f"the oracle's timed sample covers the single-scan steps {', '.join(REFERENCE_WORKLOADS)}, "
            f"not {args.workload}"))), flush=True)
        return
    G, _, gd, loss = workload(args.workload, 0)
    nv = args.cpu_views or auto_views(args.workload)
    if args.warmup > 0:
        oracle_sample(G, gd, loss, 1)
    times, rays = [], 0
    for _ in range(args.steps):
        s, rays = oracle_sample(G, gd, loss, nv)
        times.append(s)
    from oracle import oracle
    tot = sum(times)
    value = rays * args.steps / tot
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * tot / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic",
                config=dict(workload=WORKLOADS[args.workload],
                            sample=f"{nv} of {gd['n_views']} views per step"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=oracle.max_threads(), kind="oracle",
                                  sample=f"FP64 oracle fwd+loss+bwd, {nv} of {gd['n_views']} "
                                         f"views ({rays} rays) per step"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return dict(sm_mhz=float(np.median(sm)), sm_max_mhz=float(max(mx)), samples=len(sm),
                    reasons=sorted(reasons))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def measured_peaks():
    """HBM copy bandwidth (GB/s) measured on this machine's GPUs, and where it came from."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            m = json.load(f)
        return dict(hbm_gbs=float(m["hbm_gbs"]), sm_max_mhz=float(m.get("sm_max_mhz", 0.0)),
                    source="measured (MEASURED_PEAKS.json)")
    except (OSError, KeyError, ValueError):
        return dict(hbm_gbs=6800.0, sm_max_mhz=0.0, source="fallback (6.8 TB/s)")


def sources_digest():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def sort_passes(tiles, n_views=1):
    """Radix passes of the tile sort: 8-bit digits over the tile within the
    view plus an 8-bit position code (each view's keys are sorted on their
    own while view << bits of the tile fits 24 bits; else over the tile id of
    all the views)."""
    tpv = max(1, tiles // max(1, n_views))
    lb = math.ceil(math.log2(tpv)) if tpv > 1 else 0
    if (n_views << lb) < (1 << 24):
        return (lb + 8 + 7) // 8
    bits = max(1, math.ceil(math.log2(max(tiles, 2)))) + 8
    return (bits + 7) // 8


def binning_bytes(n_gauss, n_views, keys, tiles):
    """Algorithmic DRAM bytes of one binning (cull, scan, emit, sort, ranges):
    per (view, Gaussian) the 48-byte culling record read and its count and
    pixel box written (60 B), the scan's read and write (8 B), the emit's
    reads (16 B); per key the emit's write (8 B), 16 B per sort pass and the
    ranges' 4-byte read; 8 B per tile range."""
    e = float(n_gauss) * n_views
    parts = dict(k_cull=60.0 * e, scan=8.0 * e, k_emit=16.0 * e + 8.0 * keys,
                 radix_sort=16.0 * sort_passes(tiles, n_views) * keys, k_ranges=4.0 * keys + 8.0 * tiles)
    return parts


def roofline(kernels, pairs, keys, n_gauss, n_views, tiles, n_sm, sm_mhz, clock_note, peaks, workload,
             traffic_table=None, n_tof=0):
    """Roofline of the integration kernels (FP32 issue and MUFU against the
    SM count read from the device and the sampled clock) and of the binning
    kernels (HBM against the measured copy bandwidth).  The top-level
    figures are those of the dominant integration kernel."""
    f = sm_mhz * 1e6
    fp32_peak = n_sm * FP32_LANES_PER_SM * f / 1e12
    mufu_peak = n_sm * MUFU_LANES_PER_SM * f / 1e12
    digest = sources_digest()
    out = {}
    mufu = MUFU_PER_PAIR + n_tof * MUFU_PER_BIN
    ops_f = OPS_PER_PAIR_FWD + n_tof * OPS_PER_BIN_FWD
    ops_a = OPS_PER_PAIR_ADJ + n_tof * OPS_PER_BIN_ADJ
    for name, ops in (("k_forward", ops_f), ("k_adjoint", ops_a)):
        kms = kernels[name]["ms"] / max(kernels[name]["launches"], 1)
        # pairs are counted per step: work per step / the kernel's time per step
        step_ms = kernels[name]["ms"] / max(STEPS_TIMED[0], 1)
        ach = pairs * ops / (step_ms / 1e3) / 1e12 if step_ms > 0 else 0.0
        sfu = pairs * mufu / (step_ms / 1e3) / 1e12 if step_ms > 0 else 0.0
        tr = None
        if traffic_table:
            ent = traffic_table.get((workload, name))
            if ent and ent[1] == digest:
                tr = ent[0]
        out[name] = dict(bound="alu", achieved=ach, peak=fp32_peak, unit="T FP32 op/s", frac=ach / fp32_peak,
                         sfu=dict(achieved=sfu, peak=mufu_peak, unit="T MUFU op/s", frac=sfu / mufu_peak),
                         kernel_ms_per_step=step_ms, launches_per_step=kernels[name]["launches"] / max(STEPS_TIMED[0], 1),
                         ms_per_launch=kms, traffic=tr)
    bb = binning_bytes(n_gauss, n_views, keys, tiles)
    bin_ms = sum(kernels[k]["ms"] for k in bb) / max(STEPS_TIMED[0], 1)
    tot = sum(bb.values())
    gbs = tot / (bin_ms / 1e3) / 1e9 if bin_ms > 0 else 0.0
    per = {}
    for k, v in bb.items():
        ms = kernels[k]["ms"] / max(STEPS_TIMED[0], 1)
        per[k] = dict(bytes=v, ms=ms, gbs=(v / (ms / 1e3) / 1e9 if ms > 0 else 0.0),
                      frac=(v / (ms / 1e3) / 1e9 / peaks["hbm_gbs"] if ms > 0 else 0.0))
    dom = max(("k_forward", "k_adjoint"), key=lambda k: out[k]["kernel_ms_per_step"])
    d = out[dom]
    return dict(bound="alu", achieved=d["achieved"], peak=d["peak"], unit=d["unit"], frac=d["frac"],
                traffic=d["traffic"], kernel=dom, forward=out["k_forward"], adjoint=out["k_adjoint"],
                sfu=dict(kernel=dom, **d["sfu"]),
                binning_hbm=dict(bound="hbm", achieved=gbs, peak=peaks["hbm_gbs"], unit="GB/s",
                                 frac=gbs / peaks["hbm_gbs"], bytes_per_step=tot, ms_per_step=bin_ms,
                                 kernels=per, peak_source=peaks["source"]),
                n_sm=n_sm, sm_mhz=sm_mhz, clock=clock_note, sources_digest=digest,
                note=(f"FP32 work = {ops_f:g} (forward) / {ops_a:g} (adjoint) operations "
                      f"and {mufu:g} MUFU per kept pair (m <= 9"
                      + (f"; {n_tof} TOF bins" if n_tof else "") + "), per step / kernel time per step; "
                      f"peaks = {n_sm} SMs x {FP32_LANES_PER_SM} FP32 (x {MUFU_LANES_PER_SM} MUFU) lanes x "
                      f"{sm_mhz:.0f} MHz; binning bytes as documented in binning_bytes()"))


STEPS_TIMED = [1]


def measure_step(args, name, rgrt, ctx, dev, seed, world, rank, local, cpu=True, tile=None):
    """One full optimisation step (records, binning, forward, loss, adjoint,
    parameter chain, Adam) of workload `name`: the JSON fields of its line."""
    import torch
    G, Gt, gd, loss = workload(name, seed, args.pet3d_angles)
    R = synth.num_rays(gd)
    t_auto = None
    tile = tile or args.tile
    if tile == "auto":
        # tile shape from the autotuner (forward + adjoint over all views: the
        # sort's pass count depends on the total number of tiles), outside the timing
        ga = rgrt.Gaussians(ctx, *[torch.from_numpy(G[k]).to(dev) for k in ("mu", "ls", "q", "rho")])
        tw, th, t_auto = rgrt.autotune_tile(ctx, ga, gd, max_views=0)
        ga.close()
    else:
        tw, th = (int(x) for x in tile.split("x"))
    gd = dict(gd, tile_w=tw, tile_h=th)
    geom = rgrt.Geometry(ctx, gd)
    # measured data: projections of the perturbed ("true") Gaussians
    tt = {k: torch.from_numpy(v).to(dev) for k, v in Gt.items()}
    gtrue = rgrt.Gaussians(ctx, tt["mu"], tt["ls"], tt["q"], tt["rho"])
    ytrue = torch.empty(R, device=dev)
    rgrt.project_forward(ctx, gtrue, geom, ytrue)
    gtrue.close()
    if loss == "poisson":
        kappa = 1e8 / float(ytrue.sum())
        gen = torch.Generator(device=dev).manual_seed(1234 + rank)
        y = torch.poisson(kappa * ytrue, generator=gen)
        eps = 1e-9 * float((kappa * ytrue).max())
        hp = rgrt.adam_params(kappa=kappa, poisson_eps=eps)
        lkind = rgrt.RGRT_LOSS_POISSON
    else:
        y = ytrue
        hp = rgrt.adam_params()
        lkind = rgrt.RGRT_LOSS_L2
    t0 = {k: torch.from_numpy(v).to(dev) for k, v in G.items()}
    gs = rgrt.Gaussians(ctx, t0["mu"], t0["ls"], t0["q"], t0["rho"])
    loss_dev = torch.zeros(1, device=dev)
    flush = None if args.no_flush else torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    step = 0
    for wi in range(args.warmup):
        step += 1
        ctx.stats_enable(wi == args.warmup - 1)    # pair counts from the last warm-up step
        rgrt.loss_step(ctx, gs, geom, y, lkind, hp, step, loss_dev)
    torch.cuda.synchronize()
    st = ctx.stats()
    ctx.stats_enable(False)
    # timed region
    ctx.prof_enable(True)
    ctx.prof_reset()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = rgrt.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        if flush is not None:
            flush.fill_(k & 0xff)      # evict L2 between timed steps (outside the events)
        ev[k][0].record(stream)
        step += 1
        rgrt.loss_step(ctx, gs, geom, y, lkind, hp, step, loss_dev)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    launches = rgrt.launch_count() - launches0
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_max = max_over_ranks(ms, world)
    kernels = {}
    for kname in ("k_records", "k_cull", "scan", "k_emit", "radix_sort", "k_ranges", "k_forward",
                  "k_loss", "k_adjoint", "k_param_chain", "k_adam"):
        n, t = ctx.prof_get(kname)
        kernels[kname] = dict(launches=n, ms=t)
    ctx.prof_enable(False)
    value = weak_value(R, args.steps, world, ms_max)
    pairs = st["pairs_kept"]
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks()
    if clk and clk.get("sm_mhz", 0) > 0:
        sm_mhz, note = clk["sm_mhz"], "median SM clock sampled during the timed region"
    else:
        sm_mhz = peaks["sm_max_mhz"] or 2070.0
        note = "no clock samples: the maximum SM clock"
    STEPS_TIMED[0] = args.steps
    n_views = synth.num_rays(gd) // (int(gd["n_rows"]) * int(gd["n_cols"]) * max(1, int(gd.get("n_tof", 0))))
    tiles = n_views * geom.tiles_per_view
    roof = roofline(kernels, pairs, st["keys"], int(G["mu"].shape[0]), n_views, tiles, n_sm, sm_mhz, note,
                    peaks, name, TRAFFIC, n_tof=int(gd.get("n_tof", 0)))
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms_max / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=WORKLOADS[name], rays_per_step=R,
                            gaussians=int(G["mu"].shape[0]),
                            **({"angles": int(gd["n_views"])} if name == "pet3d" else {}),
                            tile=f"{tw}x{th}" + (" (autotuner)" if t_auto is not None else ""),
                            seed=seed,
                            l2=("flushed between timed steps (256 MiB write outside the events)"
                                if flush is not None else "not flushed"),
                            parallelism=f"{world} independent scans (one per GPU)"),
                pairs_per_s=pairs * world / (ms_max / 1e3 / args.steps),
                pairs_kept_per_step=pairs, pairs_evaluated_per_step=st["pairs_evaluated"],
                keys_per_step=st["keys"], kernels=kernels, roofline=roof,
                gpu_launches=launches, wall_s=wall)
    if clk:
        line["clocks"] = clk
    # end to end: host parameters in, step, host loss + parameters out
    if not args.no_e2e:
        line["e2e"] = e2e(args, rgrt, ctx, geom, G, y, lkind, hp, R, world)
    if name == "c3-tof":
        line["vs_explicit_rays"] = tof_vs_explicit(rgrt, G, dev)
    if name in ("c2", "c3") and not args.no_fitted:
        line["fitted"] = fitted(args, rgrt, ctx, geom, gs, y, lkind, hp, step, R, world)
    if cpu and rank == 0 and not args.no_cpu_baseline:
        nv = args.cpu_views or auto_views(name)
        line["cpu_baseline"] = cpu_baseline(G, gd, loss, nv, rgrt, ctx)
    gs.close()
    geom.close()
    del flush
    return line


def tof_vs_explicit(rgrt, G, dev, n_angles=32, reps=3):
    """Forward and adjoint of the TOF sinogram against the same LORs and TOF
    kernels as explicit rays (geometry_set_rays_tof), on the first n_angles
    angles of the sinogram: ms per pass of each and the ratio."""
    import torch
    ctx = rgrt.Context(dev.index or 0)
    sub = synth.geom_pet(288, 329, 63, 400.0, 576, 2.0)
    sub["angles"] = (math.pi * np.arange(n_angles) / 288.0).astype(np.float64)
    sub["n_views"] = n_angles
    gd = synth.with_tof_bins(sub, *TOF_BINS)
    nl = synth.num_rays(sub)
    o, d, ta, tb = synth.pet_lors(sub)
    nb, h, sig = TOF_BINS
    centres = (np.arange(nb) - 0.5 * (nb - 1)) * h
    R = dict(kind="rays", o=np.tile(o, (nb, 1)).astype(np.float32), d=np.tile(d, (nb, 1)).astype(np.float32),
             t=np.tile(np.stack([ta, tb], 1), (nb, 1)).astype(np.float32),
             tof=np.stack([np.repeat(centres, nl) + np.tile(0.5 * (ta + tb), nb), np.full(nb * nl, sig)],
                          1).astype(np.float32))
    gs = rgrt.Gaussians(ctx, *[torch.from_numpy(G[k]).to(dev) for k in ("mu", "ls", "q", "rho")])
    out = {}
    for name, desc in (("sinogram", gd), ("explicit_rays", R)):
        geom = rgrt.Geometry(ctx, desc)
        I = torch.empty(geom.n_rays, device=dev)
        w = torch.ones(geom.n_rays, device=dev)
        grads = [torch.empty(sz, device=dev) for sz in ((gs.n, 3), (gs.n, 3), (gs.n, 4), (gs.n,))]
        rgrt.project_forward(ctx, gs, geom, I)
        rgrt.project_backward(ctx, gs, geom, w, *grads)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        for _ in range(reps):
            rgrt.project_forward(ctx, gs, geom, I)
        e[1].record()
        for _ in range(reps):
            rgrt.project_backward(ctx, gs, geom, w, *grads)
        e[2].record()
        torch.cuda.synchronize()
        out[name] = dict(forward_ms=e[0].elapsed_time(e[1]) / reps, backward_ms=e[1].elapsed_time(e[2]) / reps)
        geom.close()
    gs.close()
    ctx.close()
    s, x = out["sinogram"], out["explicit_rays"]
    return dict(angles=n_angles, outputs=nb * nl, sinogram=s, explicit_rays=x,
                speedup=(x["forward_ms"] + x["backward_ms"]) / (s["forward_ms"] + s["backward_ms"]),
                note="forward + adjoint of the same LORs and TOF kernels (first angles of the sinogram)")


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2602_01057_gb300 import build, rgrt
    build.build()
    dev = torch.device("cuda", local)
    ctx = rgrt.Context(local)
    line = measure_step(args, args.workload, rgrt, ctx, dev, args.seed + rank, world, rank, local)
    # the other workloads of the benchmark (one GPU, default run only): the
    # PET step, batching against plain steps, serving against a one-job server
    if world == 1 and args.workload == "c2" and not args.no_extras:
        extra = {}
        try:
            extra["c3"] = measure_step(args, "c3", rgrt, ctx, dev, args.seed, 1, 0, local)
        except Exception as e:   # noqa: BLE001 -- reported in the line, not hidden
            extra["c3"] = dict(error=repr(e))
        ctx.close()
        torch.cuda.empty_cache()
        try:
            extra["c4"] = c4_measure(args, steps=EXTRA_STEPS, warmup=EXTRA_WARMUP)
        except Exception as e:   # noqa: BLE001
            extra["c4"] = dict(error=repr(e))
        torch.cuda.empty_cache()
        try:
            extra["c5"] = c5_measure(args, full=True)
        except Exception as e:   # noqa: BLE001
            extra["c5"] = dict(error=repr(e))
        line["extra"] = extra
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


EXTRA_STEPS, EXTRA_WARMUP = 3, 2
# time of flight of the TOF PET workload: bins, spacing (mm), kernel width (mm)
TOF_BINS = (13, 47.0, 31.85)


def fitted(args, rgrt, ctx, geom, gs, y, lkind, hp, step, R, world):
    """The same step timed again after 100 more optimisation steps (the
    Gaussians have moved towards the measured object): rays/s and pairs."""
    import torch
    for _ in range(100):
        step += 1
        rgrt.loss_step(ctx, gs, geom, y, lkind, hp, step, None)
    ctx.stats_enable(True)
    step += 1
    rgrt.loss_step(ctx, gs, geom, y, lkind, hp, step, None)
    torch.cuda.synchronize()
    st = ctx.stats()
    ctx.stats_enable(False)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    flush = None if args.no_flush else torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    barrier(world)
    torch.cuda.synchronize()
    for k in range(args.steps):
        if flush is not None:
            flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        step += 1
        rgrt.loss_step(ctx, gs, geom, y, lkind, hp, step, None)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world)
    return dict(after_steps=100 + args.warmup + args.steps, value=weak_value(R, args.steps, world, ms),
                unit=UNIT, ms_per_step=ms / args.steps, pairs_kept_per_step=st["pairs_kept"],
                pairs_evaluated_per_step=st["pairs_evaluated"], keys_per_step=st["keys"])


def e2e(args, rgrt, ctx, geom, G, y, lkind, hp, R, world):
    """Same step through the C ABI with host buffers: parameters and
    measurements copied in from pinned host memory, loss and updated
    parameters read back, every step."""
    import torch
    n = G["mu"].shape[0]
    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in G.items()}
    yh = y.cpu().pin_memory()
    out = {k: torch.empty_like(v).pin_memory() for k, v in host.items()}
    lh = torch.zeros(1).pin_memory()
    gs = rgrt.Gaussians(ctx, host["mu"], host["ls"], host["q"], host["rho"])
    steps = max(3, args.steps // 2)
    step = 0
    for _ in range(2):
        step += 1
        gs.set(host["mu"], host["ls"], host["q"], host["rho"])
        rgrt.loss_step(ctx, gs, geom, yh, lkind, hp, step, lh)
        gs.get(out["mu"], out["ls"], out["q"], out["rho"])
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        step += 1
        gs.set(host["mu"], host["ls"], host["q"], host["rho"])
        rgrt.loss_step(ctx, gs, geom, yh, lkind, hp, step, lh)
        gs.get(out["mu"], out["ls"], out["q"], out["rho"])
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, world)
    gs.close()
    h2d = 4 * 11 * n + 4 * R
    d2h = 4 + 4 * 11 * n
    return dict(value=R * steps * world / dt, unit=UNIT, h2d_bytes_per_step=h2d,
                d2h_bytes_per_step=d2h, steps=steps)


def c4_scans(n_scans, seed=0, small=False):
    """The batching workload: uneven cone-beam scans (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    lo, hi, vmin, vmax, sides = ((1_000, 20_000, 16, 64, [64, 96, 128]) if small else
                                 (5_000, 500_000, 30, 360, [128, 256, 384, 512]))
    for i in range(n_scans):
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        v = int(rng.integers(vmin, vmax + 1))
        side = int(rng.choice(sides))
        G, gd = synth.workload_c2(10_000 + i, n=n, n_views=v, side=side)
        out.append((_params(G), gd))
    return out


def c4_measure(args, steps, warmup, small=False):
    """Batched step over uneven scans vs one plain step per scan (rays/s):
    the fields of the batching line."""
    import torch
    from paper_2602_01057_gb300 import build, rgrt
    build.build()
    dev = torch.device("cuda", 0)
    scans = c4_scans(args.scans, small=small)
    ctx = rgrt.Context(0)
    # tile shape from the autotuner, on the median-size scan
    order = sorted(range(len(scans)), key=lambda i: scans[i][0]["mu"].shape[0])
    G, gd = scans[order[len(order) // 2]]
    gt = rgrt.Gaussians(ctx, *[torch.from_numpy(G[k]).to(dev) for k in ("mu", "ls", "q", "rho")])
    tw, th, _ = rgrt.autotune_tile(ctx, gt, gd, max_views=12)
    gt.close()
    geoms, gb, gp, ys = [], [], [], []
    rays = 0
    for i, (G, gd) in enumerate(scans):
        gd = dict(gd, tile_w=tw, tile_h=th)
        geom = rgrt.Geometry(ctx, gd)
        tr = synth.perturbed(G, 20_000 + i, pos_std=0.01)
        g_true = rgrt.Gaussians(ctx, *[torch.from_numpy(tr[k]).to(dev) for k in ("mu", "ls", "q", "rho")])
        y = torch.empty(geom.n_rays, device=dev)
        rgrt.project_forward(ctx, g_true, geom, y)
        g_true.close()
        geoms.append(geom)
        ys.append(y)
        gb.append(rgrt.Gaussians(ctx, *[torch.from_numpy(G[k]).to(dev) for k in ("mu", "ls", "q", "rho")]))
        gp.append(rgrt.Gaussians(ctx, *[torch.from_numpy(G[k]).to(dev) for k in ("mu", "ls", "q", "rho")]))
        rays += geom.n_rays
    hp = rgrt.adam_params()
    batch = rgrt.Batch(ctx, gb, geoms)
    stream = torch.cuda.current_stream()
    step = 0
    for _ in range(warmup):
        step += 1
        batch.loss_step(ys, rgrt.RGRT_LOSS_L2, hp, step)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    l0 = rgrt.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step += 1
        batch.loss_step(ys, rgrt.RGRT_LOSS_L2, hp, step)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3 / steps
    launches = rgrt.launch_count() - l0
    # one plain loss_step per scan (each with its own binning read-back)
    lo = torch.zeros(1, device=dev)
    pstep = 0
    for _ in range(warmup):
        pstep += 1
        for g, geom, y in zip(gp, geoms, ys):
            rgrt.loss_step(ctx, g, geom, y, rgrt.RGRT_LOSS_L2, hp, pstep, lo)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        pstep += 1
        for g, geom, y in zip(gp, geoms, ys):
            rgrt.loss_step(ctx, g, geom, y, rgrt.RGRT_LOSS_L2, hp, pstep, lo)
    e1.record(stream)
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3 / steps
    clk = clocks.stop()
    info = batch.info()
    batch.close()
    for x in gb + gp + geoms:
        x.close()
    ctx.close()
    name = "c4-small" if small else "c4"
    line = dict(metric=METRIC, value=rays / t_batch, unit=UNIT, n_gpus=1, steps=steps,
                warmup=warmup, ms_per_step=1e3 * t_batch, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=WORKLOADS[name], scans=len(scans), rays_per_step=rays,
                            tile=f"{tw}x{th}", gaussians=int(sum(G["mu"].shape[0] for G, _ in scans)),
                            l2=("step working set far above L2 (not flushed)" if not small else
                                "not flushed: the whole step is timed, small scans partly L2-resident")),
                plain=dict(value=rays / t_plain, ms_per_step=1e3 * t_plain,
                           note=f"the same step as {len(scans)} loss_step calls, one scan at a time"),
                speedup_vs_plain=t_plain / t_batch, batch=info, gpu_launches=launches,
                timing="CUDA events on the launching stream around all timed steps", e2e=None)
    if clk:
        line["clocks"] = clk
    return line


def run_c4(args):
    print(json.dumps(c4_measure(args, args.steps, args.warmup, small=args.workload == "c4-small")), flush=True)


C5_CT_N = (20_000, 1_000_000)   # Gaussians (log-uniform)
C5_CT_VIEWS = (30, 720)         # views (uniform)
C5_CT_SIDE = (128, 512)         # detector side (uniform, multiple of 16)
C5_PET_N = (50_000, 400_000)
C5_ITERS, C5_VIEWS_PER_ITER = 200, 8
C5_PET_COUNTS = 1e8


def c5_jobs(n_jobs, rate, seed, rgrt, serve, ctx, dev):
    """The serving stream (seeded): kinds, sizes, measurements, arrival offsets.

    Measurements are the library's projection of a perturbed copy of each
    job's Gaussians (CT), or Poisson counts of it scaled to 1e8 in total (PET);
    both are made before any timing."""
    import torch
    rng = np.random.default_rng(seed)
    ct_ph = synth.ellipsoid_phantom(12, seed=1000 + seed, semi=(0.05, 0.6), dens=(0.1, 1.0))
    pet_ph = synth.pet_phantom(seed)
    jobs, gaps = [], rng.exponential(1.0 / rate, n_jobs)
    for i in range(n_jobs):
        kind = serve.GRAD if rng.uniform() < 0.7 else serve.RECON
        pet = rng.uniform() < 0.5
        if pet:
            n = int(round(math.exp(rng.uniform(*np.log(C5_PET_N)))))
            G = synth.phantom_gaussians_mixture(pet_ph, n, seed=50_000 + i)
            gd = synth.geom_c3()
        else:
            n = int(round(math.exp(rng.uniform(*np.log(C5_CT_N)))))
            v = int(rng.integers(C5_CT_VIEWS[0], C5_CT_VIEWS[1] + 1))
            side = 16 * int(rng.integers(C5_CT_SIDE[0] // 16, C5_CT_SIDE[1] // 16 + 1))
            G = synth.phantom_gaussians_mixture(ct_ph, n, seed=50_000 + i)
            gd = synth.geom_c2(n_views=v, side=side)
        G = _params(G)
        true = synth.perturbed(G, 60_000 + i, pos_std=1.0 if pet else 0.01)
        geom = rgrt.Geometry(ctx, gd)
        gt = rgrt.Gaussians(ctx, *[torch.from_numpy(true[k]).to(dev) for k in ("mu", "ls", "q", "rho")])
        I = torch.empty(geom.n_rays, device=dev)
        rgrt.project_forward(ctx, gt, geom, I)
        I = I.cpu().numpy().astype(np.float64)
        gt.close()
        geom.close()
        if pet:
            kappa = C5_PET_COUNTS / max(I.sum(), 1e-30)
            y = rng.poisson(kappa * I).astype(np.float32)
            hp, loss = dict(kappa=float(kappa), poisson_eps=1e-3), rgrt.RGRT_LOSS_POISSON
        else:
            y = I.astype(np.float32)
            hp, loss = None, rgrt.RGRT_LOSS_L2
        jobs.append(dict(kind=kind, G=G, geom=gd, y=y, loss=loss, hp=hp, n_iter=C5_ITERS,
                         views_per_iter=C5_VIEWS_PER_ITER, seed=70_000 + i,
                         tag=("pet" if pet else "ct", kind, n)))
    return jobs, np.cumsum(gaps) - gaps[0]


def c5_run(serve, rgrt, specs, offsets, n_slots, budget, rate_scale=1.0):
    """Replay the stream on a server with n_slots slots; arrival i at
    offsets[i] / rate_scale seconds after the start."""
    import torch
    srv = serve.Server(n_slots=n_slots, hbm_budget_bytes=budget, device=0)
    jobs = [serve.Job(**sp) for sp in specs]
    l0 = rgrt.launch_count()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    futs = []
    for j, off in zip(jobs, offsets / rate_scale):
        wait = t0 + off - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        j.t_arrive = t0 + off
        futs.append(srv.submit(j))
    for f in futs:
        f.result()
    t1 = time.perf_counter()
    srv.close()
    launches = rgrt.launch_count() - l0
    lat = np.array([j.t_done - j.t_arrive for j in jobs])
    rays = sum(j.rays for j in jobs)
    # host<->device bytes of the jobs: parameters and measurements in;
    # gradients (+ loss) or fitted parameters (+ loss history) out
    h2d = sum(44 * j.G["mu"].shape[0] + (0 if j.y is None else 4 * j.y.size) for j in jobs)
    d2h = sum(44 * j.G["mu"].shape[0] + 4 * (j.n_iter if j.kind == serve.RECON else 1) for j in jobs)
    by_kind = {}
    for k in (serve.GRAD, serve.RECON):
        sel = np.array([j.kind == k for j in jobs])
        if sel.any():
            by_kind[k] = dict(jobs=int(sel.sum()), p50_s=float(np.percentile(lat[sel], 50)),
                              p99_s=float(np.percentile(lat[sel], 99)))
    ov = srv.device_overlap()
    return dict(slots=n_slots, jobs=len(jobs), wall_s=t1 - t0, jobs_per_s=len(jobs) / (t1 - t0),
                device_overlap=dict(ov, note="jobs' device intervals (CUDA events on their streams): sum, "
                                             "union, time covered by two or more, most at once"),
                rays_per_s=rays / (t1 - t0), p50_s=float(np.percentile(lat, 50)),
                p99_s=float(np.percentile(lat, 99)), mean_s=float(lat.mean()), by_kind=by_kind,
                peak_running=srv.peak_running, peak_budget_gb=srv.peak_used / 1e9,
                gpu_launches=int(launches), h2d_bytes_per_job=h2d / len(jobs),
                d2h_bytes_per_job=d2h / len(jobs))


def c5_measure(args, full=False):
    """Serving: the same job stream through a continuous-batching server and
    a one-job-at-a-time server, at the stated arrival rate and at a rate the
    one-job server can sustain; the fields of the serving line."""
    import torch
    from paper_2602_01057_gb300 import build, rgrt, serve
    build.build()
    dev = torch.device("cuda", 0)
    ctx = rgrt.Context(0)
    budget = 150 * 10**9
    n_jobs = EXTRA_JOBS if full else args.jobs
    specs, offsets = c5_jobs(n_jobs, args.rate, 0, rgrt, serve, ctx, dev)
    ctx.close()
    torch.cuda.empty_cache()
    # warm-up: a few jobs through the continuous server (module load, allocator)
    warm = [dict(sp, n_iter=5) for sp in specs[:max(args.warmup, 1)]]
    c5_run(serve, rgrt, warm, np.zeros(len(warm)), args.slots, budget)
    clocks = ClockSampler(0)
    clocks.start()
    cont = c5_run(serve, rgrt, specs, offsets, args.slots, budget)
    fifo = c5_run(serve, rgrt, specs, offsets, 1, budget)
    # a load the one-job server sustains: 80% of its measured throughput
    lam80 = 0.8 * fifo["jobs_per_s"]
    scale = lam80 / args.rate
    cont80 = c5_run(serve, rgrt, specs, offsets, args.slots, budget, rate_scale=scale)
    fifo80 = c5_run(serve, rgrt, specs, offsets, 1, budget, rate_scale=scale)
    ck = clocks.stop()
    n_ct = sum(1 for sp in specs if sp["tag"][0] == "ct")
    n_recon = sum(1 for sp in specs if sp["kind"] == serve.RECON)
    ct_sizes = [(sp["tag"][2], sp["geom"]["n_views"], sp["geom"]["n_rows"]) for sp in specs if sp["tag"][0] == "ct"]
    line = dict(metric=METRIC, value=cont["rays_per_s"], unit=UNIT, n_gpus=1, steps=len(specs),
                warmup=len(warm), ms_per_step=1e3 * cont["wall_s"] / len(specs), higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=WORKLOADS["c5"], jobs=len(specs), ct_jobs=n_ct, recon_jobs=n_recon,
                            rate_per_s=args.rate, slots=args.slots, hbm_budget_gb=150,
                            sizes=(f"CT Gaussians log-uniform {C5_CT_N[0]}-{C5_CT_N[1]}, views "
                                   f"U{{{C5_CT_VIEWS[0]}..{C5_CT_VIEWS[1]}}}, side U{{{C5_CT_SIDE[0]}.."
                                   f"{C5_CT_SIDE[1]}}} (multiples of 16); PET the 288x329x63 geometry with "
                                   f"{C5_PET_N[0]}-{C5_PET_N[1]} Gaussians; reconstructions {C5_ITERS} "
                                   f"iterations of {C5_VIEWS_PER_ITER} views"),
                            ct_largest=dict(gaussians=max(x[0] for x in ct_sizes) if ct_sizes else None,
                                            views=max(x[1] for x in ct_sizes) if ct_sizes else None,
                                            side=max(x[2] for x in ct_sizes) if ct_sizes else None),
                            l2="not flushed: jobs far above L2"),
                serving=dict(continuous=cont, fifo=fifo,
                             at_80pct_fifo_capacity=dict(rate_per_s=lam80, continuous=cont80, fifo=fifo80),
                             throughput_vs_fifo=cont["jobs_per_s"] / fifo["jobs_per_s"],
                             p99_vs_fifo_at_80pct=cont80["p99_s"] / fifo80["p99_s"]),
                gpu_launches=cont["gpu_launches"], clocks=ck,
                e2e=dict(value=cont["rays_per_s"], unit=UNIT,
                         h2d_bytes_per_step=cont["h2d_bytes_per_job"],
                         d2h_bytes_per_step=cont["d2h_bytes_per_job"],
                         note="a step is one job; jobs enter and leave as host arrays, every copy "
                              "inside the timed run"))
    return line


def run_c5(args):
    print(json.dumps(c5_measure(args)), flush=True)


EXTRA_JOBS = 32


OPS_PER_PAIR_VOX = 15   # per kept (voxel, Gaussian) pair: delta 3, P delta 9, the form 3 (plus the exponential)


def run_vox(args):
    """Voxelisation of the cone-beam workload's Gaussians: voxels/s."""
    import torch
    from paper_2602_01057_gb300 import build, rgrt
    build.build()
    G, _ = synth.workload_c2(0)
    G = _params(G)
    n = 256
    h = 2.0 / n
    vol = dict(origin=(-1 + h / 2,) * 3, size=(h, h, h), dims=(n, n, n))
    ctx = rgrt.Context(0)
    gs = rgrt.Gaussians(ctx, *[torch.from_numpy(G[k]).cuda() for k in ("mu", "ls", "q", "rho")])
    out = torch.empty((n, n, n), device="cuda")
    flush = None if args.no_flush else torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        rgrt.gaussians_voxelize(ctx, gs, vol, out)
    torch.cuda.synchronize()
    ctx.prof_enable(True)
    ctx.prof_reset()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    l0 = rgrt.launch_count()
    for k in range(args.steps):
        if flush is not None:
            flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        rgrt.gaussians_voxelize(ctx, gs, vol, out)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = rgrt.launch_count() - l0
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    nk, kms = ctx.prof_get("k_voxelize")
    nb, bms = ctx.prof_get("vox_bin")
    ctx.prof_enable(False)
    # kept pairs, counted analytically: voxels inside each Gaussian's 3-sigma
    # ellipsoid = (4/3) pi 27 sqrt(det Sigma) / h^3 (the grid is fine against sigma)
    s = np.exp(G["ls"].astype(np.float64))
    pairs = float(np.sum(4.0 / 3.0 * math.pi * 27.0 * np.prod(s, axis=1)) / h ** 3)
    per = kms / max(nk, 1)
    achieved = pairs * OPS_PER_PAIR_VOX / (per / 1e3) / 1e12
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    sm_mhz = clk["sm_mhz"] if clk and clk.get("sm_mhz", 0) > 0 else (measured_peaks()["sm_max_mhz"] or 2070.0)
    peak = n_sm * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    # end to end: the volume read back to pinned host memory every call
    host = torch.empty((n, n, n)).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(3, args.steps // 2)):
        rgrt.gaussians_voxelize(ctx, gs, vol, out)
        host.copy_(out)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / max(3, args.steps // 2)
    line = dict(metric="voxels/s", value=n ** 3 / (ms / 1e3), unit="voxels/s", n_gpus=1, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32", data="synthetic",
                config=dict(workload=WORKLOADS["vox"], voxels=n ** 3, gaussians=int(G["mu"].shape[0]),
                            l2=("flushed between timed calls (256 MiB write outside the events)"
                                if flush is not None else "not flushed")),
                kernels=dict(vox_bin=dict(launches=nb, ms=bms), k_voxelize=dict(launches=nk, ms=kms)),
                pairs_kept_per_step=pairs,
                roofline=dict(bound="alu", achieved=achieved, peak=peak, unit="T FP32 op/s", frac=achieved / peak,
                              traffic=None, kernel="k_voxelize", kernel_ms=per, n_sm=n_sm, sm_mhz=sm_mhz,
                              note="15 FP32 operations per kept (voxel, Gaussian) pair, pairs counted "
                                   "analytically; peak = SMs x 128 lanes x sampled SM clock"),
                gpu_launches=launches,
                e2e=dict(value=n ** 3 / e2e_s, unit="voxels/s", h2d_bytes_per_step=0,
                         d2h_bytes_per_step=4 * n ** 3))
    if clk:
        line["clocks"] = clk
    print(json.dumps(line), flush=True)


def run_recon(args):
    """Reconstruction quality and speed: Adam on the exact phantom projections,
    PSNR of the voxelised Gaussians every 50 steps."""
    import torch
    from paper_2602_01057_gb300 import build, rgrt
    build.build()
    ph = synth.ellipsoid_phantom(12, seed=1000, semi=(0.05, 0.6), dens=(0.1, 1.0))   # the C2 phantom
    G, gd = synth.workload_c2(0)
    G = _params(G)
    y = torch.from_numpy(synth.phantom_projection(ph, *synth.detector_rays(gd)).astype(np.float32)).cuda()
    vol = synth.voxel_grid(128)
    ref = synth.phantom_volume(ph, vol)
    ctx = rgrt.Context(0)
    geom = rgrt.Geometry(ctx, gd)
    gs = rgrt.Gaussians(ctx, *[torch.from_numpy(G[k]).cuda() for k in ("mu", "ls", "q", "rho")])
    hp = rgrt.adam_params()
    lo = torch.zeros(1, device="cuda")
    curve = []
    stream = torch.cuda.current_stream()
    ms_total = 0.0
    for it in range(args.iters + 1):
        if it % 50 == 0 or it == args.iters:
            V = rgrt.gaussians_voxelize(ctx, gs, vol)
            curve.append(dict(step=it, loss=float(lo.item()) if it else None, psnr_db=synth.psnr(V, ref)))
        if it == args.iters:
            break
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rgrt.loss_step(ctx, gs, geom, y, rgrt.RGRT_LOSS_L2, hp, it + 1, lo)
        b.record(stream)
        b.synchronize()
        ms_total += a.elapsed_time(b)
    R = synth.num_rays(gd)
    line = dict(metric=METRIC, value=R * args.iters / (ms_total / 1e3), unit=UNIT, n_gpus=1, steps=args.iters,
                warmup=0, ms_per_step=ms_total / args.iters, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=WORKLOADS["recon"], rays_per_step=R, gaussians=int(G["mu"].shape[0]),
                            voxels=int(np.prod(vol["dims"])), l2="not flushed"),
                recon=dict(psnr_db_start=curve[0]["psnr_db"], psnr_db_end=curve[-1]["psnr_db"], curve=curve,
                           note="PSNR against the phantom density at voxel centres, peak = max density"),
                e2e=None)
    print(json.dumps(line), flush=True)


POINT_SOURCES = ((0.0, 10.0, 0.0), (0.0, 100.0, 0.0), (0.0, 200.0, 0.0))


def point_source_study(rgrt, ctx, iters=1500, counts=5e6, seed=0, n_angles=288, grid=4.0):
    """Reconstruct three point sources from raw-mode data three ways -- the
    raw sinogram with the raw geometry ("raw"), its arc-corrected resampling
    with the arc-corrected geometry ("arc"), and the raw sinogram taken for
    arc-corrected ("raw_as_arc", the model a uniform-bin projector assumes)
    -- and measure the FWHM of each reconstructed source along x (the
    tangential direction, the paper's horizontal line profile) and y
    (radial) through its peak voxel, its offset from the true centre and the
    peak values."""
    import torch
    g_raw = synth.geom_pet(n_angles, 329, 5, 400.0, 576, 2.0, arc_mode=1)
    g_arc = dict(g_raw, arc_mode=0)
    clean = synth.point_source_sinogram(g_raw, POINT_SOURCES, radius=1.0)
    kappa = counts / clean.sum()
    noisy = np.random.default_rng(seed).poisson(kappa * clean) / kappa
    modes = dict(raw=(g_raw, noisy), arc=(g_arc, synth.arc_resample(noisy, g_raw)), raw_as_arc=(g_arc, noisy))
    h = 0.1
    out = {}
    for name, (gd, y) in modes.items():
        G = synth.grid_gaussians(230.0, grid, sigma=2.0, rho=0.005)
        geom = rgrt.Geometry(ctx, gd)
        gs = rgrt.Gaussians(ctx, *[torch.from_numpy(G[k]).cuda() for k in ("mu", "ls", "q", "rho")])
        yd = torch.from_numpy(np.ascontiguousarray(y, np.float32).reshape(-1)).cuda()
        hp = rgrt.adam_params(lr_mu=0.02, lr_logscale=5e-3, lr_quat=1e-3, lr_rho=2e-3)
        lo = torch.zeros(1, device="cuda")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for it in range(iters):
            rgrt.loss_step(ctx, gs, geom, yd, rgrt.RGRT_LOSS_L2, hp, it + 1, lo)
        ev1.record()
        torch.cuda.synchronize()
        res = dict(loss=float(lo.item()), ms_per_step=ev0.elapsed_time(ev1) / iters, sources=[])
        for c in POINT_SOURCES:
            n = 301
            vol = dict(origin=(c[0] - h * (n - 1) / 2, c[1] - h * (n - 1) / 2, 0.0), size=(h, h, h),
                       dims=(n, n, 1))
            V = rgrt.gaussians_voxelize(ctx, gs, vol)[0]          # [y][x]
            j, i = np.unravel_index(int(np.argmax(V)), V.shape)
            res["sources"].append(dict(
                centre_mm=list(c), peak=float(V[j, i]),
                peak_offset_mm=[float((i - (n - 1) / 2) * h), float((j - (n - 1) / 2) * h)],
                fwhm_x_mm=synth.fwhm(V[j, :], h), fwhm_y_mm=synth.fwhm(V[:, i], h)))
        peaks = [x["peak"] for x in res["sources"]]
        res["peak_max_over_min"] = max(peaks) / min(peaks) if min(peaks) > 0 else None
        out[name] = res
        gs.close()
        geom.close()
    return out


def run_points(args):
    import torch
    from paper_2602_01057_gb300 import build, rgrt
    build.build()
    ctx = rgrt.Context(0)
    t0 = time.perf_counter()
    res = point_source_study(rgrt, ctx, iters=args.point_iters, seed=args.seed)
    wall = time.perf_counter() - t0
    rays = 288 * 329 * 5
    ms = res["raw"]["ms_per_step"]
    line = dict(metric=METRIC, value=rays / (ms / 1e3), unit=UNIT, n_gpus=1, steps=None, warmup=0,
                ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
                data="synthetic", config=dict(workload=WORKLOADS["points"], rays_per_step=rays),
                points=res, wall_s=wall, e2e=None,
                note="FWHM in mm (radial bin 2.18 mm at the centre); the synthetic data has no crystal "
                     "penetration or positron range, so resolution loss with radius comes from sampling only")
    print(json.dumps(line), flush=True)


def run_pet3d(args):
    """The LORs of the 3-D PET workload through the explicit-ray path: rays/s
    of a full step."""
    G, _ = synth.workload_c3(0)
    run_explicit(args, "pet3d-rays", G, synth.pet_rays_3d(max_ring_diff=5), "poisson", pos_std=1.0,
                 note="explicit-ray path (no detector structure): the binning tests every Gaussian against "
                      "every 128-ray block")


def run_helical(args):
    """Helical cone-beam CT through the explicit-ray path: the cone-beam
    workload's Gaussians, one turn of 180 views of 256 x 256, rays/s of a
    full step."""
    G, gd = synth.workload_c2(0)
    R = synth.rays_helical(180, 256, 256, gd["pitch_u"], gd["dso"], gd["dsd"], z_per_turn=1.0)
    run_explicit(args, "helical", G, R, "l2", pos_std=0.01,
                 note="explicit-ray path: 128 consecutive rays (half a detector row) per block")


def run_explicit(args, name, G, R, loss, pos_std, note):
    import torch
    from paper_2602_01057_gb300 import build, rgrt
    build.build()
    G = _params(G)
    n_rays = R["o"].shape[0]
    ctx = rgrt.Context(0)
    geom = rgrt.Geometry(ctx, R)
    true = synth.perturbed(G, 101, pos_std=pos_std)
    gt = rgrt.Gaussians(ctx, *[torch.from_numpy(true[k]).cuda() for k in ("mu", "ls", "q", "rho")])
    ytrue = torch.empty(n_rays, device="cuda")
    rgrt.project_forward(ctx, gt, geom, ytrue)
    gt.close()
    if loss == "poisson":
        kappa = 1e8 / float(ytrue.sum())
        y = torch.poisson(kappa * ytrue, generator=torch.Generator(device="cuda").manual_seed(7))
        hp = rgrt.adam_params(kappa=kappa, poisson_eps=1e-9 * float((kappa * ytrue).max()))
        lkind = rgrt.RGRT_LOSS_POISSON
    else:
        y, hp, lkind = ytrue, rgrt.adam_params(), rgrt.RGRT_LOSS_L2
    gs = rgrt.Gaussians(ctx, *[torch.from_numpy(G[k]).cuda() for k in ("mu", "ls", "q", "rho")])
    lo = torch.zeros(1, device="cuda")
    step = 0
    for _ in range(args.warmup):
        step += 1
        rgrt.loss_step(ctx, gs, geom, y, lkind, hp, step, lo)
    torch.cuda.synchronize()
    ctx.prof_enable(True)
    ctx.prof_reset()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    l0 = rgrt.launch_count()
    for k in range(args.steps):
        ev[k][0].record(stream)
        step += 1
        rgrt.loss_step(ctx, gs, geom, y, lkind, hp, step, lo)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = rgrt.launch_count() - l0
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    kernels = {}
    for kname in ("k_records", "rays_bin", "rays_emit", "k_rays_forward", "k_loss", "k_rays_adjoint",
                  "k_param_chain", "k_adam"):
        nk, t = ctx.prof_get(kname)
        kernels[kname] = dict(launches=nk, ms=t)
    line = dict(metric=METRIC, value=n_rays / (ms / 1e3), unit=UNIT, n_gpus=1, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32", data="synthetic",
                config=dict(workload=WORKLOADS[name], rays_per_step=n_rays, gaussians=int(G["mu"].shape[0]),
                            l2="not flushed: the step's working set is far above L2"),
                kernels=kernels, keys_per_step=None, gpu_launches=launches, roofline=None, note=note, e2e=None)
    if clk:
        line["clocks"] = clk
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("c4", "c4-small"):
        run_c4(args)
    elif args.workload == "c5":
        run_c5(args)
    elif args.workload == "vox":
        run_vox(args)
    elif args.workload == "recon":
        run_recon(args)
    elif args.workload == "pet3d-rays":
        run_pet3d(args)
    elif args.workload == "helical":
        run_helical(args)
    elif args.workload == "points":
        run_points(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
