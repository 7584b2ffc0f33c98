"""Thin Python binding of librgrt's C ABI (include/rgrt.h).

Argument marshalling only: every step of the projector runs in the CUDA
library.  The functions carry the C names (``gaussians_create``,
``geometry_set``, ``project_forward``, ``project_backward``, ``loss_step``);
arrays may be torch tensors (CUDA or CPU) or numpy arrays, passed by pointer.
PyTorch provides device memory and streams.  If the library is not built the
import of a call fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

RGRT_OK = 0
RGRT_COPY, RGRT_BORROW = 0, 1
RGRT_LOSS_L2, RGRT_LOSS_POISSON = 0, 1
RGRT_KERNEL_GAUSSIAN, RGRT_KERNEL_EPANECHNIKOV = 0, 1
KERNELS = {"gaussian": RGRT_KERNEL_GAUSSIAN, "epanechnikov": RGRT_KERNEL_EPANECHNIKOV}
_KIND = {"parallel": 0, "cone": 1, "pet": 2, "pet3d": 3}


class RgrtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rgrt error {code}: {msg}")
        self.code = code


class GeomDesc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("n_views", ctypes.c_int32),
        ("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32),
        ("angles", ctypes.POINTER(ctypes.c_double)),
        ("pitch_u", ctypes.c_double), ("pitch_v", ctypes.c_double),
        ("t_a", ctypes.c_double), ("t_b", ctypes.c_double),
        ("dso", ctypes.c_double), ("dsd", ctypes.c_double), ("radius", ctypes.c_double),
        ("n_crystals", ctypes.c_int32), ("arc_mode", ctypes.c_int32),
        ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
        ("max_ring_diff", ctypes.c_int32),
    ]


class VolumeDesc(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("size", ctypes.c_double * 3), ("dims", ctypes.c_int32 * 3)]


class Adam(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in (
        "lr_mu", "lr_logscale", "lr_quat", "lr_rho", "beta1", "beta2", "eps", "kappa",
        "poisson_eps")]


_lib = None
_VP = ctypes.c_void_p
_EXPORTS = {
    "rgrt_ctx_create": ([ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_size_t], ctypes.c_int),
    "rgrt_ctx_destroy": ([_VP], ctypes.c_int),
    "gaussians_create": ([_VP, ctypes.c_int64, _VP, _VP, _VP, _VP, ctypes.c_int,
                          ctypes.POINTER(_VP)], ctypes.c_int),
    "gaussians_destroy": ([_VP], ctypes.c_int),
    "gaussians_set_kernel": ([_VP, ctypes.c_int], ctypes.c_int),
    "gaussians_get": ([_VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "gaussians_set": ([_VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "gaussians_count": ([_VP], ctypes.c_int64),
    "geometry_set": ([_VP, ctypes.POINTER(GeomDesc), ctypes.POINTER(_VP)], ctypes.c_int),
    "geometry_set_corrections": ([_VP, _VP, _VP], ctypes.c_int),
    "geometry_set_tof": ([_VP, ctypes.c_int, ctypes.c_float, ctypes.c_float], ctypes.c_int),
    "geometry_set_rays_tof": ([_VP, ctypes.c_int64, _VP, _VP, _VP, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "geometry_set_rays": ([_VP, ctypes.c_int64, _VP, _VP, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "geometry_destroy": ([_VP], ctypes.c_int),
    "geometry_num_rays": ([_VP], ctypes.c_int64),
    "project_forward": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "project_backward": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "loss_step": ([_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(Adam), ctypes.c_int, _VP, _VP],
                  ctypes.c_int),
    "loss_grad": ([_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(Adam), _VP, _VP, _VP, _VP, _VP, _VP],
                  ctypes.c_int),
    "gaussians_voxelize": ([_VP, _VP, ctypes.POINTER(VolumeDesc), _VP, _VP], ctypes.c_int),
    "rgrt_batch_create": ([_VP, ctypes.c_int, _VP, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "rgrt_batch_destroy": ([_VP], ctypes.c_int),
    "rgrt_batch_forward": ([_VP, _VP, _VP], ctypes.c_int),
    "rgrt_batch_loss_step": ([_VP, _VP, ctypes.c_int, ctypes.POINTER(Adam), ctypes.c_int, _VP, _VP],
                             ctypes.c_int),
    "rgrt_batch_debug_tile_lists": ([_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), _VP, _VP,
                                     ctypes.c_int64], ctypes.c_int),
    "rgrt_batch_info": ([_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                         ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "rgrt_autotune_tile": ([_VP, _VP, ctypes.POINTER(GeomDesc), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "project_forward_noalloc": ([ctypes.POINTER(GeomDesc), ctypes.c_int64, _VP, _VP, _VP, _VP,
                                 _VP, _VP], ctypes.c_int),
    "rgrt_last_error": ([], ctypes.c_char_p),
    "rgrt_launch_count": ([], ctypes.c_int64),
    "rgrt_debug_records": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "rgrt_debug_tile_lists": ([_VP, _VP, _VP, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_int64), _VP, _VP, ctypes.c_int64, _VP],
                              ctypes.c_int),
    "rgrt_prof_enable": ([_VP, ctypes.c_int], ctypes.c_int),
    "rgrt_prof_reset": ([_VP], ctypes.c_int),
    "rgrt_prof_get": ([_VP, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64),
                       ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "rgrt_stats_enable": ([_VP, ctypes.c_int], ctypes.c_int),
    "rgrt_stats_get": ([_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load librgrt.so; raise if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"librgrt is not built ({_build.LIB}); run "
                               "paper_2602_01057_gb300.build.build() first")
        L = ctypes.CDLL(_build.LIB)
        for name, (args, res) in _EXPORTS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(_EXPORTS)


def _check(rc):
    if rc != RGRT_OK:
        raise RgrtError(rc, lib().rgrt_last_error().decode())
    return rc


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().rgrt_launch_count())


def last_error() -> str:
    return lib().rgrt_last_error().decode()


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _f32c(a):
    """float32 C-contiguous view of a numpy array (copied if needed) or a tensor."""
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float32)
    return a


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# objects
# ---------------------------------------------------------------------------

class Context:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        h = _VP()
        _check(lib().rgrt_ctx_create(ctypes.byref(h), device, hbm_budget_bytes))
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            lib().rgrt_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def prof_enable(self, on=True):
        _check(lib().rgrt_prof_enable(self.h, int(on)))

    def prof_reset(self):
        _check(lib().rgrt_prof_reset(self.h))

    def prof_get(self, name: str):
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        _check(lib().rgrt_prof_get(self.h, name.encode(), ctypes.byref(n), ctypes.byref(ms)))
        return int(n.value), float(ms.value)

    def stats_enable(self, on=True):
        _check(lib().rgrt_stats_enable(self.h, int(on)))

    def stats(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().rgrt_stats_get(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return dict(pairs_evaluated=a.value, pairs_kept=b.value, keys=c.value)


class Gaussians:
    """Handle of n Gaussians (mu[n,3], logscale[n,3], quat[n,4] (w,x,y,z), rho[n])."""

    def __init__(self, ctx: Context, mu, ls, q, rho, borrow: bool = False):
        n = int(mu.shape[0])
        h = _VP()
        self._keep = (mu, ls, q, rho) if borrow else None
        _check(lib().gaussians_create(ctx.h, n, _ptr(mu), _ptr(ls), _ptr(q), _ptr(rho),
                                      RGRT_BORROW if borrow else RGRT_COPY, ctypes.byref(h)))
        self.h = h
        self.n = n
        self.ctx = ctx

    def close(self):
        # after its context has been closed the handle is only dropped (its
        # device memory stays allocated until the process ends): destroying it
        # would reach into the freed context
        if self.h and self.ctx.h:
            lib().gaussians_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_kernel(self, kernel):
        """"gaussian" or "epanechnikov" (or an RGRT_KERNEL_* code)."""
        k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        _check(lib().gaussians_set_kernel(self.h, k))
        return self

    def get(self, mu=None, ls=None, q=None, rho=None, stream=None):
        _check(lib().gaussians_get(self.h, _ptr(mu), _ptr(ls), _ptr(q), _ptr(rho), _stream(stream)))

    def set(self, mu=None, ls=None, q=None, rho=None, stream=None):
        _check(lib().gaussians_set(self.h, _ptr(mu), _ptr(ls), _ptr(q), _ptr(rho), _stream(stream)))

    def numpy(self):
        n = self.n
        out = dict(mu=np.zeros((n, 3), np.float32), ls=np.zeros((n, 3), np.float32),
                   q=np.zeros((n, 4), np.float32), rho=np.zeros(n, np.float32))
        self.get(out["mu"], out["ls"], out["q"], out["rho"])
        return out


def make_desc(d: dict):
    """ctypes description from a synth geometry dict (keeps the angle array alive)."""
    angles = np.ascontiguousarray(d.get("angles", np.zeros(0)), dtype=np.float64)
    # no angles: null (a PET sinogram then spaces its n_views angles evenly over pi)
    aptr = (angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if angles.size
            else ctypes.POINTER(ctypes.c_double)())
    desc = GeomDesc(
        _KIND[d["kind"]], int(d["n_views"]), int(d["n_rows"]), int(d["n_cols"]),
        aptr,
        float(d.get("pitch_u", 0.0)), float(d.get("pitch_v", 0.0)),
        float(d.get("t_a", 0.0)), float(d.get("t_b", 0.0)),
        float(d.get("dso", 0.0)), float(d.get("dsd", 0.0)), float(d.get("radius", 0.0)),
        int(d.get("n_crystals", 0)), int(d.get("arc_mode", 0)),
        int(d.get("tile_w", 16)), int(d.get("tile_h", 16)), int(d.get("max_ring_diff", 0)))
    return desc, angles


class Geometry:
    """A geometry from a description dict: a detector geometry (geometry_set)
    or, for kind "rays", explicit rays o[R,3], d[R,3], t[R,2] and optionally
    tof[R,2] = (centre, width) (geometry_set_rays[_tof]; numpy arrays or
    contiguous float32 tensors)."""

    def __init__(self, ctx: Context, d: dict):
        h = _VP()
        if d["kind"] == "rays":
            o = _f32c(d["o"])
            dd = _f32c(d["d"])
            t = _f32c(d["t"])
            n = int(o.shape[0])
            if d.get("tof") is not None:
                tof = _f32c(d["tof"])
                _check(lib().geometry_set_rays_tof(ctx.h, n, _ptr(o), _ptr(dd), _ptr(t), _ptr(tof),
                                                   ctypes.byref(h)))
            else:
                _check(lib().geometry_set_rays(ctx.h, n, _ptr(o), _ptr(dd), _ptr(t), ctypes.byref(h)))
            self.tiles_per_view = 0
        else:
            desc, angles = make_desc(d)
            _check(lib().geometry_set(ctx.h, ctypes.byref(desc), ctypes.byref(h)))
            if int(d.get("n_tof", 0)) > 0:
                rc = lib().geometry_set_tof(h, int(d["n_tof"]), float(d["tof_spacing"]), float(d["tof_sigma"]))
                if rc != RGRT_OK:
                    msg = lib().rgrt_last_error().decode()
                    lib().geometry_destroy(h)
                    raise RgrtError(rc, msg)
            tw, th = int(d.get("tile_w", 16)), int(d.get("tile_h", 16))
            self.tiles_per_view = ((int(d["n_cols"]) + tw - 1) // tw) * ((int(d["n_rows"]) + th - 1) // th)
        self.h = h
        self.ctx = ctx
        self.desc = d
        self.n_rays = int(lib().geometry_num_rays(h))

    def set_corrections(self, mult=None, add=None):
        """Per-ray measurement model of the losses: mult I + add (see the C header)."""
        mult = _f32c(mult) if mult is not None else None
        add = _f32c(add) if add is not None else None
        _check(lib().geometry_set_corrections(self.h, _ptr(mult), _ptr(add)))
        return self

    def close(self):
        # after its context has been closed the handle is only dropped (its
        # device memory stays allocated until the process ends): destroying it
        # would reach into the freed context
        if self.h and self.ctx.h:
            lib().geometry_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# the five calls, C names
# ---------------------------------------------------------------------------

def gaussians_create(ctx, mu, ls, q, rho, borrow=False) -> Gaussians:
    return Gaussians(ctx, mu, ls, q, rho, borrow)


def geometry_set(ctx, desc: dict) -> Geometry:
    return Geometry(ctx, desc)


def project_forward(ctx, gauss, geom, out, stream=None):
    _check(lib().project_forward(ctx.h, gauss.h, geom.h, _ptr(out), _stream(stream)))
    return out


def project_backward(ctx, gauss, geom, dLdI, g_mu=None, g_ls=None, g_q=None, g_rho=None,
                     stream=None):
    _check(lib().project_backward(ctx.h, gauss.h, geom.h, _ptr(dLdI), _ptr(g_mu), _ptr(g_ls),
                                  _ptr(g_q), _ptr(g_rho), _stream(stream)))
    return g_mu, g_ls, g_q, g_rho


def project_forward_noalloc(desc: dict, mu, ls, q, rho, out, stream=None):
    """Forward projection that allocates no memory (static device scratch);
    all arrays must be contiguous float32 CUDA tensors of the current device:
    mu, ls (n, 3), q (n, 4), rho (n,), out (number of rays,).  The library
    only sees raw pointers, so shapes and dtypes are checked here (ValueError)
    before the call."""
    import torch
    n = int(mu.shape[0]) if hasattr(mu, "shape") and len(mu.shape) >= 1 else -1
    dev = torch.cuda.current_device() if torch.cuda.is_available() else -1
    for name, a, shape in (("mu", mu, (n, 3)), ("ls", ls, (n, 3)), ("q", q, (n, 4)), ("rho", rho, (n,))):
        if not isinstance(a, torch.Tensor) or not a.is_cuda or a.device.index != dev:
            raise ValueError(f"{name}: a CUDA tensor of the current device is required")
        if a.dtype != torch.float32 or tuple(a.shape) != shape or not a.is_contiguous():
            raise ValueError(f"{name}: contiguous float32 of shape {shape} required, got "
                             f"{a.dtype} {tuple(a.shape)}")
    rays = int(desc["n_views"]) * (2 * int(desc.get("max_ring_diff", 0)) + 1 if desc["kind"] == "pet3d" else 1) \
        * int(desc["n_rows"]) * int(desc["n_cols"])
    if (not isinstance(out, torch.Tensor) or not out.is_cuda or out.device.index != dev
            or out.dtype != torch.float32 or out.numel() != rays or not out.is_contiguous()):
        raise ValueError(f"out: a contiguous float32 CUDA tensor of {rays} elements on the current "
                         "device is required")
    d, angles = make_desc(desc)
    _check(lib().project_forward_noalloc(ctypes.byref(d), n, _ptr(mu), _ptr(ls), _ptr(q), _ptr(rho),
                                         _ptr(out), _stream(stream)))
    del angles
    return out


class Batch:
    """Many independent scans stepped together: one persistent launch per pass
    over every (scan, tile) work item, the whole step replayed from a CUDA graph."""

    def __init__(self, ctx: Context, gauss: list, geoms: list):
        assert len(gauss) == len(geoms) and gauss
        self.ctx = ctx
        self.gauss = list(gauss)
        self.geoms = list(geoms)
        self.n = len(gauss)
        gh = (_VP * self.n)(*[g.h for g in gauss])
        mh = (_VP * self.n)(*[g.h for g in geoms])
        h = _VP()
        _check(lib().rgrt_batch_create(ctx.h, self.n, ctypes.cast(gh, _VP), ctypes.cast(mh, _VP),
                                       ctypes.byref(h)))
        self.h = h

    def close(self):
        # after its context has been closed the handle is only dropped (its
        # device memory stays allocated until the process ends): destroying it
        # would reach into the freed context
        if self.h and self.ctx.h:
            lib().rgrt_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, outs, stream=None):
        arr = (_VP * self.n)(*[_ptr(o) for o in outs])
        _check(lib().rgrt_batch_forward(self.h, ctypes.cast(arr, _VP), _stream(stream)))
        return outs

    def loss_step(self, ys, loss=RGRT_LOSS_L2, hp=None, t=1, stream=None):
        hp = hp or adam_params()
        arr = (_VP * self.n)(*[_ptr(y) for y in ys])
        out = np.zeros(self.n, np.float32)
        _check(lib().rgrt_batch_loss_step(self.h, ctypes.cast(arr, _VP), int(loss), ctypes.byref(hp),
                                          int(t), _ptr(out), _stream(stream)))
        return out

    def debug_tile_lists(self, scan):
        """(tile_start[T+1], gid[K]) of scan `scan` as the last forward or
        step binned it (numpy arrays)."""
        g = self.geoms[scan]
        d = g.desc
        T = int(d["n_views"]) * g.tiles_per_view
        start = np.zeros(T + 1, np.uint32)
        nk = ctypes.c_int64()
        rc = lib().rgrt_batch_debug_tile_lists(self.h, int(scan), ctypes.byref(nk), _ptr(start), None, 0)
        if rc not in (RGRT_OK, -3):
            _check(rc)
        gid = np.zeros(max(nk.value, 1), np.uint32)
        _check(lib().rgrt_batch_debug_tile_lists(self.h, int(scan), ctypes.byref(nk), _ptr(start), _ptr(gid),
                                                 gid.size))
        return start.astype(np.int64), gid[: nk.value].astype(np.int64)

    def info(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(lib().rgrt_batch_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return dict(work_items=a.value, key_capacity=b.value, replans=c.value)


def autotune_tile(ctx, gauss, desc: dict, max_views=12):
    """(tile_w, tile_h, ms) of the fastest tile shape for this scan."""
    d, angles = make_desc(desc)
    tw, th, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().rgrt_autotune_tile(ctx.h, gauss.h, ctypes.byref(d), int(max_views), ctypes.byref(tw),
                                    ctypes.byref(th), ctypes.byref(ms)))
    del angles
    return tw.value, th.value, ms.value


def adam_params(lr_mu=2e-4, lr_logscale=5e-3, lr_quat=1e-3, lr_rho=1e-2, beta1=0.9, beta2=0.999,
                eps=1e-8, kappa=1.0, poisson_eps=1e-9) -> Adam:
    return Adam(lr_mu, lr_logscale, lr_quat, lr_rho, beta1, beta2, eps, kappa, poisson_eps)


def loss_step(ctx, gauss, geom, y, loss=RGRT_LOSS_L2, hp: Adam | None = None, t: int = 1,
              loss_out=None, stream=None):
    hp = hp or adam_params()
    _check(lib().loss_step(ctx.h, gauss.h, geom.h, _ptr(y), int(loss), ctypes.byref(hp), int(t),
                           _ptr(loss_out), _stream(stream)))
    return loss_out


def loss_grad(ctx, gauss, geom, y, loss=RGRT_LOSS_L2, hp: Adam | None = None, loss_out=None,
              g_mu=None, g_ls=None, g_q=None, g_rho=None, stream=None):
    """Loss and dL/d(mu, logscale, quat, rho) without updating the Gaussians."""
    hp = hp or adam_params()
    _check(lib().loss_grad(ctx.h, gauss.h, geom.h, _ptr(y), int(loss), ctypes.byref(hp), _ptr(loss_out),
                           _ptr(g_mu), _ptr(g_ls), _ptr(g_q), _ptr(g_rho), _stream(stream)))
    return loss_out


def gaussians_voxelize(ctx, gauss, vol: dict, out=None, stream=None):
    """Density field on the grid vol = dict(origin, size, dims=(nx, ny, nz));
    out: [nz, ny, nx] float32 (host numpy or device tensor; a new host array
    when None)."""
    d = VolumeDesc((ctypes.c_double * 3)(*vol["origin"]), (ctypes.c_double * 3)(*vol["size"]),
                   (ctypes.c_int32 * 3)(*(int(x) for x in vol["dims"])))
    if out is None:
        nx, ny, nz = (int(x) for x in vol["dims"])
        out = np.zeros((nz, ny, nx), np.float32)
    _check(lib().gaussians_voxelize(ctx.h, gauss.h, ctypes.byref(d), _ptr(out), _stream(stream)))
    return out


def debug_records(ctx, gauss):
    out = np.zeros((gauss.n, 6), np.float32)
    _check(lib().rgrt_debug_records(ctx.h, gauss.h, _ptr(out), _stream(None)))
    return out


def debug_tile_lists(ctx, gauss, geom, v0=0, v1=None):
    """(tile_start[T+1], gid[K]) of views [v0, v1) as numpy arrays."""
    d = geom.desc
    if v1 is None:
        v1 = int(d["n_views"]) * (2 * int(d.get("max_ring_diff", 0)) + 1 if d["kind"] == "pet3d" else 1)
    T = (v1 - v0) * geom.tiles_per_view
    start = np.zeros(T + 1, np.uint32)
    nk = ctypes.c_int64()
    rc = lib().rgrt_debug_tile_lists(ctx.h, gauss.h, geom.h, v0, v1, ctypes.byref(nk), _ptr(start),
                                     None, 0, _stream(None))
    if rc not in (RGRT_OK, -3):
        _check(rc)
    gid = np.zeros(max(nk.value, 1), np.uint32)
    _check(lib().rgrt_debug_tile_lists(ctx.h, gauss.h, geom.h, v0, v1, ctypes.byref(nk), _ptr(start),
                                       _ptr(gid), gid.size, _stream(None)))
    return start.astype(np.int64), gid[: nk.value].astype(np.int64)


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------

def _autograd():
    import torch

    class GaussianProject(torch.autograd.Function):
        """I = project(mu, logscale, quat, rho) on a Geometry; backward is the
        library's hand-written adjoint.  Inputs: contiguous float32 CUDA tensors."""

        @staticmethod
        def forward(fctx, mu, ls, q, rho, geom):
            g = Gaussians(geom.ctx, mu, ls, q, rho, borrow=True)
            out = torch.empty(geom.n_rays, device=mu.device, dtype=torch.float32)
            project_forward(geom.ctx, g, geom, out)
            fctx.g = g
            fctx.geom = geom
            fctx.save_for_backward(mu, ls, q, rho)
            return out

        @staticmethod
        def backward(fctx, gout):
            mu, ls, q, rho = fctx.saved_tensors
            gout = gout.contiguous().float()
            gm = torch.empty_like(mu)
            gl = torch.empty_like(ls)
            gq = torch.empty_like(q)
            gr = torch.empty_like(rho)
            project_backward(fctx.geom.ctx, fctx.g, fctx.geom, gout, gm, gl, gq, gr)
            fctx.g.close()
            return gm, gl, gq, gr, None

    return GaussianProject


_GP = None


def gaussian_project(mu, ls, q, rho, geom):
    """Differentiable projection (torch.autograd.Function over the C ABI)."""
    global _GP
    if _GP is None:
        _GP = _autograd()
    return _GP.apply(mu, ls, q, rho, geom)
