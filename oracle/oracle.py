"""Python face of the FP64 CPU oracle (``oracle.c``) plus the loss and Adam
references, written in numpy.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never imports
it, and it never imports the product library.

Parity unpinned: none.  Every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, quadrature, finite differences, invariants or library
routines (see the test docstrings).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("n_views", ctypes.c_int32),
        ("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32),
        ("angles", ctypes.POINTER(ctypes.c_double)),
        ("pitch_u", ctypes.c_double), ("pitch_v", ctypes.c_double),
        ("t_a", ctypes.c_double), ("t_b", ctypes.c_double),
        ("dso", ctypes.c_double), ("dsd", ctypes.c_double), ("radius", ctypes.c_double),
        ("n_crystals", ctypes.c_int32), ("arc_mode", ctypes.c_int32),
        ("max_ring_diff", ctypes.c_int32),
        ("n_tof", ctypes.c_int32), ("tof_spacing", ctypes.c_double), ("tof_sigma", ctypes.c_double),
    ]


_KIND = {"parallel": 0, "cone": 1, "pet": 2, "pet3d": 3}
_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.or_num_rays.restype = ctypes.c_int64
        _lib.or_max_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Geometry:
    """ctypes geometry built from a synth geometry description dict."""

    def __init__(self, desc: dict):
        self.desc = desc
        self._angles = _f64(desc.get("angles", np.zeros(0)))
        # no angles: null (PET then spaces its n_views angles evenly over pi)
        aptr = (self._angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if self._angles.size
                else ctypes.POINTER(ctypes.c_double)())
        self.s = _Geom(
            _KIND[desc["kind"]], int(desc["n_views"]), int(desc["n_rows"]), int(desc["n_cols"]),
            aptr,
            float(desc.get("pitch_u", 0.0)), float(desc.get("pitch_v", 0.0)),
            float(desc.get("t_a", 0.0)), float(desc.get("t_b", 0.0)),
            float(desc.get("dso", 0.0)), float(desc.get("dsd", 0.0)),
            float(desc.get("radius", 0.0)), int(desc.get("n_crystals", 0)),
            int(desc.get("arc_mode", 0)), int(desc.get("max_ring_diff", 0)),
            int(desc.get("n_tof", 0)), float(desc.get("tof_spacing", 0.0)), float(desc.get("tof_sigma", 0.0)))
        self.n_views = int(desc["n_views"]) * (2 * int(desc.get("max_ring_diff", 0)) + 1
                                               if desc["kind"] == "pet3d" else 1)
        # outputs: with time of flight, n_tof per LOR (TOF bin outermost)
        self.n_lors = self.n_views * int(desc["n_rows"]) * int(desc["n_cols"])
        self.n_rays = self.n_lors * max(1, int(desc.get("n_tof", 0)))

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _geom(g):
    return g if isinstance(g, Geometry) else Geometry(g)


KERNELS = {"gaussian": 0, "epanechnikov": 1}
KAPPA2 = 7.0   # Epanechnikov support: Mahalanobis distance squared < 7


def _set_kernel(kernel):
    lib().or_set_kernel(ctypes.c_int(KERNELS[kernel]))


def _gauss(G):
    """Parameter arrays of a Gaussian set; selects its kernel (G["kernel"],
    default "gaussian") for the call that follows."""
    _set_kernel(G.get("kernel", "gaussian"))
    mu = _f32(G["mu"], (-1, 3))
    n = mu.shape[0]
    return n, mu, _f32(G["ls"], (n, 3)), _f32(G["q"], (n, 4)), _f32(G["rho"], (n,))


def max_threads() -> int:
    return int(lib().or_max_threads())


# ---------------------------------------------------------------------------
# projector
# ---------------------------------------------------------------------------

CUT2 = 9.0          # pairs with m <= 3^2 count (the 3-sigma reading of "negligible")
BAND = 9.0e-4       # |m - 9| <= 1e-4 * 9: ambiguous between FP32 and FP64


def pair(o, d, ta, tb, mu, ls, q, rho, kernel="gaussian"):
    """(value, m, A, B, C) of one Gaussian on one ray (no cut-off)."""
    _set_kernel(kernel)
    out = np.zeros(5)
    lib().or_pair(_p(_f64(o)), _p(_f64(d)), ctypes.c_double(ta), ctypes.c_double(tb),
                  _p(_f32(mu)), _p(_f32(ls)), _p(_f32(q)), ctypes.c_float(rho), _p(out))
    return out


def pair_grad(o, d, ta, tb, mu, ls, q, rho, kernel="gaussian"):
    """d value / d(mu[3], l[3], q[4], rho) of one pair (no cut-off)."""
    _set_kernel(kernel)
    out = np.zeros(11)
    lib().or_pair_grad(_p(_f64(o)), _p(_f64(d)), ctypes.c_double(ta), ctypes.c_double(tb),
                       _p(_f32(mu)), _p(_f32(ls)), _p(_f32(q)), ctypes.c_float(rho), _p(out))
    return out


def cov(ls, q):
    """(Sigma, P) as FP64 [n,3,3] arrays."""
    ls = _f32(ls, (-1, 3))
    n = ls.shape[0]
    q = _f32(q, (n, 4))
    sig = np.zeros((n, 3, 3))
    p = np.zeros((n, 3, 3))
    lib().or_cov(ctypes.c_int64(n), _p(ls), _p(q), _p(sig), _p(p))
    return sig, p


def rays(geom, idx):
    g = _geom(geom)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    n = idx.size
    o = np.zeros((n, 3)); d = np.zeros((n, 3)); ta = np.zeros(n); tb = np.zeros(n)
    lib().or_rays(g.ref, ctypes.c_int64(n), _p(idx), _p(o), _p(d), _p(ta), _p(tb))
    return o, d, ta, tb


def tables(geom):
    g = _geom(geom)
    u = np.zeros(int(g.desc["n_cols"]))
    v = np.zeros(int(g.desc["n_rows"]))
    lib().or_tables(g.ref, _p(u), _p(v))
    return u, v


def forward(geom, G, cut2=CUT2, band=BAND, brute=False, nthreads=0):
    """FP64 projection of every ray: dict(I, I_lo, I_hi, pairs)."""
    g = _geom(geom)
    n, mu, ls, q, rho = _gauss(G)
    I = np.zeros(g.n_rays); Ilo = np.zeros(g.n_rays); Ihi = np.zeros(g.n_rays)
    pairs = ctypes.c_int64(0)
    lib().or_forward(g.ref, ctypes.c_int64(n), _p(mu), _p(ls), _p(q), _p(rho),
                     ctypes.c_double(cut2), ctypes.c_double(band), ctypes.c_int(int(brute)),
                     ctypes.c_int(nthreads), _p(I), _p(Ilo), _p(Ihi), ctypes.byref(pairs))
    return dict(I=I, I_lo=Ilo, I_hi=Ihi, pairs=int(pairs.value))


def forward_rays(geom, G, idx, cut2=CUT2, band=BAND, nthreads=0):
    """Brute-force FP64 projection of selected rays (flat output indices)."""
    g = _geom(geom)
    n, mu, ls, q, rho = _gauss(G)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    nr = idx.size
    I = np.zeros(nr); Ilo = np.zeros(nr); Ihi = np.zeros(nr)
    lib().or_forward_rays(g.ref, ctypes.c_int64(n), _p(mu), _p(ls), _p(q), _p(rho),
                          ctypes.c_double(cut2), ctypes.c_double(band), ctypes.c_int64(nr),
                          _p(idx), ctypes.c_int(nthreads), _p(I), _p(Ilo), _p(Ihi))
    return dict(I=I, I_lo=Ilo, I_hi=Ihi)


def backward(geom, G, dLdI, sel=None, cut2=CUT2, band=BAND, brute=False, nthreads=0):
    """FP64 adjoint: dict(mu, ls, q, rho) of dL/dparameter (pairs with m <= cut2),
    plus 'lo' and 'hi' dicts bracketing every admissible choice for pairs
    within ``band`` of the cut.  ``sel`` restricts the Gaussians evaluated
    (rows of the others are NaN)."""
    g = _geom(geom)
    n, mu, ls, q, rho = _gauss(G)
    w = _f64(dLdI).reshape(-1)
    assert w.size == g.n_rays
    gm = np.full((n, 3), np.nan); gl = np.full((n, 3), np.nan)
    gq = np.full((n, 4), np.nan); gr = np.full(n, np.nan)
    lohi = np.full((n, 22), np.nan)
    if sel is None:
        nsel, selp = n, None
    else:
        sel_a = np.ascontiguousarray(sel, dtype=np.int64)
        nsel, selp = sel_a.size, _p(sel_a)
    lib().or_backward(g.ref, ctypes.c_int64(n), _p(mu), _p(ls), _p(q), _p(rho),
                      ctypes.c_double(cut2), ctypes.c_double(band), _p(w), ctypes.c_int64(nsel),
                      selp, ctypes.c_int(int(brute)), ctypes.c_int(nthreads),
                      _p(gm), _p(gl), _p(gq), _p(gr), _p(lohi))

    def split(a):
        return dict(mu=a[:, 0:3], ls=a[:, 3:6], q=a[:, 6:10], rho=a[:, 10])
    return dict(mu=gm, ls=gl, q=gq, rho=gr, lo=split(lohi[:, :11]), hi=split(lohi[:, 11:]))


def _ray_arrays(o, d, t):
    o = _f64(o).reshape(-1, 3)
    d = _f64(d).reshape(-1, 3)
    t = _f64(t).reshape(-1, 2)
    assert o.shape[0] == d.shape[0] == t.shape[0]
    return o, d, t


def _tof(tof, nr):
    if tof is None:
        return None
    tof = _f64(tof).reshape(-1, 2)
    assert tof.shape[0] == nr
    return tof


def forward_list(o, d, t, G, cut2=CUT2, band=BAND, nthreads=0, tof=None):
    """FP64 projection of explicit rays (o[R,3], d[R,3] any length, t[R,2]
    along the unit direction; tof[R,2] = time-of-flight centre and width, or
    None): dict(I, I_lo, I_hi, pairs); every pair evaluated."""
    o, d, t = _ray_arrays(o, d, t)
    tf = _tof(tof, o.shape[0])
    nr = o.shape[0]
    n, mu, ls, q, rho = _gauss(G)
    I = np.zeros(nr); Ilo = np.zeros(nr); Ihi = np.zeros(nr)
    pairs = ctypes.c_int64(0)
    lib().or_forward_list(ctypes.c_int64(nr), _p(o), _p(d), _p(t), None if tf is None else _p(tf),
                          ctypes.c_int64(n), _p(mu), _p(ls),
                          _p(q), _p(rho), ctypes.c_double(cut2), ctypes.c_double(band),
                          ctypes.c_int(nthreads), _p(I), _p(Ilo), _p(Ihi), ctypes.byref(pairs))
    return dict(I=I, I_lo=Ilo, I_hi=Ihi, pairs=int(pairs.value))


def backward_list(o, d, t, G, dLdI, cut2=CUT2, band=BAND, nthreads=0, tof=None):
    """FP64 adjoint for explicit rays; same outputs as backward()."""
    o, d, t = _ray_arrays(o, d, t)
    tf = _tof(tof, o.shape[0])
    nr = o.shape[0]
    n, mu, ls, q, rho = _gauss(G)
    w = _f64(dLdI).reshape(-1)
    assert w.size == nr
    gm = np.zeros((n, 3)); gl = np.zeros((n, 3)); gq = np.zeros((n, 4)); gr = np.zeros(n)
    lohi = np.zeros((n, 22))
    lib().or_backward_list(ctypes.c_int64(nr), _p(o), _p(d), _p(t), None if tf is None else _p(tf),
                           ctypes.c_int64(n), _p(mu), _p(ls),
                           _p(q), _p(rho), ctypes.c_double(cut2), ctypes.c_double(band), _p(w),
                           ctypes.c_int(nthreads), _p(gm), _p(gl), _p(gq), _p(gr), _p(lohi))

    def split(a):
        return dict(mu=a[:, 0:3], ls=a[:, 3:6], q=a[:, 6:10], rho=a[:, 10])
    return dict(mu=gm, ls=gl, q=gq, rho=gr, lo=split(lohi[:, :11]), hi=split(lohi[:, 11:]))


def voxelize(vol, G, cut2=CUT2, band=BAND, brute=False, nthreads=0):
    """FP64 density field on a voxel grid vol = dict(origin=(x, y, z) of voxel
    (0, 0, 0), size=(vx, vy, vz), dims=(nx, ny, nz)): dict(V, V_lo, V_hi) with
    arrays [nz, ny, nx]."""
    origin = _f64(vol["origin"])
    size = _f64(vol["size"])
    dims = np.ascontiguousarray(vol["dims"], dtype=np.int32)
    nx, ny, nz = (int(x) for x in dims)
    n, mu, ls, q, rho = _gauss(G)
    V = np.zeros((nz, ny, nx)); Vlo = np.zeros_like(V); Vhi = np.zeros_like(V)
    lib().or_voxelize(_p(origin), _p(size), _p(dims), ctypes.c_int64(n), _p(mu), _p(ls), _p(q), _p(rho),
                      ctypes.c_double(cut2), ctypes.c_double(band), ctypes.c_int(int(brute)),
                      ctypes.c_int(nthreads), _p(V), _p(Vlo), _p(Vhi))
    return dict(V=V, V_lo=Vlo, V_hi=Vhi)


# ---------------------------------------------------------------------------
# FP32 culling specification (bit-exact tile lists)
# ---------------------------------------------------------------------------

def records_fp32(ls, q):
    """FP32 Sigma packed (00,01,02,11,12,22) as the culling specification defines it."""
    ls = _f32(ls, (-1, 3))
    n = ls.shape[0]
    q = _f32(q, (n, 4))
    out = np.zeros((n, 6), dtype=np.float32)
    lib().or_records_fp32(ctypes.c_int64(n), _p(ls), _p(q), _p(out))
    return out


def cull_fp32(geom, G, tile_w, tile_h, views=None):
    """FP32 cull of views [v0, v1) (``views`` = (v0, v1); default every view,
    3-D PET counting one per ring difference and angle): (pixel box[V, n, 4]
    = i0, i1, j0, j1; tile rectangle[V, n, 4] = tx0, tx1, ty0, ty1; tile
    count[V, n]), V = v1 - v0."""
    g = _geom(geom)
    n, mu, ls, q, rho = _gauss(G)
    v0, v1 = (0, g.n_views) if views is None else (int(views[0]), int(views[1]))
    if not 0 <= v0 < v1 <= g.n_views:
        raise ValueError(f"view range {v0}..{v1} outside 0..{g.n_views}")
    V = v1 - v0
    box = np.zeros((V, n, 4), dtype=np.int32)
    cnt = np.zeros((V, n), dtype=np.int32)
    lib().or_cull_fp32_range(g.ref, ctypes.c_int64(n), _p(mu), _p(ls), _p(q),
                             ctypes.c_int(tile_w), ctypes.c_int(tile_h), ctypes.c_int(v0),
                             ctypes.c_int(v1), _p(box), _p(cnt))
    rect = np.where(box >= 0, box // np.array([tile_w, tile_w, tile_h, tile_h]), -1).astype(np.int32)
    return box, rect, cnt


def tile_lists_fp32(geom, G, tile_w, tile_h, views=None):
    """Per-tile Gaussian sets implied by the FP32 cull of views [v0, v1), in
    CSR form: (start[T+1], gid[K]); tile id = (view - v0) * tiles_per_view +
    ty * tiles_x + tx.  A tile's list is a set (the projection needs no
    depth order), written here in increasing Gaussian id."""
    desc = geom.desc if isinstance(geom, Geometry) else geom
    box, rect, cnt = cull_fp32(geom, G, tile_w, tile_h, views)
    V, n = cnt.shape
    tx_n = (int(desc["n_cols"]) + tile_w - 1) // tile_w
    ty_n = (int(desc["n_rows"]) + tile_h - 1) // tile_h
    T = V * tx_n * ty_n
    # every (view, Gaussian) with a non-empty rectangle, expanded to one entry
    # per tile of the rectangle (row-major within it)
    v_idx, k_idx = np.nonzero(cnt)
    r = rect[v_idx, k_idx].astype(np.int64)
    nx = r[:, 1] - r[:, 0] + 1
    c = cnt[v_idx, k_idx].astype(np.int64)
    first = np.repeat(np.cumsum(c) - c, c)
    j = np.arange(int(c.sum()), dtype=np.int64) - first        # position in the rectangle
    ent = np.repeat(np.arange(c.size), c)
    ty = r[ent, 2] + j // nx[ent]
    tx = r[ent, 0] + j % nx[ent]
    tiles = v_idx[ent].astype(np.int64) * tx_n * ty_n + ty * tx_n + tx
    gids = k_idx[ent].astype(np.int64)
    order = np.lexsort((gids, tiles))
    tiles, gids = tiles[order], gids[order]
    start = np.zeros(T + 1, dtype=np.int64)
    np.add.at(start, tiles + 1, 1)
    start = np.cumsum(start)
    return start, gids


# ---------------------------------------------------------------------------
# losses and Adam (numpy, FP64)
# ---------------------------------------------------------------------------

def loss_l2(I, y, mult=None, add=None):
    """L = 1/2 sum (m I + a - y)^2, dL/dI = m (m I + a - y); m = mult (default 1),
    a = add (default 0): the measurement model's per-ray factor and background."""
    m = 1.0 if mult is None else np.asarray(mult, np.float64)
    a = 0.0 if add is None else np.asarray(add, np.float64)
    r = m * np.asarray(I, np.float64) + a - np.asarray(y, np.float64)
    return 0.5 * float(np.sum(r * r)), m * r


def loss_poisson(I, y, kappa, eps, mult=None, add=None):
    """L = sum (lam - y log lam), lam = kappa m I + a + eps,
    dL/dI = kappa m (1 - y/lam); m = mult (default 1), a = add (default 0)."""
    m = 1.0 if mult is None else np.asarray(mult, np.float64)
    a = 0.0 if add is None else np.asarray(add, np.float64)
    lam = kappa * m * np.asarray(I, np.float64) + a + eps
    y = np.asarray(y, np.float64)
    return float(np.sum(lam - y * np.log(lam))), kappa * m * (1.0 - y / lam)


def adam(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba), bias-corrected; returns (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
