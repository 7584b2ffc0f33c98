"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module draws random numbers and writes down geometry *descriptions*
(counts, pitches, distances, view angles).  It holds none of the projector's
arithmetic: no ray set-up, no covariance, no line integral.  Both the CUDA path
and the FP64 oracle receive exactly these arrays and build everything else on
their own.

Workloads (sizes of the paper's experiments, section 4.1; constants where the
paper is silent are this project's readings):

* ``c1``  parallel-beam CT, 1,000 Gaussians with centres U[-1,1]^3, log-scales
  N(log 0.05, 0.3^2), random unit quaternions, rho ~ U(0,1); 16 views over 180
  degrees, 64x64 detector of pitch 2/64, rays over t in [-2, 2].
* ``c2``  cone-beam CT, 50,000 Gaussians fitted to a 12-ellipsoid phantom in
  [-1,1]^3 (1 unit = 128 mm); 180 views over 360 degrees, 256x256 detector,
  source-to-origin 1000 mm, source-to-detector 1500 mm, detector pitch
  chosen so the magnified 256 mm field of view fills the panel.  The cone-beam
  sparse-view CT data of the paper (TIGRE-simulated volumes) is not available;
  this phantom stands in for it.
* ``c3``  PET ring of radius 400 mm, 32 rings, 576 crystals per ring;
  arc-corrected sinogram of 288 angles x 329 radial bins x 63 planes, 200,000
  Gaussians fitted to a 20-ellipsoid activity phantom.  Stands in for the
  STIR/GATE-simulated PET data of the paper.
"""
from __future__ import annotations

import math

import numpy as np

# 1 world unit = 128 mm for the CT workloads
CT_MM_PER_UNIT = 128.0


def _random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def gaussians_uniform(n: int, seed: int, half_box: float = 1.0,
                      log_sigma: float = math.log(0.05), log_sigma_std: float = 0.3,
                      rho_range=(0.0, 1.0)) -> dict:
    """Gaussians with centres U[-half_box, half_box]^3 (the c1 recipe)."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-half_box, half_box, size=(n, 3)).astype(np.float32)
    ls = rng.normal(log_sigma, log_sigma_std, size=(n, 3)).astype(np.float32)
    q = _random_quaternions(rng, n)
    rho = rng.uniform(rho_range[0], rho_range[1], size=n).astype(np.float32)
    return dict(mu=mu, ls=ls, q=q, rho=rho)


def _random_rotations(rng: np.random.Generator, k: int) -> np.ndarray:
    """Random rotation matrices (QR of Gaussian matrices, sign-fixed)."""
    out = np.empty((k, 3, 3))
    for i in range(k):
        a = rng.normal(size=(3, 3))
        qm, rm = np.linalg.qr(a)
        qm = qm * np.sign(np.diag(rm))
        if np.linalg.det(qm) < 0:
            qm[:, 0] = -qm[:, 0]
        out[i] = qm
    return out


def ellipsoid_phantom(k: int, seed: int, semi=(0.05, 0.6), dens=(0.1, 1.0),
                      centre_box: float = 1.0, semi_axial=None) -> dict:
    """k random ellipsoids: semi-axes U(semi), random rotation, centre inside the
    box so the ellipsoid stays inside it, additive density U(dens)."""
    rng = np.random.default_rng(seed)
    axes = rng.uniform(semi[0], semi[1], size=(k, 3))
    if semi_axial is not None:
        axes[:, 2] = rng.uniform(semi_axial[0], semi_axial[1], size=k)
    rot = _random_rotations(rng, k)
    amax = axes.max(axis=1)
    lim = np.maximum(centre_box - amax, 0.0)
    centre = rng.uniform(-1.0, 1.0, size=(k, 3)) * lim[:, None]
    dens_v = rng.uniform(dens[0], dens[1], size=k)
    return dict(axes=axes, rot=rot, centre=centre, density=dens_v)


def _phantom_density(ph: dict, x: np.ndarray) -> np.ndarray:
    """Additive density of the ellipsoid phantom at points x[n,3]."""
    dsum = np.zeros(x.shape[0])
    for a, r, c, dv in zip(ph["axes"], ph["rot"], ph["centre"], ph["density"]):
        local = (x - c) @ r  # coordinates along the ellipsoid axes
        inside = np.sum((local / a) ** 2, axis=1) <= 1.0
        dsum += dv * inside
    return dsum


def phantom_fitted_gaussians(ph: dict, n: int, seed: int, box_lo, box_hi,
                             log_sigma_std: float = 0.3) -> dict:
    """Initial Gaussians for a phantom: centres drawn with probability
    proportional to the phantom density (rejection sampling in the box),
    isotropic size h = (V_support / n)^(1/3) with log-scale N(log h, 0.3^2) per
    axis, random rotation, and rho chosen so each Gaussian's mass matches the
    density at its centre times h^3."""
    rng = np.random.default_rng(seed)
    box_lo = np.asarray(box_lo, dtype=np.float64)
    box_hi = np.asarray(box_hi, dtype=np.float64)
    vol_box = float(np.prod(box_hi - box_lo))
    dmax = float(np.sum(ph["density"]))
    probe = rng.uniform(box_lo, box_hi, size=(200_000, 3))
    frac = float(np.mean(_phantom_density(ph, probe) > 0))
    v_support = max(frac * vol_box, 1e-12)
    h = (v_support / n) ** (1.0 / 3.0)
    pts = []
    need = n
    while need > 0:
        cand = rng.uniform(box_lo, box_hi, size=(max(4 * need, 1024), 3))
        dens = _phantom_density(ph, cand)
        keep = rng.uniform(0.0, dmax, size=cand.shape[0]) < dens
        sel = cand[keep][:need]
        pts.append(sel)
        need -= sel.shape[0]
    mu = np.concatenate(pts, axis=0)[:n]
    ls = rng.normal(math.log(h), log_sigma_std, size=(n, 3))
    q = _random_quaternions(rng, n)
    dens_mu = _phantom_density(ph, mu)
    rho = dens_mu * h ** 3 / ((2.0 * math.pi) ** 1.5 * np.exp(ls.sum(axis=1)))
    return dict(mu=mu.astype(np.float32), ls=ls.astype(np.float32), q=q,
                rho=rho.astype(np.float32), h=h)


# ---------------------------------------------------------------------------
# geometry descriptions
# ---------------------------------------------------------------------------

def geom_parallel(n_views: int, n_rows: int, n_cols: int, pitch_u: float, pitch_v: float,
                  t_a: float, t_b: float, span: float = math.pi, tile=(16, 16)) -> dict:
    angles = np.array([span * v / n_views for v in range(n_views)], dtype=np.float64)
    return dict(kind="parallel", n_views=n_views, n_rows=n_rows, n_cols=n_cols,
                angles=angles, pitch_u=pitch_u, pitch_v=pitch_v, t_a=t_a, t_b=t_b,
                dso=0.0, dsd=0.0, radius=0.0, n_crystals=0, arc_mode=0,
                tile_w=tile[0], tile_h=tile[1])


def geom_cone(n_views: int, n_rows: int, n_cols: int, pitch_u: float, pitch_v: float,
              dso: float, dsd: float, span: float = 2.0 * math.pi, tile=(16, 16)) -> dict:
    angles = np.array([span * v / n_views for v in range(n_views)], dtype=np.float64)
    return dict(kind="cone", n_views=n_views, n_rows=n_rows, n_cols=n_cols,
                angles=angles, pitch_u=pitch_u, pitch_v=pitch_v, t_a=0.0, t_b=0.0,
                dso=dso, dsd=dsd, radius=0.0, n_crystals=0, arc_mode=0,
                tile_w=tile[0], tile_h=tile[1])


def geom_pet(n_angles: int, n_radial: int, n_planes: int, radius: float, n_crystals: int,
             plane_pitch: float, arc_mode: int = 0, tile=(16, 16)) -> dict:
    return dict(kind="pet", n_views=n_angles, n_rows=n_planes, n_cols=n_radial,
                angles=np.zeros(0, dtype=np.float64), pitch_u=0.0, pitch_v=plane_pitch,
                t_a=0.0, t_b=0.0, dso=0.0, dsd=0.0, radius=radius,
                n_crystals=n_crystals, arc_mode=arc_mode, tile_w=tile[0], tile_h=tile[1])


def geom_pet3d(n_angles: int, n_radial: int, n_rings: int, radius: float, n_crystals: int,
               ring_pitch: float, max_ring_diff: int, arc_mode: int = 0, tile=(16, 16)) -> dict:
    """Fully 3-D PET sinograms: one view per (ring difference delta in
    [-max_ring_diff, max_ring_diff], angle), delta-major; row j of a view is
    the ring pair (min ring j, ring difference delta), rows j >= n_rings -
    |delta| carry no LOR (their output is 0).  Output [delta][angle][ring
    pair][radial]."""
    return dict(kind="pet3d", n_views=n_angles, n_rows=n_rings, n_cols=n_radial,
                angles=np.zeros(0, dtype=np.float64), pitch_u=0.0, pitch_v=ring_pitch,
                t_a=0.0, t_b=0.0, dso=0.0, dsd=0.0, radius=radius, n_crystals=n_crystals,
                arc_mode=arc_mode, max_ring_diff=max_ring_diff, tile_w=tile[0], tile_h=tile[1])


def geom_c1(tile=(16, 16)) -> dict:
    return geom_parallel(16, 64, 64, 2.0 / 64, 2.0 / 64, -2.0, 2.0, span=math.pi, tile=tile)


def geom_c2(n_views: int = 180, side: int = 256, tile=(16, 16)) -> dict:
    dso = 1000.0 / CT_MM_PER_UNIT          # 7.8125
    dsd = 1500.0 / CT_MM_PER_UNIT          # 11.71875
    # magnified 256 mm field of view fills 256 pixels: 1.5 mm pitch at 256
    pitch = (1.5 * 256.0 / side) / CT_MM_PER_UNIT
    return geom_cone(n_views, side, side, pitch, pitch, dso, dsd, span=2.0 * math.pi, tile=tile)


def geom_c3(n_angles: int = 288, n_radial: int = 329, n_planes: int = 63, arc_mode: int = 0,
            tile=(16, 16)) -> dict:
    # 32 rings at a 4 mm ring pitch: 63 planes (direct + cross) 2 mm apart
    return geom_pet(n_angles, n_radial, n_planes, radius=400.0, n_crystals=576,
                    plane_pitch=2.0, arc_mode=arc_mode, tile=tile)


def geom_c3_3d(max_ring_diff: int = 5, arc_mode: int = 0, tile=(16, 16)) -> dict:
    """The ring of geom_c3 as a fully 3-D scanner: its 32 rings at a 4 mm
    pitch (the 63 planes of geom_c3 are the direct and cross planes of these
    rings) with every ring pair up to the given ring difference."""
    return geom_pet3d(288, 329, 32, radius=400.0, n_crystals=576, ring_pitch=4.0,
                      max_ring_diff=max_ring_diff, arc_mode=arc_mode, tile=tile)


def num_rays(g: dict) -> int:
    """Outputs of a geometry: one per ray, or per (time-of-flight bin, LOR)."""
    if g["kind"] == "rays":
        return int(np.asarray(g["o"]).shape[0])
    v = int(g["n_views"])
    if g["kind"] == "pet3d":
        v *= 2 * int(g["max_ring_diff"]) + 1
    return v * int(g["n_rows"]) * int(g["n_cols"]) * max(1, int(g.get("n_tof", 0)))


def with_tof_bins(g: dict, n_tof: int, spacing: float, sigma: float) -> dict:
    """A PET sinogram geometry with time of flight: n_tof bins per LOR, bin k
    centred at (k - (n_tof - 1)/2) spacing along the LOR from its midpoint,
    Gaussian TOF kernel of width sigma (output [bin][sinogram])."""
    assert g["kind"] in ("pet", "pet3d")
    return dict(g, n_tof=int(n_tof), tof_spacing=float(spacing), tof_sigma=float(sigma))


# ---------------------------------------------------------------------------
# ground truth of the phantoms: detector rays, line integrals, voxel grids
# ---------------------------------------------------------------------------

def detector_rays(g: dict):
    """(o, d, t_a, t_b) in FP64 of every ray of a CT geometry (output order
    [view][row][col]), d unit: parallel o = u e_u + v e_v, d = e_w, t in
    [t_a, t_b]; cone o = S = -dso e_w, d towards the pixel D = S + dsd e_w +
    u e_u + v e_v, t in [0, |D - S|]; e_w = (cos th, sin th, 0),
    e_u = (-sin th, cos th, 0), e_v = z, u_i = (i - (W-1)/2) pitch_u."""
    V, H, W = int(g["n_views"]), int(g["n_rows"]), int(g["n_cols"])
    th = np.asarray(g["angles"], np.float64)
    ew = np.stack([np.cos(th), np.sin(th), np.zeros_like(th)], 1)[:, None, None, :]
    eu = np.stack([-np.sin(th), np.cos(th), np.zeros_like(th)], 1)[:, None, None, :]
    ev = np.array([0.0, 0.0, 1.0])
    u = ((np.arange(W) - 0.5 * (W - 1)) * g["pitch_u"])[None, None, :, None]
    v = ((np.arange(H) - 0.5 * (H - 1)) * g["pitch_v"])[None, :, None, None]
    if g["kind"] == "parallel":
        o = u * eu + v * ev
        d = np.broadcast_to(ew, o.shape)
        ta = np.full(o.shape[:3], float(g["t_a"]))
        tb = np.full(o.shape[:3], float(g["t_b"]))
    elif g["kind"] == "cone":
        S = -g["dso"] * ew
        D = S + g["dsd"] * ew + u * eu + v * ev
        dv = D - S
        L = np.linalg.norm(dv, axis=-1)
        o = np.broadcast_to(S, D.shape)
        d = dv / L[..., None]
        ta, tb = np.zeros_like(L), L
    else:
        raise ValueError("detector_rays covers the CT geometries")
    return (o.reshape(-1, 3), d.reshape(-1, 3), ta.reshape(-1), tb.reshape(-1))


def pet_lors(g: dict):
    """(o, d, t_a, t_b) in FP64 of every LOR of a PET ring sinogram (output
    order [plane][angle][radial]): o = s e_u + z e_v at the chord's midpoint,
    d = e_w, t in [-h, h] with h = sqrt(R^2 - s^2); e_u = (cos phi, sin phi,
    0), e_w = (sin phi, -cos phi, 0), phi_j = pi j / n_views (or the listed
    angles), s_k = (k - (W-1)/2) pi R / n_crystals (arc-corrected) or
    R sin((k - (W-1)/2) pi / n_crystals) (raw), z_p = (p - (H-1)/2) pitch."""
    assert g["kind"] == "pet"
    V, H, W = int(g["n_views"]), int(g["n_rows"]), int(g["n_cols"])
    ang = np.asarray(g.get("angles", np.zeros(0)), np.float64)
    phi = ang if ang.size else math.pi * np.arange(V) / V
    R = float(g["radius"])
    k = np.arange(W) - 0.5 * (W - 1)
    s = k * math.pi * R / g["n_crystals"] if g["arc_mode"] == 0 else R * np.sin(k * math.pi / g["n_crystals"])
    z = (np.arange(H) - 0.5 * (H - 1)) * g["pitch_v"]
    eu = np.stack([np.cos(phi), np.sin(phi), np.zeros(V)], 1)
    ew = np.stack([np.sin(phi), -np.cos(phi), np.zeros(V)], 1)
    o = s[None, None, :, None] * eu[None, :, None, :] + z[:, None, None, None] * np.array([0.0, 0.0, 1.0])
    d = np.broadcast_to(ew[None, :, None, :], o.shape)
    h = np.sqrt(np.maximum(R * R - s * s, 0.0))
    hb = np.broadcast_to(h[None, None, :], o.shape[:3])
    return o.reshape(-1, 3), d.reshape(-1, 3), -hb.reshape(-1), hb.reshape(-1)


def phantom_projection(ph: dict, o, d, ta, tb) -> np.ndarray:
    """Exact line integrals of the ellipsoid phantom (additive densities):
    sum_k D_k |{t in [t_a, t_b]: o + t d inside ellipsoid k}|, d unit, from the
    roots of the quadratic |A^-1 R^T (o + t d - c)|^2 = 1."""
    o = np.asarray(o, np.float64)
    d = np.asarray(d, np.float64)
    out = np.zeros(o.shape[0])
    for a, r, c, dens in zip(ph["axes"], ph["rot"], ph["centre"], ph["density"]):
        p = ((o - c) @ r) / a
        q = (d @ r) / a
        A = np.sum(q * q, axis=1)
        B = np.sum(p * q, axis=1)
        C = np.sum(p * p, axis=1) - 1.0
        disc = B * B - A * C
        hit = disc > 0
        sq = np.sqrt(np.where(hit, disc, 0.0))
        t1 = (-B - sq) / A
        t2 = (-B + sq) / A
        lo = np.maximum(t1, ta)
        hi = np.minimum(t2, tb)
        out += dens * np.where(hit, np.maximum(hi - lo, 0.0), 0.0)
    return out


def voxel_grid(n: int, half: float = 1.0) -> dict:
    """n^3 voxel centres covering [-half, half]^3."""
    h = 2.0 * half / n
    return dict(origin=(-half + h / 2,) * 3, size=(h, h, h), dims=(n, n, n))


def phantom_volume(ph: dict, vol: dict) -> np.ndarray:
    """The phantom's density at the voxel centres, [nz, ny, nx]."""
    nx, ny, nz = (int(x) for x in vol["dims"])
    x = vol["origin"][0] + vol["size"][0] * np.arange(nx)
    y = vol["origin"][1] + vol["size"][1] * np.arange(ny)
    z = vol["origin"][2] + vol["size"][2] * np.arange(nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    return _phantom_density(ph, pts).reshape(nz, ny, nx)


def psnr(vol: np.ndarray, ref: np.ndarray) -> float:
    """Peak signal-to-noise ratio (dB) of vol against ref, peak = max(ref)."""
    mse = float(np.mean((np.asarray(vol, np.float64) - ref) ** 2))
    return 10.0 * math.log10(float(ref.max()) ** 2 / max(mse, 1e-300))


# ---------------------------------------------------------------------------
# point sources in a PET ring (the arc vs raw sampling study)
# ---------------------------------------------------------------------------

def pet_radial_positions(g: dict) -> np.ndarray:
    """Radial positions s_i of a PET geometry's bins (arc-corrected: uniform
    pi R / n_crystals apart; raw: R sin of the crystal-pair angle)."""
    k = np.arange(int(g["n_cols"])) - 0.5 * (int(g["n_cols"]) - 1)
    R, n = float(g["radius"]), int(g["n_crystals"])
    if int(g.get("arc_mode", 0)) == 0:
        return k * (math.pi * R / n)
    return R * np.sin(k * math.pi / n)


def point_source_sinogram(g: dict, centres, radius: float, density: float = 1.0, n_sub: int = 5) -> np.ndarray:
    """Expected sinogram [plane][angle][radial] of small uniform spheres
    (point sources of the given radius and density) on a 2-D PET ring
    geometry: chord lengths 2 sqrt(a^2 - r^2)_+ through each sphere, r^2 =
    (c . e_u - s)^2 + (c_z - z_p)^2, each bin averaged over n_sub positions
    across its width (raw bins: crystal-pair angles within half a crystal
    step either side, so their width shrinks as cos; arc-corrected bins: a
    uniform width)."""
    V, H, W = int(g["n_views"]), int(g["n_rows"]), int(g["n_cols"])
    R, n = float(g["radius"]), int(g["n_crystals"])
    k = np.arange(W) - 0.5 * (W - 1)
    off = (np.arange(n_sub) + 0.5) / n_sub - 0.5          # sub-positions across a bin, in bin units
    if int(g.get("arc_mode", 0)) == 0:
        s = (k[:, None] + off[None, :]) * (math.pi * R / n)
    else:
        s = R * np.sin((k[:, None] + off[None, :]) * math.pi / n)
    phi = math.pi * np.arange(V) / V
    z = (np.arange(H) - 0.5 * (H - 1)) * float(g["pitch_v"])
    out = np.zeros((H, V, W))
    for c in np.asarray(centres, np.float64):
        cu = c[0] * np.cos(phi) + c[1] * np.sin(phi)                 # [V]
        r2 = (cu[None, :, None, None] - s[None, None, :, :]) ** 2 + ((c[2] - z) ** 2)[:, None, None, None]
        out += density * (2.0 * np.sqrt(np.maximum(radius * radius - r2, 0.0))).mean(axis=3)
    return out


def arc_resample(y: np.ndarray, g_raw: dict) -> np.ndarray:
    """Arc correction of a raw-mode sinogram [plane][angle][radial]: every
    projection linearly interpolated from the raw positions R sin(.) onto the
    uniform positions of the arc-corrected geometry (same bins, arc_mode 0);
    positions beyond the outermost raw bin get 0."""
    s_raw = pet_radial_positions(dict(g_raw, arc_mode=1))
    s_arc = pet_radial_positions(dict(g_raw, arc_mode=0))
    H, V, W = y.shape
    flat = y.reshape(-1, W)
    out = np.empty_like(flat, dtype=np.float64)
    for r in range(flat.shape[0]):
        out[r] = np.interp(s_arc, s_raw, flat[r], left=0.0, right=0.0)
    return out.reshape(H, V, W)


def grid_gaussians(radius: float, spacing: float, sigma: float, rho: float, z: float = 0.0) -> dict:
    """Isotropic Gaussians on a square grid (one layer at height z) filling
    the disk of the given radius: a blind start for reconstructions."""
    a = np.arange(-radius, radius + spacing / 2, spacing)
    X, Y = np.meshgrid(a, a, indexing="ij")
    keep = X ** 2 + Y ** 2 <= radius ** 2
    n = int(keep.sum())
    mu = np.stack([X[keep], Y[keep], np.full(n, z)], 1).astype(np.float32)
    return dict(mu=mu, ls=np.full((n, 3), math.log(sigma), np.float32),
                q=np.tile(np.array([1.0, 0.0, 0.0, 0.0], np.float32), (n, 1)),
                rho=np.full(n, rho, np.float32))


def fwhm(profile: np.ndarray, spacing: float) -> float:
    """Full width at half maximum of a sampled single-peaked profile, the
    half-maximum crossings found by linear interpolation either side of the
    peak (nan if a crossing is missing)."""
    p = np.asarray(profile, np.float64)
    i = int(np.argmax(p))
    half = 0.5 * p[i]
    lo = i
    while lo > 0 and p[lo] > half:
        lo -= 1
    hi = i
    while hi < p.size - 1 and p[hi] > half:
        hi += 1
    if p[lo] > half or p[hi] > half:
        return float("nan")
    xl = lo + (half - p[lo]) / (p[lo + 1] - p[lo])
    xh = hi - (half - p[hi]) / (p[hi - 1] - p[hi])
    return float((xh - xl) * spacing)


# ---------------------------------------------------------------------------
# explicit ray sets
# ---------------------------------------------------------------------------

def rays_helical(n_views: int, n_rows: int, n_cols: int, pitch: float, dso: float, dsd: float,
                 z_per_turn: float, turns: float = 1.0) -> dict:
    """Helical cone-beam CT as explicit rays: the source at angle th_k =
    2 pi turns k / n_views sits at (-dso e_w, z_k), z_k = z_per_turn th_k / 2 pi
    - the middle height, with the flat detector frame of the circular cone beam
    (e_w = (cos th, sin th, 0), e_u = (-sin th, cos th, 0), e_v = z) moving with
    it; each ray runs from the source (t = 0) to its pixel (t = |D - S|).
    Layout [view][row][col]."""
    k = np.arange(n_views, dtype=np.float64)
    th = 2.0 * math.pi * turns * k / n_views
    z = z_per_turn * th / (2.0 * math.pi)
    z -= 0.5 * (z[0] + z[-1])
    ew = np.stack([np.cos(th), np.sin(th), np.zeros_like(th)], 1)
    eu = np.stack([-np.sin(th), np.cos(th), np.zeros_like(th)], 1)
    ev = np.array([0.0, 0.0, 1.0])
    u = (np.arange(n_cols) - 0.5 * (n_cols - 1)) * pitch
    v = (np.arange(n_rows) - 0.5 * (n_rows - 1)) * pitch
    S = -dso * ew + z[:, None] * ev                                   # [V,3]
    D = (S[:, None, None, :] + dsd * ew[:, None, None, :] + u[None, None, :, None] * eu[:, None, None, :]
         + v[None, :, None, None] * ev[None, None, None, :])           # [V,H,W,3]
    dvec = D - S[:, None, None, :]
    L = np.linalg.norm(dvec, axis=-1)
    o = np.broadcast_to(S[:, None, None, :], D.shape).reshape(-1, 3)
    t = np.stack([np.zeros(L.size), L.reshape(-1)], 1)
    return dict(kind="rays", o=o.astype(np.float32), d=dvec.reshape(-1, 3).astype(np.float32),
                t=t.astype(np.float32))


def _morton2(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Interleave the bits of a (even positions) and b (odd positions)."""
    code = np.zeros(a.shape, np.int64)
    for bit in range(16):
        code |= ((a >> bit) & 1) << (2 * bit)
        code |= ((b >> bit) & 1) << (2 * bit + 1)
    return code


def pet_rays_3d(n_rings: int = 32, ring_pitch: float = 4.0, radius: float = 400.0, n_crystals: int = 576,
                n_angles: int = 288, n_radial: int = 329, max_ring_diff: int = 5, arc_mode: int = 0) -> dict:
    """Fully 3-D PET: the LORs between every pair of rings (r1, r2) with
    |r1 - r2| <= max_ring_diff, at the sinogram angles phi_j = pi j / n_angles
    and radial positions s_k of the 2-D ring geometry (arc-corrected or raw
    chords).  Ring r sits at z_r = (r - (n_rings - 1)/2) ring_pitch; the LOR
    runs from s e_u - h e_w + z_r1 e_z to s e_u + h e_w + z_r2 e_z,
    h = sqrt(R^2 - s^2), e_u = (cos phi, sin phi, 0), e_w = (sin phi, -cos phi, 0).
    Order: by ring difference, then angle, then the (ring pair, radial bin)
    grid of that difference and angle along a Morton curve (radial bits on
    the even positions), so that any 128 consecutive rays lie close together;
    the returned dict carries each ray's (ring1, ring2, angle, radial)."""
    c = 0.5 * (n_radial - 1)
    k = np.arange(n_radial) - c
    s = k * (math.pi * radius / n_crystals) if arc_mode == 0 else radius * np.sin(k * math.pi / n_crystals)
    h = np.sqrt(radius * radius - s * s)
    zr = (np.arange(n_rings) - 0.5 * (n_rings - 1)) * ring_pitch
    phi = math.pi * np.arange(n_angles) / n_angles
    out_o, out_d, out_t, idx = [], [], [], []
    ez = np.array([0.0, 0.0, 1.0])
    for dlt in range(-max_ring_diff, max_ring_diff + 1):
        r1s = np.array([r for r in range(n_rings) if 0 <= r + dlt < n_rings])
        if r1s.size == 0:
            continue
        pp, kk = np.meshgrid(np.arange(r1s.size), np.arange(n_radial), indexing="ij")
        order = np.argsort(_morton2(kk.ravel(), pp.ravel()), kind="stable")
        r1 = r1s[pp.ravel()[order]]
        r2 = r1 + dlt
        kq = kk.ravel()[order]
        for j in range(n_angles):
            eu = np.array([math.cos(phi[j]), math.sin(phi[j]), 0.0])
            ew = np.array([math.sin(phi[j]), -math.cos(phi[j]), 0.0])
            a = s[kq, None] * eu - h[kq, None] * ew + zr[r1, None] * ez
            b = s[kq, None] * eu + h[kq, None] * ew + zr[r2, None] * ez
            dv = b - a
            out_o.append(a)
            out_d.append(dv)
            out_t.append(np.stack([np.zeros(kq.size), np.linalg.norm(dv, axis=1)], 1))
            idx.append(np.stack([r1, r2, np.full(kq.size, j), kq], 1))
    return dict(kind="rays", o=np.concatenate(out_o).astype(np.float32),
                d=np.concatenate(out_d).astype(np.float32), t=np.concatenate(out_t).astype(np.float32),
                index=np.concatenate(idx).astype(np.int32), n_rings=n_rings, ring_pitch=ring_pitch)


def with_tof(R: dict, n_bins: int, spacing: float, sigma: float) -> dict:
    """Time-of-flight version of a ray set: every ray repeated n_bins times
    (ray-major), bin k with the TOF kernel centred at the segment's middle +
    (k - (n_bins - 1)/2) spacing (along the unit direction) and width sigma."""
    t = np.asarray(R["t"], np.float64)
    mid = np.where(np.isfinite(t).all(axis=1), 0.5 * (t[:, 0] + t[:, 1]), 0.0)
    off = (np.arange(n_bins) - 0.5 * (n_bins - 1)) * spacing
    out = {k: np.repeat(np.asarray(v), n_bins, axis=0) for k, v in R.items()
           if isinstance(v, np.ndarray) and v.ndim >= 1 and v.shape[0] == t.shape[0]}
    out.update({k: v for k, v in R.items() if k not in out})
    centres = (mid[:, None] + off[None, :]).reshape(-1)
    out["tof"] = np.stack([centres, np.full(centres.size, sigma)], 1).astype(np.float32)
    return out


def rays_random(n: int, seed: int, radius: float = 1.0, seg: float | None = None) -> dict:
    """Incoherent rays: lines through uniform points of the ball of the given
    radius along uniform directions (unnormalised: length U(0.5, 2)), the
    segment [-seg, seg] around that point (infinite when seg is None)."""
    rng = np.random.default_rng(seed)
    p = rng.normal(size=(n, 3))
    p *= (radius * rng.uniform(0, 1, n) ** (1 / 3) / np.linalg.norm(p, axis=1))[:, None]
    d = rng.normal(size=(n, 3))
    d *= (rng.uniform(0.5, 2.0, n) / np.linalg.norm(d, axis=1))[:, None]
    t = np.full((n, 2), np.inf)
    t[:, 0] = -np.inf
    if seg is not None:
        t[:, 0], t[:, 1] = -seg, seg
    return dict(kind="rays", o=p.astype(np.float32), d=d.astype(np.float32), t=t.astype(np.float32))


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def workload_c1(seed: int = 0) -> tuple[dict, dict]:
    return gaussians_uniform(1000, seed), geom_c1()


def workload_c2(seed: int = 0, n: int = 50_000, n_views: int = 180, side: int = 256) -> tuple[dict, dict]:
    ph = ellipsoid_phantom(12, seed=1000 + seed, semi=(0.05, 0.6), dens=(0.1, 1.0))
    gs = phantom_fitted_gaussians(ph, n, seed=2000 + seed, box_lo=(-1, -1, -1), box_hi=(1, 1, 1))
    return gs, geom_c2(n_views=n_views, side=side)


def pet_phantom(seed: int = 0) -> dict:
    """20 activity ellipsoids inside a cylinder of radius 250 mm, |z| <= 60 mm."""
    rng = np.random.default_rng(3000 + seed)
    k = 20
    axes = np.column_stack([rng.uniform(5, 80, k), rng.uniform(5, 80, k), rng.uniform(5, 40, k)])
    rot = _random_rotations(rng, k)
    amax = axes.max(axis=1)
    r_lim = np.maximum(250.0 - amax, 0.0)
    rad = r_lim * np.sqrt(rng.uniform(0, 1, k))
    ang = rng.uniform(0, 2 * math.pi, k)
    z_lim = np.maximum(60.0 - axes[:, 2], 0.0)
    centre = np.column_stack([rad * np.cos(ang), rad * np.sin(ang), rng.uniform(-1, 1, k) * z_lim])
    return dict(axes=axes, rot=rot, centre=centre, density=rng.uniform(0.1, 1.0, k))


def workload_c3(seed: int = 0, n: int = 200_000, n_angles: int = 288, n_radial: int = 329,
                n_planes: int = 63) -> tuple[dict, dict]:
    ph = pet_phantom(seed)
    gs = phantom_fitted_gaussians(ph, n, seed=4000 + seed, box_lo=(-250, -250, -60),
                                  box_hi=(250, 250, 60))
    return gs, geom_c3(n_angles, n_radial, n_planes)


def phantom_gaussians_mixture(ph: dict, n: int, seed: int, log_sigma_std: float = 0.3) -> dict:
    """The recipe of phantom_fitted_gaussians without rejection sampling (for
    large counts): the additive density is a mixture of uniform ellipsoids
    with weights density x volume, so centres are drawn by picking an
    ellipsoid with that probability and a uniform point inside it.  The
    support volume (union of the ellipsoids) is sum_k vol_k E_k[1/cover(x)],
    cover(x) = number of ellipsoids holding x, estimated from 4096 points
    per ellipsoid."""
    rng = np.random.default_rng(seed)
    axes, rot, centre, dens = ph["axes"], ph["rot"], ph["centre"], ph["density"]
    k = axes.shape[0]
    vol = 4.0 / 3.0 * math.pi * np.prod(axes, axis=1)

    def inside_points(idx):
        m = idx.size
        d = rng.normal(size=(m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        r = rng.uniform(0.0, 1.0, m) ** (1.0 / 3.0)
        local = d * r[:, None] * axes[idx]
        return centre[idx] + np.einsum("nij,nj->ni", rot[idx], local)

    v_union = 0.0
    for e in range(k):
        x = inside_points(np.full(4096, e))
        cover = np.zeros(x.shape[0])
        for a, r, c in zip(axes, rot, centre):
            cover += np.sum((((x - c) @ r) / a) ** 2, axis=1) <= 1.0
        v_union += vol[e] * float(np.mean(1.0 / np.maximum(cover, 1.0)))
    h = (v_union / n) ** (1.0 / 3.0)
    w = dens * vol
    which = rng.choice(k, size=n, p=w / w.sum())
    mu = inside_points(which)
    ls = rng.normal(math.log(h), log_sigma_std, size=(n, 3))
    q = _random_quaternions(rng, n)
    rho = _phantom_density(ph, mu) * h ** 3 / ((2.0 * math.pi) ** 1.5 * np.exp(ls.sum(axis=1)))
    return dict(mu=mu.astype(np.float32), ls=ls.astype(np.float32), q=q,
                rho=rho.astype(np.float32), h=h)


def perturbed(gs: dict, seed: int, pos_std: float, ls_std: float = 0.05) -> dict:
    """A second Gaussian set near gs (same count): the 'measured object'
    whose projections serve as data when fitting gs."""
    rng = np.random.default_rng(seed)
    mu = gs["mu"] + rng.normal(0, pos_std, gs["mu"].shape).astype(np.float32)
    ls = gs["ls"] + rng.normal(0, ls_std, gs["ls"].shape).astype(np.float32)
    q = _random_quaternions(rng, gs["q"].shape[0])
    rho = gs["rho"] * rng.uniform(0.8, 1.2, gs["rho"].shape).astype(np.float32)
    return dict(mu=mu.astype(np.float32), ls=ls.astype(np.float32), q=q, rho=rho.astype(np.float32))


def random_weights(n_rays: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Per-ray adjoint weights (dL/dI) for parity checks of the adjoint."""
    rng = np.random.default_rng(seed)
    return (scale * rng.normal(size=n_rays)).astype(np.float32)
