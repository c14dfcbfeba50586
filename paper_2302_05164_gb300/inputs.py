"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only describes workloads: mesh descriptors, material constants, laser paths and
seeded random fields. It holds none of the method's arithmetic, so both the CUDA path and the
oracle can take their inputs from it without sharing any computation.

Workloads (synthetic stand-ins shaped like the paper's; no paper dataset is used):
  c1  uniform Q1 brick 64x32x16 cells on 1.0x0.5x0.25 mm, constant Ti-6Al-4V-like material,
      one scan track (y = 0.25 mm, +x at 0.8 m/s), Dirichlet bottom.
  c2  Q2 octree mesh on 2x2x1 mm (40 um trees, 3 levels -> 5 um cells) refined inside a
      150 um ball around the laser spot, nonlinear k(T) and apparent capacity, 10 serpentine
      hatch tracks at 100 um spacing, v = 1 m/s.
  c3  the c1 brick with an extra tree row above it, used for a newly activated powder layer
      of three cells (46.875 um) and an implicit cool-down.
  c4  Q2 brick 1.0x0.5x0.25 mm refined to 7.8 um within a distance of the scan line,
      16 laser-power segments and a conductivity scale per instance.
Material constants of the paper's bridge example (Table mat_params) are given as BRIDGE.
"""
from __future__ import annotations

import numpy as np

# region kinds
BALL = 0
BOX = 1

DIRICHLET_BOTTOM = 1 << 4

# ---------------------------------------------------------------------------------------
# materials: rho, c, conductivity ramp (k0 at Tk0 .. k1 at Tk1), latent heat Gaussian
# (latent, Tm, sigma; sigma = 0 disables it), powder conductivity factor, Dirichlet value,
# and T_ref, the offset the FP32 operator subtracts before rounding.
# ---------------------------------------------------------------------------------------

TI64_CONST = dict(rho=4430.0, c=526.0, k0=6.7, k1=6.7, Tk0=300.0, Tk1=300.0,
                  latent=0.0, Tm=1903.0, sigma=0.0, powder_k_scale=0.1,
                  T_dirichlet=353.0, T_ref=353.0)

LUMP_QUADRATURE = 0  # row sum of the consistent capacity, c_app at quadrature points
LUMP_NODAL = 1       # c_app at the node times the row-sum lumped mass (positive for Q2)

TI64_NONLIN = dict(rho=4430.0, c=526.0, k0=6.7, k1=28.0, Tk0=300.0, Tk1=1928.0,
                   latent=2.86e5, Tm=1903.0, sigma=12.5, powder_k_scale=0.1,
                   T_dirichlet=353.0, T_ref=353.0, lumping=LUMP_QUADRATURE)

# the Q2 workloads: nodal apparent capacity (see LUMP_NODAL)
TI64_NONLIN_Q2 = dict(TI64_NONLIN, lumping=LUMP_NODAL)

# Paper, Table mat_params (stainless steel, bridge example): k = 20, rho = 7430, c = 965
BRIDGE = dict(rho=7430.0, c=965.0, k0=20.0, k1=20.0, Tk0=303.0, Tk1=303.0,
              latent=0.0, Tm=1700.0, sigma=0.0, powder_k_scale=0.01,
              T_dirichlet=303.0, T_ref=303.0)

T0 = 353.0

# Phase-dependent conductivity with history (Eqs. liquid_fraction .. material_parameter_interp)
# with the paper's material table (Sec. 5.1): solidus 1500 K, liquidus 1900 K, powder 0.2 W/mK,
# melt and solid 20 W/mK.
PHASE = dict(T_s=1500.0, T_l=1900.0, k_p=0.2, k_m=20.0, k_s=20.0)

# Radiation and evaporation on the free top surface (Eqs. bc_radiation, bc_evaporation) with
# the constants of the paper's material table (Sec. 5.1): emissivity 0.7, boiling point
# 3000 K, C_P = 54 kPa, C_T = 50,000 K, C_M = 0.001 K s^2/m^2, latent heat of evaporation
# 6.0 MJ/kg, enthalpy reference 663 K, [T] capped at T_v + 1000 K; the ambient temperature and
# the heat capacity of the enthalpy term follow the Ti-6Al-4V-like workloads (353 K, 526 J/kgK).
SURFACE_LOSS = dict(emissivity=0.7, T_amb=T0, C_P=54.0e3, C_T=5.0e4, C_M=1.0e-3, T_v=3000.0, h_v=6.0e6, c_h=526.0,
                    T_h0=663.0, T_max=4000.0)


def mesh_desc(ntree, tree_h, degree, max_level, regions=(), origin=(0.0, 0.0, 0.0),
              active_top_z=1e30, dirichlet_faces=DIRICHLET_BOTTOM, tree_exists=None,
              powder_z0=1e30, powder_z1=1e30):
    """Plain dict describing a forest of axis-aligned octrees on a brick of trees.

    regions: sequence of (kind, a[3], b[3], radius, level). A leaf is refined to `level`
    when its box lies closer than `radius` to the region core (a point for BALL, the box
    [a, b] for BOX)."""
    return dict(origin=tuple(float(v) for v in origin), ntree=tuple(int(v) for v in ntree),
                tree_h=tuple(float(v) for v in tree_h), degree=int(degree),
                max_level=int(max_level),
                regions=[(int(k), tuple(map(float, a)), tuple(map(float, b)), float(r), int(lv))
                         for (k, a, b, r, lv) in regions],
                active_top_z=float(active_top_z), dirichlet_faces=int(dirichlet_faces),
                tree_exists=None if tree_exists is None else np.ascontiguousarray(tree_exists, np.uint8),
                powder_z0=float(powder_z0), powder_z1=float(powder_z1))


def uniform_region(level, big=1e6):
    """A box region covering any domain, refining every leaf to `level`."""
    return (BOX, (-big, -big, -big), (big, big, big), 1e-9, level)


def laser(segments, power, eta=0.35, radius=40e-6, volumetric=False, h_powder=40e-6):
    """segments [n][6] = (x0, y0, x1, y1, t0, t1); power [n] or [batch][n] in W."""
    return dict(seg=np.ascontiguousarray(segments, np.float64),
                power=np.ascontiguousarray(power, np.float64), eta=float(eta),
                radius=float(radius), volumetric=int(bool(volumetric)), h_powder=float(h_powder))


def track(x0, y, x1, v, t0=0.0):
    return (x0, y, x1, y, t0, t0 + abs(x1 - x0) / v)


# ---------------------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------------------

def c1_mesh(ntree_z=4, active_top_z=1e30):
    return mesh_desc((16, 8, ntree_z), (62.5e-6,) * 3, 1, 2, [uniform_region(2)],
                     active_top_z=active_top_z)


def c1_laser(power=200.0):
    return laser([track(0.0, 0.25e-3, 1.0e-3, 0.8)], [power], eta=0.35, radius=40e-6)


def c2_spot_regions(x, y, z_top=1.0e-3, radius=150e-6, level=3):
    return [(BALL, (x, y, z_top), (x, y, z_top), radius, level)]


def c2_mesh(spot=(0.5e-3, 0.55e-3)):
    return mesh_desc((50, 50, 25), (40e-6,) * 3, 2, 3, c2_spot_regions(*spot))


def c2_laser(power=200.0, v=1.0, n_tracks=10):
    segs, t = [], 0.0
    for k in range(n_tracks):
        y = 0.55e-3 + 1e-4 * k
        a, b = (0.5e-3, 1.5e-3) if k % 2 == 0 else (1.5e-3, 0.5e-3)
        segs.append(track(a, y, b, v, t))
        t = segs[-1][5]
    return laser(segs, [power] * n_tracks, eta=0.35, radius=40e-6)


def c3_mesh(active_top_z=0.25e-3):
    """c1 brick plus one more tree row; cells above active_top_z are inactive."""
    return c1_mesh(ntree_z=5, active_top_z=active_top_z)


C3_LAYER_TOP = 0.25e-3 + 3 * 15.625e-6


def c4_mesh(radius=80e-6):
    line = (BOX, (0.0, 0.25e-3, 0.25e-3), (1.0e-3, 0.25e-3, 0.25e-3), radius, 3)
    return mesh_desc((16, 8, 4), (62.5e-6,) * 3, 2, 3, [uniform_region(1), line])


def c4_laser(powers, v=0.8, n_seg=16, steps_per_seg=125, dt=None, y=0.25e-3):
    """Single track split into n_seg pieces of equal duration; powers [batch][n_seg]."""
    powers = np.atleast_2d(np.asarray(powers, np.float64))
    if dt is None:
        seg_len = 1.0e-3 / n_seg
        segs = [track(k * seg_len, y, (k + 1) * seg_len, v, k * seg_len / v) for k in range(n_seg)]
    else:
        dur = steps_per_seg * dt
        segs = [(v * k * dur, y, v * (k + 1) * dur, y, k * dur, (k + 1) * dur) for k in range(n_seg)]
    return laser(segs, powers, eta=0.35, radius=40e-6)


C5_TREE_H = (0.625e-3, 0.625e-3, 0.64e-3)
C5_BASE_TOP = 3 * C5_TREE_H[2]        # baseplate: three tree layers, 1.92 mm
C5_LAYER = 40e-6
C5_RIBS_X = (1, 3, 6, 9, 12, 14)      # tree columns of the 12 support ribs (6 x 2 pillars)
C5_RIBS_Y = (2, 5)


def c5_mesh(layer=1, level=5, haz_layers=4, degree=2):
    """Synthetic cantilever-like part on a baseplate (a stand-in for the part-scale build of
    configuration 5): trees of 0.625 x 0.625 x 0.64 mm, 16 x 8 footprint (10 x 5 mm), three
    tree layers of baseplate (1.92 mm) and two of build chamber; in the chamber only the 12
    rib pillars (one tree each) exist. Layer `layer` of 40 um is active and is powder; the
    layer and `haz_layers` layers below it (the heat-affected zone, 4 x 40 um as in the paper)
    are refined to `level` (level 4: 39 x 39 x 40 um cells, one per layer; level 5: two), with
    2:1 grading below. Dirichlet bottom."""
    nt = (16, 8, 5)
    exists = np.zeros(nt[::-1], np.uint8)
    exists[:3] = 1
    for x in C5_RIBS_X:
        for y in C5_RIBS_Y:
            exists[3:, y, x] = 1
    top = C5_BASE_TOP + layer * C5_LAYER
    lo = top - (1 + haz_layers) * C5_LAYER
    region = (BOX, (0.0, 0.0, lo), (nt[0] * C5_TREE_H[0], nt[1] * C5_TREE_H[1], top), 1e-9, level)
    return mesh_desc(nt, C5_TREE_H, degree, level, [region], active_top_z=top, tree_exists=exists,
                     powder_z0=top - C5_LAYER, powder_z1=top)


def c5_laser(layer=1, rib=(0, 0), power=180.0, v=0.9, spacing=90e-6, angle_deg=67.0):
    """Hatch of one rib's cross-section in layer `layer` of the part-scale stand-in: parallel
    tracks at `spacing`, rotated by angle_deg x layer, clipped to the rib's square (tree
    column C5_RIBS_X[rib[0]], row C5_RIBS_Y[rib[1]]), scanned back and forth at speed v."""
    th = np.deg2rad(angle_deg * layer)
    u = np.array([np.cos(th), np.sin(th)])
    nv = np.array([-u[1], u[0]])
    x0 = C5_RIBS_X[rib[0]] * C5_TREE_H[0]
    y0 = C5_RIBS_Y[rib[1]] * C5_TREE_H[1]
    lo = np.array([x0, y0])
    hi = lo + np.array(C5_TREE_H[:2])
    c = 0.5 * (lo + hi)
    half = 0.5 * np.hypot(*C5_TREE_H[:2])
    segs, t, k = [], 0.0, 0
    for o in np.arange(-half, half, spacing):
        p = c + o * nv
        smin, smax = -np.inf, np.inf
        for d in range(2):  # slab clipping of the line p + s u to the square
            if abs(u[d]) < 1e-15:
                if not lo[d] <= p[d] <= hi[d]:
                    smin, smax = 1.0, 0.0
                continue
            a, b = (lo[d] - p[d]) / u[d], (hi[d] - p[d]) / u[d]
            smin, smax = max(smin, min(a, b)), min(smax, max(a, b))
        if smax - smin < 1e-6:
            continue
        a, b = p + smin * u, p + smax * u
        if k % 2:
            a, b = b, a
        dur = np.hypot(*(b - a)) / v
        segs.append((a[0], a[1], b[0], b[1], t, t + dur))
        t += dur
        k += 1
    return laser(segs[:kMaxSegC5], [power] * min(len(segs), kMaxSegC5), eta=0.35, radius=40e-6)


kMaxSegC5 = 64  # the library takes at most 64 laser segments per call


def c4_params(batch, n_seg=16, seed=2302):
    """Per-instance laser powers P ~ U[150, 250] W and conductivity scales s ~ U[0.8, 1.2]."""
    rng = np.random.default_rng(seed)
    P = rng.uniform(150.0, 250.0, size=(batch, n_seg))
    s = rng.uniform(0.8, 1.2, size=batch)
    return P, s


# ---------------------------------------------------------------------------------------
# seeded fields
# ---------------------------------------------------------------------------------------

def random_field(n, seed, lo=T0, hi=2600.0, batch=None):
    rng = np.random.default_rng(seed)
    shape = (n,) if batch is None else (n, batch)
    return rng.uniform(lo, hi, size=shape)


def smooth_field(coords, seed, lo=T0, hi=2600.0, batch=None):
    """Smooth seeded temperature field from dof coordinates (physical units, [n][3]):
    a sum of a few random Gaussian bumps, clipped to [lo, hi]."""
    rng = np.random.default_rng(seed)
    nb = 1 if batch is None else batch
    out = np.empty((coords.shape[0], nb))
    ext = coords.max(axis=0) - coords.min(axis=0) + 1e-12
    for b in range(nb):
        v = np.full(coords.shape[0], lo)
        for _ in range(4):
            c = coords.min(axis=0) + rng.uniform(0, 1, 3) * ext
            w = rng.uniform(0.1, 0.4) * ext.max()
            amp = rng.uniform(0.3, 1.0) * (hi - lo)
            d2 = ((coords - c) ** 2).sum(axis=1)
            v = v + amp * np.exp(-d2 / (w * w))
        out[:, b] = np.clip(v, lo, hi)
    return out[:, 0] if batch is None else out


def melt_pool_field(coords, center, peak=2600.0, width=50e-6, base=T0, seed=None, noise=0.0):
    """Melt-pool-shaped temperature: base + (peak - base) exp(-|x - center|^2 / width^2), with
    optional seeded noise of relative amplitude `noise` (coords physical, [n][3])."""
    d2 = ((np.asarray(coords) - np.asarray(center)) ** 2).sum(axis=1)
    T = base + (peak - base) * np.exp(-d2 / (width * width))
    if noise:
        rng = np.random.default_rng(seed)
        T = T * (1.0 + noise * rng.uniform(-1, 1, T.shape))
    return T


def start_vector(n, seed=7):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=n)


# ---------------------------------------------------------------------------------------
# temporal-convergence experiment (Appendix A): a 1.0 x 0.2 x 0.2 mm plate with two powder
# layers of 40 um, one track per layer along +x through the middle of the plate's width, the
# explicit scan, an interlayer cool-down (explicit, then implicit) and the second layer.
# Material and loss constants are the paper's (Table mat_params: phase model, radiation and
# evaporation, T_0 = T_inf = 303 K; no latent heat), the scan speed and beam radius those of
# the cantilever (Table scan_params_cantilever: 960 mm/s, R = 60 um) with the paper's
# cylinder source. The paper states no power: W_eff = 100 W is a reading.
# ---------------------------------------------------------------------------------------

APPA_T0 = 303.0
APPA_PLATE_TOP = 0.2e-3
APPA_LAYER = 40e-6
APPA_MATERIAL = dict(rho=7430.0, c=965.0, k0=20.0, k1=20.0, Tk0=303.0, Tk1=303.0, latent=0.0, Tm=1700.0,
                     sigma=0.0, powder_k_scale=0.01, T_dirichlet=APPA_T0, T_ref=APPA_T0)
APPA_PHASE = dict(T_s=1500.0, T_l=1900.0, k_p=0.2, k_m=20.0, k_s=20.0)
APPA_LOSS = dict(emissivity=0.7, T_amb=APPA_T0, C_P=54.0e3, C_T=5.0e4, C_M=1.0e-3, T_v=3000.0, h_v=6.0e6,
                 c_h=965.0, T_h0=663.0, T_max=4000.0)
APPA_OBS = (0.5e-3, 0.0, APPA_PLATE_TOP + APPA_LAYER)  # top of the first layer, middle of the track
APPA_DT_EXPLICIT = 2e-5  # the paper's reference steps
APPA_DT_IMPLICIT = 2e-2
APPA_COOL = 0.06  # s between the layers
APPA_COOL_EXPLICIT = 0.02  # s of it (1000 reference steps) explicit, as in the paper's examples


def appa_mesh(layers=1):
    """Q1 trees of 40 um (25 x 5 x 7 on y in [-0.1, 0.1] mm), refined once (20 um cells);
    `layers` powder layers active; Dirichlet bottom."""
    return mesh_desc((25, 5, 7), (40e-6,) * 3, 1, 1, [uniform_region(1)], origin=(0.0, -0.1e-3, 0.0),
                     active_top_z=APPA_PLATE_TOP + layers * APPA_LAYER, powder_z0=APPA_PLATE_TOP,
                     powder_z1=APPA_PLATE_TOP + 2 * APPA_LAYER)


def appa_laser(t0=0.0, power=200.0, eta=0.5, v=0.96):
    """The track of one layer (x from 0 to 1 mm at y = 0) starting at t0; W_eff = eta P."""
    return laser([track(0.0, 0.0, 1.0e-3, v, t0)], [power], eta=eta, radius=60e-6, volumetric=True,
                 h_powder=APPA_LAYER)
