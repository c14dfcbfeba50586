"""The temporal-convergence experiment of the paper's Appendix A, run through the library's
public API: a plate with two powder layers, one track per layer, the combined scheme of
Sec. 3.2 (forward Euler while the laser scans and for the first part of the interlayer
cool-down, backward Euler by Newton's method for the rest of it), the activation of the
second layer with the state and the consolidation history moved to the grown mesh, and the
temperature at the observation point (0.5, 0.0, 0.24) mm, for the reference step sizes
scaled by `dt_scale` (the paper compares dt_ref, dt_ref / 2 and dt_ref / 4).

The workload (geometry, material, loss constants, laser) is `inputs.appa_*`.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I

SCAN_STEPS_REF = 52      # 1 mm at 0.96 m/s in steps of 2e-5 s
COOL_EXPLICIT_REF = 1000  # explicit reference steps at the start of the cool-down
COOL_IMPLICIT_REF = 2     # implicit reference steps (2e-2 s) for the rest of it


def _obs_index(tables, desc):
    xyz = np.array(desc["origin"]) + np.array(desc["tree_h"]) * tables["dof_coord"] / (
        desc["degree"] * 2.0 ** desc["max_level"])
    hit = np.where(np.all(np.isclose(xyz, I.APPA_OBS, rtol=0.0, atol=1e-12), axis=1))[0]
    assert len(hit) == 1
    return int(hit[0])


def run(pbf, torch, dt_scale=1.0, precision=None, newton_rtol=1e-10, cheb_bounds=(None, None), stream=None):
    """Returns {"t": times, "T": temperatures at the observation point} sampled after every
    step of the scans and of the cool-down's implicit part and every 50 reference steps of its
    explicit part, plus the final fields, the Newton iteration counts and the step sizes.
    cheb_bounds: the Chebyshev bounds of the implicit steps on the first and the second mesh
    (None: estimated by the library)."""
    precision = pbf.PBF_F64 if precision is None else precision
    k = int(round(1.0 / dt_scale))
    assert abs(k * dt_scale - 1.0) < 1e-12, "dt_scale must be 1 / integer"
    dte, dti = I.APPA_DT_EXPLICIT * dt_scale, I.APPA_DT_IMPLICIT * dt_scale
    mat = I.APPA_MATERIAL
    desc1 = I.appa_mesh(1)
    mesh = pbf.Mesh(desc1)

    def context():
        ctx = pbf.Context(mesh, mat, precision)
        pbf.pbf_ctx_set_phase(ctx.h, I.APPA_PHASE)
        pbf.pbf_ctx_set_surface_loss(ctx.h, I.APPA_LOSS)
        return ctx

    ctx = context()
    obs = _obs_index(mesh.tables(), desc1)
    n = mesh.info()["n_dofs"]
    T = torch.full((n,), I.APPA_T0, dtype=torch.float64, device="cuda")
    times, temps, newton = [0.0], [I.APPA_T0], []
    t = 0.0

    def sample():
        times.append(t)
        temps.append(float(T[obs].item()))

    def scan(ls):
        nonlocal t
        for _ in range(SCAN_STEPS_REF * k):
            pbf.pbf_explicit_step(ctx.h, T, ls, t, dte, 1, stream=stream)
            t += dte
            sample()

    def cool(bounds):
        nonlocal t
        chunk = 50 * k
        for _ in range(COOL_EXPLICIT_REF // 50):
            pbf.pbf_explicit_step(ctx.h, T, None, t, dte, chunk, stream=stream)
            t += chunk * dte
            sample()
        for _ in range(COOL_IMPLICIT_REF * k):
            st, nit, lit, rel = pbf.pbf_implicit_newton(ctx.h, T, dti, 1, newton_rtol, 30, 1e-4, 2000, 5,
                                                        None if bounds is None else np.asarray(bounds), stream=stream)
            assert st == 0, ("Newton did not converge", rel)
            newton.append((int(nit[0]), int(lit[0])))
            t += dti
            sample()

    scan(I.appa_laser(t0=t))
    cool(cheb_bounds[0])
    # the second layer: activation, the state and the history on the grown mesh
    pbf.pbf_mesh_activate_layer(mesh.h, I.APPA_PLATE_TOP + 2 * I.APPA_LAYER, 1, I.APPA_T0)
    T2 = torch.empty(mesh.info()["n_dofs"], dtype=torch.float64, device="cuda")
    pbf.pbf_mesh_transfer(mesh.h, T, T2, stream=stream)
    ctx2 = context()
    pbf.pbf_ctx_transfer_history(ctx.h, ctx2.h, stream=stream)
    ctx.close()
    ctx, T = ctx2, T2
    layer1_end = len(times)
    scan(I.appa_laser(t0=t))
    out = {"t": np.array(times), "T": np.array(temps), "layer2_from": layer1_end, "newton": newton,
           "dt_explicit": dte, "dt_implicit": dti, "T_final": T.cpu().numpy()}
    ctx.close()
    mesh.close()
    return out


def common_samples(coarse, fine, k):
    """The fine run's samples at the coarse run's sample times (the fine run samples k times
    as often in the scans and the implicit steps, equally often in the explicit cool-down)."""
    idx, j = [], 0
    tf = fine["t"]
    for tc in coarse["t"]:
        while j < len(tf) and tf[j] < tc - 1e-12 * max(1.0, abs(tc)):
            j += 1
        assert j < len(tf) and abs(tf[j] - tc) <= 1e-9 * max(1.0, abs(tc)), (tc, tf[j] if j < len(tf) else None)
        idx.append(j)
    return fine["T"][np.array(idx)]
