"""Benchmark of the explicit hot path on the adaptive Q2 multi-track workload.

Workload C2: Q2 octree mesh on a 2 x 2 x 1 mm block (40 um trees,
3 refinement levels -> 5 um cells inside a 150 um ball around the laser spot, 2:1 balanced
with hanging nodes; 1,066,531 dofs, 132,423 cells), k(T) linear 6.7 -> 28 W/mK over
300-1928 K, apparent capacity with latent heat 2.86e5 J/kg (Gaussian around 1903 K, nodal
lumping), surface
Gaussian laser (P = 200 W, eta = 0.35, r = 40 um, v = 1 m/s, serpentine tracks), forward
Euler at half the CFL bound. Synthetic seeded initial field: a 2600 K melt pool (50 um) at the
spot on a 353 K part, 1% seeded noise.

One benchmark step = 50 explicit time steps (the re-adaptation interval of the workload) on
the resident mesh. value = dof-updates per second over all ranks (GDoF/s). Between timed
steps the L2 cache is flushed by writing a 256 MB buffer (the working set would otherwise stay
in the 129 MB L2); each step is timed with CUDA events on the stream the kernels run on.

--impl reference runs the repository's serial FP64 oracle on the host cores instead (a
bounded sample of the same workload per step) and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "explicit-step DoF-updates/s (GDoF/s) and % HBM roofline, FP32-op vs FP64 at stated error"
WORKLOAD = "C2: Q2 AMR 2x2x1 mm, 5 um cells in a 150 um ball, 1.07M dofs, nonlinear k(T) + latent heat"
CHUNK = 50                 # explicit steps per benchmark step
SHAPES = ["per-cell kernel, 128 threads", "per-cell kernel, 128 threads, 5 blocks/SM",
          "per-cell kernel, 128 threads, 6 blocks/SM", "per-cell kernel, 64 threads, 10 blocks/SM",
          "fused step, 64-cell patches", "fused step, 64-cell patches, programmatic dependent launch",
          "fused steps, one persistent cooperative launch per call",
          "lean fused step (tables through L1), 14 blocks/SM", "lean fused step (tables through L1), 12 blocks/SM",
          "lean fused step (tables through L1), 10 blocks/SM"]
KERNELS = ["k_cell<2,float,RESIDUAL,nonlinear>"] * 4 + ["k_step<2,nonlinear,nodal> (fused step)"] * 2 + \
    ["k_steps<2,nonlinear,nodal> (persistent fused steps)"] + \
    [f"k_step_lean<2,nonlinear,nodal,{b}> (lean fused step)" for b in (14, 12, 10)]
BYTES_PER_DOF_UPDATE = 16  # read T_n and write T_{n+1} in FP64 (c_app(T) recomputed in-kernel)


def flops_per_cell_q2_nonlinear():
    """Floating-point operations of one cell in the FP32 cell kernel (FMA = 2), counted from
    its arithmetic: 1D passes over the 3 x 3 x 3 tensor with the nonzeros of the Gauss-point
    tables (S: 7 per line, D: 8 per line), plus the pointwise quadrature-point work. The
    apparent capacity of the workload is nodal (evaluated in the update, not in this kernel)."""
    lines = 9
    s_pass = lines * 7 * 2
    d_pass = lines * 8 * 2
    passes = 3 * s_pass                    # values at quadrature points
    passes += 3 * (d_pass + d_pass)        # gradient and its transpose, three directions
    passes += 3 * s_pass                   # final integration
    pointwise = 27 * (5 + 6)               # k(T), metric scaling
    return passes + pointwise


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_ms=50):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []  # (host time of arrival, line)
        self.window = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def wait_first(self, timeout=5.0):
        """Blocks until the sampler has printed its first line (the process is up)."""
        t0 = time.perf_counter()
        while self.proc and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)

    def mark(self, t_begin, t_end):
        """The host-time window of the timed region."""
        self.window = (t_begin, t_end)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        """Median SM clock and the throttle reasons of the samples taken inside the timed
        window; when the window is shorter than a few sampling periods, the samples of the
        whole sampled span (warm-up included, the same kernels) are reported beside them."""
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        rows = []
        for t, ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm, mx = float(parts[0]), float(parts[1])
            except ValueError:
                continue
            rows.append((t, sm, mx, {n for n, v in zip(names, parts[3:7]) if v.lower() in ("active", "1")}))

        def agg(rs):
            return {"sm_mhz": float(np.median([r[1] for r in rs])) if rs else None,
                    "sm_max_mhz": max([r[2] for r in rs], default=0.0) or None,
                    "reasons": sorted(set().union(*[r[3] for r in rs])) if rs else [], "samples": len(rs)}

        inside = [r for r in rows if self.window and self.window[0] <= r[0] <= self.window[1] + 0.5 * self.period_ms / 1e3]
        out = agg(inside if inside else rows)
        out["sampling_ms"] = self.period_ms
        if self.window:
            out["timed_window_ms"] = round(1e3 * (self.window[1] - self.window[0]), 1)
        if len(inside) < 3:
            out["sampled_span"] = agg(rows)
            out["note"] = ("fewer than 3 samples fell inside the timed window; sampled_span covers the warm-up and "
                           "timed steps around it (the same kernels)")
        return out


def c2_initial(I, xyz, rank=0):
    """The workload's initial field: a 2600 K melt pool (50 um) at the spot on a 353 K part,
    1% seeded noise (seed 21 + rank)."""
    return I.melt_pool_field(xyz, (0.5e-3, 0.55e-3, 1.0e-3), 2600.0, 50e-6, seed=21 + rank, noise=0.01)


def oracle_dt(I, O):
    """Half the critical explicit step of the finest cells (Eq. explicit_time_step): the
    oracle's power iteration on a block of 5 um Q2 cells with the largest conductivity."""
    ob = O.Mesh(I.mesh_desc((1, 1, 1), (40e-6,) * 3, 2, 3, [I.uniform_region(3)], dirichlet_faces=0))
    lam, _ = ob.lambda_max(dict(I.TI64_NONLIN_Q2, k0=28.0), I.start_vector(ob.n_dofs), max_iter=300, rtol=1e-8)
    return 0.5 * 2.0 / lam


def time_oracle(steps, max_seconds=None):
    """Serial FP64 oracle explicit steps of the full workload (C2 mesh, initial field, laser and
    material) at the oracle's own half-critical step. Returns (dof-updates/s, n_dofs, steps
    done, seconds, T after the steps, T_0, dt)."""
    from oracle import oracle as O
    from paper_2302_05164_gb300 import inputs as I
    O.build()
    m = O.Mesh(I.c2_mesh())
    T0 = c2_initial(I, m.dof_xyz())
    ls = I.c2_laser()
    dt = oracle_dt(I, O)
    T = T0
    done, t0 = 0, time.perf_counter()
    for k in range(steps):
        T = m.explicit(I.TI64_NONLIN_Q2, T, ls, k * dt, dt, 1)
        done += 1
        if max_seconds and time.perf_counter() - t0 > max_seconds:
            break
    el = time.perf_counter() - t0
    return m.n_dofs * done / el, m.n_dofs, done, el, T, T0, dt


def bench_batched(pbf, I, torch, stream, flush, peaks, K, batch=64, chunk=50, shape=-1):
    """Configuration 4 forward steps: Q2 brick refined to 7.8 um along the track (278,581 dofs),
    64 instances with their own segment powers and conductivity scales, one launch per kernel
    for all instances, 50 explicit steps per call (as C2). The state (143 MB per vector)
    exceeds the L2."""
    desc = I.c4_mesh()
    mat = I.TI64_NONLIN_Q2
    mesh = pbf.Mesh(desc)
    n = mesh.info()["n_dofs"]
    P, s = I.c4_params(batch)
    ls = I.c4_laser(P, n_seg=16, steps_per_seg=125, dt=2e-8)
    ctx = pbf.Context(mesh, mat, pbf.PBF_F32OP, batch)
    pbf.pbf_ctx_set_k_scale(ctx.h, s)
    tab = mesh.tables()
    xyz = np.array(desc["origin"]) + np.array(desc["tree_h"]) * tab["dof_coord"] / (2 * 2.0 ** desc["max_level"])
    T0 = I.melt_pool_field(xyz, (0.05e-3, 0.25e-3, 0.25e-3), 2500.0, 50e-6, seed=5)
    T = torch.tensor(np.repeat(T0[:, None], batch, axis=1), dtype=torch.float64, device="cuda")
    dt = 2e-8
    shape_us = [-1.0] * len(SHAPES)
    if shape >= 0:
        variant = shape
        pbf.pbf_ctx_set_kernel_shape(ctx.h, shape)
    else:
        variant, shape_us = pbf.pbf_ctx_autotune(ctx.h, T, reps=3, stream=stream, times=True)
    for k in range(3):
        pbf.pbf_explicit_step(ctx.h, T, ls, k * chunk * dt, dt, chunk, batch=batch, stream=stream)
    K = max(1, min(K, 2000 // chunk - 3))  # warm-up and timed steps within the 2,000-step scan
    pbf.pbf_ctx_kernel_time(ctx.h)
    pbf.pbf_ctx_set_timing(ctx.h, True)
    torch.cuda.synchronize()
    ms = 0.0
    for k in range(K):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pbf.pbf_explicit_step(ctx.h, T, ls, (3 + k) * chunk * dt, dt, chunk, batch=batch, stream=stream)
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    pbf.pbf_ctx_set_timing(ctx.h, False)
    cell_ms, cell_n = pbf.pbf_ctx_kernel_time(ctx.h)
    rate = n * batch * chunk * K / (ms * 1e-3) / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)
    n_cells = mesh.info()["n_active"]
    cell_us = 1e3 * cell_ms / max(cell_n, 1)
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    cell_tflops = flops_per_cell_q2_nonlinear() * n_cells * batch / (cell_us * 1e-6) / 1e12
    meta = metadata_bytes(pbf, mesh, False, batch)  # both batched forms read the per-cell tables
    ctx.close()
    mesh.close()
    return {"workload": f"C4: Q2 1.0x0.5x0.25 mm, {n} dofs x {batch} instances (own powers and k scales)",
            "value": rate, "unit": "GDoF/s", "explicit_steps_per_step": chunk, "steps": K,
            "cell_kernel_avg_us": cell_us, "step_shape": SHAPES[variant] if variant < 4 else "batched fused step",
            "autotune_us_per_step": {("batched fused step" if i == 4 else SHAPES[i]): round(u, 2)
                                     for i, u in enumerate(shape_us) if u > 0},
            "cell_kernel_roofline": {"bound": "alu", "achieved": cell_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                                     "frac": cell_tflops / fp32_peak, "cells_x_instances": n_cells * batch},
            "hbm_fraction": rate * BYTES_PER_DOF_UPDATE / hbm, "l2": "state > L2; flushed between timed steps",
            "metadata": meta}


def bench_large(pbf, I, torch, stream, flush, peaks, K=5, chunk=20):
    """The C2 block and material with a 500 um refinement ball (5 um cells): 2.29 M cells,
    18.2 M dofs, one instance. Its state and tables (about 0.7 GB) exceed the L2, so the fused
    step runs from HBM over about 24 waves of patches instead of 1.4."""
    desc = I.mesh_desc((50, 50, 25), (40e-6,) * 3, 2, 3, I.c2_spot_regions(1.0e-3, 1.0e-3, radius=500e-6))
    mat = I.TI64_NONLIN_Q2
    t0 = time.perf_counter()
    mesh = pbf.Mesh(desc)
    info = mesh.info()
    n = info["n_dofs"]
    tab = mesh.tables()
    xyz = np.array(desc["origin"]) + np.array(desc["tree_h"]) * tab["dof_coord"] / (2 * 2.0 ** desc["max_level"])
    T0 = I.melt_pool_field(xyz, (1.0e-3, 1.0e-3, 1.0e-3), 2600.0, 50e-6, seed=23, noise=0.01)
    ls = I.laser([(0.6e-3, 1.0e-3, 1.4e-3, 1.0e-3, 0.0, 4e-4)], [200.0], eta=0.35, radius=40e-6)
    ctx = pbf.Context(mesh, mat, pbf.PBF_F32OP)
    setup_s = time.perf_counter() - t0
    T = torch.tensor(T0, dtype=torch.float64, device="cuda")
    dt = 2e-8
    variant, shape_us = pbf.pbf_ctx_autotune(ctx.h, T, reps=3, stream=stream, times=True)
    for k in range(2):
        pbf.pbf_explicit_step(ctx.h, T, ls, k * chunk * dt, dt, chunk, stream=stream)
    torch.cuda.synchronize()
    ms = 0.0
    for k in range(K):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pbf.pbf_explicit_step(ctx.h, T, ls, (2 + k) * chunk * dt, dt, chunk, stream=stream)
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    rate = n * chunk * K / (ms * 1e-3) / 1e9
    ok = bool(torch.isfinite(T).all().item())
    meta = metadata_bytes(pbf, mesh, variant >= 4)
    ctx.close()
    mesh.close()
    out = {"workload": f"C2 block and material, 500 um refinement ball: {info['n_active']} cells, {n} dofs, one instance",
           "value": rate, "unit": "GDoF/s", "us_per_explicit_step": 1e3 * ms / (K * chunk), "step_shape": SHAPES[variant],
           "hbm_fraction": rate * BYTES_PER_DOF_UPDATE / peaks.get("hbm_gbs", 6800.0), "finite": ok,
           "host_setup_s": setup_s, "l2": "state and tables > L2; flushed between timed steps", "metadata": meta}
    if variant >= 7:  # measured DRAM bytes per launch of the lean step on this mesh (ncu record)
        t = traffic_for_kernel("lean_large", variant)
        out["traffic_bytes_per_launch"] = t
        if t:
            out["traffic_over_algorithmic"] = t / (BYTES_PER_DOF_UPDATE * n)
    return out


def bench_adjoint(pbf, I, torch, stream, batch=8, nsteps=200, ckpt=10):
    """Adjoint sweep of configuration 4 on a reduced window: 8 instances, 200 steps, 10 stored
    states (binomial schedule), FP32 operator, gradients for 16 segment powers and s."""
    desc = I.c4_mesh()
    mat = I.TI64_NONLIN_Q2
    mesh = pbf.Mesh(desc)
    n = mesh.info()["n_dofs"]
    P, s = I.c4_params(batch)
    dt = 2e-8
    ls = I.c4_laser(P, n_seg=16, steps_per_seg=-(-nsteps // 16), dt=dt)
    ctx = pbf.Context(mesh, mat, pbf.PBF_F32OP, batch)
    pbf.pbf_ctx_set_k_scale(ctx.h, s)
    tab = mesh.tables()
    xyz = np.array(desc["origin"]) + np.array(desc["tree_h"]) * tab["dof_coord"] / (2 * 2.0 ** desc["max_level"])
    T0 = I.melt_pool_field(xyz, (0.05e-3, 0.25e-3, 0.25e-3), 2500.0, 50e-6, seed=5)
    T = torch.tensor(np.repeat(T0[:, None], batch, axis=1), dtype=torch.float64, device="cuda")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    J, g, fwd = pbf.pbf_adjoint_sweep(ctx.h, T, ls, 0.0, dt, nsteps, ckpt, batch=batch, stream=stream)
    b.record(stream)
    b.synchronize()
    ctx.close()
    mesh.close()
    return {"workload": f"C4 mesh ({n} dofs) x {batch} instances, {nsteps} steps, {ckpt} stored states",
            "seconds": a.elapsed_time(b) * 1e-3, "forward_steps": fwd, "finite": bool(np.isfinite(g).all())}


def bench_implicit(pbf, I, torch, stream, nsteps=20):
    """Configuration 3: the interlayer cool-down. The C1 brick with a newly activated three-cell
    powder layer (42,900 dofs), backward Euler at dt = 1e-2 s with bounds from 30 Lanczos
    steps: Chebyshev(5)-Jacobi CG to a 1e-8 relative residual with the FP64 and the FP32
    operator (the latter's result compared with the former's), the FP32 operator inside Newton /
    FP64 iterative refinement to a 1e-8 relative FP64 residual, and the nonlinear material by
    Newton's method."""
    mesh = pbf.Mesh(I.c3_mesh())
    pbf.pbf_mesh_activate_layer(mesh.h, I.C3_LAYER_TOP, 1, I.T0)
    n = mesh.info()["n_dofs"]
    desc = I.c3_mesh(active_top_z=I.C3_LAYER_TOP)
    tab = mesh.tables()
    T0 = I.melt_pool_field(dof_xyz(desc, tab), (0.5e-3, 0.25e-3, 0.25e-3), 1500.0, 120e-6, seed=4, noise=0.01)
    T0[tab["dirichlet"] != 0] = I.TI64_CONST["T_dirichlet"]  # the state satisfies the boundary condition
    out = {"workload": f"C3: C1 brick + 3-cell powder layer, {n} dofs, backward Euler dt = 1e-2 s, {nsteps} steps",
           "rtol": 1e-8, "cheb_degree": 5}
    dt = 1e-2
    final = {}

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        b.record(stream)
        b.synchronize()
        return r, a.elapsed_time(b)

    for name, prec in (("f64", pbf.PBF_F64), ("f32op", pbf.PBF_F32OP)):
        ctx = pbf.Context(mesh, I.TI64_CONST, prec)
        lo, hi = pbf.pbf_cheb_bounds(ctx.h, dt, None, 30, stream=stream)
        bounds = np.array((lo, 1.1 * hi))
        T = torch.tensor(T0, dtype=torch.float64, device="cuda")
        pbf.pbf_implicit_solve(ctx.h, T, dt, 2, 1e-8, 500, 5, bounds, stream=stream)  # warm-up
        T = torch.tensor(T0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        (st, iters), ms = timed(lambda: pbf.pbf_implicit_solve(ctx.h, T, dt, nsteps, 1e-8, 500, 5, bounds,
                                                               stream=stream))
        final[name] = T.clone()
        out[name] = {"status": int(st), "ms_per_step": ms / nsteps, "cg_iterations_per_step": float(np.mean(iters)),
                     "us_per_cg_iteration": 1e3 * ms / max(1, int(np.sum(iters)))}
        if prec == pbf.PBF_F32OP:
            # the FP32-operator CG stops on its recurrence residual; against the FP64 CG result:
            d = (final["f32op"] - final["f64"]).abs().max()
            out[name]["rel_diff_vs_f64_cg_of_increment"] = float(d / (final["f64"] - torch.tensor(
                T0, dtype=torch.float64, device="cuda")).abs().max())
            # the same steps by FP64 iterative refinement (Newton with the FP64 residual)
            T = torch.tensor(T0, dtype=torch.float64, device="cuda")
            (st, nit, lit, worst), ms = timed(lambda: pbf.pbf_implicit_newton(
                ctx.h, T, dt, nsteps, 1e-8, 10, 1e-4, 500, 5, bounds, stream=stream))
            d = (T - final["f64"]).abs().max()
            out["f32op_refined"] = {"status": int(st), "ms_per_step": ms / nsteps,
                                    "corrections_per_step": float(np.mean(nit)),
                                    "bicgstab_iterations_per_step": float(np.mean(lit)),
                                    "true_fp64_rel_residual": worst,
                                    "rel_diff_vs_f64_cg": float(d / final["f64"].abs().max())}
        ctx.close()
    # nonlinear conductivity (k 6.7 -> 28 W/mK) by Newton, FP64 and FP32 operators
    for name, prec in (("newton_nonlinear_f64", pbf.PBF_F64), ("newton_nonlinear_f32op", pbf.PBF_F32OP)):
        ctx = pbf.Context(mesh, I.TI64_NONLIN, prec)
        lo, hi = pbf.pbf_cheb_bounds(ctx.h, dt, None, 30, stream=stream)
        bounds = np.array((lo, 1.1 * hi))
        T = torch.tensor(T0, dtype=torch.float64, device="cuda")
        pbf.pbf_implicit_newton(ctx.h, T, dt, 1, 1e-8, 20, 1e-4, 500, 5, bounds, stream=stream)  # warm-up
        T = torch.tensor(T0, dtype=torch.float64, device="cuda")
        (st, nit, lit, worst), ms = timed(lambda: pbf.pbf_implicit_newton(
            ctx.h, T, dt, nsteps, 1e-8, 20, 1e-4, 500, 5, bounds, stream=stream))
        out[name] = {"status": int(st), "ms_per_step": ms / nsteps, "corrections_per_step": float(np.mean(nit)),
                     "bicgstab_iterations_per_step": float(np.mean(lit)), "rel_residual": worst}
        ctx.close()
    mesh.close()
    return out


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def spot_at(ls, t):
    """The laser spot at time t (the first segment with t0 <= t < t1), or None."""
    for x0, y0, x1, y1, t0, t1 in ls["seg"]:
        if t0 <= t < t1:
            a = (t - t0) / (t1 - t0)
            return x0 + (x1 - x0) * a, y0 + (y1 - y0) * a
    return None


def dof_xyz(desc, tab):
    return np.array(desc["origin"]) + np.array(desc["tree_h"]) * tab["dof_coord"] / (
        desc["degree"] * 2.0 ** desc["max_level"])


def bench_c2_adapt(pbf, I, torch, stream, T0, dt, shape, cycles=8):
    """Configuration 2 with its re-adaptation: after every 50 explicit steps the mesh is
    re-targeted to the 150 um refinement ball around the current spot (host), the state is
    moved to the new mesh (device: prolongation / injection) and the context is rebuilt (host
    tables and device set-up). Each part is timed on its own; the step rate is over the steps
    alone."""
    mat = I.TI64_NONLIN_Q2
    ls = I.c2_laser()
    mesh = pbf.Mesh(I.c2_mesh())
    T = torch.tensor(T0, dtype=torch.float64, device="cuda")
    ctx = pbf.Context(mesh, mat, pbf.PBF_F32OP)
    pbf.pbf_ctx_set_kernel_shape(ctx.h, shape)
    pbf.pbf_explicit_step(ctx.h, T, ls, 0.0, dt, 2, stream=stream)  # warm-up (not counted)
    torch.cuda.synchronize()
    step_ms = transfer_ms = 0.0
    adapt_s = ctx_s = 0.0
    updates, t, dofs = 0, 0.0, []
    for c in range(cycles):
        n = mesh.info()["n_dofs"]
        dofs.append(n)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pbf.pbf_explicit_step(ctx.h, T, ls, t, dt, CHUNK, stream=stream)
        b.record(stream)
        b.synchronize()
        step_ms += a.elapsed_time(b)
        updates += n * CHUNK
        t += CHUNK * dt
        x, y = spot_at(ls, t) or spot_at(ls, 0.0)
        h0 = time.perf_counter()
        pbf.pbf_mesh_adapt(mesh.h, I.c2_spot_regions(x, y))
        adapt_s += time.perf_counter() - h0
        Tn = torch.empty(mesh.info()["n_dofs"], dtype=torch.float64, device="cuda")
        a.record(stream)
        pbf.pbf_mesh_transfer(mesh.h, T, Tn, stream=stream)
        b.record(stream)
        b.synchronize()
        transfer_ms += a.elapsed_time(b)
        ctx.close()
        h0 = time.perf_counter()
        ctx = pbf.Context(mesh, mat, pbf.PBF_F32OP)
        pbf.pbf_ctx_set_kernel_shape(ctx.h, shape)
        ctx_s += time.perf_counter() - h0
        T = Tn
    ok = bool(torch.isfinite(T).all().item())
    ctx.close()
    mesh.close()
    return {"workload": f"C2 re-adapted every {CHUNK} steps to the ball around the moving spot, {cycles} cycles",
            "dofs_per_cycle": dofs, "steps_value": updates / (step_ms * 1e-3) / 1e9, "unit": "GDoF/s",
            "us_per_explicit_step": 1e3 * step_ms / (cycles * CHUNK),
            "host_adapt_ms_per_cycle": 1e3 * adapt_s / cycles,
            "device_transfer_us_per_cycle": 1e3 * transfer_ms / cycles,
            "context_rebuild_ms_per_cycle": 1e3 * ctx_s / cycles,
            "with_adaptation_value": updates / (step_ms * 1e-3 + adapt_s + transfer_ms * 1e-3 + ctx_s) / 1e9,
            "finite": ok}


def metadata_bytes(pbf, mesh, fused, batch=1):
    """Mesh metadata an explicit step reads at least once, the same whatever the number of
    instances in a batch (so it is amortised by batching and counted apart from the 16 B of
    state per dof-update). Every form reads, per active cell, its level, material and top flag
    (3 B) and, on the top surface, its FP32 corner (12 B), and per dof the FP32 inverse lumped
    mass (4 B). The fused step adds its patch tables. The per-cell form adds its cell-to-dof
    table (4 B per cell node) and the hanging-node rows (offsets, masters and FP32 weights)."""
    try:
        info = mesh.info()
        n_cells, n_dofs = info["n_active"], info["n_dofs"]
        common = 3 * n_cells + 12 * info["n_top_faces"] + 4 * n_dofs
        if fused:
            st = pbf.pbf_mesh_step_tables(mesh.h)
            tables = int(sum(st[k].nbytes for k in ("ptr", "cnt", "slot", "cell", "loc", "hloc", "hw")))
        else:
            tables = 4 * info["nodes_per_cell"] * n_cells + 4 * (info["n_hanging"] + 1) + 8 * info["n_con_entries"]
    except Exception as e:  # a side record: its failure is reported, the measurements stand
        return {"error": repr(e)}
    total = common + tables
    return {"form": "fused step" if fused else "per-cell", "tables_bytes": tables, "cell_and_dof_bytes": common,
            "bytes_per_step": total, "bytes_per_dof_update": total / (n_dofs * batch), "instances": batch,
            "algorithmic_state_bytes_per_dof_update": BYTES_PER_DOF_UPDATE}


def bench_laplace(pbf, I, torch, stream, flush, mesh, T0, dt, variant, K, full_gdofs):
    """The constant-coefficient instantiation of the same step. Sec. 5 compares the paper's
    full explicit step with a constant-coefficient Laplace operator on the same CPUs; the full
    step reached 44% of its throughput. Here the comparison uses the C2 mesh, the same kernel
    shape and step size, and the same timing: constant conductivity (powder included) and
    capacity, and no source, against the headline's nonlinear k(T), apparent capacity and
    laser."""
    mat = dict(I.TI64_CONST, powder_k_scale=1.0)
    ctx = pbf.Context(mesh, mat, pbf.PBF_F32OP)
    try:
        pbf.pbf_ctx_set_kernel_shape(ctx.h, variant)
        T = torch.tensor(T0, dtype=torch.float64, device="cuda")
        for k in range(3):
            pbf.pbf_explicit_step(ctx.h, T, None, k * CHUNK * dt, dt, CHUNK, stream=stream)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for k in range(K):
            flush.fill_(k & 0xFF)
            evs[k][0].record(stream)
            pbf.pbf_explicit_step(ctx.h, T, None, (3 + k) * CHUNK * dt, dt, CHUNK, stream=stream)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs)
    finally:
        ctx.close()
    n = mesh.info()["n_dofs"]
    value = n * CHUNK * K / (ms * 1e-3) / 1e9
    return {"value": value, "unit": "GDoF/s", "ms_per_step": ms / K, "steps": K, "step_shape": SHAPES[variant],
            "material": "constant k = 6.7 W/(m K) and c, no source",
            "full_step_over_laplace": full_gdofs / value, "paper_full_step_over_laplace": 0.44}


def bench_c5(pbf, I, torch, stream, flush, peaks, K=4, level=5):
    """Configuration 5, first layer of the part-scale stand-in (synthetic ribbed part on a
    baseplate, Q2, refined to level 5 in the layer and the heat-affected zone below it): FP32
    operator explicit steps at half the critical step (from the FP64 power iteration of the
    library) under a 67-degree hatch of one rib (P = 180 W, v = 0.9 m/s), the FP64 operator on
    the same steps, their difference, and a short implicit cool-down (dt = 5e-2 s) by Newton's
    method with the FP64 residual."""
    t0 = time.perf_counter()
    desc = I.c5_mesh(level=level)
    mesh = pbf.Mesh(desc)
    info = mesh.info()
    n = info["n_dofs"]
    host_mesh_s = time.perf_counter() - t0
    mat = I.TI64_NONLIN_Q2
    ls = I.c5_laser()
    cfl = pbf.Context(mesh, dict(mat, k0=mat["k1"], k1=mat["k1"], sigma=0.0, latent=0.0), pbf.PBF_F64)
    lam, dt_crit, _ = pbf.pbf_estimate_dt(cfl.h, None, 200, 1e-6)
    cfl.close()
    dt = 0.5 * dt_crit
    t0 = time.perf_counter()
    ctx = pbf.Context(mesh, mat, pbf.PBF_F32OP)
    ctx_s = time.perf_counter() - t0
    T0 = torch.full((n,), float(I.T0), dtype=torch.float64, device="cuda")
    variant, shape_us = pbf.pbf_ctx_autotune(ctx.h, T0, reps=3, stream=stream, times=True)
    T = T0.clone()
    pbf.pbf_explicit_step(ctx.h, T, ls, 0.0, dt, 3, stream=stream)  # warm-up
    T.copy_(T0)
    torch.cuda.synchronize()
    ms = 0.0
    for k in range(K):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pbf.pbf_explicit_step(ctx.h, T, ls, k * CHUNK * dt, dt, CHUNK, stream=stream)
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    value = n * CHUNK * K / (ms * 1e-3) / 1e9
    ctx64 = pbf.Context(mesh, mat, pbf.PBF_F64)
    T64 = T0.clone()
    pbf.pbf_explicit_step(ctx64.h, T64, ls, 0.0, dt, 1, stream=stream)  # warm-up
    T64.copy_(T0)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(K):
        pbf.pbf_explicit_step(ctx64.h, T64, ls, k * CHUNK * dt, dt, CHUNK, stream=stream)
    b.record(stream)
    b.synchronize()
    v64 = n * CHUNK * K / (a.elapsed_time(b) * 1e-3) / 1e9
    d = (T - T64).abs()
    err = {"rel_max": float(d.max() / T64.abs().max()),
           "rel_increment": float(d.max() / (T64 - T0).abs().max()),
           "rel_l2": float(torch.linalg.norm(T - T64) / torch.linalg.norm(T64)),
           "max_change_K": float((T64 - T0).abs().max())}
    ctx64.close()
    # the cool-down after the layer: Newton with the FP64 residual in the FP32-operator context
    Tc = T.clone()
    a.record(stream)
    st, nit, lit, worst = pbf.pbf_implicit_newton(ctx.h, Tc, 5e-2, 2, 1e-8, 20, 1e-3, 300, 5, None, stream=stream)
    b.record(stream)
    b.synchronize()
    cool = {"status": int(st), "ms_per_step": a.elapsed_time(b) / 2, "newton_corrections": [int(v) for v in nit],
            "bicgstab_iterations": [int(v) for v in lit], "rel_residual": worst, "dt_s": 5e-2,
            "bounds": "from 30 Lanczos steps (included in the first step's time)"}
    ok = bool(torch.isfinite(T).all().item())
    meta = metadata_bytes(pbf, mesh, variant >= 4)
    ctx.close()
    mesh.close()
    return {"workload": f"C5 stand-in, first layer: ribbed part on a baseplate, Q2 level {level}, "
                        f"{info['n_active']} cells, {n} dofs, 67-degree hatch of one rib",
            "value": value, "unit": "GDoF/s", "us_per_explicit_step": 1e3 * ms / (K * CHUNK), "dt_s": dt,
            "step_shape": SHAPES[variant],
            "hbm_fraction": value * BYTES_PER_DOF_UPDATE / peaks.get("hbm_gbs", 6800.0),
            "fp64": {"value": v64, "unit": "GDoF/s", "f32op_speedup": value / v64},
            "error_f32op_vs_f64_after_steps": dict(err, steps=K * CHUNK), "cooldown": cool,
            "host_mesh_s": host_mesh_s, "context_setup_s": ctx_s, "finite": ok,
            "l2": "state > L2; flushed between timed steps", "metadata": meta}



def bench_appendix_a(pbf, torch, stream):
    """The temporal-convergence experiment of Appendix A (two powder layers, explicit scan,
    explicit-then-implicit cool-down, activation of the second layer) at dt_ref, dt_ref / 2 and
    dt_ref / 4 through the library: the observation point's deviation from the finest run and
    the wall time of each run."""
    from paper_2302_05164_gb300 import temporal as TM
    runs, secs = {}, {}
    for k in (1, 2, 4):
        t0 = time.perf_counter()
        runs[k] = TM.run(pbf, torch, dt_scale=1.0 / k, stream=stream)
        secs[k] = time.perf_counter() - t0
    ref = TM.common_samples(runs[1], runs[4], 4)
    errs = {k: float(np.max(np.abs(TM.common_samples(runs[1], runs[k], k) - ref))) for k in (1, 2)}
    rise = float(np.max(runs[4]["T"]) - runs[4]["T"][0])
    return {"workload": "Appendix A: 1.0 x 0.2 x 0.2 mm plate + two 40 um powder layers, one track each, "
                        "0.06 s cool-down (0.02 s explicit, then implicit), observation point (0.5, 0, 0.24) mm",
            "max_dev_from_finest_K": {"dt_ref": errs[1], "dt_ref/2": errs[2]}, "ratio": errs[1] / errs[2],
            "order_note": "first order gives a ratio of 3 against the dt_ref/4 run",
            "peak_rise_K": rise, "wall_s": {f"dt_ref/{k}": secs[k] for k in (1, 2, 4)},
            "newton_corrections_and_bicgstab_at_dt_ref": runs[1]["newton"]}

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    return ws, rank


def max_over_ranks(ms, ws):
    """The job's time: the largest per-rank time, by an all-reduce MAX over the process group
    (NCCL on GPUs, gloo on CPU ranks)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ws, ms):
    """Whole-job throughput in G units per second: every rank's units over the job's time."""
    return units_per_rank * ws / (ms * 1e-3) / 1e9


def run_reference(args):
    ws, rank = dist_setup()
    if rank != 0:
        return
    # one warm-up step at most (the oracle has nothing to warm), and the timed steps bounded to
    # about three minutes of host time, so the run ends within a few minutes for any K
    time_oracle(min(args.warmup, 1))
    rate, n_dofs, done, seconds, _, _, _ = time_oracle(args.steps, max_seconds=180.0)
    value = rate / 1e9
    sample = f"1 serial FP64 oracle explicit step of the full workload ({n_dofs} dofs) per benchmark step, " \
             f"{done} of {args.steps} steps in {seconds:.1f} s (bounded to about 180 s)"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * seconds / max(done, 1),
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "one explicit step per step"},
                      "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                                       "cpu_model": cpu_model(), "sample": sample},
                      "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# dominant kernel -> (ncu traffic record, sources it was captured from: the kernel, its
# headers, and the host builder of the fused steps' patch tables)
_STEP_SRC = ["cell_ops.cuh", "step.cuh", "step_layout.hpp", "vec_kernels.cuh", "internal.cuh", "step_tables.cpp"]
TRAFFIC_RECORDS = {
    "cell": ("cell_kernel_c2_traffic.txt", ["kernels_cell.cu", "cell_ops.cuh", "internal.cuh"]),
    "step": ("step_kernel_c2_traffic.txt", ["kernels_step.cu"] + _STEP_SRC),
    "lean": ("step_lean_kernel_c2_traffic.txt", ["kernels_step_lean.cu"] + _STEP_SRC),
    # the lean step on the 18.2 M-dof mesh (the `large` entry), beyond L2
    "lean_large": ("step_lean_kernel_large_traffic.txt", ["kernels_step_lean.cu"] + _STEP_SRC),
}


def sources_sha256(names):
    import hashlib
    h = hashlib.sha256()
    for nm in names:
        h.update(open(os.path.join(ROOT, "paper_2302_05164_gb300", "csrc", nm), "rb").read())
    return h.hexdigest()


def traffic_for_kernel(kind, variant=None):
    """DRAM bytes per launch of the dominant kernel from the committed ncu record, if the
    kernel's sources are unchanged since that capture and the record covers this launch shape
    (else null)."""
    fname, srcs = TRAFFIC_RECORDS[kind]
    try:
        with open(os.path.join(ROOT, "profiles", fname)) as f:
            rec = json.load(f)
        if rec.get("sources_sha256") != sources_sha256(srcs):
            return None
        if variant is not None and "shape" in rec and rec["shape"] != variant:
            return None
        return rec["dram_bytes_per_launch"]
    except (OSError, KeyError, ValueError):
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="timed loop only (for profiler launch lists)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c4", "large"],
                    help="c4 / large: only the batched C4 steps / the 18 M-dof single instance (profiler runs)")
    ap.add_argument("--shape", type=int, default=-1,
                    help="explicit-step kernel shape to use instead of the autotuner's pick (0-6)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    from paper_2302_05164_gb300 import inputs as I
    from paper_2302_05164_gb300 import pbf

    ws, rank = dist_setup()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    W, K = max(3, args.warmup), args.steps
    if args.workload in ("c4", "large"):
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        if args.workload == "c4":
            out = bench_batched(pbf, I, torch, torch.cuda.current_stream(), flush, load_peaks()[0], K, shape=args.shape)
        else:
            out = bench_large(pbf, I, torch, torch.cuda.current_stream(), flush, load_peaks()[0], K=K)
        if rank == 0:
            print(json.dumps(out))
        return

    desc = I.c2_mesh()
    mat = I.TI64_NONLIN_Q2
    mesh = pbf.Mesh(desc)
    info = mesh.info()
    n = info["n_dofs"]
    tab = mesh.tables()
    xyz = np.array(desc["origin"]) + np.array(desc["tree_h"]) * tab["dof_coord"] / (2 * 2.0 ** desc["max_level"])
    T0 = c2_initial(I, xyz, rank)
    ls = I.c2_laser()
    ctx = pbf.Context(mesh, mat, pbf.PBF_F32OP)
    # critical step from the CFL estimate with the largest conductivity (Eq. explicit_time_step)
    if args.quick:
        dt = 1e-8  # profiler runs: no setup launches before the timed kernels
    else:
        cfl = pbf.Context(mesh, dict(mat, k0=mat["k1"], k1=mat["k1"], sigma=0.0, latent=0.0), pbf.PBF_F64)
        lam, dt_crit, _ = pbf.pbf_estimate_dt(cfl.h, None, 200, 1e-6)
        cfl.close()
        dt = 0.5 * dt_crit
    T = torch.tensor(T0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    if args.shape >= 0:
        variant, shape_us = args.shape, [-1.0] * len(SHAPES)
        pbf.pbf_ctx_set_kernel_shape(ctx.h, variant)
    else:
        variant, shape_us = pbf.pbf_ctx_autotune(ctx.h, T, reps=5, stream=stream, times=True)

    def bench_step(k):
        pbf.pbf_explicit_step(ctx.h, T, ls, k * CHUNK * dt, dt, CHUNK, stream=stream)

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(dev) as clocks:
        clocks.wait_first()
        for k in range(W):
            bench_step(k)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        launches0 = pbf.pbf_ctx_launch_count(ctx.h)
        t_begin = time.perf_counter()
        for k in range(K):
            flush.fill_(k & 0xFF)
            evs[k][0].record(stream)
            bench_step(W + k)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        clocks.mark(t_begin, time.perf_counter())
    ms = sum(a.elapsed_time(b) for a, b in evs)
    gpu_launches = pbf.pbf_ctx_launch_count(ctx.h) - launches0
    # the dominant kernel's launch duration: the same K benchmark steps again, with an event
    # pair around every launch of it on the library's stream (kept out of the timed loop
    # above: an event between two launches stops their programmatic overlap)
    pbf.pbf_ctx_kernel_time(ctx.h)
    pbf.pbf_ctx_set_timing(ctx.h, True)
    for k in range(K):
        flush.fill_(k & 0xFF)
        bench_step(W + K + k)
    torch.cuda.synchronize()
    pbf.pbf_ctx_set_timing(ctx.h, False)
    cell_ms, cell_launches = pbf.pbf_ctx_kernel_time(ctx.h)
    ms = max_over_ranks(ms, ws)
    value = job_rate(n * CHUNK * K, ws, ms)
    peaks, peak_src = load_peaks()
    out = {"metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": ws, "steps": K, "warmup": W,
           "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "precision": "FP32 operator arithmetic and accumulation; within a call the state is an FP32 pair "
                                "(about 48 bits) updated without rounding error, FP64 between calls",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "n_dofs": n, "n_cells": info["n_active"], "n_hanging": info["n_hanging"],
                      "explicit_steps_per_step": CHUNK, "dt_s": dt, "l2": "flushed between timed steps (256 MB write)",
                      "parallelism": f"replicas x{ws} (independent instances)",
                      "step_shape": SHAPES[variant],
                      "autotune_us_per_step": {k: round(u, 2) for k, u in zip(SHAPES, shape_us) if u > 0}},
           "gpu_launches": gpu_launches}
    # roofline of the dominant kernel. Algorithmic bytes: 16 B per dof-update (read T_n and
    # write T_{n+1} in FP64) x n dofs per launch (one launch per explicit step). Duration: the
    # timed region itself (CUDA events on the library's stream around each benchmark step of
    # CHUNK launches, the step kernel being ~97% of the device time in the ncu launch list), so
    # the figure slightly understates the kernel's own rate; the per-launch events of the
    # second pass (which stop the programmatic overlap of consecutive launches) are reported
    # beside it.
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    launch_s = ms * 1e-3 / (K * CHUNK) if variant != 6 else ms * 1e-3 / K
    bytes_launch = BYTES_PER_DOF_UPDATE * n * (CHUNK if variant == 6 else 1)
    hbm = peaks.get("hbm_gbs", 6800.0)
    achieved = bytes_launch / launch_s / 1e9
    kind = "lean" if variant >= 7 else ("step" if variant >= 4 else "cell")
    out["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                       "traffic": traffic_for_kernel(kind, variant), "kernel": KERNELS[variant],
                       "algorithmic_bytes_per_launch": bytes_launch,
                       "avg_launch_us": launch_s * 1e6,
                       "avg_launch_us_isolated": 1e3 * cell_ms / max(cell_launches, 1),
                       "launches_isolated": cell_launches,
                       "duration_source": "CUDA events around the K timed benchmark steps (CHUNK launches each) on the "
                                          "library's stream",
                       "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src}) - of measured"}
    # the FP32 ALU roof of the same kernel (the operator's flops; the lower of the two roofs)
    fpc = flops_per_cell_q2_nonlinear()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    flops_launch = fpc * info["n_active"] * (CHUNK if variant == 6 else 1)
    alu = flops_launch / launch_s / 1e12
    out["roofline_alu"] = {"bound": "alu", "achieved": alu, "peak": fp32_peak, "unit": "TFLOP/s",
                           "frac": alu / fp32_peak, "flops_per_cell": fpc,
                           "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (nominal)",
                           "note": "the ALU roof (338 GDoF/s at 238 flops per dof-update) lies below the HBM roof "
                                   "(423 GDoF/s); the kernel reaches neither: it is bound by latency and instruction "
                                   "issue within each patch (ncu: issue active ~37%, FMA pipe ~19%)"}
    out["hbm_fraction"] = {"algorithmic_bytes_per_dof_update": BYTES_PER_DOF_UPDATE,
                           "achieved_gbs": value * BYTES_PER_DOF_UPDATE,
                           "peak_gbs": hbm, "frac": value * BYTES_PER_DOF_UPDATE / hbm,
                           "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"}
    # shapes 4-9 read the patch tables (the lean forms through L1), shapes 0-3 the per-cell tables
    out["metadata"] = metadata_bytes(pbf, mesh, variant >= 4)
    out["device"] = {"name": props.name, "sms": n_sm}
    out["clocks"] = clocks.summary()
    if not args.quick:
        # FP64 operator on the same workload, timed over K benchmark steps as well
        ctx64 = pbf.Context(mesh, mat, pbf.PBF_F64)
        T64 = torch.tensor(T0, dtype=torch.float64, device="cuda")
        pbf.pbf_explicit_step(ctx64.h, T64, ls, 0.0, dt, 2, stream=stream)
        torch.cuda.synchronize()
        ms64 = 0.0
        K64 = max(1, min(K, 5))
        for k in range(K64):
            flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pbf.pbf_explicit_step(ctx64.h, T64, ls, k * CHUNK * dt, dt, CHUNK, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms64 += e0.elapsed_time(e1)
        v64 = n * CHUNK * K64 / (ms64 * 1e-3) / 1e9
        out["fp64"] = {"value": v64, "unit": "GDoF/s", "f32op_speedup": value / ws / v64, "steps": K64}
        # errors: FP32 operator against the FP64 operator after CHUNK steps, and both against
        # the oracle after two steps of the full workload at the oracle's own step size (the
        # oracle run is also the CPU baseline)
        Ta = torch.tensor(T0, dtype=torch.float64, device="cuda")
        Tb = torch.tensor(T0, dtype=torch.float64, device="cuda")
        pbf.pbf_explicit_step(ctx.h, Ta, ls, 0.0, dt, CHUNK, stream=stream)
        pbf.pbf_explicit_step(ctx64.h, Tb, ls, 0.0, dt, CHUNK, stream=stream)
        torch.cuda.synchronize()
        T0d = torch.tensor(T0, dtype=torch.float64, device="cuda")

        def errors(got, ref, start):
            d = (got - ref).abs()
            return {"rel_max": float(d.max() / ref.abs().max()),
                    "rel_increment": float(d.max() / (ref - start).abs().max()),
                    "rel_l2": float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref)),
                    "max_change_K": float((ref - start).abs().max())}

        out["error"] = {"f32op_vs_f64_after_steps": dict(errors(Ta, Tb, T0d), steps=CHUNK), "tolerance": 2e-4}
        if rank == 0:
            rate, n_s, done, secs, T_or, T0_or, dt_or = time_oracle(2)
            Tr = torch.tensor(T_or, dtype=torch.float64, device="cuda")
            Ts = torch.tensor(T0_or, dtype=torch.float64, device="cuda")
            vs = {}
            for name, c in (("f32op", ctx), ("f64", ctx64)):
                Tg = Ts.clone()
                pbf.pbf_explicit_step(c.h, Tg, ls, 0.0, dt_or, done, stream=stream)
                torch.cuda.synchronize()
                vs[name] = errors(Tg, Tr, Ts)
            out["error"]["vs_oracle"] = dict(vs, steps=done, dt_s=dt_or, n_dofs=n_s)
            out["cpu_baseline"] = {"value": rate / 1e9, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                                   "cpu_model": cpu_model(),
                                   "sample": f"{done} serial FP64 oracle explicit steps of the full workload ({n_s} "
                                             f"dofs, same mesh, material, laser and initial field), {secs:.1f} s"}
        ctx64.close()
        # end to end through the C ABI with host buffers: pinned H2D of the state, 50 steps,
        # D2H of the state, every step
        Th = torch.tensor(T0, dtype=torch.float64).pin_memory()
        Tout = torch.empty_like(Th).pin_memory()
        Td = torch.empty(n, dtype=torch.float64, device="cuda")
        for k in range(2):
            Td.copy_(Th, non_blocking=True)
            pbf.pbf_explicit_step(ctx.h, Td, ls, k * CHUNK * dt, dt, CHUNK, stream=stream)
            Tout.copy_(Td, non_blocking=True)
        torch.cuda.synchronize()
        e_ms = 0.0
        for k in range(K):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            Td.copy_(Th, non_blocking=True)
            pbf.pbf_explicit_step(ctx.h, Td, ls, k * CHUNK * dt, dt, CHUNK, stream=stream)
            Tout.copy_(Td, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e_ms += a.elapsed_time(b)
        e_ms = max_over_ranks(e_ms, ws)
        out["e2e"] = {"value": job_rate(n * CHUNK * K, ws, e_ms), "unit": "GDoF/s",
                      "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8}
        out["c2_adapt"] = bench_c2_adapt(pbf, I, torch, stream, T0, dt, variant)
        out["batched"] = bench_batched(pbf, I, torch, stream, flush, peaks, K)
        out["adjoint"] = bench_adjoint(pbf, I, torch, stream, batch=64, nsteps=2000, ckpt=40)
        out["implicit"] = bench_implicit(pbf, I, torch, stream)
        out["large"] = bench_large(pbf, I, torch, stream, flush, peaks)
        out["c5"] = bench_c5(pbf, I, torch, stream, flush, peaks)
        out["appendix_a"] = bench_appendix_a(pbf, torch, stream)
        try:
            out["laplace"] = bench_laplace(pbf, I, torch, stream, flush, mesh, T0, dt, variant, K, value / ws)
        except Exception as e:  # a side entry: its failure is reported, the headline stands
            out["laplace"] = {"error": repr(e)}
    ctx.close()
    mesh.close()
    if ws > 1:
        torch.distributed.barrier()
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
