"""GPU parity of the explicit hot path (cell operator, material, laser, lumped capacity,
fused Euler update, CFL estimate) against the oracle, through the C ABI.

Tolerances (tests/gates.py): FP64 operator 1e-10 relative max-norm (max |gpu - oracle| /
max |oracle|); FP32 operator 2e-4 relative max-norm and L2 on temperatures and 1e-3 of the
change the steps made (max |gpu - oracle| / max |oracle - T_0|); single residual evaluations
in FP32 are held to 2e-5 of max |f| (FP32 rounding of ~30-term sums of O(1) relative size)."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from tests.gates import TOL32_F, TOL64, check_f32_steps, check_f64_steps, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05164_gb300 import pbf
    return pbf


def amr_q2():
    regions = [(I.BALL, (0.3e-3, 0.25e-3, 0.25e-3), (0, 0, 0), 120e-6, 3),
               (I.BOX, (0.6e-3, 0.1e-3, 0.1e-3), (0.7e-3, 0.2e-3, 0.2e-3), 20e-6, 2)]
    return I.mesh_desc((8, 4, 2), (125e-6,) * 3, 2, 3, regions, powder_z0=0.15e-3, powder_z1=0.2e-3)


def amr_q1():
    d = amr_q2()
    d["degree"] = 1
    return d


def laser_over(desc, t_end=1e-3, power=200.0):
    y = desc["ntree"][1] * desc["tree_h"][1] / 2
    return I.laser([(0.1e-3, y, 0.9e-3, y, 0.0, t_end)], [power], eta=0.35, radius=40e-6)


def to_dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def gpu_residual(P, desc, mat, T, ls, t, prec, batch=1, kscale=None):
    m = P.Mesh(desc)
    ctx = P.Context(m, mat, prec, batch)
    if kscale is not None:
        P.pbf_ctx_set_k_scale(ctx.h, kscale)
    n = m.info()["n_dofs"]
    Td = to_dev(T)
    out = [torch.zeros(n * batch, dtype=torch.float64, device="cuda") for _ in range(3)]
    P.pbf_eval_residual(ctx.h, Td, ls, t, *out, batch=batch)
    torch.cuda.synchronize()
    return [o.cpu().numpy().reshape(n, batch) if batch > 1 else o.cpu().numpy() for o in out]


MATS = {"const": I.TI64_CONST, "nonlin": I.TI64_NONLIN, "nonlin_nodal": I.TI64_NONLIN_Q2}


@pytest.mark.parametrize("desc_fn", [amr_q1, amr_q2])
@pytest.mark.parametrize("mat", ["const", "nonlin", "nonlin_nodal"])
def test_residual_parity_f64(P, oracle_mod, desc_fn, mat):
    desc = desc_fn()
    material = MATS[mat]
    om = oracle_mod.Mesh(desc)
    T = I.smooth_field(om.dof_xyz(), seed=3, lo=353.0, hi=2900.0)
    ls = laser_over(desc)
    t = 4e-4
    fd, fv, Cm = om.residual(material, T, ls, t)
    gd, gv, gC = gpu_residual(P, desc, material, T, ls, t, P.PBF_F64)
    assert rel(gd, fd) < TOL64 and rel(gv, fv) < TOL64 and rel(gC, Cm) < TOL64
    assert np.abs(fv).max() > 0


@pytest.mark.parametrize("mat", ["nonlin", "nonlin_nodal"])
def test_residual_parity_f32(P, oracle_mod, mat):
    desc = amr_q2()
    om = oracle_mod.Mesh(desc)
    T = I.smooth_field(om.dof_xyz(), seed=5, lo=353.0, hi=2900.0)
    ls = laser_over(desc)
    fd, fv, Cm = om.residual(MATS[mat], T, ls, 4e-4)
    gd, gv, gC = gpu_residual(P, desc, MATS[mat], T, ls, 4e-4, P.PBF_F32OP)
    assert rel(gd, fd) < TOL32_F and rel(gv, fv) < TOL32_F and rel(gC, Cm) < TOL32_F


def run_gpu_steps(P, desc, mat, T0, ls, t0, dt, nsteps, prec, batch=1, kscale=None):
    m = P.Mesh(desc)
    ctx = P.Context(m, mat, prec, batch)
    if kscale is not None:
        P.pbf_ctx_set_k_scale(ctx.h, kscale)
    Td = to_dev(T0)
    P.pbf_explicit_step(ctx.h, Td, ls, t0, dt, nsteps, batch=batch)
    torch.cuda.synchronize()
    return Td.cpu().numpy()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_c1_single_track_200_steps(P, oracle_mod, prec):
    """Configuration 1: uniform Q1 brick, constant material, one track, 200 steps at half the
    CFL bound (dt from the oracle's power iteration, passed as the same double)."""
    desc = I.c1_mesh()
    om = oracle_mod.Mesh(desc)
    lam, _ = om.lambda_max(I.TI64_CONST, I.start_vector(om.n_dofs), max_iter=400, rtol=1e-8)
    dt = 0.5 * 2.0 / lam
    T0 = np.full(om.n_dofs, I.T0)
    ls = I.c1_laser()
    ref = om.explicit(I.TI64_CONST, T0, ls, 0.0, dt, 200)
    assert ref.max() > 900.0  # the track has heated the block well above T0
    got = run_gpu_steps(P, desc, I.TI64_CONST, T0, ls, 0.0, dt, 200, P.PBF_F64 if prec == "f64" else P.PBF_F32OP)
    if prec == "f64":
        check_f64_steps(got, ref, T0)
    else:
        print("C1 200 steps, FP32 operator:", check_f32_steps(got, ref, T0, min_change=500.0))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_amr_q2_nonlinear_latent_steps(P, oracle_mod, prec):
    desc = amr_q2()
    om = oracle_mod.Mesh(desc)
    mat = I.TI64_NONLIN_Q2  # nodal apparent capacity: positive lumped capacity for Q2
    lam, _ = om.lambda_max(dict(mat, k0=28.0), I.start_vector(om.n_dofs), max_iter=300, rtol=1e-8)
    dt = 0.5 * 2.0 / lam
    T0 = I.melt_pool_field(om.dof_xyz(), (0.3e-3, 0.25e-3, 0.25e-3), 2600.0, 60e-6, seed=9, noise=0.01)
    assert om.lumped_capacity(mat, T0).min() > 0
    ls = laser_over(desc, power=300.0)
    ref = om.explicit(mat, T0, ls, 1e-4, dt, 25)
    got = run_gpu_steps(P, desc, mat, T0, ls, 1e-4, dt, 25, P.PBF_F64 if prec == "f64" else P.PBF_F32OP)
    if prec == "f64":
        check_f64_steps(got, ref, T0)
    else:
        print("AMR Q2 25 steps, FP32 operator:", check_f32_steps(got, ref, T0, min_change=50.0))


@pytest.mark.parametrize("shape", list(range(10)))
def test_every_kernel_shape_matches_oracle(P, oracle_mod, shape):
    """Each explicit-step shape the autotuner can pick (the per-cell kernel's launch shapes,
    and the fused patch step kernel with and without programmatic dependent launch) gives the
    oracle's explicit steps on an AMR Q2 mesh."""
    desc = amr_q2()
    om = oracle_mod.Mesh(desc)
    mat = I.TI64_NONLIN_Q2
    lam, _ = om.lambda_max(dict(mat, k0=28.0), I.start_vector(om.n_dofs), max_iter=300, rtol=1e-8)
    dt = 0.5 * 2.0 / lam
    T0 = I.melt_pool_field(om.dof_xyz(), (0.3e-3, 0.25e-3, 0.25e-3), 2600.0, 60e-6, seed=4, noise=0.01)
    ls = laser_over(desc, power=300.0)
    ref = om.explicit(mat, T0, ls, 1e-4, dt, 10)
    m = P.Mesh(desc)
    ctx = P.Context(m, mat, P.PBF_F32OP)
    P.pbf_ctx_set_kernel_shape(ctx.h, shape)
    Td = to_dev(T0)
    P.pbf_explicit_step(ctx.h, Td, ls, 1e-4, dt, 10)
    torch.cuda.synchronize()
    check_f32_steps(Td.cpu().numpy(), ref, T0, min_change=20.0)
    # a residual evaluation after the steps finds every accumulator cleared
    fd, fv, Cm = om.residual(mat, Td.cpu().numpy(), ls, 1e-4)
    out = [torch.zeros(om.n_dofs, dtype=torch.float64, device="cuda") for _ in range(3)]
    P.pbf_eval_residual(ctx.h, Td, ls, 1e-4, *out)
    assert rel(out[0].cpu().numpy(), fd) < TOL32_F and rel(out[1].cpu().numpy(), fv) < TOL32_F


def test_batched_instances_match_independent_runs(P, oracle_mod):
    """Instances of a batch (layout [n_dofs][batch]) carry their own laser powers and
    conductivity scales; each equals an independent oracle run. Batch 3 is ragged."""
    desc = amr_q1()
    om = oracle_mod.Mesh(desc)
    mat = I.TI64_NONLIN
    B = 3
    powers = np.array([[150.0], [200.0], [260.0]])
    s = np.array([0.8, 1.0, 1.2])
    ls = laser_over(desc)
    ls["power"] = powers
    T0 = I.smooth_field(om.dof_xyz(), seed=2, lo=353.0, hi=1800.0, batch=B)
    lam, _ = om.lambda_max(dict(mat, k0=28.0 * 1.2), I.start_vector(om.n_dofs), max_iter=300, rtol=1e-8)
    dt = 0.4 * 2.0 / lam
    got = run_gpu_steps(P, desc, mat, T0, ls, 0.0, dt, 10, P.PBF_F64, batch=B, kscale=s).reshape(-1, B)
    for b in range(B):
        ref = om.explicit(mat, T0[:, b], ls, 0.0, dt, 10, s=s[b], instance=b)
        check_f64_steps(got[:, b], ref, T0[:, b])


def test_cfl_estimate_matches_oracle(P, oracle_mod):
    desc = amr_q2()
    om = oracle_mod.Mesh(desc)
    x0 = I.start_vector(om.n_dofs)
    lam_o, it_o = om.lambda_max(I.TI64_CONST, x0, max_iter=60, rtol=0.0)
    m = P.Mesh(desc)
    ctx = P.Context(m, I.TI64_CONST, P.PBF_F64)
    lam_g, dtc, it_g = P.pbf_estimate_dt(ctx.h, to_dev(x0), max_iter=60, rtol=0.0)
    assert it_g == it_o == 60
    assert abs(lam_g - lam_o) < 1e-9 * lam_o and abs(dtc - 2.0 / lam_g) < 1e-15


def test_edge_cases(P, oracle_mod):
    desc = amr_q1()
    om = oracle_mod.Mesh(desc)
    T0 = I.smooth_field(om.dof_xyz(), seed=1)
    # zero steps: state untouched
    got = run_gpu_steps(P, desc, I.TI64_CONST, T0, None, 0.0, 1e-7, 0, P.PBF_F64)
    assert np.array_equal(got, T0)
    # laser whose only segment lies in the future: no source, same as no laser
    ls = laser_over(desc)
    ls["seg"] = ls["seg"].copy()
    ls["seg"][0, 4:] = [1.0, 2.0]
    a = run_gpu_steps(P, desc, I.TI64_CONST, T0, ls, 0.0, 1e-7, 3, P.PBF_F64)
    b = run_gpu_steps(P, desc, I.TI64_CONST, T0, None, 0.0, 1e-7, 3, P.PBF_F64)
    assert rel(a, b) < 1e-14  # atomic scatter: equal up to summation order
    # every cell inactive: no dofs, a context still works
    empty = dict(desc, active_top_z=-1.0)
    m = P.Mesh(empty)
    assert m.info()["n_dofs"] == 0
    ctx = P.Context(m, I.TI64_CONST, P.PBF_F64)
    Td = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.pbf_explicit_step(ctx.h, Td, None, 0.0, 1e-7, 2)
    torch.cuda.synchronize()


def test_c2_full_size_residual_and_step(P, oracle_mod):
    """Configuration 2 at full size (Q2, ~1.07M dofs, 39.6k hanging nodes): the residual, and
    five explicit steps at half the critical step in both precisions and in every launch
    configuration the benchmark chooses from."""
    desc = I.c2_mesh()
    om = oracle_mod.Mesh(desc)
    mat = I.TI64_NONLIN_Q2
    T = I.melt_pool_field(om.dof_xyz(), (0.51e-3, 0.55e-3, 1.0e-3), 2800.0, 50e-6, seed=21, noise=0.02)
    ls = I.c2_laser()
    t = 1e-5
    fd, fv, Cm = om.residual(mat, T, ls, t)
    gd, gv, gC = gpu_residual(P, desc, mat, T, ls, t, P.PBF_F64)
    assert rel(gd, fd) < TOL64 and rel(gv, fv) < TOL64 and rel(gC, Cm) < TOL64
    gd, gv, gC = gpu_residual(P, desc, mat, T, ls, t, P.PBF_F32OP)
    assert rel(gd, fd) < TOL32_F and rel(gC, Cm) < TOL32_F
    # steps at half the critical step of the finest cells (k at its largest value), taken from
    # the oracle's power iteration on a uniform block of 5 um Q2 cells
    ob = oracle_mod.Mesh(I.mesh_desc((2, 2, 2), (40e-6,) * 3, 2, 3, [I.uniform_region(3)], dirichlet_faces=0))
    lam, _ = ob.lambda_max(dict(mat, k0=28.0), I.start_vector(ob.n_dofs), max_iter=300, rtol=1e-8)
    dt = 0.5 * 2.0 / lam
    nsteps = 5
    ref = om.explicit(mat, T, ls, t, dt, nsteps)
    got = run_gpu_steps(P, desc, mat, T, ls, t, dt, nsteps, P.PBF_F64)
    check_f64_steps(got, ref, T)
    got = run_gpu_steps(P, desc, mat, T, ls, t, dt, nsteps, P.PBF_F32OP)
    print("C2 full size, 5 steps, FP32 operator (autotuner's default shape):", check_f32_steps(got, ref, T, 20.0))
    # the fused shapes the benchmark chooses from; at this size the persistent form has
    # fewer blocks than patches (blocks take several patches per step)
    m = P.Mesh(desc)
    ctx = P.Context(m, mat, P.PBF_F32OP)
    for shape in (4, 5, 6, 7, 8, 9):
        P.pbf_ctx_set_kernel_shape(ctx.h, shape)
        Td = to_dev(T)
        P.pbf_explicit_step(ctx.h, Td, ls, t, dt, nsteps)
        torch.cuda.synchronize()
        print(f"C2 full size, shape {shape}:", check_f32_steps(Td.cpu().numpy(), ref, T, 20.0))
    ctx.close()
    m.close()
