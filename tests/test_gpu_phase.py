"""GPU parity of the phase-dependent conductivity with its consolidated-fraction history
(Sec. 2, Eqs. liquid_fraction, consolidated_fraction, phase_fractions,
material_parameter_interp) with the oracle, through the C ABI: residual terms at the initial
history, explicit steps that melt part of a powder layer (history stored per quadrature point),
and a residual at a cool state afterwards that must see the consolidated material; FP64 and
FP32 operators, Q1 and Q2 with hanging nodes; the fused step kernel with the model; the adjoint
sweep with the history against the oracle's adjoint.

Tolerances: FP64 1e-10 relative; FP32 operator 2e-5 of max|f| (residual terms), 2e-4 relative
max-norm on temperatures, and 5e-3 of max|f| for a residual that reads a history built by FP32
steps."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from tests.gates import check_f32_steps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32_F, TOL32_T = 1e-10, 2e-5, 2e-4
PH = dict(I.PHASE, k_m=30.0, k_s=25.0)


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05164_gb300 import pbf
    return pbf


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def to_dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def mesh(degree):
    regions = [(I.BALL, (0.3e-3, 0.25e-3, 0.25e-3), (0, 0, 0), 120e-6, 3)]
    return I.mesh_desc((8, 4, 2), (125e-6,) * 3, degree, 3, regions, powder_z0=0.17e-3, powder_z1=1.0)


def gpu_residual(P, ctx, T, n):
    out = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(3)]
    P.pbf_eval_residual(ctx.h, to_dev(T), None, 0.0, *out)
    return out[0].cpu().numpy()


@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_phase_residual_matches_oracle(P, oracle_mod, degree, prec):
    desc = mesh(degree)
    om = oracle_mod.Mesh(desc)
    om.set_phase(PH)
    T = I.smooth_field(om.dof_xyz(), seed=51, lo=1200.0, hi=2300.0)
    fd, _, _ = om.residual(I.TI64_CONST, T)
    m = P.Mesh(desc)
    ctx = P.Context(m, I.TI64_CONST, P.PBF_F64 if prec == "f64" else P.PBF_F32OP)
    P.pbf_ctx_set_phase(ctx.h, PH)
    gd = gpu_residual(P, ctx, T, om.n_dofs)
    assert rel(gd, fd) < (TOL64 if prec == "f64" else TOL32_F)
    # residual evaluations do not store the history: a second one is the same
    assert rel(gpu_residual(P, ctx, T, om.n_dofs), fd) < (TOL64 if prec == "f64" else TOL32_F)


def gpu_history(P, ctx, n_cells, nq):
    out = torch.zeros(nq * n_cells, dtype=torch.float64, device="cuda")
    P.pbf_ctx_get_history(ctx.h, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(nq, n_cells).T  # the oracle's [cell][q]


# FP32 shapes: 1 the per-cell form; 4 and 5 the fused step kernel (the phase model read and
# stored per quadrature point inside it); 8 a lean shape, which runs as 5 with the phase model
@pytest.mark.parametrize("prec,shape", [("f64", 5), ("f32", 1), ("f32", 4), ("f32", 5), ("f32", 8)])
def test_phase_history_through_explicit_steps(P, oracle_mod, prec, shape):
    desc = mesh(2)
    om = oracle_mod.Mesh(desc)
    om.set_phase(PH)
    mat = I.TI64_CONST
    lam, _ = oracle_mod.Mesh(desc).lambda_max(dict(mat, k0=30.0, k1=30.0, powder_k_scale=1.0),
                                              I.start_vector(om.n_dofs), max_iter=300, rtol=1e-8)
    dt = 0.4 * 2.0 / lam
    T0 = I.melt_pool_field(om.dof_xyz(), (0.3e-3, 0.25e-3, 0.25e-3), 2600.0, 60e-6, seed=52, noise=0.01)
    ref = om.explicit(mat, T0, None, 0.0, dt, 8)
    m = P.Mesh(desc)
    ctx = P.Context(m, mat, P.PBF_F64 if prec == "f64" else P.PBF_F32OP)
    P.pbf_ctx_set_phase(ctx.h, PH)
    P.pbf_ctx_set_kernel_shape(ctx.h, shape)
    Td = to_dev(T0)
    n0 = P.pbf_ctx_launch_count(ctx.h)
    P.pbf_explicit_step(ctx.h, Td, None, 0.0, dt, 8)
    torch.cuda.synchronize()
    if prec == "f32" and shape >= 4:
        assert P.pbf_ctx_launch_count(ctx.h) - n0 == 8 + 1  # fused: one launch per step and the last update
    if prec == "f64":
        assert rel(Td.cpu().numpy(), ref) < TOL64
    else:
        check_f32_steps(Td.cpu().numpy(), ref, T0)
    assert np.abs(ref - T0).max() > 1.0
    # the phase model moved the field by far more than the GPU's error: a form without it fails
    ref_plain = oracle_mod.Mesh(desc).explicit(mat, T0, None, 0.0, dt, 8)
    assert np.max(np.abs(Td.cpu().numpy() - ref)) < 0.1 * np.max(np.abs(ref - ref_plain))
    # the stored history (r_c after the last step's state T_7) equals the oracle's: exactly up
    # to FP64 rounding, and for the FP32 operator within dT / (T_l - T_s) of its state error
    h_ref = om.history()
    assert np.any((h_ref > 0.0) & (h_ref < 1.0))
    h_got = gpu_history(P, ctx, om.n_active, 27)
    assert np.max(np.abs(h_got - h_ref)) < (1e-10 if prec == "f64" else 5e-3)
    # a cool state now sees the consolidated powder where the steps melted it
    cool = I.smooth_field(om.dof_xyz(), seed=53, lo=400.0, hi=1400.0)
    fd, _, _ = om.residual(mat, cool)
    fresh = oracle_mod.Mesh(desc)
    fresh.set_phase(PH)
    fd0, _, _ = fresh.residual(mat, cool)
    assert rel(fd0, fd) > 1e-3  # the history changed the operator
    # the FP32 form's history follows its own states (within 2e-4 of the oracle's); g(T) turns a
    # state difference dT into dT / (T_l - T_s) of r_c, about 1e-3 here
    assert rel(gpu_residual(P, ctx, cool, om.n_dofs), fd) < (TOL64 if prec == "f64" else 5e-3)


@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("prec,shape", [("f64", 5), ("f32", 1), ("f32", 5)])
def test_phase_model_with_surface_loss_and_laser(P, oracle_mod, degree, prec, shape):
    """The paper's material model (phase-dependent conductivity with its history) with the
    radiation / evaporation loss and the surface laser, Q1 and Q2 with hanging nodes: six
    explicit steps in the fused step kernel with both options (FP32, shape 5) and in the
    per-cell form, against the oracle; temperatures and stored history."""
    desc = mesh(degree)
    om = oracle_mod.Mesh(desc)
    om.set_phase(PH)
    om.set_surface_loss(I.SURFACE_LOSS)
    mat = I.TI64_CONST
    lam, _ = oracle_mod.Mesh(desc).lambda_max(dict(mat, k0=30.0, k1=30.0, powder_k_scale=1.0),
                                              I.start_vector(om.n_dofs), max_iter=300, rtol=1e-8)
    dt = 0.4 * 2.0 / lam
    T0 = I.melt_pool_field(om.dof_xyz(), (0.3e-3, 0.25e-3, 0.25e-3), 3600.0, 60e-6, seed=54, noise=0.01)
    ls = I.laser([(0.1e-3, 0.25e-3, 0.9e-3, 0.25e-3, 0.0, 1e-3)], [200.0], eta=0.35, radius=40e-6)
    ref = om.explicit(mat, T0, ls, 1e-4, dt, 6)
    m = P.Mesh(desc)
    ctx = P.Context(m, mat, P.PBF_F64 if prec == "f64" else P.PBF_F32OP)
    P.pbf_ctx_set_phase(ctx.h, PH)
    P.pbf_ctx_set_surface_loss(ctx.h, I.SURFACE_LOSS)
    P.pbf_ctx_set_kernel_shape(ctx.h, shape)
    Td = to_dev(T0)
    n0 = P.pbf_ctx_launch_count(ctx.h)
    P.pbf_explicit_step(ctx.h, Td, ls, 1e-4, dt, 6)
    torch.cuda.synchronize()
    if prec == "f32" and shape >= 4:
        assert P.pbf_ctx_launch_count(ctx.h) - n0 == 6 + 1
    got = Td.cpu().numpy()
    if prec == "f64":
        assert rel(got, ref) < TOL64
    else:
        print(f"phase model + surface loss, Q{degree}, shape {shape}:", check_f32_steps(got, ref, T0))
    nq = (degree + 1) ** 3
    h_ref = om.history()
    assert np.max(np.abs(gpu_history(P, ctx, om.n_active, nq) - h_ref)) < (1e-10 if prec == "f64" else 5e-3)
    ctx.close()
    m.close()


@pytest.mark.parametrize("p,prec,ckpt", [(1, "f64", 3), (2, "f64", 4), (2, "f32", 3)])
def test_adjoint_with_phase_model_matches_oracle(P, oracle_mod, p, prec, ckpt):
    """The adjoint sweep with the phase model (the history as a state of the stepper, stored
    with every snapshot, its adjoint carried backward) equals the oracle's adjoint, which
    stores every state and history, for a batch of two instances with their own powers,
    conductivity scales and initial fields; the laser track partly melts the powder layer.
    FP64 1e-10, FP32 operator 1e-3; the phase model moves the gradients by far more than the
    tolerance; the context's history is as before the call."""
    d = I.mesh_desc((4, 2, 2), (125e-6,) * 3, p, 1, [I.uniform_region(1)], powder_z0=0.19e-3, powder_z1=1.0)
    om = oracle_mod.Mesh(d)
    mat = dict(I.TI64_CONST)
    lam, _ = om.lambda_max(dict(mat, k0=30.0, k1=30.0, powder_k_scale=1.0), I.start_vector(om.n_dofs), max_iter=300,
                           rtol=1e-8)
    dt, nsteps, Tt, B = 0.3 * 2.0 / lam, 12, 1800.0, 2
    P_, s = I.c4_params(B, n_seg=3, seed=2304)
    ls = I.c4_laser(P_, n_seg=3, steps_per_seg=4, dt=dt, v=1.0, y=0.125e-3)
    ls["seg"][:, 0] += 0.15e-3
    ls["seg"][:, 2] += 0.15e-3
    xyz = om.dof_xyz()
    T0 = np.stack([I.melt_pool_field(xyz, (0.2e-3, 0.125e-3, 0.25e-3), 1950.0 + 30 * b, 110e-6, seed=11 + b,
                                     noise=0.01) for b in range(B)], axis=1)
    ref0 = [om.adjoint(mat, T0[:, b], ls, 0.0, dt, nsteps, T_target=Tt, s=s[b], instance=b) for b in range(B)]
    om.set_phase(PH)
    ref = [om.adjoint(mat, T0[:, b], ls, 0.0, dt, nsteps, T_target=Tt, s=s[b], instance=b) for b in range(B)]
    m = P.Mesh(d)
    ctx = P.Context(m, mat, P.PBF_F64 if prec == "f64" else P.PBF_F32OP, B)
    P.pbf_ctx_set_k_scale(ctx.h, s)
    P.pbf_ctx_set_phase(ctx.h, PH)
    nq = (p + 1) ** 3
    h_before = torch.zeros(nq * om.n_active * B, dtype=torch.float64, device="cuda")
    P.pbf_ctx_get_history(ctx.h, h_before)
    J, g, fwd = P.pbf_adjoint_sweep(ctx.h, to_dev(T0), ls, 0.0, dt, nsteps, ckpt, T_target=Tt, batch=B)
    tol = 1e-10 if prec == "f64" else 1e-3
    for b in range(B):
        Jr, gr = ref[b]
        assert abs(J[b] - Jr) < tol * abs(Jr)
        assert np.max(np.abs(g[b] - gr)) < tol * np.max(np.abs(gr)), (g[b], gr)
        assert np.max(np.abs(gr - ref0[b][1])) > 100 * tol * np.max(np.abs(gr))
    assert fwd > nsteps
    h_after = torch.zeros_like(h_before)
    P.pbf_ctx_get_history(ctx.h, h_after)
    assert torch.equal(h_before, h_after)
    ctx.close()
    m.close()


def test_implicit_covers_the_phase_model_and_bad_parameters_refused(P):
    m = P.Mesh(mesh(1))
    ctx = P.Context(m, I.TI64_CONST, P.PBF_F64)
    with pytest.raises(P.PbfError):
        P.pbf_ctx_set_phase(ctx.h, dict(PH, T_l=1400.0))  # liquidus below solidus
    P.pbf_ctx_set_phase(ctx.h, PH)
    n = m.info()["n_dofs"]
    T = torch.full((n,), 500.0, dtype=torch.float64, device="cuda")
    status, _ = P.pbf_implicit_solve(ctx.h, T, 1e-2, 1, 1e-8, 200, 5, np.array([0.5, 2.0]))
    assert status == 0  # the implicit solve covers it by Newton's method (tests/test_gpu_newton.py)
    with pytest.raises(P.PbfError):  # the phase model needs the constant or nodal capacity
        P.pbf_ctx_set_phase(P.Context(m, I.TI64_NONLIN, P.PBF_F64).h, PH)
