"""GPU parity of the radiation / evaporation surface loss on the free top surface (Sec. 2,
Eqs. bc_rad_evap, bc_radiation, bc_evaporation) with the oracle, through the C ABI:
residual terms and explicit steps on adaptive Q1/Q2 meshes with hanging nodes on the top
surface, a field that crosses the boiling point and the evaporation cap, FP64 and FP32
operators; the adjoint sweep with the loss against the oracle's adjoint.

Tolerances as for the other parity tests: FP64 1e-10 relative; FP32 operator 2e-5 of max|f|
for residual terms and 2e-4 relative max-norm on temperatures."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from tests.gates import check_f32_steps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32_F, TOL32_T = 1e-10, 2e-5, 2e-4


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
    return I.mesh_desc((8, 4, 2), (125e-6,) * 3, degree, 3, regions)


def hot_field(om):
    # up to 4300 K at the top: radiation everywhere, evaporation above 3000 K, cap at 4000 K
    return I.melt_pool_field(om.dof_xyz(), (0.3e-3, 0.25e-3, 0.25e-3), 4300.0, 70e-6, seed=41, noise=0.01)


@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_surface_loss_residual_matches_oracle(P, oracle_mod, degree, prec):
    desc = mesh(degree)
    om = oracle_mod.Mesh(desc)
    om.set_surface_loss(I.SURFACE_LOSS)
    mat = I.TI64_NONLIN_Q2
    T = hot_field(om)
    ls = I.laser([(0.1e-3, 0.25e-3, 0.9e-3, 0.25e-3, 0.0, 1e-3)], [200.0], eta=0.35, radius=40e-6)
    fd, fv, _ = om.residual(mat, T, ls, 2e-4)
    m = P.Mesh(desc)
    ctx = P.Context(m, mat, P.PBF_F64 if prec == "f64" else P.PBF_F32OP)
    P.pbf_ctx_set_surface_loss(ctx.h, I.SURFACE_LOSS)
    out = [torch.zeros(om.n_dofs, dtype=torch.float64, device="cuda") for _ in range(3)]
    P.pbf_eval_residual(ctx.h, to_dev(T), ls, 2e-4, *out)
    gd, gv = out[0].cpu().numpy(), out[1].cpu().numpy()
    tol = TOL64 if prec == "f64" else TOL32_F
    assert rel(gd, fd) < tol and rel(gv, fv) < tol
    # the loss dominates the top rows here: without it the source term differs
    _, fv0, _ = oracle_mod.Mesh(desc).residual(mat, T, ls, 2e-4)
    assert rel(fv0, fv) > 1e-2


@pytest.mark.parametrize("prec,shape", [("f64", 5), ("f32", 1), ("f32", 4), ("f32", 5), ("f32", 9)])
def test_explicit_steps_with_surface_loss_match_oracle(P, oracle_mod, prec, shape):
    """Six steps with the laser on. FP32 shapes: 1 the per-cell form (a face kernel after the
    cell kernel); 4 and 5 the fused step kernel, which adds the loss of each top face in its
    cell phase; 9 a lean shape, which runs as 5 with the surface loss."""
    desc = mesh(2)
    om = oracle_mod.Mesh(desc)
    om.set_surface_loss(I.SURFACE_LOSS)
    mat = I.TI64_NONLIN_Q2
    T0 = I.melt_pool_field(om.dof_xyz(), (0.3e-3, 0.25e-3, 0.25e-3), 3700.0, 70e-6, seed=42, noise=0.01)
    ls = I.laser([(0.1e-3, 0.25e-3, 0.9e-3, 0.25e-3, 0.0, 1e-3)], [200.0], eta=0.35, radius=40e-6)
    lam, _ = oracle_mod.Mesh(desc).lambda_max(dict(mat, k0=28.0), I.start_vector(om.n_dofs), max_iter=300,
                                              rtol=1e-8)
    dt = 0.4 * 2.0 / lam
    ref = om.explicit(mat, T0, ls, 1e-4, dt, 6)
    m = P.Mesh(desc)
    ctx = P.Context(m, mat, P.PBF_F64 if prec == "f64" else P.PBF_F32OP)
    P.pbf_ctx_set_surface_loss(ctx.h, I.SURFACE_LOSS)
    P.pbf_ctx_set_kernel_shape(ctx.h, shape)
    Td = to_dev(T0)
    n0 = P.pbf_ctx_launch_count(ctx.h)
    P.pbf_explicit_step(ctx.h, Td, ls, 1e-4, dt, 6)
    torch.cuda.synchronize()
    if prec == "f32" and shape >= 4:
        assert P.pbf_ctx_launch_count(ctx.h) - n0 == 6 + 1  # fused: one launch per step and the last update
    got = Td.cpu().numpy()
    if prec == "f64":
        assert rel(got, ref) < TOL64
    else:
        check_f32_steps(got, ref, T0)
    assert np.abs(ref - T0).max() > 1.0
    # switched off again: the plain operator (the oracle without the loss)
    P.pbf_ctx_set_surface_loss(ctx.h, None)
    Td = to_dev(T0)
    P.pbf_explicit_step(ctx.h, Td, ls, 1e-4, dt, 6)
    torch.cuda.synchronize()
    ref0 = oracle_mod.Mesh(desc).explicit(mat, T0, ls, 1e-4, dt, 6)
    # the loss moved the field by far more than the GPU's error: a form without it fails
    assert np.max(np.abs(got - ref)) < 0.1 * np.max(np.abs(ref - ref0))
    if prec == "f64":
        assert rel(Td.cpu().numpy(), ref0) < TOL64
    else:
        check_f32_steps(Td.cpu().numpy(), ref0, T0)


@pytest.mark.parametrize("p,prec", [(1, "f64"), (2, "f64"), (2, "f32")])
def test_adjoint_with_surface_loss_matches_oracle(P, oracle_mod, p, prec):
    """The adjoint sweep with radiation and evaporation on the top surface (the loss's face
    term in the transposed step, the laser's part of f_vol in the power gradients) equals the
    oracle's adjoint for a batch of two instances with their own powers, conductivity scales
    and initial fields, with binomial checkpoints (3 stored states for 12 steps); the top
    reaches 3600 K, so evaporation is active. FP64 1e-10, FP32 operator 1e-3 (as the adjoint
    without the loss). The loss moves the gradients by far more than the tolerance."""
    d = I.mesh_desc((4, 2, 2), (125e-6,) * 3, p, 1, [I.uniform_region(1)])
    om = oracle_mod.Mesh(d)
    mat = dict(I.TI64_NONLIN, lumping=I.LUMP_QUADRATURE if p == 1 else I.LUMP_NODAL)
    dt, nsteps, Tt, B = 5e-6, 12, 3000.0, 2
    P_, s = I.c4_params(B, n_seg=3, seed=2303)
    ls = I.c4_laser(P_, n_seg=3, steps_per_seg=4, dt=dt, v=0.5, y=0.125e-3)
    xyz = om.dof_xyz()
    T0 = np.stack([I.melt_pool_field(xyz, (0.25e-3, 0.125e-3, 0.25e-3), 3550.0 + 50 * b, 90e-6, seed=11 + b,
                                     noise=0.01) for b in range(B)], axis=1)
    ref0 = [om.adjoint(mat, T0[:, b], ls, 0.0, dt, nsteps, T_target=Tt, s=s[b], instance=b) for b in range(B)]
    om.set_surface_loss(I.SURFACE_LOSS)
    ref = [om.adjoint(mat, T0[:, b], ls, 0.0, dt, nsteps, T_target=Tt, s=s[b], instance=b) for b in range(B)]
    m = P.Mesh(d)
    ctx = P.Context(m, mat, P.PBF_F64 if prec == "f64" else P.PBF_F32OP, B)
    P.pbf_ctx_set_k_scale(ctx.h, s)
    P.pbf_ctx_set_surface_loss(ctx.h, I.SURFACE_LOSS)
    T0d = to_dev(T0)
    J, g, fwd = P.pbf_adjoint_sweep(ctx.h, T0d, ls, 0.0, dt, nsteps, 3, T_target=Tt, batch=B)
    tol = 1e-10 if prec == "f64" else 1e-3
    for b in range(B):
        Jr, gr = ref[b]
        assert abs(J[b] - Jr) < tol * abs(Jr)
        assert np.max(np.abs(g[b] - gr)) < tol * np.max(np.abs(gr)), (g[b], gr)
        assert np.max(np.abs(gr - ref0[b][1])) > 100 * tol * np.max(np.abs(gr))
    assert fwd > nsteps
    ctx.close()
    m.close()


def test_implicit_covers_the_surface_loss_and_cap_checked(P):
    desc = mesh(1)
    m = P.Mesh(desc)
    ctx = P.Context(m, I.TI64_CONST, P.PBF_F64)
    P.pbf_ctx_set_surface_loss(ctx.h, I.SURFACE_LOSS)
    n = m.info()["n_dofs"]
    T = torch.full((n,), 500.0, dtype=torch.float64, device="cuda")
    status, _ = P.pbf_implicit_solve(ctx.h, T, 1e-2, 1, 1e-8, 200, 5, np.array([0.5, 2.0]))
    assert status == 0  # the implicit solve covers it by Newton's method (tests/test_gpu_newton.py)
    with pytest.raises(P.PbfError):
        P.pbf_ctx_set_surface_loss(ctx.h, dict(I.SURFACE_LOSS, T_max=2000.0))  # cap below T_v
