"""GPU parity of the implicit cool-down path (implicit operator, Jacobi diagonal,
Chebyshev(5)-Jacobi preconditioned CG with FP64 dot products, Lanczos bounds) on the
configuration-3 mesh with a newly activated powder layer, against the oracle.

Tolerances: FP64 operator with both solvers converged to 1e-12 relative residual: 1e-10
relative max-norm on T; FP32 operator: 2e-4."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from tests.gates import check_f32_steps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05164_gb300 import pbf
    return pbf


RTOL = 1e-11


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def to_dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def c3(oracle_mod):
    """Configuration 3: the c1 brick with a three-cell powder layer activated on top (powder
    conductivity x 0.1), a hot track left in the part, and the oracle's Lanczos bounds."""
    old = oracle_mod.Mesh(I.c3_mesh())
    om = oracle_mod.Mesh(I.c3_mesh(active_top_z=I.C3_LAYER_TOP))
    t_old, t_new = old.tables(), om.tables()
    act_old = t_old["leaves"][:, 4] == 1
    act_new = t_new["leaves"][:, 4] == 1
    newly = act_new & ~act_old
    om.set_material(newly[act_new].astype(np.uint8))
    T_old = I.melt_pool_field(old.dof_xyz(), (0.5e-3, 0.25e-3, 0.25e-3), 1500.0, 120e-6, seed=4, noise=0.01)
    T = oracle_mod.transfer(old, T_old, om, I.T0)
    dt = 1e-2
    b = I.start_vector(om.n_dofs, seed=3)
    lmin, lmax = om.lanczos_bounds(I.TI64_CONST, dt, b, 30)
    bounds = (lmin, 1.1 * lmax)
    ref, it_ref, st = om.implicit(I.TI64_CONST, T, dt, 1, RTOL, 400, 5, *bounds)
    assert st == 0
    return dict(old=old, om=om, T_old=T_old, T=T, dt=dt, b=b, bounds=bounds, ref=ref, it_ref=it_ref)


def gpu_c3(P):
    m = P.Mesh(I.c3_mesh())
    P.pbf_mesh_activate_layer(m.h, I.C3_LAYER_TOP, 1, I.T0)
    return m


def test_activation_transfer_matches_oracle(P, c3):
    m = P.Mesh(I.c3_mesh())
    Told = to_dev(c3["T_old"])
    P.pbf_mesh_activate_layer(m.h, I.C3_LAYER_TOP, 1, I.T0)
    Tnew = torch.zeros(m.info()["n_dofs"], dtype=torch.float64, device="cuda")
    P.pbf_mesh_transfer(m.h, Told, Tnew)
    got = Tnew.cpu().numpy()
    assert np.array_equal(got, c3["T"])  # shared nodes copied exactly, new nodes T_init
    with pytest.raises(P.PbfError):
        P.pbf_mesh_transfer(m.h, Told, Tnew)  # the transfer was consumed


def test_adapt_transfer_matches_oracle(P, oracle_mod):
    d0 = I.mesh_desc((8, 4, 2), (125e-6,) * 3, 2, 3, I.c2_spot_regions(0.3e-3, 0.25e-3, 0.25e-3, 150e-6), )
    d1 = I.mesh_desc((8, 4, 2), (125e-6,) * 3, 2, 3, I.c2_spot_regions(0.5e-3, 0.25e-3, 0.25e-3, 150e-6))
    o0, o1 = oracle_mod.Mesh(d0), oracle_mod.Mesh(d1)
    T0 = I.smooth_field(o0.dof_xyz(), seed=6)
    ref = oracle_mod.transfer(o0, T0, o1, -1.0)
    m = P.Mesh(d0)
    P.pbf_mesh_adapt(m.h, d1["regions"])
    Tn = torch.zeros(m.info()["n_dofs"], dtype=torch.float64, device="cuda")
    P.pbf_mesh_transfer(m.h, to_dev(T0), Tn)
    assert rel(Tn.cpu().numpy(), ref) < 1e-13


def test_cheb_bounds_match_oracle(P, c3):
    m = gpu_c3(P)
    ctx = P.Context(m, I.TI64_CONST, P.PBF_F64)
    lo, hi = P.pbf_cheb_bounds(ctx.h, c3["dt"], to_dev(c3["b"]), 30)
    ref_lo, ref_hi = c3["bounds"][0], c3["bounds"][1] / 1.1
    assert abs(lo - ref_lo) < 1e-8 * ref_lo and abs(hi - ref_hi) < 1e-8 * ref_hi


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_implicit_cooldown_matches_oracle(P, c3, prec):
    T, dt, ref, it_ref = c3["T"], c3["dt"], c3["ref"], c3["it_ref"]
    m = gpu_c3(P)
    ctx = P.Context(m, I.TI64_CONST, P.PBF_F64 if prec == "f64" else P.PBF_F32OP)
    Td = to_dev(T)
    status, iters = P.pbf_implicit_solve(ctx.h, Td, dt, 1, RTOL, 400, 5, np.array(c3["bounds"]))
    assert status == 0
    got = Td.cpu().numpy()
    if prec == "f64":
        assert rel(got, ref) < 1e-10
    else:
        print("C3 backward-Euler step, FP32 operator:", check_f32_steps(got, ref, T))
    if prec == "f64":
        assert abs(int(iters[0]) - int(it_ref[0])) <= 1
    assert got.max() < T.max()  # the hot track cools


def test_implicit_changing_dt_and_bounds_on_one_context(P, c3):
    """The preconditioner runs as a CUDA graph captured for one (dt, bounds, degree); solves
    with another dt and other bounds on the same context, and back, still match the oracle
    (the graph is rebuilt whenever its parameters change)."""
    om, T = c3["om"], c3["T"]
    dt2 = 2.5e-3
    lmin, lmax = om.lanczos_bounds(I.TI64_CONST, dt2, c3["b"], 30)
    bounds2 = (lmin, 1.1 * lmax)
    ref2, it2, st = om.implicit(I.TI64_CONST, T, dt2, 1, RTOL, 400, 5, *bounds2)
    assert st == 0
    m = gpu_c3(P)
    ctx = P.Context(m, I.TI64_CONST, P.PBF_F64)
    for dt, bounds, ref in ((c3["dt"], c3["bounds"], c3["ref"]), (dt2, bounds2, ref2),
                            (c3["dt"], c3["bounds"], c3["ref"])):
        Td = to_dev(T)
        status, iters = P.pbf_implicit_solve(ctx.h, Td, dt, 1, RTOL, 400, 5, np.array(bounds))
        assert status == 0
        assert rel(Td.cpu().numpy(), ref) < 1e-10


def test_implicit_reports_nonconvergence_and_bad_inputs(P, c3):
    m = gpu_c3(P)
    ctx = P.Context(m, I.TI64_CONST, P.PBF_F64)
    Td = to_dev(c3["T"])
    status, iters = P.pbf_implicit_solve(ctx.h, Td, c3["dt"], 1, 1e-12, 1, 5, np.array(c3["bounds"]))
    assert status == 4 and iters[0] == 1  # PBF_ENOCONV, state holds the last iterate
    bctx = P.Context(m, I.TI64_CONST, P.PBF_F64, 2)
    status, _ = P.pbf_implicit_solve(bctx.h, torch.zeros(2 * m.info()["n_dofs"], dtype=torch.float64,
                                                        device="cuda"), c3["dt"], 1, 1e-8, 10, 5, None)
    assert status == 1  # batches: one instance only
    # default bounds (library Lanczos from its SplitMix64 start vector) also converge
    Td = to_dev(c3["T"])
    status, iters = P.pbf_implicit_solve(ctx.h, Td, c3["dt"], 1, 1e-8, 400, 5, None)
    assert status == 0 and iters[0] < 100


def test_volumetric_source_matches_oracle(P, oracle_mod):
    """The paper's cylinder source (Eq. heat_soruce_cylindrical, -h_powder < z^ < 0)."""
    regions = [(I.BALL, (0.3e-3, 0.25e-3, 0.25e-3), (0, 0, 0), 120e-6, 3)]
    desc = I.mesh_desc((8, 4, 2), (125e-6,) * 3, 2, 3, regions, active_top_z=0.25e-3)
    om = oracle_mod.Mesh(desc)
    ls = I.laser([(0.2e-3, 0.25e-3, 0.6e-3, 0.25e-3, 0.0, 1e-3)], [200.0], volumetric=True, h_powder=40e-6)
    T = np.full(om.n_dofs, I.T0)
    _, fv, _ = om.residual(I.TI64_CONST, T, ls, 2e-4)
    assert fv.sum() > 0
    m = P.Mesh(desc)
    ctx = P.Context(m, I.TI64_CONST, P.PBF_F64)
    out = [torch.zeros(om.n_dofs, dtype=torch.float64, device="cuda") for _ in range(3)]
    P.pbf_eval_residual(ctx.h, to_dev(T), ls, 2e-4, *out)
    assert rel(out[1].cpu().numpy(), fv) < 1e-10
