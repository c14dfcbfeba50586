"""GPU parity of the fused explicit step (one launch per forward-Euler step: the patch-staged
cell operator that completes the previous step while staging) against the oracle, through
the C ABI: degrees 1 and 2 on adaptive meshes with hanging nodes, constant / nonlinear
conductivity, nodal apparent capacity, surface and volumetric lasers, Dirichlet dofs that
start away from T_D, short sequences that exercise the accumulator rotation (1, 2, 3 steps)
and consecutive calls mixing the fused and per-cell forms.

Tolerances (tests/gates.py): FP32 operator, 2e-4 relative max-norm and L2 on temperatures and
1e-3 of the change the steps made (as for the per-cell form)."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from tests.gates import check_f32_steps, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FUSED, FUSED_PDL, PERSISTENT, PER_CELL = 4, 5, 6, 1
LEAN = (7, 8, 9)


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05164_gb300 import pbf
    return pbf


def amr(degree):
    regions = [(I.BALL, (0.3e-3, 0.25e-3, 0.25e-3), (0, 0, 0), 120e-6, 3),
               (I.BOX, (0.6e-3, 0.1e-3, 0.1e-3), (0.7e-3, 0.2e-3, 0.2e-3), 20e-6, 2)]
    return I.mesh_desc((8, 4, 2), (125e-6,) * 3, degree, 3, regions, powder_z0=0.15e-3, powder_z1=0.2e-3)


def track_laser(desc, power=300.0, volumetric=False):
    y = desc["ntree"][1] * desc["tree_h"][1] / 2
    return I.laser([(0.1e-3, y, 0.9e-3, y, 0.0, 1e-3)], [power], eta=0.35, radius=40e-6, volumetric=volumetric,
                   h_powder=40e-6)


def to_dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def stable_dt(om, mat):
    lam, _ = om.lambda_max(dict(mat, k0=max(mat["k0"], mat["k1"])), I.start_vector(om.n_dofs), max_iter=300,
                           rtol=1e-8)
    return 0.5 * 2.0 / lam


def fused_run(P, desc, mat, T0, ls, t0, dt, calls, shape=FUSED):
    """calls: list of (shape, nsteps) run back to back on one context."""
    m = P.Mesh(desc)
    ctx = P.Context(m, mat, P.PBF_F32OP)
    Td = to_dev(T0)
    t = t0
    for sh, n in calls:
        P.pbf_ctx_set_kernel_shape(ctx.h, sh)
        P.pbf_explicit_step(ctx.h, Td, ls, t, dt, n)
        t += n * dt
    torch.cuda.synchronize()
    return Td.cpu().numpy(), ctx, m


@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("mat", ["const", "nonlin_nodal"])
@pytest.mark.parametrize("shape", [FUSED, FUSED_PDL, PERSISTENT, *LEAN])
def test_fused_steps_match_oracle(P, oracle_mod, degree, mat, shape):
    desc = amr(degree)
    material = I.TI64_CONST if mat == "const" else I.TI64_NONLIN_Q2
    om = oracle_mod.Mesh(desc)
    dt = stable_dt(om, material)
    T0 = I.melt_pool_field(om.dof_xyz(), (0.3e-3, 0.25e-3, 0.25e-3), 2600.0, 60e-6, seed=11, noise=0.01)
    ls = track_laser(desc)
    ref = om.explicit(material, T0, ls, 1e-4, dt, 12)
    got, _, _ = fused_run(P, desc, material, T0, ls, 1e-4, dt, [(shape, 12)])
    check_f32_steps(got, ref, T0)
    assert np.abs(ref - T0).max() > 1.0  # the steps changed the field


@pytest.mark.parametrize("shape", [FUSED, PERSISTENT, LEAN[0]])
@pytest.mark.parametrize("nsteps", [1, 2, 3])
def test_short_sequences_rotate_accumulators(P, oracle_mod, nsteps, shape):
    """1, 2 and 3 steps (every position of the three-buffer rotation at the final update),
    each followed by a residual that must find all accumulators cleared."""
    desc = amr(2)
    om = oracle_mod.Mesh(desc)
    mat = I.TI64_NONLIN_Q2
    dt = stable_dt(om, mat)
    T0 = I.smooth_field(om.dof_xyz(), seed=12, lo=353.0, hi=2400.0)
    ls = track_laser(desc)
    ref = om.explicit(mat, T0, ls, 2e-4, dt, nsteps)
    got, ctx, m = fused_run(P, desc, mat, T0, ls, 2e-4, dt, [(shape, nsteps)])
    check_f32_steps(got, ref, T0)
    fd, fv, _ = om.residual(mat, got, ls, 3e-4)
    out = [torch.zeros(om.n_dofs, dtype=torch.float64, device="cuda") for _ in range(3)]
    P.pbf_eval_residual(ctx.h, to_dev(got), ls, 3e-4, *out)
    assert rel(out[0].cpu().numpy(), fd) < 2e-5 and rel(out[1].cpu().numpy(), fv) < 2e-5


def test_dirichlet_dofs_start_away_from_td(P, oracle_mod):
    """The first step evaluates the operator at the state as given, Dirichlet dofs included;
    from then on they hold T_D (the oracle's order)."""
    desc = amr(2)
    om = oracle_mod.Mesh(desc)
    mat = I.TI64_CONST
    dt = stable_dt(om, mat)
    T0 = I.smooth_field(om.dof_xyz(), seed=13, lo=400.0, hi=2000.0)
    tab = om.tables()
    assert T0[tab["dirichlet"] != 0].min() > mat["T_dirichlet"]
    ls = track_laser(desc, power=0.0)
    for n, shape in ((1, FUSED), (4, FUSED), (1, PERSISTENT), (4, PERSISTENT), (1, LEAN[0]), (4, LEAN[1])):
        ref = om.explicit(mat, T0, ls, 0.0, dt, n)
        got, _, _ = fused_run(P, desc, mat, T0, ls, 0.0, dt, [(shape, n)])
        check_f32_steps(got, ref, T0)
        assert np.all(got[tab["dirichlet"] != 0] == mat["T_dirichlet"])


def test_volumetric_source_in_fused_steps(P, oracle_mod):
    desc = amr(2)
    desc = dict(desc, active_top_z=0.25e-3)
    om = oracle_mod.Mesh(desc)
    mat = I.TI64_NONLIN_Q2
    dt = stable_dt(om, mat)
    T0 = np.full(om.n_dofs, I.T0)
    ls = track_laser(desc, power=250.0, volumetric=True)
    ref = om.explicit(mat, T0, ls, 1e-4, dt, 8)
    got, _, _ = fused_run(P, desc, mat, T0, ls, 1e-4, dt, [(FUSED_PDL, 4), (PERSISTENT, 4)])
    assert ref.max() > I.T0 + 1.0
    check_f32_steps(got, ref, T0)
    got, _, _ = fused_run(P, desc, mat, T0, ls, 1e-4, dt, [(LEAN[1], 8)])
    assert ref.max() > I.T0 + 1.0
    check_f32_steps(got, ref, T0)


def test_consecutive_calls_mix_forms(P, oracle_mod):
    """Fused, per-cell and fused calls back to back on one context equal one oracle run."""
    desc = amr(2)
    om = oracle_mod.Mesh(desc)
    mat = I.TI64_NONLIN_Q2
    dt = stable_dt(om, mat)
    T0 = I.melt_pool_field(om.dof_xyz(), (0.5e-3, 0.25e-3, 0.25e-3), 2400.0, 80e-6, seed=14, noise=0.01)
    ls = track_laser(desc)
    ref = om.explicit(mat, T0, ls, 0.0, dt, 29)
    got, _, _ = fused_run(P, desc, mat, T0, ls, 0.0, dt,
                          [(FUSED, 5), (PER_CELL, 4), (PERSISTENT, 3), (FUSED_PDL, 8), (LEAN[0], 3), (PERSISTENT, 2),
                           (LEAN[2], 4)])
    check_f32_steps(got, ref, T0)


def test_quadrature_capacity_falls_back(P, oracle_mod):
    """The fused form covers the constant and nodal capacities; with the quadrature-point
    capacity shapes 4/5 run the per-cell form and still match the oracle."""
    desc = amr(1)
    om = oracle_mod.Mesh(desc)
    mat = I.TI64_NONLIN
    dt = stable_dt(om, mat)
    T0 = I.melt_pool_field(om.dof_xyz(), (0.3e-3, 0.25e-3, 0.25e-3), 2600.0, 60e-6, seed=15, noise=0.01)
    ls = track_laser(desc)
    ref = om.explicit(mat, T0, ls, 1e-4, dt, 6)
    got, _, _ = fused_run(P, desc, mat, T0, ls, 1e-4, dt, [(FUSED, 6)])
    check_f32_steps(got, ref, T0)


def test_autotune_times_every_step_form(P):
    desc = amr(2)
    m = P.Mesh(desc)
    ctx = P.Context(m, I.TI64_NONLIN_Q2, P.PBF_F32OP)
    T = torch.full((m.info()["n_dofs"],), 900.0, dtype=torch.float64, device="cuda")
    T0 = T.clone()
    v, us = P.pbf_ctx_autotune(ctx.h, T, reps=3, times=True)
    assert len(us) == 10 and all(u > 0 for u in us) and us[v] == min(us)
    assert torch.equal(T, T0)  # the state is not modified
    print(f"autotune, one instance ({m.info()['n_dofs']} dofs), us per step by shape:", [round(u, 1) for u in us])
    bctx = P.Context(m, I.TI64_NONLIN_Q2, P.PBF_F32OP, 2)  # a batch: the per-cell shapes and shape 4
    Tb = torch.full((2 * m.info()["n_dofs"],), 900.0, dtype=torch.float64, device="cuda")
    v, us = P.pbf_ctx_autotune(bctx.h, Tb, reps=2, times=True)
    print("autotune, batch of 2, us per step by shape:", [round(u, 1) for u in us])
    assert us[4] > 0 and all(u < 0 for u in us[5:]) and v <= 4  # shape 4: the batched fused form


def test_persistent_barrier_time_out_is_reported(P, oracle_mod):
    """The persistent form's grid barrier ends its waits after one second: with the test hook
    the barrier waits for blocks that do not exist, the call returns PBF_ETIMEOUT, and the
    context stays usable (the next call matches the oracle)."""
    import time
    desc = amr(1)
    om = oracle_mod.Mesh(desc)
    mat = I.TI64_CONST
    dt = stable_dt(om, mat)
    T0 = I.smooth_field(om.dof_xyz(), seed=16, lo=353.0, hi=1500.0)
    ls = track_laser(desc)
    m = P.Mesh(desc)
    ctx = P.Context(m, mat, P.PBF_F32OP)
    P.pbf_ctx_set_kernel_shape(ctx.h, PERSISTENT)
    P.pbf_ctx_set_barrier_test(ctx.h, 1)
    Td = to_dev(T0)
    t0 = time.perf_counter()
    with pytest.raises(P.PbfError) as err:
        P.pbf_explicit_step(ctx.h, Td, ls, 0.0, dt, 3)
    assert err.value.status == 6  # PBF_ETIMEOUT
    assert time.perf_counter() - t0 < 10.0
    P.pbf_ctx_set_barrier_test(ctx.h, 0)
    Td = to_dev(T0)
    P.pbf_explicit_step(ctx.h, Td, ls, 0.0, dt, 3)
    torch.cuda.synchronize()
    check_f32_steps(Td.cpu().numpy(), om.explicit(mat, T0, ls, 0.0, dt, 3), T0)


@pytest.mark.parametrize("degree,mat", [(1, "nonlin_nodal"), (2, "nonlin_nodal"), (2, "const")])
def test_batched_fused_steps_match_independent_oracle_runs(P, oracle_mod, degree, mat):
    """The fused step of a batch (shape 4 with batch > 1: one launch per step for all
    instances, the update applied in the gather, hanging nodes from the constraint rows, the
    spot computed on the device, the step sequence replayed as one CUDA graph): a ragged batch
    of three instances with their own segment powers, conductivity scales and initial fields
    equals three independent oracle runs, over two consecutive calls (the second replays the
    graph with a new start time) and after a per-cell call on the same context. The powers keep
    the peak near 5,000-8,000 K: with several hundred kelvin per step across the 12.5 K wide
    latent-heat peak the trajectory amplifies rounding differences by orders of magnitude (FP64
    GPU and oracle then differ by 1e-10 instead of 1e-15), which no FP32 gate survives."""
    desc = amr(degree)
    material = {"nonlin_nodal": I.TI64_NONLIN_Q2, "const": I.TI64_CONST}[mat]
    om = oracle_mod.Mesh(desc)
    B = 3
    s = np.array([0.8, 1.0, 1.2])
    dt = stable_dt(om, dict(material, k0=max(material["k0"], material["k1"]) * 1.2,
                            k1=max(material["k0"], material["k1"]) * 1.2))
    ls = track_laser(desc)
    ls["power"] = np.array([[40.0], [55.0], [70.0]])
    xyz = om.dof_xyz()
    T0 = np.stack([I.melt_pool_field(xyz, (0.3e-3, 0.25e-3, 0.25e-3), 2300.0 + 100 * b, 60e-6, seed=40 + b,
                                     noise=0.01) for b in range(B)], axis=1)
    m = P.Mesh(desc)
    ctx = P.Context(m, material, P.PBF_F32OP, B)
    P.pbf_ctx_set_k_scale(ctx.h, s)
    Td = to_dev(T0.reshape(-1))
    plan = [(FUSED, 6, 1e-4), (FUSED, 6, 1e-4 + 6 * dt), (PER_CELL, 3, 1e-4 + 12 * dt), (FUSED, 5, 1e-4 + 15 * dt)]
    for shape, n, t in plan:
        P.pbf_ctx_set_kernel_shape(ctx.h, shape)
        P.pbf_explicit_step(ctx.h, Td, ls, t, dt, n, batch=B)
    torch.cuda.synchronize()
    got = Td.cpu().numpy().reshape(-1, B)
    for b in range(B):
        ref = om.explicit(material, T0[:, b], ls, 1e-4, dt, 20, s=s[b], instance=b)
        print(f"batched fused, degree {degree}, {mat}, instance {b}:", check_f32_steps(got[:, b], ref, T0[:, b]))
    assert P.pbf_ctx_launch_count(ctx.h) > 0
    ctx.close()
    m.close()
