"""GPU parity of the phase model's history across a mesh change (Sec. 4.1 coarsening rule with
r_coarsen = 0.9; Sec. 2, the consolidated fraction r_c as history data): explicit steps that
melt part of a powder band store r_c on both sides (FP64, 1e-10); the per-cell minima agree;
the gated adaptation gives the oracle's mesh bit-exactly; the transferred history equals the
oracle's transfer exactly (a pure copy); and steps on the new mesh with that history match
the oracle again."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def gpu_history(P, ctx, n_cells, nq):
    out = torch.zeros(nq * n_cells, dtype=torch.float64, device="cuda")
    P.pbf_ctx_get_history(ctx.h, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(nq, n_cells).T  # the oracle's [cell][q]


@pytest.mark.parametrize("p", [1, 2])
def test_history_through_gated_adaptation(P, oracle_mod, p):
    nq = (p + 1) ** 3
    spot0, spot1 = (0.30e-3, 0.25e-3), (0.55e-3, 0.25e-3)
    top = 0.25e-3

    def regions(spot):
        return [I.uniform_region(1), (I.BALL, (spot[0], spot[1], top), (0, 0, 0), 80e-6, 3)]

    d0 = I.mesh_desc((8, 4, 2), (125e-6,) * 3, p, 3, regions(spot0), powder_z0=0.2e-3, powder_z1=0.3e-3)
    mat = I.TI64_CONST
    om = oracle_mod.Mesh(d0)
    om.set_phase(I.PHASE)
    T0 = I.melt_pool_field(om.dof_xyz(), (spot0[0], spot0[1], top), 2200.0, 60e-6, seed=61, noise=0.01)
    lam, _ = oracle_mod.Mesh(d0).lambda_max(dict(mat, k0=30.0, k1=30.0, powder_k_scale=1.0),
                                            I.start_vector(om.n_dofs), max_iter=300, rtol=1e-8)
    dt = 0.4 * 2.0 / lam
    ref = om.explicit(mat, T0, None, 0.0, dt, 6)
    h0 = om.history()
    assert np.any((h0 > 0.0) & (h0 < 0.9)) and np.any(h0 == 0.0)  # partly melted powder
    m = P.Mesh(d0)
    ctx0 = P.Context(m, mat, P.PBF_F64)
    P.pbf_ctx_set_phase(ctx0.h, I.PHASE)
    Td = to_dev(T0)
    P.pbf_explicit_step(ctx0.h, Td, None, 0.0, dt, 6)
    torch.cuda.synchronize()
    assert rel(Td.cpu().numpy(), ref) < 1e-10
    assert np.max(np.abs(gpu_history(P, ctx0, om.n_active, nq) - h0)) < 1e-10
    rc_min = P.pbf_ctx_history_cell_min(ctx0.h, om.n_active)
    assert np.max(np.abs(rc_min - h0.min(axis=1))) < 1e-10
    # the oracle's history in the GPU context, so that the transfer can be compared exactly
    P.pbf_ctx_set_history(ctx0.h, to_dev(h0.T.reshape(-1)))
    # gated adaptation to the moved ball
    r_min = h0.min(axis=1)
    pins = om.gate_pins(r_min, 0.9)
    assert len(pins) > 0
    d1 = dict(d0, regions=regions(spot1) + pins)
    om1 = oracle_mod.Mesh(d1)
    P.pbf_mesh_adapt_gated(m.h, regions(spot1), r_min, 0.9)
    got_t, ref_t = m.tables(), om1.tables()
    for k in ("leaves", "cell_dofs", "con_ptr", "con_idx", "con_w", "dirichlet"):
        assert np.array_equal(got_t[k], ref_t[k]), k
    # the state and the history on the new mesh
    T1 = torch.zeros(om1.n_dofs, dtype=torch.float64, device="cuda")
    P.pbf_mesh_transfer(m.h, Td, T1)
    T1_ref = oracle_mod.transfer(om, ref, om1, -1.0)
    assert rel(T1.cpu().numpy(), T1_ref) < 1e-10
    ctx1 = P.Context(m, mat, P.PBF_F64)
    P.pbf_ctx_set_phase(ctx1.h, I.PHASE)
    P.pbf_ctx_transfer_history(ctx0.h, ctx1.h)
    h1_ref = oracle_mod.transfer_history(om, h0, om1)
    assert np.array_equal(gpu_history(P, ctx1, om1.n_active, nq), h1_ref)
    # steps on the new mesh with the moved history
    om1.set_phase(I.PHASE)
    om1.set_history(h1_ref)
    ref2 = om1.explicit(mat, T1_ref, None, 6 * dt, dt, 4)
    P.pbf_explicit_step(ctx1.h, T1, None, 6 * dt, dt, 4)
    torch.cuda.synchronize()
    assert rel(T1.cpu().numpy(), ref2) < 1e-10
    assert np.max(np.abs(gpu_history(P, ctx1, om1.n_active, nq) - om1.history())) < 1e-10
    # the stale context is refused as a target, and a context of another generation as a source
    with pytest.raises(P.PbfError):
        P.pbf_ctx_transfer_history(ctx1.h, ctx0.h)
    ctx0.close()
    ctx1.close()
    m.close()
