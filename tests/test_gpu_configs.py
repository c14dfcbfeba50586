"""GPU parity at the stated sizes of the configurations that the other tests cover on small
meshes: the part-scale stand-in's first layer (configuration 5, level 4: 1.72 M Q2 dofs,
hanging nodes below the refined band, powder layer, 67-degree hatch) for explicit steps in
both operator precisions, and the adjoint sweep on the full configuration-4 mesh (278,581 Q2
dofs) for two instances over a short window. Tolerances as elsewhere (tests/gates.py; the
adjoint: 1e-10 FP64, 1e-3 FP32)."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from tests.gates import check_f32_steps, check_f64_steps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_05164_gb300 import pbf
    return pbf


def to_dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_c5_first_layer_explicit_steps(P, oracle_mod):
    desc = I.c5_mesh(level=4)
    om = oracle_mod.Mesh(desc)
    assert om.n_dofs > 1_500_000 and om.n_hanging > 0
    mat = I.TI64_NONLIN_Q2
    ls = I.c5_laser()
    # half the critical step of the finest cells (k at its largest), from a small block of them
    h = [t / 16 for t in I.C5_TREE_H]
    ob = oracle_mod.Mesh(I.mesh_desc((1, 1, 1), tuple(4 * v for v in h), 2, 2, [I.uniform_region(2)],
                                     dirichlet_faces=0))
    lam, _ = ob.lambda_max(dict(mat, k0=28.0), I.start_vector(ob.n_dofs), max_iter=500, rtol=1e-9)
    dt = 0.5 * 2.0 / lam
    x0, y0 = ls["seg"][0][0], ls["seg"][0][1]
    top = I.C5_BASE_TOP + I.C5_LAYER
    T0 = I.melt_pool_field(om.dof_xyz(), (x0, y0, top), 2200.0, 80e-6, seed=51, noise=0.01)
    nsteps = 2
    ref = om.explicit(mat, T0, ls, 0.0, dt, nsteps)
    m = P.Mesh(desc)
    for prec in (P.PBF_F64, P.PBF_F32OP):
        ctx = P.Context(m, mat, prec)
        Td = to_dev(T0)
        P.pbf_explicit_step(ctx.h, Td, ls, 0.0, dt, nsteps)
        torch.cuda.synchronize()
        got = Td.cpu().numpy()
        if prec == P.PBF_F64:
            print("C5 level 4, FP64:", check_f64_steps(got, ref, T0))
        else:
            print("C5 level 4, FP32 operator (default shape):", check_f32_steps(got, ref, T0, min_change=10.0))
            for shape in (5, 7):
                P.pbf_ctx_set_kernel_shape(ctx.h, shape)
                Td = to_dev(T0)
                P.pbf_explicit_step(ctx.h, Td, ls, 0.0, dt, nsteps)
                torch.cuda.synchronize()
                print(f"C5 level 4, shape {shape}:", check_f32_steps(Td.cpu().numpy(), ref, T0, min_change=10.0))
        ctx.close()
    m.close()


@pytest.fixture(scope="module")
def c4ref(oracle_mod):
    """The oracle's adjoint on the full configuration-4 mesh: two instances with their own
    segment powers and conductivity scales, six steps over three segments."""
    desc = I.c4_mesh()
    om = oracle_mod.Mesh(desc)
    assert om.n_dofs > 250_000
    mat = I.TI64_NONLIN_Q2
    batch, nsteps, seg = 2, 6, 3
    dt = 2e-8
    Pw, s = I.c4_params(batch, n_seg=seg)
    ls = I.c4_laser(Pw, n_seg=seg, steps_per_seg=nsteps // seg, dt=dt)
    xyz = om.dof_xyz()
    T0 = np.stack([I.melt_pool_field(xyz, (0.05e-3, 0.25e-3, 0.25e-3), 2500.0 + 50 * b, 50e-6, seed=5 + b,
                                     noise=0.01) for b in range(batch)], axis=1)
    ref = [om.adjoint(mat, T0[:, b], ls, 0.0, dt, nsteps, s=s[b], instance=b) for b in range(batch)]
    return dict(desc=desc, mat=mat, batch=batch, nsteps=nsteps, dt=dt, s=s, ls=ls, T0=T0, ref=ref)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_c4_adjoint_full_mesh_two_instances(P, c4ref, prec):
    c = c4ref
    m = P.Mesh(c["desc"])
    ctx = P.Context(m, c["mat"], P.PBF_F64 if prec == "f64" else P.PBF_F32OP, c["batch"])
    P.pbf_ctx_set_k_scale(ctx.h, c["s"])
    J, g, fwd = P.pbf_adjoint_sweep(ctx.h, to_dev(c["T0"]), c["ls"], 0.0, c["dt"], c["nsteps"], 3, batch=c["batch"])
    tol = 1e-10 if prec == "f64" else 1e-3
    for b in range(c["batch"]):
        Jr, gr = c["ref"][b]
        assert abs(J[b] - Jr) < tol * abs(Jr), (b, J[b], Jr)
        assert np.max(np.abs(g[b] - gr)) < tol * np.max(np.abs(gr)), (b, g[b], gr)
    ctx.close()
    m.close()
