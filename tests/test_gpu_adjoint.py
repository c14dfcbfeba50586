"""GPU parity of the adjoint sweep (transposed linearised cell operator incl. the k'(T) term
and the capacity derivative, parameter gradients, binomial checkpointing) with the oracle's
adjoint, which stores every state. Tolerances: FP64 operator 1e-10 relative on J and on the
gradient vector (max-norm); FP32 operator 1e-3."""
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


def setup(p, lumping, batch, nsteps=12, seg=3):
    d = I.mesh_desc((4, 2, 2), (62.5e-6,) * 3, p, 2,
                    [I.uniform_region(1), (I.BALL, (0.1e-3, 0.06e-3, 0.125e-3), (0, 0, 0), 40e-6, 2)])
    mat = dict(I.TI64_NONLIN, lumping=lumping)
    dt = 1e-7 if p == 1 else 4e-8
    steps_per_seg = -(-nsteps // seg)
    P_, s = I.c4_params(batch, n_seg=seg, seed=2302)
    ls = I.c4_laser(P_, n_seg=seg, steps_per_seg=steps_per_seg, dt=dt, v=0.5, y=0.06e-3)
    return d, mat, dt, ls, s


def oracle_ref(oracle_mod, d, mat, T0, ls, dt, nsteps, s):
    om = oracle_mod.Mesh(d)
    out = []
    for b in range(len(s)):
        J, g = om.adjoint(mat, T0[:, b] if T0.ndim == 2 else T0, ls, 0.0, dt, nsteps, s=s[b], instance=b)
        out.append((J, g))
    return out


@pytest.mark.parametrize("p,lumping,prec,batch,ckpt", [
    (1, I.LUMP_QUADRATURE, "f64", 2, 3),
    (2, I.LUMP_NODAL, "f64", 1, 4),
    (1, I.LUMP_QUADRATURE, "f64", 1, 1),
    (2, I.LUMP_NODAL, "f32", 2, 3),
])
def test_adjoint_matches_oracle(P, oracle_mod, p, lumping, prec, batch, ckpt):
    d, mat, dt, ls, s = setup(p, lumping, batch)
    om = oracle_mod.Mesh(d)
    xyz = om.dof_xyz()
    T0 = np.stack([I.melt_pool_field(xyz, (0.08e-3, 0.06e-3, 0.125e-3), 2500.0 + 50 * b, 50e-6, seed=b, noise=0.01)
                   for b in range(batch)], axis=1)
    nsteps = 12
    ref = oracle_ref(oracle_mod, d, mat, T0, ls, dt, nsteps, s)
    m = P.Mesh(d)
    ctx = P.Context(m, mat, P.PBF_F64 if prec == "f64" else P.PBF_F32OP, batch)
    P.pbf_ctx_set_k_scale(ctx.h, s)
    T0d = torch.tensor(np.ascontiguousarray(T0), dtype=torch.float64, device="cuda")
    J, g, fwd = P.pbf_adjoint_sweep(ctx.h, T0d, ls, 0.0, dt, nsteps, ckpt, batch=batch)
    tol = 1e-10 if prec == "f64" else 1e-3
    for b in range(batch):
        Jr, gr = ref[b]
        assert abs(J[b] - Jr) < tol * abs(Jr)
        assert np.max(np.abs(g[b] - gr)) < tol * np.max(np.abs(gr)), (g[b], gr)
    assert fwd >= nsteps
    if ckpt == 1:
        assert fwd == nsteps + nsteps * (nsteps - 1) // 2  # no snapshots: quadratic recomputation
    # the state passed in is not modified
    assert np.array_equal(T0d.cpu().numpy(), T0)


@pytest.mark.parametrize("p,lumping", [(1, I.LUMP_QUADRATURE), (2, I.LUMP_NODAL)])
def test_adjoint_matches_central_differences(P, oracle_mod, p, lumping):
    """The GPU adjoint's gradient against central finite differences of the GPU's own
    objective (h = 1e-4 relative per parameter, FP64 operator). The perturbed runs are extra
    instances of the same batch: instance 0 holds the parameters, instances 2k+1 / 2k+2 the
    +h / -h perturbation of parameter k (three segment powers, then the conductivity scale)."""
    d = I.mesh_desc((4, 2, 2), (62.5e-6,) * 3, p, 1, [I.uniform_region(1)])
    xyz = oracle_mod.Mesh(d).dof_xyz()
    mat = dict(I.TI64_NONLIN, lumping=lumping)
    T0 = I.smooth_field(xyz, seed=11, lo=353.0, hi=2400.0)
    dt, nst = 2e-7, 12
    P0, s0 = np.array([180.0, 220.0, 240.0]), 1.05
    params = np.concatenate([P0, [s0]])
    m_par = params.size
    h = 1e-4 * params
    B = 1 + 2 * m_par
    powers = np.tile(P0, (B, 1))
    scales = np.full(B, s0)
    for k in range(m_par):
        for sign, b in ((1.0, 2 * k + 1), (-1.0, 2 * k + 2)):
            if k < P0.size:
                powers[b, k] += sign * h[k]
            else:
                scales[b] += sign * h[k]
    ls = I.c4_laser(powers, n_seg=3, steps_per_seg=4, dt=dt, v=0.5, y=0.25e-3)
    m = P.Mesh(d)
    ctx = P.Context(m, mat, P.PBF_F64, B)
    P.pbf_ctx_set_k_scale(ctx.h, scales)
    T0d = torch.tensor(np.repeat(T0[:, None], B, axis=1), dtype=torch.float64, device="cuda")
    J, g, _ = P.pbf_adjoint_sweep(ctx.h, T0d, ls, 0.0, dt, nst, 4, batch=B)
    assert J[0] > 0 and np.all(np.isfinite(g))
    fd = np.array([(J[2 * k + 1] - J[2 * k + 2]) / (2 * h[k]) for k in range(m_par)])
    for k in range(m_par):
        assert abs(g[0, k] - fd[k]) < 1e-5 * max(abs(fd[k]), 1e-3 * np.abs(g[0]).max()), (k, g[0, k], fd[k])


def test_autograd_function_gives_the_adjoint_gradient(P, oracle_mod):
    """ThermalObjective (torch.autograd.Function over pbf_adjoint_sweep): J and the gradients
    that torch's backward delivers for P and s, with a non-uniform upstream gradient, equal
    the oracle's adjoint per instance (FP64 operator, 1e-10)."""
    from paper_2302_05164_gb300.autograd import ThermalObjective
    batch = 2
    d, mat, dt, ls, s = setup(2, I.LUMP_NODAL, batch)
    om = oracle_mod.Mesh(d)
    T0 = np.stack([I.melt_pool_field(om.dof_xyz(), (0.08e-3, 0.06e-3, 0.125e-3), 2500.0 + 50 * b, 50e-6, seed=b,
                                     noise=0.01) for b in range(batch)], axis=1)
    nsteps = 12
    ref = oracle_ref(oracle_mod, d, mat, T0, ls, dt, nsteps, s)
    m = P.Mesh(d)
    ctx = P.Context(m, mat, P.PBF_F64, batch)
    T0d = torch.tensor(np.ascontiguousarray(T0), dtype=torch.float64, device="cuda")
    Pt = torch.tensor(np.asarray(ls["power"]), dtype=torch.float64, requires_grad=True)
    st = torch.tensor(s, dtype=torch.float64, requires_grad=True)
    J = ThermalObjective.apply(Pt, st, ctx.h, T0d, ls, 0.0, dt, nsteps, 4)
    w = torch.tensor([0.7, -1.3], dtype=torch.float64)
    (w * J).sum().backward()
    n_seg = Pt.shape[1]
    for b in range(batch):
        Jr, gr = ref[b]
        assert abs(float(J[b].detach()) - Jr) < 1e-10 * abs(Jr)
        got = np.concatenate([Pt.grad[b].numpy(), [float(st.grad[b])]])
        assert got.shape == (n_seg + 1,)
        assert np.max(np.abs(got - float(w[b]) * gr)) < 1e-10 * np.max(np.abs(gr))
    assert np.array_equal(T0d.cpu().numpy(), T0)
