"""Pins of the oracle's finite-element operator, time steppers, solvers and adjoint against
what the paper and the mathematics fix: textbook element matrices, closed forms, the paper's
printed critical time step, conservation, exact polynomial reproduction and finite
differences. A plausible slip anywhere in the oracle (dropped term, wrong sign, transposed
index, wrong metric factor) fails at least one of these."""
import math
import os

import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from tests import textbook as TB

def golden(name):
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


UNIT = dict(rho=1.0, c=1.0, k0=1.0, k1=1.0, Tk0=0.0, Tk1=0.0, latent=0.0, Tm=0.0, sigma=0.0,
            powder_k_scale=0.1, T_dirichlet=0.0)


def amr_desc(p, dirichlet=0, top=1e30):
    regions = [(I.BALL, (0.35, 0.4, 0.9), (0, 0, 0), 0.45, 3),
               (I.BOX, (1.2, 0.2, 0.3), (1.3, 0.3, 0.5), 0.05, 2)]
    return I.mesh_desc((2, 1, 1), (1.0, 1.0, 1.0), p, 3, regions, dirichlet_faces=dirichlet, active_top_z=top)


def interior(m, desc):
    c = m.tables()["dof_coord"]
    N = np.array(desc["ntree"]) * desc["degree"] << desc["max_level"]
    return np.all((c > 0) & (c < N), axis=1)


@pytest.mark.parametrize("p", [1, 2])
def test_operator_equals_textbook_kronecker(oracle_mod, p):
    ntree, L = (3, 2, 1), 1
    th = (0.4, 0.3, 0.5)
    d = I.mesh_desc(ntree, th, p, L, [I.uniform_region(L)])
    m = oracle_mod.Mesh(d)
    ncell = [n << L for n in ntree]
    h = [t / (1 << L) for t in th]
    K, M = TB.brick_matrices(p, ncell, h)
    lex = TB.lex_index(m.tables()["dof_coord"], p, ncell)
    mat = dict(UNIT, k0=2.5, k1=2.5, rho=3.0, c=0.7)
    T = np.random.default_rng(0).normal(size=m.n_dofs)
    Tl = np.zeros(K.shape[0])
    Tl[lex] = T
    fd, fv, Cm = m.residual(mat, T)
    ref = -2.5 * (K @ Tl)[lex]
    assert np.max(np.abs(fd - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.allclose(Cm, 3.0 * 0.7 * M.sum(axis=1)[lex], rtol=1e-13, atol=0)
    assert np.all(fv == 0)


@pytest.mark.parametrize("p", [1, 2])
def test_patch_test_across_hanging_faces(oracle_mod, p):
    d = amr_desc(p)
    m = oracle_mod.Mesh(d)
    assert m.n_hanging > 0
    x = m.dof_xyz()
    inner = interior(m, d)
    k = 1.7
    mat = dict(UNIT, k0=k, k1=k)
    if p == 1:
        # linear field: zero residual on every interior dof
        u = 0.3 + 1.1 * x[:, 0] - 0.7 * x[:, 1] + 2.0 * x[:, 2]
        fd, _, Cm = m.residual(mat, u)
        assert np.max(np.abs(fd[inner])) < 1e-12
    else:
        # quadratic field, Laplacian 2*(1 + 2 - 0.5): f_i = k lap(u) int N_i on interior dofs
        u = x[:, 0] ** 2 + 2 * x[:, 1] ** 2 - 0.5 * x[:, 2] ** 2 + 0.3 * x[:, 0] * x[:, 1] + x[:, 2]
        fd, _, Cm = m.residual(mat, u)
        lap = 2 * (1 + 2 - 0.5)
        err = fd[inner] - k * lap * Cm[inner]
        assert np.max(np.abs(err)) < 1e-12 * np.max(np.abs(fd[inner]))


def test_nonlinear_conductivity_closed_form(oracle_mod):
    """u = Ta + a x with k(T) linear on the ramp: div(k grad u) = k' a^2 exactly (Q2)."""
    d = amr_desc(2)
    m = oracle_mod.Mesh(d)
    x = m.dof_xyz()
    mat = dict(UNIT, k0=6.7, k1=28.0, Tk0=300.0, Tk1=1928.0)
    a = 400.0
    u = 700.0 + a * x[:, 0]  # 700..1500 K over x in [0, 2]: inside the ramp
    fd, _, Cm = m.residual(mat, u)
    inner = interior(m, d)
    kp = (28.0 - 6.7) / (1928.0 - 300.0)
    ref = kp * a * a * Cm[inner]
    assert np.max(np.abs(fd[inner] - ref)) < 1e-10 * np.max(np.abs(ref))
    # powder cells scale k; a conductivity scale s scales f_diff linearly
    fd2, _, _ = m.residual(mat, u, s=1.3)
    assert np.allclose(fd2, 1.3 * fd, rtol=1e-12, atol=1e-12 * np.abs(fd).max())


@pytest.mark.parametrize("p", [1, 2])
def test_conservation_symmetry_capacity(oracle_mod, p):
    d = amr_desc(p, top=0.8)
    m = oracle_mod.Mesh(d)
    rng = np.random.default_rng(1)
    mat = dict(I.TI64_NONLIN)
    T = rng.uniform(300, 2600, m.n_dofs)
    fd, _, Cm = m.residual(mat, T)
    assert abs(fd.sum()) < 1e-12 * np.abs(fd).sum()          # K 1 = 0: no flux leaves
    lin = dict(UNIT, k0=2.0, k1=2.0)
    xa, xb = rng.normal(size=(2, m.n_dofs))
    ka, _, _ = m.residual(lin, xa)
    kb, _, _ = m.residual(lin, xb)
    assert abs(xb @ ka - xa @ kb) < 1e-12 * abs(xb @ ka)      # symmetric stiffness
    Cc = m.lumped_capacity(dict(UNIT, rho=2.0, c=3.0), T)
    lv = m.tables()["leaves"]
    vol = float(((0.5 ** lv[:, 3]) ** 3 * lv[:, 4]).sum())   # union of active cells
    assert np.all(Cc > 0) and abs(Cc.sum() - 6.0 * vol) < 1e-12 * 6.0 * vol


def test_apparent_capacity_integrates_latent_heat(oracle_mod):
    mat = I.TI64_NONLIN
    T = np.linspace(mat["Tm"] - 20 * mat["sigma"], mat["Tm"] + 20 * mat["sigma"], 40001)
    c = np.array([oracle_mod.capp(mat, t) for t in T])
    lat = np.trapezoid(c - mat["c"], T)
    assert abs(lat - mat["latent"]) < 1e-8 * mat["latent"]
    peak = mat["c"] + mat["latent"] / (mat["sigma"] * math.sqrt(2 * math.pi))
    assert abs(oracle_mod.capp(mat, mat["Tm"]) - peak) < 1e-9 * peak
    # conductivity: clamped linear ramp
    assert oracle_mod.cond(mat, 100.0) == 6.7 and oracle_mod.cond(mat, 5000.0) == 28.0
    assert abs(oracle_mod.cond(mat, 1114.0) - (6.7 + 21.3 * 0.5)) < 1e-12
    assert abs(oracle_mod.cond(mat, 1114.0, 1, 1.2) - 0.1 * 1.2 * (6.7 + 21.3 * 0.5)) < 1e-12
    # uniform state: lumped capacity integrates rho c_app(T*)
    m = oracle_mod.Mesh(amr_desc(2))
    Cm = m.lumped_capacity(mat, np.full(m.n_dofs, 1900.0))
    assert abs(Cm.sum() - mat["rho"] * oracle_mod.capp(mat, 1900.0) * 2.0) < 1e-10 * Cm.sum()


def test_lumped_capacity_sign_q1_q2(oracle_mod):
    """Row-sum lumping of a capacity with a sharp c_app(T) peak: Q1 bases are non-negative, so
    C~_ii = int rho c_app(T_h) N_i > 0; Q2 vertex bases are negative inside the cell, so the
    same row sum turns negative where the latent peak sits there, while the nodal form
    rho c_app(T_i) sum_j M_ij stays positive. Both forms agree for constant c."""
    rng = np.random.default_rng(8)
    for p in (1, 2):
        d = I.mesh_desc((2, 2, 2), (1e-4,) * 3, p, 2, [I.uniform_region(2)])
        m = oracle_mod.Mesh(d)
        T = I.T0 + rng.uniform(1850.0, 1960.0, m.n_dofs) - I.T0  # nodes around the latent peak
        Cq = m.lumped_capacity(I.TI64_NONLIN, T)
        Cn = m.lumped_capacity(dict(I.TI64_NONLIN, lumping=I.LUMP_NODAL), T)
        assert Cn.min() > 0
        if p == 1:
            assert Cq.min() > 0
        else:
            assert Cq.min() < 0
        const = np.full(m.n_dofs, 600.0)
        a = m.lumped_capacity(I.TI64_NONLIN, const)
        b = m.lumped_capacity(dict(I.TI64_NONLIN, lumping=I.LUMP_NODAL), const)
        assert np.allclose(a, b, rtol=1e-12, atol=0)
    # nodal form: c_app evaluated at the node, times the constant-coefficient lumped mass
    m = oracle_mod.Mesh(I.mesh_desc((2, 1, 1), (1e-4,) * 3, 2, 1, [I.uniform_region(1)]))
    T = rng.uniform(1850.0, 1960.0, m.n_dofs)
    M = m.lumped_capacity(dict(I.TI64_CONST, rho=1.0, c=1.0), T)
    Cn = m.lumped_capacity(dict(I.TI64_NONLIN, lumping=I.LUMP_NODAL), T)
    ref = np.array([I.TI64_NONLIN["rho"] * oracle_mod.capp(I.TI64_NONLIN, t) for t in T]) * M
    assert np.allclose(Cn, ref, rtol=1e-12, atol=0)


def test_laser_total_power(oracle_mod):
    """The surface Gaussian 2 eta P/(pi r^2) exp(-2 d^2/r^2) integrates to eta P."""
    d = I.mesh_desc((4, 4, 1), (100e-6, 100e-6, 100e-6), 2, 3, [I.uniform_region(3)])
    m = oracle_mod.Mesh(d)
    ls = I.laser([(0.2e-3, 0.2e-3, 0.2e-3, 0.2e-3, 0.0, 1.0)], [200.0], eta=0.35, radius=40e-6)
    _, fv, _ = m.residual(I.TI64_CONST, np.full(m.n_dofs, 353.0), ls, t=0.5)
    assert abs(fv.sum() - 70.0) < 1e-4 * 70.0
    # off-time: no source; segment timing is [t0, t1)
    _, fv0, _ = m.residual(I.TI64_CONST, np.full(m.n_dofs, 353.0), ls, t=1.0)
    assert np.all(fv0 == 0)


def test_volumetric_source_total_power_and_depth(oracle_mod):
    """The cylinder source 2 eta P/(pi r^2 h_p) exp(-2 d^2/r^2) on -h_p < z^ < 0 (Eq.
    heat_soruce_cylindrical, bound read as below the active top) integrates to eta P when the
    cylinder lies inside the domain with cell faces at depth h_p, and loads only the dofs of
    cells that reach into the powder band."""
    d = I.mesh_desc((4, 4, 1), (100e-6, 100e-6, 100e-6), 2, 3, [I.uniform_region(3)], active_top_z=0.1e-3)
    m = oracle_mod.Mesh(d)
    ls = I.laser([(0.2e-3, 0.2e-3, 0.2e-3, 0.2e-3, 0.0, 1.0)], [200.0], eta=0.35, radius=40e-6, volumetric=True,
                 h_powder=50e-6)
    _, fv, _ = m.residual(I.TI64_CONST, np.full(m.n_dofs, 353.0), ls, t=0.5)
    assert abs(fv.sum() - 70.0) < 1e-4 * 70.0
    z = m.dof_xyz()[:, 2]
    assert np.all(fv[z < 0.05e-3 - 1e-12] == 0.0) and fv[z > 0.05e-3 + 1e-12].max() > 0.0


def test_critical_time_step_closed_form_and_paper_value(oracle_mod):
    # uniform Q1, lumped capacity, Neumann: lambda_max(C~^-1 K) = 4 alpha / h^2 exactly
    d = I.mesh_desc((2, 2, 2), (1.0, 1.0, 1.0), 1, 2, [I.uniform_region(2)], dirichlet_faces=0)
    m = oracle_mod.Mesh(d)
    mat = dict(UNIT, k0=3.0, k1=3.0, rho=2.0, c=1.5)
    lam, it = m.lambda_max(mat, I.start_vector(m.n_dofs), max_iter=2000, rtol=1e-13)
    alpha, h = 3.0 / 3.0, 0.25
    assert abs(lam - 4 * alpha / h ** 2) < 1e-6 * lam
    # Paper, Sec. 5.1: bridge material (Table mat_params) on 40 um Q1 cells gives
    # dt_max = 2.9e-4 s from Eq. (explicit_time_step)
    g = golden("bridge_critical_dt.txt")
    mat = dict(I.BRIDGE, k0=g["k_W_per_mK"], k1=g["k_W_per_mK"], rho=g["rho_kg_per_m3"], c=g["c_J_per_kgK"])
    d = I.mesh_desc((2, 2, 2), (4 * g["h_m"],) * 3, 1, 2, [I.uniform_region(2)])
    m = oracle_mod.Mesh(d)
    lam, it = m.lambda_max(mat, I.start_vector(m.n_dofs), max_iter=3000, rtol=1e-10)
    dt = 2.0 / lam
    assert round(dt, 5) == g["dt_max_s"]


def test_explicit_cosine_mode_multiplier(oracle_mod):
    """Q1 lumped, Neumann: cos(pi x) at the nodes is an eigenvector of C~^-1 K with
    eigenvalue alpha (2/h^2)(1 - cos(pi h)); one Euler step multiplies it by 1 - dt lambda."""
    n = 16
    d = I.mesh_desc((n, 1, 1), (1.0 / n,) * 3, 1, 0, [], dirichlet_faces=0)
    m = oracle_mod.Mesh(d)
    x = m.dof_xyz()[:, 0]
    h = 1.0 / n
    mat = dict(UNIT, k0=0.8, k1=0.8, rho=2.0, c=0.5)
    alpha = 0.8
    lam = alpha * 2 / h ** 2 * (1 - math.cos(math.pi * h))
    dt = 0.9 / (4 * alpha / h ** 2)  # stable: dt lambda_max = 0.9 < 2
    T0 = 10.0 + np.cos(math.pi * x)
    T1 = m.explicit(mat, T0, None, 0.0, dt, 3)
    assert np.max(np.abs(T1 - (10.0 + (1 - dt * lam) ** 3 * np.cos(math.pi * x)))) < 1e-13


def test_explicit_q2_converges_to_exact_decay(oracle_mod):
    errs = []
    for n in (4, 8):
        d = I.mesh_desc((n, 1, 1), (1.0 / n,) * 3, 2, 0, [], dirichlet_faces=0)
        m = oracle_mod.Mesh(d)
        x = m.dof_xyz()[:, 0]
        lam, _ = m.lambda_max(UNIT, I.start_vector(m.n_dofs), max_iter=500, rtol=1e-10)
        t_end = 0.02
        nst = int(math.ceil(t_end / (0.25 / lam)))
        dt = t_end / nst
        T = m.explicit(UNIT, np.cos(math.pi * x), None, 0.0, dt, nst)
        errs.append(np.max(np.abs(T - math.exp(-math.pi ** 2 * t_end) * np.cos(math.pi * x))))
    assert errs[1] < errs[0] / 3.5


def kron_implicit(p, ntree, L, th, mat, dt):
    ncell = [n << L for n in ntree]
    h = [t / (1 << L) for t in th]
    K, M = TB.brick_matrices(p, ncell, h)
    return mat["rho"] * mat["c"] / dt * M + mat["k0"] * K


def test_implicit_step_matches_dense_solve(oracle_mod):
    p, ntree, L, th = 1, (2, 2, 1), 2, (1e-4, 1e-4, 1e-4)
    d = I.mesh_desc(ntree, th, p, L, [I.uniform_region(L)])
    m = oracle_mod.Mesh(d)
    mat = dict(I.TI64_CONST)
    dt = 1e-2
    A = kron_implicit(p, ntree, L, th, mat, dt)
    t = m.tables()
    lex = TB.lex_index(t["dof_coord"], p, [n << L for n in ntree])
    free = t["dirichlet"] == 0
    rng = np.random.default_rng(5)
    T = 353.0 + np.where(free, rng.uniform(0, 1000, m.n_dofs), 0.0)
    lmin, lmax = m.lanczos_bounds(mat, dt, I.start_vector(m.n_dofs))
    T1, iters, st = m.implicit(mat, T, dt, 1, 1e-13, 200, 5, lmin, 1.1 * lmax)
    assert st == 0
    # dense: (C/dt + K) dT = -K T on free rows, dT = 0 on Dirichlet rows
    Al = np.zeros_like(A)
    Al[np.ix_(lex, lex)] = 0
    P = np.zeros((m.n_dofs, A.shape[0]))
    P[np.arange(m.n_dofs), lex] = 1.0
    Ad = P @ A @ P.T
    Kd = P @ (kron_implicit(p, ntree, L, th, dict(mat, rho=0.0), dt)) @ P.T
    rhs = -(Kd @ T)
    f = free
    dT = np.zeros(m.n_dofs)
    dT[f] = np.linalg.solve(Ad[np.ix_(f, f)], rhs[f])
    assert np.max(np.abs(T1 - (T + dT))) < 1e-9 * np.max(np.abs(dT))
    assert iters[0] < 60


def test_chebyshev_is_the_shifted_chebyshev_polynomial(oracle_mod):
    p, ntree, L, th = 1, (2, 1, 1), 1, (1e-4, 1e-4, 1e-4)
    d = I.mesh_desc(ntree, th, p, L, [I.uniform_region(L)])
    m = oracle_mod.Mesh(d)
    mat = dict(I.TI64_CONST)
    dt = 1e-3
    t = m.tables()
    lex = TB.lex_index(t["dof_coord"], p, [n << L for n in ntree])
    P = np.zeros((m.n_dofs, len(lex)))
    P[np.arange(m.n_dofs), lex] = 1.0
    A = P @ kron_implicit(p, ntree, L, th, mat, dt) @ P.T
    f = t["dirichlet"] == 0
    Af = A[np.ix_(f, f)]
    D = np.diag(Af).copy()
    assert np.allclose(m.implicit_diagonal(mat, dt)[f], D, rtol=1e-13)
    S = Af / np.sqrt(np.outer(D, D))
    ev, V = np.linalg.eigh(S)
    lmin, lmax = 0.9 * ev.min(), 1.1 * ev.max()
    r = np.zeros(m.n_dofs)
    r[f] = np.random.default_rng(2).normal(size=f.sum())
    deg = 5
    z = m.chebyshev(mat, dt, deg, lmin, lmax, r)
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    kdeg = deg + 1  # residual polynomial degree after deg+1 Chebyshev steps
    resid = np.cos(kdeg * np.arccos(np.clip((theta - ev) / delta, -1, 1))) / np.cosh(kdeg * np.arccosh(theta / delta))
    poly = (1 - resid) / ev                     # z = p(D^-1 A) D^-1 r, 1 - lambda p = residual
    zs = V @ (poly * (V.T @ (r[f] / np.sqrt(D))))
    zref = zs / np.sqrt(D)
    assert np.max(np.abs(z[f] - zref)) < 1e-10 * np.max(np.abs(zref))
    # Lanczos bounds from 30 Jacobi-PCG steps approach the extreme eigenvalues of D^-1 A
    lo, hi = m.lanczos_bounds(mat, dt, I.start_vector(m.n_dofs), 30)
    assert abs(hi - ev.max()) < 1e-6 * ev.max() and abs(lo - ev.min()) < 1e-6 * ev.min()


@pytest.mark.parametrize("p,lumping", [(1, I.LUMP_QUADRATURE), (2, I.LUMP_NODAL)])
def test_adjoint_matches_central_differences(oracle_mod, p, lumping):
    d = I.mesh_desc((4, 2, 2), (62.5e-6,) * 3, p, 1, [I.uniform_region(1)])
    m = oracle_mod.Mesh(d)
    mat = dict(I.TI64_NONLIN, lumping=lumping)
    T0 = I.smooth_field(m.dof_xyz(), seed=11, lo=353.0, hi=2400.0)
    dt, nst = 2e-7, 12
    ls = I.c4_laser([[180.0, 220.0, 240.0]], n_seg=3, steps_per_seg=4, dt=dt, v=0.5, y=0.25e-3)
    s = 1.05
    J, g = m.adjoint(mat, T0, ls, 0.0, dt, nst, s=s)
    assert J > 0 and np.all(np.isfinite(g))
    for k in range(4):
        pw = ls["power"].copy()
        if k < 3:
            h = 1e-4 * pw[0, k]
            lp, lm = dict(ls, power=pw.copy()), dict(ls, power=pw.copy())
            lp["power"][0, k] += h
            lm["power"][0, k] -= h
            fd = (m.objective(mat, T0, lp, 0.0, dt, nst, s=s) - m.objective(mat, T0, lm, 0.0, dt, nst, s=s)) / (2 * h)
        else:
            h = 1e-4 * s
            fd = (m.objective(mat, T0, ls, 0.0, dt, nst, s=s + h) - m.objective(mat, T0, ls, 0.0, dt, nst, s=s - h)) / (2 * h)
        assert abs(g[k] - fd) < 1e-5 * max(abs(fd), 1e-3 * np.abs(g).max()), (k, g[k], fd)


@pytest.mark.parametrize("p", [1, 2])
def test_transfer_reproduces_polynomials_and_fills_new_cells(oracle_mod, p):
    a = oracle_mod.Mesh(amr_desc(p, top=0.75))
    regions = [(I.BALL, (1.5, 0.5, 0.9), (0, 0, 0), 0.3, 3)]
    b = oracle_mod.Mesh(I.mesh_desc((2, 1, 1), (1.0,) * 3, p, 3, regions, active_top_z=0.875))
    rng = np.random.default_rng(4)
    coef = rng.normal(size=(p + 1, p + 1, p + 1))

    def u(x):
        return sum(coef[i, j, k] * x[:, 0] ** i * x[:, 1] ** j * x[:, 2] ** k
                   for i in range(p + 1) for j in range(p + 1) for k in range(p + 1))
    xa, xb = a.dof_xyz(), b.dof_xyz()
    Tb = oracle_mod.transfer(a, u(xa), b, -7.0)
    lv = a.tables()["leaves"]
    act = lv[lv[:, 4] == 1]
    lo = act[:, :3] * p
    hi = lo + p * (1 << (3 - act[:, 3]))[:, None]
    cb = b.tables()["dof_coord"]
    old = np.array([np.any(np.all((lo <= c) & (c <= hi), axis=1)) for c in cb])
    assert old.sum() < b.n_dofs
    assert np.max(np.abs(Tb[old] - u(xb[old]))) < 1e-12 * np.abs(u(xb)).max()
    assert np.all(Tb[~old] == -7.0)


# ---- radiation and evaporation on the free top surface (Eqs. bc_rad_evap, bc_radiation,
# bc_evaporation) ------------------------------------------------------------------------

def paper_surface_flux(q, T):
    """Transcription of Eqs. bc_radiation and bc_evaporation for the checks below."""
    out = q["emissivity"] * 5.670374419e-8 * (T ** 4 - q["T_amb"] ** 4)
    Tc = min(T, q["T_max"])
    if q["C_P"] > 0 and Tc > q["T_v"]:
        mdot = 0.82 * q["C_P"] * math.exp(-q["C_T"] * (1.0 / Tc - 1.0 / q["T_v"])) * math.sqrt(q["C_M"] / Tc)
        out += mdot * (q["h_v"] + q["c_h"] * (Tc - q["T_h0"]))
    return out


def test_surface_flux_branches(oracle_mod):
    q = I.SURFACE_LOSS
    for T in (353.0, 1500.0, 2999.0, 3000.0, 3001.0, 3500.0, 4000.0, 4500.0):
        got = oracle_mod.surface_flux(q, T)
        assert abs(got - paper_surface_flux(q, T)) <= 1e-13 * abs(got) + 1e-9
    # capped: the evaporation part is constant above T_max, radiation keeps growing
    rad = lambda T: q["emissivity"] * 5.670374419e-8 * (T ** 4 - q["T_amb"] ** 4)
    e1 = oracle_mod.surface_flux(q, 4200.0) - rad(4200.0)
    e2 = oracle_mod.surface_flux(q, 4700.0) - rad(4700.0)
    assert abs(e1 - e2) < 1e-9 * abs(e1) and e1 > 0
    assert oracle_mod.surface_flux(q, q["T_amb"]) == 0.0
    assert oracle_mod.surface_flux(dict(q, emissivity=0.0), 2900.0) == 0.0


def test_surface_flux_derivative_matches_differences(oracle_mod):
    """q'(T) of the adjoint's face term against Richardson-extrapolated central differences of
    the transcribed Eqs. bc_radiation and bc_evaporation, inside each branch: radiation only,
    radiation with evaporation, and above the evaporation cap (radiation only again)."""
    q = I.SURFACE_LOSS

    def cd(T, h):
        return (paper_surface_flux(q, T + h) - paper_surface_flux(q, T - h)) / (2 * h)

    for T in (353.0, 1500.0, 2900.0, 3100.0, 3500.0, 3900.0, 4200.0, 5000.0):
        # 1 K: Richardson is exact for T^4, the evaporation part varies on T^2 / C_T ~ 200 K,
        # and a smaller step loses digits to the large capped flux above T_max
        h = 1.0
        ref = (4 * cd(T, h / 2) - cd(T, h)) / 3
        got = oracle_mod.surface_flux_deriv(q, T)
        assert abs(got - ref) <= 1e-8 * abs(ref), (T, got, ref)
    # the evaporation part dominates the derivative between T_v and T_max
    assert oracle_mod.surface_flux_deriv(q, 3500.0) > 100 * oracle_mod.surface_flux_deriv(dict(q, C_P=0.0), 3500.0)


@pytest.mark.parametrize("p", [1, 2])
def test_adjoint_with_surface_loss_matches_central_differences(oracle_mod, p):
    """With radiation and evaporation on the top surface (explicit, at each step's state) the
    adjoint gradient (dJ/dP per segment and dJ/ds) equals central differences of the objective
    to 1e-5, on a brick whose top reaches 3600 K under the laser track, so that evaporation is
    active; the loss's face term moves every gradient component by a large fraction of itself,
    so a dropped or wrong term fails. The step, 5 us, stays inside the loss term's own
    stability limit (dt q'(T) 2 / (rho c h) below 1 at 3600 K)."""
    d = I.mesh_desc((4, 2, 2), (125e-6,) * 3, p, 1, [I.uniform_region(1)])
    m = oracle_mod.Mesh(d)
    mat = dict(I.TI64_NONLIN, lumping=I.LUMP_QUADRATURE if p == 1 else I.LUMP_NODAL)
    dt, nst, s, Tt = 5e-6, 12, 1.05, 3000.0
    T0 = I.melt_pool_field(m.dof_xyz(), (0.25e-3, 0.125e-3, 0.25e-3), 3600.0, 90e-6, seed=11, noise=0.01)
    ls = I.c4_laser([[180.0, 220.0, 240.0]], n_seg=3, steps_per_seg=4, dt=dt, v=0.5, y=0.125e-3)
    _, g0 = m.adjoint(mat, T0, ls, 0.0, dt, nst, s=s, T_target=Tt)
    m.set_surface_loss(I.SURFACE_LOSS)
    J, g = m.adjoint(mat, T0, ls, 0.0, dt, nst, s=s, T_target=Tt)
    assert J > 0 and np.all(np.isfinite(g))

    def obj(ls_, s_):
        return m.objective(mat, T0, ls_, 0.0, dt, nst, s=s_, T_target=Tt)

    for k in range(4):
        pw = ls["power"].copy()
        if k < 3:
            h = 1e-4 * pw[0, k]
            lp, lm = dict(ls, power=pw.copy()), dict(ls, power=pw.copy())
            lp["power"][0, k] += h
            lm["power"][0, k] -= h
            fd = (obj(lp, s) - obj(lm, s)) / (2 * h)
        else:
            h = 1e-4 * s
            fd = (obj(ls, s + h) - obj(ls, s - h)) / (2 * h)
        assert abs(g[k] - fd) < 1e-5 * abs(fd), (k, g[k], fd)
        assert abs(g[k] - g0[k]) > 0.05 * abs(fd), (k, g[k], g0[k])


@pytest.mark.parametrize("p", [1, 2])
def test_adjoint_with_phase_model_matches_central_differences(oracle_mod, p):
    """With the phase model (k(T, r_c), r_c = max(r_c, g(T)) stored by every step) the adjoint
    carries the history's own adjoint backward (through the max where the stored value wins,
    into lambda through g'(T) where g wins) and the gradient equals central differences of the
    objective to 1e-5, on a brick with a powder top layer that the laser track partly melts (the
    history grows at about a hundred quadrature points). The phase model moves every gradient
    component by a large fraction; dropping the history term moves them by 1e-3 to 5e-2 (checked
    when the pin was written). The adjoint and the objective leave the stored history as they
    found it."""
    ph = dict(I.PHASE, k_m=30.0, k_s=25.0)
    d = I.mesh_desc((4, 2, 2), (125e-6,) * 3, p, 1, [I.uniform_region(1)], powder_z0=0.19e-3, powder_z1=1.0)
    m = oracle_mod.Mesh(d)
    mat = dict(I.TI64_CONST)
    lam, _ = m.lambda_max(dict(mat, k0=30.0, k1=30.0, powder_k_scale=1.0), I.start_vector(m.n_dofs), max_iter=300,
                          rtol=1e-8)
    dt, nst, s, Tt = 0.3 * 2.0 / lam, 12, 1.05, 1800.0
    T0 = I.melt_pool_field(m.dof_xyz(), (0.2e-3, 0.125e-3, 0.25e-3), 1950.0, 110e-6, seed=11, noise=0.01)
    ls = I.c4_laser([[180.0, 220.0, 240.0]], n_seg=3, steps_per_seg=4, dt=dt, v=1.0, y=0.125e-3)
    ls["seg"][:, 0] += 0.15e-3
    ls["seg"][:, 2] += 0.15e-3
    _, g0 = m.adjoint(mat, T0, ls, 0.0, dt, nst, s=s, T_target=Tt)
    m.set_phase(ph)
    h0 = m.history()
    J, g = m.adjoint(mat, T0, ls, 0.0, dt, nst, s=s, T_target=Tt)
    assert J > 0 and np.all(np.isfinite(g))
    assert np.array_equal(m.history(), h0)
    stepped = oracle_mod.Mesh(d)
    stepped.set_phase(ph)
    stepped.explicit(mat, T0, ls, 0.0, dt, nst, s=s)
    assert np.sum(stepped.history() > h0) > 50  # the track melts powder: the history grows

    def obj(ls_, s_):
        return m.objective(mat, T0, ls_, 0.0, dt, nst, s=s_, T_target=Tt)

    for k in range(4):
        pw = ls["power"].copy()
        if k < 3:
            h = 1e-4 * pw[0, k]
            lp, lm = dict(ls, power=pw.copy()), dict(ls, power=pw.copy())
            lp["power"][0, k] += h
            lm["power"][0, k] -= h
            fd = (obj(lp, s) - obj(lm, s)) / (2 * h)
        else:
            h = 1e-4 * s
            fd = (obj(ls, s + h) - obj(ls, s - h)) / (2 * h)
        assert abs(g[k] - fd) < 1e-5 * abs(fd), (k, g[k], fd)
        assert abs(g[k] - g0[k]) > 0.05 * abs(fd), (k, g[k], g0[k])
    assert np.array_equal(m.history(), h0)


@pytest.mark.parametrize("p", [1, 2])
def test_surface_loss_of_a_constant_field(oracle_mod, p):
    """Constant T: the boundary term is -q(T) int_top N_i dA: it sums to -q(T) times the top
    area (partition of unity, constraint rows summing to 1 across hanging faces), vanishes off
    the top surface, and for a uniform Q1 brick each top node carries a quarter face per
    adjacent top face."""
    q = I.SURFACE_LOSS
    regions = [(I.BALL, (0.3e-3, 0.25e-3, 0.25e-3), (0, 0, 0), 120e-6, 2)] if p == 2 else [I.uniform_region(1)]
    d = I.mesh_desc((4, 2, 2), (125e-6,) * 3, p, 2, regions)
    m = oracle_mod.Mesh(d)
    m.set_surface_loss(q)
    Tc = 3400.0
    T = np.full(m.n_dofs, Tc)
    fd, fv, _ = m.residual(I.TI64_CONST, T)
    area = 4 * 125e-6 * 2 * 125e-6
    assert abs(fv.sum() + paper_surface_flux(q, Tc) * area) < 1e-12 * paper_surface_flux(q, Tc) * area
    assert np.abs(fd).max() < 1e-9 * np.abs(fv).max()
    z = m.dof_xyz()[:, 2]
    assert np.all(fv[z < z.max() - 1e-12] == 0.0) and np.all(fv[z > z.max() - 1e-12] < 0.0)
    if p == 1:  # uniform 62.5 um cells: weights h^2/4 per adjacent top face
        h = 62.5e-6
        xy = m.dof_xyz()[:, :2]
        top = z > z.max() - 1e-12
        on_x = (np.abs(xy[:, 0]) < 1e-12) | (np.abs(xy[:, 0] - 0.5e-3) < 1e-12)
        on_y = (np.abs(xy[:, 1]) < 1e-12) | (np.abs(xy[:, 1] - 0.25e-3) < 1e-12)
        faces = np.where(on_x & on_y, 1, np.where(on_x | on_y, 2, 4))
        expect = -paper_surface_flux(q, Tc) * faces * h * h / 4
        assert np.abs(fv[top] - expect[top]).max() < 1e-12 * np.abs(expect[top]).max()
    m.set_surface_loss(None)
    _, fv0, _ = m.residual(I.TI64_CONST, T)
    assert np.all(fv0 == 0.0)


def test_radiating_slab_reaches_the_flux_balance(oracle_mod):
    """A column (1 mm, Dirichlet bottom at 2500 K, insulated sides, radiating top) relaxes to
    the steady state of the continuum problem: a linear profile whose conductive flux
    k (T_D - T_top) / L equals the radiation q_rad(T_top), with T_top the root of that scalar
    equation (bisection here). Q1 represents the linear profile exactly, so the nodal values
    agree with the continuum solution once the transient has decayed."""
    q = dict(I.SURFACE_LOSS, C_P=0.0)
    mat = dict(I.TI64_CONST, T_dirichlet=2500.0)
    L, kk = 1.0e-3, mat["k0"]
    d = I.mesh_desc((1, 1, 8), (125e-6,) * 3, 1, 0, [])
    m = oracle_mod.Mesh(d)
    m.set_surface_loss(q)
    lam, _ = m.lambda_max(mat, I.start_vector(m.n_dofs), max_iter=400, rtol=1e-10)
    dt = 0.5 * 2.0 / lam
    T = m.explicit(mat, np.full(m.n_dofs, 2500.0), None, 0.0, dt, int(4.0 / dt))
    lo, hi = 353.0, 2500.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if kk * (2500.0 - mid) / L > paper_surface_flux(q, mid):
            lo = mid
        else:
            hi = mid
    T_top = 0.5 * (lo + hi)
    z = m.dof_xyz()[:, 2]
    expect = 2500.0 + (T_top - 2500.0) * z / L
    assert 2000.0 < T_top < 2450.0
    assert np.abs(T - expect).max() < 1e-6


# ---- phase-dependent conductivity with history (Eqs. liquid_fraction, consolidated_fraction,
# phase_fractions, material_parameter_interp) ---------------------------------------------

def _phase_mesh(oracle_mod, p, powder):
    regions = [(I.BALL, (0.3e-3, 0.25e-3, 0.25e-3), (0, 0, 0), 120e-6, 2)]
    z0, z1 = (-1.0, 1.0) if powder else (1e30, 1e30)
    return oracle_mod.Mesh(I.mesh_desc((4, 2, 2), (125e-6,) * 3, p, 2, regions, powder_z0=z0, powder_z1=z1))


def _ramp(k_lo, k_hi, ph):
    return dict(I.TI64_CONST, k0=k_lo, k1=k_hi, Tk0=ph["T_s"], Tk1=ph["T_l"], powder_k_scale=1.0)


@pytest.mark.parametrize("p", [1, 2])
def test_phase_conductivity_of_consolidated_material_is_the_solid_to_melt_ramp(oracle_mod, p):
    """r_c = 1: k = k_s + g(T) (k_m - k_s), i.e. the clamped linear ramp from k_s at T_s to
    k_m at T_l; the residual of a field across solid, mushy and melt equals the ramp
    material's."""
    ph = dict(I.PHASE, k_m=30.0)
    m = _phase_mesh(oracle_mod, p, powder=False)
    T = I.smooth_field(m.dof_xyz(), seed=31, lo=1200.0, hi=2300.0)
    ref, _, _ = m.residual(_ramp(ph["k_s"], ph["k_m"], ph), T)
    m.set_phase(ph)
    fd, _, _ = m.residual(I.TI64_CONST, T)
    assert np.abs(fd - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(ref).max() > 0


@pytest.mark.parametrize("p", [1, 2])
def test_phase_conductivity_of_powder_before_and_after_melting(oracle_mod, p):
    """Powder (r_c = 0 before): k = k_p + g (k_m - k_p), the ramp from k_p to k_m (the residual
    reads r_c = max(stored, g) without storing it). After an explicit step at a melted state the
    history holds r_c = 1: a field below T_s then sees k_s, not k_p (irreversible
    consolidation)."""
    ph = dict(I.PHASE, k_m=30.0, k_s=25.0)
    m = _phase_mesh(oracle_mod, p, powder=True)
    m.set_phase(ph)
    T = I.smooth_field(m.dof_xyz(), seed=32, lo=1200.0, hi=2300.0)
    fd, _, _ = m.residual(I.TI64_CONST, T)
    ref, _, _ = _phase_mesh(oracle_mod, p, powder=True).residual(_ramp(ph["k_p"], ph["k_m"], ph), T)
    assert np.abs(fd - ref).max() < 1e-12 * np.abs(ref).max()
    cool = I.smooth_field(m.dof_xyz(), seed=33, lo=400.0, hi=1400.0)
    plain = _phase_mesh(oracle_mod, p, powder=True)
    k_p_res, _, _ = plain.residual(dict(I.TI64_CONST, k0=ph["k_p"], k1=ph["k_p"], powder_k_scale=1.0), cool)
    fd, _, _ = m.residual(I.TI64_CONST, cool)
    assert np.abs(fd - k_p_res).max() < 1e-12 * np.abs(k_p_res).max()  # residuals did not consolidate
    m.explicit(I.TI64_CONST, np.full(m.n_dofs, 2600.0), None, 0.0, 1e-12, 1)
    k_s_res, _, _ = plain.residual(dict(I.TI64_CONST, k0=ph["k_s"], k1=ph["k_s"], powder_k_scale=1.0), cool)
    fd, _, _ = m.residual(I.TI64_CONST, cool)
    assert np.abs(fd - k_s_res).max() < 1e-12 * np.abs(k_s_res).max()
    m.set_phase(ph)  # setting the model again restarts the history
    fd, _, _ = m.residual(I.TI64_CONST, cool)
    assert np.abs(fd - k_p_res).max() < 1e-12 * np.abs(k_p_res).max()
