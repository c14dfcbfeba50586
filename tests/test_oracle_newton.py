"""Pins of the oracle's nonlinear backward Euler (Sec. 3.2, Eq. backward_euler_nonlinear) and
its Newton-Raphson solve (Eqs. Newton_1, Newton_2): the residual against brute-force
assembled matrices for a linear material, the Jacobian-vector product (with the k'(T) term
L_e of Eq. matrix_free_eval) against differences of the residual, the converged step against
a dense Newton iteration on a tiny mesh with hanging nodes, and the linear case against a
dense solve."""
import numpy as np
import pytest

from paper_2302_05164_gb300 import inputs as I
from tests.assembly import assemble, small_amr

LIN = dict(rho=3.0, c=0.7, k0=2.5, k1=2.5, Tk0=0.0, Tk1=0.0, latent=0.0, Tm=0.0, sigma=0.0, powder_k_scale=0.1,
           T_dirichlet=1.0)
# conductivity ramp 2.5 -> 9 over [0.5, 3.5]; the fields below stay inside the ramp (no kink)
NONLIN = dict(LIN, k1=9.0, Tk0=0.5, Tk1=3.5)


def mesh(oracle_mod, p):
    desc = small_amr(p)
    desc["powder_z0"], desc["powder_z1"] = 0.75, 2.0
    m = oracle_mod.Mesh(desc)
    assert m.n_hanging > 0
    return m, desc


def field(m, lo, hi, seed):
    return I.smooth_field(m.dof_xyz(), seed=seed, lo=lo, hi=hi)


@pytest.mark.parametrize("p", [1, 2])
def test_newton_residual_of_a_linear_material_is_the_assembled_one(oracle_mod, p):
    """r(T) = M (T - T_n)/dt + K T on free rows (M, K assembled from textbook element
    matrices with the explicit constraint matrix), 0 on Dirichlet rows."""
    m, desc = mesh(oracle_mod, p)
    dt = 0.3
    kf = lambda mt: 2.5 * (0.1 if mt == 1 else 1.0)
    K, t = assemble(m, desc, kf, 0.0)
    M, _ = assemble(m, desc, lambda mt: 0.0, 3.0 * 0.7)
    free = t["dirichlet"] == 0
    T, Tn = field(m, 1.0, 3.0, 1), field(m, 1.0, 3.0, 2)
    ref = np.where(free, M @ (T - Tn) / dt + K @ T, 0.0)
    r = m.newton_residual(LIN, T, Tn, dt)
    assert np.max(np.abs(r - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("p", [1, 2])
def test_newton_jacobian_matches_differences_of_the_residual(oracle_mod, p):
    """J(T) v (Eq. Newton_1: C/dt - df_diff/dT, including the k'(T) term L_e) equals
    Richardson-extrapolated central differences of r(T) in the direction v (error O(eps^4))
    on free rows, and v itself on Dirichlet rows."""
    m, _ = mesh(oracle_mod, p)
    dt = 0.05
    T, Tn = field(m, 0.8, 3.2, 3), field(m, 0.8, 3.2, 4)
    free = m.tables()["dirichlet"] == 0
    v = np.random.default_rng(5).normal(size=m.n_dofs) * free

    def cd(eps):
        return (m.newton_residual(NONLIN, T + eps * v, Tn, dt) - m.newton_residual(NONLIN, T - eps * v, Tn, dt)) / (
            2 * eps)

    eps = 1e-3
    ref = (4 * cd(eps / 2) - cd(eps)) / 3
    Jv = m.newton_jacobian(NONLIN, T, dt, v)
    assert np.max(np.abs(Jv[free] - ref[free])) <= 1e-8 * np.max(np.abs(ref))
    # the k' term matters here: without it the product moves by far more than the tolerance
    Jlin = m.newton_jacobian(dict(NONLIN, k1=NONLIN["k0"], Tk1=NONLIN["Tk0"]), T, dt, v)
    assert np.max(np.abs(Jlin - Jv)) > 1e-3 * np.max(np.abs(Jv))
    w = np.random.default_rng(6).normal(size=m.n_dofs) * (~free)
    assert np.array_equal(m.newton_jacobian(NONLIN, T, dt, w)[~free], w[~free])


def dense_jacobian(m, mat, T, dt):
    n = m.n_dofs
    J = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        J[:, j] = m.newton_jacobian(mat, T, dt, e)
    return J


@pytest.mark.parametrize("p", [1, 2])
def test_newton_step_matches_dense_newton(oracle_mod, p):
    """One nonlinear backward-Euler step: the oracle's Newton iteration (BiCGStab with the
    Chebyshev-Jacobi preconditioner) equals a dense Newton iteration (numpy solves of the
    assembled Jacobian) to 1e-11, the dense iteration converges quadratically, and the
    oracle needs only a few corrections."""
    m, _ = mesh(oracle_mod, p)
    free = m.tables()["dirichlet"] == 0
    dt = 0.05
    Tn = field(m, 1.0, 3.0, 7)
    Tn[~free] = NONLIN["T_dirichlet"]
    lmin, lmax = m.lanczos_bounds(NONLIN, dt, np.random.default_rng(8).normal(size=m.n_dofs), 30)
    got, nit, lit, st = m.implicit_newton(NONLIN, Tn, dt, 1, 1e-13, 20, 1e-12, 400, 5, lmin, 1.1 * lmax)
    assert st == 0 and 2 <= nit[0] <= 6, (nit, lit)
    T = Tn.copy()
    norms = []
    for _ in range(8):
        r = m.newton_residual(NONLIN, T, Tn, dt)
        norms.append(np.linalg.norm(r))
        if norms[-1] <= 1e-14 * norms[0]:
            break
        T = T + np.linalg.solve(dense_jacobian(m, NONLIN, T, dt), -r)
    assert norms[-1] <= 1e-13 * norms[0]
    # quadratic convergence: each reduction factor at most the previous residual's relative size
    rel = np.array(norms) / norms[0]
    for a, b in zip(rel[1:-1], rel[2:]):
        if a < 1e-3:
            assert b <= 10 * a * a + 1e-15, rel
    assert np.max(np.abs(got - T)) <= 1e-11 * np.max(np.abs(T))
    assert np.max(np.abs(got - Tn)) > 1e-2  # the step moved the field


@pytest.mark.parametrize("p", [1, 2])
def test_newton_on_a_linear_material_is_one_dense_solve(oracle_mod, p):
    """With constant k the Newton iteration is one linear solve: (M/dt + K) (T - T_n) = -K T_n
    on free rows (the increment form of the linear backward Euler), equal to a dense solve of
    the assembled system to 1e-11."""
    m, desc = mesh(oracle_mod, p)
    dt = 0.05
    kf = lambda mt: 2.5 * (0.1 if mt == 1 else 1.0)
    A, t = assemble(m, desc, kf, 3.0 * 0.7 / dt)
    K, _ = assemble(m, desc, kf, 0.0)
    free = t["dirichlet"] == 0
    Tn = field(m, 1.0, 3.0, 9)
    Tn[~free] = LIN["T_dirichlet"]
    lmin, lmax = m.lanczos_bounds(LIN, dt, np.random.default_rng(8).normal(size=m.n_dofs), 30)
    got, nit, lit, st = m.implicit_newton(LIN, Tn, dt, 1, 1e-12, 5, 1e-13, 400, 5, lmin, 1.1 * lmax)
    assert st == 0 and nit[0] == 1
    ref = Tn.copy()
    ff = np.ix_(free, free)
    ref[free] += np.linalg.solve(A[ff], -(K @ Tn)[free])
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


PHASE = dict(T_s=1.5, T_l=2.5, k_p=0.2, k_m=9.0, k_s=6.0)
# evaporation switched on below the fields (T_v = 1) with an O(1) flux, radiation negligible at T ~ 2
LOSS = dict(emissivity=0.7, T_amb=1.0, C_P=1.0, C_T=0.0, C_M=1.0, T_v=1.0, h_v=1.0, c_h=0.0, T_h0=0.0, T_max=1e9)


def phase_mesh(oracle_mod, p):
    """The tiny mesh with the phase model: cells of the upper band are powder (r_c = 0, never
    melted), the rest consolidated (r_c = 1); the field spans the melting range."""
    m, desc = mesh(oracle_mod, p)
    m.set_phase(PHASE)
    return m, desc


@pytest.mark.parametrize("p", [1, 2])
def test_newton_jacobian_with_phase_model_and_surface_loss(oracle_mod, p):
    """With the phase model (Eq. material_parameter_interp, r_c = max(stored, g(T))) the
    Jacobian's k'(T) follows the branch of the max, and the surface loss enters the residual at
    T_n only (Eq. backward_euler_nonlinear): J v equals differences of the residual. The stored
    history is 0 (powder) or 1 (consolidated), so no quadrature point sits on the max's kink."""
    m, _ = phase_mesh(oracle_mod, p)
    m.set_surface_loss(LOSS)
    dt = 0.05
    T, Tn = field(m, 1.6, 2.4, 13), field(m, 1.6, 2.4, 14)
    free = m.tables()["dirichlet"] == 0
    v = np.random.default_rng(15).normal(size=m.n_dofs) * free

    def cd(eps):
        return (m.newton_residual(NONLIN, T + eps * v, Tn, dt) - m.newton_residual(NONLIN, T - eps * v, Tn, dt)) / (
            2 * eps)

    eps = 1e-4
    ref = (4 * cd(eps / 2) - cd(eps)) / 3
    Jv = m.newton_jacobian(NONLIN, T, dt, v)
    assert np.max(np.abs(Jv[free] - ref[free])) <= 1e-7 * np.max(np.abs(ref))
    # the surface loss moves the residual (evaluated at T_n), not the Jacobian
    r_loss = m.newton_residual(NONLIN, T, Tn, dt)
    m.set_surface_loss(None)
    assert np.max(np.abs(m.newton_residual(NONLIN, T, Tn, dt) - r_loss)) > 1e-6 * np.max(np.abs(r_loss))
    assert np.array_equal(m.newton_jacobian(NONLIN, T, dt, v), Jv)


@pytest.mark.parametrize("p", [1, 2])
def test_newton_step_with_phase_model_matches_dense_newton(oracle_mod, p):
    """The oracle's Newton step with the phase model and the surface loss equals a dense Newton
    iteration on its residual and Jacobian to 1e-11, and the converged step stores the history
    r_c = max(r_c, g(T_{n+1}))."""
    m, _ = phase_mesh(oracle_mod, p)
    m.set_surface_loss(LOSS)
    free = m.tables()["dirichlet"] == 0
    dt = 0.05
    Tn = field(m, 1.6, 2.8, 16)
    Tn[~free] = NONLIN["T_dirichlet"]
    h0 = m.history()
    lmin, lmax = m.lanczos_bounds(NONLIN, dt, np.random.default_rng(8).normal(size=m.n_dofs), 30)
    T = Tn.copy()
    norms = []
    for _ in range(10):
        r = m.newton_residual(NONLIN, T, Tn, dt)
        norms.append(np.linalg.norm(r))
        if norms[-1] <= 1e-14 * norms[0]:
            break
        T = T + np.linalg.solve(dense_jacobian(m, NONLIN, T, dt), -r)
    assert norms[-1] <= 1e-13 * norms[0]
    got, nit, lit, st = m.implicit_newton(NONLIN, Tn, dt, 1, 1e-13, 20, 1e-12, 400, 5, lmin, 1.1 * lmax)
    assert st == 0
    assert np.max(np.abs(got - T)) <= 1e-11 * np.max(np.abs(T))
    h1 = m.history()
    assert np.all(h1 >= h0) and np.any(h1 > h0)  # melted powder consolidated
