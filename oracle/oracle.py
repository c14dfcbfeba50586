"""ctypes wrapper around the serial FP64 oracle (pbf_oracle.cpp).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of the
benchmark may import this module; the GPU library never does. It marshals plain Python
dicts (as produced by the package's `inputs` module) into the oracle's own C structs.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pbf_oracle.cpp")
LIB = os.path.join(HERE, "_build", "libpbf_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, so rounding follows the source)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


class _Desc(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("ntree", C.c_int * 3), ("tree_h", C.c_double * 3),
                ("degree", C.c_int), ("max_level", C.c_int), ("tree_exists", C.c_void_p),
                ("active_top_z", C.c_double), ("dirichlet_faces", C.c_uint),
                ("n_regions", C.c_int), ("regions", C.c_void_p),
                ("powder_z0", C.c_double), ("powder_z1", C.c_double)]


class _Mat(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("rho", "c", "k0", "k1", "Tk0", "Tk1", "latent", "Tm",
                                          "sigma", "powder_k_scale", "T_dirichlet")] + [("lumping", C.c_int)]


class _Loss(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("emissivity", "T_amb", "C_P", "C_T", "C_M", "T_v", "h_v", "c_h", "T_h0",
                                          "T_max")]


class _Phase(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("T_s", "T_l", "k_p", "k_m", "k_s")]


def surface_loss(q: dict) -> _Loss:
    return _Loss(*[float(q[n]) for n, _ in _Loss._fields_])


class _Laser(C.Structure):
    _fields_ = [("n_seg", C.c_int), ("seg", C.c_void_p), ("power", C.c_void_p),
                ("eta", C.c_double), ("radius", C.c_double), ("volumetric", C.c_int),
                ("h_powder", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.or_mesh_build.restype = C.c_void_p
        L.or_mesh_build.argtypes = [C.POINTER(_Desc)]
        L.or_mesh_free.argtypes = [C.c_void_p]
        L.or_lambda_max.restype = C.c_double
        L.or_adjoint.restype = C.c_double
        L.or_objective.restype = C.c_double
        L.or_capp.restype = C.c_double
        L.or_cond.restype = C.c_double
        L.or_surface_flux.restype = C.c_double
        L.or_surface_flux_deriv.restype = C.c_double
        L.or_implicit.restype = C.c_int
        L.or_implicit_newton.restype = C.c_int
        L.or_gate_pins.restype = C.c_int
    return _lib


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else C.c_void_p(0)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def material(m: dict) -> _Mat:
    return _Mat(*[float(m[n]) for n, _ in _Mat._fields_[:-1]], int(m.get("lumping", 0)))


class _LaserHolder:
    def __init__(self, ls: dict, instance: int = 0):
        self.seg = _f64(ls["seg"])
        pw = np.atleast_2d(_f64(ls["power"]))
        self.power = np.ascontiguousarray(pw[instance])
        self.s = _Laser(self.seg.shape[0], _ptr(self.seg), _ptr(self.power), ls["eta"], ls["radius"],
                        int(ls.get("volumetric", 0)), float(ls.get("h_powder", 40e-6)))

    @property
    def ref(self):
        return C.byref(self.s)


class Mesh:
    """Oracle mesh built from a descriptor dict (see inputs.mesh_desc)."""

    def __init__(self, desc: dict):
        self.desc = desc
        regs = np.zeros((max(1, len(desc["regions"])), 9))
        for i, (k, a, b, r, lv) in enumerate(desc["regions"]):
            regs[i] = [k, *a, *b, r, lv]
        self._regs = regs
        te = desc.get("tree_exists")
        self._te = None if te is None else np.ascontiguousarray(te, np.uint8)
        d = _Desc((C.c_double * 3)(*desc["origin"]), (C.c_int * 3)(*desc["ntree"]),
                  (C.c_double * 3)(*desc["tree_h"]), desc["degree"], desc["max_level"],
                  _ptr(self._te), desc["active_top_z"], desc["dirichlet_faces"],
                  len(desc["regions"]), _ptr(regs), desc["powder_z0"], desc["powder_z1"])
        self.h = lib().or_mesh_build(C.byref(d))
        cnt = np.zeros(8, np.int64)
        lib().or_mesh_counts(C.c_void_p(self.h), _ptr(cnt))
        (self.n_leaves, self.n_active, self.n_dofs, self.n_hanging, self.n_con, self.n_colours,
         self.n_top, self.npc) = (int(v) for v in cnt)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_mesh_free(C.c_void_p(self.h))
            self.h = None

    def tables(self) -> dict:
        t = dict(leaves=np.zeros((self.n_leaves, 5), np.int64),
                 material=np.zeros(self.n_leaves, np.uint8),
                 cell_dofs=np.zeros((self.n_active, self.npc), np.int32),
                 con_ptr=np.zeros(self.n_hanging + 1, np.int32),
                 con_idx=np.zeros(self.n_con, np.int32),
                 con_w=np.zeros(self.n_con, np.float64),
                 hang_coord=np.zeros((self.n_hanging, 3), np.int64),
                 dof_coord=np.zeros((self.n_dofs, 3), np.int64),
                 dirichlet=np.zeros(self.n_dofs, np.uint8),
                 colour=np.zeros(self.n_active, np.int32),
                 top=np.zeros(self.n_active, np.uint8))
        lib().or_mesh_tables(C.c_void_p(self.h), *[_ptr(t[k]) for k in
                             ("leaves", "material", "cell_dofs", "con_ptr", "con_idx", "con_w",
                              "hang_coord", "dof_coord", "dirichlet", "colour", "top")])
        return t

    def dof_xyz(self) -> np.ndarray:
        """Physical dof coordinates [n][3] (for building smooth seeded fields)."""
        c = self.tables()["dof_coord"].astype(np.float64)
        d = self.desc
        L, p = d["max_level"], d["degree"]
        return np.array(d["origin"]) + np.array(d["tree_h"]) * c / (p * 2.0 ** L)

    def set_material(self, mat_active: np.ndarray):
        m = np.ascontiguousarray(mat_active, np.uint8)
        lib().or_mesh_set_material(C.c_void_p(self.h), _ptr(m))

    def set_phase(self, ph):
        """Phase-dependent conductivity k(T, r_c) with the consolidated-fraction history per
        quadrature point (dict T_s, T_l, k_p, k_m, k_s; None: off); setting it restarts the
        history from the cell materials. Explicit steps update the history, residuals read it."""
        self._phase = None if ph is None else _Phase(*[float(ph[n]) for n, _ in _Phase._fields_])
        lib().or_set_phase(C.c_void_p(self.h), None if ph is None else C.byref(self._phase))

    def set_surface_loss(self, q):
        """Radiation / evaporation on the top faces (dict of `surface_loss` fields; None: off)
        for every later residual and explicit step; the adjoint and objective refuse it."""
        self._loss = None if q is None else surface_loss(q)
        lib().or_set_surface_loss(C.c_void_p(self.h), None if q is None else C.byref(self._loss))

    # ---- operators -------------------------------------------------------------------
    def residual(self, mat, T, ls=None, t=0.0, s=1.0, instance=0):
        T = _f64(T)
        fd, fv, Cm = (np.zeros(self.n_dofs) for _ in range(3))
        lh = _LaserHolder(ls, instance) if ls is not None else None
        lib().or_residual(C.c_void_p(self.h), C.byref(material(mat)), C.c_double(s), _ptr(T),
                          lh.ref if lh else None, C.c_double(t), _ptr(fd), _ptr(fv), _ptr(Cm))
        return fd, fv, Cm

    def explicit(self, mat, T, ls, t0, dt, nsteps, s=1.0, instance=0):
        T = _f64(T).copy()
        lh = _LaserHolder(ls, instance) if ls is not None else None
        lib().or_explicit(C.c_void_p(self.h), C.byref(material(mat)), C.c_double(s), _ptr(T),
                          lh.ref if lh else None, C.c_double(t0), C.c_double(dt), C.c_int(nsteps))
        return T

    def lambda_max(self, mat, x0, max_iter=200, rtol=1e-6, s=1.0):
        x0 = _f64(x0)  # bound to a name: the array must outlive the C call
        it = C.c_int(0)
        lam = lib().or_lambda_max(C.c_void_p(self.h), C.byref(material(mat)), C.c_double(s), _ptr(x0),
                                  C.c_int(max_iter), C.c_double(rtol), C.byref(it))
        return lam, it.value

    def lumped_capacity(self, mat, T):
        out = np.zeros(self.n_dofs)
        T = _f64(T)  # keep the (possibly copied) array alive during the call
        lib().or_lumped_capacity(C.c_void_p(self.h), C.byref(material(mat)), _ptr(T), _ptr(out))
        return out

    def apply_implicit(self, mat, dt, x):
        y = np.zeros(self.n_dofs)
        x = _f64(x)
        lib().or_apply_implicit(C.c_void_p(self.h), C.byref(material(mat)), C.c_double(dt), _ptr(x), _ptr(y))
        return y

    def implicit_diagonal(self, mat, dt):
        y = np.zeros(self.n_dofs)
        lib().or_implicit_diagonal(C.c_void_p(self.h), C.byref(material(mat)), C.c_double(dt), _ptr(y))
        return y

    def chebyshev(self, mat, dt, degree, lmin, lmax, r):
        z = np.zeros(self.n_dofs)
        r = _f64(r)
        lib().or_chebyshev(C.c_void_p(self.h), C.byref(material(mat)), C.c_double(dt), C.c_int(degree),
                           C.c_double(lmin), C.c_double(lmax), _ptr(r), _ptr(z))
        return z

    def lanczos_bounds(self, mat, dt, b, n_iter=30):
        out = np.zeros(2)
        b = _f64(b)
        lib().or_lanczos_bounds(C.c_void_p(self.h), C.byref(material(mat)), C.c_double(dt), _ptr(b),
                                C.c_int(n_iter), _ptr(out))
        return float(out[0]), float(out[1])

    def implicit(self, mat, T, dt, nsteps, rtol, max_it, degree, lmin, lmax):
        T = _f64(T).copy()
        iters = np.zeros(nsteps, np.int32)
        st = lib().or_implicit(C.c_void_p(self.h), C.byref(material(mat)), _ptr(T), C.c_double(dt),
                               C.c_int(nsteps), C.c_double(rtol), C.c_int(max_it), C.c_int(degree),
                               C.c_double(lmin), C.c_double(lmax), _ptr(iters))
        return T, iters, st

    def newton_residual(self, mat, T, Tn, dt):
        """r(T) = C (T - T_n)/dt - f_diff(T) on free dofs, 0 on Dirichlet dofs."""
        T, Tn = _f64(T), _f64(Tn)
        r = np.zeros(self.n_dofs)
        lib().or_newton_residual(C.c_void_p(self.h), C.byref(material(mat)), _ptr(T), _ptr(Tn), C.c_double(dt),
                                 _ptr(r))
        return r

    def newton_jacobian(self, mat, T, dt, v):
        """J(T) v of the nonlinear backward-Euler residual (identity rows on Dirichlet dofs)."""
        T, v = _f64(T), _f64(v)
        y = np.zeros(self.n_dofs)
        lib().or_newton_jacobian(C.c_void_p(self.h), C.byref(material(mat)), _ptr(T), C.c_double(dt), _ptr(v),
                                 _ptr(y))
        return y

    def implicit_newton(self, mat, T, dt, nsteps, newton_rtol, newton_max, lin_rtol, lin_max, degree, lmin, lmax):
        T = _f64(T).copy()
        nit = np.zeros(nsteps, np.int32)
        lit = np.zeros(nsteps, np.int32)
        st = lib().or_implicit_newton(C.c_void_p(self.h), C.byref(material(mat)), _ptr(T), C.c_double(dt),
                                      C.c_int(nsteps), C.c_double(newton_rtol), C.c_int(newton_max),
                                      C.c_double(lin_rtol), C.c_int(lin_max), C.c_int(degree), C.c_double(lmin),
                                      C.c_double(lmax), _ptr(nit), _ptr(lit))
        return T, nit, lit, st

    def adjoint(self, mat, T0, ls, t0, dt, nsteps, T_target=2300.0, p_exp=16.0, s=1.0, instance=0):
        lh = _LaserHolder(ls, instance)
        grad = np.zeros(lh.seg.shape[0] + 1)
        T0 = _f64(T0)
        J = lib().or_adjoint(C.c_void_p(self.h), C.byref(material(mat)), C.c_double(s), _ptr(T0), lh.ref,
                             C.c_double(t0), C.c_double(dt), C.c_int(nsteps), C.c_double(T_target),
                             C.c_double(p_exp), _ptr(grad))
        return J, grad

    def step_transpose(self, mat, T, ls, t, dt, w, s=1.0, instance=0):
        """(dT_{n+1}/dT_n)^T w for one explicit step at state T and time t (Dirichlet rows zero)."""
        T, w = _f64(T), _f64(w)
        out = np.zeros(self.n_dofs)
        lh = _LaserHolder(ls, instance) if ls is not None else None
        lib().or_step_transpose(C.c_void_p(self.h), C.byref(material(mat)), C.c_double(s), _ptr(T),
                                lh.ref if lh else None, C.c_double(t), C.c_double(dt), _ptr(w), _ptr(out))
        return out

    def objective(self, mat, T0, ls, t0, dt, nsteps, T_target=2300.0, p_exp=16.0, s=1.0, instance=0):
        lh = _LaserHolder(ls, instance)
        T0 = _f64(T0)
        return lib().or_objective(C.c_void_p(self.h), C.byref(material(mat)), C.c_double(s), _ptr(T0),
                                  lh.ref, C.c_double(t0), C.c_double(dt), C.c_int(nsteps),
                                  C.c_double(T_target), C.c_double(p_exp))

    def history(self):
        """r_c per active cell and quadrature point, [n_active][(p+1)^3] (x fastest)."""
        nq3 = (self.desc["degree"] + 1) ** 3
        out = np.zeros((self.n_active, nq3))
        lib().or_history_get(C.c_void_p(self.h), _ptr(out))
        return out

    def set_history(self, rc):
        rc = _f64(rc)
        lib().or_history_set(C.c_void_p(self.h), _ptr(rc))

    def gate_pins(self, rc_min, r_coarsen=0.9):
        """Pin regions that keep every family with a cell of r_c below r_coarsen from merging
        (region tuples as in inputs.mesh_desc)."""
        rc_min = _f64(rc_min)
        out = np.zeros((max(1, self.n_active), 9))
        n = lib().or_gate_pins(C.c_void_p(self.h), _ptr(rc_min), C.c_double(r_coarsen), _ptr(out),
                               C.c_int(out.shape[0]))
        return [(int(r[0]), tuple(r[1:4]), tuple(r[4:7]), float(r[7]), int(r[8])) for r in out[:n]]

    def surface_weights(self):
        w = np.zeros(self.n_dofs)
        lib().or_surface_weights(C.c_void_p(self.h), _ptr(w))
        return w


def transfer(old: Mesh, T_old, new: Mesh, T_init):
    out = np.zeros(new.n_dofs)
    T_old = _f64(T_old)
    lib().or_transfer(C.c_void_p(old.h), _ptr(T_old), C.c_void_p(new.h), C.c_double(T_init), _ptr(out))
    return out


def transfer_history(old: Mesh, rc_old, new: Mesh):
    """r_c moved to a changed mesh: nearest old quadrature point in the first old active cell
    holding each new point; new parts start at 0 (powder) or 1."""
    nq3 = (new.desc["degree"] + 1) ** 3
    out = np.zeros((new.n_active, nq3))
    rc_old = _f64(rc_old)
    lib().or_transfer_history(C.c_void_p(old.h), _ptr(rc_old), C.c_void_p(new.h), _ptr(out))
    return out


def surface_flux(q, T):
    return lib().or_surface_flux(C.byref(surface_loss(q)), C.c_double(T))


def surface_flux_deriv(q, T):
    return lib().or_surface_flux_deriv(C.byref(surface_loss(q)), C.c_double(T))


def capp(mat, T):
    return lib().or_capp(C.byref(material(mat)), C.c_double(T))


def cond(mat, T, mat_id=0, s=1.0):
    return lib().or_cond(C.byref(material(mat)), C.c_double(T), C.c_int(mat_id), C.c_double(s))
