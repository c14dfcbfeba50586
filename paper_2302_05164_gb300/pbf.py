"""Python binding of the C ABI in include/pbf.h (argument marshalling only).

Every numerical step runs in the CUDA library `_build/libpbf.so`; this module converts Python
objects (dicts from `inputs`, numpy arrays, torch CUDA tensors) into the C structs and
pointers of the ABI and raises `PbfError` on a non-zero status. There is no fallback: when the
library is missing, importing the binding fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpbf.so")

PBF_F64, PBF_F32OP = 0, 1
STATUS = {0: "PBF_OK", 1: "PBF_EINVAL", 2: "PBF_ENOMEM", 3: "PBF_ECUDA", 4: "PBF_ENOCONV", 5: "PBF_ENAN",
          6: "PBF_ETIMEOUT", 7: "PBF_EFAULT", 8: "PBF_ESTATE"}


class PbfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Region(C.Structure):
    _fields_ = [("kind", C.c_int), ("level", C.c_int), ("a", C.c_double * 3), ("b", C.c_double * 3),
                ("radius", C.c_double)]


class SurfaceLoss(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("emissivity", "T_amb", "C_P", "C_T", "C_M", "T_v", "h_v", "c_h", "T_h0",
                                          "T_max")]


class Phase(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("T_s", "T_l", "k_p", "k_m", "k_s")]


class MeshDesc(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("ntree", C.c_int * 3), ("tree_h", C.c_double * 3),
                ("degree", C.c_int), ("max_level", C.c_int), ("tree_exists", C.c_void_p),
                ("active_top_z", C.c_double), ("dirichlet_faces", C.c_uint32), ("n_regions", C.c_int),
                ("regions", C.c_void_p), ("powder_z0", C.c_double), ("powder_z1", C.c_double)]


class MeshInfo(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("n_leaves", "n_active", "n_dofs", "n_hanging", "n_con_entries",
                                         "n_colours", "n_top_faces", "nodes_per_cell", "generation")]


class MeshTables(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("leaves", "material", "cell_dofs", "con_ptr", "con_idx", "con_w",
                                          "hang_coord", "dof_coord", "dirichlet", "colour", "top")]


class StepTables(C.Structure):
    _fields_ = [("n_patches", C.c_int64), ("n_slots", C.c_int64), ("n_hent", C.c_int64),
                ("cells_per_patch", C.c_int32), ("max_slots", C.c_int32), ("max_hent", C.c_int32)] + \
               [(n, C.c_void_p) for n in ("ptr", "cnt", "slot", "cell", "loc", "hloc", "hw")]


class TransferMapC(C.Structure):
    _fields_ = [("n_old", C.c_int64), ("n_new", C.c_int64), ("n_entries", C.c_int64), ("fill", C.c_double),
                ("ptr", C.c_void_p), ("idx", C.c_void_p), ("w", C.c_void_p)]


class Material(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("rho", "c", "k0", "k1", "Tk0", "Tk1", "latent", "Tm", "sigma",
                                          "powder_k_scale", "T_dirichlet", "T_ref")] + [("lumping", C.c_int)]


class Laser(C.Structure):
    _fields_ = [("n_seg", C.c_int), ("seg", C.c_void_p), ("power", C.c_void_p), ("eta", C.c_double),
                ("radius", C.c_double), ("volumetric", C.c_int), ("h_powder", C.c_double)]


_lib = None

_SIGS = {
    "pbf_last_error": ([], C.c_char_p),
    "pbf_version": ([], C.c_char_p),
    "pbf_mesh_create": ([C.POINTER(MeshDesc), C.POINTER(C.c_void_p)], C.c_int),
    "pbf_mesh_destroy": ([C.c_void_p], C.c_int),
    "pbf_mesh_info": ([C.c_void_p, C.POINTER(MeshInfo)], C.c_int),
    "pbf_mesh_export": ([C.c_void_p, C.POINTER(MeshTables)], C.c_int),
    "pbf_mesh_step_tables": ([C.c_void_p, C.POINTER(StepTables)], C.c_int),
    "pbf_mesh_transfer_map": ([C.c_void_p, C.POINTER(TransferMapC)], C.c_int),
    "pbf_mesh_history_map": ([C.c_void_p, C.POINTER(C.c_int64), C.c_void_p], C.c_int),
    "pbf_mesh_activate_layer": ([C.c_void_p, C.c_double, C.c_int, C.c_double], C.c_int),
    "pbf_mesh_adapt": ([C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "pbf_mesh_adapt_gated": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double], C.c_int),
    "pbf_ctx_history_cell_min": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "pbf_ctx_get_history": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "pbf_ctx_set_history": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "pbf_ctx_transfer_history": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "pbf_mesh_transfer": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "pbf_ctx_create": ([C.c_void_p, C.POINTER(Material), C.c_int, C.c_int, C.POINTER(C.c_void_p)], C.c_int),
    "pbf_ctx_destroy": ([C.c_void_p], C.c_int),
    "pbf_ctx_set_k_scale": ([C.c_void_p, C.c_void_p], C.c_int),
    "pbf_eval_residual": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p], C.c_int),
    "pbf_explicit_step": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_void_p], C.c_int),
    "pbf_estimate_dt": ([C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double),
                         C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p], C.c_int),
    "pbf_estimate_dt_noalloc": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p], C.c_int),
    "pbf_cheb_bounds": ([C.c_void_p, C.c_double, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "pbf_implicit_solve": ([C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_double, C.c_int, C.c_int,
                            C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "pbf_implicit_newton": ([C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_double, C.c_int, C.c_double, C.c_int,
                             C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p],
                            C.c_int),
    "pbf_adjoint_sweep": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int,
                           C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.POINTER(C.c_longlong),
                           C.c_void_p], C.c_int),
    "pbf_revolve_cost": ([C.c_int, C.c_int, C.POINTER(C.c_longlong)], C.c_int),
    "pbf_round_to_f32": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "pbf_widen_to_f64": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "pbf_ctx_autotune": ([C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_void_p], C.c_int),
    "pbf_ctx_set_kernel_shape": ([C.c_void_p, C.c_int], C.c_int),
    "pbf_ctx_set_barrier_test": ([C.c_void_p, C.c_int], C.c_int),
    "pbf_ctx_set_surface_loss": ([C.c_void_p, C.POINTER(SurfaceLoss)], C.c_int),
    "pbf_ctx_set_phase": ([C.c_void_p, C.POINTER(Phase)], C.c_int),
    "pbf_ctx_set_timing": ([C.c_void_p, C.c_int], C.c_int),
    "pbf_ctx_kernel_time": ([C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)], C.c_int),
    "pbf_ctx_launch_count": ([C.c_void_p, C.POINTER(C.c_longlong)], C.c_int),
}


def lib():
    """Loads the CUDA library; raises ImportError when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                              "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise PbfError(status, lib().pbf_last_error().decode())


def _ptr(x):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


# ---- marshalling helpers -----------------------------------------------------------------

def _regions(regions):
    arr = (Region * max(1, len(regions)))()
    for i, (k, a, b, r, lv) in enumerate(regions):
        arr[i] = Region(int(k), int(lv), (C.c_double * 3)(*a), (C.c_double * 3)(*b), float(r))
    return arr


def _material(m: dict) -> Material:
    return Material(*[float(m.get(n, 0.0)) for n, _ in Material._fields_[:-1]], int(m.get("lumping", 0)))


class _LaserArg:
    def __init__(self, ls, batch):
        if ls is None:
            self.ref = None
            return
        self.seg = np.ascontiguousarray(ls["seg"], np.float64)
        n = self.seg.shape[0]
        pw = np.asarray(ls["power"], np.float64)
        if pw.ndim == 1:
            pw = np.broadcast_to(pw, (batch, n))
        self.power = np.ascontiguousarray(pw)
        self.s = Laser(n, _ptr(self.seg), _ptr(self.power), ls["eta"], ls["radius"],
                       int(ls.get("volumetric", 0)), float(ls.get("h_powder", 40e-6)))
        self.ref = C.byref(self.s)


# ---- C-ABI functions (same names) -----------------------------------------------------------

def pbf_mesh_create(desc: dict):
    regs = _regions(desc["regions"])
    te = desc.get("tree_exists")
    te = None if te is None else np.ascontiguousarray(te, np.uint8)
    d = MeshDesc((C.c_double * 3)(*desc["origin"]), (C.c_int * 3)(*desc["ntree"]),
                 (C.c_double * 3)(*desc["tree_h"]), desc["degree"], desc["max_level"], _ptr(te),
                 desc["active_top_z"], desc["dirichlet_faces"], len(desc["regions"]),
                 C.cast(regs, C.c_void_p), desc["powder_z0"], desc["powder_z1"])
    h = C.c_void_p()
    _check(lib().pbf_mesh_create(C.byref(d), C.byref(h)))
    return h


def pbf_mesh_destroy(h):
    _check(lib().pbf_mesh_destroy(h))


def pbf_mesh_info(h) -> dict:
    info = MeshInfo()
    _check(lib().pbf_mesh_info(h, C.byref(info)))
    return {n: int(getattr(info, n)) for n, _ in MeshInfo._fields_}


def pbf_mesh_export(h) -> dict:
    i = pbf_mesh_info(h)
    npc = i["nodes_per_cell"]
    t = dict(leaves=np.zeros((i["n_leaves"], 5), np.int64), material=np.zeros(i["n_leaves"], np.uint8),
             cell_dofs=np.zeros((i["n_active"], npc), np.int32), con_ptr=np.zeros(i["n_hanging"] + 1, np.int32),
             con_idx=np.zeros(i["n_con_entries"], np.int32), con_w=np.zeros(i["n_con_entries"], np.float64),
             hang_coord=np.zeros((i["n_hanging"], 3), np.int64), dof_coord=np.zeros((i["n_dofs"], 3), np.int64),
             dirichlet=np.zeros(i["n_dofs"], np.uint8), colour=np.zeros(i["n_active"], np.int32),
             top=np.zeros(i["n_active"], np.uint8))
    tab = MeshTables(*[_ptr(t[n]) for n, _ in MeshTables._fields_])
    _check(lib().pbf_mesh_export(h, C.byref(tab)))
    return t


def pbf_mesh_step_tables(h) -> dict:
    """Patch tables of the fused explicit step (host only): sizes first, then the arrays."""
    t = StepTables()
    _check(lib().pbf_mesh_step_tables(h, C.byref(t)))
    npc = pbf_mesh_info(h)["nodes_per_cell"]
    npat, cpp = int(t.n_patches), int(t.cells_per_patch)
    out = dict(ptr=np.zeros(npat, np.int32), cnt=np.zeros((npat, 4), np.int32), slot=np.zeros(t.n_slots, np.int32),
               cell=np.zeros((npat, cpp), np.int32), loc=np.zeros((npat, npc, cpp), np.uint16),
               hloc=np.zeros(t.n_hent, np.uint16), hw=np.zeros(t.n_hent, np.float32))
    if npat:
        for n in ("ptr", "cnt", "slot", "cell", "loc", "hloc", "hw"):
            setattr(t, n, _ptr(out[n]))
        _check(lib().pbf_mesh_step_tables(h, C.byref(t)))
    out.update(cells_per_patch=cpp, max_slots=int(t.max_slots), max_hent=int(t.max_hent))
    return out


def pbf_mesh_transfer_map(h) -> dict:
    """The pending transfer's map (host only): sizes first, then the arrays."""
    t = TransferMapC()
    _check(lib().pbf_mesh_transfer_map(h, C.byref(t)))
    out = dict(ptr=np.zeros(t.n_new + 1, np.int32), idx=np.zeros(t.n_entries, np.int32),
               w=np.zeros(t.n_entries, np.float64))
    t.ptr, t.idx, t.w = (_ptr(out[n]) for n in ("ptr", "idx", "w"))
    _check(lib().pbf_mesh_transfer_map(h, C.byref(t)))
    out.update(n_old=int(t.n_old), n_new=int(t.n_new), fill=float(t.fill))
    return out


def pbf_mesh_history_map(h):
    """The history map of the mesh's last change (host only): ([n_active][(p+1)^3] int32, the old
    mesh's active cells)."""
    i = pbf_mesh_info(h)
    out = np.zeros((i["n_active"], i["nodes_per_cell"]), np.int32)
    n_old = C.c_int64()
    _check(lib().pbf_mesh_history_map(h, C.byref(n_old), _ptr(out)))
    return out, int(n_old.value)


def pbf_mesh_activate_layer(h, z_new_top, material, T_init):
    _check(lib().pbf_mesh_activate_layer(h, float(z_new_top), int(material), float(T_init)))


def pbf_mesh_adapt(h, regions):
    regs = _regions(regions)
    _check(lib().pbf_mesh_adapt(h, len(regions), C.cast(regs, C.c_void_p)))


def pbf_mesh_transfer(h, T_old, T_new, batch=1, stream=None):
    _check(lib().pbf_mesh_transfer(h, _ptr(T_old), _ptr(T_new), int(batch), _stream(stream)))


def pbf_ctx_create(mesh, material: dict, precision=PBF_F64, batch=1):
    h = C.c_void_p()
    m = _material(material)
    _check(lib().pbf_ctx_create(mesh, C.byref(m), int(precision), int(batch), C.byref(h)))
    return h


def pbf_ctx_destroy(h):
    _check(lib().pbf_ctx_destroy(h))


def pbf_ctx_set_k_scale(h, s):
    s = np.ascontiguousarray(s, np.float64)
    _check(lib().pbf_ctx_set_k_scale(h, _ptr(s)))


def pbf_eval_residual(h, T, laser, t, fdiff, fvol, Cm, batch=1, stream=None):
    la = _LaserArg(laser, batch)
    _check(lib().pbf_eval_residual(h, _ptr(T), la.ref, float(t), _ptr(fdiff), _ptr(fvol), _ptr(Cm), _stream(stream)))


def pbf_explicit_step(h, T, laser, t0, dt, nsteps, batch=1, stream=None):
    la = _LaserArg(laser, batch)
    _check(lib().pbf_explicit_step(h, _ptr(T), la.ref, float(t0), float(dt), int(nsteps), _stream(stream)))


def pbf_estimate_dt(h, x0=None, max_iter=200, rtol=1e-6, stream=None):
    lam, dtc, it = C.c_double(), C.c_double(), C.c_int()
    _check(lib().pbf_estimate_dt(h, _ptr(x0), int(max_iter), float(rtol), C.byref(lam), C.byref(dtc),
                                 C.byref(it), _stream(stream)))
    return lam.value, dtc.value, it.value


def pbf_estimate_dt_noalloc(h, x, y, max_iter=200, rtol=1e-6, stream=None):
    """Allocation-free power iteration: x (device, start vector in, last iterate out) and y
    (device work vector) are supplied by the caller."""
    lam, dtc, it = C.c_double(), C.c_double(), C.c_int()
    _check(lib().pbf_estimate_dt_noalloc(h, _ptr(x), _ptr(y), int(max_iter), float(rtol), C.byref(lam),
                                         C.byref(dtc), C.byref(it), _stream(stream)))
    return lam.value, dtc.value, it.value


def pbf_cheb_bounds(h, dt, b=None, n_iter=30, stream=None):
    out = np.zeros(2)
    _check(lib().pbf_cheb_bounds(h, float(dt), _ptr(b), int(n_iter), _ptr(out), _stream(stream)))
    return float(out[0]), float(out[1])


def pbf_implicit_solve(h, T, dt, nsteps, rtol=1e-8, max_it=500, cheb_degree=5, cheb_bounds=None, stream=None):
    iters = np.zeros(max(1, nsteps), np.int32)
    cb = None if cheb_bounds is None else np.ascontiguousarray(cheb_bounds, np.float64)
    st = lib().pbf_implicit_solve(h, _ptr(T), float(dt), int(nsteps), float(rtol), int(max_it), int(cheb_degree),
                                  _ptr(cb), _ptr(iters), _stream(stream))
    return st, iters[:nsteps]


def pbf_implicit_newton(h, T, dt, nsteps, newton_rtol=1e-8, newton_max=50, lin_rtol=1e-4, lin_max=500,
                        cheb_degree=5, cheb_bounds=None, stream=None):
    """Returns (status, Newton corrections per step, BiCGStab iterations per step, largest
    relative residual); PBF_ENOCONV (4) is returned, other failures raise PbfError."""
    nit = np.zeros(max(1, nsteps), np.int32)
    lit = np.zeros(max(1, nsteps), np.int32)
    rel = C.c_double(0.0)
    cb = None if cheb_bounds is None else np.ascontiguousarray(cheb_bounds, np.float64)
    st = lib().pbf_implicit_newton(h, _ptr(T), float(dt), int(nsteps), float(newton_rtol), int(newton_max),
                                   float(lin_rtol), int(lin_max), int(cheb_degree), _ptr(cb), _ptr(nit), _ptr(lit),
                                   C.byref(rel), _stream(stream))
    if st not in (0, 4):
        _check(st)
    return st, nit[:nsteps], lit[:nsteps], rel.value


def pbf_adjoint_sweep(h, T0, laser, t0, dt, nsteps, n_checkpoints, T_target=2300.0, p_exp=16.0, batch=1,
                      stream=None):
    la = _LaserArg(laser, batch)
    n_seg = la.seg.shape[0]
    J = np.zeros(batch)
    grad = np.zeros((batch, n_seg + 1))
    fwd = C.c_longlong()
    _check(lib().pbf_adjoint_sweep(h, _ptr(T0), la.ref, float(t0), float(dt), int(nsteps), int(n_checkpoints),
                                   float(T_target), float(p_exp), _ptr(J), _ptr(grad), C.byref(fwd), _stream(stream)))
    return J, grad, fwd.value


def pbf_revolve_cost(nsteps, n_snaps):
    out = C.c_longlong()
    _check(lib().pbf_revolve_cost(int(nsteps), int(n_snaps), C.byref(out)))
    return out.value


def pbf_round_to_f32(x, y, n, stream=None):
    _check(lib().pbf_round_to_f32(_ptr(x), _ptr(y), int(n), _stream(stream)))


def pbf_widen_to_f64(x, y, n, stream=None):
    _check(lib().pbf_widen_to_f64(_ptr(x), _ptr(y), int(n), _stream(stream)))


N_SHAPES = 10


def pbf_ctx_autotune(h, T, reps=5, stream=None, times=False):
    """Picks the fastest explicit-step shape of an FP32-operator context; returns its index
    (and the microseconds per step of every shape, -1 where a shape does not apply, when
    times=True)."""
    v = C.c_int()
    us = np.zeros(N_SHAPES, np.float32)
    _check(lib().pbf_ctx_autotune(h, _ptr(T), int(reps), C.byref(v), _ptr(us), _stream(stream)))
    return (v.value, us.tolist()) if times else v.value


def pbf_ctx_set_kernel_shape(h, shape):
    _check(lib().pbf_ctx_set_kernel_shape(h, int(shape)))


def pbf_ctx_set_surface_loss(h, q):
    """q: dict with the SurfaceLoss fields, or None to switch the surface loss off."""
    if q is None:
        _check(lib().pbf_ctx_set_surface_loss(h, None))
    else:
        s = SurfaceLoss(*[float(q[n]) for n, _ in SurfaceLoss._fields_])
        _check(lib().pbf_ctx_set_surface_loss(h, C.byref(s)))


def pbf_mesh_adapt_gated(h, regions, cell_rc_min, r_coarsen=0.9):
    regs = _regions(regions)
    rc = np.ascontiguousarray(cell_rc_min, np.float64)
    _check(lib().pbf_mesh_adapt_gated(h, len(regions), C.cast(regs, C.c_void_p), _ptr(rc), float(r_coarsen)))


def pbf_ctx_history_cell_min(h, n_cells, stream=None):
    out = np.zeros(max(1, n_cells))
    _check(lib().pbf_ctx_history_cell_min(h, _ptr(out), _stream(stream)))
    return out[:n_cells]


def pbf_ctx_get_history(h, rc, stream=None):
    """rc: FP64 device tensor [(p+1)^3][n_cells][batch]."""
    _check(lib().pbf_ctx_get_history(h, _ptr(rc), _stream(stream)))


def pbf_ctx_set_history(h, rc, stream=None):
    _check(lib().pbf_ctx_set_history(h, _ptr(rc), _stream(stream)))


def pbf_ctx_transfer_history(h_from, h_to, stream=None):
    _check(lib().pbf_ctx_transfer_history(h_from, h_to, _stream(stream)))


def pbf_ctx_set_phase(h, ph):
    """ph: dict with the Phase fields (T_s, T_l, k_p, k_m, k_s), or None to switch it off."""
    if ph is None:
        _check(lib().pbf_ctx_set_phase(h, None))
    else:
        p = Phase(*[float(ph[n]) for n, _ in Phase._fields_])
        _check(lib().pbf_ctx_set_phase(h, C.byref(p)))


def pbf_ctx_set_barrier_test(h, extra_blocks):
    _check(lib().pbf_ctx_set_barrier_test(h, int(extra_blocks)))


def pbf_ctx_set_timing(h, enable):
    _check(lib().pbf_ctx_set_timing(h, int(bool(enable))))


def pbf_ctx_kernel_time(h):
    ms, n = C.c_double(), C.c_longlong()
    _check(lib().pbf_ctx_kernel_time(h, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def pbf_ctx_launch_count(h):
    n = C.c_longlong()
    _check(lib().pbf_ctx_launch_count(h, C.byref(n)))
    return n.value


# ---- small object wrappers ---------------------------------------------------------------------

class Mesh:
    def __init__(self, desc: dict):
        self.h = pbf_mesh_create(desc)

    def info(self):
        return pbf_mesh_info(self.h)

    def tables(self):
        return pbf_mesh_export(self.h)

    def close(self):
        if self.h:
            pbf_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    def __init__(self, mesh: Mesh, material: dict, precision=PBF_F64, batch=1):
        self.mesh = mesh
        self.batch = batch
        self.h = pbf_ctx_create(mesh.h, material, precision, batch)

    def close(self):
        if self.h:
            pbf_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
