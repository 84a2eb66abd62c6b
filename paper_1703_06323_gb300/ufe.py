"""Thin ctypes binding of libufe (include/ufe.h), with the C ABI's own names.

Only argument marshalling happens here: numpy arrays are passed as host
pointers (UFE_MEM_HOST), torch CUDA tensors as device pointers (UFE_MEM_DEVICE)
on torch's current stream.  Every step of the solver runs in the CUDA library;
if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build_ext

OK = 0
ERR_INVALID_ARG, ERR_OUT_OF_MEMORY, ERR_CUDA = -1, -2, -3
ERR_SINGULAR_LOCAL, ERR_SINGULAR_COARSE, ERR_BREAKDOWN = -4, -5, -6
ERR_NO_CONVERGENCE, ERR_UNSUPPORTED, ERR_TIMEOUT = -7, -8, -9
MEM_HOST, MEM_DEVICE = 0, 1
CELL_EXTERNAL, CELL_CUT, CELL_INTERNAL = 0, 1, 2
OBJ_CORNER, OBJ_EDGE, OBJ_FACE = 0, 1, 2
WEIGHT_STIFFNESS, WEIGHT_TOPOLOGICAL = 0, 1
OBJECTS_STANDARD, OBJECTS_VARIANT1, OBJECTS_VARIANT2 = 0, 1, 2
COARSE_C, COARSE_CE, COARSE_CEF = 0, 1, 2
PREC_FP64, PREC_MIXED = 0, 1
COARSE_SOLVER_AUTO, COARSE_SOLVER_DENSE, COARSE_SOLVER_CR, COARSE_SOLVER_BDDC = 0, 1, 2, 3
PIN_NONE, PIN_AUTO = -1, -2


class UfeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ufe status {status}: {msg}")
        self.status = status


class MeshInfo(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_cells", ctypes.c_int64), ("n_active_cells", ctypes.c_int64),
                ("n_cut_cells", ctypes.c_int64), ("n_dof", ctypes.c_int64), ("n_subdomains", ctypes.c_int64),
                ("n_interface_dofs", ctypes.c_int64), ("pinned_node", ctypes.c_int64),
                ("n_constrained", ctypes.c_int64), ("max_interior", ctypes.c_int32),
                ("max_interface", ctypes.c_int32)]


class BddcOpts(ctypes.Structure):
    _fields_ = [("weighting", ctypes.c_int32), ("objects", ctypes.c_int32), ("coarse", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("coarse_solver", ctypes.c_int32), ("coarse_group", ctypes.c_int32),
                ("coarse_keep_corners", ctypes.c_int32)]


class BddcInfo(ctypes.Structure):
    _fields_ = [("n_objects", ctypes.c_int64), ("n_corners", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("n_faces", ctypes.c_int64), ("n_coarse", ctypes.c_int64), ("max_local_coarse", ctypes.c_int32),
                ("setup_ms", ctypes.c_double), ("inverse_flops_local", ctypes.c_double),
                ("inverse_flops_coarse", ctypes.c_double), ("bytes_interior_inverse", ctypes.c_double),
                ("bytes_neumann", ctypes.c_double), ("bytes_coarse_basis", ctypes.c_double),
                ("bytes_offdiag", ctypes.c_double), ("bytes_coarse_inverse", ctypes.c_double),
                ("interior_slots", ctypes.c_int64), ("interface_slots", ctypes.c_int64),
                ("fp64_refactor", ctypes.c_int32), ("coarse_solver", ctypes.c_int32), ("cphi_error", ctypes.c_double),
                ("coarse_layers", ctypes.c_int32), ("coarse_levels", ctypes.c_int32),
                ("local_tensor_cores", ctypes.c_int32), ("prec_cluster", ctypes.c_int32),
                ("prec_stages", ctypes.c_int32), ("fp64_subdomains", ctypes.c_int32),
                ("level2_subdomains", ctypes.c_int32), ("level3_coarse", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxit", ctypes.c_int32), ("flexible", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("true_rel_residual", ctypes.c_double), ("solve_ms", ctypes.c_double)]


def _load():
    path = build_ext.LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libufe is not built ({path}); run paper_1703_06323_gb300.build_ext.build()")
    lib = ctypes.CDLL(path)
    P, I32, I64, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "ufe_last_error": (ctypes.c_char_p, []),
        "ufe_version": (ctypes.c_int, []),
        "ufe_kernel_launches": (ctypes.c_int64, []),
        "ufe_timing_enable": (None, [ctypes.c_int]),
        "ufe_timing_reset": (None, []),
        "ufe_timing_get": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int64)]),
        "ufe_probe_fma_rate": (ctypes.c_int, [ctypes.c_int, P, ctypes.POINTER(ctypes.c_double)]),
        "ufe_mesh_create": (ctypes.c_int, [P, P, P, P, P, ctypes.c_int, U32, I64, P, ctypes.POINTER(P)]),
        "ufe_mesh_get_info": (ctypes.c_int, [P, ctypes.POINTER(MeshInfo)]),
        "ufe_mesh_get_cell_types": (ctypes.c_int, [P, P, ctypes.c_int]),
        "ufe_mesh_get_dof_map": (ctypes.c_int, [P, P, ctypes.c_int]),
        "ufe_mesh_get_subdomains": (ctypes.c_int, [P, P, ctypes.c_int]),
        "ufe_mesh_get_neighbours": (ctypes.c_int, [P, P, ctypes.c_int]),
        "ufe_mesh_destroy": (None, [P]),
        "ufe_assemble": (ctypes.c_int, [P, P, P, P, P, ctypes.c_int, ctypes.POINTER(P)]),
        "ufe_assemble_elastic": (ctypes.c_int, [P, ctypes.c_double, ctypes.c_double, P, P, P, P, ctypes.c_int,
                                                ctypes.POINTER(P)]),
        "ufe_assemble_nitsche": (ctypes.c_int, [P, P, P, ctypes.c_int, ctypes.POINTER(P)]),
        "ufe_system_get_nitsche_beta": (ctypes.c_int, [P, P, ctypes.c_int]),
        "ufe_system_get_info": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
        "ufe_system_get_rhs": (ctypes.c_int, [P, P, ctypes.c_int]),
        "ufe_system_apply": (ctypes.c_int, [P, P, P, ctypes.c_int]),
        "ufe_system_set_kappa": (ctypes.c_int, [P, P, ctypes.c_int]),
        "ufe_system_get_cut_data": (ctypes.c_int, [P, P, P, P, P, ctypes.c_int]),
        "ufe_system_destroy": (None, [P]),
        "ufe_bddc_setup": (ctypes.c_int, [P, ctypes.POINTER(BddcOpts), ctypes.POINTER(P)]),
        "ufe_bddc_get_info": (ctypes.c_int, [P, ctypes.POINTER(BddcInfo)]),
        "ufe_bddc_get_objects": (ctypes.c_int, [P, P, P, P, ctypes.c_int]),
        "ufe_bddc_apply": (ctypes.c_int, [P, P, P, ctypes.c_int]),
        "ufe_bddc_apply_noalloc": (ctypes.c_int, [P, P, P]),
        "ufe_bddc_destroy": (None, [P]),
        "ufe_pcg_solve": (ctypes.c_int, [P, P, P, P, ctypes.c_int, ctypes.POINTER(SolveOpts),
                                         ctypes.POINTER(SolveInfo)]),
        "ufe_pcg_solve_batched": (ctypes.c_int, [ctypes.c_int32, P, P, P, P, ctypes.c_int,
                                                 ctypes.POINTER(SolveOpts), P]),
        "ufe_adjoint": (ctypes.c_int, [P, P, P, P, P, P, ctypes.c_int, ctypes.POINTER(SolveOpts),
                                       ctypes.POINTER(SolveInfo)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()
EXPORTED = ("ufe_last_error", "ufe_version", "ufe_kernel_launches", "ufe_timing_enable", "ufe_timing_reset",
            "ufe_timing_get", "ufe_probe_fma_rate", "ufe_mesh_create", "ufe_mesh_get_info", "ufe_mesh_get_cell_types",
            "ufe_mesh_get_dof_map", "ufe_mesh_get_subdomains", "ufe_mesh_get_neighbours", "ufe_mesh_destroy",
            "ufe_assemble", "ufe_assemble_elastic", "ufe_assemble_nitsche", "ufe_system_get_nitsche_beta", "ufe_system_get_info", "ufe_system_get_rhs", "ufe_system_apply", "ufe_system_set_kappa",
            "ufe_system_get_cut_data",
            "ufe_system_destroy", "ufe_bddc_setup", "ufe_bddc_get_info", "ufe_bddc_get_objects", "ufe_bddc_apply",
            "ufe_bddc_apply_noalloc",
            "ufe_bddc_destroy", "ufe_pcg_solve", "ufe_pcg_solve_batched", "ufe_adjoint")


def _check(status):
    if status != OK:
        raise UfeError(status, LIB.ufe_last_error().decode())


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, mem, keepalive) of an array argument; None passes NULL."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return ctypes.c_void_p(a.data_ptr()), (MEM_DEVICE if a.is_cuda else MEM_HOST), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), MEM_HOST, arr


def _mem_of(*args):
    mems = {m for (_, m, _) in args if m is not None}
    if len(mems) > 1:
        raise TypeError("mix of host and device arrays in one call")
    return mems.pop() if mems else MEM_HOST


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def ufe_version():
    return LIB.ufe_version()


def ufe_kernel_launches():
    return LIB.ufe_kernel_launches()


def ufe_timing_enable(on=True):
    LIB.ufe_timing_enable(1 if on else 0)


def ufe_timing_reset():
    LIB.ufe_timing_reset()


def ufe_timing_get(kernel):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(LIB.ufe_timing_get(kernel.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def ufe_probe_fma_rate(kind, stream=None):
    """Measured FMA rate (TFLOP/s) of the current device: kind "fp64" or "fp32"."""
    out = ctypes.c_double()
    _check(LIB.ufe_probe_fma_rate({"fp64": 0, "fp32": 1}[kind], _stream(stream), ctypes.byref(out)))
    return out.value


def ufe_mesh_create(box_lo, box_hi, cells, sub_cells, phi_nodes, dirichlet_face_mask=0, pin_node=PIN_AUTO,
                    stream=None):
    lo = (ctypes.c_double * 3)(*box_lo)
    hi = (ctypes.c_double * 3)(*box_hi)
    c = (ctypes.c_int32 * 3)(*cells)
    s = (ctypes.c_int32 * 3)(*sub_cells)
    phi = _ptr(phi_nodes, np.float64)
    out = ctypes.c_void_p()
    _check(LIB.ufe_mesh_create(lo, hi, c, s, phi[0], phi[1], int(dirichlet_face_mask), int(pin_node),
                               _stream(stream), ctypes.byref(out)))
    return out


def ufe_mesh_get_info(mesh):
    info = MeshInfo()
    _check(LIB.ufe_mesh_get_info(mesh, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in MeshInfo._fields_}


def _get(fn, handle, n, dtype):
    out = np.empty(n, dtype=dtype)
    _check(fn(handle, ctypes.c_void_p(out.ctypes.data), MEM_HOST))
    return out


def ufe_mesh_get_cell_types(mesh):
    return _get(LIB.ufe_mesh_get_cell_types, mesh, ufe_mesh_get_info(mesh)["n_cells"], np.uint8)


def ufe_mesh_get_dof_map(mesh):
    return _get(LIB.ufe_mesh_get_dof_map, mesh, ufe_mesh_get_info(mesh)["n_nodes"], np.int32)


def ufe_mesh_get_subdomains(mesh):
    return _get(LIB.ufe_mesh_get_subdomains, mesh, ufe_mesh_get_info(mesh)["n_cells"], np.int32)


def ufe_mesh_get_neighbours(mesh):
    n = ufe_mesh_get_info(mesh)["n_dof"]
    return _get(LIB.ufe_mesh_get_neighbours, mesh, n * 8, np.int32).reshape(n, 8)


def ufe_mesh_destroy(mesh):
    LIB.ufe_mesh_destroy(mesh)


def ufe_assemble(mesh, kappa_cells=None, f_nodes=None, flux_nodes=None, dirichlet_values=None):
    args = [_ptr(kappa_cells, np.float64), _ptr(f_nodes, np.float64), _ptr(flux_nodes, np.float64),
            _ptr(dirichlet_values, np.float64)]
    mem = _mem_of(*args)
    out = ctypes.c_void_p()
    _check(LIB.ufe_assemble(mesh, args[0][0], args[1][0], args[2][0], args[3][0], mem, ctypes.byref(out)))
    return out


def ufe_assemble_nitsche(mesh, f_nodes, dirichlet_values):
    """Poisson with weak (Nitsche) Dirichlet data on the unfitted boundary; dirichlet_values
    are also the strong values at the constrained box nodes."""
    args = [_ptr(f_nodes, np.float64), _ptr(dirichlet_values, np.float64)]
    mem = _mem_of(*args)
    out = ctypes.c_void_p()
    _check(LIB.ufe_assemble_nitsche(mesh, args[0][0], args[1][0], mem, ctypes.byref(out)))
    return out


def ufe_system_get_nitsche_beta(system, n_cut):
    return _get(LIB.ufe_system_get_nitsche_beta, system, n_cut, np.float64)


def ufe_assemble_elastic(mesh, E, nu, E_scale_cells=None, f_nodes=None, stress_nodes=None, dirichlet_values=None):
    """Q1^3 linear elasticity: f (n_nodes, 3), stress (n_nodes, 9) or None, Dirichlet values (n_nodes, 3)."""
    def flat(a):
        return None if a is None else (a.reshape(-1) if _is_torch(a) else np.asarray(a).reshape(-1))
    args = [_ptr(flat(E_scale_cells), np.float64), _ptr(flat(f_nodes), np.float64),
            _ptr(flat(stress_nodes), np.float64), _ptr(flat(dirichlet_values), np.float64)]
    mem = _mem_of(*args)
    out = ctypes.c_void_p()
    _check(LIB.ufe_assemble_elastic(mesh, float(E), float(nu), args[0][0], args[1][0], args[2][0], args[3][0], mem,
                                    ctypes.byref(out)))
    return out


def ufe_system_get_info(system):
    nc = ctypes.c_int32()
    n = ctypes.c_int64()
    _check(LIB.ufe_system_get_info(system, ctypes.byref(nc), ctypes.byref(n)))
    return {"ncomp": nc.value, "n": n.value}


def ufe_system_get_rhs(system, n):
    """The assembled right-hand side (n = ncomp * n_dof doubles)."""
    return _get(LIB.ufe_system_get_rhs, system, n, np.float64)


def ufe_system_apply(system, x, y=None):
    xp = _ptr(x, np.float64)
    if y is None:
        y = np.empty(len(x), dtype=np.float64) if xp[1] == MEM_HOST else x.new_empty(x.shape)
    yp = _ptr(y, np.float64)
    _check(LIB.ufe_system_apply(system, xp[0], yp[0], _mem_of(xp, yp)))
    return y


def ufe_system_set_kappa(system, kappa):
    kp = _ptr(kappa, np.float64)
    _check(LIB.ufe_system_set_kappa(system, kp[0], kp[1]))


def ufe_system_get_cut_data(system, n_cut):
    ne = 8 * ufe_system_get_info(system)["ncomp"]
    cells = np.empty(n_cut, np.int32)
    K = np.empty(n_cut * ne * ne, np.float64)
    load = np.empty(n_cut * ne, np.float64)
    eta = np.empty(n_cut, np.float64)
    ptrs = [ctypes.c_void_p(a.ctypes.data) for a in (cells, K, load, eta)]
    _check(LIB.ufe_system_get_cut_data(system, *ptrs, MEM_HOST))
    return cells, K.reshape(n_cut, ne, ne), load.reshape(n_cut, ne), eta


def ufe_system_destroy(system):
    LIB.ufe_system_destroy(system)


def ufe_bddc_setup(system, weighting=WEIGHT_STIFFNESS, objects=OBJECTS_VARIANT1, coarse=COARSE_CEF,
                   precision=PREC_FP64, coarse_solver=0, coarse_group=0, coarse_keep_corners=0):
    opts = BddcOpts(weighting, objects, coarse, precision, coarse_solver, coarse_group, coarse_keep_corners)
    out = ctypes.c_void_p()
    _check(LIB.ufe_bddc_setup(system, ctypes.byref(opts), ctypes.byref(out)))
    return out


def ufe_bddc_get_info(bddc):
    info = BddcInfo()
    _check(LIB.ufe_bddc_get_info(bddc, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in BddcInfo._fields_}


def ufe_bddc_get_objects(bddc, n_dof):
    n_obj = ufe_bddc_get_info(bddc)["n_objects"]
    obj = np.empty(n_dof, np.int32)
    kind = np.empty(max(n_obj, 1), np.int32)
    coarse = np.empty(max(n_obj, 1), np.int32)
    _check(LIB.ufe_bddc_get_objects(bddc, ctypes.c_void_p(obj.ctypes.data), ctypes.c_void_p(kind.ctypes.data),
                                    ctypes.c_void_p(coarse.ctypes.data), MEM_HOST))
    return obj, kind[:n_obj], coarse[:n_obj]


def ufe_bddc_apply(bddc, r, z=None):
    rp = _ptr(r, np.float64)
    if z is None:
        z = np.empty(len(r), dtype=np.float64) if rp[1] == MEM_HOST else r.new_empty(r.shape)
    zp = _ptr(z, np.float64)
    _check(LIB.ufe_bddc_apply(bddc, rp[0], zp[0], _mem_of(rp, zp)))
    return z


def ufe_bddc_apply_noalloc(bddc, r, z):
    """z = M r into a preallocated device tensor, without any device allocation."""
    if not (_is_torch(r) and _is_torch(z) and r.is_cuda and z.is_cuda):
        raise TypeError("ufe_bddc_apply_noalloc takes CUDA tensors")
    rp = _ptr(r, np.float64)
    zp = _ptr(z, np.float64)
    _check(LIB.ufe_bddc_apply_noalloc(bddc, rp[0], zp[0]))
    return z


def ufe_bddc_destroy(bddc):
    LIB.ufe_bddc_destroy(bddc)


def ufe_pcg_solve(system, bddc, b, x, rtol=1e-8, maxit=1000, flexible=-1, check_every=8, raise_on_error=True):
    """Solve in place into x (numpy float64 or torch CUDA float64); returns (status, info dict)."""
    bp = _ptr(b, np.float64)
    xp = _ptr(x, np.float64)
    mem = _mem_of(bp, xp)
    opts = SolveOpts(float(rtol), int(maxit), int(flexible), int(check_every), 0)
    info = SolveInfo()
    st = LIB.ufe_pcg_solve(system, bddc, bp[0], xp[0], mem, ctypes.byref(opts), ctypes.byref(info))
    if xp[1] == MEM_HOST and not _is_torch(x) and xp[2] is not x:
        x[:] = xp[2]
    if raise_on_error:
        _check(st)
    return st, {k: getattr(info, k) for k, _ in SolveInfo._fields_}


def ufe_pcg_solve_batched(systems, bddcs, bs, xs, rtol=1e-8, maxit=1000, flexible=-1, raise_on_error=True):
    """Solve every (system, bddc) pair at once into xs[i] (numpy or torch CUDA float64;
    bs None or a list with None for the assembled right-hand side); returns (status, infos)."""
    n = len(systems)
    if not (len(bddcs) == n and len(xs) == n and (bs is None or len(bs) == n)):
        raise ValueError("systems, bddcs, xs (and bs) must have the same length")
    xp = [_ptr(x, np.float64) for x in xs]
    bp = [_ptr(b, np.float64) for b in bs] if bs is not None else [(None, None, None)] * n
    mem = _mem_of(*xp, *bp)
    Parr = ctypes.c_void_p * max(n, 1)
    sys_a = Parr(*[ctypes.cast(h, ctypes.c_void_p) for h in systems])
    bd_a = Parr(*[ctypes.cast(h, ctypes.c_void_p) for h in bddcs])
    b_a = Parr(*[p[0] for p in bp])
    x_a = Parr(*[p[0] for p in xp])
    infos = (SolveInfo * max(n, 1))()
    opts = SolveOpts(float(rtol), int(maxit), int(flexible), 0, 0)
    st = LIB.ufe_pcg_solve_batched(n, sys_a, bd_a, b_a, x_a, mem, ctypes.byref(opts), infos)
    for x, p in zip(xs, xp):
        if p[1] == MEM_HOST and not _is_torch(x) and p[2] is not x:
            x[:] = p[2]
    if raise_on_error:
        _check(st)
    return st, [{k: getattr(infos[i], k) for k, _ in SolveInfo._fields_} for i in range(n)]


def ufe_adjoint(system, bddc, u, dJdu, lam, dJdkappa, rtol=1e-8, maxit=1000, flexible=-1, check_every=8):
    args = [_ptr(a, np.float64) for a in (u, dJdu, lam, dJdkappa)]
    mem = _mem_of(*args)
    opts = SolveOpts(float(rtol), int(maxit), int(flexible), int(check_every), 0)
    info = SolveInfo()
    _check(LIB.ufe_adjoint(system, bddc, args[0][0], args[1][0], args[2][0], args[3][0], mem, ctypes.byref(opts),
                           ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in SolveInfo._fields_}
