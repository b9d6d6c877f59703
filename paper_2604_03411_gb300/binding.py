"""Thin ctypes binding of the C ABI declared in include/gd.h.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device arrays are passed as torch CUDA tensors (their data pointers);
host arrays as numpy arrays.  Importing this module loads
``_build/libgd.so`` and raises if it has not been built -- there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libgd.so")

GD_OK = 0
STATUS = {0: "GD_OK", 1: "GD_ERR_ARG", 2: "GD_ERR_MESH", 3: "GD_ERR_CUDA", 4: "GD_ERR_OOM",
          5: "GD_ERR_NOT_CONVERGED", 6: "GD_ERR_NAN", 7: "GD_ERR_KRYLOV", 8: "GD_ERR_LOCAL_SOLVE",
          9: "GD_ERR_TIMEOUT", 10: "GD_ERR_STATE"}
globals().update({name: code for code, name in STATUS.items()})
GD_ENERGY_ICNN_RAW, GD_ENERGY_ICNN_ISO, GD_ENERGY_NEO_HOOKE = 0, 1, 2
GD_FP64, GD_MIXED = 0, 1
GD_ASM_RESIDUAL, GD_ASM_TANGENT = 0, 1
GD_INNER_AUTO, GD_INNER_FP64, GD_INNER_REFINED = 0, 1, 2
GD_MONOLITHIC, GD_STAGGERED, GD_STAGGERED_ITERATED = 0, 1, 2
GD_BICGSTAB, GD_GMRES = 0, 1
GD_ICNN_AUTO, GD_ICNN_CUDA_CORES, GD_ICNN_BF16, GD_ICNN_BF16X3 = 0, 1, 2, 3
GD_NOALLOC_MAX_DOFS = 131072

_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i8p = ctypes.POINTER(ctypes.c_int8)
_i64p = ctypes.POINTER(ctypes.c_int64)


class GdMesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_nodes", ctypes.c_int64), ("n_elems", ctypes.c_int64),
                ("coords", _dp), ("conn", _i32p),
                ("n_bc", ctypes.c_int64), ("bc_node", _i32p), ("bc_comp", _i8p), ("bc_scale", _dp),
                ("n_react", ctypes.c_int64), ("react_node", _i32p), ("react_comp", ctypes.c_int32)]


class GdIcnn(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("width", ctypes.c_int32), ("params", _dp)]


class GdMaterial(ctypes.Structure):
    _fields_ = [("mu_e", ctypes.c_double), ("lambda_e", ctypes.c_double), ("eta_d", ctypes.c_double),
                ("kappa_d", ctypes.c_double), ("beta_d", ctypes.c_double), ("c_d", ctypes.c_double),
                ("gamma_d", ctypes.c_double), ("energy", ctypes.c_int32)]


class GdLoadPath(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int32), ("load", _dp)]


class GdOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double),
                ("newton_max", ctypes.c_int32), ("line_search_max", ctypes.c_int32), ("krylov", ctypes.c_int32),
                ("krylov_rtol", ctypes.c_double), ("krylov_max", ctypes.c_int32), ("gmres_m", ctypes.c_int32),
                ("local_max", ctypes.c_int32), ("checkpoint_every", ctypes.c_int32),
                ("max_step_cuts", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p), ("inner_solve", ctypes.c_int32),
                ("coarse", ctypes.c_int32), ("scheme", ctypes.c_int32), ("stagger_max", ctypes.c_int32),
                ("asm_grid_max", ctypes.c_int32), ("krylov_row_cache", ctypes.c_int32), ("icnn_mma", ctypes.c_int32)]


class GdNewtonReport(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("krylov_iterations", ctypes.c_int32), ("line_search_cuts", ctypes.c_int32),
                ("local_failures", ctypes.c_int32), ("loading_points", ctypes.c_int32),
                ("step_cuts", ctypes.c_int32), ("assemblies", ctypes.c_int32),
                ("residual0", ctypes.c_double), ("residual", ctypes.c_double), ("reaction", ctypes.c_double),
                ("max_damage", ctypes.c_double), ("assembly_ms", ctypes.c_double), ("krylov_ms", ctypes.c_double),
                ("yield_evals", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("krylov_fp32_iterations", ctypes.c_int32), ("noise_passes", ctypes.c_int32),
                ("noise", ctypes.c_double), ("noise_ms", ctypes.c_double)]


class GdPathReport(ctypes.Structure):
    _fields_ = [("steps_done", ctypes.c_int32), ("total_newton", ctypes.c_int32),
                ("total_krylov", ctypes.c_int32), ("step_cuts", ctypes.c_int32), ("assemblies", ctypes.c_int32),
                ("assembly_ms", ctypes.c_double), ("krylov_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]


class GdTuneReport(ctypes.Structure):
    _fields_ = [("asm_warps", ctypes.c_int32), ("krylov_ctas_per_sm", ctypes.c_int32),
                ("asm_ms", ctypes.c_double * 3), ("krylov_us", ctypes.c_double * 4),
                ("krylov_up", ctypes.c_int32), ("krylov_us_up", ctypes.c_double * 3),
                ("krylov_lanes", ctypes.c_int32), ("krylov_us_lanes", ctypes.c_double * 3)]


_H = ctypes.c_void_p

# name -> (restype, argtypes); mirrors include/gd.h
PROTOTYPES = {
    "gd_default_options": (None, [ctypes.POINTER(GdOptions)]),
    "gd_create": (ctypes.c_int, [ctypes.POINTER(GdMesh), ctypes.POINTER(GdIcnn), ctypes.POINTER(GdIcnn),
                                 ctypes.POINTER(GdMaterial), ctypes.POINTER(GdLoadPath), ctypes.POINTER(GdOptions),
                                 ctypes.POINTER(_H)]),
    "gd_create_batch": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(GdMesh), ctypes.POINTER(GdIcnn),
                                       ctypes.POINTER(GdIcnn), ctypes.POINTER(GdMaterial), ctypes.POINTER(GdLoadPath),
                                       ctypes.POINTER(GdOptions), ctypes.POINTER(_H)]),
    "gd_batch_layout": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int32), _i64p, _i64p,
                                       ctypes.POINTER(ctypes.c_int32)]),
    "gd_set_params": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p]),
    "gd_csr_pattern": (ctypes.c_int, [_H, _i64p, _i64p, _i32p, _i32p]),
    "gd_build_pattern": (ctypes.c_int, [ctypes.POINTER(GdMesh), _i64p, _i64p, _i32p, _i32p, _i32p]),
    "gd_coarse_info": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "gd_coarse_aggregates": (ctypes.c_int, [ctypes.POINTER(GdMesh), ctypes.c_int32, _i32p,
                                            ctypes.POINTER(ctypes.c_int32)]),
    "gd_coarse_basis": (ctypes.c_int, [ctypes.POINTER(GdMesh), ctypes.c_int32, _i32p, ctypes.POINTER(ctypes.c_int32),
                                       _i32p, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)]),
    "gd_assemble": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "gd_spmv": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "gd_solve": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                _dp]),
    "gd_solve_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_double, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_int32), _dp]),
    "gd_autotune": (ctypes.c_int, [_H, ctypes.POINTER(GdTuneReport)]),
    "gd_newton_step": (ctypes.c_int, [_H, ctypes.POINTER(GdNewtonReport)]),
    "gd_run_load_path": (ctypes.c_int, [_H, _dp, ctypes.POINTER(GdPathReport)]),
    "gd_backward": (ctypes.c_int, [_H, _dp, _dp]),
    "gd_get_fields": (ctypes.c_int, [_H, _dp, _dp, _dp]),
    "gd_set_state": (ctypes.c_int, [_H, _dp, _dp, _dp, _dp, ctypes.c_int32]),
    "gd_get_state": (ctypes.c_int, [_H, _dp, _dp, _dp, _dp, ctypes.POINTER(ctypes.c_int32)]),
    "gd_last_error": (ctypes.c_char_p, [_H]),
    "gd_destroy": (None, [_H]),
}

_lib = None


def lib():
    """The loaded library; raises FileNotFoundError when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FileNotFoundError(f"{LIB_PATH} is missing: build it with "
                                    "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class GDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st, h=None):
    if st != GD_OK:
        msg = lib().gd_last_error(h)
        raise GDError(st, msg.decode() if msg else "")


def _dptr(t) -> int:
    """Device pointer of a torch tensor (or 0 for None)."""
    if t is None:
        return 0
    assert t.is_cuda and t.is_contiguous(), "device arrays must be contiguous CUDA tensors"
    return t.data_ptr()


def _hp(a: Optional[np.ndarray], typ=_dp):
    if a is None:
        return ctypes.cast(None, typ)
    return a.ctypes.data_as(typ)


def gd_default_options(**overrides) -> GdOptions:
    o = GdOptions()
    lib().gd_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


class Handle:
    """Owns a gd_handle; keeps the host arrays alive only during gd_create."""

    def __init__(self, ptr, meta):
        self.ptr = ptr
        self.meta = meta
        # bumped by every call that changes the committed path or the weights (the
        # autograd view checks that the path it differentiates is still the handle's)
        self.generation = 0

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lib().gd_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def _mesh_struct(m):
    """(GdMesh, arrays to keep alive) for a mesh with the fields of inputs.Mesh."""
    coords = np.ascontiguousarray(m.coords, np.float64)
    conn = np.ascontiguousarray(m.conn, np.int32)
    bcn = np.ascontiguousarray(m.bc_node, np.int32)
    bcc = np.ascontiguousarray(m.bc_comp, np.int8)
    bcs = np.ascontiguousarray(m.bc_scale, np.float64)
    rn = np.ascontiguousarray(m.react_node, np.int32)
    mesh = GdMesh(m.dim, coords.shape[0], conn.shape[0], _hp(coords), _hp(conn, _i32p), bcn.size, _hp(bcn, _i32p),
                  _hp(bcc, _i8p), _hp(bcs), rn.size, _hp(rn, _i32p), int(m.react_comp))
    return mesh, (coords, conn, bcn, bcc, bcs, rn)


def gd_build_pattern(m):
    """Host-only: (rowptr, colidx, slot) of the CSR pattern gd_create builds."""
    mesh, keep = _mesh_struct(m)
    nr = ctypes.c_int64()
    nnz = ctypes.c_int64()
    _check(lib().gd_build_pattern(ctypes.byref(mesh), ctypes.byref(nr), ctypes.byref(nnz), None, None, None), None)
    nen = 4 if m.dim == 2 else 8
    rowptr = np.zeros(nr.value + 1, np.int32)
    colidx = np.zeros(nnz.value, np.int32)
    slot = np.zeros(keep[1].shape[0] * nen * nen, np.int32)
    _check(lib().gd_build_pattern(ctypes.byref(mesh), None, None, _hp(rowptr, _i32p), _hp(colidx, _i32p),
                                  _hp(slot, _i32p)), None)
    return rowptr, colidx, slot.reshape(-1, nen, nen)


def gd_coarse_aggregates(m, target_nodes: int):
    """Host-only: (agg [n_nodes], n_aggregates) of the two-level preconditioner's aggregation."""
    mesh, keep = _mesh_struct(m)
    agg = np.zeros(m.n_nodes, np.int32)
    na = ctypes.c_int32()
    _check(lib().gd_coarse_aggregates(ctypes.byref(mesh), int(target_nodes), _hp(agg, _i32p), ctypes.byref(na)), None)
    return agg, na.value


def gd_coarse_basis(m, target_nodes: int):
    """Host-only: (agg [n_nodes], coff [n_agg + 1], P [n_nodes, ndof, n_modes]) of the
    two-level preconditioner's coarse basis."""
    mesh, keep = _mesh_struct(m)
    ndof = m.dim + 1
    nm_max = ndof + (1 if m.dim == 2 else 3)
    agg = np.zeros(m.n_nodes, np.int32)
    coff = np.zeros(m.n_nodes + 1, np.int32)
    P = np.zeros(m.n_nodes * ndof * nm_max, np.float32)
    na = ctypes.c_int32()
    nm = ctypes.c_int32()
    _check(lib().gd_coarse_basis(ctypes.byref(mesh), int(target_nodes), _hp(agg, _i32p), ctypes.byref(na),
                                 _hp(coff, _i32p), P.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                 ctypes.byref(nm)), None)
    return agg, coff[: na.value + 1], P.reshape(m.n_nodes, ndof, nm.value)


def gd_coarse_info(h: Handle):
    """(aggregates, coarse unknowns) of the handle's two-level preconditioner ((0, 0): off)."""
    na = ctypes.c_int32()
    nc = ctypes.c_int32()
    _check(lib().gd_coarse_info(h.ptr, ctypes.byref(na), ctypes.byref(nc)), h.ptr)
    return na.value, nc.value


def gd_create(problem, options: Optional[GdOptions] = None) -> Handle:
    """gd_create from a problem description with fields mesh, psi, yld, mat, load
    (see paper_2604_03411_gb300.inputs)."""
    m = problem.mesh
    mesh, keep = _mesh_struct(m)
    coords, conn = keep[0], keep[1]
    pp = np.ascontiguousarray(problem.psi.params, np.float64) if problem.psi is not None else None
    yp = np.ascontiguousarray(problem.yld.params, np.float64) if problem.yld.width > 0 else None
    psi = GdIcnn(3, problem.psi.width if problem.psi is not None else 0, _hp(pp))
    yld = GdIcnn(1, problem.yld.width, _hp(yp))
    mt = problem.mat
    mat = GdMaterial(mt.mu_e, mt.lambda_e, mt.eta_d, mt.kappa_d, mt.beta_d, mt.c_d, mt.gamma_d, int(mt.energy))
    load = np.ascontiguousarray(problem.load, np.float64)
    path = GdLoadPath(load.size, _hp(load))
    opt = options if options is not None else gd_default_options()
    h = _H()
    _check(lib().gd_create(ctypes.byref(mesh), ctypes.byref(psi), ctypes.byref(yld), ctypes.byref(mat),
                           ctypes.byref(path), ctypes.byref(opt), ctypes.byref(h)), None)
    nen = 4 if m.dim == 2 else 8
    meta = dict(dim=m.dim, n_nodes=coords.shape[0], n_elems=conn.shape[0], ndof=m.dim + 1, nq=nen, nen=nen,
                n_steps=load.size, precision=opt.precision,
                n_psi=pp.size if pp is not None else 0, n_yield=yp.size if yp is not None else 0)
    return Handle(h, meta)


def gd_create_batch(problems, options: Optional[GdOptions] = None) -> Handle:
    """gd_create_batch from a list of problem descriptions (one per specimen; the
    material and options of the first apply to all)."""
    n = len(problems)
    meshes = (GdMesh * n)()
    psis = (GdIcnn * n)()
    ylds = (GdIcnn * n)()
    paths = (GdLoadPath * n)()
    keep = []
    for i, p in enumerate(problems):
        meshes[i], k = _mesh_struct(p.mesh)
        keep.append(k)
        pp = np.ascontiguousarray(p.psi.params, np.float64) if p.psi is not None else None
        yp = np.ascontiguousarray(p.yld.params, np.float64) if p.yld.width > 0 else None
        ld = np.ascontiguousarray(p.load, np.float64)
        keep += [pp, yp, ld]
        psis[i] = GdIcnn(3, p.psi.width if p.psi is not None else 0, _hp(pp))
        ylds[i] = GdIcnn(1, p.yld.width, _hp(yp))
        paths[i] = GdLoadPath(ld.size, _hp(ld))
    mt = problems[0].mat
    mat = GdMaterial(mt.mu_e, mt.lambda_e, mt.eta_d, mt.kappa_d, mt.beta_d, mt.c_d, mt.gamma_d, int(mt.energy))
    opt = options if options is not None else gd_default_options()
    h = _H()
    _check(lib().gd_create_batch(n, meshes, psis, ylds, ctypes.byref(mat), paths, ctypes.byref(opt),
                                 ctypes.byref(h)), None)
    dim = problems[0].mesh.dim
    nen = 4 if dim == 2 else 8
    n_nodes = sum(p.mesh.coords.shape[0] for p in problems)
    n_elems = sum(p.mesh.conn.shape[0] for p in problems)
    meta = dict(dim=dim, n_nodes=n_nodes, n_elems=n_elems, ndof=dim + 1, nq=nen, nen=nen,
                n_steps=max(p.load.size for p in problems), n_spec=n, precision=opt.precision, n_psi=0, n_yield=0)
    return Handle(h, meta)


def gd_batch_layout(h: Handle):
    """(node_off, elem_off, n_steps) of the handle's specimens; offsets have n_spec + 1 entries."""
    ns = ctypes.c_int32()
    st = ctypes.c_int32()
    _check(lib().gd_batch_layout(h.ptr, ctypes.byref(ns), None, None, ctypes.byref(st)), h.ptr)
    no = np.zeros(ns.value + 1, np.int64)
    eo = np.zeros(ns.value + 1, np.int64)
    _check(lib().gd_batch_layout(h.ptr, None, _hp(no, _i64p), _hp(eo, _i64p), None), h.ptr)
    return no, eo, st.value


def gd_set_params(h: Handle, theta_psi=None, theta_yield=None):
    """theta_* may be numpy arrays (host) or CUDA tensors (device), or None to keep."""
    h.generation += 1
    keep = []

    def ptr(a):
        if a is None:
            return None
        if hasattr(a, "is_cuda"):
            if a.is_cuda:
                return _dptr(a)
            a = a.numpy()
        a = np.ascontiguousarray(a, np.float64)
        keep.append(a)
        return a.ctypes.data

    _check(lib().gd_set_params(h.ptr, ptr(theta_psi), ptr(theta_yield)), h.ptr)


def gd_csr_pattern(h: Handle):
    nr = ctypes.c_int64()
    nnz = ctypes.c_int64()
    _check(lib().gd_csr_pattern(h.ptr, ctypes.byref(nr), ctypes.byref(nnz), None, None), h.ptr)
    rowptr = np.zeros(nr.value + 1, np.int32)
    colidx = np.zeros(nnz.value, np.int32)
    _check(lib().gd_csr_pattern(h.ptr, None, None, _hp(rowptr, _i32p), _hp(colidx, _i32p)), h.ptr)
    return rowptr, colidx


def gd_assemble(h: Handle, dofs, kappa_n=None, R=None, csr_vals=None, kappa_trial=None, loading=None,
                mode: int = GD_ASM_TANGENT):
    """All array arguments are contiguous CUDA tensors (or None)."""
    st = lib().gd_assemble(h.ptr, _dptr(dofs), _dptr(kappa_n), _dptr(R), _dptr(csr_vals), _dptr(kappa_trial),
                           _dptr(loading), mode)
    _check(st, h.ptr)


def gd_spmv(h: Handle, x, y, free_only: int = 0):
    _check(lib().gd_spmv(h.ptr, _dptr(x), _dptr(y), int(free_only)), h.ptr)


def gd_solve(h: Handle, b, x, csr_vals=None):
    """Solve K x = b (device FP64 tensors); returns (iterations, relative residual)."""
    it = ctypes.c_int32()
    rel = ctypes.c_double()
    _check(lib().gd_solve(h.ptr, _dptr(csr_vals), _dptr(b), _dptr(x), ctypes.byref(it), ctypes.byref(rel)), h.ptr)
    return it.value, rel.value


def gd_solve_noalloc(ndof, n_nodes, rowptr, colidx, vals, fixed, b, x, rtol, max_it, stream=None):
    """All arrays are contiguous CUDA tensors; returns (iterations, relative residual)."""
    it = ctypes.c_int32()
    rel = ctypes.c_double()
    st = lib().gd_solve_noalloc(int(ndof), int(n_nodes), _dptr(rowptr), _dptr(colidx), _dptr(vals), _dptr(fixed),
                                _dptr(b), _dptr(x), float(rtol), int(max_it), stream, ctypes.byref(it),
                                ctypes.byref(rel))
    _check(st, None)
    return it.value, rel.value


def gd_autotune(h: Handle) -> GdTuneReport:
    rep = GdTuneReport()
    _check(lib().gd_autotune(h.ptr, ctypes.byref(rep)), h.ptr)
    return rep


def gd_newton_step(h: Handle) -> GdNewtonReport:
    h.generation += 1
    rep = GdNewtonReport()
    _check(lib().gd_newton_step(h.ptr, ctypes.byref(rep)), h.ptr)
    return rep


def gd_run_load_path(h: Handle):
    """(reaction [n_steps], report); a batch returns reaction [n_steps, n_spec]."""
    h.generation += 1
    ns = h.meta.get("n_spec", 1)
    reac = np.zeros(max(h.meta["n_steps"], 1) * ns)
    rep = GdPathReport()
    st = lib().gd_run_load_path(h.ptr, _hp(reac), ctypes.byref(rep))
    _check(st, h.ptr)
    if "n_spec" in h.meta:
        return reac[:h.meta["n_steps"] * ns].reshape(h.meta["n_steps"], ns), rep
    return reac[:h.meta["n_steps"]], rep


def gd_backward(h: Handle, dL_dreaction: np.ndarray) -> np.ndarray:
    g = np.ascontiguousarray(dL_dreaction, np.float64)
    out = np.zeros(h.meta["n_psi"] + h.meta["n_yield"])
    _check(lib().gd_backward(h.ptr, _hp(g), _hp(out)), h.ptr)
    return out


def gd_get_fields(h: Handle, damage: bool = False):
    """(dofs, kappa [n_elems, nq]) of the committed state, plus the damage field
    d = 1 - f_d(kappa) [n_elems, nq] when damage=True."""
    d = np.zeros(h.meta["n_nodes"] * h.meta["ndof"])
    k = np.zeros(h.meta["n_elems"] * h.meta["nq"])
    dm = np.zeros_like(k) if damage else None
    _check(lib().gd_get_fields(h.ptr, _hp(d), _hp(k), _hp(dm)), h.ptr)
    shape = (h.meta["n_elems"], h.meta["nq"])
    if damage:
        return d, k.reshape(shape), dm.reshape(shape)
    return d, k.reshape(shape)


def gd_set_state(h: Handle, dofs=None, kappa=None, next_step: int = 0, dofs_prev=None, dofs_prev2=None):
    h.generation += 1
    d = np.ascontiguousarray(dofs, np.float64).ravel() if dofs is not None else None
    dp = np.ascontiguousarray(dofs_prev, np.float64).ravel() if dofs_prev is not None else None
    dpp = np.ascontiguousarray(dofs_prev2, np.float64).ravel() if dofs_prev2 is not None else None
    k = np.ascontiguousarray(kappa, np.float64).ravel() if kappa is not None else None
    _check(lib().gd_set_state(h.ptr, _hp(d), _hp(dp), _hp(dpp), _hp(k), int(next_step)), h.ptr)


def gd_get_state(h: Handle):
    """(dofs, dofs_prev, kappa [n_elems, nq], next_step, dofs_prev2) of the committed state."""
    d = np.zeros(h.meta["n_nodes"] * h.meta["ndof"])
    dp = np.zeros_like(d)
    dpp = np.zeros_like(d)
    k = np.zeros(h.meta["n_elems"] * h.meta["nq"])
    ns = ctypes.c_int32()
    _check(lib().gd_get_state(h.ptr, _hp(d), _hp(dp), _hp(dpp), _hp(k), ctypes.byref(ns)), h.ptr)
    return d, dp, k.reshape(h.meta["n_elems"], h.meta["nq"]), ns.value, dpp


def gd_last_error(h: Optional[Handle] = None) -> str:
    r = lib().gd_last_error(h.ptr if h is not None else None)
    return r.decode() if r else ""


def gd_destroy(h: Handle):
    if h.ptr:
        lib().gd_destroy(h.ptr)
        h.ptr = None
