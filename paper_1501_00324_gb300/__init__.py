"""Python binding of libfespmv (include/fespmv.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: device vectors are torch CUDA tensors (their
``data_ptr()`` is passed), host arrays are numpy arrays, and the stream
defaults to torch's current CUDA stream.  The compiled library must be present
(it is built in-tree by ``__graft_entry__.build()`` or on first import); if it
cannot be loaded, importing this package raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

# ---- constants mirrored from include/fespmv.h -------------------------------------
FESPMV_OK = 0
FESPMV_ERR_INVALID_ARG = -1
FESPMV_ERR_BAD_CSR = -2
FESPMV_ERR_OOM = -3
FESPMV_ERR_CUDA = -4
FESPMV_ERR_BREAKDOWN = -5
FESPMV_ERR_NOT_CONVERGED = -6
FESPMV_ERR_UNSUPPORTED = -7
FESPMV_ERR_CANCELLED = -8
FESPMV_PENDING = 1

FESPMV_FMT_CSR = 0
FESPMV_FMT_SLICED = 1
FESPMV_REORDER_NONE = 0
FESPMV_REORDER_MORTON = 1
FESPMV_COLS_SORTED = 0
FESPMV_COLS_RENUMBERED = 1
FESPMV_COLS_ORIGINAL = 2
FESPMV_PREC_F64 = 1
FESPMV_PREC_F32 = 2
FESPMV_PREC_BF16 = 4
FESPMV_PREC_DF64 = 8
FESPMV_IO_PERMUTED = 1
FESPMV_IO_HOST = 2
FESPMV_EXPORT_PERM = 0
FESPMV_EXPORT_META = 1
FESPMV_EXPORT_COLS = 2
FESPMV_EXPORT_VALUES = 3
FESPMV_EXPORT_SRCMAP = 4
FESPMV_EXPORT_DIAG = 5
FESPMV_EXPORT_VALUES_F32 = 6
FESPMV_EXPORT_VALUES_BF16 = 7
FESPMV_EXPORT_SCALE = 8
FESPMV_EXPORT_TILES = 9
FESPMV_EXPORT_TILE_COLS = 10
FESPMV_EXPORT_TILE_INDEX = 11
FESPMV_EXPORT_NB_META = 12
FESPMV_EXPORT_NB_COLS = 13
FESPMV_EXPORT_NB_VALUES_F32 = 14
FESPMV_EXPORT_NB_VALUES_BF16 = 15
FESPMV_EXPORT_NB_MAP = 16
FESPMV_EXPORT_NB_TILES = 17
FESPMV_EXPORT_NB_TILE_NODES = 18
FESPMV_EXPORT_NB_TILE_INDEX = 19
FESPMV_CG_F64 = 0
FESPMV_CG_F32_REFINE = 1
FESPMV_CG_BF16_REFINE = 2
FESPMV_CG_X0 = 4
FESPMV_CG_NO_PRECOND = 8
FESPMV_CG_SINGLE_REDUCTION = 16
FESPMV_CG_RELIABLE = 32
FESPMV_CG_FLEXIBLE = 64
FESPMV_CG_NO_CLUSTER = 128


class FespmvError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class fespmv_options(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in
                ("format", "reorder", "sigma", "threshold", "vec", "csr_lanes", "precisions",
                 "block", "tiles", "node_blocks", "col_order")]


class fespmv_mesh_info(ctypes.Structure):
    _fields_ = [("dofs_per_node", ctypes.c_int32), ("node_xyz", ctypes.c_void_p)]


class fespmv_info(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_slices", ctypes.c_int64),
                ("packed_len", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("format", ctypes.c_int32), ("vec", ctypes.c_int32), ("n_tiles", ctypes.c_int64),
                ("tile_dict_len", ctypes.c_int64), ("tile_max_cols", ctypes.c_int32),
                ("node_blocks", ctypes.c_int32), ("nb_slices", ctypes.c_int64), ("nb_len", ctypes.c_int64),
                ("nb_tiles", ctypes.c_int64), ("nb_tile_dict_len", ctypes.c_int64)]


class cg_options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("max_restarts", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("inner_steps", ctypes.c_int32), ("pad", ctypes.c_int32)]


class cg_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("outer", ctypes.c_int32), ("relres", ctypes.c_double),
                ("true_relres", ctypes.c_double)]


class fe_newton_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps", ctypes.c_int32), ("cg_iters", ctypes.c_int64),
                ("res_norm0", ctypes.c_double), ("res_norm", ctypes.c_double), ("dx_norm", ctypes.c_double),
                ("last_cg", cg_result)]


# int (*)(const double* phi, double* Ke, double* Re, void* user, stream)
FE_ELEMENT_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p)


class srv_timing(ctypes.Structure):
    _fields_ = [("t_queue_s", ctypes.c_double), ("t_solve_s", ctypes.c_double),
                ("t_total_s", ctypes.c_double)]


class srv_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "queued", "active",
                                              "peak_active", "workspace_bytes",
                                              "peak_workspace_bytes", "grouped")]


def _load():
    path = _build.build()
    try:
        return ctypes.CDLL(path)
    except OSError as e:  # pragma: no cover - a broken build is an error, not a fallback
        raise ImportError(f"libfespmv could not be loaded from {path}: {e}") from e


LIB_PATH = _build.SO
_lib = _load()
_P = ctypes.c_void_p
_i32, _i64 = ctypes.c_int32, ctypes.c_int64
_lib.spmv_create.argtypes = [ctypes.POINTER(_P), _i64, _P, _P, _P, ctypes.POINTER(fespmv_mesh_info),
                             ctypes.POINTER(fespmv_options), _P]
_lib.spmv_create.restype = ctypes.c_int
_lib.spmv_destroy.argtypes = [_P]
_lib.spmv_destroy.restype = None
_lib.spmv_apply.argtypes = [_P, _P, _P, _i32, _P]
_lib.spmv_apply.restype = ctypes.c_int
_lib.spmv_apply_scaled.argtypes = [_P, _P, _P, _i32, _i32, _P]
_lib.spmv_apply_scaled.restype = ctypes.c_int
_lib.spmv_apply_multi.argtypes = [_P, _P, _P, _i32, _i32, _i32, _P]
_lib.spmv_apply_multi.restype = ctypes.c_int
_lib.spmv_permute.argtypes = [_P, _P, _P, _i32, _P]
_lib.spmv_permute.restype = ctypes.c_int
_lib.spmv_update_values.argtypes = [_P, _P, _i32, _P]
_lib.spmv_update_values.restype = ctypes.c_int
_lib.spmv_get_info.argtypes = [_P, ctypes.POINTER(fespmv_info)]
_lib.spmv_get_info.restype = ctypes.c_int
_lib.spmv_export.argtypes = [_P, _i32, _P, ctypes.c_size_t, _P]
_lib.spmv_export.restype = ctypes.c_int
_lib.spmv_plan.argtypes = [_i64, _P, _P, ctypes.POINTER(fespmv_mesh_info),
                           ctypes.POINTER(fespmv_options), ctypes.POINTER(fespmv_info), _P, _P, _P, _P]
_lib.spmv_plan.restype = ctypes.c_int
_lib.spmv_plan_tiles.argtypes = [_i64, _i64, _P, _i64, _P, _P, _P, _P, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
_lib.spmv_plan_tiles.restype = ctypes.c_int
_lib.cg_solve.argtypes = [_P, _P, _P, ctypes.POINTER(cg_options), ctypes.POINTER(cg_result), _P]
_lib.cg_solve.restype = ctypes.c_int
_lib.cg_solve_multi.argtypes = [_P, _P, _P, _i32, ctypes.POINTER(cg_options), _P, _P]
_lib.cg_solve_multi.restype = ctypes.c_int
_lib.assembly_create.argtypes = [ctypes.POINTER(_P), _P, _P, _P, _i64, _i32, _i32, _P, _P, _P]
_lib.assembly_create.restype = ctypes.c_int
_lib.assembly_matrix.argtypes = [_P, _P, _i32, _P]
_lib.assembly_matrix.restype = ctypes.c_int
_lib.assembly_vector.argtypes = [_P, _P, _P, _i32, _P]
_lib.assembly_vector.restype = ctypes.c_int
_lib.assembly_get_info.argtypes = [_P, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
_lib.assembly_get_info.restype = ctypes.c_int
_lib.assembly_destroy.argtypes = [_P]
_lib.assembly_destroy.restype = None
_lib.fe_newton_step.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.POINTER(cg_options),
                                ctypes.POINTER(fe_newton_result), _P]
_lib.fe_newton_step.restype = ctypes.c_int
_lib.fe_newton_solve.argtypes = [_P, _P, FE_ELEMENT_FN, _P, _P, _P, _P, _P, ctypes.c_double, _i32,
                                 ctypes.POINTER(cg_options), ctypes.POINTER(fe_newton_result), _P]
_lib.fe_newton_solve.restype = ctypes.c_int
_lib.srv_create.argtypes = [ctypes.POINTER(_P), _i64, _i32]
_lib.srv_create.restype = ctypes.c_int
_lib.srv_set_grouping.argtypes = [_P, _i32]
_lib.srv_set_grouping.restype = ctypes.c_int
_lib.srv_register.argtypes = [_P, _P, ctypes.POINTER(_i32)]
_lib.srv_register.restype = ctypes.c_int
_lib.srv_submit.argtypes = [_P, _i32, _P, ctypes.POINTER(cg_options), ctypes.POINTER(_i64)]
_lib.srv_submit.restype = ctypes.c_int
_lib.srv_poll.argtypes = [_P, _i64, _i32, _P, ctypes.POINTER(cg_result), ctypes.POINTER(srv_timing)]
_lib.srv_poll.restype = ctypes.c_int
_lib.srv_get_stats.argtypes = [_P, ctypes.POINTER(srv_stats)]
_lib.srv_get_stats.restype = ctypes.c_int
_lib.srv_cancel_queued.argtypes = [_P, ctypes.POINTER(_i64)]
_lib.srv_cancel_queued.restype = ctypes.c_int
_lib.srv_destroy.argtypes = [_P]
_lib.srv_destroy.restype = None
_PP = ctypes.POINTER(_P)
_lib.batch_create.argtypes = [ctypes.POINTER(_P), _i32, _P, _P, _P, _P, _P, ctypes.POINTER(fespmv_options), _P]
_lib.batch_create.restype = ctypes.c_int
_lib.batch_destroy.argtypes = [_P]
_lib.batch_destroy.restype = None
_lib.batch_spmv.argtypes = [_P, _P, _P, _P]
_lib.batch_spmv.restype = ctypes.c_int
_lib.batch_cg_solve.argtypes = [_P, _P, _P, ctypes.POINTER(cg_options), _P, _P]
_lib.batch_cg_solve.restype = ctypes.c_int
_lib.batch_get_info.argtypes = [_P, ctypes.POINTER(fespmv_info), ctypes.POINTER(_i64)]
_lib.batch_get_info.restype = ctypes.c_int
_lib.spmv_autotune.argtypes = [_i64, _P, _P, _P, ctypes.POINTER(fespmv_mesh_info),
                               ctypes.POINTER(fespmv_options), _i32, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(_i32), _P]
_lib.spmv_autotune.restype = ctypes.c_int
_lib.fespmv_status_string.argtypes = [ctypes.c_int]
_lib.fespmv_status_string.restype = ctypes.c_char_p
_lib.fespmv_last_error.argtypes = []
_lib.fespmv_last_error.restype = ctypes.c_char_p


def lib():
    """The loaded ctypes library (for callers that marshal arguments themselves)."""
    return _lib


def _check(rc: int):
    if rc != FESPMV_OK:
        msg = _lib.fespmv_last_error().decode() or _lib.fespmv_status_string(rc).decode()
        raise FespmvError(rc, msg)


def last_error() -> str:
    """The calling thread's last error message of the library (fespmv_last_error)."""
    return _lib.fespmv_last_error().decode()


def _stream(stream):
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(a):
    """Address of a torch tensor or numpy array (contiguity is the caller's job)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(a.data_ptr())


class Matrix:
    """A handle returned by spmv_create (owns device memory until spmv_destroy)."""

    def __init__(self, handle: ctypes.c_void_p, n_rows: int, nnz: int):
        self.handle = handle
        self.n_rows = n_rows
        self.nnz = nnz

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            try:
                _lib.spmv_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def spmv_create(rowptr, colind, values, node_xyz=None, dofs_per_node=1, format=FESPMV_FMT_SLICED,
                reorder=None, sigma=0, threshold=0, vec=0, csr_lanes=0, precisions=0, block=0,
                tiles=0, node_blocks=0, col_order=0, stream=None) -> Matrix:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    values = np.ascontiguousarray(values, dtype=np.float64)
    xyz = None if node_xyz is None else np.ascontiguousarray(node_xyz, dtype=np.float64)
    if reorder is None:
        reorder = FESPMV_REORDER_MORTON if xyz is not None else FESPMV_REORDER_NONE
    opts = fespmv_options(format, reorder, sigma, threshold, vec, csr_lanes, precisions, block, tiles,
                          node_blocks, col_order)
    mesh = fespmv_mesh_info(dofs_per_node, None if xyz is None else xyz.ctypes.data)
    h = _P()
    n = len(rowptr) - 1
    _check(_lib.spmv_create(ctypes.byref(h), n, _ptr(rowptr), _ptr(colind), _ptr(values),
                            ctypes.byref(mesh), ctypes.byref(opts), _stream(stream)))
    return Matrix(h, n, int(rowptr[-1]))


def status_string(status: int) -> str:
    return _lib.fespmv_status_string(status).decode()


def spmv_destroy(A: Matrix):
    if A.handle:
        _lib.spmv_destroy(A.handle)
        A.handle = None


def spmv_apply(A: Matrix, x, y, flags=0, stream=None):
    if isinstance(x, np.ndarray):
        flags |= FESPMV_IO_HOST
    _check(_lib.spmv_apply(A.handle, _ptr(x), _ptr(y), flags, _stream(stream)))
    return y


def spmv_apply_scaled(A: Matrix, x, y, precision=FESPMV_PREC_F32, flags=0, stream=None):
    _check(_lib.spmv_apply_scaled(A.handle, _ptr(x), _ptr(y), precision, flags, _stream(stream)))
    return y


def spmv_apply_multi(A: Matrix, X, Y, precision=FESPMV_PREC_F64, flags=0, stream=None):
    """Y = A X for X of shape (n_rows, k), k <= 32 (torch CUDA tensors)."""
    k = X.shape[1] if X.dim() == 2 else 1
    _check(_lib.spmv_apply_multi(A.handle, _ptr(X), _ptr(Y), k, precision, flags, _stream(stream)))
    return Y


def spmv_permute(A: Matrix, x, out, direction=0, stream=None):
    _check(_lib.spmv_permute(A.handle, _ptr(x), _ptr(out), direction, _stream(stream)))
    return out


def spmv_update_values(A: Matrix, values, flags=0, stream=None):
    if isinstance(values, np.ndarray):
        values = np.ascontiguousarray(values, dtype=np.float64)
        flags |= FESPMV_IO_HOST
    _check(_lib.spmv_update_values(A.handle, _ptr(values), flags, _stream(stream)))


def spmv_plan(rowptr, colind, node_xyz=None, dofs_per_node=1, reorder=None, sigma=0,
              threshold=0, vec=0, node_blocks=0, col_order=0) -> dict:
    """Host-only planning: returns perm, meta (S x 4), cols and srcmap as numpy arrays."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    xyz = None if node_xyz is None else np.ascontiguousarray(node_xyz, dtype=np.float64)
    if reorder is None:
        reorder = FESPMV_REORDER_MORTON if xyz is not None else FESPMV_REORDER_NONE
    opts = fespmv_options(FESPMV_FMT_SLICED, reorder, sigma, threshold, vec, 0, 0, 0, 0, node_blocks, col_order)
    mesh = fespmv_mesh_info(dofs_per_node, None if xyz is None else xyz.ctypes.data)
    info = fespmv_info()
    n = len(rowptr) - 1
    args = (n, _ptr(rowptr), _ptr(colind), ctypes.byref(mesh), ctypes.byref(opts), ctypes.byref(info))
    _check(_lib.spmv_plan(*args, None, None, None, None))
    perm = np.zeros(max(n, 1), np.int32)
    meta = np.zeros(max(info.n_slices * 4, 1), np.uint32)
    cols = np.zeros(max(info.packed_len, 1), np.int32)
    src = np.zeros(max(info.packed_len, 1), np.int64)
    _check(_lib.spmv_plan(*args, _ptr(perm), _ptr(meta), _ptr(cols), _ptr(src)))
    return dict(perm=perm[:n], meta=meta[:info.n_slices * 4].reshape(-1, 4),
                cols=cols[:info.packed_len], srcmap=src[:info.packed_len])


def spmv_plan_tiles(n_rows, meta, cols):
    """Host-only tiles of a packed layout from spmv_plan: (tiles int32[n, 4], tile
    columns int32, index uint16[packed_len]), or None when a slice is too wide."""
    meta = np.ascontiguousarray(meta, dtype=np.uint32).reshape(-1)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    ns, plen = len(meta) // 4, len(cols)
    tiles = np.zeros(max(4 * ns, 1), np.int32)
    tcols = np.zeros(max(plen, 1), np.int32)
    index = np.zeros(max(plen, 1), np.uint16)
    nt, nc = _i64(0), _i64(0)
    _check(_lib.spmv_plan_tiles(n_rows, ns, _ptr(meta), plen, _ptr(cols), _ptr(tiles), _ptr(tcols),
                                _ptr(index), ctypes.byref(nt), ctypes.byref(nc)))
    if nt.value == 0 and ns > 0:
        return None
    return tiles[:4 * nt.value].reshape(-1, 4), tcols[:nc.value], index[:plen]


def spmv_autotune(rowptr, colind, values, node_xyz=None, dofs_per_node=1, reorder=None, sigma=0,
                  reps=0, tiles=0, precisions=0, stream=None) -> dict:
    """Time candidate layouts (products in FP32/BF16 when precisions names that copy, else
    FP64); returns dict(vec, threshold, block, tiles, sigma, reorder, best_us, tried)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    values = np.ascontiguousarray(values, dtype=np.float64)
    xyz = None if node_xyz is None else np.ascontiguousarray(node_xyz, dtype=np.float64)
    if reorder is None:
        reorder = FESPMV_REORDER_MORTON if xyz is not None else FESPMV_REORDER_NONE
    opts = fespmv_options(FESPMV_FMT_SLICED, reorder, sigma, 0, 0, 0, precisions, 0, tiles)
    mesh = fespmv_mesh_info(dofs_per_node, None if xyz is None else xyz.ctypes.data)
    best = ctypes.c_double(0)
    tried = _i32(0)
    _check(_lib.spmv_autotune(len(rowptr) - 1, _ptr(rowptr), _ptr(colind), _ptr(values), ctypes.byref(mesh),
                              ctypes.byref(opts), reps, ctypes.byref(best), ctypes.byref(tried),
                              _stream(stream)))
    return dict(vec=opts.vec, threshold=opts.threshold, block=opts.block, tiles=opts.tiles, sigma=sigma,
                reorder=reorder, best_us=best.value, tried=tried.value)


def spmv_get_info(A: Matrix) -> dict:
    info = fespmv_info()
    _check(_lib.spmv_get_info(A.handle, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in fespmv_info._fields_}


_EXPORT_DTYPES = {FESPMV_EXPORT_PERM: (np.int32, "n_rows"), FESPMV_EXPORT_META: (np.uint32, "meta"),
                  FESPMV_EXPORT_COLS: (np.int32, "packed_len"),
                  FESPMV_EXPORT_VALUES: (np.float64, "packed_len"),
                  FESPMV_EXPORT_SRCMAP: (np.int64, "packed_len"),
                  FESPMV_EXPORT_DIAG: (np.float64, "n_rows"),
                  FESPMV_EXPORT_VALUES_F32: (np.float32, "packed_len"),
                  FESPMV_EXPORT_VALUES_BF16: (np.uint16, "packed_len"),
                  FESPMV_EXPORT_SCALE: (np.float64, "n_rows"),
                  FESPMV_EXPORT_TILES: (np.int32, "tiles"),
                  FESPMV_EXPORT_NB_META: (np.uint32, "nb_meta"),
                  FESPMV_EXPORT_NB_COLS: (np.int32, "nb_len"),
                  FESPMV_EXPORT_NB_VALUES_F32: (np.float32, "nb_values"),
                  FESPMV_EXPORT_NB_VALUES_BF16: (np.uint16, "nb_values"),
                  FESPMV_EXPORT_NB_MAP: (np.int64, "nb_values"),
                  FESPMV_EXPORT_NB_TILES: (np.int32, "nb_tiles4"),
                  FESPMV_EXPORT_NB_TILE_NODES: (np.int32, "nb_tile_dict_len"),
                  FESPMV_EXPORT_NB_TILE_INDEX: (np.uint16, "nb_len"),
                  FESPMV_EXPORT_TILE_COLS: (np.int32, "tile_dict_len"),
                  FESPMV_EXPORT_TILE_INDEX: (np.uint16, "packed_len")}


def spmv_export(A: Matrix, what: int, stream=None) -> np.ndarray:
    info = spmv_get_info(A)
    dt, key = _EXPORT_DTYPES[what]
    count = {"meta": info["n_slices"] * 4, "tiles": info["n_tiles"] * 4, "nb_meta": info["nb_slices"] * 4,
             "nb_values": info["nb_len"] * 9, "nb_tiles4": info["nb_tiles"] * 4}.get(key) or info.get(key, 0)
    out = np.zeros(max(count, 1), dtype=dt)
    _check(_lib.spmv_export(A.handle, what, _ptr(out), out.nbytes, _stream(stream)))
    out = out[:count]
    return out.reshape(-1, 4) if key in ("meta", "tiles", "nb_meta", "nb_tiles4") else out


def cg_solve(A: Matrix, b, x, tol=1e-10, max_iter=0, precision=FESPMV_CG_F64, flags=0,
             max_restarts=0, check_every=0, max_outer=0, inner_tol=0.0, inner_steps=0, stream=None) -> dict:
    """Solve A x = b; returns the cg_result fields as a dict.

    CG outcomes (converged, not converged, breakdown) are reported in
    result["status"]; argument and CUDA errors raise FespmvError."""
    if isinstance(b, np.ndarray):
        flags |= FESPMV_IO_HOST
    o = cg_options(tol, max_iter, precision, flags, max_restarts, check_every, max_outer, inner_tol,
                   inner_steps)
    r = cg_result()
    rc = _lib.cg_solve(A.handle, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(r), _stream(stream))
    if rc not in (FESPMV_OK, FESPMV_ERR_NOT_CONVERGED, FESPMV_ERR_BREAKDOWN):
        _check(rc)
    return {k: getattr(r, k) for k, _ in cg_result._fields_}


def cg_solve_multi(A: Matrix, B, X, tol=1e-10, max_iter=0, precision=FESPMV_CG_F64, flags=0,
                   max_restarts=0, check_every=0, max_outer=0, inner_tol=0.0, stream=None):
    """Solve A X = B for B of shape (n_rows, k), k <= 32, column by column in lockstep;
    returns (status, list of k per-column result dicts).  numpy arrays are host I/O."""
    if isinstance(B, np.ndarray):
        flags |= FESPMV_IO_HOST
    k = B.shape[1] if B.ndim == 2 else 1
    o = cg_options(tol, max_iter, precision, flags, max_restarts, check_every, max_outer, inner_tol)
    res = (cg_result * k)()
    rc = _lib.cg_solve_multi(A.handle, _ptr(B), _ptr(X), k, ctypes.byref(o), ctypes.cast(res, _P),
                             _stream(stream))
    if rc not in (FESPMV_OK, FESPMV_ERR_NOT_CONVERGED, FESPMV_ERR_BREAKDOWN):
        _check(rc)
    return rc, [{f: getattr(r, f) for f, _ in cg_result._fields_} for r in res]


class Assembly:
    """An element-to-entry map (assembly_create); destroy it with assembly_destroy."""

    def __init__(self, handle, A, n_rows):
        self.handle = handle
        self.A = A              # keeps the matrix handle alive
        self.n_rows = n_rows

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.assembly_destroy(self.handle)
            self.handle = None


def assembly_create(A: Matrix, rowptr, colind, elem_nodes, dofs_per_node=1, dirichlet=None,
                    stream=None) -> Assembly:
    """elem_nodes: (n_elems, nodes_per_elem) int array of input node numbers."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    en = np.ascontiguousarray(elem_nodes, dtype=np.int32)
    mk = None if dirichlet is None else np.ascontiguousarray(dirichlet, dtype=np.uint8)
    h = _P()
    _check(_lib.assembly_create(ctypes.byref(h), A.handle, _ptr(rowptr), _ptr(colind), en.shape[0],
                                en.shape[1] if en.ndim == 2 else 1, dofs_per_node, _ptr(en), _ptr(mk),
                                _stream(stream)))
    return Assembly(h, A, A.n_rows)


def assembly_destroy(P: Assembly):
    if P.handle:
        _lib.assembly_destroy(P.handle)
        P.handle = None


def assembly_matrix(P: Assembly, elem_mats, flags=0, stream=None):
    """A's values from element matrices (torch CUDA tensor, or numpy for host I/O)."""
    if isinstance(elem_mats, np.ndarray):
        elem_mats = np.ascontiguousarray(elem_mats, dtype=np.float64)
        flags |= FESPMV_IO_HOST
    _check(_lib.assembly_matrix(P.handle, _ptr(elem_mats), flags, _stream(stream)))


def assembly_vector(P: Assembly, elem_vecs, r, flags=0, stream=None):
    _check(_lib.assembly_vector(P.handle, _ptr(elem_vecs), _ptr(r), flags, _stream(stream)))
    return r


def _newton_dict(r):
    out = {f: getattr(r, f) for f, _ in fe_newton_result._fields_ if f != "last_cg"}
    out["last_cg"] = {f: getattr(r.last_cg, f) for f, _ in cg_result._fields_}
    return out


def fe_newton_step(P: Assembly, elem_mats, elem_vecs, R, dx, phi=None, tol=1e-10, max_iter=0,
                   precision=FESPMV_CG_F64, flags=0, max_restarts=0, check_every=0, max_outer=0,
                   inner_tol=0.0, stream=None) -> dict:
    """One Newton update (Sec. 2): R and K assembled from the element quantities,
    K dx = R solved by CG, phi -= dx.  All arrays are torch CUDA tensors (input
    numbering).  Solve outcomes are in result["status"]; other errors raise."""
    o = cg_options(tol, max_iter, precision, flags, max_restarts, check_every, max_outer, inner_tol)
    r = fe_newton_result()
    rc = _lib.fe_newton_step(P.handle, _ptr(elem_mats), _ptr(elem_vecs), _ptr(R), _ptr(dx), _ptr(phi),
                             ctypes.byref(o), ctypes.byref(r), _stream(stream))
    if rc not in (FESPMV_OK, FESPMV_ERR_NOT_CONVERGED, FESPMV_ERR_BREAKDOWN):
        _check(rc)
    return _newton_dict(r)


def fe_newton_solve(P: Assembly, phi, element_fn, Ke, Re, R, dx, newton_tol=1e-8, max_steps=20,
                    tol=1e-10, max_iter=0, precision=FESPMV_CG_F64, flags=0, max_restarts=0,
                    check_every=0, max_outer=0, inner_tol=0.0, stream=None) -> dict:
    """Newton's loop of Sec. 2 for one time step.  element_fn(phi, Ke, Re) fills the
    element tangents Ke and residuals Re (torch CUDA tensors, written in place) for
    the current phi; it is called from the library, on the calling thread."""
    def cb(phi_p, ke_p, re_p, user, stream_p):
        try:
            element_fn(phi, Ke, Re)
            return 0
        except Exception:   # a failing callback stops the loop with an error
            import traceback
            traceback.print_exc()
            return 1
    fn = FE_ELEMENT_FN(cb)
    o = cg_options(tol, max_iter, precision, flags, max_restarts, check_every, max_outer, inner_tol)
    r = fe_newton_result()
    rc = _lib.fe_newton_solve(P.handle, _ptr(phi), fn, None, _ptr(Ke), _ptr(Re), _ptr(R), _ptr(dx),
                              float(newton_tol), int(max_steps), ctypes.byref(o), ctypes.byref(r),
                              _stream(stream))
    if rc not in (FESPMV_OK, FESPMV_ERR_NOT_CONVERGED, FESPMV_ERR_BREAKDOWN):
        _check(rc)
    return _newton_dict(r)


def assembly_get_info(P: Assembly) -> dict:
    nc, nb = _i64(), _i64()
    _check(_lib.assembly_get_info(P.handle, ctypes.byref(nc), ctypes.byref(nb)))
    return {"contributions": nc.value, "device_bytes": nb.value}


class Server:
    """A solve server (srv_create); destroy it with srv_destroy."""

    def __init__(self, handle, sizes):
        self.handle = handle
        self.sizes = sizes          # matrix id -> n_rows

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.srv_destroy(self.handle)
            self.handle = None


def srv_create(workspace_budget_bytes: int, max_active: int) -> Server:
    h = _P()
    _check(_lib.srv_create(ctypes.byref(h), workspace_budget_bytes, max_active))
    return Server(h, {})


def srv_set_grouping(S: Server, width: int):
    """Solve requests on one matrix together in lockstep groups (0 off, 4/8/16/32, -1 by size)."""
    _check(_lib.srv_set_grouping(S.handle, width))


def srv_register(S: Server, A: Matrix) -> int:
    mid = _i32()
    _check(_lib.srv_register(S.handle, A.handle, ctypes.byref(mid)))
    S.sizes[mid.value] = A.n_rows
    return mid.value


def srv_submit(S: Server, matrix_id: int, b, tol=1e-10, max_iter=0, precision=FESPMV_CG_F64,
               flags=0, max_restarts=0, check_every=0, max_outer=0, inner_tol=0.0) -> int:
    b = np.ascontiguousarray(b, dtype=np.float64)
    o = cg_options(tol, max_iter, precision, flags, max_restarts, check_every, max_outer, inner_tol)
    t = _i64()
    _check(_lib.srv_submit(S.handle, matrix_id, _ptr(b), ctypes.byref(o), ctypes.byref(t)))
    return t.value


def srv_poll(S: Server, ticket: int, n_rows: int, wait=True):
    """Returns None while pending (wait=False), else (status, x, result dict, timing dict).
    n_rows = 0 skips copying x."""
    x = np.zeros(max(n_rows, 1)) if n_rows > 0 else None
    r = cg_result()
    tm = srv_timing()
    rc = _lib.srv_poll(S.handle, ticket, 1 if wait else 0, _ptr(x) if x is not None else None,
                       ctypes.byref(r), ctypes.byref(tm))
    if rc == FESPMV_PENDING:
        return None
    if rc not in (FESPMV_OK, FESPMV_ERR_NOT_CONVERGED, FESPMV_ERR_BREAKDOWN, FESPMV_ERR_CANCELLED):
        _check(rc)
    return (rc, x[:n_rows] if x is not None else None, {k: getattr(r, k) for k, _ in cg_result._fields_},
            {k: getattr(tm, k) for k, _ in srv_timing._fields_})


def srv_get_stats(S: Server) -> dict:
    st = srv_stats()
    _check(_lib.srv_get_stats(S.handle, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in srv_stats._fields_}


def srv_cancel_queued(S: Server) -> int:
    n = _i64()
    _check(_lib.srv_cancel_queued(S.handle, ctypes.byref(n)))
    return n.value


def srv_destroy(S: Server):
    if S.handle:
        _lib.srv_destroy(S.handle)
        S.handle = None


class Batch:
    """A batch handle (batch_create); destroy with batch_destroy."""

    def __init__(self, handle, n_rows):
        self.handle = handle
        self.n_rows = list(n_rows)
        self.offsets = np.concatenate([[0], np.cumsum(self.n_rows)]).astype(np.int64)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.batch_destroy(self.handle)
            self.handle = None


def batch_create(problems, sigma=0, threshold=0, vec=0, precisions=0, block=0, reorder=None,
                 stream=None) -> Batch:
    """problems: sequence of (rowptr, colind, values, node_xyz or None, dofs_per_node)."""
    keep = []
    n = len(problems)
    n_rows = np.array([len(p[0]) - 1 for p in problems], dtype=np.int64)
    rp = (_P * n)()
    ci = (_P * n)()
    va = (_P * n)()
    mesh = (fespmv_mesh_info * n)()
    any_xyz = False
    for j, (r, c, v, xyz, dpn) in enumerate(problems):
        r = np.ascontiguousarray(r, dtype=np.int64)
        c = np.ascontiguousarray(c, dtype=np.int32)
        v = np.ascontiguousarray(v, dtype=np.float64)
        keep += [r, c, v]
        rp[j], ci[j], va[j] = r.ctypes.data, c.ctypes.data, v.ctypes.data
        if xyz is not None:
            xyz = np.ascontiguousarray(xyz, dtype=np.float64)
            keep.append(xyz)
            any_xyz = True
        mesh[j] = fespmv_mesh_info(dpn, None if xyz is None else xyz.ctypes.data)
    if reorder is None:
        reorder = FESPMV_REORDER_MORTON if any_xyz else FESPMV_REORDER_NONE
    opts = fespmv_options(FESPMV_FMT_SLICED, reorder, sigma, threshold, vec, 0, precisions, block, 0)
    h = _P()
    _check(_lib.batch_create(ctypes.byref(h), n, _ptr(n_rows), ctypes.cast(rp, _P),
                             ctypes.cast(ci, _P), ctypes.cast(va, _P), ctypes.cast(mesh, _P),
                             ctypes.byref(opts), _stream(stream)))
    return Batch(h, n_rows)


def batch_destroy(B: Batch):
    if B.handle:
        _lib.batch_destroy(B.handle)
        B.handle = None


def batch_spmv(B: Batch, x, y, stream=None):
    _check(_lib.batch_spmv(B.handle, _ptr(x), _ptr(y), _stream(stream)))
    return y


def batch_cg_solve(B: Batch, b, x, tol=1e-10, max_iter=0, precision=FESPMV_CG_F32_REFINE, flags=0,
                   check_every=0, max_outer=0, inner_tol=0.0, stream=None):
    """Returns (status, list of per-problem result dicts)."""
    if isinstance(b, np.ndarray):
        flags |= FESPMV_IO_HOST
    o = cg_options(tol, max_iter, precision, flags, 0, check_every, max_outer, inner_tol)
    res = (cg_result * len(B.n_rows))()
    rc = _lib.batch_cg_solve(B.handle, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.cast(res, _P),
                             _stream(stream))
    if rc not in (FESPMV_OK, FESPMV_ERR_NOT_CONVERGED, FESPMV_ERR_BREAKDOWN):
        _check(rc)
    return rc, [{k: getattr(r, k) for k, _ in cg_result._fields_} for r in res]


def batch_get_info(B: Batch) -> dict:
    info = fespmv_info()
    pad = _i64()
    _check(_lib.batch_get_info(B.handle, ctypes.byref(info), ctypes.byref(pad)))
    d = {k: getattr(info, k) for k, _ in fespmv_info._fields_}
    d["padded_rows"] = pad.value
    return d
