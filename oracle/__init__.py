"""CPU oracle for the FE SpMV + CG path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library:
``oracle.c`` holds the FP64 sparse product, Jacobi-PCG and the
mixed-precision refinement; ``layout.py`` holds the numpy definitions of the
row/column permutation and the warp-slice packing.

``oracle.c`` also holds a flexible CG (Notay 2000) preconditioned by a few
steps of low-precision CG on S A S, and assembles global values and vectors from element quantities
(the sum of the element contributions to each entry, Sec. 4).

Pins (tests that tie the oracle to something other than itself) live in
``tests/test_oracle_pins.py``: dense brute-force products, the paper's worked
permutation example (Sec. 5.2/5.3), zero row sums of Neumann Laplacians,
symmetry and positive definiteness, dense direct solves, finite termination of
CG in exact-arithmetic terms, and recovery of manufactured solutions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import layout  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib_handle = None

STATUS = {0: "converged", 1: "not_converged", 2: "breakdown", 3: "bad_input"}


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc -O2 -ffp-contract=off: no fused multiply-add)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.oracle_set_threads.argtypes = [i32]
        lib.oracle_set_threads.restype = None
        lib.oracle_get_threads.argtypes = []
        lib.oracle_get_threads.restype = i32
        lib.oracle_csr_spmv.argtypes = [i64, P, P, P, P, P]
        lib.oracle_csr_spmv.restype = None
        lib.oracle_pcg.argtypes = [i64, P, P, P, P, P, dbl, i32, i32, i32, P, P, P]
        lib.oracle_pcg.restype = i32
        lib.oracle_pcg_single_reduction.argtypes = [i64, P, P, P, P, P, dbl, i32, i32, i32, P, P, P]
        lib.oracle_pcg_single_reduction.restype = i32
        lib.oracle_refine.argtypes = [i64, P, P, P, P, P, dbl, dbl, i32, i32, i32, P, P, P]
        lib.oracle_refine.restype = i32
        lib.oracle_refine_reliable.argtypes = [i64, P, P, P, P, P, dbl, dbl, i32, i32, P, P, P]
        lib.oracle_refine_reliable.restype = i32
        lib.oracle_fcg.argtypes = [i64, P, P, P, P, P, dbl, i32, i32, i32, P, P, P]
        lib.oracle_fcg.restype = i32
        lib.oracle_scaled_values.argtypes = [i64, P, P, P, i32, P]
        lib.oracle_scaled_values.restype = i32
        lib.oracle_csr_spmv_f32.argtypes = [i64, P, P, P, P, P]
        lib.oracle_csr_spmv_f32.restype = None
        lib.oracle_round_bf16.argtypes = [ctypes.c_float]
        lib.oracle_round_bf16.restype = ctypes.c_float
        lib.oracle_assemble_matrix.argtypes = [i64, P, P, i64, i32, i32, P, P, P, P]
        lib.oracle_assemble_matrix.restype = i32
        lib.oracle_assemble_vector.argtypes = [i64, i64, i32, i32, P, P, P, P]
        lib.oracle_assemble_vector.restype = None
        _lib_handle = lib
    return _lib_handle


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(rowptr, colind, values):
    return (np.ascontiguousarray(rowptr, dtype=np.int64),
            np.ascontiguousarray(colind, dtype=np.int32),
            np.ascontiguousarray(values, dtype=np.float64))


def set_threads(threads: int) -> None:
    """Host threads of the product's row loop (default 1).  Every row stays one
    sequential sum, so results do not depend on it; only the CPU-baseline
    timing uses more than one."""
    _lib().oracle_set_threads(int(threads))


def get_threads() -> int:
    return int(_lib().oracle_get_threads())


def csr_spmv(rowptr, colind, values, x) -> np.ndarray:
    """y = A x (FP64, sequential row sums in stored order)."""
    rp, ci, va = _csr(rowptr, colind, values)
    n = len(rp) - 1
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n, dtype=np.float64)
    _lib().oracle_csr_spmv(n, _p(rp), _p(ci), _p(va), _p(x), _p(y))
    return y


def pcg(rowptr, colind, values, b, x0=None, tol=1e-10, max_iter=100000, jacobi=True,
        max_restarts=3, single_reduction=False):
    """Jacobi-PCG; returns (x, info) with info = dict(status, iters, relres, true_relres).
    single_reduction=True runs the one-reduction (Chronopoulos-Gear) arrangement."""
    rp, ci, va = _csr(rowptr, colind, values)
    n = len(rp) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    tr = ctypes.c_double(0)
    fn = _lib().oracle_pcg_single_reduction if single_reduction else _lib().oracle_pcg
    st = fn(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), tol, max_iter,
                           1 if jacobi else 0, max_restarts, ctypes.byref(it), ctypes.byref(rr),
                           ctypes.byref(tr))
    return x, dict(status=STATUS[st], iters=it.value, relres=rr.value, true_relres=tr.value)


def round_bf16(values) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    f = _lib().oracle_round_bf16
    return np.array([f(float(v)) for v in np.asarray(values, dtype=np.float32)],
                    dtype=np.float32)


def scaled_values(rowptr, colind, values, storage="f32") -> np.ndarray:
    """Values of B = S A S (S = diag(A)^-1/2) rounded to float or bfloat16 (as float32)."""
    rp, ci, va = _csr(rowptr, colind, values)
    out = np.empty(len(va), dtype=np.float32)
    st = _lib().oracle_scaled_values(len(rp) - 1, _p(rp), _p(ci), _p(va),
                                     {"f32": 0, "bf16": 1}[storage], _p(out))
    if st != 0:
        raise ValueError("non-positive diagonal")
    return out


def csr_spmv_f32(rowptr, colind, bvalues, x) -> np.ndarray:
    """y = B x with float values, float vector and float left-to-right row sums."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    bv = np.ascontiguousarray(bvalues, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty(len(rp) - 1, dtype=np.float32)
    _lib().oracle_csr_spmv_f32(len(rp) - 1, _p(rp), _p(ci), _p(bv), _p(x), _p(y))
    return y


def refine(rowptr, colind, values, b, x0=None, tol=1e-10, inner_tol=1e-3, max_outer=50,
           max_inner=20000, storage="f32"):
    """FP64 refinement around a float/bfloat16 inner CG on S A S."""
    rp, ci, va = _csr(rowptr, colind, values)
    n = len(rp) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    o = ctypes.c_int(0)
    i = ctypes.c_int(0)
    tr = ctypes.c_double(0)
    st = _lib().oracle_refine(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), tol, inner_tol,
                              max_outer, max_inner, {"f32": 0, "bf16": 1}[storage],
                              ctypes.byref(o), ctypes.byref(i), ctypes.byref(tr))
    return x, dict(status=STATUS[st], outer=o.value, inner=i.value, true_relres=tr.value)


def refine_reliable(rowptr, colind, values, b, x0=None, tol=1e-10, delta=0.1, max_iter=20000,
                    storage="f32"):
    """One float/bfloat16 CG on S A S with FP64 reliable updates (no restarts);
    info: status, updates (residual replacements), iters (CG steps), true_relres."""
    rp, ci, va = _csr(rowptr, colind, values)
    n = len(rp) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    u = ctypes.c_int(0)
    i = ctypes.c_int(0)
    tr = ctypes.c_double(0)
    st = _lib().oracle_refine_reliable(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), tol, delta, max_iter,
                                       {"f32": 0, "bf16": 1}[storage], ctypes.byref(u), ctypes.byref(i),
                                       ctypes.byref(tr))
    return x, dict(status=STATUS[st], updates=u.value, iters=i.value, true_relres=tr.value)


def fcg(rowptr, colind, values, b, tol=1e-10, inner_steps=8, max_iter=20000, storage="bf16"):
    """Flexible CG (one previous direction kept) preconditioned by `inner_steps` steps
    of CG on S A S in float / bfloat16 ('f32', 'bf16') or exact FP64 ('f64');
    info: status, iters (outer steps), inner (inner steps), true_relres."""
    rp, ci, va = _csr(rowptr, colind, values)
    n = len(rp) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n)
    it = ctypes.c_int(0)
    inn = ctypes.c_int(0)
    tr = ctypes.c_double(0)
    st = _lib().oracle_fcg(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), tol, inner_steps, max_iter,
                           {"f32": 0, "bf16": 1, "f64": 2}[storage], ctypes.byref(it), ctypes.byref(inn),
                           ctypes.byref(tr))
    return x, dict(status={0: "converged", 1: "not_converged", 2: "breakdown", 3: "bad_input"}[st],
                   iters=it.value, inner=inn.value, true_relres=tr.value)


def assemble_matrix(rowptr, colind, elem_nodes, elem_mats, dofs_per_node, mask=None) -> np.ndarray:
    """Global values (CSR order of the given pattern) as the sums of the element
    contributions in ascending element order; masked rows are identity rows and
    entries with a masked row or column get no contribution (Sec. 4)."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    en = np.ascontiguousarray(elem_nodes, dtype=np.int32)
    ke = np.ascontiguousarray(elem_mats, dtype=np.float64)
    n = len(rp) - 1
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    out = np.zeros(int(rp[-1]), dtype=np.float64)
    rc = _lib().oracle_assemble_matrix(n, _p(rp), _p(ci), en.shape[0], en.shape[1], dofs_per_node, _p(en),
                                       _p(ke), None if mk is None else _p(mk), _p(out))
    if rc != 0:
        raise ValueError("an element contribution has no stored position in the pattern")
    return out


def assemble_vector(n_rows, elem_nodes, elem_vecs, dofs_per_node, mask=None) -> np.ndarray:
    """Global vector as the sums of the element vectors' entries, ascending element
    order; 0 on masked rows (Sec. 4)."""
    en = np.ascontiguousarray(elem_nodes, dtype=np.int32)
    re = np.ascontiguousarray(elem_vecs, dtype=np.float64)
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    out = np.zeros(n_rows, dtype=np.float64)
    _lib().oracle_assemble_vector(n_rows, en.shape[0], en.shape[1], dofs_per_node, _p(en), _p(re),
                                  None if mk is None else _p(mk), _p(out))
    return out
