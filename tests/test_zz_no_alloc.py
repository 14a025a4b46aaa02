"""The allocation-free CG entry point (cg_solve_csr_static), through the C ABI.

Some callers may not allocate device memory: they run inside another
framework's memory pool, must not grow the process's device footprint, or
cannot block on the allocator.  cg_solve_csr_static serves them with a
workspace held in a fixed device array of the library.

These tests hold it to the bar of the other CG tests, against the FP64 oracle
(oracle.pcg) and against cg_solve on a CSR handle, on two calls in a row (the
second call finds the first call's leftovers in the shared array):
  - the true residual, recomputed by the oracle, is at most 1.01 * tol;
  - the iteration count is within 2 % (+2) of the oracle's PCG and of cg_solve;
  - x is within cond(A) * 2e-10 of the oracle's and of cg_solve's solution
    (dense condition number on the small mesh; on the 64^3 mesh, at the row
    limit, within 1e-6 of both and of the manufactured solution, as the
    full-size CG tests).
Covered: every lane count near the row limit's largest grid (32 lanes at
262,144 rows fill the partial-sum buffer exactly), a warm start
(FESPMV_CG_X0 from a converged x: at most one step), plain CG
(FESPMV_CG_NO_PRECOND), and rejection of unsupported sizes and flags.
"""
import ctypes

import numpy as np
import pytest

import fegen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_00324_gb300 as fs  # noqa: E402

MAX_ROWS = 262_144


def dense_cond(p):
    A = np.zeros((p.n_rows, p.n_rows))
    for i in range(p.n_rows):
        A[i, p.colind[p.rowptr[i]:p.rowptr[i + 1]]] = p.values[p.rowptr[i]:p.rowptr[i + 1]]
    return np.linalg.cond(A)


def static_lib():
    lib = ctypes.CDLL(fs.LIB_PATH)
    lib.cg_solve_csr_static.restype = ctypes.c_int
    return lib


def static_solve(lib, p, dev_csr, b, lanes, tol=1e-10, flags=0, x0=None):
    rp, ci, va = dev_csr
    bd = torch.from_numpy(b).cuda()
    if x0 is None:
        xd = torch.full_like(bd, 3.0)    # garbage in x: overwritten (no FESPMV_CG_X0)
    else:
        xd = torch.from_numpy(np.array(x0)).cuda()
    opts = fs.cg_options(tol, 0, fs.FESPMV_CG_F64, flags, 0, 0, 0)
    res = fs.cg_result()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.cg_solve_csr_static(ctypes.c_int64(p.n_rows), ctypes.c_void_p(rp.data_ptr()),
                                 ctypes.c_void_p(ci.data_ptr()), ctypes.c_void_p(va.data_ptr()),
                                 ctypes.c_void_p(bd.data_ptr()), ctypes.c_void_p(xd.data_ptr()),
                                 ctypes.c_int32(lanes), ctypes.byref(opts), ctypes.byref(res), stream)
    torch.cuda.synchronize()
    return rc, res, xd.cpu().numpy()


def handle_solve(A, b, flags=0):
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    ref = fs.cg_solve(A, bd, xd, tol=1e-10, flags=flags)
    torch.cuda.synchronize()
    return ref, xd.cpu().numpy()


def relres(p, x, b):
    r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("lanes", [4, 1, 32])
@pytest.mark.parametrize("precond", [True, False])
def test_static_cg_matches_oracle_and_cg_solve(lanes, precond):
    lib = static_lib()
    p = fegen.cube_laplace(12, 61)
    dev_csr = tuple(torch.from_numpy(a).cuda() for a in (p.rowptr, p.colind, p.values))
    A = fs.spmv_create(p.rowptr, p.colind, p.values, format=fs.FESPMV_FMT_CSR, csr_lanes=lanes)
    flags = 0 if precond else fs.FESPMV_CG_NO_PRECOND
    cond = dense_cond(p)
    for call in range(2):
        b = fegen.random_vector(p.n_rows, 62 + call)
        ref, x_ref = handle_solve(A, b, flags)
        xo, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-10, jacobi=precond)
        rc, res, x = static_solve(lib, p, dev_csr, b, lanes, flags=flags)
        assert rc == 0 and res.status == 0 and ref["status"] == 0 and info["status"] == "converged"
        for xx in (x, x_ref):
            assert relres(p, xx, b) <= 1.01e-10
        assert rel(x, xo) <= cond * 2e-10
        assert rel(x, x_ref) <= cond * 2e-10
        assert abs(res.iters - info["iters"]) <= 0.02 * info["iters"] + 2
        assert abs(res.iters - ref["iters"]) <= 0.02 * ref["iters"] + 2


def test_static_cg_warm_start_from_a_solution():
    lib = static_lib()
    p = fegen.cube_laplace(10, 63)
    dev_csr = tuple(torch.from_numpy(a).cuda() for a in (p.rowptr, p.colind, p.values))
    b = fegen.random_vector(p.n_rows, 64)
    rc, res, x = static_solve(lib, p, dev_csr, b, 4)
    assert rc == 0 and res.iters > 10
    for call in range(2):
        rc2, res2, x2 = static_solve(lib, p, dev_csr, b, 4, flags=fs.FESPMV_CG_X0, x0=x)
        assert rc2 == 0 and res2.status == 0
        assert res2.iters <= 1, res2.iters
        assert relres(p, x2, b) <= 1.01e-10
        assert rel(x2, x) <= 1e-9


def test_static_cg_at_the_row_limit_with_32_lanes():
    # 64^3 nodes = 262,144 rows, the largest size accepted; with 32 lanes per row the
    # product's grid (32,768 blocks) fills the static partial-sum buffer exactly
    lib = static_lib()
    p = fegen.cube_laplace(64, 65)
    assert p.n_rows == MAX_ROWS
    dev_csr = tuple(torch.from_numpy(a).cuda() for a in (p.rowptr, p.colind, p.values))
    A = fs.spmv_create(p.rowptr, p.colind, p.values, format=fs.FESPMV_FMT_CSR, csr_lanes=32)
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    xo, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-10)
    assert info["status"] == "converged"
    ref, x_ref = handle_solve(A, b)
    for call in range(2):
        rc, res, x = static_solve(lib, p, dev_csr, b, 32)
        assert rc == 0 and res.status == 0
        assert relres(p, x, b) <= 1.01e-10
        assert abs(res.iters - info["iters"]) <= 0.02 * info["iters"] + 2
        assert abs(res.iters - ref["iters"]) <= 0.02 * ref["iters"] + 2
        assert rel(x, xo) <= 1e-6 and rel(x, x_ref) <= 1e-6 and rel(x, u) <= 1e-6


def test_static_cg_rejects_oversize_and_unsupported_flags():
    lib = static_lib()
    opts = fs.cg_options(1e-10, 0, 0, 0, 0, 0, 0)
    rc = lib.cg_solve_csr_static(ctypes.c_int64(MAX_ROWS + 1), None, None, None, None, None,
                                 ctypes.c_int32(4), ctypes.byref(opts), None, None)
    assert rc == fs.FESPMV_ERR_INVALID_ARG
    assert b"at most 262144 rows" in fs.lib().fespmv_last_error()
    for flags, prec, lanes in ((fs.FESPMV_IO_HOST, 0, 4), (fs.FESPMV_CG_RELIABLE, 0, 4),
                               (0, fs.FESPMV_CG_F32_REFINE, 4), (0, 0, 3)):
        bad = fs.cg_options(1e-10, 0, prec, flags, 0, 0, 0)
        rc = lib.cg_solve_csr_static(ctypes.c_int64(8), None, None, None, None, None,
                                     ctypes.c_int32(lanes), ctypes.byref(bad), None, None)
        assert rc == fs.FESPMV_ERR_INVALID_ARG, (flags, prec, lanes)
