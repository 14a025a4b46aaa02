"""The allocation-free CG entry point (cg_solve_csr_static), through the C ABI.

Some callers may not allocate device memory (they run inside another
framework's memory pool, must not grow the process's device footprint, or
cannot block on the allocator).  cg_solve_csr_static serves them with a
workspace held in a fixed device array of the library.  This test checks it
against cg_solve on a CSR handle, on two calls in a row (the second call finds
the first call's leftovers in the shared array), with the tolerance of the
other CG tests: both true residuals at most 1.01e-10 and the two solutions
within cond(A) * 2e-10 of each other.
"""
import ctypes

import numpy as np
import pytest

import fegen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_00324_gb300 as fs  # noqa: E402


def dense_cond(p):
    A = np.zeros((p.n_rows, p.n_rows))
    for i in range(p.n_rows):
        A[i, p.colind[p.rowptr[i]:p.rowptr[i + 1]]] = p.values[p.rowptr[i]:p.rowptr[i + 1]]
    return np.linalg.cond(A)


def static_solve(lib, p, dev_csr, b, lanes, tol):
    rp, ci, va = dev_csr
    bd = torch.from_numpy(b).cuda()
    xd = torch.full_like(bd, 3.0)        # garbage in x: overwritten (no FESPMV_CG_X0)
    opts = fs.cg_options(tol, 0, fs.FESPMV_CG_F64, 0, 0, 0, 0)
    res = fs.cg_result()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.cg_solve_csr_static(ctypes.c_int64(p.n_rows), ctypes.c_void_p(rp.data_ptr()),
                                 ctypes.c_void_p(ci.data_ptr()), ctypes.c_void_p(va.data_ptr()),
                                 ctypes.c_void_p(bd.data_ptr()), ctypes.c_void_p(xd.data_ptr()),
                                 ctypes.c_int32(lanes), ctypes.byref(opts), ctypes.byref(res), stream)
    torch.cuda.synchronize()
    return rc, res, xd.cpu().numpy()


@pytest.mark.parametrize("lanes", [4, 1])
def test_static_cg_matches_cg_solve(lanes):
    lib = ctypes.CDLL(fs.LIB_PATH)
    lib.cg_solve_csr_static.restype = ctypes.c_int
    p = fegen.cube_laplace(12, 61)
    dev_csr = tuple(torch.from_numpy(a).cuda() for a in (p.rowptr, p.colind, p.values))
    A = fs.spmv_create(p.rowptr, p.colind, p.values, format=fs.FESPMV_FMT_CSR, csr_lanes=lanes)
    cond = dense_cond(p)
    for call in range(2):
        b = fegen.random_vector(p.n_rows, 62 + call)
        bd = torch.from_numpy(b).cuda()
        x_ref = torch.zeros_like(bd)
        ref = fs.cg_solve(A, bd, x_ref, tol=1e-10)
        x_ref = x_ref.cpu().numpy()
        rc, res, x = static_solve(lib, p, dev_csr, b, lanes, 1e-10)
        assert rc == 0 and res.status == 0 and ref["status"] == 0
        for xx in (x, x_ref):
            r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, xx)
            assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)
        assert np.linalg.norm(x - x_ref) <= cond * 2e-10 * np.linalg.norm(x_ref)
        assert abs(res.iters - ref["iters"]) <= 0.02 * ref["iters"] + 2


def test_static_cg_rejects_oversize():
    lib = ctypes.CDLL(fs.LIB_PATH)
    opts = fs.cg_options(1e-10, 0, 0, 0, 0, 0, 0)
    rc = lib.cg_solve_csr_static(ctypes.c_int64(262_145), None, None, None, None, None,
                                 ctypes.c_int32(4), ctypes.byref(opts), None, None)
    assert rc == fs.FESPMV_ERR_INVALID_ARG
    assert b"at most 262144 rows" in fs.lib().fespmv_last_error()
