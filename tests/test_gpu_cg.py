"""GPU conjugate gradients through the C ABI, checked against the FP64 oracle.

Pass criteria: the true residual ||b - A x|| / ||b||, recomputed by the oracle
from the GPU's x, is at most the requested tolerance (plus 1 % for the
oracle's own rounding); x agrees with the oracle's PCG solution within
cond(A) * tol (both are tol-accurate solutions of the same system); the
iteration count is within 2 % (+2) of the oracle's, since the two differ only
in rounding order.
"""
import numpy as np
import pytest

import fegen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_00324_gb300 as fs  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def true_relres(p, x, b):
    r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


def solve(A, b, **kw):
    bd = dev(b)
    xd = torch.zeros_like(bd)
    res = fs.cg_solve(A, bd, xd, **kw)
    torch.cuda.synchronize()
    return xd.cpu().numpy(), res


def make(p, **kw):
    return fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node, **kw)


FORMATS = [dict(format=fs.FESPMV_FMT_SLICED, sigma=512), dict(format=fs.FESPMV_FMT_CSR, csr_lanes=4),
           dict(format=fs.FESPMV_FMT_SLICED, sigma=64, threshold=4, vec=1),
           dict(format=fs.FESPMV_FMT_SLICED, sigma=512, precisions=fs.FESPMV_PREC_DF64),
           dict(format=fs.FESPMV_FMT_SLICED, sigma=512, tiles=-1)]


@pytest.mark.parametrize("fmt", range(len(FORMATS)))
@pytest.mark.parametrize("name", ["cube_laplace_20", "elasticity_8", "shell_5x16x24"])
def test_cg_matches_oracle(name, fmt):
    p = {"cube_laplace_20": lambda: fegen.cube_laplace(20, 1501),
         "elasticity_8": lambda: fegen.cube_elasticity(8, 51),
         "shell_5x16x24": lambda: fegen.shell_laplace(5, 16, 24, 52)}[name]()
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    A = make(p, **FORMATS[fmt])
    x, res = solve(A, b, tol=1e-10)
    assert res["status"] == 0, res
    assert true_relres(p, x, b) <= 1.01e-10
    assert res["true_relres"] <= 1e-10
    xo, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-10)
    assert info["status"] == "converged"
    assert abs(res["iters"] - info["iters"]) <= 0.02 * info["iters"] + 2
    # both are 1e-10-residual solutions: their gap is bounded by cond(A) * 2e-10
    from test_oracle_pins import dense_of
    if p.n_rows <= 3000:
        cond = np.linalg.cond(dense_of(p.rowptr, p.colind, p.values, p.n_rows))
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= cond * 2e-10
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-6


def test_cg_is_bitwise_reproducible_and_host_io():
    p = fegen.cube_elasticity(9, 53)
    b = fegen.random_vector(p.n_rows, 54)
    A = make(p, sigma=256)
    x1, r1 = solve(A, b)
    x2, r2 = solve(A, b)
    assert r1["iters"] == r2["iters"] and np.array_equal(x1.view(np.uint64), x2.view(np.uint64))
    xh = np.zeros(p.n_rows)
    r3 = fs.cg_solve(A, b, xh)          # numpy arrays: host I/O through the same entry point
    assert r3["status"] == 0 and np.array_equal(xh.view(np.uint64), x1.view(np.uint64))


def test_cg_options_and_status_codes():
    p = fegen.cube_laplace(10, 55)
    b = fegen.random_vector(p.n_rows, 56)
    A = make(p, sigma=128)
    # iteration limit
    x, res = solve(A, b, tol=1e-12, max_iter=5, max_restarts=-1)
    assert res["status"] == fs.FESPMV_ERR_NOT_CONVERGED and res["iters"] == 5
    # plain CG agrees with the oracle's plain CG
    x, res = solve(A, b, tol=1e-10, flags=fs.FESPMV_CG_NO_PRECOND)
    xo, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-10, jacobi=False)
    assert res["status"] == 0 and abs(res["iters"] - info["iters"]) <= 0.02 * info["iters"] + 2
    # warm start from the solution: converged before the first iteration
    bd = dev(b)
    xd = dev(x)
    res = fs.cg_solve(A, bd, xd, flags=fs.FESPMV_CG_X0)
    assert res["status"] == 0 and res["iters"] == 0
    # b = 0 gives x = 0
    z = torch.zeros(p.n_rows, dtype=torch.float64, device="cuda")
    xd = torch.ones_like(z)
    res = fs.cg_solve(A, z, xd)
    assert res["status"] == 0 and not xd.any().item()
    # every graph size reaches the same iterate
    xs = [solve(A, b, check_every=c)[0] for c in (1, 7, 64)]
    assert all(np.array_equal(xs[0], xi) for xi in xs[1:])


def test_cg_breakdown_on_indefinite_and_bad_diagonal():
    # diag(1, -1): Jacobi rejects the diagonal; plain CG meets p.Ap <= 0
    A = fs.spmv_create(np.array([0, 1, 2]), np.array([0, 1]), np.array([1.0, -1.0]),
                       format=fs.FESPMV_FMT_CSR)
    b = np.array([1.0, 1.0])
    x, res = solve(A, b)
    assert res["status"] == fs.FESPMV_ERR_BREAKDOWN
    x, res = solve(A, b, flags=fs.FESPMV_CG_NO_PRECOND)
    assert res["status"] == fs.FESPMV_ERR_BREAKDOWN


@pytest.mark.parametrize("prec", [0, fs.FESPMV_PREC_DF64])
def test_cg_full_size_elasticity_64(prec):
    """The benchmark system (786,432 rows): residual checked by the oracle's product."""
    p = fegen.cube_elasticity(64, 1502)
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    A = make(p, sigma=1024, precisions=prec)
    x, res = solve(A, b, tol=1e-10)
    assert res["status"] == 0, res
    assert true_relres(p, x, b) <= 1.01e-10
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-5


SR = fs.FESPMV_CG_SINGLE_REDUCTION


@pytest.mark.parametrize("fmt", [0, 1, 3, 4])
@pytest.mark.parametrize("name", ["cube_laplace_20", "elasticity_8", "shell_5x16x24"])
def test_single_reduction_cg_matches_oracle(name, fmt):
    """Chronopoulos-Gear PCG against the oracle's own single-reduction PCG."""
    p = {"cube_laplace_20": lambda: fegen.cube_laplace(20, 1501),
         "elasticity_8": lambda: fegen.cube_elasticity(8, 51),
         "shell_5x16x24": lambda: fegen.shell_laplace(5, 16, 24, 52)}[name]()
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    A = make(p, **FORMATS[fmt])
    x, res = solve(A, b, tol=1e-10, flags=SR)
    assert res["status"] == 0, res
    assert true_relres(p, x, b) <= 1.01e-10
    xo, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-10, single_reduction=True)
    assert info["status"] == "converged"
    assert abs(res["iters"] - info["iters"]) <= 0.02 * info["iters"] + 2
    from test_oracle_pins import dense_of
    if p.n_rows <= 3000:
        cond = np.linalg.cond(dense_of(p.rowptr, p.colind, p.values, p.n_rows))
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= cond * 2e-10
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-6


def test_single_reduction_cg_options_and_status_codes():
    p = fegen.cube_laplace(10, 55)
    b = fegen.random_vector(p.n_rows, 56)
    A = make(p, sigma=128)
    x, res = solve(A, b, tol=1e-12, max_iter=5, max_restarts=-1, flags=SR)
    assert res["status"] == fs.FESPMV_ERR_NOT_CONVERGED and res["iters"] == 5
    # the first 5 iterates agree with the oracle's (same recurrences, different rounding)
    xo, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-12, max_iter=5, single_reduction=True)
    assert info["iters"] == 5
    assert np.linalg.norm(x - xo) <= 1e-11 * np.linalg.norm(xo)
    x, res = solve(A, b, tol=1e-10, flags=SR | fs.FESPMV_CG_NO_PRECOND)
    xo, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-10, jacobi=False, single_reduction=True)
    assert res["status"] == 0 and abs(res["iters"] - info["iters"]) <= 0.02 * info["iters"] + 2
    res = fs.cg_solve(A, dev(b), dev(x), flags=SR | fs.FESPMV_CG_X0)
    assert res["status"] == 0 and res["iters"] == 0
    z = torch.zeros(p.n_rows, dtype=torch.float64, device="cuda")
    xd = torch.ones_like(z)
    assert fs.cg_solve(A, z, xd, flags=SR)["status"] == 0 and not xd.any().item()
    xs = [solve(A, b, check_every=c, flags=SR)[0] for c in (1, 7, 64)]
    assert all(np.array_equal(xs[0], xi) for xi in xs[1:])
    x2, _ = solve(A, b, flags=SR)
    assert np.array_equal(xs[0].view(np.uint64), x2.view(np.uint64))
    # breakdown on an indefinite matrix; refinement precisions reject the flag
    B = fs.spmv_create(np.array([0, 1, 2]), np.array([0, 1]), np.array([1.0, -1.0]),
                       format=fs.FESPMV_FMT_CSR)
    assert solve(B, np.array([1.0, 1.0]), flags=SR | fs.FESPMV_CG_NO_PRECOND)[1]["status"] == \
        fs.FESPMV_ERR_BREAKDOWN
    C = make(p, sigma=128, precisions=fs.FESPMV_PREC_F64 | fs.FESPMV_PREC_F32)
    with pytest.raises(fs.FespmvError):
        solve(C, b, precision=fs.FESPMV_CG_F32_REFINE, flags=SR)


def test_single_reduction_cg_full_size_elasticity_64():
    p = fegen.cube_elasticity(64, 1502)
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    A = make(p, sigma=1024)
    x, res = solve(A, b, tol=1e-10, flags=SR)
    assert res["status"] == 0, res
    assert true_relres(p, x, b) <= 1.01e-10
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-5


@pytest.mark.parametrize("flags", [0, fs.FESPMV_CG_NO_CLUSTER])
@pytest.mark.parametrize("name", ["cube_laplace_20", "elasticity_8"])
def test_small_handles_cluster_and_graph_paths(name, flags):
    """Small handles run reliable-update refinement in one cluster launch unless
    FESPMV_CG_NO_CLUSTER keeps the graphs: both meet the oracle's bar (true residual,
    step and update counts), reproducibly, with a warm start and a step limit; FP64
    PCG (graphs either way) alongside."""
    p = {"cube_laplace_20": lambda: fegen.cube_laplace(20, 1501),
         "elasticity_8": lambda: fegen.cube_elasticity(8, 51)}[name]()
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    A = make(p, sigma=256, precisions=fs.FESPMV_PREC_F32)
    x, res = solve(A, b, tol=1e-10, flags=flags)
    assert res["status"] == 0 and true_relres(p, x, b) <= 1.01e-10
    xo, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-10)
    assert abs(res["iters"] - info["iters"]) <= 0.02 * info["iters"] + 2
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-6
    # repeated solves are bitwise equal
    x2, res2 = solve(A, b, tol=1e-10, flags=flags)
    assert res2["iters"] == res["iters"] and np.array_equal(x.view(np.uint64), x2.view(np.uint64))
    # warm start from the solution: no iteration
    bd, xd = dev(b), dev(x)
    r3 = fs.cg_solve(A, bd, xd, tol=1e-10, flags=flags | fs.FESPMV_CG_X0)
    assert r3["status"] == 0 and r3["iters"] == 0
    # an iteration limit
    _, r4 = solve(A, b, tol=1e-10, max_iter=5, max_restarts=-1, flags=flags)
    assert r4["status"] == fs.FESPMV_ERR_NOT_CONVERGED and r4["iters"] == 5
    # reliable-update refinement
    kw = dict(tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE, flags=flags | fs.FESPMV_CG_RELIABLE)
    xr, rr = solve(A, b, **kw)
    assert rr["status"] == 0 and true_relres(p, xr, b) <= 1.01e-10
    _, ir = oracle.refine_reliable(p.rowptr, p.colind, p.values, b, tol=1e-10)
    assert abs(rr["iters"] - ir["iters"]) <= 0.1 * ir["iters"] + 5
    assert abs(rr["outer"] - ir["updates"]) <= 2
    xr2, rr2 = solve(A, b, **kw)
    assert rr2["iters"] == rr["iters"] and np.array_equal(xr.view(np.uint64), xr2.view(np.uint64))
    r5 = fs.cg_solve(A, bd, dev(xr), **dict(kw, flags=kw["flags"] | fs.FESPMV_CG_X0))
    assert r5["status"] == 0 and r5["iters"] == 0
    _, r6 = solve(A, b, **dict(kw, max_iter=7))
    assert r6["status"] == fs.FESPMV_ERR_NOT_CONVERGED and r6["iters"] <= 7


class TinyProblem:
    """A problem record (the fields the tests read) for matrices that are not meshes."""


def tridiagonal_problem(n):
    """SPD tridiagonal n x n: diagonal 4 + i/n, off-diagonal -1 (eigenvalues in [2, 7])."""
    cols, vals, ends = [], [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                cols.append(j)
                vals.append(4.0 + i / n if j == i else -1.0)
        ends.append(len(cols))
    p = TinyProblem()
    p.rowptr = np.array([0] + ends, dtype=np.int64)
    p.colind = np.array(cols, dtype=np.int32)
    p.values = np.array(vals)
    p.n_rows, p.node_xyz, p.dofs_per_node = n, None, 1
    return p


@pytest.mark.parametrize("n", [1, 2, 31, 33])
def test_tiny_systems_through_every_path(n):
    """1, 2, 31 and 33 rows (one row, a few, one short of a warp's 32-row slice and
    one past it) through every product format and the FP64, single-reduction and
    reliable-update solves: products within the componentwise bound, solves at the
    oracle's bar.  The matrix is SPD tridiagonal, diagonal 4 + i/n, off-diagonal -1."""
    p = tridiagonal_problem(n)
    u = fegen.random_vector(n, 60 + n)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    xo, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-10)
    assert info["status"] == "converged" and info["iters"] <= n
    bound = 1e-12 * oracle.csr_spmv(p.rowptr, p.colind, np.abs(p.values), np.abs(u))
    for kw in FORMATS + [dict(format=fs.FESPMV_FMT_SLICED, sigma=512, precisions=fs.FESPMV_PREC_F32)]:
        A = make(p, **kw)
        yd = torch.empty(n, dtype=torch.float64, device="cuda")
        fs.spmv_apply(A, dev(u), yd)
        assert np.all(np.abs(yd.cpu().numpy() - b) <= bound), kw
        for flags in (0, fs.FESPMV_CG_SINGLE_REDUCTION):
            x, res = solve(A, b, tol=1e-10, flags=flags)
            assert res["status"] == 0, (kw, flags, res)
            assert true_relres(p, x, b) <= 1.01e-10
            assert abs(res["iters"] - info["iters"]) <= 0.02 * info["iters"] + 2
            assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
        if kw.get("precisions") == fs.FESPMV_PREC_F32:
            for flags in (fs.FESPMV_CG_RELIABLE, fs.FESPMV_CG_RELIABLE | fs.FESPMV_CG_NO_CLUSTER):
                x, res = solve(A, b, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE, flags=flags)
                assert res["status"] == 0, (flags, res)
                assert true_relres(p, x, b) <= 1.01e-10
