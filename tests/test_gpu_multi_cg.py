"""Lockstep CG for many right-hand sides (cg_solve_multi), checked against the oracle.

Each column is an independent Jacobi-PCG solve of the same matrix, so the
oracle is the single-RHS oracle run once per column.  Pass criteria per column,
as for cg_solve: the true residual ||b - A x|| / ||b||, recomputed by the
oracle, is at most the tolerance (+1 % for the oracle's own rounding); x agrees
with the oracle's PCG solution within cond(A) * 2 tol where cond(A) is small
enough to compute; FP64 iteration counts are within 2 % (+2) of the oracle's.
Columns do not interact: a column's x and iteration count are bitwise the same
whatever the other columns hold, and the same in any column slot.
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


def make(p, **kw):
    kw.setdefault("sigma", 256)
    return fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node,
                          precisions=fs.FESPMV_PREC_F32 | kw.pop("prec", 0), **kw)


def rhs(p, k, seed):
    B = np.stack([fegen.random_vector(p.n_rows, seed + j) for j in range(k)], axis=1)
    B[:, 0] = oracle.csr_spmv(p.rowptr, p.colind, p.values, fegen.manufactured_solution(p))
    return B


def solve(A, B, **kw):
    Bd = dev(B)
    Xd = torch.zeros_like(Bd)
    rc, res = fs.cg_solve_multi(A, Bd, Xd, **kw)
    torch.cuda.synchronize()
    return rc, Xd.cpu().numpy(), res


def true_relres(p, x, b):
    return np.linalg.norm(b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)) / np.linalg.norm(b)


def cond_of(p):
    from test_oracle_pins import dense_of
    return np.linalg.cond(dense_of(p.rowptr, p.colind, p.values, p.n_rows))


PROBLEMS = {"cube_laplace_14": lambda: fegen.cube_laplace(14, 301),
            "elasticity_8": lambda: fegen.cube_elasticity(8, 302),
            "shell_5x16x20": lambda: fegen.shell_laplace(5, 16, 20, 303)}


@pytest.mark.parametrize("k", [1, 5, 17, 32])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_multi_cg_f64_matches_oracle(name, k):
    p = PROBLEMS[name]()
    B = rhs(p, k, 310)
    A = make(p)
    rc, X, res = solve(A, B, tol=1e-10)
    assert rc == fs.FESPMV_OK
    cond = cond_of(p) if p.n_rows <= 3000 else None
    for j in range(k):
        assert res[j]["status"] == 0, (j, res[j])
        assert true_relres(p, X[:, j], B[:, j]) <= 1.01e-10
        xo, info = oracle.pcg(p.rowptr, p.colind, p.values, B[:, j], tol=1e-10)
        assert info["status"] == "converged"
        assert abs(res[j]["iters"] - info["iters"]) <= 0.02 * info["iters"] + 2, (j, res[j], info)
        if cond is not None:
            assert np.linalg.norm(X[:, j] - xo) / np.linalg.norm(xo) <= cond * 2e-10


@pytest.mark.parametrize("variant", ["float_pair_handle", "no_precond"])
def test_multi_cg_f64_variants(variant):
    """FP64 on a handle holding float pairs (its outer residual products use them) and
    FP64 without Jacobi (the oracle's unpreconditioned CG): per column within tolerance,
    iteration counts within 2 % (+2) of the oracle's."""
    p = fegen.cube_elasticity(8, 395)
    B = rhs(p, 6, 396)
    pairs = variant == "float_pair_handle"
    A = make(p, prec=fs.FESPMV_PREC_DF64 if pairs else 0)
    flags = 0 if pairs else fs.FESPMV_CG_NO_PRECOND
    rc, X, res = solve(A, B, tol=1e-10, flags=flags)
    assert rc == fs.FESPMV_OK
    for j in range(6):
        assert res[j]["status"] == 0, (j, res[j])
        assert true_relres(p, X[:, j], B[:, j]) <= 1.01e-10
        _, info = oracle.pcg(p.rowptr, p.colind, p.values, B[:, j], tol=1e-10, jacobi=pairs)
        assert abs(res[j]["iters"] - info["iters"]) <= 0.02 * info["iters"] + 2, (j, res[j], info)


@pytest.mark.parametrize("check_every", [1, 3, 64])
def test_multi_cg_graph_chunks(check_every):
    """Graphs of 1, 3 and 64 inner iterations (outer-step grids of 8, 24 and 512): the
    same per-column convergence; the FP64 recurrence is the same whatever the chunk."""
    p = fegen.cube_laplace(11, 397)
    B = rhs(p, 5, 398)
    A = make(p)
    rc, X, res = solve(A, B, tol=1e-10, check_every=check_every)
    _, X16, res16 = solve(A, B, tol=1e-10)
    assert rc == 0
    for j in range(5):
        assert true_relres(p, X[:, j], B[:, j]) <= 1.01e-10
        assert res[j]["iters"] == res16[j]["iters"]
        assert np.array_equal(X[:, j].view(np.uint64), X16[:, j].view(np.uint64))
    rc, X, res = solve(A, B, tol=1e-10, check_every=check_every, precision=fs.FESPMV_CG_F32_REFINE,
                       flags=fs.FESPMV_CG_RELIABLE)
    assert rc == 0
    for j in range(5):
        assert true_relres(p, X[:, j], B[:, j]) <= 1.01e-10


@pytest.mark.parametrize("reliable", [False, True])
@pytest.mark.parametrize("k", [3, 8, 32])
def test_multi_cg_f32_refinement_reaches_fp64_tolerance(k, reliable):
    p = fegen.cube_elasticity(8, 320)
    B = rhs(p, k, 321)
    A = make(p)
    flags = fs.FESPMV_CG_RELIABLE if reliable else 0
    rc, X, res = solve(A, B, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE, flags=flags)
    assert rc == fs.FESPMV_OK
    cond = cond_of(p)
    for j in range(k):
        assert res[j]["status"] == 0 and res[j]["outer"] >= 1, (j, res[j])
        assert true_relres(p, X[:, j], B[:, j]) <= 1.01e-10
        xo, _ = oracle.pcg(p.rowptr, p.colind, p.values, B[:, j], tol=1e-10)
        assert np.linalg.norm(X[:, j] - xo) / np.linalg.norm(xo) <= cond * 2e-10
        if reliable:   # same bound as the oracle's reliable-update solve
            _, info = oracle.refine_reliable(p.rowptr, p.colind, p.values, B[:, j], tol=1e-10)
            assert res[j]["iters"] <= 1.3 * info["iters"] + 5, (j, res[j], info)


@pytest.mark.parametrize("precision,flags", [(fs.FESPMV_CG_F64, 0),
                                             (fs.FESPMV_CG_F32_REFINE, fs.FESPMV_CG_RELIABLE),
                                             (fs.FESPMV_CG_F32_REFINE, 0)])
def test_multi_cg_columns_are_independent(precision, flags):
    """Bitwise: a column solved beside other right-hand sides, in another slot,
    or beside copies of itself gives the same x and iteration count."""
    p = fegen.cube_laplace(13, 330)
    k = 29                                     # padded width 32 in every call below
    B = np.stack([fegen.random_vector(p.n_rows, 331 + j) for j in range(k)], axis=1)
    A = make(p)
    kw = dict(tol=1e-10, precision=precision, flags=flags)
    _, X1, r1 = solve(A, B, **kw)
    order = np.arange(k)[::-1]
    _, X2, r2 = solve(A, B[:, order], **kw)
    other = np.stack([fegen.random_vector(p.n_rows, 900 + j) for j in range(k)], axis=1)
    other[:, 7] = B[:, 3]
    _, X3, r3 = solve(A, other, **kw)
    for j in range(k):
        jj = int(np.where(order == j)[0][0])
        assert np.array_equal(X1[:, j].view(np.uint64), X2[:, jj].view(np.uint64)), j
        assert r1[j]["iters"] == r2[jj]["iters"]
    assert np.array_equal(X1[:, 3].view(np.uint64), X3[:, 7].view(np.uint64))
    assert r1[3]["iters"] == r3[7]["iters"]
    # repeated solves are bitwise equal
    _, X4, r4 = solve(A, B, **kw)
    assert np.array_equal(X1.view(np.uint64), X4.view(np.uint64))
    assert [r["iters"] for r in r1] == [r["iters"] for r in r4]


def test_multi_cg_column_matches_single_solve():
    """A column of the lockstep FP64 solve and cg_solve of that column take the
    same recurrence: iteration counts within 2 % (+2), both within tolerance."""
    p = fegen.cube_elasticity(9, 340)
    B = rhs(p, 6, 341)
    A = make(p)
    rc, X, res = solve(A, B, tol=1e-10)
    assert rc == 0
    for j in range(6):
        bd = dev(B[:, j])
        xd = torch.zeros_like(bd)
        r1 = fs.cg_solve(A, bd, xd, tol=1e-10)
        assert r1["status"] == 0
        assert abs(res[j]["iters"] - r1["iters"]) <= 0.02 * r1["iters"] + 2


def test_multi_cg_host_io_permuted_and_initial_guess():
    p = fegen.cube_elasticity(7, 350)
    k = 6
    B = rhs(p, k, 351)
    A = make(p)
    # host arrays
    Xh = np.zeros_like(B)
    rc, res = fs.cg_solve_multi(A, B, Xh, tol=1e-10)
    assert rc == 0
    for j in range(k):
        assert true_relres(p, Xh[:, j], B[:, j]) <= 1.01e-10
    # permuted numbering: the same solutions, permuted
    P = fs.spmv_export(A, fs.FESPMV_EXPORT_PERM)
    rc, Xp, res_p = solve(A, B[P], tol=1e-10, flags=fs.FESPMV_IO_PERMUTED)
    assert rc == 0
    Xu = np.empty_like(Xp)
    Xu[P] = Xp
    assert np.array_equal(Xu.view(np.uint64), Xh.view(np.uint64))
    # initial guess: the solution itself needs no iteration; a nearby guess needs fewer
    Bd = dev(B)
    Xd = dev(Xh)
    rc, r0 = fs.cg_solve_multi(A, Bd, Xd, tol=1e-8, flags=fs.FESPMV_CG_X0)
    assert rc == 0 and all(r["iters"] == 0 for r in r0)
    near = Xh + 1e-6 * np.stack([fegen.random_vector(p.n_rows, 360 + j) for j in range(k)], axis=1)
    Xd = dev(near)
    rc, r1 = fs.cg_solve_multi(A, Bd, Xd, tol=1e-10, flags=fs.FESPMV_CG_X0)
    assert rc == 0
    X1 = Xd.cpu().numpy()
    for j in range(k):
        assert r1[j]["iters"] < res[j]["iters"]
        assert true_relres(p, X1[:, j], B[:, j]) <= 1.01e-10


def test_multi_cg_zero_and_duplicate_columns():
    p = fegen.cube_laplace(10, 370)
    B = np.stack([fegen.random_vector(p.n_rows, 371 + j) for j in range(7)], axis=1)
    B[:, 2] = 0.0
    B[:, 5] = B[:, 1]
    A = make(p)
    for precision in (fs.FESPMV_CG_F64, fs.FESPMV_CG_F32_REFINE):
        rc, X, res = solve(A, B, tol=1e-10, precision=precision)
        assert rc == 0
        assert np.all(X[:, 2] == 0.0) and res[2]["iters"] == 0 and res[2]["relres"] == 0.0
        assert np.array_equal(X[:, 5].view(np.uint64), X[:, 1].view(np.uint64))
        assert res[5]["iters"] == res[1]["iters"]


def test_multi_cg_rejects_bad_arguments_and_reports_limits():
    p = fegen.cube_laplace(8, 380)
    A = make(p)
    B = dev(np.ones((p.n_rows, 33)))
    with pytest.raises(fs.FespmvError) as e:
        fs.cg_solve_multi(A, B, B.clone())
    assert e.value.status == fs.FESPMV_ERR_INVALID_ARG
    B4 = dev(np.ones((p.n_rows, 4)))
    for kw, code in ((dict(precision=fs.FESPMV_CG_BF16_REFINE), fs.FESPMV_ERR_UNSUPPORTED),
                     (dict(flags=fs.FESPMV_CG_SINGLE_REDUCTION), fs.FESPMV_ERR_UNSUPPORTED),
                     (dict(flags=fs.FESPMV_CG_RELIABLE), fs.FESPMV_ERR_UNSUPPORTED)):
        with pytest.raises(fs.FespmvError) as e:
            fs.cg_solve_multi(A, B4, B4.clone(), **kw)
        assert e.value.status == code
    K2 = make(p, threshold=2)
    with pytest.raises(fs.FespmvError) as e:
        fs.cg_solve_multi(K2, B4, B4.clone())
    assert e.value.status == fs.FESPMV_ERR_UNSUPPORTED
    F64only = fs.spmv_create(p.rowptr, p.colind, p.values, sigma=64)
    with pytest.raises(fs.FespmvError) as e:
        fs.cg_solve_multi(F64only, B4, B4.clone(), precision=fs.FESPMV_CG_F32_REFINE)
    assert e.value.status == fs.FESPMV_ERR_UNSUPPORTED
    # an iteration limit stops every column with NOT_CONVERGED and that count
    rc, X, res = solve(A, np.ones((p.n_rows, 4)), tol=1e-12, max_iter=5)
    assert rc == fs.FESPMV_ERR_NOT_CONVERGED
    assert all(r["status"] == fs.FESPMV_ERR_NOT_CONVERGED and r["iters"] == 5 for r in res)


def test_multi_cg_non_positive_diagonal_is_breakdown():
    p = fegen.cube_laplace(6, 390)
    vals = p.values.copy()
    rows = np.repeat(np.arange(p.n_rows), np.diff(p.rowptr))
    vals[(rows == 4) & (p.colind == 4)] = -1.0
    A = fs.spmv_create(p.rowptr, p.colind, vals, sigma=64)
    rc, X, res = solve(A, np.ones((p.n_rows, 3)), tol=1e-10)
    assert rc == fs.FESPMV_ERR_BREAKDOWN
    assert all(r["status"] == fs.FESPMV_ERR_BREAKDOWN for r in res)


def test_multi_cg_empty_matrix():
    A = fs.spmv_create(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), sigma=8)
    B = torch.zeros((0, 4), dtype=torch.float64, device="cuda")
    rc, res = fs.cg_solve_multi(A, B, B.clone())
    assert rc == 0 and all(r["iters"] == 0 for r in res)


def test_multi_cg_full_size_elasticity_64_32_rhs():
    """The 64^3 elasticity matrix with 32 right-hand sides, FP32 values with FP64
    reliable updates: every column reaches 1e-10 on the FP64 residual that the
    oracle recomputes (sampled columns)."""
    p = fegen.cube_elasticity(64, 1502)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=1024, vec=4,
                       precisions=fs.FESPMV_PREC_F32)
    k = 32
    B = np.stack([fegen.random_vector(p.n_rows, 1700 + j) for j in range(k)], axis=1)
    rc, X, res = solve(A, B, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE, flags=fs.FESPMV_CG_RELIABLE)
    assert rc == 0
    assert all(r["status"] == 0 and r["true_relres"] <= 1e-10 for r in res)
    for j in (0, 17, 31):
        assert true_relres(p, X[:, j], B[:, j]) <= 1.01e-10


@pytest.mark.parametrize("reliable", [True, False])
def test_multi_cg_on_node_blocks(reliable):
    """The lockstep FP32 solves with their products on 3x3 node blocks: every column
    meets the FP64 tolerance, agrees with the oracle's PCG, stays within the
    reliable-update step bound, and is bitwise independent of the other columns."""
    p = fegen.cube_elasticity(8, 340)
    k = 13
    B = rhs(p, k, 341)
    A = make(p, node_blocks=3)
    assert fs.spmv_get_info(A)["node_blocks"] == 3
    flags = fs.FESPMV_CG_RELIABLE if reliable else 0
    kw = dict(tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE, flags=flags)
    rc, X, res = solve(A, B, **kw)
    assert rc == fs.FESPMV_OK
    cond = cond_of(p)
    for j in range(k):
        assert res[j]["status"] == 0, (j, res[j])
        assert true_relres(p, X[:, j], B[:, j]) <= 1.01e-10
        xo, _ = oracle.pcg(p.rowptr, p.colind, p.values, B[:, j], tol=1e-10)
        assert np.linalg.norm(X[:, j] - xo) / np.linalg.norm(xo) <= cond * 2e-10
        if reliable:
            _, info = oracle.refine_reliable(p.rowptr, p.colind, p.values, B[:, j], tol=1e-10)
            assert res[j]["iters"] <= 1.3 * info["iters"] + 5, (j, res[j], info)
    order = np.arange(k)[::-1]
    _, X2, r2 = solve(A, B[:, order], **kw)
    for j in range(k):
        jj = int(np.where(order == j)[0][0])
        assert np.array_equal(X[:, j].view(np.uint64), X2[:, jj].view(np.uint64)), j
        assert res[j]["iters"] == r2[jj]["iters"]


@pytest.mark.parametrize("n,k", [(1, 1), (1, 32), (2, 3), (33, 32)])
def test_tiny_systems_many_right_hand_sides(n, k):
    """1, 2 and 33 rows with 1, 3 or 32 columns: every column at the oracle's bar in
    FP64 and with FP32 reliable updates (the products of one handle on all columns)."""
    from test_gpu_cg import tridiagonal_problem
    p = tridiagonal_problem(n)
    A = make(p)
    B = np.stack([fegen.random_vector(n, 70 + j) for j in range(k)], axis=1)
    for kw in (dict(tol=1e-10), dict(tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE, flags=fs.FESPMV_CG_RELIABLE)):
        rc, X, res = solve(A, B, **kw)
        assert rc == 0, (kw, res)
        for j in range(k):
            assert res[j]["status"] == 0, (kw, j, res[j])
            assert true_relres(p, X[:, j], B[:, j]) <= 1.01e-10
            if "precision" not in kw:
                _, info = oracle.pcg(p.rowptr, p.colind, p.values, B[:, j], tol=1e-10)
                assert abs(res[j]["iters"] - info["iters"]) <= 0.02 * info["iters"] + 2
