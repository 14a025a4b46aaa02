"""Multi-RHS products Y = A X (k <= 32 columns, one pass over the matrix).

FP64: each column within the componentwise bound of the single-vector tests,
1e-12 * (|A||x|)_i.  FP32 (B = S A S): each column within 2 L 2^-24 (|B||x|)_i
of the oracle's float product (both are float sums of the same products).
"""
import numpy as np
import pytest

import fegen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_00324_gb300 as fs  # noqa: E402


def handle(p, **kw):
    return fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node,
                          precisions=fs.FESPMV_PREC_F32, **kw)


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("k", [1, 3, 4, 7, 8, 16, 17, 32])
@pytest.mark.parametrize("vec", [1, 2, 4])
def test_multi_fp64_parity(k, vec, pairs):
    """FP64 products by DFMA, or (handles with FESPMV_PREC_DF64) by float pairs on the
    FP32 pipe: both within the FP64 bound."""
    p = fegen.cube_elasticity(7, 110)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node, vec=vec, sigma=128,
                       precisions=fs.FESPMV_PREC_F32 | (fs.FESPMV_PREC_DF64 if pairs else 0))
    X = np.stack([fegen.random_vector(p.n_rows, 111 + j) for j in range(k)], axis=1)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Yd = torch.full_like(Xd, float("nan"))
    fs.spmv_apply_multi(A, Xd, Yd, fs.FESPMV_PREC_F64)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy()
    for j in range(k):
        yo = oracle.csr_spmv(p.rowptr, p.colind, p.values, X[:, j])
        bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(p.values), np.abs(X[:, j]))
        assert np.all(np.abs(Y[:, j] - yo) <= 1e-12 * bound)


def check_f32(p, X, Y):
    bv = oracle.scaled_values(p.rowptr, p.colind, p.values, "f32")
    L = np.diff(p.rowptr).max()
    for j in range(X.shape[1]):
        yo = oracle.csr_spmv_f32(p.rowptr, p.colind, bv, X[:, j])
        bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(bv).astype(np.float64),
                                np.abs(X[:, j]).astype(np.float64))
        assert np.all(np.abs(Y[:, j].astype(np.float64) - yo) <= 2 * L * 2.0 ** -24 * bound)


@pytest.mark.parametrize("k", [5, 12, 32])
@pytest.mark.parametrize("vec", [1, 2, 4])
@pytest.mark.parametrize("permuted", [False, True])
def test_multi_fp32_parity(permuted, vec, k):
    p = fegen.shell_laplace(5, 16, 30, 112)
    A = handle(p, sigma=256, vec=vec)
    X = np.stack([fegen.random_vector(p.n_rows, 113 + j) for j in range(k)], axis=1).astype(np.float32)
    if permuted:
        P = fs.spmv_export(A, fs.FESPMV_EXPORT_PERM)
        Xd = torch.from_numpy(np.ascontiguousarray(X[P])).cuda()
    else:
        Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Yd = torch.full_like(Xd, float("nan"))
    fs.spmv_apply_multi(A, Xd, Yd, fs.FESPMV_PREC_F32, fs.FESPMV_IO_PERMUTED if permuted else 0)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy()
    if permuted:
        Yu = np.empty_like(Y)
        Yu[P] = Y
        Y = Yu
    check_f32(p, X, Y)


def test_multi_rejects_k2_layout_and_bad_k():
    p = fegen.cube_laplace(6, 114)
    A = handle(p, threshold=2)
    X = torch.zeros((p.n_rows, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(fs.FespmvError) as e:
        fs.spmv_apply_multi(A, X, X.clone())
    assert e.value.status == fs.FESPMV_ERR_UNSUPPORTED
    B = handle(p)
    X33 = torch.zeros((p.n_rows, 33), dtype=torch.float64, device="cuda")
    with pytest.raises(fs.FespmvError):
        fs.spmv_apply_multi(B, X33, X33.clone())


def test_multi_fp32_full_size_elasticity_64():
    p = fegen.cube_elasticity(64, 1502)
    A = handle(p, sigma=1024)
    k = 32
    X = np.stack([fegen.random_vector(p.n_rows, 1600 + j) for j in range(k)], axis=1).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Yd = torch.empty_like(Xd)
    fs.spmv_apply_multi(A, Xd, Yd, fs.FESPMV_PREC_F32)
    torch.cuda.synchronize()
    check_f32(p, X[:, [0, 13, 31]], Yd.cpu().numpy()[:, [0, 13, 31]])


@pytest.mark.parametrize("prec", [fs.FESPMV_PREC_F64, fs.FESPMV_PREC_F32])
def test_multi_nan_ragged_rows_and_unaligned_buffers(prec):
    """Padding entries never touch X: a NaN in row c of X poisons exactly the
    rows that store column c (in that column of Y only); empty rows (FP64) give 0;
    buffers that are not 16-byte aligned (views offset by one row of k = 5)
    take the staging path, in both numberings."""
    n = 37
    rng = np.random.default_rng(5)
    lens = np.array([0 if i % 7 == 0 else 1 + i % 5 for i in range(n)])
    lens[3] = n
    rows = [np.sort(rng.choice(n, lens[i], replace=False)) for i in range(n)]
    if prec == fs.FESPMV_PREC_F32:   # the FP32 copy of S A S needs a positive diagonal in every row
        rows = [np.union1d(r, [i]) for i, r in enumerate(rows)]
        lens = np.array([len(r) for r in rows])
    rowptr = np.concatenate([[0], np.cumsum(lens)])
    cols = np.concatenate(rows).astype(np.int32)
    vals = rng.uniform(0.5, 2.0, len(cols))
    A = fs.spmv_create(rowptr, cols, vals, precisions=fs.FESPMV_PREC_F64 | prec, sigma=8, vec=2)
    P = fs.spmv_export(A, fs.FESPMV_EXPORT_PERM)
    k = 5
    dt = torch.float64 if prec == fs.FESPMV_PREC_F64 else torch.float32
    X = np.stack([fegen.random_vector(n, 120 + j) for j in range(k)], axis=1)
    X[11, 2] = np.nan
    for flags in (0, fs.FESPMV_IO_PERMUTED):
        Xin = X[P] if flags else X
        big = torch.zeros(n + 1, k, dtype=dt, device="cuda")
        big[1:] = torch.from_numpy(np.ascontiguousarray(Xin)).to(dt)
        Ybig = torch.full((n + 1, k), 7.0, dtype=dt, device="cuda")
        fs.spmv_apply_multi(A, big[1:], Ybig[1:], prec, flags)
        torch.cuda.synchronize()
        assert Ybig[0].eq(7.0).all().item()
        Y = Ybig[1:].double().cpu().numpy()
        if flags:
            Yu = np.empty_like(Y)
            Yu[P] = Y
            Y = Yu
        for j in range(k):
            yo = oracle.csr_spmv(rowptr, cols, vals, X[:, j])
            assert np.array_equal(np.isnan(Y[:, j]), np.isnan(yo))
            assert np.all(Y[lens == 0, j] == 0.0)
            if prec == fs.FESPMV_PREC_F64 and j != 2:
                bound = oracle.csr_spmv(rowptr, cols, np.abs(vals), np.abs(X[:, j]))
                assert np.all(np.abs(Y[:, j] - yo) <= 1e-12 * bound)


@pytest.mark.parametrize("per_row", [4, 20, 40])
def test_multi_fp32_random_sparse_rows(per_row):
    """Random sparse rows of 4, 20 and 40 entries: slices whose rows share no
    columns (no row-to-row reuse), with many distinct columns per slice."""
    n = 4096
    rng = np.random.default_rng(per_row)
    rows = [np.union1d(rng.choice(n, per_row, replace=False), [i]) for i in range(n)]
    rowptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])])
    cols = np.concatenate(rows).astype(np.int32)
    vals = rng.uniform(-1.0, 1.0, len(cols))
    vals[cols == np.repeat(np.arange(n), np.diff(rowptr))] = 2.0 * per_row

    class Q:
        pass
    q = Q()
    q.rowptr, q.colind, q.values = rowptr, cols, vals
    for vec in (1, 2, 4):
        A = fs.spmv_create(rowptr, cols, vals, precisions=fs.FESPMV_PREC_F32, sigma=64, vec=vec)
        for k in (3, 32):
            X = np.stack([fegen.random_vector(n, 130 + j) for j in range(k)], axis=1).astype(np.float32)
            Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
            Yd = torch.full_like(Xd, float("nan"))
            fs.spmv_apply_multi(A, Xd, Yd, fs.FESPMV_PREC_F32)
            torch.cuda.synchronize()
            check_f32(q, X, Yd.cpu().numpy())


def test_multi_float_pairs_out_of_range_and_nan():
    """Entries of A or X outside the float pairs' range, and NaN, take the FP64 path."""
    p = fegen.cube_elasticity(7, 140)
    rng = np.random.default_rng(141)
    vals = p.values.copy()
    idx = rng.choice(p.nnz, 30, replace=False)
    vals[idx[:15]] *= 1e-30
    vals[idx[15:]] *= 1e30
    A = fs.spmv_create(p.rowptr, p.colind, vals, p.node_xyz, 3, sigma=128, precisions=fs.FESPMV_PREC_DF64)
    k = 8
    X = np.stack([fegen.random_vector(p.n_rows, 142 + j) for j in range(k)], axis=1)
    X[rng.choice(p.n_rows, 20, replace=False), 3] *= 1e200
    X[rng.choice(p.n_rows, 20, replace=False), 5] *= 1e-200
    X[9, 6] = np.nan
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Yd = torch.full_like(Xd, float("nan"))
    fs.spmv_apply_multi(A, Xd, Yd, fs.FESPMV_PREC_F64)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy()
    for j in range(k):
        yo = oracle.csr_spmv(p.rowptr, p.colind, vals, X[:, j])
        assert np.array_equal(np.isnan(Y[:, j]), np.isnan(yo))
        ok = ~np.isnan(yo)
        bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(vals), np.abs(X[:, j]))
        assert np.all(np.abs(Y[ok, j] - yo[ok]) <= 1e-12 * bound[ok])


@pytest.mark.parametrize("n", [1, 33])
def test_multi_tiny_systems(n):
    """1 row and 33 rows (one past a 32-row slice) with 1, 5 and 32 columns: FP64
    within the FP64 bound, FP32 within the float bound of the oracle's product."""
    from test_gpu_cg import tridiagonal_problem
    p = tridiagonal_problem(n)
    A = handle(p, sigma=256)
    for k in (1, 5, 32):
        X = np.stack([fegen.random_vector(n, 120 + j) for j in range(k)], axis=1)
        Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        Yd = torch.full_like(Xd, float("nan"))
        fs.spmv_apply_multi(A, Xd, Yd, fs.FESPMV_PREC_F64)
        X32 = np.ascontiguousarray(X.astype(np.float32))
        X32d = torch.from_numpy(X32).cuda()
        Y32d = torch.full_like(X32d, float("nan"))
        fs.spmv_apply_multi(A, X32d, Y32d, fs.FESPMV_PREC_F32)
        torch.cuda.synchronize()
        Y = Yd.cpu().numpy()
        for j in range(k):
            yo = oracle.csr_spmv(p.rowptr, p.colind, p.values, X[:, j])
            bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(p.values), np.abs(X[:, j]))
            assert np.all(np.abs(Y[:, j] - yo) <= 1e-12 * bound), (k, j)
        check_f32(p, X32, Y32d.cpu().numpy())
