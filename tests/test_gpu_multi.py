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


@pytest.mark.parametrize("k", [1, 7, 32])
@pytest.mark.parametrize("vec", [1, 2, 4])
def test_multi_fp64_parity(k, vec):
    p = fegen.cube_elasticity(7, 110)
    A = handle(p, vec=vec, sigma=128)
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


@pytest.mark.parametrize("permuted", [False, True])
def test_multi_fp32_parity(permuted):
    p = fegen.shell_laplace(5, 16, 30, 112)
    A = handle(p, sigma=256)
    k = 32
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
