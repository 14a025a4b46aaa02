"""Batches of independent FE problems (block-diagonal SLICED handle) on the GPU.

Every problem's product is checked against the oracle with the componentwise
FP64 bound of the single-matrix tests (1e-12 * (|A||x|)_i); every problem's
refined solve must meet the tolerance on its true residual (recomputed by the
oracle) and agree with the oracle's FP64 PCG solution within cond(A) * 2e-10.
"""
import numpy as np
import pytest

import fegen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_00324_gb300 as fs  # noqa: E402


def mixed_problems():
    return [fegen.cube_laplace(3, 90), fegen.cube_laplace(9, 91), fegen.cube_elasticity(5, 92),
            fegen.shell_laplace(4, 10, 16, 93), fegen.cube_laplace(13, 94), fegen.cube_laplace(4, 95),
            fegen.cube_elasticity(7, 96), fegen.shell_laplace(3, 6, 9, 97)]


def as_batch(ps, **kw):
    return fs.batch_create([(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node) for p in ps],
                           **kw)


@pytest.mark.parametrize("kw", [dict(sigma=256), dict(sigma=64, threshold=4, vec=1), dict(vec=4)])
def test_batch_spmv_parity(kw):
    ps = mixed_problems()
    B = as_batch(ps, **kw)
    xs = [fegen.random_vector(p.n_rows, 100 + j) for j, p in enumerate(ps)]
    xd = torch.from_numpy(np.concatenate(xs)).cuda()
    yd = torch.full_like(xd, float("nan"))
    fs.batch_spmv(B, xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    for j, p in enumerate(ps):
        yj = y[B.offsets[j]:B.offsets[j + 1]]
        yo = oracle.csr_spmv(p.rowptr, p.colind, p.values, xs[j])
        bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(p.values), np.abs(xs[j]))
        assert np.all(np.abs(yj - yo) <= 1e-12 * bound)
    info = fs.batch_get_info(B)
    assert info["n_rows"] == sum(p.n_rows for p in ps) and info["padded_rows"] % 32 == 0


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_batch_refined_cg(storage):
    ps = mixed_problems()
    prec = fs.FESPMV_PREC_F32 | fs.FESPMV_PREC_BF16
    B = as_batch(ps, sigma=256, precisions=prec)
    us = [fegen.manufactured_solution(p) for p in ps]
    bs = [oracle.csr_spmv(p.rowptr, p.colind, p.values, u) for p, u in zip(ps, us)]
    b = np.concatenate(bs)
    x = np.zeros_like(b)
    cgp = fs.FESPMV_CG_F32_REFINE if storage == "f32" else fs.FESPMV_CG_BF16_REFINE
    rc, res = fs.batch_cg_solve(B, b, x, tol=1e-10, precision=cgp)   # host vectors
    from test_oracle_pins import dense_of
    for j, p in enumerate(ps):
        if storage == "bf16":
            # bf16 refinement contracts only when cond(B) * 2^-8 < 1: compare with the oracle's outcome
            _, ir = oracle.refine(p.rowptr, p.colind, p.values, bs[j], tol=1e-10, inner_tol=1e-2,
                                  storage="bf16")
            if ir["status"] != "converged":
                assert res[j]["status"] != 0
                continue
        assert res[j]["status"] == 0, (j, res[j])
        xj = x[B.offsets[j]:B.offsets[j + 1]]
        r = bs[j] - oracle.csr_spmv(p.rowptr, p.colind, p.values, xj)
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bs[j])
        xo, _ = oracle.pcg(p.rowptr, p.colind, p.values, bs[j], tol=1e-12)
        cond = np.linalg.cond(dense_of(p.rowptr, p.colind, p.values, p.n_rows))
        assert np.linalg.norm(xj - xo) <= cond * 2e-10 * np.linalg.norm(xo)
    if storage == "f32":
        assert rc == 0


def test_batch_many_cubes_device_vectors():
    # 64 cubes, node counts log-uniform in [64, 8000]
    rng = np.random.default_rng(98)
    sizes = np.exp(rng.uniform(np.log(64), np.log(8000), size=64))
    ps = [fegen.valid_seed(lambda sd: fegen.cube_laplace(max(3, round(N ** (1 / 3))), sd), 2000 + i)
          for i, N in enumerate(sizes)]
    B = as_batch(ps, sigma=256)
    bs = [fegen.random_vector(p.n_rows, 3000 + j) for j, p in enumerate(ps)]
    bd = torch.from_numpy(np.concatenate(bs)).cuda()
    xd = torch.zeros_like(bd)
    rc, res = fs.batch_cg_solve(B, bd, xd, tol=1e-10)
    torch.cuda.synchronize()
    assert rc == 0
    x = xd.cpu().numpy()
    for j, p in enumerate(ps):
        xj = x[B.offsets[j]:B.offsets[j + 1]]
        r = bs[j] - oracle.csr_spmv(p.rowptr, p.colind, p.values, xj)
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bs[j])
        # the single-problem refined solver takes the same number of refinement steps
        A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=256,
                           precisions=fs.FESPMV_PREC_F32)
        xs = np.zeros(p.n_rows)
        r1 = fs.cg_solve(A, bs[j], xs, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE)
        assert abs(r1["outer"] - res[j]["outer"]) <= 1


def test_batch_rejects_bad_input():
    p = fegen.cube_laplace(4, 99)
    bad = p.colind.copy()
    bad[3] = p.n_rows + 5
    with pytest.raises(fs.FespmvError) as e:
        fs.batch_create([(p.rowptr, p.colind, p.values, None, 1), (p.rowptr, bad, p.values, None, 1)])
    assert e.value.status == fs.FESPMV_ERR_BAD_CSR and "problem 1" in str(e.value)


def test_batch_reliable_updates_match_single_solves():
    """Reliable updates in the batch: every problem meets the tolerance (oracle residual),
    takes about the steps of the oracle's reliable-update solve, and fewer steps than the
    batch's restarted refinement."""
    rng = np.random.default_rng(99)
    sizes = np.exp(rng.uniform(np.log(200), np.log(6000), size=24))
    ps = [fegen.valid_seed(lambda sd: fegen.cube_laplace(max(3, round(N ** (1 / 3))), sd), 4000 + i)
          for i, N in enumerate(sizes)] + [fegen.cube_elasticity(6, 4100), fegen.shell_laplace(4, 12, 16, 4101)]
    B = as_batch(ps, sigma=256)
    bs = [fegen.random_vector(p.n_rows, 5000 + j) for j, p in enumerate(ps)]
    b = np.concatenate(bs)
    x = np.zeros_like(b)
    rc, res = fs.batch_cg_solve(B, b, x, tol=1e-10, flags=fs.FESPMV_CG_RELIABLE)
    assert rc == 0
    x2 = np.zeros_like(b)
    rc2, res2 = fs.batch_cg_solve(B, b, x2, tol=1e-10)
    assert rc2 == 0
    for j, p in enumerate(ps):
        xj = x[B.offsets[j]:B.offsets[j + 1]]
        r = bs[j] - oracle.csr_spmv(p.rowptr, p.colind, p.values, xj)
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bs[j])
        _, io = oracle.refine_reliable(p.rowptr, p.colind, p.values, bs[j], tol=1e-10, delta=0.1)
        assert io["status"] == "converged"
        assert abs(res[j]["iters"] - io["iters"]) <= 0.1 * io["iters"] + 5
    assert sum(r["iters"] for r in res) < sum(r["iters"] for r in res2)


def test_batch_of_tiny_systems():
    """A batch holding 1-, 2- and 33-row problems beside a mesh: products within the
    bound and every problem solved (FP32 refinement, reliable updates, and FP64).
    Morton ordering needs coordinates for every problem, so none is given here."""
    from test_gpu_cg import tridiagonal_problem
    ps = [tridiagonal_problem(1), fegen.cube_laplace(4, 98), tridiagonal_problem(2), tridiagonal_problem(33)]
    B = fs.batch_create([(p.rowptr, p.colind, p.values, None, 1) for p in ps], sigma=256,
                        precisions=fs.FESPMV_PREC_F32)
    xs = [fegen.random_vector(p.n_rows, 110 + j) for j, p in enumerate(ps)]
    xd = torch.from_numpy(np.concatenate(xs)).cuda()
    yd = torch.full_like(xd, float("nan"))
    fs.batch_spmv(B, xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    bs = []
    for j, p in enumerate(ps):
        yo = oracle.csr_spmv(p.rowptr, p.colind, p.values, xs[j])
        bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(p.values), np.abs(xs[j]))
        assert np.all(np.abs(y[B.offsets[j]:B.offsets[j + 1]] - yo) <= 1e-12 * bound)
        bs.append(yo)
    b = np.concatenate(bs)
    for prec, flags in ((fs.FESPMV_CG_F32_REFINE, 0), (fs.FESPMV_CG_F32_REFINE, fs.FESPMV_CG_RELIABLE),
                        (fs.FESPMV_CG_F64, 0)):
        x = np.zeros_like(b)
        rc, res = fs.batch_cg_solve(B, b, x, tol=1e-10, precision=prec, flags=flags)
        assert rc == 0, (prec, flags, res)
        for j, p in enumerate(ps):
            xj = x[B.offsets[j]:B.offsets[j + 1]]
            r = bs[j] - oracle.csr_spmv(p.rowptr, p.colind, p.values, xj)
            assert res[j]["status"] == 0 and np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bs[j]), (prec, flags, j)
