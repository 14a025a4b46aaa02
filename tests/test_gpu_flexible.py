"""Flexible CG with low-precision inner steps (cg_solve with FESPMV_CG_FLEXIBLE).

Checked against oracle.fcg, the same method in plain C: the true residual
(recomputed by the oracle) meets the tolerance, the outer step count is within
10 % + 3 of the oracle's (the inner float arithmetic differs in rounding order
and FMA use), every outer step takes the stated number of inner steps, and x
agrees with the oracle's FP64 PCG solution within cond(A) * 2e-10.  BF16 values,
with which restarted refinement and reliable updates stall on these matrices,
reach 1e-10 here, at full size on the 24 x 256 x 512 shell as well.
"""
import numpy as np
import pytest

import fegen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_00324_gb300 as fs  # noqa: E402

CG = {"f32": fs.FESPMV_CG_F32_REFINE, "bf16": fs.FESPMV_CG_BF16_REFINE}
PREC = fs.FESPMV_PREC_F32 | fs.FESPMV_PREC_BF16


def solve(A, b, **kw):
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    res = fs.cg_solve(A, bd, xd, **kw)
    torch.cuda.synchronize()
    return xd.cpu().numpy(), res


def relres(p, x, b):
    r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("fmt", [dict(sigma=256), dict(sigma=256, tiles=-1),
                                 dict(format=fs.FESPMV_FMT_CSR, csr_lanes=4)])
@pytest.mark.parametrize("storage,m", [("bf16", 8), ("bf16", 3), ("f32", 8)])
@pytest.mark.parametrize("mesh", ["shell_5x16x24", "elasticity_7"])
def test_flexible_cg_matches_oracle(mesh, storage, m, fmt):
    p = {"shell_5x16x24": lambda: fegen.shell_laplace(5, 16, 24, 52),
         "elasticity_7": lambda: fegen.cube_elasticity(7, 81)}[mesh]()
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node, precisions=PREC, **fmt)
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    x, res = solve(A, b, tol=1e-10, precision=CG[storage], flags=fs.FESPMV_CG_FLEXIBLE, inner_steps=m)
    assert res["status"] == 0, res
    assert relres(p, x, b) <= 1.01e-10 and res["true_relres"] <= 1e-10
    _, info = oracle.fcg(p.rowptr, p.colind, p.values, b, tol=1e-10, inner_steps=m, storage=storage)
    assert info["status"] == "converged"
    assert abs(res["iters"] - info["iters"]) <= 0.1 * info["iters"] + 3
    assert res["outer"] == m * res["iters"]            # every outer step takes m inner steps
    xo, _ = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-10)
    from test_oracle_pins import dense_of
    cond = np.linalg.cond(dense_of(p.rowptr, p.colind, p.values, p.n_rows))
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= cond * 2e-10


def test_flexible_cg_warm_start_reproducibility_and_options():
    p = fegen.cube_elasticity(6, 82)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=128, precisions=PREC)
    b = fegen.random_vector(p.n_rows, 83)
    kw = dict(tol=1e-10, precision=fs.FESPMV_CG_BF16_REFINE, flags=fs.FESPMV_CG_FLEXIBLE)
    x1, r1 = solve(A, b, **kw)
    x2, r2 = solve(A, b, **kw)
    assert r1["status"] == 0 and r1["iters"] == r2["iters"]
    assert np.array_equal(x1.view(np.uint64), x2.view(np.uint64))
    # warm start from the solution: converged before any step
    bd = torch.from_numpy(b).cuda()
    xd = torch.from_numpy(x1.copy()).cuda()
    r3 = fs.cg_solve(A, bd, xd, tol=1e-10, precision=fs.FESPMV_CG_BF16_REFINE,
                     flags=fs.FESPMV_CG_FLEXIBLE | fs.FESPMV_CG_X0)
    assert r3["status"] == 0 and r3["iters"] == 0
    # the iteration limit
    _, r4 = solve(A, b, tol=1e-10, max_iter=3, max_restarts=-1, precision=fs.FESPMV_CG_F32_REFINE,
                  flags=fs.FESPMV_CG_FLEXIBLE)
    assert r4["status"] == fs.FESPMV_ERR_NOT_CONVERGED and r4["iters"] == 3
    # unsupported combinations
    for prec, fl in ((fs.FESPMV_CG_F64, fs.FESPMV_CG_FLEXIBLE),
                     (fs.FESPMV_CG_F32_REFINE, fs.FESPMV_CG_FLEXIBLE | fs.FESPMV_CG_RELIABLE)):
        with pytest.raises(fs.FespmvError):
            solve(A, b, precision=prec, flags=fl)
    B = torch.from_numpy(np.stack([b, b], axis=1)).cuda()
    with pytest.raises(fs.FespmvError):
        fs.cg_solve_multi(A, B, torch.zeros_like(B), precision=fs.FESPMV_CG_F32_REFINE,
                          flags=fs.FESPMV_CG_FLEXIBLE)


def test_flexible_bf16_full_size_shell():
    """The 24 x 256 x 512 shell (3.1 M rows) with BF16 values reaches 1e-10."""
    p = fegen.shell_laplace(24, 256, 512, 1503)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=1024, precisions=fs.FESPMV_PREC_BF16)
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    x, res = solve(A, b, tol=1e-10, precision=fs.FESPMV_CG_BF16_REFINE, flags=fs.FESPMV_CG_FLEXIBLE)
    assert res["status"] == 0, res
    assert relres(p, x, b) <= 1.01e-10
