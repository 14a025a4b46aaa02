"""Low-precision copies of B = S A S and the mixed-precision refined CG, on the GPU.

- The FP32 / BF16 values of B are compared bit for bit with the oracle's
  (same formula round((s_i * a_ij) * s_j), IEEE division and square root).
- y = B x in float is compared componentwise with the oracle's float product:
  both are float sums of the same products in different order, so each is
  within L * 2^-24 * (|B||x|)_i of the exact value (L = row length); the test
  allows twice that.
- The refined solve must reach the FP64 tolerance on the true residual
  (recomputed by the oracle) and agree with the oracle's FP64 PCG solution
  within cond(A) * 2e-10.
"""
import numpy as np
import pytest

import fegen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_00324_gb300 as fs  # noqa: E402

PREC = {"f32": fs.FESPMV_PREC_F32, "bf16": fs.FESPMV_PREC_BF16}
CG = {"f32": fs.FESPMV_CG_F32_REFINE, "bf16": fs.FESPMV_CG_BF16_REFINE}


def make(p, prec_bits, **kw):
    return fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node,
                          precisions=prec_bits, **kw)


FORMATS = [dict(format=fs.FESPMV_FMT_SLICED, sigma=256), dict(format=fs.FESPMV_FMT_CSR, csr_lanes=4),
           dict(format=fs.FESPMV_FMT_SLICED, sigma=64, threshold=3, vec=4),
           dict(format=fs.FESPMV_FMT_SLICED, sigma=256, tiles=-1)]


@pytest.mark.parametrize("fmt", range(len(FORMATS)))
def test_scaled_values_bit_exact(fmt):
    p = fegen.cube_elasticity(7, 71)
    A = make(p, fs.FESPMV_PREC_F32 | fs.FESPMV_PREC_BF16, **FORMATS[fmt])
    b32 = oracle.scaled_values(p.rowptr, p.colind, p.values, "f32")
    b16 = oracle.scaled_values(p.rowptr, p.colind, p.values, "bf16")
    g32 = fs.spmv_export(A, fs.FESPMV_EXPORT_VALUES_F32)
    g16 = fs.spmv_export(A, fs.FESPMV_EXPORT_VALUES_BF16)
    if FORMATS[fmt]["format"] == fs.FESPMV_FMT_SLICED:
        src = fs.spmv_export(A, fs.FESPMV_EXPORT_SRCMAP)
        live = src >= 0
        assert np.array_equal(g32[live].view(np.uint32), b32[src[live]].view(np.uint32))
        assert np.array_equal(g16[live], (b16[src[live]].view(np.uint32) >> 16).astype(np.uint16))
        assert not g32[~live].any() and not g16[~live].any()
    else:
        assert np.array_equal(g32.view(np.uint32), b32.view(np.uint32))
        assert np.array_equal(g16, (b16.view(np.uint32) >> 16).astype(np.uint16))


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("fmt", range(len(FORMATS)))
def test_scaled_spmv_parity(storage, fmt):
    p = fegen.shell_laplace(5, 20, 32, 72)
    A = make(p, PREC[storage], **FORMATS[fmt])
    bv = oracle.scaled_values(p.rowptr, p.colind, p.values, storage)
    x = fegen.random_vector(p.n_rows, 73).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    fs.spmv_apply_scaled(A, xd, yd, PREC[storage])
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    yo = oracle.csr_spmv_f32(p.rowptr, p.colind, bv, x)
    bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(bv).astype(np.float64), np.abs(x).astype(np.float64))
    L = np.diff(p.rowptr).max()
    assert np.all(np.abs(y.astype(np.float64) - yo) <= 2 * L * 2.0 ** -24 * bound)


def solve(A, b, **kw):
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    res = fs.cg_solve(A, bd, xd, **kw)
    torch.cuda.synchronize()
    return xd.cpu().numpy(), res


@pytest.mark.parametrize("name", ["cube_laplace_20", "elasticity_8", "shell_5x16x24"])
@pytest.mark.parametrize("fmt", [0, 1])
def test_f32_refinement_reaches_fp64_tolerance(name, fmt):
    p = {"cube_laplace_20": lambda: fegen.cube_laplace(20, 1501),
         "elasticity_8": lambda: fegen.cube_elasticity(8, 74),
         "shell_5x16x24": lambda: fegen.shell_laplace(5, 16, 24, 75)}[name]()
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    A = make(p, fs.FESPMV_PREC_F32, **FORMATS[fmt])
    x, res = solve(A, b, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE)
    assert res["status"] == 0, res
    r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)
    xo, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-12)
    from test_oracle_pins import dense_of
    if p.n_rows <= 3000:
        cond = np.linalg.cond(dense_of(p.rowptr, p.colind, p.values, p.n_rows))
        assert np.linalg.norm(x - xo) <= cond * 2e-10 * np.linalg.norm(xo)
    # the oracle's refinement reaches the same tolerance in a similar number of outer steps
    xr, ir = oracle.refine(p.rowptr, p.colind, p.values, b, tol=1e-10, inner_tol=1e-2)
    assert ir["status"] == "converged"
    assert abs(res["outer"] - ir["outer"]) <= 2


def test_bf16_refinement_small_system_and_stagnation_report():
    p = fegen.cube_laplace(8, 27)
    b = fegen.random_vector(p.n_rows, 28)
    A = make(p, fs.FESPMV_PREC_BF16)
    x, res = solve(A, b, tol=1e-10, precision=fs.FESPMV_CG_BF16_REFINE)
    xr, ir = oracle.refine(p.rowptr, p.colind, p.values, b, tol=1e-10, inner_tol=1e-2,
                           storage="bf16")
    assert ir["status"] == "converged" and res["status"] == 0
    r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)
    # a precision the handle does not hold is refused
    B = make(p, 0)
    with pytest.raises(fs.FespmvError):
        solve(B, b, precision=fs.FESPMV_CG_F32_REFINE)


def test_f32_refinement_full_size_elasticity_64():
    p = fegen.cube_elasticity(64, 1502)
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    A = make(p, fs.FESPMV_PREC_F32, sigma=1024)
    x, res = solve(A, b, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE)
    assert res["status"] == 0, res
    r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)


REL = fs.FESPMV_CG_RELIABLE


@pytest.mark.parametrize("name", ["cube_laplace_20", "elasticity_8", "shell_5x16x24"])
@pytest.mark.parametrize("fmt", [0, 1, 3])
def test_reliable_refinement_matches_oracle(name, fmt):
    """FP32 CG with reliable updates against the oracle's: true residual, solution,
    step and update counts (float sums in another order: counts within 10 % + 5)."""
    p = {"cube_laplace_20": lambda: fegen.cube_laplace(20, 1501),
         "elasticity_8": lambda: fegen.cube_elasticity(8, 74),
         "shell_5x16x24": lambda: fegen.shell_laplace(5, 16, 24, 75)}[name]()
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    A = make(p, fs.FESPMV_PREC_F32, **FORMATS[fmt])
    x, res = solve(A, b, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE, flags=REL, inner_tol=0.1)
    assert res["status"] == 0, res
    r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)
    xo, info = oracle.refine_reliable(p.rowptr, p.colind, p.values, b, tol=1e-10, delta=0.1)
    assert info["status"] == "converged"
    assert abs(res["iters"] - info["iters"]) <= 0.1 * info["iters"] + 5
    assert abs(res["outer"] - info["updates"]) <= 3
    from test_oracle_pins import dense_of
    if p.n_rows <= 3000:
        cond = np.linalg.cond(dense_of(p.rowptr, p.colind, p.values, p.n_rows))
        assert np.linalg.norm(x - xo) <= cond * 2e-10 * np.linalg.norm(xo)
    # fewer steps than restarted refinement on the same system
    _, rr = solve(A, b, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE)
    assert res["iters"] < rr["iters"]


def test_reliable_refinement_limits_and_options():
    p = fegen.cube_laplace(10, 76)
    b = fegen.random_vector(p.n_rows, 77)
    A = make(p, fs.FESPMV_PREC_F32 | fs.FESPMV_PREC_BF16)
    x, res = solve(A, b, tol=1e-12, precision=fs.FESPMV_CG_F32_REFINE, flags=REL, max_iter=7)
    assert res["status"] == fs.FESPMV_ERR_NOT_CONVERGED and res["iters"] == 7
    # the same first 7 steps as the oracle's (no update reached yet at delta = 1e-6)
    x7, res7 = solve(A, b, tol=1e-12, precision=fs.FESPMV_CG_F32_REFINE, flags=REL, max_iter=7,
                     inner_tol=1e-6)
    xo, io = oracle.refine_reliable(p.rowptr, p.colind, p.values, b, tol=1e-12, delta=1e-6, max_iter=7)
    assert io["status"] == "not_converged" and io["updates"] == 0
    assert np.linalg.norm(x7 - xo) <= 1e-5 * np.linalg.norm(xo)
    # BF16 with reliable updates (default delta 0.1) on a small system converges, as the
    # oracle's does; with delta 0.01 both stop without converging (B in bfloat16 is too
    # far from S A S for updates that rare)
    xb, rb = solve(A, b, tol=1e-10, precision=fs.FESPMV_CG_BF16_REFINE, flags=REL)
    _, ob = oracle.refine_reliable(p.rowptr, p.colind, p.values, b, tol=1e-10, delta=0.1, storage="bf16")
    assert rb["status"] == 0 and ob["status"] == "converged"
    _, rb2 = solve(A, b, tol=1e-10, precision=fs.FESPMV_CG_BF16_REFINE, flags=REL, inner_tol=1e-2,
                   max_iter=3000)
    _, ob2 = oracle.refine_reliable(p.rowptr, p.colind, p.values, b, tol=1e-10, delta=1e-2, storage="bf16",
                                    max_iter=3000)
    assert rb2["status"] != 0 and ob2["status"] != "converged"
    # b = 0; FP64 refuses the flag; graph sizes reach the same iterate
    z = torch.zeros(p.n_rows, dtype=torch.float64, device="cuda")
    xz = torch.ones_like(z)
    assert fs.cg_solve(A, z, xz, precision=fs.FESPMV_CG_F32_REFINE, flags=REL)["status"] == 0
    assert not xz.any().item()
    with pytest.raises(fs.FespmvError):
        solve(A, b, precision=fs.FESPMV_CG_F64, flags=REL)
    xs = [solve(A, b, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE, flags=REL, check_every=c)[0]
          for c in (1, 16)]
    assert np.array_equal(xs[0], xs[1])


def test_reliable_refinement_full_size_elasticity_64():
    p = fegen.cube_elasticity(64, 1502)
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    A = make(p, fs.FESPMV_PREC_F32, sigma=1024)
    x, res = solve(A, b, tol=1e-10, precision=fs.FESPMV_CG_F32_REFINE, flags=REL, inner_tol=0.1)
    assert res["status"] == 0, res
    r = b - oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)
