"""GPU parity of every SpMV kernel against the FP64 oracle, through the C ABI.

Tolerance (componentwise, FP64):  |y_gpu - y_oracle| <= 1e-12 * (|A| |x|)_i.
Both sides compute the exact row sum rounded with different association (the
oracle sums left to right without FMA; the kernels use FMA per lane and a
shuffle tree), so the true gap is a few ulps of (|A||x|)_i; 1e-12 is the
bound the method must meet.  Index work (permutation, packing, value map) is
compared bit for bit.
"""
import numpy as np
import pytest

import fegen
import oracle
from oracle import layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1501_00324_gb300 as fs  # noqa: E402

TOL = 1e-12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_parity(p, y, x, values=None):
    vals = p.values if values is None else values
    yo = oracle.csr_spmv(p.rowptr, p.colind, vals, x)
    bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(vals), np.abs(x))
    err = np.abs(y - yo)
    bad = ~(err <= TOL * bound)
    assert not bad.any(), (f"{bad.sum()} rows off; worst rel "
                           f"{(err / np.maximum(bound, 1e-300)).max():.3e}")


def apply(A, x, flags=0):
    xd = dev(x)
    yd = torch.full_like(xd, float("nan"))
    fs.spmv_apply(A, xd, yd, flags)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


PROBLEMS = {
    "cube_laplace_20": lambda: fegen.cube_laplace(20, 1501),
    "cube_laplace_13_neumann": lambda: fegen.cube_laplace(13, 41, dirichlet=False),
    "elasticity_9": lambda: fegen.cube_elasticity(9, 42),
    "shell_6x20x36": lambda: fegen.shell_laplace(6, 20, 36, 43),
}
_cache = {}


def problem(name):
    if name not in _cache:
        _cache[name] = PROBLEMS[name]()
    return _cache[name]


KERNELS = [
    dict(format=fs.FESPMV_FMT_CSR, csr_lanes=1),
    dict(format=fs.FESPMV_FMT_CSR, csr_lanes=4),
    dict(format=fs.FESPMV_FMT_CSR, csr_lanes=8),
    dict(format=fs.FESPMV_FMT_CSR, csr_lanes=32),
    dict(format=fs.FESPMV_FMT_SLICED, vec=1, sigma=0, threshold=0),
    dict(format=fs.FESPMV_FMT_SLICED, vec=2, sigma=256, threshold=0),
    dict(format=fs.FESPMV_FMT_SLICED, vec=4, sigma=10**9, threshold=0),
    dict(format=fs.FESPMV_FMT_SLICED, vec=2, sigma=256, threshold=4),
    dict(format=fs.FESPMV_FMT_SLICED, vec=1, sigma=64, threshold=2, block=128),
    dict(format=fs.FESPMV_FMT_SLICED, vec=2, sigma=64, threshold=0, reorder=fs.FESPMV_REORDER_NONE),
    # x gathered from L1/L2 instead of staged per tile in shared memory
    dict(format=fs.FESPMV_FMT_SLICED, vec=2, sigma=256, threshold=0, tiles=-1),
    dict(format=fs.FESPMV_FMT_SLICED, vec=1, sigma=64, threshold=2, tiles=-1),
    dict(format=fs.FESPMV_FMT_SLICED, vec=4, sigma=10**9, threshold=4, tiles=-1),
    # float-pair FP64 products on the FP32 pipe
    dict(format=fs.FESPMV_FMT_SLICED, vec=2, sigma=256, precisions=fs.FESPMV_PREC_DF64),
    dict(format=fs.FESPMV_FMT_SLICED, vec=1, sigma=64, threshold=2, precisions=fs.FESPMV_PREC_DF64),
    dict(format=fs.FESPMV_FMT_SLICED, vec=4, sigma=10**9, threshold=4, precisions=fs.FESPMV_PREC_DF64),
    dict(format=fs.FESPMV_FMT_SLICED, vec=2, sigma=256, precisions=fs.FESPMV_PREC_DF64, tiles=-1),
]


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("k", range(len(KERNELS)))
def test_spmv_parity(name, k):
    p = problem(name)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node, **KERNELS[k])
    x = fegen.random_vector(p.n_rows, 7 + k)
    check_parity(p, apply(A, x), x)
    # host buffers through the same entry point
    y = np.zeros(p.n_rows)
    fs.spmv_apply(A, x, y)
    check_parity(p, y, x)


@pytest.mark.parametrize("name", ["elasticity_9", "shell_6x20x36"])
def test_device_layout_bit_exact_and_permuted_io(name):
    p = problem(name)
    sigma, thr, V = 128, 3, 2
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node,
                       sigma=sigma, threshold=thr, vec=V)
    P = layout.row_permutation(p.rowptr, p.dofs_per_node, p.node_xyz, "morton", sigma)
    rp2, ci2, v2, vmap = layout.permute_csr(p.rowptr, p.colind, p.values, P)
    meta, col, val, pmap = layout.pack(rp2, ci2, v2, thr, V)
    src = np.full(len(col), -1, dtype=np.int64)
    src[pmap[vmap]] = np.arange(p.nnz)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_PERM), P.astype(np.int32))
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_META), meta)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_COLS), col)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_SRCMAP), src)
    got = fs.spmv_export(A, fs.FESPMV_EXPORT_VALUES)
    assert np.array_equal(got.view(np.uint64), val.view(np.uint64))
    dg = fs.spmv_export(A, fs.FESPMV_EXPORT_DIAG)
    Ad = {(i, c): v for i in range(p.n_rows)
          for c, v in zip(ci2[rp2[i]:rp2[i + 1]], v2[rp2[i]:rp2[i + 1]])}
    assert np.array_equal(dg, np.array([Ad.get((i, i), 0.0) for i in range(p.n_rows)]))
    # permuted I/O: y' = A' x' with x' = x[P] equals y[P]
    x = fegen.random_vector(p.n_rows, 77)
    yp = apply(A, x[P], fs.FESPMV_IO_PERMUTED)
    yo = oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(p.values), np.abs(x))
    assert np.all(np.abs(yp - yo[P]) <= TOL * bound[P])
    # spmv_permute round trip is exact
    xd = dev(x)
    xp = torch.empty_like(xd)
    back = torch.empty_like(xd)
    fs.spmv_permute(A, xd, xp, 0)
    fs.spmv_permute(A, xp, back, 1)
    torch.cuda.synchronize()
    assert np.array_equal(xp.cpu().numpy(), x[P]) and np.array_equal(back.cpu().numpy(), x)


@pytest.mark.parametrize("fmt", [fs.FESPMV_FMT_CSR, fs.FESPMV_FMT_SLICED])
def test_update_values(fmt):
    p = problem("elasticity_9")
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, format=fmt, sigma=64)
    rng = np.random.default_rng(3)
    new = p.values * rng.uniform(0.5, 2.0, size=p.nnz)
    x = fegen.random_vector(p.n_rows, 8)
    fs.spmv_update_values(A, new)                         # host values
    check_parity(p, apply(A, x), x, values=new)
    fs.spmv_update_values(A, dev(p.values))               # device values
    torch.cuda.synchronize()
    check_parity(p, apply(A, x), x)


def test_edge_cases_empty_ragged_and_nonfinite():
    # empty matrix
    A = fs.spmv_create(np.array([0]), np.array([], np.int32), np.array([]))
    fs.spmv_apply(A, torch.zeros(0, dtype=torch.float64, device="cuda"),
                  torch.zeros(0, dtype=torch.float64, device="cuda"))
    # 37 rows (ragged last warp), empty rows, one long row spanning a whole warp
    n = 37
    rng = np.random.default_rng(5)
    lens = np.array([0 if i % 7 == 0 else 1 + i % 5 for i in range(n)])
    lens[3] = n
    rowptr = np.concatenate([[0], np.cumsum(lens)])
    cols = np.concatenate([np.sort(rng.choice(n, lens[i], replace=False)) for i in range(n)])
    vals = rng.standard_normal(len(cols))

    class Q:  # minimal problem record for check_parity
        pass
    q = Q()
    q.rowptr, q.colind, q.values, q.n_rows = rowptr, cols.astype(np.int32), vals, n
    for kw in KERNELS:
        kw = {k: v for k, v in kw.items() if k != "reorder"}
        A = fs.spmv_create(rowptr, cols, vals, **kw)
        x = fegen.random_vector(n, 9)
        y = apply(A, x)
        check_parity(q, y, x)
        assert np.all(y[lens == 0] == 0.0)
        # a NaN in x poisons exactly the rows that store that column, never an empty row
        xn = x.copy()
        xn[11] = np.nan
        yn = apply(A, xn)
        yo = oracle.csr_spmv(rowptr, cols, vals, xn)
        assert np.array_equal(np.isnan(yn), np.isnan(yo))


@pytest.mark.parametrize("fmt,kw", [(fs.FESPMV_FMT_SLICED, dict(sigma=1024, vec=1, threshold=0, tiles=0)),
                                    (fs.FESPMV_FMT_SLICED, dict(sigma=1024, vec=2)),
                                    (fs.FESPMV_FMT_SLICED, dict(sigma=1024, vec=2, tiles=-1)),
                                    (fs.FESPMV_FMT_SLICED, dict(sigma=1024, vec=2,
                                                                precisions=fs.FESPMV_PREC_DF64)),
                                    (fs.FESPMV_FMT_CSR, dict(csr_lanes=4))])
def test_full_size_elasticity_64(fmt, kw):
    """The benchmark's matrix (64^3 nodes, 786,432 rows, ~34M nnz), every row checked;
    the first layout is the one the benchmark times (one entry per lane per load, sort
    windows of 1,024 rows, K1 slices, x staged per tile), also in the permuted
    numbering the timed product runs in."""
    p = fegen.cube_elasticity(64, 1502)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, format=fmt, **kw)
    x = fegen.random_vector(p.n_rows, 1504)
    check_parity(p, apply(A, x), x)
    if fmt == fs.FESPMV_FMT_SLICED and kw.get("vec") == 1:
        info = fs.spmv_get_info(A)
        assert info["vec"] == 1 and info["n_tiles"] > 0
        xd = torch.from_numpy(x).cuda()
        xp, yp, y = torch.empty_like(xd), torch.empty_like(xd), torch.empty_like(xd)
        fs.spmv_permute(A, xd, xp, 0)
        fs.spmv_apply(A, xp, yp, fs.FESPMV_IO_PERMUTED)
        fs.spmv_permute(A, yp, y, 1)
        check_parity(p, y.cpu().numpy(), x)


@pytest.mark.parametrize("tiles", [0, -1])
@pytest.mark.parametrize("vec", [1, 2, 4])
def test_float_pair_product_out_of_range_entries(vec, tiles):
    """Values and x entries outside [2^-50, 2^50], and Inf/NaN, take the exact FP64 path."""
    p = problem("elasticity_9")
    rng = np.random.default_rng(11)
    vals = p.values.copy()
    idx = rng.choice(p.nnz, 40, replace=False)
    vals[idx[:20]] *= 1e-30
    vals[idx[20:]] *= 1e30
    A = fs.spmv_create(p.rowptr, p.colind, vals, p.node_xyz, 3, sigma=64, vec=vec,
                       precisions=fs.FESPMV_PREC_DF64, tiles=tiles)
    x = fegen.random_vector(p.n_rows, 12)
    x[rng.choice(p.n_rows, 30, replace=False)] *= 1e-200
    x[rng.choice(p.n_rows, 30, replace=False)] *= 1e200
    x[rng.choice(p.n_rows, 5, replace=False)] = 0.0
    check_parity(p, apply(A, x), x, values=vals)
    xn = x.copy()
    xn[7] = np.inf
    xn[19] = np.nan
    yn = apply(A, xn)
    yo = oracle.csr_spmv(p.rowptr, p.colind, vals, xn)
    assert np.array_equal(np.isnan(yn), np.isnan(yo)) and np.array_equal(np.isinf(yn), np.isinf(yo))


def test_autotuner_returns_a_valid_fast_layout():
    p = problem("shell_6x20x36")
    t = fs.spmv_autotune(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=256, reps=5)
    assert t["tried"] >= 9 and t["best_us"] > 0
    assert t["vec"] in (1, 2, 4) and t["block"] in (128, 256) and t["threshold"] >= 0 and t["tiles"] in (0, -1)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=256, vec=t["vec"],
                       threshold=t["threshold"], block=t["block"], tiles=t["tiles"])
    assert fs.spmv_get_info(A)["n_tiles"] > 0 or t["tiles"] == -1
    # with tiles off in the base options only cache-gather layouts are tried
    u = fs.spmv_autotune(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=256, reps=3, tiles=-1)
    assert u["tiles"] == -1 and u["tried"] < t["tried"]
    x = fegen.random_vector(p.n_rows, 21)
    check_parity(p, apply(A, x), x)
    # timed in the low precision the options name: the winner is a valid FP32 layout
    for prec in (fs.FESPMV_PREC_F32, fs.FESPMV_PREC_BF16):
        w = fs.spmv_autotune(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=256, reps=3, tiles=-1,
                             precisions=prec)
        assert w["tiles"] == -1 and w["tried"] == u["tried"] and w["best_us"] > 0
        B = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=256, vec=w["vec"],
                           threshold=w["threshold"], block=w["block"], tiles=-1, precisions=prec)
        assert fs.spmv_get_info(B)["vec"] == w["vec"]


@pytest.mark.parametrize("name,thr,V", [("elasticity_9", 0, 2), ("shell_6x20x36", 3, 1),
                                        ("cube_laplace_20", 2, 4)])
def test_tiles_bit_exact_against_oracle(name, thr, V):
    p = problem(name)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node, sigma=128,
                       threshold=thr, vec=V)
    meta = fs.spmv_export(A, fs.FESPMV_EXPORT_META)
    col = fs.spmv_export(A, fs.FESPMV_EXPORT_COLS)
    t, d, idx = layout.tiles(meta, col, 8, 4096)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_TILES), t)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_TILE_COLS), d)
    assert np.array_equal(fs.spmv_export(A, fs.FESPMV_EXPORT_TILE_INDEX), idx)
    info = fs.spmv_get_info(A)
    assert info["n_tiles"] == len(t) and info["tile_max_cols"] == t[:, 3].max()
    B = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, p.dofs_per_node, sigma=128, tiles=-1)
    assert fs.spmv_get_info(B)["n_tiles"] == 0


def test_slice_wider_than_a_tile_gathers_from_cache():
    """A slice with more distinct columns than a tile holds leaves the handle untiled."""
    n = 8192
    rng = np.random.default_rng(17)
    rows = [np.union1d(rng.choice(n, 200, replace=False), [i]) if i < 32 else np.array([i])
            for i in range(n)]
    rowptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])])
    cols = np.concatenate(rows).astype(np.int32)
    vals = rng.standard_normal(len(cols))
    A = fs.spmv_create(rowptr, cols, vals, sigma=0)
    assert fs.spmv_get_info(A)["n_tiles"] == 0

    class Q:
        pass
    q = Q()
    q.rowptr, q.colind, q.values, q.n_rows = rowptr, cols, vals, n
    x = fegen.random_vector(n, 18)
    check_parity(q, apply(A, x), x)


@pytest.mark.parametrize("k", [1, 5, 10, 13])
def test_pinned_host_buffers_are_read_and_written_in_place(k):
    """Page-locked host x and y (the in-place permutation path) give the same bits as
    device vectors (on tiled handles: the product with the permutations folded in);
    pageable host buffers (staging copies) too."""
    p = problem("elasticity_9")
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, **KERNELS[k])
    x = fegen.random_vector(p.n_rows, 31)
    yd = apply(A, x)
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.full((p.n_rows,), float("nan"), dtype=torch.float64).pin_memory()
    fs.spmv_apply(A, xh.numpy(), yh.numpy())
    assert np.array_equal(yh.numpy().view(np.uint64), yd.view(np.uint64))
    y2 = np.zeros(p.n_rows)
    fs.spmv_apply(A, x, y2)
    assert np.array_equal(y2.view(np.uint64), yd.view(np.uint64))
    # pinned views that are not 16-byte aligned (one double in)
    xb = torch.zeros(p.n_rows + 1, dtype=torch.float64).pin_memory()
    yb = torch.full((p.n_rows + 1,), 7.0, dtype=torch.float64).pin_memory()
    xb[1:] = torch.from_numpy(x)
    fs.spmv_apply(A, xb.numpy()[1:], yb.numpy()[1:])
    assert np.array_equal(yb.numpy()[1:].view(np.uint64), yd.view(np.uint64)) and yb[0].item() == 7.0


def test_full_size_shell_24x256x512():
    """The shell workload (3,145,728 rows, ~46 M nnz, more tiles than the cube): every
    row of the tiled FP64 product, and of the FP32 product of S A S, against the oracle."""
    p = fegen.shell_laplace(24, 256, 512, 1503)
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 1, sigma=1024,
                       precisions=fs.FESPMV_PREC_F32)
    assert fs.spmv_get_info(A)["n_tiles"] > 0
    x = fegen.random_vector(p.n_rows, 1505)
    check_parity(p, apply(A, x), x)
    bv = oracle.scaled_values(p.rowptr, p.colind, p.values, "f32")
    x32 = x.astype(np.float32)
    xd = dev(x32)
    yd = torch.empty_like(xd)
    fs.spmv_apply_scaled(A, xd, yd, fs.FESPMV_PREC_F32)
    torch.cuda.synchronize()
    yo = oracle.csr_spmv_f32(p.rowptr, p.colind, bv, x32)
    bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(bv).astype(np.float64), np.abs(x32).astype(np.float64))
    L = np.diff(p.rowptr).max()
    assert np.all(np.abs(yd.cpu().numpy().astype(np.float64) - yo) <= 2 * L * 2.0 ** -24 * bound)


@pytest.mark.parametrize("tiles", [0, -1])
@pytest.mark.parametrize("col_order", [fs.FESPMV_COLS_RENUMBERED, fs.FESPMV_COLS_ORIGINAL])
def test_column_orders_k1_and_k1r(col_order, tiles):
    """K1 (input column numbers) and K1r (renumbered, unsorted) handles: the FP64
    product within the componentwise bound, input and host I/O; K1 handles take x
    in the input numbering only and carry no CG."""
    p = problem("elasticity_9")
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, sigma=128, tiles=tiles,
                       col_order=col_order)
    x = fegen.random_vector(p.n_rows, 31)
    check_parity(p, apply(A, x), x)
    yh = np.zeros(p.n_rows)
    fs.spmv_apply(A, x.copy(), yh)
    check_parity(p, yh, x)
    xd = torch.from_numpy(x).cuda()
    if col_order == fs.FESPMV_COLS_ORIGINAL:
        with pytest.raises(fs.FespmvError):
            fs.spmv_apply(A, xd, torch.empty_like(xd), fs.FESPMV_IO_PERMUTED)
        with pytest.raises(fs.FespmvError):
            fs.cg_solve(A, xd, torch.zeros_like(xd))
    else:
        res = fs.cg_solve(A, xd, torch.zeros_like(xd), tol=1e-10)
        assert res["status"] == 0


@pytest.mark.parametrize("k", [4, 5, 6, 7, 8])
def test_input_numbering_folds_the_permutations(k):
    """On tiled handles the input-numbering product stages x[P[c']] per tile and stores
    y[P[i']]: bitwise the permuted-numbering product between two gathers."""
    p = problem("elasticity_9")
    A = fs.spmv_create(p.rowptr, p.colind, p.values, p.node_xyz, 3, **KERNELS[k])
    assert fs.spmv_get_info(A)["n_tiles"] > 0
    x = fegen.random_vector(p.n_rows, 32)
    xd = dev(x)
    xp, yp, y = torch.empty_like(xd), torch.full_like(xd, float("nan")), torch.empty_like(xd)
    fs.spmv_permute(A, xd, xp, 0)
    fs.spmv_apply(A, xp, yp, fs.FESPMV_IO_PERMUTED)
    fs.spmv_permute(A, yp, y, 1)
    torch.cuda.synchronize()
    yi = apply(A, x)
    assert np.array_equal(yi.view(np.uint64), y.cpu().numpy().view(np.uint64))
    check_parity(p, yi, x)
