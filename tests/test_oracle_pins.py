"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test ties one oracle routine to something it does not compute itself:
a dense brute-force product, the paper's worked example, a closed form, a
dense direct solve, or a property exact arithmetic guarantees.  A dropped
term, a wrong sign or index, or a transposed operand in the oracle fails at
least one of them.
"""
import json
import os

import numpy as np
import pytest

import fegen
import oracle
from oracle import layout

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_of(rowptr, colind, values, n):
    """Dense matrix built entry by entry (duplicates summed)."""
    A = np.zeros((n, n))
    for i in range(n):
        for p in range(rowptr[i], rowptr[i + 1]):
            A[i, colind[p]] += values[p]
    return A


def small_problems():
    return [fegen.cube_laplace(4, 7, dirichlet=False), fegen.cube_laplace(5, 8),
            fegen.cube_elasticity(3, 9, dirichlet=False), fegen.cube_elasticity(4, 10),
            fegen.shell_laplace(3, 5, 8, 11, dirichlet=False), fegen.shell_laplace(4, 6, 8, 12)]


# ---------------------------------------------------------------- sparse product

def test_spmv_integer_matrix_exact():
    # 3x3 matrix with integer entries: every product and sum is exact in FP64
    rowptr = np.array([0, 2, 2, 5])
    colind = np.array([2, 0, 0, 1, 2])
    values = np.array([3.0, -1.0, 2.0, 5.0, -4.0])
    x = np.array([7.0, -2.0, 0.5])
    y = oracle.csr_spmv(rowptr, colind, values, x)
    assert y.tolist() == [3 * 0.5 - 7.0, 0.0, 2 * 7.0 - 10.0 - 2.0]


@pytest.mark.parametrize("k", range(6))
def test_spmv_matches_dense_brute_force(k):
    p = small_problems()[k]
    A = dense_of(p.rowptr, p.colind, p.values, p.n_rows)
    x = fegen.random_vector(p.n_rows, 100 + k)
    y = oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    yd = A @ x
    bound = np.abs(A) @ np.abs(x)
    assert np.all(np.abs(y - yd) <= 1e-14 * bound + 1e-300)


def test_spmv_empty_rows_and_empty_matrix():
    rowptr = np.array([0, 0, 1, 1])
    y = oracle.csr_spmv(rowptr, np.array([2]), np.array([4.0]), np.array([1.0, 2.0, 3.0]))
    assert y.tolist() == [0.0, 12.0, 0.0]
    y0 = oracle.csr_spmv(np.array([0]), np.array([], dtype=np.int32), np.array([]), np.array([]))
    assert y0.shape == (0,)


def test_worked_example_k1r_k1rs():
    g = json.load(open(os.path.join(GOLDEN, "worked_example_k1r.json")))
    x, P, A, c = (np.array(g[k]) for k in ("x", "P", "A", "c"))
    # x'(.) = x(P(.))
    assert x[P - 1].tolist() == g["x_prime"]
    # c' = P^-1 applied to c
    cp = layout.worked_example_renumber(c, P)
    assert cp.tolist() == g["c_prime"]
    order = np.argsort(cp, kind="stable")
    assert cp[order].tolist() == g["c_dprime"]
    assert A[order].tolist() == g["A_dprime"]
    # the row's product is unchanged by the renumbering, through the oracle
    n = len(x)
    rowptr = np.array([0, len(A)] + [len(A)] * (n - 1))
    y = oracle.csr_spmv(rowptr, c - 1, A.astype(float), x.astype(float))
    assert y[0] == g["row_dot"]
    xp = x[P - 1].astype(float)
    y2 = oracle.csr_spmv(rowptr, np.array(g["c_dprime"]) - 1,
                         np.array(g["A_dprime"], dtype=float), xp)
    assert y2[0] == g["row_dot"]


# ------------------------------------------------------------- permutation + packing

@pytest.mark.parametrize("k", range(6))
def test_permute_csr_is_PAPt(k):
    p = small_problems()[k]
    A = dense_of(p.rowptr, p.colind, p.values, p.n_rows)
    P = layout.row_permutation(p.rowptr, p.dofs_per_node, p.node_xyz, "morton", sigma=16)
    assert sorted(P.tolist()) == list(range(p.n_rows))
    rp2, ci2, v2, vmap = layout.permute_csr(p.rowptr, p.colind, p.values, P)
    A2 = dense_of(rp2, ci2, v2, p.n_rows)
    assert np.array_equal(A2, A[np.ix_(P, P)])
    for i in range(p.n_rows):
        assert np.all(np.diff(ci2[rp2[i]:rp2[i + 1]]) > 0)
    assert np.array_equal(v2[vmap], p.values)
    # y' = A' x' with x' = x[P] gives y[P]
    x = fegen.random_vector(p.n_rows, 5)
    y = oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    y2 = oracle.csr_spmv(rp2, ci2, v2, x[P])
    assert np.all(np.abs(y2 - y[P]) <= 1e-14 * (np.abs(A) @ np.abs(x))[P] + 1e-300)


def test_morton_codes_of_cube_corners():
    corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float)
    code = layout.morton_codes(corners)
    full = (1 << layout.MORTON_BITS) - 1
    expect = []
    for i, j, k in corners.astype(int):
        c = 0
        for b in range(layout.MORTON_BITS):
            c |= ((i * full >> b) & 1) << (3 * b + 2)
            c |= ((j * full >> b) & 1) << (3 * b + 1)
            c |= ((k * full >> b) & 1) << (3 * b)
        expect.append(c)
    assert code.tolist() == expect
    assert code[-1] == (1 << 63) - 1
    # z-order of the corners: x most significant, then y, then z
    assert np.argsort(code).tolist() == list(range(8))


def test_length_sort_is_stable_and_windowed():
    lens = np.array([3, 5, 5, 1, 7, 2, 2, 9])
    rowptr = np.concatenate([[0], np.cumsum(lens)])
    P = layout.row_permutation(rowptr, 1, None, "none", sigma=4)
    assert P.tolist() == [1, 2, 0, 3, 7, 4, 5, 6]
    Pg = layout.row_permutation(rowptr, 1, None, "none", sigma=100)
    assert Pg.tolist() == [7, 4, 1, 2, 0, 5, 6, 3]


def test_slice_plan_k1_and_k2_threshold_rule():
    # one group of 32 rows: row 0 has 100 entries, the rest 5
    lens = np.array([100] + [5] * 31)
    rowptr = np.concatenate([[0], np.cumsum(lens)])
    k1 = layout.slice_plan(rowptr, threshold=0, V=1)
    assert k1 == [(0, 32, 1, 100)]
    # tau = 7: T = 16 (ceil(100/16) = 7 <= 7, ceil(100/8) = 13 > 7); 16 warps of 2 rows
    k2 = layout.slice_plan(rowptr, threshold=7, V=1)
    assert len(k2) == 16
    assert k2[0] == (0, 2, 16, 7)
    assert k2[1] == (2, 2, 16, 1)
    # V = 2 rounds each width up to even
    assert layout.slice_plan(rowptr, threshold=7, V=2)[1] == (2, 2, 16, 2)
    # tau larger than any row keeps T = 1; row > 32*tau uses a whole warp per row
    assert layout.slice_plan(rowptr, threshold=200, V=1) == k1
    big = np.concatenate([[0], np.cumsum(np.array([2000] + [1] * 3))])
    plan = layout.slice_plan(big, threshold=10, V=1)
    assert plan[0] == (0, 1, 32, 63) and len(plan) == 4


@pytest.mark.parametrize("threshold,V", [(0, 1), (0, 2), (4, 2), (3, 4)])
def test_pack_roundtrip_reproduces_rows(threshold, V):
    p = fegen.cube_elasticity(3, 13)
    P = layout.row_permutation(p.rowptr, 3, p.node_xyz, "morton", sigma=64)
    rp2, ci2, v2, _ = layout.permute_csr(p.rowptr, p.colind, p.values, P)
    meta, col, val, pmap = layout.pack(rp2, ci2, v2, threshold, V)
    assert np.array_equal(col[pmap], ci2) and np.array_equal(val[pmap], v2)
    pad = np.ones(len(col), bool)
    pad[pmap] = False
    assert np.all(col[pad] == -1) and np.all(val[pad] == 0)
    # walk the slices the way a warp does and rebuild every row's entries
    seen = {}
    for off32, w, r0, lt in meta:
        T = 1 << int(lt)
        for lane in range(32):
            r = r0 + lane // T
            for step in range(w):
                pos = off32 * 32 + (step // V) * 32 * V + lane * V + step % V
                if col[pos] >= 0:
                    seen.setdefault(r, []).append((step * T + lane % T, col[pos], val[pos]))
    for i in range(p.n_rows):
        ents = sorted(seen.get(i, []))
        assert [e[1] for e in ents] == ci2[rp2[i]:rp2[i + 1]].tolist()
        assert [e[2] for e in ents] == v2[rp2[i]:rp2[i + 1]].tolist()


# ------------------------------------------------------------------ conjugate gradient

def test_pcg_matches_dense_solve():
    p = fegen.cube_laplace(6, 21)
    A = dense_of(p.rowptr, p.colind, p.values, p.n_rows)
    b = fegen.random_vector(p.n_rows, 22)
    x, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-12)
    assert info["status"] == "converged" and info["true_relres"] <= 1e-12
    xd = np.linalg.solve(A, b)
    cond = np.linalg.cond(A)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 10 * cond * 1e-12


def test_pcg_recovers_manufactured_solution():
    p = fegen.cube_elasticity(5, 23)
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    x, info = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-12)
    assert info["status"] == "converged"
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-8


def test_cg_finite_termination_distinct_eigenvalues():
    # block-diagonal SPD matrix with exactly 3 distinct eigenvalues {1, 3, 4}:
    # blocks [[2,1],[1,2]] (eigenvalues 1, 3) and diagonal 4s; plain CG ends in 3 steps
    n_blocks, n4 = 5, 4
    rows, cols, vals = [], [], []
    for b in range(n_blocks):
        i = 2 * b
        for (r, c, v) in ((i, i, 2.0), (i, i + 1, 1.0), (i + 1, i, 1.0), (i + 1, i + 1, 2.0)):
            rows.append(r), cols.append(c), vals.append(v)
    for k in range(n4):
        i = 2 * n_blocks + k
        rows.append(i), cols.append(i), vals.append(4.0)
    n = 2 * n_blocks + n4
    order = np.lexsort((cols, rows))
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))])
    b = fegen.random_vector(n, 3)
    x, info = oracle.pcg(rowptr, np.array(cols)[order], np.array(vals)[order], b,
                         tol=1e-13, jacobi=False, max_restarts=0)
    assert info["status"] == "converged" and info["iters"] == 3


def test_jacobi_pcg_on_diagonal_matrix_is_one_step():
    n = 9
    d = np.arange(1, n + 1, dtype=float)
    b = fegen.random_vector(n, 4)
    x, info = oracle.pcg(np.arange(n + 1), np.arange(n), d, b, tol=1e-14, max_restarts=0)
    assert info["iters"] == 1
    assert np.allclose(x, b / d, rtol=1e-15, atol=0)


def test_cg_error_decreases_in_A_norm():
    p = fegen.cube_laplace(6, 24)
    A = dense_of(p.rowptr, p.colind, p.values, p.n_rows)
    b = fegen.random_vector(p.n_rows, 25)
    xs = np.linalg.solve(A, b)
    errs = []
    for k in range(1, 25):
        x, _ = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=0.0, max_iter=k, max_restarts=0)
        e = x - xs
        errs.append(e @ A @ e)
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))


@pytest.mark.parametrize("jacobi", [True, False])
def test_single_reduction_pcg_matches_dense_and_textbook(jacobi):
    p = fegen.cube_elasticity(4, 31)
    A = dense_of(p.rowptr, p.colind, p.values, p.n_rows)
    b = fegen.random_vector(p.n_rows, 32)
    x1, i1 = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-12, jacobi=jacobi,
                        single_reduction=True)
    x0, i0 = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-12, jacobi=jacobi)
    assert i1["status"] == "converged" and i1["true_relres"] <= 1e-12
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x1 - xd) / np.linalg.norm(xd) <= 10 * np.linalg.cond(A) * 1e-12
    # same recurrences in exact arithmetic: the step counts agree to rounding
    assert abs(i1["iters"] - i0["iters"]) <= 0.02 * i0["iters"] + 2
    # the first iterates agree closely (before rounding differences grow)
    xa, _ = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=0.0, max_iter=5, jacobi=jacobi,
                       max_restarts=0)
    xb, _ = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=0.0, max_iter=5, jacobi=jacobi,
                       max_restarts=0, single_reduction=True)
    assert np.linalg.norm(xa - xb) <= 1e-10 * np.linalg.norm(xa)


def test_single_reduction_pcg_finite_termination_and_status():
    n_blocks, n4 = 5, 4
    rows, cols, vals = [], [], []
    for b_ in range(n_blocks):
        i = 2 * b_
        for (r, c, v) in ((i, i, 2.0), (i, i + 1, 1.0), (i + 1, i, 1.0), (i + 1, i + 1, 2.0)):
            rows.append(r), cols.append(c), vals.append(v)
    for k in range(n4):
        i = 2 * n_blocks + k
        rows.append(i), cols.append(i), vals.append(4.0)
    n = 2 * n_blocks + n4
    order = np.lexsort((cols, rows))
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))])
    b = fegen.random_vector(n, 3)
    _, info = oracle.pcg(rowptr, np.array(cols)[order], np.array(vals)[order], b, tol=1e-13,
                         jacobi=False, max_restarts=0, single_reduction=True)
    assert info["status"] == "converged" and info["iters"] == 3
    _, info = oracle.pcg(np.arange(3), np.arange(2), np.array([1.0, -1.0]), np.ones(2),
                         jacobi=False, single_reduction=True)
    assert info["status"] == "breakdown"


def test_pcg_status_codes():
    # indefinite diagonal: Jacobi rejects it, plain CG breaks down (p.q <= 0)
    rowptr, colind = np.arange(3), np.arange(2)
    vals = np.array([1.0, -1.0])
    b = np.array([1.0, 1.0])
    _, info = oracle.pcg(rowptr, colind, vals, b)
    assert info["status"] == "bad_input"
    _, info = oracle.pcg(rowptr, colind, vals, b, jacobi=False)
    assert info["status"] == "breakdown"
    p = fegen.cube_laplace(6, 26)
    _, info = oracle.pcg(p.rowptr, p.colind, p.values, fegen.random_vector(p.n_rows, 1),
                         tol=1e-12, max_iter=3, max_restarts=0)
    assert info["status"] == "not_converged" and info["iters"] == 3
    x, info = oracle.pcg(p.rowptr, p.colind, p.values, np.zeros(p.n_rows))
    assert info["status"] == "converged" and not x.any()


# ------------------------------------------------------------- mixed-precision refinement

def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    v = np.concatenate([rng.standard_normal(2000).astype(np.float32),
                        np.array([1.0, -0.0, 1e-40, 3.0e38, 1.00390625, 1.01171875], np.float32)])
    ours = oracle.round_bf16(v)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_refinement_reaches_fp64_solution(storage):
    p = fegen.cube_laplace(8, 27)
    b = fegen.random_vector(p.n_rows, 28)
    xr, info = oracle.refine(p.rowptr, p.colind, p.values, b, tol=1e-10, inner_tol=1e-3,
                             storage=storage)
    assert info["status"] == "converged" and info["true_relres"] <= 1e-10
    x64, _ = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-12)
    A = dense_of(p.rowptr, p.colind, p.values, p.n_rows)
    cond = np.linalg.cond(A)
    assert np.linalg.norm(xr - x64) / np.linalg.norm(x64) <= cond * 1e-10


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_scaled_values_match_dense_scaling(storage):
    p = fegen.cube_elasticity(3, 29)
    A = dense_of(p.rowptr, p.colind, p.values, p.n_rows)
    s = 1.0 / np.sqrt(np.diag(A))
    Bd = (s[:, None] * A) * s[None, :]
    bv = oracle.scaled_values(p.rowptr, p.colind, p.values, storage)
    B = dense_of(p.rowptr, p.colind, bv.astype(np.float64), p.n_rows)
    u = 2.0 ** -24 if storage == "f32" else 2.0 ** -8   # unit roundoff, 24- or 8-bit significand
    assert np.all(np.abs(B - Bd) <= u * np.abs(Bd) * 1.0001)
    assert np.array_equal(B, B.T)                        # symmetric scaling keeps symmetry
    assert np.all(np.abs(np.diag(B) - 1.0) <= u)
    # float products: within the float rounding bound of the dense FP64 product
    x = fegen.random_vector(p.n_rows, 30).astype(np.float32)
    y = oracle.csr_spmv_f32(p.rowptr, p.colind, bv, x)
    yd = B @ x.astype(np.float64)
    L = np.diff(p.rowptr).max()
    assert np.all(np.abs(y - yd) <= (L + 1) * 2.0 ** -24 * (np.abs(B) @ np.abs(x)))


def test_float_spmv_integer_matrix_exact():
    # Small integers: every product and partial sum is exact in float, so the
    # float product must equal the integer product exactly (an empty row gives 0).
    rng = np.random.default_rng(31)
    n = 40
    counts = rng.integers(0, 9, size=n)
    counts[7] = 0
    rowptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    colind = np.concatenate([np.sort(rng.choice(n, size=c, replace=False)) for c in counts]).astype(np.int32)
    values = rng.integers(-20, 21, size=rowptr[-1]).astype(np.float32)
    x = rng.integers(-15, 16, size=n).astype(np.float32)
    y = oracle.csr_spmv_f32(rowptr, colind, values, x)
    A = dense_of(rowptr, colind, values.astype(np.float64), n).astype(np.int64)
    assert y.dtype == np.float32
    assert np.array_equal(y.astype(np.int64), A @ x.astype(np.int64))
    assert y[7] == 0.0


def _one_step_slices(cols_per_slice):
    """meta/col for slices of one step (w = 1) each: slice s holds 32 entries."""
    meta, col = [], []
    for s, cs in enumerate(cols_per_slice):
        meta.append((s, 1, 32 * s, 0))
        col.extend(list(cs) + [-1] * (32 - len(cs)))
    return np.array(meta, dtype=np.uint32), np.array(col, dtype=np.int32)


def test_tiles_hand_example():
    # slices with columns {0,1,2}, {2,3}, {4,5,6}, {6}: with max_cols = 5 the first two
    # share a tile (4 columns), the third would make 7, so it opens a new tile with the fourth
    meta, col = _one_step_slices([[0, 1, 2], [3, 2], [4, 5, 6], [6]])
    t, d, idx = layout.tiles(meta, col, max_slices=8, max_cols=5)
    assert t.tolist() == [[0, 2, 0, 4], [2, 2, 4, 3]]
    assert d.tolist() == [0, 1, 2, 3, 4, 5, 6]
    assert idx[:3].tolist() == [0, 1, 2] and idx[32:34].tolist() == [3, 2]
    assert idx[3] == 4 and idx[64 + 3] == 3          # padding -> the tile's zero slot D
    # max_slices closes tiles too; a slice wider than max_cols means no tiles
    t2, _, _ = layout.tiles(meta, col, max_slices=1, max_cols=5)
    assert t2[:, 1].tolist() == [1, 1, 1, 1]
    assert layout.tiles(meta, col, max_slices=8, max_cols=2) is None


@pytest.mark.parametrize("maker", ["elasticity", "shell"])
def test_tiles_reconstruct_columns_and_are_greedy(maker):
    p = fegen.cube_elasticity(6, 71) if maker == "elasticity" else fegen.shell_laplace(4, 12, 16, 72)
    P = layout.row_permutation(p.rowptr, p.dofs_per_node, p.node_xyz, "morton", 128)
    rp2, ci2, v2, _ = layout.permute_csr(p.rowptr, p.colind, p.values, P)
    meta, col, _, _ = layout.pack(rp2, ci2, v2, 3, 2)
    meta = np.asarray(meta).reshape(-1, 4)
    max_slices, max_cols = 4, 160
    t, d, idx = layout.tiles(meta, col, max_slices, max_cols)

    def cols_of(first, count):
        b = int(meta[first, 0]) * 32
        e = int(meta[first + count - 1, 0]) * 32 + 32 * int(meta[first + count - 1, 1])
        return col[b:e], b, e

    assert t[0, 0] == 0 and t[-1, 0] + t[-1, 1] == len(meta)
    assert np.all(t[1:, 0] == t[:-1, 0] + t[:-1, 1])                     # contiguous, in order
    for k, (first, count, off, D) in enumerate(t):
        cs, b, e = cols_of(first, count)
        real = cs[cs >= 0]
        u, first_pos = np.unique(real, return_index=True)
        assert D == len(u) <= max_cols and 1 <= count <= max_slices
        assert np.array_equal(d[off:off + D], real[np.sort(first_pos)])  # first-use order
        ii = idx[b:e].astype(np.int64)
        assert np.array_equal(d[off + ii[cs >= 0]], real)               # index -> column
        assert np.all(ii[cs < 0] == D)
        if k + 1 < len(t):                                               # greedy: the next slice
            nxt, _, _ = cols_of(first + count, 1)                        # would break a limit
            union = np.union1d(real, nxt[nxt >= 0])
            assert count == max_slices or len(union) > max_cols


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_reliable_refinement_reaches_dense_solution(storage):
    p = fegen.cube_laplace(7, 31)
    b = fegen.random_vector(p.n_rows, 32)
    x, info = oracle.refine_reliable(p.rowptr, p.colind, p.values, b, tol=1e-10, storage=storage)
    assert info["status"] == "converged" and info["true_relres"] <= 1e-10
    A = dense_of(p.rowptr, p.colind, p.values, p.n_rows)
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= np.linalg.cond(A) * 1e-10
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1.01e-10   # recomputed densely
    # about log(1e-10) / log(delta) replacements
    assert 8 <= info["updates"] <= 16


def test_reliable_refinement_keeps_the_krylov_space():
    """No restarts: the float CG with residual replacement needs close to as many steps
    as FP64 Jacobi-PCG (the same method in exact arithmetic, since CG on S A S is
    Jacobi-PCG on A; float rounding delays it somewhat), while restarted refinement,
    at any inner tolerance, needs clearly more."""
    p = fegen.cube_elasticity(6, 33)
    b = fegen.random_vector(p.n_rows, 34)
    _, rel = oracle.refine_reliable(p.rowptr, p.colind, p.values, b, tol=1e-10)
    _, pcg = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-10)
    assert rel["status"] == "converged" and pcg["status"] == "converged"
    assert pcg["iters"] <= rel["iters"] <= 1.3 * pcg["iters"] + 5
    for inner_tol in (1e-1, 1e-2, 1e-3):
        _, rst = oracle.refine(p.rowptr, p.colind, p.values, b, tol=1e-10, inner_tol=inner_tol)
        assert rst["inner"] > 1.3 * rel["iters"]


def test_reliable_refinement_special_cases():
    # diagonal matrix: B = S A S = I up to rounding, so CG needs a step per update
    n = 50
    rowptr = np.arange(n + 1)
    colind = np.arange(n, dtype=np.int32)
    vals = np.linspace(1.0, 100.0, n)
    b = fegen.random_vector(n, 35)
    x, info = oracle.refine_reliable(rowptr, colind, vals, b, tol=1e-12)
    assert info["status"] == "converged" and info["iters"] <= 4
    assert np.allclose(x, b / vals, rtol=1e-11, atol=0)
    # b = 0 gives x = 0 at once; a non-positive diagonal is rejected
    x0, i0 = oracle.refine_reliable(rowptr, colind, vals, np.zeros(n))
    assert i0["status"] == "converged" and i0["iters"] == 0 and not x0.any()
    _, bad = oracle.refine_reliable(rowptr, colind, -vals, b)
    assert bad["status"] == "breakdown"
    # iteration limit
    p = fegen.cube_laplace(8, 36)
    bb = fegen.random_vector(p.n_rows, 37)
    _, lim = oracle.refine_reliable(p.rowptr, p.colind, p.values, bb, tol=1e-12, max_iter=3)
    assert lim["status"] == "not_converged" and lim["iters"] == 3


# ---------------------------------------------------------------- assembly (Sec. 4)

@pytest.mark.parametrize("maker", [lambda d: fegen.cube_laplace(6, 21, dirichlet=d, elements=True),
                                   lambda d: fegen.cube_elasticity(5, 22, dirichlet=d, elements=True),
                                   lambda d: fegen.shell_laplace(3, 8, 10, 23, dirichlet=d, elements=True)])
@pytest.mark.parametrize("dirichlet", [True, False])
def test_assembly_equals_the_generators_rowwise_assembly(maker, dirichlet):
    """The oracle sums element contributions element by element; the generator
    sums them row by row (its own traversal of the tets around each node, then
    the symmetric elimination).  Both add in ascending element order, so the
    values agree bit for bit."""
    p = maker(dirichlet)
    mask = p.dirichlet if dirichlet else None
    v = oracle.assemble_matrix(p.rowptr, p.colind, p.elem_nodes, p.elem_mats, p.dofs_per_node, mask)
    assert np.array_equal(v.view(np.uint64), p.values.view(np.uint64))


def test_assembly_hand_example():
    """Two elements on nodes {0,1,2} and {1,2,3} (scalar dofs): entries shared by
    both are the sums, the others one element's value; node 3 constrained."""
    en = np.array([[0, 1, 2], [1, 2, 3]], dtype=np.int32)
    K1 = np.array([[4., -1., -2.], [-1., 5., -3.], [-2., -3., 6.]])
    K2 = np.array([[7., -4., -1.], [-4., 8., -2.], [-1., -2., 9.]])
    rows = [[0, 1, 2], [0, 1, 2, 3], [0, 1, 2, 3], [1, 2, 3]]
    rowptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    colind = np.concatenate(rows).astype(np.int32)
    v = oracle.assemble_matrix(rowptr, colind, en, np.stack([K1, K2]), 1)
    dense = np.zeros((4, 4))
    for r, cs in enumerate(rows):
        for k, c in enumerate(cs):
            dense[r, c] = v[rowptr[r] + k]
    expect = np.array([[4., -1., -2., 0.],
                       [-1., 5. + 7., -3. - 4., -1.],
                       [-2., -3. - 4., 6. + 8., -2.],
                       [0., -1., -2., 9.]])
    assert np.array_equal(dense, expect)
    mask = np.array([0, 0, 0, 1], dtype=np.uint8)
    rows_m = [[0, 1, 2], [0, 1, 2], [0, 1, 2], [3]]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows_m])]).astype(np.int64)
    vm = oracle.assemble_matrix(rp, np.concatenate(rows_m).astype(np.int32), en, np.stack([K1, K2]), 1, mask)
    assert np.array_equal(vm, [4., -1., -2., -1., 12., -7., -2., -7., 14., 1.])
    r = oracle.assemble_vector(4, en, np.array([[1., 2., 3.], [10., 20., 30.]]), 1, mask)
    assert np.array_equal(r, [1., 12., 23., 0.])
    with pytest.raises(ValueError):   # a contribution with no stored position
        oracle.assemble_matrix(rp, np.concatenate(rows_m).astype(np.int32), en, np.stack([K1, K2]), 1)


@pytest.mark.parametrize("maker", [lambda: fegen.cube_elasticity(5, 24, elements=True),
                                   lambda: fegen.shell_laplace(3, 8, 10, 25, elements=True)])
def test_vector_assembly_of_element_products_is_the_global_product(maker):
    """Linearity: assembling the element vectors K_e u_e gives K u (u zero on the
    constrained dofs), up to rounding."""
    p = maker()
    u = fegen.random_vector(p.n_rows, 26)
    u[p.dirichlet.astype(bool)] = 0.0
    dpn = p.dofs_per_node
    idx = (dpn * p.elem_nodes[:, :, None] + np.arange(dpn)[None, None, :]).reshape(p.n_elems, -1)
    re = np.einsum("eij,ej->ei", p.elem_mats, u[idx])
    r = oracle.assemble_vector(p.n_rows, p.elem_nodes, re, dpn, p.dirichlet)
    ku = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    ku[p.dirichlet.astype(bool)] = 0.0
    bound = oracle.csr_spmv(p.rowptr, p.colind, np.abs(p.values), np.abs(u))
    assert np.all(np.abs(r - ku) <= 1e-13 * (bound + 1e-300) * 30)


def test_threaded_product_is_bitwise_the_sequential_one():
    # the CPU baseline runs the product's row loop on all host cores; each row is
    # still one sequential sum, so the result must not change by a single bit
    p = fegen.cube_elasticity(10, 77)
    x = fegen.random_vector(p.n_rows, 78)
    y1 = oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
    try:
        oracle.set_threads(4)
        y4 = oracle.csr_spmv(p.rowptr, p.colind, p.values, x)
        xo4, info4 = oracle.pcg(p.rowptr, p.colind, p.values, x, tol=1e-8)
    finally:
        oracle.set_threads(1)
    xo1, info1 = oracle.pcg(p.rowptr, p.colind, p.values, x, tol=1e-8)
    assert np.array_equal(y1.view(np.uint64), y4.view(np.uint64))
    assert info1["iters"] == info4["iters"]
    assert np.array_equal(xo1.view(np.uint64), xo4.view(np.uint64))


def test_node_blocks_hand_example():
    # two nodes, six rows; node 0's rows touch column nodes 0 and 1, so do node 1's
    rowptr = np.array([0, 3, 4, 6, 7, 9, 11], dtype=np.int64)
    colind = np.array([0, 1, 4, 1, 2, 5, 3, 0, 4, 2, 5], dtype=np.int32)
    meta, col, vidx = layout.node_blocks(rowptr, colind)
    assert meta.tolist() == [[0, 2, 0, 0]]
    want_col = np.full(64, -1)
    want_col[[0, 32, 1, 33]] = [0, 1, 0, 1]
    assert np.array_equal(col, want_col)
    want = np.full(9 * 64, -1)
    # (value index) -> CSR position, worked out by hand from index = 288*step + 32*k + lane
    # (k = 3a + b: row a of the node, column b of the block's column node)
    for idx, p in ((0, 0), (32, 1), (320, 2), (128, 3), (256, 4), (544, 5),
                   (289, 6), (97, 7), (417, 8), (257, 9), (545, 10)):
        want[idx] = p
    assert np.array_equal(vidx, want)


@pytest.mark.parametrize("n,sigma", [(5, 96), (6, 0)])
def test_node_blocks_hold_every_entry_once(n, sigma):
    p = fegen.cube_elasticity(n, 60 + n)
    P = layout.node_row_permutation(p.rowptr, p.node_xyz, "morton", sigma)
    # whole nodes: rows 3k..3k+2 are the three dofs of one node
    assert np.all(P.reshape(-1, 3) // 3 == (P.reshape(-1, 3) // 3)[:, :1])
    assert np.array_equal(P.reshape(-1, 3) % 3, np.tile(np.arange(3), (len(P) // 3, 1)))
    rp2, c2, v2, _ = layout.permute_csr(p.rowptr, p.colind, p.values, P)
    meta, col, vidx = layout.node_blocks(rp2, c2)
    live = vidx[vidx >= 0]
    assert np.array_equal(np.sort(live), np.arange(p.nnz))
    # the blocks rebuild the permuted matrix
    nr = p.n_rows
    D = np.zeros((nr, nr))
    for s, (o32, w, first, _) in enumerate(meta):
        o = int(o32) * 32
        for lane in range(32):
            I = int(first) + lane
            if I >= nr // 3:
                break
            for st in range(int(w)):
                J = col[o + 32 * st + lane]
                if J < 0:
                    continue
                for k in range(9):
                    q = vidx[9 * (o + 32 * st) + 32 * k + lane]
                    a, b = divmod(k, 3)
                    D[3 * I + a, 3 * J + b] += v2[q] if q >= 0 else 0.0
    assert np.array_equal(D, dense_of(rp2, c2, v2, nr))
    # and the library's host planner orders the rows the same way
    pl = fs_plan(p, sigma)
    assert np.array_equal(pl["perm"], P)


def fs_plan(p, sigma):
    fs = pytest.importorskip("paper_1501_00324_gb300")
    return fs.spmv_plan(p.rowptr, p.colind, p.node_xyz, 3, sigma=sigma, vec=1, node_blocks=3)


# ---- flexible CG with a low-precision inner CG (oracle_fcg) ----------------------

def test_fcg_with_one_exact_inner_step_is_jacobi_pcg():
    # one FP64 inner step on S A S gives z = c D^-1 r: the flexible directions are
    # Jacobi-PCG's up to scale, so the iterates are PCG's
    p = fegen.shell_laplace(5, 16, 24, 52)
    u = fegen.manufactured_solution(p)
    b = oracle.csr_spmv(p.rowptr, p.colind, p.values, u)
    xo, io = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-10)
    x, info = oracle.fcg(p.rowptr, p.colind, p.values, b, tol=1e-10, inner_steps=1, storage="f64")
    assert info["status"] == "converged" and abs(info["iters"] - io["iters"]) <= 1
    assert info["inner"] == info["iters"]
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-11


def test_fcg_finite_termination_and_diagonal():
    # Jacobi-scaled, the 3-eigenvalue matrix of the PCG pin has eigenvalues {1/2, 1, 3/2}
    n_blocks, n4 = 5, 4
    rows, cols, vals = [], [], []
    for blk in range(n_blocks):
        i = 2 * blk
        for (r, c, v) in ((i, i, 2.0), (i, i + 1, 1.0), (i + 1, i, 1.0), (i + 1, i + 1, 2.0)):
            rows.append(r), cols.append(c), vals.append(v)
    for k in range(n4):
        i = 2 * n_blocks + k
        rows.append(i), cols.append(i), vals.append(4.0)
    n = 2 * n_blocks + n4
    order = np.lexsort((cols, rows))
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))])
    b = fegen.random_vector(n, 3)
    x, info = oracle.fcg(rowptr, np.array(cols)[order], np.array(vals)[order], b, tol=1e-13,
                         inner_steps=1, storage="f64")
    assert info["status"] == "converged" and info["iters"] == 3
    # a diagonal matrix: S A S = I, the (FP64) inner solve is exact, one outer step
    d = np.arange(1, 10, dtype=float)
    bd = fegen.random_vector(9, 4)
    x, info = oracle.fcg(np.arange(10), np.arange(9), d, bd, tol=1e-14, inner_steps=3, storage="f64")
    assert info["iters"] == 1 and np.allclose(x, bd / d, rtol=1e-14)


@pytest.mark.parametrize("storage", ["bf16", "f32"])
def test_fcg_low_precision_inner_matches_dense_solve(storage):
    p = fegen.cube_elasticity(4, 24)
    A = dense_of(p.rowptr, p.colind, p.values, p.n_rows)
    b = fegen.random_vector(p.n_rows, 25)
    x, info = oracle.fcg(p.rowptr, p.colind, p.values, b, tol=1e-12, inner_steps=6, storage=storage)
    assert info["status"] == "converged" and info["true_relres"] <= 1e-12
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 10 * np.linalg.cond(A) * 1e-12
    # the inner steps pay: fewer outer steps than Jacobi-PCG's iterations
    _, io = oracle.pcg(p.rowptr, p.colind, p.values, b, tol=1e-12)
    assert info["iters"] < io["iters"] / 2
