"""Reference definitions of the reordering and packing (TEST INFRASTRUCTURE).

Plain numpy statements of the integer work the library does on the host before
any kernel runs; the tests compare the library's exported arrays with these bit
for bit.  Nothing here is imported by the product path.

Paper mapping:

* Row sort (Sec. 5.1, ELL-WARP): rows are sorted by length, longest first.  Here
  the sort is stable and confined to windows of ``sigma`` rows of a locality
  order (sigma >= n_rows reproduces the paper's global sort).
* Symmetric renumbering (Sec. 5.2, K1r): x'(.) = x(P(.)), c'(.) = P^-1(c(.)),
  i.e. new column index = Pinv[old column]; the worked example of Sec. 5.2
  (P = [2 5 7 3 1 4 6], c = [1 2 4 5 6] -> c' = [5 1 6 2 7]) pins this reading.
* Sorted columns (Sec. 5.3, K1rs): within each row, entries are ordered by the
  new column index and the values move with them.
* Warp slices (Sec. 5.1 and Sec. 5.4, K1/K2): 32 consecutive rows form a group;
  with threshold tau > 0 the group's rows get T lanes each, T the smallest power
  of two with ceil(maxlen/T) <= tau (at most 32), and the group splits into T
  warps of 32/T rows.  tau = 0 is K1 (T = 1).  Each warp's entries are padded
  to its own width and stored "column-major": entry k of local row r goes to
  lane r*T + k%T, step k//T.  Steps are grouped V at a time so that each lane
  reads V consecutive entries (V = 1 is the paper's layout).

Layout of one slice (warp), width w steps (a multiple of V), offset ``off``::

    position(lane, step) = off + (step // V) * 32 * V + lane * V + step % V

Padding entries hold value 0 and column -1.  The per-slice metadata row is
``(off // 32, w, first_row, log2 T)`` as uint32.

Tiles (this library's x staging, not in the paper): slices are taken in order
and grouped greedily into runs of at most ``max_slices`` slices whose distinct
columns number at most ``max_cols``; a tile's dictionary lists its distinct
columns in order of first use (packed order), and each packed entry stores its
column's index in that list (padding: the list's length).  A slice that alone
has more than ``max_cols`` distinct columns means no tiles at all.

The locality order (a design choice of this library, not the paper's) is the
Morton (Z-order) curve of the node coordinates: each coordinate is mapped to
q = floor((x - min) / (max - min) * 2097151) (q = 0 on a flat axis), the 21
bits of (qx, qy, qz) are interleaved with x the most significant, and nodes are
sorted by (code, node number).  The dofs of a node stay adjacent.
"""
from __future__ import annotations

import numpy as np

MORTON_BITS = 21
MORTON_SCALE = float((1 << MORTON_BITS) - 1)


def worked_example_renumber(c: np.ndarray, P: np.ndarray):
    """Sec. 5.2 renumbering for 1-based arrays: returns (c', x-permutation).

    c'_k = Pinv[c_k] where Pinv is the inverse of P (both 1-based)."""
    P = np.asarray(P)
    Pinv = np.empty_like(P)
    Pinv[P - 1] = np.arange(1, len(P) + 1)
    return Pinv[np.asarray(c) - 1]


def morton_codes(node_xyz: np.ndarray) -> np.ndarray:
    xyz = np.asarray(node_xyz, dtype=np.float64)
    q = np.zeros(xyz.shape, dtype=np.uint64)
    for d in range(3):
        lo = xyz[:, d].min()
        hi = xyz[:, d].max()
        if hi > lo:
            t = (xyz[:, d] - lo) / (hi - lo) * MORTON_SCALE
            q[:, d] = np.floor(t).astype(np.uint64)
    code = np.zeros(xyz.shape[0], dtype=np.uint64)
    for b in range(MORTON_BITS):
        for d in range(3):
            bit = (q[:, d] >> np.uint64(b)) & np.uint64(1)
            code |= bit << np.uint64(3 * b + (2 - d))
    return code


def node_order(node_xyz, n_nodes: int, reorder: str) -> np.ndarray:
    """Node numbers in locality order ('none' keeps the input order)."""
    if reorder == "none" or node_xyz is None:
        return np.arange(n_nodes, dtype=np.int64)
    if reorder == "morton":
        code = morton_codes(node_xyz)
        return np.lexsort((np.arange(n_nodes), code)).astype(np.int64)
    raise ValueError(reorder)


def row_permutation(rowptr: np.ndarray, dofs_per_node: int, node_xyz=None,
                    reorder: str = "morton", sigma: int = 0) -> np.ndarray:
    """P with P[new_row] = old_row: locality order, then a stable longest-first
    sort inside consecutive windows of sigma rows (sigma = 0: no length sort)."""
    n = len(rowptr) - 1
    d = dofs_per_node
    assert n % d == 0
    nodes = node_order(node_xyz, n // d, reorder)
    P = (nodes[:, None] * d + np.arange(d)[None, :]).ravel()
    if sigma > 0:
        lens = np.diff(rowptr)[P]
        out = np.empty_like(P)
        for s in range(0, n, sigma):
            seg = slice(s, min(n, s + sigma))
            order = np.argsort(-lens[seg], kind="stable")
            out[seg] = P[seg][order]
        P = out
    return P.astype(np.int64)


def inverse(P: np.ndarray) -> np.ndarray:
    Pinv = np.empty_like(P)
    Pinv[P] = np.arange(len(P), dtype=P.dtype)
    return Pinv


def permute_csr(rowptr, colind, values, P, col_order: str = "sorted"):
    """Row-permuted CSR: rows in the order P.  col_order 'sorted' (K1rs, Sec. 5.3):
    columns renumbered by Pinv and sorted per row; 'renumbered' (K1r, Sec. 5.2):
    renumbered, each row in the input's order; 'original' (K1, Sec. 5.1): the
    input's column numbers and order.

    Returns (rowptr2, colind2, values2, vmap) with vmap[old_position] =
    position of the same entry in the permuted CSR."""
    n = len(rowptr) - 1
    Pinv = inverse(P)
    lens = np.diff(rowptr)
    lens2 = lens[P]
    rowptr2 = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens2, out=rowptr2[1:])
    nnz = int(rowptr[-1])
    old_row = np.repeat(np.arange(n), lens)
    new_row = Pinv[old_row]
    if col_order == "original":
        new_col = colind.astype(np.int64)
    else:
        new_col = Pinv[colind.astype(np.int64)]
    if col_order == "sorted":
        order = np.lexsort((new_col, new_row))       # row-major, columns ascending
    else:
        order = np.lexsort((np.arange(nnz), new_row))  # row-major, the input's order in a row
    colind2 = new_col[order].astype(np.int32)
    values2 = np.asarray(values)[order]
    vmap = np.empty(nnz, dtype=np.int64)
    vmap[order] = np.arange(nnz, dtype=np.int64)
    return rowptr2, colind2, values2, vmap


def slice_plan(rowptr2, threshold: int = 0, V: int = 2):
    """Per-slice (first_row, n_rows, T, width) following the K1/K2 rule."""
    n = len(rowptr2) - 1
    lens = np.diff(rowptr2)
    slices = []
    for g0 in range(0, n, 32):
        m = min(32, n - g0)
        maxlen = int(lens[g0:g0 + m].max()) if m else 0
        T = 1
        if threshold > 0:
            while T < 32 and -(-maxlen // T) > threshold:
                T *= 2
        rpw = 32 // T
        for j in range(T):
            r0 = g0 + j * rpw
            if r0 >= g0 + m:
                break
            nr = min(rpw, g0 + m - r0)
            ml = int(lens[r0:r0 + nr].max())
            w = -(-ml // T)
            w = -(-w // V) * V
            slices.append((r0, nr, T, w))
    return slices


def pack(rowptr2, colind2, values2, threshold: int = 0, V: int = 2):
    """Packed slice arrays of the permuted CSR.

    Returns (meta uint32 [S,4], col int32 [L], val float64 [L], pmap int64 [nnz])
    with pmap[permuted CSR position] = packed position."""
    slices = slice_plan(rowptr2, threshold, V)
    total = sum(32 * w for (_, _, _, w) in slices)
    col = np.full(total, -1, dtype=np.int32)
    val = np.zeros(total, dtype=np.asarray(values2).dtype)
    pmap = np.empty(int(rowptr2[-1]), dtype=np.int64)
    meta = np.zeros((len(slices), 4), dtype=np.uint32)
    off = 0
    for s, (r0, nr, T, w) in enumerate(slices):
        meta[s] = (off // 32, w, r0, T.bit_length() - 1)
        for r in range(nr):
            a, b = int(rowptr2[r0 + r]), int(rowptr2[r0 + r + 1])
            k = np.arange(b - a)
            lane = r * T + k % T
            step = k // T
            pos = off + (step // V) * 32 * V + lane * V + step % V
            col[pos] = colind2[a:b]
            val[pos] = values2[a:b]
            pmap[a:b] = pos
        off += 32 * w
    return meta, col, val, pmap


def tiles(meta: np.ndarray, col: np.ndarray, max_slices: int = 8, max_cols: int = 4096):
    """Greedy tiles of consecutive slices; returns (tiles int32[n_tiles, 4] =
    (first slice, slices, dictionary offset, size D), dictionary int32[],
    index uint16[packed_len]) or None when one slice has too many columns."""
    meta = np.asarray(meta).reshape(-1, 4)
    col = np.asarray(col)
    out_tiles, out_dict = [], []
    index = np.zeros(len(col), dtype=np.uint16)
    pos = {}           # column -> index in the open tile's dictionary
    first, count = 0, 0

    def close():
        D = len(pos)
        out_tiles.append((first, count, len(out_dict) - D, D))
        for t in range(first, first + count):
            b = int(meta[t, 0]) * 32
            e = b + 32 * int(meta[t, 1])
            for p in range(b, e):
                if col[p] < 0:
                    index[p] = D

    for sl in range(len(meta)):
        b = int(meta[sl, 0]) * 32
        e = b + 32 * int(meta[sl, 1])
        cols = [int(c) for c in col[b:e] if c >= 0]
        distinct = set(cols)
        if len(distinct) > max_cols:
            return None
        fresh = distinct - set(pos)
        if count > 0 and (count == max_slices or len(pos) + len(fresh) > max_cols):
            close()
            pos, first, count = {}, sl, 0
        if count == 0:
            first = sl
        for p in range(b, e):
            c = int(col[p])
            if c < 0:
                continue
            if c not in pos:
                pos[c] = len(pos)
                out_dict.append(c)
            index[p] = pos[c]
        count += 1
    if count > 0:
        close()
    return (np.array(out_tiles, dtype=np.int32).reshape(-1, 4), np.array(out_dict, dtype=np.int32), index)


# ---------------------------------------------------------------------------
# 3x3 node blocks (this library's layout for three dofs per node; not in the
# paper, which stores one column per value).  The node locality order is sorted
# stably, longest first, inside windows of ceil(sigma / 3) nodes, a node's
# length being the longest of its three rows; its dofs stay at rows 3k + c.
# Block row I holds rows 3I..3I+2; its blocks are the column nodes J that any
# of those rows touches, ascending.  Slices: 32 node rows each (K1, one block
# row per lane), width = the longest block row of the slice, block (lane l, step
# s) at slot off + 32 s + l; each block's value k = 3a + b (row 3I+a, column
# 3J+b) at index 9 off + k (32 w) + 32 s + l, zero where the matrix stores no
# entry.  Metadata per slice: (off // 32, w, first node row, 0).

def node_row_permutation(rowptr: np.ndarray, node_xyz=None, reorder: str = "morton",
                         sigma: int = 0) -> np.ndarray:
    """P (P[new_row] = old_row) for 3 dofs per node with whole nodes sorted."""
    n = len(rowptr) - 1
    assert n % 3 == 0
    nn = n // 3
    nodes = node_order(node_xyz, nn, reorder)
    if sigma > 0:
        lens = np.diff(rowptr).reshape(nn, 3).max(axis=1)[nodes]
        wn = -(-sigma // 3)
        out = np.empty_like(nodes)
        for s in range(0, nn, wn):
            seg = slice(s, min(nn, s + wn))
            out[seg] = nodes[seg][np.argsort(-lens[seg], kind="stable")]
        nodes = out
    return (nodes[:, None] * 3 + np.arange(3)[None, :]).ravel().astype(np.int64)


def node_blocks(rowptr2, colind2):
    """Node-block arrays of a node-ordered permuted CSR: (meta uint32 [S,4],
    col int32 [L], vidx int64 [9L]) with vidx[value index] = permuted CSR
    position of that block value, -1 where the block stores a zero."""
    n = len(rowptr2) - 1
    assert n % 3 == 0
    nn = n // 3
    blocks = []
    for I in range(nn):
        a, b = int(rowptr2[3 * I]), int(rowptr2[3 * I + 3])
        blocks.append(sorted(set(int(c) // 3 for c in colind2[a:b])))
    S = -(-nn // 32)
    meta = np.zeros((S, 4), dtype=np.uint32)
    widths = []
    off = 0
    for s in range(S):
        rows = range(32 * s, min(nn, 32 * s + 32))
        w = max((len(blocks[I]) for I in rows), default=0)
        meta[s] = (off // 32, w, 32 * s, 0)
        widths.append(w)
        off += 32 * w
    col = np.full(off, -1, dtype=np.int32)
    vidx = np.full(9 * off, -1, dtype=np.int64)
    for s in range(S):
        o, w = int(meta[s, 0]) * 32, widths[s]
        for I in range(32 * s, min(nn, 32 * s + 32)):
            lane = I - 32 * s
            where = {J: st for st, J in enumerate(blocks[I])}
            for J, st in where.items():
                col[o + 32 * st + lane] = J
            for a in range(3):
                for p in range(int(rowptr2[3 * I + a]), int(rowptr2[3 * I + a + 1])):
                    J, b = divmod(int(colind2[p]), 3)
                    vidx[9 * (o + 32 * where[J]) + 32 * (3 * a + b) + lane] = p
    return meta, col, vidx
