// Host planner: locality order, windowed row-length sort, symmetric renumbering
// with sorted columns, and warp-slice packing.
//
// Paper mapping (arXiv:1501.00324):
//   Sec. 5.1 (ELL-WARP, K1): sort rows by length, group 32 rows per warp, pad
//            each warp to its own longest row, store column-major.
//   Sec. 5.2 (K1r): renumber x and the columns with the same permutation,
//            x'(.) = x(P(.)), c' = P^-1(c), so results need no remap on store.
//   Sec. 5.3 (K1rs): sort the renumbered columns inside each row, moving the
//            values with them.
//   Sec. 5.4 (K2): with a threshold tau, a 32-row group whose longest row
//            needs more than tau steps per lane gets T = 2, 4, ... 32 lanes per
//            row (T the smallest power of two with ceil(maxlen/T) <= tau) and
//            splits into T warps of 32/T rows.
// Design choices of this library (not in the paper): the length sort is stable
// and confined to windows of `sigma` rows of a locality order (the Morton curve
// of the node coordinates, dofs of a node kept adjacent), so that rows handled
// by one warp stay close in the mesh and their x gathers share cache lines; and
// each lane reads V consecutive entries per load (V = 1 is the paper's layout).
//
// Compiled with -ffp-contract=off: the Morton quantisation is a floating-point
// decision that must round the same way as the reference definition.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace fespmv {

static const int kMortonBits = 21;

int validate_csr(int64_t n, const int64_t* rowptr, const int32_t* colind) {
    if (rowptr[0] != 0) {
        set_error("rowptr[0] = %lld, expected 0", (long long)rowptr[0]);
        return FESPMV_ERR_BAD_CSR;
    }
    for (int64_t i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) {
            set_error("rowptr decreases at row %lld", (long long)i);
            return FESPMV_ERR_BAD_CSR;
        }
    const int64_t nnz = rowptr[n];
    for (int64_t p = 0; p < nnz; ++p)
        if (colind[p] < 0 || (int64_t)colind[p] >= n) {
            set_error("column index %d at position %lld outside [0, %lld)", colind[p],
                      (long long)p, (long long)n);
            return FESPMV_ERR_BAD_CSR;
        }
    return FESPMV_OK;
}

// Nodes in Morton order of their coordinates (ties by node number).
static void morton_node_order(int64_t n_nodes, const double* xyz, std::vector<int64_t>& order) {
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = hi[d] = n_nodes ? xyz[d] : 0.0;
    }
    for (int64_t i = 0; i < n_nodes; ++i)
        for (int d = 0; d < 3; ++d) {
            double v = xyz[i * 3 + d];
            if (v < lo[d]) lo[d] = v;
            if (v > hi[d]) hi[d] = v;
        }
    const double scale = (double)((1u << kMortonBits) - 1u);
    std::vector<uint64_t> code((size_t)n_nodes);
    for (int64_t i = 0; i < n_nodes; ++i) {
        uint64_t q[3];
        for (int d = 0; d < 3; ++d) {
            if (hi[d] > lo[d]) {
                double t = (xyz[i * 3 + d] - lo[d]) / (hi[d] - lo[d]);
                t = t * scale;
                q[d] = (uint64_t)std::floor(t);
            } else {
                q[d] = 0;
            }
        }
        uint64_t c = 0;
        for (int b = 0; b < kMortonBits; ++b)
            for (int d = 0; d < 3; ++d) c |= ((q[d] >> b) & 1ull) << (3 * b + (2 - d));
        code[(size_t)i] = c;
    }
    order.resize((size_t)n_nodes);
    std::iota(order.begin(), order.end(), (int64_t)0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return code[(size_t)a] < code[(size_t)b]; });
}

int order_and_permute(int64_t n, const int64_t* rowptr, const int32_t* colind, int dpn,
                      const double* node_xyz, int reorder, int sigma, Permuted& out, bool node_sort,
                      int col_order) {
    if (dpn <= 0) dpn = 1;
    if (n % dpn != 0) {
        set_error("n_rows %lld is not a multiple of dofs_per_node %d", (long long)n, dpn);
        return FESPMV_ERR_INVALID_ARG;
    }
    const int64_t n_nodes = n / dpn;

    // 1. locality order of nodes, expanded to rows (dofs of a node adjacent)
    std::vector<int64_t> nodes;
    if (reorder == FESPMV_REORDER_MORTON && node_xyz) {
        morton_node_order(n_nodes, node_xyz, nodes);
    } else {
        nodes.resize((size_t)n_nodes);
        std::iota(nodes.begin(), nodes.end(), (int64_t)0);
    }
    // 2a. (node_sort) stable longest-first sort of whole nodes inside windows of
    //     ceil(sigma / dpn) nodes, a node's length being its longest row
    if (node_sort && sigma > 0) {
        const int64_t wn = (sigma + dpn - 1) / dpn;
        auto len = [&](int64_t node) {
            int64_t m = 0;
            for (int c = 0; c < dpn; ++c) m = std::max(m, rowptr[node * dpn + c + 1] - rowptr[node * dpn + c]);
            return m;
        };
        for (int64_t s = 0; s < n_nodes; s += wn) {
            int64_t e = std::min<int64_t>(n_nodes, s + wn);
            std::stable_sort(nodes.begin() + s, nodes.begin() + e,
                             [&](int64_t a, int64_t b) { return len(a) > len(b); });
        }
    }
    out.perm.resize((size_t)n);
    for (int64_t k = 0; k < n_nodes; ++k)
        for (int c = 0; c < dpn; ++c) out.perm[(size_t)(k * dpn + c)] = (int32_t)(nodes[(size_t)k] * dpn + c);

    // 2. stable longest-first sort inside windows of sigma rows
    if (sigma > 0 && !node_sort) {
        for (int64_t s = 0; s < n; s += sigma) {
            int64_t e = std::min<int64_t>(n, s + sigma);
            std::stable_sort(out.perm.begin() + s, out.perm.begin() + e, [&](int32_t a, int32_t b) {
                return (rowptr[a + 1] - rowptr[a]) > (rowptr[b + 1] - rowptr[b]);
            });
        }
    }
    out.pinv.assign((size_t)n, 0);
    for (int64_t i = 0; i < n; ++i) out.pinv[(size_t)out.perm[(size_t)i]] = (int32_t)i;

    // 3. permuted rows with renumbered, sorted columns: (new col, input position)
    out.rp2.assign((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = out.perm[(size_t)i];
        out.rp2[(size_t)i + 1] = out.rp2[(size_t)i] + (rowptr[o + 1] - rowptr[o]);
    }
    const int64_t nnz = out.rp2[(size_t)n];
    out.c2.resize((size_t)nnz);
    out.s2.resize((size_t)nnz);
    out.diagpos.assign((size_t)n, -1);
    std::vector<std::pair<int32_t, int64_t>> row;
    std::vector<int32_t> seen;
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = out.perm[(size_t)i];
        row.clear();
        // K1 keeps the input's column numbers; K1r / K1rs renumber them (c' = P^-1[c])
        for (int64_t p = rowptr[o]; p < rowptr[o + 1]; ++p)
            row.emplace_back(col_order == FESPMV_COLS_ORIGINAL ? colind[p] : out.pinv[(size_t)colind[p]], p);
        if (col_order == FESPMV_COLS_SORTED) {
            std::sort(row.begin(), row.end());
        }
        seen.clear();
        for (const auto& e : row) seen.push_back(e.first);
        std::sort(seen.begin(), seen.end());
        for (size_t k = 1; k < seen.size(); ++k)
            if (seen[k] == seen[k - 1]) {
                set_error("duplicate column in row %lld", (long long)o);
                return FESPMV_ERR_BAD_CSR;
            }
        // the diagonal: new column i, or old column o when columns keep the input numbering
        const int32_t dcol = col_order == FESPMV_COLS_ORIGINAL ? (int32_t)o : (int32_t)i;
        for (size_t k = 0; k < row.size(); ++k) {
            out.c2[(size_t)out.rp2[(size_t)i] + k] = row[k].first;
            out.s2[(size_t)out.rp2[(size_t)i] + k] = row[k].second;
            if (row[k].first == dcol) out.diagpos[(size_t)i] = row[k].second;
        }
    }
    return FESPMV_OK;
}

int pack_slices(const std::vector<int64_t>& rp2, const std::vector<int32_t>& c2,
                const std::vector<int64_t>& s2, int threshold, int V, Plan& out, bool with_ppos) {
    const int64_t n = (int64_t)rp2.size() - 1;
    // slice plan: per 32-row group choose T, split into T warps of 32/T rows
    struct Slice { int64_t r0; int nr; int T; int64_t w; };
    std::vector<Slice> slices;
    for (int64_t g0 = 0; g0 < n; g0 += 32) {
        int m = (int)std::min<int64_t>(32, n - g0);
        int64_t maxlen = 0;
        for (int r = 0; r < m; ++r) maxlen = std::max(maxlen, rp2[(size_t)(g0 + r + 1)] - rp2[(size_t)(g0 + r)]);
        int T = 1;
        if (threshold > 0)
            while (T < 32 && (maxlen + T - 1) / T > threshold) T *= 2;
        int rpw = 32 / T;
        for (int j = 0; j < T; ++j) {
            int64_t r0 = g0 + (int64_t)j * rpw;
            if (r0 >= g0 + m) break;
            int nr = (int)std::min<int64_t>(rpw, g0 + m - r0);
            int64_t ml = 0;
            for (int r = 0; r < nr; ++r) ml = std::max(ml, rp2[(size_t)(r0 + r + 1)] - rp2[(size_t)(r0 + r)]);
            int64_t w = (ml + T - 1) / T;
            w = (w + V - 1) / V * V;
            slices.push_back({r0, nr, T, w});
        }
    }
    out.n_slices = (int64_t)slices.size();
    int64_t total = 0;
    for (const Slice& s : slices) total += 32 * s.w;
    if (total / 32 > (int64_t)UINT32_MAX || n > (int64_t)UINT32_MAX) {
        set_error("packed matrix too large for 32-bit slice offsets");
        return FESPMV_ERR_UNSUPPORTED;
    }
    out.packed_len = total;
    out.col.assign((size_t)total, -1);
    out.src.assign((size_t)total, -1);
    out.meta.assign((size_t)out.n_slices * 4, 0);
    if (with_ppos) out.ppos.assign(c2.size(), -1);
    int64_t off = 0;
    for (size_t si = 0; si < slices.size(); ++si) {
        const Slice& s = slices[si];
        int lt = 0;
        while ((1 << lt) < s.T) ++lt;
        out.meta[si * 4 + 0] = (uint32_t)(off / 32);
        out.meta[si * 4 + 1] = (uint32_t)s.w;
        out.meta[si * 4 + 2] = (uint32_t)s.r0;
        out.meta[si * 4 + 3] = (uint32_t)lt;
        for (int r = 0; r < s.nr; ++r) {
            int64_t a = rp2[(size_t)(s.r0 + r)], b = rp2[(size_t)(s.r0 + r + 1)];
            for (int64_t k = 0; k < b - a; ++k) {
                int64_t lane = (int64_t)r * s.T + k % s.T;
                int64_t step = k / s.T;
                int64_t pos = off + (step / V) * 32 * V + lane * V + step % V;
                out.col[(size_t)pos] = c2[(size_t)(a + k)];
                out.src[(size_t)pos] = s2[(size_t)(a + k)];
                if (with_ppos) out.ppos[(size_t)(a + k)] = pos;
            }
        }
        off += 32 * s.w;
    }
    return FESPMV_OK;
}

bool build_tiles(const std::vector<uint32_t>& meta, const std::vector<int32_t>& col, int64_t n,
                 int max_slices, int max_cols, Tiles& out) {
    const int64_t ns = (int64_t)meta.size() / 4;
    out = Tiles();
    out.lidx.assign(col.size(), 0);
    std::vector<int32_t> tile_of((size_t)n, -1), seen((size_t)n, -1), local((size_t)n, 0);
    int32_t tile = -1;
    int D = 0, first = 0, count = 0;
    auto slice_range = [&](int64_t sl, int64_t& b, int64_t& e) {
        b = (int64_t)meta[(size_t)sl * 4] * 32;
        e = b + 32 * (int64_t)meta[(size_t)sl * 4 + 1];
    };
    auto close = [&]() {
        out.tiles.insert(out.tiles.end(), {first, count, (int32_t)(out.dict.size() - (size_t)D), D});
        out.dmax = std::max(out.dmax, D);
        for (int64_t sl = first; sl < (int64_t)first + count; ++sl) {  // padding -> zero slot D
            int64_t b, e;
            slice_range(sl, b, e);
            for (int64_t p = b; p < e; ++p)
                if (col[(size_t)p] < 0) out.lidx[(size_t)p] = (uint16_t)D;
        }
    };
    for (int64_t sl = 0; sl < ns; ++sl) {
        int64_t b, e;
        slice_range(sl, b, e);
        if (count == 0) {  // open a tile
            ++tile;
            D = 0;
            first = (int)sl;
        }
        int fresh = 0;  // distinct columns of the slice not yet in the tile
        for (int64_t p = b; p < e; ++p) {
            const int32_t c = col[(size_t)p];
            if (c >= 0 && tile_of[(size_t)c] != tile && seen[(size_t)c] != (int32_t)sl) {
                seen[(size_t)c] = (int32_t)sl;
                ++fresh;
            }
        }
        if (count > 0 && (count == max_slices || D + fresh > max_cols)) {
            close();
            ++tile;
            D = 0;
            first = (int)sl;
            count = 0;
            fresh = 0;
            for (int64_t p = b; p < e; ++p) {
                const int32_t c = col[(size_t)p];
                if (c >= 0 && seen[(size_t)c] != (int32_t)(-2 - sl)) {
                    seen[(size_t)c] = (int32_t)(-2 - sl);
                    ++fresh;
                }
            }
        }
        if (fresh > max_cols) {
            out = Tiles();
            return false;
        }
        for (int64_t p = b; p < e; ++p) {
            const int32_t c = col[(size_t)p];
            if (c < 0) continue;
            if (tile_of[(size_t)c] != tile) {
                tile_of[(size_t)c] = tile;
                local[(size_t)c] = D++;
                out.dict.push_back(c);
            }
            out.lidx[(size_t)p] = (uint16_t)local[(size_t)c];
        }
        ++count;
    }
    if (count > 0) close();
    return true;
}

// The node blocks of Sec. 5's slices for 3-dof nodes: block row I holds rows
// 3I..3I+2, its blocks are the column nodes J any of them touches (ascending),
// one block row per lane, 32 per slice, padded to the slice's longest block row.
int pack_node_blocks(const std::vector<int64_t>& rp2, const std::vector<int32_t>& c2,
                     const std::vector<int64_t>& ppos, NodeBlocks& out) {
    const int64_t n = (int64_t)rp2.size() - 1;
    if (n % 3 != 0) {
        set_error("node blocks need n_rows divisible by 3 (got %lld)", (long long)n);
        return FESPMV_ERR_INVALID_ARG;
    }
    const int64_t nn = n / 3;
    // block columns of every node row
    std::vector<int64_t> bp((size_t)nn + 1, 0);
    std::vector<int32_t> bc;
    std::vector<int32_t> cols;
    for (int64_t I = 0; I < nn; ++I) {
        cols.clear();
        for (int a = 0; a < 3; ++a)
            for (int64_t p = rp2[(size_t)(3 * I + a)]; p < rp2[(size_t)(3 * I + a + 1)]; ++p)
                cols.push_back(c2[(size_t)p] / 3);
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
        bc.insert(bc.end(), cols.begin(), cols.end());
        bp[(size_t)I + 1] = (int64_t)bc.size();
    }
    out = NodeBlocks();
    out.n_slices = (nn + 31) / 32;
    out.meta.assign((size_t)out.n_slices * 4, 0);
    int64_t total = 0;
    for (int64_t s = 0; s < out.n_slices; ++s) {
        int64_t w = 0;
        for (int64_t I = 32 * s; I < std::min<int64_t>(nn, 32 * s + 32); ++I)
            w = std::max(w, bp[(size_t)I + 1] - bp[(size_t)I]);
        out.meta[(size_t)s * 4 + 0] = (uint32_t)(total / 32);
        out.meta[(size_t)s * 4 + 1] = (uint32_t)w;
        out.meta[(size_t)s * 4 + 2] = (uint32_t)(32 * s);
        total += 32 * w;
    }
    if (total / 32 > (int64_t)UINT32_MAX) {
        set_error("node blocks too large for 32-bit slice offsets");
        return FESPMV_ERR_UNSUPPORTED;
    }
    out.len = total;
    out.col.assign((size_t)total, -1);
    out.map.assign((size_t)total * 9, -1);
    for (int64_t s = 0; s < out.n_slices; ++s) {
        const int64_t off = 32 * (int64_t)out.meta[(size_t)s * 4], w = out.meta[(size_t)s * 4 + 1];
        for (int64_t I = 32 * s; I < std::min<int64_t>(nn, 32 * s + 32); ++I) {
            const int64_t lane = I - 32 * s;
            for (int64_t k = bp[(size_t)I]; k < bp[(size_t)I + 1]; ++k) {
                const int64_t step = k - bp[(size_t)I];
                out.col[(size_t)(off + 32 * step + lane)] = bc[(size_t)k];
            }
            // the entries of the three rows, each to its block's value slot
            for (int a = 0; a < 3; ++a) {
                int64_t k = bp[(size_t)I];
                for (int64_t p = rp2[(size_t)(3 * I + a)]; p < rp2[(size_t)(3 * I + a + 1)]; ++p) {
                    const int32_t J = c2[(size_t)p] / 3, b = c2[(size_t)p] % 3;
                    while (bc[(size_t)k] != J) ++k;   // columns ascend within the row
                    const int64_t step = k - bp[(size_t)I];
                    out.map[(size_t)(9 * (off + 32 * step) + 32 * (3 * a + b) + lane)] = ppos[(size_t)p];
                }
            }
        }
    }
    return FESPMV_OK;
}

int build_plan(int64_t n, const int64_t* rowptr, const int32_t* colind, int dpn,
               const double* node_xyz, int reorder, int sigma, int threshold, int V, Plan& out,
               NodeBlocks* nb, int col_order) {
    Permuted pm;
    int rc = order_and_permute(n, rowptr, colind, dpn, node_xyz, reorder, sigma, pm, nb != nullptr, col_order);
    if (rc) return rc;
    rc = pack_slices(pm.rp2, pm.c2, pm.s2, threshold, V, out, nb != nullptr);
    if (rc) return rc;
    if (nb) {
        if ((rc = pack_node_blocks(pm.rp2, pm.c2, out.ppos, *nb))) return rc;
        // tiles of up to 8 node-block slices whose column nodes (at most 2048) are staged
        build_tiles(nb->meta, nb->col, n / 3, 8, 2048, nb->tiles);
    }
    out.perm.swap(pm.perm);
    out.pinv.swap(pm.pinv);
    out.diagpos.swap(pm.diagpos);
    return FESPMV_OK;
}

}  // namespace fespmv
