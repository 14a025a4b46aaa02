// C ABI entry points (include/fespmv.h): handle lifetime, SpMV, permutation,
// value refresh and inspection.  Every entry point catches C++ exceptions and
// turns them into status codes.
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>

#include "internal.h"

namespace fespmv {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("%s failed: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FESPMV_ERR_OOM : FESPMV_ERR_CUDA;
}

int device_alloc(fespmv_mat* A, void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;  // keep every pointer valid for empty matrices
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMalloc(%zu bytes) for %s failed: %s", bytes, what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? FESPMV_ERR_OOM : FESPMV_ERR_CUDA;
    }
    A->device_bytes += (int64_t)bytes;
    return FESPMV_OK;
}

void free_handle(fespmv_mat* A) {
    if (!A) return;
    free_cg(A);
    free_multi_cg(A);
    void* ptrs[] = {A->d_rowptr, A->d_colind, A->d_val, A->d_meta, A->d_col, A->d_perm, A->d_pinv,
                    A->d_src, A->d_diagpos, A->d_diag, A->d_xp, A->d_yp, A->d_xh, A->d_yh,
                    A->d_vals_in, A->d_val32, A->d_val16, A->d_scale, A->d_flag, A->d_xs,
                    A->d_ys, A->d_xk, A->d_yk, A->d_vdf, A->d_xdf, A->d_tiles, A->d_tdict,
                    A->d_tlidx, A->d_xkdf, A->d_nbmeta, A->d_nbcol, A->d_nbmap, A->d_nb32, A->d_nb16,
                    A->d_nbtiles, A->d_nbtdict, A->d_nbtlidx};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete A;
}

static int ck(cudaError_t e, const char* what) {
    return e == cudaSuccess ? FESPMV_OK : cuda_fail(e, what);
}

#define TRY(expr)                 \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ != FESPMV_OK) {   \
            free_handle(A);       \
            return rc_;           \
        }                         \
    } while (0)

// Storage for S and the low-precision copies of S A S requested at create.
int alloc_scaled(fespmv_mat* A, int64_t len) {
    if (!(A->precisions & (FESPMV_PREC_F32 | FESPMV_PREC_BF16))) return FESPMV_OK;
    int rc = device_alloc(A, (void**)&A->d_scale, sizeof(double) * A->n, "scale S");
    if (!rc) rc = device_alloc(A, (void**)&A->d_flag, sizeof(int), "diagonal flag");
    if (!rc && (A->precisions & FESPMV_PREC_F32))
        rc = device_alloc(A, (void**)&A->d_val32, sizeof(float) * len, "FP32 values");
    if (!rc && (A->precisions & FESPMV_PREC_BF16))
        rc = device_alloc(A, (void**)&A->d_val16, sizeof(uint16_t) * len, "BF16 values");
    if (!rc) rc = device_alloc(A, (void**)&A->d_xs, sizeof(float) * A->n, "float x scratch");
    if (!rc) rc = device_alloc(A, (void**)&A->d_ys, sizeof(float) * A->n, "float y scratch");
    return rc;
}

// Device arrays of a SLICED handle from a host plan (perm/pinv/diagpos of n rows).
int upload_sliced(fespmv_mat* A, const Plan& plan, cudaStream_t s) {
    const int64_t n = A->n;
    A->n_slices = plan.n_slices;
    A->packed_len = plan.packed_len;
    A->max_lanes_log2 = 0;
    for (int64_t i = 0; i < plan.n_slices; ++i)
        A->max_lanes_log2 = std::max<int>(A->max_lanes_log2, (int)plan.meta[(size_t)i * 4 + 3]);
    int rc;
    if ((rc = device_alloc(A, (void**)&A->d_meta, sizeof(uint4) * plan.n_slices, "slice metadata")) ||
        (rc = device_alloc(A, (void**)&A->d_col, sizeof(int32_t) * plan.packed_len, "packed columns")) ||
        (rc = device_alloc(A, (void**)&A->d_val, sizeof(double) * plan.packed_len, "packed values")) ||
        (rc = device_alloc(A, (void**)&A->d_src, sizeof(int64_t) * plan.packed_len, "value map")) ||
        (rc = device_alloc(A, (void**)&A->d_perm, sizeof(int32_t) * n, "permutation")) ||
        (rc = device_alloc(A, (void**)&A->d_pinv, sizeof(int32_t) * n, "inverse permutation")) ||
        (rc = device_alloc(A, (void**)&A->d_xp, sizeof(double) * n, "permuted x")) ||
        (rc = device_alloc(A, (void**)&A->d_yp, sizeof(double) * n, "permuted y")) ||
        (rc = ck(cudaMemcpyAsync(A->d_meta, plan.meta.data(), sizeof(uint4) * plan.n_slices, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")) ||
        (rc = ck(cudaMemcpyAsync(A->d_col, plan.col.data(), sizeof(int32_t) * plan.packed_len, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")) ||
        (rc = ck(cudaMemcpyAsync(A->d_src, plan.src.data(), sizeof(int64_t) * plan.packed_len, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")) ||
        (rc = ck(cudaMemcpyAsync(A->d_perm, plan.perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")) ||
        (rc = ck(cudaMemcpyAsync(A->d_pinv, plan.pinv.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")) ||
        (rc = ck(cudaMemcpyAsync(A->d_diagpos, plan.diagpos.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")))
        return rc;
    return FESPMV_OK;
}

// Tile arrays of a SLICED handle (x staged through shared memory); leaves the
// handle untiled when a slice has more distinct columns than a tile holds.
static const int kTileSlices = 8, kTileCols = 4096;

int upload_tiles(fespmv_mat* A, const Plan& plan, Tiles& t, cudaStream_t s) {
    if (plan.n_slices == 0 || !build_tiles(plan.meta, plan.col, A->n, kTileSlices, kTileCols, t))
        return FESPMV_OK;
    A->n_tiles = (int64_t)t.tiles.size() / 4;
    A->tile_dmax = t.dmax;
    A->tile_dict_len = (int64_t)t.dict.size();
    int rc;
    if ((rc = device_alloc(A, (void**)&A->d_tiles, sizeof(int4) * (size_t)std::max<int64_t>(1, A->n_tiles), "tiles")) ||
        (rc = device_alloc(A, (void**)&A->d_tdict, sizeof(int32_t) * std::max<size_t>(1, t.dict.size()), "tile columns")) ||
        (rc = device_alloc(A, (void**)&A->d_tlidx, sizeof(uint16_t) * (size_t)std::max<int64_t>(1, plan.packed_len), "tile indices")) ||
        (rc = ck(cudaMemcpyAsync(A->d_tiles, t.tiles.data(), sizeof(int32_t) * t.tiles.size(), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")) ||
        (rc = ck(cudaMemcpyAsync(A->d_tdict, t.dict.data(), sizeof(int32_t) * t.dict.size(), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")) ||
        (rc = ck(cudaMemcpyAsync(A->d_tlidx, t.lidx.data(), sizeof(uint16_t) * t.lidx.size(), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")))
        return rc;
    A->tiled = 1;
    return FESPMV_OK;
}

// Node-block arrays of a SLICED handle (values filled by launch_nb3_refresh).
static int upload_node_blocks(fespmv_mat* A, const NodeBlocks& nb, bool tiles, cudaStream_t s) {
    A->nb_slices = nb.n_slices;
    A->nb_len = nb.len;
    const size_t len = (size_t)std::max<int64_t>(1, nb.len);
    int rc;
    if ((rc = device_alloc(A, (void**)&A->d_nbmeta, sizeof(uint4) * (size_t)std::max<int64_t>(1, nb.n_slices), "node-block slices")) ||
        (rc = device_alloc(A, (void**)&A->d_nbcol, sizeof(int32_t) * len, "node-block columns")) ||
        (rc = device_alloc(A, (void**)&A->d_nbmap, sizeof(int64_t) * 9 * len, "node-block map")) ||
        ((A->precisions & FESPMV_PREC_F32) &&
         (rc = device_alloc(A, (void**)&A->d_nb32, sizeof(float) * 9 * len, "node-block FP32 values"))) ||
        ((A->precisions & FESPMV_PREC_BF16) &&
         (rc = device_alloc(A, (void**)&A->d_nb16, sizeof(uint16_t) * 9 * len, "node-block BF16 values"))) ||
        (rc = ck(cudaMemcpyAsync(A->d_nbmeta, nb.meta.data(), sizeof(uint32_t) * nb.meta.size(), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")) ||
        (rc = ck(cudaMemcpyAsync(A->d_nbcol, nb.col.data(), sizeof(int32_t) * nb.col.size(), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")) ||
        (rc = ck(cudaMemcpyAsync(A->d_nbmap, nb.map.data(), sizeof(int64_t) * nb.map.size(), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")))
        return rc;
    const Tiles& t = nb.tiles;
    if (tiles && !t.tiles.empty()) {
        A->nb_tiles = (int64_t)t.tiles.size() / 4;
        A->nb_tile_dmax = t.dmax;
        A->nb_tile_dict_len = (int64_t)t.dict.size();
        if ((rc = device_alloc(A, (void**)&A->d_nbtiles, sizeof(int4) * (size_t)A->nb_tiles, "node-block tiles")) ||
            (rc = device_alloc(A, (void**)&A->d_nbtdict, sizeof(int32_t) * std::max<size_t>(1, t.dict.size()), "node-block tile nodes")) ||
            (rc = device_alloc(A, (void**)&A->d_nbtlidx, sizeof(uint16_t) * len, "node-block tile indices")) ||
            (rc = ck(cudaMemcpyAsync(A->d_nbtiles, t.tiles.data(), sizeof(int32_t) * t.tiles.size(), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")) ||
            (rc = ck(cudaMemcpyAsync(A->d_nbtdict, t.dict.data(), sizeof(int32_t) * t.dict.size(), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")) ||
            (rc = ck(cudaMemcpyAsync(A->d_nbtlidx, t.lidx.data(), sizeof(uint16_t) * t.lidx.size(), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync")))
            return rc;
    }
    A->nb = 3;
    return FESPMV_OK;
}

static bool pow2_upto32(int v) { return v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32; }

static int create_impl(fespmv_mat_t* out, int64_t n, const int64_t* rowptr, const int32_t* colind,
                       const double* values, const fespmv_mesh_info* mesh,
                       const fespmv_options* opts_in, cudaStream_t s) {
    if (!out) { set_error("out is NULL"); return FESPMV_ERR_INVALID_ARG; }
    *out = nullptr;
    if (n < 0 || n > (int64_t)INT32_MAX - 1) {
        set_error("n_rows %lld outside [0, 2^31-1)", (long long)n);
        return FESPMV_ERR_INVALID_ARG;
    }
    if (!rowptr || (n > 0 && rowptr[n] > 0 && (!colind || !values))) {
        set_error("rowptr, colind or values is NULL");
        return FESPMV_ERR_INVALID_ARG;
    }
    fespmv_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts_in) o = *opts_in;
    if (o.format != FESPMV_FMT_CSR && o.format != FESPMV_FMT_SLICED) {
        set_error("unknown format %d", o.format); return FESPMV_ERR_INVALID_ARG;
    }
    if (o.vec == 0) o.vec = 2;
    if (o.vec != 1 && o.vec != 2 && o.vec != 4) {
        set_error("vec must be 1, 2 or 4 (got %d)", o.vec); return FESPMV_ERR_INVALID_ARG;
    }
    if (o.csr_lanes == 0) o.csr_lanes = 1;
    if (!pow2_upto32(o.csr_lanes)) {
        set_error("csr_lanes must be a power of two <= 32 (got %d)", o.csr_lanes);
        return FESPMV_ERR_INVALID_ARG;
    }
    if (o.tiles < -1 || o.tiles > 0) {
        set_error("tiles must be 0 (on) or -1 (off) (got %d)", o.tiles); return FESPMV_ERR_INVALID_ARG;
    }
    if (o.block == 0) o.block = 256;
    if (o.block < 32 || o.block > 1024 || o.block % 32) {
        set_error("block must be a multiple of 32 in [32, 1024] (got %d)", o.block);
        return FESPMV_ERR_INVALID_ARG;
    }
    if (o.format == FESPMV_FMT_SLICED && o.block > 256) {
        set_error("SLICED kernels take at most 256 threads per block (got %d)", o.block);
        return FESPMV_ERR_INVALID_ARG;
    }
    if (o.sigma < 0 || o.threshold < 0) {
        set_error("sigma and threshold must be >= 0"); return FESPMV_ERR_INVALID_ARG;
    }
    if (o.reorder == FESPMV_REORDER_MORTON && (!mesh || !mesh->node_xyz) && o.format == FESPMV_FMT_SLICED) {
        set_error("REORDER_MORTON needs mesh->node_xyz"); return FESPMV_ERR_INVALID_ARG;
    }
    if (o.precisions & FESPMV_PREC_DF64 && o.format != FESPMV_FMT_SLICED) {
        set_error("FESPMV_PREC_DF64 needs a SLICED handle"); return FESPMV_ERR_INVALID_ARG;
    }
    if (o.precisions & ~(FESPMV_PREC_F64 | FESPMV_PREC_F32 | FESPMV_PREC_BF16 | FESPMV_PREC_DF64)) {
        set_error("unknown precision bits 0x%x", o.precisions); return FESPMV_ERR_INVALID_ARG;
    }
    if (o.col_order < FESPMV_COLS_SORTED || o.col_order > FESPMV_COLS_ORIGINAL) {
        set_error("unknown col_order %d", o.col_order); return FESPMV_ERR_INVALID_ARG;
    }
    if (o.col_order == FESPMV_COLS_ORIGINAL &&
        (o.format != FESPMV_FMT_SLICED || o.node_blocks || (o.precisions & ~FESPMV_PREC_F64))) {
        set_error("FESPMV_COLS_ORIGINAL: SLICED handles with FP64 values only");
        return FESPMV_ERR_INVALID_ARG;
    }
    if (o.node_blocks != 0 &&
        (o.node_blocks != 3 || o.format != FESPMV_FMT_SLICED || !mesh || mesh->dofs_per_node != 3 ||
         !(o.precisions & (FESPMV_PREC_F32 | FESPMV_PREC_BF16)))) {
        set_error("node_blocks = 3 needs a SLICED handle, dofs_per_node = 3 and FP32 or BF16 values (got %d)",
                  o.node_blocks);
        return FESPMV_ERR_INVALID_ARG;
    }
    int rc = validate_csr(n, rowptr, colind);
    if (rc) return rc;
    const int64_t nnz = rowptr[n];
    int dpn = (mesh && mesh->dofs_per_node > 0) ? mesh->dofs_per_node : 1;

    fespmv_mat* A = new fespmv_mat();
    A->n = n;
    A->nnz = nnz;
    A->format = o.format;
    A->block = o.block;
    A->csr_lanes = o.csr_lanes;
    A->vec = o.vec;
    A->precisions = o.precisions | FESPMV_PREC_F64;

    // values reach the device once; the packed array is filled by a gather kernel
    TRY(device_alloc(A, (void**)&A->d_vals_in, sizeof(double) * nnz, "input values"));
    TRY(ck(cudaMemcpyAsync(A->d_vals_in, values, sizeof(double) * nnz, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync"));
    TRY(device_alloc(A, (void**)&A->d_diagpos, sizeof(int64_t) * n, "diagonal map"));
    TRY(device_alloc(A, (void**)&A->d_diag, sizeof(double) * n, "diagonal"));

    if (o.format == FESPMV_FMT_CSR) {
        // check duplicates and locate diagonals
        std::vector<int64_t> diagpos((size_t)n, -1);
        std::vector<int32_t> cols;
        for (int64_t i = 0; i < n; ++i) {
            cols.assign(colind + rowptr[i], colind + rowptr[i + 1]);
            std::sort(cols.begin(), cols.end());
            for (size_t k = 1; k < cols.size(); ++k)
                if (cols[k] == cols[k - 1]) {
                    set_error("duplicate column %d in row %lld", cols[k], (long long)i);
                    free_handle(A);
                    return FESPMV_ERR_BAD_CSR;
                }
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
                if (colind[p] == i) diagpos[(size_t)i] = p;
        }
        TRY(device_alloc(A, (void**)&A->d_rowptr, sizeof(int64_t) * (n + 1), "rowptr"));
        TRY(device_alloc(A, (void**)&A->d_colind, sizeof(int32_t) * nnz, "colind"));
        TRY(device_alloc(A, (void**)&A->d_val, sizeof(double) * nnz, "values"));
        TRY(ck(cudaMemcpyAsync(A->d_rowptr, rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync"));
        TRY(ck(cudaMemcpyAsync(A->d_colind, colind, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync"));
        TRY(ck(cudaMemcpyAsync(A->d_diagpos, diagpos.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync"));
        TRY(alloc_scaled(A, nnz));
        TRY(launch_fill_values(A, A->d_vals_in, s));
        TRY(ck(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
    } else {
        Plan plan;
        NodeBlocks nb;   // host arrays stay alive until the stream synchronisation below
        A->col_order = o.col_order;
        TRY(build_plan(n, rowptr, colind, dpn, mesh ? mesh->node_xyz : nullptr, o.reorder, o.sigma,
                       o.threshold, o.vec, plan, o.node_blocks ? &nb : nullptr, o.col_order));
        TRY(upload_sliced(A, plan, s));
        if (o.node_blocks) TRY(upload_node_blocks(A, nb, o.tiles >= 0, s));
        Tiles tiles;  // host arrays stay alive until the stream synchronisation below
        if (o.tiles >= 0) TRY(upload_tiles(A, plan, tiles, s));
        if (A->precisions & FESPMV_PREC_DF64) {
            TRY(device_alloc(A, (void**)&A->d_vdf, sizeof(float2) * plan.packed_len, "float-pair values"));
            TRY(device_alloc(A, (void**)&A->d_xdf, sizeof(float2) * n, "float-pair x"));
        }
        TRY(alloc_scaled(A, plan.packed_len));
        TRY(launch_fill_values(A, A->d_vals_in, s));
        // host vectors must stay alive until the copies finish
        TRY(ck(cudaStreamSynchronize(s), "cudaStreamSynchronize"));
    }
    if (A->d_flag) {
        int bad = 0;
        TRY(ck(cudaMemcpy(&bad, A->d_flag, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy"));
        if (bad) {
            set_error("FP32/BF16 copies of S A S need a positive, finite diagonal");
            free_handle(A);
            return FESPMV_ERR_INVALID_ARG;
        }
    }
    cudaFree(A->d_vals_in);     // staging is re-allocated by spmv_update_values when needed
    A->device_bytes -= (int64_t)(nnz > 0 ? sizeof(double) * nnz : 16);
    A->d_vals_in = nullptr;
    *out = A;
    return FESPMV_OK;
}

}  // namespace fespmv

using namespace fespmv;

#define GUARD_BEGIN try {
#define GUARD_END                                                    \
    }                                                                \
    catch (const std::bad_alloc&) {                                  \
        set_error("host allocation failed");                         \
        return FESPMV_ERR_OOM;                                       \
    }                                                                \
    catch (...) {                                                    \
        set_error("unexpected C++ exception");                       \
        return FESPMV_ERR_INVALID_ARG;                               \
    }

extern "C" {

int spmv_create(fespmv_mat_t* out, int64_t n_rows, const int64_t* rowptr, const int32_t* colind,
                const double* values, const fespmv_mesh_info* mesh, const fespmv_options* opts,
                fespmv_stream_t stream) {
    GUARD_BEGIN
    return create_impl(out, n_rows, rowptr, colind, values, mesh, opts, (cudaStream_t)stream);
    GUARD_END
}

void spmv_destroy(fespmv_mat_t A) {
    try {
        free_handle(A);
    } catch (...) {
    }
}

static int ensure_host_staging(fespmv_mat* A) {
    if (!A->d_xh) {
        int rc = device_alloc(A, (void**)&A->d_xh, sizeof(double) * A->n, "host-I/O x");
        if (rc) return rc;
    }
    if (!A->d_yh) {
        int rc = device_alloc(A, (void**)&A->d_yh, sizeof(double) * A->n, "host-I/O y");
        if (rc) return rc;
    }
    return FESPMV_OK;
}

// Device address of a pinned (page-locked, mapped) host buffer, or nullptr for
// pageable memory and anything else.
static void* mapped_view(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int spmv_apply(fespmv_mat_t A, const double* x, double* y, int32_t flags, fespmv_stream_t stream) {
    GUARD_BEGIN
    if (!A || (A->n > 0 && (!x || !y))) { set_error("null argument"); return FESPMV_ERR_INVALID_ARG; }
    if (flags & ~(FESPMV_IO_PERMUTED | FESPMV_IO_HOST)) {
        set_error("unknown flags 0x%x", flags); return FESPMV_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (A->n == 0) return FESPMV_OK;
    if (A->col_order == FESPMV_COLS_ORIGINAL) {
        // K1: x in the input numbering feeds the kernel as it is; y leaves through P^-1
        if (flags & FESPMV_IO_PERMUTED) {
            set_error("a FESPMV_COLS_ORIGINAL handle reads x in the input numbering only");
            return FESPMV_ERR_UNSUPPORTED;
        }
        const double* xk = x;
        if (flags & FESPMV_IO_HOST) {
            int rc = ensure_host_staging(A);
            if (rc) return rc;
            FESPMV_CUDA(cudaMemcpyAsync(A->d_xh, x, sizeof(double) * A->n, cudaMemcpyHostToDevice, s));
            xk = A->d_xh;
        }
        double* yk = (flags & FESPMV_IO_HOST) ? A->d_yh : y;
        int rc;
        if ((rc = launch_spmv(A, xk, A->d_yp, s)) || (rc = launch_gather(A->d_yp, A->d_pinv, yk, A->n, s)))
            return rc;
        if (flags & FESPMV_IO_HOST) {
            FESPMV_CUDA(cudaMemcpyAsync(y, yk, sizeof(double) * A->n, cudaMemcpyDeviceToHost, s));
            FESPMV_CUDA(cudaStreamSynchronize(s));
        }
        return FESPMV_OK;
    }
    const double* xd = x;
    double* yd = y;
    if (A->format == FESPMV_FMT_SLICED && A->tiled && !A->d_vdf && !(flags & (FESPMV_IO_PERMUTED | FESPMV_IO_HOST)))
        // device x and y in the input numbering on a tiled handle: the permutations fold
        // into the product (x[P[c']] staged per tile, y[P[i']] stored per row)
        return launch_spmv_tiled_io(A, x, y, s);
    if ((flags & FESPMV_IO_HOST) && A->format == FESPMV_FMT_SLICED && !(flags & FESPMV_IO_PERMUTED) &&
        !A->d_vdf) {
        // pinned host buffers: the permutations read x and write y in place over the host link
        const double* xv = static_cast<const double*>(mapped_view(x));
        double* yv = static_cast<double*>(mapped_view(y));
        if (xv && yv) {
            int rc;
            if ((rc = launch_scatter(xv, A->d_pinv, A->d_xp, A->n, s)) ||
                (rc = launch_spmv(A, A->d_xp, A->d_yp, s)) ||
                (rc = launch_gather(A->d_yp, A->d_pinv, yv, A->n, s)))
                return rc;
            FESPMV_CUDA(cudaStreamSynchronize(s));
            return FESPMV_OK;
        }
    }
    if (flags & FESPMV_IO_HOST) {
        int rc = ensure_host_staging(A);
        if (rc) return rc;
        FESPMV_CUDA(cudaMemcpyAsync(A->d_xh, x, sizeof(double) * A->n, cudaMemcpyHostToDevice, s));
        xd = A->d_xh;
        yd = A->d_yh;
    }
    int rc;
    if (A->d_vdf) {   // float-pair FP64 product
        const double* xp = xd;
        if (!(flags & FESPMV_IO_PERMUTED)) {
            if ((rc = launch_gather_split(xd, A->d_perm, A->d_xp, A->d_xdf, A->n, s))) return rc;
            xp = A->d_xp;
        } else if ((rc = launch_split(xd, A->d_xdf, A->n, s))) {
            return rc;
        }
        double* yp = (flags & FESPMV_IO_PERMUTED) ? yd : A->d_yp;
        if ((rc = launch_spmv_df(A, A->d_xdf, xp, yp, s))) return rc;
        if (!(flags & FESPMV_IO_PERMUTED) && (rc = launch_gather(A->d_yp, A->d_pinv, yd, A->n, s))) return rc;
    } else if (A->format == FESPMV_FMT_SLICED && !(flags & FESPMV_IO_PERMUTED)) {
        if ((rc = launch_gather(xd, A->d_perm, A->d_xp, A->n, s))) return rc;
        if ((rc = launch_spmv(A, A->d_xp, A->d_yp, s))) return rc;
        if ((rc = launch_gather(A->d_yp, A->d_pinv, yd, A->n, s))) return rc;
    } else {
        if ((rc = launch_spmv(A, xd, yd, s))) return rc;
    }
    if (flags & FESPMV_IO_HOST) {
        FESPMV_CUDA(cudaMemcpyAsync(y, yd, sizeof(double) * A->n, cudaMemcpyDeviceToHost, s));
        FESPMV_CUDA(cudaStreamSynchronize(s));
    }
    return FESPMV_OK;
    GUARD_END
}

int spmv_apply_scaled(fespmv_mat_t A, const float* x, float* y, int32_t precision, int32_t flags,
                      fespmv_stream_t stream) {
    GUARD_BEGIN
    if (!A || (A->n > 0 && (!x || !y)) || (flags & ~FESPMV_IO_PERMUTED) ||
        (precision != FESPMV_PREC_F32 && precision != FESPMV_PREC_BF16)) {
        set_error("bad argument"); return FESPMV_ERR_INVALID_ARG;
    }
    if ((precision == FESPMV_PREC_F32 && !A->d_val32) || (precision == FESPMV_PREC_BF16 && !A->d_val16)) {
        set_error("the handle holds no %s copy (FESPMV_PREC_* at create)",
                  precision == FESPMV_PREC_F32 ? "FP32" : "BF16");
        return FESPMV_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (A->n == 0) return FESPMV_OK;
    int rc;
    if (A->format == FESPMV_FMT_SLICED && !(flags & FESPMV_IO_PERMUTED)) {
        if ((rc = launch_gather_f32(x, A->d_perm, A->d_xs, A->n, s))) return rc;
        if ((rc = launch_spmv_low(A, precision, A->d_xs, A->d_ys, s))) return rc;
        return launch_gather_f32(A->d_ys, A->d_pinv, y, A->n, s);
    }
    return launch_spmv_low(A, precision, x, y, s);
    GUARD_END
}

int spmv_permute(fespmv_mat_t A, const double* in, double* out, int32_t direction,
                 fespmv_stream_t stream) {
    GUARD_BEGIN
    if (!A || (A->n > 0 && (!in || !out)) || (direction != 0 && direction != 1)) {
        set_error("bad argument"); return FESPMV_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (A->n == 0) return FESPMV_OK;
    if (A->format != FESPMV_FMT_SLICED) {
        FESPMV_CUDA(cudaMemcpyAsync(out, in, sizeof(double) * A->n, cudaMemcpyDeviceToDevice, s));
        return FESPMV_OK;
    }
    return launch_gather(in, direction == 0 ? A->d_perm : A->d_pinv, out, A->n, s);
    GUARD_END
}

int spmv_update_values(fespmv_mat_t A, const double* values, int32_t flags, fespmv_stream_t stream) {
    GUARD_BEGIN
    if (!A || (A->nnz > 0 && !values) || (flags & ~FESPMV_IO_HOST)) {
        set_error("bad argument"); return FESPMV_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const double* src = values;
    if (flags & FESPMV_IO_HOST) {
        if (!A->d_vals_in) {
            int rc = device_alloc(A, (void**)&A->d_vals_in, sizeof(double) * A->nnz, "value staging");
            if (rc) return rc;
        }
        FESPMV_CUDA(cudaMemcpyAsync(A->d_vals_in, values, sizeof(double) * A->nnz, cudaMemcpyHostToDevice, s));
        src = A->d_vals_in;
    }
    int rc = launch_fill_values(A, src, s);
    if (rc) return rc;
    if (flags & FESPMV_IO_HOST) FESPMV_CUDA(cudaStreamSynchronize(s));
    return FESPMV_OK;
    GUARD_END
}

int spmv_plan(int64_t n, const int64_t* rowptr, const int32_t* colind, const fespmv_mesh_info* mesh,
              const fespmv_options* opts_in, fespmv_info* info, int32_t* perm, uint32_t* meta,
              int32_t* cols, int64_t* srcmap) {
    GUARD_BEGIN
    if (!rowptr || !info || n < 0 || n > (int64_t)INT32_MAX - 1) {
        set_error("bad argument"); return FESPMV_ERR_INVALID_ARG;
    }
    fespmv_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts_in) o = *opts_in;
    if (o.vec == 0) o.vec = 2;
    if ((o.vec != 1 && o.vec != 2 && o.vec != 4) || o.sigma < 0 || o.threshold < 0) {
        set_error("bad options"); return FESPMV_ERR_INVALID_ARG;
    }
    if (o.reorder == FESPMV_REORDER_MORTON && (!mesh || !mesh->node_xyz)) {
        set_error("REORDER_MORTON needs mesh->node_xyz"); return FESPMV_ERR_INVALID_ARG;
    }
    if (n > 0 && rowptr[n] > 0 && !colind) { set_error("colind is NULL"); return FESPMV_ERR_INVALID_ARG; }
    int rc = validate_csr(n, rowptr, colind);
    if (rc) return rc;
    const int dpn = (mesh && mesh->dofs_per_node > 0) ? mesh->dofs_per_node : 1;
    if (o.node_blocks != 0 && (o.node_blocks != 3 || dpn != 3)) {
        set_error("node_blocks = 3 needs dofs_per_node = 3"); return FESPMV_ERR_INVALID_ARG;
    }
    Plan plan;
    NodeBlocks nb;
    if (o.col_order < FESPMV_COLS_SORTED || o.col_order > FESPMV_COLS_ORIGINAL) {
        set_error("unknown col_order %d", o.col_order); return FESPMV_ERR_INVALID_ARG;
    }
    rc = build_plan(n, rowptr, colind, dpn, mesh ? mesh->node_xyz : nullptr, o.reorder, o.sigma, o.threshold,
                    o.vec, plan, o.node_blocks ? &nb : nullptr, o.col_order);
    if (rc) return rc;
    info->n_rows = n;
    info->nnz = rowptr[n];
    info->n_slices = plan.n_slices;
    info->packed_len = plan.packed_len;
    info->device_bytes = 0;
    info->format = FESPMV_FMT_SLICED;
    info->vec = o.vec;
    if (perm) std::memcpy(perm, plan.perm.data(), sizeof(int32_t) * (size_t)n);
    if (meta) std::memcpy(meta, plan.meta.data(), sizeof(uint32_t) * 4 * (size_t)plan.n_slices);
    if (cols) std::memcpy(cols, plan.col.data(), sizeof(int32_t) * (size_t)plan.packed_len);
    if (srcmap) std::memcpy(srcmap, plan.src.data(), sizeof(int64_t) * (size_t)plan.packed_len);
    return FESPMV_OK;
    GUARD_END
}

int spmv_plan_tiles(int64_t n, int64_t n_slices, const uint32_t* meta, int64_t packed_len,
                    const int32_t* cols, int32_t* tiles, int32_t* tile_cols, uint16_t* index,
                    int64_t* n_tiles, int64_t* n_tile_cols) {
    GUARD_BEGIN
    if (n < 0 || n_slices < 0 || packed_len < 0 || !n_tiles || !n_tile_cols ||
        (n_slices > 0 && !meta) || (packed_len > 0 && !cols)) {
        set_error("bad argument"); return FESPMV_ERR_INVALID_ARG;
    }
    for (int64_t sl = 0; sl < n_slices; ++sl) {
        const int64_t b = (int64_t)meta[sl * 4] * 32, e = b + 32 * (int64_t)meta[sl * 4 + 1];
        if (e > packed_len) { set_error("slice %lld outside the packed arrays", (long long)sl); return FESPMV_ERR_INVALID_ARG; }
    }
    for (int64_t q = 0; q < packed_len; ++q)
        if (cols[q] < -1 || (int64_t)cols[q] >= n) {
            set_error("column %d at position %lld out of range", cols[q], (long long)q);
            return FESPMV_ERR_INVALID_ARG;
        }
    std::vector<uint32_t> m(meta, meta + 4 * n_slices);
    std::vector<int32_t> c(cols, cols + packed_len);
    Tiles t;
    *n_tiles = 0;
    *n_tile_cols = 0;
    if (!build_tiles(m, c, n, kTileSlices, kTileCols, t)) return FESPMV_OK;
    *n_tiles = (int64_t)t.tiles.size() / 4;
    *n_tile_cols = (int64_t)t.dict.size();
    if (tiles) std::memcpy(tiles, t.tiles.data(), sizeof(int32_t) * t.tiles.size());
    if (tile_cols) std::memcpy(tile_cols, t.dict.data(), sizeof(int32_t) * t.dict.size());
    if (index) std::memcpy(index, t.lidx.data(), sizeof(uint16_t) * t.lidx.size());
    return FESPMV_OK;
    GUARD_END
}

int spmv_autotune(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* values,
                  const fespmv_mesh_info* mesh, fespmv_options* opts, int32_t reps, double* best_us,
                  int32_t* n_tried, fespmv_stream_t stream) {
    GUARD_BEGIN
    if (!opts || !rowptr || n < 0) { set_error("bad argument"); return FESPMV_ERR_INVALID_ARG; }
    if (reps <= 0) reps = 20;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = validate_csr(n, rowptr, colind);
    if (rc) return rc;
    int64_t maxlen = 0;
    for (int64_t i = 0; i < n; ++i) maxlen = std::max(maxlen, rowptr[i + 1] - rowptr[i]);
    std::vector<int> thresholds = {0};
    for (int64_t d : {4, 8}) {
        const int t = (int)std::max<int64_t>(1, (maxlen + d - 1) / d);
        if (t < maxlen && std::find(thresholds.begin(), thresholds.end(), t) == thresholds.end())
            thresholds.push_back(t);
    }
    double* x = nullptr;
    double* y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&] {
        if (x) cudaFree(x);
        if (y) cudaFree(y);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&x, sizeof(double) * std::max<int64_t>(n, 1)) != cudaSuccess ||
        cudaMalloc(&y, sizeof(double) * std::max<int64_t>(n, 1)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return cuda_fail(cudaGetLastError(), "spmv_autotune setup");
    }
    cudaMemsetAsync(x, 0, sizeof(double) * n, s);
    fespmv_options best = *opts;
    best.format = FESPMV_FMT_SLICED;
    double best_t = 1e300;
    int tried = 0;
    // the products are timed in the precision the caller will run: the FP32 (or BF16)
    // copy of S A S when the base options keep one, else FP64
    const int tprec = (opts->precisions & FESPMV_PREC_F32) ? FESPMV_PREC_F32
                    : (opts->precisions & FESPMV_PREC_BF16) ? FESPMV_PREC_BF16 : 0;
    auto product = [&](fespmv_mat_t A) {
        return tprec ? spmv_apply_scaled(A, reinterpret_cast<const float*>(x), reinterpret_cast<float*>(y), tprec,
                                         FESPMV_IO_PERMUTED, stream)
                     : spmv_apply(A, x, y, FESPMV_IO_PERMUTED, stream);
    };
    // layouts: x staged per tile (block fixed by the tiled kernels), or gathered from
    // cache with 128 or 256 threads per block; tiles only when the base options allow them
    struct Shape { int tiles, block; };
    std::vector<Shape> shapes;
    if (opts->tiles >= 0) shapes.push_back({0, 256});
    shapes.push_back({-1, 128});
    shapes.push_back({-1, 256});
    for (int vec : {1, 2, 4})
        for (int thr : thresholds)
            for (const Shape& sh : shapes) {
                fespmv_options o = *opts;
                o.format = FESPMV_FMT_SLICED;
                o.vec = vec;
                o.threshold = thr;
                o.block = sh.block;
                o.tiles = sh.tiles;
                o.precisions = FESPMV_PREC_F64 | tprec;
                fespmv_mat_t A = nullptr;
                rc = spmv_create(&A, n, rowptr, colind, values, mesh, &o, stream);
                if (rc) { cleanup(); return rc; }
                for (int w = 0; w < 2; ++w) rc |= product(A);
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps; ++r) rc |= product(A);
                cudaEventRecord(e1, s);
                cudaError_t e = cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                spmv_destroy(A);
                if (rc || e != cudaSuccess) {
                    cleanup();
                    return rc ? rc : cuda_fail(e, "spmv_autotune timing");
                }
                ++tried;
                const double us = 1e3 * ms / reps;
                if (us < best_t) {
                    best_t = us;
                    best = o;
                }
            }
    cleanup();
    opts->format = FESPMV_FMT_SLICED;
    opts->vec = best.vec;
    opts->threshold = best.threshold;
    opts->block = best.block;
    opts->tiles = best.tiles;
    if (best_us) *best_us = best_t;
    if (n_tried) *n_tried = tried;
    return FESPMV_OK;
    GUARD_END
}

int spmv_get_info(fespmv_mat_t A, fespmv_info* info) {
    if (!A || !info) { set_error("null argument"); return FESPMV_ERR_INVALID_ARG; }
    info->n_rows = A->n;
    info->nnz = A->nnz;
    info->n_slices = A->n_slices;
    info->packed_len = A->format == FESPMV_FMT_SLICED ? A->packed_len : A->nnz;
    info->device_bytes = A->device_bytes;
    info->format = A->format;
    info->vec = A->vec;
    info->n_tiles = A->tiled ? A->n_tiles : 0;
    info->tile_dict_len = A->tiled ? A->tile_dict_len : 0;
    info->tile_max_cols = A->tiled ? A->tile_dmax : 0;
    info->node_blocks = A->nb;
    info->nb_slices = A->nb_slices;
    info->nb_len = A->nb_len;
    info->nb_tiles = A->nb_tiles;
    info->nb_tile_dict_len = A->nb_tile_dict_len;
    return FESPMV_OK;
}

int spmv_export(fespmv_mat_t A, int32_t what, void* out, size_t bytes, fespmv_stream_t stream) {
    GUARD_BEGIN
    if (!A || !out) { set_error("null argument"); return FESPMV_ERR_INVALID_ARG; }
    const void* src = nullptr;
    size_t need = 0;
    bool sliced = A->format == FESPMV_FMT_SLICED;
    switch (what) {
        case FESPMV_EXPORT_PERM: src = A->d_perm; need = 4 * (size_t)A->n; break;
        case FESPMV_EXPORT_META: src = A->d_meta; need = 16 * (size_t)A->n_slices; break;
        case FESPMV_EXPORT_COLS: src = A->d_col; need = 4 * (size_t)A->packed_len; break;
        case FESPMV_EXPORT_VALUES:
            src = A->d_val; need = 8 * (size_t)(sliced ? A->packed_len : A->nnz); break;
        case FESPMV_EXPORT_SRCMAP: src = A->d_src; need = 8 * (size_t)A->packed_len; break;
        case FESPMV_EXPORT_DIAG: src = A->d_diag; need = 8 * (size_t)A->n; break;
        case FESPMV_EXPORT_VALUES_F32:
            src = A->d_val32; need = 4 * (size_t)(sliced ? A->packed_len : A->nnz); break;
        case FESPMV_EXPORT_VALUES_BF16:
            src = A->d_val16; need = 2 * (size_t)(sliced ? A->packed_len : A->nnz); break;
        case FESPMV_EXPORT_SCALE: src = A->d_scale; need = 8 * (size_t)A->n; break;
        case FESPMV_EXPORT_TILES: src = A->d_tiles; need = 16 * (size_t)A->n_tiles; break;
        case FESPMV_EXPORT_TILE_COLS: src = A->d_tdict; need = 4 * (size_t)A->tile_dict_len; break;
        case FESPMV_EXPORT_TILE_INDEX: src = A->d_tlidx; need = 2 * (size_t)A->packed_len; break;
        case FESPMV_EXPORT_NB_META: src = A->d_nbmeta; need = 16 * (size_t)A->nb_slices; break;
        case FESPMV_EXPORT_NB_COLS: src = A->d_nbcol; need = 4 * (size_t)A->nb_len; break;
        case FESPMV_EXPORT_NB_VALUES_F32: src = A->d_nb32; need = 36 * (size_t)A->nb_len; break;
        case FESPMV_EXPORT_NB_VALUES_BF16: src = A->d_nb16; need = 18 * (size_t)A->nb_len; break;
        case FESPMV_EXPORT_NB_MAP: src = A->d_nbmap; need = 72 * (size_t)A->nb_len; break;
        case FESPMV_EXPORT_NB_TILES: src = A->d_nbtiles; need = 16 * (size_t)A->nb_tiles; break;
        case FESPMV_EXPORT_NB_TILE_NODES: src = A->d_nbtdict; need = 4 * (size_t)A->nb_tile_dict_len; break;
        case FESPMV_EXPORT_NB_TILE_INDEX: src = A->d_nbtlidx; need = 2 * (size_t)A->nb_len; break;
        default: set_error("unknown export %d", what); return FESPMV_ERR_INVALID_ARG;
    }
    if (!src) { set_error("array %d is not held by this handle", what); return FESPMV_ERR_UNSUPPORTED; }
    if (!sliced && (what == FESPMV_EXPORT_PERM || what == FESPMV_EXPORT_META ||
                    what == FESPMV_EXPORT_COLS || what == FESPMV_EXPORT_SRCMAP)) {
        set_error("array %d exists only for SLICED handles", what); return FESPMV_ERR_UNSUPPORTED;
    }
    if (bytes < need) { set_error("buffer of %zu bytes, need %zu", bytes, need); return FESPMV_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    if (need) FESPMV_CUDA(cudaMemcpyAsync(out, src, need, cudaMemcpyDeviceToHost, s));
    FESPMV_CUDA(cudaStreamSynchronize(s));
    return FESPMV_OK;
    GUARD_END
}

const char* fespmv_status_string(int status) {
    switch (status) {
        case FESPMV_OK: return "ok";
        case FESPMV_ERR_INVALID_ARG: return "invalid argument";
        case FESPMV_ERR_BAD_CSR: return "malformed CSR";
        case FESPMV_ERR_OOM: return "out of memory";
        case FESPMV_ERR_CUDA: return "CUDA error";
        case FESPMV_ERR_BREAKDOWN: return "CG breakdown";
        case FESPMV_ERR_NOT_CONVERGED: return "CG not converged";
        case FESPMV_ERR_UNSUPPORTED: return "unsupported";
        case FESPMV_PENDING: return "pending";
        case FESPMV_ERR_CANCELLED: return "cancelled";
        default: return "unknown status";
    }
}

const char* fespmv_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
