// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "fespmv.h"

namespace fespmv {

// Per-thread last error message (fespmv_last_error).
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

#define FESPMV_CUDA(call)                                         \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return ::fespmv::cuda_fail(e_, #call); \
    } while (0)

// Host-side result of reordering and packing (see plan.cpp).
struct Plan {
    std::vector<int32_t> perm;      // P[new] = old
    std::vector<int32_t> pinv;      // Pinv[old] = new
    std::vector<uint32_t> meta;     // 4 per slice: offset/32, width, first row, log2 T
    std::vector<int32_t> col;       // packed columns (new numbering), -1 = padding
    std::vector<int64_t> src;       // packed entry -> input CSR position, -1 = padding
    std::vector<int64_t> diagpos;   // new row -> input CSR position of its diagonal, -1 none
    int64_t n_slices = 0;
    int64_t packed_len = 0;
    std::vector<int64_t> ppos;      // permuted CSR entry -> packed position (when asked for)
};


// Tiles of consecutive slices for the x-staging kernels: each tile's distinct
// columns form its dictionary (first-use order); every packed entry carries its
// 16-bit index into the dictionary, padding the index D of a zero slot.
struct Tiles {
    std::vector<int32_t> tiles;     // 4 per tile: first slice, slices, dictionary offset, size D
    std::vector<int32_t> dict;      // concatenated dictionaries
    std::vector<uint16_t> lidx;     // per packed entry
    int dmax = 0;                   // largest D
};

// Greedy runs of at most max_slices slices, closed before the dictionary would
// exceed max_cols.  Returns false (and leaves `out` empty) when one slice alone
// has more than max_cols distinct columns.
bool build_tiles(const std::vector<uint32_t>& meta, const std::vector<int32_t>& col, int64_t n,
                 int max_slices, int max_cols, Tiles& out);

// 3x3 node blocks of a node-ordered permuted CSR (rows 3I..3I+2 of node I): K1
// slices of 32 node rows, one block row per lane, blocks column-major in the
// slice; each block one int32 block column and 9 values stored step-major
// (value k = 3a + b of the block at step s, lane l of a slice at offset off:
// index 9 (off + 32 s) + 32 k + l, so that a warp reads one contiguous run per step).
struct NodeBlocks {
    std::vector<uint32_t> meta;     // 4 per slice: offset/32 (block slots), width, first node row, 0
    std::vector<int32_t> col;       // per block slot: block column (node), -1 = padding
    std::vector<int64_t> map;       // per value: packed position of the entry, -1 = zero fill
    int64_t n_slices = 0;
    int64_t len = 0;                // block slots including padding
    Tiles tiles;                    // tiles of node-block slices (x of the column nodes staged)
};
int pack_node_blocks(const std::vector<int64_t>& rp2, const std::vector<int32_t>& c2,
                     const std::vector<int64_t>& ppos, NodeBlocks& out);

// Permuted CSR (stage 1 of planning): P, Pinv, rows in new order with columns
// renumbered and sorted, each entry's input position, each row's diagonal position.
struct Permuted {
    std::vector<int32_t> perm, pinv;
    std::vector<int64_t> rp2;
    std::vector<int32_t> c2;
    std::vector<int64_t> s2;      // input CSR position; -2 = constant 1.0 (batch padding)
    std::vector<int64_t> diagpos;
};
// node_sort: the windowed length sort moves whole nodes (windows of ceil(sigma /
// dofs_per_node) nodes, key = the longest row of the node), so that the dofs of
// every node stay adjacent at rows dofs_per_node * k + c.
// col_order: FESPMV_COLS_SORTED (Sec. 5.3, K1rs), _RENUMBERED (Sec. 5.2, K1r: renumbered,
// in the input's order) or _ORIGINAL (Sec. 5.1, K1: the input numbering, not renumbered).
int order_and_permute(int64_t n, const int64_t* rowptr, const int32_t* colind, int dofs_per_node,
                      const double* node_xyz, int reorder, int sigma, Permuted& out, bool node_sort = false,
                      int col_order = 0);
// Stage 2: the K1/K2 warp slices of a permuted CSR (meta, col, src, sizes of `out`;
// with_ppos: also each permuted entry's packed position).
int pack_slices(const std::vector<int64_t>& rp2, const std::vector<int32_t>& c2,
                const std::vector<int64_t>& s2, int threshold, int vec, Plan& out, bool with_ppos = false);

// Builds the locality order, windowed length sort, symmetric renumbering with
// sorted columns and the warp-slice packing.  Returns FESPMV_OK or an error code
// (message set).
int build_plan(int64_t n, const int64_t* rowptr, const int32_t* colind, int dofs_per_node,
               const double* node_xyz, int reorder, int sigma, int threshold, int vec,
               Plan& out, NodeBlocks* nb = nullptr, int col_order = 0);

// Validates a host CSR (monotone offsets, columns in range); duplicates are
// detected by build_plan for SLICED and by validate_csr_rows for CSR.
int validate_csr(int64_t n, const int64_t* rowptr, const int32_t* colind);

}  // namespace fespmv

namespace fespmv {
struct CgWork;     // cg.cu
struct MultiWork;  // multi_cg.cu
}

// The opaque handle.
struct fespmv_mat {
    int64_t n = 0;
    int64_t nnz = 0;
    int format = FESPMV_FMT_CSR;
    int block = 256;
    int precisions = FESPMV_PREC_F64;
    int64_t device_bytes = 0;

    // FESPMV_FMT_CSR
    int csr_lanes = 1;
    int64_t* d_rowptr = nullptr;
    int32_t* d_colind = nullptr;
    double* d_val = nullptr;          // CSR values, or packed values for SLICED

    // FESPMV_FMT_SLICED
    int vec = 2;
    int col_order = 0;                // FESPMV_COLS_*; ORIGINAL: x in the input numbering
    int64_t n_slices = 0;
    int64_t packed_len = 0;
    uint4* d_meta = nullptr;
    int32_t* d_col = nullptr;
    int32_t* d_perm = nullptr;
    int32_t* d_pinv = nullptr;
    int64_t* d_src = nullptr;

    // both formats
    int64_t* d_diagpos = nullptr;     // row (handle numbering) -> input CSR position of diagonal
    double* d_diag = nullptr;         // diag(A) in handle numbering
    double* d_xp = nullptr;           // permuted-I/O scratch (n each)
    double* d_yp = nullptr;
    double* d_xh = nullptr;           // host-I/O staging (n each), allocated on first use
    double* d_yh = nullptr;
    double* d_vals_in = nullptr;      // update_values staging (nnz), allocated on first use
    float* d_val32 = nullptr;         // B = S A S in FP32 (same positions as d_val)
    uint16_t* d_val16 = nullptr;      // B in bfloat16 bits
    double* d_scale = nullptr;        // S = diag(A)^-1/2 (handle numbering)
    int* d_flag = nullptr;            // set to 1 when diag(A) has a non-positive entry
    float2* d_vdf = nullptr;          // FP64 values as float pairs (FESPMV_PREC_DF64)
    float2* d_xdf = nullptr;          // float-pair x scratch (n)
    double* d_xk = nullptr;           // multi-RHS permuted-I/O scratch (32 n doubles each)
    double* d_yk = nullptr;
    float2* d_xkdf = nullptr;         // multi-RHS X as float pairs (handles with FESPMV_PREC_DF64)
    int max_lanes_log2 = 0;           // largest log2(lanes per row) over the slices
    // x staged through shared memory (SLICED, options.tiles >= 0): Tiles on the device
    int tiled = 0;                    // 1 when the tile arrays below are in use
    int64_t n_tiles = 0;
    int tile_dmax = 0;
    int64_t tile_dict_len = 0;
    int4* d_tiles = nullptr;
    int32_t* d_tdict = nullptr;
    uint16_t* d_tlidx = nullptr;
    float* d_xs = nullptr;            // float permuted-I/O scratch (n each)
    float* d_ys = nullptr;
    // 3x3 node blocks (SLICED, options.node_blocks = 3): the FP32 / BF16 copies of S A S
    int nb = 0;                       // 3 when in use
    int64_t nb_slices = 0;
    int64_t nb_len = 0;               // block slots including padding
    uint4* d_nbmeta = nullptr;
    int32_t* d_nbcol = nullptr;
    int64_t* d_nbmap = nullptr;       // 9 per slot: packed position, -1 = zero
    float* d_nb32 = nullptr;          // 9 per slot
    uint16_t* d_nb16 = nullptr;       // 9 per slot, bfloat16 bits
    int64_t nb_tiles = 0;             // tiles of node-block slices (0: x gathered from L1/L2)
    int nb_tile_dmax = 0;             // largest tile node list
    int64_t nb_tile_dict_len = 0;
    int4* d_nbtiles = nullptr;
    int32_t* d_nbtdict = nullptr;     // the tiles' column nodes
    uint16_t* d_nbtlidx = nullptr;    // per slot: index of its column node in the tile's list

    fespmv::CgWork* cg = nullptr;     // CG workspace, allocated by the first cg_solve
    fespmv::MultiWork* mcg = nullptr; // multi-RHS CG workspace, allocated by the first cg_solve_multi
};

namespace fespmv {

int device_alloc(fespmv_mat* A, void** p, size_t bytes, const char* what);

// Kernel launchers (spmv_kernels.cu); all enqueue on `s` and return FESPMV_OK or
// FESPMV_ERR_CUDA.
int launch_spmv(const fespmv_mat* A, const double* x, double* y, cudaStream_t s);
int launch_spmv_tiled(const fespmv_mat* A, const double* x, double* y, cudaStream_t s);
// The same FP64 product with x and y in the input numbering (the permutations folded
// into the tile staging and the row store).
int launch_spmv_tiled_io(const fespmv_mat* A, const double* x, double* y, cudaStream_t s);
int launch_spmv_low_tiled(const fespmv_mat* A, int precision, const float* x, float* y, cudaStream_t s);
int launch_spmv_df_tiled(const fespmv_mat* A, const float2* xdf, const double* x, double* y, cudaStream_t s);
int launch_gather(const double* in, const int32_t* idx, double* out, int64_t n, cudaStream_t s);
int launch_scatter(const double* in, const int32_t* idx, double* out, int64_t n, cudaStream_t s);
int launch_fill_values(fespmv_mat* A, const double* vals_in, cudaStream_t s);
unsigned grid_for(int64_t work, int block);
// Rebuilds S and the FP32/BF16 copies of S A S from the FP64 values (if held).
int launch_build_scaled(fespmv_mat* A, cudaStream_t s);
int launch_nb3_refresh(fespmv_mat* A, cudaStream_t s);   // node-block copies from the scalar ones
int launch_nb3_product(const fespmv_mat* A, int precision, const float* x, float* y, cudaStream_t s);
int launch_nb3_multi(const fespmv_mat* A, const float* X, float* Y, int kw, cudaStream_t s);  // FP32, KW = kw
// The lockstep CG's FP32 product with per-block column sums of p.q (part == nullptr:
// only the grid, i.e. the number of partial rows, is returned).
unsigned launch_nb3_multi_dot(const fespmv_mat* A, const float* P, float* Q, int kw, double* part, cudaStream_t s);
// y = B x with the FP32 (precision FESPMV_PREC_F32) or BF16 copy, handle numbering.
int launch_spmv_low(const fespmv_mat* A, int precision, const float* x, float* y, cudaStream_t s);
int launch_gather_f32(const float* in, const int32_t* idx, float* out, int64_t n, cudaStream_t s);
// Float-pair FP64 product (FESPMV_PREC_DF64): y = A x with x given as double and split.
int launch_spmv_df(const fespmv_mat* A, const float2* xs, const double* x, double* y, cudaStream_t s);
int launch_split(const double* v, float2* out, int64_t len, cudaStream_t s);
int launch_gather_split(const double* x, const int32_t* idx, double* xp, float2* xs, int64_t n,
                        cudaStream_t s);

// Multi-RHS kernels (multi.cu), X and Y row-major with row stride kw (4, 8, 16 or 32),
// handle numbering.  launch_multi_dot: Q = A P with the FP64 (f64) or FP32 copy
// of S A S, plus per-block FP64 sums of p_ij q_ij at part[block * kw + j]; returns
// its grid (with part == nullptr it only returns the grid).
unsigned launch_multi_dot(const fespmv_mat* A, const void* P, void* Q, int kw, bool f64, double* part,
                          cudaStream_t s);
// The same product and sums on a FESPMV_PREC_DF64 handle as float pairs: P is split
// into Pdf (n x kw pairs, the caller's scratch) first.
unsigned launch_multi_dot_pairs(const fespmv_mat* A, const double* P, double* Q, float2* Pdf, int kw, double* part,
                                cudaStream_t s);
// Y = A X in FP64 (float pairs on FESPMV_PREC_DF64 handles).
int launch_multi_f64(fespmv_mat* A, const double* X, double* Y, int kw, cudaStream_t s);
// dst[i, j] = src[idx[i], j] (idx null: identity) for j < k, 0 for k <= j < ldd.
void launch_gather_rows_f64(const double* src, int lds, const int32_t* idx, double* dst, int ldd, int64_t n,
                            int k, cudaStream_t s);
int multi_width(int k);   // the padded width kw for k columns

// Handle plumbing (capi.cpp)
void free_handle(fespmv_mat* A);
int alloc_scaled(fespmv_mat* A, int64_t len);
int upload_sliced(fespmv_mat* A, const Plan& plan, cudaStream_t s);

// CG (cg.cu) and the multi-RHS CG (multi_cg.cu)
void free_cg(fespmv_mat* A);
void free_multi_cg(fespmv_mat* A);

}  // namespace fespmv

struct fespmv_assembly;
namespace fespmv {
fespmv_mat* assembly_handle(fespmv_assembly* P);   // the matrix an assembly map writes
}  // namespace fespmv
