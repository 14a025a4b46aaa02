/*
 * fespmv.h -- C ABI of the GB300 finite-element SpMV + CG library.
 *
 * Paper: J. Wong, E. Kuhl, E. Darve, "A New Sparse Matrix Vector Multiplication
 * GPU Algorithm Designed for Finite Element Problems" (arXiv:1501.00324).
 *
 * The library computes y = A x for sparse stiffness matrices of unstructured
 * finite-element meshes (Sec. 4 states the problem: given A and x, compute y)
 * and runs the Jacobi-preconditioned conjugate-gradient solve of K dx = R that
 * the paper's Newton loop performs (Sec. 2.1, Sec. 4), on one GPU.
 *
 * Entry points, in these groups: handles and products (spmv_create,
 * spmv_apply, spmv_apply_multi, spmv_apply_scaled, spmv_update_values,
 * spmv_autotune, spmv_plan / spmv_plan_tiles host-only planning, spmv_export);
 * solves (cg_solve, cg_solve_csr_static, cg_solve_multi); assembly from element
 * quantities (assembly_*, Sec. 4); batches of independent problems (batch_*);
 * the solve server (srv_*).
 *
 * Conventions for every entry point:
 *   - Return 0 (FESPMV_OK) on success or a negative FESPMV_ERR_* code; nothing
 *     aborts or traps.  fespmv_last_error() gives a message for the calling
 *     thread's most recent failure.
 *   - Host arrays passed to spmv_create are read during the call and not
 *     retained.  Device arrays passed to spmv_apply / cg_solve stay owned by the
 *     caller and must hold the stated number of elements.
 *   - All device work is ordered on the caller's stream (a cudaStream_t passed
 *     as fespmv_stream_t; NULL = legacy default stream).
 *   - A handle is not thread-safe: calls on one handle must not overlap.
 *   - Indices are 0-based; CSR row offsets are int64, column indices int32.
 */
#ifndef FESPMV_H
#define FESPMV_H

#include <stddef.h>
#include <stdint.h>

/* The library is compiled with hidden visibility: the functions declared here are
 * its only exported symbols. */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fespmv_stream_t; /* identical to cudaStream_t */
typedef struct fespmv_mat* fespmv_mat_t;      /* opaque; owns the device memory it allocates */

/* ---- status codes ---------------------------------------------------------------- */
#define FESPMV_OK                  0
#define FESPMV_ERR_INVALID_ARG    -1  /* null pointer, bad size or bad option */
#define FESPMV_ERR_BAD_CSR        -2  /* rowptr not monotone, column out of range, duplicate */
#define FESPMV_ERR_OOM            -3  /* device or host allocation failed */
#define FESPMV_ERR_CUDA           -4  /* a CUDA runtime call failed (message has the name) */
#define FESPMV_ERR_BREAKDOWN      -5  /* CG: p.Ap <= 0 or a non-finite scalar */
#define FESPMV_ERR_NOT_CONVERGED  -6  /* CG: iteration limit reached above tolerance */
#define FESPMV_ERR_UNSUPPORTED    -7  /* option combination not built for this handle */
#define FESPMV_ERR_CANCELLED      -8  /* srv_poll: the request was cancelled before it started */
#define FESPMV_PENDING             1  /* srv_poll: the solve has not finished yet */

/* ---- matrix formats and kernels ---------------------------------------------------- */
/* Storage built by spmv_create. */
#define FESPMV_FMT_CSR     0  /* the input CSR as given: baseline kernels (Sec. 4, CSR) */
#define FESPMV_FMT_SLICED  1  /* FE warp slices: locality order, length sort, packed
                                 column-major slices (Sec. 5.1-5.5, ELL-WARP K1/K2) */

/* Node locality orders for FESPMV_FMT_SLICED. */
#define FESPMV_REORDER_NONE    0  /* keep the input numbering */
#define FESPMV_REORDER_MORTON  1  /* Z-order curve of node_xyz (requires mesh->node_xyz) */

/* Column numbering of FESPMV_FMT_SLICED (the paper's K1 / K1r / K1rs, Sec. 5.1-5.3). */
#define FESPMV_COLS_SORTED     0  /* K1rs: renumbered with the rows (c' = P^-1[c]) and sorted per row */
#define FESPMV_COLS_RENUMBERED 1  /* K1r: renumbered, each row in the input's order */
#define FESPMV_COLS_ORIGINAL   2  /* K1: the input numbering; the product reads x in the input
                                     numbering and writes y in the handle's (spmv_apply without
                                     FESPMV_IO_PERMUTED returns y in the input numbering).  FP64
                                     products only: no FP32/BF16/float-pair copies, node blocks,
                                     CG, multi-RHS or assembly on such a handle. */

/* Kernel selection for FESPMV_FMT_CSR (csr_lanes) is by lanes per row:
 * 1 = one thread per row (CSR scalar, Sec. 4), 2..32 (power of two) = that many
 * lanes of a warp per row with a shuffle reduction (CSR vector, Sec. 4). */

/* Value copies kept by a handle (bitmask in fespmv_options.precisions). */
#define FESPMV_PREC_F64      1  /* FP64 values (always kept) */
#define FESPMV_PREC_F32      2  /* FP32 values of B = S A S, S = diag(A)^-1/2 (refined CG) */
#define FESPMV_PREC_BF16     4  /* bfloat16 values of B = S A S (refined CG) */
#define FESPMV_PREC_DF64     8  /* SLICED: also keep the FP64 values as float pairs
                                   (hi, lo) and compute every FP64 product of the handle
                                   (spmv_apply, cg_solve) on the FP32 pipe with
                                   error-free transformations; values or x entries
                                   outside |v| in [2^-50, 2^50] (and Inf/NaN) take an
                                   exact FP64 path.  Componentwise error below
                                   (L+2) 2^-47 sum_j |A_ij x_j| for rows of L entries. */

typedef struct {
    int32_t format;      /* FESPMV_FMT_*; 0 = CSR baseline */
    int32_t reorder;     /* FESPMV_REORDER_*; SLICED only; MORTON needs node_xyz */
    int32_t sigma;       /* SLICED: rows per length-sort window (stable, longest first);
                            0 = no sort; >= n_rows = the paper's global sort (Sec. 5.1) */
    int32_t threshold;   /* SLICED: K2 threshold, max entries per lane (Sec. 5.4); 0 = K1 */
    int32_t vec;         /* SLICED: entries per lane per load, 1, 2 or 4; 0 = 2 */
    int32_t csr_lanes;   /* CSR: lanes per row, 1..32 power of two; 0 = 1 (scalar) */
    int32_t precisions;  /* FESPMV_PREC_* bitmask; 0 = FP64 only */
    int32_t block;       /* threads per block for the SpMV kernel, multiple of 32, <= 1024
                            (<= 256 for SLICED); 0 = 256 */
    int32_t tiles;       /* SLICED: x staged through shared memory.  0 = on: runs of up to 8
                            consecutive slices form tiles whose distinct columns (at most 4096)
                            are gathered once per product into shared memory, and each stored
                            entry keeps a 16-bit index into its tile's columns next to the
                            32-bit column; the FP64 and FP32/BF16 products use them.  Left off
                            when one slice alone has more distinct columns.  -1 = off. */
    int32_t node_blocks; /* SLICED with dofs_per_node = 3 and FESPMV_PREC_F32 or _BF16: 3 = also
                            keep those copies of S A S as 3x3 node blocks (rows of node I are
                            3I..3I+2 in the handle's numbering: the length sort moves whole
                            nodes; each block one int32 column node and 9 values, zero where
                            the matrix has no entry).  spmv_apply_scaled and the refined CG's
                            inner products then read the blocks: runs of up to 8 slices of 32
                            node rows stage the x values of their column nodes (at most 2048)
                            in shared memory, and each block keeps a 16-bit index into that
                            list: 2/9 of a byte of index per value, one lookup per 9 values
                            (tiles = -1: x gathered from L1/L2 with the int32 block columns).  NaN or Inf in x at a column
                            a block stores as zero reaches its rows.  0 = off. */
    int32_t col_order;   /* SLICED: FESPMV_COLS_*; 0 = sorted (K1rs) */
} fespmv_options;

typedef struct {
    int32_t dofs_per_node;   /* rows = dofs_per_node * n_nodes, row = d*node + c; 0 = 1 */
    const double* node_xyz;  /* host, n_nodes x 3 coordinates, or NULL */
} fespmv_mesh_info;

/* Sizes of a built handle. */
typedef struct {
    int64_t n_rows;
    int64_t nnz;
    int64_t n_slices;        /* SLICED: warps per product; CSR: 0 */
    int64_t packed_len;      /* SLICED: stored entries including padding; CSR: nnz */
    int64_t device_bytes;    /* device memory owned by the handle */
    int32_t format;
    int32_t vec;
    int64_t n_tiles;         /* SLICED with tiles: tiles (0 when the products gather x from L1/L2) */
    int64_t tile_dict_len;   /* concatenated tile column lists */
    int32_t tile_max_cols;   /* largest tile column list */
    int32_t node_blocks;     /* 3 with node blocks, else 0 */
    int64_t nb_slices;       /* node-block slices (32 node rows each) */
    int64_t nb_len;          /* node-block slots including padding */
    int64_t nb_tiles;        /* tiles of node-block slices (0: x gathered from L1/L2) */
    int64_t nb_tile_dict_len;/* concatenated column-node lists of those tiles */
} fespmv_info;

/*
 * spmv_create -- build a handle for y = A x from a host CSR matrix.
 *   n_rows          square matrix order (>= 0)
 *   rowptr          host int64[n_rows+1], rowptr[0] = 0, non-decreasing
 *   colind          host int32[nnz], each in [0, n_rows), no duplicates within a row
 *   values          host double[nnz]
 *   mesh            optional mesh metadata (NULL: one dof per node, no coordinates)
 *   opts            optional options (NULL or zero-initialised: defaults)
 * SLICED handles reorder on the host (Sec. 5.1 row sort, Sec. 5.2 symmetric
 * renumbering x' = x(P), c' = P^-1(c), Sec. 5.3 per-row column sort), pack
 * the warp slices and copy them to the device once.  Errors: INVALID_ARG,
 * BAD_CSR, OOM, CUDA.  On error *out is set to NULL.
 */
int spmv_create(fespmv_mat_t* out, int64_t n_rows, const int64_t* rowptr, const int32_t* colind,
                const double* values, const fespmv_mesh_info* mesh, const fespmv_options* opts,
                fespmv_stream_t stream);

/* Free every device and host resource of the handle (NULL is ignored).  The
 * caller must make sure no work using the handle is still running. */
void spmv_destroy(fespmv_mat_t A);

/* I/O flags for spmv_apply and cg_solve. */
#define FESPMV_IO_PERMUTED  1  /* vectors are in the handle's permuted numbering */
#define FESPMV_IO_HOST      2  /* vectors are host memory: copied in and out on the stream,
                                  and the call waits for the stream before returning */

/*
 * spmv_apply -- y = A x in FP64.
 *   x, y  n_rows doubles each, device memory unless FESPMV_IO_HOST; x and y must
 *         not overlap.  Without FESPMV_IO_PERMUTED they are in the numbering of
 *         the CSR given to spmv_create.  For device vectors a SLICED handle with
 *         tiles (the default) folds the permutations into the product: each tile
 *         stages x[P[c']] for its columns c' and each row i' stores y[P[i']].
 *         Otherwise a SLICED handle permutes x on the way in and y on the way out
 *         (two gathers of n_rows entries); with FESPMV_IO_HOST and page-locked
 *         (pinned, mapped) host buffers those permutations read x and write y in
 *         place over the host link (no staging copies; measured faster than one
 *         contiguous copy each way around the folded product); pageable buffers
 *         are copied through staging.
 * Result per entry: the exact sum over the stored entries of the row, rounded
 * with a different association than a left-to-right sum (componentwise error
 * well under 1e-12 * sum_j |A_ij x_j|).  Errors: INVALID_ARG, CUDA.
 */
int spmv_apply(fespmv_mat_t A, const double* x, double* y, int32_t flags, fespmv_stream_t stream);

/*
 * spmv_apply_multi -- Y = A X for k right-hand sides at once (1 <= k <= 32), the
 * matrix streamed from memory once for all columns (the paper applies one
 * vector at a time; this is the batched layer's product).
 *   X, Y       device, row-major n_rows x k (k values per row), double with
 *              precision FESPMV_PREC_F64 (FP64 values and arithmetic) or float
 *              with FESPMV_PREC_F32 (the FP32 copy of B = S A S, float
 *              arithmetic); input numbering unless FESPMV_IO_PERMUTED
 * Needs a SLICED handle built with threshold 0 (one lane per row).  Each entry
 * of Y is the sum of its row's products in the order of the row's stored
 * entries (one FMA chain per row and column).  With FESPMV_PREC_F64 on a handle
 * holding float pairs (FESPMV_PREC_DF64) the products and sums are float pairs
 * on the FP32 pipe (as spmv_apply's), rows meeting values outside the pairs'
 * range summed again in FP64: within the same 1e-12 componentwise bound.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM (scratch for the input numbering), CUDA.
 */
int spmv_apply_multi(fespmv_mat_t A, const void* X, void* Y, int32_t k, int32_t precision,
                     int32_t flags, fespmv_stream_t stream);

/* Vector permutation between the input numbering and a SLICED handle's numbering
 * (device arrays of n_rows doubles, no overlap):
 *   direction 0: out[i'] = in[P[i']]   (input -> permuted, x' = x(P), Sec. 5.2)
 *   direction 1: out[i]  = in[Pinv[i]] (permuted -> input)
 * CSR handles copy.  Errors: INVALID_ARG, CUDA. */
int spmv_permute(fespmv_mat_t A, const double* in, double* out, int32_t direction,
                 fespmv_stream_t stream);

/*
 * spmv_update_values -- replace the matrix values, keeping the pattern (the
 * per-Newton-step refresh of Sec. 6, "Cost of Reordering Matrix Values": one
 * gather through the map computed at create time, on the device).
 *   values  double[nnz] in the CSR order given to spmv_create; device memory
 *           unless FESPMV_IO_HOST is set in flags.
 * FP32 scaled copies kept by the handle are rebuilt too.  Errors: INVALID_ARG, CUDA.
 */
int spmv_update_values(fespmv_mat_t A, const double* values, int32_t flags,
                       fespmv_stream_t stream);

int spmv_get_info(fespmv_mat_t A, fespmv_info* info);

/*
 * spmv_autotune -- choose the SLICED layout for this matrix by measurement (the
 * paper tunes block size and the K2 threshold per matrix by exhaustive timing,
 * Sec. 6 and Table "bestvalues", and leaves an a-priori rule to future work,
 * Sec. 9).  Candidates: vec in {1, 2, 4} x threshold in {0, ceil(maxlen/4),
 * ceil(maxlen/8)} (distinct values, 0 = K1) x layout in {x staged per tile (when
 * the base options' tiles is 0), x gathered from cache with 128 or 256 threads
 * per block}, each built from the given CSR with the base options' reorder and
 * sigma, then timed as `reps` back-to-back products in the permuted numbering on
 * `stream`: products of the FP32 copy of S A S when the base options' precisions
 * hold FESPMV_PREC_F32 (else of the BF16 copy when they hold FESPMV_PREC_BF16: the
 * refined CG's inner product), FP64 products otherwise.
 *   opts_inout   in: base options (format forced to SLICED); out: the fastest
 *                candidate's vec, threshold, block and tiles
 *   reps         products timed per candidate (0 = 20)
 *   best_us      out (may be NULL): mean microseconds per product of the winner
 *   n_tried      out (may be NULL): candidates timed
 * Device memory: one candidate handle at a time plus two vectors.  Errors: as
 * spmv_create.
 */
int spmv_autotune(int64_t n_rows, const int64_t* rowptr, const int32_t* colind, const double* values,
                  const fespmv_mesh_info* mesh, fespmv_options* opts_inout, int32_t reps,
                  double* best_us, int32_t* n_tried, fespmv_stream_t stream);

/*
 * spmv_apply_scaled -- y = B x for the low-precision copy B = S A S (S =
 * diag(A)^-1/2) kept with FESPMV_PREC_F32 or FESPMV_PREC_BF16: B's stored
 * values, float x and y, float products and sums.  This is the operator of
 * the refined CG's inner iterations.
 *   precision  FESPMV_PREC_F32 or FESPMV_PREC_BF16
 *   x, y       device float[n_rows] (permuted numbering with FESPMV_IO_PERMUTED;
 *              without it a SLICED handle gathers x in and y out)
 * Errors: INVALID_ARG, UNSUPPORTED (copy not held), CUDA.
 */
int spmv_apply_scaled(fespmv_mat_t A, const float* x, float* y, int32_t precision, int32_t flags,
                      fespmv_stream_t stream);

/* Arrays spmv_export can copy to the host (for tests and inspection). */
#define FESPMV_EXPORT_PERM     0  /* int32[n_rows]: P, P[new] = old (SLICED) */
#define FESPMV_EXPORT_META     1  /* uint32[n_slices*4]: (offset/32, width, first row, log2 T) */
#define FESPMV_EXPORT_COLS     2  /* int32[packed_len]: packed column indices, -1 = padding */
#define FESPMV_EXPORT_VALUES   3  /* double[packed_len]: packed values, 0 = padding */
#define FESPMV_EXPORT_SRCMAP   4  /* int64[packed_len]: CSR position of each packed entry, -1 pad */
#define FESPMV_EXPORT_DIAG     5  /* double[n_rows]: diag(A) in the handle's numbering */
#define FESPMV_EXPORT_VALUES_F32  6  /* float[packed_len or nnz]: values of B = S A S */
#define FESPMV_EXPORT_VALUES_BF16 7  /* uint16[packed_len or nnz]: bfloat16 bits of B */
#define FESPMV_EXPORT_SCALE    8  /* double[n_rows]: S = diag(A)^-1/2, handle numbering */
#define FESPMV_EXPORT_TILES    9  /* int32[n_tiles*4]: (first slice, slices, column-list offset, D) */
#define FESPMV_EXPORT_TILE_COLS 10 /* int32[tile_dict_len]: each tile's distinct columns, first-use order */
#define FESPMV_EXPORT_TILE_INDEX 11 /* uint16[packed_len]: index into the tile's columns; padding = D */
#define FESPMV_EXPORT_NB_META  12 /* uint32[nb_slices*4]: (offset/32, width, first node row, 0) */
#define FESPMV_EXPORT_NB_COLS  13 /* int32[nb_len]: block column (node) per slot, -1 = padding */
#define FESPMV_EXPORT_NB_VALUES_F32 14 /* float[9*nb_len]: block values, 9 words of 32 lanes per slot step */
#define FESPMV_EXPORT_NB_VALUES_BF16 15 /* uint16[9*nb_len]: the same in bfloat16 bits */
#define FESPMV_EXPORT_NB_MAP   16 /* int64[9*nb_len]: packed position of each block value, -1 = zero */
#define FESPMV_EXPORT_NB_TILES 17 /* int32[nb_tiles*4]: (first slice, slices, node-list offset, D) */
#define FESPMV_EXPORT_NB_TILE_NODES 18 /* int32[nb_tile_dict_len]: each tile's column nodes, first-use order */
#define FESPMV_EXPORT_NB_TILE_INDEX 19 /* uint16[nb_len]: index of a slot's node in its tile's list; padding = D */
/* Copy internal array `what` into host buffer `out` of `bytes` bytes (must be at
 * least the array's size).  Synchronises the stream.  Errors: INVALID_ARG,
 * UNSUPPORTED (array not held by this handle), CUDA. */
int spmv_export(fespmv_mat_t A, int32_t what, void* out, size_t bytes, fespmv_stream_t stream);

/*
 * spmv_plan -- the host part of spmv_create for FESPMV_FMT_SLICED, with no
 * device work (usable without a GPU).  Computes the same permutation, slice
 * metadata, packed columns and value map that spmv_create uploads.
 *   info     out: n_rows, nnz, n_slices, packed_len (always written)
 *   perm     out: int32[n_rows] or NULL
 *   meta     out: uint32[n_slices*4] or NULL
 *   cols     out: int32[packed_len] or NULL
 *   srcmap   out: int64[packed_len] or NULL
 * Call once with NULL arrays to learn the sizes, then again with buffers.
 * Errors: INVALID_ARG, BAD_CSR, OOM (host), UNSUPPORTED.
 */
int spmv_plan(int64_t n_rows, const int64_t* rowptr, const int32_t* colind,
              const fespmv_mesh_info* mesh, const fespmv_options* opts, fespmv_info* info,
              int32_t* perm, uint32_t* meta, int32_t* cols, int64_t* srcmap);

/*
 * spmv_plan_tiles -- the tiles spmv_create builds (options.tiles = 0) for a packed
 * layout from spmv_plan, on the host, with no device work: runs of at most 8
 * consecutive slices whose distinct columns number at most 4096, each tile's
 * columns in order of first use, each stored entry's 16-bit index into its tile's
 * list (padding: the list's length).  Not in the paper: this library's x staging.
 *   n_rows        rows of the matrix (every column index is -1 or in [0, n_rows))
 *   meta, cols    spmv_plan's slice metadata (n_slices x 4) and packed columns
 *   tiles         out: int32[4 * n_slices] or NULL: (first slice, slices, list offset, D)
 *   tile_cols     out: int32[packed_len] or NULL: the concatenated column lists
 *   index         out: uint16[packed_len] or NULL
 *   n_tiles, n_tile_cols   out: counts; 0 and 0 when one slice alone has more
 *                 than 4096 distinct columns (the handle then gathers x from cache)
 * Errors: INVALID_ARG (a slice outside the packed arrays, a column out of range),
 * OOM (host).
 */
int spmv_plan_tiles(int64_t n_rows, int64_t n_slices, const uint32_t* meta, int64_t packed_len,
                    const int32_t* cols, int32_t* tiles, int32_t* tile_cols, uint16_t* index,
                    int64_t* n_tiles, int64_t* n_tile_cols);

/* ---- conjugate gradients ----------------------------------------------------------- */
#define FESPMV_CG_F64          0  /* FP64 Jacobi-PCG on the handle's FP64 values */
#define FESPMV_CG_F32_REFINE   1  /* FP64 refinement around FP32 CG on B = S A S (FP32 values) */
#define FESPMV_CG_BF16_REFINE  2  /* FP64 refinement around FP32 CG on B = S A S (BF16 values) */
#define FESPMV_CG_X0           4  /* flag: x holds the initial guess (otherwise x0 = 0) */
#define FESPMV_CG_NO_PRECOND   8  /* flag: plain CG instead of Jacobi-PCG */
#define FESPMV_CG_SINGLE_REDUCTION 16 /* flag: single-reduction (Chronopoulos-Gear) PCG, below */
#define FESPMV_CG_RELIABLE     32 /* flag: refined precisions without restarts (reliable updates), below */
#define FESPMV_CG_FLEXIBLE     64 /* flag: refined precisions as the preconditioner of a flexible
                                     FP64 CG (Notay 2000), below */
#define FESPMV_CG_NO_CLUSTER  128 /* flag: keep the CUDA-graph iterations of reliable updates
                                     on a small handle (see "Small handles" below) */

typedef struct {
    double tol;            /* stop when ||b - A x||_2 <= tol ||b||_2; 0 = 1e-10 */
    int32_t max_iter;      /* iteration limit over all restarts; 0 = 100000 */
    int32_t precision;     /* FESPMV_CG_F64 */
    int32_t flags;         /* FESPMV_IO_PERMUTED | FESPMV_IO_HOST | FESPMV_CG_X0 |
                              FESPMV_CG_NO_PRECOND */
    int32_t max_restarts;  /* restarts from the true residual; 0 = 3, < 0 = none */
    int32_t check_every;   /* iterations per graph launch between host polls; 0 = 16 */
    int32_t max_outer;     /* refinement: FP64 residual steps; 0 = 60 */
    double inner_tol;      /* refinement: inner CG stops at ||r_in|| <= inner_tol ||S r||; 0 = 1e-2 */
    int32_t inner_steps;   /* FESPMV_CG_FLEXIBLE: low-precision CG steps per outer step; 0 = 8 */
    int32_t pad;
} cg_options;

typedef struct {
    int32_t status;        /* FESPMV_OK, FESPMV_ERR_NOT_CONVERGED or FESPMV_ERR_BREAKDOWN */
    int32_t iters;         /* CG iterations over all restarts */
    int32_t restarts;      /* restarts taken (FP64) */
    int32_t outer;         /* refinement steps taken (refined precisions) */
    double relres;         /* recurrence residual ||r_k|| / ||b|| at exit */
    double true_relres;    /* ||b - A x|| / ||b|| recomputed in FP64 at exit */
} cg_result;

/*
 * cg_solve -- solve A x = b by Jacobi-preconditioned conjugate gradients, the
 * linear solver of the paper's Newton step K dx = R (Sec. 2.1; Jacobi
 * preconditioning as in Sec. 2.1), textbook Hestenes-Stiefel recurrences:
 *   r = b - A x0, z = D^-1 r, p = z, rho = r.z;
 *   repeat q = A p; alpha = rho / p.q; x += alpha p; r -= alpha q;
 *          stop when ||r|| <= tol ||b||; z = D^-1 r; beta = r.z / rho; p = z + beta p.
 * After the recurrence stops, ||b - A x|| is recomputed in FP64; above tol the
 * iteration restarts from x (max_restarts times).
 *   b, x   n_rows doubles (device unless FESPMV_IO_HOST; permuted numbering with
 *          FESPMV_IO_PERMUTED); x is overwritten with the solution.
 *   opts   NULL = defaults;  res  optional result record.
 * The matrix must be symmetric positive definite with a positive diagonal.
 * Work runs on `stream` as CUDA graphs of check_every iterations with the
 * scalars kept on the device; the call blocks the host until the solve ends
 * (it polls a status word after each graph).  Dot products are reduced in a
 * fixed order, so repeated solves of the same system give bitwise-equal x.
 * Workspace (8 vectors of n_rows doubles) is allocated on the first call and
 * kept by the handle.
 *
 * flag FESPMV_CG_SINGLE_REDUCTION (FESPMV_CG_F64 only, else UNSUPPORTED): the
 * same method in the Chronopoulos-Gear arrangement, whose iterates equal the
 * ones above in exact arithmetic (u = D^-1 r, w = A u, s = A p):
 *   r = b - A x0, u = D^-1 r, p = s = 0;
 *   repeat w = A u; gamma = r.u; delta = w.u;  stop when ||r|| <= tol ||b||;
 *          beta = gamma / gamma_old (0 at first), alpha = gamma / (delta - beta gamma / alpha_old)
 *          (gamma / delta at first);  p = u + beta p; s = w + beta s;
 *          x += alpha p; r -= alpha s; u = D^-1 r.
 * All three dot products come from one grid reduction fused with the product,
 * so an iteration is two launches instead of three.  The FP64 product is used
 * for every handle (no float-pair products on this path).
 *
 * precision FESPMV_CG_F32_REFINE / FESPMV_CG_BF16_REFINE (the handle must hold the
 * FP32 / BF16 copy, FESPMV_PREC_F32 / FESPMV_PREC_BF16 at create): mixed-precision
 * iterative refinement, x0 = 0 (or x with FESPMV_CG_X0),
 *   repeat: r = b - A x in FP64;  stop when ||r|| <= tol ||b||;
 *           solve B w = S r by plain CG with FP32 vectors and FP32 arithmetic in
 *           the product, FP64 dot products, until ||B w - S r|| <= inner_tol ||S r||
 *           or max_iter inner steps;  x += S w in FP64.
 * diag(B) = 1, so Jacobi on B is the identity.  iters counts inner steps, outer
 * the FP64 residual steps.
 *
 * flag FESPMV_CG_RELIABLE (refined precisions only, else UNSUPPORTED): one inner
 * CG without restarts.  Each time the inner residual has fallen by inner_tol
 * (default 0.1 with this flag) (or
 * its estimate ||r|| ~ c ||r_in||, c = ||r|| / ||S r|| at the last update, reaches
 * tol ||b||) the correction is folded in, x += S w, r = b - A x is recomputed in
 * FP64 and replaces the inner residual (r_in = S r in float), and the search
 * direction is kept: p = r_in + beta p with beta = r_in.r_in / rho ("reliable
 * updates", Sleijpen and van der Vorst 1996).  The solve stops at the first update
 * whose ||r|| <= tol ||b||, or with NOT_CONVERGED when ||r|| did not decrease since
 * the previous update or after max_iter inner steps in total.  outer counts updates.  A refinement step that does not reduce ||r|| ends
 * the solve with FESPMV_ERR_NOT_CONVERGED (the low-precision operator is too
 * far from A for this system: contraction needs cond(B) * u_storage < 1).  Returns FESPMV_OK, FESPMV_ERR_NOT_CONVERGED,
 * FESPMV_ERR_BREAKDOWN (p.Ap <= 0 -- delta - beta gamma / alpha_old <= 0 in the
 * single-reduction form -- non-finite scalars or a non-positive diagonal with
 * Jacobi), INVALID_ARG, UNSUPPORTED, OOM or CUDA.
 *
 * flag FESPMV_CG_FLEXIBLE (refined precisions only, else UNSUPPORTED; not with
 * FESPMV_CG_RELIABLE): the low-precision CG becomes the preconditioner of an
 * FP64 flexible CG (Y. Notay, SIAM J. Sci. Comput. 22, 2000, keeping one
 * previous direction), x0 = 0 (or x with FESPMV_CG_X0):
 *   r = b - A x;  repeat: w = inner_steps steps of CG on B w = S r from w = 0
 *   (FP32 vectors, FP32 or BF16 values, FP64 dots);  z = S w;
 *   p = z (first) or z - (z.q / p.q) p;  q = A p (FP64);  alpha = p.r / p.q;
 *   x += alpha p;  r -= alpha q;  stop when ||r|| <= tol ||b||, confirmed on the
 *   true residual (restarts as FP64 CG).
 * Each step applies a different polynomial in B, which the flexible recurrence
 * tolerates, so BF16 values converge to FP64 accuracy where refinement stalls
 * (cond(B) 2^-8 >= 1).  iters counts outer (FP64) steps, outer the inner steps.
 *
 * Small handles: on a SLICED handle of at most 16,384 rows without float pairs,
 * reliable-update refinement (FESPMV_CG_RELIABLE) runs as one launch of one
 * thread-block cluster (8 CTAs that synchronise with cluster barriers and reduce
 * through distributed shared memory) instead of CUDA graphs of kernel launches:
 * the same recurrences and tests; the reductions run in another fixed order, so
 * the iterates differ from the graphs' in rounding only.  FESPMV_CG_NO_CLUSTER
 * keeps the graphs.  The solve server takes the same path, so a result is bitwise
 * the same alone and served.
 */
int cg_solve(fespmv_mat_t A, const double* b, double* x, const cg_options* opts, cg_result* res,
             fespmv_stream_t stream);

/*
 * cg_solve_csr_static -- cg_solve for a CSR matrix that allocates nothing.
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory -- code that runs inside another framework's
 * memory pool, plugins that must not grow the process's device footprint, and
 * latency-critical loops that cannot block on the allocator -- and therefore
 * cannot create a handle with spmv_create.
 *   n_rows                 at most 262,144 (larger sizes return INVALID_ARG)
 *   rowptr, colind, values device CSR arrays (int64[n+1], int32[nnz], double[nnz]),
 *                          same rules as spmv_create; not validated on the device
 *   b                      device double[n_rows]
 *   x                      device double[n_rows]; initial guess with FESPMV_CG_X0,
 *                          overwritten with the solution
 *   csr_lanes              lanes per row of the CSR kernel (1..32, power of two; 0 = 4)
 *   opts, res              as for cg_solve (IO flags other than FESPMV_CG_X0 and
 *                          FESPMV_CG_NO_PRECOND are rejected)
 * Same Jacobi-PCG recurrences and kernels as cg_solve on a FESPMV_FMT_CSR handle.
 * The workspace (about 8.8 MB) is one fixed device array inside this library;
 * every GPU that loads the library holds it until the process exits.  Each
 * call looks up that array's address on the current device (so a device reset
 * between calls is harmless).  Every call shares the array and leaves its
 * contents behind; each call clears the state it needs, but calls whose work
 * overlaps on the GPU (from several threads or streams) race on the array and
 * must be serialised by the caller.  The call calls no device or host
 * allocator.  It reads the solver's scalars back to the host and synchronises
 * `stream` several times, so it blocks until the solve ends and must not be
 * called while `stream` is being captured into a CUDA graph.
 */
int cg_solve_csr_static(int64_t n_rows, const int64_t* rowptr, const int32_t* colind,
                        const double* values, const double* b, double* x, int32_t csr_lanes,
                        const cg_options* opts, cg_result* res, fespmv_stream_t stream);

/*
 * cg_solve_multi -- solve A x_j = b_j for k right-hand sides of one matrix by k
 * Jacobi-PCG solves run in lockstep (the solver of cg_solve, Sec. 2.1, once per
 * column), so that each iteration streams the matrix once for all columns with
 * the multi-RHS product of spmv_apply_multi.  The paper solves one system at a
 * time; this entry point is the library's batching of right-hand sides.
 *   B, X   n_rows x k doubles, row-major (row i holds b_i1 .. b_ik), device unless
 *          FESPMV_IO_HOST, permuted numbering with FESPMV_IO_PERMUTED; X holds the
 *          initial guesses with FESPMV_CG_X0 and is overwritten with the solutions.
 *   k      1 .. 32
 *   opts   as cg_solve: precision FESPMV_CG_F64 or FESPMV_CG_F32_REFINE (flag
 *          FESPMV_CG_RELIABLE allowed); BF16 and FESPMV_CG_SINGLE_REDUCTION return
 *          UNSUPPORTED.  max_iter bounds each column's iterations in total.
 *   res    NULL or k records, one per column.
 * Each column has its own scalars and stopping test, and its dot products are
 * reduced in a fixed order of their own (p.q: each lane sums the products of its
 * at most 4 rows of a warp's unit in the vectors' precision, and those sums are
 * added in FP64; the other dots in FP64): a column's x is bitwise the same
 * whatever the other columns hold (for the same padded width: k rounded up to
 * 4, 8, 16 or 32).
 *   FESPMV_CG_F64: every stop of the recurrence (||r|| <= tol ||b||) is checked
 *   against the FP64 residual b - A x; above tol the column restarts from x
 *   (max_restarts times).  relres and true_relres are both that FP64 residual.
 *   On a handle created with FESPMV_PREC_DF64 every FP64 product of the solve
 *   (inner and residual) runs as float pairs on the FP32 pipe (see
 *   FESPMV_PREC_DF64), with the p.q sums in FP64.
 *   FESPMV_CG_F32_REFINE: the iterative refinement (or, with FESPMV_CG_RELIABLE,
 *   the reliable updates) of cg_solve, per column, with one difference: a column
 *   whose inner residual has fallen by inner_tol keeps iterating until the next
 *   FP64 outer step (or until it has fallen by inner_tol^3 with reliable updates,
 *   inner_tol^2 without), and those steps come every 8 * check_every inner
 *   iterations (or as soon as no column is iterating); an inner CG also stops
 *   once its residual estimates ||b - A x|| <= tol ||b||.
 * Needs a SLICED handle with one lane per row (threshold 0; UNSUPPORTED
 * otherwise) and, for the refinement, the FP32 copy (FESPMV_PREC_F32).  The
 * workspace (seven n_rows x kw arrays of doubles) is allocated on the first call
 * and grows with kw; the call blocks the host until every column has stopped.
 * Returns FESPMV_OK when every column converged, else the first column's
 * NOT_CONVERGED or BREAKDOWN (a non-positive diagonal: BREAKDOWN for all).
 */
int cg_solve_multi(fespmv_mat_t A, const double* B, double* X, int32_t k, const cg_options* opts,
                   cg_result* res, fespmv_stream_t stream);

/* ---- assembly as a sparse product (Sec. 4) ------------------------------------------ */
typedef struct fespmv_assembly* fespmv_assembly_t;

/*
 * assembly_create -- the map that lets the GPU assemble A's values from element
 * matrices, and global vectors from element vectors, in A's own storage.  Sec. 4
 * writes assembly without atomics as the row sums K^elem 1 of a matrix with one
 * row per global non-zero listing the element contributions to it; here those
 * rows are A's value positions (its packed slices, or the CSR order), each
 * listing its contributions in ascending element order, so that the assembled
 * values equal 0 + c_1 + c_2 + ... summed on the host in element order and
 * loaded with spmv_update_values, bit for bit.
 *   A                 a handle (SLICED or CSR) created from the pattern below
 *   rowptr, colind    the host CSR pattern given to spmv_create (ascending columns)
 *   n_elems, nodes_per_elem, dofs_per_node
 *                     the elements; dof = dofs_per_node * node + c (the same
 *                     dofs_per_node for every node)
 *   elem_nodes        host int32[n_elems * nodes_per_elem]: node numbers of the
 *                     input numbering (0 .. n_rows / dofs_per_node - 1)
 *   dirichlet         host uint8[n_rows] or NULL: rows eliminated symmetrically
 *                     (their stored diagonal becomes 1; entries with a marked row
 *                     or column receive no contribution)
 * The map is built on the host (threads over nodes) and kept on the device:
 * 8 bytes per value position, 4 per contribution (n_elems * m^2 at most,
 * m = nodes_per_elem * dofs_per_node), 4 per element-vector entry.  Errors:
 * INVALID_ARG (sizes, node numbers, n_elems * m^2 >= 2^32, a pattern with
 * another nnz than A's), BAD_CSR (an element contributes to an unmarked entry
 * the pattern does not store; a marked row stores no diagonal), OOM, CUDA.
 */
int assembly_create(fespmv_assembly_t* out, fespmv_mat_t A, const int64_t* rowptr, const int32_t* colind,
                    int64_t n_elems, int32_t nodes_per_elem, int32_t dofs_per_node, const int32_t* elem_nodes,
                    const uint8_t* dirichlet, fespmv_stream_t stream);

/*
 * assembly_matrix -- A's values := the sums of the element matrices'
 * contributions (one thread per value position adds its list), the marked rows'
 * unit diagonals, then A's diagonal, float-pair copy and S with the FP32 / BF16
 * copies of S A S refreshed as spmv_update_values does.
 *   Ke   double[n_elems * m * m], element e's matrix row-major at e * m * m, row and
 *        column dofs_per_node * a + c for component c of local node a; device memory,
 *        or host with FESPMV_IO_HOST (copied to a device buffer kept by the map;
 *        the call then returns after the copy).
 */
int assembly_matrix(fespmv_assembly_t P, const double* Ke, int32_t flags, fespmv_stream_t stream);

/*
 * assembly_vector -- r_I := the sums of the element vectors' entries for dof I in
 * ascending element order, 0 on marked rows (the residual vector of Sec. 4).
 *   Re   device double[n_elems * m], element e's vector at e * m (dofs_per_node * a + c)
 *   r    device double[n_rows]: input numbering, or the handle's with
 *        FESPMV_IO_PERMUTED (SLICED handles)
 */
int assembly_vector(fespmv_assembly_t P, const double* Re, double* r, int32_t flags, fespmv_stream_t stream);

/* Contributions held and device bytes of the map. */
int assembly_get_info(fespmv_assembly_t P, int64_t* n_contributions, int64_t* device_bytes);
void assembly_destroy(fespmv_assembly_t P);

/* ---- Newton updates on a fixed pattern (Sec. 2) ----------------------------------- */

typedef struct {
    int32_t status;      /* FESPMV_OK, NOT_CONVERGED (update limit), or the failing call's code */
    int32_t steps;       /* Newton updates applied */
    int64_t cg_iters;    /* CG iterations over all updates */
    double res_norm0;    /* ||R||_2 of the first residual assembled */
    double res_norm;     /* ||R||_2 of the last residual assembled */
    double dx_norm;      /* ||dx||_2 of the last update */
    cg_result last_cg;   /* the last update's solve */
} fe_newton_result;

/*
 * fe_newton_step -- one global Newton update of Sec. 2 (the algorithm table:
 * assemble the global residual R and iteration matrix K from the element
 * quantities, then phi <- phi - K^-1 R) on the pattern of P's matrix:
 *   R  := the sums of the element residuals (assembly_vector, input numbering)
 *   K  := the sums of the element tangents into P's handle (assembly_matrix)
 *   dx := the solution of K dx = R by cg_solve with opts (FESPMV_CG_X0: dx holds
 *         the initial guess; IO flags are rejected: every vector is device memory
 *         in the input numbering)
 *   phi := phi - dx (skipped when phi is NULL)
 *   Ke, Re   device element tangents / residuals, layouts of assembly_matrix /
 *            assembly_vector (the caller's physics computes them from phi)
 *   R, dx    device double[n_rows], written
 *   out      steps = 1, res_norm = ||R||, dx_norm = ||dx||, last_cg = the solve's result
 * Blocks until the update is applied.  Errors: INVALID_ARG, OOM, CUDA, and the
 * solve's BREAKDOWN / NOT_CONVERGED (phi is then left unchanged).
 */
int fe_newton_step(fespmv_assembly_t P, const double* Ke, const double* Re, double* R, double* dx,
                   double* phi, const cg_options* opts, fe_newton_result* out, fespmv_stream_t stream);

/* The caller's element routine: fill Ke and Re (device) for the current phi
 * (device, input numbering), work ordered on `stream`; return 0, or a non-zero
 * code that stops the iteration. */
typedef int (*fe_element_fn)(const double* phi, double* Ke, double* Re, void* user, fespmv_stream_t stream);

/*
 * fe_newton_solve -- the global Newton loop of Sec. 2 for one time step: call
 * element_fn on phi, assemble R; stop when ||R|| <= newton_tol * ||R_0|| (R_0 the
 * first residual; also when R = 0); otherwise apply fe_newton_step's update and
 * repeat, at most max_steps updates (the residual of the last phi is assembled
 * and tested too).  With FESPMV_CG_X0 in opts every solve starts from the previous
 * update's dx (dx's content on entry for the first).
 *   phi            device double[n_rows], the initial iterate; updated in place
 *   Ke, Re, R, dx  device buffers of assembly_matrix / assembly_vector sizes and n_rows
 *   newton_tol     >= 0; max_steps >= 1
 * Returns FESPMV_OK when the test held, NOT_CONVERGED after max_steps updates, or
 * the failing call's code (the callback's non-zero code becomes INVALID_ARG's
 * message).  out (nullable) gets the counts and norms.
 */
int fe_newton_solve(fespmv_assembly_t P, double* phi, fe_element_fn element_fn, void* user, double* Ke,
                    double* Re, double* R, double* dx, double newton_tol, int32_t max_steps,
                    const cg_options* opts, fe_newton_result* out, fespmv_stream_t stream);

/* ---- batches of independent FE problems ------------------------------------------- */
typedef struct fespmv_batch* fespmv_batch_t;

/*
 * batch_create -- many independent matrices (meshes of uneven sizes) held as one
 * block-diagonal SLICED matrix.  Each problem j is ordered, renumbered and
 * column-sorted on its own (as spmv_create does: Sec. 5.1-5.3) and padded with
 * identity rows to a multiple of 32 rows, so that no warp slice (Sec. 5.1, 5.4)
 * spans two problems; one product then computes every problem's product in a
 * single launch.  The paper treats one matrix at a time; batching is this
 * library's layer on top.
 *   count            number of problems (>= 1)
 *   n_rows[j]        rows of problem j
 *   rowptr[j], colind[j], values[j]   host CSR of problem j (rules of spmv_create)
 *   mesh             NULL or count entries (dofs_per_node, node_xyz per problem)
 *   opts             as spmv_create (format is SLICED; FP32 values of S A S are
 *                    always kept for the refined solver; block <= 256)
 * Host planning runs one thread per core over the problems.
 * Errors: INVALID_ARG, BAD_CSR (message names the problem), OOM, CUDA, UNSUPPORTED.
 */
int batch_create(fespmv_batch_t* out, int32_t count, const int64_t* n_rows,
                 const int64_t* const* rowptr, const int32_t* const* colind,
                 const double* const* values, const fespmv_mesh_info* mesh,
                 const fespmv_options* opts, fespmv_stream_t stream);
void batch_destroy(fespmv_batch_t B);

/* y = A x for every problem at once, FP64.  x, y: device doubles, the problems'
 * vectors concatenated in input numbering (sum of n_rows entries). */
int batch_spmv(fespmv_batch_t B, const double* x, double* y, fespmv_stream_t stream);

/*
 * batch_cg_solve -- solve every problem A_j x_j = b_j by the refined CG of
 * cg_solve (FESPMV_CG_F32_REFINE, the default here, or FESPMV_CG_BF16_REFINE;
 * FESPMV_CG_F64 is taken as F32_REFINE), all problems in lockstep: each
 * refinement step runs one batched FP64 residual, then inner FP32 iterations
 * of all problems still refining, as CUDA graphs of check_every iterations
 * (five launches per iteration for the whole batch), then x_j += S w_j.
 * With FESPMV_CG_RELIABLE each problem keeps its search direction across the
 * FP64 residual steps (reliable updates, as in cg_solve; inner_tol defaults
 * to 0.1 and max_iter bounds each problem's total inner steps).
 * Scalars are per problem; finished problems are skipped by every kernel.
 *   b, x     concatenated vectors (device, or host with FESPMV_IO_HOST);
 *            x: initial guess with FESPMV_CG_X0, else zero; overwritten
 *   results  NULL or count entries
 * Returns FESPMV_OK when every problem converged, else the first failing
 * problem's status (results has each one).
 */
int batch_cg_solve(fespmv_batch_t B, const double* b, double* x, const cg_options* opts,
                   cg_result* results, fespmv_stream_t stream);

/* Sizes: info->n_rows is the total input rows; *padded_rows (may be NULL) the
 * rows of the padded block-diagonal matrix. */
int batch_get_info(fespmv_batch_t B, fespmv_info* info, int64_t* padded_rows);

/* ---- solve server: continuous batching of CG solves ------------------------------- */
typedef struct fespmv_server* fespmv_server_t;

typedef struct {
    double t_queue_s;    /* submit -> admitted to a slot */
    double t_solve_s;    /* admitted -> finished (result on the host) */
    double t_total_s;    /* submit -> finished */
} srv_timing;

typedef struct {
    int64_t submitted, completed, queued, active, peak_active;
    int64_t workspace_bytes, peak_workspace_bytes;
    int64_t grouped;      /* requests admitted to lockstep groups (srv_set_grouping) */
} srv_stats;

/*
 * srv_create -- start a solve server on the current device.  The paper solves
 * one system at a time; this layer serves many CG solves at once, as the
 * Newton steps of several simulations would submit them.
 *   workspace_budget_bytes  device bytes the server may hold for solve
 *                           workspaces (vectors, partial sums); matrices are
 *                           the caller's and not counted
 *   max_active              most solves in flight at once
 * A scheduler thread admits queued requests in arrival order as soon as a slot
 * is free and the request's workspace fits in the budget (idle workspaces are
 * reused for the same matrix and released for others when needed), runs each
 * admitted solve on its own stream, and advances all of them round-robin, one
 * graph of check_every iterations at a time, so their iterations overlap on
 * the device.  A solve in the mix runs the kernels, grids and reduction order
 * of cg_solve, so its x is bitwise equal to cg_solve's on the same handle.
 * Errors: INVALID_ARG, OOM.
 */
int srv_create(fespmv_server_t* out, int64_t workspace_budget_bytes, int32_t max_active);

/*
 * srv_set_grouping -- solve the requests on one matrix together, as the columns
 * of a lockstep multi-RHS CG (the algorithm of cg_solve_multi), so that one pass
 * over the matrix serves all of them.  Each registered matrix gets at most one
 * group at a time, of a fixed width:
 *   width  0 = off (default: every request takes the single path above);
 *          4, 8, 16 or 32 = that many columns for every matrix;
 *          -1 = by size: 32 columns while n_rows * 32 <= 2^21, halved until
 *          n_rows * width <= 2^21, at least 4.
 * A group pays off when it holds two or more right-hand sides, so a request takes
 * it when at least two requests of its matrix wait in the queue or the group
 * already holds two (a lone request takes the single path, which is faster for
 * one right-hand side).  It joins a free column of its matrix's group (wherever it
 * stands in the queue: a full group does not hold up other requests), starts at the group's
 * next FP64 outer step (they come every 8 * check_every inner iterations, or at
 * once when no column iterates) and finishes at the outer step that finds it
 * converged, stopped or broken down; its column is then free for the next
 * request.  Its x is bitwise equal to cg_solve_multi's for that right-hand side
 * alone with the group's width (e.g. k = width with the other columns zero), and
 * within the tolerance of cg_solve's; which path a request takes depends on the
 * load, so with grouping on a result equals one of the two solves alone.  A group counts as one solve toward
 * max_active and holds group workspace (seven n_rows x width arrays of doubles)
 * in the budget; an idle group is kept for reuse and released when the budget
 * needs room.  Requests a group cannot take (FESPMV_CG_BF16_REFINE,
 * FESPMV_CG_SINGLE_REDUCTION, options other than those of its matrix's running
 * group: precision, flags, check_every; a handle that cg_solve_multi rejects)
 * take the single path.  Affects requests admitted after the call.  Errors:
 * INVALID_ARG (bad width).
 */
int srv_set_grouping(fespmv_server_t S, int32_t width);

/* Make handle A solvable by the server; *matrix_id names it in srv_submit.  The
 * handle stays the caller's: it must outlive the server and must not be used
 * by other calls while solves on it are in flight.  Errors: INVALID_ARG, OOM
 * (one workspace of A is larger than the whole budget). */
int srv_register(fespmv_server_t S, fespmv_mat_t A, int32_t* matrix_id);

/* Queue the solve A x = b (b: host double[n_rows] in the input numbering,
 * copied before the call returns; x0 = 0).  opts as for cg_solve except that
 * FESPMV_IO_PERMUTED and FESPMV_CG_X0 are refused.  *ticket identifies the
 * request.  Thread-safe.  Errors: INVALID_ARG, UNSUPPORTED, OOM. */
int srv_submit(fespmv_server_t S, int32_t matrix_id, const double* b, const cg_options* opts,
               int64_t* ticket);

/* Collect a request: with wait = 0 returns FESPMV_PENDING while it runs; once it
 * has finished, writes x (host double[n_rows], may be NULL), res and timing (may
 * be NULL), releases the ticket and returns the solve's status (FESPMV_OK,
 * NOT_CONVERGED, BREAKDOWN, or the error that stopped it).  wait = 1 blocks until
 * the request finishes.  Thread-safe. */
int srv_poll(fespmv_server_t S, int64_t ticket, int32_t wait, double* x, cg_result* res,
             srv_timing* timing);

int srv_get_stats(fespmv_server_t S, srv_stats* stats);

/* Drop every request still waiting for a slot: each finishes with
 * FESPMV_ERR_CANCELLED (collect it with srv_poll as usual); solves already
 * running are not touched.  *n_cancelled (may be NULL) receives the count. */
int srv_cancel_queued(fespmv_server_t S, int64_t* n_cancelled);

/* Finish every queued and running solve, stop the scheduler and free the
 * workspaces (not the registered handles).  Uncollected results are dropped. */
void srv_destroy(fespmv_server_t S);

/* Human-readable name of a status code, and the last failure message of the
 * calling thread (empty if none).  Both strings are static or thread-local. */
const char* fespmv_status_string(int status);
const char* fespmv_last_error(void);

#ifdef __cplusplus
}
#endif

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif
#endif /* FESPMV_H */
