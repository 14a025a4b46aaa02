// Products of 3x3 node blocks (SLICED handles created with node_blocks = 3).
//
// For three dofs per node (linear elasticity) the stiffness matrix is a matrix
// of 3x3 blocks: the rows of node I touch the same column nodes J.  Storing one
// int32 block column per 9 values instead of one column index per value cuts
// the index stream from 2-4 bytes per value to 4/9 of a byte, and one gather of
// x[3J..3J+2] serves nine products.  The slices are those of Sec. 5.1 (K1, one
// warp per 32 rows, column-major, padded to the longest row) over node rows:
// a lane holds the three rows of one node and walks its blocks in ascending
// column order, so each row's sum runs over its columns in ascending order,
// as the scalar slices do.  Values are B = S A S in FP32 or BF16 (the refined
// CG's inner operator); a block stores zeros where the matrix has no entry.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "spmv_device.cuh"
#include "nodeblock_device.cuh"

namespace fespmv {

// y = B x over node blocks: one warp per slice.
template <typename VT, int U>
__global__ void __launch_bounds__(256) nb3_product(const uint4* __restrict__ meta, const int32_t* __restrict__ col,
                                                   const VT* __restrict__ val, const float* __restrict__ x,
                                                   float* __restrict__ y, int64_t n_nodes, int64_t n_slices) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (warp >= n_slices) return;
    const int lane = threadIdx.x & 31;
    float s[3];
    const uint4 m = meta[warp];
    nb3_row_sums<VT, U>(m, col, val, x, lane, s);
    const int64_t node = (int64_t)m.z + lane;
    if (node < n_nodes) {
        y[3 * node] = s[0];
        y[3 * node + 1] = s[1];
        y[3 * node + 2] = s[2];
    }
}

// The same with x staged per tile (one block per tile of at most 8 slices).
template <typename VT, int U>
__global__ void __launch_bounds__(256, 8) nb3_product_tiled(const uint4* __restrict__ meta,
                                                         const uint16_t* __restrict__ lidx,
                                                         const VT* __restrict__ val, const int4* __restrict__ tiles,
                                                         const int32_t* __restrict__ dict,
                                                         const float* __restrict__ x, float* __restrict__ y,
                                                         int64_t n_nodes) {
    extern __shared__ __align__(16) unsigned char nb_smem[];
    float* xs = reinterpret_cast<float*>(nb_smem);
    const int4 tl = nb3_stage(tiles + blockIdx.x, dict, x, xs);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wid >= tl.y) return;
    const uint4 m = meta[tl.x + wid];
    float s[3];
    nb3_row_sums_tiled<VT, U>(m, lidx, val, xs, lane, s);
    const int64_t node = (int64_t)m.z + lane;
    if (node < n_nodes) {
        y[3 * node] = s[0];
        y[3 * node + 1] = s[1];
        y[3 * node + 2] = s[2];
    }
}

// Node-block copies of the FP32 / BF16 values: each value slot takes the packed
// scalar copy's value at its mapped position (0 where the block has no entry),
// so both layouts hold the same bits.
__global__ void nb3_gather(const int64_t* __restrict__ map, const float* __restrict__ v32,
                           const uint16_t* __restrict__ v16, float* __restrict__ o32, uint16_t* __restrict__ o16,
                           int64_t len) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = map[i];
        if (o32) o32[i] = p >= 0 ? v32[p] : 0.0f;
        if (o16) o16[i] = p >= 0 ? v16[p] : (uint16_t)0;
    }
}

int launch_nb3_refresh(fespmv_mat* A, cudaStream_t s) {
    if (!A->nb || A->nb_len == 0) return FESPMV_OK;
    const int64_t len = 9 * A->nb_len;
    nb3_gather<<<grid_for(len, 256), 256, 0, s>>>(A->d_nbmap, A->d_val32, A->d_val16, A->d_nb32, A->d_nb16, len);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

int launch_nb3_product(const fespmv_mat* A, int precision, const float* x, float* y, cudaStream_t s) {
    if (A->n == 0) return FESPMV_OK;
    if (A->nb_tiles > 0) {
        const size_t smem = sizeof(float) * 3 * (size_t)(A->nb_tile_dmax + 1);
        const unsigned g = (unsigned)A->nb_tiles;
        if (precision == FESPMV_PREC_F32)
            nb3_product_tiled<float, 2><<<g, 256, smem, s>>>(A->d_nbmeta, A->d_nbtlidx, A->d_nb32, A->d_nbtiles,
                                                             A->d_nbtdict, x, y, A->n / 3);
        else
            nb3_product_tiled<__nv_bfloat16, 4><<<g, 256, smem, s>>>(
                A->d_nbmeta, A->d_nbtlidx, reinterpret_cast<const __nv_bfloat16*>(A->d_nb16), A->d_nbtiles,
                A->d_nbtdict, x, y, A->n / 3);
        FESPMV_CUDA(cudaGetLastError());
        return FESPMV_OK;
    }
    const unsigned g = grid_for(A->nb_slices * 32, 256);
    if (precision == FESPMV_PREC_F32)
        nb3_product<float, 2><<<g, 256, 0, s>>>(A->d_nbmeta, A->d_nbcol, A->d_nb32, x, y, A->n / 3, A->nb_slices);
    else
        nb3_product<__nv_bfloat16, 2><<<g, 256, 0, s>>>(A->d_nbmeta, A->d_nbcol,
                                                        reinterpret_cast<const __nv_bfloat16*>(A->d_nb16), x, y,
                                                        A->n / 3, A->nb_slices);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

}  // namespace fespmv
