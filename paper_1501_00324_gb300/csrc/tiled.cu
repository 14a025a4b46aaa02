// Products with x staged through shared memory (SLICED handles with tiles).
//
// The K1/K2 warp slices of Sec. 5.1/5.4 are grouped into tiles of consecutive
// slices (at most one slice per warp of the block).  A tile's distinct columns
// form its dictionary; next to each packed value the layout stores the entry's
// 16-bit index into that dictionary instead of a 32-bit column.  A block
// gathers the tile's x values into shared memory once (each is then read by
// about six entries of an FE slice), and its warps walk their slices exactly as
// the global-gather kernels do, reading x from shared memory.  Padding entries
// index a zero slot after the dictionary, so they add 0 whatever x holds.
//
// Bytes from HBM per stored entry: value + 2 (index) instead of value + 4, plus
// the dictionaries (4 bytes per distinct column per tile, ~0.2-0.4 per entry).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "internal.h"
#include "tiled_device.cuh"

namespace fespmv {

// y = A x (FP64 values), or y = B x with B's FP32 / BF16 values and float x, y.
template <typename VT, int V, int U>
__global__ void __launch_bounds__(kTiledBlock) sliced_tiled(const uint4* __restrict__ meta,
                                                            const uint16_t* __restrict__ lidx,
                                                            const VT* __restrict__ val,
                                                            const int4* __restrict__ tiles,
                                                            const int32_t* __restrict__ dict,
                                                            const typename SumOf<VT>::type* __restrict__ x,
                                                            typename SumOf<VT>::type* __restrict__ y, int64_t n) {
    using ST = typename SumOf<VT>::type;
    extern __shared__ __align__(16) unsigned char tile_smem[];
    ST* xs = reinterpret_cast<ST*>(tile_smem);
    const int4 tl = stage_tile<ST>(tiles + blockIdx.x, dict, x, xs);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wid >= tl.y) return;
    const uint4 m = meta[tl.x + wid];
    const ST sum = tiled_row_sum<VT, V, U>(m, lidx, val, xs, lane);
    const int lt = (int)m.w;
    const int64_t row = (int64_t)m.z + (lane >> lt);
    if ((lane & ((1 << lt) - 1)) == 0 && row < n) y[row] = sum;
}

// y = A x with float-pair products (FESPMV_PREC_DF64 handles), x pairs staged per tile.
template <int V, int U>
__global__ void __launch_bounds__(kTiledBlock) sliced_tiled_df(const uint4* __restrict__ meta,
                                                               const uint16_t* __restrict__ lidx,
                                                               const float2* __restrict__ vdf,
                                                               const double* __restrict__ val,
                                                               const int32_t* __restrict__ col,
                                                               const int4* __restrict__ tiles,
                                                               const int32_t* __restrict__ dict,
                                                               const float2* __restrict__ xdf,
                                                               const double* __restrict__ x,
                                                               double* __restrict__ y, int64_t n) {
    extern __shared__ __align__(16) unsigned char tile_smem[];
    float2* xs = reinterpret_cast<float2*>(tile_smem);
    const int4 tl = stage_tile<float2>(tiles + blockIdx.x, dict, xdf, xs);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wid >= tl.y) return;
    const uint4 m = meta[tl.x + wid];
    const double sum = tiled_row_sum_df<V, U>(m, lidx, vdf, val, col, xs, x, lane);
    const int lt = (int)m.w;
    const int64_t row = (int64_t)m.z + (lane >> lt);
    if ((lane & ((1 << lt) - 1)) == 0 && row < n) y[row] = sum;
}

int launch_spmv_df_tiled(const fespmv_mat* A, const float2* xdf, const double* x, double* y, cudaStream_t s) {
    if (A->n == 0) return FESPMV_OK;
    const size_t smem = sizeof(float2) * (size_t)(A->tile_dmax + 1);
    const unsigned g = (unsigned)A->n_tiles;
    switch (A->vec) {
        case 1: sliced_tiled_df<1, 8><<<g, kTiledBlock, smem, s>>>(A->d_meta, A->d_tlidx, A->d_vdf, A->d_val, A->d_col, A->d_tiles, A->d_tdict, xdf, x, y, A->n); break;
        case 4: sliced_tiled_df<4, 2><<<g, kTiledBlock, smem, s>>>(A->d_meta, A->d_tlidx, A->d_vdf, A->d_val, A->d_col, A->d_tiles, A->d_tdict, xdf, x, y, A->n); break;
        default: sliced_tiled_df<2, 4><<<g, kTiledBlock, smem, s>>>(A->d_meta, A->d_tlidx, A->d_vdf, A->d_val, A->d_col, A->d_tiles, A->d_tdict, xdf, x, y, A->n); break;
    }
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

template <typename VT, int V>
static void launch_tiled_t(const fespmv_mat* A, const VT* val, const typename SumOf<VT>::type* x,
                           typename SumOf<VT>::type* y, cudaStream_t s) {
    using ST = typename SumOf<VT>::type;
    constexpr int U = (V == 1) ? 8 : (V == 2 ? 4 : 2);
    const size_t smem = sizeof(ST) * (size_t)(A->tile_dmax + 1);
    sliced_tiled<VT, V, U><<<(unsigned)A->n_tiles, kTiledBlock, smem, s>>>(A->d_meta, A->d_tlidx, val, A->d_tiles,
                                                                          A->d_tdict, x, y, A->n);
}

template <typename VT>
static void dispatch_tiled(const fespmv_mat* A, const VT* val, const typename SumOf<VT>::type* x,
                           typename SumOf<VT>::type* y, cudaStream_t s) {
    switch (A->vec) {
        case 1: launch_tiled_t<VT, 1>(A, val, x, y, s); break;
        case 4: launch_tiled_t<VT, 4>(A, val, x, y, s); break;
        default: launch_tiled_t<VT, 2>(A, val, x, y, s); break;
    }
}

int launch_spmv_tiled(const fespmv_mat* A, const double* x, double* y, cudaStream_t s) {
    if (A->n == 0) return FESPMV_OK;
    dispatch_tiled<double>(A, A->d_val, x, y, s);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

int launch_spmv_low_tiled(const fespmv_mat* A, int precision, const float* x, float* y, cudaStream_t s) {
    if (A->n == 0) return FESPMV_OK;
    if (precision == FESPMV_PREC_F32)
        dispatch_tiled<float>(A, A->d_val32, x, y, s);
    else
        dispatch_tiled<__nv_bfloat16>(A, reinterpret_cast<const __nv_bfloat16*>(A->d_val16), x, y, s);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

}  // namespace fespmv
