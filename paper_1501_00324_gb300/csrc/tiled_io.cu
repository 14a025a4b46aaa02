// The FP64 tiled product for vectors in the input numbering (spmv_apply without
// FESPMV_IO_PERMUTED on a tiled SLICED handle): the row permutation P of the
// locality order and length sort (Sec. 5.1-5.3) folds into the tile staging and
// the row store instead of running as two gathers around the product.
#include <cuda_runtime.h>

#include "internal.h"
#include "tiled_device.cuh"

namespace fespmv {

// y = A x in FP64 with x and y in the input numbering: column c' of the handle's
// numbering is staged from x[P[c']] and row i' stores y[P[i']], so that no separate
// gather runs; the sums are those of sliced_tiled, term for term.
template <int V, int U>
__global__ void __launch_bounds__(kTiledBlock) sliced_tiled_io(const uint4* __restrict__ meta,
                                                               const uint16_t* __restrict__ lidx,
                                                               const double* __restrict__ val,
                                                               const int4* __restrict__ tiles,
                                                               const int32_t* __restrict__ dict,
                                                               const int32_t* __restrict__ perm,
                                                               const double* __restrict__ x, double* __restrict__ y,
                                                               int64_t n) {
    extern __shared__ __align__(16) unsigned char tile_smem[];
    double* xs = reinterpret_cast<double*>(tile_smem);
    const int4 tl = tiles[blockIdx.x];
    for (int e = threadIdx.x; e <= tl.w; e += blockDim.x)
        xs[e] = e < tl.w ? __ldg(x + __ldg(perm + __ldg(dict + tl.z + e))) : 0.0;
    __syncthreads();
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wid >= tl.y) return;
    const uint4 m = meta[tl.x + wid];
    const double sum = tiled_row_sum<double, V, U>(m, lidx, val, xs, lane);
    const int lt = (int)m.w;
    const int64_t row = (int64_t)m.z + (lane >> lt);
    if ((lane & ((1 << lt) - 1)) == 0 && row < n) y[__ldg(perm + row)] = sum;
}

int launch_spmv_tiled_io(const fespmv_mat* A, const double* x, double* y, cudaStream_t s) {
    if (A->n == 0) return FESPMV_OK;
    const size_t smem = sizeof(double) * (size_t)(A->tile_dmax + 1);
    const unsigned g = (unsigned)A->n_tiles;
    switch (A->vec) {
        case 1: sliced_tiled_io<1, 8><<<g, kTiledBlock, smem, s>>>(A->d_meta, A->d_tlidx, A->d_val, A->d_tiles, A->d_tdict, A->d_perm, x, y, A->n); break;
        case 4: sliced_tiled_io<4, 2><<<g, kTiledBlock, smem, s>>>(A->d_meta, A->d_tlidx, A->d_val, A->d_tiles, A->d_tdict, A->d_perm, x, y, A->n); break;
        default: sliced_tiled_io<2, 4><<<g, kTiledBlock, smem, s>>>(A->d_meta, A->d_tlidx, A->d_val, A->d_tiles, A->d_tdict, A->d_perm, x, y, A->n); break;
    }
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

}  // namespace fespmv
