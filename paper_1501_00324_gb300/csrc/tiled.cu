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
#include "spmv_device.cuh"

namespace fespmv {

constexpr int kTiledBlock = 256;  // 8 warps: a tile holds at most 8 slices

// V consecutive stream entries of 16-bit indices / values, converted for the sum.
template <int V>
__device__ __forceinline__ void ld_idx(const uint16_t* p, int (&c)[V]) {
    if constexpr (V == 1) {
        c[0] = ld_stream(reinterpret_cast<const unsigned short*>(p));
    } else if constexpr (V == 2) {
        const unsigned u = ld_stream(reinterpret_cast<const unsigned*>(p));
        c[0] = (int)(u & 0xffffu); c[1] = (int)(u >> 16);
    } else {
        const uint2 u = ld_stream(reinterpret_cast<const uint2*>(p));
        c[0] = (int)(u.x & 0xffffu); c[1] = (int)(u.x >> 16);
        c[2] = (int)(u.y & 0xffffu); c[3] = (int)(u.y >> 16);
    }
}

template <int V>
__device__ __forceinline__ void ld_val(const double* p, double (&v)[V]) {
    if constexpr (V == 1) {
        v[0] = ld_stream(p);
    } else {
#pragma unroll
        for (int h = 0; h < V; h += 2) {
            const double2 t = ld_stream(reinterpret_cast<const double2*>(p + h));
            v[h] = t.x; v[h + 1] = t.y;
        }
    }
}
template <int V>
__device__ __forceinline__ void ld_val(const float* p, float (&v)[V]) {
    if constexpr (V == 1) {
        v[0] = ld_stream(p);
    } else if constexpr (V == 2) {
        const float2 t = ld_stream(reinterpret_cast<const float2*>(p));
        v[0] = t.x; v[1] = t.y;
    } else {
        const float4 t = ld_stream(reinterpret_cast<const float4*>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
}
template <int V>
__device__ __forceinline__ void ld_val(const __nv_bfloat16* p, float (&v)[V]) {
    if constexpr (V == 1) {
        const unsigned short u = ld_stream(reinterpret_cast<const unsigned short*>(p));
        v[0] = __uint_as_float((unsigned)u << 16);
    } else if constexpr (V == 2) {
        const unsigned u = ld_stream(reinterpret_cast<const unsigned*>(p));
        v[0] = __uint_as_float(u << 16); v[1] = __uint_as_float(u & 0xffff0000u);
    } else {
        const uint2 u = ld_stream(reinterpret_cast<const uint2*>(p));
        v[0] = __uint_as_float(u.x << 16); v[1] = __uint_as_float(u.x & 0xffff0000u);
        v[2] = __uint_as_float(u.y << 16); v[3] = __uint_as_float(u.y & 0xffff0000u);
    }
}

template <typename VT> struct SumOf { using type = float; };   // float and bf16 values: float sums
template <> struct SumOf<double> { using type = double; };

// Stage the tile's x values (and the zero slot) into xs; returns the tile.
template <typename XT>
__device__ __forceinline__ int4 stage_tile(const int4* __restrict__ tiles, const int32_t* __restrict__ dict,
                                           const XT* __restrict__ x, XT* xs) {
    const int4 tl = tiles[blockIdx.x];
    for (int e = threadIdx.x; e <= tl.w; e += blockDim.x) xs[e] = e < tl.w ? __ldg(x + __ldg(dict + tl.z + e)) : XT(0);
    __syncthreads();
    return tl;
}

// One slice's row sums from shared-memory x: lanes with (lane & (T-1)) == 0 hold
// their row's sum (the slice layout of Sec. 5.1/5.4, U chunks of V steps in flight).
template <typename VT, int V, int U>
__device__ __forceinline__ typename SumOf<VT>::type tiled_row_sum(const uint4 m, const uint16_t* __restrict__ lidx,
                                                                  const VT* __restrict__ val,
                                                                  const typename SumOf<VT>::type* xs, int lane) {
    using ST = typename SumOf<VT>::type;
    const int64_t off = (int64_t)m.x * 32 + lane * V;
    const int w = (int)m.y;
    const VT* vp = val + off;
    const uint16_t* cp = lidx + off;
    ST sum = ST(0);
    int s = 0;
    for (; s + U * V <= w; s += U * V) {
        ST v[U][V];
        int c[U][V];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ld_val<V>(vp + u * 32 * V, v[u]);
            ld_idx<V>(cp + u * 32 * V, c[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < V; ++k) sum = fma(v[u][k], xs[c[u][k]], sum);
        vp += U * 32 * V;
        cp += U * 32 * V;
    }
    for (; s < w; s += V) {
        ST v[V];
        int c[V];
        ld_val<V>(vp, v);
        ld_idx<V>(cp, c);
#pragma unroll
        for (int k = 0; k < V; ++k) sum = fma(v[k], xs[c[k]], sum);
        vp += 32 * V;
        cp += 32 * V;
    }
    const int T = 1 << (int)m.w;
    for (int o = T >> 1; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    return sum;
}

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
    const int4 tl = stage_tile<ST>(tiles, dict, x, xs);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wid >= tl.y) return;
    const uint4 m = meta[tl.x + wid];
    const ST sum = tiled_row_sum<VT, V, U>(m, lidx, val, xs, lane);
    const int lt = (int)m.w;
    const int64_t row = (int64_t)m.z + (lane >> lt);
    if ((lane & ((1 << lt) - 1)) == 0 && row < n) y[row] = sum;
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
