// Device cores of the x-staging (tiled) products, shared by the plain products
// (tiled.cu) and the CG kernels (cg.cu).
//
// A tile is a run of consecutive K1/K2 warp slices (Sec. 5.1/5.4); its distinct
// columns are gathered once into shared memory, and each stored entry carries a
// 16-bit index into that list (padding: the zero slot after it).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

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

template <typename XT> __device__ __forceinline__ XT zero_of() { return XT(0); }
template <> __device__ __forceinline__ float2 zero_of<float2>() { return make_float2(0.0f, 0.0f); }

// Stage the x values of tile *tile (and the zero slot) into xs; returns the tile.
template <typename XT>
__device__ __forceinline__ int4 stage_tile(const int4* __restrict__ tile, const int32_t* __restrict__ dict,
                                           const XT* __restrict__ x, XT* xs) {
    const int4 tl = *tile;
    for (int e = threadIdx.x; e <= tl.w; e += blockDim.x)
        xs[e] = e < tl.w ? __ldg(x + __ldg(dict + tl.z + e)) : zero_of<XT>();
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

// V consecutive float pairs (16-byte loads for V >= 2).
template <int V>
__device__ __forceinline__ void ld_pairs(const float2* p, float2 (&a)[V]) {
    if constexpr (V == 1) {
        a[0] = ld_stream(p);
    } else {
#pragma unroll
        for (int h = 0; h < V; h += 2) {
            const float4 t = ld_stream(reinterpret_cast<const float4*>(p + h));
            a[h] = make_float2(t.x, t.y);
            a[h + 1] = make_float2(t.z, t.w);
        }
    }
}

// One slice's row sums with float-pair products (values and x as (hi, lo) float
// pairs, double-float sums on the FP32 pipe; see df_add_product), x pairs from
// shared memory.  Rows that meet a marked pair (a value or x outside the pairs'
// range, NaN, Inf) are summed again in FP64 from val, col and x64, as in
// sliced_row_sum_df.
template <int V, int U>
__device__ __forceinline__ double tiled_row_sum_df(const uint4 m, const uint16_t* __restrict__ lidx,
                                                   const float2* __restrict__ vdf,
                                                   const double* __restrict__ val,
                                                   const int32_t* __restrict__ col, const float2* xs,
                                                   const double* __restrict__ x64, int lane) {
    const int64_t off = (int64_t)m.x * 32;
    const int w = (int)m.y;
    const int lt = (int)m.w;
    const float2* vp = vdf + off + lane * V;
    const uint16_t* cp = lidx + off + lane * V;
    DfAcc s;
    int st = 0;
    for (; st + U * V <= w; st += U * V) {
        float2 a[U][V];
        int c[U][V];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ld_pairs<V>(vp + u * 32 * V, a[u]);
            ld_idx<V>(cp + u * 32 * V, c[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const float2 xv = xs[c[u][k]];
                df_add_product(s, a[u][k].x, a[u][k].y, xv.x, xv.y);
            }
        vp += U * 32 * V;
        cp += U * 32 * V;
    }
    for (; st < w; st += V) {
        int c[V];
        float2 a[V];
        ld_pairs<V>(vp, a);
        ld_idx<V>(cp, c);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const float2 xv = xs[c[k]];
            df_add_product(s, a[k].x, a[k].y, xv.x, xv.y);
        }
        vp += 32 * V;
        cp += 32 * V;
    }
    const int T = 1 << lt;
    for (int o = T >> 1; o > 0; o >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, s.hi, o);
        const float ol = __shfl_down_sync(0xffffffffu, s.lo, o);
        df_add(s, oh, ol);
    }
    const bool bad = isnan(s.hi) || isnan(s.lo) || isinf(s.hi);
    const bool row_bad = __shfl_sync(0xffffffffu, bad, lane & ~(T - 1));
    double r = df_value(s);
    if (__any_sync(0xffffffffu, row_bad)) {
        double d = 0.0;
        if (row_bad)
            for (int q = 0; q < w; ++q) {
                const int64_t pos = off + (int64_t)(q / V) * 32 * V + lane * V + q % V;
                const int32_t c = col[pos];
                if (c >= 0) d = fma(val[pos], __ldg(x64 + c), d);
            }
        for (int o = T >> 1; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        if (row_bad) r = d;
    }
    return r;
}

}  // namespace fespmv
