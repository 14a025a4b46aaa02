// Device-side row-sum cores shared by the plain SpMV kernels and the CG kernels.
//
// sliced_row_sum: one warp walks one slice of the packed K1/K2 layout
// (Sec. 5.1, Sec. 5.4) in the renumbered space of Sec. 5.2/5.3.  Lane l owns local
// row l >> log2T; after the call, lanes with (l & (T-1)) == 0 hold their row's sum.
// csr_row_sum: L lanes share one CSR row (L = 1 is CSR scalar, Sec. 4), reduced
// with shuffles inside groups of L lanes; lane sub == 0 holds the sum.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fespmv {

// Matrix stream loads: cache-streaming (evict-first) so that the gathered vector
// keeps its L1/L2 lines.
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }

template <int V> struct Chunk;
template <> struct Chunk<1> {
    double v[1]; int32_t c[1];
    __device__ __forceinline__ void load(const double* vp, const int32_t* cp) {
        v[0] = ld_stream(vp); c[0] = ld_stream(cp);
    }
};
template <> struct Chunk<2> {
    double v[2]; int32_t c[2];
    __device__ __forceinline__ void load(const double* vp, const int32_t* cp) {
        double2 a = ld_stream(reinterpret_cast<const double2*>(vp));
        int2 b = ld_stream(reinterpret_cast<const int2*>(cp));
        v[0] = a.x; v[1] = a.y; c[0] = b.x; c[1] = b.y;
    }
};
template <> struct Chunk<4> {
    double v[4]; int32_t c[4];
    __device__ __forceinline__ void load(const double* vp, const int32_t* cp) {
        double2 a = ld_stream(reinterpret_cast<const double2*>(vp));
        double2 a2 = ld_stream(reinterpret_cast<const double2*>(vp) + 1);
        int4 b = ld_stream(reinterpret_cast<const int4*>(cp));
        v[0] = a.x; v[1] = a.y; v[2] = a2.x; v[3] = a2.y;
        c[0] = b.x; c[1] = b.y; c[2] = b.z; c[3] = b.w;
    }
};

template <int V>
__device__ __forceinline__ void fma_chunk(const Chunk<V>& e, const double* __restrict__ x, double& sum) {
    double xv[V];
#pragma unroll
    for (int k = 0; k < V; ++k) xv[k] = e.c[k] >= 0 ? __ldg(x + e.c[k]) : 0.0;
#pragma unroll
    for (int k = 0; k < V; ++k) sum = fma(e.v[k], xv[k], sum);
}

// U chunks of V steps are loaded before any is consumed: each lane keeps
// U*(8V + 4V) bytes of the matrix stream in flight.
template <int V, int U>
__device__ __forceinline__ double sliced_row_sum_f64(const uint4 m, const int32_t* __restrict__ col,
                                                     const double* __restrict__ val,
                                                     const double* __restrict__ x, int lane) {
    const int64_t off = (int64_t)m.x * 32;
    const int w = (int)m.y;
    const int lt = (int)m.w;
    const double* vp = val + off + lane * V;
    const int32_t* cp = col + off + lane * V;
    double sum = 0.0;
    int s = 0;
    for (; s + U * V <= w; s += U * V) {
        Chunk<V> e[U];
#pragma unroll
        for (int u = 0; u < U; ++u) e[u].load(vp + u * 32 * V, cp + u * 32 * V);
#pragma unroll
        for (int u = 0; u < U; ++u) fma_chunk<V>(e[u], x, sum);
        vp += U * 32 * V;
        cp += U * 32 * V;
    }
    for (; s < w; s += V) {
        Chunk<V> e;
        e.load(vp, cp);
        fma_chunk<V>(e, x, sum);
        vp += 32 * V;
        cp += 32 * V;
    }
    const int T = 1 << lt;
    for (int o = T >> 1; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    return sum;
}

template <int L>
__device__ __forceinline__ double csr_row_sum_f64(int64_t row, int sub, int64_t n,
                                                  const int64_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ col,
                                                  const double* __restrict__ val,
                                                  const double* __restrict__ x) {
    double sum = 0.0;
    if (row < n) {
        const int64_t e = rowptr[row + 1];
        for (int64_t p = rowptr[row] + sub; p < e; p += L) sum = fma(val[p], __ldg(x + col[p]), sum);
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o, L);
    return sum;
}

}  // namespace fespmv

// ---------------------------------------------------------------- low-precision cores
// Values of B = S A S stored as float or bfloat16, x and the sums in float.
#include <cuda_bf16.h>

namespace fespmv {

template <typename VT, int V> struct LowChunk;
template <int V> struct LowChunk<float, V> {
    float v[V]; int32_t c[V];
    __device__ __forceinline__ void load(const float* vp, const int32_t* cp) {
        if constexpr (V == 1) {
            v[0] = ld_stream(vp); c[0] = ld_stream(cp);
        } else if constexpr (V == 2) {
            float2 a = ld_stream(reinterpret_cast<const float2*>(vp));
            int2 b = ld_stream(reinterpret_cast<const int2*>(cp));
            v[0] = a.x; v[1] = a.y; c[0] = b.x; c[1] = b.y;
        } else {
            float4 a = ld_stream(reinterpret_cast<const float4*>(vp));
            int4 b = ld_stream(reinterpret_cast<const int4*>(cp));
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            c[0] = b.x; c[1] = b.y; c[2] = b.z; c[3] = b.w;
        }
    }
};
template <int V> struct LowChunk<__nv_bfloat16, V> {
    float v[V]; int32_t c[V];
    __device__ __forceinline__ void load(const __nv_bfloat16* vp, const int32_t* cp) {
        if constexpr (V == 1) {
            unsigned short u = ld_stream(reinterpret_cast<const unsigned short*>(vp));
            v[0] = __uint_as_float((unsigned)u << 16);
            c[0] = ld_stream(cp);
        } else if constexpr (V == 2) {
            unsigned u = ld_stream(reinterpret_cast<const unsigned*>(vp));
            v[0] = __uint_as_float(u << 16); v[1] = __uint_as_float(u & 0xffff0000u);
            int2 b = ld_stream(reinterpret_cast<const int2*>(cp));
            c[0] = b.x; c[1] = b.y;
        } else {
            uint2 u = ld_stream(reinterpret_cast<const uint2*>(vp));
            v[0] = __uint_as_float(u.x << 16); v[1] = __uint_as_float(u.x & 0xffff0000u);
            v[2] = __uint_as_float(u.y << 16); v[3] = __uint_as_float(u.y & 0xffff0000u);
            int4 b = ld_stream(reinterpret_cast<const int4*>(cp));
            c[0] = b.x; c[1] = b.y; c[2] = b.z; c[3] = b.w;
        }
    }
};

template <typename VT, int V, int U>
__device__ __forceinline__ float sliced_row_sum_low(const uint4 m, const int32_t* __restrict__ col,
                                                    const VT* __restrict__ val,
                                                    const float* __restrict__ x, int lane) {
    const int64_t off = (int64_t)m.x * 32;
    const int w = (int)m.y;
    const int lt = (int)m.w;
    const VT* vp = val + off + lane * V;
    const int32_t* cp = col + off + lane * V;
    float sum = 0.0f;
    int s = 0;
    for (; s + U * V <= w; s += U * V) {
        LowChunk<VT, V> e[U];
#pragma unroll
        for (int u = 0; u < U; ++u) e[u].load(vp + u * 32 * V, cp + u * 32 * V);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < V; ++k)
                sum = fmaf(e[u].v[k], e[u].c[k] >= 0 ? __ldg(x + e[u].c[k]) : 0.0f, sum);
        vp += U * 32 * V;
        cp += U * 32 * V;
    }
    for (; s < w; s += V) {
        LowChunk<VT, V> e;
        e.load(vp, cp);
#pragma unroll
        for (int k = 0; k < V; ++k) sum = fmaf(e.v[k], e.c[k] >= 0 ? __ldg(x + e.c[k]) : 0.0f, sum);
        vp += 32 * V;
        cp += 32 * V;
    }
    const int T = 1 << lt;
    for (int o = T >> 1; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    return sum;
}

template <typename VT>
__device__ __forceinline__ float low_to_float(VT v);
template <> __device__ __forceinline__ float low_to_float<float>(float v) { return v; }
template <> __device__ __forceinline__ float low_to_float<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

template <typename VT, int L>
__device__ __forceinline__ float csr_row_sum_low(int64_t row, int sub, int64_t n,
                                                 const int64_t* __restrict__ rowptr,
                                                 const int32_t* __restrict__ col,
                                                 const VT* __restrict__ val,
                                                 const float* __restrict__ x) {
    float sum = 0.0f;
    if (row < n) {
        const int64_t e = rowptr[row + 1];
        for (int64_t p = rowptr[row] + sub; p < e; p += L)
            sum = fmaf(low_to_float<VT>(val[p]), __ldg(x + col[p]), sum);
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o, L);
    return sum;
}

}  // namespace fespmv
