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

// ---------------------------------------------------------------- float-pair FP64 product
// An FP64 value v in the fast range (|v| in [2^-50, 2^50], or 0) is held as two
// floats hi = fl32(v), lo = fl32(v - hi): 48 significant bits, error <= 2^-48 |v|.
// Any other value (tiny, huge, Inf, NaN) is marked by hi = NaN and its product is
// taken in FP64 from the original double (exact slow path).  A product
// a*x = (ah + al)(xh + xl) is formed on the FP32 pipe with an error-free
// product (Dekker/Ogita-Rump-Oishi TwoProduct via FMA) and accumulated with an
// error-free sum (Knuth TwoSum) and a renormalisation after every term, so each
// term adds at most ~2^-47 of (|a x| + |partial sum|) to the error: a row of L
// entries stays within ~(L+2) 2^-47 sum|a x|, under 1e-12 for L < 140.
namespace fespmv {

constexpr float kDfLo = 8.8817841970012523e-16f;   // 2^-50
constexpr float kDfHi = 1.125899906842624e15f;     // 2^50

struct DfAcc {
    float hi = 0.0f, lo = 0.0f;
};

__device__ __forceinline__ void df_add_product(DfAcc& s, float ah, float al, float xh, float xl) {
    const float p = ah * xh;
    const float e = fmaf(ah, xh, -p);
    const float c = fmaf(ah, xl, fmaf(al, xh, e));
    const float t0 = s.hi + p;
    const float bp = t0 - s.hi;
    const float err = (s.hi - (t0 - bp)) + (p - bp);
    const float t = (s.lo + err) + c;
    s.hi = t0 + t;
    s.lo = t - (s.hi - t0);
}

// (a.hi, a.lo) += (b.hi, b.lo): TwoSum of the high parts, then renormalise.
__device__ __forceinline__ void df_add(DfAcc& a, float bh, float bl) {
    const float t0 = a.hi + bh;
    const float bp = t0 - a.hi;
    const float err = (a.hi - (t0 - bp)) + (bh - bp);
    const float t = (a.lo + err) + bl;
    a.hi = t0 + t;
    a.lo = t - (a.hi - t0);
}

__device__ __forceinline__ double df_value(const DfAcc& s) {
    return (double)s.hi + (double)s.lo;
}

// Split with integer operations (no FP64 pipe): hi = v rounded to nearest even
// at 24 bits, lo = v - hi rounded to nearest (exact scaling by 2^(e-52)).  Equal
// to (fl32(v), fl32(v - fl32(v))) for every v in the fast range; 0 -> (0, 0);
// anything else -> (NaN, 0).
__device__ __forceinline__ float2 df_split(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    if ((u << 1) == 0ull) return make_float2(0.0f, 0.0f);
    const int e = (int)((u >> 52) & 0x7ffull) - 1023;
    if (e < -50 || e >= 50) return make_float2(__int_as_float(0x7fc00000), 0.0f);
    const unsigned long long m = u & 0xfffffffffffffull;
    unsigned mh = (unsigned)(m >> 29);
    const long long rem = (long long)(m & 0x1fffffffull);
    const bool up = rem > (1ll << 28) || (rem == (1ll << 28) && (mh & 1u));
    int eh = e;
    if (up && ++mh == (1u << 23)) {   // rounding carried into the exponent
        mh = 0;
        ++eh;
    }
    const unsigned sign = (unsigned)(u >> 63) << 31;
    const float hi = __uint_as_float(sign | ((unsigned)(eh + 127) << 23) | mh);
    const long long d = rem - (up ? (1ll << 29) : 0ll);   // v - hi in units of 2^(e-52)
    float lo = __ll2float_rn(d) * __uint_as_float((unsigned)(e - 52 + 127) << 23);
    if (sign) lo = -lo;
    return make_float2(hi, lo);
}

template <int V> struct DfChunk;
template <> struct DfChunk<1> {
    float2 v[1]; int32_t c[1];
    __device__ __forceinline__ void load(const float2* vp, const int32_t* cp) {
        v[0] = ld_stream(vp); c[0] = ld_stream(cp);
    }
};
template <> struct DfChunk<2> {
    float2 v[2]; int32_t c[2];
    __device__ __forceinline__ void load(const float2* vp, const int32_t* cp) {
        float4 a = ld_stream(reinterpret_cast<const float4*>(vp));
        int2 b = ld_stream(reinterpret_cast<const int2*>(cp));
        v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w); c[0] = b.x; c[1] = b.y;
    }
};
template <> struct DfChunk<4> {
    float2 v[4]; int32_t c[4];
    __device__ __forceinline__ void load(const float2* vp, const int32_t* cp) {
        float4 a = ld_stream(reinterpret_cast<const float4*>(vp));
        float4 a2 = ld_stream(reinterpret_cast<const float4*>(vp) + 1);
        int4 b = ld_stream(reinterpret_cast<const int4*>(cp));
        v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
        v[2] = make_float2(a2.x, a2.y); v[3] = make_float2(a2.z, a2.w);
        c[0] = b.x; c[1] = b.y; c[2] = b.z; c[3] = b.w;
    }
};

// Fast path for one entry: marked values (NaN high parts) make the row's sum NaN,
// which sliced_row_sum_df detects and recomputes in FP64.
__device__ __forceinline__ void df_entry(DfAcc& s, float2 a, int32_t c, const float2* __restrict__ xs) {
    if (c < 0) return;
    const float2 xv = __ldg(xs + c);
    df_add_product(s, a.x, a.y, xv.x, xv.y);
}

template <int V, int U>
__device__ __forceinline__ double sliced_row_sum_df(const uint4 m, const int32_t* __restrict__ col,
                                                    const float2* __restrict__ vdf,
                                                    const double* __restrict__ val,
                                                    const float2* __restrict__ xs,
                                                    const double* __restrict__ x64, int lane) {
    const int64_t off = (int64_t)m.x * 32;
    const int w = (int)m.y;
    const int lt = (int)m.w;
    const int64_t base = off + lane * V;
    DfAcc s;
    int st = 0;
    for (; st + U * V <= w; st += U * V) {
        DfChunk<V> e[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            e[u].load(vdf + base + (int64_t)(st + u * V) * 32, col + base + (int64_t)(st + u * V) * 32);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < V; ++k) df_entry(s, e[u].v[k], e[u].c[k], xs);
    }
    for (; st < w; st += V) {
        DfChunk<V> e;
        e.load(vdf + base + (int64_t)st * 32, col + base + (int64_t)st * 32);
#pragma unroll
        for (int k = 0; k < V; ++k) df_entry(s, e.v[k], e.c[k], xs);
    }
    const int T = 1 << lt;
    for (int o = T >> 1; o > 0; o >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, s.hi, o);
        const float ol = __shfl_down_sync(0xffffffffu, s.lo, o);
        df_add(s, oh, ol);
    }
    // Rows that met a marked value (or a genuine NaN/Inf) are recomputed in FP64
    // from the double values: every lane of such a row sums its own entries again.
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
