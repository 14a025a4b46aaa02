// Products with many right-hand sides sharing one pass over the matrix
// (spmv_apply_multi in fespmv.h): Y = A X, X and Y row-major n x k, k <= 32.
//
// The kernel works on X and Y with a padded row stride KW (4, 8, 16 or 32 >= k)
// in the renumbered space of Sec. 5.2.  A warp covers RW rows of one K1 slice
// (Sec. 5.1, one lane per row in the stored layout); its lanes form G groups of
// KW/4 lanes, each lane owning 4 consecutive right-hand sides, and group g owns
// RW/G consecutive rows of the slice.  Per stored step a group reads the V
// entries of each of its rows, gathers the KW-wide row of X named by each column
// index with one 16-byte (FP32) or 32-byte (FP64) load per lane, and applies it
// with 4 FMAs per lane.  So one warp instruction advances G entries, the matrix
// streams from HBM once for all k columns, and every gather is a full, aligned
// line of X.
//
// Row-to-row reuse: in an FE matrix the dofs of one node have the same columns,
// and the locality order keeps them adjacent, so consecutive rows of a group
// often name the same column at the same step.  A gather is predicated off when
// the column equals the previous row's at that step; the registers still hold
// that row of X.  The FMAs of padding entries (column -1) are skipped, so a NaN
// in X never reaches a row that does not store its column.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "spmv_device.cuh"

namespace fespmv {

// Four consecutive X values at p, loaded only when `take` is set (otherwise the
// registers keep their contents).  Read-only path: X is not written here.
__device__ __forceinline__ void ld_x4(const float* p, bool take, float (&v)[4]) {
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
        "@q ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%5];\n\t}"
        : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3])
        : "r"((int)take), "l"(p));
}
__device__ __forceinline__ void ld_x4(const double* p, bool take, double (&v)[4]) {
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
        "@q ld.global.nc.v2.f64 {%0, %1}, [%5];\n\t"
        "@q ld.global.nc.v2.f64 {%2, %3}, [%5+16];\n\t}"
        : "+d"(v[0]), "+d"(v[1]), "+d"(v[2]), "+d"(v[3])
        : "r"((int)take), "l"(p));
}

// V consecutive stream entries (column indices or values) at p.
template <int V> __device__ __forceinline__ void ld_v(const int32_t* p, int32_t (&c)[V]) {
    if constexpr (V == 1) {
        c[0] = ld_stream(p);
    } else if constexpr (V == 2) {
        const int2 t = ld_stream(reinterpret_cast<const int2*>(p));
        c[0] = t.x; c[1] = t.y;
    } else {
        const int4 t = ld_stream(reinterpret_cast<const int4*>(p));
        c[0] = t.x; c[1] = t.y; c[2] = t.z; c[3] = t.w;
    }
}
template <int V> __device__ __forceinline__ void ld_v(const float* p, float (&a)[V]) {
    if constexpr (V == 1) {
        a[0] = ld_stream(p);
    } else if constexpr (V == 2) {
        const float2 t = ld_stream(reinterpret_cast<const float2*>(p));
        a[0] = t.x; a[1] = t.y;
    } else {
        const float4 t = ld_stream(reinterpret_cast<const float4*>(p));
        a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
    }
}
template <int V> __device__ __forceinline__ void ld_v(const double* p, double (&a)[V]) {
    if constexpr (V == 1) {
        a[0] = ld_stream(p);
    } else {
#pragma unroll
        for (int h = 0; h < V; h += 2) {
            const double2 t = ld_stream(reinterpret_cast<const double2*>(p + h));
            a[h] = t.x; a[h + 1] = t.y;
        }
    }
}

// One warp's unit of work: RW rows of one slice (unit gw = slice * 32/RW + part),
// all KW columns; stores the rows of Y and leaves the sums in acc (per group
// row i, this lane's 4 columns).
template <typename VT, typename XT, int V, int KW, int RW>
__device__ __forceinline__ void multi_unit(const uint4* __restrict__ meta, const int32_t* __restrict__ col,
                                           const VT* __restrict__ val, const XT* __restrict__ X,
                                           XT* __restrict__ Y, int64_t gw, int64_t n, int lane,
                                           XT (&acc)[RW / (32 / (KW / 4))][4]) {
    constexpr int LPG = KW / 4;  // lanes per group
    constexpr int G = 32 / LPG;  // groups per warp
    constexpr int R = RW / G;    // rows per group
    constexpr int WPS = 32 / RW; // warps per slice
    static_assert(R >= 1 && RW * WPS == 32, "bad multi-RHS tiling");
    const int64_t slice = gw / WPS;
    const int g = lane / LPG, q = lane % LPG;
    const uint4 m = meta[slice];
    const int first_row = (int)(gw % WPS) * RW + g * R;  // first local row of this group
    const int64_t off = (int64_t)m.x * 32 + (int64_t)first_row * V;
    const int w = (int)m.y;
    const int32_t* cp = col + off;
    const VT* vp = val + off;
    const XT* Xq = X + 4 * q;

#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = XT(0);
    XT xr[V][4];
#pragma unroll
    for (int t = 0; t < V; ++t)
#pragma unroll
        for (int j = 0; j < 4; ++j) xr[t][j] = XT(0);

    for (int s = 0; s < w; s += V) {
        // this group's rows at V steps; more warps in flight (registers freed by not
        // double-buffering these loads) hide their latency better than a prefetch
        int32_t c[R][V];
        VT a[R][V];
        const int64_t o = (int64_t)s * 32;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            ld_v<V>(cp + o + i * V, c[i]);
            ld_v<V>(vp + o + i * V, a[i]);
        }
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
            for (int t = 0; t < V; ++t) {
                const int cc = c[i][t];
                const bool take = cc >= 0 && (i == 0 || cc != c[i - 1][t]);
                ld_x4(Xq + (int64_t)cc * KW, take, xr[t]);
                if (cc >= 0) {
                    const XT av = (XT)a[i][t];
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(av, xr[t][j], acc[i][j]);
                }
            }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int64_t row = (int64_t)m.z + first_row + i;
        if (row < n) {
            XT* yp = Y + row * KW + 4 * q;
            if constexpr (std::is_same<XT, float>::value) {
                *reinterpret_cast<float4*>(yp) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            } else {
                reinterpret_cast<double2*>(yp)[0] = make_double2(acc[i][0], acc[i][1]);
                reinterpret_cast<double2*>(yp)[1] = make_double2(acc[i][2], acc[i][3]);
            }
        }
    }
}

template <typename VT, typename XT, int V, int KW, int RW>
__global__ void __launch_bounds__(128, 4) sliced_multi(const uint4* __restrict__ meta,
                                                       const int32_t* __restrict__ col,
                                                       const VT* __restrict__ val,
                                                       const XT* __restrict__ X, XT* __restrict__ Y,
                                                       int64_t n_slices, int64_t n) {
    constexpr int R = RW / (32 / (KW / 4));
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (gw >= n_slices * (32 / RW)) return;
    XT acc[R][4];
    multi_unit<VT, XT, V, KW, RW>(meta, col, val, X, Y, gw, n, threadIdx.x & 31, acc);
}

// The product of the lockstep CG of cg_solve_multi: Q = A P as sliced_multi
// computes it, and for every column j the sum of p_ij q_ij over the rows this
// block covered at part[blockIdx.x * KW + j].  Each lane sums the products of
// its (at most 4) rows of a unit in the vectors' precision and accumulates those
// sums in FP64: FP32 inner vectors then spend one conversion and one FP64 add per
// unit and column instead of two conversions and a DFMA per row (the FP64 pipe,
// which the conversions also occupy, was 45 % busy); the FP32 bound (6 blocks of
// 128 threads per SM) gives it the occupancy of the plain product.
// The grid is resident (persistent): each warp strides over the units, so the
// partial sums stay few.
template <typename VT, typename XT, int V, int KW, int RW>
__global__ void __launch_bounds__(128, sizeof(XT) == 4 ? 6 : 4) sliced_multi_dot(const uint4* __restrict__ meta,
                                                           const int32_t* __restrict__ col,
                                                           const VT* __restrict__ val,
                                                           const XT* __restrict__ P, XT* __restrict__ Q,
                                                           int64_t n_slices, int64_t n,
                                                           double* __restrict__ part) {
    constexpr int LPG = KW / 4, G = 32 / LPG, R = RW / G, WPS = 32 / RW;
    __shared__ double sh[4][KW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int g = lane / LPG, q = lane % LPG;
    double d[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t units = n_slices * WPS;
    for (int64_t gw = (int64_t)blockIdx.x * 4 + wib; gw < units; gw += (int64_t)gridDim.x * 4) {
        XT acc[R][4];
        multi_unit<VT, XT, V, KW, RW>(meta, col, val, P, Q, gw, n, lane, acc);
        const int64_t row0 = (int64_t)meta[gw / WPS].z + (int)(gw % WPS) * RW + g * R;
        XT t[4] = {XT(0), XT(0), XT(0), XT(0)};
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (row0 + i < n) {
                XT pv[4] = {XT(0), XT(0), XT(0), XT(0)};
                ld_x4(P + (row0 + i) * KW + 4 * q, true, pv);
#pragma unroll
                for (int j = 0; j < 4; ++j) t[j] = fma(pv[j], acc[i][j], t[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) d[j] += (double)t[j];
    }
    // lanes with the same q hold the same columns: sum over the warp's groups
#pragma unroll
    for (int o = LPG; o < 32; o <<= 1)
#pragma unroll
        for (int j = 0; j < 4; ++j) d[j] += __shfl_xor_sync(0xffffffffu, d[j], o);
    if (g == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j) sh[wib][4 * q + j] = d[j];
    __syncthreads();
    if (threadIdx.x < KW)
        part[(int64_t)blockIdx.x * KW + threadIdx.x] =
            ((sh[0][threadIdx.x] + sh[1][threadIdx.x]) + sh[2][threadIdx.x]) + sh[3][threadIdx.x];
}

// ---------------------------------------------------------------- FP64 by float pairs
// FESPMV_PREC_DF64 handles: the same lane groups and row-to-row reuse, with every
// product and sum as float pairs on the FP32 pipe (df_add_product: the pair
// product with its FMA error terms, double-float sums), X split into pairs.  One
// DFMA per stored entry and right-hand side is what bounds the FP64 kernel above
// (GB300 retires ~1.9 FP64 lanes per clock per SM); the FP32 pipe is ~58x wider.
// Rows whose pair sums meet a marked pair (a value or an X entry outside the
// pairs' range, NaN, Inf) are summed again in FP64 from val, col and X64.

// Four float pairs at p (32 bytes), loaded only when `take` is set.
__device__ __forceinline__ void ld_x4_pairs(const float2* p, bool take, float2 (&v)[4]) {
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %8, 0;\n\t"
        "@q ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%9];\n\t"
        "@q ld.global.nc.v4.f32 {%4, %5, %6, %7}, [%9+16];\n\t}"
        : "+f"(v[0].x), "+f"(v[0].y), "+f"(v[1].x), "+f"(v[1].y), "+f"(v[2].x), "+f"(v[2].y),
          "+f"(v[3].x), "+f"(v[3].y)
        : "r"((int)take), "l"(p));
}

template <int V>
__device__ __forceinline__ void ld_v_pairs(const float2* p, float2 (&a)[V]) {
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

// One warp's unit of a float-pair product: as multi_unit, every product and sum as
// float pairs; rows whose pair sums meet a marked pair are summed again in FP64.
// Stores the rows of Y and leaves their values in out.
template <int V, int KW, int RW>
__device__ __forceinline__ void multi_unit_df(const uint4* __restrict__ meta, const int32_t* __restrict__ col,
                                              const float2* __restrict__ vdf, const double* __restrict__ val,
                                              const float2* __restrict__ Xdf, const double* __restrict__ X64,
                                              double* __restrict__ Y, int64_t gw, int64_t n, int lane,
                                              double (&out)[RW / (32 / (KW / 4))][4]) {
    constexpr int LPG = KW / 4, G = 32 / LPG, R = RW / G, WPS = 32 / RW;
    static_assert(R >= 1 && RW * WPS == 32, "bad multi-RHS tiling");
    const int64_t slice = gw / WPS;
    const int g = lane / LPG, q = lane % LPG;
    const uint4 m = meta[slice];
    const int first_row = (int)(gw % WPS) * RW + g * R;
    const int64_t off = (int64_t)m.x * 32 + (int64_t)first_row * V;
    const int w = (int)m.y;
    const int32_t* cp = col + off;
    const float2* vp = vdf + off;
    const float2* Xq = Xdf + 4 * q;

    DfAcc acc[R][4];
    float2 xr[V][4];
#pragma unroll
    for (int t = 0; t < V; ++t)
#pragma unroll
        for (int j = 0; j < 4; ++j) xr[t][j] = make_float2(0.f, 0.f);
    for (int s = 0; s < w; s += V) {
        int32_t c[R][V];
        float2 a[R][V];
        const int64_t o = (int64_t)s * 32;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            ld_v<V>(cp + o + i * V, c[i]);
            ld_v_pairs<V>(vp + o + i * V, a[i]);
        }
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
            for (int t = 0; t < V; ++t) {
                const int cc = c[i][t];
                const bool take = cc >= 0 && (i == 0 || cc != c[i - 1][t]);
                ld_x4_pairs(Xq + (int64_t)cc * KW, take, xr[t]);
                if (cc >= 0) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) df_add_product(acc[i][j], a[i][t].x, a[i][t].y, xr[t][j].x, xr[t][j].y);
                }
            }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int64_t row = (int64_t)m.z + first_row + i;
        double* yv = out[i];
        bool bad = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            bad |= isnan(acc[i][j].hi) || isnan(acc[i][j].lo) || isinf(acc[i][j].hi);
            yv[j] = df_value(acc[i][j]);
        }
        if (bad) {   // this lane's four sums of the row again, in FP64
#pragma unroll
            for (int j = 0; j < 4; ++j) yv[j] = 0.0;
            for (int s2 = 0; s2 < w; ++s2) {
                const int64_t pos = (int64_t)m.x * 32 + (int64_t)(s2 / V) * 32 * V + (int64_t)(first_row + i) * V + s2 % V;
                const int32_t cc = col[pos];
                if (cc >= 0) {
                    const double av = val[pos];
#pragma unroll
                    for (int j = 0; j < 4; ++j) yv[j] = fma(av, X64[(int64_t)cc * KW + 4 * q + j], yv[j]);
                }
            }
        }
        if (row < n) {
            double* yp = Y + row * KW + 4 * q;
            reinterpret_cast<double2*>(yp)[0] = make_double2(yv[0], yv[1]);
            reinterpret_cast<double2*>(yp)[1] = make_double2(yv[2], yv[3]);
        }
    }
}

template <int V, int KW, int RW>
__global__ void __launch_bounds__(128, 4) sliced_multi_df(const uint4* __restrict__ meta,
                                                          const int32_t* __restrict__ col,
                                                          const float2* __restrict__ vdf,
                                                          const double* __restrict__ val,
                                                          const float2* __restrict__ Xdf,
                                                          const double* __restrict__ X64,
                                                          double* __restrict__ Y, int64_t n_slices,
                                                          int64_t n) {
    constexpr int R = RW / (32 / (KW / 4));
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (gw >= n_slices * (32 / RW)) return;
    double out[R][4];
    multi_unit_df<V, KW, RW>(meta, col, vdf, val, Xdf, X64, Y, gw, n, threadIdx.x & 31, out);
}

// The FP64 product of the lockstep CG on a float-pair handle: Q = A P as
// sliced_multi_df computes it (P given in double and split into pairs), and the
// per-column sums of p_ij q_ij as sliced_multi_dot forms them, in FP64.
template <int V, int KW, int RW>
__global__ void __launch_bounds__(128, 4) sliced_multi_df_dot(const uint4* __restrict__ meta,
                                                              const int32_t* __restrict__ col,
                                                              const float2* __restrict__ vdf,
                                                              const double* __restrict__ val,
                                                              const float2* __restrict__ Pdf,
                                                              const double* __restrict__ P,
                                                              double* __restrict__ Q, int64_t n_slices,
                                                              int64_t n, double* __restrict__ part) {
    constexpr int LPG = KW / 4, G = 32 / LPG, R = RW / G, WPS = 32 / RW;
    __shared__ double sh[4][KW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int g = lane / LPG, q = lane % LPG;
    double d[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t units = n_slices * WPS;
    for (int64_t gw = (int64_t)blockIdx.x * 4 + wib; gw < units; gw += (int64_t)gridDim.x * 4) {
        double out[R][4];
        multi_unit_df<V, KW, RW>(meta, col, vdf, val, Pdf, P, Q, gw, n, lane, out);
        const int64_t row0 = (int64_t)meta[gw / WPS].z + (int)(gw % WPS) * RW + g * R;
        double t[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (row0 + i < n) {
                double pv[4] = {0.0, 0.0, 0.0, 0.0};
                ld_x4(P + (row0 + i) * KW + 4 * q, true, pv);
#pragma unroll
                for (int j = 0; j < 4; ++j) t[j] = fma(pv[j], out[i][j], t[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) d[j] += t[j];
    }
#pragma unroll
    for (int o = LPG; o < 32; o <<= 1)
#pragma unroll
        for (int j = 0; j < 4; ++j) d[j] += __shfl_xor_sync(0xffffffffu, d[j], o);
    if (g == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j) sh[wib][4 * q + j] = d[j];
    __syncthreads();
    if (threadIdx.x < KW)
        part[(int64_t)blockIdx.x * KW + threadIdx.x] =
            ((sh[0][threadIdx.x] + sh[1][threadIdx.x]) + sh[2][threadIdx.x]) + sh[3][threadIdx.x];
}

// X in pairs (df_split: marked pairs for values outside the fast range).
__global__ void split_rows(const double* __restrict__ X, float2* __restrict__ Xdf, int64_t len) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < len) Xdf[t] = df_split(X[t]);
}

// Dst[i, j] = Src[idx[i], j] (idx == nullptr: identity) for j < k, 0 for k <= j < ldd.
template <typename XT>
__global__ void gather_rows(const XT* __restrict__ src, int lds, const int32_t* __restrict__ idx,
                            XT* __restrict__ dst, int ldd, int64_t n, int k) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n * ldd) {
        const int64_t i = t / ldd;
        const int j = (int)(t % ldd);
        const int64_t r = idx ? (int64_t)idx[i] : i;
        dst[t] = j < k ? src[r * lds + j] : XT(0);
    }
}

// Rows per warp: four rows per lane group (row-to-row reuse chains of four: longer
// chains serialise the gathers of a warp, shorter ones reuse less), at most 32,
// and small enough that the per-lane registers (accumulators, V stream entries
// per row, V rows of X) stay near 100 so that four 128-thread blocks fit on an SM
// without spilling.
template <typename VT, typename XT, int V, int KW>
constexpr int multi_rows_per_warp() {
    const int sx = (int)sizeof(XT) / 4, sv = (int)sizeof(VT) / 4, groups = 128 / KW;
    int rw = 4 * groups > 32 ? 32 : 4 * groups;
    while (rw / 2 >= groups) {
        const int r = rw / groups;
        if (r * 4 * sx + r * V * (1 + sv) + V * 4 * sx <= 104) break;
        rw /= 2;
    }
    return rw;
}

template <typename VT, typename XT, int V, int KW>
static void launch_multi_kw(const fespmv_mat* A, const VT* val, const XT* X, XT* Y, cudaStream_t s) {
    constexpr int RW = multi_rows_per_warp<VT, XT, V, KW>();
    const unsigned g = grid_for(A->n_slices * (32 / RW) * 32, 128);
    sliced_multi<VT, XT, V, KW, RW><<<g, 128, 0, s>>>(A->d_meta, A->d_col, val, X, Y, A->n_slices, A->n);
}

template <typename VT, typename XT, int V>
static void launch_multi_v(const fespmv_mat* A, const VT* val, const XT* X, XT* Y, int kw, cudaStream_t s) {
    switch (kw) {
        case 4: launch_multi_kw<VT, XT, V, 4>(A, val, X, Y, s); break;
        case 8: launch_multi_kw<VT, XT, V, 8>(A, val, X, Y, s); break;
        case 16: launch_multi_kw<VT, XT, V, 16>(A, val, X, Y, s); break;
        default: launch_multi_kw<VT, XT, V, 32>(A, val, X, Y, s); break;
    }
}

template <typename VT, typename XT>
static void launch_multi(const fespmv_mat* A, const VT* val, const XT* X, XT* Y, int kw, cudaStream_t s) {
    switch (A->vec) {
        case 1: launch_multi_v<VT, XT, 1>(A, val, X, Y, kw, s); break;
        case 4: launch_multi_v<VT, XT, 4>(A, val, X, Y, kw, s); break;
        default: launch_multi_v<VT, XT, 2>(A, val, X, Y, kw, s); break;
    }
}

// The product-and-dot kernel: its grid is the blocks resident at once (at most
// one block per four units); with part == nullptr nothing is launched.
template <typename VT, typename XT, int V, int KW>
static unsigned multi_dot_kw(const fespmv_mat* A, const VT* val, const XT* P, XT* Q, double* part,
                             cudaStream_t s) {
    constexpr int RW = multi_rows_per_warp<VT, XT, V, KW>();
    auto kernel = sliced_multi_dot<VT, XT, V, KW, RW>;
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0);
    const int64_t units = A->n_slices * (32 / RW);
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)sms * std::max(per_sm, 1), (units + 3) / 4));
    if (part) kernel<<<grid, 128, 0, s>>>(A->d_meta, A->d_col, val, P, Q, A->n_slices, A->n, part);
    return grid;
}

template <typename VT, typename XT, int V>
static unsigned multi_dot_v(const fespmv_mat* A, const VT* val, const XT* P, XT* Q, int kw, double* part,
                            cudaStream_t s) {
    switch (kw) {
        case 4: return multi_dot_kw<VT, XT, V, 4>(A, val, P, Q, part, s);
        case 8: return multi_dot_kw<VT, XT, V, 8>(A, val, P, Q, part, s);
        case 16: return multi_dot_kw<VT, XT, V, 16>(A, val, P, Q, part, s);
        default: return multi_dot_kw<VT, XT, V, 32>(A, val, P, Q, part, s);
    }
}

template <typename VT, typename XT>
static unsigned multi_dot(const fespmv_mat* A, const VT* val, const XT* P, XT* Q, int kw, double* part,
                          cudaStream_t s) {
    switch (A->vec) {
        case 1: return multi_dot_v<VT, XT, 1>(A, val, P, Q, kw, part, s);
        case 4: return multi_dot_v<VT, XT, 4>(A, val, P, Q, kw, part, s);
        default: return multi_dot_v<VT, XT, 2>(A, val, P, Q, kw, part, s);
    }
}

template <int V, int KW>
static void launch_multi_df_kw(const fespmv_mat* A, const float2* Xdf, const double* X, double* Y,
                               cudaStream_t s) {
    constexpr int RW = multi_rows_per_warp<double, double, V, KW>();
    const unsigned g = grid_for(A->n_slices * (32 / RW) * 32, 128);
    sliced_multi_df<V, KW, RW><<<g, 128, 0, s>>>(A->d_meta, A->d_col, A->d_vdf, A->d_val, Xdf, X, Y,
                                                 A->n_slices, A->n);
}

template <int V, int KW>
static unsigned multi_df_dot_kw(const fespmv_mat* A, const double* P, double* Q, const float2* Pdf, double* part,
                                cudaStream_t s) {
    constexpr int RW = multi_rows_per_warp<double, double, V, KW>();
    auto kernel = sliced_multi_df_dot<V, KW, RW>;
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0);
    const int64_t units = A->n_slices * (32 / RW);
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)sms * std::max(per_sm, 1), (units + 3) / 4));
    if (part)
        kernel<<<grid, 128, 0, s>>>(A->d_meta, A->d_col, A->d_vdf, A->d_val, Pdf, P, Q, A->n_slices, A->n, part);
    return grid;
}

template <int V>
static unsigned multi_df_dot_v(const fespmv_mat* A, const double* P, double* Q, const float2* Pdf, int kw,
                               double* part, cudaStream_t s) {
    switch (kw) {
        case 4: return multi_df_dot_kw<V, 4>(A, P, Q, Pdf, part, s);
        case 8: return multi_df_dot_kw<V, 8>(A, P, Q, Pdf, part, s);
        case 16: return multi_df_dot_kw<V, 16>(A, P, Q, Pdf, part, s);
        default: return multi_df_dot_kw<V, 32>(A, P, Q, Pdf, part, s);
    }
}

template <int V>
static void launch_multi_df_v(const fespmv_mat* A, const float2* Xdf, const double* X, double* Y, int kw,
                              cudaStream_t s) {
    switch (kw) {
        case 4: launch_multi_df_kw<V, 4>(A, Xdf, X, Y, s); break;
        case 8: launch_multi_df_kw<V, 8>(A, Xdf, X, Y, s); break;
        case 16: launch_multi_df_kw<V, 16>(A, Xdf, X, Y, s); break;
        default: launch_multi_df_kw<V, 32>(A, Xdf, X, Y, s); break;
    }
}

static int launch_multi_df(fespmv_mat* A, const double* X, double* Y, int kw, cudaStream_t s) {
    if (!A->d_xkdf) {
        int rc = device_alloc(A, (void**)&A->d_xkdf, sizeof(float2) * 32 * (size_t)A->n, "multi-RHS pair scratch");
        if (rc) return rc;
    }
    const int64_t len = A->n * kw;
    split_rows<<<grid_for(len, 256), 256, 0, s>>>(X, A->d_xkdf, len);
    switch (A->vec) {
        case 1: launch_multi_df_v<1>(A, A->d_xkdf, X, Y, kw, s); break;
        case 4: launch_multi_df_v<4>(A, A->d_xkdf, X, Y, kw, s); break;
        default: launch_multi_df_v<2>(A, A->d_xkdf, X, Y, kw, s); break;
    }
    return FESPMV_OK;
}

static int ensure_multi_scratch(fespmv_mat* A) {
    if (A->d_xk) return FESPMV_OK;
    const size_t bytes = sizeof(double) * 32 * (size_t)A->n;
    int rc = device_alloc(A, (void**)&A->d_xk, bytes, "multi-RHS x scratch");
    if (!rc) rc = device_alloc(A, (void**)&A->d_yk, bytes, "multi-RHS y scratch");
    return rc;
}

static int padded_width(int k) {
    int kw = 4;
    while (kw < k) kw *= 2;
    return kw;
}

template <typename XT>
static int apply_multi_t(fespmv_mat* A, const XT* X, XT* Y, int k, int flags, cudaStream_t s) {
    const bool permute = !(flags & FESPMV_IO_PERMUTED);
    const int kw = padded_width(k);
    const size_t align = 4 * sizeof(XT);
    // the caller's buffers serve directly when they already have the kernel's layout
    const bool direct = !permute && kw == k && (uintptr_t)X % align == 0 && (uintptr_t)Y % align == 0;
    const XT* xs = X;
    XT* ys = Y;
    if (!direct) {
        int rc = ensure_multi_scratch(A);
        if (rc) return rc;
        xs = reinterpret_cast<const XT*>(A->d_xk);
        ys = reinterpret_cast<XT*>(A->d_yk);
        gather_rows<XT><<<grid_for(A->n * kw, 256), 256, 0, s>>>(X, k, permute ? A->d_perm : nullptr,
                                                                 const_cast<XT*>(xs), kw, A->n, k);
    }
    if constexpr (std::is_same<XT, double>::value) {
        if (A->d_vdf) {                                              // FP64 by float pairs
            int rc = launch_multi_df(A, xs, ys, kw, s);
            if (rc) return rc;
        } else {
            launch_multi<double, double>(A, A->d_val, xs, ys, kw, s);  // FP64 values and sums
        }
    } else if (A->nb && A->d_nb32) {
        int rc = launch_nb3_multi(A, xs, ys, kw, s);                 // FP32 node blocks
        if (rc) return rc;
    } else {
        launch_multi<float, float>(A, A->d_val32, xs, ys, kw, s);   // FP32 copy of S A S
    }
    if (!direct)
        gather_rows<XT><<<grid_for(A->n * k, 256), 256, 0, s>>>(ys, kw, permute ? A->d_pinv : nullptr, Y, k,
                                                                A->n, k);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

unsigned launch_multi_dot(const fespmv_mat* A, const void* P, void* Q, int kw, bool f64, double* part,
                          cudaStream_t s) {
    if (f64)
        return multi_dot<double, double>(A, A->d_val, (const double*)P, (double*)Q, kw, part, s);
    if (A->nb && A->d_nb32) return launch_nb3_multi_dot(A, (const float*)P, (float*)Q, kw, part, s);
    return multi_dot<float, float>(A, A->d_val32, (const float*)P, (float*)Q, kw, part, s);
}

unsigned launch_multi_dot_pairs(const fespmv_mat* A, const double* P, double* Q, float2* Pdf, int kw, double* part,
                                cudaStream_t s) {
    if (part) {
        const int64_t len = A->n * kw;
        split_rows<<<grid_for(len, 256), 256, 0, s>>>(P, Pdf, len);
    }
    switch (A->vec) {
        case 1: return multi_df_dot_v<1>(A, P, Q, Pdf, kw, part, s);
        case 4: return multi_df_dot_v<4>(A, P, Q, Pdf, kw, part, s);
        default: return multi_df_dot_v<2>(A, P, Q, Pdf, kw, part, s);
    }
}

int launch_multi_f64(fespmv_mat* A, const double* X, double* Y, int kw, cudaStream_t s) {
    if (A->d_vdf) return launch_multi_df(A, X, Y, kw, s);
    launch_multi<double, double>(A, A->d_val, X, Y, kw, s);
    return FESPMV_OK;
}

void launch_gather_rows_f64(const double* src, int lds, const int32_t* idx, double* dst, int ldd, int64_t n,
                            int k, cudaStream_t s) {
    gather_rows<double><<<grid_for(n * ldd, 256), 256, 0, s>>>(src, lds, idx, dst, ldd, n, k);
}

int multi_width(int k) { return padded_width(k); }

}  // namespace fespmv

using namespace fespmv;

extern "C" int spmv_apply_multi(fespmv_mat_t A, const void* X, void* Y, int32_t k,
                                int32_t precision, int32_t flags, fespmv_stream_t stream) {
    try {
        if (!A || (A->n > 0 && (!X || !Y)) || k < 1 || k > 32 || (flags & ~FESPMV_IO_PERMUTED) ||
            (precision != FESPMV_PREC_F64 && precision != FESPMV_PREC_F32)) {
            set_error("spmv_apply_multi: bad argument");
            return FESPMV_ERR_INVALID_ARG;
        }
        if (A->format != FESPMV_FMT_SLICED || A->max_lanes_log2 != 0 || A->col_order == FESPMV_COLS_ORIGINAL) {
            set_error("spmv_apply_multi needs a SLICED handle with one lane per row (threshold 0)");
            return FESPMV_ERR_UNSUPPORTED;
        }
        if (precision == FESPMV_PREC_F32 && !A->d_val32) {
            set_error("spmv_apply_multi: the handle holds no FP32 copy");
            return FESPMV_ERR_UNSUPPORTED;
        }
        if (A->n == 0) return FESPMV_OK;
        cudaStream_t s = (cudaStream_t)stream;
        if (precision == FESPMV_PREC_F64)
            return apply_multi_t<double>(A, (const double*)X, (double*)Y, k, flags, s);
        return apply_multi_t<float>(A, (const float*)X, (float*)Y, k, flags, s);
    } catch (...) {
        set_error("unexpected C++ exception");
        return FESPMV_ERR_INVALID_ARG;
    }
}
