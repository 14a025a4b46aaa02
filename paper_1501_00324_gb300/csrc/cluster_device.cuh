// Device core of the cluster solvers: a whole reliable-update solve of one problem
// run by one thread-block cluster (batch.cu: one problem per cluster from a work
// counter; cluster_cg.cu: a small handle's cg_solve in one launch).
//
// The CTAs of the cluster split the problem's slices (warps) and rows (threads);
// they synchronise only among themselves (hardware cluster barriers through
// cooperative_groups) and reduce dot products through distributed shared memory:
// every CTA adds the CTAs' partial sums in rank order, so all CTAs hold the same
// bits and take the same decisions, and every CTA passes the same sequence of
// barriers.
#pragma once

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_run.h"
#include "dot2.cuh"
#include "spmv_device.cuh"

namespace fespmv {

namespace cgx = cooperative_groups;
constexpr int kClusterCtas = 8;      // CTAs per cluster (the portable maximum) and
constexpr int kClusterThreads = 256; // threads per CTA: two CTAs per SM, 38 clusters at once

struct ClusterRed {
    double slot[2][4];   // per-CTA partial sums, two slots used in turn
    int job;
};

// What a cluster solve reports.
struct ClusterOut {
    int status, iters, outer;   // outer: reliable updates
    double rr, bb, true_rr;
};

__device__ __forceinline__ double cl_warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of K values over the cluster (fixed order: a block tree per CTA, then the
// CTAs in rank order); every thread of every CTA returns the same sums.
template <int K>
__device__ __forceinline__ void cluster_sum(cgx::cluster_group& cl, ClusterRed& red, int& turn, double (&v)[K]) {
    __shared__ double sh[K][kClusterThreads / 32];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = cl_warp_sum(v[k]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sh[k][warp] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = 0.0;
            for (int w = 0; w < kClusterThreads / 32; ++w) t += sh[k][w];
            red.slot[turn][k] = t;
        }
    cl.sync();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0.0;
    for (unsigned r = 0; r < cl.num_blocks(); ++r) {
        const double* rp = cl.map_shared_rank(&red.slot[turn][0], r);
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += rp[k];
    }
    turn ^= 1;
}

// The cluster's threads over a problem's rows [r0, r1) (the vector updates).
struct ClusterPart {
    int64_t tid, nthreads;
    __device__ ClusterPart(const cgx::cluster_group& cl) {
        tid = (int64_t)cl.block_rank() * kClusterThreads + threadIdx.x;
        nthreads = (int64_t)cl.num_blocks() * kClusterThreads;
    }
};

// Loads of vectors that the cluster wrote earlier in the same launch (p, x): plain
// global loads, which the cluster barriers order (acquire), never the read-only
// non-coherent path of __ldg, whose lines may be stale within one launch.
__device__ __forceinline__ float ld_vec(const float* a) {
    float v;
    asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(a));
    return v;
}
__device__ __forceinline__ double ld_vec(const double* a) {
    double v;
    asm volatile("ld.global.f64 %0, [%1];" : "=d"(v) : "l"(a));
    return v;
}

// A CTA's 8 warps walk many slices each, one after another, so the latency of a
// slice is what counts: all of a slice's entries are loaded in rounds of UM
// chunks of V per lane (one round for slices up to UM*V wide), then all its
// gathers issued, then the sums.  The summation order is that of
// sliced_row_sum_low / sliced_row_sum_f64 (entry by entry), so the sums are the
// graph path's bit for bit.
template <typename VT, int V, int UM>
__device__ __forceinline__ float cl_slice_sum_low(const uint4 m, const int32_t* __restrict__ col,
                                                  const VT* __restrict__ val, const float* x, int lane) {
    const int64_t off = (int64_t)m.x * 32;
    const int w = (int)m.y;
    const VT* vp = val + off + lane * V;
    const int32_t* cp = col + off + lane * V;
    float sum = 0.0f;
    for (int s = 0; s < w; s += UM * V) {
        LowChunk<VT, V> e[UM];
#pragma unroll
        for (int u = 0; u < UM; ++u)
            if (s + u * V < w) e[u].load(vp + u * 32 * V, cp + u * 32 * V);
        float xv[UM][V];
#pragma unroll
        for (int u = 0; u < UM; ++u)
#pragma unroll
            for (int k = 0; k < V; ++k) xv[u][k] = (s + u * V < w && e[u].c[k] >= 0) ? ld_vec(x + e[u].c[k]) : 0.0f;
#pragma unroll
        for (int u = 0; u < UM; ++u)
            if (s + u * V < w)
#pragma unroll
                for (int k = 0; k < V; ++k) sum = fmaf(e[u].v[k], xv[u][k], sum);
        vp += UM * 32 * V;
        cp += UM * 32 * V;
    }
    const int T = 1 << (int)m.w;
    for (int o = T >> 1; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    return sum;
}

template <int V, int UM>
__device__ __forceinline__ double cl_slice_sum_f64(const uint4 m, const int32_t* __restrict__ col,
                                                   const double* __restrict__ val, const double* x, int lane) {
    const int64_t off = (int64_t)m.x * 32;
    const int w = (int)m.y;
    const double* vp = val + off + lane * V;
    const int32_t* cp = col + off + lane * V;
    double sum = 0.0;
    for (int s = 0; s < w; s += UM * V) {
        Chunk<V> e[UM];
#pragma unroll
        for (int u = 0; u < UM; ++u)
            if (s + u * V < w) e[u].load(vp + u * 32 * V, cp + u * 32 * V);
        double xv[UM][V];
#pragma unroll
        for (int u = 0; u < UM; ++u)
#pragma unroll
            for (int k = 0; k < V; ++k) xv[u][k] = (s + u * V < w && e[u].c[k] >= 0) ? ld_vec(x + e[u].c[k]) : 0.0;
#pragma unroll
        for (int u = 0; u < UM; ++u)
            if (s + u * V < w)
#pragma unroll
                for (int k = 0; k < V; ++k) sum = fma(e[u].v[k], xv[u][k], sum);
        vp += UM * 32 * V;
        cp += UM * 32 * V;
    }
    const int T = 1 << (int)m.w;
    for (int o = T >> 1; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    return sum;
}

// Entries per lane loaded in one round of the slice sums above.
template <int V> constexpr int cl_round_chunks() { return V == 4 ? 4 : (V == 2 ? 8 : 16); }

// q = A x (FP64) over this CTA's slices [s0, s1) (its warps every eighth slice), the
// next slice's metadata loaded while the current one is summed; ends with the
// cluster synchronised.
template <int V, int U>
__device__ __forceinline__ void cluster_product_f64(cgx::cluster_group& cl, const uint4* __restrict__ meta,
                                                    const int32_t* __restrict__ col, const double* __restrict__ val,
                                                    const double* x, double* q, int64_t s0, int64_t s1) {
    const int lane = threadIdx.x & 31;
    int64_t sl = s0 + (threadIdx.x >> 5);
    uint4 m = sl < s1 ? meta[sl] : make_uint4(0, 0, 0, 0);
    while (sl < s1) {
        const int64_t nx = sl + kClusterThreads / 32;
        const uint4 mn = nx < s1 ? meta[nx] : make_uint4(0, 0, 0, 0);
        const double sum = cl_slice_sum_f64<V, cl_round_chunks<V>() / 2>(m, col, val, x, lane);
        const int lt = (int)m.w;
        if ((lane & ((1 << lt) - 1)) == 0) q[(int64_t)m.z + (lane >> lt)] = sum;
        sl = nx;
        m = mn;
    }
    cl.sync();
}

// One group of four rows of the inner CG update: w += a p, r_in -= a q, and the
// rows' r_in^2 added to acc in row order.
__device__ __forceinline__ void update4(float a, const float4& p, const float4& q, float4& r, float4& w,
                                        Dot2& acc) {
    w.x = fmaf(a, p.x, w.x);
    w.y = fmaf(a, p.y, w.y);
    w.z = fmaf(a, p.z, w.z);
    w.w = fmaf(a, p.w, w.w);
    r.x = fmaf(-a, q.x, r.x);
    r.y = fmaf(-a, q.y, r.y);
    r.z = fmaf(-a, q.z, r.z);
    r.w = fmaf(-a, q.w, r.w);
    acc.add(r.x, r.x);
    acc.add(r.y, r.y);
    acc.add(r.z, r.z);
    acc.add(r.w, r.w);
}

// Reliable-update refinement of one problem (the algorithm of cg_solve with
// FESPMV_CG_RELIABLE): inner CG on B = S A S with float vectors; when the inner
// residual has fallen below thresh_in, x += S w and the residual is replaced by
// b - A x in FP64, the direction kept.  The inner system is carried scaled by a
// power of two, 2^k, chosen at every replacement so that |r_in| is near 1: the
// scaling is exact, so every rounding of the iteration is that of the unscaled one,
// and the inner dot products, float pairs (Dot2) summed in FP64 over the cluster,
// cannot overflow.  Rows past n (padding) must be
// rows the matrix stores as identity rows with b = 0, or lie outside [r0, r1).
// r0 must be a multiple of 4 and the float vectors 16-byte aligned.
template <typename VT, int V, int U>
__device__ ClusterOut cluster_reliable(cgx::cluster_group& cl, ClusterRed& red, int& turn,
                                       const uint4* __restrict__ meta, const int32_t* __restrict__ col,
                                       const VT* __restrict__ val32, const double* __restrict__ val64,
                                       const double* __restrict__ scale, const double* __restrict__ b,
                                       double* __restrict__ x, double* __restrict__ q64, float* __restrict__ w,
                                       float* __restrict__ rin, float* __restrict__ p, float* __restrict__ q32,
                                       int64_t s0, int64_t s1, int64_t r0, int64_t r1, double tol2, double in2,
                                       int has_x0, int max_iter, int max_outer) {
    const ClusterPart cp(cl);
    const int lane = threadIdx.x & 31;
    // the products: CTA r takes the r-th contiguous run of the slices, its warps
    // every eighth slice of the run, so that an SM's gathers stay near one another
    // (locality order) and hit in its L1
    const unsigned rank = cl.block_rank(), nct = cl.num_blocks();
    const int64_t cs0 = s0 + (s1 - s0) * rank / nct, cs1 = s0 + (s1 - s0) * (rank + 1) / nct;
    const int warp = threadIdx.x >> 5;
    ClusterOut out{CG_RUNNING, 0, 0, 0.0, 0.0, 0.0};
    double rho = 0.0, thresh2 = 0.0, thresh_in = 0.0, prev = INFINITY;
    int ksc = 0;   // r_in, p and w hold the inner system scaled by 2^ksc
    bool first = true;
    for (;;) {
        // ---- FP64 residual: r = b - A x, r_in = float(S r), w = 0 (x += S w first after a step)
        if (!first) {   // w solves the scaled system: x += S w 2^-k (exact rescaling)
            for (int64_t i = r0 + cp.tid; i < r1; i += cp.nthreads)
                x[i] = fma(scale[i], ldexp((double)w[i], -ksc), x[i]);
            cl.sync();
        }
        const bool ax = !first || has_x0;
        if (ax) cluster_product_f64<V, U>(cl, meta, col, val64, x, q64, cs0, cs1);
        double v3[3] = {0.0, 0.0, 0.0};
        for (int64_t i = r0 + cp.tid; i < r1; i += cp.nthreads) {
            const double bi = b[i];
            const double ri = ax ? bi - q64[i] : bi;
            const float rs = (float)(scale[i] * ri);
            w[i] = 0.0f;
            rin[i] = rs;
            v3[0] = fma(ri, ri, v3[0]);
            v3[1] = fma((double)rs, (double)rs, v3[1]);
            v3[2] = fma(bi, bi, v3[2]);
        }
        cluster_sum<3>(cl, red, turn, v3);
        out.rr = v3[0];
        const double rhs2 = v3[1];
        if (first) {
            out.bb = v3[2];
            thresh2 = tol2 * out.bb;
        }
        if (!isfinite(out.rr) || !isfinite(rhs2)) { out.status = CG_BREAKDOWN; break; }
        if (out.rr <= thresh2) { out.status = CG_CONVERGED; break; }
        if (out.outer >= max_outer || out.iters >= max_iter || !(out.rr < prev)) { out.status = CG_MAXITER; break; }
        prev = out.rr;
        // the scale of the new inner system: 2^(2k) rhs2 in [1, 4)
        const int knew = rhs2 > 0.0 ? -(ilogb(rhs2) >> 1) : 0;
        const double rhs2s = ldexp(rhs2, 2 * knew);
        // the kept direction takes the replaced residual: p = r_in + beta p (p = r_in
        // first), p brought from the old scale to the new one through beta
        const double beta0 = first ? 0.0 : rhs2s / rho;
        const float bt = (float)ldexp(beta0, ksc - knew);
        rho = rhs2s;
        thresh_in = fmax(in2 * rhs2s, out.rr > 0.0 ? tol2 * out.bb * rhs2s / out.rr : 0.0);
        for (int64_t i = r0 + cp.tid; i < r1; i += cp.nthreads) {
            const float ri = ldexpf(rin[i], knew);
            rin[i] = ri;
            p[i] = first ? ri : fmaf(bt, p[i], ri);
        }
        ksc = knew;
        first = false;
        cl.sync();
        // ---- inner CG steps on B until the reliable-update test
        for (;;) {
            Dot2 d1;
            {
                int64_t sl = cs0 + warp;
                uint4 m = sl < cs1 ? meta[sl] : make_uint4(0, 0, 0, 0);
                while (sl < cs1) {
                    const int64_t nx = sl + kClusterThreads / 32;
                    const uint4 mn = nx < cs1 ? meta[nx] : make_uint4(0, 0, 0, 0);
                    const float sum = cl_slice_sum_low<VT, V, cl_round_chunks<V>()>(m, col, val32, p, lane);
                    if ((lane & ((1 << (int)m.w) - 1)) == 0) {
                        const int64_t row = (int64_t)m.z + (lane >> (int)m.w);
                        q32[row] = sum;
                        d1.add(p[row], sum);
                    }
                    sl = nx;
                    m = mn;
                }
            }
            double v1[1] = {d1.value()};
            cluster_sum<1>(cl, red, turn, v1);
            const double pq = v1[0];
            if (!(pq > 0.0) || !isfinite(pq)) { out.status = CG_BREAKDOWN; break; }
            const float a = (float)(rho / pq);
            Dot2 d2;
            // w += a p, r_in -= a q: rows four at a time (r0 is a multiple of 4), two
            // groups of four in flight per thread, then the rows past the last group
            {
                float4* W4 = reinterpret_cast<float4*>(w);
                float4* R4 = reinterpret_cast<float4*>(rin);
                const float4* P4 = reinterpret_cast<const float4*>(p);
                const float4* Q4 = reinterpret_cast<const float4*>(q32);
                const int64_t g1 = r1 >> 2;
                for (int64_t g = (r0 >> 2) + cp.tid; g < g1; g += 2 * cp.nthreads) {
                    const int64_t h = g + cp.nthreads;
                    const bool two = h < g1;
                    float4 pa = P4[g], qa = Q4[g], ra = R4[g], wa = W4[g];
                    float4 pb = pa, qb = qa, rb = ra, wb = wa;
                    if (two) { pb = P4[h]; qb = Q4[h]; rb = R4[h]; wb = W4[h]; }
                    update4(a, pa, qa, ra, wa, d2);
                    W4[g] = wa;
                    R4[g] = ra;
                    if (two) {
                        update4(a, pb, qb, rb, wb, d2);
                        W4[h] = wb;
                        R4[h] = rb;
                    }
                }
                for (int64_t i = 4 * g1 + cp.tid; i < r1; i += cp.nthreads) {
                    w[i] = fmaf(a, p[i], w[i]);
                    const float ri = fmaf(-a, q32[i], rin[i]);
                    rin[i] = ri;
                    d2.add(ri, ri);
                }
            }
            double v2[1] = {d2.value()};
            cluster_sum<1>(cl, red, turn, v2);
            const double rn = v2[0];
            ++out.iters;
            if (!isfinite(rn)) { out.status = CG_BREAKDOWN; break; }
            if (rn <= thresh_in || out.iters >= max_iter) break;   // -> reliable update
            const float bt = (float)(rn / rho);
            rho = rn;
            {   // p = r_in + bt p, as above
                float4* P4 = reinterpret_cast<float4*>(p);
                const float4* R4 = reinterpret_cast<const float4*>(rin);
                const int64_t g1 = r1 >> 2;
                for (int64_t g = (r0 >> 2) + cp.tid; g < g1; g += 2 * cp.nthreads) {
                    const int64_t h = g + cp.nthreads;
                    const bool two = h < g1;
                    float4 pa = P4[g], ra = R4[g];
                    float4 pb = pa, rb = ra;
                    if (two) { pb = P4[h]; rb = R4[h]; }
                    P4[g] = make_float4(fmaf(bt, pa.x, ra.x), fmaf(bt, pa.y, ra.y), fmaf(bt, pa.z, ra.z),
                                        fmaf(bt, pa.w, ra.w));
                    if (two)
                        P4[h] = make_float4(fmaf(bt, pb.x, rb.x), fmaf(bt, pb.y, rb.y), fmaf(bt, pb.z, rb.z),
                                            fmaf(bt, pb.w, rb.w));
                }
                for (int64_t i = 4 * g1 + cp.tid; i < r1; i += cp.nthreads) p[i] = fmaf(bt, p[i], rin[i]);
            }
            cl.sync();
        }
        if (out.status != CG_RUNNING) break;
        ++out.outer;
    }
    out.true_rr = out.rr;
    return out;
}

}  // namespace fespmv
