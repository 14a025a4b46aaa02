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

// The cluster's share of a problem: slices [s0, s1) by warps, rows [r0, r1) by threads.
struct ClusterPart {
    int64_t gw, nwarps, tid, nthreads;
    __device__ ClusterPart(const cgx::cluster_group& cl) {
        const unsigned rank = cl.block_rank(), C = cl.num_blocks();
        gw = (int64_t)rank * (kClusterThreads / 32) + (threadIdx.x >> 5);
        nwarps = (int64_t)C * (kClusterThreads / 32);
        tid = (int64_t)rank * kClusterThreads + threadIdx.x;
        nthreads = (int64_t)C * kClusterThreads;
    }
};

// q = A x (FP64) over slices [s0, s1); ends with the cluster synchronised.
template <int V, int U>
__device__ __forceinline__ void cluster_product_f64(cgx::cluster_group& cl, const ClusterPart& cp,
                                                    const uint4* __restrict__ meta, const int32_t* __restrict__ col,
                                                    const double* __restrict__ val, const double* __restrict__ x,
                                                    double* __restrict__ q, int64_t s0, int64_t s1) {
    const int lane = threadIdx.x & 31;
    for (int64_t sl = s0 + cp.gw; sl < s1; sl += cp.nwarps) {
        const uint4 m = meta[sl];
        const double sum = sliced_row_sum_f64<V, U>(m, col, val, x, lane);
        const int lt = (int)m.w;
        if ((lane & ((1 << lt) - 1)) == 0) q[(int64_t)m.z + (lane >> lt)] = sum;
    }
    cl.sync();
}

// Reliable-update refinement of one problem (the algorithm of cg_solve with
// FESPMV_CG_RELIABLE): inner CG on B = S A S with float vectors and FP64 dots;
// when the inner residual has fallen below thresh_in, x += S w and the residual is
// replaced by b - A x in FP64, the direction kept.  Rows past n (padding) must be
// rows the matrix stores as identity rows with b = 0, or lie outside [r0, r1).
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
    ClusterOut out{CG_RUNNING, 0, 0, 0.0, 0.0, 0.0};
    double rho = 0.0, thresh2 = 0.0, thresh_in = 0.0, prev = INFINITY;
    bool first = true;
    for (;;) {
        // ---- FP64 residual: r = b - A x, r_in = float(S r), w = 0 (x += S w first after a step)
        if (!first) {
            for (int64_t i = r0 + cp.tid; i < r1; i += cp.nthreads) x[i] = fma(scale[i], (double)w[i], x[i]);
            cl.sync();
        }
        const bool ax = !first || has_x0;
        if (ax) cluster_product_f64<V, U>(cl, cp, meta, col, val64, x, q64, s0, s1);
        double v3[3] = {0.0, 0.0, 0.0};
        for (int64_t i = r0 + cp.tid; i < r1; i += cp.nthreads) {
            const double bi = b[i];
            const double ri = ax ? bi - q64[i] : bi;
            const float rs = (float)(scale[i] * ri);
            w[i] = 0.0f;
            rin[i] = rs;
            if (first) p[i] = rs;
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
        // the kept direction takes the replaced residual: p = r_in + beta p (p = r_in first)
        const double beta0 = first ? 0.0 : rhs2 / rho;
        rho = rhs2;
        thresh_in = fmax(in2 * rhs2, out.rr > 0.0 ? tol2 * out.bb * rhs2 / out.rr : 0.0);
        if (!first) {
            const float bt = (float)beta0;
            for (int64_t i = r0 + cp.tid; i < r1; i += cp.nthreads) p[i] = fmaf(bt, p[i], rin[i]);
        }
        first = false;
        cl.sync();
        // ---- inner CG steps on B until the reliable-update test
        for (;;) {
            double v1[1] = {0.0};
            for (int64_t sl = s0 + cp.gw; sl < s1; sl += cp.nwarps) {
                const uint4 m = meta[sl];
                const float sum = sliced_row_sum_low<VT, V, U>(m, col, val32, p, lane);
                const int lt = (int)m.w;
                if ((lane & ((1 << lt) - 1)) == 0) {
                    const int64_t row = (int64_t)m.z + (lane >> lt);
                    q32[row] = sum;
                    v1[0] = fma((double)p[row], (double)sum, v1[0]);
                }
            }
            cluster_sum<1>(cl, red, turn, v1);
            const double pq = v1[0];
            if (!(pq > 0.0) || !isfinite(pq)) { out.status = CG_BREAKDOWN; break; }
            const float a = (float)(rho / pq);
            double v2[1] = {0.0};
            for (int64_t i = r0 + cp.tid; i < r1; i += cp.nthreads) {
                w[i] = fmaf(a, p[i], w[i]);
                const float ri = fmaf(-a, q32[i], rin[i]);
                rin[i] = ri;
                v2[0] = fma((double)ri, (double)ri, v2[0]);
            }
            cluster_sum<1>(cl, red, turn, v2);
            const double rn = v2[0];
            ++out.iters;
            if (!isfinite(rn)) { out.status = CG_BREAKDOWN; break; }
            if (rn <= thresh_in || out.iters >= max_iter) break;   // -> reliable update
            const float bt = (float)(rn / rho);
            rho = rn;
            for (int64_t i = r0 + cp.tid; i < r1; i += cp.nthreads) p[i] = fmaf(bt, p[i], rin[i]);
            cl.sync();
        }
        if (out.status != CG_RUNNING) break;
        ++out.outer;
    }
    out.true_rr = out.rr;
    return out;
}

}  // namespace fespmv
