// Jacobi-preconditioned conjugate gradients on the device (cg_solve).
//
// The paper solves K dx = R with Jacobi-preconditioned CG inside each Newton
// step (Sec. 2.1, Sec. 4); the recurrences are the textbook Hestenes-Stiefel
// ones.  GB300 layout of one iteration, three kernels, all scalars on the device:
//   1. cg_spmv_dot   q = A p (the SpMV kernel of the handle) fused with p.q;
//                    the last block to finish reduces the per-block partial sums
//                    in a fixed order and forms alpha = rho / p.q
//   2. cg_update     x += alpha p, r -= alpha q, z = D^-1 r on the fly, r.z and
//                    r.r; the last block forms beta, counts the iteration and
//                    sets the status word (converged / breakdown / limit)
//   3. cg_pupdate    p = D^-1 r + beta p (z is never stored)
// Every kernel returns at once when the status word is no longer RUNNING, so a
// CUDA graph of `check_every` iterations can be launched repeatedly and the
// host only polls the status between graphs.  All reductions have a fixed
// order, so a solve is bitwise reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "dot2.cuh"
#include "internal.h"
#include "spmv_device.cuh"
#include "tiled_device.cuh"
#include "nodeblock_device.cuh"
#include "cg_run.h"

namespace fespmv {

// ------------------------------------------------------------------ reductions

// Sum over the block of K values (fixed order); the result is valid in thread 0.
// The lane values go to shared memory and one warp adds them: lane l sums
// entries l, l + 32, ... sequentially, then a shuffle tree.  This takes about
// a third of the FP64 adds of a shuffle tree in every warp, which matters on a
// part whose FP64 pipe retires about two lanes per clock per SM.
template <int K, int MAXB = 256>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
    __shared__ double sh[K][MAXB];
    const int t = threadIdx.x, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k][t] = v[k];
    __syncthreads();
    if (t < 32) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = sh[k][t];
            for (int w = 1; w < nw; ++w) s += sh[k][w * 32 + t];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            v[k] = s;
        }
    }
    __syncthreads();
}

// Deterministic grid-wide sum: block sums go to partials[k*gridDim.x + block];
// the last block to arrive sums them in block order (every thread issues its
// loads before adding) and returns true (result in thread 0's v).  counters[0]
// is zero between kernels (the last block resets it).
constexpr int64_t grid_sum_doubles(int64_t g) { return 3 * g + 8; }

template <int K, int MAXB = 256>
__device__ __forceinline__ bool grid_sum(double (&v)[K], double* partials, unsigned int* counters) {
    __shared__ bool last;
    const unsigned G = gridDim.x;
    block_sum<K, MAXB>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) partials[k * G + blockIdx.x] = v[k];
        __threadfence();
        last = atomicAdd(&counters[0], 1u) == G - 1;
    }
    __syncthreads();
    if (!last) return false;
    constexpr int UR = K == 1 ? 8 : (K == 2 ? 4 : 2);
    double t[K];
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = 0.0;
    for (unsigned i0 = threadIdx.x; i0 < G; i0 += UR * blockDim.x) {
        double x[UR][K];
#pragma unroll
        for (int u = 0; u < UR; ++u) {
            const unsigned i = i0 + u * blockDim.x;
#pragma unroll
            for (int k = 0; k < K; ++k) x[u][k] = i < G ? __ldcg(partials + k * G + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < UR; ++u)
#pragma unroll
            for (int k = 0; k < K; ++k) t[k] += x[u][k];
    }
    block_sum<K, MAXB>(t);
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = t[k];
    if (threadIdx.x == 0) counters[0] = 0;
    return true;
}

__device__ __forceinline__ void finish_pq(double pq, CgScalars* sc) {
    sc->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) sc->status = CG_BREAKDOWN;
    else sc->alpha = sc->rho / pq;
}

// ------------------------------------------------------------------ kernels

template <int V, int U>
__global__ void __launch_bounds__(256, V == 4 ? 6 : 8) cg_spmv_dot_sliced(const uint4* __restrict__ meta,
                                                          const int32_t* __restrict__ col,
                                                          const double* __restrict__ val,
                                                          const double* __restrict__ p,
                                                          double* __restrict__ q, int64_t n_slices,
                                                          int64_t n, double* partials,
                                                          CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    double v[1] = {0.0};
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = warp; sl < n_slices; sl += nw) {   // persistent warps stride over slices
        const uint4 m = meta[sl];
        const double sum = sliced_row_sum_f64<V, U>(m, col, val, p, lane);
        const int lt = (int)m.w;
        const int64_t row = (int64_t)m.z + (lane >> lt);
        if ((lane & ((1 << lt) - 1)) == 0 && row < n) {
            q[row] = sum;
            v[0] = fma(p[row], sum, v[0]);
        }
    }
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) finish_pq(v[0], sc);
}

// The same products with x staged through shared memory per tile (handles with
// tiles): persistent blocks stride over the tiles, staging each tile's x then
// walking its slices, and reduce once at the end as above.
template <int V, int U>
__global__ void __launch_bounds__(kTiledBlock) cg_spmv_dot_tiled(const uint4* __restrict__ meta,
                                                                 const uint16_t* __restrict__ lidx,
                                                                 const double* __restrict__ val,
                                                                 const int4* __restrict__ tiles,
                                                                 const int32_t* __restrict__ dict,
                                                                 const double* __restrict__ p,
                                                                 double* __restrict__ q, int64_t n,
                                                                 int64_t n_tiles, double* partials,
                                                                 CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    extern __shared__ __align__(16) unsigned char tile_smem[];
    double* xs = reinterpret_cast<double*>(tile_smem);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v[1] = {0.0};
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {   // persistent blocks stride over tiles
        const int4 tl = stage_tile<double>(tiles + t, dict, p, xs);
        if (wid < tl.y) {
            const uint4 m = meta[tl.x + wid];
            const double sum = tiled_row_sum<double, V, U>(m, lidx, val, xs, lane);
            const int lt = (int)m.w;
            const int64_t row = (int64_t)m.z + (lane >> lt);
            if ((lane & ((1 << lt) - 1)) == 0 && row < n) {
                q[row] = sum;
                v[0] = fma(p[row], sum, v[0]);
            }
        }
        __syncthreads();  // the next tile overwrites xs
    }
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) finish_pq(v[0], sc);
}

template <int V, int U>
__global__ void __launch_bounds__(256) cg_spmv_dot_df(const uint4* __restrict__ meta,
                                                      const int32_t* __restrict__ col,
                                                      const float2* __restrict__ vdf,
                                                      const double* __restrict__ val,
                                                      const double* __restrict__ p,
                                                      const float2* __restrict__ pdf,
                                                      double* __restrict__ q, int64_t n_slices,
                                                      int64_t n, double* partials, CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    double v[1] = {0.0};
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = warp; sl < n_slices; sl += nw) {   // persistent warps stride over slices
        const uint4 m = meta[sl];
        const double sum = sliced_row_sum_df<V, U>(m, col, vdf, val, pdf, p, lane);
        const int lt = (int)m.w;
        const int64_t row = (int64_t)m.z + (lane >> lt);
        if ((lane & ((1 << lt) - 1)) == 0 && row < n) {
            q[row] = sum;
            v[0] = fma(p[row], sum, v[0]);
        }
    }
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) finish_pq(v[0], sc);
}

template <int V, int U>
__global__ void __launch_bounds__(kTiledBlock) cg_spmv_dot_tiled_df(const uint4* __restrict__ meta,
                                                                    const uint16_t* __restrict__ lidx,
                                                                    const float2* __restrict__ vdf,
                                                                    const double* __restrict__ val,
                                                                    const int32_t* __restrict__ col,
                                                                    const int4* __restrict__ tiles,
                                                                    const int32_t* __restrict__ dict,
                                                                    const double* __restrict__ p,
                                                                    const float2* __restrict__ pdf,
                                                                    double* __restrict__ q, int64_t n,
                                                                    int64_t n_tiles, double* partials,
                                                                    CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    extern __shared__ __align__(16) unsigned char tile_smem[];
    float2* xs = reinterpret_cast<float2*>(tile_smem);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v[1] = {0.0};
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int4 tl = stage_tile<float2>(tiles + t, dict, pdf, xs);
        if (wid < tl.y) {
            const uint4 m = meta[tl.x + wid];
            const double sum = tiled_row_sum_df<V, U>(m, lidx, vdf, val, col, xs, p, lane);
            const int lt = (int)m.w;
            const int64_t row = (int64_t)m.z + (lane >> lt);
            if ((lane & ((1 << lt) - 1)) == 0 && row < n) {
                q[row] = sum;
                v[0] = fma(p[row], sum, v[0]);
            }
        }
        __syncthreads();
    }
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) finish_pq(v[0], sc);
}

template <int L>
__global__ void cg_spmv_dot_csr(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ p,
                                double* __restrict__ q, int64_t n, double* partials, CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = t / L;
    const int sub = (int)(t % L);
    double v[1] = {0.0};
    const double sum = csr_row_sum_f64<L>(row, sub, n, rowptr, col, val, p);
    if (row < n && sub == 0) {
        q[row] = sum;
        v[0] = p[row] * sum;
    }
    if (grid_sum<1, 1024>(v, partials, sc->counters) && threadIdx.x == 0) finish_pq(v[0], sc);
}

__global__ void __launch_bounds__(256, 4) cg_update(int64_t n, double* __restrict__ x,
                                                 double* __restrict__ r,
                                                 const double* __restrict__ p,
                                                 const double* __restrict__ q,
                                                 const double* __restrict__ dinv, double* partials,
                                                 CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const double a = sc->alpha;
    double v[2] = {0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fma(a, p[i], x[i]);
        const double ri = fma(-a, q[i], r[i]);
        r[i] = ri;
        v[0] = fma(ri, dinv[i] * ri, v[0]);
        v[1] = fma(ri, ri, v[1]);
    }
    if (grid_sum<2>(v, partials, sc->counters) && threadIdx.x == 0) {
        sc->iters += 1;
        sc->rr = v[1];
        if (!isfinite(v[0]) || !isfinite(v[1])) sc->status = CG_BREAKDOWN;
        else if (v[1] <= sc->thresh2) sc->status = CG_CONVERGED;
        else if (sc->iters >= sc->max_iter) sc->status = CG_MAXITER;
        else {
            sc->beta = v[0] / sc->rho;
            sc->rho = v[0];
        }
    }
}

__global__ void __launch_bounds__(256, 4) cg_pupdate(int64_t n, double* __restrict__ p,
                                                  const double* __restrict__ r,
                                                  const double* __restrict__ dinv,
                                                  float2* __restrict__ pdf, const CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const double beta = sc->beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double pi = fma(beta, p[i], dinv[i] * r[i]);
        p[i] = pi;
        if (pdf) pdf[i] = df_split(pi);
    }
}

// dinv = 1/diag (Jacobi) or 1; a non-positive or non-finite diagonal marks BADDIAG.
__global__ void cg_dinv(int64_t n, const double* __restrict__ diag, double* __restrict__ dinv,
                        int jacobi, CgScalars* sc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double d = diag[i];
        if (!jacobi) {
            dinv[i] = 1.0;
        } else if (d > 0.0 && isfinite(d)) {
            dinv[i] = 1.0 / d;
        } else {
            dinv[i] = 0.0;
            sc->status = CG_BADDIAG;
        }
    }
}

// r = b - Ax (Ax = q, or 0 when q is null), p = D^-1 r; rho = r.z, rr = r.r, bb = b.b.
__global__ void __launch_bounds__(256) cg_init(int64_t n, const double* __restrict__ b,
                                               const double* __restrict__ q, double* __restrict__ r,
                                               double* __restrict__ p,
                                               const double* __restrict__ dinv, double tol2,
                                               double* partials, CgScalars* sc,
                                               float2* __restrict__ pdf) {
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double bi = b[i];
        const double ri = q ? bi - q[i] : bi;
        const double zi = dinv[i] * ri;
        r[i] = ri;
        p[i] = zi;
        if (pdf) pdf[i] = df_split(zi);
        v[0] = fma(ri, zi, v[0]);
        v[1] = fma(ri, ri, v[1]);
        v[2] = fma(bi, bi, v[2]);
    }
    if (grid_sum<3>(v, partials, sc->counters) && threadIdx.x == 0) {
        sc->rho = v[0];
        sc->rr = v[1];
        sc->bb = v[2];
        sc->thresh2 = tol2 * v[2];
        sc->first = 1;
        if (sc->status == CG_BADDIAG) return;
        if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2])) sc->status = CG_BREAKDOWN;
        else if (v[1] <= sc->thresh2) sc->status = CG_CONVERGED;
        else if (sc->iters >= sc->max_iter) sc->status = CG_MAXITER;
        else sc->status = CG_RUNNING;
    }
}

// true_rr = ||b - q||^2 with q = A x.
__global__ void __launch_bounds__(256, 8) cg_true_residual(int64_t n, const double* __restrict__ b,
                                                        const double* __restrict__ q,
                                                        double* partials, CgScalars* sc) {
    double v[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double d = b[i] - q[i];
        v[0] = fma(d, d, v[0]);
    }
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) sc->true_rr = v[0];
}

// ------------------------------------------------------------------ single-reduction CG
// Chronopoulos-Gear arrangement (FESPMV_CG_SINGLE_REDUCTION): per iteration one
// product w = A u fused with gamma = r.u, delta = w.u and r.r (one grid
// reduction, scalars formed by the last block), then one streaming update
//   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = D^-1 r.

__device__ __forceinline__ void finish_cg1(double gam, double del, double rr, CgScalars* sc) {
    sc->rr = rr;
    if (!sc->first) sc->iters += 1;
    if (!isfinite(gam) || !isfinite(del) || !isfinite(rr)) {
        sc->status = CG_BREAKDOWN;
        return;
    }
    if (rr <= sc->thresh2) {
        sc->status = CG_CONVERGED;
        return;
    }
    if (sc->iters >= sc->max_iter) {
        sc->status = CG_MAXITER;
        return;
    }
    double beta = 0.0, denom = del;
    if (!sc->first) {
        beta = gam / sc->rho;
        denom = del - beta * gam / sc->alpha;
    }
    if (!(denom > 0.0)) {
        sc->status = CG_BREAKDOWN;
        return;
    }
    sc->alpha = gam / denom;
    sc->beta = beta;
    sc->rho = gam;
    sc->first = 0;
}

template <int V, int U>
__global__ void __launch_bounds__(256, 6) cg1_spmv_dots_sliced(const uint4* __restrict__ meta,
                                                               const int32_t* __restrict__ col,
                                                               const double* __restrict__ val,
                                                               const double* __restrict__ u,
                                                               const double* __restrict__ r,
                                                               double* __restrict__ w, int64_t n_slices,
                                                               int64_t n, double* partials, CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    double v[3] = {0.0, 0.0, 0.0};
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = warp; sl < n_slices; sl += nw) {
        const uint4 m = meta[sl];
        const double sum = sliced_row_sum_f64<V, U>(m, col, val, u, lane);
        const int lt = (int)m.w;
        const int64_t row = (int64_t)m.z + (lane >> lt);
        if ((lane & ((1 << lt) - 1)) == 0 && row < n) {
            w[row] = sum;
            const double ur = u[row], rr = r[row];
            v[0] = fma(rr, ur, v[0]);
            v[1] = fma(sum, ur, v[1]);
            v[2] = fma(rr, rr, v[2]);
        }
    }
    if (grid_sum<3>(v, partials, sc->counters) && threadIdx.x == 0) finish_cg1(v[0], v[1], v[2], sc);
}

template <int V, int U>
__global__ void __launch_bounds__(kTiledBlock) cg1_spmv_dots_tiled(const uint4* __restrict__ meta,
                                                                   const uint16_t* __restrict__ lidx,
                                                                   const double* __restrict__ val,
                                                                   const int4* __restrict__ tiles,
                                                                   const int32_t* __restrict__ dict,
                                                                   const double* __restrict__ u,
                                                                   const double* __restrict__ r,
                                                                   double* __restrict__ w, int64_t n,
                                                                   int64_t n_tiles, double* partials,
                                                                   CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    extern __shared__ __align__(16) unsigned char tile_smem[];
    double* xs = reinterpret_cast<double*>(tile_smem);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int4 tl = stage_tile<double>(tiles + t, dict, u, xs);
        if (wid < tl.y) {
            const uint4 m = meta[tl.x + wid];
            const double sum = tiled_row_sum<double, V, U>(m, lidx, val, xs, lane);
            const int lt = (int)m.w;
            const int64_t row = (int64_t)m.z + (lane >> lt);
            if ((lane & ((1 << lt) - 1)) == 0 && row < n) {
                w[row] = sum;
                const double ur = u[row], rr = r[row];
                v[0] = fma(rr, ur, v[0]);
                v[1] = fma(sum, ur, v[1]);
                v[2] = fma(rr, rr, v[2]);
            }
        }
        __syncthreads();
    }
    if (grid_sum<3>(v, partials, sc->counters) && threadIdx.x == 0) finish_cg1(v[0], v[1], v[2], sc);
}

template <int L>
__global__ void cg1_spmv_dots_csr(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const double* __restrict__ val, const double* __restrict__ u,
                                  const double* __restrict__ r, double* __restrict__ w, int64_t n,
                                  double* partials, CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = t / L;
    const int sub = (int)(t % L);
    double v[3] = {0.0, 0.0, 0.0};
    const double sum = csr_row_sum_f64<L>(row, sub, n, rowptr, col, val, u);
    if (row < n && sub == 0) {
        w[row] = sum;
        const double ur = u[row], rr = r[row];
        v[0] = rr * ur;
        v[1] = sum * ur;
        v[2] = rr * rr;
    }
    if (grid_sum<3, 1024>(v, partials, sc->counters) && threadIdx.x == 0) finish_cg1(v[0], v[1], v[2], sc);
}

__global__ void __launch_bounds__(256, 4) cg1_update(int64_t n, double* __restrict__ x,
                                                     double* __restrict__ r, double* __restrict__ u,
                                                     double* __restrict__ p, double* __restrict__ s,
                                                     const double* __restrict__ w,
                                                     const double* __restrict__ dinv, const CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const double a = sc->alpha, b = sc->beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double pi = fma(b, p[i], u[i]);
        const double si = fma(b, s[i], w[i]);
        p[i] = pi;
        s[i] = si;
        x[i] = fma(a, pi, x[i]);
        const double ri = fma(-a, si, r[i]);
        r[i] = ri;
        u[i] = dinv[i] * ri;
    }
}

// ------------------------------------------------------------------ refinement kernels
// Inner CG on B = S A S with float vectors and float products; dot products and
// all scalars in FP64 (the oracle's refinement, step by step).

__device__ __forceinline__ void finish_pq_inner(double pq, CgScalars* sc) {
    sc->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) sc->status = CG_BREAKDOWN;
    else sc->alpha = sc->rho / pq;
}

template <typename VT, int V, int U>
__global__ void __launch_bounds__(256, 8) cg32_spmv_dot_sliced(const uint4* __restrict__ meta,
                                                            const int32_t* __restrict__ col,
                                                            const VT* __restrict__ val,
                                                            const float* __restrict__ p,
                                                            float* __restrict__ q, int64_t n_slices,
                                                            int64_t n, double* partials,
                                                            CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    double v[1] = {0.0};
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = warp; sl < n_slices; sl += nw) {   // persistent warps stride over slices
        const uint4 m = meta[sl];
        const float sum = sliced_row_sum_low<VT, V, U>(m, col, val, p, lane);
        const int lt = (int)m.w;
        const int64_t row = (int64_t)m.z + (lane >> lt);
        if ((lane & ((1 << lt) - 1)) == 0 && row < n) {
            q[row] = sum;
            v[0] = fma((double)p[row], (double)sum, v[0]);
        }
    }
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) finish_pq_inner(v[0], sc);
}

template <typename VT, int V, int U>
__global__ void __launch_bounds__(kTiledBlock) cg32_spmv_dot_tiled(const uint4* __restrict__ meta,
                                                                   const uint16_t* __restrict__ lidx,
                                                                   const VT* __restrict__ val,
                                                                   const int4* __restrict__ tiles,
                                                                   const int32_t* __restrict__ dict,
                                                                   const float* __restrict__ p,
                                                                   float* __restrict__ q, int64_t n,
                                                                   int64_t n_tiles, double* partials,
                                                                   CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    extern __shared__ __align__(16) unsigned char tile_smem[];
    float* xs = reinterpret_cast<float*>(tile_smem);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v[1] = {0.0};
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int4 tl = stage_tile<float>(tiles + t, dict, p, xs);
        if (wid < tl.y) {
            const uint4 m = meta[tl.x + wid];
            const float sum = tiled_row_sum<VT, V, U>(m, lidx, val, xs, lane);
            const int lt = (int)m.w;
            const int64_t row = (int64_t)m.z + (lane >> lt);
            if ((lane & ((1 << lt) - 1)) == 0 && row < n) {
                q[row] = sum;
                v[0] = fma((double)p[row], (double)sum, v[0]);
            }
        }
        __syncthreads();
    }
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) finish_pq_inner(v[0], sc);
}

// The inner product on 3x3 node blocks (handles with node_blocks): persistent
// warps over the node-block slices, three rows per lane.
template <typename VT, int U>
__global__ void __launch_bounds__(256) cg32_spmv_dot_nb(const uint4* __restrict__ meta,
                                                        const int32_t* __restrict__ col,
                                                        const VT* __restrict__ val, const float* __restrict__ p,
                                                        float* __restrict__ q, int64_t n_slices, int64_t n_nodes,
                                                        double* partials, CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    double v[1] = {0.0};
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = warp; sl < n_slices; sl += nw) {
        const uint4 m = meta[sl];
        float s[3];
        nb3_row_sums<VT, U>(m, col, val, p, lane, s);
        const int64_t node = (int64_t)m.z + lane;
        if (node < n_nodes) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                q[3 * node + a] = s[a];
                v[0] = fma((double)p[3 * node + a], (double)s[a], v[0]);
            }
        }
    }
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) finish_pq_inner(v[0], sc);
}

// The same with x staged per tile: persistent blocks over the node-block tiles.
template <typename VT, int U>
__global__ void __launch_bounds__(256, 8) cg32_spmv_dot_nb_tiled(const uint4* __restrict__ meta,
                                                              const uint16_t* __restrict__ lidx,
                                                              const VT* __restrict__ val,
                                                              const int4* __restrict__ tiles,
                                                              const int32_t* __restrict__ dict,
                                                              const float* __restrict__ p, float* __restrict__ q,
                                                              int64_t n_tiles, int64_t n_nodes, double* partials,
                                                              CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    extern __shared__ __align__(16) unsigned char tile_smem[];
    float* xs = reinterpret_cast<float*>(tile_smem);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v[1] = {0.0};
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int4 tl = nb3_stage(tiles + t, dict, p, xs);
        if (wid < tl.y) {
            const uint4 m = meta[tl.x + wid];
            float s[3];
            nb3_row_sums_tiled<VT, U>(m, lidx, val, xs, lane, s);
            const int64_t node = (int64_t)m.z + lane;
            if (node < n_nodes) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    q[3 * node + a] = s[a];
                    v[0] = fma((double)p[3 * node + a], (double)s[a], v[0]);
                }
            }
        }
        __syncthreads();   // the next tile overwrites xs
    }
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) finish_pq_inner(v[0], sc);
}

template <typename VT, int L>
__global__ void cg32_spmv_dot_csr(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const VT* __restrict__ val, const float* __restrict__ p,
                                  float* __restrict__ q, int64_t n, double* partials, CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = t / L;
    const int sub = (int)(t % L);
    double v[1] = {0.0};
    const float sum = csr_row_sum_low<VT, L>(row, sub, n, rowptr, col, val, p);
    if (row < n && sub == 0) {
        q[row] = sum;
        v[0] = (double)p[row] * (double)sum;
    }
    if (grid_sum<1, 1024>(v, partials, sc->counters) && threadIdx.x == 0) finish_pq_inner(v[0], sc);
}

// Inner step of the refinement: w += a p, r_in -= a q, r_in.r_in.  Rows four at a
// time (float4; the vectors are 16-byte aligned) and the rows past the last group
// one by one.  Each thread sums its rows' squares as a float pair (Dot2) on the
// FP32 pipe; where its |r_in| leave [2^-60, 2^60] (the squares would leave the
// float range, or NaN/Inf) it sums them again in FP64.
__global__ void __launch_bounds__(256, 4) cg32_update(int64_t n, float* __restrict__ w,
                                                   float* __restrict__ r,
                                                   const float* __restrict__ p,
                                                   const float* __restrict__ q, double* partials,
                                                   CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const float a = (float)sc->alpha;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = n >> 2;
    float4* W4 = reinterpret_cast<float4*>(w);
    float4* R4 = reinterpret_cast<float4*>(r);
    const float4* P4 = reinterpret_cast<const float4*>(p);
    const float4* Q4 = reinterpret_cast<const float4*>(q);
    Dot2 acc;
    float amax = 0.0f;
    for (int64_t g = tid; g < n4; g += nth) {
        const float4 pv = P4[g], qv = Q4[g];
        float4 rv = R4[g], wv = W4[g];
        wv.x = fmaf(a, pv.x, wv.x);
        wv.y = fmaf(a, pv.y, wv.y);
        wv.z = fmaf(a, pv.z, wv.z);
        wv.w = fmaf(a, pv.w, wv.w);
        rv.x = fmaf(-a, qv.x, rv.x);
        rv.y = fmaf(-a, qv.y, rv.y);
        rv.z = fmaf(-a, qv.z, rv.z);
        rv.w = fmaf(-a, qv.w, rv.w);
        W4[g] = wv;
        R4[g] = rv;
        acc.add(rv.x, rv.x);
        acc.add(rv.y, rv.y);
        acc.add(rv.z, rv.z);
        acc.add(rv.w, rv.w);
        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(rv.x), fabsf(rv.y)), fmaxf(fabsf(rv.z), fabsf(rv.w))));
    }
    for (int64_t i = 4 * n4 + tid; i < n; i += nth) {
        w[i] = fmaf(a, p[i], w[i]);
        const float ri = fmaf(-a, q[i], r[i]);
        r[i] = ri;
        acc.add(ri, ri);
        amax = fmaxf(amax, fabsf(ri));
    }
    double v[1] = {acc.value()};
    if (!(amax <= 0x1p60f) || (amax > 0.0f && amax < 0x1p-60f) || !isfinite(v[0])) {
        double t = 0.0;
        for (int64_t g = tid; g < n4; g += nth) {
            const float4 rv = R4[g];
            t = fma((double)rv.x, (double)rv.x, t);
            t = fma((double)rv.y, (double)rv.y, t);
            t = fma((double)rv.z, (double)rv.z, t);
            t = fma((double)rv.w, (double)rv.w, t);
        }
        for (int64_t i = 4 * n4 + tid; i < n; i += nth) t = fma((double)r[i], (double)r[i], t);
        v[0] = t;
    }
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) {
        sc->iters += 1;
        sc->iters_in += 1;
        sc->rr = v[0];
        if (!isfinite(v[0])) sc->status = CG_BREAKDOWN;
        else if (v[0] <= sc->thresh_in) sc->status = CG_CONVERGED;
        else if (sc->iters_in >= sc->max_iter) sc->status = CG_MAXITER;
        else {
            sc->beta = v[0] / sc->rho;
            sc->rho = v[0];
        }
    }
}

// p = r_in + beta p, four rows at a time.
__global__ void __launch_bounds__(256, 4) cg32_pupdate(int64_t n, float* __restrict__ p,
                                                    const float* __restrict__ r, const CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const float beta = (float)sc->beta;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = n >> 2;
    float4* P4 = reinterpret_cast<float4*>(p);
    const float4* R4 = reinterpret_cast<const float4*>(r);
    for (int64_t g = tid; g < n4; g += nth) {
        const float4 pv = P4[g], rv = R4[g];
        P4[g] = make_float4(fmaf(beta, pv.x, rv.x), fmaf(beta, pv.y, rv.y), fmaf(beta, pv.z, rv.z),
                            fmaf(beta, pv.w, rv.w));
    }
    for (int64_t i = 4 * n4 + tid; i < n; i += nth) p[i] = fmaf(beta, p[i], r[i]);
}

// Outer step: r = b - Ax (FP64; Ax = q or 0), rhs = float(S r); inner state
// w = 0, r_in = p = rhs.  Sums: r.r (outer), rhs.rhs (inner rho), b.b.
// Reliable updates (keep_p): the same residual replaces the inner recurrence
// residual but p is kept; beta = rho' / rho for the p update that follows, the
// inner step count runs on, and the inner stop threshold is the smaller
// reduction of delta^2 rho' and the estimate c^2 rho' <= tol^2 b.b, where
// c = ||r|| / ||S r|| (the scaled residual's norm against the true one).
__global__ void __launch_bounds__(256) refine_residual(int64_t n, const double* __restrict__ b,
                                                       const double* __restrict__ q,
                                                       const double* __restrict__ scale,
                                                       float* __restrict__ w, float* __restrict__ r_in,
                                                       float* __restrict__ p, double tol2,
                                                       double inner_tol2, int reliable, int keep_p,
                                                       double* partials, CgScalars* sc) {
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double bi = b[i];
        const double ri = q ? bi - q[i] : bi;
        const float rs = (float)(scale[i] * ri);
        w[i] = 0.0f;
        r_in[i] = rs;
        if (!keep_p) p[i] = rs;
        v[0] = fma(ri, ri, v[0]);
        v[1] = fma((double)rs, (double)rs, v[1]);
        v[2] = fma(bi, bi, v[2]);
    }
    if (grid_sum<3>(v, partials, sc->counters) && threadIdx.x == 0) {
        sc->true_rr = v[0];
        if (keep_p) sc->beta = v[1] / sc->rho;
        sc->rho = v[1];
        sc->bb = v[2];
        sc->thresh2 = tol2 * v[2];
        if (reliable) {
            sc->thresh_in = fmax(inner_tol2 * v[1], v[0] > 0.0 ? tol2 * v[2] * v[1] / v[0] : 0.0);
        } else {
            sc->thresh_in = inner_tol2 * v[1];
            sc->iters_in = 0;
        }
        if (!isfinite(v[0]) || !isfinite(v[1])) sc->status = CG_BREAKDOWN;
        else if (v[0] <= sc->thresh2) sc->status = CG_CONVERGED;
        else sc->status = CG_RUNNING;
    }
}

// x += S w in FP64.
__global__ void __launch_bounds__(256, 8) refine_update(int64_t n, double* __restrict__ x,
                                                     const double* __restrict__ scale,
                                                     const float* __restrict__ w) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = fma(scale[i], (double)w[i], x[i]);
}

// ------------------------------------------------------------------ flexible CG (FESPMV_CG_FLEXIBLE)
// Notay's flexible CG with one kept direction, in FP64, preconditioned by a fixed
// number of low-precision CG steps on B = S A S (the inner kernels above, with a
// scalar block of their own).  Per outer step: inner start, m inner steps,
// beta = -z.q / p.q, p = z + beta p with p.r, q = A p with p.q (alpha = p.r / p.q),
// then x, r and ||r||.  z = S w is formed on the fly and never stored.

// Inner start from the outer residual: r_in = float(S r), w = 0, p_in = r_in.
__global__ void __launch_bounds__(256) fcg_inner_init(int64_t n, const double* __restrict__ r,
                                                      const double* __restrict__ scale, float* __restrict__ w,
                                                      float* __restrict__ rin, float* __restrict__ pin, int m,
                                                      double* partials, CgScalars* sc_in, const CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    double v[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float rs = (float)(scale[i] * r[i]);
        w[i] = 0.0f;
        rin[i] = rs;
        pin[i] = rs;
        v[0] = fma((double)rs, (double)rs, v[0]);
    }
    if (grid_sum<1>(v, partials, sc_in->counters) && threadIdx.x == 0) {
        sc_in->rho = v[0];
        sc_in->iters_in = 0;
        sc_in->max_iter = m;
        sc_in->thresh_in = 0.0;
        sc_in->status = !isfinite(v[0]) ? CG_BREAKDOWN : (v[0] > 0.0 ? CG_RUNNING : CG_CONVERGED);
    }
}

// beta = -(S w).q / p.q with q = A p of the previous direction (0 at the first step).
__global__ void __launch_bounds__(256) fcg_beta(int64_t n, const float* __restrict__ w,
                                                const double* __restrict__ scale, const double* __restrict__ q,
                                                double* partials, CgScalars* sc) {
    if (sc->status != CG_RUNNING || sc->first) return;
    double v[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v[0] = fma(scale[i] * (double)w[i], q[i], v[0]);
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) {
        sc->beta = -v[0] / sc->pq;
        if (!isfinite(sc->beta)) sc->status = CG_BREAKDOWN;
    }
}

// p = S w + beta p (p = S w at the first step) and p.r, the numerator of alpha.
__global__ void __launch_bounds__(256) fcg_direction(int64_t n, const float* __restrict__ w,
                                                     const double* __restrict__ scale, double* __restrict__ p,
                                                     const double* __restrict__ r, float2* __restrict__ pdf,
                                                     double* partials, CgScalars* sc) {
    if (sc->status != CG_RUNNING) return;
    const bool first = sc->first;
    const double beta = sc->beta;
    double v[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double z = scale[i] * (double)w[i];
        const double pi = first ? z : fma(beta, p[i], z);
        p[i] = pi;
        if (pdf) pdf[i] = df_split(pi);
        v[0] = fma(pi, r[i], v[0]);
    }
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) {
        sc->rho = v[0];
        sc->first = 0;
        if (!isfinite(v[0])) sc->status = CG_BREAKDOWN;
    }
}

// x += alpha p, r -= alpha q, ||r||^2; counts the outer step and copies the inner
// step count for the host.
__global__ void __launch_bounds__(256, 4) fcg_update(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                     const double* __restrict__ p, const double* __restrict__ q,
                                                     double* partials, CgScalars* sc, const CgScalars* sc_in) {
    if (sc->status != CG_RUNNING) return;
    const double a = sc->alpha;
    double v[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fma(a, p[i], x[i]);
        const double ri = fma(-a, q[i], r[i]);
        r[i] = ri;
        v[0] = fma(ri, ri, v[0]);
    }
    if (grid_sum<1>(v, partials, sc->counters) && threadIdx.x == 0) {
        sc->iters += 1;
        sc->iters_in = sc_in->iters;
        sc->rr = v[0];
        if (!isfinite(v[0])) sc->status = CG_BREAKDOWN;
        else if (v[0] <= sc->thresh2) sc->status = CG_CONVERGED;
        else if (sc->iters >= sc->max_iter) sc->status = CG_MAXITER;
    }
}

// ------------------------------------------------------------------ host side
//
// A solve in flight is a CgRun: a small state machine that enqueues work on
// its stream and advances when the event of its last status copy has fired.
// cg_solve drives one run to the end (blocking); the solve server advances
// many runs round-robin, each on its own stream and workspace, so their
// iterations overlap on the device.

// SLICED CG products run persistent: at most 8 blocks per SM, warps stride over slices.
static unsigned spmv_grid(const fespmv_mat* A) {
    if (A->format == FESPMV_FMT_SLICED) {
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const unsigned full = grid_for(A->n_slices * 32, A->block);
        const unsigned cap = (unsigned)sms * (2048u / (unsigned)A->block);
        return std::max(1u, std::min(full, cap));
    }
    return grid_for(A->n * A->csr_lanes, A->block);
}

// A persistent tiled kernel's grid: the blocks of `kernel` resident at once (with
// its shared memory), at most one per tile.
template <typename Kernel>
static unsigned tiled_grid(const fespmv_mat* A, Kernel kernel, size_t smem) {
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kTiledBlock, smem);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(A->n_tiles, (int64_t)sms * std::max(per_sm, 1)));
}

// A persistent SLICED kernel's grid: spmv_grid, capped at the blocks of `kernel`
// that are resident at once (kernels holding more than 32 registers fit fewer).
template <typename Kernel>
static unsigned resident_grid(const fespmv_mat* A, Kernel kernel) {
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, A->block, 0);
    return std::max(1u, std::min(spmv_grid(A), (unsigned)(sms * std::max(per_sm, 1))));
}

void destroy_work(CgWork* w) {
    if (!w) return;
    if (w->graph) cudaGraphExecDestroy(w->graph);
    if (w->graph_cg1) cudaGraphExecDestroy(w->graph_cg1);
    for (cudaGraphExec_t g : w->graph_low)
        if (g) cudaGraphExecDestroy(g);
    for (cudaGraphExec_t g : w->graph_flex)
        if (g) cudaGraphExecDestroy(g);
    for (cudaEvent_t e : w->ev)
        if (e) cudaEventDestroy(e);
    if (w->cap) cudaStreamDestroy(w->cap);
    void* ptrs[] = {w->x, w->r, w->p, w->q, w->b, w->dinv, w->partials, w->sc, w->sc_in,
                    w->w32, w->r32, w->p32, w->q32, w->pdf, w->u, w->s};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (w->h_sc) cudaFreeHost(w->h_sc);
    if (w->h_io) cudaFreeHost(w->h_io);
    delete w;
}

void free_cg(fespmv_mat* A) {
    destroy_work(A->cg);
    A->cg = nullptr;
}

static int work_alloc(CgWork* w, void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMalloc(%zu bytes) for %s failed: %s", bytes, what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? FESPMV_ERR_OOM : FESPMV_ERR_CUDA;
    }
    w->bytes += (int64_t)bytes;
    return FESPMV_OK;
}

// Workspace bytes one solve of A needs (FP64 vectors, partial sums, scalars and,
// for refined precisions, the float vectors).
int64_t work_bytes(const fespmv_mat* A, bool refine) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t upd = std::max(1u, std::min(grid_for(A->n, 256), (unsigned)(sms * 8)));
    const int64_t np = grid_sum_doubles(
        std::max<int64_t>({(int64_t)spmv_grid(A), upd, A->tiled ? A->n_tiles : 0, A->nb_tiles}));
    int64_t b = 8 * 8 * A->n + 8 * np + 2 * (int64_t)sizeof(CgScalars);
    if (A->d_vdf) b += 8 * A->n;
    if (refine) b += 4 * 4 * A->n;
    return b;
}

int create_work(const fespmv_mat* A, bool host_staging, CgWork** out) {
    *out = nullptr;
    CgWork* w = new CgWork();
    w->n = A->n;
    int dev = 0, sms = 0, rc;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
        destroy_work(w);
        return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    w->upd_grid = std::max(1u, std::min(grid_for(A->n, 256), (unsigned)(sms * 4)));
    const size_t nb = sizeof(double) * (size_t)A->n;
    double** vecs[] = {&w->x, &w->r, &w->p, &w->q, &w->b, &w->dinv, &w->u, &w->s};
    for (double** v : vecs)
        if ((rc = work_alloc(w, (void**)v, nb, "CG vector"))) { destroy_work(w); return rc; }
    if (A->d_vdf && (rc = work_alloc(w, (void**)&w->pdf, sizeof(float2) * (size_t)A->n, "CG float-pair p"))) {
        destroy_work(w);
        return rc;
    }
    // one partial per block of the largest reduction grid: the persistent products, the
    // vector updates, or the tiled products (at most one block per tile)
    const size_t np = (size_t)grid_sum_doubles(
        std::max<int64_t>({(int64_t)spmv_grid(A), (int64_t)w->upd_grid, A->tiled ? A->n_tiles : 0, A->nb_tiles}));
    if ((rc = work_alloc(w, (void**)&w->partials, sizeof(double) * np, "CG partial sums")) ||
        (rc = work_alloc(w, (void**)&w->sc, sizeof(CgScalars), "CG scalars")) ||
        (rc = work_alloc(w, (void**)&w->sc_in, sizeof(CgScalars), "inner CG scalars"))) {
        destroy_work(w);
        return rc;
    }
    if ((e = cudaMallocHost((void**)&w->h_sc, 2 * sizeof(CgScalars))) != cudaSuccess ||
        (host_staging && (e = cudaMallocHost((void**)&w->h_io, nb ? nb : 16)) != cudaSuccess) ||
        (e = cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&w->ev[0], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&w->ev[1], cudaEventDisableTiming)) != cudaSuccess) {
        destroy_work(w);
        return cuda_fail(e, "CG workspace setup");
    }
    *out = w;
    return FESPMV_OK;
}

static int ensure_workspace(fespmv_mat* A) {
    if (A->cg) return FESPMV_OK;
    int rc = create_work(A, false, &A->cg);
    if (rc == FESPMV_OK) A->device_bytes += A->cg->bytes;
    return rc;
}

template <int V>
static void launch_spmv_dot_sliced(const fespmv_mat* A, CgWork* w, cudaStream_t s) {
    constexpr int U = (V == 1) ? 8 : (V == 2 ? 4 : 2);
    if (A->tiled) {
        const size_t smem = sizeof(double) * (A->tile_dmax + 1);
        const unsigned g = tiled_grid(A, cg_spmv_dot_tiled<V, U>, smem);
        cg_spmv_dot_tiled<V, U><<<g, kTiledBlock, smem, s>>>(A->d_meta, A->d_tlidx, A->d_val, A->d_tiles,
                                                             A->d_tdict, w->p, w->q, A->n, A->n_tiles,
                                                             w->partials, w->sc);
        return;
    }
    const unsigned g = resident_grid(A, cg_spmv_dot_sliced<V, U>);
    cg_spmv_dot_sliced<V, U><<<g, A->block, 0, s>>>(A->d_meta, A->d_col, A->d_val, w->p, w->q, A->n_slices,
                                                    A->n, w->partials, w->sc);
}

template <int L>
static void launch_spmv_dot_csr(const fespmv_mat* A, CgWork* w, cudaStream_t s) {
    cg_spmv_dot_csr<L><<<spmv_grid(A), A->block, 0, s>>>(A->d_rowptr, A->d_colind, A->d_val, w->p,
                                                         w->q, A->n, w->partials, w->sc);
}

template <int V>
static void launch_spmv_dot_df(const fespmv_mat* A, CgWork* w, cudaStream_t s) {
    constexpr int U = (V == 4) ? 2 : 4;
    if (A->tiled) {
        const size_t smem = sizeof(float2) * (A->tile_dmax + 1);
        const unsigned g = tiled_grid(A, cg_spmv_dot_tiled_df<V, U>, smem);
        cg_spmv_dot_tiled_df<V, U><<<g, kTiledBlock, smem, s>>>(A->d_meta, A->d_tlidx, A->d_vdf, A->d_val,
                                                                A->d_col, A->d_tiles, A->d_tdict, w->p, w->pdf,
                                                                w->q, A->n, A->n_tiles, w->partials, w->sc);
        return;
    }
    cg_spmv_dot_df<V, U><<<spmv_grid(A), A->block, 0, s>>>(A->d_meta, A->d_col, A->d_vdf, A->d_val, w->p,
                                                           w->pdf, w->q, A->n_slices, A->n,
                                                           w->partials, w->sc);
}

// q = A p with p.q (alpha = rho / p.q), the FP64 product of the handle.
static void launch_spmv_dot(const fespmv_mat* A, CgWork* w, cudaStream_t s) {
    if (A->d_vdf) {
        switch (A->vec) {
            case 1: launch_spmv_dot_df<1>(A, w, s); break;
            case 4: launch_spmv_dot_df<4>(A, w, s); break;
            default: launch_spmv_dot_df<2>(A, w, s); break;
        }
    } else if (A->format == FESPMV_FMT_SLICED) {
        switch (A->vec) {
            case 1: launch_spmv_dot_sliced<1>(A, w, s); break;
            case 4: launch_spmv_dot_sliced<4>(A, w, s); break;
            default: launch_spmv_dot_sliced<2>(A, w, s); break;
        }
    } else {
        switch (A->csr_lanes) {
            case 1: launch_spmv_dot_csr<1>(A, w, s); break;
            case 2: launch_spmv_dot_csr<2>(A, w, s); break;
            case 4: launch_spmv_dot_csr<4>(A, w, s); break;
            case 8: launch_spmv_dot_csr<8>(A, w, s); break;
            case 16: launch_spmv_dot_csr<16>(A, w, s); break;
            default: launch_spmv_dot_csr<32>(A, w, s); break;
        }
    }
}

static void launch_iteration(const fespmv_mat* A, CgWork* w, cudaStream_t s) {
    launch_spmv_dot(A, w, s);
    cg_update<<<w->upd_grid, 256, 0, s>>>(A->n, w->x, w->r, w->p, w->q, w->dinv, w->partials, w->sc);
    cg_pupdate<<<w->upd_grid, 256, 0, s>>>(A->n, w->p, w->r, w->dinv, w->pdf, w->sc);
}

template <int V>
static void launch_cg1_sliced(const fespmv_mat* A, CgWork* w, cudaStream_t s) {
    constexpr int U = (V == 1) ? 8 : (V == 2 ? 4 : 2);
    if (A->tiled) {
        const size_t smem = sizeof(double) * (A->tile_dmax + 1);
        const unsigned g = tiled_grid(A, cg1_spmv_dots_tiled<V, U>, smem);
        cg1_spmv_dots_tiled<V, U><<<g, kTiledBlock, smem, s>>>(A->d_meta, A->d_tlidx, A->d_val, A->d_tiles,
                                                               A->d_tdict, w->u, w->r, w->q, A->n,
                                                               A->n_tiles, w->partials, w->sc);
        return;
    }
    const unsigned g = resident_grid(A, cg1_spmv_dots_sliced<V, U>);
    cg1_spmv_dots_sliced<V, U><<<g, A->block, 0, s>>>(A->d_meta, A->d_col, A->d_val, w->u, w->r,
                                                                 w->q, A->n_slices, A->n, w->partials,
                                                                 w->sc);
}

template <int L>
static void launch_cg1_csr(const fespmv_mat* A, CgWork* w, cudaStream_t s) {
    cg1_spmv_dots_csr<L><<<spmv_grid(A), A->block, 0, s>>>(A->d_rowptr, A->d_colind, A->d_val, w->u, w->r,
                                                           w->q, A->n, w->partials, w->sc);
}

// One single-reduction iteration: w (= q) = A u with the three dots, then the update.
static void launch_iteration_cg1(const fespmv_mat* A, CgWork* w, cudaStream_t s) {
    if (A->format == FESPMV_FMT_SLICED) {
        switch (A->vec) {
            case 1: launch_cg1_sliced<1>(A, w, s); break;
            case 4: launch_cg1_sliced<4>(A, w, s); break;
            default: launch_cg1_sliced<2>(A, w, s); break;
        }
    } else {
        switch (A->csr_lanes) {
            case 1: launch_cg1_csr<1>(A, w, s); break;
            case 2: launch_cg1_csr<2>(A, w, s); break;
            case 4: launch_cg1_csr<4>(A, w, s); break;
            case 8: launch_cg1_csr<8>(A, w, s); break;
            case 16: launch_cg1_csr<16>(A, w, s); break;
            default: launch_cg1_csr<32>(A, w, s); break;
        }
    }
    cg1_update<<<w->upd_grid, 256, 0, s>>>(A->n, w->x, w->r, w->u, w->p, w->s, w->q, w->dinv, w->sc);
}

template <typename VT, int V>
static void launch_inner_dot_sliced(const fespmv_mat* A, CgWork* w, const VT* val, cudaStream_t s) {
    constexpr int U = (V == 4) ? 4 : 8;
    if (A->tiled) {
        constexpr int UT = (V == 1) ? 8 : (V == 2 ? 4 : 2);
        const size_t smem = sizeof(float) * (A->tile_dmax + 1);
        const unsigned g = tiled_grid(A, cg32_spmv_dot_tiled<VT, V, UT>, smem);
        cg32_spmv_dot_tiled<VT, V, UT><<<g, kTiledBlock, smem, s>>>(A->d_meta, A->d_tlidx, val, A->d_tiles,
                                                                    A->d_tdict, w->p32, w->q32, A->n,
                                                                    A->n_tiles, w->partials, w->sc);
        return;
    }
    cg32_spmv_dot_sliced<VT, V, U><<<spmv_grid(A), A->block, 0, s>>>(A->d_meta, A->d_col, val, w->p32,
                                                                     w->q32, A->n_slices, A->n,
                                                                     w->partials, w->sc);
}

template <typename VT, int L>
static void launch_inner_dot_csr(const fespmv_mat* A, CgWork* w, const VT* val, cudaStream_t s) {
    cg32_spmv_dot_csr<VT, L><<<spmv_grid(A), A->block, 0, s>>>(A->d_rowptr, A->d_colind, val, w->p32,
                                                               w->q32, A->n, w->partials, w->sc);
}

template <typename VT>
static void launch_inner_dot(const fespmv_mat* A, CgWork* w, const VT* val, cudaStream_t s) {
    if (A->nb) {
        const VT* nbv = std::is_same<VT, float>::value ? reinterpret_cast<const VT*>(A->d_nb32)
                                                       : reinterpret_cast<const VT*>(A->d_nb16);
        if (A->nb_tiles > 0) {
            // one block per tile: a tile is a large unit (256 node rows), so blocks striding
            // over tiles would leave the last round of tiles to a few SMs
            const size_t smem = sizeof(float) * 3 * (size_t)(A->nb_tile_dmax + 1);
            const unsigned g = (unsigned)A->nb_tiles;
            cg32_spmv_dot_nb_tiled<VT, std::is_same<VT, float>::value ? 2 : 4><<<g, 256, smem, s>>>(A->d_nbmeta, A->d_nbtlidx, nbv, A->d_nbtiles,
                                                               A->d_nbtdict, w->p32, w->q32, A->nb_tiles, A->n / 3,
                                                               w->partials, w->sc);
            return;
        }
        const unsigned g = std::max(1u, std::min(spmv_grid(A), grid_for(A->nb_slices * 32, 256)));
        cg32_spmv_dot_nb<VT, 2><<<g, 256, 0, s>>>(A->d_nbmeta, A->d_nbcol, nbv, w->p32, w->q32, A->nb_slices,
                                                  A->n / 3, w->partials, w->sc);
        return;
    }
    if (A->format == FESPMV_FMT_SLICED) {
        switch (A->vec) {
            case 1: launch_inner_dot_sliced<VT, 1>(A, w, val, s); break;
            case 4: launch_inner_dot_sliced<VT, 4>(A, w, val, s); break;
            default: launch_inner_dot_sliced<VT, 2>(A, w, val, s); break;
        }
    } else {
        switch (A->csr_lanes) {
            case 1: launch_inner_dot_csr<VT, 1>(A, w, val, s); break;
            case 2: launch_inner_dot_csr<VT, 2>(A, w, val, s); break;
            case 4: launch_inner_dot_csr<VT, 4>(A, w, val, s); break;
            case 8: launch_inner_dot_csr<VT, 8>(A, w, val, s); break;
            case 16: launch_inner_dot_csr<VT, 16>(A, w, val, s); break;
            default: launch_inner_dot_csr<VT, 32>(A, w, val, s); break;
        }
    }
}

static void launch_inner_iteration(const fespmv_mat* A, CgWork* w, int bf16, cudaStream_t s) {
    if (bf16)
        launch_inner_dot<__nv_bfloat16>(A, w, reinterpret_cast<const __nv_bfloat16*>(A->d_val16), s);
    else
        launch_inner_dot<float>(A, w, A->d_val32, s);
    cg32_update<<<w->upd_grid, 256, 0, s>>>(A->n, w->w32, w->r32, w->p32, w->q32, w->partials, w->sc);
    cg32_pupdate<<<w->upd_grid, 256, 0, s>>>(A->n, w->p32, w->r32, w->sc);
}

// One outer step of the flexible CG: inner start, m inner steps on the inner
// scalars, then the FP64 direction, product and update.
static void launch_flexible_iteration(const fespmv_mat* A, CgWork* w, int bf16, int m, cudaStream_t s) {
    fcg_inner_init<<<w->upd_grid, 256, 0, s>>>(A->n, w->r, A->d_scale, w->w32, w->r32, w->p32, m, w->partials,
                                               w->sc_in, w->sc);
    CgScalars* outer = w->sc;
    w->sc = w->sc_in;   // the inner kernels read the workspace's scalar block
    for (int j = 0; j < m; ++j) launch_inner_iteration(A, w, bf16, s);
    w->sc = outer;
    fcg_beta<<<w->upd_grid, 256, 0, s>>>(A->n, w->w32, A->d_scale, w->q, w->partials, w->sc);
    fcg_direction<<<w->upd_grid, 256, 0, s>>>(A->n, w->w32, A->d_scale, w->p, w->r, w->pdf, w->partials, w->sc);
    launch_spmv_dot(A, w, s);
    fcg_update<<<w->upd_grid, 256, 0, s>>>(A->n, w->x, w->r, w->p, w->q, w->partials, w->sc, w->sc_in);
}

// Graph of `chunk` iterations (kind 0: FP64; 1: FP32 inner; 2: BF16 inner; 3:
// single-reduction FP64; 4, 5: flexible CG outer steps with FP32 / BF16 inner
// steps, `m` of them) for this workspace; kernel arguments are the workspace's
// fixed pointers.
static int ensure_graph(const fespmv_mat* A, CgWork* w, int kind, int chunk, int m = 0) {
    cudaGraphExec_t& slot = kind == 0 ? w->graph
                          : kind == 3 ? w->graph_cg1
                          : kind >= 4 ? w->graph_flex[kind - 4] : w->graph_low[kind - 1];
    int& slot_chunk = kind == 0 ? w->graph_chunk
                    : kind == 3 ? w->chunk_cg1
                    : kind >= 4 ? w->chunk_flex[kind - 4] : w->chunk_low[kind - 1];
    if (slot && slot_chunk == chunk && (kind < 4 || w->steps_flex[kind - 4] == m)) return FESPMV_OK;
    if (slot) {
        cudaGraphExecDestroy(slot);
        slot = nullptr;
    }
    cudaGraph_t g = nullptr;
    FESPMV_CUDA(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk; ++i) {
        if (kind == 0) launch_iteration(A, w, w->cap);
        else if (kind == 3) launch_iteration_cg1(A, w, w->cap);
        else if (kind >= 4) launch_flexible_iteration(A, w, kind - 4, m, w->cap);
        else launch_inner_iteration(A, w, kind - 1, w->cap);
    }
    cudaError_t e = cudaStreamEndCapture(w->cap, &g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&slot, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    slot_chunk = chunk;
    if (kind >= 4) w->steps_flex[kind - 4] = m;
    return FESPMV_OK;
}

int ensure_low_work(CgWork* w) {
    if (w->w32) return FESPMV_OK;
    const size_t nb = sizeof(float) * (size_t)w->n;
    float** vecs[] = {&w->w32, &w->r32, &w->p32, &w->q32};
    for (float** v : vecs) {
        int rc = work_alloc(w, (void**)v, nb, "refinement vector");
        if (rc) return rc;
    }
    return FESPMV_OK;
}

__global__ void cg_copy_flag(CgScalars* sc, const int* flag) {
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->pad = flag ? *flag : 0;
}


int normalize_options(cg_options& o) {
    if (o.tol == 0.0) o.tol = 1e-10;
    if (o.max_iter == 0) o.max_iter = 100000;
    if (o.max_restarts == 0) o.max_restarts = 3;
    if (o.max_restarts < 0) o.max_restarts = 0;
    if (o.check_every == 0) o.check_every = 16;
    if (o.max_outer == 0) o.max_outer = 60;
    if (o.inner_tol == 0.0) o.inner_tol = (o.flags & FESPMV_CG_RELIABLE) ? 1e-1 : 1e-2;
    if (o.inner_steps == 0) o.inner_steps = 8;
    if (!(o.tol > 0.0) || o.max_iter < 0 || o.check_every < 1 || o.check_every > 4096 ||
        o.precision < FESPMV_CG_F64 || o.precision > FESPMV_CG_BF16_REFINE || o.max_outer < 0 ||
        !(o.inner_tol > 0.0 && o.inner_tol < 1.0) ||
        o.inner_steps < 1 || o.inner_steps > 1024 ||
        (o.flags & ~(FESPMV_IO_PERMUTED | FESPMV_IO_HOST | FESPMV_CG_X0 | FESPMV_CG_NO_PRECOND |
                     FESPMV_CG_SINGLE_REDUCTION | FESPMV_CG_RELIABLE | FESPMV_CG_FLEXIBLE |
                     FESPMV_CG_NO_CLUSTER))) {
        set_error("bad cg_options");
        return FESPMV_ERR_INVALID_ARG;
    }
    if ((o.flags & FESPMV_CG_SINGLE_REDUCTION) && o.precision != FESPMV_CG_F64) {
        set_error("FESPMV_CG_SINGLE_REDUCTION applies to FESPMV_CG_F64 only");
        return FESPMV_ERR_UNSUPPORTED;
    }
    if ((o.flags & FESPMV_CG_RELIABLE) && o.precision == FESPMV_CG_F64) {
        set_error("FESPMV_CG_RELIABLE applies to the refined precisions only");
        return FESPMV_ERR_UNSUPPORTED;
    }
    if ((o.flags & FESPMV_CG_FLEXIBLE) && (o.precision == FESPMV_CG_F64 || (o.flags & FESPMV_CG_RELIABLE))) {
        set_error("FESPMV_CG_FLEXIBLE applies to the refined precisions, without FESPMV_CG_RELIABLE");
        return FESPMV_ERR_UNSUPPORTED;
    }
    return FESPMV_OK;
}

int check_precision(const fespmv_mat* A, int precision) {
    if (A->col_order == FESPMV_COLS_ORIGINAL) {
        set_error("CG needs x and A x in one numbering: not on a FESPMV_COLS_ORIGINAL handle");
        return FESPMV_ERR_UNSUPPORTED;
    }
    if (precision == FESPMV_CG_F32_REFINE && !A->d_val32) {
        set_error("FESPMV_CG_F32_REFINE needs a handle created with FESPMV_PREC_F32");
        return FESPMV_ERR_UNSUPPORTED;
    }
    if (precision == FESPMV_CG_BF16_REFINE && !A->d_val16) {
        set_error("FESPMV_CG_BF16_REFINE needs a handle created with FESPMV_PREC_BF16");
        return FESPMV_ERR_UNSUPPORTED;
    }
    return FESPMV_OK;
}

// Copies the status word to the host and records the event of slot `k`.
static int enqueue_status(CgRun& r, int k) {
    FESPMV_CUDA(cudaMemcpyAsync(&r.w->h_sc[k], r.w->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, r.s));
    FESPMV_CUDA(cudaEventRecord(r.w->ev[k], r.s));
    return FESPMV_OK;
}

static int enqueue_graph(CgRun& r) {
    const int k = (r.head + r.queued) & 1;
    FESPMV_CUDA(cudaGraphLaunch(r.graph, r.s));
    int rc = enqueue_status(r, k);
    if (rc) return rc;
    ++r.queued;
    --r.graphs_left;
    return FESPMV_OK;
}

static int start_graphs(CgRun& r, int kind, int max_iter) {
    int rc = ensure_graph(r.A, r.w, kind, r.o.check_every, r.o.inner_steps);
    if (rc) return rc;
    r.graph = kind == 0 ? r.w->graph
            : kind == 3 ? r.w->graph_cg1
            : kind >= 4 ? r.w->graph_flex[kind - 4] : r.w->graph_low[kind - 1];
    r.graphs_left = (int64_t)max_iter / r.o.check_every + 3;
    r.head = 0;
    r.queued = 0;
    if ((rc = enqueue_graph(r))) return rc;
    if (r.graphs_left > 0 && (rc = enqueue_graph(r))) return rc;
    r.phase = PH_ITER;
    return FESPMV_OK;
}

static int enqueue_init(CgRun& r, bool ax) {
    CgWork* w = r.w;
    int rc;
    const bool cg1 = r.o.flags & FESPMV_CG_SINGLE_REDUCTION;
    if (ax && (rc = launch_spmv(r.A, w->x, w->q, r.s))) return rc;
    if (cg1) {
        FESPMV_CUDA(cudaMemsetAsync(w->p, 0, sizeof(double) * (size_t)r.A->n, r.s));
        FESPMV_CUDA(cudaMemsetAsync(w->s, 0, sizeof(double) * (size_t)r.A->n, r.s));
    }
    cg_init<<<w->upd_grid, 256, 0, r.s>>>(r.A->n, w->b, ax ? w->q : nullptr, w->r, cg1 ? w->u : w->p,
                                          w->dinv, r.o.tol * r.o.tol, w->partials, w->sc,
                                          cg1 ? nullptr : w->pdf);
    FESPMV_CUDA(cudaGetLastError());
    r.phase = PH_INIT_WAIT;
    return enqueue_status(r, 0);
}

static int enqueue_residual(CgRun& r, bool ax) {
    CgWork* w = r.w;
    int rc;
    const int reliable = (r.o.flags & FESPMV_CG_RELIABLE) ? 1 : 0;
    const int keep_p = reliable && r.outer > 0;
    if (ax && (rc = launch_spmv(r.A, w->x, w->q, r.s))) return rc;
    refine_residual<<<w->upd_grid, 256, 0, r.s>>>(r.A->n, w->b, ax ? w->q : nullptr, r.A->d_scale, w->w32,
                                                  w->r32, w->p32, r.o.tol * r.o.tol,
                                                  r.o.inner_tol * r.o.inner_tol, reliable, keep_p,
                                                  w->partials, w->sc);
    // reliable update: the kept direction takes the replaced residual, p = r_in + beta p
    if (keep_p) cg32_pupdate<<<w->upd_grid, 256, 0, r.s>>>(r.A->n, w->p32, w->r32, w->sc);
    FESPMV_CUDA(cudaGetLastError());
    r.phase = PH_RES_WAIT;
    return enqueue_status(r, 0);
}

int run_begin(CgRun& r) {
    CgWork* w = r.w;
    int rc;
    r.restarts = 0;
    r.outer = 0;
    r.prev = INFINITY;
    r.status = CG_RUNNING;
    r.error = FESPMV_OK;
    r.queued = 0;
    r.head = 0;
    CgScalars init;
    std::memset(&init, 0, sizeof(init));
    init.max_iter = r.o.max_iter;
    init.status = CG_RUNNING;
    // the pinned slot doubles as the upload buffer: it is not read until the first status copy
    w->h_sc[1] = init;
    FESPMV_CUDA(cudaMemcpyAsync(w->sc, &w->h_sc[1], sizeof(CgScalars), cudaMemcpyHostToDevice, r.s));
    // small handles: reliable-update refinement in one cluster launch
    const bool reliable_only = (r.o.flags & FESPMV_CG_RELIABLE) && !(r.o.flags & FESPMV_CG_FLEXIBLE);
    if (r.A->format == FESPMV_FMT_SLICED && r.A->n <= kClusterSolveMaxRows && !r.A->d_vdf &&
        !(r.o.flags & FESPMV_CG_NO_CLUSTER) && reliable_only) {
        if ((rc = ensure_low_work(w))) return rc;
        cg_copy_flag<<<1, 32, 0, r.s>>>(w->sc, r.A->d_flag);
        FESPMV_CUDA(cudaGetLastError());
        rc = launch_cluster_cg_reliable(r.A, w, r.o.precision == FESPMV_CG_BF16_REFINE ? 1 : 0, r.o.tol * r.o.tol,
                                        r.o.inner_tol * r.o.inner_tol, r.has_x0 ? 1 : 0, r.o.max_iter,
                                        r.o.max_outer, r.s);
        if (rc) return rc;
        r.phase = PH_CLUSTER_WAIT;
        return enqueue_status(r, 0);
    }
    const bool flexible = r.o.flags & FESPMV_CG_FLEXIBLE;
    if (flexible) {   // the inner scalars (their reduction counters and step count) start at zero
        if ((rc = ensure_low_work(w))) return rc;
        FESPMV_CUDA(cudaMemsetAsync(w->sc_in, 0, sizeof(CgScalars), r.s));
    }
    if (r.o.precision == FESPMV_CG_F64 || flexible) {
        cg_dinv<<<w->upd_grid, 256, 0, r.s>>>(r.A->n, r.A->d_diag, w->dinv,
                                              (r.o.flags & FESPMV_CG_NO_PRECOND) ? 0 : 1, w->sc);
        FESPMV_CUDA(cudaGetLastError());
        return enqueue_init(r, r.has_x0);
    }
    if ((rc = ensure_low_work(w))) return rc;
    cg_copy_flag<<<1, 32, 0, r.s>>>(w->sc, r.A->d_flag);
    FESPMV_CUDA(cudaGetLastError());
    return enqueue_residual(r, r.has_x0);
}

static int finish(CgRun& r, int status) {
    r.status = status;
    CgWork* w = r.w;
    const size_t nb = sizeof(double) * (size_t)r.A->n;
    double* dst = r.out_host ? w->q : r.x_out;
    int rc;
    if (r.permute) {
        if ((rc = launch_gather(w->x, r.A->d_pinv, dst, r.A->n, r.s))) return rc;
    } else {
        FESPMV_CUDA(cudaMemcpyAsync(dst, w->x, nb, cudaMemcpyDeviceToDevice, r.s));
    }
    if (r.out_host) FESPMV_CUDA(cudaMemcpyAsync(r.x_out, w->q, nb, cudaMemcpyDeviceToHost, r.s));
    FESPMV_CUDA(cudaEventRecord(w->ev[0], r.s));
    r.phase = PH_OUT_WAIT;
    return FESPMV_OK;
}

// Advance the run by at most one phase.  Returns FESPMV_OK with *progress set
// when something happened, or an error.  block: wait for the pending event.
int run_step(CgRun& r, bool block, bool* progress) {
    *progress = false;
    if (r.phase == PH_DONE) return FESPMV_OK;
    CgWork* w = r.w;
    const int k = r.phase == PH_ITER ? r.head : 0;
    cudaEvent_t ev = w->ev[k];
    if (block) {
        FESPMV_CUDA(cudaEventSynchronize(ev));
    } else {
        cudaError_t q = cudaEventQuery(ev);
        if (q == cudaErrorNotReady) return FESPMV_OK;
        if (q != cudaSuccess) return cuda_fail(q, "cudaEventQuery");
    }
    *progress = true;
    const CgScalars h = w->h_sc[k];
    int rc = FESPMV_OK;
    switch (r.phase) {
        case PH_INIT_WAIT:
            r.last = h;
            if (h.status == CG_BADDIAG) {
                set_error("Jacobi preconditioning needs a positive, finite diagonal");
                r.error = FESPMV_ERR_BREAKDOWN;
                r.phase = PH_DONE;
                return FESPMV_OK;
            }
            if (h.bb == 0.0) {  // b = 0: x = 0
                FESPMV_CUDA(cudaMemsetAsync(w->x, 0, sizeof(double) * (size_t)r.A->n, r.s));
                r.last.true_rr = 0.0;
                return finish(r, CG_CONVERGED);
            }
            if (h.status == CG_RUNNING) {
                const int kind = (r.o.flags & FESPMV_CG_FLEXIBLE) ? (r.o.precision == FESPMV_CG_BF16_REFINE ? 5 : 4)
                               : (r.o.flags & FESPMV_CG_SINGLE_REDUCTION) ? 3 : 0;
                return start_graphs(r, kind, r.o.max_iter);
            }
            // converged (or failed) before iterating: confirm on the true residual
            if ((rc = launch_spmv(r.A, w->x, w->q, r.s))) return rc;
            cg_true_residual<<<w->upd_grid, 256, 0, r.s>>>(r.A->n, w->b, w->q, w->partials, w->sc);
            FESPMV_CUDA(cudaGetLastError());
            r.phase = PH_TRUE_WAIT;
            return enqueue_status(r, 0);
        case PH_ITER: {
            r.last = h;
            --r.queued;
            r.head ^= 1;
            if (h.status == CG_RUNNING && r.graphs_left > 0) return enqueue_graph(r);
            if (r.queued > 0) return FESPMV_OK;  // let the no-op graphs drain
            if (r.o.precision == FESPMV_CG_F64 || (r.o.flags & FESPMV_CG_FLEXIBLE)) {
                if ((rc = launch_spmv(r.A, w->x, w->q, r.s))) return rc;
                cg_true_residual<<<w->upd_grid, 256, 0, r.s>>>(r.A->n, w->b, w->q, w->partials, w->sc);
                FESPMV_CUDA(cudaGetLastError());
                r.phase = PH_TRUE_WAIT;
                return enqueue_status(r, 0);
            }
            refine_update<<<w->upd_grid, 256, 0, r.s>>>(r.A->n, w->x, r.A->d_scale, w->w32);
            FESPMV_CUDA(cudaGetLastError());
            ++r.outer;
            return enqueue_residual(r, true);
        }
        case PH_TRUE_WAIT: {
            r.last = h;
            int st = h.status == CG_RUNNING ? CG_MAXITER : h.status;
            if (st == CG_CONVERGED && !(h.true_rr <= h.thresh2)) {
                if (r.restarts < r.o.max_restarts && h.iters < r.o.max_iter) {
                    ++r.restarts;
                    return enqueue_init(r, true);
                }
                st = CG_MAXITER;
            }
            return finish(r, st);
        }
        case PH_RES_WAIT:
            r.last = h;
            if (h.pad) {
                set_error("refinement needs a positive, finite diagonal (S = diag(A)^-1/2)");
                r.error = FESPMV_ERR_BREAKDOWN;
                r.phase = PH_DONE;
                return FESPMV_OK;
            }
            if (h.bb == 0.0) {
                FESPMV_CUDA(cudaMemsetAsync(w->x, 0, sizeof(double) * (size_t)r.A->n, r.s));
                return finish(r, CG_CONVERGED);
            }
            if (h.status == CG_CONVERGED || h.status == CG_BREAKDOWN) return finish(r, h.status);
            if (r.outer >= r.o.max_outer) return finish(r, CG_MAXITER);
            if ((r.o.flags & FESPMV_CG_RELIABLE) && h.iters >= r.o.max_iter) return finish(r, CG_MAXITER);
            if (!(h.true_rr < r.prev)) {  // no progress: the low-precision operator is too far from A
                set_error("refinement stagnated: ||b - A x|| did not decrease");
                return finish(r, CG_MAXITER);
            }
            r.prev = h.true_rr;
            return start_graphs(r, r.o.precision == FESPMV_CG_BF16_REFINE ? 2 : 1, r.o.max_iter);
        case PH_CLUSTER_WAIT: {   // the one-launch solve has finished
            r.last = h;
            if (h.pad) {
                set_error("refinement needs a positive, finite diagonal (S = diag(A)^-1/2)");
                r.error = FESPMV_ERR_BREAKDOWN;
                r.phase = PH_DONE;
                return FESPMV_OK;
            }
            r.outer = h.iters_in;
            return finish(r, h.status == CG_RUNNING ? CG_MAXITER : h.status);
        }
        case PH_OUT_WAIT:
            r.phase = PH_DONE;
            return FESPMV_OK;
        default:
            return FESPMV_OK;
    }
}

int run_result(const CgRun& r, cg_result* res) {
    if (r.error) {
        if (res) res->status = r.error;
        return r.error;
    }
    const int out = r.status == CG_CONVERGED ? FESPMV_OK
                  : r.status == CG_BREAKDOWN ? FESPMV_ERR_BREAKDOWN : FESPMV_ERR_NOT_CONVERGED;
    if (res) {
        const CgScalars& h = r.last;
        res->status = out;
        res->iters = h.iters;
        res->restarts = r.restarts;
        res->outer = (r.o.flags & FESPMV_CG_FLEXIBLE) ? h.iters_in : r.outer;
        if (r.o.precision == FESPMV_CG_F64 || (r.o.flags & FESPMV_CG_FLEXIBLE)) {
            res->relres = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
            res->true_relres = h.bb > 0 ? std::sqrt(h.true_rr / h.bb) : 0.0;
        } else {
            res->relres = h.bb > 0 ? std::sqrt(h.true_rr / h.bb) : 0.0;
            res->true_relres = res->relres;
        }
    }
    if (out == FESPMV_ERR_BREAKDOWN) set_error("CG breakdown (p.Ap <= 0 or a non-finite scalar)");
    if (out == FESPMV_ERR_NOT_CONVERGED && (r.o.precision == FESPMV_CG_F64 || (r.o.flags & FESPMV_CG_FLEXIBLE)))
        set_error("CG stopped above the tolerance");
    return out;
}

// Stage b (and x0) into the workspace's permuted vectors on stream s.
int stage_inputs(CgRun& r, const double* b, const double* x0, bool host) {
    CgWork* w = r.w;
    const size_t nb = sizeof(double) * (size_t)r.A->n;
    int rc;
    const double* bsrc = b;
    if (host) {
        FESPMV_CUDA(cudaMemcpyAsync(w->q, b, nb, cudaMemcpyHostToDevice, r.s));
        bsrc = w->q;
    }
    if (r.permute) {
        if ((rc = launch_gather(bsrc, r.A->d_perm, w->b, r.A->n, r.s))) return rc;
    } else {
        FESPMV_CUDA(cudaMemcpyAsync(w->b, bsrc, nb, cudaMemcpyDeviceToDevice, r.s));
    }
    if (x0) {
        const double* xsrc = x0;
        if (host) {
            FESPMV_CUDA(cudaMemcpyAsync(w->q, x0, nb, cudaMemcpyHostToDevice, r.s));
            xsrc = w->q;
        }
        if (r.permute) {
            if ((rc = launch_gather(xsrc, r.A->d_perm, w->x, r.A->n, r.s))) return rc;
        } else {
            FESPMV_CUDA(cudaMemcpyAsync(w->x, xsrc, nb, cudaMemcpyDeviceToDevice, r.s));
        }
    } else {
        FESPMV_CUDA(cudaMemsetAsync(w->x, 0, nb, r.s));
    }
    return FESPMV_OK;
}

static int cg_solve_impl(fespmv_mat* A, const double* b, double* x, const cg_options* opts,
                         cg_result* res, cudaStream_t s) {
    cg_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    int rc = normalize_options(o);
    if (rc) return rc;
    if ((rc = check_precision(A, o.precision))) return rc;
    if (res) std::memset(res, 0, sizeof(*res));
    if (A->n == 0) return FESPMV_OK;
    if ((rc = ensure_workspace(A))) return rc;
    CgRun r;
    r.A = A;
    r.w = A->cg;
    r.s = s;
    r.o = o;
    r.permute = A->format == FESPMV_FMT_SLICED && !(o.flags & FESPMV_IO_PERMUTED);
    r.has_x0 = o.flags & FESPMV_CG_X0;
    r.out_host = o.flags & FESPMV_IO_HOST;
    r.x_out = x;
    if ((rc = stage_inputs(r, b, r.has_x0 ? x : nullptr, r.out_host))) return rc;
    if ((rc = run_begin(r))) return rc;
    while (r.phase != PH_DONE) {
        bool progress;
        if ((rc = run_step(r, true, &progress))) return rc;
    }
    FESPMV_CUDA(cudaStreamSynchronize(s));
    return run_result(r, res);
}

// ------------------------------------------------------------------ allocation-free CSR solve
//
// cg_solve_csr_static serves callers that cannot allocate device memory: code
// running where cudaMalloc is forbidden or unavailable (inside a framework's
// own memory pool, a plugin that must not grow the process's device
// footprint, or a real-time loop that may not block on the allocator).  The
// caller passes the CSR matrix, b and x in device memory; the CG workspace
// (r, p, q, D^-1, partial sums, scalars) lives in the fixed array below, which
// every GPU that loads this library holds until the process exits.
constexpr int64_t kStaticMaxRows = int64_t(1) << 18;     // 262,144 rows
constexpr int64_t kStaticPartials = 3 * 32768 + 8;       // grid_sum storage for the largest grid
constexpr size_t kStaticVecBytes = sizeof(double) * kStaticMaxRows;
constexpr size_t kStaticBytes = 4 * kStaticVecBytes + sizeof(double) * kStaticPartials + 512;
static_assert(sizeof(CgScalars) <= 512, "the static scratch reserves 512 bytes for the scalars");

static __device__ __align__(256) unsigned char g_cg_static_scratch[kStaticBytes];

// Device address of the array for the current device, looked up on every call.
// The lookup is cheap once the module is loaded, and a cached address could go
// stale: a cudaDeviceReset (or any teardown of the primary context) loads the
// module again, and the array may then sit elsewhere.
static int static_scratch(void** out) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_cg_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_cg_static_scratch)");
    *out = ptr;
    return FESPMV_OK;
}

__global__ void cg_static_reset(CgScalars* sc, int max_iter) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        CgScalars z = {};
        z.max_iter = max_iter;
        z.status = CG_RUNNING;
        *sc = z;
    }
}

__global__ void csr_diag(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                         const double* __restrict__ val, double* __restrict__ diag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (col[p] == i) d += val[p];
        diag[i] = d;
    }
}

template <int L>
__global__ void csr_spmv_static(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ x,
                                double* __restrict__ y, int64_t n) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = t / L;
    const int sub = (int)(t % L);
    const double sum = csr_row_sum_f64<L>(row, sub, n, rowptr, col, val, x);
    if (row < n && sub == 0) y[row] = sum;
}

struct StaticCsr {
    int64_t n;
    const int64_t* rowptr;
    const int32_t* col;
    const double* val;
    int lanes;
    unsigned spmv_grid;
};

template <int L>
static void static_launch(const StaticCsr& m, bool dot, const double* x, double* y, double* partials,
                          CgScalars* sc, cudaStream_t s) {
    if (dot)
        cg_spmv_dot_csr<L><<<m.spmv_grid, 256, 0, s>>>(m.rowptr, m.col, m.val, x, y, m.n, partials, sc);
    else
        csr_spmv_static<L><<<m.spmv_grid, 256, 0, s>>>(m.rowptr, m.col, m.val, x, y, m.n);
}

static void static_spmv(const StaticCsr& m, bool dot, const double* x, double* y, double* partials,
                        CgScalars* sc, cudaStream_t s) {
    switch (m.lanes) {
        case 1: static_launch<1>(m, dot, x, y, partials, sc, s); break;
        case 2: static_launch<2>(m, dot, x, y, partials, sc, s); break;
        case 4: static_launch<4>(m, dot, x, y, partials, sc, s); break;
        case 8: static_launch<8>(m, dot, x, y, partials, sc, s); break;
        case 16: static_launch<16>(m, dot, x, y, partials, sc, s); break;
        default: static_launch<32>(m, dot, x, y, partials, sc, s); break;
    }
}

static int static_read(CgScalars* h, const CgScalars* sc, cudaStream_t s) {
    FESPMV_CUDA(cudaMemcpyAsync(h, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    FESPMV_CUDA(cudaStreamSynchronize(s));
    return FESPMV_OK;
}

static int cg_static_impl(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* values,
                          const double* b, double* x, int lanes, const cg_options* opts,
                          cg_result* res, cudaStream_t s) {
    cg_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.tol == 0.0) o.tol = 1e-10;
    if (o.max_iter == 0) o.max_iter = 100000;
    if (o.max_restarts == 0) o.max_restarts = 3;
    if (o.max_restarts < 0) o.max_restarts = 0;
    if (o.check_every == 0) o.check_every = 16;
    if (lanes == 0) lanes = 4;
    if (res) std::memset(res, 0, sizeof(*res));
    if (n < 0 || n > kStaticMaxRows) {
        set_error("cg_solve_csr_static handles at most %lld rows (got %lld)",
                  (long long)kStaticMaxRows, (long long)n);
        return FESPMV_ERR_INVALID_ARG;
    }
    if (!(o.tol > 0.0) || o.max_iter < 0 || o.check_every < 1 || o.precision != FESPMV_CG_F64 ||
        (o.flags & ~(FESPMV_CG_X0 | FESPMV_CG_NO_PRECOND)) ||
        !(lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32)) {
        set_error("bad options for cg_solve_csr_static");
        return FESPMV_ERR_INVALID_ARG;
    }
    if (n == 0) return FESPMV_OK;
    if (!rowptr || !colind || !values || !b || !x) {
        set_error("null argument");
        return FESPMV_ERR_INVALID_ARG;
    }
    void* base = nullptr;
    int rc = static_scratch(&base);
    if (rc) return rc;
    unsigned char* sp = static_cast<unsigned char*>(base);
    double* r = reinterpret_cast<double*>(sp);
    double* p = reinterpret_cast<double*>(sp + kStaticVecBytes);
    double* q = reinterpret_cast<double*>(sp + 2 * kStaticVecBytes);
    double* dinv = reinterpret_cast<double*>(sp + 3 * kStaticVecBytes);
    double* partials = reinterpret_cast<double*>(sp + 4 * kStaticVecBytes);
    CgScalars* sc = reinterpret_cast<CgScalars*>(sp + 4 * kStaticVecBytes + sizeof(double) * kStaticPartials);

    int dev = 0, sms = 0;
    FESPMV_CUDA(cudaGetDevice(&dev));
    FESPMV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned upd = std::max(1u, std::min(grid_for(n, 256), (unsigned)(sms * 8)));
    StaticCsr m{n, rowptr, colind, values, lanes, grid_for(n * lanes, 256)};
    if (grid_sum_doubles(m.spmv_grid) > kStaticPartials || grid_sum_doubles(upd) > kStaticPartials) {
        set_error("grid too large for the static partial-sum buffer");
        return FESPMV_ERR_UNSUPPORTED;
    }

    // every call starts from cleared scalars; vectors are fully written before use
    cg_static_reset<<<1, 32, 0, s>>>(sc, o.max_iter);
    csr_diag<<<upd, 256, 0, s>>>(n, rowptr, colind, values, q);
    cg_dinv<<<upd, 256, 0, s>>>(n, q, dinv, (o.flags & FESPMV_CG_NO_PRECOND) ? 0 : 1, sc);
    const bool has_x0 = o.flags & FESPMV_CG_X0;
    if (!has_x0) FESPMV_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, s));
    FESPMV_CUDA(cudaGetLastError());

    const double tol2 = o.tol * o.tol;
    CgScalars h;
    int restarts = 0;
    bool need_ax = has_x0;
    int status = CG_RUNNING;
    for (;;) {
        if (need_ax) static_spmv(m, false, x, q, partials, sc, s);
        cg_init<<<upd, 256, 0, s>>>(n, b, need_ax ? q : nullptr, r, p, dinv, tol2, partials, sc, nullptr);
        FESPMV_CUDA(cudaGetLastError());
        if ((rc = static_read(&h, sc, s))) return rc;
        if (h.status == CG_BADDIAG) {
            set_error("Jacobi preconditioning needs a positive, finite diagonal");
            if (res) res->status = FESPMV_ERR_BREAKDOWN;
            return FESPMV_ERR_BREAKDOWN;
        }
        if (h.bb == 0.0) {
            FESPMV_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, s));
            FESPMV_CUDA(cudaStreamSynchronize(s));
            h.true_rr = 0.0;
            status = CG_CONVERGED;
            break;
        }
        while (h.status == CG_RUNNING) {
            for (int k = 0; k < o.check_every; ++k) {
                static_spmv(m, true, p, q, partials, sc, s);
                cg_update<<<upd, 256, 0, s>>>(n, x, r, p, q, dinv, partials, sc);
                cg_pupdate<<<upd, 256, 0, s>>>(n, p, r, dinv, nullptr, sc);
            }
            FESPMV_CUDA(cudaGetLastError());
            if ((rc = static_read(&h, sc, s))) return rc;
        }
        static_spmv(m, false, x, q, partials, sc, s);
        cg_true_residual<<<upd, 256, 0, s>>>(n, b, q, partials, sc);
        FESPMV_CUDA(cudaGetLastError());
        if ((rc = static_read(&h, sc, s))) return rc;
        status = h.status;
        if (status == CG_CONVERGED && !(h.true_rr <= h.thresh2)) {
            if (restarts < o.max_restarts && h.iters < o.max_iter) {
                ++restarts;
                need_ax = true;
                continue;
            }
            status = CG_MAXITER;
        }
        break;
    }
    const int out = status == CG_CONVERGED ? FESPMV_OK
                  : status == CG_BREAKDOWN ? FESPMV_ERR_BREAKDOWN : FESPMV_ERR_NOT_CONVERGED;
    if (res) {
        res->status = out;
        res->iters = h.iters;
        res->restarts = restarts;
        res->relres = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
        res->true_relres = h.bb > 0 ? std::sqrt(h.true_rr / h.bb) : 0.0;
    }
    if (out == FESPMV_ERR_BREAKDOWN) set_error("CG breakdown (p.Ap <= 0 or a non-finite scalar)");
    if (out == FESPMV_ERR_NOT_CONVERGED) set_error("CG stopped above the tolerance");
    return out;
}

}  // namespace fespmv

extern "C" int cg_solve(fespmv_mat_t A, const double* b, double* x, const cg_options* opts,
                        cg_result* res, fespmv_stream_t stream) {
    try {
        if (!A || (A->n > 0 && (!b || !x))) {
            fespmv::set_error("null argument");
            return FESPMV_ERR_INVALID_ARG;
        }
        return fespmv::cg_solve_impl(A, b, x, opts, res, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        fespmv::set_error("host allocation failed");
        return FESPMV_ERR_OOM;
    } catch (...) {
        fespmv::set_error("unexpected C++ exception");
        return FESPMV_ERR_INVALID_ARG;
    }
}

extern "C" int cg_solve_csr_static(int64_t n_rows, const int64_t* rowptr, const int32_t* colind,
                                   const double* values, const double* b, double* x,
                                   int32_t csr_lanes, const cg_options* opts, cg_result* res,
                                   fespmv_stream_t stream) {
    try {
        return fespmv::cg_static_impl(n_rows, rowptr, colind, values, b, x, csr_lanes, opts, res,
                                      (cudaStream_t)stream);
    } catch (...) {
        fespmv::set_error("unexpected C++ exception");
        return FESPMV_ERR_INVALID_ARG;
    }
}
