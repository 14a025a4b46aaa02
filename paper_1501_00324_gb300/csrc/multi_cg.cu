// Conjugate gradients for many right-hand sides of one matrix (cg_solve_multi in
// fespmv.h): k <= 32 independent Jacobi-PCG solves A x_j = b_j (the solver of
// the paper's Newton step, Sec. 2.1, once per column) run in lockstep, so that
// every iteration streams the matrix once for all of them.  The same lockstep
// solve, with columns filled and emptied while it runs, serves the solve
// server's groups (multi_group.h).
//
// The solves share nothing but the product: each column has its own scalars
// (alpha, beta, rho, thresholds, status), the vectors are row-major n x kw blocks
// in the handle's numbering (kw = k padded to 4, 8, 16 or 32; the padding
// columns are zero right-hand sides, converged from the start), and each
// column's dot products are reduced in a fixed order that does not depend on
// the other columns.  So a column's iterates -- and its x -- are bitwise the
// same whatever the other columns hold, for a given width kw.
//
// One inner iteration is five launches, captured check_every times in one CUDA
// graph: the product Q = B P with the per-column sums of p.q fused in (multi.cu),
// the alpha of each column, the update w += alpha p, r -= alpha q with the sums
// of r.r (and r.z), the beta of each column, and p = z + beta p.  Columns that
// have stopped are skipped by the updates (their vectors stay as they were).
//
// Around the inner iteration sits the FP64 outer step of cg_solve: r = b - A x
// in FP64 (the multi-RHS FP64 product), per-column convergence test, and then
// either iterative refinement with an FP32 inner CG on B = S A S (restarted, or
// reliable updates that keep p), or for FESPMV_CG_F64 the FP64 inner CG on A
// itself with Jacobi z = D^-1 r, whose true-residual checks are the restarts.
//
// In lockstep the columns reach their refinement points at different
// iterations.  A column whose inner residual has fallen by inner_tol is marked
// due and keeps iterating (until it has fallen by inner_tol^3 with reliable
// updates, inner_tol^2 without: further the float recurrence drifts from the
// true residual); outer steps come every kOuterChunks graph launches (or at once
// when no column is iterating) and act only on the columns that are due or whose
// inner CG has stopped.  No column waits for the others, and the grid of outer
// steps is fixed, so the independence above still holds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <type_traits>

#include "cg_run.h"
#include "internal.h"
#include "multi_group.h"

namespace fespmv {

struct MScal {
    double rho, alpha, beta, rr_in, thresh_in, thresh_due, rr, bb, thresh2, prev;
    double tol2, in2;   // this column's tol^2 and inner_tol^2
    int iters, iters_in, status_in, status_out, outer, max_iter, max_outer;
    int due;    // the inner residual has fallen by inner_tol: replace it at the next outer step
    int act;    // this outer step acts on the column: 1 its inner CG has stopped, 2 it is due
                // and still iterating (its p already follows the last residual), 3 it is new
                // (x = x0, nothing to fold in), 0 none of these
    int fresh;  // set for a column whose first outer step is still to come
};

struct MultiWork {
    int kw = 0;                                  // allocated width
    double *x = nullptr, *b = nullptr, *q64 = nullptr, *dinv = nullptr;
    void *w = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;  // inner vectors (float or double)
    double* part = nullptr;
    int64_t part_len = 0;
    MScal* sc = nullptr;
    MScal* h_sc = nullptr;                       // pinned mirror
    float2* pdf = nullptr;                       // p as float pairs (FESPMV_PREC_DF64 handles)
    int64_t bytes = 0;                           // device bytes held
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    int g_kw = 0, g_f64 = -1, g_pre = -1, g_chunk = 0;
};

namespace {

constexpr int kUpdBlock = 256;
constexpr int kOuterChunks = 8;   // graph launches between outer steps

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Column c of the partial sums part[b * stride + c], b < nb, summed by one block
// in a fixed order (valid in thread 0).
__device__ double column_sum(const double* __restrict__ part, int64_t nb, int stride, int c) {
    __shared__ double sh[32];
    double t = 0.0;
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) t += part[b * stride + c];
    t = warp_sum_d(t);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[warp] = t;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        r = warp_sum_d(r);
    }
    __syncthreads();
    return r;
}

// Four consecutive entries of a row-major block (16 or 32 bytes, aligned).
template <typename T> struct Quad;
template <> struct Quad<float> {
    static __device__ __forceinline__ void load(const float* p, float (&v)[4]) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    static __device__ __forceinline__ void store(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Quad<double> {
    static __device__ __forceinline__ void load(const double* p, double (&v)[4]) {
        const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void store(double* p, const double (&v)[4]) {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
};

// Per-column sums of NQ quantities over a block: s[k][j] of each thread (its 4
// columns 4 qd + j, qd = thread % (KW/4)) summed over the warp's lanes of equal qd,
// then over the warps in order; written to part[(k * nb + block) * KW + c].
template <int KW, int NQ>
__device__ __forceinline__ void block_columns(double (&s)[NQ][4], double* __restrict__ part, int64_t nb) {
    constexpr int LPG = KW / 4;
    constexpr int NW = kUpdBlock / 32;
    __shared__ double sh[NQ][NW][KW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = LPG; o < 32; o <<= 1)
#pragma unroll
        for (int k = 0; k < NQ; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) s[k][j] += __shfl_xor_sync(0xffffffffu, s[k][j], o);
    if (lane < LPG)
#pragma unroll
        for (int k = 0; k < NQ; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) sh[k][warp][4 * lane + j] = s[k][j];
    __syncthreads();
    if (threadIdx.x < KW)
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) t += sh[k][w][threadIdx.x];
            part[((int64_t)k * nb + blockIdx.x) * KW + threadIdx.x] = t;
        }
}

// ------------------------------------------------------------------ inner iteration

__global__ void mc_finalize_pq(const double* __restrict__ part, int64_t nb, int kw, MScal* sc) {
    const int c = blockIdx.x;
    if (sc[c].status_in != CG_RUNNING) return;
    const double pq = column_sum(part, nb, kw, c);
    if (threadIdx.x == 0) {
        MScal& s = sc[c];
        if (!(pq > 0.0) || !isfinite(pq)) s.status_in = CG_BREAKDOWN;
        else s.alpha = s.rho / pq;
    }
}

// w += alpha p, r -= alpha q for the running columns; sums of r.r and (PRE) r.z,
// z = dinv r.
template <typename T, int KW, bool PRE>
__global__ void __launch_bounds__(kUpdBlock) mc_update(int64_t n, T* __restrict__ w, T* __restrict__ r,
                                                       const T* __restrict__ p, const T* __restrict__ q,
                                                       const double* __restrict__ dinv,
                                                       double* __restrict__ part, const MScal* __restrict__ sc) {
    constexpr int LPG = KW / 4, NQ = PRE ? 2 : 1;
    __shared__ double s_alpha[KW];
    __shared__ int s_run[KW];
    if (threadIdx.x < KW) {
        s_alpha[threadIdx.x] = sc[threadIdx.x].alpha;
        s_run[threadIdx.x] = sc[threadIdx.x].status_in == CG_RUNNING;
    }
    __syncthreads();
    const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int qd = (int)(first % LPG);   // the stride is a multiple of LPG: fixed per thread
    T a[4];
    bool run[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        a[j] = (T)s_alpha[4 * qd + j];
        run[j] = s_run[4 * qd + j] != 0;
    }
    double s[NQ][4] = {};
    const bool any = run[0] || run[1] || run[2] || run[3];
    if (any) {
        for (int64_t t = first; t < n * LPG; t += (int64_t)gridDim.x * blockDim.x) {
            const int64_t row = t / LPG, o = row * KW + 4 * qd;
            T pv[4], qv[4], wv[4], rv[4];
            Quad<T>::load(p + o, pv);
            Quad<T>::load(q + o, qv);
            Quad<T>::load(w + o, wv);
            Quad<T>::load(r + o, rv);
            const double di = PRE ? dinv[row] : 1.0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (run[j]) {
                    wv[j] = fma(a[j], pv[j], wv[j]);
                    rv[j] = fma(-a[j], qv[j], rv[j]);
                    const double rd = (double)rv[j];
                    s[0][j] = fma(rd, rd, s[0][j]);
                    if constexpr (PRE) s[NQ - 1][j] = fma(rd, di * rd, s[NQ - 1][j]);
                }
            }
            Quad<T>::store(w + o, wv);
            Quad<T>::store(r + o, rv);
        }
    }
    const int64_t nb = gridDim.x;
    block_columns<KW, NQ>(s, part, nb);
}

// rr -> convergence test, beta and rho; rz (r.z) is the preconditioned product
// (the same sums as rr without preconditioning).
__global__ void mc_finalize_rr(const double* __restrict__ part, int64_t nb, int kw, int pre, MScal* sc) {
    const int c = blockIdx.x;
    if (sc[c].status_in != CG_RUNNING) return;
    const double rr = column_sum(part, nb, kw, c);
    const double rz = pre ? column_sum(part + nb * kw, nb, kw, c) : rr;
    if (threadIdx.x == 0) {
        MScal& s = sc[c];
        s.iters += 1;
        s.iters_in += 1;
        s.rr_in = rr;
        if (!isfinite(rr) || !isfinite(rz)) s.status_in = CG_BREAKDOWN;
        else if (rr <= s.thresh_in) s.status_in = CG_CONVERGED;   // tol reached (estimate): stop
        else if (s.iters >= s.max_iter) s.status_in = CG_MAXITER;
        else {
            if (rr <= s.thresh_due) s.due = 1;   // keeps iterating until the outer step
            s.beta = rz / s.rho;
            s.rho = rz;
        }
    }
}

// p = z + beta p (z = dinv r with PRE, else r) for the running columns (ACT: only
// those whose inner CG had stopped when the outer step acted on them).
template <typename T, int KW, bool PRE, bool ACT>
__global__ void __launch_bounds__(kUpdBlock) mc_pupdate(int64_t n, T* __restrict__ p, const T* __restrict__ r,
                                                        const double* __restrict__ dinv,
                                                        const MScal* __restrict__ sc) {
    constexpr int LPG = KW / 4;
    __shared__ double s_beta[KW];
    __shared__ int s_run[KW];
    if (threadIdx.x < KW) {
        s_beta[threadIdx.x] = sc[threadIdx.x].beta;
        s_run[threadIdx.x] = sc[threadIdx.x].status_in == CG_RUNNING && (!ACT || sc[threadIdx.x].act == 1);
    }
    __syncthreads();
    const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int qd = (int)(first % LPG);
    T bt[4];
    bool run[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        bt[j] = (T)s_beta[4 * qd + j];
        run[j] = s_run[4 * qd + j] != 0;
    }
    if (!(run[0] || run[1] || run[2] || run[3])) return;
    for (int64_t t = first; t < n * LPG; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / LPG, o = row * KW + 4 * qd;
        T pv[4], rv[4];
        Quad<T>::load(p + o, pv);
        Quad<T>::load(r + o, rv);
        const T di = PRE ? (T)dinv[row] : T(1);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (run[j]) pv[j] = fma(bt[j], pv[j], PRE ? di * rv[j] : rv[j]);
        Quad<T>::store(p + o, pv);
    }
}

// ------------------------------------------------------------------ outer step

// dinv = 1/diag (Jacobi) or 1; a non-positive or non-finite diagonal sets *bad.
__global__ void mc_dinv(int64_t n, const double* __restrict__ diag, double* __restrict__ dinv, int jacobi,
                        int* bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = diag[i];
        if (!jacobi) {
            dinv[i] = 1.0;
        } else if (d > 0.0 && isfinite(d)) {
            dinv[i] = 1.0 / d;
        } else {
            dinv[i] = 0.0;
            *bad = 1;
        }
    }
}

// For the columns the outer step acts on: r = b - Ax (Ax = q64, or 0 when q64 is null);
// the inner right-hand side r_in = float(S r) (refinement, T = float) or r itself
// (T = double); w = 0; p = dinv r_in (dinv = 1 without PRE), unless reliable
// updates keep p after the first step.  Sums per column: r.r, r_in.r_in, b.b and
// r_in.(dinv r_in).
template <typename T, int KW, bool PRE>
__global__ void __launch_bounds__(kUpdBlock) mc_residual(int64_t n, const double* __restrict__ b,
                                                         const double* __restrict__ q64,
                                                         const double* __restrict__ scale,
                                                         const double* __restrict__ dinv, T* __restrict__ w,
                                                         T* __restrict__ r, T* __restrict__ p, int reliable,
                                                         double* __restrict__ part, const MScal* __restrict__ sc) {
    constexpr int LPG = KW / 4;
    constexpr bool SCALED = std::is_same<T, float>::value;   // refinement: B = S A S
    __shared__ int s_run[KW], s_keep[KW];
    if (threadIdx.x < KW) {
        const MScal& c = sc[threadIdx.x];
        s_run[threadIdx.x] = c.act != 0;
        // reliable updates keep p; a column caught while iterating already holds
        // p = r + beta p_old, which becomes r_new + beta p_old by adding r_new - r
        s_keep[threadIdx.x] = reliable && c.outer > 0 ? c.act : 0;
    }
    __syncthreads();
    const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int qd = (int)(first % LPG);
    bool run[4];
    int keep[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        run[j] = s_run[4 * qd + j] != 0;
        keep[j] = s_keep[4 * qd + j];
    }
    double s[4][4] = {};
    if (run[0] || run[1] || run[2] || run[3]) {
        for (int64_t t = first; t < n * LPG; t += (int64_t)gridDim.x * blockDim.x) {
            const int64_t row = t / LPG, o = row * KW + 4 * qd;
            double bv[4], qv[4] = {0.0, 0.0, 0.0, 0.0};
            T wv[4], rv[4], pv[4];
            Quad<double>::load(b + o, bv);
            if (q64) Quad<double>::load(q64 + o, qv);
            Quad<T>::load(w + o, wv);
            Quad<T>::load(r + o, rv);
            Quad<T>::load(p + o, pv);
            const double sc_i = SCALED ? scale[row] : 1.0;
            const double di = PRE ? dinv[row] : 1.0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (run[j]) {
                    const double ri = bv[j] - qv[j];
                    const T rin = (T)(sc_i * ri);
                    wv[j] = T(0);
                    if (keep[j] == 2) pv[j] += rin - rv[j];
                    else if (!keep[j]) pv[j] = PRE ? (T)(di * (double)rin) : rin;
                    rv[j] = rin;
                    const double rd = (double)rin;
                    s[0][j] = fma(ri, ri, s[0][j]);
                    s[1][j] = fma(rd, rd, s[1][j]);
                    s[2][j] = fma(bv[j], bv[j], s[2][j]);
                    s[3][j] = fma(rd, di * rd, s[3][j]);
                }
            }
            Quad<T>::store(w + o, wv);
            Quad<T>::store(r + o, rv);
            Quad<T>::store(p + o, pv);
        }
    }
    block_columns<KW, 4>(s, part, gridDim.x);
}

// Per column acted on: the FP64 convergence test and the start of the next inner
// phase.  Refinement: due when the inner residual has fallen by inner_tol, stopped
// when it estimates ||b - A x|| <= tol ||b|| (||r|| ~ ||r_in|| ||r|| / ||S r|| at
// this step).  FP64 (f64): the inner CG runs to tol ||b|| on its own recurrence;
// rho = r.z.
__global__ void mc_finalize_res(const double* __restrict__ part, int64_t nb, int kw, MScal* sc, int reliable,
                                int f64) {
    const int c = blockIdx.x;
    if (!sc[c].act) return;
    const double rr = column_sum(part, nb, kw, c);
    const double rhs2 = column_sum(part + nb * kw, nb, kw, c);
    const double bb = column_sum(part + 2 * nb * kw, nb, kw, c);
    const double rz = column_sum(part + 3 * nb * kw, nb, kw, c);
    if (threadIdx.x == 0) {
        MScal& s = sc[c];
        const double tol2 = s.tol2, in2 = s.in2;
        s.rr = rr;
        s.bb = bb;
        s.thresh2 = tol2 * bb;
        s.due = 0;
        s.fresh = 0;
        s.status_in = CG_CONVERGED;    // idle unless another inner phase starts below
        if (!isfinite(rr) || !isfinite(rhs2) || !isfinite(rz)) s.status_out = CG_BREAKDOWN;
        else if (rr <= s.thresh2) s.status_out = CG_CONVERGED;
        else if (s.outer >= s.max_outer) s.status_out = CG_MAXITER;
        else if (s.iters >= s.max_iter) s.status_out = CG_MAXITER;
        else if (!(rr < s.prev)) s.status_out = CG_MAXITER;   // stagnation
        else {
            s.prev = rr;
            s.iters_in = 0;
            if (f64) {
                s.thresh_in = tol2 * bb;
                s.thresh_due = -1.0;
                s.rho = rz;
            } else {
                // reliable updates replace the residual and keep p (p = r_in + beta p follows
                // for a column whose inner CG had stopped); restarted refinement starts again
                // from p = r_in.  A due column iterates on until the next outer step unless
                // its residual falls by inner_tol^3 (reliable) or inner_tol^2 (restarted)
                // first, or it estimates ||b - A x|| <= tol ||b||.
                if (reliable) s.beta = (s.outer > 0 && s.act == 1) ? rhs2 / s.rho : 0.0;
                s.thresh_due = in2 * rhs2;
                s.thresh_in = fmax((reliable ? in2 * in2 * in2 : in2 * in2) * rhs2,
                                   rr > 0.0 ? tol2 * bb * rhs2 / rr : 0.0);
                s.rho = rhs2;
            }
            if (!(s.rho > 0.0)) s.status_out = CG_BREAKDOWN;   // z.r <= 0: D or A not positive
            else s.status_in = CG_RUNNING;
        }
    }
}

// x += S w (refinement) or x += w (FP64) for the columns the outer step acts on
// (not the new ones: their w is another column's leftover).
template <typename T, int KW>
__global__ void __launch_bounds__(kUpdBlock) mc_xupdate(int64_t n, double* __restrict__ x,
                                                        const double* __restrict__ scale, const T* __restrict__ w,
                                                        const MScal* __restrict__ sc) {
    constexpr int LPG = KW / 4;
    __shared__ int s_run[KW];
    if (threadIdx.x < KW) s_run[threadIdx.x] = sc[threadIdx.x].act == 1 || sc[threadIdx.x].act == 2;
    __syncthreads();
    const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int qd = (int)(first % LPG);
    bool run[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) run[j] = s_run[4 * qd + j] != 0;
    if (!(run[0] || run[1] || run[2] || run[3])) return;
    for (int64_t t = first; t < n * LPG; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / LPG, o = row * KW + 4 * qd;
        double xv[4];
        T wv[4];
        Quad<double>::load(x + o, xv);
        Quad<T>::load(w + o, wv);
        const double sc_i = scale ? scale[row] : 1.0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (run[j]) xv[j] = fma(sc_i, (double)wv[j], xv[j]);
        Quad<double>::store(x + o, xv);
    }
}

// The columns this outer step acts on; the finished inner phases are counted.
__global__ void mc_mark_act(int kw, MScal* sc) {
    const int c = threadIdx.x;
    if (c < kw) {
        MScal& s = sc[c];
        s.act = s.status_out != CG_RUNNING ? 0 : s.fresh ? 3 : s.status_in != CG_RUNNING ? 1 : s.due ? 2 : 0;
        if (s.act == 1 || s.act == 2) s.outer += 1;
    }
}

// ------------------------------------------------------------------ host side

struct Shape {
    int kw;
    bool f64, pre;
};

template <typename T, int KW, bool PRE>
static void inner_kw(const fespmv_mat* A, MultiWork* w, unsigned dot_grid, unsigned upd_grid, cudaStream_t s) {
    T* wv = static_cast<T*>(w->w);
    T* rv = static_cast<T*>(w->r);
    T* pv = static_cast<T*>(w->p);
    T* qv = static_cast<T*>(w->q);
    if constexpr (std::is_same<T, double>::value) {
        // FP64 products as float pairs on handles that keep them (the FP32 pipe)
        if (w->pdf) launch_multi_dot_pairs(A, pv, qv, w->pdf, KW, w->part, s);
        else launch_multi_dot(A, pv, qv, KW, true, w->part, s);
    } else {
        launch_multi_dot(A, pv, qv, KW, false, w->part, s);
    }
    mc_finalize_pq<<<KW, 256, 0, s>>>(w->part, dot_grid, KW, w->sc);
    mc_update<T, KW, PRE><<<upd_grid, kUpdBlock, 0, s>>>(A->n, wv, rv, pv, qv, w->dinv, w->part, w->sc);
    mc_finalize_rr<<<KW, 256, 0, s>>>(w->part, upd_grid, KW, PRE ? 1 : 0, w->sc);
    mc_pupdate<T, KW, PRE, false><<<upd_grid, kUpdBlock, 0, s>>>(A->n, pv, rv, w->dinv, w->sc);
}

template <typename T, bool PRE>
static void inner_t(const fespmv_mat* A, MultiWork* w, int kw, unsigned dot_grid, unsigned upd_grid,
                    cudaStream_t s) {
    switch (kw) {
        case 4: inner_kw<T, 4, PRE>(A, w, dot_grid, upd_grid, s); break;
        case 8: inner_kw<T, 8, PRE>(A, w, dot_grid, upd_grid, s); break;
        case 16: inner_kw<T, 16, PRE>(A, w, dot_grid, upd_grid, s); break;
        default: inner_kw<T, 32, PRE>(A, w, dot_grid, upd_grid, s); break;
    }
}

static void launch_inner(const fespmv_mat* A, MultiWork* w, Shape sh, unsigned dot_grid, unsigned upd_grid,
                         cudaStream_t s) {
    if (sh.f64) {
        if (sh.pre) inner_t<double, true>(A, w, sh.kw, dot_grid, upd_grid, s);
        else inner_t<double, false>(A, w, sh.kw, dot_grid, upd_grid, s);
    } else {
        inner_t<float, false>(A, w, sh.kw, dot_grid, upd_grid, s);
    }
}

template <typename T, int KW, bool PRE>
static void residual_kw(const fespmv_mat* A, MultiWork* w, bool ax, int reliable, unsigned upd_grid,
                        cudaStream_t s) {
    mc_residual<T, KW, PRE><<<upd_grid, kUpdBlock, 0, s>>>(
        A->n, w->b, ax ? w->q64 : nullptr, A->d_scale, w->dinv, static_cast<T*>(w->w), static_cast<T*>(w->r),
        static_cast<T*>(w->p), reliable, w->part, w->sc);
}

template <typename T, int KW>
static void xupdate_kw(const fespmv_mat* A, MultiWork* w, bool scaled, unsigned upd_grid, cudaStream_t s) {
    mc_xupdate<T, KW><<<upd_grid, kUpdBlock, 0, s>>>(A->n, w->x, scaled ? A->d_scale : nullptr,
                                                     static_cast<const T*>(w->w), w->sc);
}

template <typename T, bool PRE>
static void outer_t(const fespmv_mat* A, MultiWork* w, int kw, bool ax, int reliable, unsigned upd_grid,
                    cudaStream_t s) {
    switch (kw) {
        case 4: residual_kw<T, 4, PRE>(A, w, ax, reliable, upd_grid, s); break;
        case 8: residual_kw<T, 8, PRE>(A, w, ax, reliable, upd_grid, s); break;
        case 16: residual_kw<T, 16, PRE>(A, w, ax, reliable, upd_grid, s); break;
        default: residual_kw<T, 32, PRE>(A, w, ax, reliable, upd_grid, s); break;
    }
}

template <typename T>
static void xupdate_t(const fespmv_mat* A, MultiWork* w, int kw, bool scaled, unsigned upd_grid, cudaStream_t s) {
    switch (kw) {
        case 4: xupdate_kw<T, 4>(A, w, scaled, upd_grid, s); break;
        case 8: xupdate_kw<T, 8>(A, w, scaled, upd_grid, s); break;
        case 16: xupdate_kw<T, 16>(A, w, scaled, upd_grid, s); break;
        default: xupdate_kw<T, 32>(A, w, scaled, upd_grid, s); break;
    }
}

// p = r_in + beta p after a residual replacement (reliable updates), acted-on columns.
static void replaced_pupdate(const fespmv_mat* A, MultiWork* w, int kw, unsigned upd_grid, cudaStream_t s) {
    float* p = static_cast<float*>(w->p);
    const float* r = static_cast<const float*>(w->r);
    switch (kw) {
        case 4: mc_pupdate<float, 4, false, true><<<upd_grid, kUpdBlock, 0, s>>>(A->n, p, r, w->dinv, w->sc); break;
        case 8: mc_pupdate<float, 8, false, true><<<upd_grid, kUpdBlock, 0, s>>>(A->n, p, r, w->dinv, w->sc); break;
        case 16: mc_pupdate<float, 16, false, true><<<upd_grid, kUpdBlock, 0, s>>>(A->n, p, r, w->dinv, w->sc); break;
        default: mc_pupdate<float, 32, false, true><<<upd_grid, kUpdBlock, 0, s>>>(A->n, p, r, w->dinv, w->sc); break;
    }
}

static unsigned update_grid(int64_t n, int kw) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t quads = n * (kw / 4);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 4, (quads + kUpdBlock - 1) / kUpdBlock));
}

static void destroy_multi_work(MultiWork* w) {
    if (!w) return;
    if (w->graph) cudaGraphExecDestroy(w->graph);
    if (w->cap) cudaStreamDestroy(w->cap);
    void* ptrs[] = {w->x, w->b, w->q64, w->dinv, w->w, w->r, w->p, w->q, w->part, w->sc, w->pdf};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (w->h_sc) cudaFreeHost(w->h_sc);
    delete w;
}

static int mw_alloc(MultiWork* w, void** p, size_t bytes, const char* what) {
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

// Grid of the FP64 inner product: float pairs on handles that keep them.
static unsigned dot_grid_of(const fespmv_mat* A, int kw, bool f64) {
    if (f64 && A->d_vdf) return launch_multi_dot_pairs(A, nullptr, nullptr, nullptr, kw, nullptr, nullptr);
    return launch_multi_dot(A, nullptr, nullptr, kw, f64, nullptr, nullptr);
}

// Partial sums for either precision's grids at width kw.
static int64_t multi_part_len(const fespmv_mat* A, int kw) {
    const unsigned g32 = dot_grid_of(A, kw, false);
    const unsigned g64 = dot_grid_of(A, kw, true);
    return (int64_t)std::max({g32, g64, 4 * update_grid(A->n, kw)}) * kw;
}

// Workspace of a lockstep solve of width kw: x, b, A x (FP64) and w, r, p, q (8-byte
// entries, used as float by the refinement), n x kw each; 1/diag; partial sums;
// per-column scalars (device and pinned host); a stream for graph capture.
static int create_multi_work(const fespmv_mat* A, int kw, MultiWork** out) {
    *out = nullptr;
    MultiWork* w = new MultiWork();
    const size_t bytes = sizeof(double) * (size_t)A->n * kw;
    const int64_t pl = multi_part_len(A, kw);
    int rc;
    if ((rc = mw_alloc(w, (void**)&w->x, bytes, "multi-RHS x")) ||
        (rc = mw_alloc(w, (void**)&w->b, bytes, "multi-RHS b")) ||
        (rc = mw_alloc(w, (void**)&w->q64, bytes, "multi-RHS A x")) ||
        (rc = mw_alloc(w, &w->w, bytes, "multi-RHS w")) || (rc = mw_alloc(w, &w->r, bytes, "multi-RHS r")) ||
        (rc = mw_alloc(w, &w->p, bytes, "multi-RHS p")) || (rc = mw_alloc(w, &w->q, bytes, "multi-RHS q")) ||
        (rc = mw_alloc(w, (void**)&w->dinv, sizeof(double) * (size_t)A->n, "multi-RHS dinv")) ||
        (rc = mw_alloc(w, (void**)&w->part, sizeof(double) * (size_t)pl, "multi-RHS partial sums")) ||
        (rc = mw_alloc(w, (void**)&w->sc, sizeof(MScal) * 32, "multi-RHS scalars")) ||
        (A->d_vdf && (rc = mw_alloc(w, (void**)&w->pdf, sizeof(float2) * (size_t)A->n * kw, "multi-RHS p pairs")))) {
        destroy_multi_work(w);
        return rc;
    }
    cudaError_t e = cudaMallocHost((void**)&w->h_sc, sizeof(MScal) * 32);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        destroy_multi_work(w);
        return cuda_fail(e, "multi-RHS workspace");
    }
    w->kw = kw;
    w->part_len = pl;
    *out = w;
    return FESPMV_OK;
}

// The handle's own workspace (cg_solve_multi), grown to width kw.
static int ensure_handle_work(fespmv_mat* A, int kw) {
    if (A->mcg && A->mcg->kw >= kw) return FESPMV_OK;
    if (A->mcg) {
        A->device_bytes -= A->mcg->bytes;
        destroy_multi_work(A->mcg);
        A->mcg = nullptr;
    }
    MultiWork* w = nullptr;
    int rc = create_multi_work(A, kw, &w);
    if (rc) return rc;
    A->mcg = w;
    A->device_bytes += w->bytes;
    return FESPMV_OK;
}

static int multi_graph(const fespmv_mat* A, MultiWork* w, Shape sh, int chunk, unsigned dot_grid,
                       unsigned upd_grid) {
    if (w->graph && w->g_kw == sh.kw && w->g_f64 == (int)sh.f64 && w->g_pre == (int)sh.pre && w->g_chunk == chunk)
        return FESPMV_OK;
    if (w->graph) {
        cudaGraphExecDestroy(w->graph);
        w->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    FESPMV_CUDA(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk; ++i) launch_inner(A, w, sh, dot_grid, upd_grid, w->cap);
    cudaError_t e = cudaStreamEndCapture(w->cap, &g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&w->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    w->g_kw = sh.kw;
    w->g_f64 = sh.f64;
    w->g_pre = sh.pre;
    w->g_chunk = chunk;
    return FESPMV_OK;
}

static int read_scalars(MultiWork* w, int kw, cudaStream_t s) {
    FESPMV_CUDA(cudaMemcpyAsync(w->h_sc, w->sc, sizeof(MScal) * kw, cudaMemcpyDeviceToHost, s));
    FESPMV_CUDA(cudaStreamSynchronize(s));
    return FESPMV_OK;
}

// 1/diag (Jacobi of the FP64 solve; 1 with NO_PRECOND) and the check of diag(A) > 0
// that Jacobi and S = D^-1/2 need.  Returns FESPMV_ERR_BREAKDOWN for a bad diagonal.
static int prepare_diag(const fespmv_mat* A, MultiWork* w, Shape sh, cudaStream_t s) {
    int* bad = reinterpret_cast<int*>(w->part);   // scratch: the partial sums are rewritten later
    FESPMV_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    mc_dinv<<<grid_for(A->n, 256), 256, 0, s>>>(A->n, A->d_diag, w->dinv, (!sh.f64 || sh.pre) ? 1 : 0, bad);
    FESPMV_CUDA(cudaGetLastError());
    int h_bad = 0;
    FESPMV_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    FESPMV_CUDA(cudaStreamSynchronize(s));
    if (h_bad) {
        set_error("the diagonal has a non-positive or non-finite entry");
        return FESPMV_ERR_BREAKDOWN;
    }
    return FESPMV_OK;
}

// Scalars of a column before its first outer step.
static MScal new_column(const cg_options& o, bool f64) {
    MScal z;
    std::memset(&z, 0, sizeof(z));
    z.status_out = CG_RUNNING;
    z.status_in = CG_CONVERGED;
    z.fresh = 1;
    z.prev = INFINITY;
    z.tol2 = o.tol * o.tol;
    z.in2 = o.inner_tol * o.inner_tol;
    z.max_iter = o.max_iter;
    z.max_outer = f64 ? o.max_restarts + 1 : o.max_outer;   // FP64: the first solve and its restarts
    return z;
}

static cg_result column_result(const MScal& h, bool f64) {
    cg_result r;
    std::memset(&r, 0, sizeof(r));
    r.status = h.status_out == CG_CONVERGED ? FESPMV_OK
             : h.status_out == CG_BREAKDOWN ? FESPMV_ERR_BREAKDOWN : FESPMV_ERR_NOT_CONVERGED;
    r.iters = h.iters;
    r.restarts = f64 ? std::max(h.outer - 1, 0) : 0;
    r.outer = f64 ? 0 : h.outer;
    r.relres = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
    r.true_relres = r.relres;
    return r;
}

// One outer step for the columns it acts on (see mc_mark_act): fold the inner
// corrections into x, r = b - A x in FP64 (ax: A x computed; else x = 0), the
// convergence tests and the start of the next inner phases.
static int enqueue_outer(fespmv_mat* A, MultiWork* w, Shape sh, int reliable, bool ax, unsigned upd_grid,
                         cudaStream_t s) {
    const int kw = sh.kw;
    mc_mark_act<<<1, 32, 0, s>>>(kw, w->sc);
    if (sh.f64) xupdate_t<double>(A, w, kw, false, upd_grid, s);
    else xupdate_t<float>(A, w, kw, true, upd_grid, s);
    if (ax) {
        int rc = launch_multi_f64(A, w->x, w->q64, kw, s);
        if (rc) return rc;
    }
    if (sh.f64) {
        if (sh.pre) outer_t<double, true>(A, w, kw, ax, 0, upd_grid, s);
        else outer_t<double, false>(A, w, kw, ax, 0, upd_grid, s);
    } else {
        outer_t<float, false>(A, w, kw, ax, reliable, upd_grid, s);
    }
    mc_finalize_res<<<kw, 256, 0, s>>>(w->part, upd_grid, kw, w->sc, reliable, sh.f64 ? 1 : 0);
    // reliable updates: the kept directions take the replaced residuals
    if (reliable) replaced_pupdate(A, w, kw, upd_grid, s);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

// Where a column stands after a scalar read: still iterating, or waiting for an
// outer step (due, or its inner CG stopped).
static void column_flags(const MScal& h, bool& iterating, bool& acted) {
    iterating |= h.status_in == CG_RUNNING;
    acted |= h.status_out == CG_RUNNING && (h.status_in != CG_RUNNING || h.due);
}

// Options shared by cg_solve_multi and the server's groups.
static int check_multi_options(const fespmv_mat* A, const cg_options& o, const char* who) {
    if (o.flags & FESPMV_CG_SINGLE_REDUCTION) {
        set_error("%s: FESPMV_CG_SINGLE_REDUCTION is not supported", who);
        return FESPMV_ERR_UNSUPPORTED;
    }
    if (o.precision == FESPMV_CG_BF16_REFINE) {
        set_error("%s: FESPMV_CG_BF16_REFINE is not supported (FP64 or FP32 refinement)", who);
        return FESPMV_ERR_UNSUPPORTED;
    }
    if (A->format != FESPMV_FMT_SLICED || A->max_lanes_log2 != 0) {
        set_error("%s needs a SLICED handle with one lane per row (threshold 0)", who);
        return FESPMV_ERR_UNSUPPORTED;
    }
    return check_precision(A, o.precision);
}

static Shape shape_of(int kw, const cg_options& o) {
    const bool f64 = o.precision == FESPMV_CG_F64;
    return Shape{kw, f64, f64 && !(o.flags & FESPMV_CG_NO_PRECOND)};
}

static int solve_multi_impl(fespmv_mat* A, const double* B, double* X, int k, const cg_options* opts,
                            cg_result* res, cudaStream_t s) {
    cg_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    int rc = normalize_options(o);
    if (rc || (rc = check_multi_options(A, o, "cg_solve_multi"))) return rc;
    if (o.flags & FESPMV_CG_FLEXIBLE) {
        set_error("cg_solve_multi: FESPMV_CG_FLEXIBLE is not supported");
        return FESPMV_ERR_UNSUPPORTED;
    }
    if (A->n == 0) {   // empty system: every column is solved by x = 0
        if (res)
            for (int j = 0; j < k; ++j) std::memset(&res[j], 0, sizeof(cg_result));
        return FESPMV_OK;
    }
    const Shape sh = shape_of(multi_width(k), o);
    const bool f64 = sh.f64;
    const int kw = sh.kw;
    const int64_t n = A->n;
    const unsigned dot_grid = dot_grid_of(A, kw, f64);
    const unsigned upd_grid = update_grid(n, kw);
    if ((rc = ensure_handle_work(A, kw))) return rc;
    MultiWork* w = A->mcg;
    if ((rc = multi_graph(A, w, sh, o.check_every, dot_grid, upd_grid))) return rc;
    if ((rc = prepare_diag(A, w, sh, s))) {
        if (res)
            for (int j = 0; j < k; ++j) {
                std::memset(&res[j], 0, sizeof(cg_result));
                res[j].status = rc;
            }
        set_error("cg_solve_multi: the diagonal has a non-positive or non-finite entry");
        return rc;
    }

    // b (and x0) into the handle's numbering, row stride kw
    const bool host = o.flags & FESPMV_IO_HOST;
    const int32_t* perm = (o.flags & FESPMV_IO_PERMUTED) ? nullptr : A->d_perm;
    const size_t nk = sizeof(double) * (size_t)n * k;
    const double* bsrc = B;
    if (host) {
        FESPMV_CUDA(cudaMemcpyAsync(w->q64, B, nk, cudaMemcpyHostToDevice, s));
        bsrc = w->q64;
    }
    launch_gather_rows_f64(bsrc, k, perm, w->b, kw, n, k, s);
    const bool x0 = o.flags & FESPMV_CG_X0;
    if (x0) {
        const double* xsrc = X;
        if (host) {
            FESPMV_CUDA(cudaMemcpyAsync(w->q64, X, nk, cudaMemcpyHostToDevice, s));
            xsrc = w->q64;
        }
        launch_gather_rows_f64(xsrc, k, perm, w->x, kw, n, k, s);
    } else {
        FESPMV_CUDA(cudaMemsetAsync(w->x, 0, sizeof(double) * (size_t)n * kw, s));
    }
    // inner vectors start at zero: kept directions and frozen columns read defined values
    for (void* v : {w->w, w->r, w->p, w->q})
        FESPMV_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * (size_t)n * kw, s));
    for (int j = 0; j < kw; ++j) w->h_sc[j] = new_column(o, f64);
    FESPMV_CUDA(cudaMemcpyAsync(w->sc, w->h_sc, sizeof(MScal) * kw, cudaMemcpyHostToDevice, s));
    const int reliable = (o.flags & FESPMV_CG_RELIABLE) ? 1 : 0;
    // Outer steps come on a fixed grid of `period` inner iterations (and when no
    // column is iterating, the next grid point is taken at once: the idle steps in
    // between change nothing).  So when a column is acted on depends on its own
    // iterates only.
    const int64_t period = (int64_t)o.check_every * kOuterChunks;
    int64_t it = 0;   // inner iterations on the grid
    for (int step = 0;; ++step) {
        if ((rc = enqueue_outer(A, w, sh, reliable, x0 || step > 0, upd_grid, s))) return rc;
        if ((rc = read_scalars(w, kw, s))) return rc;
        bool running = false;
        for (int j = 0; j < kw; ++j) running |= w->h_sc[j].status_in == CG_RUNNING;
        if (!running) break;   // every column has stopped
        for (;;) {
            FESPMV_CUDA(cudaGraphLaunch(w->graph, s));
            it += o.check_every;
            if ((rc = read_scalars(w, kw, s))) return rc;
            bool iterating = false, acted = false;
            for (int j = 0; j < kw; ++j) column_flags(w->h_sc[j], iterating, acted);
            if (!iterating) {
                it = (it + period - 1) / period * period;
                break;
            }
            if (it % period == 0 && acted) break;
        }
    }
    // x back to the caller's numbering and row stride k
    double* xdst = host ? w->q64 : X;
    launch_gather_rows_f64(w->x, kw, (o.flags & FESPMV_IO_PERMUTED) ? nullptr : A->d_pinv, xdst, k, n, k, s);
    FESPMV_CUDA(cudaGetLastError());
    if (host) FESPMV_CUDA(cudaMemcpyAsync(X, w->q64, nk, cudaMemcpyDeviceToHost, s));
    FESPMV_CUDA(cudaStreamSynchronize(s));
    int worst = FESPMV_OK;
    for (int j = 0; j < k; ++j) {
        const cg_result r = column_result(w->h_sc[j], f64);
        if (r.status != FESPMV_OK && worst == FESPMV_OK) worst = r.status;
        if (res) res[j] = r;
    }
    if (worst != FESPMV_OK) set_error("cg_solve_multi: at least one right-hand side did not converge");
    return worst;
}

// ------------------------------------------------------------------ groups of the solve server

// out[i] = M[pinv[i], c] (row stride kw): one column of x in the input numbering.
__global__ void mc_extract_column(const double* __restrict__ M, int kw, int c, const int32_t* __restrict__ pinv,
                                  double* __restrict__ out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = M[(int64_t)pinv[i] * kw + c];
}

// M[i, c] = in[perm[i]] (in == nullptr: 0): one column of b, or x = 0.
__global__ void mc_insert_column(const double* __restrict__ in, const int32_t* __restrict__ perm,
                                 double* __restrict__ M, int kw, int c, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) M[i * kw + c] = in ? in[perm[i]] : 0.0;
}

}  // namespace

struct GroupColumn {
    int state = 0;            // 0 free, 1 waiting for an outer step, 2 solving
    int64_t tag = 0;
    std::vector<double> b;
    cg_options o{};
};

struct MultiGroup {
    fespmv_mat* A = nullptr;
    MultiWork* w = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;     // the outer step's scalars are back
    Shape sh{};
    int reliable = 0, precision = 0, flags = 0, chunk = 16;
    int64_t period = 0, it = 0;
    unsigned upd_grid = 0;
    int phase = 0;            // 0 nothing enqueued, 1 an outer step, 2 graphs of inner iterations
    // graphs in flight (at most 2, oldest at qhead): their scalars, events and end points
    cudaEvent_t gev[2] = {nullptr, nullptr};
    MScal* h_slot[2] = {nullptr, nullptr};
    int64_t q_end[2] = {0, 0};
    int nq = 0, qhead = 0;
    std::vector<GroupColumn> cols;
    double* d_io = nullptr;   // one column in or out (n doubles)
};

namespace {

void group_free(MultiGroup* g) {
    if (!g) return;
    if (g->s) cudaStreamSynchronize(g->s);
    destroy_multi_work(g->w);
    if (g->d_io) cudaFree(g->d_io);
    if (g->ev) cudaEventDestroy(g->ev);
    for (int k = 0; k < 2; ++k) {
        if (g->gev[k]) cudaEventDestroy(g->gev[k]);
        if (g->h_slot[k]) cudaFreeHost(g->h_slot[k]);
    }
    if (g->s) cudaStreamDestroy(g->s);
    delete g;
}

// Queue graphs of inner iterations, up to two in flight.  A graph may start at a
// grid point only once the graph ending there has been examined (the outer-step
// decision is taken on its scalars); between grid points a graph is queued before
// the previous one's scalars are back, which keeps the GPU busy.  A queued graph
// that turns out to follow the last column's stop changes nothing.
int group_top_up(MultiGroup* g) {
    const int kw = g->sh.kw;
    int64_t tail = g->nq ? g->q_end[(g->qhead + g->nq - 1) % 2] : g->it;
    while (g->nq < 2) {
        if (tail % g->period == 0 && tail != g->it) break;
        const int slot = (g->qhead + g->nq) % 2;
        FESPMV_CUDA(cudaGraphLaunch(g->w->graph, g->s));
        FESPMV_CUDA(cudaMemcpyAsync(g->h_slot[slot], g->w->sc, sizeof(MScal) * kw, cudaMemcpyDeviceToHost, g->s));
        FESPMV_CUDA(cudaEventRecord(g->gev[slot], g->s));
        tail += g->chunk;
        g->q_end[slot] = tail;
        ++g->nq;
    }
    g->phase = 2;
    return FESPMV_OK;
}

// Inject the waiting columns, enqueue an outer step and the read of the scalars.
int group_start_outer(MultiGroup* g) {
    fespmv_mat* A = g->A;
    MultiWork* w = g->w;
    const int kw = g->sh.kw;
    const unsigned gr = grid_for(A->n, 256);
    for (int c = 0; c < kw; ++c) {
        GroupColumn& col = g->cols[(size_t)c];
        if (col.state != 1) continue;
        FESPMV_CUDA(cudaMemcpyAsync(g->d_io, col.b.data(), sizeof(double) * (size_t)A->n, cudaMemcpyHostToDevice,
                                    g->s));
        mc_insert_column<<<gr, 256, 0, g->s>>>(g->d_io, A->d_perm, w->b, kw, c, A->n);
        mc_insert_column<<<gr, 256, 0, g->s>>>(nullptr, A->d_perm, w->x, kw, c, A->n);
        w->h_sc[c] = new_column(col.o, g->sh.f64);
        FESPMV_CUDA(cudaMemcpyAsync(w->sc + c, &w->h_sc[c], sizeof(MScal), cudaMemcpyHostToDevice, g->s));
        col.state = 2;
    }
    int rc = enqueue_outer(A, w, g->sh, g->reliable, true, g->upd_grid, g->s);
    if (rc) return rc;
    FESPMV_CUDA(cudaMemcpyAsync(w->h_sc, w->sc, sizeof(MScal) * kw, cudaMemcpyDeviceToHost, g->s));
    FESPMV_CUDA(cudaEventRecord(g->ev, g->s));
    g->phase = 1;
    return FESPMV_OK;
}

}  // namespace

// ---- the server's interface (multi_group.h)

int group_width_auto(const fespmv_mat* A) {
    int kw = 32;
    while (kw > 4 && A->n * (int64_t)kw > ((int64_t)1 << 21)) kw /= 2;
    return kw;
}

int64_t group_bytes(const fespmv_mat* A, int kw) {
    return (int64_t)sizeof(double) * (7 * kw + 2) * A->n + (int64_t)sizeof(double) * multi_part_len(A, kw) +
           (int64_t)sizeof(MScal) * 32 + (A->d_vdf ? (int64_t)sizeof(float2) * kw * A->n : 0);
}

int group_create(fespmv_mat* A, int kw, const cg_options& o, MultiGroup** out) {
    *out = nullptr;
    int rc = check_multi_options(A, o, "solve group");
    if (rc) return rc;
    if (A->n == 0) {
        set_error("solve group: empty matrix");
        return FESPMV_ERR_INVALID_ARG;
    }
    MultiGroup* g = new MultiGroup();
    g->A = A;
    g->sh = shape_of(kw, o);
    g->reliable = (o.flags & FESPMV_CG_RELIABLE) ? 1 : 0;
    g->precision = o.precision;
    g->flags = o.flags & (FESPMV_CG_RELIABLE | FESPMV_CG_NO_PRECOND);
    g->chunk = o.check_every;
    g->period = (int64_t)o.check_every * kOuterChunks;
    g->cols.resize((size_t)kw);
    g->upd_grid = update_grid(A->n, kw);
    const unsigned dot_grid = dot_grid_of(A, kw, g->sh.f64);
    cudaError_t e = cudaStreamCreateWithFlags(&g->s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&g->gev[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&g->h_slot[k], sizeof(MScal) * 32);
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->d_io, sizeof(double) * (size_t)A->n);
    if (e != cudaSuccess) {
        group_free(g);
        return cuda_fail(e, "solve group");
    }
    if ((rc = create_multi_work(A, kw, &g->w)) || (rc = multi_graph(A, g->w, g->sh, g->chunk, dot_grid, g->upd_grid)) ||
        (rc = prepare_diag(A, g->w, g->sh, g->s))) {
        group_free(g);
        return rc;
    }
    // inner vectors start at zero (columns that never ran still pass through the product)
    for (void* v : {g->w->w, g->w->r, g->w->p, g->w->q}) {
        e = cudaMemsetAsync(v, 0, sizeof(double) * (size_t)A->n * kw, g->s);
        if (e != cudaSuccess) {
            group_free(g);
            return cuda_fail(e, "cudaMemsetAsync");
        }
    }
    // every column starts finished and idle
    MScal idle;
    std::memset(&idle, 0, sizeof(idle));
    idle.status_out = CG_CONVERGED;
    idle.status_in = CG_CONVERGED;
    for (int c = 0; c < kw; ++c) g->w->h_sc[c] = idle;
    e = cudaMemcpyAsync(g->w->sc, g->w->h_sc, sizeof(MScal) * kw, cudaMemcpyHostToDevice, g->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
    if (e != cudaSuccess) {
        group_free(g);
        return cuda_fail(e, "solve group");
    }
    *out = g;
    return FESPMV_OK;
}

void group_destroy(MultiGroup* g) { group_free(g); }

int64_t group_device_bytes(const MultiGroup* g) {
    return g->w->bytes + (int64_t)sizeof(double) * g->A->n;
}

bool group_matches(const MultiGroup* g, const cg_options& o) {
    return g->precision == o.precision && g->flags == (o.flags & (FESPMV_CG_RELIABLE | FESPMV_CG_NO_PRECOND)) &&
           g->chunk == o.check_every;
}

int group_free_columns(const MultiGroup* g) {
    int k = 0;
    for (const GroupColumn& c : g->cols) k += c.state == 0;
    return k;
}

int group_width_of(const MultiGroup* g) { return g->sh.kw; }

bool group_empty(const MultiGroup* g) {
    return g->phase == 0 && group_free_columns(g) == (int)g->cols.size();
}

int group_add(MultiGroup* g, int64_t tag, const double* b, const cg_options& o) {
    for (GroupColumn& c : g->cols)
        if (c.state == 0) {
            c.state = 1;
            c.tag = tag;
            c.b.assign(b, b + g->A->n);
            c.o = o;
            return FESPMV_OK;
        }
    set_error("solve group: no free column");
    return FESPMV_ERR_INVALID_ARG;
}

int group_step(MultiGroup* g, bool* progress, std::vector<GroupDone>& done) {
    *progress = false;
    const int kw = g->sh.kw;
    if (g->phase == 0) {
        bool waiting = false;
        for (const GroupColumn& c : g->cols) waiting |= c.state == 1;
        if (!waiting) return FESPMV_OK;
        *progress = true;
        return group_start_outer(g);
    }
    const int slot = g->qhead;
    cudaError_t q = cudaEventQuery(g->phase == 1 ? g->ev : g->gev[slot]);
    if (q == cudaErrorNotReady) return FESPMV_OK;
    if (q != cudaSuccess) return cuda_fail(q, "solve group");
    *progress = true;
    const MScal* h;
    const bool after_graph = g->phase == 2;
    if (after_graph) {
        h = g->h_slot[slot];
        g->it = g->q_end[slot];
        g->qhead = (g->qhead + 1) % 2;
        --g->nq;
    } else {   // the columns this outer step finished: x out, results
        h = g->w->h_sc;
        for (int c = 0; c < kw; ++c) {
            GroupColumn& col = g->cols[(size_t)c];
            if (col.state != 2 || h[c].status_out == CG_RUNNING) continue;
            GroupDone d;
            d.tag = col.tag;
            d.res = column_result(h[c], g->sh.f64);
            d.x.resize((size_t)g->A->n);
            mc_extract_column<<<grid_for(g->A->n, 256), 256, 0, g->s>>>(g->w->x, kw, c, g->A->d_pinv, g->d_io,
                                                                         g->A->n);
            FESPMV_CUDA(cudaMemcpyAsync(d.x.data(), g->d_io, sizeof(double) * (size_t)g->A->n,
                                        cudaMemcpyDeviceToHost, g->s));
            FESPMV_CUDA(cudaStreamSynchronize(g->s));
            done.push_back(std::move(d));
            col.state = 0;
            col.b.clear();
            col.b.shrink_to_fit();
        }
    }
    bool iterating = false, acted = false, waiting = false;
    for (int c = 0; c < kw; ++c) {
        const GroupColumn& col = g->cols[(size_t)c];
        if (col.state == 2) column_flags(h[c], iterating, acted);
        waiting |= col.state == 1;
    }
    if (!iterating) {
        // graphs still queued change nothing now; stream order runs them before what follows
        g->nq = 0;
        if (!acted && !waiting) {   // nothing left: the next column starts a fresh grid
            g->phase = 0;
            g->it = 0;
            return FESPMV_OK;
        }
        g->it = (g->it + g->period - 1) / g->period * g->period;
        return group_start_outer(g);
    }
    // a graph that ends on a grid point is examined before anything is queued past it
    if (after_graph && g->it % g->period == 0 && (acted || waiting)) return group_start_outer(g);
    return group_top_up(g);
}

void free_multi_cg(fespmv_mat* A) {
    if (A && A->mcg) {
        A->device_bytes -= A->mcg->bytes;
        destroy_multi_work(A->mcg);
        A->mcg = nullptr;
    }
}

}  // namespace fespmv

using namespace fespmv;

extern "C" int cg_solve_multi(fespmv_mat_t A, const double* B, double* X, int32_t k, const cg_options* opts,
                              cg_result* res, fespmv_stream_t stream) {
    try {
        if (!A || k < 1 || k > 32 || (A->n > 0 && (!B || !X))) {
            set_error("cg_solve_multi: bad argument");
            return FESPMV_ERR_INVALID_ARG;
        }
        return solve_multi_impl(A, B, X, k, opts, res, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FESPMV_ERR_OOM;
    } catch (...) {
        set_error("unexpected C++ exception");
        return FESPMV_ERR_INVALID_ARG;
    }
}
