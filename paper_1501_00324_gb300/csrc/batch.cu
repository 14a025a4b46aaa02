// Batched FE matrices (batch_* in fespmv.h): many independent problems of
// uneven sizes held as one block-diagonal SLICED matrix and solved together.
//
// Each problem is ordered and renumbered on its own (Morton order of its own
// nodes, windowed length sort, sorted columns: Sec. 5.1-5.3) and padded with
// identity rows to a multiple of 32 rows, so that no 32-row group -- and hence
// no warp slice (Sec. 5.1, 5.4) -- spans two problems.  One product of the
// block-diagonal matrix is then every problem's product in one launch.
//
// The solver is the FP64 iterative refinement of cg_solve around an FP32 inner
// CG on B = S A S, run for all problems in lockstep with per-problem scalars:
// per-slice and per-warp partial sums are reduced per problem (one block per
// problem, fixed order), problems that have finished are skipped by every
// kernel, and one CUDA graph holds `check_every` inner iterations of the whole
// batch (five launches per iteration, whatever the number of problems).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "cg_run.h"
#include "cluster_device.cuh"
#include "internal.h"
#include "spmv_device.cuh"

namespace fespmv {

struct BScal {
    double rho, pq, alpha, beta, rr_in, thresh_in, rr, bb, rhs2, thresh2, prev;
    int iters, iters_in, status_in, status_out, outer, max_iter, max_outer, pad;
};

}  // namespace fespmv

struct fespmv_batch {
    int32_t count = 0;
    fespmv_mat* M = nullptr;              // block-diagonal padded matrix
    int64_t n_in = 0;                     // sum of the problems' rows
    std::vector<int64_t> n_rows, in_off, row_off, pslice, pwarp;
    int32_t* d_slice_prob = nullptr;      // slice -> problem
    int32_t* d_warp_prob = nullptr;       // 32-row group -> problem
    int64_t* d_pslice = nullptr;          // problem -> first slice (count + 1)
    int64_t* d_pwarp = nullptr;           // problem -> first 32-row group (count + 1)
    int32_t* d_perm_g = nullptr;          // padded permuted row -> input row, -1 = padding
    int32_t* d_pinv_g = nullptr;          // input row -> padded permuted row
    // solver workspace (first batch_cg_solve)
    double *x = nullptr, *b = nullptr, *q = nullptr, *part = nullptr;
    float *w32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    fespmv::BScal* sc = nullptr;
    fespmv::BScal* h_sc = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_chunk = 0, graph_bf16 = -1;
    // the cluster solver (reliable updates): problems largest first, a work counter
    int32_t* d_order = nullptr;
    unsigned* d_next = nullptr;
};

namespace fespmv {

// ------------------------------------------------------------------ kernels

__global__ void gather_pad_f64(const double* __restrict__ in, const int32_t* __restrict__ idx,
                               double* __restrict__ out, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const int32_t s = idx[i];
        out[i] = s >= 0 ? __ldg(in + s) : 0.0;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of part[b, e) over one block in a fixed order (valid in thread 0).
__device__ double block_range_sum(const double* __restrict__ part, int64_t b, int64_t e) {
    __shared__ double sh[32];
    double t = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) t += part[i];
    t = warp_sum(t);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[warp] = t;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

template <typename VT, int V, int U>
__global__ void __launch_bounds__(256) b_spmv32_dot(const uint4* __restrict__ meta,
                                                    const int32_t* __restrict__ col,
                                                    const VT* __restrict__ val,
                                                    const float* __restrict__ p,
                                                    float* __restrict__ q, int64_t n_slices,
                                                    const int32_t* __restrict__ slice_prob,
                                                    double* __restrict__ part,
                                                    const BScal* __restrict__ sc) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_slices) return;
    if (sc[slice_prob[warp]].status_in != CG_RUNNING) return;
    const uint4 m = meta[warp];
    const float sum = sliced_row_sum_low<VT, V, U>(m, col, val, p, lane);
    const int lt = (int)m.w;
    const int64_t row = (int64_t)m.z + (lane >> lt);
    double c = 0.0;
    if ((lane & ((1 << lt) - 1)) == 0) {   // every group is full: all rows are real or padding
        q[row] = sum;
        c = (double)p[row] * (double)sum;
    }
    c = warp_sum(c);
    if (lane == 0) part[warp] = c;
}

__global__ void b_finalize_pq(const double* __restrict__ part, const int64_t* __restrict__ pslice,
                              BScal* sc) {
    const int j = blockIdx.x;
    if (sc[j].status_in != CG_RUNNING) return;
    const double pq = block_range_sum(part, pslice[j], pslice[j + 1]);
    if (threadIdx.x == 0) {
        sc[j].pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) sc[j].status_in = CG_BREAKDOWN;
        else sc[j].alpha = sc[j].rho / pq;
    }
}

__global__ void __launch_bounds__(256) b_update32(int64_t np, float* __restrict__ w,
                                                  float* __restrict__ r,
                                                  const float* __restrict__ p,
                                                  const float* __restrict__ q,
                                                  const int32_t* __restrict__ warp_prob,
                                                  double* __restrict__ part,
                                                  const BScal* __restrict__ sc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;                   // np is a multiple of 32: whole warps leave
    const int64_t g = i >> 5;
    const BScal& s = sc[warp_prob[g]];
    if (s.status_in != CG_RUNNING) return;
    const float a = (float)s.alpha;
    w[i] = fmaf(a, p[i], w[i]);
    const float ri = fmaf(-a, q[i], r[i]);
    r[i] = ri;
    const double c = warp_sum((double)ri * (double)ri);
    if ((threadIdx.x & 31) == 0) part[g] = c;
}

__global__ void b_finalize_rr(const double* __restrict__ part, const int64_t* __restrict__ pwarp,
                              BScal* sc) {
    const int j = blockIdx.x;
    if (sc[j].status_in != CG_RUNNING) return;
    const double rr = block_range_sum(part, pwarp[j], pwarp[j + 1]);
    if (threadIdx.x == 0) {
        BScal& s = sc[j];
        s.iters += 1;
        s.iters_in += 1;
        s.rr_in = rr;
        if (!isfinite(rr)) s.status_in = CG_BREAKDOWN;
        else if (rr <= s.thresh_in) s.status_in = CG_CONVERGED;
        else if (s.iters_in >= s.max_iter) s.status_in = CG_MAXITER;
        else {
            s.beta = rr / s.rho;
            s.rho = rr;
        }
    }
}

__global__ void __launch_bounds__(256) b_pupdate32(int64_t np, float* __restrict__ p,
                                                   const float* __restrict__ r,
                                                   const int32_t* __restrict__ warp_prob,
                                                   const BScal* __restrict__ sc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const BScal& s = sc[warp_prob[i >> 5]];
    if (s.status_in != CG_RUNNING) return;
    p[i] = fmaf((float)s.beta, p[i], r[i]);
}

// r = b - Ax (Ax = q or 0), rhs = float(S r), w = 0, r_in = p = rhs for problems
// still refining; per-group partials of r.r, rhs.rhs, b.b.
__global__ void __launch_bounds__(256) b_residual(int64_t np, const double* __restrict__ b,
                                                  const double* __restrict__ q,
                                                  const double* __restrict__ scale,
                                                  float* __restrict__ w, float* __restrict__ r32,
                                                  float* __restrict__ p32,
                                                  const int32_t* __restrict__ warp_prob,
                                                  double* __restrict__ part, int64_t ngroups,
                                                  int reliable, const BScal* __restrict__ sc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int64_t g = i >> 5;
    const BScal& s = sc[warp_prob[g]];
    if (s.status_out != CG_RUNNING) return;
    const double bi = b[i];
    const double ri = q ? bi - q[i] : bi;
    const float rs = (float)(scale[i] * ri);
    w[i] = 0.0f;
    r32[i] = rs;
    if (!(reliable && s.outer > 0)) p32[i] = rs;   // reliable updates keep the direction
    const double c0 = warp_sum(ri * ri);
    const double c1 = warp_sum((double)rs * (double)rs);
    const double c2 = warp_sum(bi * bi);
    if ((threadIdx.x & 31) == 0) {
        part[g] = c0;
        part[ngroups + g] = c1;
        part[2 * ngroups + g] = c2;
    }
}

__global__ void b_finalize_res(const double* __restrict__ part, int64_t ngroups,
                               const int64_t* __restrict__ pwarp, BScal* sc, double tol2,
                               double in2, int reliable) {
    const int j = blockIdx.x;
    if (sc[j].status_out != CG_RUNNING) return;
    const double rr = block_range_sum(part, pwarp[j], pwarp[j + 1]);
    const double rhs2 = block_range_sum(part + ngroups, pwarp[j], pwarp[j + 1]);
    const double bb = block_range_sum(part + 2 * ngroups, pwarp[j], pwarp[j + 1]);
    if (threadIdx.x == 0) {
        BScal& s = sc[j];
        s.rr = rr;
        s.bb = bb;
        s.thresh2 = tol2 * bb;
        s.status_in = CG_CONVERGED;        // idle unless another inner solve starts below
        if (!isfinite(rr) || !isfinite(rhs2)) s.status_out = CG_BREAKDOWN;
        else if (rr <= s.thresh2) s.status_out = CG_CONVERGED;
        else if (s.outer >= s.max_outer) s.status_out = CG_MAXITER;
        else if (reliable && s.iters >= s.max_iter) s.status_out = CG_MAXITER;
        else if (!(rr < s.prev)) s.status_out = CG_MAXITER;   // stagnation
        else {
            s.prev = rr;
            if (reliable) {   // replace the residual, keep p: p = r_in + beta p follows
                s.beta = s.outer > 0 ? rhs2 / s.rho : 0.0;
                s.thresh_in = fmax(in2 * rhs2, rr > 0.0 ? tol2 * bb * rhs2 / rr : 0.0);
            } else {
                s.thresh_in = in2 * rhs2;
                s.iters_in = 0;
            }
            s.rho = rhs2;
            s.status_in = CG_RUNNING;
        }
    }
}

// x += S w for problems that ran an inner solve in this refinement step.
__global__ void __launch_bounds__(256) b_xupdate(int64_t np, double* __restrict__ x,
                                                 const double* __restrict__ scale,
                                                 const float* __restrict__ w,
                                                 const int32_t* __restrict__ warp_prob,
                                                 const BScal* __restrict__ sc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    if (sc[warp_prob[i >> 5]].status_out != CG_RUNNING) return;
    x[i] = fma(scale[i], (double)w[i], x[i]);
}

__global__ void b_outer_count(int count, BScal* sc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < count && sc[j].status_out == CG_RUNNING) sc[j].outer += 1;
}

// ------------------------------------------------------------------ cluster solver
//
// Reliable-update refinement for the whole batch in one persistent launch:
// thread-block clusters take problems from a work counter (largest first) and
// each runs its problem's solve to the end (cluster_reliable in
// cluster_device.cuh), synchronising only within the cluster.  No grid-wide
// synchronisation and no host polling: finished problems cost nothing, and a
// small problem's iterations cost a few cluster barriers each.
template <typename VT, int V, int U>
__global__ void __launch_bounds__(kClusterThreads, 2) b_cluster_reliable(
    const uint4* __restrict__ meta, const int32_t* __restrict__ col, const VT* __restrict__ val32,
    const double* __restrict__ val64, const double* __restrict__ scale, const double* __restrict__ b,
    double* __restrict__ x, double* __restrict__ q64, float* __restrict__ w, float* __restrict__ rin,
    float* __restrict__ p, float* __restrict__ q32, const int64_t* __restrict__ pslice,
    const int64_t* __restrict__ pwarp, const int32_t* __restrict__ order, int count, unsigned* next,
    BScal* sc, double tol2, double in2, int has_x0, int max_iter, int max_outer) {
    cgx::cluster_group cl = cgx::this_cluster();
    __shared__ ClusterRed red;
    const unsigned rank = cl.block_rank();
    int turn = 0;
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) red.job = (int)atomicAdd(next, 1u);
        cl.sync();
        const int job = *cl.map_shared_rank(&red.job, 0);
        if (job >= count) break;
        const int j = order[job];
        const ClusterOut o = cluster_reliable<VT, V, U>(cl, red, turn, meta, col, val32, val64, scale, b, x, q64, w,
                                                        rin, p, q32, pslice[j], pslice[j + 1], 32 * pwarp[j],
                                                        32 * pwarp[j + 1], tol2, in2, has_x0, max_iter, max_outer);
        if (rank == 0 && threadIdx.x == 0) {
            BScal& s = sc[j];
            s.status_out = o.status;
            s.status_in = CG_CONVERGED;
            s.iters = o.iters;
            s.outer = o.outer;
            s.rr = o.rr;
            s.bb = o.bb;
        }
        cl.sync();   // the job word and the reduction slots are reused by the next problem
    }
    cl.sync();       // no CTA leaves while another may still read its shared memory
}

// ------------------------------------------------------------------ host side

static void destroy_batch(fespmv_batch* B) {
    if (!B) return;
    if (B->graph) cudaGraphExecDestroy(B->graph);
    if (B->cap) cudaStreamDestroy(B->cap);
    void* ptrs[] = {B->d_slice_prob, B->d_warp_prob, B->d_pslice, B->d_pwarp, B->d_perm_g, B->d_pinv_g,
                    B->x, B->b, B->q, B->part, B->w32, B->r32, B->p32, B->q32, B->sc, B->d_order, B->d_next};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (B->h_sc) cudaFreeHost(B->h_sc);
    if (B->M) free_handle(B->M);
    delete B;
}

static int batch_create_impl(fespmv_batch_t* out, int32_t count, const int64_t* n_rows,
                             const int64_t* const* rowptr, const int32_t* const* colind,
                             const double* const* values, const fespmv_mesh_info* mesh,
                             const fespmv_options* opts_in, cudaStream_t s) {
    if (!out || count <= 0 || !n_rows || !rowptr || !colind || !values) {
        set_error("batch_create: null argument or count <= 0");
        return FESPMV_ERR_INVALID_ARG;
    }
    *out = nullptr;
    fespmv_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts_in) o = *opts_in;
    if (o.vec == 0) o.vec = 2;
    if (o.block == 0) o.block = 256;
    if ((o.vec != 1 && o.vec != 2 && o.vec != 4) || o.block < 32 || o.block > 256 || o.block % 32 ||
        o.sigma < 0 || o.threshold < 0 ||
        (o.precisions & ~(FESPMV_PREC_F64 | FESPMV_PREC_F32 | FESPMV_PREC_BF16))) {
        set_error("batch_create: bad options");
        return FESPMV_ERR_INVALID_ARG;
    }
    if (!(o.precisions & (FESPMV_PREC_F32 | FESPMV_PREC_BF16))) o.precisions |= FESPMV_PREC_F32;
    // validate and order every problem (independent: in parallel)
    std::vector<Permuted> pm((size_t)count);
    std::vector<int> rcs((size_t)count, FESPMV_OK);
    std::vector<std::string> errs((size_t)count);
    for (int j = 0; j < count; ++j)
        if (n_rows[j] < 0 || (n_rows[j] > 0 && (!rowptr[j] || (rowptr[j][n_rows[j]] > 0 && (!colind[j] || !values[j]))))) {
            set_error("batch_create: problem %d has a null array or negative size", j);
            return FESPMV_ERR_INVALID_ARG;
        }
    {
        const int nt = std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
        std::vector<std::thread> th;
        for (int t = 0; t < nt; ++t)
            th.emplace_back([&, t] {
                for (int j = t; j < count; j += nt) {
                    const bool xyz = mesh && mesh[j].node_xyz;
                    if (o.reorder == FESPMV_REORDER_MORTON && !xyz) {
                        rcs[(size_t)j] = FESPMV_ERR_INVALID_ARG;
                        errs[(size_t)j] = "REORDER_MORTON needs node_xyz for every problem";
                        continue;
                    }
                    int rc = validate_csr(n_rows[j], rowptr[j], colind[j]);
                    if (!rc)
                        rc = order_and_permute(n_rows[j], rowptr[j], colind[j],
                                               mesh && mesh[j].dofs_per_node > 0 ? mesh[j].dofs_per_node : 1,
                                               xyz ? mesh[j].node_xyz : nullptr, o.reorder, o.sigma,
                                               pm[(size_t)j]);
                    rcs[(size_t)j] = rc;
                    if (rc) errs[(size_t)j] = fespmv_last_error();
                }
            });
        for (auto& t : th) t.join();
    }
    for (int j = 0; j < count; ++j)
        if (rcs[(size_t)j]) {
            set_error("batch_create: problem %d: %s", j, errs[(size_t)j].c_str());
            return rcs[(size_t)j];
        }

    fespmv_batch* B = new fespmv_batch();
    B->count = count;
    B->n_rows.assign(n_rows, n_rows + count);
    B->in_off.assign((size_t)count + 1, 0);
    B->row_off.assign((size_t)count + 1, 0);
    std::vector<int64_t> nnz_off((size_t)count + 1, 0);
    for (int j = 0; j < count; ++j) {
        B->in_off[(size_t)j + 1] = B->in_off[(size_t)j] + n_rows[j];
        B->row_off[(size_t)j + 1] = B->row_off[(size_t)j] + (n_rows[j] + 31) / 32 * 32;
        nnz_off[(size_t)j + 1] = nnz_off[(size_t)j] + (n_rows[j] ? rowptr[j][n_rows[j]] : 0);
    }
    const int64_t np = B->row_off[(size_t)count];
    B->n_in = B->in_off[(size_t)count];
    if (np > (int64_t)INT32_MAX - 1) {
        set_error("batch_create: %lld padded rows exceed 32-bit indices", (long long)np);
        destroy_batch(B);
        return FESPMV_ERR_UNSUPPORTED;
    }
    // global permuted CSR: problem blocks on the diagonal, padding rows = identity
    std::vector<int64_t> rp(1, 0);
    rp.reserve((size_t)np + 1);
    std::vector<int32_t> cc;
    std::vector<int64_t> ss;
    cc.reserve((size_t)nnz_off[(size_t)count] + (size_t)(np - B->n_in));
    ss.reserve(cc.capacity());
    Plan plan;
    plan.perm.resize((size_t)np);
    plan.pinv.resize((size_t)np);
    plan.diagpos.resize((size_t)np);
    std::vector<int32_t> perm_g((size_t)np, -1), pinv_g((size_t)B->n_in);
    for (int j = 0; j < count; ++j) {
        const Permuted& P = pm[(size_t)j];
        const int64_t ro = B->row_off[(size_t)j], io = B->in_off[(size_t)j], no = nnz_off[(size_t)j];
        const int64_t nj = n_rows[j], padj = B->row_off[(size_t)j + 1] - ro;
        for (int64_t i = 0; i < padj; ++i) {
            if (i < nj) {
                for (int64_t k = P.rp2[(size_t)i]; k < P.rp2[(size_t)i + 1]; ++k) {
                    cc.push_back((int32_t)(ro + P.c2[(size_t)k]));
                    ss.push_back(no + P.s2[(size_t)k]);
                }
                plan.diagpos[(size_t)(ro + i)] = P.diagpos[(size_t)i] >= 0 ? no + P.diagpos[(size_t)i] : -1;
                perm_g[(size_t)(ro + i)] = (int32_t)(io + P.perm[(size_t)i]);
                pinv_g[(size_t)(io + P.perm[(size_t)i])] = (int32_t)(ro + i);
            } else {
                cc.push_back((int32_t)(ro + i));      // padding: unit diagonal
                ss.push_back(-2);
                plan.diagpos[(size_t)(ro + i)] = -2;
            }
            rp.push_back((int64_t)cc.size());
        }
    }
    for (int64_t i = 0; i < np; ++i) plan.perm[(size_t)i] = plan.pinv[(size_t)i] = (int32_t)i;
    int rc = pack_slices(rp, cc, ss, o.threshold, o.vec, plan);
    if (rc) {
        destroy_batch(B);
        return rc;
    }
    // slice / group -> problem maps
    std::vector<int32_t> slice_prob((size_t)plan.n_slices), warp_prob((size_t)(np / 32));
    B->pslice.assign((size_t)count + 1, 0);
    B->pwarp.assign((size_t)count + 1, 0);
    {
        int j = 0;
        for (int64_t sl = 0; sl < plan.n_slices; ++sl) {
            const int64_t r0 = plan.meta[(size_t)sl * 4 + 2];
            while (r0 >= B->row_off[(size_t)j + 1]) B->pslice[(size_t)(++j)] = sl;
            slice_prob[(size_t)sl] = j;
        }
        while (j < count) B->pslice[(size_t)(++j)] = plan.n_slices;
        for (int p = 0; p < count; ++p) {
            B->pwarp[(size_t)p + 1] = B->row_off[(size_t)p + 1] / 32;
            for (int64_t g = B->row_off[(size_t)p] / 32; g < B->row_off[(size_t)p + 1] / 32; ++g)
                warp_prob[(size_t)g] = p;
        }
    }
    // the block-diagonal matrix as an ordinary SLICED handle
    fespmv_mat* M = new fespmv_mat();
    B->M = M;
    M->n = np;
    M->nnz = nnz_off[(size_t)count];
    M->format = FESPMV_FMT_SLICED;
    M->block = o.block;
    M->vec = o.vec;
    M->precisions = o.precisions | FESPMV_PREC_F64;
    std::vector<double> vals((size_t)std::max<int64_t>(M->nnz, 1));
    for (int j = 0; j < count; ++j)
        if (n_rows[j]) std::memcpy(vals.data() + nnz_off[(size_t)j], values[j], sizeof(double) * rowptr[j][n_rows[j]]);
    auto fail = [&](int code) { destroy_batch(B); return code; };
    if ((rc = device_alloc(M, (void**)&M->d_vals_in, sizeof(double) * M->nnz, "input values")) ||
        (rc = device_alloc(M, (void**)&M->d_diagpos, sizeof(int64_t) * np, "diagonal map")) ||
        (rc = device_alloc(M, (void**)&M->d_diag, sizeof(double) * np, "diagonal")))
        return fail(rc);
    if (cudaMemcpyAsync(M->d_vals_in, vals.data(), sizeof(double) * M->nnz, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "cudaMemcpyAsync"));
    if ((rc = upload_sliced(M, plan, s)) || (rc = alloc_scaled(M, plan.packed_len)) ||
        (rc = launch_fill_values(M, M->d_vals_in, s)))
        return fail(rc);
    if ((rc = device_alloc(M, (void**)&B->d_slice_prob, sizeof(int32_t) * plan.n_slices, "slice map")) ||
        (rc = device_alloc(M, (void**)&B->d_warp_prob, sizeof(int32_t) * (np / 32), "group map")) ||
        (rc = device_alloc(M, (void**)&B->d_pslice, sizeof(int64_t) * (count + 1), "problem slices")) ||
        (rc = device_alloc(M, (void**)&B->d_pwarp, sizeof(int64_t) * (count + 1), "problem groups")) ||
        (rc = device_alloc(M, (void**)&B->d_perm_g, sizeof(int32_t) * np, "batch permutation")) ||
        (rc = device_alloc(M, (void**)&B->d_pinv_g, sizeof(int32_t) * B->n_in, "batch inverse permutation")))
        return fail(rc);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(B->d_slice_prob, slice_prob.data(), sizeof(int32_t) * plan.n_slices, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_warp_prob, warp_prob.data(), sizeof(int32_t) * (np / 32), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_pslice, B->pslice.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_pwarp, B->pwarp.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_perm_g, perm_g.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_pinv_g, pinv_g.data(), sizeof(int32_t) * B->n_in, cudaMemcpyHostToDevice, s)) ||
        (e = cudaStreamSynchronize(s)))
        return fail(cuda_fail(e, "batch upload"));
    int bad = 0;
    if ((e = cudaMemcpy(&bad, M->d_flag, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(cuda_fail(e, "cudaMemcpy"));
    if (bad) {
        set_error("batch_create: every problem needs a positive, finite diagonal");
        return fail(FESPMV_ERR_INVALID_ARG);
    }
    cudaFree(M->d_vals_in);
    M->d_vals_in = nullptr;
    *out = B;
    return FESPMV_OK;
}

static int batch_ensure_work(fespmv_batch* B) {
    if (B->sc) return FESPMV_OK;
    fespmv_mat* M = B->M;
    const int64_t np = M->n, ng = np / 32;
    const size_t nd = sizeof(double) * (size_t)np, nf = sizeof(float) * (size_t)np;
    int rc;
    if ((rc = device_alloc(M, (void**)&B->x, nd, "batch x")) ||
        (rc = device_alloc(M, (void**)&B->b, nd, "batch b")) ||
        (rc = device_alloc(M, (void**)&B->q, std::max(nd, sizeof(double) * (size_t)B->n_in), "batch q")) ||
        (rc = device_alloc(M, (void**)&B->part, sizeof(double) * (size_t)std::max<int64_t>(M->n_slices, 3 * ng), "batch partial sums")) ||
        (rc = device_alloc(M, (void**)&B->w32, nf, "batch w")) ||
        (rc = device_alloc(M, (void**)&B->r32, nf, "batch r")) ||
        (rc = device_alloc(M, (void**)&B->p32, nf, "batch p")) ||
        (rc = device_alloc(M, (void**)&B->q32, nf, "batch q32")) ||
        (rc = device_alloc(M, (void**)&B->sc, sizeof(BScal) * B->count, "batch scalars")))
        return rc;
    FESPMV_CUDA(cudaMallocHost((void**)&B->h_sc, sizeof(BScal) * B->count));
    FESPMV_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
    return FESPMV_OK;
}

template <typename VT, int V>
static void launch_b_spmv(fespmv_batch* B, const VT* val, cudaStream_t s) {
    constexpr int U = (V == 4) ? 4 : 8;
    fespmv_mat* M = B->M;
    b_spmv32_dot<VT, V, U><<<grid_for(M->n_slices * 32, M->block), M->block, 0, s>>>(
        M->d_meta, M->d_col, val, B->p32, B->q32, M->n_slices, B->d_slice_prob, B->part, B->sc);
}

template <typename VT>
static void launch_b_spmv_v(fespmv_batch* B, const VT* val, cudaStream_t s) {
    switch (B->M->vec) {
        case 1: launch_b_spmv<VT, 1>(B, val, s); break;
        case 4: launch_b_spmv<VT, 4>(B, val, s); break;
        default: launch_b_spmv<VT, 2>(B, val, s); break;
    }
}

static void launch_b_inner(fespmv_batch* B, int bf16, cudaStream_t s) {
    fespmv_mat* M = B->M;
    const int64_t np = M->n;
    if (bf16)
        launch_b_spmv_v<__nv_bfloat16>(B, reinterpret_cast<const __nv_bfloat16*>(M->d_val16), s);
    else
        launch_b_spmv_v<float>(B, M->d_val32, s);
    b_finalize_pq<<<B->count, 256, 0, s>>>(B->part, B->d_pslice, B->sc);
    b_update32<<<grid_for(np, 256), 256, 0, s>>>(np, B->w32, B->r32, B->p32, B->q32, B->d_warp_prob,
                                                 B->part, B->sc);
    b_finalize_rr<<<B->count, 256, 0, s>>>(B->part, B->d_pwarp, B->sc);
    b_pupdate32<<<grid_for(np, 256), 256, 0, s>>>(np, B->p32, B->r32, B->d_warp_prob, B->sc);
}

static int batch_graph(fespmv_batch* B, int bf16, int chunk) {
    if (B->graph && B->graph_chunk == chunk && B->graph_bf16 == bf16) return FESPMV_OK;
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    FESPMV_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk; ++i) launch_b_inner(B, bf16, B->cap);
    cudaError_t e = cudaStreamEndCapture(B->cap, &g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&B->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    B->graph_chunk = chunk;
    B->graph_bf16 = bf16;
    return FESPMV_OK;
}

// The cluster solver's launch: as many clusters of kClusterCtas CTAs as are resident
// at once (at most one per problem), a work counter set to zero first.
template <typename VT, int V>
static int launch_cluster_t(fespmv_batch* B, const VT* val32, double tol2, double in2, int has_x0,
                            int max_iter, int max_outer, cudaStream_t s) {
    constexpr int U = (V == 4) ? 2 : (V == 2 ? 4 : 8);
    fespmv_mat* M = B->M;
    auto kernel = b_cluster_reliable<VT, V, U>;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0, csize = kClusterCtas;
    for (; csize >= 1; csize /= 2) {   // the largest cluster size the device places
        attr[0].val.clusterDim.x = csize;
        cfg.gridDim = dim3(csize);
        if (cudaOccupancyMaxActiveClusters(&clusters, (void*)kernel, &cfg) == cudaSuccess && clusters > 0) break;
        cudaGetLastError();
    }
    if (csize < 1 || clusters < 1) {
        set_error("batch_cg_solve: no thread-block cluster fits the device");
        return FESPMV_ERR_UNSUPPORTED;
    }
    clusters = std::min(clusters, (int)B->count);
    cfg.gridDim = dim3((unsigned)(clusters * csize));
    FESPMV_CUDA(cudaMemsetAsync(B->d_next, 0, sizeof(unsigned), s));
    FESPMV_CUDA(cudaLaunchKernelEx(&cfg, kernel, (const uint4*)M->d_meta, (const int32_t*)M->d_col, val32,
                                   (const double*)M->d_val, (const double*)M->d_scale, (const double*)B->b, B->x,
                                   B->q, B->w32, B->r32, B->p32, B->q32, (const int64_t*)B->d_pslice,
                                   (const int64_t*)B->d_pwarp, (const int32_t*)B->d_order, (int)B->count,
                                   B->d_next, B->sc, tol2, in2, has_x0, max_iter, max_outer));
    return FESPMV_OK;
}

template <typename VT>
static int launch_cluster_v(fespmv_batch* B, const VT* val32, double tol2, double in2, int has_x0, int max_iter,
                            int max_outer, cudaStream_t s) {
    switch (B->M->vec) {
        case 1: return launch_cluster_t<VT, 1>(B, val32, tol2, in2, has_x0, max_iter, max_outer, s);
        case 4: return launch_cluster_t<VT, 4>(B, val32, tol2, in2, has_x0, max_iter, max_outer, s);
        default: return launch_cluster_t<VT, 2>(B, val32, tol2, in2, has_x0, max_iter, max_outer, s);
    }
}

// Problems in decreasing order of their rows (the largest start first) and the
// work counter, on the first cluster solve.
static int ensure_cluster_work(fespmv_batch* B, cudaStream_t s) {
    if (B->d_order) return FESPMV_OK;
    std::vector<int32_t> order((size_t)B->count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) {
        return B->pwarp[(size_t)a + 1] - B->pwarp[(size_t)a] > B->pwarp[(size_t)c + 1] - B->pwarp[(size_t)c];
    });
    int rc;
    if ((rc = device_alloc(B->M, (void**)&B->d_order, sizeof(int32_t) * (size_t)B->count, "batch order")) ||
        (rc = device_alloc(B->M, (void**)&B->d_next, sizeof(unsigned), "batch work counter")))
        return rc;
    FESPMV_CUDA(cudaMemcpyAsync(B->d_order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice, s));
    FESPMV_CUDA(cudaStreamSynchronize(s));
    return FESPMV_OK;
}

static int read_bsc(fespmv_batch* B, cudaStream_t s) {
    FESPMV_CUDA(cudaMemcpyAsync(B->h_sc, B->sc, sizeof(BScal) * B->count, cudaMemcpyDeviceToHost, s));
    FESPMV_CUDA(cudaStreamSynchronize(s));
    return FESPMV_OK;
}

static int batch_solve_impl(fespmv_batch* B, const double* b, double* x, const cg_options* opts,
                            cg_result* res, cudaStream_t s) {
    cg_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.precision == FESPMV_CG_F64) o.precision = FESPMV_CG_F32_REFINE;
    int rc = normalize_options(o);
    if (rc) return rc;
    if (o.flags & (FESPMV_IO_PERMUTED | FESPMV_CG_NO_PRECOND | FESPMV_CG_FLEXIBLE)) {
        set_error("batch_cg_solve: IO_PERMUTED, NO_PRECOND and FLEXIBLE are not supported");
        return FESPMV_ERR_INVALID_ARG;
    }
    fespmv_mat* M = B->M;
    const int bf16 = o.precision == FESPMV_CG_BF16_REFINE ? 1 : 0;
    if ((bf16 && !M->d_val16) || (!bf16 && !M->d_val32)) {
        set_error("batch_cg_solve: the batch holds no %s copy", bf16 ? "BF16" : "FP32");
        return FESPMV_ERR_UNSUPPORTED;
    }
    if ((rc = batch_ensure_work(B)) || (rc = batch_graph(B, bf16, o.check_every))) return rc;
    const int64_t np = M->n, ng = np / 32;
    const bool host = o.flags & FESPMV_IO_HOST;
    const size_t nin = sizeof(double) * (size_t)B->n_in;
    // b (and x0) into the padded permuted layout
    const double* bsrc = b;
    if (host) {
        FESPMV_CUDA(cudaMemcpyAsync(B->q, b, nin, cudaMemcpyHostToDevice, s));
        bsrc = B->q;
    }
    gather_pad_f64<<<grid_for(np, 256), 256, 0, s>>>(bsrc, B->d_perm_g, B->b, np);
    const bool x0 = o.flags & FESPMV_CG_X0;
    if (x0) {
        const double* xsrc = x;
        if (host) {
            FESPMV_CUDA(cudaMemcpyAsync(B->q, x, nin, cudaMemcpyHostToDevice, s));
            xsrc = B->q;
        }
        gather_pad_f64<<<grid_for(np, 256), 256, 0, s>>>(xsrc, B->d_perm_g, B->x, np);
    } else {
        FESPMV_CUDA(cudaMemsetAsync(B->x, 0, sizeof(double) * (size_t)np, s));
    }
    for (int j = 0; j < B->count; ++j) {
        BScal z;
        std::memset(&z, 0, sizeof(z));
        z.status_out = CG_RUNNING;
        z.status_in = CG_CONVERGED;
        z.prev = INFINITY;
        z.max_iter = o.max_iter;
        z.max_outer = o.max_outer;
        B->h_sc[j] = z;
    }
    FESPMV_CUDA(cudaMemcpyAsync(B->sc, B->h_sc, sizeof(BScal) * B->count, cudaMemcpyHostToDevice, s));
    const double tol2 = o.tol * o.tol, in2 = o.inner_tol * o.inner_tol;
    const int reliable = (o.flags & FESPMV_CG_RELIABLE) ? 1 : 0;
    const int64_t max_graphs = (int64_t)o.max_iter / o.check_every + 3;
    if (reliable) {   // every problem to the end in one launch of thread-block clusters
        if ((rc = ensure_cluster_work(B, s))) return rc;
        rc = bf16 ? launch_cluster_v<__nv_bfloat16>(B, reinterpret_cast<const __nv_bfloat16*>(M->d_val16), tol2, in2,
                                                      x0 ? 1 : 0, o.max_iter, o.max_outer, s)
                  : launch_cluster_v<float>(B, M->d_val32, tol2, in2, x0 ? 1 : 0, o.max_iter, o.max_outer, s);
        if (rc) return rc;
        if ((rc = read_bsc(B, s))) return rc;
    }
    for (int step = 0; !reliable; ++step) {
        const bool ax = x0 || step > 0;
        if (ax && (rc = launch_spmv(M, B->x, B->q, s))) return rc;
        b_residual<<<grid_for(np, 256), 256, 0, s>>>(np, B->b, ax ? B->q : nullptr, M->d_scale, B->w32,
                                                     B->r32, B->p32, B->d_warp_prob, B->part, ng, reliable,
                                                     B->sc);
        b_finalize_res<<<B->count, 256, 0, s>>>(B->part, ng, B->d_pwarp, B->sc, tol2, in2, reliable);
        // reliable updates: the kept directions take the replaced residuals (beta = 0 at the
        // first step, where p = r_in already)
        if (reliable) b_pupdate32<<<grid_for(np, 256), 256, 0, s>>>(np, B->p32, B->r32, B->d_warp_prob, B->sc);
        FESPMV_CUDA(cudaGetLastError());
        if ((rc = read_bsc(B, s))) return rc;
        bool any = false;
        for (int j = 0; j < B->count; ++j) any |= B->h_sc[j].status_in == CG_RUNNING;
        if (!any) break;
        for (int64_t k = 0; k < max_graphs; ++k) {
            FESPMV_CUDA(cudaGraphLaunch(B->graph, s));
            if ((rc = read_bsc(B, s))) return rc;
            bool running = false;
            for (int j = 0; j < B->count; ++j) running |= B->h_sc[j].status_in == CG_RUNNING;
            if (!running) break;
        }
        b_xupdate<<<grid_for(np, 256), 256, 0, s>>>(np, B->x, M->d_scale, B->w32, B->d_warp_prob, B->sc);
        b_outer_count<<<(B->count + 255) / 256, 256, 0, s>>>(B->count, B->sc);
        FESPMV_CUDA(cudaGetLastError());
    }
    // x back to the input numbering
    double* xdst = host ? B->q : x;
    gather_pad_f64<<<grid_for(B->n_in, 256), 256, 0, s>>>(B->x, B->d_pinv_g, xdst, B->n_in);
    FESPMV_CUDA(cudaGetLastError());
    if (host) FESPMV_CUDA(cudaMemcpyAsync(x, B->q, nin, cudaMemcpyDeviceToHost, s));
    FESPMV_CUDA(cudaStreamSynchronize(s));
    int worst = FESPMV_OK;
    for (int j = 0; j < B->count; ++j) {
        const BScal& h = B->h_sc[j];
        const int st = h.status_out == CG_CONVERGED ? FESPMV_OK
                     : h.status_out == CG_BREAKDOWN ? FESPMV_ERR_BREAKDOWN : FESPMV_ERR_NOT_CONVERGED;
        if (st != FESPMV_OK && worst == FESPMV_OK) worst = st;
        if (res) {
            res[j].status = st;
            res[j].iters = h.iters;
            res[j].restarts = 0;
            res[j].outer = h.outer;
            res[j].relres = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
            res[j].true_relres = res[j].relres;
        }
    }
    if (worst != FESPMV_OK) set_error("batch_cg_solve: at least one problem did not converge");
    return worst;
}

}  // namespace fespmv

using namespace fespmv;

extern "C" {

int batch_create(fespmv_batch_t* out, int32_t count, const int64_t* n_rows,
                 const int64_t* const* rowptr, const int32_t* const* colind,
                 const double* const* values, const fespmv_mesh_info* mesh,
                 const fespmv_options* opts, fespmv_stream_t stream) {
    try {
        return batch_create_impl(out, count, n_rows, rowptr, colind, values, mesh, opts,
                                 (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FESPMV_ERR_OOM;
    } catch (...) {
        set_error("unexpected C++ exception");
        return FESPMV_ERR_INVALID_ARG;
    }
}

void batch_destroy(fespmv_batch_t B) {
    try {
        destroy_batch(B);
    } catch (...) {
    }
}

int batch_spmv(fespmv_batch_t B, const double* x, double* y, fespmv_stream_t stream) {
    if (!B || (B->n_in > 0 && (!x || !y))) {
        set_error("null argument");
        return FESPMV_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    fespmv_mat* M = B->M;
    if (M->n == 0) return FESPMV_OK;
    gather_pad_f64<<<grid_for(M->n, 256), 256, 0, s>>>(x, B->d_perm_g, M->d_xp, M->n);
    int rc = launch_spmv(M, M->d_xp, M->d_yp, s);
    if (rc) return rc;
    gather_pad_f64<<<grid_for(B->n_in, 256), 256, 0, s>>>(M->d_yp, B->d_pinv_g, y, B->n_in);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

int batch_cg_solve(fespmv_batch_t B, const double* b, double* x, const cg_options* opts,
                   cg_result* results, fespmv_stream_t stream) {
    try {
        if (!B || (B->n_in > 0 && (!b || !x))) {
            set_error("null argument");
            return FESPMV_ERR_INVALID_ARG;
        }
        return batch_solve_impl(B, b, x, opts, results, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FESPMV_ERR_OOM;
    } catch (...) {
        set_error("unexpected C++ exception");
        return FESPMV_ERR_INVALID_ARG;
    }
}

int batch_get_info(fespmv_batch_t B, fespmv_info* info, int64_t* padded_rows) {
    if (!B || !info) {
        set_error("null argument");
        return FESPMV_ERR_INVALID_ARG;
    }
    int rc = spmv_get_info(B->M, info);
    info->n_rows = B->n_in;
    if (padded_rows) *padded_rows = B->M->n;
    return rc;
}

}  // extern "C"
