// Host-side types of the CG solver shared by cg.cu and the solve server.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace fespmv {

enum : int { CG_RUNNING = 0, CG_CONVERGED = 1, CG_BREAKDOWN = 2, CG_MAXITER = 3, CG_BADDIAG = 4 };

struct CgScalars {
    double rho, pq, alpha, beta, rr, bb, thresh2, true_rr;
    int iters, max_iter, status, pad;
    unsigned int counters[1];    // grid_sum's arrival counter (zero between kernels)
    unsigned int pad2;
    double thresh_in;   // refinement: inner stop threshold on r_in.r_in
    int iters_in, first; // refinement: inner steps of the current outer step; single-reduction: first step
};

struct CgWork {
    int64_t n = 0;
    double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *b = nullptr, *dinv = nullptr;
    double* partials = nullptr;
    CgScalars* sc = nullptr;
    CgScalars* sc_in = nullptr;   // flexible CG: the inner (low-precision) CG's scalars
    CgScalars* h_sc = nullptr;  // pinned host mirror, 2 slots
    unsigned upd_grid = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_chunk = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // refinement (float inner CG): w, r_in, p, q
    float *w32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    cudaGraphExec_t graph_low[2] = {nullptr, nullptr};  // FP32, BF16 inner iterations
    int chunk_low[2] = {0, 0};
    cudaGraphExec_t graph_flex[2] = {nullptr, nullptr}; // flexible CG outer steps, FP32 / BF16 inner
    int chunk_flex[2] = {0, 0}, steps_flex[2] = {0, 0};
    double* h_io = nullptr;     // pinned host staging of n doubles (solve server)
    float2* pdf = nullptr;      // float-pair split of p (handles with FESPMV_PREC_DF64)
    double *u = nullptr, *s = nullptr;  // single-reduction CG: u = D^-1 r, s = A p
    cudaGraphExec_t graph_cg1 = nullptr;
    int chunk_cg1 = 0;
    int64_t bytes = 0;          // device bytes held
};

// One solve in flight (see the host side below).
struct CgRun {
    fespmv_mat* A = nullptr;
    CgWork* w = nullptr;
    cudaStream_t s = nullptr;
    cg_options o{};
    bool permute = false, has_x0 = false, out_host = false;
    double* x_out = nullptr;
    int phase = 5;             // PH_DONE
    int restarts = 0, outer = 0;
    double prev = 0.0;
    int64_t graphs_left = 0;
    int queued = 0, head = 0;
    int status = 0, error = 0;
    cudaGraphExec_t graph = nullptr;
    CgScalars last{};
};

enum Phase { PH_INIT_WAIT, PH_ITER, PH_TRUE_WAIT, PH_RES_WAIT, PH_OUT_WAIT, PH_DONE, PH_CLUSTER_WAIT };

// Handles with at most this many rows run reliable-update refinement in one
// cluster launch (cluster_cg.cu).
constexpr int64_t kClusterSolveMaxRows = 16384;
int launch_cluster_cg_reliable(const fespmv_mat* A, CgWork* w, int bf16, double tol2, double in2, int has_x0,
                               int max_iter, int max_outer, cudaStream_t s);

// Workspace for one solve of A (vectors, partial sums, scalars, graphs, stream
// for capture, events; pinned staging of n doubles when host_staging).
int create_work(const fespmv_mat* A, bool host_staging, CgWork** out);
void destroy_work(CgWork* w);
int64_t work_bytes(const fespmv_mat* A, bool refine);
int ensure_low_work(CgWork* w);  // float vectors of the refined precisions
int normalize_options(cg_options& o);
int check_precision(const fespmv_mat* A, int precision);
// Stage b (and x0) into the run's workspace (host = pointers are host memory).
int stage_inputs(CgRun& r, const double* b, const double* x0, bool host);
// Enqueue the start of the solve; then advance with run_step until PH_DONE.
int run_begin(CgRun& r);
int run_step(CgRun& r, bool block, bool* progress);
int run_result(const CgRun& r, cg_result* res);

}  // namespace fespmv
