// The reliable-update refinement of a small handle in one launch of one
// thread-block cluster.
//
// A graph iteration of the refined solve costs three kernel boundaries; on a
// problem of a few thousand rows they cost more than the iteration's work (20 us
// per inner step on 8,000 rows).  Here the whole solve runs in one cluster of
// kClusterCtas CTAs that synchronise with hardware cluster barriers and reduce
// through distributed shared memory (cluster_device.cuh): 14 us per step.  Larger
// handles keep the graphs: a cluster's 64 warps walk their share of the slices
// one after another, which on 30,000 rows already costs more than the graphs'
// boundaries.  The solve server takes the same path for the same handles, so a
// result is the same alone and in the mix.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "cg_run.h"
#include "cluster_device.cuh"
#include "internal.h"

namespace fespmv {

template <typename VT, int V, int U>
__global__ void __launch_bounds__(kClusterThreads, 2) cl_solve_reliable(
    const uint4* __restrict__ meta, const int32_t* __restrict__ col, const VT* __restrict__ val32,
    const double* __restrict__ val64, const double* __restrict__ scale, const double* __restrict__ b,
    double* __restrict__ x, double* __restrict__ q64, float* __restrict__ w, float* __restrict__ rin,
    float* __restrict__ p, float* __restrict__ q32, int64_t n_slices, int64_t n, double tol2, double in2,
    int has_x0, int max_iter, int max_outer, CgScalars* sc) {
    // S needs a positive diagonal (the copy flag cg_copy_flag left in pad)
    if (*reinterpret_cast<const volatile int*>(&sc->pad)) return;
    cgx::cluster_group cl = cgx::this_cluster();
    __shared__ ClusterRed red;
    int turn = 0;
    const ClusterOut o = cluster_reliable<VT, V, U>(cl, red, turn, meta, col, val32, val64, scale, b, x, q64, w, rin,
                                                    p, q32, 0, n_slices, 0, n, tol2, in2, has_x0, max_iter, max_outer);
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
        sc->status = o.status;
        sc->iters = o.iters;
        sc->rr = o.rr;
        sc->bb = o.bb;
        sc->true_rr = o.true_rr;
        sc->thresh2 = tol2 * o.bb;
        sc->iters_in = o.outer;
    }
    cl.sync();
}

namespace {

template <typename Kernel, typename... Args>
int launch_one_cluster(Kernel kernel, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(kClusterCtas);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FESPMV_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
    return FESPMV_OK;
}

template <typename VT, int V>
int cluster_rel_v(const fespmv_mat* A, CgWork* w, const VT* val32, double tol2, double in2, int has_x0,
                  int max_iter, int max_outer, cudaStream_t s) {
    constexpr int U = (V == 4) ? 2 : (V == 2 ? 4 : 8);
    return launch_one_cluster(cl_solve_reliable<VT, V, U>, s, (const uint4*)A->d_meta, (const int32_t*)A->d_col,
                              val32, (const double*)A->d_val, (const double*)A->d_scale, (const double*)w->b, w->x,
                              w->q, w->w32, w->r32, w->p32, w->q32, A->n_slices, A->n, tol2, in2, has_x0,
                              max_iter, max_outer, w->sc);
}

}  // namespace

int launch_cluster_cg_reliable(const fespmv_mat* A, CgWork* w, int bf16, double tol2, double in2, int has_x0,
                               int max_iter, int max_outer, cudaStream_t s) {
    if (bf16) {
        const __nv_bfloat16* v = reinterpret_cast<const __nv_bfloat16*>(A->d_val16);
        switch (A->vec) {
            case 1: return cluster_rel_v<__nv_bfloat16, 1>(A, w, v, tol2, in2, has_x0, max_iter, max_outer, s);
            case 4: return cluster_rel_v<__nv_bfloat16, 4>(A, w, v, tol2, in2, has_x0, max_iter, max_outer, s);
            default: return cluster_rel_v<__nv_bfloat16, 2>(A, w, v, tol2, in2, has_x0, max_iter, max_outer, s);
        }
    }
    switch (A->vec) {
        case 1: return cluster_rel_v<float, 1>(A, w, A->d_val32, tol2, in2, has_x0, max_iter, max_outer, s);
        case 4: return cluster_rel_v<float, 4>(A, w, A->d_val32, tol2, in2, has_x0, max_iter, max_outer, s);
        default: return cluster_rel_v<float, 2>(A, w, A->d_val32, tol2, in2, has_x0, max_iter, max_outer, s);
    }
}

}  // namespace fespmv
