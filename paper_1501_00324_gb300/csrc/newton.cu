// Newton updates on a fixed sparsity pattern (fe_newton_step, fe_newton_solve).
//
// Sec. 2 of the paper advances the monodomain model by backward Euler; every
// time step runs a global Newton iteration whose update assembles the element
// tangents and residuals into the global K and R (Sec. 4: as sparse products
// with a vector of ones), solves K dx = R with Jacobi-preconditioned CG and sets
// phi <- phi - dx (the algorithm table of Sec. 2).  The pattern of K never
// changes, so every step reuses the handle, its layout and the assembly map;
// only values, R and the solve are new.  The element quantities themselves are
// the caller's physics (here a callback), which this library does not model.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "internal.h"

namespace fespmv {
namespace {

constexpr int kNewtonBlocks = 256;
constexpr int kNewtonThreads = 256;

// Per-block sums of a.a (fixed order: grid-stride sums per thread, then a
// shared-memory tree), written to partial[blockIdx.x].
__device__ __forceinline__ void block_tree(double v, double* partial) {
    __shared__ double sh[kNewtonThreads];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = kNewtonThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *partial = sh[0];
}

__global__ void __launch_bounds__(kNewtonThreads) newton_sq(const double* __restrict__ a, int64_t n,
                                                            double* __restrict__ partial) {
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kNewtonThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kNewtonThreads)
        v = fma(a[i], a[i], v);
    block_tree(v, partial + blockIdx.x);
}

// phi -= dx (when phi is given) and the per-block sums of dx.dx.
__global__ void __launch_bounds__(kNewtonThreads) newton_apply(double* __restrict__ phi,
                                                               const double* __restrict__ dx, int64_t n,
                                                               double* __restrict__ partial) {
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kNewtonThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kNewtonThreads) {
        const double d = dx[i];
        if (phi) phi[i] = phi[i] - d;
        v = fma(d, d, v);
    }
    block_tree(v, partial + blockIdx.x);
}

// One block adds the partial sums in block order.
__global__ void newton_total(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += partial[b];
        *out = s;
    }
}

struct Scratch {
    double* d = nullptr;   // kNewtonBlocks partial sums + 1 total
    ~Scratch() {
        if (d) cudaFree(d);
    }
};

int norm2(const double* a, int64_t n, bool apply_to_phi, double* phi, Scratch& w, double* out, cudaStream_t s) {
    const unsigned g = std::max(1u, std::min((unsigned)kNewtonBlocks, grid_for(n, kNewtonThreads)));
    if (apply_to_phi)
        newton_apply<<<g, kNewtonThreads, 0, s>>>(phi, a, n, w.d);
    else
        newton_sq<<<g, kNewtonThreads, 0, s>>>(a, n, w.d);
    newton_total<<<1, 32, 0, s>>>(w.d, (int)g, w.d + kNewtonBlocks);
    FESPMV_CUDA(cudaGetLastError());
    double h = 0.0;
    FESPMV_CUDA(cudaMemcpyAsync(&h, w.d + kNewtonBlocks, sizeof(double), cudaMemcpyDeviceToHost, s));
    FESPMV_CUDA(cudaStreamSynchronize(s));
    *out = std::sqrt(h);
    return FESPMV_OK;
}

int step_impl(fespmv_assembly_t P, const double* Ke, const double* Re, double* R, double* dx, double* phi,
              const cg_options* opts, cg_result* res, double* r_norm, double* dx_norm, Scratch& w,
              cudaStream_t s, bool r_ready) {
    fespmv_mat* A = assembly_handle(P);
    const int64_t n = A->n;
    int rc;
    if (!r_ready) {
        if ((rc = assembly_vector(P, Re, R, 0, (fespmv_stream_t)s))) return rc;
        if ((rc = norm2(R, n, false, nullptr, w, r_norm, s))) return rc;
    }
    if ((rc = assembly_matrix(P, Ke, 0, (fespmv_stream_t)s))) return rc;
    cg_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.flags & (FESPMV_IO_HOST | FESPMV_IO_PERMUTED)) {
        set_error("Newton updates take device vectors in the input numbering");
        return FESPMV_ERR_INVALID_ARG;
    }
    rc = cg_solve(A, R, dx, &o, res, (fespmv_stream_t)s);
    if (rc) return rc;
    return norm2(dx, n, true, phi, w, dx_norm, s);
}

int alloc_scratch(Scratch& w) {
    cudaError_t e = cudaMalloc(&w.d, sizeof(double) * (kNewtonBlocks + 1));
    if (e != cudaSuccess) {
        w.d = nullptr;
        set_error("cudaMalloc for the Newton norms failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? FESPMV_ERR_OOM : FESPMV_ERR_CUDA;
    }
    return FESPMV_OK;
}

bool bad_vectors(fespmv_assembly_t P, const void* a, const void* b, const void* c) {
    fespmv_mat* A = assembly_handle(P);
    return !A || (A->n > 0 && (!a || !b || !c));
}

}  // namespace
}  // namespace fespmv

using namespace fespmv;

extern "C" {

int fe_newton_step(fespmv_assembly_t P, const double* Ke, const double* Re, double* R, double* dx, double* phi,
                   const cg_options* opts, fe_newton_result* out, fespmv_stream_t stream) {
    try {
        if (!P || bad_vectors(P, Re, R, dx) || (assembly_handle(P)->n > 0 && !Ke)) {
            set_error("fe_newton_step: null argument");
            return FESPMV_ERR_INVALID_ARG;
        }
        fe_newton_result r;
        std::memset(&r, 0, sizeof(r));
        Scratch w;
        int rc = alloc_scratch(w);
        if (!rc) rc = step_impl(P, Ke, Re, R, dx, phi, opts, &r.last_cg, &r.res_norm, &r.dx_norm, w,
                                (cudaStream_t)stream, false);
        r.steps = rc ? 0 : 1;
        r.res_norm0 = r.res_norm;
        r.cg_iters = r.last_cg.iters;
        r.status = rc;
        if (out) *out = r;
        return rc;
    } catch (...) {
        set_error("unexpected C++ exception");
        return FESPMV_ERR_INVALID_ARG;
    }
}

int fe_newton_solve(fespmv_assembly_t P, double* phi, fe_element_fn element_fn, void* user, double* Ke,
                    double* Re, double* R, double* dx, double newton_tol, int32_t max_steps,
                    const cg_options* opts, fe_newton_result* out, fespmv_stream_t stream) {
    try {
        if (!P || !element_fn || bad_vectors(P, phi, R, dx) || bad_vectors(P, Ke, Re, R) || !(newton_tol >= 0.0) ||
            max_steps < 1) {
            set_error("fe_newton_solve: bad argument");
            return FESPMV_ERR_INVALID_ARG;
        }
        cudaStream_t s = (cudaStream_t)stream;
        fe_newton_result r;
        std::memset(&r, 0, sizeof(r));
        r.status = FESPMV_ERR_NOT_CONVERGED;
        Scratch w;
        int rc = alloc_scratch(w);
        for (int k = 0; !rc; ++k) {
            const int cb = element_fn(phi, Ke, Re, user, stream);
            if (cb) {
                set_error("fe_newton_solve: the element callback returned %d", cb);
                rc = FESPMV_ERR_INVALID_ARG;
                break;
            }
            // the residual of the current phi decides whether another update is due
            if ((rc = assembly_vector(P, Re, R, 0, stream))) break;
            double rn = 0.0;
            if ((rc = norm2(R, assembly_handle(P)->n, false, nullptr, w, &rn, s))) break;
            if (k == 0) r.res_norm0 = rn;
            r.res_norm = rn;
            if (rn <= newton_tol * r.res_norm0 || rn == 0.0) {
                r.status = FESPMV_OK;
                break;
            }
            if (k == max_steps) break;
            if ((rc = step_impl(P, Ke, Re, R, dx, phi, opts, &r.last_cg, &rn, &r.dx_norm, w, s, true))) break;
            r.steps += 1;
            r.cg_iters += r.last_cg.iters;
        }
        if (rc) r.status = rc;
        if (out) *out = r;
        if (!rc && r.status == FESPMV_ERR_NOT_CONVERGED)
            set_error("Newton stopped after %d updates with ||R|| / ||R_0|| = %g", r.steps,
                      r.res_norm0 > 0 ? r.res_norm / r.res_norm0 : 0.0);
        return r.status;
    } catch (...) {
        set_error("unexpected C++ exception");
        return FESPMV_ERR_INVALID_ARG;
    }
}

}  // extern "C"
