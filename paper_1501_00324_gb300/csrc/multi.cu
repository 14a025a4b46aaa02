// Products with many right-hand sides sharing one pass over the matrix
// (spmv_apply_multi in fespmv.h): Y = A X, X and Y row-major n x k, k <= 32.
//
// One warp walks one K1 slice (32 rows, one lane per row in the layout of
// Sec. 5.1).  Instead of each lane reading its own row's entry, the whole warp
// reads a chunk of the slice (32*V entries: V steps of all 32 rows) with
// uniform vector loads -- every lane fetches the same 16 bytes, one L1
// wavefront per load -- and then lane j applies every entry to right-hand side
// j: acc[row] += a * X[c][j].  A row of X is k contiguous values, so each
// gather is one coalesced 128 B (FP32) or 256 B (FP64) access, and the matrix
// is streamed from HBM once for all k columns.  The entry -> row mapping of a
// chunk is fixed at compile time (row = e / V), so the 32 accumulators stay in
// registers.
#include <cuda_runtime.h>

#include <type_traits>

#include "internal.h"
#include "spmv_device.cuh"

namespace fespmv {

template <typename T> struct U16;   // 16-byte uniform loads
template <> struct U16<double> { using type = double2; static constexpr int n = 2; };
template <> struct U16<float> { using type = float4; static constexpr int n = 4; };

template <typename VT, typename XT, int V>
__global__ void __launch_bounds__(128) sliced_multi(const uint4* __restrict__ meta,
                                                    const int32_t* __restrict__ col,
                                                    const VT* __restrict__ val,
                                                    const XT* __restrict__ X, XT* __restrict__ Y,
                                                    int64_t n_slices, int64_t n, int k) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_slices) return;
    const uint4 m = meta[warp];
    const int64_t off = (int64_t)m.x * 32;
    const int w = (int)m.y;
    const bool active = lane < k;
    XT acc[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) acc[r] = XT(0);
    constexpr int NV = U16<VT>::n;
    using VV = typename U16<VT>::type;
    for (int s = 0; s < w; s += V) {
        const VT* vp = val + off + (int64_t)s * 32;
        const int32_t* cp = col + off + (int64_t)s * 32;
#pragma unroll
        for (int e0 = 0; e0 < 32 * V; e0 += 4) {
            const int4 c4 = ld_stream(reinterpret_cast<const int4*>(cp + e0));
            VT v[4];
#pragma unroll
            for (int h = 0; h < 4; h += NV) {
                const VV t = ld_stream(reinterpret_cast<const VV*>(vp + e0 + h));
                if constexpr (NV == 2) {
                    v[h] = t.x; v[h + 1] = t.y;
                } else {
                    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
                }
            }
            const int32_t cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int e = e0 + h;
                if (cc[h] >= 0 && active)
                    acc[e / V] = fma((XT)v[h], __ldg(X + (int64_t)cc[h] * k + lane), acc[e / V]);
            }
        }
    }
    if (active) {
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const int64_t row = (int64_t)m.z + r;
            if (row < n) Y[row * k + lane] = acc[r];
        }
    }
}

// Y[i, :] = X[idx[i], :] for k columns.
template <typename XT>
__global__ void gather_rows(const XT* __restrict__ X, const int32_t* __restrict__ idx,
                            XT* __restrict__ Y, int64_t n, int k) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n * k) {
        const int64_t i = t / k;
        const int j = (int)(t % k);
        Y[t] = X[(int64_t)idx[i] * k + j];
    }
}

template <typename VT, typename XT>
static void launch_multi(const fespmv_mat* A, const VT* val, const XT* X, XT* Y, int k, cudaStream_t s) {
    const unsigned g = grid_for(A->n_slices * 32, 128);
    switch (A->vec) {
        case 1: sliced_multi<VT, XT, 1><<<g, 128, 0, s>>>(A->d_meta, A->d_col, val, X, Y, A->n_slices, A->n, k); break;
        case 4: sliced_multi<VT, XT, 4><<<g, 128, 0, s>>>(A->d_meta, A->d_col, val, X, Y, A->n_slices, A->n, k); break;
        default: sliced_multi<VT, XT, 2><<<g, 128, 0, s>>>(A->d_meta, A->d_col, val, X, Y, A->n_slices, A->n, k); break;
    }
}

static int ensure_multi_scratch(fespmv_mat* A) {
    if (A->d_xk) return FESPMV_OK;
    const size_t bytes = sizeof(double) * 32 * (size_t)A->n;
    int rc = device_alloc(A, (void**)&A->d_xk, bytes, "multi-RHS x scratch");
    if (!rc) rc = device_alloc(A, (void**)&A->d_yk, bytes, "multi-RHS y scratch");
    return rc;
}

template <typename XT>
static int apply_multi_t(fespmv_mat* A, const XT* X, XT* Y, int k, int precision, int flags,
                         cudaStream_t s) {
    const bool permute = !(flags & FESPMV_IO_PERMUTED);
    const XT* xs = X;
    XT* ys = Y;
    if (permute) {
        int rc = ensure_multi_scratch(A);
        if (rc) return rc;
        xs = reinterpret_cast<const XT*>(A->d_xk);
        ys = reinterpret_cast<XT*>(A->d_yk);
        gather_rows<XT><<<grid_for(A->n * k, 256), 256, 0, s>>>(X, A->d_perm, const_cast<XT*>(xs), A->n, k);
    }
    (void)precision;
    if constexpr (std::is_same<XT, double>::value)
        launch_multi<double, double>(A, A->d_val, xs, ys, k, s);     // FP64 values and sums
    else
        launch_multi<float, float>(A, A->d_val32, xs, ys, k, s);     // FP32 copy of S A S
    if (permute) gather_rows<XT><<<grid_for(A->n * k, 256), 256, 0, s>>>(ys, A->d_pinv, Y, A->n, k);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

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
        if (A->format != FESPMV_FMT_SLICED || A->max_lanes_log2 != 0) {
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
            return apply_multi_t<double>(A, (const double*)X, (double*)Y, k, precision, flags, s);
        return apply_multi_t<float>(A, (const float*)X, (float*)Y, k, precision, flags, s);
    } catch (...) {
        set_error("unexpected C++ exception");
        return FESPMV_ERR_INVALID_ARG;
    }
}
