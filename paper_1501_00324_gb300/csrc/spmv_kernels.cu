// SpMV kernels for sm_103a: CSR scalar / vector baselines and the FE warp-slice
// kernel, plus the gathers that move vectors and values between numberings.
//
// CSR scalar (Sec. 4, CSR: the one-thread-per-row alternative) and CSR vector
// (Sec. 4, CSR: lanes of a warp share a row and reduce inside the warp) are the
// baselines.  The warp-slice kernel executes the K1/K2 layout of Sec. 5.1 and
// Sec. 5.4 in the renumbered space of Sec. 5.2/5.3 (no remap on store):
//   - one warp per slice; lane l works on local row l >> log2T;
//   - the slice's values and column indices are read column-major, so a step of
//     the warp reads 32*V consecutive entries (V entries per lane, one 8*V-byte
//     value load and one 4*V-byte index load per lane);
//   - x is gathered through the read-only path and stays L1/L2 resident;
//   - lanes of one row combine with __shfl_down_sync (the paper's K2 used a
//     warp-synchronous volatile shared-memory tree, which is unsafe under
//     independent thread scheduling on Volta and later);
//   - padding entries carry column -1 and contribute nothing.
#include <cuda_runtime.h>

#include "internal.h"
#include "spmv_device.cuh"

namespace fespmv {

// ---------------------------------------------------------------- CSR baselines

template <int L>
__global__ void csr_f64(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                        const double* __restrict__ val, const double* __restrict__ x,
                        double* __restrict__ y, int64_t n) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = t / L;
    const int sub = (int)(t % L);
    double sum = csr_row_sum_f64<L>(row, sub, n, rowptr, col, val, x);
    if (row < n && sub == 0) y[row] = sum;
}

// ---------------------------------------------------------------- warp slices

template <int V, int U>
__global__ void __launch_bounds__(256) sliced_f64(const uint4* __restrict__ meta,
                                                  const int32_t* __restrict__ col,
                                                  const double* __restrict__ val,
                                                  const double* __restrict__ x,
                                                  double* __restrict__ y, int64_t n_slices,
                                                  int64_t n) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_slices) return;          // whole warps leave together
    const uint4 m = meta[warp];
    const double sum = sliced_row_sum_f64<V, U>(m, col, val, x, lane);
    const int lt = (int)m.w;
    const int64_t row = (int64_t)m.z + (lane >> lt);
    if ((lane & ((1 << lt) - 1)) == 0 && row < n) y[row] = sum;
}

// ---------------------------------------------------------------- float-pair FP64 product

template <int V, int U>
__global__ void __launch_bounds__(256, 8) sliced_df64(const uint4* __restrict__ meta,
                                                   const int32_t* __restrict__ col,
                                                   const float2* __restrict__ vdf,
                                                   const double* __restrict__ val,
                                                   const float2* __restrict__ xs,
                                                   const double* __restrict__ x,
                                                   double* __restrict__ y, int64_t n_slices, int64_t n) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_slices) return;
    const uint4 m = meta[warp];
    const double sum = sliced_row_sum_df<V, U>(m, col, vdf, val, xs, x, lane);
    const int lt = (int)m.w;
    const int64_t row = (int64_t)m.z + (lane >> lt);
    if ((lane & ((1 << lt) - 1)) == 0 && row < n) y[row] = sum;
}

__global__ void split_df(const double* __restrict__ v, float2* __restrict__ out, int64_t len) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < len) out[i] = df_split(v[i]);
}

// xp[i] = x[idx[i]] and its float-pair split, in one pass.
__global__ void gather_split_df(const double* __restrict__ x, const int32_t* __restrict__ idx,
                                double* __restrict__ xp, float2* __restrict__ xs, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const double v = __ldg(x + idx[i]);
        xp[i] = v;
        xs[i] = df_split(v);
    }
}

// ---------------------------------------------------------------- low precision (B = S A S)

template <typename VT, int V, int U>
__global__ void __launch_bounds__(256) sliced_low(const uint4* __restrict__ meta,
                                                  const int32_t* __restrict__ col,
                                                  const VT* __restrict__ val,
                                                  const float* __restrict__ x,
                                                  float* __restrict__ y, int64_t n_slices, int64_t n) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_slices) return;
    const uint4 m = meta[warp];
    const float sum = sliced_row_sum_low<VT, V, U>(m, col, val, x, lane);
    const int lt = (int)m.w;
    const int64_t row = (int64_t)m.z + (lane >> lt);
    if ((lane & ((1 << lt) - 1)) == 0 && row < n) y[row] = sum;
}

template <typename VT, int L>
__global__ void csr_low(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                        const VT* __restrict__ val, const float* __restrict__ x,
                        float* __restrict__ y, int64_t n) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = t / L;
    const int sub = (int)(t % L);
    const float sum = csr_row_sum_low<VT, L>(row, sub, n, rowptr, col, val, x);
    if (row < n && sub == 0) y[row] = sum;
}

// S = diag(A)^-1/2; a non-positive or non-finite diagonal sets *bad.
__global__ void scale_from_diag(const double* __restrict__ diag, double* __restrict__ scale,
                                int64_t n, int* bad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const double d = diag[i];
        if (d > 0.0 && isfinite(d)) {
            scale[i] = 1.0 / sqrt(d);
        } else {
            scale[i] = 0.0;
            *bad = 1;
        }
    }
}

__device__ __forceinline__ void store_low(float b, float* f32, uint16_t* b16, int64_t pos) {
    if (f32) f32[pos] = b;
    if (b16) b16[pos] = __bfloat16_as_ushort(__float2bfloat16_rn(b));
}

// B = S A S entry by entry: b = (float)((s_row * a) * s_col), padding stays 0.
template <int V>
__global__ void build_scaled_sliced(const uint4* __restrict__ meta, const int32_t* __restrict__ col,
                                   const double* __restrict__ val, const double* __restrict__ scale,
                                   float* __restrict__ f32, uint16_t* __restrict__ b16, int64_t n_slices) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_slices) return;
    const uint4 m = meta[warp];
    const int64_t off = (int64_t)m.x * 32;
    const int64_t row = (int64_t)m.z + (lane >> m.w);
    const double sr = scale[row];
    // steps are independent: unrolled, a warp keeps several column -> scale gathers in flight
#pragma unroll 4
    for (int st = 0; st < (int)m.y; ++st) {
        const int64_t pos = off + (int64_t)(st / V) * 32 * V + lane * V + st % V;
        const int32_t c = col[pos];
        const float b = c >= 0 ? (float)((sr * val[pos]) * scale[c]) : 0.0f;
        store_low(b, f32, b16, pos);
    }
}

__global__ void build_scaled_csr(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, const double* __restrict__ scale,
                                 float* f32, uint16_t* b16, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            store_low((float)((scale[i] * val[p]) * scale[col[p]]), f32, b16, p);
}

// ---------------------------------------------------------------- gathers

__global__ void gather_f64(const double* __restrict__ in, const int32_t* __restrict__ idx,
                           double* __restrict__ out, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __ldg(in + idx[i]);
}

// out[idx[i]] = in[i]: reads `in` in order (a pinned host buffer read in place
// streams over the host link in full lines), scatters into device memory.  One
// entry per thread: the link's latency wants many requests in flight.
__global__ void scatter_f64(const double* __restrict__ in, const int32_t* __restrict__ idx,
                            double* __restrict__ out, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[idx[i]] = in[i];
}

__global__ void gather_f32(const float* __restrict__ in, const int32_t* __restrict__ idx,
                           float* __restrict__ out, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __ldg(in + idx[i]);
}

// packed[q] = values[src[q]]; src = -1 is padding (0), -2 a batch padding row's
// unit diagonal (1).  diag[i] = values[diagpos[i]] with the same conventions.
__global__ void fill_values_f64(const double* __restrict__ vals_in, const int64_t* __restrict__ src,
                                double* __restrict__ packed, int64_t len) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < len) {
        int64_t s = src[q];
        packed[q] = s >= 0 ? vals_in[s] : (s == -2 ? 1.0 : 0.0);
    }
}

__global__ void fill_diag_f64(const double* __restrict__ vals_in, const int64_t* __restrict__ diagpos,
                              double* __restrict__ diag, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        int64_t s = diagpos[i];
        diag[i] = s >= 0 ? vals_in[s] : (s == -2 ? 1.0 : 0.0);
    }
}

unsigned grid_for(int64_t work, int block) {
    return (unsigned)((work + block - 1) / block);
}

int launch_gather(const double* in, const int32_t* idx, double* out, int64_t n, cudaStream_t s) {
    if (n == 0) return FESPMV_OK;
    gather_f64<<<grid_for(n, 256), 256, 0, s>>>(in, idx, out, n);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

int launch_scatter(const double* in, const int32_t* idx, double* out, int64_t n, cudaStream_t s) {
    if (n == 0) return FESPMV_OK;
    scatter_f64<<<grid_for(n, 256), 256, 0, s>>>(in, idx, out, n);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

int launch_gather_f32(const float* in, const int32_t* idx, float* out, int64_t n, cudaStream_t s) {
    if (n == 0) return FESPMV_OK;
    gather_f32<<<grid_for(n, 256), 256, 0, s>>>(in, idx, out, n);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

int launch_split(const double* v, float2* out, int64_t len, cudaStream_t s) {
    if (len == 0) return FESPMV_OK;
    split_df<<<grid_for(len, 256), 256, 0, s>>>(v, out, len);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

int launch_gather_split(const double* x, const int32_t* idx, double* xp, float2* xs, int64_t n,
                        cudaStream_t s) {
    if (n == 0) return FESPMV_OK;
    gather_split_df<<<grid_for(n, 256), 256, 0, s>>>(x, idx, xp, xs, n);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

template <int V>
static void launch_df(const fespmv_mat* A, const float2* xs, const double* x, double* y, cudaStream_t s) {
    constexpr int U = (V == 4) ? 2 : 4;
    sliced_df64<V, U><<<grid_for(A->n_slices * 32, A->block), A->block, 0, s>>>(
        A->d_meta, A->d_col, A->d_vdf, A->d_val, xs, x, y, A->n_slices, A->n);
}

int launch_spmv_df(const fespmv_mat* A, const float2* xs, const double* x, double* y, cudaStream_t s) {
    if (A->n == 0) return FESPMV_OK;
    if (A->tiled) return launch_spmv_df_tiled(A, xs, x, y, s);
    switch (A->vec) {
        case 1: launch_df<1>(A, xs, x, y, s); break;
        case 4: launch_df<4>(A, xs, x, y, s); break;
        default: launch_df<2>(A, xs, x, y, s); break;
    }
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

int launch_build_scaled(fespmv_mat* A, cudaStream_t s) {
    if (!A->d_scale || A->n == 0) return FESPMV_OK;
    FESPMV_CUDA(cudaMemsetAsync(A->d_flag, 0, sizeof(int), s));
    scale_from_diag<<<grid_for(A->n, 256), 256, 0, s>>>(A->d_diag, A->d_scale, A->n, A->d_flag);
    if (!A->d_val32 && !A->d_val16) return FESPMV_OK;
    if (A->format == FESPMV_FMT_SLICED) {
        const unsigned g = grid_for(A->n_slices * 32, 256);
        switch (A->vec) {
            case 1: build_scaled_sliced<1><<<g, 256, 0, s>>>(A->d_meta, A->d_col, A->d_val, A->d_scale, A->d_val32, A->d_val16, A->n_slices); break;
            case 4: build_scaled_sliced<4><<<g, 256, 0, s>>>(A->d_meta, A->d_col, A->d_val, A->d_scale, A->d_val32, A->d_val16, A->n_slices); break;
            default: build_scaled_sliced<2><<<g, 256, 0, s>>>(A->d_meta, A->d_col, A->d_val, A->d_scale, A->d_val32, A->d_val16, A->n_slices); break;
        }
    } else {
        build_scaled_csr<<<grid_for(A->n, 256), 256, 0, s>>>(A->d_rowptr, A->d_colind, A->d_val, A->d_scale,
                                                           A->d_val32, A->d_val16, A->n);
    }
    FESPMV_CUDA(cudaGetLastError());
    return launch_nb3_refresh(A, s);
}

int launch_fill_values(fespmv_mat* A, const double* vals_in, cudaStream_t s) {
    if (A->format == FESPMV_FMT_SLICED) {
        if (A->packed_len > 0)
            fill_values_f64<<<grid_for(A->packed_len, 256), 256, 0, s>>>(vals_in, A->d_src, A->d_val,
                                                                        A->packed_len);
    } else if (A->nnz > 0) {
        FESPMV_CUDA(cudaMemcpyAsync(A->d_val, vals_in, sizeof(double) * A->nnz,
                                    cudaMemcpyDeviceToDevice, s));
    }
    if (A->n > 0)
        fill_diag_f64<<<grid_for(A->n, 256), 256, 0, s>>>(vals_in, A->d_diagpos, A->d_diag, A->n);
    FESPMV_CUDA(cudaGetLastError());
    if (A->d_vdf) {
        int rc = launch_split(A->d_val, A->d_vdf, A->packed_len, s);
        if (rc) return rc;
    }
    return launch_build_scaled(A, s);
}

template <int L>
static void launch_csr(const fespmv_mat* A, const double* x, double* y, cudaStream_t s) {
    int64_t threads = A->n * L;
    csr_f64<L><<<grid_for(threads, A->block), A->block, 0, s>>>(A->d_rowptr, A->d_colind,
                                                              A->d_val, x, y, A->n);
}

template <int V>
static void launch_sliced(const fespmv_mat* A, const double* x, double* y, cudaStream_t s) {
    constexpr int U = (V == 1) ? 8 : (V == 2 ? 4 : 2);
    int64_t threads = A->n_slices * 32;
    sliced_f64<V, U><<<grid_for(threads, A->block), A->block, 0, s>>>(A->d_meta, A->d_col, A->d_val,
                                                                     x, y, A->n_slices, A->n);
}

template <typename VT, int V>
static void launch_sliced_low(const fespmv_mat* A, const VT* val, const float* x, float* y, cudaStream_t s) {
    constexpr int U = (V == 4) ? 4 : 8;
    sliced_low<VT, V, U><<<grid_for(A->n_slices * 32, A->block), A->block, 0, s>>>(A->d_meta, A->d_col, val, x,
                                                                               y, A->n_slices, A->n);
}

template <typename VT, int L>
static void launch_csr_low(const fespmv_mat* A, const VT* val, const float* x, float* y, cudaStream_t s) {
    csr_low<VT, L><<<grid_for(A->n * L, A->block), A->block, 0, s>>>(A->d_rowptr, A->d_colind, val, x, y, A->n);
}

template <typename VT>
static void dispatch_low(const fespmv_mat* A, const VT* val, const float* x, float* y, cudaStream_t s) {
    if (A->format == FESPMV_FMT_SLICED) {
        switch (A->vec) {
            case 1: launch_sliced_low<VT, 1>(A, val, x, y, s); break;
            case 4: launch_sliced_low<VT, 4>(A, val, x, y, s); break;
            default: launch_sliced_low<VT, 2>(A, val, x, y, s); break;
        }
    } else {
        switch (A->csr_lanes) {
            case 1: launch_csr_low<VT, 1>(A, val, x, y, s); break;
            case 2: launch_csr_low<VT, 2>(A, val, x, y, s); break;
            case 4: launch_csr_low<VT, 4>(A, val, x, y, s); break;
            case 8: launch_csr_low<VT, 8>(A, val, x, y, s); break;
            case 16: launch_csr_low<VT, 16>(A, val, x, y, s); break;
            default: launch_csr_low<VT, 32>(A, val, x, y, s); break;
        }
    }
}

int launch_spmv_low(const fespmv_mat* A, int precision, const float* x, float* y, cudaStream_t s) {
    if (A->n == 0) return FESPMV_OK;
    if (A->nb) return launch_nb3_product(A, precision, x, y, s);
    if (A->tiled) return launch_spmv_low_tiled(A, precision, x, y, s);
    if (precision == FESPMV_PREC_F32)
        dispatch_low<float>(A, A->d_val32, x, y, s);
    else
        dispatch_low<__nv_bfloat16>(A, reinterpret_cast<const __nv_bfloat16*>(A->d_val16), x, y, s);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

int launch_spmv(const fespmv_mat* A, const double* x, double* y, cudaStream_t s) {
    if (A->n == 0) return FESPMV_OK;
    if (A->format == FESPMV_FMT_CSR) {
        switch (A->csr_lanes) {
            case 1: launch_csr<1>(A, x, y, s); break;
            case 2: launch_csr<2>(A, x, y, s); break;
            case 4: launch_csr<4>(A, x, y, s); break;
            case 8: launch_csr<8>(A, x, y, s); break;
            case 16: launch_csr<16>(A, x, y, s); break;
            default: launch_csr<32>(A, x, y, s); break;
        }
    } else if (A->tiled) {
        return launch_spmv_tiled(A, x, y, s);
    } else {
        switch (A->vec) {
            case 1: launch_sliced<1>(A, x, y, s); break;
            case 4: launch_sliced<4>(A, x, y, s); break;
            default: launch_sliced<2>(A, x, y, s); break;
        }
    }
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

}  // namespace fespmv
