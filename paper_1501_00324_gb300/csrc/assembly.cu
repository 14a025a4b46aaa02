// Assembly as a sparse product (assembly_* in fespmv.h).
//
// Sec. 4 of the paper assembles the global tangent matrix without atomics by
// writing it as a sparse product: a matrix K^elem with one row per global
// non-zero, whose entries are the element contributions to that non-zero, times
// a vector of ones; the residual vector the same way from the element vectors.
// Here the rows of K^elem are the handle's own value positions (the packed
// slices of Sec. 5, or the CSR order), so the row sums land directly in the
// storage the FE product reads: no host assembly, no reordering of values
// (the cost alpha of Sec. 6) when the values change between Newton steps.
//
// The plan (host, once per mesh): for every value position the indices of its
// contributions in the element-matrix array, in ascending element order, so
// the sums are 0 + c_1 + c_2 + ... exactly as the host would add them; rows of
// constrained dofs hold their unit diagonal.  The kernels: one thread per value
// position summing its list (the "product with ones", no multiplication), the
// unit diagonals, the diagonal of the handle's numbering, and the derived
// copies (float pairs, S and the FP32/BF16 values of S A S) as
// spmv_update_values refreshes them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "internal.h"

struct fespmv_assembly {
    fespmv_mat* A = nullptr;
    int64_t n_elems = 0;
    int npe = 0, dpn = 0, m = 0;
    int64_t len = 0;                 // value positions (packed_len or nnz)
    int64_t n_contrib = 0, n_vcontrib = 0, n_ones = 0;
    int64_t* d_kp = nullptr;         // len + 1 offsets into d_kidx
    uint32_t* d_kidx = nullptr;      // element-matrix entry of each contribution
    int64_t* d_ones = nullptr;       // value positions of the unit diagonals
    int64_t* d_diagpk = nullptr;     // handle row -> value position of its diagonal (-1: none)
    int64_t* d_vp = nullptr;         // n + 1 offsets into d_vidx (input rows)
    uint32_t* d_vidx = nullptr;      // element-vector entry of each contribution
    double* d_stage = nullptr;       // element matrices copied from the host
    int64_t bytes = 0;
};

namespace fespmv {
namespace {

__global__ void asm_values(const int64_t* __restrict__ kp, const uint32_t* __restrict__ kidx,
                           const double* __restrict__ Ke, double* __restrict__ val, int64_t len) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= len) return;
    double v = 0.0;
    // the loads of several contributions go out together; the sum stays in list order
#pragma unroll 4
    for (int64_t k = kp[p], e = kp[p + 1]; k < e; ++k) v += __ldg(Ke + kidx[k]);
    val[p] = v;
}

__global__ void asm_ones(const int64_t* __restrict__ pos, double* __restrict__ val, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) val[pos[i]] = 1.0;
}

__global__ void asm_diag(const int64_t* __restrict__ diagpk, const double* __restrict__ val,
                         double* __restrict__ diag, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) diag[i] = diagpk[i] >= 0 ? val[diagpk[i]] : 0.0;
}

// out[r] = sum of the contributions of input row idx[r] (idx null: r).
__global__ void asm_vector(const int64_t* __restrict__ vp, const uint32_t* __restrict__ vidx,
                           const double* __restrict__ Re, const int32_t* __restrict__ idx,
                           double* __restrict__ out, int64_t n) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t I = idx ? (int64_t)idx[r] : r;
    double v = 0.0;
#pragma unroll 4
    for (int64_t k = vp[I], e = vp[I + 1]; k < e; ++k) v += __ldg(Re + vidx[k]);
    out[r] = v;
}

int64_t find_col(const int64_t* rowptr, const int32_t* colind, int64_t i, int32_t j) {
    int64_t lo = rowptr[i], hi = rowptr[i + 1];
    const int32_t* p = std::lower_bound(colind + lo, colind + hi, j);
    return (p != colind + hi && *p == j) ? (int64_t)(p - colind) : -1;
}

int asm_alloc(fespmv_assembly* P, void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMalloc(%zu bytes) for %s failed: %s", bytes, what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? FESPMV_ERR_OOM : FESPMV_ERR_CUDA;
    }
    P->bytes += (int64_t)bytes;
    return FESPMV_OK;
}

void free_assembly(fespmv_assembly* P) {
    if (!P) return;
    void* ptrs[] = {P->d_kp, P->d_kidx, P->d_ones, P->d_diagpk, P->d_vp, P->d_vidx, P->d_stage};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete P;
}

template <typename Fn>
void parallel_rows(int64_t n, Fn fn) {
    const int nt = (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    if (nt == 1 || n < 4096) {
        fn(0, n, 0);
        return;
    }
    std::vector<std::thread> th;
    const int64_t chunk = (n + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        const int64_t b = t * chunk, e = std::min(n, b + chunk);
        if (b < e) th.emplace_back(fn, b, e, t);
    }
    for (auto& t : th) t.join();
}

int create_impl(fespmv_assembly_t* out, fespmv_mat* A, const int64_t* rowptr, const int32_t* colind,
                int64_t n_elems, int npe, int dpn, const int32_t* elem_nodes, const uint8_t* mask,
                cudaStream_t s) {
    *out = nullptr;
    const int64_t n = A->n;
    if (npe < 1 || npe > 64 || dpn < 1 || dpn > 8 || n_elems < 0 || (n_elems > 0 && !elem_nodes) ||
        n % dpn != 0 || !rowptr || (A->nnz > 0 && !colind) || rowptr[n] != A->nnz) {
        set_error("assembly_create: bad argument (sizes, or a pattern other than the handle's)");
        return FESPMV_ERR_INVALID_ARG;
    }
    if (A->format == FESPMV_FMT_SLICED && A->n > 0 && !A->d_src) {
        set_error("assembly_create: the handle holds no value map");
        return FESPMV_ERR_UNSUPPORTED;
    }
    const int m = npe * dpn;
    if ((double)n_elems * m * m >= 4294967296.0) {
        set_error("assembly_create: more than 2^32 element-matrix entries");
        return FESPMV_ERR_INVALID_ARG;
    }
    const int64_t n_nodes = n / dpn;
    for (int64_t k = 0; k < n_elems * npe; ++k)
        if (elem_nodes[k] < 0 || elem_nodes[k] >= n_nodes) {
            set_error("assembly_create: element %lld names node %d, outside [0, %lld)", (long long)(k / npe),
                      elem_nodes[k], (long long)n_nodes);
            return FESPMV_ERR_INVALID_ARG;
        }
    for (int64_t i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) {
            set_error("assembly_create: rowptr decreases at row %lld", (long long)i);
            return FESPMV_ERR_BAD_CSR;
        }
    // value position of each CSR entry
    const bool sliced = A->format == FESPMV_FMT_SLICED;
    const int64_t len = sliced ? A->packed_len : A->nnz;
    std::vector<int64_t> vpos((size_t)A->nnz);
    if (sliced) {
        std::vector<int64_t> src((size_t)len);
        if (len > 0)
            FESPMV_CUDA(cudaMemcpy(src.data(), A->d_src, sizeof(int64_t) * (size_t)len, cudaMemcpyDeviceToHost));
        for (int64_t p = 0; p < len; ++p)
            if (src[(size_t)p] >= 0) vpos[(size_t)src[(size_t)p]] = p;
    } else {
        for (int64_t q = 0; q < A->nnz; ++q) vpos[(size_t)q] = q;
    }
    // node -> (element, local vertex), ascending element
    std::vector<int64_t> np_off((size_t)n_nodes + 1, 0);
    for (int64_t k = 0; k < n_elems * npe; ++k) ++np_off[(size_t)elem_nodes[k] + 1];
    for (int64_t a = 0; a < n_nodes; ++a) np_off[(size_t)a + 1] += np_off[(size_t)a];
    std::vector<int64_t> inc((size_t)(n_elems * npe));
    {
        std::vector<int64_t> fill(np_off.begin(), np_off.end() - 1);
        for (int64_t e = 0; e < n_elems; ++e)
            for (int a = 0; a < npe; ++a) inc[(size_t)fill[(size_t)elem_nodes[e * npe + a]]++] = e * npe + a;
    }
    // count the contributions of every value position, rows in parallel (a row's
    // entries are its own: no two threads touch one position)
    std::vector<int64_t> cnt((size_t)len + 1, 0);
    std::vector<int> err(64, 0);
    std::vector<int64_t> err_row(64, -1);
    auto walk = [&](int64_t a0, int64_t a1, int t, bool fill_pass, const std::vector<int64_t>* kp,
                    std::vector<int64_t>* cursor, uint32_t* kidx) {
        for (int64_t a = a0; a < a1; ++a)
            for (int64_t q = np_off[(size_t)a]; q < np_off[(size_t)a + 1]; ++q) {
                const int64_t e = inc[(size_t)q] / npe;
                const int la = (int)(inc[(size_t)q] % npe);
                for (int ci = 0; ci < dpn; ++ci) {
                    const int64_t I = dpn * a + ci;
                    if (mask && mask[I]) continue;
                    for (int b = 0; b < npe; ++b)
                        for (int cj = 0; cj < dpn; ++cj) {
                            const int32_t J = (int32_t)(dpn * (int64_t)elem_nodes[e * npe + b] + cj);
                            if (mask && mask[J]) continue;
                            const int64_t c = find_col(rowptr, colind, I, J);
                            if (c < 0) {
                                err[(size_t)t] = 1;
                                err_row[(size_t)t] = I;
                                continue;
                            }
                            const int64_t pos = vpos[(size_t)c];
                            if (!fill_pass) {
                                ++cnt[(size_t)pos + 1];
                            } else {
                                const int64_t at = (*kp)[(size_t)pos] + (*cursor)[(size_t)pos]++;
                                kidx[at] = (uint32_t)(e * m * m + (int64_t)(dpn * la + ci) * m + dpn * b + cj);
                            }
                        }
                }
            }
    };
    parallel_rows(n_nodes, [&](int64_t a0, int64_t a1, int t) { walk(a0, a1, t, false, nullptr, nullptr, nullptr); });
    for (size_t t = 0; t < err.size(); ++t)
        if (err[t]) {
            set_error("assembly_create: an element contributes to an entry of row %lld that the pattern does not "
                      "store", (long long)err_row[t]);
            return FESPMV_ERR_BAD_CSR;
        }
    for (int64_t p = 0; p < len; ++p) cnt[(size_t)p + 1] += cnt[(size_t)p];
    const int64_t n_contrib = cnt[(size_t)len];
    std::vector<uint32_t> kidx((size_t)std::max<int64_t>(n_contrib, 1));
    {
        std::vector<int64_t> cursor((size_t)len, 0);
        parallel_rows(n_nodes, [&](int64_t a0, int64_t a1, int t) {
            walk(a0, a1, t, true, &cnt, &cursor, kidx.data());
        });
    }
    // unit diagonals of the constrained rows
    std::vector<int64_t> ones;
    if (mask)
        for (int64_t i = 0; i < n; ++i)
            if (mask[i]) {
                const int64_t c = find_col(rowptr, colind, i, (int32_t)i);
                if (c < 0) {
                    set_error("assembly_create: constrained row %lld stores no diagonal", (long long)i);
                    return FESPMV_ERR_BAD_CSR;
                }
                ones.push_back(vpos[(size_t)c]);
            }
    // diagonal of each handle row
    std::vector<int64_t> diagpk((size_t)n, -1);
    if (n > 0) {
        std::vector<int64_t> dpos((size_t)n);
        FESPMV_CUDA(cudaMemcpy(dpos.data(), A->d_diagpos, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost));
        for (int64_t r = 0; r < n; ++r)
            if (dpos[(size_t)r] >= 0) diagpk[(size_t)r] = vpos[(size_t)dpos[(size_t)r]];
    }
    // vector contributions per input row, ascending element
    std::vector<int64_t> vp((size_t)n + 1, 0);
    for (int64_t a = 0; a < n_nodes; ++a)
        for (int c = 0; c < dpn; ++c) {
            const int64_t I = dpn * a + c;
            vp[(size_t)I + 1] = vp[(size_t)I] + ((mask && mask[I]) ? 0 : np_off[(size_t)a + 1] - np_off[(size_t)a]);
        }
    std::vector<uint32_t> vidx((size_t)std::max<int64_t>(vp[(size_t)n], 1));
    for (int64_t a = 0; a < n_nodes; ++a)
        for (int c = 0; c < dpn; ++c) {
            const int64_t I = dpn * a + c;
            if (mask && mask[I]) continue;
            int64_t at = vp[(size_t)I];
            for (int64_t q = np_off[(size_t)a]; q < np_off[(size_t)a + 1]; ++q) {
                const int64_t e = inc[(size_t)q] / npe;
                const int la = (int)(inc[(size_t)q] % npe);
                vidx[(size_t)at++] = (uint32_t)(e * m + dpn * la + c);
            }
        }

    fespmv_assembly* P = new fespmv_assembly();
    P->A = A;
    P->n_elems = n_elems;
    P->npe = npe;
    P->dpn = dpn;
    P->m = m;
    P->len = len;
    P->n_contrib = n_contrib;
    P->n_vcontrib = vp[(size_t)n];
    P->n_ones = (int64_t)ones.size();
    int rc;
    if ((rc = asm_alloc(P, (void**)&P->d_kp, sizeof(int64_t) * (size_t)(len + 1), "assembly offsets")) ||
        (rc = asm_alloc(P, (void**)&P->d_kidx, sizeof(uint32_t) * kidx.size(), "assembly contributions")) ||
        (rc = asm_alloc(P, (void**)&P->d_ones, sizeof(int64_t) * std::max<size_t>(ones.size(), 1), "unit diagonals")) ||
        (rc = asm_alloc(P, (void**)&P->d_diagpk, sizeof(int64_t) * (size_t)std::max<int64_t>(n, 1), "diagonal positions")) ||
        (rc = asm_alloc(P, (void**)&P->d_vp, sizeof(int64_t) * (size_t)(n + 1), "vector offsets")) ||
        (rc = asm_alloc(P, (void**)&P->d_vidx, sizeof(uint32_t) * vidx.size(), "vector contributions"))) {
        free_assembly(P);
        return rc;
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(P->d_kp, cnt.data(), sizeof(int64_t) * (size_t)(len + 1), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(P->d_kidx, kidx.data(), sizeof(uint32_t) * kidx.size(), cudaMemcpyHostToDevice, s)) ||
        (!ones.empty() && (e = cudaMemcpyAsync(P->d_ones, ones.data(), sizeof(int64_t) * ones.size(),
                                               cudaMemcpyHostToDevice, s))) ||
        (n > 0 && (e = cudaMemcpyAsync(P->d_diagpk, diagpk.data(), sizeof(int64_t) * (size_t)n,
                                       cudaMemcpyHostToDevice, s))) ||
        (e = cudaMemcpyAsync(P->d_vp, vp.data(), sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(P->d_vidx, vidx.data(), sizeof(uint32_t) * vidx.size(), cudaMemcpyHostToDevice, s)) ||
        (e = cudaStreamSynchronize(s))) {
        free_assembly(P);
        return cuda_fail(e, "assembly upload");
    }
    *out = P;
    return FESPMV_OK;
}

int matrix_impl(fespmv_assembly* P, const double* Ke, int32_t flags, cudaStream_t s) {
    fespmv_mat* A = P->A;
    const double* src = Ke;
    if (flags & FESPMV_IO_HOST) {
        const size_t bytes = sizeof(double) * (size_t)P->n_elems * P->m * P->m;
        if (!P->d_stage && bytes > 0) {
            int rc = asm_alloc(P, (void**)&P->d_stage, bytes, "element matrices");
            if (rc) return rc;
        }
        if (bytes > 0) FESPMV_CUDA(cudaMemcpyAsync(P->d_stage, Ke, bytes, cudaMemcpyHostToDevice, s));
        src = P->d_stage;
    }
    if (P->len > 0) asm_values<<<grid_for(P->len, 256), 256, 0, s>>>(P->d_kp, P->d_kidx, src, A->d_val, P->len);
    if (P->n_ones > 0) asm_ones<<<grid_for(P->n_ones, 256), 256, 0, s>>>(P->d_ones, A->d_val, P->n_ones);
    if (A->n > 0) asm_diag<<<grid_for(A->n, 256), 256, 0, s>>>(P->d_diagpk, A->d_val, A->d_diag, A->n);
    FESPMV_CUDA(cudaGetLastError());
    if (A->d_vdf) {
        int rc = launch_split(A->d_val, A->d_vdf, A->packed_len, s);
        if (rc) return rc;
    }
    int rc = launch_build_scaled(A, s);
    if (rc) return rc;
    if (flags & FESPMV_IO_HOST) FESPMV_CUDA(cudaStreamSynchronize(s));
    return FESPMV_OK;
}

}  // namespace

fespmv_mat* assembly_handle(fespmv_assembly* P) { return P ? P->A : nullptr; }

}  // namespace fespmv

using namespace fespmv;

extern "C" {

int assembly_create(fespmv_assembly_t* out, fespmv_mat_t A, const int64_t* rowptr, const int32_t* colind,
                    int64_t n_elems, int32_t nodes_per_elem, int32_t dofs_per_node, const int32_t* elem_nodes,
                    const uint8_t* dirichlet, fespmv_stream_t stream) {
    try {
        if (!out || !A) {
            set_error("null argument");
            return FESPMV_ERR_INVALID_ARG;
        }
        if (A->col_order == FESPMV_COLS_ORIGINAL) {
            set_error("assembly needs a handle with renumbered columns (not FESPMV_COLS_ORIGINAL)");
            return FESPMV_ERR_UNSUPPORTED;
        }
        return create_impl(out, A, rowptr, colind, n_elems, nodes_per_elem, dofs_per_node, elem_nodes, dirichlet,
                           (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return FESPMV_ERR_OOM;
    } catch (...) {
        set_error("unexpected C++ exception");
        return FESPMV_ERR_INVALID_ARG;
    }
}

int assembly_matrix(fespmv_assembly_t P, const double* Ke, int32_t flags, fespmv_stream_t stream) {
    if (!P || (P->n_elems > 0 && !Ke) || (flags & ~FESPMV_IO_HOST)) {
        set_error("assembly_matrix: bad argument");
        return FESPMV_ERR_INVALID_ARG;
    }
    return matrix_impl(P, Ke, flags, (cudaStream_t)stream);
}

int assembly_vector(fespmv_assembly_t P, const double* Re, double* r, int32_t flags, fespmv_stream_t stream) {
    if (!P || (P->n_elems > 0 && !Re) || (P->A->n > 0 && !r) || (flags & ~FESPMV_IO_PERMUTED)) {
        set_error("assembly_vector: bad argument");
        return FESPMV_ERR_INVALID_ARG;
    }
    fespmv_mat* A = P->A;
    if ((flags & FESPMV_IO_PERMUTED) && A->format != FESPMV_FMT_SLICED) {
        set_error("assembly_vector: FESPMV_IO_PERMUTED needs a SLICED handle");
        return FESPMV_ERR_INVALID_ARG;
    }
    if (A->n == 0) return FESPMV_OK;
    cudaStream_t s = (cudaStream_t)stream;
    asm_vector<<<grid_for(A->n, 256), 256, 0, s>>>(P->d_vp, P->d_vidx, Re,
                                                   (flags & FESPMV_IO_PERMUTED) ? A->d_perm : nullptr, r, A->n);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

int assembly_get_info(fespmv_assembly_t P, int64_t* n_contributions, int64_t* device_bytes) {
    if (!P) {
        set_error("null argument");
        return FESPMV_ERR_INVALID_ARG;
    }
    if (n_contributions) *n_contributions = P->n_contrib;
    if (device_bytes) *device_bytes = P->bytes;
    return FESPMV_OK;
}

void assembly_destroy(fespmv_assembly_t P) {
    try {
        free_assembly(P);
    } catch (...) {
    }
}

}  // extern "C"
