// Products of 3x3 node blocks (SLICED handles created with node_blocks = 3).
//
// For three dofs per node (linear elasticity) the stiffness matrix is a matrix
// of 3x3 blocks: the rows of node I touch the same column nodes J.  Storing one
// int32 block column per 9 values instead of one column index per value cuts
// the index stream from 2-4 bytes per value to 4/9 of a byte, and one gather of
// x[3J..3J+2] serves nine products.  The slices are those of Sec. 5.1 (K1, one
// warp per 32 rows, column-major, padded to the longest row) over node rows:
// a lane holds the three rows of one node and walks its blocks in ascending
// column order, so each row's sum runs over its columns in ascending order,
// as the scalar slices do.  Values are B = S A S in FP32 or BF16 (the refined
// CG's inner operator); a block stores zeros where the matrix has no entry.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "spmv_device.cuh"
#include "nodeblock_device.cuh"

namespace fespmv {

// y = B x over node blocks: one warp per slice.
template <typename VT, int U>
__global__ void __launch_bounds__(256) nb3_product(const uint4* __restrict__ meta, const int32_t* __restrict__ col,
                                                   const VT* __restrict__ val, const float* __restrict__ x,
                                                   float* __restrict__ y, int64_t n_nodes, int64_t n_slices) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (warp >= n_slices) return;
    const int lane = threadIdx.x & 31;
    float s[3];
    const uint4 m = meta[warp];
    nb3_row_sums<VT, U>(m, col, val, x, lane, s);
    const int64_t node = (int64_t)m.z + lane;
    if (node < n_nodes) {
        y[3 * node] = s[0];
        y[3 * node + 1] = s[1];
        y[3 * node + 2] = s[2];
    }
}

// The same with x staged per tile (one block per tile of at most 8 slices).
template <typename VT, int U>
__global__ void __launch_bounds__(256, 8) nb3_product_tiled(const uint4* __restrict__ meta,
                                                         const uint16_t* __restrict__ lidx,
                                                         const VT* __restrict__ val, const int4* __restrict__ tiles,
                                                         const int32_t* __restrict__ dict,
                                                         const float* __restrict__ x, float* __restrict__ y,
                                                         int64_t n_nodes) {
    extern __shared__ __align__(16) unsigned char nb_smem[];
    float* xs = reinterpret_cast<float*>(nb_smem);
    const int4 tl = nb3_stage(tiles + blockIdx.x, dict, x, xs);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wid >= tl.y) return;
    const uint4 m = meta[tl.x + wid];
    float s[3];
    nb3_row_sums_tiled<VT, U>(m, lidx, val, xs, lane, s);
    const int64_t node = (int64_t)m.z + lane;
    if (node < n_nodes) {
        y[3 * node] = s[0];
        y[3 * node + 1] = s[1];
        y[3 * node + 2] = s[2];
    }
}

// One node row's products with its 3 x 4 accumulators (rows 3I+a, the lane's four
// right-hand sides): per block (ascending column node J) rows a = 0..2 add
// v[3a+b] * X[3J+b] for b = 0..2.  The block columns of the next U steps are
// loaded one iteration ahead, so that a step's X gathers (three 16-byte loads, one
// per X row of the column node) are issued together with its value loads instead
// of after a dependent column load.
template <int KW, int U>
__device__ __forceinline__ void nb3_multi_rows(const int32_t* cp, const float* vp,
                                               const float* xc, int w, float (&acc)[3][4]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[a][j] = 0.0f;
    int32_t Jn[U];
#pragma unroll
    for (int u = 0; u < U; ++u) Jn[u] = u < w ? ld_stream(cp + 32 * u) : -1;
    for (int st = 0; st < w; st += U) {
        int32_t J[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            J[u] = Jn[u];
            Jn[u] = st + U + u < w ? ld_stream(cp + 32 * (st + U + u)) : -1;
        }
        float4 xb[U][3];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                xb[u][b] = J[u] >= 0 ? __ldg(reinterpret_cast<const float4*>(xc + (3 * (int64_t)J[u] + b) * KW))
                                     : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float v[U][9];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < 9; ++k) v[u][k] = st + u < w ? ld_stream(vp + 288 * (st + u) + 32 * k) : 0.0f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (J[u] < 0) continue;   // a padding slot
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    acc[a][0] = fmaf(v[u][3 * a + b], xb[u][b].x, acc[a][0]);
                    acc[a][1] = fmaf(v[u][3 * a + b], xb[u][b].y, acc[a][1]);
                    acc[a][2] = fmaf(v[u][3 * a + b], xb[u][b].z, acc[a][2]);
                    acc[a][3] = fmaf(v[u][3 * a + b], xb[u][b].w, acc[a][3]);
                }
        }
    }
}

// Y = B X for X, Y row-major n x KW (KW = 4..32 right-hand sides, FP32): KW / 4
// lanes per node row, each lane 4 consecutive right-hand sides of the node's 3
// rows; per block the 9 values (the same words for the row's lanes) and one
// 16-byte load of each of the 3 X rows the block's column node names, so one X
// row serves the 3 rows of the node.  The matrix streams once for all columns.
template <int KW, int U>
__global__ void __launch_bounds__(256, 1) nb3_multi(const uint4* __restrict__ meta, const int32_t* __restrict__ col,
                                                 const float* __restrict__ val, const float* __restrict__ X,
                                                 float* __restrict__ Y, int64_t n_nodes, int64_t n_slices) {
    constexpr int LPR = KW / 4, RPW = 32 / LPR;   // lanes per node row, node rows per warp
    const int lane = threadIdx.x & 31, g = lane / LPR, c = lane % LPR;
    const int64_t nr = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * RPW + g;   // node row slot
    if (nr >= n_slices * 32) return;   // RPW divides 32: a warp never straddles two slices
    const uint4 m = meta[nr >> 5];
    const int ls = (int)(nr & 31);
    const int64_t off = (int64_t)m.x * 32;
    float acc[3][4];
    nb3_multi_rows<KW, U>(col + off + ls, val + 9 * off + ls, X + 4 * c, (int)m.y, acc);
    const int64_t node = (int64_t)m.z + ls;
    if (node < n_nodes)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            *reinterpret_cast<float4*>(Y + (3 * node + a) * KW + 4 * c) =
                make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
}

template <int KW, int U>
static void nb3_multi_launch(const fespmv_mat* A, const float* X, float* Y, cudaStream_t s) {
    const int64_t warps = A->nb_slices * 32 / (32 / (KW / 4));
    nb3_multi<KW, U><<<grid_for(warps * 32, 256), 256, 0, s>>>(A->d_nbmeta, A->d_nbcol, A->d_nb32, X, Y,
                                                               A->n / 3, A->nb_slices);
}

int launch_nb3_multi(const fespmv_mat* A, const float* X, float* Y, int kw, cudaStream_t s) {
    if (A->n == 0) return FESPMV_OK;
    switch (kw) {
        case 4: nb3_multi_launch<4, 2>(A, X, Y, s); break;
        case 8: nb3_multi_launch<8, 2>(A, X, Y, s); break;
        case 16: nb3_multi_launch<16, 2>(A, X, Y, s); break;
        default: nb3_multi_launch<32, 2>(A, X, Y, s); break;
    }
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

// The lockstep multi-RHS CG's product on node blocks: Q = B P as nb3_multi, and
// for every column j the sum of p_ij q_ij over the rows this block covered at
// part[blockIdx.x * KW + j] (per lane in float over its node's 3 rows, then in
// FP64 over its units, then over the groups of a warp and the warps in order).
// Persistent: warps stride over units of 32 / (KW / 4) node rows.
template <int KW, int U>
__global__ void __launch_bounds__(128, 6) nb3_multi_dot(const uint4* __restrict__ meta,
                                                        const int32_t* __restrict__ col,
                                                        const float* __restrict__ val, const float* __restrict__ P,
                                                        float* __restrict__ Q, int64_t n_nodes, int64_t n_slices,
                                                        double* __restrict__ part) {
    constexpr int LPR = KW / 4, RPW = 32 / LPR;
    __shared__ double sh[4][KW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, g = lane / LPR, c = lane % LPR;
    double d[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t units = n_slices * 32 / RPW;
    for (int64_t u = (int64_t)blockIdx.x * 4 + wib; u < units; u += (int64_t)gridDim.x * 4) {
        const int64_t nr = u * RPW + g;
        const uint4 m = meta[nr >> 5];
        const int ls = (int)(nr & 31);
        const int64_t off = (int64_t)m.x * 32;
        float acc[3][4];
        nb3_multi_rows<KW, U>(col + off + ls, val + 9 * off + ls, P + 4 * c, (int)m.y, acc);
        const int64_t node = (int64_t)m.z + ls;
        if (node < n_nodes) {
            float t[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int64_t row = 3 * node + a;
                *reinterpret_cast<float4*>(Q + row * KW + 4 * c) =
                    make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
                const float4 pv = __ldg(reinterpret_cast<const float4*>(P + row * KW + 4 * c));
                t[0] = fmaf(pv.x, acc[a][0], t[0]);
                t[1] = fmaf(pv.y, acc[a][1], t[1]);
                t[2] = fmaf(pv.z, acc[a][2], t[2]);
                t[3] = fmaf(pv.w, acc[a][3], t[3]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) d[j] += (double)t[j];
        }
    }
    // lanes with the same c hold the same columns: sum over the warp's groups
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1)
#pragma unroll
        for (int j = 0; j < 4; ++j) d[j] += __shfl_xor_sync(0xffffffffu, d[j], o);
    if (g == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j) sh[wib][4 * c + j] = d[j];
    __syncthreads();
    if (threadIdx.x < KW)
        part[(int64_t)blockIdx.x * KW + threadIdx.x] =
            ((sh[0][threadIdx.x] + sh[1][threadIdx.x]) + sh[2][threadIdx.x]) + sh[3][threadIdx.x];
}

template <int KW>
static unsigned nb3_multi_dot_kw(const fespmv_mat* A, const float* P, float* Q, double* part, cudaStream_t s) {
    auto kernel = nb3_multi_dot<KW, 2>;
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0);
    const int64_t units = A->nb_slices * 32 / (32 / (KW / 4));
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)sms * std::max(per_sm, 1), (units + 3) / 4));
    if (part) kernel<<<grid, 128, 0, s>>>(A->d_nbmeta, A->d_nbcol, A->d_nb32, P, Q, A->n / 3, A->nb_slices, part);
    return grid;
}

unsigned launch_nb3_multi_dot(const fespmv_mat* A, const float* P, float* Q, int kw, double* part, cudaStream_t s) {
    switch (kw) {
        case 4: return nb3_multi_dot_kw<4>(A, P, Q, part, s);
        case 8: return nb3_multi_dot_kw<8>(A, P, Q, part, s);
        case 16: return nb3_multi_dot_kw<16>(A, P, Q, part, s);
        default: return nb3_multi_dot_kw<32>(A, P, Q, part, s);
    }
}

// Node-block copies of the FP32 / BF16 values: each value slot takes the packed
// scalar copy's value at its mapped position (0 where the block has no entry),
// so both layouts hold the same bits.
__global__ void nb3_gather(const int64_t* __restrict__ map, const float* __restrict__ v32,
                           const uint16_t* __restrict__ v16, float* __restrict__ o32, uint16_t* __restrict__ o16,
                           int64_t len) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = map[i];
        if (o32) o32[i] = p >= 0 ? v32[p] : 0.0f;
        if (o16) o16[i] = p >= 0 ? v16[p] : (uint16_t)0;
    }
}

int launch_nb3_refresh(fespmv_mat* A, cudaStream_t s) {
    if (!A->nb || A->nb_len == 0) return FESPMV_OK;
    const int64_t len = 9 * A->nb_len;
    nb3_gather<<<grid_for(len, 256), 256, 0, s>>>(A->d_nbmap, A->d_val32, A->d_val16, A->d_nb32, A->d_nb16, len);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

int launch_nb3_product(const fespmv_mat* A, int precision, const float* x, float* y, cudaStream_t s) {
    if (A->n == 0) return FESPMV_OK;
    if (A->nb_tiles > 0) {
        const size_t smem = sizeof(float) * 3 * (size_t)(A->nb_tile_dmax + 1);
        const unsigned g = (unsigned)A->nb_tiles;
        if (precision == FESPMV_PREC_F32)
            nb3_product_tiled<float, 2><<<g, 256, smem, s>>>(A->d_nbmeta, A->d_nbtlidx, A->d_nb32, A->d_nbtiles,
                                                             A->d_nbtdict, x, y, A->n / 3);
        else
            nb3_product_tiled<__nv_bfloat16, 4><<<g, 256, smem, s>>>(
                A->d_nbmeta, A->d_nbtlidx, reinterpret_cast<const __nv_bfloat16*>(A->d_nb16), A->d_nbtiles,
                A->d_nbtdict, x, y, A->n / 3);
        FESPMV_CUDA(cudaGetLastError());
        return FESPMV_OK;
    }
    const unsigned g = grid_for(A->nb_slices * 32, 256);
    if (precision == FESPMV_PREC_F32)
        nb3_product<float, 2><<<g, 256, 0, s>>>(A->d_nbmeta, A->d_nbcol, A->d_nb32, x, y, A->n / 3, A->nb_slices);
    else
        nb3_product<__nv_bfloat16, 2><<<g, 256, 0, s>>>(A->d_nbmeta, A->d_nbcol,
                                                        reinterpret_cast<const __nv_bfloat16*>(A->d_nb16), x, y,
                                                        A->n / 3, A->nb_slices);
    FESPMV_CUDA(cudaGetLastError());
    return FESPMV_OK;
}

}  // namespace fespmv
