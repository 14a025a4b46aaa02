// Device core of the 3x3 node-block products (nodeblock.cu, cg.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "spmv_device.cuh"

namespace fespmv {

__device__ __forceinline__ float nb3_value(const float* p) { return ld_stream(p); }
__device__ __forceinline__ float nb3_value(const __nv_bfloat16* p) {
    const unsigned short u = ld_stream(reinterpret_cast<const unsigned short*>(p));
    return __uint_as_float((unsigned)u << 16);
}

// The three row sums of node row m.z + lane of one slice (metadata m): per block
// (ascending block column J) rows a = 0..2 add v[3a+b] * x[3J+b] for b = 0..2.
// U blocks are loaded ahead of their sums.
template <typename VT, int U>
__device__ __forceinline__ void nb3_row_sums(const uint4 m, const int32_t* __restrict__ col,
                                             const VT* __restrict__ val, const float* __restrict__ x, int lane,
                                             float (&s)[3]) {
    const int64_t off = (int64_t)m.x * 32;
    const int w = (int)m.y;
    const int32_t* cp = col + off + lane;
    const VT* vp = val + 9 * off + lane;
    s[0] = s[1] = s[2] = 0.0f;
    int st = 0;
    for (; st + U <= w; st += U) {
        int32_t J[U];
        float v[U][9];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            J[u] = ld_stream(cp + 32 * (st + u));
#pragma unroll
            for (int k = 0; k < 9; ++k) v[u][k] = nb3_value(vp + 288 * (st + u) + 32 * k);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (J[u] < 0) continue;
            const float* xp = x + 3 * (int64_t)J[u];
            const float x0 = __ldg(xp), x1 = __ldg(xp + 1), x2 = __ldg(xp + 2);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                s[a] = fmaf(v[u][3 * a], x0, s[a]);
                s[a] = fmaf(v[u][3 * a + 1], x1, s[a]);
                s[a] = fmaf(v[u][3 * a + 2], x2, s[a]);
            }
        }
    }
    for (; st < w; ++st) {
        const int32_t J = ld_stream(cp + 32 * st);
        float v[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) v[k] = nb3_value(vp + 288 * st + 32 * k);
        if (J < 0) continue;
        const float* xp = x + 3 * (int64_t)J;
        const float x0 = __ldg(xp), x1 = __ldg(xp + 1), x2 = __ldg(xp + 2);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s[a] = fmaf(v[3 * a], x0, s[a]);
            s[a] = fmaf(v[3 * a + 1], x1, s[a]);
            s[a] = fmaf(v[3 * a + 2], x2, s[a]);
        }
    }
}

// Stage the x values of tile tl's column nodes (3 per node) into xs, then the
// zero slot D (three zeros: padding slots index it).
__device__ __forceinline__ int4 nb3_stage(const int4* __restrict__ tile, const int32_t* __restrict__ dict,
                                          const float* __restrict__ x, float* xs) {
    const int4 tl = *tile;
    for (int e = threadIdx.x; e < 3 * (tl.w + 1); e += blockDim.x) {
        const int node = e / 3, c = e - 3 * node;
        xs[e] = node < tl.w ? __ldg(x + 3 * (int64_t)__ldg(dict + tl.z + node) + c) : 0.0f;
    }
    __syncthreads();
    return tl;
}

// nb3_row_sums with x from a staged tile: each slot's 16-bit index names its
// column node in the tile's list (padding: the zero slot).
template <typename VT, int U>
__device__ __forceinline__ void nb3_row_sums_tiled(const uint4 m, const uint16_t* __restrict__ lidx,
                                                   const VT* __restrict__ val, const float* xs, int lane,
                                                   float (&s)[3]) {
    const int64_t off = (int64_t)m.x * 32;
    const int w = (int)m.y;
    const unsigned short* cp = reinterpret_cast<const unsigned short*>(lidx) + off + lane;
    const VT* vp = val + 9 * off + lane;
    s[0] = s[1] = s[2] = 0.0f;
    int st = 0;
    for (; st + U <= w; st += U) {
        int li[U];
        float v[U][9];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            li[u] = ld_stream(cp + 32 * (st + u));
#pragma unroll
            for (int k = 0; k < 9; ++k) v[u][k] = nb3_value(vp + 288 * (st + u) + 32 * k);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float x0 = xs[3 * li[u]], x1 = xs[3 * li[u] + 1], x2 = xs[3 * li[u] + 2];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                s[a] = fmaf(v[u][3 * a], x0, s[a]);
                s[a] = fmaf(v[u][3 * a + 1], x1, s[a]);
                s[a] = fmaf(v[u][3 * a + 2], x2, s[a]);
            }
        }
    }
    for (; st < w; ++st) {
        const int li = ld_stream(cp + 32 * st);
        float v[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) v[k] = nb3_value(vp + 288 * st + 32 * k);
        const float x0 = xs[3 * li], x1 = xs[3 * li + 1], x2 = xs[3 * li + 2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s[a] = fmaf(v[3 * a], x0, s[a]);
            s[a] = fmaf(v[3 * a + 1], x1, s[a]);
            s[a] = fmaf(v[3 * a + 2], x2, s[a]);
        }
    }
}

}  // namespace fespmv
