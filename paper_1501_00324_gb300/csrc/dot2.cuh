// Float-pair dot products for the low-precision CG kernels (cg.cu, the cluster
// solvers).
#pragma once

#include <cuda_runtime.h>

namespace fespmv {

// A dot product of floats accumulated as a float pair on the FP32 pipe: Dot2 of
// Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput.,
// 2005): each product split exactly by an FMA (TwoProduct), added to the running
// sum by Knuth's TwoSum, the two rounding errors gathered in lo.  The result is
// as accurate as a sum taken in twice float precision, and none of it runs on
// the FP64 pipe, which on this GPU costs ~60 times the FP32 pipe per operation.
// The intrinsics keep the compiler from contracting the error terms into FMAs.
struct Dot2 {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        const float s = __fadd_rn(hi, p);
        const float z = __fsub_rn(s, hi);
        const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(p, z));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(t, e));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

}  // namespace fespmv
