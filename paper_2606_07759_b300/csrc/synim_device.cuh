// synim_device.cuh -- small device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>

namespace synim {

// a + b with the rounding error added to err (Knuth's two-sum; exact).
__device__ __forceinline__ float two_sum(float a, float b, float &err) {
    const float s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    err = __fadd_rn(err, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z)));
    return s;
}

// (Ah + Al) j + (Bh + Bl) i + (ch + cl) - off, evaluated with error-free
// products and sums so that the only rounding is the final one.
__device__ __forceinline__ float exact_affine(float Ah, float Al, float Bh, float Bl, float ch, float cl,
                                              int j, int i, int off) {
    const float fj = (float)j, fi = (float)i;
    const float p1 = __fmul_rn(Ah, fj), p2 = __fmul_rn(Bh, fi);
    float err = __fadd_rn(__fadd_rn(fmaf(Ah, fj, -p1), fmaf(Bh, fi, -p2)),
                          __fadd_rn(fmaf(Al, fj, __fmul_rn(Bl, fi)), cl));
    float sum = two_sum(p1, p2, err);
    sum = two_sum(sum, ch, err);
    sum = two_sum(sum, (float)(-off), err);
    return __fadd_rn(sum, err);
}

}  // namespace synim
