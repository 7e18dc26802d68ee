// Complex numbers as float pairs (hi + lo per component, ~2^-44 relative) for FP64-quality
// arithmetic on the fp32 pipe, which is ~64x GB300's FP64 pipe: the error-free transforms
// TwoSum and TwoProduct (with fmaf) and a fused (h, l) += x y.  Device code only.
#pragma once

namespace afqmc {

struct __align__(16) ffc {   // 16-byte aligned: a peer CTA can receive it as one 16-byte store
    float rh, rl, ih, il;
};
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float v = s - a;
    e = (a - (s - v)) + (b - v);
}
// (h, l) + x y for float pairs: TwoProduct of the leading parts, first-order cross terms
__device__ __forceinline__ void ff_fma(float& h, float& l, float xh, float xl, float yh, float yl) {
    const float p = xh * yh;
    float pe = fmaf(xh, yh, -p);
    pe = fmaf(xh, yl, fmaf(xl, yh, pe));
    float s, e;
    two_sum(h, p, s, e);
    e += l + pe;
    h = s + e;
    l = e - (h - s);
}

}  // namespace afqmc
