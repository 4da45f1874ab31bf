// Per-(pixel, Gaussian) evaluation of the closed-form opacity shared by the forward and
// backward blend kernels.  Every operation is written out (fmaf / __fmul_rn / __fadd_rn) so
// the two kernels compute identical bits and therefore take identical skip decisions.
#pragma once

#include "vg_internal.cuh"

namespace vg {

constexpr float kHalfLog2e = 0.72134752044448170f;   // 0.5 * log2(e)
constexpr float kLog2eF = 1.44269504088896341f;

// Pixel-constant part: pixel coordinates and log2 |d_c| of the un-normalised camera ray
// d_c = ((x + 0.5 - cx)/fx, (y + 0.5 - cy)/fy, 1).
struct PixelRay {
    float xf, yf, Lp;
};

__device__ __forceinline__ PixelRay pixel_ray(const ViewInfo &V, int x, int y) {
    PixelRay p;
    p.xf = (float)x;
    p.yf = (float)y;
    const float u = __fdiv_rn(__fsub_rn(__fadd_rn(p.xf, 0.5f), V.cx), V.fx);
    const float v = __fdiv_rn(__fsub_rn(__fadd_rn(p.yf, 0.5f), V.cy), V.fy);
    p.Lp = 0.5f * __log2f(fmaf(u, u, fmaf(v, v, 1.0f)));
    return p;
}

// Record layout (6 x float4):
//   r0 = (A0.x, A0.y, A0.z, A1.x)  r1 = (A1.y, A1.z, A2.x, A2.y)  r2 = (A2.z, C0.x, C0.y, C0.z)
//   r3 = (C1.x, C1.y, C1.z, C2.x)  r4 = (C2.y, C2.z, px0, py0)     r5 = (log2(kappa sqrt(2pi)), r, g, b)
// d' = A0 dx + A1 dy + A2, o' x d' = C0 dx + C1 dy + C2 with (dx, dy) = pixel - (px0, py0);
//   tau = kappa sqrt(2 pi) |d_c| / |d'| exp(-|o' x d'|^2 / (2 |d'|^2))   (Eq. 19, unit-ray form).
struct PairEval {
    float dx, dy;
    float dp[3], cr[3];
    float rs, m2, tau;
};

__device__ __forceinline__ void eval_pair(const float4 &r0, const float4 &r1, const float4 &r2, const float4 &r3,
                                          const float4 &r4, const float4 &r5, const PixelRay &p, PairEval &e) {
    e.dx = __fsub_rn(p.xf, r4.z);
    e.dy = __fsub_rn(p.yf, r4.w);
    e.dp[0] = fmaf(r0.x, e.dx, fmaf(r0.w, e.dy, r1.z));
    e.dp[1] = fmaf(r0.y, e.dx, fmaf(r1.x, e.dy, r1.w));
    e.dp[2] = fmaf(r0.z, e.dx, fmaf(r1.y, e.dy, r2.x));
    e.cr[0] = fmaf(r2.y, e.dx, fmaf(r3.x, e.dy, r3.w));
    e.cr[1] = fmaf(r2.z, e.dx, fmaf(r3.y, e.dy, r4.x));
    e.cr[2] = fmaf(r2.w, e.dx, fmaf(r3.z, e.dy, r4.y));
    const float a = fmaf(e.dp[0], e.dp[0], fmaf(e.dp[1], e.dp[1], __fmul_rn(e.dp[2], e.dp[2])));
    const float q = fmaf(e.cr[0], e.cr[0], fmaf(e.cr[1], e.cr[1], __fmul_rn(e.cr[2], e.cr[2])));
    e.rs = rsqrt_approx(a);
    e.m2 = __fmul_rn(q, __fmul_rn(e.rs, e.rs));
    e.tau = __fmul_rn(ex2_approx(fmaf(e.m2, -kHalfLog2e, __fadd_rn(r5.x, p.Lp))), e.rs);
}

}  // namespace vg
