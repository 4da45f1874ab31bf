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

// A thread owns P pixels of a 16x16 tile (P = 1, 2 or 4); 256 / P threads per tile.
//   P = 1: pixel (t % 16, t / 16)
//   P = 2: pixels (t % 16, 2 (t / 16) + k), k = 0, 1            (a warp covers 16 x 4 pixels)
//   P = 4: pixels (2 (t % 8) + (k & 1), 2 (t / 8) + (k >> 1))    (a warp covers 16 x 8 pixels)
// d' and o' x d' are affine in the pixel offset, so a thread's other pixels follow from its
// first by one add per component.  Forward and backward both use pair_eval_at(), so they
// compute the same bits and take the same skip decisions.
template <int P>
struct PixLayout {
    static constexpr int kThreads = kTilePix / P;
    __device__ static void origin(int t, int &x, int &y) {
        if (P == 1) {
            x = t & 15;
            y = t >> 4;
        } else if (P == 2) {
            x = t & 15;
            y = 2 * (t >> 4);
        } else {
            x = 2 * (t & 7);
            y = 2 * (t >> 3);
        }
    }
    __host__ __device__ static constexpr int ox(int k) { return P == 4 ? (k & 1) : 0; }
    __host__ __device__ static constexpr int oy(int k) { return P == 4 ? (k >> 1) : (P == 2 ? k : 0); }
};

// Bounds of the pixels a warp owns, for the warp-uniform footprint test of each record.
struct WarpBox {
    int x0, y0, x1, y1;
};

template <int P>
__device__ __forceinline__ WarpBox warp_box(int x0, int y0) {
    int xmin = x0, xmax = x0, ymin = y0, ymax = y0;
#pragma unroll
    for (int k = 1; k < P; ++k) {
        xmax = max(xmax, x0 + PixLayout<P>::ox(k));
        ymax = max(ymax, y0 + PixLayout<P>::oy(k));
    }
    WarpBox b;
    b.x0 = __reduce_min_sync(0xffffffffu, xmin);
    b.y0 = __reduce_min_sync(0xffffffffu, ymin);
    b.x1 = __reduce_max_sync(0xffffffffu, xmax);
    b.y1 = __reduce_max_sync(0xffffffffu, ymax);
    return b;
}

__device__ __forceinline__ bool box_misses(const WarpBox &b, const short4 &r) {
    return r.z < b.x0 || r.x > b.x1 || r.w < b.y0 || r.y > b.y1;
}

__device__ __forceinline__ bool box_inside(const WarpBox &b, const short4 &r) {
    return r.x <= b.x0 && r.z >= b.x1 && r.y <= b.y0 && r.w >= b.y1;
}

__device__ __forceinline__ bool pixel_outside(int x, int y, const short4 &r) {
    return x < r.x || x > r.z || y < r.y || y > r.w;
}

struct QuadBase {
    float dx, dy;          // offset of the thread's first pixel from the reference pixel
    float dp[3], cr[3];    // d' and o' x d' there
};

__device__ __forceinline__ void quad_base(const float4 &r0, const float4 &r1, const float4 &r2, const float4 &r3,
                                          const float4 &r4, float x0, float y0, QuadBase &b) {
    b.dx = __fsub_rn(x0, r4.z);
    b.dy = __fsub_rn(y0, r4.w);
    b.dp[0] = fmaf(r0.x, b.dx, fmaf(r0.w, b.dy, r1.z));
    b.dp[1] = fmaf(r0.y, b.dx, fmaf(r1.x, b.dy, r1.w));
    b.dp[2] = fmaf(r0.z, b.dx, fmaf(r1.y, b.dy, r2.x));
    b.cr[0] = fmaf(r2.y, b.dx, fmaf(r3.x, b.dy, r3.w));
    b.cr[1] = fmaf(r2.z, b.dx, fmaf(r3.y, b.dy, r4.x));
    b.cr[2] = fmaf(r2.w, b.dx, fmaf(r3.z, b.dy, r4.y));
}

// d', o' x d', (dx, dy) of the pixel at offset (sx, sy) from the thread's first pixel, and
// its tau (unclamped).
__device__ __forceinline__ void pair_eval_at(const float4 &r0, const float4 &r1, const float4 &r2, const float4 &r3,
                                             const float4 &r5, const QuadBase &b, bool sx, bool sy, float Lp,
                                             PairEval &e) {
    const float A0[3] = {r0.x, r0.y, r0.z}, A1[3] = {r0.w, r1.x, r1.y};
    const float C0[3] = {r2.y, r2.z, r2.w}, C1[3] = {r3.x, r3.y, r3.z};
    e.dx = sx ? __fadd_rn(b.dx, 1.0f) : b.dx;
    e.dy = sy ? __fadd_rn(b.dy, 1.0f) : b.dy;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float dpc = b.dp[c], crc = b.cr[c];
        if (sx) {
            dpc = __fadd_rn(dpc, A0[c]);
            crc = __fadd_rn(crc, C0[c]);
        }
        if (sy) {
            dpc = __fadd_rn(dpc, A1[c]);
            crc = __fadd_rn(crc, C1[c]);
        }
        e.dp[c] = dpc;
        e.cr[c] = crc;
    }
    const float a = fmaf(e.dp[0], e.dp[0], fmaf(e.dp[1], e.dp[1], __fmul_rn(e.dp[2], e.dp[2])));
    const float q = fmaf(e.cr[0], e.cr[0], fmaf(e.cr[1], e.cr[1], __fmul_rn(e.cr[2], e.cr[2])));
    e.rs = rsqrt_approx(a);
    e.m2 = __fmul_rn(q, __fmul_rn(e.rs, e.rs));
    e.tau = __fmul_rn(ex2_approx(fmaf(e.m2, -kHalfLog2e, __fadd_rn(r5.x, Lp))), e.rs);
}

// Warp reduce-scatter of NP per-lane values (NP a power of two, 2..32).  Each exchange step
// with partner lane^w keeps half of the lane's values and sends the other half while more than
// one value is left (NP/2 + NP/4 + ... shuffles), then plain butterfly adds finish the sum.
// Afterwards lane l holds the warp sum of value scatter_index<NP>(l); the 32/NP lanes that
// differ only in their low log2(32/NP) bits hold the same value.
template <int NP>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[NP], int lane) {
    static_assert(NP >= 2 && NP <= 32 && (NP & (NP - 1)) == 0, "NP must be a power of two");
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int w = 16 >> s;
        const int c = NP >> s;   // values the lane still holds
        if (c > 1) {
            const int h = c / 2;
            const bool hi = (lane & w) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const float keep = hi ? v[i + h] : v[i];
                const float send = hi ? v[i] : v[i + h];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
            }
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], w);
        }
    }
    return v[0];
}

template <int NP>
__device__ __forceinline__ int scatter_index(int lane) {
    int idx = 0;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int c = NP >> s;
        if (c > 1 && (lane & (16 >> s))) idx += c / 2;
    }
    return idx;
}

// True for the one lane of each group that holds the same reduce-scatter result.
template <int NP>
__device__ __forceinline__ bool scatter_writer(int lane) {
    return (lane & (32 / NP - 1)) == 0;
}

}  // namespace vg
