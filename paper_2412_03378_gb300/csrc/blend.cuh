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
// Every pixel is evaluated by the same operations, whatever the pixel layout of the kernel:
//   dx = x - px0, dy = y - py0 (rounded), d'_c = fma(A1_c, dy, fma(A0_c, dx, A2_c)) and the same
//   for o' x d' with C.
// The inner term depends on the pixel column only, so the pixels of a thread that share a column
// share it (ColBase), and forward and backward compute identical bits for a pixel -- and take
// identical skip and clamp decisions -- with any pixels-per-thread setting of either kernel.
struct PairEval {
    float dx, dy;
    float dp[3], cr[3];
    float rs, m2, tau;
};

// A thread owns P pixels of a tile of tw x th pixels (16 x 16, 32 x 16 or 16 x 8; P = 1, 2 or 4);
// tw th / P threads per tile.  Warps own near-square pixel boxes, which the footprint tests below
// cull best, laid out row by row over the tile; with w = t / 32, l = t % 32, the warp's box column
// wx = w % (tw / bw) and row wy = w / (tw / bw):
//   P = 1: box 8 x 4,  pixel (8 wx + l % 8, 4 wy + l / 8)
//   P = 2: box 8 x 8,  pixels (8 wx + l % 8, 8 wy + 2 (l / 8) + k)
//   P = 4: box 16 x 8, pixels (16 wx + 2 (l % 8) + (k & 1), 8 wy + 2 (l / 8) + (k >> 1))
// A thread's pixels lie in one column (P = 1, 2) or two (P = 4), and it forms each
// column's inner terms (col_base) once per record.
template <int P>
struct PixLayout {
    static constexpr int kBoxW = P == 4 ? 16 : 8;
    // register caps that keep the occupancy of 16 x 16 tiles (forward / backward)
    static constexpr int kFwdRegs = P == 2 ? 73 : 85;
    static constexpr int kBwdRegs = P == 1 ? 56 : (P == 2 ? 96 : 128);
    __device__ static void origin(int t, int tw, int &x, int &y) {
        const int w = t >> 5, l = t & 31;
        const int nwx = tw / kBoxW, wx = w % nwx, wy = w / nwx;
        if (P == 1) {
            x = 8 * wx + (l & 7);
            y = 4 * wy + (l >> 3);
        } else if (P == 2) {
            x = 8 * wx + (l & 7);
            y = 8 * wy + 2 * (l >> 3);
        } else {
            x = 16 * wx + 2 * (l & 7);
            y = 8 * wy + 2 * (l >> 3);
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

// Conservative opacity test of one record against a warp's pixel box, for blending with
// tau_skip >= tau_cut (pairs with tau < tau_skip are skipped by the blend itself).  With
// u = (dx, dy, 1) in the record's pixel offsets, tau = K |d_c| / |A u| exp(-m^2 / 2) and
// m^2 = |C u|^2 / |A u|^2.  Over the box, |A u| >= |A u_c| - |A0| hx - |A1| hy (u_c the box
// centre, hx, hy its half-widths) and |d_c| <= its largest corner value, which bounds the
// amplitude by Amax; tau >= tau_skip then needs m^2 <= r^2 = 2 ln(Amax / tau_skip), i.e.
// Q(u) = |C u|^2 - r^2 |A u|^2 <= 0 somewhere in the box.  The box minimum of the quadratic
// Q is found from the interior stationary point (kept when it lies within a pixel of the box)
// or the four edges; r^2 is inflated by a relative 1e-3 plus 1e-2 so that FP32 rounding never
// turns a blended pair into a culled one.  Returns false only when every pixel of the box has
// tau < tau_skip.
struct BoxCull {
    float x0, y0, x1, y1;   // pixel box (inclusive pixel indices)
    float l2dmax;           // log2 of the largest |d_c| over the box
    float l2tskip;          // log2(tau_skip)
};

__device__ __forceinline__ BoxCull box_cull(const ViewInfo &V, const WarpBox &b, float tau_skip) {
    BoxCull c;
    c.x0 = (float)b.x0;
    c.y0 = (float)b.y0;
    c.x1 = (float)b.x1;
    c.y1 = (float)b.y1;
    float m = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {   // |d_c|^2 is convex in the pixel position: largest at a corner
        const float u = ((k & 1 ? c.x1 : c.x0) + 0.5f - V.cx) / V.fx;
        const float v = ((k & 2 ? c.y1 : c.y0) + 0.5f - V.cy) / V.fy;
        m = fmaxf(m, fmaf(u, u, fmaf(v, v, 1.0f)));
    }
    c.l2dmax = 0.5f * __log2f(m) + 1e-4f;
    c.l2tskip = __log2f(tau_skip);
    return c;
}

__device__ __forceinline__ float quad_edge_min(float h, float rh, float hc, float c0, float lo, float hi) {
    // min over s in [lo, hi] of h s^2 + 2 hc s + c0 (h > 0, rh ~ 1/h): a misplaced vertex only
    // raises the value by h ds^2, far inside the margins of box_may_blend
    const float s = fminf(fmaxf(-hc * rh, lo), hi);
    return fmaf(fmaf(h, s, 2.0f * hc), s, c0);
}

// Per record, the Gram matrices the test needs: G = A^T A and K = C^T C over the columns
// (A0, A1, A2), (C0, C1, C2), packed as (g00 g01 g02 g11) (g12 g22 k00 k01) (k02 k11 k12 k22).
constexpr int kCullF4 = 3;

__device__ __forceinline__ void cull_row(const float4 &r0, const float4 &r1, const float4 &r2, const float4 &r3,
                                         const float4 &r4, float4 out[kCullF4]) {
    const float A0[3] = {r0.x, r0.y, r0.z}, A1[3] = {r0.w, r1.x, r1.y}, A2[3] = {r1.z, r1.w, r2.x};
    const float C0[3] = {r2.y, r2.z, r2.w}, C1[3] = {r3.x, r3.y, r3.z}, C2[3] = {r3.w, r4.x, r4.y};
    auto dot = [](const float *a, const float *b) { return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2])); };
    out[0] = make_float4(dot(A0, A0), dot(A0, A1), dot(A0, A2), dot(A1, A1));
    out[1] = make_float4(dot(A1, A2), dot(A2, A2), dot(C0, C0), dot(C0, C1));
    out[2] = make_float4(dot(C0, C2), dot(C1, C1), dot(C1, C2), dot(C2, C2));
}

// The test of the record (px0, py0, log2 K from the record; Gram matrices from cull_row; sg00 =
// sqrtf(g00) = |A0| and sg11 = sqrtf(g11) = |A1|, formed once per staged record by the thread that
// stages it rather than once per warp that tests it).
__device__ __forceinline__ bool box_may_blend(const float4 &ga, const float4 &gb, const float4 &gc, float px0,
                                              float py0, float l2K, float sg00, float sg11, const BoxCull &bc) {
    const float g00 = ga.x, g01 = ga.y, g02 = ga.z, g11 = ga.w, g12 = gb.x, g22 = gb.y;
    const float k00 = gb.z, k01 = gb.w, k02 = gc.x, k11 = gc.y, k12 = gc.z, k22 = gc.w;
    const float ex0 = bc.x0 - px0, ex1 = bc.x1 - px0, ey0 = bc.y0 - py0, ey1 = bc.y1 - py0;
    const float cx = 0.5f * (ex0 + ex1), cy = 0.5f * (ey0 + ey1), hx = 0.5f * (ex1 - ex0), hy = 0.5f * (ey1 - ey0);
    // |A u_c|^2 = u_c^T G u_c with u_c = (cx, cy, 1)
    const float au2 = fmaf(cx, fmaf(g00, cx, 2.0f * fmaf(g01, cy, g02)), fmaf(cy, fmaf(g11, cy, 2.0f * g12), g22));
    const float low = sqrtf(fmaxf(au2, 0.0f)) * 0.9999f - sg00 * hx - sg11 * hy;
    if (!(low > 0.0f)) return true;                      // no useful amplitude bound: keep
    const float t = l2K + bc.l2dmax - __log2f(low) - bc.l2tskip;   // log2(Amax / tau_skip)
    if (!(t > -1e-3f)) return false;                     // Amax < tau_skip: no pixel blends
    const float r2s = fmaf(1.3862944f * 1.001f, fmaxf(t, 0.0f), 1e-2f);   // 2 ln 2 t, inflated
    const float h00 = fmaf(-r2s, g00, k00), h01 = fmaf(-r2s, g01, k01), h11 = fmaf(-r2s, g11, k11);
    const float b0 = fmaf(-r2s, g02, k02), b1 = fmaf(-r2s, g12, k12), c0 = fmaf(-r2s, g22, k22);
    const float det = fmaf(h00, h11, -h01 * h01);
    if (!(h00 > 0.0f) || !(h11 > 0.0f) || !(det > 0.0f)) return true;   // not an ellipse: keep
    const float rdet = rcp_approx(det);
    const float xs = (h01 * b1 - h11 * b0) * rdet, ys = (h01 * b0 - h00 * b1) * rdet;
    // the ellipse centre within a pixel of the box: keep (its neighbourhood is the minimum)
    if (xs >= ex0 - 1.0f && xs <= ex1 + 1.0f && ys >= ey0 - 1.0f && ys <= ey1 + 1.0f) return true;
    // otherwise the minimum lies on an edge: y = ey0 / ey1 (quadratic in x), x = ex0 / ex1 (in y)
    const float rh00 = rcp_approx(h00), rh11 = rcp_approx(h11);
    float q = quad_edge_min(h00, rh00, fmaf(h01, ey0, b0), fmaf(fmaf(h11, ey0, 2.0f * b1), ey0, c0), ex0, ex1);
    q = fminf(q, quad_edge_min(h00, rh00, fmaf(h01, ey1, b0), fmaf(fmaf(h11, ey1, 2.0f * b1), ey1, c0), ex0, ex1));
    q = fminf(q, quad_edge_min(h11, rh11, fmaf(h01, ex0, b1), fmaf(fmaf(h00, ex0, 2.0f * b0), ex0, c0), ey0, ey1));
    q = fminf(q, quad_edge_min(h11, rh11, fmaf(h01, ex1, b1), fmaf(fmaf(h00, ex1, 2.0f * b0), ex1, c0), ey0, ey1));
    return q <= 0.0f;
}

struct ColBase {
    float dx;              // x - px0 of the column
    float ip[3], ic[3];    // fma(A0, dx, A2) and fma(C0, dx, C2)
};

__device__ __forceinline__ void col_base(const float4 &r0, const float4 &r1, const float4 &r2, const float4 &r3,
                                         const float4 &r4, float x, ColBase &b) {
    b.dx = __fsub_rn(x, r4.z);
    b.ip[0] = fmaf(r0.x, b.dx, r1.z);
    b.ip[1] = fmaf(r0.y, b.dx, r1.w);
    b.ip[2] = fmaf(r0.z, b.dx, r2.x);
    b.ic[0] = fmaf(r2.y, b.dx, r3.w);
    b.ic[1] = fmaf(r2.z, b.dx, r4.x);
    b.ic[2] = fmaf(r2.w, b.dx, r4.y);
}

// d', o' x d', (dx, dy) and tau (unclamped) of the pixel in row y of the column b.
__device__ __forceinline__ void pair_eval_col(const float4 &r0, const float4 &r1, const float4 &r3, const float4 &r4,
                                              const float4 &r5, const ColBase &b, float y, float Lp, PairEval &e) {
    e.dx = b.dx;
    e.dy = __fsub_rn(y, r4.w);
    e.dp[0] = fmaf(r0.w, e.dy, b.ip[0]);
    e.dp[1] = fmaf(r1.x, e.dy, b.ip[1]);
    e.dp[2] = fmaf(r1.y, e.dy, b.ip[2]);
    e.cr[0] = fmaf(r3.x, e.dy, b.ic[0]);
    e.cr[1] = fmaf(r3.y, e.dy, b.ic[1]);
    e.cr[2] = fmaf(r3.z, e.dy, b.ic[2]);
    const float a = fmaf(e.dp[0], e.dp[0], fmaf(e.dp[1], e.dp[1], __fmul_rn(e.dp[2], e.dp[2])));
    const float q = fmaf(e.cr[0], e.cr[0], fmaf(e.cr[1], e.cr[1], __fmul_rn(e.cr[2], e.cr[2])));
    e.rs = rsqrt_approx(a);
    e.m2 = __fmul_rn(q, __fmul_rn(e.rs, e.rs));
    e.tau = __fmul_rn(ex2_approx(fmaf(e.m2, -kHalfLog2e, __fadd_rn(r5.x, Lp))), e.rs);
}

// ------------------------------------------------------------------ splat mode (Eq. 5-7)
// The record's C rows hold L^T (Sigma'^-1 = L L^T) relative to the reference pixel, its third
// row zero: q = |C u|^2 = w' Sigma'^-1 w needs two components per pixel, and
//   alpha = min(o exp(-q/2), alpha_max) = min(ex2(log2 o - q log2(e)/2), alpha_max).
// The blend runs on tau = -ln(1 - alpha) (log1pf, exact to rounding for small alpha), so the
// transmittance update, the stored S = sum tau and the backward's log-space replay are those
// of the default mode.  Forward and backward evaluate with the same operations.
struct SplatCol {
    float dx;        // x - px0 of the column
    float i0, i1;    // fma(C0, dx, C2), two components
};

__device__ __forceinline__ void splat_col(const float4 &r2, const float4 &r3, const float4 &r4, float x, SplatCol &b) {
    b.dx = __fsub_rn(x, r4.z);
    b.i0 = fmaf(r2.y, b.dx, r3.w);
    b.i1 = fmaf(r2.z, b.dx, r4.x);
}

// (dx, dy) and q = |C u|^2 of the pixel in row y of the column b (the same operations for every
// pixel layout); returns the unclamped opacity o G'(p).
__device__ __forceinline__ float splat_at(const float4 &r3, const float4 &r4, const float4 &r5, const SplatCol &b,
                                          float y, float &dx, float &dy, float &q) {
    dx = b.dx;
    dy = __fsub_rn(y, r4.w);
    const float c0 = fmaf(r3.x, dy, b.i0), c1 = fmaf(r3.y, dy, b.i1);
    q = fmaf(c0, c0, __fmul_rn(c1, c1));
    return ex2_approx(fmaf(q, -kHalfLog2e, r5.x));
}

// The opacity box test of the splat mode: box_may_blend with the record's A = (0, 0, e_z)
// (|A u| = 1) and the amplitude o alone, so the radius is r^2 = 2 ln(o / alpha_min).
__device__ __forceinline__ BoxCull box_cull_splat(const WarpBox &b, float alpha_min) {
    BoxCull c;
    c.x0 = (float)b.x0;
    c.y0 = (float)b.y0;
    c.x1 = (float)b.x1;
    c.y1 = (float)b.y1;
    c.l2dmax = 1e-4f;
    c.l2tskip = __log2f(alpha_min);
    return c;
}

// Asynchronous global-to-shared copies (cp.async): 16 bytes (both addresses 16-byte aligned)
// and 8 bytes (8-byte aligned); cp_async_wait() waits for all of the thread's copies.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// mbarrier objects in shared memory (CTA scope).  arrive has release semantics and try_wait
// acquire semantics (the PTX defaults), so stores before an arrive are visible to a thread whose
// wait saw that phase complete, and loads before an arrive are done before any store that
// follows such a wait.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the completion of the barrier phase of the given parity: returns false
// once limit_ns have passed, or as soon as *abort is set by another warp of the CTA that gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned long long limit_ns,
                                          const volatile int *abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (*abort || globaltimer_ns() - t0 > limit_ns) return false;
    return true;
}

// Vector reductions into global memory (red.global.add.v2/v4.f32, no return value): p must be
// 8- / 16-byte aligned.
__device__ __forceinline__ void red_add_v2(float *p, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// Partial warp reduce-scatter of NP per-lane values (NP a power of two): in exchange step s
// (partner lane^(16>>s)) the lane keeps one half of the values it still holds, adds the
// partner's copy of that half and hands over the other half.  After S steps the lane's
// v[0 .. NP>>S) hold the sums, over the 2^S lanes that differ only in lane bits 4 .. 5-S, of
// the values [base, base + (NP>>S)); base is returned.  NP>>S values cost NP - (NP>>S) shuffles.
template <int NP, int S>
__device__ __forceinline__ int warp_reduce_scatter_part(float (&v)[NP], int lane) {
    static_assert(S >= 1 && (NP >> S) >= 1 && S <= 5, "bad step count");
    int base = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int w = 16 >> s;
        const int h = (NP >> s) / 2;
        const bool hi = (lane & w) != 0;
        if (hi) base += h;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float keep = hi ? v[i + h] : v[i];
            const float send = hi ? v[i] : v[i + h];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return base;
}

}  // namespace vg
