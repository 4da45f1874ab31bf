// Per-(view, Gaussian) geometry used by the preprocess kernel and recomputed by the
// backward chain kernel, so that both see bit-identical records.
#pragma once

#include <type_traits>

#include <float.h>

#include "vg_internal.cuh"

namespace vg {

// FP32 with explicit rounding: these wrappers keep nvcc from fusing a multiply and an add,
// so the key function below yields the same bits as any IEEE implementation of the same
// operation sequence.
#define VG_MUL(a, b) __fmul_rn((a), (b))
#define VG_ADD(a, b) __fadd_rn((a), (b))
#define VG_SUB(a, b) __fsub_rn((a), (b))
#define VG_DIV(a, b) __fdiv_rn((a), (b))
#define VG_SQRT(a) __fsqrt_rn(a)

// log2(sqrt(2 pi))
constexpr float kLog2Sqrt2Pi = 1.32574806473615935f;
constexpr float kLog2e = 1.44269504088896341f;

template <typename RT>
__device__ __forceinline__ void load_gauss(const GaussIn &g, long long i, float mu[3], float s[3], float q[4],
                                           float &kap) {
    const RT *m = (const RT *)g.mu, *sc = (const RT *)g.scale, *qq = (const RT *)g.quat, *k = (const RT *)g.kappa;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        mu[c] = g.mu_f32 ? ld_f<float>((const float *)g.mu, 3 * i + c) : ld_f<RT>(m, 3 * i + c);
        s[c] = ld_f<RT>(sc, 3 * i + c);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = ld_f<RT>(qq, 4 * i + c);
    kap = ld_f<RT>(k, i);
}

// ------------------------------------------------------------------ density (Eq. 20)
// With GaussIn::density_theta the density input is theta in [0, 1] and
//   kappa = -ln(1 - 0.99 theta) (1/s_x + 1/s_y + 1/s_z) / 3   (Eq. 20).
// kap_key, which sizes the footprint in the bit-exact key function, is an upper bound of kappa
// made of correctly rounded operations and the binary exponent only: with x = 0.99 theta and
// 1 - x = m 2^e (m in [0.5, 1)), -ln(1 - x) <= min(x / (1 - x), (1 - e) ln 2).
struct Density {
    float kap_key;   // key function (validity and footprint)
    float kap;       // the record's amplitude
    float lnv;       // -ln(1 - 0.99 theta)    (density_theta only)
    float m;         // (1/s_x + 1/s_y + 1/s_z) / 3
};

__device__ __forceinline__ Density density_of(const GaussIn &g, float kin, const float s[3]) {
    Density d;
    if (!g.density_theta) {
        d.kap_key = d.kap = kin;
        d.lnv = d.m = 0.0f;
        return d;
    }
    d.m = __fmul_rn(__fadd_rn(__fadd_rn(__fdiv_rn(1.0f, s[0]), __fdiv_rn(1.0f, s[1])), __fdiv_rn(1.0f, s[2])),
                    0.33333334f);
    if (!(kin > 0.0f && kin <= 1.0f)) {   // outside (0, 1] (or NaN): no density, culled
        d.kap_key = d.kap = d.lnv = 0.0f;
        return d;
    }
    const float x = __fmul_rn(0.99f, kin);
    const float om = __fsub_rn(1.0f, x);
    const float b1 = __fdiv_rn(x, om);
    const int e = (int)((__float_as_uint(om) >> 23) & 0xFFu) - 126;   // om = m 2^e, m in [0.5, 1)
    const float b2 = __fmul_rn((float)(1 - e), 0.6931472f);
    d.kap_key = __fmul_rn(fminf(b1, b2), d.m);
    d.lnv = -log1pf(-x);
    d.kap = d.lnv * d.m;
    return d;
}

// Colour activation and its derivative: the clamp at 0, or the softplus (1/beta) ln(1 + e^(beta x))
__device__ __forceinline__ float colour_act(float x, float beta) {
    if (!(beta > 0.0f)) return fmaxf(x, 0.0f);
    const float t = beta * x;
    return (t > 0.0f ? t + log1pf(__expf(-t)) : log1pf(__expf(t))) / beta;
}

__device__ __forceinline__ float colour_act_grad(float x, float beta) {
    if (!(beta > 0.0f)) return x > 0.0f ? 1.0f : 0.0f;
    return 1.0f / (1.0f + __expf(-beta * x));
}

// Validity, unit quaternion, rotation Rq and world covariance Sigma = Rq S^2 Rq^T, FP32 with
// a fixed operation order (the key function's first stage).
__device__ __forceinline__ bool key_cov(const float mu[3], const float s[3], const float q[4], float kap,
                                        float Sig[9], float Rq[9], float qn[4], float &smax) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (!isfinite(mu[k]) || !isfinite(s[k]) || !(s[k] > 0.0f)) return false;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (!isfinite(q[k])) return false;
    if (!isfinite(kap) || !(kap > 0.0f)) return false;
    float n2 = VG_ADD(VG_ADD(VG_ADD(VG_MUL(q[0], q[0]), VG_MUL(q[1], q[1])), VG_MUL(q[2], q[2])), VG_MUL(q[3], q[3]));
    if (!(n2 > 0.0f) || !isfinite(n2)) return false;
    float inv = VG_DIV(1.0f, VG_SQRT(n2));
    float w = VG_MUL(q[0], inv), x = VG_MUL(q[1], inv), y = VG_MUL(q[2], inv), z = VG_MUL(q[3], inv);
    qn[0] = w;
    qn[1] = x;
    qn[2] = y;
    qn[3] = z;
    Rq[0] = VG_SUB(1.0f, VG_MUL(2.0f, VG_ADD(VG_MUL(y, y), VG_MUL(z, z))));
    Rq[1] = VG_MUL(2.0f, VG_SUB(VG_MUL(x, y), VG_MUL(w, z)));
    Rq[2] = VG_MUL(2.0f, VG_ADD(VG_MUL(x, z), VG_MUL(w, y)));
    Rq[3] = VG_MUL(2.0f, VG_ADD(VG_MUL(x, y), VG_MUL(w, z)));
    Rq[4] = VG_SUB(1.0f, VG_MUL(2.0f, VG_ADD(VG_MUL(x, x), VG_MUL(z, z))));
    Rq[5] = VG_MUL(2.0f, VG_SUB(VG_MUL(y, z), VG_MUL(w, x)));
    Rq[6] = VG_MUL(2.0f, VG_SUB(VG_MUL(x, z), VG_MUL(w, y)));
    Rq[7] = VG_MUL(2.0f, VG_ADD(VG_MUL(y, z), VG_MUL(w, x)));
    Rq[8] = VG_SUB(1.0f, VG_MUL(2.0f, VG_ADD(VG_MUL(x, x), VG_MUL(y, y))));
    float v0 = VG_MUL(s[0], s[0]), v1 = VG_MUL(s[1], s[1]), v2 = VG_MUL(s[2], s[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Sig[3 * i + j] = VG_ADD(VG_ADD(VG_MUL(VG_MUL(Rq[3 * i], v0), Rq[3 * j]),
                                           VG_MUL(VG_MUL(Rq[3 * i + 1], v1), Rq[3 * j + 1])),
                                    VG_MUL(VG_MUL(Rq[3 * i + 2], v2), Rq[3 * j + 2]));
    smax = fmaxf(fmaxf(s[0], s[1]), s[2]);
    return true;
}

// k^2 with tau >= tau_cut => Mahalanobis m^2 <= k^2: tau <= kappa sqrt(2 pi) s_max exp(-m^2/2)
// and ln x <= e ln 2 for x = m 2^e, m in [0.5, 1).  No transcendental function involved.
__device__ __forceinline__ bool key_k2(float kap, float smax, float tau_cut, float &k2) {
    float xr = VG_DIV(VG_MUL(VG_MUL(kap, 2.5066283f), smax), tau_cut);
    if (!(xr > 1.0f)) return false;
    int e = (xr > FLT_MAX) ? 128 : (int)((__float_as_uint(xr) >> 23) & 0xFFu) - 126;
    k2 = VG_MUL((float)e, 1.3862944f);
    return true;
}

// Pixel indices whose centre coordinate lies in [lo, hi] after a small outward pad;
// returns lo > hi when empty.
__device__ __forceinline__ void pixel_span(float lo, float hi, int n, int &ilo, int &ihi) {
    lo = VG_SUB(lo, VG_ADD(0.02f, VG_MUL(1e-5f, fabsf(lo))));
    hi = VG_ADD(hi, VG_ADD(0.02f, VG_MUL(1e-5f, fabsf(hi))));
    if (!(hi >= 0.0f) || !(lo <= (float)(n - 1))) {
        ilo = 1;
        ihi = 0;
        return;
    }
    ilo = (lo <= 0.0f) ? 0 : (int)ceilf(lo);
    ihi = (hi >= (float)(n - 1)) ? n - 1 : (int)floorf(hi);
}

// Key function of one (view, Gaussian): camera depth of the mean (FP32 bits), the
// conservative pixel rectangle of the Mahalanobis-k ellipsoid's screen bounding box (a
// Gaussian contributes only to these pixels) and the tile rectangle covering it.
// Returns 0 = invalid/behind z_near, 1 = valid but no footprint, 2 = visible.
__device__ __forceinline__ int key_persp(const ViewInfo &V, const float mu[3], const float Sig[9], float smax,
                                         float kap, float z_near, float tau_cut, uint32_t &depth, short4 &rect,
                                         short4 &prect, float &Zf) {
    const float *C = V.R;
    float X = VG_ADD(VG_ADD(VG_ADD(VG_MUL(C[0], mu[0]), VG_MUL(C[1], mu[1])), VG_MUL(C[2], mu[2])), V.t[0]);
    float Y = VG_ADD(VG_ADD(VG_ADD(VG_MUL(C[3], mu[0]), VG_MUL(C[4], mu[1])), VG_MUL(C[5], mu[2])), V.t[1]);
    float Z = VG_ADD(VG_ADD(VG_ADD(VG_MUL(C[6], mu[0]), VG_MUL(C[7], mu[1])), VG_MUL(C[8], mu[2])), V.t[2]);
    Zf = Z;
    if (!(Z > z_near)) return 0;
    depth = __float_as_uint(Z);
    float k2;
    if (!key_k2(kap, smax, tau_cut, k2)) return 1;
    float T[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = VG_ADD(VG_ADD(VG_MUL(C[3 * i], Sig[j]), VG_MUL(C[3 * i + 1], Sig[3 + j])),
                                  VG_MUL(C[3 * i + 2], Sig[6 + j]));
    float sxx = VG_ADD(VG_ADD(VG_MUL(T[0], C[0]), VG_MUL(T[1], C[1])), VG_MUL(T[2], C[2]));
    float sxz = VG_ADD(VG_ADD(VG_MUL(T[0], C[6]), VG_MUL(T[1], C[7])), VG_MUL(T[2], C[8]));
    float syy = VG_ADD(VG_ADD(VG_MUL(T[3], C[3]), VG_MUL(T[4], C[4])), VG_MUL(T[5], C[5]));
    float syz = VG_ADD(VG_ADD(VG_MUL(T[3], C[6]), VG_MUL(T[4], C[7])), VG_MUL(T[5], C[8]));
    float szz = VG_ADD(VG_ADD(VG_MUL(T[6], C[6]), VG_MUL(T[7], C[7])), VG_MUL(T[8], C[8]));
    float ZZ = VG_MUL(Z, Z);
    float a2 = VG_SUB(ZZ, VG_MUL(k2, szz));
    if (!(a2 > 0.0f)) {   // the cutoff ellipsoid reaches the camera plane: the whole view
        rect = make_short4(0, 0, (short)(V.tiles_x - 1), (short)(V.tiles_y - 1));
        prect = make_short4(0, 0, (short)(V.W - 1), (short)(V.H - 1));
        return 2;
    }
    float k22 = VG_MUL(k2, k2);
    float XZ = VG_MUL(X, Z), YZ = VG_MUL(Y, Z);
    float bu = VG_SUB(XZ, VG_MUL(k2, sxz));
    float qu = VG_ADD(VG_SUB(VG_MUL(ZZ, sxx), VG_MUL(2.0f, VG_MUL(XZ, sxz))), VG_MUL(VG_MUL(X, X), szz));
    float du = VG_SUB(VG_MUL(k2, qu), VG_MUL(k22, VG_SUB(VG_MUL(sxx, szz), VG_MUL(sxz, sxz))));
    if (!(du > 0.0f)) du = 0.0f;
    float ru = VG_SQRT(du);
    float ulo = VG_DIV(VG_SUB(bu, ru), a2), uhi = VG_DIV(VG_ADD(bu, ru), a2);
    float bv = VG_SUB(YZ, VG_MUL(k2, syz));
    float qv = VG_ADD(VG_SUB(VG_MUL(ZZ, syy), VG_MUL(2.0f, VG_MUL(YZ, syz))), VG_MUL(VG_MUL(Y, Y), szz));
    float dv = VG_SUB(VG_MUL(k2, qv), VG_MUL(k22, VG_SUB(VG_MUL(syy, szz), VG_MUL(syz, syz))));
    if (!(dv > 0.0f)) dv = 0.0f;
    float rv = VG_SQRT(dv);
    float vlo = VG_DIV(VG_SUB(bv, rv), a2), vhi = VG_DIV(VG_ADD(bv, rv), a2);
    float xlo = VG_SUB(VG_ADD(VG_MUL(ulo, V.fx), V.cx), 0.5f), xhi = VG_SUB(VG_ADD(VG_MUL(uhi, V.fx), V.cx), 0.5f);
    float ylo = VG_SUB(VG_ADD(VG_MUL(vlo, V.fy), V.cy), 0.5f), yhi = VG_SUB(VG_ADD(VG_MUL(vhi, V.fy), V.cy), 0.5f);
    int ix0, ix1, iy0, iy1;
    pixel_span(xlo, xhi, V.W, ix0, ix1);
    pixel_span(ylo, yhi, V.H, iy0, iy1);
    if (ix0 > ix1 || iy0 > iy1) return 1;
    rect = make_short4((short)(ix0 / V.tw), (short)(iy0 / V.th), (short)(ix1 / V.tw), (short)(iy1 / V.th));
    prect = make_short4((short)ix0, (short)iy0, (short)ix1, (short)iy1);
    return 2;
}

// Splat-mode key function (the 3DGS comparison mode, Eq. 5-7): the depth key of key_persp and
// the pixel bounding box of the 2D Gaussian's ellipse w' Sigma'^-1 w <= k^2, Sigma' = J W Sigma
// W^T J^T + dil I with J the projection's Jacobian at the mean, k^2 = 2 ln 2 * e where
// opacity / alpha_cut = m 2^e (so that every pixel outside has o G' < alpha_cut).  Its
// half-widths are k sqrt(Sigma'_xx) and k sqrt(Sigma'_yy).  FP32, fixed operation order.
// Returns 0 = invalid/behind z_near, 1 = valid but no footprint, 2 = visible.
__device__ __forceinline__ int key_splat(const ViewInfo &V, const float mu[3], const float Sig[9], float opac,
                                         float z_near, float alpha_cut, float dil, uint32_t &depth, short4 &rect,
                                         short4 &prect) {
    const float *C = V.R;
    float X = VG_ADD(VG_ADD(VG_ADD(VG_MUL(C[0], mu[0]), VG_MUL(C[1], mu[1])), VG_MUL(C[2], mu[2])), V.t[0]);
    float Y = VG_ADD(VG_ADD(VG_ADD(VG_MUL(C[3], mu[0]), VG_MUL(C[4], mu[1])), VG_MUL(C[5], mu[2])), V.t[1]);
    float Z = VG_ADD(VG_ADD(VG_ADD(VG_MUL(C[6], mu[0]), VG_MUL(C[7], mu[1])), VG_MUL(C[8], mu[2])), V.t[2]);
    if (!(Z > z_near)) return 0;
    depth = __float_as_uint(Z);
    const float xr = VG_DIV(opac, alpha_cut);
    if (!(xr > 1.0f)) return 1;
    const int e = (xr > FLT_MAX) ? 128 : (int)((__float_as_uint(xr) >> 23) & 0xFFu) - 126;
    const float k2 = VG_MUL((float)e, 1.3862944f);
    float T[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = VG_ADD(VG_ADD(VG_MUL(C[3 * i], Sig[j]), VG_MUL(C[3 * i + 1], Sig[3 + j])),
                                  VG_MUL(C[3 * i + 2], Sig[6 + j]));
    const float sxx = VG_ADD(VG_ADD(VG_MUL(T[0], C[0]), VG_MUL(T[1], C[1])), VG_MUL(T[2], C[2]));
    const float sxz = VG_ADD(VG_ADD(VG_MUL(T[0], C[6]), VG_MUL(T[1], C[7])), VG_MUL(T[2], C[8]));
    const float syy = VG_ADD(VG_ADD(VG_MUL(T[3], C[3]), VG_MUL(T[4], C[4])), VG_MUL(T[5], C[5]));
    const float syz = VG_ADD(VG_ADD(VG_MUL(T[3], C[6]), VG_MUL(T[4], C[7])), VG_MUL(T[5], C[8]));
    const float szz = VG_ADD(VG_ADD(VG_MUL(T[6], C[6]), VG_MUL(T[7], C[7])), VG_MUL(T[8], C[8]));
    const float u = VG_DIV(X, Z), v = VG_DIV(Y, Z);
    const float jx = VG_DIV(V.fx, Z), jy = VG_DIV(V.fy, Z);
    float exx = VG_ADD(VG_SUB(sxx, VG_MUL(2.0f, VG_MUL(u, sxz))), VG_MUL(VG_MUL(u, u), szz));
    float eyy = VG_ADD(VG_SUB(syy, VG_MUL(2.0f, VG_MUL(v, syz))), VG_MUL(VG_MUL(v, v), szz));
    if (!(exx > 0.0f)) exx = 0.0f;
    if (!(eyy > 0.0f)) eyy = 0.0f;
    const float vx = VG_ADD(VG_MUL(VG_MUL(jx, jx), exx), dil), vy = VG_ADD(VG_MUL(VG_MUL(jy, jy), eyy), dil);
    const float hx = VG_SQRT(VG_MUL(k2, vx)), hy = VG_SQRT(VG_MUL(k2, vy));
    const float mx = VG_SUB(VG_ADD(VG_MUL(u, V.fx), V.cx), 0.5f), my = VG_SUB(VG_ADD(VG_MUL(v, V.fy), V.cy), 0.5f);
    int ix0, ix1, iy0, iy1;
    pixel_span(VG_SUB(mx, hx), VG_ADD(mx, hx), V.W, ix0, ix1);
    pixel_span(VG_SUB(my, hy), VG_ADD(my, hy), V.H, iy0, iy1);
    if (ix0 > ix1 || iy0 > iy1) return 1;
    rect = make_short4((short)(ix0 / V.tw), (short)(iy0 / V.th), (short)(ix1 / V.tw), (short)(iy1 / V.th));
    prect = make_short4((short)ix0, (short)iy0, (short)ix1, (short)iy1);
    return 2;
}

// ------------------------------------------------------------------ double-float arithmetic
// Error-free transformations in FP32: two_sum (Knuth) gives s + e == a + b exactly, two_prod
// (via FMA) gives p + e == a * b exactly.  Sums of products accumulated with them as in the
// Dot2 algorithm (Ogita, Rump, Oishi: "Accurate Sum and Dot Product", SIAM J. Sci. Comput. 2005)
// are as accurate as if computed in twice the working precision, i.e. ~48 significant bits,
// on the FP32 pipe (GB300's FP64 rate is a small fraction of its FP32 rate).
struct DF {
    float hi, lo;   // unevaluated sum hi + lo
};

__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF{s, e};
}

__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return DF{p, fmaf(a, b, -p)};
}

// acc + a * b with the product and the leading sum error-free (one Dot2 step)
__device__ __forceinline__ DF df_fma(DF acc, float a, float b) {
    const DF p = two_prod(a, b);
    const DF s = two_sum(acc.hi, p.hi);
    return DF{s.hi, __fadd_rn(acc.lo, __fadd_rn(s.lo, p.lo))};
}

// acc + a * (b.hi + b.lo)
__device__ __forceinline__ DF df_fma(DF acc, float a, DF b) {
    DF r = df_fma(acc, a, b.hi);
    r.lo = fmaf(a, b.lo, r.lo);
    return r;
}

__device__ __forceinline__ DF df_add(DF acc, DF b) {
    const DF s = two_sum(acc.hi, b.hi);
    return DF{s.hi, __fadd_rn(acc.lo, __fadd_rn(s.lo, b.lo))};
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

__device__ __forceinline__ float df_float(DF a) { return __fadd_rn(a.hi, a.lo); }

// renormalised so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ DF df_norm(DF a) {
    const float s = __fadd_rn(a.hi, a.lo);
    return DF{s, __fsub_rn(a.lo, __fsub_rn(s, a.hi))};
}

// ------------------------------------------------------------------ record geometry
// Blend-record geometry of one (view, Gaussian).  With B = Rc Rq and M = S^-1 B^T the
// whitening in camera coordinates, a pixel ray d_c = (u, v, 1) maps to d' = M d_c and the
// camera centre to o' = -M mu_c.  Pixels are addressed relative to the projected mean
// (px0, py0), so that d' = A0 dx + A1 dy + A2 and o' x d' = C0 dx + C1 dy + C2 with
// C2 ~ 0: the cancellation-prone cross product is formed per Gaussian in extra precision
// (double-float) instead of per pixel.
struct ItemGeom {
    float M[9];        // row-major
    DF muc[3];         // camera-space mean, double-float
    DF opx[3];         // o' = -M mu_c, double-float
    float op[3];       // o' rounded to FP32
    float px0, py0;    // reference pixel: the projected mean in FP32
    float dc0[3];      // camera ray through the reference pixel
    float Dx, Dy;      // reference pixel minus the exact projection, in pixels
    float A[9];        // A0, A1, A2 (rows of 3)
    float Cc[9];       // C0, C1, C2
};

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ void item_geom(const ViewInfo &V, const float mu[3], const float s[3], const float Rq[9],
                                          ItemGeom &G) {
    const float *Rc = V.R;
    float B[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            B[3 * i + j] = Rc[3 * i] * Rq[j] + Rc[3 * i + 1] * Rq[3 + j] + Rc[3 * i + 2] * Rq[6 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float is = 1.0f / s[i];
#pragma unroll
        for (int j = 0; j < 3; ++j) G.M[3 * i + j] = B[3 * j + i] * is;
    }
    // mu_c = Rc mu + t and o' = -M mu_c, both to ~48 bits
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        DF acc = DF{V.t[k], 0.0f};
        acc = df_fma(acc, Rc[3 * k], mu[0]);
        acc = df_fma(acc, Rc[3 * k + 1], mu[1]);
        acc = df_fma(acc, Rc[3 * k + 2], mu[2]);
        G.muc[k] = df_norm(acc);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        DF acc = DF{0.0f, 0.0f};
        acc = df_fma(acc, -G.M[3 * i], G.muc[0]);
        acc = df_fma(acc, -G.M[3 * i + 1], G.muc[1]);
        acc = df_fma(acc, -G.M[3 * i + 2], G.muc[2]);
        G.opx[i] = df_norm(acc);
        G.op[i] = G.opx[i].hi;
    }
    const float Xf = G.muc[0].hi, Yf = G.muc[1].hi, Zf = G.muc[2].hi;
    const float izf = 1.0f / Zf;
    G.px0 = fmaf(V.fx, Xf * izf, V.cx - 0.5f);
    G.py0 = fmaf(V.fy, Yf * izf, V.cy - 0.5f);
    // (px0 + 0.5 - cx) exactly as a double-float; then D = (e Z - f X) / Z to ~48 bits before rounding
    const DF ex = df_add(two_sum(G.px0, 0.5f), DF{-V.cx, 0.0f});
    const DF ey = df_add(two_sum(G.py0, 0.5f), DF{-V.cy, 0.0f});
    DF nx = df_fma(DF{0.0f, 0.0f}, ex.hi, G.muc[2]);
    nx.lo = fmaf(ex.lo, G.muc[2].hi, nx.lo);
    nx = df_fma(nx, -V.fx, G.muc[0]);
    DF ny = df_fma(DF{0.0f, 0.0f}, ey.hi, G.muc[2]);
    ny.lo = fmaf(ey.lo, G.muc[2].hi, ny.lo);
    ny = df_fma(ny, -V.fy, G.muc[1]);
    G.Dx = df_float(nx) * izf;
    G.Dy = df_float(ny) * izf;
    G.dc0[0] = df_float(ex) / V.fx;
    G.dc0[1] = df_float(ey) / V.fy;
    G.dc0[2] = 1.0f;
    float ifx = 1.0f / V.fx, ify = 1.0f / V.fy;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        G.A[i] = G.M[3 * i] * ifx;
        G.A[3 + i] = G.M[3 * i + 1] * ify;
        G.A[6 + i] = G.M[3 * i] * G.dc0[0] + G.M[3 * i + 1] * G.dc0[1] + G.M[3 * i + 2];
    }
    cross3(G.op, &G.A[0], &G.Cc[0]);
    cross3(G.op, &G.A[3], &G.Cc[3]);
#pragma unroll
    for (int i = 0; i < 3; ++i) G.Cc[6 + i] = G.Cc[i] * G.Dx + G.Cc[3 + i] * G.Dy;
}

// ------------------------------------------------------------------ splat-mode geometry
// a b - c d to within about 1.5 ulp with one FMA-exact product (Kahan's 2x2 determinant;
// Jeannerod, Louvet, Muller, "Further analysis of Kahan's algorithm for the accurate
// computation of 2x2 determinants", Math. Comp. 82, 2013).
__device__ __forceinline__ float diff_prod(float a, float b, float c, float d) {
    const float w = __fmul_rn(c, d);
    const float e = fmaf(-c, d, w);
    const float f = fmaf(a, b, -w);
    return __fadd_rn(f, e);
}

// x / y in double-float: the remainder x.hi - q1 y.hi of the rounded quotient is exact
// through an FMA, the low parts enter its correction.
__device__ __forceinline__ DF df_div(DF x, DF y) {
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const float r = __fsub_rn(__fadd_rn(fmaf(-q1, y.hi, x.hi), x.lo), __fmul_rn(q1, y.lo));
    return DF{q1, __fdiv_rn(r, y.hi)};
}

// The 2D Gaussian of one (view, Gaussian) in the 3DGS comparison mode (Eq. 5-7).  With t the
// camera-space mean, u = tx/tz, v = ty/tz, jx = fx/tz, jy = fy/tz, the rows of J W are
// a_0 = jx (W_0 - u W_2) and a_1 = jy (W_1 - v W_2) (W_i the rows of the view rotation), and
// with B_ik = s_k (a_i . r_k) (r_k the Gaussian's axes) Sigma' = B B^T + dil I.  Its
// determinant is formed without cancellation, det = |n|^2 + dil (|b_0|^2 + |b_1|^2) + dil^2
// with n = b_0 x b_1 from Kahan's 2x2 determinants, so that thin footprints keep their
// accuracy in FP32.  The mean mu' = (fx u + cx - 1/2, fy v + cy - 1/2) (pixel index
// coordinates) is formed in double-float from the double-float camera-space mean and split
// into the reference pixel (px0, py0) (its leading part) and the remainder (mx, my).
struct SplatGeom {
    float u, v, jx, jy, iz;   // iz = 1 / tz
    float a[2][3];            // rows of J W
    float ar[2][3];           // a_i . r_k
    float B[2][3];
    float n[3];               // b_0 x b_1
    float g00, g01, g11, det; // Sigma' = [[g00, g01], [g01, g11]] and its determinant
    float px0, py0, mx, my;
};

__device__ __forceinline__ bool splat_geom(const ViewInfo &V, const float mu[3], const float s[3], const float Rq[9],
                                           float dil, SplatGeom &G) {
    const float *W = V.R;
    DF t[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        DF acc = DF{V.t[k], 0.0f};
        acc = df_fma(acc, W[3 * k], mu[0]);
        acc = df_fma(acc, W[3 * k + 1], mu[1]);
        acc = df_fma(acc, W[3 * k + 2], mu[2]);
        t[k] = df_norm(acc);
    }
    if (!(t[2].hi > 0.0f)) return false;
    const DF ud = df_div(t[0], t[2]), vd = df_div(t[1], t[2]);
    G.u = ud.hi;
    G.v = vd.hi;
    G.iz = 1.0f / t[2].hi;
    G.jx = V.fx * G.iz;
    G.jy = V.fy * G.iz;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        G.a[0][c] = G.jx * fmaf(-G.u, W[6 + c], W[c]);
        G.a[1][c] = G.jy * fmaf(-G.v, W[6 + c], W[3 + c]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            G.ar[i][k] = fmaf(G.a[i][0], Rq[k], fmaf(G.a[i][1], Rq[3 + k], G.a[i][2] * Rq[6 + k]));
            G.B[i][k] = s[k] * G.ar[i][k];
        }
    const float *b0 = G.B[0], *b1 = G.B[1];
    G.n[0] = diff_prod(b0[1], b1[2], b0[2], b1[1]);
    G.n[1] = diff_prod(b0[2], b1[0], b0[0], b1[2]);
    G.n[2] = diff_prod(b0[0], b1[1], b0[1], b1[0]);
    const float s00 = fmaf(b0[0], b0[0], fmaf(b0[1], b0[1], b0[2] * b0[2]));
    const float s11 = fmaf(b1[0], b1[0], fmaf(b1[1], b1[1], b1[2] * b1[2]));
    G.g00 = s00 + dil;
    G.g11 = s11 + dil;
    G.g01 = fmaf(b0[0], b1[0], fmaf(b0[1], b1[1], b0[2] * b1[2]));
    G.det = fmaf(G.n[0], G.n[0], fmaf(G.n[1], G.n[1], G.n[2] * G.n[2])) + dil * (s00 + s11 + dil);
    DF mx = df_norm(df_add(df_fma(DF{V.cx, 0.0f}, V.fx, ud), DF{-0.5f, 0.0f}));
    DF my = df_norm(df_add(df_fma(DF{V.cy, 0.0f}, V.fy, vd), DF{-0.5f, 0.0f}));
    G.px0 = mx.hi;
    G.py0 = my.hi;
    G.mx = mx.lo;
    G.my = my.lo;
    return G.det > 0.0f && isfinite(G.det);
}

// Splat-mode blend record in the layout of the default mode: q = w' Sigma'^-1 w = |C u|^2 with
// u = (dx, dy, 1), w = (dx - mx, dy - my) and C's rows L^T (Sigma'^-1 = L L^T, Cholesky):
//   L00 = sqrt(g11 / det), L10 = -g01 / sqrt(g11 det), L11 = 1 / sqrt(g11);
// A = (0, 0, e_z) makes |A u| = 1, unused by the splat kernels except in the opacity box test.
// A non-finite factor (a footprint far below a pixel) yields alpha = 0 through log2 o = -inf.
// Writes A, C and the reference pixel to out[0..19]; returns the record's log2 o.
__device__ __forceinline__ float splat_record(const SplatGeom &G, float opac, float out[20]) {
    float L00 = sqrtf(G.g11 / G.det), L10 = -G.g01 / sqrtf(G.g11 * G.det), L11 = 1.0f / sqrtf(G.g11);
    float l2o = log2f(opac);
    if (!(isfinite(L00) && isfinite(L10) && isfinite(L11))) {
        L00 = L10 = L11 = 0.0f;
        l2o = -INFINITY;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k] = 0.0f;
    out[8] = 1.0f;
    out[9] = L00;
    out[10] = 0.0f;
    out[11] = 0.0f;
    out[12] = L10;
    out[13] = L11;
    out[14] = 0.0f;
    out[15] = -fmaf(L00, G.mx, L10 * G.my);
    out[16] = -(L11 * G.my);
    out[17] = 0.0f;
    out[18] = G.px0;
    out[19] = G.py0;
    return l2o;
}

// ------------------------------------------------------------------ spherical harmonics
// Real spherical harmonics to degree 3 (Condon-Shortley phase); Y[k] for k < (deg+1)^2.
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float Y[16]) {
    Y[0] = 0.28209479177387814f;
    if (deg < 1) return;
    Y[1] = -0.48860251190291992f * y;
    Y[2] = 0.48860251190291992f * z;
    Y[3] = -0.48860251190291992f * x;
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = 1.0925484305920792f * x * y;
    Y[5] = -1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);
    Y[7] = -1.0925484305920792f * x * z;
    Y[8] = 0.54627421529603959f * (xx - yy);
    if (deg < 3) return;
    Y[9] = -0.59004358992664352f * y * (3.0f * xx - yy);
    Y[10] = 2.8906114426405538f * x * y * z;
    Y[11] = -0.45704579946446572f * y * (4.0f * zz - xx - yy);
    Y[12] = 0.37317633259011540f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -0.45704579946446572f * x * (4.0f * zz - xx - yy);
    Y[14] = 1.4453057213202769f * z * (xx - yy);
    Y[15] = -0.59004358992664352f * x * (xx - 3.0f * yy);
}

// Gradient of the basis polynomials with respect to (x, y, z), dY[k][c].
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float dY[16][3]) {
    dY[0][0] = dY[0][1] = dY[0][2] = 0.0f;
    if (deg < 1) return;
    const float c1 = 0.48860251190291992f;
    dY[1][0] = 0.0f; dY[1][1] = -c1; dY[1][2] = 0.0f;
    dY[2][0] = 0.0f; dY[2][1] = 0.0f; dY[2][2] = c1;
    dY[3][0] = -c1; dY[3][1] = 0.0f; dY[3][2] = 0.0f;
    if (deg < 2) return;
    const float a = 1.0925484305920792f, b = 0.31539156525252005f, c = 0.54627421529603959f;
    float xx = x * x, yy = y * y, zz = z * z;
    dY[4][0] = a * y;        dY[4][1] = a * x;        dY[4][2] = 0.0f;
    dY[5][0] = 0.0f;         dY[5][1] = -a * z;       dY[5][2] = -a * y;
    dY[6][0] = -2.0f * b * x; dY[6][1] = -2.0f * b * y; dY[6][2] = 4.0f * b * z;
    dY[7][0] = -a * z;       dY[7][1] = 0.0f;         dY[7][2] = -a * x;
    dY[8][0] = 2.0f * c * x; dY[8][1] = -2.0f * c * y; dY[8][2] = 0.0f;
    if (deg < 3) return;
    const float e = 0.59004358992664352f, f = 2.8906114426405538f, g = 0.45704579946446572f,
                h = 0.37317633259011540f, i = 1.4453057213202769f;
    dY[9][0] = -6.0f * e * x * y;  dY[9][1] = -3.0f * e * (xx - yy);  dY[9][2] = 0.0f;
    dY[10][0] = f * y * z;         dY[10][1] = f * x * z;             dY[10][2] = f * x * y;
    dY[11][0] = 2.0f * g * x * y;  dY[11][1] = -g * (4.0f * zz - xx - 3.0f * yy); dY[11][2] = -8.0f * g * y * z;
    dY[12][0] = -6.0f * h * x * z; dY[12][1] = -6.0f * h * y * z;     dY[12][2] = h * (6.0f * zz - 3.0f * xx - 3.0f * yy);
    dY[13][0] = -g * (4.0f * zz - 3.0f * xx - yy); dY[13][1] = 2.0f * g * x * y; dY[13][2] = -8.0f * g * x * z;
    dY[14][0] = 2.0f * i * x * z;  dY[14][1] = -2.0f * i * y * z;     dY[14][2] = i * (xx - yy);
    dY[15][0] = -3.0f * e * (xx - yy); dY[15][1] = 6.0f * e * x * y;  dY[15][2] = 0.0f;
}

// g = sum_k w_k grad Y_k(x, y, z): the basis gradients of sh_basis_grad, weighted and summed
// term by term without materialising them.
__device__ __forceinline__ void sh_grad_dot(int deg, float x, float y, float z, const float w[16], float g[3]) {
    g[0] = g[1] = g[2] = 0.0f;
    if (deg < 1) return;
    const float c1 = 0.48860251190291992f;
    g[0] = -c1 * w[3];
    g[1] = -c1 * w[1];
    g[2] = c1 * w[2];
    if (deg < 2) return;
    const float a = 1.0925484305920792f, b = 0.31539156525252005f, c = 0.54627421529603959f;
    const float xx = x * x, yy = y * y, zz = z * z;
    g[0] += a * y * w[4] - 2.0f * b * x * w[6] - a * z * w[7] + 2.0f * c * x * w[8];
    g[1] += a * x * w[4] - a * z * w[5] - 2.0f * b * y * w[6] - 2.0f * c * y * w[8];
    g[2] += -a * y * w[5] + 4.0f * b * z * w[6] - a * x * w[7];
    if (deg < 3) return;
    const float e = 0.59004358992664352f, f = 2.8906114426405538f, gg = 0.45704579946446572f,
                h = 0.37317633259011540f, i = 1.4453057213202769f;
    g[0] += -6.0f * e * x * y * w[9] + f * y * z * w[10] + 2.0f * gg * x * y * w[11] - 6.0f * h * x * z * w[12] -
            gg * (4.0f * zz - 3.0f * xx - yy) * w[13] + 2.0f * i * x * z * w[14] - 3.0f * e * (xx - yy) * w[15];
    g[1] += -3.0f * e * (xx - yy) * w[9] + f * x * z * w[10] - gg * (4.0f * zz - xx - 3.0f * yy) * w[11] -
            6.0f * h * y * z * w[12] + 2.0f * gg * x * y * w[13] - 2.0f * i * y * z * w[14] + 6.0f * e * x * y * w[15];
    g[2] += f * x * y * w[10] - 8.0f * gg * y * z * w[11] + h * (6.0f * zz - 3.0f * xx - 3.0f * yy) * w[12] -
            8.0f * gg * x * z * w[13] + i * (xx - yy) * w[14];
}

template <typename ST>
__device__ __forceinline__ void eval_colour(const GaussIn &g, long long gi, const float dir[3], float rgb[3],
                                            float raw[3]) {
    float Y[16];
    sh_basis(g.sh_degree, dir[0], dir[1], dir[2], Y);
    const int K = (g.sh_degree + 1) * (g.sh_degree + 1);
    const ST *sh = (const ST *)g.sh + (long long)gi * K * 3;
    float acc[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int k = 0; k < 16; ++k) {   // unrolled so that Y stays in registers
        if (k >= K) break;
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] = fmaf(ld_f<ST>(sh, 3 * k + c), Y[k], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        raw[c] = acc[c];
        rgb[c] = fmaxf(acc[c], 0.0f);
    }
}

// ------------------------------------------------------------------ warp staging of per-Gaussian rows
// Per-Gaussian rows (SH coefficients, blend records) are contiguous in global memory, one row per
// Gaussian.  A warp that owns 32 consecutive Gaussians moves their rows through shared memory so
// that every global load and store instruction covers consecutive addresses; each lane then
// works on its own row, padded to an odd stride (conflict-free across lanes).
constexpr int kRowStride = 49;   // >= 48 SH floats (degree 3) and >= 24 record floats; odd

// floor(e / w) as (e * row_inv(w)) >> 20, exact for e < 2^20 / w (here e < 32 * 48)
__host__ __device__ __forceinline__ uint32_t row_inv(int w) { return ((1u << 20) + (uint32_t)w - 1u) / (uint32_t)w; }

template <typename T>
__device__ __forceinline__ void warp_load_rows(const T *src, int rows, int w, float *buf, int lane) {
    const uint32_t inv = row_inv(w), total = (uint32_t)(rows * w);
#pragma unroll 4
    for (uint32_t e = lane; e < total; e += 32) {
        const uint32_t r = (e * inv) >> 20, c = e - r * (uint32_t)w;
        buf[r * kRowStride + c] = ld_f<T>(src, e);
    }
}

// FP32 rows: asynchronous 4-byte global-to-shared copies (cp.async), so that all of the warp's
// loads are in flight at once without passing through registers.  The caller waits with
// rows_wait() before __syncwarp().
template <>
__device__ __forceinline__ void warp_load_rows<float>(const float *src, int rows, int w, float *buf, int lane) {
    const uint32_t inv = row_inv(w), total = (uint32_t)(rows * w);
    for (uint32_t e = lane; e < total; e += 32) {
        const uint32_t r = (e * inv) >> 20, c = e - r * (uint32_t)w;
        const unsigned sa = (unsigned)__cvta_generic_to_shared(buf + r * kRowStride + c);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src + e) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// completes this thread's outstanding row copies
__device__ __forceinline__ void rows_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void warp_store_rows(float *dst, int rows, int w, const float *buf, int lane,
                                                int stride = kRowStride) {
    const uint32_t inv = row_inv(w), total = (uint32_t)(rows * w);
    for (uint32_t e = lane; e < total; e += 32) {
        const uint32_t r = (e * inv) >> 20, c = e - r * (uint32_t)w;
        dst[e] = buf[r * (uint32_t)stride + c];
    }
}

// FP32 rows of degree-3 SH (48 floats = 12 x 16 bytes per Gaussian) in 16-byte pieces: a warp's
// 32 rows are one contiguous 6,144-byte block, copied piece by piece with consecutive lanes on
// consecutive pieces (coalesced), into rows of kRow16 float4 -- an odd count, so that 8 lanes
// reading their own rows' piece j with 128-bit loads hit 8 different bank groups.
constexpr int kRow16 = 13;
constexpr int kSh3Pieces = 12;   // 16-byte pieces of one degree-3 FP32 SH row

// piece c of the block: row c / 12, piece c % 12 (c < 384: (c * 2731) >> 15 == c / 12)
__device__ __forceinline__ void sh3_piece(uint32_t c, uint32_t &r, uint32_t &j) {
    r = (c * 2731u) >> 15;
    j = c - r * (uint32_t)kSh3Pieces;
}

// Whether the SH rows of g take the 16-byte path: FP32, degree 3, a 16-byte aligned array.
template <typename ST>
inline bool sh3_rows(const GaussIn &g) {
    return std::is_same<ST, float>::value && g.sh != nullptr && g.sh_degree == 3 &&
           ((uintptr_t)g.sh & 15u) == 0;
}

// Asynchronous copies of `rows` rows (src 16-byte aligned); wait with rows_wait() before __syncwarp().
__device__ __forceinline__ void warp_load_sh3(const float *src, int rows, float4 *buf, int lane) {
    const uint32_t total = (uint32_t)rows * kSh3Pieces;
    for (uint32_t c = lane; c < total; c += 32) {
        uint32_t r, j;
        sh3_piece(c, r, j);
        const unsigned sa = (unsigned)__cvta_generic_to_shared(buf + r * kRow16 + j);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src + 4 * c) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void warp_store_sh3(float *dst, int rows, const float4 *buf, int lane) {
    const uint32_t total = (uint32_t)rows * kSh3Pieces;
    for (uint32_t c = lane; c < total; c += 32) {
        uint32_t r, j;
        sh3_piece(c, r, j);
        reinterpret_cast<float4 *>(dst)[c] = buf[r * kRow16 + j];
    }
}

// the colour of eval_colour_row from a degree-3 row staged by warp_load_sh3, in the same
// operation order (coefficient k, channel c), read 4 coefficients (three float4) at a time
__device__ __forceinline__ void eval_colour_sh3(const float4 *row, const float dir[3], float rgb[3], float raw[3],
                                                float beta = 0.0f) {
    float Y[16];
    sh_basis(3, dir[0], dir[1], dir[2], Y);
    float acc[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 a = row[3 * q], b = row[3 * q + 1], c = row[3 * q + 2];
        const float v[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) acc[ch] = fmaf(v[3 * kk + ch], Y[4 * q + kk], acc[ch]);
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        raw[ch] = acc[ch];
        rgb[ch] = colour_act(acc[ch], beta);
    }
}

// view-dependent colour from a staged SH row (same operation order as eval_colour)
__device__ __forceinline__ void eval_colour_row(int deg, const float *row, const float dir[3], float rgb[3],
                                                float raw[3], float beta = 0.0f) {
    float Y[16];
    sh_basis(deg, dir[0], dir[1], dir[2], Y);
    const int K = (deg + 1) * (deg + 1);
    float acc[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (k >= K) break;
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] = fmaf(row[3 * k + c], Y[k], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        raw[c] = acc[c];
        rgb[c] = colour_act(acc[c], beta);
    }
}

__device__ __forceinline__ void view_dir(const ViewInfo &V, const float mu[3], float dir[3], float &len) {
    float d0 = mu[0] - V.of[0], d1 = mu[1] - V.of[1], d2 = mu[2] - V.of[2];
    float n2 = d0 * d0 + d1 * d1 + d2 * d2;
    len = sqrtf(n2);
    float inv = 1.0f / len;
    dir[0] = d0 * inv;
    dir[1] = d1 * inv;
    dir[2] = d2 * inv;
}

}  // namespace vg
