// Tomography mode (Sec. 6.2, Eq. 21): parallel-beam projection proj = exp(-sum_g tau_g) of the
// same closed-form line integrals (Eq. 19), and its backward.
//
// For a parallel beam the ray direction d is fixed per angle, so per (angle, Gaussian) the
// line integral over the detector is an exact 2D Gaussian.  With W = S^-1 Rq^T the whitening,
// d' = W d and w_u = W e_u, w_v = W e_v, the whitened offset of the ray through detector pixel
// (i, j) from the centre is y = ((i - i_mu) pu (w_u x d') + (j - j_mu) pv (w_v x d')) / |d'|,
// a vector in the plane orthogonal to d'.  Expressed in an orthonormal basis (e1, e2) of that
// plane the record holds y = c0 dx + c1 dy (2D) and
//     tau = kappa sqrt(2 pi) / |d'| * exp(-|y|^2 / 2),
// i.e. ~10 FP32 operations and one ex2 per (pixel, Gaussian) pair.
#include "blend.cuh"
#include "geometry.cuh"

namespace vg {

constexpr int kTomoGradN = 8;   // per-item accumulator: dc0 (2), dc1 (2), sum dL/dy (2), dlnA, pad

// Orthonormal basis of the plane orthogonal to the unit vector n (Duff, Burgess, Christensen,
// Hill, Liani, Trotter, Raimondo: "Building an Orthonormal Basis, Revisited", JCGT 2017).
__device__ __forceinline__ void onb(const float n[3], float b1[3], float b2[3]) {
    const float sign = copysignf(1.0f, n[2]);
    const float a = -1.0f / (sign + n[2]);
    const float b = n[0] * n[1] * a;
    b1[0] = 1.0f + sign * n[0] * n[0] * a;
    b1[1] = sign * b;
    b1[2] = -sign * n[0];
    b2[0] = b;
    b2[1] = sign + n[1] * n[1] * a;
    b2[2] = -n[1];
}

// Per-item tomography geometry (shared by the preprocess and the chain kernels).
struct TomoGeom {
    float W[9];          // row-major whitening S^-1 Rq^T
    float dp[3], wu[3], wv[3];
    float C0[3], C1[3];  // pu (w_u x d'), pv (w_v x d')
    float n;             // |d'|
    float e1[3], e2[3];
    float c0[2], c1[2];  // (C . e) / n
    float imu, jmu;
};

__device__ __forceinline__ void tomo_geom(const float mu[3], const float s[3], const float Rq[9], float ct, float st,
                                          float pu, float pv, float u0, float v0, TomoGeom &G) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float is = 1.0f / s[i];
#pragma unroll
        for (int j = 0; j < 3; ++j) G.W[3 * i + j] = Rq[3 * j + i] * is;
        G.dp[i] = G.W[3 * i] * ct + G.W[3 * i + 1] * st;
        G.wu[i] = -G.W[3 * i] * st + G.W[3 * i + 1] * ct;
        G.wv[i] = G.W[3 * i + 2];
    }
    cross3(G.wu, G.dp, G.C0);
    cross3(G.wv, G.dp, G.C1);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        G.C0[i] *= pu;
        G.C1[i] *= pv;
    }
    G.n = sqrtf(G.dp[0] * G.dp[0] + G.dp[1] * G.dp[1] + G.dp[2] * G.dp[2]);
    const float in = 1.0f / G.n;
    const float nn[3] = {G.dp[0] * in, G.dp[1] * in, G.dp[2] * in};
    onb(nn, G.e1, G.e2);
    G.c0[0] = (G.C0[0] * G.e1[0] + G.C0[1] * G.e1[1] + G.C0[2] * G.e1[2]) * in;
    G.c0[1] = (G.C0[0] * G.e2[0] + G.C0[1] * G.e2[1] + G.C0[2] * G.e2[2]) * in;
    G.c1[0] = (G.C1[0] * G.e1[0] + G.C1[1] * G.e1[1] + G.C1[2] * G.e1[2]) * in;
    G.c1[1] = (G.C1[0] * G.e2[0] + G.C1[1] * G.e2[1] + G.C1[2] * G.e2[2]) * in;
    const float um = -st * mu[0] + ct * mu[1];
    G.imu = (um - u0) / pu - 0.5f;
    G.jmu = (mu[2] - v0) / pv - 0.5f;
}

// ---------------------------------------------------------------------------- preprocess
template <typename RT>
__global__ void __launch_bounds__(256)
k_tomo_preprocess(GaussIn g, const float *__restrict__ cs, int n_angles, int det_w, int det_h, float pu, float pv,
                  float u0, float v0, float tau_cut, float4 *__restrict__ rec, uint32_t *__restrict__ count,
                  short4 *__restrict__ rect, short4 *__restrict__ prect) {
    pdl_entry();
    const long long n_items = (long long)g.n * n_angles;
    const int tiles_x = (det_w + kTile - 1) / kTile;
    (void)tiles_x;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < n_items;
         it += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(it / g.n);
        const long long gi = it - (long long)a * g.n;
        const float ct = cs[2 * a], st = cs[2 * a + 1];
        float mu[3], s[3], q[4], kin, Sig[9], Rq[9], qn[4], smax, k2;
        load_gauss<RT>(g, gi, mu, s, q, kin);
        const Density dn = density_of(g, kin, s);
        const float kap = dn.kap;
        short4 rc = make_short4(-1, -1, -1, -1), prc = rc;
        uint32_t cnt = 0;
        if (key_cov(mu, s, q, dn.kap_key, Sig, Rq, qn, smax) && key_k2(dn.kap_key, smax, tau_cut, k2)) {
            // key function: orthographic bounding box of the Mahalanobis-k ellipsoid (FP32, fixed order)
            const float um = VG_ADD(VG_MUL(-st, mu[0]), VG_MUL(ct, mu[1]));
            const float vm = mu[2];
            float suu = VG_ADD(VG_SUB(VG_MUL(VG_MUL(st, st), Sig[0]), VG_MUL(2.0f, VG_MUL(VG_MUL(st, ct), Sig[1]))),
                               VG_MUL(VG_MUL(ct, ct), Sig[4]));
            if (!(suu > 0.0f)) suu = 0.0f;
            const float svv = Sig[8];
            const float hu = VG_SQRT(VG_MUL(k2, suu)), hv = VG_SQRT(VG_MUL(k2, svv));
            const float xlo = VG_SUB(VG_DIV(VG_SUB(VG_SUB(um, hu), u0), pu), 0.5f);
            const float xhi = VG_SUB(VG_DIV(VG_SUB(VG_ADD(um, hu), u0), pu), 0.5f);
            const float ylo = VG_SUB(VG_DIV(VG_SUB(VG_SUB(vm, hv), v0), pv), 0.5f);
            const float yhi = VG_SUB(VG_DIV(VG_SUB(VG_ADD(vm, hv), v0), pv), 0.5f);
            int ix0, ix1, iy0, iy1;
            pixel_span(xlo, xhi, det_w, ix0, ix1);
            pixel_span(ylo, yhi, det_h, iy0, iy1);
            if (ix0 <= ix1 && iy0 <= iy1) {
                rc = make_short4((short)(ix0 / kTile), (short)(iy0 / kTile), (short)(ix1 / kTile), (short)(iy1 / kTile));
                prc = make_short4((short)ix0, (short)iy0, (short)ix1, (short)iy1);
                cnt = (uint32_t)(rc.z - rc.x + 1) * (uint32_t)(rc.w - rc.y + 1);
                TomoGeom G;
                tomo_geom(mu, s, Rq, ct, st, pu, pv, u0, v0, G);
                const float lnA2 = log2f(kap) + kLog2Sqrt2Pi - log2f(G.n);
                rec[2 * it] = make_float4(G.imu, G.jmu, G.c0[0], G.c0[1]);
                rec[2 * it + 1] = make_float4(G.c1[0], G.c1[1], lnA2, 0.0f);
            }
        }
        count[it] = cnt;
        rect[it] = rc;
        prect[it] = prc;
    }
}

cudaError_t launch_tomo_preprocess(const GaussIn &g, const float *cs_d, int n_angles, int det_w, int det_h,
                                   float pitch_u, float pitch_v, float u0, float v0, float tau_cut, float4 *rec,
                                   uint32_t *count, short4 *rect, short4 *prect, cudaStream_t st,
                                   long long *launches) {
    const long long n_items = (long long)g.n * n_angles;
    long long b = (n_items + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    *launches += 1;
    if (g.rec_dtype == VG_BF16)
        pdl_launch(k_tomo_preprocess<__nv_bfloat16>, (unsigned)b, 256, 0, st, g, cs_d, n_angles, det_w, det_h, pitch_u, pitch_v,
                                                                      u0, v0, tau_cut, rec, count, rect, prect);
    else if (g.rec_dtype == VG_F16)
        pdl_launch(k_tomo_preprocess<__half>, (unsigned)b, 256, 0, st, g, cs_d, n_angles, det_w, det_h, pitch_u, pitch_v, u0,
                                                               v0, tau_cut, rec, count, rect, prect);
    else
        pdl_launch(k_tomo_preprocess<float>, (unsigned)b, 256, 0, st, g, cs_d, n_angles, det_w, det_h, pitch_u, pitch_v, u0,
                                                              v0, tau_cut, rec, count, rect, prect);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- projector
// One CTA of 64 threads per detector tile, a 2x2 pixel quad per thread; y advances by c0 or c1
// from one quad pixel to the next.
constexpr int kQuadThreads = kTilePix / 4;   // 64 threads, a 2x2 quad each
constexpr int kTomoChunk = kQuadThreads;

__global__ void __launch_bounds__(kQuadThreads, 12)
k_tomo_fwd(const uint2 *__restrict__ ranges, int tiles_x, int tiles_per_view, int det_w, int det_h,
           const uint32_t *__restrict__ sorted_item, const float4 *__restrict__ rec, const short4 *__restrict__ prect,
           float *__restrict__ proj) {
    pdl_entry();
    __shared__ float4 srec[kTomoChunk * 2];
    __shared__ short4 srect[kTomoChunk];
    const int tile = blockIdx.x;
    const int view = tile / tiles_per_view, local = tile - view * tiles_per_view;
    const int ty = local / tiles_x, tx = local - ty * tiles_x;
    const int x0 = tx * kTile + 2 * (threadIdx.x & 7), y0 = ty * kTile + 2 * (threadIdx.x >> 3);
    const float xf = (float)x0, yf = (float)y0;
    const WarpBox wb = warp_box<4>(x0, y0);
    const int lane = threadIdx.x & 31;
    const uint2 rg = ranges[tile];
    float sum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (uint32_t base = rg.x; base < rg.y; base += kTomoChunk) {
        const uint32_t n = min((uint32_t)kTomoChunk, rg.y - base);
        __syncthreads();
        if (threadIdx.x < n) {
            const uint32_t item = sorted_item[base + threadIdx.x];
            const float4 *src = rec + 2 * (size_t)item;
            srec[2 * threadIdx.x] = __ldg(src);
            srec[2 * threadIdx.x + 1] = __ldg(src + 1);
            srect[threadIdx.x] = prect[item];
        }
        __syncthreads();
        // the warp ballots the records whose footprint touches its pixels and whether it lies
        // inside the footprint; it visits only those records
        for (int w0 = 0; w0 < (int)n; w0 += 32) {
            const int jl = w0 + lane;
            bool need = false, full = false;
            if (jl < (int)n) {
                const short4 pr = srect[jl];
                need = !box_misses(wb, pr);
                full = box_inside(wb, pr);
            }
            unsigned m = __ballot_sync(0xffffffffu, need);
            const unsigned mf = __ballot_sync(0xffffffffu, full);
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int j = w0 + b;
                const float4 r0 = srec[2 * j], r1 = srec[2 * j + 1];
                const float dx = xf - r0.x, dy = yf - r0.y;
                const float ya0 = fmaf(r0.z, dx, r1.x * dy), ya1 = fmaf(r0.w, dx, r1.y * dy);   // pixel (0,0)
                const float yb0 = ya0 + r0.z, yb1 = ya1 + r0.w;                                   // (1,0)
                const float yc0 = ya0 + r1.x, yc1 = ya1 + r1.y;                                   // (0,1)
                const float yd0 = yb0 + r1.x, yd1 = yb1 + r1.y;                                   // (1,1)
                const float ta = ex2_approx(fmaf(fmaf(ya0, ya0, ya1 * ya1), -kHalfLog2e, r1.z));
                const float tb = ex2_approx(fmaf(fmaf(yb0, yb0, yb1 * yb1), -kHalfLog2e, r1.z));
                const float tc = ex2_approx(fmaf(fmaf(yc0, yc0, yc1 * yc1), -kHalfLog2e, r1.z));
                const float td = ex2_approx(fmaf(fmaf(yd0, yd0, yd1 * yd1), -kHalfLog2e, r1.z));
                if ((mf >> b) & 1u) {                // every pixel of the warp is inside
                    sum[0] += ta;
                    sum[1] += tb;
                    sum[2] += tc;
                    sum[3] += td;
                } else {                             // footprint rectangle, separable in x and y
                    const short4 pr = srect[j];
                    const bool xa = x0 >= pr.x && x0 <= pr.z, xb = x0 + 1 >= pr.x && x0 + 1 <= pr.z;
                    const bool ya = y0 >= pr.y && y0 <= pr.w, yb = y0 + 1 >= pr.y && y0 + 1 <= pr.w;
                    sum[0] += (xa && ya) ? ta : 0.0f;
                    sum[1] += (xb && ya) ? tb : 0.0f;
                    sum[2] += (xa && yb) ? tc : 0.0f;
                    sum[3] += (xb && yb) ? td : 0.0f;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = x0 + (k & 1), y = y0 + (k >> 1);
        if (x < det_w && y < det_h) proj[((long long)view * det_h + y) * det_w + x] = ex2_approx(-kLog2eF * sum[k]);
    }
}

cudaError_t launch_tomo_fwd(const uint2 *ranges, long long n_tiles, int tiles_x, int tiles_per_view, int det_w,
                            int det_h, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                            float *proj, cudaStream_t st, long long *launches) {
    if (n_tiles <= 0) return cudaSuccess;
    pdl_launch(k_tomo_fwd, (unsigned)n_tiles, kQuadThreads, 0, st, ranges, tiles_x, tiles_per_view, det_w, det_h,
                                                           sorted_item, rec, prect, proj);
    *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- backward
// proj = exp(-sum tau)  =>  dL/dtau = -proj dL/dproj for every Gaussian on the ray;
// ln tau = lnA - |y|^2/2  =>  dL/dy = -dL/dln(tau) y.  Seven partials per (pixel, Gaussian)
// are summed over the quad and added to the per-item accumulator (8 floats, 32-byte aligned)
// with vector reductions in L2: directly by each contributing lane (two v4 reductions) when
// at most kTomoDirectLanes lanes of the warp contribute, otherwise after two shuffle exchange
// steps that leave every lane 2 values summed over 4 lanes (one v2 reduction per lane).  With
// 100,000 Gaussians, 256 parallel-beam angles and 512^2 detectors this backward takes 118 ms
// per step against 140 ms with a full reduce-scatter and 7 scalar reductions per (warp,
// Gaussian).
__global__ void __launch_bounds__(kQuadThreads, 12)
k_tomo_bwd(const uint2 *__restrict__ ranges, int tiles_x, int tiles_per_view, int det_w, int det_h,
           const uint32_t *__restrict__ sorted_item, const float4 *__restrict__ rec, const short4 *__restrict__ prect,
           const float *__restrict__ proj, const float *__restrict__ dL_dproj, float *__restrict__ grad_acc) {
    pdl_entry();
    constexpr int NP = 8;   // 7 partials, padded to a power of two (the accumulator's 8 floats)
    constexpr int kTomoDirectLanes = 16;
    __shared__ float4 srec[kTomoChunk * 2];
    __shared__ short4 srect[kTomoChunk];
    __shared__ uint32_t sitem[kTomoChunk];
    const int tile = blockIdx.x;
    const int view = tile / tiles_per_view, local = tile - view * tiles_per_view;
    const int ty = local / tiles_x, tx = local - ty * tiles_x;
    const int x0 = tx * kTile + 2 * (threadIdx.x & 7), y0 = ty * kTile + 2 * (threadIdx.x >> 3);
    const float xf = (float)x0, yf = (float)y0;
    const int lane = threadIdx.x & 31;
    float gtau[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = x0 + (k & 1), y = y0 + (k >> 1);
        gtau[k] = 0.0f;
        if (x < det_w && y < det_h) {
            const long long pix = ((long long)view * det_h + y) * det_w + x;
            gtau[k] = -proj[pix] * dL_dproj[pix];
        }
    }
    const WarpBox wb = warp_box<4>(x0, y0);
    const uint2 rg = ranges[tile];
    for (uint32_t base = rg.x; base < rg.y; base += kTomoChunk) {
        const uint32_t n = min((uint32_t)kTomoChunk, rg.y - base);
        if (threadIdx.x < n) {
            const uint32_t item = sorted_item[base + threadIdx.x];
            sitem[threadIdx.x] = item;
            srec[2 * threadIdx.x] = __ldg(rec + 2 * (size_t)item);
            srec[2 * threadIdx.x + 1] = __ldg(rec + 2 * (size_t)item + 1);
            srect[threadIdx.x] = prect[item];
        }
        __syncthreads();
        for (int w0 = 0; w0 < (int)n; w0 += 32) {
            const int jl = w0 + lane;
            const bool need = jl < (int)n && !box_misses(wb, srect[jl]);
            unsigned m = __ballot_sync(0xffffffffu, need);
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int j = w0 + b;
                const short4 pr = srect[j];
                const float4 r0 = srec[2 * j], r1 = srec[2 * j + 1];
                float v[NP];
#pragma unroll
                for (int k = 0; k < NP; ++k) v[k] = 0.0f;
                const float dx0 = xf - r0.x, dy0 = yf - r0.y;
                const float ya0 = fmaf(r0.z, dx0, r1.x * dy0), ya1 = fmaf(r0.w, dx0, r1.y * dy0);
                const float yb0 = ya0 + r0.z, yb1 = ya1 + r0.w;
                const float q0[4] = {ya0, yb0, ya0 + r1.x, yb0 + r1.x}, q1[4] = {ya1, yb1, ya1 + r1.y, yb1 + r1.y};
                // footprint rectangle, separable in x and y; all-true when the warp lies inside it
                const bool full = box_inside(wb, pr);
                const bool xa = full || (x0 >= pr.x && x0 <= pr.z), xb = full || (x0 + 1 >= pr.x && x0 + 1 <= pr.z);
                const bool ya = full || (y0 >= pr.y && y0 <= pr.w), yb = full || (y0 + 1 >= pr.y && y0 + 1 <= pr.w);
                // the quad's pixels sit at (dx0 + (k & 1), dy0 + (k >> 1)): the dx- and dy-weighted
                // sums follow from the plain sums and those of the odd columns and rows
                float ox0 = 0.0f, ox1 = 0.0f, oy0 = 0.0f, oy1 = 0.0f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float y0v = q0[k], y1v = q1[k];
                    const float m2 = fmaf(y0v, y0v, y1v * y1v);
                    const float tau = ex2_approx(fmaf(m2, -kHalfLog2e, r1.z));
                    const bool in = ((k & 1) ? xb : xa) && ((k & 2) ? yb : ya);
                    const float G = in ? gtau[k] * tau : 0.0f;      // dL / d ln(tau)
                    const float gy0 = -G * y0v, gy1 = -G * y1v;
                    if (k & 1) {
                        ox0 += gy0;
                        ox1 += gy1;
                    }
                    if (k & 2) {
                        oy0 += gy0;
                        oy1 += gy1;
                    }
                    v[4] += gy0;
                    v[5] += gy1;
                    v[6] += G;
                }
                v[0] = fmaf(v[4], dx0, ox0);
                v[1] = fmaf(v[5], dx0, ox1);
                v[2] = fmaf(v[4], dy0, oy0);
                v[3] = fmaf(v[5], dy0, oy1);
                const bool any = (xa || xb) && (ya || yb);   // some pixel of the quad contributes
                const unsigned act = __ballot_sync(0xffffffffu, any);
                float *dst = grad_acc + (size_t)sitem[j] * kTomoGradN;
                if (__popc(act) <= kTomoDirectLanes) {
                    if (any) {
                        red_add_v4(dst, v[0], v[1], v[2], v[3]);
                        red_add_v4(dst + 4, v[4], v[5], v[6], 0.0f);
                    }
                } else {
                    const int b0 = warp_reduce_scatter_part<NP, 2>(v, lane);
                    red_add_v2(dst + b0, v[0], v[1]);
                }
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_tomo_bwd(const uint2 *ranges, long long n_tiles, int tiles_x, int tiles_per_view, int det_w,
                            int det_h, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                            const float *proj, const float *dL_dproj, float *grad_acc, cudaStream_t st,
                            long long *launches) {
    if (n_tiles <= 0) return cudaSuccess;
    pdl_launch(k_tomo_bwd, (unsigned)n_tiles, kQuadThreads, 0, st, ranges, tiles_x, tiles_per_view, det_w, det_h,
                                                           sorted_item, rec, prect, proj, dL_dproj, grad_acc);
    *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- chain
template <typename RT>
__global__ void __launch_bounds__(128)
k_tomo_chain(GaussIn g, const float *__restrict__ cs, int n_angles, long long item0, long long n_items, float pu,
             float pv, float u0, float v0, const float *__restrict__ grad_acc, float *__restrict__ dmu,
             float *__restrict__ dscale, float *__restrict__ dquat, float *__restrict__ dkappa) {
    pdl_entry();
    (void)n_angles;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_items;
         k += (long long)gridDim.x * blockDim.x) {
        const float4 a4 = *(const float4 *)(grad_acc + k * kTomoGradN);
        const float4 b4 = *(const float4 *)(grad_acc + k * kTomoGradN + 4);
        if (a4.x == 0.0f && a4.y == 0.0f && a4.z == 0.0f && a4.w == 0.0f && b4.x == 0.0f && b4.y == 0.0f &&
            b4.z == 0.0f)
            continue;
        const long long it = item0 + k;
        const int a = (int)(it / g.n);
        const long long gi = it - (long long)a * g.n;
        const float ct = cs[2 * a], st = cs[2 * a + 1];
        float mu[3], s[3], q[4], kin, Sig[9], Rq[9], qn[4], smax;
        load_gauss<RT>(g, gi, mu, s, q, kin);
        const Density dns = density_of(g, kin, s);
        const float kap = dns.kap;
        if (!key_cov(mu, s, q, dns.kap_key, Sig, Rq, qn, smax)) continue;
        TomoGeom G;
        tomo_geom(mu, s, Rq, ct, st, pu, pv, u0, v0, G);
        const float dc0[2] = {a4.x, a4.y}, dc1[2] = {a4.z, a4.w}, dys[2] = {b4.x, b4.y};
        const float dlnA = b4.z;
        // c_k = (C_k . e) / n (2D, in the plane orthogonal to d'); lnA = ln(kappa sqrt(2pi)) - ln n
        const float in = 1.0f / G.n;
        float gC0[3], gC1[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gC0[i] = (dc0[0] * G.e1[i] + dc0[1] * G.e2[i]) * in;
            gC1[i] = (dc1[0] * G.e1[i] + dc1[1] * G.e2[i]) * in;
        }
        const float dn = -(gC0[0] * G.C0[0] + gC0[1] * G.C0[1] + gC0[2] * G.C0[2] + gC1[0] * G.C1[0] +
                           gC1[1] * G.C1[1] + gC1[2] * G.C1[2]) * in - dlnA * in;
        float gdp[3], gwu[3], gwv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) gdp[i] = dn * G.dp[i] * in;
        // C0 = pu (w_u x d'), C1 = pv (w_v x d')
        float t[3];
        cross3(gC0, G.wu, t);
#pragma unroll
        for (int i = 0; i < 3; ++i) gdp[i] += pu * t[i];
        cross3(gC1, G.wv, t);
#pragma unroll
        for (int i = 0; i < 3; ++i) gdp[i] += pv * t[i];
        cross3(G.dp, gC0, gwu);
        cross3(G.dp, gC1, gwv);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gwu[i] *= pu;
            gwv[i] *= pv;
        }
        // d' = W d, w_u = W e_u, w_v = W e_v with d = (ct, st, 0), e_u = (-st, ct, 0), e_v = (0, 0, 1)
        float dW[9];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dW[3 * i + 0] = gdp[i] * ct - gwu[i] * st;
            dW[3 * i + 1] = gdp[i] * st + gwu[i] * ct;
            dW[3 * i + 2] = gwv[i];
        }
        // W[i][j] = Rq[j][i] / s_i
        float dsc[3], dR[9];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float is = 1.0f / s[i];
            dsc[i] = -(dW[3 * i] * G.W[3 * i] + dW[3 * i + 1] * G.W[3 * i + 1] + dW[3 * i + 2] * G.W[3 * i + 2]) * is;
#pragma unroll
            for (int j = 0; j < 3; ++j) dR[3 * j + i] = dW[3 * i + j] * is;
        }
        const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
        float dqn[4];
        dqn[0] = 2.0f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
        dqn[1] = 2.0f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.0f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                         2.0f * x * dR[8]);
        dqn[2] = 2.0f * (-2.0f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                         2.0f * y * dR[8]);
        dqn[3] = 2.0f * (-2.0f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.0f * z * dR[4] + y * dR[5] +
                         x * dR[6] + y * dR[7]);
        const float qnorm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const float dot = qn[0] * dqn[0] + qn[1] * dqn[1] + qn[2] * dqn[2] + qn[3] * dqn[3];
        // i_mu = (e_u . mu - u0)/pu - 1/2, j_mu = (mu_z - v0)/pv - 1/2; dL/di_mu = -c0 . sum dL/dy
        const float gi_mu = -(G.c0[0] * dys[0] + G.c0[1] * dys[1]);
        const float gj_mu = -(G.c1[0] * dys[0] + G.c1[1] * dys[1]);
        const float dm[3] = {-st * gi_mu / pu, ct * gi_mu / pu, gj_mu / pv};
        float dk = dlnA / kap;   // dL/dkappa; with Eq. 20 it becomes dL/dtheta plus a share of dL/ds
        if (g.density_theta) {
#pragma unroll
            for (int c = 0; c < 3; ++c) dsc[c] -= dk * dns.lnv / (3.0f * s[c] * s[c]);
            dk = dk * 0.99f / (1.0f - 0.99f * kin) * dns.m;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicAdd(&dmu[3 * gi + c], dm[c]);
            atomicAdd(&dscale[3 * gi + c], dsc[c]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) atomicAdd(&dquat[4 * gi + c], (dqn[c] - qn[c] * dot) / qnorm);
        atomicAdd(&dkappa[gi], dk);
    }
}

cudaError_t launch_tomo_chain(const GaussIn &g, const float *cs_d, int n_angles, long long item0, long long n_items,
                              float pitch_u, float pitch_v, float u0, float v0, const float *grad_acc, float *dmu,
                              float *dscale, float *dquat, float *dkappa, cudaStream_t st, long long *launches) {
    long long b = (n_items + 127) / 128;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    *launches += 1;
    if (g.rec_dtype == VG_BF16)
        pdl_launch(k_tomo_chain<__nv_bfloat16>, (unsigned)b, 128, 0, st, g, cs_d, n_angles, item0, n_items, pitch_u, pitch_v, u0,
                                                                 v0, grad_acc, dmu, dscale, dquat, dkappa);
    else if (g.rec_dtype == VG_F16)
        pdl_launch(k_tomo_chain<__half>, (unsigned)b, 128, 0, st, g, cs_d, n_angles, item0, n_items, pitch_u, pitch_v, u0, v0,
                                                          grad_acc, dmu, dscale, dquat, dkappa);
    else
        pdl_launch(k_tomo_chain<float>, (unsigned)b, 128, 0, st, g, cs_d, n_angles, item0, n_items, pitch_u, pitch_v, u0, v0,
                                                         grad_acc, dmu, dscale, dquat, dkappa);
    return cudaGetLastError();
}

}  // namespace vg
