// Ray-marching reference of the volume rendering equation (Eq. 1) with the fields of Supp. A,
// sigma(x) = sum kappa_i G_i(x) and c(x) = sum c_i kappa_i G_i(x) / sigma(x), for measuring the
// blend's no-overlap approximation (Sec. 4.1) on the GPU: per pixel, NeRF's quadrature on
// midpoint samples t_k = t_near + (k + 1/2) delta of the unit ray from the camera centre,
//   C = sum_k T_k (1 - exp(-sigma_k delta)) c(x_k) + T bg,  T_k = exp(-delta sum_{j<k} sigma_j).
//
// Along a pixel's ray each Gaussian is a 1D Gaussian in t (Supp. B): with the record's
// d' = A u and o' x d' = C u (u = (dx, dy, 1)) and E = (o'.A0, o'.A1, o'.A2),
//   kappa G(o + t d) = kappa exp(-m^2/2) exp(-(t - gamma)^2 / (2 beta^2)),
//   m^2 = |C u|^2 / |A u|^2,  gamma = -(E . u) |d_c| / |A u|^2,  beta^2 = |d_c|^2 / |A u|^2,
// so a sample costs one FMA chain and one ex2 per (pixel, Gaussian).  The Gaussians near a pixel
// are those of its tile list whose footprint rectangle holds the pixel (every other one adds less
// than tau_cut to the ray's optical depth); the march needs no order.  One CTA per tile, one
// pixel per thread; samples are processed 16 at a time in registers, each pass walking the
// tile's list (records staged in shared memory) and skipping Gaussians whose 1D Gaussian is
// below 2^-50 on the pass's samples.
#include "blend.cuh"
#include "geometry.cuh"

namespace vg {

constexpr int kMarchS = 16;        // samples per pass
constexpr int kMarchChunk = 128;   // records per shared-memory chunk

// E = (o'.A0, o'.A1, o'.A2) of every visible item.
template <typename RT>
__global__ void __launch_bounds__(256)
k_march_prep(GaussIn g, const ViewInfo *__restrict__ views, long long n_items, const uint32_t *__restrict__ count,
             float4 *__restrict__ E) {
    pdl_entry();
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < n_items;
         it += (long long)gridDim.x * blockDim.x) {
        float4 e = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (count[it] != 0) {
            const int v = (int)(it / g.n);
            const long long gi = it - (long long)v * g.n;
            float mu[3], s[3], q[4], kin, Sig[9], Rq[9], qn[4], smax;
            load_gauss<RT>(g, gi, mu, s, q, kin);
            const Density dn = density_of(g, kin, s);
            if (key_cov(mu, s, q, dn.kap_key, Sig, Rq, qn, smax)) {
                ItemGeom G;
                item_geom(views[v], mu, s, Rq, G);
                e.x = G.op[0] * G.A[0] + G.op[1] * G.A[1] + G.op[2] * G.A[2];
                e.y = G.op[0] * G.A[3] + G.op[1] * G.A[4] + G.op[2] * G.A[5];
                e.z = G.op[0] * G.A[6] + G.op[1] * G.A[7] + G.op[2] * G.A[8];
            }
        }
        E[it] = e;
    }
}

__global__ void __launch_bounds__(kMaxTilePix)
k_ray_march(const ViewInfo *__restrict__ views, const int *__restrict__ tile_view, const uint2 *__restrict__ ranges,
            const uint32_t *__restrict__ sorted_item, const float4 *__restrict__ rec, const float4 *__restrict__ E,
            const short4 *__restrict__ prect, float t_near, float delta, int n_samples, float T_stop, float bg0,
            float bg1, float bg2, const float *__restrict__ raster, float *__restrict__ rgb, float *__restrict__ T_out,
            float *__restrict__ err) {
    pdl_entry();
    __shared__ float4 srec[kMarchChunk * (kRecF4 + 1)];
    __shared__ short4 srect[kMarchChunk];
    const int tile = blockIdx.x;
    const ViewInfo &V = views[tile_view[tile]];
    const int local = tile - V.tile_base;
    const int tyi = local / V.tiles_x, txi = local - tyi * V.tiles_x;
    const int x = txi * V.tw + (int)(threadIdx.x % V.tw), y = tyi * V.th + (int)(threadIdx.x / V.tw);
    const bool inside = x < V.W && y < V.H;
    const float xf = (float)x, yf = (float)y;
    const float pu = ((float)x + 0.5f - V.cx) / V.fx, pv = ((float)y + 0.5f - V.cy) / V.fy;
    const float dcn2 = fmaf(pu, pu, fmaf(pv, pv, 1.0f)), dcn = sqrtf(dcn2);
    const uint2 rg = ranges[tile];
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    bool live = inside;
    for (int k0 = 0; k0 < n_samples; k0 += kMarchS) {
        if (!__syncthreads_or(live)) break;
        float sg[kMarchS], a0[kMarchS], a1[kMarchS], a2[kMarchS];
#pragma unroll
        for (int s = 0; s < kMarchS; ++s) sg[s] = a0[s] = a1[s] = a2[s] = 0.0f;
        const float tk0 = fmaf((float)k0 + 0.5f, delta, t_near);
        for (uint32_t base = rg.x; base < rg.y; base += kMarchChunk) {
            const int n = (int)min((uint32_t)kMarchChunk, rg.y - base);
            __syncthreads();
            for (int r = threadIdx.x; r < n; r += blockDim.x) {
                const uint32_t item = sorted_item[base + r];
#pragma unroll
                for (int c = 0; c < kRecF4; ++c) srec[r * (kRecF4 + 1) + c] = __ldg(rec + (size_t)item * kRecF4 + c);
                srec[r * (kRecF4 + 1) + kRecF4] = __ldg(E + item);
                srect[r] = prect[item];
            }
            __syncthreads();
            if (!live) continue;
            for (int j = 0; j < n; ++j) {
                if (pixel_outside(x, y, srect[j])) continue;
                const float4 *rr = &srec[j * (kRecF4 + 1)];
                const float4 r0 = rr[0], r1 = rr[1], r2 = rr[2], r3 = rr[3], r4 = rr[4], r5 = rr[5], e4 = rr[6];
                const float dx = xf - r4.z, dy = yf - r4.w;
                const float d0 = fmaf(r0.x, dx, fmaf(r0.w, dy, r1.z));
                const float d1 = fmaf(r0.y, dx, fmaf(r1.x, dy, r1.w));
                const float d2 = fmaf(r0.z, dx, fmaf(r1.y, dy, r2.x));
                const float q0 = fmaf(r2.y, dx, fmaf(r3.x, dy, r3.w));
                const float q1 = fmaf(r2.z, dx, fmaf(r3.y, dy, r4.x));
                const float q2 = fmaf(r2.w, dx, fmaf(r3.z, dy, r4.y));
                const float a = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
                const float qq = fmaf(q0, q0, fmaf(q1, q1, q2 * q2));
                const float bq = fmaf(e4.x, dx, fmaf(e4.y, dy, e4.z));
                const float ia = 1.0f / a;
                const float lp = fmaf(-qq * ia, kHalfLog2e, r5.x - kLog2Sqrt2Pi);   // log2(kappa exp(-m^2/2))
                const float gam = -bq * dcn * ia;
                const float h = kHalfLog2e * a / dcn2;                                // log2(e) / (2 beta^2)
                const float room = lp + 50.0f;                                        // value >= 2^-50 only
                if (!(room > 0.0f)) continue;
                const float half = sqrtf(room / h);
                const float slo = (gam - half - tk0) / delta, shi = (gam + half - tk0) / delta;
                if (shi < 0.0f || slo > (float)(kMarchS - 1)) continue;
#pragma unroll
                for (int s = 0; s < kMarchS; ++s) {
                    const float dt = fmaf((float)s, delta, tk0) - gam;
                    const float v = ex2_approx(fmaf(-dt * dt, h, lp));
                    sg[s] += v;
                    a0[s] = fmaf(r5.y, v, a0[s]);
                    a1[s] = fmaf(r5.z, v, a1[s]);
                    a2[s] = fmaf(r5.w, v, a2[s]);
                }
            }
        }
        if (live) {
#pragma unroll
            for (int s = 0; s < kMarchS; ++s) {
                if (k0 + s >= n_samples || !live) continue;
                const float sig = sg[s];
                if (sig > 0.0f) {
                    const float xs = sig * delta;
                    const float w = T * (-expm1f(-xs) / sig);   // T (1 - e^{-sigma delta}) / sigma
                    C0 = fmaf(w, a0[s], C0);
                    C1 = fmaf(w, a1[s], C1);
                    C2 = fmaf(w, a2[s], C2);
                    T *= expf(-xs);
                }
                if (T < T_stop) live = false;
            }
        }
    }
    if (!inside) return;
    const long long pix = V.pix_base + (long long)y * V.W + x;
    const float c0 = fmaf(T, bg0, C0), c1 = fmaf(T, bg1, C1), c2 = fmaf(T, bg2, C2);
    if (rgb) {
        rgb[3 * pix] = c0;
        rgb[3 * pix + 1] = c1;
        rgb[3 * pix + 2] = c2;
    }
    if (T_out) T_out[pix] = T;
    if (err && raster)
        err[pix] = fmaxf(fabsf(c0 - raster[3 * pix]), fmaxf(fabsf(c1 - raster[3 * pix + 1]), fabsf(c2 - raster[3 * pix + 2])));
}

cudaError_t launch_ray_march(const GaussIn &g, const ViewInfo *views_d, const int *tile_view, long long n_tiles,
                             int tile_px,
                             long long n_items, const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec,
                             const uint32_t *count, const short4 *prect, float4 *E, float t_near, float t_far,
                             int n_samples, float T_stop, const float bg[3], const float *raster, float *rgb,
                             float *T_out, float *err, cudaStream_t st, long long *launches) {
    if (n_items > 0) {
        long long b = (n_items + 255) / 256;
        if (b > 152 * 32) b = 152 * 32;
        if (g.rec_dtype == VG_BF16)
            pdl_launch(k_march_prep<__nv_bfloat16>, (unsigned)b, 256, 0, st, g, views_d, n_items, count, E);
        else if (g.rec_dtype == VG_F16)
            pdl_launch(k_march_prep<__half>, (unsigned)b, 256, 0, st, g, views_d, n_items, count, E);
        else
            pdl_launch(k_march_prep<float>, (unsigned)b, 256, 0, st, g, views_d, n_items, count, E);
        *launches += 1;
    }
    if (n_tiles > 0) {
        const float delta = (t_far - t_near) / (float)n_samples;
        pdl_launch(k_ray_march, (unsigned)n_tiles, (unsigned)tile_px, 0, st, views_d, tile_view, ranges, sorted_item, rec, E, prect, t_near,
                                                          delta, n_samples, T_stop, bg[0], bg[1], bg[2], raster, rgb,
                                                          T_out, err);
        *launches += 1;
    }
    return cudaGetLastError();
}

}  // namespace vg
