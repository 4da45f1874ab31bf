/* FP64 CPU oracle for the volumetrically consistent Gaussian rasterizer (arXiv 2412.03378).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA library
 * is checked against.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg load it; the product path never does.  It shares no code with the CUDA library.
 *
 * What it computes, with the passage each part follows:
 *   - density mixture sigma(x) = sum_i kappa_i G_i(x), G_i unnormalised (Sec. 3.2, Eq. 3-4);
 *   - per-Gaussian transmittance along a ray over the whole line (Sec. 4.2, Eq. 15-19):
 *       a = d'P d, b = d'P(o-mu), c = (o-mu)'P(o-mu), P = Sigma^-1, d a unit direction,
 *       tau = kappa sqrt(2 pi / a) exp(-(c - b^2/a)/2),  alpha = 1 - exp(-tau);
 *   - front-to-back alpha blending of the depth-sorted per-tile list (Sec. 4.1, Eq. 14);
 *   - analytic gradient of the blend by the chain rule through a, b, c (derived from Eq. 19);
 *   - tomography: proj = exp(-sum_i tau_i) on a parallel beam (Sec. 6.2, Eq. 21);
 *   - the 3DGS comparison mode (Sec. 3.2, Eq. 5-7): alpha = o G'(p) with the splatted 2D
 *     Gaussian of covariance J W Sigma W^T J^T, blended with the same Eq. 14 / Eq. 5;
 *   - the per-tile binning that the paper inherits from 3DGS (Sec. 7, "per-tile sorting"),
 *     with a conservative footprint computed by an FP32 key function (readings in the
 *     design notes: the footprint is the screen bounding box of the Mahalanobis-k
 *     ellipsoid, k^2 = 2 ln 2 * e where kappa sqrt(2 pi) s_max / tau_cut = m 2^e).
 *
 * Everything except the key function is double precision.  The key function decides
 * integers (tile rectangles, depth keys); it is written in FP32 with an explicit
 * operation order and must be compiled without floating-point contraction
 * (-ffp-contract=off) so the GPU's decisions can be compared bit for bit.
 */
#include "vg_oracle.h"

#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel regions (n < 1: all cores); returns the count now in use. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* =============================== FP32 key function =============================== */

/* Validity, unit quaternion, rotation and world covariance Sigma = R S^2 R^T, all FP32. */
static int cov_fp32(const float *mu, const float *s, const float *q, float kap, float Sig[9],
                    float *smax)
{
    for (int k = 0; k < 3; ++k)
        if (!isfinite(mu[k]) || !isfinite(s[k]) || !(s[k] > 0.0f)) return 0;
    for (int k = 0; k < 4; ++k)
        if (!isfinite(q[k])) return 0;
    if (!isfinite(kap) || !(kap > 0.0f)) return 0;
    float n2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    if (!(n2 > 0.0f) || !isfinite(n2)) return 0;
    float inv = 1.0f / sqrtf(n2);
    float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
    float R[9];
    R[0] = 1.0f - 2.0f * (y * y + z * z);
    R[1] = 2.0f * (x * y - w * z);
    R[2] = 2.0f * (x * z + w * y);
    R[3] = 2.0f * (x * y + w * z);
    R[4] = 1.0f - 2.0f * (x * x + z * z);
    R[5] = 2.0f * (y * z - w * x);
    R[6] = 2.0f * (x * z - w * y);
    R[7] = 2.0f * (y * z + w * x);
    R[8] = 1.0f - 2.0f * (x * x + y * y);
    float v0 = s[0] * s[0], v1 = s[1] * s[1], v2 = s[2] * s[2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Sig[3 * i + j] = ((R[3 * i + 0] * v0) * R[3 * j + 0] + (R[3 * i + 1] * v1) * R[3 * j + 1]) +
                             (R[3 * i + 2] * v2) * R[3 * j + 2];
    *smax = fmaxf(fmaxf(s[0], s[1]), s[2]);
    return 1;
}

/* k^2 bound: tau >= tau_cut needs m^2 <= 2 ln(kappa sqrt(2 pi) beta / tau_cut) with
 * beta <= s_max; ln x <= e ln 2 for x = m 2^e, m in [0.5, 1). */
static int k2_bound(float kap, float smax, float tau_cut, float *k2)
{
    float xr = ((kap * 2.5066283f) * smax) / tau_cut;
    if (!(xr > 1.0f)) return 0;
    int e;
    if (xr > FLT_MAX)
        e = 128;
    else
        (void)frexpf(xr, &e);
    *k2 = (float)e * 1.3862944f;
    return 1;
}

/* Pixel indices i whose centre coordinate lies in [lo, hi] after a small outward pad. */
static void pixel_span(float lo, float hi, int n, int *ilo, int *ihi)
{
    lo = lo - (0.02f + 1e-5f * fabsf(lo));
    hi = hi + (0.02f + 1e-5f * fabsf(hi));
    if (!(hi >= 0.0f) || !(lo <= (float)(n - 1))) {
        *ilo = 1;
        *ihi = 0;
        return;
    }
    *ilo = (lo <= 0.0f) ? 0 : (int)ceilf(lo);
    *ihi = (hi >= (float)(n - 1)) ? n - 1 : (int)floorf(hi);
}

static int key_persp(const float *mu, const float *s, const float *q, float kap, const float *cf,
                     int W, int H, int tw, int th, float z_near, float tau_cut, uint32_t *depth,
                     int32_t rect[4], int32_t prect[4])
{
    rect[0] = rect[1] = rect[2] = rect[3] = -1;
    prect[0] = prect[1] = prect[2] = prect[3] = -1;
    *depth = 0xFFFFFFFFu;
    float Sig[9], smax;
    if (!cov_fp32(mu, s, q, kap, Sig, &smax)) return 0;
    const float *C = cf;
    const float *t = cf + 9;
    float X = ((C[0] * mu[0] + C[1] * mu[1]) + C[2] * mu[2]) + t[0];
    float Y = ((C[3] * mu[0] + C[4] * mu[1]) + C[5] * mu[2]) + t[1];
    float Z = ((C[6] * mu[0] + C[7] * mu[1]) + C[8] * mu[2]) + t[2];
    if (!(Z > z_near)) return 0;
    memcpy(depth, &Z, 4);
    float k2;
    if (!k2_bound(kap, smax, tau_cut, &k2)) return 0;
    float T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = (C[3 * i] * Sig[j] + C[3 * i + 1] * Sig[3 + j]) + C[3 * i + 2] * Sig[6 + j];
    float sxx = (T[0] * C[0] + T[1] * C[1]) + T[2] * C[2];
    float sxz = (T[0] * C[6] + T[1] * C[7]) + T[2] * C[8];
    float syy = (T[3] * C[3] + T[4] * C[4]) + T[5] * C[5];
    float syz = (T[3] * C[6] + T[4] * C[7]) + T[5] * C[8];
    float szz = (T[6] * C[6] + T[7] * C[7]) + T[8] * C[8];
    int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
    float ZZ = Z * Z;
    float a2 = ZZ - k2 * szz;
    if (!(a2 > 0.0f)) { /* the cutoff ellipsoid reaches the camera plane: whole view */
        rect[0] = 0;
        rect[1] = 0;
        rect[2] = tiles_x - 1;
        rect[3] = tiles_y - 1;
        prect[0] = 0;
        prect[1] = 0;
        prect[2] = W - 1;
        prect[3] = H - 1;
        return 1;
    }
    float k22 = k2 * k2;
    float XZ = X * Z, YZ = Y * Z;
    float bu = XZ - k2 * sxz;
    float qu = (ZZ * sxx - 2.0f * (XZ * sxz)) + (X * X) * szz;
    float du = k2 * qu - k22 * (sxx * szz - sxz * sxz);
    if (!(du > 0.0f)) du = 0.0f;
    float ru = sqrtf(du);
    float ulo = (bu - ru) / a2, uhi = (bu + ru) / a2;
    float bv = YZ - k2 * syz;
    float qv = (ZZ * syy - 2.0f * (YZ * syz)) + (Y * Y) * szz;
    float dv = k2 * qv - k22 * (syy * szz - syz * syz);
    if (!(dv > 0.0f)) dv = 0.0f;
    float rv = sqrtf(dv);
    float vlo = (bv - rv) / a2, vhi = (bv + rv) / a2;
    float xlo = (ulo * cf[12] + cf[14]) - 0.5f, xhi = (uhi * cf[12] + cf[14]) - 0.5f;
    float ylo = (vlo * cf[13] + cf[15]) - 0.5f, yhi = (vhi * cf[13] + cf[15]) - 0.5f;
    int ix0, ix1, iy0, iy1;
    pixel_span(xlo, xhi, W, &ix0, &ix1);
    pixel_span(ylo, yhi, H, &iy0, &iy1);
    if (ix0 > ix1 || iy0 > iy1) return 0;
    rect[0] = ix0 / tw;
    rect[1] = iy0 / th;
    rect[2] = ix1 / tw;
    rect[3] = iy1 / th;
    prect[0] = ix0;
    prect[1] = iy0;
    prect[2] = ix1;
    prect[3] = iy1;
    return 1;
}

int64_t orc_keys(int n, const float *mu, const float *scale, const float *quat, const float *kappa,
                 int n_views, const float *cam_f, const int32_t *cam_wh, int tile_w, int tile_h,
                 float z_near, float tau_cut, uint32_t *depth_bits, int32_t *rect, int32_t *prect)
{
    int64_t total = 0;
    for (int v = 0; v < n_views; ++v) {
        for (int g = 0; g < n; ++g) {
            int64_t it = (int64_t)v * n + g;
            int32_t *r = rect + 4 * it;
            if (key_persp(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g], cam_f + 16 * v,
                          cam_wh[2 * v], cam_wh[2 * v + 1], tile_w, tile_h, z_near, tau_cut,
                          depth_bits + it, r, prect + 4 * it))
                total += (int64_t)(r[2] - r[0] + 1) * (r[3] - r[1] + 1);
        }
    }
    return total;
}

/* Splat-mode key function (the 3DGS comparison mode, Eq. 5-7), FP32, fixed operation order.
 * The depth key is the camera z of the mean, as in key_persp.  The footprint is the pixel
 * bounding box of the ellipse w' Sigma'^-1 w <= k^2 of the 2D Gaussian, Sigma' = J W Sigma W' J'
 * + dilation I (Eq. 7, J the affine Jacobian of the projection at the mean), with
 * k^2 = 2 ln 2 * e where opacity / alpha_cut = m 2^e, so that every pixel outside it has
 * alpha = o G' < alpha_cut.  Its half-widths are k sqrt(Sigma'_xx) and k sqrt(Sigma'_yy). */
static int key_splat(const float *mu, const float *s, const float *q, float opac, const float *cf,
                     int W, int H, int tw, int th, float z_near, float alpha_cut, float dil,
                     uint32_t *depth, int32_t rect[4], int32_t prect[4])
{
    rect[0] = rect[1] = rect[2] = rect[3] = -1;
    prect[0] = prect[1] = prect[2] = prect[3] = -1;
    *depth = 0xFFFFFFFFu;
    float Sig[9], smax;
    if (!cov_fp32(mu, s, q, opac, Sig, &smax)) return 0;
    const float *C = cf;
    const float *t = cf + 9;
    float X = ((C[0] * mu[0] + C[1] * mu[1]) + C[2] * mu[2]) + t[0];
    float Y = ((C[3] * mu[0] + C[4] * mu[1]) + C[5] * mu[2]) + t[1];
    float Z = ((C[6] * mu[0] + C[7] * mu[1]) + C[8] * mu[2]) + t[2];
    if (!(Z > z_near)) return 0;
    memcpy(depth, &Z, 4);
    float xr = opac / alpha_cut;
    if (!(xr > 1.0f)) return 0;
    int e;
    if (xr > FLT_MAX)
        e = 128;
    else
        (void)frexpf(xr, &e);
    float k2 = (float)e * 1.3862944f;
    float T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = (C[3 * i] * Sig[j] + C[3 * i + 1] * Sig[3 + j]) + C[3 * i + 2] * Sig[6 + j];
    float sxx = (T[0] * C[0] + T[1] * C[1]) + T[2] * C[2];
    float sxz = (T[0] * C[6] + T[1] * C[7]) + T[2] * C[8];
    float syy = (T[3] * C[3] + T[4] * C[4]) + T[5] * C[5];
    float syz = (T[3] * C[6] + T[4] * C[7]) + T[5] * C[8];
    float szz = (T[6] * C[6] + T[7] * C[7]) + T[8] * C[8];
    float u = X / Z, v = Y / Z;
    float jx = cf[12] / Z, jy = cf[13] / Z;
    float exx = (sxx - 2.0f * (u * sxz)) + (u * u) * szz;
    float eyy = (syy - 2.0f * (v * syz)) + (v * v) * szz;
    if (!(exx > 0.0f)) exx = 0.0f;
    if (!(eyy > 0.0f)) eyy = 0.0f;
    float vx = (jx * jx) * exx + dil, vy = (jy * jy) * eyy + dil;
    float hx = sqrtf(k2 * vx), hy = sqrtf(k2 * vy);
    float mx = (u * cf[12] + cf[14]) - 0.5f, my = (v * cf[13] + cf[15]) - 0.5f;
    int ix0, ix1, iy0, iy1;
    pixel_span(mx - hx, mx + hx, W, &ix0, &ix1);
    pixel_span(my - hy, my + hy, H, &iy0, &iy1);
    if (ix0 > ix1 || iy0 > iy1) return 0;
    rect[0] = ix0 / tw;
    rect[1] = iy0 / th;
    rect[2] = ix1 / tw;
    rect[3] = iy1 / th;
    prect[0] = ix0;
    prect[1] = iy0;
    prect[2] = ix1;
    prect[3] = iy1;
    return 1;
}

int64_t orc_keys_splat(int n, const float *mu, const float *scale, const float *quat, const float *opac,
                       int n_views, const float *cam_f, const int32_t *cam_wh, int tile_w, int tile_h,
                       float z_near, float alpha_cut, float dilation, uint32_t *depth_bits, int32_t *rect,
                       int32_t *prect)
{
    int64_t total = 0;
    for (int v = 0; v < n_views; ++v) {
        for (int g = 0; g < n; ++g) {
            int64_t it = (int64_t)v * n + g;
            int32_t *r = rect + 4 * it;
            if (key_splat(mu + 3 * g, scale + 3 * g, quat + 4 * g, opac[g], cam_f + 16 * v, cam_wh[2 * v],
                          cam_wh[2 * v + 1], tile_w, tile_h, z_near, alpha_cut, dilation, depth_bits + it, r,
                          prect + 4 * it))
                total += (int64_t)(r[2] - r[0] + 1) * (r[3] - r[1] + 1);
        }
    }
    return total;
}

int64_t orc_tomo_keys(int n, const float *mu, const float *scale, const float *quat,
                      const float *kappa, int n_angles, const float *angles, int det_w, int det_h,
                      float pitch_u, float pitch_v, float u0, float v0, int tile_w, int tile_h,
                      float tau_cut, int32_t *rect, int32_t *prect)
{
    int64_t total = 0;
    for (int a = 0; a < n_angles; ++a) {
        float ct = (float)cos((double)angles[a]);
        float st = (float)sin((double)angles[a]);
        for (int g = 0; g < n; ++g) {
            int32_t *r = rect + 4 * ((int64_t)a * n + g);
            int32_t *pr = prect + 4 * ((int64_t)a * n + g);
            r[0] = r[1] = r[2] = r[3] = -1;
            pr[0] = pr[1] = pr[2] = pr[3] = -1;
            float Sig[9], smax, k2;
            const float *m = mu + 3 * g;
            if (!cov_fp32(m, scale + 3 * g, quat + 4 * g, kappa[g], Sig, &smax)) continue;
            if (!k2_bound(kappa[g], smax, tau_cut, &k2)) continue;
            float um = (-st) * m[0] + ct * m[1];
            float vm = m[2];
            float suu = ((st * st) * Sig[0] - 2.0f * ((st * ct) * Sig[1])) + (ct * ct) * Sig[4];
            if (!(suu > 0.0f)) suu = 0.0f;
            float svv = Sig[8];
            float hu = sqrtf(k2 * suu), hv = sqrtf(k2 * svv);
            float xlo = ((um - hu) - u0) / pitch_u - 0.5f, xhi = ((um + hu) - u0) / pitch_u - 0.5f;
            float ylo = ((vm - hv) - v0) / pitch_v - 0.5f, yhi = ((vm + hv) - v0) / pitch_v - 0.5f;
            int ix0, ix1, iy0, iy1;
            pixel_span(xlo, xhi, det_w, &ix0, &ix1);
            pixel_span(ylo, yhi, det_h, &iy0, &iy1);
            if (ix0 > ix1 || iy0 > iy1) continue;
            r[0] = ix0 / tile_w;
            r[1] = iy0 / tile_h;
            r[2] = ix1 / tile_w;
            r[3] = iy1 / tile_h;
            pr[0] = ix0;
            pr[1] = iy0;
            pr[2] = ix1;
            pr[3] = iy1;
            total += (int64_t)(r[2] - r[0] + 1) * (r[3] - r[1] + 1);
        }
    }
    return total;
}

/* ================================ binning / sort ================================ */

typedef struct {
    int64_t tile;
    uint32_t depth;
    int32_t g;
} inst_t;

static int cmp_inst(const void *pa, const void *pb)
{
    const inst_t *a = (const inst_t *)pa, *b = (const inst_t *)pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    if (a->g != b->g) return a->g < b->g ? -1 : 1;
    return 0;
}

int64_t orc_bin(int n, int n_views, const uint32_t *depth_bits, const int32_t *rect,
                const int32_t *view_tiles_x, const int32_t *view_tile_base, int64_t n_tiles_total,
                int64_t capacity, int64_t *tile_start, int32_t *sorted_g)
{
    int64_t total = 0;
    for (int64_t it = 0; it < (int64_t)n_views * n; ++it) {
        const int32_t *r = rect + 4 * it;
        if (r[0] >= 0) total += (int64_t)(r[2] - r[0] + 1) * (r[3] - r[1] + 1);
    }
    if (total > capacity) return total;
    inst_t *inst = (inst_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(inst_t));
    int64_t k = 0;
    for (int v = 0; v < n_views; ++v) {
        for (int g = 0; g < n; ++g) {
            int64_t it = (int64_t)v * n + g;
            const int32_t *r = rect + 4 * it;
            if (r[0] < 0) continue;
            for (int ty = r[1]; ty <= r[3]; ++ty)
                for (int tx = r[0]; tx <= r[2]; ++tx) {
                    inst[k].tile = (int64_t)view_tile_base[v] + (int64_t)ty * view_tiles_x[v] + tx;
                    inst[k].depth = depth_bits ? depth_bits[it] : 0u;
                    inst[k].g = g;
                    ++k;
                }
        }
    }
    qsort(inst, (size_t)total, sizeof(inst_t), cmp_inst);
    for (int64_t t = 0; t <= n_tiles_total; ++t) tile_start[t] = 0;
    for (int64_t i = 0; i < total; ++i) {
        sorted_g[i] = inst[i].g;
        tile_start[inst[i].tile + 1] += 1;
    }
    for (int64_t t = 0; t < n_tiles_total; ++t) tile_start[t + 1] += tile_start[t];
    free(inst);
    return total;
}

/* ============================ FP64 Gaussian geometry ============================ */

typedef struct {
    double mu[3];
    double qn[4];   /* unit quaternion (w, x, y, z) */
    double qnorm;   /* |q| of the input */
    double R[9];    /* rotation, row-major; column k is principal axis k */
    double s[3];
    double P[9];    /* precision Sigma^-1 = R diag(1/s^2) R^T */
    double kap;
} gauss64;

static int valid64(const double *mu, const double *s, const double *q, double kap)
{
    for (int k = 0; k < 3; ++k)
        if (!isfinite(mu[k]) || !isfinite(s[k]) || !(s[k] > 0)) return 0;
    double n2 = 0;
    for (int k = 0; k < 4; ++k) {
        if (!isfinite(q[k])) return 0;
        n2 += q[k] * q[k];
    }
    return isfinite(kap) && kap > 0 && n2 > 0 && isfinite(n2);
}

static void prep64(const double *mu, const double *s, const double *q, double kap, gauss64 *G)
{
    for (int k = 0; k < 3; ++k) {
        G->mu[k] = mu[k];
        G->s[k] = s[k];
    }
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    G->qnorm = n;
    double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    G->qn[0] = w;
    G->qn[1] = x;
    G->qn[2] = y;
    G->qn[3] = z;
    double *R = G->R;
    R[0] = 1 - 2 * (y * y + z * z);
    R[1] = 2 * (x * y - w * z);
    R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);
    R[4] = 1 - 2 * (x * x + z * z);
    R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);
    R[7] = 2 * (y * z + w * x);
    R[8] = 1 - 2 * (x * x + y * y);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * R[3 * j + k] / (G->s[k] * G->s[k]);
            G->P[3 * i + j] = acc;
        }
    G->kap = kap;
}

/* tau of one Gaussian along the line o + t d (d unit), Eq. 19 in the a, b, c form. */
static double tau64(const gauss64 *G, const double o[3], const double d[3], double *pa,
                    double *pb, double *pc, double p[3])
{
    for (int k = 0; k < 3; ++k) p[k] = o[k] - G->mu[k];
    double Pd[3], Pp[3];
    for (int i = 0; i < 3; ++i) {
        Pd[i] = G->P[3 * i] * d[0] + G->P[3 * i + 1] * d[1] + G->P[3 * i + 2] * d[2];
        Pp[i] = G->P[3 * i] * p[0] + G->P[3 * i + 1] * p[1] + G->P[3 * i + 2] * p[2];
    }
    double a = d[0] * Pd[0] + d[1] * Pd[1] + d[2] * Pd[2];
    double b = d[0] * Pp[0] + d[1] * Pp[1] + d[2] * Pp[2];
    double c = p[0] * Pp[0] + p[1] * Pp[1] + p[2] * Pp[2];
    *pa = a;
    *pb = b;
    *pc = c;
    /* Eq. 19 as printed: tau = kappa G(o + gamma d) sqrt(2 pi) beta with gamma = -b/a the
     * maximiser along the ray and beta = a^-1/2.  G is evaluated at the maximiser itself
     * (stationary in gamma), which avoids the cancellation in c - b^2/a. */
    double gam = -b / a, e[3], Pe[3];
    for (int k = 0; k < 3; ++k) e[k] = p[k] + gam * d[k];
    for (int i = 0; i < 3; ++i) Pe[i] = G->P[3 * i] * e[0] + G->P[3 * i + 1] * e[1] + G->P[3 * i + 2] * e[2];
    double m2 = e[0] * Pe[0] + e[1] * Pe[1] + e[2] * Pe[2];
    return G->kap * exp(-0.5 * m2) * sqrt(2.0 * ORC_PI) / sqrt(a);
}

void orc_tau(const double *mu, const double *scale, const double *quat, double kappa, const double *o,
             const double *d, double *out)
{
    gauss64 G;
    prep64(mu, scale, quat, kappa, &G);
    double a, b, c, p[3];
    double t = tau64(&G, o, d, &a, &b, &c, p);
    out[0] = t;
    out[1] = a;
    out[2] = b;
    out[3] = c;
    out[4] = -b / a;                          /* gamma: the maximiser of G along the ray   */
    out[5] = 1.0 / sqrt(a);                   /* beta: standard deviation along the ray     */
    out[6] = t / (G.kap * sqrt(2.0 * ORC_PI / a)); /* G_j(o + gamma d): maximum along the ray */
}

/* Real spherical harmonics up to degree 3 (Condon-Shortley phase), evaluated on complex
 * arguments so that the gradient can be taken by the complex-step method. */
static void sh_eval_c(int deg, double complex x, double complex y, double complex z,
                      double complex *out)
{
    const double c0 = 0.5 * sqrt(1.0 / ORC_PI);
    const double c1 = sqrt(3.0 / (4.0 * ORC_PI));
    const double c2a = 0.5 * sqrt(15.0 / ORC_PI), c2b = 0.25 * sqrt(5.0 / ORC_PI),
                 c2c = 0.25 * sqrt(15.0 / ORC_PI);
    const double c3a = 0.25 * sqrt(35.0 / (2.0 * ORC_PI)), c3b = 0.5 * sqrt(105.0 / ORC_PI),
                 c3c = 0.25 * sqrt(21.0 / (2.0 * ORC_PI)), c3d = 0.25 * sqrt(7.0 / ORC_PI),
                 c3e = 0.25 * sqrt(105.0 / ORC_PI);
    double complex xx = x * x, yy = y * y, zz = z * z;
    out[0] = c0;
    if (deg < 1) return;
    out[1] = -c1 * y;
    out[2] = c1 * z;
    out[3] = -c1 * x;
    if (deg < 2) return;
    out[4] = c2a * x * y;
    out[5] = -c2a * y * z;
    out[6] = c2b * (2.0 * zz - xx - yy);
    out[7] = -c2a * x * z;
    out[8] = c2c * (xx - yy);
    if (deg < 3) return;
    out[9] = -c3a * y * (3.0 * xx - yy);
    out[10] = c3b * x * y * z;
    out[11] = -c3c * y * (4.0 * zz - xx - yy);
    out[12] = c3d * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    out[13] = -c3c * x * (4.0 * zz - xx - yy);
    out[14] = c3e * z * (xx - yy);
    out[15] = -c3a * x * (xx - 3.0 * yy);
}

void orc_sh_basis(int degree, const double *dir, double *out)
{
    double complex v[16];
    sh_eval_c(degree, dir[0], dir[1], dir[2], v);
    int K = (degree + 1) * (degree + 1);
    for (int k = 0; k < K; ++k) out[k] = creal(v[k]);
}

/* d Y_k / d dir_j by the complex-step method: exact to rounding for polynomials. */
static void sh_grad(int deg, const double dir[3], double dY[16][3])
{
    const double h = 1e-30;
    double complex v[16];
    for (int j = 0; j < 3; ++j) {
        double complex a = dir[0], b = dir[1], c = dir[2];
        if (j == 0) a += I * h;
        if (j == 1) b += I * h;
        if (j == 2) c += I * h;
        sh_eval_c(deg, a, b, c, v);
        int K = (deg + 1) * (deg + 1);
        for (int k = 0; k < K; ++k) dY[k][j] = cimag(v[k]) / h;
    }
}

typedef struct {
    double R[9], t[3], fx, fy, cx, cy, o[3];
    int W, H;
} cam64;

static void cam_setup(const float *cf, const int32_t *wh, cam64 *c)
{
    for (int k = 0; k < 9; ++k) c->R[k] = cf[k];
    for (int k = 0; k < 3; ++k) c->t[k] = cf[9 + k];
    c->fx = cf[12];
    c->fy = cf[13];
    c->cx = cf[14];
    c->cy = cf[15];
    c->W = wh[0];
    c->H = wh[1];
    for (int k = 0; k < 3; ++k)   /* o = -R^T t */
        c->o[k] = -(c->R[k] * c->t[0] + c->R[3 + k] * c->t[1] + c->R[6 + k] * c->t[2]);
}

/* Unit world direction of the ray through the centre of pixel (x, y) (Sec. 4.1). */
static void pixel_dir(const cam64 *c, int x, int y, double d[3])
{
    double dc[3] = {(x + 0.5 - c->cx) / c->fx, (y + 0.5 - c->cy) / c->fy, 1.0};
    double n2 = 0;
    for (int k = 0; k < 3; ++k) {
        d[k] = c->R[k] * dc[0] + c->R[3 + k] * dc[1] + c->R[6 + k] * dc[2];
        n2 += d[k] * d[k];
    }
    double n = sqrt(n2);
    for (int k = 0; k < 3; ++k) d[k] /= n;
}

/* ------------------------------------------------------------------ splat mode (Eq. 5-7)
 * The 3DGS comparison mode: alpha = o G'(p) (Eq. 6), G' the 2D Gaussian with mean mu' the
 * projection of mu and covariance Sigma' = J W Sigma W^T J^T (Eq. 7) plus an optional isotropic
 * dilation, J the Jacobian of the pinhole projection at the camera-space mean t:
 *   J = [[fx/tz, 0, -fx tx/tz^2], [0, fy/tz, -fy ty/tz^2]].
 * Pixel (x, y) has its centre at index coordinates (x, y), so mu' = (fx tx/tz + cx - 1/2,
 * fy ty/tz + cy - 1/2) in the same coordinates. */
typedef struct {
    double t[3];     /* camera-space mean */
    double J[6];     /* row-major 2 x 3 */
    double V[9];     /* camera-space covariance W Sigma W^T */
    double S2[4];    /* Sigma' (2 x 2, row-major) */
    double Q[4];     /* Sigma'^-1 */
    double m[2];     /* mu' */
    int ok;
} splat64;

static void splat_setup(const gauss64 *G, const cam64 *c, double dil, splat64 *S)
{
    S->ok = 0;
    for (int i = 0; i < 3; ++i)
        S->t[i] = c->R[3 * i] * G->mu[0] + c->R[3 * i + 1] * G->mu[1] + c->R[3 * i + 2] * G->mu[2] + c->t[i];
    const double tx = S->t[0], ty = S->t[1], tz = S->t[2];
    if (!(tz > 0)) return;
    double Sig[9], WS[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += G->R[3 * i + k] * G->s[k] * G->s[k] * G->R[3 * j + k];
            Sig[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += c->R[3 * i + k] * Sig[3 * k + j];
            WS[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += WS[3 * i + k] * c->R[3 * j + k];
            S->V[3 * i + j] = acc;
        }
    double *J = S->J;
    J[0] = c->fx / tz;
    J[1] = 0;
    J[2] = -c->fx * tx / (tz * tz);
    J[3] = 0;
    J[4] = c->fy / tz;
    J[5] = -c->fy * ty / (tz * tz);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += J[3 * i + a] * S->V[3 * a + b] * J[3 * j + b];
            S->S2[2 * i + j] = acc + (i == j ? dil : 0.0);
        }
    const double det = S->S2[0] * S->S2[3] - S->S2[1] * S->S2[2];
    if (!(det > 0)) return;
    S->Q[0] = S->S2[3] / det;
    S->Q[1] = -S->S2[1] / det;
    S->Q[2] = -S->S2[2] / det;
    S->Q[3] = S->S2[0] / det;
    S->m[0] = c->fx * tx / tz + c->cx - 0.5;
    S->m[1] = c->fy * ty / tz + c->cy - 0.5;
    S->ok = 1;
}

/* o G'(p) at pixel (x, y): returns the unclamped opacity, w = p - mu' and q = w' Q w. */
static double splat_alpha(const splat64 *S, double opac, int x, int y, double w[2], double *q)
{
    w[0] = x - S->m[0];
    w[1] = y - S->m[1];
    *q = S->Q[0] * w[0] * w[0] + (S->Q[1] + S->Q[2]) * w[0] * w[1] + S->Q[3] * w[1] * w[1];
    return opac * exp(-0.5 * *q);
}

/* Largest splat opacity: the clamp 1 - exp(-tau_max) (0.99 in the 3DGS convention), and at most
 * 1 - 2^-24, so that 1 - alpha and the log-transmittance stay finite. */
static double splat_alpha_max(double tau_max)
{
    double a = -expm1(-tau_max);
    const double cap = 1.0 - 5.9604644775390625e-8;
    return a < cap ? a : cap;
}

void orc_splat2d(const double *mu, const double *scale, const double *quat, const float *cam_f,
                 const int32_t *cam_wh, double dil, double *out)
{
    gauss64 G;
    prep64(mu, scale, quat, 1.0, &G);
    cam64 cam;
    cam_setup(cam_f, cam_wh, &cam);
    splat64 S;
    splat_setup(&G, &cam, dil, &S);
    out[0] = S.m[0];
    out[1] = S.m[1];
    out[2] = S.S2[0];
    out[3] = S.S2[1];
    out[4] = S.S2[3];
    out[5] = S.ok;
}

/* Output activation of the colour: the clamp max(x, 0), or with beta > 0 the softplus
 * (1/beta) ln(1 + e^(beta x)) (Supp. D, beta = 10), and its derivative. */
static double colour_act(double x, double beta)
{
    if (!(beta > 0)) return x > 0 ? x : 0;
    const double t = beta * x;
    return (t > 0 ? t + log1p(exp(-t)) : log1p(exp(t))) / beta;
}

static double colour_act_grad(double x, double beta)
{
    if (!(beta > 0)) return x > 0 ? 1.0 : 0.0;
    return 1.0 / (1.0 + exp(-beta * x));
}

/* View-dependent colour: rgb = act(sum_k sh_k Y_k(dir) + 0.5), dir = (mu - o)/|mu - o|, act the
 * clamp at 0 or the softplus (see colour_act). */
static void colour64(const double *sh, int deg, const gauss64 *G, const double o[3], double rgb[3],
                     double raw[3], double beta)
{
    double dir[3], n2 = 0;
    for (int k = 0; k < 3; ++k) {
        dir[k] = G->mu[k] - o[k];
        n2 += dir[k] * dir[k];
    }
    double n = sqrt(n2);
    for (int k = 0; k < 3; ++k) dir[k] /= n;
    double Y[16];
    orc_sh_basis(deg, dir, Y);
    int K = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.5;
        for (int k = 0; k < K; ++k) acc += sh[3 * k + ch] * Y[k];
        raw[ch] = acc;
        rgb[ch] = colour_act(acc, beta);
    }
}

typedef struct {
    int64_t g;
    uint32_t depth;
} order_t;

static int cmp_order(const void *pa, const void *pb)
{
    const order_t *a = (const order_t *)pa, *b = (const order_t *)pb;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    return a->g < b->g ? -1 : (a->g > b->g);
}

static double tau_skip_of(double alpha_min)
{
    if (!(alpha_min > 0)) return 0.0;
    if (alpha_min >= 1) return INFINITY;
    return -log1p(-alpha_min);
}

/* A Gaussian contributes to the pixels of its footprint rectangle (inclusive pixel
 * bounds from the key function); tile lists are the coarse version of the same set. */
static int outside(const int32_t *prect, int64_t item, int x, int y)
{
    if (!prect) return 0;
    const int32_t *r = prect + 4 * item;
    return x < r[0] || x > r[2] || y < r[1] || y > r[3];
}

/* ================================ forward render ================================ */

void orc_render(int n, const double *mu, const double *scale, const double *quat, const double *kappa,
                const double *sh, int sh_degree, int n_views, const float *cam_f,
                const int32_t *cam_wh, int tile_w, int tile_h, const double *opts,
                const int64_t *tile_start, const int32_t *sorted_g, const int32_t *view_tile_base,
                int brute, const uint32_t *depth_bits, const int32_t *prect,
                const int64_t *pix_base, const int32_t *pix_mask, double *rgb, double *T_final,
                int32_t *n_blend, int64_t *last_pos, double *diag)
{
    const double tau_skip = tau_skip_of(opts[0]);
    const double tau_max = opts[2], T_stop = opts[3];
    const double bg[3] = {opts[4], opts[5], opts[6]};
    const int splat = opts[9] != 0;
    const double amax = splat_alpha_max(tau_max);
    const int K = (sh_degree + 1) * (sh_degree + 1);
    gauss64 *G = (gauss64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(gauss64));
    double *col = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    order_t *ord = (order_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(order_t));
    splat64 *SP = (splat64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(splat64));
    for (int g = 0; g < n; ++g) prep64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g], &G[g]);
    for (int v = 0; v < n_views; ++v) {
        cam64 cam;
        cam_setup(cam_f + 16 * v, cam_wh + 2 * v, &cam);
        double raw[3];
        for (int g = 0; g < n; ++g) {
            colour64(sh + (size_t)g * K * 3, sh_degree, &G[g], cam.o, col + 3 * g, raw, opts[8]);
            if (splat) splat_setup(&G[g], &cam, opts[10], &SP[g]);
        }
        int64_t n_ord = 0;
        if (brute) {
            for (int g = 0; g < n; ++g) {
                uint32_t dk = depth_bits[(int64_t)v * n + g];
                if (dk != 0xFFFFFFFFu) {
                    ord[n_ord].g = g;
                    ord[n_ord].depth = dk;
                    ++n_ord;
                }
            }
            qsort(ord, (size_t)n_ord, sizeof(order_t), cmp_order);
        }
        const int W = cam.W, H = cam.H;
        const int tiles_x = (W + tile_w - 1) / tile_w;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t pix = 0; pix < (int64_t)W * H; ++pix) {
            int64_t gp = pix_base[v] + pix;
            if (pix_mask && !pix_mask[gp]) continue;
            int x = (int)(pix % W), y = (int)(pix / W);
            double d[3];
            pixel_dir(&cam, x, y, d);
            int64_t lo, hi;
            if (brute) {
                lo = 0;
                hi = n_ord;
            } else {
                int64_t tile = view_tile_base[v] + (int64_t)(y / tile_h) * tiles_x + x / tile_w;
                lo = tile_start[tile];
                hi = tile_start[tile + 1];
            }
            double T = 1.0, C[3] = {0, 0, 0}, S = 0.0;
            /* how close each threshold decision of this pixel came to going the other way
             * (relative distance to alpha_min / tau_max / T_stop; INFINITY: no such decision) */
            double m_skip = INFINITY, m_clamp = INFINITY, m_stop = INFINITY;
            int nb = 0;
            int64_t last = lo;
            for (int64_t k = lo; k < hi; ++k) {
                int64_t g = brute ? ord[k].g : sorted_g[k];
                if (!brute && outside(prect, (int64_t)v * n + g, x, y)) continue;
                double tau, alpha;
                if (splat) {   /* Eq. 6: alpha = o G'(p), clamped; tau = -ln(1 - alpha) */
                    if (!SP[g].ok) continue;
                    double w[2], q;
                    alpha = splat_alpha(&SP[g], G[g].kap, x, y, w, &q);
                    if (amax < 1.0) m_clamp = fmin(m_clamp, fabs(alpha - amax) / amax);
                    if (alpha > amax) alpha = amax;
                    if (opts[0] > 0) m_skip = fmin(m_skip, fabs(alpha - opts[0]) / opts[0]);
                    if (alpha < opts[0]) continue;
                    tau = -log1p(-alpha);
                } else {
                    double a, b, c, p[3];
                    tau = tau64(&G[g], cam.o, d, &a, &b, &c, p);
                    if (isfinite(tau_max)) m_clamp = fmin(m_clamp, fabs(tau - tau_max) / tau_max);
                    if (tau > tau_max) tau = tau_max;
                    if (tau_skip > 0) m_skip = fmin(m_skip, fabs(tau - tau_skip) / tau_skip);
                    if (tau < tau_skip) continue;
                    alpha = -expm1(-tau);
                }
                for (int ch = 0; ch < 3; ++ch) C[ch] += col[3 * g + ch] * alpha * T;
                T *= exp(-tau);
                S += tau;
                ++nb;
                last = k + 1;
                if (T_stop > 0) m_stop = fmin(m_stop, fabs(T - T_stop) / T_stop);
                if (T < T_stop) break;
            }
            for (int ch = 0; ch < 3; ++ch) rgb[3 * gp + ch] = C[ch] + T * bg[ch];
            T_final[gp] = T;
            if (n_blend) n_blend[gp] = nb;
            if (last_pos) last_pos[gp] = last - lo;
            if (diag) {
                diag[4 * gp] = S;
                diag[4 * gp + 1] = m_skip;
                diag[4 * gp + 2] = m_clamp;
                diag[4 * gp + 3] = m_stop;
            }
        }
    }
    free(G);
    free(col);
    free(ord);
    free(SP);
}

/* ============================ analytic gradient ============================ */

/* Per-(view, Gaussian) accumulators: dL/dP (full 3x3), geometric dL/dmu, dL/dkappa, dL/drgb. */
#define ACC_N 16

static void atomic_add(double *p, double v)
{
#pragma omp atomic
    *p += v;
}

/* Accumulate dL/dtau for one (pixel, Gaussian) pair into dL/dP, dL/dmu and dL/dkappa.
 * ln tau = ln kappa + ln sqrt(2 pi) - ln(a)/2 - c/2 + b^2/(2a). */
static void acc_tau(double *acc, const gauss64 *G, double dLdtau, double tau, double a, double b,
                    const double d[3], const double p[3])
{
    double dl = dLdtau * tau; /* dL/d ln tau */
    double La = dl * (-0.5 / a - 0.5 * b * b / (a * a));
    double Lb = dl * (b / a);
    double Lc = dl * (-0.5);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            atomic_add(&acc[3 * i + j], La * d[i] * d[j] + Lb * d[i] * p[j] + Lc * p[i] * p[j]);
    for (int i = 0; i < 3; ++i) {
        double Pd = G->P[3 * i] * d[0] + G->P[3 * i + 1] * d[1] + G->P[3 * i + 2] * d[2];
        double Pp = G->P[3 * i] * p[0] + G->P[3 * i + 1] * p[1] + G->P[3 * i + 2] * p[2];
        atomic_add(&acc[9 + i], -Lb * Pd - 2.0 * Lc * Pp);
    }
    atomic_add(&acc[12], dl / G->kap);
}

static void chain_R(const gauss64 *G, const double dR[9], double *dquat);

/* Chain dL/dP into dL/dscale and dL/dquat (through the unit quaternion). */
static void chain_P(const gauss64 *G, const double Gm[9], double *dscale, double *dquat)
{
    const double *R = G->R;
    double Dg[3];
    for (int k = 0; k < 3; ++k) Dg[k] = 1.0 / (G->s[k] * G->s[k]);
    /* P = sum_k s_k^-2 r_k r_k^T  =>  dL/ds_k = -2 s_k^-3 r_k^T G r_k */
    for (int k = 0; k < 3; ++k) {
        double acc = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) acc += R[3 * i + k] * Gm[3 * i + j] * R[3 * j + k];
        dscale[k] += -2.0 * acc / (G->s[k] * G->s[k] * G->s[k]);
    }
    /* dL/dR = (G + G^T) R D */
    double dR[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += (Gm[3 * a + j] + Gm[3 * j + a]) * R[3 * j + b];
            dR[3 * a + b] = acc * Dg[b];
        }
    chain_R(G, dR, dquat);
}

/* Chain dL/dR (row-major) into dL/dquat through the unit quaternion. */
static void chain_R(const gauss64 *G, const double dR[9], double *dquat)
{
    /* R(w, x, y, z) entries differentiated by hand. */
    double w = G->qn[0], x = G->qn[1], y = G->qn[2], z = G->qn[3];
    double J[9][4] = {
        {0, 0, -4 * y, -4 * z},         {-2 * z, 2 * y, 2 * x, -2 * w}, {2 * y, 2 * z, 2 * w, 2 * x},
        {2 * z, 2 * y, 2 * x, 2 * w},   {0, -4 * x, 0, -4 * z},         {-2 * x, -2 * w, 2 * z, 2 * y},
        {-2 * y, 2 * z, -2 * w, 2 * x}, {2 * x, 2 * w, 2 * z, 2 * y},   {0, -4 * x, -4 * y, 0},
    };
    double dqn[4] = {0, 0, 0, 0};
    for (int e = 0; e < 9; ++e)
        for (int c = 0; c < 4; ++c) dqn[c] += dR[e] * J[e][c];
    /* q_n = q / |q|  =>  dL/dq = (dqn - q_n (q_n . dqn)) / |q| */
    double dot = 0;
    for (int c = 0; c < 4; ++c) dot += G->qn[c] * dqn[c];
    for (int c = 0; c < 4; ++c) dquat[c] += (dqn[c] - G->qn[c] * dot) / G->qnorm;
}

/* Splat mode: chain the per-(view, Gaussian) sums dL/dQ = sum dL/dq w w^T (A[0..2] = xx, xy, yy)
 * and dL/dmu' (A[4..5]) through Q = Sigma'^-1, Sigma' = J V J^T + dil I, V = W Sigma W^T,
 * Sigma = R diag(s^2) R^T, mu' = (fx tx/tz, fy ty/tz) + const and J(t), t = W mu + t_cam. */
static void chain_splat(const gauss64 *G, const splat64 *S, const cam64 *c, const double *A, double *dmu,
                        double *dscale, double *dquat)
{
    const double dQ[4] = {A[0], A[1], A[1], A[2]};
    const double *Q = S->Q, *J = S->J, *V = S->V, *W = c->R;
    double T1[4], dS[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) T1[2 * i + j] = Q[2 * i] * dQ[j] + Q[2 * i + 1] * dQ[2 + j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) dS[2 * i + j] = -(T1[2 * i] * Q[j] + T1[2 * i + 1] * Q[2 + j]);
    double dV[9], dJ[6];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) acc += J[3 * i + a] * dS[2 * i + j] * J[3 * j + b];
            dV[3 * a + b] = acc;
        }
    for (int i = 0; i < 2; ++i)
        for (int a = 0; a < 3; ++a) {
            double acc = 0;
            for (int j = 0; j < 2; ++j)
                for (int b = 0; b < 3; ++b) acc += dS[2 * i + j] * J[3 * j + b] * V[3 * b + a];
            dJ[3 * i + a] = 2.0 * acc;
        }
    double dSig[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) acc += W[3 * i + a] * dV[3 * i + j] * W[3 * j + b];
            dSig[3 * a + b] = acc;
        }
    const double *R = G->R;
    for (int k = 0; k < 3; ++k) {
        double acc = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) acc += R[3 * i + k] * dSig[3 * i + j] * R[3 * j + k];
        dscale[k] += 2.0 * G->s[k] * acc;
    }
    double dR[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += (dSig[3 * a + j] + dSig[3 * j + a]) * R[3 * j + b];
            dR[3 * a + b] = acc * G->s[b] * G->s[b];
        }
    chain_R(G, dR, dquat);
    const double tx = S->t[0], ty = S->t[1], tz = S->t[2], fx = c->fx, fy = c->fy;
    const double iz = 1.0 / tz, iz2 = iz * iz, iz3 = iz2 * iz;
    double dt[3];
    dt[0] = A[4] * fx * iz - dJ[2] * fx * iz2;
    dt[1] = A[5] * fy * iz - dJ[5] * fy * iz2;
    dt[2] = -A[4] * fx * tx * iz2 - A[5] * fy * ty * iz2 - dJ[0] * fx * iz2 + dJ[2] * 2.0 * fx * tx * iz3 -
            dJ[4] * fy * iz2 + dJ[5] * 2.0 * fy * ty * iz3;
    for (int k = 0; k < 3; ++k) dmu[k] += W[k] * dt[0] + W[3 + k] * dt[1] + W[6 + k] * dt[2];
}

typedef struct {
    int64_t g;
    double tau, alpha, T;
    int clamped;
} blend_rec;

void orc_render_grad(int n, const double *mu, const double *scale, const double *quat,
                     const double *kappa, const double *sh, int sh_degree, int n_views,
                     const float *cam_f, const int32_t *cam_wh, int tile_w, int tile_h,
                     const double *opts, const int64_t *tile_start, const int32_t *sorted_g,
                     const int32_t *view_tile_base, const int32_t *prect, const int64_t *pix_base,
                     const double *dL_drgb, const double *dL_dT, const int32_t *pix_mask,
                     double *dmu, double *dscale, double *dquat, double *dkappa, double *dsh)
{
    const double tau_skip = tau_skip_of(opts[0]);
    const double tau_max = opts[2], T_stop = opts[3];
    const double bg[3] = {opts[4], opts[5], opts[6]};
    const int splat = opts[9] != 0;
    const double amax = splat_alpha_max(tau_max);
    const int K = (sh_degree + 1) * (sh_degree + 1);
    gauss64 *G = (gauss64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(gauss64));
    double *col = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    double *acc = (double *)calloc((size_t)(n > 0 ? n : 1) * ACC_N, sizeof(double));
    splat64 *SP = (splat64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(splat64));
    for (int g = 0; g < n; ++g) prep64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g], &G[g]);
    int64_t maxlen = 1;
    for (int v = 0; v < n_views; ++v) {
        int tx = (cam_wh[2 * v] + tile_w - 1) / tile_w, ty = (cam_wh[2 * v + 1] + tile_h - 1) / tile_h;
        for (int64_t t = view_tile_base[v]; t < view_tile_base[v] + (int64_t)tx * ty; ++t)
            if (tile_start[t + 1] - tile_start[t] > maxlen) maxlen = tile_start[t + 1] - tile_start[t];
    }
    for (int v = 0; v < n_views; ++v) {
        cam64 cam;
        cam_setup(cam_f + 16 * v, cam_wh + 2 * v, &cam);
        double raw[3];
        for (int g = 0; g < n; ++g) {
            colour64(sh + (size_t)g * K * 3, sh_degree, &G[g], cam.o, col + 3 * g, raw, opts[8]);
            if (splat) splat_setup(&G[g], &cam, opts[10], &SP[g]);
        }
        memset(acc, 0, (size_t)(n > 0 ? n : 1) * ACC_N * sizeof(double));
        const int W = cam.W, H = cam.H;
        const int tiles_x = (W + tile_w - 1) / tile_w;
#pragma omp parallel
        {
            blend_rec *rec = (blend_rec *)malloc((size_t)maxlen * sizeof(blend_rec));
#pragma omp for schedule(dynamic, 16)
            for (int64_t pix = 0; pix < (int64_t)W * H; ++pix) {
                int64_t gp = pix_base[v] + pix;
                if (pix_mask && !pix_mask[gp]) continue;
                int x = (int)(pix % W), y = (int)(pix / W);
                double d[3];
                pixel_dir(&cam, x, y, d);
                int64_t tile = view_tile_base[v] + (int64_t)(y / tile_h) * tiles_x + x / tile_w;
                int64_t lo = tile_start[tile], hi = tile_start[tile + 1];
                double T = 1.0;
                int nr = 0;
                for (int64_t k = lo; k < hi; ++k) {
                    int64_t g = sorted_g[k];
                    if (outside(prect, (int64_t)v * n + g, x, y)) continue;
                    double tau, alpha;
                    int clamped = 0;
                    if (splat) {
                        if (!SP[g].ok) continue;
                        double w[2], q;
                        alpha = splat_alpha(&SP[g], G[g].kap, x, y, w, &q);
                        if (alpha > amax) {
                            alpha = amax;
                            clamped = 1;
                        }
                        if (alpha < opts[0]) continue;
                        tau = -log1p(-alpha);
                    } else {
                        double a, b, c, p[3];
                        tau = tau64(&G[g], cam.o, d, &a, &b, &c, p);
                        if (tau > tau_max) {
                            tau = tau_max;
                            clamped = 1;
                        }
                        if (tau < tau_skip) continue;
                        alpha = -expm1(-tau);
                    }
                    rec[nr].g = g;
                    rec[nr].tau = tau;
                    rec[nr].alpha = alpha;
                    rec[nr].T = T;
                    rec[nr].clamped = clamped;
                    ++nr;
                    T *= exp(-tau);
                    if (T < T_stop) break;
                }
                const double *gc = dL_drgb + 3 * gp;
                double gT = dL_dT ? dL_dT[gp] : 0.0;
                double Tend = T;
                double Rs[3] = {Tend * bg[0], Tend * bg[1], Tend * bg[2]};
                for (int r = nr - 1; r >= 0; --r) {
                    int64_t g = rec[r].g;
                    double al = rec[r].alpha, Ti = rec[r].T, Tn = Ti * exp(-rec[r].tau);
                    double dLdtau = -gT * Tend;
                    for (int ch = 0; ch < 3; ++ch) {
                        double cc = col[3 * g + ch];
                        atomic_add(&acc[ACC_N * g + 13 + ch], gc[ch] * al * Ti);
                        dLdtau += gc[ch] * (cc * Tn - Rs[ch]);
                        Rs[ch] += cc * al * Ti;
                    }
                    if (!rec[r].clamped && splat) {
                        /* tau = -ln(1 - alpha), alpha = o exp(-q/2), q = w' Q w, w = p - mu' */
                        double w[2], q;
                        const splat64 *S = &SP[g];
                        splat_alpha(S, G[g].kap, x, y, w, &q);
                        const double dLda = dLdtau / (1.0 - al);
                        const double dLdq = -0.5 * al * dLda;
                        double *A = &acc[ACC_N * g];
                        atomic_add(&A[0], dLdq * w[0] * w[0]);
                        atomic_add(&A[1], dLdq * w[0] * w[1]);
                        atomic_add(&A[2], dLdq * w[1] * w[1]);
                        atomic_add(&A[4], -2.0 * dLdq * (S->Q[0] * w[0] + S->Q[1] * w[1]));
                        atomic_add(&A[5], -2.0 * dLdq * (S->Q[2] * w[0] + S->Q[3] * w[1]));
                        atomic_add(&A[12], dLda * al / G[g].kap);
                    } else if (!rec[r].clamped) {
                        double a, b, c, p[3];
                        double tau = tau64(&G[g], cam.o, d, &a, &b, &c, p);
                        acc_tau(&acc[ACC_N * g], &G[g], dLdtau, tau, a, b, d, p);
                    }
                }
            }
            free(rec);
        }
        /* chain the per-view accumulators into parameter gradients */
        for (int g = 0; g < n; ++g) {
            double *A = &acc[ACC_N * g];
            int any = 0;
            for (int k = 0; k < ACC_N; ++k) any |= (A[k] != 0.0);
            if (!any) continue;
            if (splat) {
                chain_splat(&G[g], &SP[g], &cam, A, dmu + 3 * g, dscale + 3 * g, dquat + 4 * g);
            } else {
                chain_P(&G[g], A, dscale + 3 * g, dquat + 4 * g);
                for (int k = 0; k < 3; ++k) dmu[3 * g + k] += A[9 + k];
            }
            dkappa[g] += A[12];
            /* colour: rgb = act(sh . Y(dir) + 0.5), dir = (mu - o)/|mu - o| */
            double rgb[3], rw[3], dir[3], n2 = 0;
            colour64(sh + (size_t)g * K * 3, sh_degree, &G[g], cam.o, rgb, rw, opts[8]);
            for (int k = 0; k < 3; ++k) {
                dir[k] = G[g].mu[k] - cam.o[k];
                n2 += dir[k] * dir[k];
            }
            double nrm = sqrt(n2);
            for (int k = 0; k < 3; ++k) dir[k] /= nrm;
            double Y[16], dY[16][3];
            orc_sh_basis(sh_degree, dir, Y);
            sh_grad(sh_degree, dir, dY);
            double gdir[3] = {0, 0, 0};
            for (int ch = 0; ch < 3; ++ch) {
                const double gch = A[13 + ch] * colour_act_grad(rw[ch], opts[8]);
                if (gch == 0) continue;
                for (int k = 0; k < K; ++k) {
                    dsh[((size_t)g * K + k) * 3 + ch] += gch * Y[k];
                    for (int j = 0; j < 3; ++j) gdir[j] += gch * sh[((size_t)g * K + k) * 3 + ch] * dY[k][j];
                }
            }
            double dotd = gdir[0] * dir[0] + gdir[1] * dir[1] + gdir[2] * dir[2];
            for (int j = 0; j < 3; ++j) dmu[3 * g + j] += (gdir[j] - dir[j] * dotd) / nrm;
        }
    }
    free(G);
    free(col);
    free(acc);
    free(SP);
}

/* ======================== ray-marching reference (Supp. A) ======================== */
/* Eq. 1 discretised with the quadrature of NeRF (Mildenhall et al. 2020, its Eq. 3) on
 * n_samples midpoint samples t_k = t_near + (k + 1/2) delta of [t_near, t_far] along each pixel's
 * unit ray from the camera centre, with the fields of Supp. A (with kappa, reading 11):
 *   sigma(x) = sum_i kappa_i G_i(x),  c(x) = sum_i c_i kappa_i G_i(x) / sigma(x),
 *   C = sum_k T_k (1 - exp(-sigma_k delta)) c(x_k) + T bg,  T_k = exp(-delta sum_{j<k} sigma_j).
 * c_i is the Gaussian's colour for the view (the rasterizer's).  Every Gaussian with a valid depth
 * key takes part, with no lists and no order; T_stop (opts[3]) ends a pixel's march. */
void orc_ray_march(int n, const double *mu, const double *scale, const double *quat, const double *kappa,
                   const double *sh, int sh_degree, int n_views, const float *cam_f, const int32_t *cam_wh,
                   const double *opts, const uint32_t *depth_bits, double t_near, double t_far, int n_samples,
                   const int64_t *pix_base, const int32_t *pix_mask, double *rgb, double *T_final)
{
    const double T_stop = opts[3];
    const double bg[3] = {opts[4], opts[5], opts[6]};
    const int K = (sh_degree + 1) * (sh_degree + 1);
    const double delta = (t_far - t_near) / n_samples;
    gauss64 *G = (gauss64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(gauss64));
    double *col = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    int *use = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    for (int g = 0; g < n; ++g) prep64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g], &G[g]);
    for (int v = 0; v < n_views; ++v) {
        cam64 cam;
        cam_setup(cam_f + 16 * v, cam_wh + 2 * v, &cam);
        double raw[3];
        int nu = 0;
        for (int g = 0; g < n; ++g) {
            if (depth_bits[(int64_t)v * n + g] == 0xFFFFFFFFu) continue;
            colour64(sh + (size_t)g * K * 3, sh_degree, &G[g], cam.o, col + 3 * g, raw, opts[8]);
            use[nu++] = g;
        }
        const int W = cam.W, H = cam.H;
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t pix = 0; pix < (int64_t)W * H; ++pix) {
            const int64_t gp = pix_base[v] + pix;
            if (pix_mask && !pix_mask[gp]) continue;
            const int x = (int)(pix % W), y = (int)(pix / W);
            double d[3];
            pixel_dir(&cam, x, y, d);
            double T = 1.0, C[3] = {0, 0, 0};
            for (int k = 0; k < n_samples; ++k) {
                const double t = t_near + (k + 0.5) * delta;
                double xk[3], sig = 0, cs[3] = {0, 0, 0};
                for (int a = 0; a < 3; ++a) xk[a] = cam.o[a] + t * d[a];
                for (int u = 0; u < nu; ++u) {
                    const gauss64 *Gg = &G[use[u]];
                    double e[3], m2 = 0;
                    for (int a = 0; a < 3; ++a) e[a] = xk[a] - Gg->mu[a];
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) m2 += e[a] * Gg->P[3 * a + b] * e[b];
                    const double val = Gg->kap * exp(-0.5 * m2);
                    sig += val;
                    for (int ch = 0; ch < 3; ++ch) cs[ch] += col[3 * use[u] + ch] * val;
                }
                if (sig > 0) {
                    const double w = -expm1(-sig * delta) / sig;   /* (1 - e^{-sigma delta}) / sigma */
                    for (int ch = 0; ch < 3; ++ch) C[ch] += T * w * cs[ch];
                    T *= exp(-sig * delta);
                }
                if (T < T_stop) break;
            }
            for (int ch = 0; ch < 3; ++ch) rgb[3 * gp + ch] = C[ch] + T * bg[ch];
            T_final[gp] = T;
        }
    }
    free(G);
    free(col);
    free(use);
}

/* ================================ voxel density ================================ */
/* Density on a grid (for volumetric metrics): sigma(x) = sum_g kappa_g G_g(x) (Eq. 3-4) at the
 * voxel centres x = origin + (i + 1/2, j + 1/2, k + 1/2) * voxel.  Each Gaussian is truncated
 * to the voxel box of its ellipsoid (x - mu)' P (x - mu) <= k^2 with k^2 = 2 ln 2 e, where
 * kappa / sigma_cut = m 2^e (sigma >= sigma_cut needs m^2 <= 2 ln(kappa / sigma_cut)): the
 * box is computed in FP32 with a fixed operation order so that both sides agree bit for bit. */
int64_t orc_voxel_boxes(int n, const float *mu, const float *scale, const float *quat, const float *kappa,
                        const float *origin, const float *voxel, const int32_t *dims, float sigma_cut,
                        int32_t *box /* [n][6] x0 y0 z0 x1 y1 z1, -1 when empty */)
{
    int64_t total = 0;
    for (int g = 0; g < n; ++g) {
        int32_t *b = box + 6 * (int64_t)g;
        for (int k = 0; k < 6; ++k) b[k] = -1;
        float Sig[9], smax;
        if (!cov_fp32(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g], Sig, &smax)) continue;
        const float xr = kappa[g] / sigma_cut;
        if (!(xr > 1.0f)) continue;
        int e;
        if (xr > FLT_MAX)
            e = 128;
        else
            (void)frexpf(xr, &e);
        const float k2 = (float)e * 1.3862944f;
        int lo[3], hi[3], ok = 1;
        for (int a = 0; a < 3; ++a) {
            const float h = sqrtf(k2 * Sig[4 * a]);
            const float c = mu[3 * g + a] - origin[a];
            const float flo = (c - h) / voxel[a] - 0.5f, fhi = (c + h) / voxel[a] - 0.5f;
            pixel_span(flo, fhi, dims[a], &lo[a], &hi[a]);
            if (lo[a] > hi[a]) ok = 0;
        }
        if (!ok) continue;
        for (int a = 0; a < 3; ++a) {
            b[a] = lo[a];
            b[3 + a] = hi[a];
        }
        total += (int64_t)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
    }
    return total;
}

/* sigma at the voxels (masked ones only when mask is given), summing every Gaussian whose box
 * contains the voxel (or, brute force, every valid Gaussian). */
void orc_voxel_density(int n, const double *mu, const double *scale, const double *quat, const double *kappa,
                       const int32_t *box, int brute, const float *origin, const float *voxel,
                       const int32_t *dims, const int32_t *mask, double *out)
{
    gauss64 *G = (gauss64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(gauss64));
    char *ok = (char *)malloc((size_t)(n > 0 ? n : 1));
    for (int g = 0; g < n; ++g) {
        ok[g] = (char)valid64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g]);
        if (ok[g]) prep64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g], &G[g]);
    }
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t v = 0; v < nx * ny * nz; ++v) {
        if (mask && !mask[v]) continue;
        const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / (nx * ny));
        const double x[3] = {(double)origin[0] + (i + 0.5) * (double)voxel[0],
                             (double)origin[1] + (j + 0.5) * (double)voxel[1],
                             (double)origin[2] + (k + 0.5) * (double)voxel[2]};
        double sum = 0;
        for (int g = 0; g < n; ++g) {
            if (!ok[g]) continue;
            if (!brute) {
                const int32_t *b = box + 6 * (int64_t)g;
                if (b[0] < 0 || i < b[0] || i > b[3] || j < b[1] || j > b[4] || k < b[2] || k > b[5]) continue;
            }
            double d[3], m2 = 0;
            for (int a = 0; a < 3; ++a) d[a] = x[a] - G[g].mu[a];
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) m2 += d[a] * G[g].P[3 * a + c] * d[c];
            sum += G[g].kap * exp(-0.5 * m2);
        }
        out[v] = sum;
    }
    free(G);
    free(ok);
}

/* ================================== cone beam ================================== */
/* Cone-beam tomography (Eq. 21 with diverging rays): a point source at the camera centre and
 * a flat detector in the camera's image plane, so each detector pixel's ray is a pixel ray of
 * the pinhole camera.  proj = exp(-sum_g tau_g) over the Gaussians of the pixel's tile list
 * whose footprint rectangle contains the pixel (or, brute force, over every valid Gaussian). */
void orc_cone(int n, const double *mu, const double *scale, const double *quat, const double *kappa,
              int n_views, const float *cam_f, const int32_t *cam_wh, int tile_w, int tile_h,
              const int64_t *tile_start, const int32_t *sorted_g, const int32_t *view_tile_base,
              const int32_t *prect, int brute, const int64_t *pix_base, const int32_t *pix_mask,
              double *line_sum, double *proj)
{
    gauss64 *G = (gauss64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(gauss64));
    char *ok = (char *)malloc((size_t)(n > 0 ? n : 1));
    for (int g = 0; g < n; ++g) {
        ok[g] = (char)valid64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g]);
        if (ok[g]) prep64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g], &G[g]);
    }
    for (int v = 0; v < n_views; ++v) {
        cam64 cam;
        cam_setup(cam_f + 16 * v, cam_wh + 2 * v, &cam);
        const int W = cam.W, H = cam.H;
        const int tiles_x = (W + tile_w - 1) / tile_w;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t pix = 0; pix < (int64_t)W * H; ++pix) {
            const int64_t gp = pix_base[v] + pix;
            if (pix_mask && !pix_mask[gp]) continue;
            const int x = (int)(pix % W), y = (int)(pix / W);
            double d[3];
            pixel_dir(&cam, x, y, d);
            double sum = 0;
            if (brute) {
                for (int g = 0; g < n; ++g) {
                    if (!ok[g]) continue;
                    double a, b, c, p[3];
                    sum += tau64(&G[g], cam.o, d, &a, &b, &c, p);
                }
            } else {
                const int64_t tile = view_tile_base[v] + (int64_t)(y / tile_h) * tiles_x + x / tile_w;
                for (int64_t k = tile_start[tile]; k < tile_start[tile + 1]; ++k) {
                    const int64_t g = sorted_g[k];
                    if (outside(prect, (int64_t)v * n + g, x, y)) continue;
                    double a, b, c, p[3];
                    sum += tau64(&G[g], cam.o, d, &a, &b, &c, p);
                }
            }
            line_sum[gp] = sum;
            proj[gp] = exp(-sum);
        }
    }
    free(G);
    free(ok);
}

/* Gradient of sum(dL_dproj * proj) for the cone beam: dL/dtau_g = -proj dL/dproj at every pair. */
void orc_cone_grad(int n, const double *mu, const double *scale, const double *quat, const double *kappa,
                   int n_views, const float *cam_f, const int32_t *cam_wh, int tile_w, int tile_h,
                   const int64_t *tile_start, const int32_t *sorted_g, const int32_t *view_tile_base,
                   const int32_t *prect, const int64_t *pix_base, const double *dL_dproj,
                   const int32_t *pix_mask, double *dmu, double *dscale, double *dquat, double *dkappa)
{
    gauss64 *G = (gauss64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(gauss64));
    double *acc = (double *)calloc((size_t)(n > 0 ? n : 1) * ACC_N, sizeof(double));
    for (int g = 0; g < n; ++g)
        if (valid64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g]))
            prep64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g], &G[g]);
    for (int v = 0; v < n_views; ++v) {
        cam64 cam;
        cam_setup(cam_f + 16 * v, cam_wh + 2 * v, &cam);
        memset(acc, 0, (size_t)(n > 0 ? n : 1) * ACC_N * sizeof(double));
        const int W = cam.W, H = cam.H;
        const int tiles_x = (W + tile_w - 1) / tile_w;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t pix = 0; pix < (int64_t)W * H; ++pix) {
            const int64_t gp = pix_base[v] + pix;
            if (pix_mask && !pix_mask[gp]) continue;
            const int x = (int)(pix % W), y = (int)(pix / W);
            double d[3];
            pixel_dir(&cam, x, y, d);
            const int64_t tile = view_tile_base[v] + (int64_t)(y / tile_h) * tiles_x + x / tile_w;
            double sum = 0;
            for (int64_t k = tile_start[tile]; k < tile_start[tile + 1]; ++k) {
                const int64_t g = sorted_g[k];
                if (outside(prect, (int64_t)v * n + g, x, y)) continue;
                double a, b, c, p[3];
                sum += tau64(&G[g], cam.o, d, &a, &b, &c, p);
            }
            const double dLdtau = -exp(-sum) * dL_dproj[gp];
            for (int64_t k = tile_start[tile]; k < tile_start[tile + 1]; ++k) {
                const int64_t g = sorted_g[k];
                if (outside(prect, (int64_t)v * n + g, x, y)) continue;
                double a, b, c, p[3];
                const double tau = tau64(&G[g], cam.o, d, &a, &b, &c, p);
                acc_tau(&acc[ACC_N * g], &G[g], dLdtau, tau, a, b, d, p);
            }
        }
        for (int g = 0; g < n; ++g) {
            double *A = &acc[ACC_N * g];
            int any = 0;
            for (int k = 0; k < ACC_N; ++k) any |= (A[k] != 0.0);
            if (!any) continue;
            chain_P(&G[g], A, dscale + 3 * g, dquat + 4 * g);
            for (int k = 0; k < 3; ++k) dmu[3 * g + k] += A[9 + k];
            dkappa[g] += A[12];
        }
    }
    free(G);
    free(acc);
}

/* ================================== tomography ================================== */

void orc_tomo(int n, const double *mu, const double *scale, const double *quat, const double *kappa,
              int n_angles, const float *angles, int det_w, int det_h, float pitch_u,
              float pitch_v, float u0, float v0, int tile_w, int tile_h,
              const int64_t *tile_start, const int32_t *sorted_g, const int32_t *prect, int brute,
              const int32_t *pix_mask, double *line_sum, double *proj)
{
    gauss64 *G = (gauss64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(gauss64));
    char *ok = (char *)malloc((size_t)(n > 0 ? n : 1));
    for (int g = 0; g < n; ++g) {
        ok[g] = (char)valid64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g]);
        if (ok[g]) prep64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g], &G[g]);
    }
    const int tiles_x = (det_w + tile_w - 1) / tile_w, tiles_y = (det_h + tile_h - 1) / tile_h;
    for (int an = 0; an < n_angles; ++an) {
        double th = angles[an];
        double d[3] = {cos(th), sin(th), 0.0};
        double eu[3] = {-sin(th), cos(th), 0.0};
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t pix = 0; pix < (int64_t)det_w * det_h; ++pix) {
            int64_t gp = (int64_t)an * det_w * det_h + pix;
            if (pix_mask && !pix_mask[gp]) continue;
            int i = (int)(pix % det_w), j = (int)(pix / det_w);
            double u = u0 + (i + 0.5) * (double)pitch_u, vv = v0 + (j + 0.5) * (double)pitch_v;
            double o[3] = {u * eu[0], u * eu[1], vv};
            double sum = 0;
            if (brute) {
                for (int g = 0; g < n; ++g) {
                    if (!ok[g]) continue;
                    double a, b, c, p[3];
                    sum += tau64(&G[g], o, d, &a, &b, &c, p);
                }
            } else {
                int64_t tile = (int64_t)an * tiles_x * tiles_y + (int64_t)(j / tile_h) * tiles_x + i / tile_w;
                for (int64_t k = tile_start[tile]; k < tile_start[tile + 1]; ++k) {
                    if (outside(prect, (int64_t)an * n + sorted_g[k], i, j)) continue;
                    double a, b, c, p[3];
                    sum += tau64(&G[sorted_g[k]], o, d, &a, &b, &c, p);
                }
            }
            line_sum[gp] = sum;
            proj[gp] = exp(-sum);
        }
    }
    free(G);
    free(ok);
}

void orc_tomo_grad(int n, const double *mu, const double *scale, const double *quat,
                   const double *kappa, int n_angles, const float *angles, int det_w, int det_h,
                   float pitch_u, float pitch_v, float u0, float v0, int tile_w, int tile_h,
                   const int64_t *tile_start, const int32_t *sorted_g, const int32_t *prect,
                   const double *dL_dproj, const int32_t *pix_mask, double *dmu, double *dscale,
                   double *dquat, double *dkappa)
{
    gauss64 *G = (gauss64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(gauss64));
    double *acc = (double *)calloc((size_t)(n > 0 ? n : 1) * ACC_N, sizeof(double));
    for (int g = 0; g < n; ++g)
        if (valid64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g]))
            prep64(mu + 3 * g, scale + 3 * g, quat + 4 * g, kappa[g], &G[g]);
    const int tiles_x = (det_w + tile_w - 1) / tile_w, tiles_y = (det_h + tile_h - 1) / tile_h;
    for (int an = 0; an < n_angles; ++an) {
        double th = angles[an];
        double d[3] = {cos(th), sin(th), 0.0};
        double eu[3] = {-sin(th), cos(th), 0.0};
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t pix = 0; pix < (int64_t)det_w * det_h; ++pix) {
            int64_t gp = (int64_t)an * det_w * det_h + pix;
            if (pix_mask && !pix_mask[gp]) continue;
            int i = (int)(pix % det_w), j = (int)(pix / det_w);
            double u = u0 + (i + 0.5) * (double)pitch_u, vv = v0 + (j + 0.5) * (double)pitch_v;
            double o[3] = {u * eu[0], u * eu[1], vv};
            int64_t tile = (int64_t)an * tiles_x * tiles_y + (int64_t)(j / tile_h) * tiles_x + i / tile_w;
            double sum = 0;
            for (int64_t k = tile_start[tile]; k < tile_start[tile + 1]; ++k) {
                if (outside(prect, (int64_t)an * n + sorted_g[k], i, j)) continue;
                double a, b, c, p[3];
                sum += tau64(&G[sorted_g[k]], o, d, &a, &b, &c, p);
            }
            /* proj = exp(-sum)  =>  dL/dtau_i = -proj dL/dproj for every Gaussian on the ray */
            double dLdtau = -exp(-sum) * dL_dproj[gp];
            for (int64_t k = tile_start[tile]; k < tile_start[tile + 1]; ++k) {
                int64_t g = sorted_g[k];
                if (outside(prect, (int64_t)an * n + g, i, j)) continue;
                double a, b, c, p[3];
                double tau = tau64(&G[g], o, d, &a, &b, &c, p);
                acc_tau(&acc[ACC_N * g], &G[g], dLdtau, tau, a, b, d, p);
            }
        }
    }
    for (int g = 0; g < n; ++g) {
        double *A = &acc[ACC_N * g];
        int any = 0;
        for (int k = 0; k < 13; ++k) any |= (A[k] != 0.0);
        if (!any) continue;
        chain_P(&G[g], A, dscale + 3 * g, dquat + 4 * g);
        for (int k = 0; k < 3; ++k) dmu[3 * g + k] += A[9 + k];
        dkappa[g] += A[12];
    }
    free(G);
    free(acc);
}
