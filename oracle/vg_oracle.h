/* FP64 CPU oracle for the volumetrically consistent Gaussian rasterizer
 * (arXiv 2412.03378).  TEST INFRASTRUCTURE ONLY: this library exists to check the
 * CUDA path.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load it; the product path never does.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Camera records are float[16] = { R[9] (row-major, world->camera), t[3], fx, fy, cx, cy }
 * with integer sizes in cam_wh[2] = { width, height }.  A world point x maps to camera
 * coordinates R x + t (OpenCV axes: x right, y down, z forward).
 *
 * The FP64 paths (render, gradient, tomography, tau) take double parameters so that
 * finite differences can perturb them; the key functions take the FP32 values the GPU sees.
 *
 * Options are double[11] = { alpha_min, tau_cut, tau_max, T_stop, bg_r, bg_g, bg_b, z_near,
 * softplus_beta, splat, splat_dilation }; softplus_beta > 0 replaces the colour clamp max(x, 0)
 * by the softplus (1/beta) ln(1 + e^(beta x)) (Supp. D).  splat != 0 selects the 3DGS comparison
 * mode (Eq. 5-7): the density array holds the peak opacity o, alpha = min(o G'(p), alpha_max)
 * with G' the projected 2D Gaussian of covariance J W Sigma W^T J^T + splat_dilation I,
 * alpha_max = min(1 - exp(-tau_max), 1 - 2^-24), pairs with alpha < alpha_min skipped, and the
 * footprint from orc_keys_splat (alpha_cut = tau_cut).  The density reparameterisation of Eq. 20 is applied
 * by the Python wrapper (kappa from theta and the scales) before these functions are called.
 */
#ifndef VG_ORACLE_H
#define VG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Key function (depth key, tile rectangle and pixel footprint rectangle) in FP32 with a
 * fixed operation order.  Tiled evaluation restricts each Gaussian to the pixels of its
 * footprint rectangle (prect, inclusive); brute-force evaluation does not. */
int64_t orc_keys(int n, const float *mu, const float *scale, const float *quat, const float *kappa,
                 int n_views, const float *cam_f, const int32_t *cam_wh, int tile_w, int tile_h,
                 float z_near, float tau_cut, uint32_t *depth_bits, int32_t *rect, int32_t *prect);
int64_t orc_tomo_keys(int n, const float *mu, const float *scale, const float *quat,
                      const float *kappa, int n_angles, const float *angles, int det_w, int det_h,
                      float pitch_u, float pitch_v, float u0, float v0, int tile_w, int tile_h,
                      float tau_cut, int32_t *rect, int32_t *prect);
/* Splat-mode key function: same depth key; footprint = pixel box of the 2D Gaussian's
 * ellipse outside which alpha < alpha_cut. */
int64_t orc_keys_splat(int n, const float *mu, const float *scale, const float *quat, const float *opac,
                       int n_views, const float *cam_f, const int32_t *cam_wh, int tile_w, int tile_h,
                       float z_near, float alpha_cut, float dilation, uint32_t *depth_bits, int32_t *rect,
                       int32_t *prect);
/* The projected 2D Gaussian of one Gaussian (FP64): out = { mu'_x, mu'_y, S'_xx, S'_xy, S'_yy, ok }. */
void orc_splat2d(const double *mu, const double *scale, const double *quat, const float *cam_f,
                 const int32_t *cam_wh, double dil, double *out);
/* Stable sort of (tile, depth, Gaussian) instances; fills tile_start[n_tiles+1], sorted_g. */
int64_t orc_bin(int n, int n_views, const uint32_t *depth_bits, const int32_t *rect,
                const int32_t *view_tiles_x, const int32_t *view_tile_base, int64_t n_tiles_total,
                int64_t capacity, int64_t *tile_start, int32_t *sorted_g);

void orc_sh_basis(int degree, const double *dir, double *out);
void orc_tau(const double *mu, const double *scale, const double *quat, double kappa,
             const double *o, const double *d, double *out /* tau, a, b, c, gamma, beta, gmax */);

void orc_render(int n, const double *mu, const double *scale, const double *quat,
                const double *kappa, const double *sh, int sh_degree, int n_views, const float *cam_f,
                const int32_t *cam_wh, int tile_w, int tile_h, const double *opts,
                const int64_t *tile_start, const int32_t *sorted_g, const int32_t *view_tile_base,
                int brute, const uint32_t *depth_bits, const int32_t *prect,
                const int64_t *pix_base, const int32_t *pix_mask, double *rgb, double *T_final,
                int32_t *n_blend, int64_t *last_pos, double *diag);
/* Optional per-pixel outputs of orc_render (each may be NULL): n_blend = blended pairs;
 * last_pos = position + 1, within the pixel's tile list, of the last blended pair (0 when none;
 * the position in the depth order in brute-force mode); diag[4] = { S = sum of the blended
 * tau, and the relative distance of the closest skip (alpha_min), clamp (tau_max) and
 * early-stop (T_stop) decision to its threshold, INFINITY when the pixel met none }. */

void orc_render_grad(int n, const double *mu, const double *scale, const double *quat,
                     const double *kappa, const double *sh, int sh_degree, int n_views,
                     const float *cam_f, const int32_t *cam_wh, int tile_w, int tile_h,
                     const double *opts, const int64_t *tile_start, const int32_t *sorted_g,
                     const int32_t *view_tile_base, const int32_t *prect, const int64_t *pix_base,
                     const double *dL_drgb, const double *dL_dT, const int32_t *pix_mask,
                     double *dmu, double *dscale, double *dquat, double *dkappa, double *dsh);

/* Ray-marching reference (Supp. A): NeRF quadrature of Eq. 1 with sigma = sum kappa G and the
 * density-weighted colour, midpoint samples on [t_near, t_far]; every Gaussian with a valid depth key. */
void orc_ray_march(int n, const double *mu, const double *scale, const double *quat, const double *kappa,
                   const double *sh, int sh_degree, int n_views, const float *cam_f, const int32_t *cam_wh,
                   const double *opts, const uint32_t *depth_bits, double t_near, double t_far, int n_samples,
                   const int64_t *pix_base, const int32_t *pix_mask, double *rgb, double *T_final);

/* Voxel density: truncation boxes (FP32 key-function style, bit-exact) and sigma at voxel centres. */
int64_t orc_voxel_boxes(int n, const float *mu, const float *scale, const float *quat, const float *kappa,
                        const float *origin, const float *voxel, const int32_t *dims, float sigma_cut,
                        int32_t *box);
void orc_voxel_density(int n, const double *mu, const double *scale, const double *quat, const double *kappa,
                       const int32_t *box, int brute, const float *origin, const float *voxel,
                       const int32_t *dims, const int32_t *mask, double *out);

/* Cone-beam projection: the source at each camera's centre, the detector its image plane. */
void orc_cone(int n, const double *mu, const double *scale, const double *quat, const double *kappa,
              int n_views, const float *cam_f, const int32_t *cam_wh, int tile_w, int tile_h,
              const int64_t *tile_start, const int32_t *sorted_g, const int32_t *view_tile_base,
              const int32_t *prect, int brute, const int64_t *pix_base, const int32_t *pix_mask,
              double *line_sum, double *proj);
void orc_cone_grad(int n, const double *mu, const double *scale, const double *quat, const double *kappa,
                   int n_views, const float *cam_f, const int32_t *cam_wh, int tile_w, int tile_h,
                   const int64_t *tile_start, const int32_t *sorted_g, const int32_t *view_tile_base,
                   const int32_t *prect, const int64_t *pix_base, const double *dL_dproj,
                   const int32_t *pix_mask, double *dmu, double *dscale, double *dquat, double *dkappa);

void orc_tomo(int n, const double *mu, const double *scale, const double *quat, const double *kappa,
              int n_angles, const float *angles, int det_w, int det_h, float pitch_u,
              float pitch_v, float u0, float v0, int tile_w, int tile_h,
              const int64_t *tile_start, const int32_t *sorted_g, const int32_t *prect, int brute,
              const int32_t *pix_mask, double *line_sum, double *proj);

void orc_tomo_grad(int n, const double *mu, const double *scale, const double *quat,
                   const double *kappa, int n_angles, const float *angles, int det_w, int det_h,
                   float pitch_u, float pitch_v, float u0, float v0, int tile_w, int tile_h,
                   const int64_t *tile_start, const int32_t *sorted_g, const int32_t *prect,
                   const double *dL_dproj, const int32_t *pix_mask, double *dmu, double *dscale, double *dquat, double *dkappa);

int orc_num_threads(void);
int orc_set_threads(int n);   /* threads of later parallel regions (n < 1: all cores) */

#ifdef __cplusplus
}
#endif
#endif
