// Internal declarations of the CUDA library (kernels, launchers, device helpers).
// Nothing here is part of the C ABI; see include/vg.h for that.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "vg.h"

namespace vg {

constexpr int kTile = 16;                 // the default tile (16 x 16 pixels); tomography's tiles
constexpr int kTilePix = kTile * kTile;
constexpr int kMaxTilePix = 512;          // the largest tile the blend kernels take (32 x 16)
constexpr int kRecF4 = 6;                 // blend record: 6 x float4 = 96 bytes
constexpr int kGradN = 16;                // per-item gradient accumulator (moments, dln kappa, colour)
constexpr int kTomoRecF4 = 2;             // tomography record: 2 x float4

// Per-view constants, device side.
struct ViewInfo {
    float R[9], t[3];
    float fx, fy, cx, cy;
    float of[3];          // camera centre o = -R^T t, FP32
    double od[3];         // camera centre, FP64
    int W, H, tiles_x, tiles_y;
    int tile_base;        // first global tile id of this view
    int tw, th;           // tile width and height in pixels (16 x 16, 32 x 16 or 16 x 8)
    int pad;
    long long pix_base;   // first pixel of this view in the concatenated image
};

struct GaussIn {
    const void *mu, *scale, *quat, *kappa, *sh;
    int rec_dtype, sh_dtype, n, sh_degree;
    int mu_f32;            // mu is float32 whatever rec_dtype says
    int density_theta;     // the density array holds Eq. 20's theta
    float softplus_beta;   // colour activation: 0 = clamp at 0, > 0 = softplus(beta)
    int splat;             // 3DGS comparison mode: the density array holds the peak opacity
    float splat_dil;       // its 2D covariance dilation (pixels^2)
};

struct BlendParams {
    float tau_skip;       // skip contributions with tau < tau_skip (alpha < alpha_min)
    float tau_max;
    float T_stop;
    float bg[3];
    int pixel_test;       // test every pixel against the Gaussian's footprint rectangle
                          // (needed when tau_skip < tau_cut; otherwise implied by the skip)
    int splat;            // 3DGS comparison mode: alpha = min(o G', alpha_max), skipped below
    float alpha_min;      // alpha_min, instead of the tau bounds above
    float alpha_max;
    int chunk_fwd;        // records staged per barrier: 64 or 128
    int chunk_bwd;
    int tile_px;          // pixels per tile (the blend kernels' block is tile_px / P threads)
};

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Programmatic dependent launch: every kernel of the library is launched with programmatic
// stream serialisation, so the next kernel's CTAs are scheduled while the previous kernel's
// last wave drains.  pdl_entry() must run first in every kernel: it blocks until the previous
// grid has completed and its writes are visible (so the usual stream order holds for all
// memory accesses after it), then lets the next grid start launching.  VG_PDL=0 at compile
// time restores plain stream-ordered launches.
#ifndef VG_PDL
#define VG_PDL 1
#endif
__device__ __forceinline__ void pdl_entry() {
#if VG_PDL
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = VG_PDL ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename T> __device__ __forceinline__ float ld_f(const T *p, long long i);
template <> __device__ __forceinline__ float ld_f<float>(const float *p, long long i) { return __ldg(p + i); }
template <> __device__ __forceinline__ float ld_f<__nv_bfloat16>(const __nv_bfloat16 *p, long long i) {
    return __bfloat162float(p[i]);
}
template <> __device__ __forceinline__ float ld_f<__half>(const __half *p, long long i) { return __half2float(p[i]); }

// ------------------------------------------------------------------ launchers
// All launchers return cudaGetLastError() after their launches and add the number of
// kernels they launched to *launches.
cudaError_t launch_preprocess(const GaussIn &g, const ViewInfo *views_d, int n_views, float z_near,
                              float tau_cut, float4 *rec, uint32_t *depth, uint32_t *count, short4 *rect,
                              short4 *prect, unsigned long long *n_visible, cudaStream_t st, long long *launches);

cudaError_t launch_tomo_preprocess(const GaussIn &g, const float *cs_d /* [A][2] cos, sin */, int n_angles,
                                   int det_w, int det_h, float pitch_u, float pitch_v, float u0, float v0,
                                   float tau_cut, float4 *rec, uint32_t *count, short4 *rect, short4 *prect,
                                   cudaStream_t st, long long *launches);

// Error bits latched in the workspace's device flag word.
constexpr uint32_t kDevErrTimeout = 1u, kDevErrCapacity = 2u;

// Single-pass exclusive scan of count[perm[i]] (perm may be NULL) into out[0..n); out[n] and
// *total64 receive the total.  tmp must hold scan_tmp_words(n) uint32; *err gets
// kDevErrTimeout if a look-back wait timed out and kDevErrCapacity if the total exceeds cap.
size_t scan_tmp_words(long long n);
cudaError_t launch_scan_gather(const uint32_t *count, const uint32_t *perm, uint32_t *out, long long n,
                               uint32_t *tmp, unsigned long long *total64, unsigned long long cap, uint32_t *err,
                               cudaStream_t st, long long *launches);

// Stable LSD radix sort of (key, value) pairs over key bits [0, bits) (n < 2^30), one kernel
// per 8-bit digit.  Reads keys_in / vals_in (vals_in NULL: values are the input positions);
// pass p writes (ka, va) for even p and (kb, vb) for odd p; the result pointers are returned
// in keys_out / vals_out.  scratch must hold radix_scratch_words(n, bits) uint32.  With n_dev
// non-NULL the kernels sort min(n, *n_dev) keys (a count known on the device only; n is then
// the capacity the launch covers).
size_t radix_scratch_words(long long n, int bits);
cudaError_t launch_radix_sort(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *ka, uint32_t *va,
                              uint32_t *kb, uint32_t *vb, long long n, const unsigned long long *n_dev, int bits,
                              uint32_t *scratch, uint32_t *err, uint32_t **keys_out, uint32_t **vals_out,
                              cudaStream_t st, long long *launches);

// A look-back over a status array (4 zero words, device) whose predecessor never publishes, with a
// spin limit of spin_limit polls; the wait gives up and sets kDevErrTimeout in *err (test path).
cudaError_t launch_lookback_selftest(void *status, int which, int spin_limit, uint32_t *err, unsigned long long *out,
                                     cudaStream_t st, long long *launches);

// Pipe-peak microbenchmark (peaks.cu): pipe 0 = FP32 FMA, 1 = ex2 (MUFU); *ops receives the
// instructions (per lane) one launch executes.
cudaError_t launch_pipe_peak(int pipe, int iters, double *ops, cudaStream_t st);

// Duplicate items into (tile key, item) instances, in the order given by perm (NULL = item
// order).  offsets[i] is the first instance slot of the i-th item in that order.
cudaError_t launch_duplicate(const uint32_t *perm, const uint32_t *offsets, const short4 *rect,
                             const ViewInfo *views, long long n_items, int n_per_view, uint32_t *inst_key,
                             uint32_t *inst_val, long long capacity, cudaStream_t st, long long *launches);

cudaError_t launch_ranges(const uint32_t *sorted_key, long long n_inst, const unsigned long long *n_dev, uint2 *ranges,
                          long long n_tiles, cudaStream_t st, long long *launches);

// The L2 image loss fused into the forward's epilogue (target NULL: none): *loss +=
// scale sum (rgb - target)^2 and grad = 2 scale (rgb - target), per pixel where rgb is written.
struct L2Fused {
    const float *target;
    float *grad;
    float *loss;
    float scale;
};

cudaError_t launch_render_fwd(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                              const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                              const BlendParams &bp, int ppt, float *rgb, float *T_user, float *T_ws, float *S_out,
                              uint32_t *nlast_out, uint32_t *tile_replay, unsigned long long *pair_count,
                              const L2Fused &l2, cudaStream_t st, long long *launches);

cudaError_t launch_render_bwd(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                              const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                              const BlendParams &bp, int ppt, const float *T_fin, const float *S_fin,
                              const uint32_t *nlast, const float *dL_drgb, const float *dL_dT, float *grad_acc,
                              unsigned long long *pair_count, uint32_t *err, cudaStream_t st, long long *launches);

// Longest-first tile order: order[] lists the tiles by descending length (bucketed): the instance
// count from ranges, or (ranges NULL) the lengths in lens.
cudaError_t launch_tile_order(const uint2 *ranges, const uint32_t *lens, long long n_tiles, uint32_t *order,
                              cudaStream_t st, long long *launches);

// Voxel density query (voxel.cu): grid origin, voxel size, voxel and brick (8^3) counts.
struct VoxelGrid {
    float ox, oy, oz, vx, vy, vz;
    int nx, ny, nz, bx, by, bz;
};
cudaError_t launch_voxel_pre(const GaussIn &g, const VoxelGrid &grid, float sigma_cut, float4 *rec, short4 *box,
                             uint32_t *count, cudaStream_t st, long long *launches);
cudaError_t launch_voxel_dup(const uint32_t *offsets, const short4 *box, const VoxelGrid &grid, long long n,
                             uint32_t *inst_key, uint32_t *inst_val, long long capacity, cudaStream_t st,
                             long long *launches);
cudaError_t launch_voxel_eval(const uint2 *ranges, const uint32_t *sorted, const float4 *rec, const short4 *box,
                              const VoxelGrid &grid, float *out, cudaStream_t st, long long *launches);

// Ray-marching reference (march.cu): one CTA of tile_px threads per tile (one pixel each); E
// receives (o'.A0, o'.A1, o'.A2) per item (scratch);
// rgb / T_out / err (max over channels of |rgb - raster|) are each optional.
cudaError_t launch_ray_march(const GaussIn &g, const ViewInfo *views_d, const int *tile_view, long long n_tiles,
                             int tile_px,
                             long long n_items, const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec,
                             const uint32_t *count, const short4 *prect, float4 *E, float t_near, float t_far,
                             int n_samples, float T_stop, const float bg[3], const float *raster, float *rgb,
                             float *T_out, float *err, cudaStream_t st, long long *launches);

// The chain reads grad_acc and leaves every item it reads zero again (an all-zero row is left
// as it is), so a following backward needs no clearing pass.
cudaError_t launch_chain(const GaussIn &g, const ViewInfo *views_d, int n_views, float *grad_acc, int zero,
                         float *dmu, float *dscale, float *dquat, float *dkappa, float *dsh, cudaStream_t st,
                         long long *launches);

cudaError_t launch_tomo_fwd(const uint2 *ranges, long long n_tiles, int tiles_x, int tiles_per_view, int det_w,
                            int det_h, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                            float *proj, cudaStream_t st, long long *launches);

cudaError_t launch_tomo_bwd(const uint2 *ranges, long long n_tiles, int tiles_x, int tiles_per_view, int det_w,
                            int det_h, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                            const float *proj, const float *dL_dproj, float *grad_acc, cudaStream_t st,
                            long long *launches);

cudaError_t launch_tomo_chain(const GaussIn &g, const float *cs_d, int n_angles, long long item0, long long n_items,
                              float pitch_u, float pitch_v, float u0, float v0, const float *grad_acc, float *dmu,
                              float *dscale, float *dquat, float *dkappa, cudaStream_t st, long long *launches);

cudaError_t launch_l2_loss(const float *x, const float *y, long long n, float scale, float *loss, float *grad,
                           cudaStream_t st, long long *launches);
// The same without zeroing *loss first (accumulates across calls).
cudaError_t launch_l2_loss_acc(const float *x, const float *y, long long n, float scale, float *loss, float *grad,
                               cudaStream_t st, long long *launches);

}  // namespace vg
