/* vg.h — C ABI of the volumetric Gaussian rasterizer (arXiv 2412.03378, "Volumetrically
 * Consistent 3D Gaussian Rasterization") for NVIDIA GB300 (sm_103a).
 *
 * The library renders a mixture of 3D Gaussians sigma(x) = sum_i kappa_i G_i(x) (Sec. 3.2,
 * Eq. 3-4) by front-to-back alpha blending (Sec. 4.1, Eq. 14) of per-Gaussian opacities
 * that are the exact line integral of each Gaussian along the pixel ray (Sec. 4.2, Eq. 19):
 *
 *     tau_i = kappa_i sqrt(2 pi / a) exp(-(c - b^2 / a) / 2),   alpha_i = 1 - exp(-tau_i),
 *     a = d' P d,  b = d' P (o - mu),  c = (o - mu)' P (o - mu),  P = Sigma^-1,
 *
 * with o the camera centre and d the unit direction through the pixel centre.  A tomography
 * mode (Sec. 6.2, Eq. 21) sums the same line integrals along parallel-beam rays and returns
 * exp(-sum).  All work runs in this library's CUDA kernels; the calls only marshal arguments.
 *
 * Conventions shared by every call
 *  - Pointers named in vg_gaussians, image buffers and gradient buffers are DEVICE pointers
 *    owned by the caller.  Camera, beam-angle and option structs are HOST memory, read
 *    during the call only.
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy
 *    default stream) unless its comment says it synchronises.
 *  - Every call returns a vg_status and never aborts.  On failure vg_last_error() gives a
 *    one-line message.  Device-side failures are latched and reported by the next call.
 *  - A workspace is not thread-safe; separate workspaces are independent.
 *  - Gradient outputs are ACCUMULATED (+=); the caller zeroes them first.
 */
#ifndef VG_H
#define VG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VG_OK = 0,
    VG_ERR_INVALID_ARG = 1,   /* a null pointer, a negative size, an unsupported layout       */
    VG_ERR_CUDA = 2,          /* a CUDA runtime call failed                                   */
    VG_ERR_OOM = 3,           /* device memory for the workspace could not be allocated       */
    VG_ERR_CAPACITY = 4,      /* fixed-capacity mode: more tile instances than reserved       */
    VG_ERR_TIMEOUT = 5,       /* a bounded device wait gave up                                */
    VG_ERR_UNSUPPORTED = 6,   /* a valid request the library does not implement               */
    VG_ERR_STATE = 7          /* calls out of order (e.g. render before bin_sort)             */
} vg_status;

typedef enum { VG_F32 = 0, VG_BF16 = 1, VG_F16 = 2 } vg_dtype;

/* Gaussian parameters (Sec. 3.2, Eq. 3-4; Sec. 5 for the colour model), structure of
 * arrays, row-major, device memory:
 *   mu    [n][3]  means (world)                           rec_dtype
 *   scale [n][3]  per-axis standard deviations, > 0       rec_dtype
 *   quat  [n][4]  rotation quaternions (w, x, y, z), normalised inside      rec_dtype
 *   kappa [n]     densities kappa >= 0                    rec_dtype
 *   sh    [n][K][3] real spherical-harmonic colour coefficients, K = (sh_degree+1)^2,
 *                 colour = max(sum_k sh_k Y_k(dir) + 0.5, 0), dir = (mu - o)/|mu - o|
 *                                                          sh_dtype (may be NULL in tomography)
 * Gaussians with a non-finite parameter, a non-positive scale, a zero quaternion or
 * kappa <= 0 are culled (counted in vg_stats.n_culled), never an error. */
typedef struct {
    const void *mu, *scale, *quat, *kappa, *sh;
    int32_t rec_dtype;   /* vg_dtype of mu, scale, quat, kappa */
    int32_t sh_dtype;    /* vg_dtype of sh */
    int32_t n;
    int32_t sh_degree;   /* 0..3 */
    int32_t mu_f32;      /* nonzero: mu is float32 whatever rec_dtype says (mixed storage: BF16 / FP16
                            records with FP32 means keep image errors near 1e-4) */
} vg_gaussians;

/* Pinhole camera, OpenCV axes (x right, y down, z forward).  A world point x maps to
 * camera coordinates R x + t; pixel (i, j) has its centre ray through
 * ((i + 0.5 - cx)/fx, (j + 0.5 - cy)/fy, 1) in camera coordinates (Sec. 4.1: the ray
 * passes through the pixel centre). */
typedef struct {
    float R[9];          /* row-major world->camera rotation */
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
} vg_camera;

/* Parallel-beam tomography geometry.  Rotation axis is world z; for angle theta the rays
 * run along d = (cos theta, sin theta, 0) and detector pixel (i, j) sits at
 * u = u0 + (i + 0.5) pitch_u along (-sin theta, cos theta, 0) and v = v0 + (j + 0.5) pitch_v
 * along (0, 0, 1).  `angles` is a HOST array of n_angles radians. */
typedef struct {
    int32_t n_angles;
    const float *angles;
    int32_t det_w, det_h;
    float pitch_u, pitch_v, u0, v0;
} vg_beam;

/* Blend options.  The paper swaps only the alpha of 3DGS (Sec. 5); thresholds follow the
 * 3DGS conventions when enabled:
 *   alpha_min  contributions with alpha < alpha_min are skipped (0: none skipped);
 *   tau_cut    tile footprints cover every pixel where tau >= tau_cut may hold (> 0);
 *   tau_max    tau is clamped to tau_max, i.e. alpha <= 1 - exp(-tau_max) (INFINITY: none);
 *   T_stop     a pixel stops once its transmittance falls below T_stop (0: never);
 *   bg         background colour added with the final transmittance;
 *   z_near     Gaussians whose mean has camera z <= z_near are culled.
 * The paper states none of these values; the two presets used by the tests are "exact"
 * (alpha_min 0, tau_max inf, T_stop 0) and the 3DGS conventions (alpha_min 1/255,
 * tau_max ln 100, T_stop 1e-4). */
typedef struct {
    float alpha_min, tau_cut, tau_max, T_stop;
    float bg[3];
    float z_near;
    uint32_t flags;      /* VG_FLAG_* */
    int32_t pixels_per_thread;  /* blend kernels: pixels owned by one thread, 1, 2 or 4;
                                   0 = the library defaults (forward 2, backward 1, the
                                   fastest measured).  Every pixel is evaluated by the same
                                   operations in every layout: images and per-pixel state are
                                   bit-identical, forward and backward take the same skip and
                                   clamp decisions, and gradients differ only in the order of
                                   the accumulator's additions. */
    float softplus_beta;  /* 0: rgb = max(sh . Y + 0.5, 0); > 0: rgb = softplus of the same with
                             this beta, ln(1 + e^(beta x)) / beta (Supp. D uses 10) */
    float splat_dilation; /* VG_FLAG_SPLAT only: added to both variances of the 2D covariance
                             (pixels^2; 0 = Eq. 7 as printed, 0.3 = the 3DGS rasterizer) */
    int32_t chunk;        /* blend kernels: records staged in shared memory per barrier, 64 or 128
                             (the backward: a ring of chunk / 16 slots of 32 records);
                             0 = the autotuned value, else 128.  Images are bit-identical;
                             gradients differ only in the order of the accumulator's
                             additions. */
    int32_t tile_w, tile_h; /* screen tile in pixels: 16x16, 32x16 or 16x8; 0x0 = the autotuned
                               shape, else 16x16.  Images are bit-identical and gradients
                               differ only in the order of the accumulator's additions; the
                               tile lists (and with them the instance count) follow the shape,
                               each list still in depth order. */
} vg_opts;

#define VG_FLAG_FIXED_CAPACITY 1u  /* vg_bin_sort never synchronises: the instance count stays
                                      on the device and the kernels cover the capacity reserved
                                      with vg_workspace_reserve.  More instances than that are
                                      dropped and latched: the next vg_query returns
                                      VG_ERR_CAPACITY.  With every buffer reserved (and the views
                                      uploaded by an earlier call with the same cameras), a
                                      step issues no allocation, copy from pageable memory or
                                      synchronisation, so it can be captured in a CUDA graph. */
#define VG_FLAG_GRAD_ZERO 4u       /* render_bwd / project_tomo zero their gradient outputs
                                      before accumulating into them                        */
#define VG_FLAG_DENSITY_THETA 8u   /* the density input holds Eq. 20's theta in [0, 1]:
                                      kappa = -ln(1 - 0.99 theta) (1/s_x + 1/s_y + 1/s_z) / 3;
                                      dkappa then receives dL/dtheta and dscale includes the
                                      scales' share through kappa.  Footprints are sized
                                      with an FP32 upper bound of kappa (exact operations
                                      only: min(x / (1 - x), (1 - e) ln 2) for -ln(1 - x),
                                      1 - x = m 2^e) */
#define VG_FLAG_COUNT_PAIRS 2u     /* render_fwd / render_bwd also count evaluated (pixel,
                                      Gaussian) pairs into vg_stats (slower; for roofline) */
#define VG_FLAG_PROJ_GIVEN 32u     /* vg_project_tomo with dL_dproj: proj already holds the
                                      projection of the same Gaussians, beam and options (from an
                                      earlier call), so it is not recomputed before the backward */
#define VG_FLAG_SPLAT 16u          /* the 3DGS comparison mode (Sec. 3.2, Eq. 5-7) in the same
                                      pipeline: the density input holds the peak opacity o and
                                      alpha = min(o G'(p), alpha_max), G' the 2D Gaussian with
                                      the projected mean and covariance J W Sigma W^T J^T +
                                      splat_dilation I (J the projection's Jacobian at the
                                      mean), alpha_max = min(1 - exp(-tau_max), 1 - 2^-24);
                                      pairs with alpha < alpha_min are skipped and footprints
                                      cover every pixel with o G' >= tau_cut.  Keys, lists,
                                      blending, the backward (dkappa receives dL/do) and the
                                      outputs are otherwise those of the default mode.  Not
                                      combined with VG_FLAG_DENSITY_THETA, tomography or the
                                      cone beam. */

typedef struct {
    int64_t n_items;          /* views x Gaussians of the last preprocess                    */
    int64_t n_visible;        /* items with a non-empty footprint                           */
    int64_t n_culled;         /* invalid parameters or behind z_near                        */
    int64_t n_instances;      /* (tile, item) instances of the last bin_sort                 */
    int64_t n_tiles;          /* tiles over all views                                       */
    int64_t n_pixels;         /* pixels over all views                                      */
    int64_t instance_capacity;
    int64_t n_pairs;          /* evaluated pairs of the last counted render_fwd              */
    int64_t launches;         /* kernels launched by this workspace since creation          */
    int64_t device_bytes;     /* device memory held by the workspace                        */
    int64_t n_pairs_bwd;      /* pairs replayed by the last counted render_bwd              */
    int64_t n_blend;          /* pairs of the last counted render_fwd with tau >= tau_skip   */
    int64_t n_blend_bwd;      /* pairs of the last counted render_bwd with tau >= tau_skip   */
} vg_stats;

/* Per-stage device time recorded with CUDA events on the launching stream while
 * profiling is enabled (vg_profile_enable).  Stage names: "preprocess", "depth_sort",
 * "scan", "duplicate", "tile_sort", "ranges", "render_fwd", "render_bwd", "chain",
 * "l2_loss", "tomo_fwd", "tomo_bwd", "voxel_eval", "ray_march" (the voxel query records its own
 * preprocess, scan, duplicate, tile_sort and ranges stages under the same names). */
typedef struct {
    char name[24];
    int64_t calls;
    double total_ms;
} vg_stage_time;

typedef struct vg_workspace vg_workspace;

/* Create / destroy a workspace: library-owned device scratch (records, keys, sort buffers,
 * per-pixel replay state, gradient intermediates).  Buffers grow on demand unless
 * VG_FLAG_FIXED_CAPACITY is set.  Destroy synchronises the device. */
vg_status vg_workspace_create(vg_workspace **ws);
vg_status vg_workspace_destroy(vg_workspace *ws);

/* Pre-size the workspace (synchronous): n_items = views x Gaussians, n_instances = tile
 * instances, n_pixels and n_tiles over all views.  Needed before fixed-capacity use; it
 * reserves every buffer a step uses except the per-view camera table, which the first
 * vg_preprocess with those cameras allocates and uploads. */
vg_status vg_workspace_reserve(vg_workspace *ws, int64_t n_items, int64_t n_instances,
                               int64_t n_pixels, int64_t n_tiles);

/* Per-(view, Gaussian) set-up (Sec. 5: the rasterizer's per-primitive phase, whose 3D
 * inverse covariances the paper notes are its extra cost, Supp. F).  For each item it
 * computes the depth key (camera z of the mean, FP32), the conservative tile rectangle of
 * the ellipsoid (x - mu)' P (x - mu) <= k^2 that bounds every pixel with tau >= tau_cut,
 * the view-dependent colour from spherical harmonics, and the blend record (whitening of
 * Sigma relative to the pixel grid).  `cams` holds n_views host structs; views are
 * rendered into one concatenated image buffer in view order. */
vg_status vg_preprocess(vg_workspace *ws, const vg_gaussians *g, const vg_camera *cams,
                        int32_t n_views, const vg_opts *opts, void *stream);

/* Tile binning and depth sort (Sec. 7: per-tile sorting of primitives front to back).
 * Emits one instance per (tile, item) the footprint covers and sorts instances by
 * (tile, depth key, Gaussian index) with a stable on-device radix sort.  Synchronises once
 * to read the instance count unless VG_FLAG_FIXED_CAPACITY is set.  Device-side errors (a
 * bounded look-back wait that gave up, a capacity overflow) are latched and returned by this
 * call's synchronisation, or by the next vg_query. */
vg_status vg_bin_sort(vg_workspace *ws, void *stream);

/* Front-to-back blend (Sec. 4.1, Eq. 14 with the Eq. 19 alpha).  Outputs, device memory:
 *   rgb     [sum_v H_v W_v][3] float32, views concatenated, row-major pixels
 *   T_final [sum_v H_v W_v]    float32 final transmittance (may be NULL)
 * The workspace keeps per-pixel replay state (blended count, log-transmittance) for
 * vg_render_bwd. */
vg_status vg_render_fwd(vg_workspace *ws, float *rgb, float *T_final, void *stream);

/* vg_render_fwd with the L2 image loss of vg_l2_loss fused into the blend's epilogue: each
 * pixel's colour is compared with the target where the blend writes it, so no second kernel
 * reads the image back.  The loss is the training loss of the benchmark workloads (an L2 loss
 * against a target image); the paper's own training losses (Supp. D) are out of scope.
 *   rgb, T_final  as vg_render_fwd (rgb must not be NULL)
 *   target   [sum_v H_v W_v][3] float32, device, the layout of rgb
 *   *loss    = scale * sum (rgb - target)^2, a device scalar (overwritten)
 *   dL_drgb  [sum_v H_v W_v][3] float32, device: 2 scale (rgb - target) (overwritten)
 * rgb, T_final and dL_drgb are bit-identical to vg_render_fwd followed by vg_l2_loss; the loss
 * differs from vg_l2_loss's only in the order of its additions.  A NULL loss, or a NULL rgb,
 * target or dL_drgb while the views have pixels: VG_ERR_INVALID_ARG. */
vg_status vg_render_fwd_l2(vg_workspace *ws, float *rgb, float *T_final, const float *target, float scale,
                           float *loss, float *dL_drgb, void *stream);

/* Backward of the last vg_render_fwd on this workspace (derived from Eq. 14 and Eq. 19 by
 * the chain rule; the forward is replayed back to front, nothing per pair is stored).
 *   dL_drgb [pixels][3] float32, dL_dT [pixels] float32 or NULL.
 * Accumulates into float32 device buffers shaped like the inputs of vg_preprocess:
 *   dmu [n][3], dscale [n][3], dquat [n][4] (w.r.t. the unnormalised input), dkappa [n],
 *   dsh [n][K][3] (may be NULL to skip colour gradients).
 * Device-side waits of the blend kernel are bounded: one that gives up (it cannot under
 * normal operation) latches VG_ERR_TIMEOUT, which the next vg_query or synchronising call
 * reports; the gradients of that call are then not valid. */
vg_status vg_render_bwd(vg_workspace *ws, const float *dL_drgb, const float *dL_dT,
                        float *dmu, float *dscale, float *dquat, float *dkappa, float *dsh,
                        void *stream);

/* Backward that allocates no device memory.  The paper has no counterpart: this is a
 * library-usage variant of vg_render_bwd with the same arguments and results.
 *
 * vg_render_bwd keeps its per-(view, Gaussian) gradient accumulator (64 bytes per item) in
 * the workspace and grows it with cudaMalloc when a larger scene arrives; cudaFree and
 * cudaMalloc can also synchronise the whole device.  Some callers cannot allow that at
 * backward time: a process whose device memory belongs to another allocator (a framework's
 * caching allocator) or to a budget fixed in advance, or a latency-critical loop that must
 * not stall on a device-wide synchronisation.  This entry point serves them: it calls no
 * cudaMalloc, cudaFree or allocating library routine, and keeps the accumulator in a
 * fixed array inside the library instead.
 *
 *  - Limit: views x Gaussians of the last vg_preprocess must be <= VG_NOALLOC_MAX_ITEMS;
 *    larger requests return VG_ERR_INVALID_ARG and launch nothing.
 *  - The array (VG_NOALLOC_MAX_ITEMS x 64 bytes = 4 MiB) is a static device allocation of
 *    the library: every GPU that loads the library holds it until the process exits.
 *  - Every call looks up the array's device address in the current context (no allocation),
 *    so the address stays valid after cudaDeviceReset.  The first call on a device, and the
 *    first after a cudaDeviceReset, loads the library's module onto it: make that call before
 *    any stream capture.
 *  - VG_FLAG_COUNT_PAIRS and the stage profiler ("render_bwd", "chain") work as in
 *    vg_render_bwd; the pair counters are the workspace's own.
 *  - Every call shares the one array.  Each call clears the part it uses before
 *    accumulating, but calls whose work overlaps on the GPU (different streams or
 *    workspaces in flight at once) race on it: serialise them.
 *  - The workspace's forward state must exist (vg_render_fwd ran on it); nothing in the
 *    workspace is resized. */
#define VG_NOALLOC_MAX_ITEMS 65536
vg_status vg_render_bwd_noalloc(vg_workspace *ws, const float *dL_drgb, const float *dL_dT,
                                float *dmu, float *dscale, float *dquat, float *dkappa,
                                float *dsh, void *stream);

/* Measured pipe peaks, the denominators of the blend and tomography kernels' roofline
 * (synchronous; allocates nothing).  pipe 0: FP32 FMA instructions per second (one FFMA = 2 flop);
 * pipe 1: ex2.approx instructions per second (the transcendental unit the closed-form opacity
 * uses).  Every thread of a grid at the occupancy limit on every SM runs 8 independent
 * dependency chains with no memory traffic; after a warm-up, three launches of about min_ms each
 * (0 < min_ms <= 10000) are event-timed on `stream` and the fastest is returned in *ops_per_s
 * (lane operations per second) and its duration in *ms (may be NULL).  The SM clock during the
 * run is the caller's to sample. */
vg_status vg_pipe_peak(vg_workspace *ws, int32_t pipe, float min_ms, double *ops_per_s, float *ms, void *stream);

/* Failure-path check of the bounded device waits (no counterpart in the paper: it tests the
 * library's own failure detection).  Runs one bounded wait that can never be satisfied --
 * which = 0: the instance scan's warp-cooperative look-back, 1: a radix pass's look-back, both
 * on a predecessor that never publishes its status, with a limit of spin_limit polls (1..2^20;
 * a few dozen take microseconds); 2: the backward blend's ring wait on a full barrier no
 * producer arrives on, with a limit of spin_limit microseconds (1..2^20).  The wait gives up,
 * latches VG_ERR_TIMEOUT in the workspace and the kernel returns; the next vg_query reports the
 * timeout (and clears it) and the workspace stays usable.  Uses the workspace's scan scratch;
 * nothing a later call reads is left changed. */
vg_status vg_selftest_timeout(vg_workspace *ws, int32_t which, int32_t spin_limit, void *stream);

/* Tomography (Sec. 6.2, Eq. 21): for every angle and detector pixel,
 *   proj[a][j][i] = exp(-sum_g tau_g(ray)),  float32 device buffer [n_angles][det_h][det_w].
 * If dL_dproj is not NULL it also runs the backward and accumulates dmu, dscale, dquat,
 * dkappa (float32, shaped as above).  Colour coefficients are ignored.  Only
 * opts->tau_cut and opts->flags are used. */
vg_status vg_project_tomo(vg_workspace *ws, const vg_gaussians *g, const vg_beam *beam,
                          const vg_opts *opts, float *proj, const float *dL_dproj, float *dmu,
                          float *dscale, float *dquat, float *dkappa, void *stream);

/* One tomography training step with the L2 loss, fused per angle batch: proj (written, as in
 * vg_project_tomo), *loss = scale * sum_i (proj_i - target_i)^2 (device scalar, overwritten) and
 * the gradients of *loss accumulated into dmu, dscale, dquat, dkappa (overwritten with
 * VG_FLAG_GRAD_ZERO).  target [n_angles][det_h][det_w] float32, device.  Each angle batch is
 * preprocessed, binned and projected once, where the two-call form (project, then project with
 * dL_dproj) does it twice. */
vg_status vg_tomo_l2_step(vg_workspace *ws, const vg_gaussians *g, const vg_beam *beam, const vg_opts *opts,
                          const float *target, float scale, float *proj, float *loss, float *dmu, float *dscale,
                          float *dquat, float *dkappa, void *stream);

/* Cone-beam tomography (Eq. 21 with diverging rays): for each of n_views cameras the
 * X-ray source is the camera centre and the detector its image plane, so detector pixel (i, j)
 * measures proj = exp(-sum_g tau_g) along that pixel's ray.  Same Gaussians (density only: sh
 * is ignored), the same key function, tile lists and pixel footprint rectangles as vg_preprocess
 * / vg_bin_sort, and the blend kernels in their exact form (no skip, clamp, early stop or
 * background), whose final transmittance is exp(-sum tau).  opts: tau_cut, z_near, flags
 * (VG_FLAG_DENSITY_THETA, VG_FLAG_GRAD_ZERO, VG_FLAG_FIXED_CAPACITY, VG_FLAG_COUNT_PAIRS) and
 * pixels_per_thread are used.  proj [sum_v H_v W_v] float32, device; with dL_dproj non-NULL
 * the gradients of sum(dL_dproj * proj) are accumulated into dmu/dscale/dquat/dkappa as in
 * vg_render_bwd. */
vg_status vg_project_cone(vg_workspace *ws, const vg_gaussians *g, const vg_camera *cams, int32_t n_views,
                          const vg_opts *opts, float *proj, const float *dL_dproj, float *dmu, float *dscale,
                          float *dquat, float *dkappa, void *stream);

/* Ray-marching reference (Supp. A) of the views binned by the last vg_preprocess / vg_bin_sort
 * (default mode only): Eq. 1 with sigma(x) = sum kappa G(x) and c(x) = sum c kappa G(x) / sigma(x)
 * (c the Gaussians' colours of the view) by NeRF's quadrature on n_samples (1..2^20) midpoint
 * samples of [t_near, t_far] (0 <= t_near < t_far) along each pixel's unit ray:
 *   rgb = sum_k T_k (1 - exp(-sigma_k delta)) c(x_k) + T bg,   T = exp(-delta sum_k sigma_k),
 * ending a pixel once T < opts.T_stop.  Unlike the blend it assumes neither order nor the absence
 * of overlap, so |rgb - blend| measures those approximations: with raster_rgb (the vg_render_fwd
 * image of the same views) err_map[p] = max over channels |rgb - raster_rgb| (the overlap-error
 * map).  Each Gaussian enters the pixels of its footprint rectangle (opts.tau_cut bounds what
 * the rest adds to a ray's optical depth).  rgb [P][3], T [P], err_map [P] are float32 device
 * buffers, each optional (err_map needs raster_rgb). */
vg_status vg_ray_march(vg_workspace *ws, float t_near, float t_far, int32_t n_samples, const float *raster_rgb,
                       float *rgb, float *T, float *err_map, void *stream);

/* Regular voxel grid: voxel (i, j, k) has its centre at origin + (i + 1/2, j + 1/2, k + 1/2) * voxel. */
typedef struct {
    float origin[3];
    float voxel[3];
    int32_t nx, ny, nz;   /* each 1..32767 */
} vg_grid;

/* Density on a grid (the density of Eq. 3-4, for volumetric comparisons):
 *   out[k][j][i] = sum_g kappa_g exp(-(x - mu_g)' Sigma_g^-1 (x - mu_g) / 2)   (float32, device)
 * at the voxel centres x.  Each Gaussian is truncated to the voxel box of its ellipsoid
 * (x - mu)' Sigma^-1 (x - mu) <= k^2, k^2 = 2 ln 2 e with kappa / sigma_cut = m 2^e, where
 * sigma_cut = opts->tau_cut; with VG_FLAG_DENSITY_THETA the density input holds Eq. 20's theta.
 * SH are not used.  Synchronises once (the instance count). */
vg_status vg_query_density(vg_workspace *ws, const vg_gaussians *g, const vg_grid *grid, const vg_opts *opts,
                           float *out, void *stream);

/* L2 image loss helper for training steps: loss = scale * sum_i (x_i - y_i)^2 written to the
 * device scalar *loss (overwritten), grad_i = 2 scale (x_i - y_i) (overwritten). */
vg_status vg_l2_loss(vg_workspace *ws, const float *x, const float *y, int64_t n, float scale,
                     float *loss, float *grad, void *stream);

/* Autotuner (synchronous; allocates scratch): after vg_bin_sort, times the forward and the
 * backward blend with 1, 2 and 4 pixels per thread (which also sets each warp's pixel box:
 * 8x4, 8x8 or 16x8 pixels) and with 64 and 128 records per staged chunk (the chunk depth),
 * `reps` timed runs each after one warm-up, for each tile shape 32x16, 16x16 and 16x8: the
 * views of the last vg_preprocess are preprocessed and binned again for each shape (binning
 * timed too, in the form VG_FLAG_FIXED_CAPACITY selects; the instance buffers grow to the
 * largest count), unless that call fixed vg_opts.tile_w / tile_h, which are then kept.  The
 * shape with the least binning + forward + backward time and its fastest settings become this
 * workspace's defaults for vg_opts.pixels_per_thread = 0, vg_opts.chunk = 0 and
 * vg_opts.tile_w = tile_h = 0, and the workspace is left binned with that shape.  The chosen
 * values are written to *ppt_fwd / *ppt_bwd / *chunk_fwd / *chunk_bwd / *tile_w / *tile_h (each
 * may be NULL).  Images and gradients do not depend on the choice; instance counts do (a
 * fixed capacity reserved for one shape may not hold another's: reserve after tuning).  Call
 * vg_render_fwd again before vg_render_bwd. */
vg_status vg_autotune(vg_workspace *ws, int32_t reps, int32_t *ppt_fwd, int32_t *ppt_bwd, int32_t *chunk_fwd,
                      int32_t *chunk_bwd, int32_t *tile_w, int32_t *tile_h, void *stream);

/* Statistics of the last calls (synchronises the stream).  *out is filled in every case; the
 * status is the first device-side error latched since the last report (VG_ERR_CAPACITY when
 * a fixed-capacity bin_sort had more instances than reserved, VG_ERR_TIMEOUT when a bounded
 * device wait gave up), which this call clears, else VG_OK. */
vg_status vg_query(vg_workspace *ws, vg_stats *out, void *stream);

/* Enable (1) or disable (0) per-stage event timing; enabling clears earlier records. */
vg_status vg_profile_enable(vg_workspace *ws, int32_t enable);

/* Restrict the event timing to some stages: bit k of stage_mask selects the k-th stage name in
 * the vg_stage_time list above ("preprocess" = bit 0 ... "ray_march" = bit 13); 0 selects all
 * (the default).  Fewer recorded stages mean fewer event records between the kernels of a
 * timed step.  Errors: VG_ERR_INVALID_ARG for a NULL workspace. */
vg_status vg_profile_stages(vg_workspace *ws, uint32_t stage_mask);

/* Aggregate the recorded stage times (synchronises on the recorded events) into `out`
 * (capacity entries, HOST memory); *n_out receives the number of stages written.  The
 * records are cleared. */
vg_status vg_profile_read(vg_workspace *ws, vg_stage_time *out, int32_t capacity, int32_t *n_out);

/* Diagnostic read-backs of the last preprocess / bin_sort into HOST buffers (synchronous):
 *   depth_bits [n_items] uint32 (0xFFFFFFFF for culled items), rect [n_items][4] int32
 *   (tile x0, y0, x1, y1 inclusive; -1 when culled); tile_start [n_tiles + 1] int64 and
 *   sorted_item [n_instances] int32 (item = view * n + Gaussian). */
vg_status vg_read_keys(vg_workspace *ws, uint32_t *depth_bits, int32_t *rect);
vg_status vg_read_bins(vg_workspace *ws, int64_t *tile_start, int32_t *sorted_item);
/* The lists of tiles [tile0, tile1) only: counts [tile1 - tile0] int64 and their items,
 * concatenated in tile order, into sorted_item (capacity `cap` entries; *n_out receives the
 * number written, VG_ERR_INVALID_ARG when cap is too small). */
vg_status vg_read_bins_range(vg_workspace *ws, int64_t tile0, int64_t tile1, int64_t *counts,
                             int32_t *sorted_item, int64_t cap, int64_t *n_out);

/* Diagnostic read-back of the per-pixel replay state of the last vg_render_fwd into HOST buffers
 * (synchronous), views concatenated as in the image:
 *   S [n_pixels] float32: sum of the tau of the pairs the pixel blended (Eq. 14: T = exp(-S)),
 *   last [n_pixels] uint32: position + 1, within the pixel's tile list, of the last pair the
 *        pixel blended (0 when it blended none).
 * Either may be NULL.  Together they identify the pixels where a threshold decision (alpha_min,
 * T_stop) went differently from another implementation.  VG_ERR_STATE before a forward. */
vg_status vg_read_pixel_state(vg_workspace *ws, float *S, uint32_t *last);

/* Message of the last failure on this workspace ("" if none).  ws may be NULL for
 * failures of vg_workspace_create. */
const char *vg_last_error(const vg_workspace *ws);

#ifdef __cplusplus
}
#endif
#endif /* VG_H */
