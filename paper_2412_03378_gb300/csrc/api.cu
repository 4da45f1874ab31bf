// C ABI of the rasterizer: workspace management, argument validation and the order of
// kernel launches for each entry point declared in include/vg.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vg_internal.cuh"

namespace vg {
// csrc/peaks.cu: one bounded mbarrier wait of the backward's ring that must give up after
// limit_us microseconds (latching kDevErrTimeout in *err).
cudaError_t launch_ring_selftest(int limit_us, uint32_t *err, cudaStream_t st, long long *launches);
}  // namespace vg

using namespace vg;

namespace {

template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
};

}  // namespace

struct vg_workspace {
    std::string err;
    int stage = 0;   // 0 empty, 1 preprocessed, 2 binned, 3 rendered
    GaussIn g{};
    vg_opts opts{};
    BlendParams bp{};
    int n_views = 0;
    std::vector<ViewInfo> views_h;
    std::vector<int> tile_view_h;
    long long n_items = 0, n_tiles = 0, n_pixels = 0, n_inst = 0;
    long long capacity = 0;
    long long launches = 0;
    bool views_valid = false;
    bool tomo_read = false;   // read-backs refer to the last tomography batch

    DBuf<ViewInfo> views;
    DBuf<int> tile_view;
    DBuf<float4> rec;
    DBuf<uint32_t> depth, count, offsets;
    DBuf<short4> rect, prect;
    DBuf<uint32_t> skey[2], sval[2];
    DBuf<uint32_t> ikey[2], ival[2];
    uint32_t *perm = nullptr;          // items in depth order (points into sval)
    uint32_t *inst_key = nullptr;      // sorted instance tile keys
    uint32_t *inst_item = nullptr;     // sorted instance items
    DBuf<uint2> ranges;
    DBuf<float> S_fin, T_fin;
    DBuf<uint32_t> nlast;
    DBuf<float> grad;
    DBuf<uint32_t> hist, scan_tmp;
    DBuf<unsigned long long> counters;   // [0] visible items; fwd [1] evaluated, [2] blended pairs; bwd [3], [4];
                                         // [6] instance total of the last scan, [7] look-back timeout flag
    DBuf<float> tomo_cs;
    DBuf<uint32_t> tord;                  // tile order buffer
    DBuf<short4> vbox;                    // voxel query: truncation boxes (2 per Gaussian)
    DBuf<float4> march_E;                 // ray march: o'.A_k per item
    DBuf<float> tomo_dl;                  // fused tomography step: dL/dproj of one angle batch
    uint32_t *tile_order = nullptr;       // longest-first tile order of the last bin_sort
    uint32_t *tile_order_bwd = nullptr;   // longest replay first, from the last forward (NULL: none)
    DBuf<uint32_t> treplay, tord_bwd;     // per-tile replay lengths and their order
    int ppt_fwd = 2, ppt_bwd = 1;         // pixels per thread of the blend kernels
    int tuned_fwd = 0, tuned_bwd = 0;     // vg_autotune's choice (0: none yet)
    int tuned_chunk_fwd = 0, tuned_chunk_bwd = 0;
    int tuned_tw = 0, tuned_th = 0;        // vg_autotune's tile shape (0: none yet)
    uint32_t *h_total = nullptr;         // pinned: [0..1] instance total (u64), [2] look-back timeout flag
    cudaEvent_t total_ev = nullptr;       // recorded after the copy into h_total (binning ahead of it)
    const float *grad_zero_p = nullptr;   // grad.p and the leading floats of it known to be zero
    size_t grad_zero_n = 0;               // (left so by the chain), which a backward need not clear

    // per-stage event timing (vg_profile_enable)
    bool prof_on = false;
    uint32_t prof_mask = ~0u;             // bit k: stage k is recorded (vg_profile_stages)
    struct ProfRec {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> prof_pool;
};

namespace {

// Measured on the 1M-Gaussian 1280x832 workload (GB300, footprint culling on): forward
// 0.53 / 0.49 / 0.74 ms and backward 1.32 / 1.16 / 1.19 ms for 1 / 2 / 4 pixels per thread.
constexpr int kDefaultPixelsFwd = 2;
constexpr int kDefaultPixelsBwd = 1;
constexpr int kDefaultChunk = 128;

enum Stage { ST_PRE, ST_DEPTH, ST_SCAN, ST_DUP, ST_TILE, ST_RANGES, ST_FWD, ST_BWD, ST_CHAIN, ST_LOSS, ST_TFWD,
             ST_TBWD, ST_VOXEL, ST_MARCH, ST_COUNT };
const char *kStageName[ST_COUNT] = {"preprocess", "depth_sort", "scan",     "duplicate", "tile_sort", "ranges",
                                    "render_fwd", "render_bwd", "chain",    "l2_loss",   "tomo_fwd",  "tomo_bwd",
                                    "voxel_eval", "ray_march"};

cudaEvent_t prof_event(vg_workspace *ws) {
    if (!ws->prof_pool.empty()) {
        cudaEvent_t e = ws->prof_pool.back();
        ws->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Records an event pair around a stage on the launching stream while profiling is on.
struct ProfScope {
    vg_workspace *ws;
    cudaStream_t st;
    int idx = -1;
    ProfScope(vg_workspace *w, int stage, cudaStream_t s) : ws(w), st(s) {
        if (!ws->prof_on || !((ws->prof_mask >> stage) & 1u)) return;
        cudaEvent_t a = prof_event(ws), b = prof_event(ws);
        if (!a || !b) return;
        cudaEventRecord(a, st);
        ws->prof.push_back({stage, a, b});
        idx = (int)ws->prof.size() - 1;
    }
    ~ProfScope() {
        if (idx >= 0) cudaEventRecord(ws->prof[idx].b, st);
    }
};

vg_status fail(vg_workspace *ws, vg_status s, const std::string &msg) {
    if (ws) ws->err = msg;
    return s;
}

#define VG_CUDA(ws, call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(ws, VG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
vg_status ensure(vg_workspace *ws, DBuf<T> &b, size_t n, const char *what) {
    if (n == 0) n = 1;
    if (b.p && b.n >= n) return VG_OK;
    if (b.p && (ws->opts.flags & VG_FLAG_FIXED_CAPACITY))
        return fail(ws, VG_ERR_CAPACITY, std::string("fixed-capacity workspace too small for ") + what);
    size_t nn = std::max(n, b.n + b.n / 4);
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        b.p = nullptr;
        b.n = 0;
        if (e != cudaSuccess) return fail(ws, VG_ERR_CUDA, std::string("cudaFree: ") + cudaGetErrorString(e));
    }
    cudaError_t e = cudaMalloc((void **)&b.p, nn * sizeof(T));
    if (e != cudaSuccess) {
        b.p = nullptr;
        (void)cudaGetLastError();
        return fail(ws, VG_ERR_OOM, std::string("cudaMalloc for ") + what + ": " + cudaGetErrorString(e));
    }
    b.n = nn;
    return VG_OK;
}

#define VG_TRY(x)                          \
    do {                                   \
        vg_status s_ = (x);                \
        if (s_ != VG_OK) return s_;        \
    } while (0)

template <typename T>
void release(DBuf<T> &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.0f; }
// the tile shapes the blend kernels' pixel layouts cover (widths a multiple of 16, heights of 8)
bool tile_shape_ok(int tw, int th) { return (tw == 16 && th == 16) || (tw == 32 && th == 16) || (tw == 16 && th == 8); }

int bits_for(long long n) {
    int b = 1;
    while (b < 32 && (1LL << b) < n) ++b;
    return b;
}

vg_status check_gauss(vg_workspace *ws, const vg_gaussians *g, bool need_sh) {
    if (!g) return fail(ws, VG_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n < 0) return fail(ws, VG_ERR_INVALID_ARG, "negative Gaussian count");
    if (g->sh_degree < 0 || g->sh_degree > 3) return fail(ws, VG_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (g->rec_dtype < VG_F32 || g->rec_dtype > VG_F16 || g->sh_dtype < VG_F32 || g->sh_dtype > VG_F16)
        return fail(ws, VG_ERR_INVALID_ARG, "unknown dtype");
    if (g->n > 0 && (!g->mu || !g->scale || !g->quat || !g->kappa || (need_sh && !g->sh)))
        return fail(ws, VG_ERR_INVALID_ARG, "a Gaussian parameter pointer is NULL");
    return VG_OK;
}

GaussIn to_in(const vg_gaussians *g) {
    GaussIn r;
    r.mu = g->mu;
    r.scale = g->scale;
    r.quat = g->quat;
    r.kappa = g->kappa;
    r.sh = g->sh;
    r.rec_dtype = g->rec_dtype;
    r.sh_dtype = g->sh_dtype;
    r.n = g->n;
    r.sh_degree = g->sh_degree;
    r.mu_f32 = g->mu_f32 ? 1 : 0;
    r.density_theta = 0;
    r.softplus_beta = 0.0f;
    r.splat = 0;
    r.splat_dil = 0.0f;
    return r;
}

}  // namespace

extern "C" {

const char *vg_last_error(const vg_workspace *ws) {
    static const char *none = "";
    static const char *nows = "workspace is NULL or could not be created";
    if (!ws) return nows;
    return ws->err.empty() ? none : ws->err.c_str();
}

vg_status vg_workspace_create(vg_workspace **out) {
    if (!out) return VG_ERR_INVALID_ARG;
    *out = nullptr;
    vg_workspace *ws = new (std::nothrow) vg_workspace();
    if (!ws) return VG_ERR_OOM;
    cudaError_t e = cudaMallocHost((void **)&ws->h_total, 64);
    if (e != cudaSuccess) {
        delete ws;
        return VG_ERR_CUDA;
    }
    e = cudaMalloc((void **)&ws->counters.p, 8 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFreeHost(ws->h_total);
        delete ws;
        return VG_ERR_OOM;
    }
    ws->counters.n = 8;
    cudaMemset(ws->counters.p, 0, 8 * sizeof(unsigned long long));
    *out = ws;
    return VG_OK;
}

vg_status vg_workspace_destroy(vg_workspace *ws) {
    if (!ws) return VG_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    release(ws->views);
    release(ws->tile_view);
    release(ws->rec);
    release(ws->depth);
    release(ws->count);
    release(ws->offsets);
    release(ws->rect);
    release(ws->prect);
    for (int k = 0; k < 2; ++k) {
        release(ws->skey[k]);
        release(ws->sval[k]);
        release(ws->ikey[k]);
        release(ws->ival[k]);
    }
    release(ws->ranges);
    release(ws->S_fin);
    release(ws->T_fin);
    release(ws->nlast);
    release(ws->grad);
    release(ws->hist);
    release(ws->scan_tmp);
    release(ws->counters);
    release(ws->tomo_cs);
    release(ws->tord);
    release(ws->treplay);
    release(ws->tord_bwd);
    release(ws->vbox);
    release(ws->march_E);
    release(ws->tomo_dl);
    if (ws->h_total) cudaFreeHost(ws->h_total);
    for (auto &r : ws->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ws->prof_pool) cudaEventDestroy(e);
    if (ws->total_ev) cudaEventDestroy(ws->total_ev);
    delete ws;
    return VG_OK;
}

static vg_status reserve_items(vg_workspace *ws, long long n_items) {
    VG_TRY(ensure(ws, ws->rec, (size_t)n_items * kRecF4, "records"));
    VG_TRY(ensure(ws, ws->depth, (size_t)n_items, "depth keys"));
    VG_TRY(ensure(ws, ws->count, (size_t)n_items, "tile counts"));
    VG_TRY(ensure(ws, ws->rect, (size_t)n_items, "tile rectangles"));
    VG_TRY(ensure(ws, ws->prect, (size_t)n_items, "pixel rectangles"));
    VG_TRY(ensure(ws, ws->offsets, (size_t)n_items + 1, "offsets"));
    for (int k = 0; k < 2; ++k) {
        VG_TRY(ensure(ws, ws->skey[k], (size_t)n_items, "sort keys"));
        VG_TRY(ensure(ws, ws->sval[k], (size_t)n_items, "sort values"));
    }
    return VG_OK;
}

static vg_status reserve_sort_scratch(vg_workspace *ws, long long n) {
    VG_TRY(ensure(ws, ws->hist, radix_scratch_words(n, 32), "radix sort scratch"));
    VG_TRY(ensure(ws, ws->scan_tmp, scan_tmp_words(n), "scan scratch"));
    return VG_OK;
}

static unsigned long long *total64_ptr(vg_workspace *ws) { return ws->counters.p + 6; }
static uint32_t *lookback_err_ptr(vg_workspace *ws) { return (uint32_t *)(ws->counters.p + 7); }
// The backward's tile order: by the replay lengths the last forward measured, else the binning's.
static const uint32_t *bwd_order(vg_workspace *ws) { return ws->tile_order_bwd ? ws->tile_order_bwd : ws->tile_order; }

// Reports (and clears) error bits latched on the device: a look-back timeout, a capacity
// overflow.  Reads h_total[2] as filled by the last copy of counters[6..7].
static vg_status latched_status(vg_workspace *ws, cudaStream_t st) {
    const uint32_t e = ws->h_total[2];
    if (e == 0) return VG_OK;
    ws->h_total[2] = 0;
    ws->grad_zero_n = 0;   // after a device-side failure the next backward clears its accumulator
    cudaMemsetAsync(lookback_err_ptr(ws), 0, sizeof(uint32_t), st);
    if (e & kDevErrTimeout) return fail(ws, VG_ERR_TIMEOUT, "a bounded device wait (scan or sort look-back, backward ring) timed out");
    return fail(ws, VG_ERR_CAPACITY, "more (tile, Gaussian) instances than the fixed capacity");
}

// Reads the instance total of the last scan and the latched error bits (synchronises st).
static vg_status read_total(vg_workspace *ws, cudaStream_t st, long long *total) {
    VG_CUDA(ws, cudaMemcpyAsync(ws->h_total, ws->counters.p + 6, 2 * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, st));
    VG_CUDA(ws, cudaStreamSynchronize(st));
    VG_TRY(latched_status(ws, st));
    *total = (long long)(((unsigned long long)ws->h_total[1] << 32) | ws->h_total[0]);
    return VG_OK;
}

// The same in two halves: the copy and an event now, the wait (on that event only, so that
// work enqueued after the copy keeps running) later.
static vg_status read_total_start(vg_workspace *ws, cudaStream_t st) {
    if (!ws->total_ev) VG_CUDA(ws, cudaEventCreateWithFlags(&ws->total_ev, cudaEventDisableTiming));
    VG_CUDA(ws, cudaMemcpyAsync(ws->h_total, ws->counters.p + 6, 2 * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, st));
    VG_CUDA(ws, cudaEventRecord(ws->total_ev, st));
    return VG_OK;
}
static vg_status read_total_finish(vg_workspace *ws, cudaStream_t st, long long *total) {
    VG_CUDA(ws, cudaEventSynchronize(ws->total_ev));
    VG_TRY(latched_status(ws, st));
    *total = (long long)(((unsigned long long)ws->h_total[1] << 32) | ws->h_total[0]);
    return VG_OK;
}

static vg_status reserve_instances(vg_workspace *ws, long long cap) {
    for (int k = 0; k < 2; ++k) {
        VG_TRY(ensure(ws, ws->ikey[k], (size_t)cap, "instance keys"));
        VG_TRY(ensure(ws, ws->ival[k], (size_t)cap, "instance items"));
    }
    ws->capacity = (long long)std::min(ws->ikey[0].n, ws->ival[0].n);
    return reserve_sort_scratch(ws, cap);
}

vg_status vg_workspace_reserve(vg_workspace *ws, int64_t n_items, int64_t n_instances, int64_t n_pixels,
                               int64_t n_tiles) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (n_items < 0 || n_instances < 0 || n_pixels < 0 || n_tiles < 0)
        return fail(ws, VG_ERR_INVALID_ARG, "negative reservation");
    const unsigned flags = ws->opts.flags;
    ws->opts.flags &= ~VG_FLAG_FIXED_CAPACITY;
    vg_status s = reserve_items(ws, n_items);
    if (s == VG_OK) s = reserve_sort_scratch(ws, n_items);
    if (s == VG_OK) s = reserve_instances(ws, n_instances);
    if (s == VG_OK) s = ensure(ws, ws->S_fin, (size_t)n_pixels, "pixel state");
    if (s == VG_OK) s = ensure(ws, ws->T_fin, (size_t)n_pixels, "pixel state");
    if (s == VG_OK) s = ensure(ws, ws->nlast, (size_t)n_pixels, "pixel state");
    if (s == VG_OK) s = ensure(ws, ws->ranges, (size_t)n_tiles, "tile ranges");
    if (s == VG_OK) s = ensure(ws, ws->tile_view, (size_t)n_tiles, "tile views");
    if (s == VG_OK) s = ensure(ws, ws->grad, (size_t)n_items * kGradN, "gradient accumulators");
    if (s == VG_OK) s = ensure(ws, ws->tord, (size_t)n_tiles, "tile order");
    ws->opts.flags = flags;
    return s;
}

static vg_status upload_views(vg_workspace *ws, const std::vector<ViewInfo> &vh, const std::vector<int> &tv,
                              cudaStream_t st);
static vg_status run_preprocess(vg_workspace *ws, cudaStream_t st);

static vg_status preprocess_impl(vg_workspace *ws, const vg_gaussians *g, const vg_camera *cams, int32_t n_views,
                                 const vg_opts *opts, void *stream, bool need_sh) {
    if (!ws) return VG_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    VG_TRY(check_gauss(ws, g, need_sh));
    if (!cams || n_views < 1) return fail(ws, VG_ERR_INVALID_ARG, "need at least one camera");
    if (!opts) return fail(ws, VG_ERR_INVALID_ARG, "opts is NULL");
    if (!finite_pos(opts->tau_cut)) return fail(ws, VG_ERR_INVALID_ARG, "tau_cut must be finite and > 0");
    if (!(opts->alpha_min >= 0.0f && opts->alpha_min < 1.0f)) return fail(ws, VG_ERR_INVALID_ARG, "alpha_min must be in [0, 1)");
    if (!(opts->tau_max > 0.0f) || !(opts->T_stop >= 0.0f && opts->T_stop < 1.0f) || !std::isfinite(opts->z_near))
        return fail(ws, VG_ERR_INVALID_ARG, "invalid tau_max, T_stop or z_near");
    if (opts->pixels_per_thread != 0 && opts->pixels_per_thread != 1 && opts->pixels_per_thread != 2 &&
        opts->pixels_per_thread != 4)
        return fail(ws, VG_ERR_INVALID_ARG, "pixels_per_thread must be 0, 1, 2 or 4");
    if (opts->chunk != 0 && opts->chunk != 64 && opts->chunk != 128)
        return fail(ws, VG_ERR_INVALID_ARG, "chunk must be 0, 64 or 128");
    int tw = opts->tile_w, th = opts->tile_h;
    if (tw == 0 && th == 0) {
        tw = ws->tuned_tw ? ws->tuned_tw : kTile;
        th = ws->tuned_th ? ws->tuned_th : kTile;
    } else if (!tile_shape_ok(tw, th)) {
        return fail(ws, VG_ERR_INVALID_ARG, "tile_w x tile_h must be 0 x 0, 16 x 16, 32 x 16 or 16 x 8");
    }
    const long long n_items = (long long)g->n * n_views;
    if (n_items >= 0xFFFFFFFFLL) return fail(ws, VG_ERR_INVALID_ARG, "views x Gaussians must be < 2^32");

    std::vector<ViewInfo> vh((size_t)n_views);
    std::vector<int> tv;
    long long tile_base = 0, pix_base = 0;
    for (int v = 0; v < n_views; ++v) {
        const vg_camera &c = cams[v];
        if (c.width <= 0 || c.height <= 0 || !finite_pos(std::fabs(c.fx)) || !finite_pos(std::fabs(c.fy)) ||
            !std::isfinite(c.cx) || !std::isfinite(c.cy))
            return fail(ws, VG_ERR_INVALID_ARG, "invalid camera intrinsics or size");
        for (int k = 0; k < 9; ++k)
            if (!std::isfinite(c.R[k])) return fail(ws, VG_ERR_INVALID_ARG, "non-finite camera rotation");
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(c.t[k])) return fail(ws, VG_ERR_INVALID_ARG, "non-finite camera translation");
        ViewInfo &V = vh[v];
        memset(&V, 0, sizeof(V));
        memcpy(V.R, c.R, sizeof(V.R));
        memcpy(V.t, c.t, sizeof(V.t));
        V.fx = c.fx;
        V.fy = c.fy;
        V.cx = c.cx;
        V.cy = c.cy;
        for (int k = 0; k < 3; ++k) {
            V.od[k] = -((double)c.R[k] * c.t[0] + (double)c.R[3 + k] * c.t[1] + (double)c.R[6 + k] * c.t[2]);
            V.of[k] = (float)V.od[k];
        }
        V.W = c.width;
        V.H = c.height;
        V.tw = tw;
        V.th = th;
        V.tiles_x = (c.width + tw - 1) / tw;
        V.tiles_y = (c.height + th - 1) / th;
        if (c.width > 32767 || c.height > 32767) return fail(ws, VG_ERR_INVALID_ARG, "image wider or taller than 32767");
        V.tile_base = (int)tile_base;
        V.pix_base = pix_base;
        for (int t = 0; t < V.tiles_x * V.tiles_y; ++t) tv.push_back(v);
        tile_base += (long long)V.tiles_x * V.tiles_y;
        pix_base += (long long)c.width * c.height;
        if (tile_base >= (1LL << 30)) return fail(ws, VG_ERR_INVALID_ARG, "too many tiles");
    }
    if (!(opts->softplus_beta >= 0.0f) || !std::isfinite(opts->softplus_beta))
        return fail(ws, VG_ERR_INVALID_ARG, "softplus_beta must be finite and >= 0");
    const bool splat = (opts->flags & VG_FLAG_SPLAT) != 0;
    if (splat && (opts->flags & VG_FLAG_DENSITY_THETA))
        return fail(ws, VG_ERR_INVALID_ARG, "VG_FLAG_SPLAT and VG_FLAG_DENSITY_THETA exclude each other");
    if (splat && !(opts->splat_dilation >= 0.0f && std::isfinite(opts->splat_dilation)))
        return fail(ws, VG_ERR_INVALID_ARG, "splat_dilation must be finite and >= 0");
    ws->opts = *opts;
    ws->g = to_in(g);
    ws->g.density_theta = (opts->flags & VG_FLAG_DENSITY_THETA) ? 1 : 0;
    ws->g.softplus_beta = opts->softplus_beta;
    ws->g.splat = splat ? 1 : 0;
    ws->g.splat_dil = splat ? opts->splat_dilation : 0.0f;
    ws->tomo_read = false;
    VG_TRY(reserve_items(ws, n_items));
    VG_TRY(upload_views(ws, vh, tv, st));
    ws->n_views = n_views;
    ws->n_items = n_items;
    ws->n_tiles = tile_base;
    ws->n_pixels = pix_base;
    ws->bp.tau_skip = opts->alpha_min > 0.0f ? (float)(-std::log1p(-(double)opts->alpha_min)) : 0.0f;
    ws->bp.tau_max = opts->tau_max;
    ws->ppt_fwd = opts->pixels_per_thread ? opts->pixels_per_thread : (ws->tuned_fwd ? ws->tuned_fwd : kDefaultPixelsFwd);
    ws->ppt_bwd = opts->pixels_per_thread ? opts->pixels_per_thread : (ws->tuned_bwd ? ws->tuned_bwd : kDefaultPixelsBwd);
    ws->bp.chunk_fwd = opts->chunk ? opts->chunk : (ws->tuned_chunk_fwd ? ws->tuned_chunk_fwd : kDefaultChunk);
    ws->bp.chunk_bwd = opts->chunk ? opts->chunk : (ws->tuned_chunk_bwd ? ws->tuned_chunk_bwd : kDefaultChunk);
    ws->bp.T_stop = opts->T_stop;
    ws->bp.tile_px = tw * th;
    for (int c = 0; c < 3; ++c) ws->bp.bg[c] = opts->bg[c];
    ws->bp.pixel_test = ws->bp.tau_skip < opts->tau_cut ? 1 : 0;
    // splat mode: alpha <= min(1 - exp(-tau_max), 1 - 2^-24) keeps 1 - alpha and S = sum tau finite
    ws->bp.splat = splat ? 1 : 0;
    ws->bp.alpha_min = opts->alpha_min;
    ws->bp.alpha_max = (float)std::min(-std::expm1(-(double)opts->tau_max), 1.0 - 5.9604644775390625e-8);
    if (splat) ws->bp.pixel_test = opts->alpha_min < opts->tau_cut ? 1 : 0;
    return run_preprocess(ws, st);
}

// The view table and the tile -> view map on the device (copied only when they changed).
static vg_status upload_views(vg_workspace *ws, const std::vector<ViewInfo> &vh, const std::vector<int> &tv,
                              cudaStream_t st) {
    VG_TRY(ensure(ws, ws->views, vh.size(), "views"));
    VG_TRY(ensure(ws, ws->tile_view, tv.size(), "tile views"));
    const bool same = ws->views_valid && ws->views_h.size() == vh.size() &&
                      memcmp(ws->views_h.data(), vh.data(), vh.size() * sizeof(ViewInfo)) == 0;
    if (!same) {
        // pageable sources: the runtime stages them before returning, so the host vectors
        // may change afterwards
        VG_CUDA(ws, cudaMemcpyAsync(ws->views.p, vh.data(), vh.size() * sizeof(ViewInfo), cudaMemcpyHostToDevice, st));
        VG_CUDA(ws, cudaMemcpyAsync(ws->tile_view.p, tv.data(), tv.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        ws->views_h = vh;
        ws->tile_view_h = tv;
        ws->views_valid = true;
    }
    return VG_OK;
}

// Per-item records, depth keys and tile footprints of the workspace's Gaussians and views.
static vg_status run_preprocess(vg_workspace *ws, cudaStream_t st) {
    VG_CUDA(ws, cudaMemsetAsync(ws->counters.p, 0, sizeof(unsigned long long), st));
    if (ws->n_items > 0) {
        ProfScope ps(ws, ST_PRE, st);
        VG_CUDA(ws, launch_preprocess(ws->g, ws->views.p, ws->n_views, ws->opts.z_near, ws->opts.tau_cut, ws->rec.p,
                                      ws->depth.p, ws->count.p, ws->rect.p, ws->prect.p, ws->counters.p, st,
                                      &ws->launches));
    }
    ws->stage = 1;
    return VG_OK;
}

// The views of the last vg_preprocess cut into tw x th tiles, preprocessed again (the tile
// footprints depend on the shape; the records do not).
static vg_status retile(vg_workspace *ws, int tw, int th, cudaStream_t st) {
    std::vector<ViewInfo> vh = ws->views_h;
    std::vector<int> tv;
    long long tile_base = 0;
    for (size_t v = 0; v < vh.size(); ++v) {
        ViewInfo &V = vh[v];
        V.tw = tw;
        V.th = th;
        V.tiles_x = (V.W + tw - 1) / tw;
        V.tiles_y = (V.H + th - 1) / th;
        V.tile_base = (int)tile_base;
        tile_base += (long long)V.tiles_x * V.tiles_y;
        if (tile_base >= (1LL << 30)) return fail(ws, VG_ERR_INVALID_ARG, "too many tiles");
        tv.insert(tv.end(), (size_t)V.tiles_x * V.tiles_y, (int)v);
    }
    VG_TRY(upload_views(ws, vh, tv, st));
    ws->n_tiles = tile_base;
    ws->bp.tile_px = tw * th;
    return run_preprocess(ws, st);
}

vg_status vg_preprocess(vg_workspace *ws, const vg_gaussians *g, const vg_camera *cams, int32_t n_views,
                        const vg_opts *opts, void *stream) {
    return preprocess_impl(ws, g, cams, n_views, opts, stream, true);
}

vg_status vg_bin_sort(vg_workspace *ws, void *stream) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (ws->stage < 1) return fail(ws, VG_ERR_STATE, "vg_bin_sort before vg_preprocess");
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = ws->n_items;
    const bool fixed = (ws->opts.flags & VG_FLAG_FIXED_CAPACITY) != 0;
    // binning ahead of the count's readback on instance buffers left by an earlier call (below);
    // the sort scratch for both sorts is reserved before anything is enqueued
    const bool ahead = !fixed && ws->capacity > 0 && ws->ikey[1].p != nullptr;
    VG_TRY(reserve_sort_scratch(ws, ahead ? std::max(n, ws->capacity) : n));
    // 1. items by depth key (stable: ties keep index order)
    {
        ProfScope ps(ws, ST_DEPTH, st);
        uint32_t *ksorted = nullptr;
        VG_CUDA(ws, launch_radix_sort(ws->depth.p, nullptr, ws->skey[0].p, ws->sval[0].p, ws->skey[1].p,
                                      ws->sval[1].p, n, nullptr, 32, ws->hist.p, lookback_err_ptr(ws), &ksorted,
                                      &ws->perm, st, &ws->launches));
    }
    // 2. instance offsets in depth order
    {
        ProfScope ps(ws, ST_SCAN, st);
        VG_CUDA(ws, launch_scan_gather(ws->count.p, ws->perm, ws->offsets.p, n, ws->scan_tmp.p, total64_ptr(ws),
                                       fixed ? (unsigned long long)ws->capacity : ~0ull, lookback_err_ptr(ws), st,
                                       &ws->launches));
    }
    // The instance count: read back (one synchronisation), or, with a fixed capacity, left on
    // the device; the kernels below then cover the capacity and read the count themselves.
    // Without a fixed capacity, when an earlier call left instance buffers, the rest of the
    // binning is enqueued on them first in the same device-count form (kernels stop at the
    // capacity) and the count is read back afterwards, so the GPU keeps working through the
    // readback; a step with more instances than the buffers hold is binned again after they grow.
    auto bin_rest = [&](long long total, const unsigned long long *total_dev) -> vg_status {
        // 3. duplicate in depth order, 4. stable sort by tile id, 5. per-tile ranges
        {
            ProfScope ps(ws, ST_DUP, st);
            VG_CUDA(ws, launch_duplicate(ws->perm, ws->offsets.p, ws->rect.p, ws->views.p, n, ws->g.n, ws->ikey[0].p,
                                         ws->ival[0].p, ws->capacity, st, &ws->launches));
        }
        {
            ProfScope ps(ws, ST_TILE, st);
            VG_CUDA(ws, launch_radix_sort(ws->ikey[0].p, ws->ival[0].p, ws->ikey[1].p, ws->ival[1].p, ws->ikey[0].p,
                                          ws->ival[0].p, total, total_dev, bits_for(ws->n_tiles), ws->hist.p,
                                          lookback_err_ptr(ws), &ws->inst_key, &ws->inst_item, st, &ws->launches));
        }
        VG_TRY(ensure(ws, ws->ranges, (size_t)ws->n_tiles, "tile ranges"));
        VG_TRY(ensure(ws, ws->tord, (size_t)ws->n_tiles, "tile order"));
        {
            ProfScope ps(ws, ST_RANGES, st);
            VG_CUDA(ws, launch_ranges(ws->inst_key, total, total_dev, ws->ranges.p, ws->n_tiles, st, &ws->launches));
            VG_CUDA(ws, launch_tile_order(ws->ranges.p, nullptr, ws->n_tiles, ws->tord.p, st, &ws->launches));
            ws->tile_order = ws->tord.p;
            ws->tile_order_bwd = nullptr;   // until a forward has measured the replay lengths
        }
        return VG_OK;
    };
    if (fixed) {
        if (ws->capacity <= 0 || !ws->ikey[1].p)
            return fail(ws, VG_ERR_CAPACITY, "fixed capacity: reserve instances with vg_workspace_reserve first");
        ws->n_inst = -1;   // known on the device only
        VG_TRY(bin_rest(ws->capacity, total64_ptr(ws)));
    } else {
        long long total;
        if (ahead) {
            VG_TRY(read_total_start(ws, st));
            VG_TRY(bin_rest(ws->capacity, total64_ptr(ws)));
            VG_TRY(read_total_finish(ws, st, &total));
        } else {
            VG_TRY(read_total(ws, st, &total));
        }
        if (total > (long long)(1u << 30) - 1)
            return fail(ws, VG_ERR_INVALID_ARG, "more than 2^30 - 1 (tile, Gaussian) instances");
        if (!ahead || total > ws->capacity) {
            // the binning enqueued ahead still uses the buffers about to be replaced
            if (ahead) VG_CUDA(ws, cudaStreamSynchronize(st));
            VG_TRY(reserve_instances(ws, total));
            VG_TRY(bin_rest(total, nullptr));
        }
        ws->n_inst = total;
    }
    ws->stage = 2;
    return VG_OK;
}

static vg_status render_fwd_impl(vg_workspace *ws, float *rgb, float *T_final, void *stream, bool rgb_optional,
                                 const L2Fused &l2 = L2Fused{}) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (ws->stage < 2) return fail(ws, VG_ERR_STATE, "vg_render_fwd before vg_bin_sort");
    if (!rgb && ws->n_pixels > 0 && !rgb_optional) return fail(ws, VG_ERR_INVALID_ARG, "rgb is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (l2.target) VG_CUDA(ws, cudaMemsetAsync(l2.loss, 0, sizeof(float), st));
    VG_TRY(ensure(ws, ws->S_fin, (size_t)ws->n_pixels, "pixel state"));
    VG_TRY(ensure(ws, ws->T_fin, (size_t)ws->n_pixels, "pixel state"));
    VG_TRY(ensure(ws, ws->nlast, (size_t)ws->n_pixels, "pixel state"));
    unsigned long long *pc = nullptr;
    if (ws->opts.flags & VG_FLAG_COUNT_PAIRS) {
        pc = ws->counters.p + 1;
        VG_CUDA(ws, cudaMemsetAsync(pc, 0, 2 * sizeof(unsigned long long), st));
    }
    VG_TRY(ensure(ws, ws->treplay, (size_t)std::max<long long>(ws->n_tiles, 1), "tile replay lengths"));
    VG_TRY(ensure(ws, ws->tord_bwd, (size_t)std::max<long long>(ws->n_tiles, 1), "backward tile order"));
    {
        ProfScope ps(ws, ST_FWD, st);
        VG_CUDA(ws, cudaMemsetAsync(ws->treplay.p, 0, sizeof(uint32_t) * (size_t)ws->n_tiles, st));
        VG_CUDA(ws, launch_render_fwd(ws->views.p, ws->tile_view.p, (const int *)ws->tile_order, ws->n_tiles,
                                      ws->ranges.p, ws->inst_item, ws->rec.p, ws->prect.p, ws->bp, ws->ppt_fwd, rgb, T_final,
                                      ws->T_fin.p, ws->S_fin.p, ws->nlast.p, ws->treplay.p, pc, l2, st, &ws->launches));
        // the backward's order: longest replay (largest last blended position in the tile) first
        VG_CUDA(ws, launch_tile_order(nullptr, ws->treplay.p, ws->n_tiles, ws->tord_bwd.p, st, &ws->launches));
        ws->tile_order_bwd = ws->tord_bwd.p;
    }
    ws->stage = 3;
    return VG_OK;
}

vg_status vg_render_fwd(vg_workspace *ws, float *rgb, float *T_final, void *stream) {
    return render_fwd_impl(ws, rgb, T_final, stream, false);
}

vg_status vg_render_fwd_l2(vg_workspace *ws, float *rgb, float *T_final, const float *target, float scale,
                           float *loss, float *dL_drgb, void *stream) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (!loss || (ws->n_pixels > 0 && (!rgb || !target || !dL_drgb)))
        return fail(ws, VG_ERR_INVALID_ARG, "invalid loss arguments");
    if (ws->n_pixels == 0) {   // no pixel: the loss is zero (the forward still records its state)
        VG_CUDA(ws, cudaMemsetAsync(loss, 0, sizeof(float), (cudaStream_t)stream));
        return render_fwd_impl(ws, rgb, T_final, stream, false);
    }
    return render_fwd_impl(ws, rgb, T_final, stream, false, L2Fused{target, dL_drgb, loss, scale});
}

static vg_status render_bwd_impl(vg_workspace *ws, const float *dL_drgb, const float *dL_dT, float *dmu, float *dscale,
                                 float *dquat, float *dkappa, float *dsh, void *stream, bool drgb_optional) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (ws->stage < 3) return fail(ws, VG_ERR_STATE, "vg_render_bwd before vg_render_fwd");
    if ((!dL_drgb && ws->n_pixels > 0 && !drgb_optional) || (ws->g.n > 0 && (!dmu || !dscale || !dquat || !dkappa)))
        return fail(ws, VG_ERR_INVALID_ARG, "a gradient pointer is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t acc_n = (size_t)ws->n_items * kGradN;
    VG_TRY(ensure(ws, ws->grad, acc_n, "gradient accumulators"));
    const bool clean = ws->grad_zero_p == ws->grad.p && ws->grad_zero_n >= acc_n;
    ws->grad_zero_n = 0;   // until the chain below has run
    if (ws->n_items > 0 && !clean) VG_CUDA(ws, cudaMemsetAsync(ws->grad.p, 0, sizeof(float) * acc_n, st));
    unsigned long long *pc = nullptr;
    if (ws->opts.flags & VG_FLAG_COUNT_PAIRS) {
        pc = ws->counters.p + 3;
        VG_CUDA(ws, cudaMemsetAsync(pc, 0, 2 * sizeof(unsigned long long), st));
    }
    {
        ProfScope ps(ws, ST_BWD, st);
        VG_CUDA(ws, launch_render_bwd(ws->views.p, ws->tile_view.p, (const int *)bwd_order(ws), ws->n_tiles,
                                      ws->ranges.p, ws->inst_item, ws->rec.p, ws->prect.p, ws->bp, ws->ppt_bwd,
                                      ws->T_fin.p,
                                      ws->S_fin.p, ws->nlast.p, dL_drgb, dL_dT, ws->grad.p, pc, lookback_err_ptr(ws),
                                      st, &ws->launches));
    }
    {
        // the chain writes every Gaussian's gradient: overwriting with VG_FLAG_GRAD_ZERO, else adding
        ProfScope ps(ws, ST_CHAIN, st);
        VG_CUDA(ws, launch_chain(ws->g, ws->views.p, ws->n_views, ws->grad.p, (ws->opts.flags & VG_FLAG_GRAD_ZERO) ? 1 : 0,
                                 dmu, dscale, dquat, dkappa, dsh, st, &ws->launches));
    }
    ws->grad_zero_p = ws->grad.p;   // the chain left the accumulator zero
    ws->grad_zero_n = acc_n;
    return VG_OK;
}

vg_status vg_render_bwd(vg_workspace *ws, const float *dL_drgb, const float *dL_dT, float *dmu, float *dscale,
                        float *dquat, float *dkappa, float *dsh, void *stream) {
    return render_bwd_impl(ws, dL_drgb, dL_dT, dmu, dscale, dquat, dkappa, dsh, stream, false);
}

vg_status vg_project_cone(vg_workspace *ws, const vg_gaussians *g, const vg_camera *cams, int32_t n_views,
                          const vg_opts *opts, float *proj, const float *dL_dproj, float *dmu, float *dscale,
                          float *dquat, float *dkappa, void *stream) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (!opts) return fail(ws, VG_ERR_INVALID_ARG, "opts is NULL");
    if (opts->flags & VG_FLAG_SPLAT) return fail(ws, VG_ERR_INVALID_ARG, "the cone beam has no splat mode");
    // With no skip, clamp or early stop the blend's final transmittance is exp(-sum tau): the
    // cone-beam projection.  Its gradient is the blend's dL/dT_final term alone.
    vg_opts o = *opts;
    o.alpha_min = 0.0f;
    o.tau_max = INFINITY;
    o.T_stop = 0.0f;
    o.bg[0] = o.bg[1] = o.bg[2] = 0.0f;
    o.softplus_beta = 0.0f;
    vg_gaussians gd = g ? *g : vg_gaussians{};
    gd.sh = nullptr;   // density only
    gd.sh_degree = 0;
    VG_TRY(preprocess_impl(ws, g ? &gd : nullptr, cams, n_views, &o, stream, false));
    VG_TRY(vg_bin_sort(ws, stream));
    if (!proj && ws->n_pixels > 0) return fail(ws, VG_ERR_INVALID_ARG, "proj is NULL");
    VG_TRY(render_fwd_impl(ws, nullptr, proj, stream, true));
    if (dL_dproj) VG_TRY(render_bwd_impl(ws, nullptr, dL_dproj, dmu, dscale, dquat, dkappa, nullptr, stream, true));
    return VG_OK;
}

vg_status vg_ray_march(vg_workspace *ws, float t_near, float t_far, int32_t n_samples, const float *raster_rgb,
                       float *rgb, float *T, float *err_map, void *stream) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (ws->stage < 2) return fail(ws, VG_ERR_STATE, "vg_ray_march before vg_bin_sort");
    if (ws->g.splat) return fail(ws, VG_ERR_INVALID_ARG, "the ray march needs the default (volumetric) mode");
    if (!(t_near >= 0.0f) || !(t_far > t_near) || !std::isfinite(t_far))
        return fail(ws, VG_ERR_INVALID_ARG, "need 0 <= t_near < t_far, finite");
    if (n_samples < 1 || n_samples > (1 << 20)) return fail(ws, VG_ERR_INVALID_ARG, "n_samples must be 1..2^20");
    if (err_map && !raster_rgb) return fail(ws, VG_ERR_INVALID_ARG, "err_map needs raster_rgb");
    cudaStream_t st = (cudaStream_t)stream;
    VG_TRY(ensure(ws, ws->march_E, (size_t)ws->n_items, "ray-march scratch"));
    ProfScope ps(ws, ST_MARCH, st);
    VG_CUDA(ws, launch_ray_march(ws->g, ws->views.p, ws->tile_view.p, ws->n_tiles, ws->bp.tile_px, ws->n_items,
                                 ws->ranges.p,
                                 ws->inst_item, ws->rec.p, ws->count.p, ws->prect.p, ws->march_E.p, t_near, t_far,
                                 n_samples, ws->opts.T_stop, ws->opts.bg, raster_rgb, rgb, T, err_map, st,
                                 &ws->launches));
    return VG_OK;
}

vg_status vg_query_density(vg_workspace *ws, const vg_gaussians *g, const vg_grid *grid, const vg_opts *opts,
                           float *out, void *stream) {
    if (!ws) return VG_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    VG_TRY(check_gauss(ws, g, false));
    if (!grid || !opts) return fail(ws, VG_ERR_INVALID_ARG, "grid or opts is NULL");
    if (!finite_pos(opts->tau_cut)) return fail(ws, VG_ERR_INVALID_ARG, "tau_cut (sigma_cut) must be finite and > 0");
    if (opts->flags & VG_FLAG_SPLAT) return fail(ws, VG_ERR_INVALID_ARG, "the density query has no splat mode");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || grid->nx > 32767 || grid->ny > 32767 || grid->nz > 32767)
        return fail(ws, VG_ERR_INVALID_ARG, "grid sizes must be 1..32767");
    for (int a = 0; a < 3; ++a)
        if (!finite_pos(grid->voxel[a]) || !std::isfinite(grid->origin[a]))
            return fail(ws, VG_ERR_INVALID_ARG, "invalid grid origin or voxel size");
    if (!out) return fail(ws, VG_ERR_INVALID_ARG, "out is NULL");
    VoxelGrid vgd;
    vgd.ox = grid->origin[0];
    vgd.oy = grid->origin[1];
    vgd.oz = grid->origin[2];
    vgd.vx = grid->voxel[0];
    vgd.vy = grid->voxel[1];
    vgd.vz = grid->voxel[2];
    vgd.nx = grid->nx;
    vgd.ny = grid->ny;
    vgd.nz = grid->nz;
    vgd.bx = (grid->nx + 7) / 8;
    vgd.by = (grid->ny + 7) / 8;
    vgd.bz = (grid->nz + 7) / 8;
    const long long bricks = (long long)vgd.bx * vgd.by * vgd.bz, n = g->n;
    if (bricks >= (1LL << 30)) return fail(ws, VG_ERR_INVALID_ARG, "too many bricks");
    ws->opts = *opts;
    ws->g = to_in(g);
    ws->g.sh = nullptr;
    ws->g.density_theta = (opts->flags & VG_FLAG_DENSITY_THETA) ? 1 : 0;
    ws->stage = 0;   // the render state of this workspace is overwritten below
    ws->views_valid = false;
    VG_TRY(reserve_items(ws, n));
    VG_TRY(reserve_sort_scratch(ws, n));
    VG_TRY(ensure(ws, ws->vbox, (size_t)n * 2, "voxel boxes"));
    {
        ProfScope ps(ws, ST_PRE, st);
        VG_CUDA(ws, launch_voxel_pre(ws->g, vgd, opts->tau_cut, ws->rec.p, ws->vbox.p, ws->count.p, st,
                                     &ws->launches));
    }
    {
        ProfScope ps(ws, ST_SCAN, st);
        VG_CUDA(ws, launch_scan_gather(ws->count.p, nullptr, ws->offsets.p, n, ws->scan_tmp.p, total64_ptr(ws), ~0ull,
                                       lookback_err_ptr(ws), st, &ws->launches));
    }
    long long total = 0;
    VG_TRY(read_total(ws, st, &total));
    if (total > (long long)(1u << 30) - 1) return fail(ws, VG_ERR_INVALID_ARG, "more than 2^30 - 1 (brick, Gaussian) pairs");
    VG_TRY(reserve_instances(ws, total));
    ws->n_inst = total;
    VG_TRY(ensure(ws, ws->ranges, (size_t)bricks, "brick ranges"));
    uint32_t *keys = nullptr, *vals = nullptr;
    {
        ProfScope ps(ws, ST_DUP, st);
        VG_CUDA(ws, launch_voxel_dup(ws->offsets.p, ws->vbox.p, vgd, n, ws->ikey[0].p, ws->ival[0].p, ws->capacity,
                                     st, &ws->launches));
    }
    {
        ProfScope ps(ws, ST_TILE, st);
        VG_CUDA(ws, launch_radix_sort(ws->ikey[0].p, ws->ival[0].p, ws->ikey[1].p, ws->ival[1].p, ws->ikey[0].p,
                                      ws->ival[0].p, total, nullptr, bits_for(bricks), ws->hist.p,
                                      lookback_err_ptr(ws), &keys, &vals, st, &ws->launches));
    }
    {
        ProfScope ps(ws, ST_RANGES, st);
        VG_CUDA(ws, launch_ranges(keys, total, nullptr, ws->ranges.p, bricks, st, &ws->launches));
    }
    {
        ProfScope ps(ws, ST_VOXEL, st);
        VG_CUDA(ws, launch_voxel_eval(ws->ranges.p, vals, ws->rec.p, ws->vbox.p, vgd, out, st, &ws->launches));
    }
    return VG_OK;
}

// ---------------------------------------------------------------- allocation-free backward
// The per-item gradient accumulator of vg_render_bwd_noalloc: a fixed array that the
// library's module brings onto every device it is loaded on.  Host code must not pass the
// symbol itself to a kernel (in host code it names a host-side stand-in); the device
// address comes from cudaGetSymbolAddress, looked up in the current context on every call.
static __device__ __align__(256) float g_noalloc_acc[(size_t)VG_NOALLOC_MAX_ITEMS * kGradN];

namespace {
// The array's device address in the current context.  cudaGetSymbolAddress allocates nothing; it
// is called on every call, so the address stays right after cudaDeviceReset (which unloads the
// module: the next call loads it again, with the array possibly elsewhere).
vg_status noalloc_scratch(vg_workspace *ws, float **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_acc);
    if (e != cudaSuccess || !p)
        return fail(ws, VG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = (float *)p;
    return VG_OK;
}
}  // namespace

vg_status vg_render_bwd_noalloc(vg_workspace *ws, const float *dL_drgb, const float *dL_dT, float *dmu,
                                float *dscale, float *dquat, float *dkappa, float *dsh, void *stream) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (ws->stage < 3) return fail(ws, VG_ERR_STATE, "vg_render_bwd_noalloc before vg_render_fwd");
    if ((!dL_drgb && ws->n_pixels > 0) || (ws->g.n > 0 && (!dmu || !dscale || !dquat || !dkappa)))
        return fail(ws, VG_ERR_INVALID_ARG, "a gradient pointer is NULL");
    if (ws->n_items > (long long)VG_NOALLOC_MAX_ITEMS)
        return fail(ws, VG_ERR_INVALID_ARG,
                    "views x Gaussians = " + std::to_string(ws->n_items) + " exceeds VG_NOALLOC_MAX_ITEMS = " +
                        std::to_string((long long)VG_NOALLOC_MAX_ITEMS) + " of the allocation-free backward");
    cudaStream_t st = (cudaStream_t)stream;
    float *acc = nullptr;
    VG_TRY(noalloc_scratch(ws, &acc));
    // the array keeps the previous call's sums: clear the part this call accumulates into
    if (ws->n_items > 0) VG_CUDA(ws, cudaMemsetAsync(acc, 0, sizeof(float) * (size_t)ws->n_items * kGradN, st));
    unsigned long long *pc = nullptr;   // the workspace's own counters: nothing is allocated for them
    if (ws->opts.flags & VG_FLAG_COUNT_PAIRS) {
        pc = ws->counters.p + 3;
        VG_CUDA(ws, cudaMemsetAsync(pc, 0, 2 * sizeof(unsigned long long), st));
    }
    {
        ProfScope ps(ws, ST_BWD, st);
        VG_CUDA(ws, launch_render_bwd(ws->views.p, ws->tile_view.p, (const int *)bwd_order(ws), ws->n_tiles,
                                      ws->ranges.p, ws->inst_item, ws->rec.p, ws->prect.p, ws->bp, ws->ppt_bwd,
                                      ws->T_fin.p, ws->S_fin.p, ws->nlast.p, dL_drgb, dL_dT, acc, pc,
                                      lookback_err_ptr(ws), st, &ws->launches));
    }
    {
        ProfScope ps(ws, ST_CHAIN, st);
        VG_CUDA(ws, launch_chain(ws->g, ws->views.p, ws->n_views, acc, (ws->opts.flags & VG_FLAG_GRAD_ZERO) ? 1 : 0,
                                 dmu, dscale, dquat, dkappa, dsh, st, &ws->launches));
    }
    return VG_OK;
}

vg_status vg_pipe_peak(vg_workspace *ws, int32_t pipe, float min_ms, double *ops_per_s, float *ms, void *stream) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if ((pipe != 0 && pipe != 1) || !ops_per_s || !(min_ms > 0.0f) || !(min_ms <= 10000.0f))
        return fail(ws, VG_ERR_INVALID_ARG, "pipe must be 0 (FMA) or 1 (ex2), min_ms in (0, 10000]");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    VG_CUDA(ws, cudaEventCreate(&a));
    cudaError_t e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return fail(ws, VG_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    }
    // one short launch to warm up and size the timed ones, then three timed launches of about
    // min_ms each; the fastest counts
    int iters = 64;
    double ops = 0.0, best = 0.0;
    float best_ms = 0.0f;
    for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) e = launch_pipe_peak(pipe, iters, &ops, st);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        ws->launches += 1;
        if (e != cudaSuccess) break;
        if (r >= 2 && t > 0.0f && ops / (t * 1e-3) > best) {
            best = ops / (t * 1e-3);
            best_ms = t;
        }
        if (r < 2 && t > 0.0f)   // resize towards min_ms per launch
            iters = (int)std::min(1.0e8, std::max(16.0, iters * (double)min_ms / t));
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return fail(ws, VG_ERR_CUDA, std::string("pipe peak: ") + cudaGetErrorString(e));
    *ops_per_s = best;
    if (ms) *ms = best_ms;
    return VG_OK;
}

vg_status vg_selftest_timeout(vg_workspace *ws, int32_t which, int32_t spin_limit, void *stream) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (which < 0 || which > 2)
        return fail(ws, VG_ERR_INVALID_ARG, "which must be 0 (scan), 1 (radix pass) or 2 (backward ring)");
    if (spin_limit < 1 || spin_limit > (1 << 20)) return fail(ws, VG_ERR_INVALID_ARG, "spin_limit must be 1..2^20");
    cudaStream_t st = (cudaStream_t)stream;
    if (which == 2) {
        VG_CUDA(ws, launch_ring_selftest(spin_limit, lookback_err_ptr(ws), st, &ws->launches));
        return VG_OK;
    }
    VG_TRY(ensure(ws, ws->scan_tmp, 4, "self-test status words"));
    // a predecessor that never publishes: its status word stays zero for the whole wait
    VG_CUDA(ws, cudaMemsetAsync(ws->scan_tmp.p, 0, 4 * sizeof(uint32_t), st));
    VG_CUDA(ws, launch_lookback_selftest(ws->scan_tmp.p, which, spin_limit, lookback_err_ptr(ws), ws->counters.p + 5,
                                         st, &ws->launches));
    return VG_OK;
}

// Parallel-beam projection in angle batches.  With dL_dproj the backward follows each batch's
// projection; with target (and dL_dproj NULL) the L2 loss scale * sum (proj - target)^2 is
// accumulated into *loss and its gradient drives the backward, so that each batch is
// preprocessed, binned and projected once for the whole training step.
static vg_status tomo_impl(vg_workspace *ws, const vg_gaussians *g, const vg_beam *beam, const vg_opts *opts,
                           float *proj, const float *dL_dproj, const float *target, float scale, float *loss,
                           float *dmu, float *dscale, float *dquat, float *dkappa, cudaStream_t st) {
    const bool fused = target != nullptr;
    const bool backward = dL_dproj != nullptr || fused;
    const bool proj_given = dL_dproj && !fused && (opts && (opts->flags & VG_FLAG_PROJ_GIVEN));
    VG_TRY(check_gauss(ws, g, false));
    if (!beam || beam->n_angles < 1 || !beam->angles || beam->det_w <= 0 || beam->det_h <= 0 ||
        !finite_pos(beam->pitch_u) || !finite_pos(beam->pitch_v) || !std::isfinite(beam->u0) ||
        !std::isfinite(beam->v0))
        return fail(ws, VG_ERR_INVALID_ARG, "invalid beam geometry");
    if (!opts || !finite_pos(opts->tau_cut)) return fail(ws, VG_ERR_INVALID_ARG, "opts->tau_cut must be finite and > 0");
    if (opts->flags & VG_FLAG_SPLAT) return fail(ws, VG_ERR_INVALID_ARG, "tomography has no splat mode");
    if (!proj) return fail(ws, VG_ERR_INVALID_ARG, "proj is NULL");
    if (backward && g->n > 0 && (!dmu || !dscale || !dquat || !dkappa))
        return fail(ws, VG_ERR_INVALID_ARG, "a gradient pointer is NULL");
    if (fused && (!loss || !std::isfinite(scale))) return fail(ws, VG_ERR_INVALID_ARG, "loss is NULL or scale not finite");
    const int A = beam->n_angles, N = g->n;
    const int tiles_x = (beam->det_w + kTile - 1) / kTile, tiles_y = (beam->det_h + kTile - 1) / kTile;
    if (tiles_x > 32767 || tiles_y > 32767) return fail(ws, VG_ERR_INVALID_ARG, "detector too large");
    const long long tpv = (long long)tiles_x * tiles_y;
    const long long det_px = (long long)beam->det_w * beam->det_h;
    ws->opts = *opts;
    ws->g = to_in(g);
    ws->g.density_theta = (opts->flags & VG_FLAG_DENSITY_THETA) ? 1 : 0;
    ws->stage = 0;   // the render state of this workspace is overwritten below
    ws->views_valid = false;
    std::vector<float> cs(2 * (size_t)A);
    for (int a = 0; a < A; ++a) {
        if (!std::isfinite(beam->angles[a])) return fail(ws, VG_ERR_INVALID_ARG, "non-finite beam angle");
        cs[2 * a] = (float)std::cos((double)beam->angles[a]);
        cs[2 * a + 1] = (float)std::sin((double)beam->angles[a]);
    }
    VG_TRY(ensure(ws, ws->tomo_cs, cs.size(), "beam angles"));
    VG_CUDA(ws, cudaMemcpyAsync(ws->tomo_cs.p, cs.data(), cs.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    if (fused) VG_CUDA(ws, cudaMemsetAsync(loss, 0, sizeof(float), st));
    if (backward && (opts->flags & VG_FLAG_GRAD_ZERO) && N > 0) {
        VG_CUDA(ws, cudaMemsetAsync(dmu, 0, (size_t)N * 3 * sizeof(float), st));
        VG_CUDA(ws, cudaMemsetAsync(dscale, 0, (size_t)N * 3 * sizeof(float), st));
        VG_CUDA(ws, cudaMemsetAsync(dquat, 0, (size_t)N * 4 * sizeof(float), st));
        VG_CUDA(ws, cudaMemsetAsync(dkappa, 0, (size_t)N * sizeof(float), st));
    }
    // angles are processed in batches of at most ~4M (angle, Gaussian) items
    const long long budget = 1LL << 22;
    int batch = N > 0 ? (int)std::max<long long>(1, std::min<long long>(A, budget / N)) : A;
    while ((long long)batch * tpv >= (1LL << 30) && batch > 1) batch /= 2;
    for (int a0 = 0; a0 < A; a0 += batch) {
        const int nb = std::min(batch, A - a0);
        const long long items = (long long)nb * N;
        if (items >= 0xFFFFFFFFLL) return fail(ws, VG_ERR_INVALID_ARG, "angles x Gaussians per batch must be < 2^32");
        const long long n_tiles = (long long)nb * tpv;
        VG_TRY(reserve_items(ws, items));
        VG_TRY(reserve_sort_scratch(ws, items));
        std::vector<ViewInfo> vh((size_t)nb);
        for (int v = 0; v < nb; ++v) {
            memset(&vh[v], 0, sizeof(ViewInfo));
            vh[v].W = beam->det_w;
            vh[v].H = beam->det_h;
            vh[v].tw = kTile;
            vh[v].th = kTile;
            vh[v].tiles_x = tiles_x;
            vh[v].tiles_y = tiles_y;
            vh[v].tile_base = (int)(v * tpv);
            vh[v].pix_base = (long long)v * det_px;
        }
        VG_TRY(ensure(ws, ws->views, vh.size(), "views"));
        VG_CUDA(ws, cudaMemcpyAsync(ws->views.p, vh.data(), vh.size() * sizeof(ViewInfo), cudaMemcpyHostToDevice, st));
        if (items > 0) {
            ProfScope ps(ws, ST_PRE, st);
            VG_CUDA(ws, cudaMemsetAsync(ws->depth.p, 0xFF, sizeof(uint32_t) * (size_t)items, st));
            VG_CUDA(ws, launch_tomo_preprocess(ws->g, ws->tomo_cs.p + 2 * (size_t)a0, nb, beam->det_w, beam->det_h,
                                               beam->pitch_u, beam->pitch_v, beam->u0, beam->v0, opts->tau_cut,
                                               ws->rec.p, ws->count.p, ws->rect.p, ws->prect.p, st, &ws->launches));
        }
        {
            ProfScope ps(ws, ST_SCAN, st);
            VG_CUDA(ws, launch_scan_gather(ws->count.p, nullptr, ws->offsets.p, items, ws->scan_tmp.p,
                                           total64_ptr(ws), ~0ull, lookback_err_ptr(ws), st, &ws->launches));
        }
        long long total = 0;
        VG_TRY(read_total(ws, st, &total));
        if (total > (long long)(1u << 30) - 1)
            return fail(ws, VG_ERR_INVALID_ARG, "more than 2^30 - 1 (tile, Gaussian) instances in an angle batch");
        VG_TRY(reserve_instances(ws, total));
        {
            ProfScope ps(ws, ST_DUP, st);
            VG_CUDA(ws, launch_duplicate(nullptr, ws->offsets.p, ws->rect.p, ws->views.p, items, N > 0 ? N : 1,
                                         ws->ikey[0].p, ws->ival[0].p, ws->capacity, st, &ws->launches));
        }
        {
            ProfScope ps(ws, ST_TILE, st);
            VG_CUDA(ws, launch_radix_sort(ws->ikey[0].p, ws->ival[0].p, ws->ikey[1].p, ws->ival[1].p, ws->ikey[0].p,
                                          ws->ival[0].p, total, nullptr, bits_for(n_tiles), ws->hist.p,
                                          lookback_err_ptr(ws), &ws->inst_key, &ws->inst_item, st, &ws->launches));
        }
        VG_TRY(ensure(ws, ws->ranges, (size_t)n_tiles, "tile ranges"));
        {
            ProfScope ps(ws, ST_RANGES, st);
            VG_CUDA(ws, launch_ranges(ws->inst_key, total, nullptr, ws->ranges.p, n_tiles, st, &ws->launches));
        }
        float *proj_b = proj + (size_t)a0 * det_px;
        if (!proj_given) {
            ProfScope ps(ws, ST_TFWD, st);
            VG_CUDA(ws, launch_tomo_fwd(ws->ranges.p, n_tiles, tiles_x, (int)tpv, beam->det_w, beam->det_h,
                                        ws->inst_item, ws->rec.p, ws->prect.p, proj_b, st, &ws->launches));
        }
        const float *dl_b = dL_dproj ? dL_dproj + (size_t)a0 * det_px : nullptr;
        if (fused) {   // the batch's share of the loss and its gradient dL/dproj
            VG_TRY(ensure(ws, ws->tomo_dl, (size_t)nb * det_px, "loss gradient"));
            ProfScope ps(ws, ST_LOSS, st);
            VG_CUDA(ws, launch_l2_loss_acc(proj_b, target + (size_t)a0 * det_px, (long long)nb * det_px, scale, loss,
                                           ws->tomo_dl.p, st, &ws->launches));
            dl_b = ws->tomo_dl.p;
        }
        if (backward && items > 0) {
            VG_TRY(ensure(ws, ws->grad, (size_t)items * 8, "gradient accumulators"));
            ws->grad_zero_n = 0;   // the tomography backward leaves its sums in the accumulator
            VG_CUDA(ws, cudaMemsetAsync(ws->grad.p, 0, sizeof(float) * (size_t)items * 8, st));
            ProfScope ps(ws, ST_TBWD, st);
            VG_CUDA(ws, launch_tomo_bwd(ws->ranges.p, n_tiles, tiles_x, (int)tpv, beam->det_w, beam->det_h,
                                        ws->inst_item, ws->rec.p, ws->prect.p, proj_b, dl_b, ws->grad.p, st,
                                        &ws->launches));
            VG_CUDA(ws, launch_tomo_chain(ws->g, ws->tomo_cs.p, A, (long long)a0 * N, items, beam->pitch_u,
                                          beam->pitch_v, beam->u0, beam->v0, ws->grad.p, dmu, dscale, dquat, dkappa,
                                          st, &ws->launches));
        }
        ws->n_items = items;
        ws->n_tiles = n_tiles;
        ws->n_inst = total;
        ws->n_views = nb;
        ws->n_pixels = (long long)nb * det_px;
    }
    ws->stage = 0;
    ws->tomo_read = true;
    return VG_OK;
}

vg_status vg_project_tomo(vg_workspace *ws, const vg_gaussians *g, const vg_beam *beam, const vg_opts *opts,
                          float *proj, const float *dL_dproj, float *dmu, float *dscale, float *dquat, float *dkappa,
                          void *stream) {
    if (!ws) return VG_ERR_INVALID_ARG;
    return tomo_impl(ws, g, beam, opts, proj, dL_dproj, nullptr, 0.0f, nullptr, dmu, dscale, dquat, dkappa,
                     (cudaStream_t)stream);
}

vg_status vg_tomo_l2_step(vg_workspace *ws, const vg_gaussians *g, const vg_beam *beam, const vg_opts *opts,
                          const float *target, float scale, float *proj, float *loss, float *dmu, float *dscale,
                          float *dquat, float *dkappa, void *stream) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (!target) return fail(ws, VG_ERR_INVALID_ARG, "target is NULL");
    return tomo_impl(ws, g, beam, opts, proj, nullptr, target, scale, loss, dmu, dscale, dquat, dkappa,
                     (cudaStream_t)stream);
}

vg_status vg_l2_loss(vg_workspace *ws, const float *x, const float *y, int64_t n, float scale, float *loss,
                     float *grad, void *stream) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (n < 0 || !loss || (n > 0 && (!x || !y || !grad))) return fail(ws, VG_ERR_INVALID_ARG, "invalid loss arguments");
    ProfScope ps(ws, ST_LOSS, (cudaStream_t)stream);
    VG_CUDA(ws, launch_l2_loss(x, y, n, scale, loss, grad, (cudaStream_t)stream, &ws->launches));
    return VG_OK;
}

vg_status vg_autotune(vg_workspace *ws, int32_t reps, int32_t *ppt_fwd, int32_t *ppt_bwd, int32_t *chunk_fwd,
                      int32_t *chunk_bwd, int32_t *tile_w, int32_t *tile_h, void *stream) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (ws->stage < 2 || !ws->views_valid) return fail(ws, VG_ERR_STATE, "vg_autotune before vg_bin_sort");
    if (reps < 1) reps = 3;
    cudaStream_t st = (cudaStream_t)stream;
    VG_TRY(ensure(ws, ws->S_fin, (size_t)ws->n_pixels, "pixel state"));
    VG_TRY(ensure(ws, ws->T_fin, (size_t)ws->n_pixels, "pixel state"));
    VG_TRY(ensure(ws, ws->nlast, (size_t)ws->n_pixels, "pixel state"));
    VG_TRY(ensure(ws, ws->grad, (size_t)ws->n_items * kGradN, "gradient accumulators"));
    // scratch image and loss gradient (zero: the timing does not depend on the values)
    float *rgb = nullptr, *dl = nullptr;
    const size_t px3 = (size_t)std::max<long long>(ws->n_pixels, 1) * 3;
    VG_CUDA(ws, cudaMalloc((void **)&rgb, px3 * sizeof(float)));
    cudaError_t e = cudaMalloc((void **)&dl, px3 * sizeof(float));
    if (e != cudaSuccess) {
        cudaFree(rgb);
        return fail(ws, VG_ERR_OOM, "autotune scratch");
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    auto elapsed = [&]() {
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    };
    // The default tile shape first, another one taken only when it is faster by more than 2%
    // (the measured differences between shapes are often within the run-to-run spread); a
    // shape set in the options of the last vg_preprocess is kept.
    const int shapes[3][2] = {{16, 16}, {32, 16}, {16, 8}};
    const int cur_tw = ws->views_h[0].tw, cur_th = ws->views_h[0].th;
    const bool fixed_shape = ws->opts.tile_w != 0;
    const int n_shapes = fixed_shape ? 1 : 3;
    const unsigned flags = ws->opts.flags;
    const int cand[3] = {1, 2, 4}, chunks[2] = {64, 128};
    float best_total = 1e30f;
    int pf = kDefaultPixelsFwd, pb = kDefaultPixelsBwd, cf = kDefaultChunk, cb = kDefaultChunk;
    int tw = cur_tw, th = cur_th, last_tw = cur_tw, last_th = cur_th;
    vg_status vs = VG_OK;
    e = cudaMemsetAsync(dl, 0, px3 * sizeof(float), st);
    for (int s = 0; s < n_shapes && e == cudaSuccess && vs == VG_OK; ++s) {
        const int sw = fixed_shape ? cur_tw : shapes[s][0], sh = fixed_shape ? cur_th : shapes[s][1];
        float t_bin = 0.0f;
        if (!fixed_shape) {
            // one binning that may grow the instance buffers, then the timed ones in the
            // fixed-capacity form (the device work of either form, without the count's readback)
            ws->opts.flags = flags & ~VG_FLAG_FIXED_CAPACITY;
            vs = retile(ws, sw, sh, st);
            if (vs == VG_OK) vs = vg_bin_sort(ws, st);
            ws->opts.flags = flags | VG_FLAG_FIXED_CAPACITY;
            last_tw = sw, last_th = sh;
            t_bin = 1e30f;
            for (int r = 0; r < reps && vs == VG_OK; ++r) {
                cudaEventRecord(a, st);
                vs = run_preprocess(ws, st);
                if (vs == VG_OK) vs = vg_bin_sort(ws, st);
                t_bin = std::min(t_bin, elapsed());
            }
            ws->opts.flags = flags;
            if (vs != VG_OK) break;
        }
        float best_f = 1e30f, best_b = 1e30f;
        int spf = pf, spb = pb, scf = cf, scb = cb;
        for (int i = 0; i < 6 && e == cudaSuccess; ++i) {
            BlendParams bp = ws->bp;
            bp.chunk_fwd = bp.chunk_bwd = chunks[i & 1];
            const int ppt = cand[i >> 1];
            float tf = 1e30f, tb = 1e30f;   // the fastest of the timed runs
            for (int r = 0; r <= reps && e == cudaSuccess; ++r) {   // the first round warms up
                cudaEventRecord(a, st);
                e = launch_render_fwd(ws->views.p, ws->tile_view.p, (const int *)ws->tile_order, ws->n_tiles,
                                      ws->ranges.p, ws->inst_item, ws->rec.p, ws->prect.p, bp, ppt, rgb, nullptr,
                                      ws->T_fin.p, ws->S_fin.p, ws->nlast.p, nullptr, nullptr, L2Fused{}, st,
                                      &ws->launches);
                float ms = elapsed();
                if (r) tf = std::min(tf, ms);
                if (e != cudaSuccess) break;
                ws->grad_zero_n = 0;   // timed backward passes without the chain leave sums behind
                e = cudaMemsetAsync(ws->grad.p, 0, sizeof(float) * (size_t)ws->n_items * kGradN, st);
                cudaEventRecord(a, st);
                if (e == cudaSuccess)
                    e = launch_render_bwd(ws->views.p, ws->tile_view.p, (const int *)ws->tile_order, ws->n_tiles,
                                          ws->ranges.p, ws->inst_item, ws->rec.p, ws->prect.p, bp, ppt, ws->T_fin.p,
                                          ws->S_fin.p, ws->nlast.p, dl, nullptr, ws->grad.p, nullptr,
                                          lookback_err_ptr(ws), st, &ws->launches);
                ms = elapsed();
                if (r) tb = std::min(tb, ms);
            }
            if (tf < best_f) best_f = tf, spf = ppt, scf = chunks[i & 1];
            if (tb < best_b) best_b = tb, spb = ppt, scb = chunks[i & 1];
        }
        const float total = t_bin + best_f + best_b;
        if (s == 0 || total < 0.98f * best_total)
            best_total = total, pf = spf, pb = spb, cf = scf, cb = scb, tw = sw, th = sh;
    }
    if (vs == VG_OK && e == cudaSuccess && (tw != last_tw || th != last_th)) {   // leave the chosen tiling binned
        ws->opts.flags = flags & ~VG_FLAG_FIXED_CAPACITY;
        vs = retile(ws, tw, th, st);
        if (vs == VG_OK) vs = vg_bin_sort(ws, st);
        ws->opts.flags = flags;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(rgb);
    cudaFree(dl);
    if (vs != VG_OK) return vs;
    if (e != cudaSuccess) return fail(ws, VG_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
    ws->tuned_fwd = ws->ppt_fwd = pf;
    ws->tuned_bwd = ws->ppt_bwd = pb;
    ws->tuned_chunk_fwd = ws->bp.chunk_fwd = cf;
    ws->tuned_chunk_bwd = ws->bp.chunk_bwd = cb;
    if (!fixed_shape) ws->tuned_tw = tw, ws->tuned_th = th;
    ws->stage = 2;   // the replay state no longer belongs to a vg_render_fwd of the caller
    if (ppt_fwd) *ppt_fwd = pf;
    if (ppt_bwd) *ppt_bwd = pb;
    if (chunk_fwd) *chunk_fwd = cf;
    if (chunk_bwd) *chunk_bwd = cb;
    if (tile_w) *tile_w = tw;
    if (tile_h) *tile_h = th;
    return VG_OK;
}

vg_status vg_query(vg_workspace *ws, vg_stats *out, void *stream) {
    if (!ws || !out) return VG_ERR_INVALID_ARG;
    VG_CUDA(ws, cudaStreamSynchronize((cudaStream_t)stream));
    unsigned long long c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    VG_CUDA(ws, cudaMemcpy(c, ws->counters.p, sizeof(c), cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof(*out));
    out->n_items = ws->n_items;
    out->n_visible = (int64_t)c[0];
    // with a fixed capacity the instance count lives on the device (c[6]); an overflow is latched
    out->n_instances = ws->n_inst >= 0 ? ws->n_inst : (int64_t)std::min<unsigned long long>(c[6], (unsigned long long)ws->capacity);
    out->n_tiles = ws->n_tiles;
    out->n_pixels = ws->n_pixels;
    out->instance_capacity = ws->capacity;
    out->n_pairs = (int64_t)c[1];
    out->n_blend = (int64_t)c[2];
    out->n_pairs_bwd = (int64_t)c[3];
    out->n_blend_bwd = (int64_t)c[4];
    out->launches = ws->launches;
    size_t bytes = ws->views.n * sizeof(ViewInfo) + ws->tile_view.n * 4 + ws->rec.n * 16 + ws->depth.n * 4 +
                   ws->count.n * 4 + ws->offsets.n * 4 + ws->rect.n * 8 + ws->ranges.n * 8 + ws->S_fin.n * 4 +
                   ws->T_fin.n * 4 + ws->nlast.n * 4 + ws->grad.n * 4 + ws->hist.n * 4 + ws->scan_tmp.n * 4;
    for (int k = 0; k < 2; ++k)
        bytes += (ws->skey[k].n + ws->sval[k].n + ws->ikey[k].n + ws->ival[k].n) * 4;
    out->device_bytes = (int64_t)bytes;
    ws->h_total[2] = (uint32_t)c[7];
    return latched_status(ws, (cudaStream_t)stream);
}

vg_status vg_profile_enable(vg_workspace *ws, int32_t enable) {
    if (!ws) return VG_ERR_INVALID_ARG;
    for (auto &r : ws->prof) {
        ws->prof_pool.push_back(r.a);
        ws->prof_pool.push_back(r.b);
    }
    ws->prof.clear();
    ws->prof_on = enable != 0;
    return VG_OK;
}

vg_status vg_profile_stages(vg_workspace *ws, uint32_t stage_mask) {
    if (!ws) return VG_ERR_INVALID_ARG;
    ws->prof_mask = stage_mask ? stage_mask : ~0u;
    return VG_OK;
}

vg_status vg_profile_read(vg_workspace *ws, vg_stage_time *out, int32_t capacity, int32_t *n_out) {
    if (!ws || !n_out || (capacity > 0 && !out)) return VG_ERR_INVALID_ARG;
    double tot[ST_COUNT] = {0};
    long long calls[ST_COUNT] = {0};
    for (auto &r : ws->prof) {
        VG_CUDA(ws, cudaEventSynchronize(r.b));
        float ms = 0.0f;
        VG_CUDA(ws, cudaEventElapsedTime(&ms, r.a, r.b));
        tot[r.stage] += ms;
        calls[r.stage] += 1;
        ws->prof_pool.push_back(r.a);
        ws->prof_pool.push_back(r.b);
    }
    ws->prof.clear();
    int n = 0;
    for (int k = 0; k < ST_COUNT; ++k) {
        if (!calls[k]) continue;
        if (n < capacity) {
            memset(out[n].name, 0, sizeof(out[n].name));
            strncpy(out[n].name, kStageName[k], sizeof(out[n].name) - 1);
            out[n].calls = calls[k];
            out[n].total_ms = tot[k];
        }
        ++n;
    }
    *n_out = n < capacity ? n : capacity;
    return VG_OK;
}

vg_status vg_read_keys(vg_workspace *ws, uint32_t *depth_bits, int32_t *rect) {
    if (!ws || !depth_bits || !rect) return VG_ERR_INVALID_ARG;
    if (ws->stage < 1 && !ws->tomo_read) return fail(ws, VG_ERR_STATE, "no preprocess to read");
    VG_CUDA(ws, cudaDeviceSynchronize());
    const size_t n = (size_t)ws->n_items;
    if (n == 0) return VG_OK;
    VG_CUDA(ws, cudaMemcpy(depth_bits, ws->depth.p, n * 4, cudaMemcpyDeviceToHost));
    std::vector<short4> r(n);
    VG_CUDA(ws, cudaMemcpy(r.data(), ws->rect.p, n * sizeof(short4), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) {
        rect[4 * i] = r[i].x;
        rect[4 * i + 1] = r[i].y;
        rect[4 * i + 2] = r[i].z;
        rect[4 * i + 3] = r[i].w;
    }
    return VG_OK;
}

vg_status vg_read_bins_range(vg_workspace *ws, int64_t tile0, int64_t tile1, int64_t *counts, int32_t *sorted_item,
                             int64_t cap, int64_t *n_out) {
    if (!ws || !counts || !n_out || tile0 < 0 || tile1 < tile0) return VG_ERR_INVALID_ARG;
    if (ws->stage < 2 && !ws->tomo_read) return fail(ws, VG_ERR_STATE, "no bin_sort to read");
    if (tile1 > ws->n_tiles) return fail(ws, VG_ERR_INVALID_ARG, "tile range beyond the last tile");
    VG_CUDA(ws, cudaDeviceSynchronize());
    *n_out = 0;
    if (tile1 == tile0) return VG_OK;
    std::vector<uint2> rg((size_t)(tile1 - tile0));
    VG_CUDA(ws, cudaMemcpy(rg.data(), ws->ranges.p + tile0, rg.size() * sizeof(uint2), cudaMemcpyDeviceToHost));
    // the lists of consecutive tiles are consecutive in the sorted instance array
    long long first = -1, last = -1, n = 0;
    for (size_t t = 0; t < rg.size(); ++t) {
        counts[t] = (int64_t)(rg[t].y - rg[t].x);
        n += counts[t];
        if (counts[t] > 0) {
            if (first < 0) first = rg[t].x;
            last = rg[t].y;
        }
    }
    if (n > cap || (n > 0 && !sorted_item)) return fail(ws, VG_ERR_INVALID_ARG, "sorted_item capacity too small");
    if (n > 0 && last - first != n) return fail(ws, VG_ERR_STATE, "tile lists are not contiguous");
    if (n > 0)
        VG_CUDA(ws, cudaMemcpy(sorted_item, ws->inst_item + first, (size_t)n * 4, cudaMemcpyDeviceToHost));
    *n_out = n;
    return VG_OK;
}

vg_status vg_read_pixel_state(vg_workspace *ws, float *S, uint32_t *last) {
    if (!ws) return VG_ERR_INVALID_ARG;
    if (ws->stage < 3) return fail(ws, VG_ERR_STATE, "no vg_render_fwd to read");
    VG_CUDA(ws, cudaDeviceSynchronize());
    const size_t n = (size_t)ws->n_pixels;
    if (n == 0) return VG_OK;
    if (S) VG_CUDA(ws, cudaMemcpy(S, ws->S_fin.p, n * sizeof(float), cudaMemcpyDeviceToHost));
    if (last) {
        VG_CUDA(ws, cudaMemcpy(last, ws->nlast.p, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        // the kernels keep positions in the sorted instance array: make them relative to the list
        std::vector<uint2> rg((size_t)ws->n_tiles);
        if (ws->n_tiles > 0)
            VG_CUDA(ws, cudaMemcpy(rg.data(), ws->ranges.p, rg.size() * sizeof(uint2), cudaMemcpyDeviceToHost));
        for (const ViewInfo &V : ws->views_h)
            for (int y = 0; y < V.H; ++y)
                for (int x = 0; x < V.W; ++x) {
                    const size_t p = (size_t)(V.pix_base + (long long)y * V.W + x);
                    last[p] -= rg[(size_t)V.tile_base + (size_t)(y / V.th) * V.tiles_x + x / V.tw].x;
                }
    }
    return VG_OK;
}

vg_status vg_read_bins(vg_workspace *ws, int64_t *tile_start, int32_t *sorted_item) {
    if (!ws || !tile_start) return VG_ERR_INVALID_ARG;
    if (ws->stage < 2 && !ws->tomo_read) return fail(ws, VG_ERR_STATE, "no bin_sort to read");
    VG_CUDA(ws, cudaDeviceSynchronize());
    long long n_inst = ws->n_inst;
    if (n_inst < 0) {   // fixed capacity: the count is on the device
        unsigned long long t = 0;
        VG_CUDA(ws, cudaMemcpy(&t, total64_ptr(ws), sizeof(t), cudaMemcpyDeviceToHost));
        n_inst = (long long)std::min<unsigned long long>(t, (unsigned long long)ws->capacity);
    }
    if (!sorted_item && n_inst > 0) return VG_ERR_INVALID_ARG;
    std::vector<uint2> rg((size_t)ws->n_tiles);
    if (ws->n_tiles > 0)
        VG_CUDA(ws, cudaMemcpy(rg.data(), ws->ranges.p, rg.size() * sizeof(uint2), cudaMemcpyDeviceToHost));
    tile_start[0] = 0;
    for (long long t = 0; t < ws->n_tiles; ++t) tile_start[t + 1] = tile_start[t] + (int64_t)(rg[t].y - rg[t].x);
    if (n_inst > 0)
        VG_CUDA(ws, cudaMemcpy(sorted_item, ws->inst_item, (size_t)n_inst * 4, cudaMemcpyDeviceToHost));
    return VG_OK;
}

}  // extern "C"
