// Backward of the blend (derived from Eq. 14 and Eq. 19 by the chain rule).
//
// k_render_bwd replays every pixel's list back to front from its stored blended count and
// log-transmittance S = sum tau (no per-pair state is kept by the forward):
//   T_i = exp(-(S_after - tau_i)),  dL/dc_i = g alpha_i T_i,
//   dL/dtau_i = g . (c_i T_{i+1} - R_i) - gT T_end,  R_i = sum_{j>i} c_j alpha_j T_j + T_end bg,
// then differentiates tau with respect to the record.  The replay is branch-free: a lane whose
// pixel does not blend the Gaussian (past its last blended record, outside the footprint or
// below the skip threshold) takes tau = 0, which leaves its state unchanged and adds zeros
// (0.421 ms against 0.464 ms with per-lane branches).  d' = A u and o' x d' = C u are linear in
// u = (dx, dy, 1), so with ga = 2 dL/da and gq = 2 dL/dq per pixel (a = |d'|^2, q = |o' x d'|^2)
//   dL/dA = A sum_p ga u u^T,   dL/dC = C sum_p gq u u^T:
// per Gaussian only the two symmetric 3x3 moment matrices (6 + 6 values), sum dL/dln(kappa) and
// the three colour partials are summed -- 16 values, added to the per-item accumulator in L2
// with vector reductions (red.global.add.v4/v2).  When at most kDirectLanes lanes of the warp
// contribute to a Gaussian, each of them adds its 16 values directly (four v4 reductions);
// otherwise three shuffle exchange steps leave every lane with 2 values summed over 8 lanes,
// and all 32 lanes add those (one v2 reduction each).  Thresholds 8 / 12 / 16 / 24 measured
// 0.411 / 0.403 / 0.411 / 0.470 ms on the 1M-Gaussian 1280x832 step (the ring kernel); two more
// butterfly steps before v2 reductions from 8 lanes only measured 0.417 ms.  Earlier, on the same
// step: 0.465 ms against 0.539 ms for a full reduce-scatter with 16 scalar reductions; a full
// reduce-scatter per Gaussian waits on five dependent shuffle rounds, while the L2 reduction
// units absorb the extra (unreturned) reductions; shared-memory float atomics measured slower
// than either.  k_chain multiplies by A and C and maps the result to dmu, dscale, dquat,
// dkappa, dsh.
#include "blend.cuh"
#include "geometry.cuh"

namespace vg {

// Accumulator layout per item: [0..5] sum ga (xx, xy, x, yy, y, 1), [6..11] the same for gq,
// [12] sum dL/dln(kappa), [13..15] dL/dcolour.
constexpr int kGradUsed = 16;
static_assert(kGradUsed == kGradN, "the vector reductions cover the whole 16-float accumulator");
constexpr int kDirectLanes = 12;   // at most this many contributing lanes: direct reductions


// Records are staged through a ring of kGroup-record slots in shared memory, back to front: the
// CTA's last warp is the producer, gathering each group's records (and, for the opacity test,
// their Gram rows) into a free slot; the other warps consume the slots in order.  Slots
// complete on mbarriers (full: the producer's 32 lanes arrive once the slot is written;
// empty: every consumer lane arrives once its warp is done with it), so a consumer warp waits
// only for data and never for the other consumers: warps whose pixels need few of a group's
// records run ahead by up to the ring's depth.  Every wait is bounded (kWaitLimitNs): a wait
// that runs out latches kDevErrTimeout in *err and the warp returns, and the CTA's other warps
// give up at their next wait.
constexpr int kGroup = 32;                               // records per ring slot
constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // 1 s

template <bool PIXTEST>
struct RingSlot {
    float4 rec[kGroup * kRecF4];                // the records, one after another
    float4 cull[PIXTEST ? 1 : kCullF4][kGroup];  // Gram rows for the opacity test, by row
    float4 ref[PIXTEST ? 1 : kGroup];            // (px0, py0, log2 K, |A0|) for the opacity test
    float sa1[PIXTEST ? 1 : kGroup];             // |A1| for the opacity test
    short4 rect[kGroup];                         // pixel footprint rectangles
    uint32_t item[kGroup];                       // item ids (accumulator rows)
};

// One CTA per tile (longest list first): tw th / P consumer threads owning P pixels each, plus
// the producer warp.  For each group a consumer warp first ballots which records it needs (some
// pixel of the warp reached the record, the record's footprint touches the warp's pixels and,
// when pairs below tau_skip are skipped, its opacity can reach tau_skip there), then visits only
// those, back to front.  The chunk setting CH gives the ring depth: CH / 16 slots (4 or 8, i.e.
// 128 or 256 records in flight).  The register cap is that of 4 / 4 / 5 CTAs of a 16 x 16 tile
// (with its producer warp) per SM for P = 1 / 2 / 4, whatever the tile shape.
template <int P, bool COUNT, bool PIXTEST, bool SPLAT, int CH>
__global__ void __maxnreg__(PixLayout<P>::kBwdRegs)
k_render_bwd(const ViewInfo *__restrict__ views, const int *__restrict__ tile_view, const int *__restrict__ tile_order,
             const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted_item, const float4 *__restrict__ rec,
             const short4 *__restrict__ prect, BlendParams bp, const float *__restrict__ T_fin, const float *__restrict__ S_fin,
             const uint32_t *__restrict__ nlast, const float *__restrict__ dL_drgb, const float *__restrict__ dL_dT,
             float *__restrict__ grad_acc, unsigned long long *__restrict__ pair_count, uint32_t *__restrict__ err) {
    pdl_entry();
    using L = PixLayout<P>;
    constexpr int kSlots = CH / 16;
    using Slot = RingSlot<PIXTEST>;
    __shared__ Slot ring[kSlots];
    __shared__ __align__(8) uint64_t full[kSlots], empty[kSlots];
    __shared__ uint32_t s_last;
    __shared__ int s_abort;

    const int n_cons = (int)blockDim.x - 32;   // consumer threads; the last warp produces
    const bool producer = (int)threadIdx.x >= n_cons;
    const int tile = tile_order ? tile_order[blockIdx.x] : (int)blockIdx.x;
    const ViewInfo &V = views[tile_view[tile]];
    const int local = tile - V.tile_base;
    const int tyi = local / V.tiles_x, txi = local - tyi * V.tiles_x;
    int ix, iy;
    L::origin(producer ? 0 : (int)threadIdx.x, V.tw, ix, iy);
    const int x0 = txi * V.tw + ix, y0 = tyi * V.th + iy;
    const uint2 rg = ranges[tile];
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_last = rg.x;
        s_abort = 0;
#pragma unroll
        for (int k = 0; k < kSlots; ++k) {
            mbar_init(&full[k], 32);
            mbar_init(&empty[k], (unsigned)n_cons);
        }
    }

    float Lp[P], S[P], Tafter[P], R0[P], R1[P], R2[P], g0[P], g1[P], g2[P], gTterm[P];
    uint32_t my_last[P];
    uint32_t thr_last = rg.x;
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const int x = x0 + L::ox(k), y = y0 + L::oy(k);
        Lp[k] = SPLAT ? 0.0f : pixel_ray(V, x, y).Lp;
        my_last[k] = rg.x;
        S[k] = 0.0f;
        float Tend = 1.0f;
        g0[k] = g1[k] = g2[k] = gTterm[k] = 0.0f;
        if (!producer && x < V.W && y < V.H) {
            const long long pix = V.pix_base + (long long)y * V.W + x;
            my_last[k] = nlast[pix];
            S[k] = S_fin[pix];
            Tend = T_fin[pix];
            if (dL_drgb) {   // absent for the cone-beam projection (dL/dT alone)
                g0[k] = dL_drgb[3 * pix];
                g1[k] = dL_drgb[3 * pix + 1];
                g2[k] = dL_drgb[3 * pix + 2];
            }
            gTterm[k] = dL_dT ? -dL_dT[pix] * Tend : 0.0f;
        }
        Tafter[k] = ex2_approx(__fmul_rn(-kLog2eF, S[k]));
        R0[k] = Tend * bp.bg[0];
        R1[k] = Tend * bp.bg[1];
        R2[k] = Tend * bp.bg[2];
        thr_last = max(thr_last, my_last[k]);
    }
    __syncthreads();   // s_last and the barriers are initialised
    if (thr_last > rg.x) atomicMax(&s_last, thr_last);
    __syncthreads();   // the last such barrier of the kernel: warps proceed independently below
    const uint32_t tile_last = s_last;
    const uint32_t n_groups = (tile_last - rg.x + kGroup - 1) / kGroup;
    // group g covers [start, end) with end = tile_last - g kGroup, start = max(rg.x, end - kGroup)
    auto group_range = [&](uint32_t g, uint32_t &start, uint32_t &end) {
        end = tile_last - g * kGroup;
        start = (end - rg.x > (uint32_t)kGroup) ? end - kGroup : rg.x;
    };
    auto give_up = [&]() {
        if (lane == 0) atomicOr(err, kDevErrTimeout);
        s_abort = 1;
    };

    if (producer) {
        for (uint32_t g = 0; g < n_groups; ++g) {
            const int sl = (int)(g % kSlots);
            if (!mbar_wait(&empty[sl], ((g / kSlots) & 1u) ^ 1u, kWaitLimitNs, &s_abort)) {
                give_up();
                return;
            }
            uint32_t start, end;
            group_range(g, start, end);
            Slot &Sl = ring[sl];
            if (lane < (int)(end - start)) {
                const uint32_t item = sorted_item[start + lane];
                const float4 *src = rec + (size_t)item * kRecF4;
                float4 q[kRecF4];
#pragma unroll
                for (int k = 0; k < kRecF4; ++k) q[k] = __ldg(src + k);
                const short4 pr = prect[item];
#pragma unroll
                for (int k = 0; k < kRecF4; ++k) Sl.rec[lane * kRecF4 + k] = q[k];
                Sl.rect[lane] = pr;
                Sl.item[lane] = item;
                if (!PIXTEST) {
                    float4 c[kCullF4];
                    cull_row(q[0], q[1], q[2], q[3], q[4], c);
#pragma unroll
                    for (int k = 0; k < kCullF4; ++k) Sl.cull[k][lane] = c[k];
                    Sl.ref[lane] = make_float4(q[4].z, q[4].w, q[5].x, sqrtf(c[0].x));
                    Sl.sa1[lane] = sqrtf(c[0].w);
                }
            }
            mbar_arrive(&full[sl]);
        }
        return;
    }

    const uint32_t warp_last = __reduce_max_sync(0xffffffffu, thr_last);
    const WarpBox wb = warp_box<P>(x0, y0);
    const BoxCull bc = SPLAT ? box_cull_splat(wb, bp.alpha_min) : box_cull(V, wb, bp.tau_skip);
    const float xf = (float)x0, yf = (float)y0;
    unsigned long long pairs = 0, blended = 0;   // evaluated / blended pairs (COUNT only)
    for (uint32_t g = 0; g < n_groups; ++g) {
        const int sl = (int)(g % kSlots);
        uint32_t start, end;
        group_range(g, start, end);
        if (!mbar_wait(&full[sl], (g / kSlots) & 1u, kWaitLimitNs, &s_abort)) {
            give_up();
            return;
        }
        if (start < warp_last) {
            const Slot &Sl = ring[sl];
            const int n = (int)(end - start);
            bool need = lane < n && start + (uint32_t)lane < warp_last && !box_misses(wb, Sl.rect[lane]);
            if (!PIXTEST && need) {   // skip records whose opacity stays below tau_skip on this warp
                const float4 r = Sl.ref[lane];
                need = box_may_blend(Sl.cull[0][lane], Sl.cull[1][lane], Sl.cull[2][lane], r.x, r.y, r.z, r.w,
                                     Sl.sa1[lane], bc);
            }
            unsigned m = __ballot_sync(0xffffffffu, need);
            while (m) {
                const int b = 31 - __clz(m);
                m ^= 1u << b;
                const int j = b;
                const uint32_t idx = start + (uint32_t)j;
                float gv[kGradUsed];
#pragma unroll
                for (int k = 0; k < kGradUsed; ++k) gv[k] = 0.0f;
                bool any = false;
                {
                    const float4 *r = &Sl.rec[j * kRecF4];
                    const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3], r4 = r[4], r5 = r[5];
                    short4 pr;
                    if (PIXTEST) pr = Sl.rect[j];
                    constexpr int kCols = P == 4 ? 2 : 1;   // pixel columns of the thread
                    ColBase cb[kCols];
                    SplatCol sc[kCols];
#pragma unroll
                    for (int c = 0; c < kCols; ++c) {
                        if constexpr (SPLAT)
                            splat_col(r2, r3, r4, c ? xf + 1.0f : xf, sc[c]);
                        else
                            col_base(r0, r1, r2, r3, r4, c ? xf + 1.0f : xf, cb[c]);
                    }
#pragma unroll
                    for (int k = 0; k < P; ++k) {
                        bool valid = idx < my_last[k];
                        if (PIXTEST) valid = valid && !pixel_outside(x0 + L::ox(k), y0 + L::oy(k), pr);
                        float tau, e2, alpha, pdx, pdy, kG, ca, cq;
                        if constexpr (SPLAT) {
                            float q;
                            const float ar = splat_at(r3, r4, r5, sc[L::ox(k)], L::oy(k) ? yf + (float)L::oy(k) : yf, pdx, pdy, q);
                            if (COUNT) pairs += valid;
                            const bool clamped = ar > bp.alpha_max;
                            const float a_c = fminf(ar, bp.alpha_max);
                            valid = valid && a_c >= bp.alpha_min;
                            alpha = valid ? a_c : 0.0f;
                            e2 = __fsub_rn(1.0f, alpha);
                            tau = -log1pf(-alpha);
                            // tau = -ln(1 - o G'): dtau/dln o = alpha / (1 - alpha); a clamp cuts it
                            kG = clamped ? 0.0f : alpha / e2;
                            ca = 0.0f;
                            cq = -1.0f;        // ln(o G') = ln o - q/2
                        } else {
                            PairEval e;
                            pair_eval_col(r0, r1, r3, r4, r5, cb[L::ox(k)], L::oy(k) ? yf + (float)L::oy(k) : yf, Lp[k], e);
                            if (COUNT) pairs += valid;
                            const bool clamped = e.tau > bp.tau_max;
                            const float t_c = fminf(e.tau, bp.tau_max);
                            valid = valid && t_c >= bp.tau_skip;
                            tau = valid ? t_c : 0.0f;
                            e2 = ex2_approx(__fmul_rn(-kLog2eF, tau));
                            alpha = __fsub_rn(1.0f, e2);
                            pdx = e.dx;
                            pdy = e.dy;
                            kG = clamped ? 0.0f : tau;   // dln(tau)/dln(amplitude) = 1; a clamp cuts it
                            const float r2s = e.rs * e.rs;
                            ca = r2s * (e.m2 - 1.0f);
                            cq = -r2s;
                        }
                        if (COUNT) blended += valid;
                        any |= valid;
                        const float Sb = S[k] - tau;
                        const float Tb = valid ? ex2_approx(-kLog2eF * Sb) : Tafter[k];
                        const float aT = alpha * Tb;
                        gv[13] = fmaf(g0[k], aT, gv[13]);
                        gv[14] = fmaf(g1[k], aT, gv[14]);
                        gv[15] = fmaf(g2[k], aT, gv[15]);
                        // per channel c T - R with one rounding each (fma): a single scalar g . R
                        // measured less accurate for flattened Gaussians under Eq. 20
                        const float dtau = g0[k] * fmaf(r5.y, Tafter[k], -R0[k]) + g1[k] * fmaf(r5.z, Tafter[k], -R1[k]) +
                                           g2[k] * fmaf(r5.w, Tafter[k], -R2[k]) + gTterm[k];
                        R0[k] = fmaf(r5.y, aT, R0[k]);
                        R1[k] = fmaf(r5.z, aT, R1[k]);
                        R2[k] = fmaf(r5.w, aT, R2[k]);
                        S[k] = Sb;
                        Tafter[k] = Tb;
                        const float G = dtau * kG;                   // dL / d ln(amplitude)
                        const float gq = G * cq;                     // 2 dL/dq
                        const float xx = pdx * pdx, xy = pdx * pdy, yy = pdy * pdy;
                        if constexpr (!SPLAT) {
                            const float ga = G * ca;                 // 2 dL/da
                            gv[0] = fmaf(ga, xx, gv[0]);
                            gv[1] = fmaf(ga, xy, gv[1]);
                            gv[2] = fmaf(ga, pdx, gv[2]);
                            gv[3] = fmaf(ga, yy, gv[3]);
                            gv[4] = fmaf(ga, pdy, gv[4]);
                            gv[5] += ga;
                        }
                        gv[6] = fmaf(gq, xx, gv[6]);
                        gv[7] = fmaf(gq, xy, gv[7]);
                        gv[8] = fmaf(gq, pdx, gv[8]);
                        gv[9] = fmaf(gq, yy, gv[9]);
                        gv[10] = fmaf(gq, pdy, gv[10]);
                        gv[11] += gq;
                        gv[12] += G;
                    }
                }
                const unsigned act = __ballot_sync(0xffffffffu, any);
                if (act) {
                    float *dst = grad_acc + (size_t)Sl.item[j] * kGradN;   // 64-byte aligned
                    if (__popc(act) <= kDirectLanes) {
                        if (any) {
                            red_add_v4(dst, gv[0], gv[1], gv[2], gv[3]);
                            red_add_v4(dst + 4, gv[4], gv[5], gv[6], gv[7]);
                            red_add_v4(dst + 8, gv[8], gv[9], gv[10], gv[11]);
                            red_add_v4(dst + 12, gv[12], gv[13], gv[14], gv[15]);
                        }
                    } else {
                        const int b0 = warp_reduce_scatter_part<kGradUsed, 3>(gv, lane);
                        red_add_v2(dst + b0, gv[0], gv[1]);
                    }
                }
            }
        }
        mbar_arrive(&empty[sl]);   // this warp is done with the slot
    }
    if (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
            blended += __shfl_xor_sync(0xffffffffu, blended, o);
        }
        if (lane == 0 && pairs) atomicAdd(pair_count, pairs);
        if (lane == 0 && blended) atomicAdd(pair_count + 1, blended);
    }
}

template <int P, bool PIXTEST, bool SPLAT, int CH>
static void launch_bwd_ptsc(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                            const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                            const BlendParams &bp, const float *T_fin, const float *S_fin, const uint32_t *nlast,
                            const float *dL_drgb, const float *dL_dT, float *grad_acc, unsigned long long *pair_count,
                            uint32_t *err, cudaStream_t st) {
    const unsigned threads = (unsigned)(bp.tile_px / P + 32);   // consumers + the producer warp
    if (pair_count)
        pdl_launch(k_render_bwd<P, true, PIXTEST, SPLAT, CH>, (unsigned)n_tiles, threads, 0, st,
            views_d, tile_view, tile_order, ranges, sorted_item, rec, prect, bp, T_fin, S_fin, nlast, dL_drgb, dL_dT,
            grad_acc, pair_count, err);
    else
        pdl_launch(k_render_bwd<P, false, PIXTEST, SPLAT, CH>, (unsigned)n_tiles, threads, 0, st,
            views_d, tile_view, tile_order, ranges, sorted_item, rec, prect, bp, T_fin, S_fin, nlast, dL_drgb, dL_dT,
            grad_acc, nullptr, err);
}

template <int P, bool PIXTEST, bool SPLAT>
static void launch_bwd_pts(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                           const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                           const BlendParams &bp, const float *T_fin, const float *S_fin, const uint32_t *nlast,
                           const float *dL_drgb, const float *dL_dT, float *grad_acc, unsigned long long *pair_count,
                           uint32_t *err, cudaStream_t st) {
    if (bp.chunk_bwd == 64)
        launch_bwd_ptsc<P, PIXTEST, SPLAT, 64>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect,
                                               bp, T_fin, S_fin, nlast, dL_drgb, dL_dT, grad_acc, pair_count, err, st);
    else
        launch_bwd_ptsc<P, PIXTEST, SPLAT, 128>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect,
                                                bp, T_fin, S_fin, nlast, dL_drgb, dL_dT, grad_acc, pair_count, err, st);
}

template <int P, bool PIXTEST>
static void launch_bwd_pt(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                          const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                          const BlendParams &bp, const float *T_fin, const float *S_fin, const uint32_t *nlast,
                          const float *dL_drgb, const float *dL_dT, float *grad_acc, unsigned long long *pair_count,
                          uint32_t *err, cudaStream_t st) {
    if (bp.splat)
        launch_bwd_pts<P, PIXTEST, true>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp,
                                         T_fin, S_fin, nlast, dL_drgb, dL_dT, grad_acc, pair_count, err, st);
    else
        launch_bwd_pts<P, PIXTEST, false>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect,
                                          bp, T_fin, S_fin, nlast, dL_drgb, dL_dT, grad_acc, pair_count, err, st);
}

template <int P>
static void launch_bwd_p(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                         const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                         const BlendParams &bp, const float *T_fin, const float *S_fin, const uint32_t *nlast,
                         const float *dL_drgb, const float *dL_dT, float *grad_acc, unsigned long long *pair_count,
                         uint32_t *err, cudaStream_t st) {
    if (bp.pixel_test)
        launch_bwd_pt<P, true>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, T_fin,
                               S_fin, nlast, dL_drgb, dL_dT, grad_acc, pair_count, err, st);
    else
        launch_bwd_pt<P, false>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, T_fin,
                                S_fin, nlast, dL_drgb, dL_dT, grad_acc, pair_count, err, st);
}

cudaError_t launch_render_bwd(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                              const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                              const BlendParams &bp, int ppt, const float *T_fin, const float *S_fin,
                              const uint32_t *nlast, const float *dL_drgb, const float *dL_dT, float *grad_acc,
                              unsigned long long *pair_count, uint32_t *err, cudaStream_t st, long long *launches) {
    if (n_tiles <= 0) return cudaSuccess;
    if (ppt == 1)
        launch_bwd_p<1>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, T_fin, S_fin, nlast,
                        dL_drgb, dL_dT, grad_acc, pair_count, err, st);
    else if (ppt == 4)
        launch_bwd_p<4>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, T_fin, S_fin, nlast,
                        dL_drgb, dL_dT, grad_acc, pair_count, err, st);
    else
        launch_bwd_p<2>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, T_fin, S_fin, nlast,
                        dL_drgb, dL_dT, grad_acc, pair_count, err, st);
    *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- chain
__device__ __forceinline__ void cross_add(const float a[3], const float b[3], float c[3]) {
    c[0] += a[1] * b[2] - a[2] * b[1];
    c[1] += a[2] * b[0] - a[0] * b[2];
    c[2] += a[0] * b[1] - a[1] * b[0];
}

// Splat mode (Eq. 5-7): the moments Mq = sum gq u u^T (gq = 2 dL/dq, u = (dx, dy, 1) from the
// reference pixel; accumulator entries 6..11) of one (view, Gaussian) give, with w = u - m,
//   dL/dQ = (1/2) sum gq w w^T,   dL/dmu' = -Q sum gq w      (q = w' Q w, Q = Sigma'^-1),
// then dL/dSigma' = -Q dL/dQ Q and, with Sigma' = B B^T + dil I, dL/dB = -2 Q dL/dQ P where
// P = Q B has the rows (b_1 x n + dil b_0) / det and (n x b_0 + dil b_1) / det (n = b_0 x b_1:
// no cancellation for thin footprints), and through B_ik = s_k (a_i . r_k), a_i the rows of
// J W, and J(t), mu'(t) to the rotation (dR, row-major), scale and mean.
__device__ __forceinline__ void splat_chain(const ViewInfo &V, const float mu[3], const float s[3], const float Rq[9],
                                            float dil, const float ga[kGradN], float dR[9], float dm[3],
                                            float dsc[3]) {
    SplatGeom G;
    if (!splat_geom(V, mu, s, Rq, dil, G)) {
#pragma unroll
        for (int k = 0; k < 9; ++k) dR[k] = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) dm[k] = dsc[k] = 0.0f;
        return;
    }
    const float mx = G.mx, my = G.my;
    const float M00 = ga[6], M01 = ga[7], M02 = ga[8], M11 = ga[9], M12 = ga[10], M22 = ga[11];
    const float Sx = fmaf(-mx, M22, M02), Sy = fmaf(-my, M22, M12);
    const float Sxx = fmaf(-mx, M02 + Sx, M00);
    const float Sxy = fmaf(-mx, Sy, fmaf(-my, M02, M01));
    const float Syy = fmaf(-my, M12 + Sy, M11);
    const float idet = 1.0f / G.det;
    const float Q00 = G.g11 * idet, Q01 = -G.g01 * idet, Q11 = G.g00 * idet;
    const float dmx = -fmaf(Q00, Sx, Q01 * Sy), dmy = -fmaf(Q01, Sx, Q11 * Sy);
    // T = Q dL/dQ with dL/dQ = (1/2) [[Sxx, Sxy], [Sxy, Syy]]
    const float T00 = 0.5f * fmaf(Q00, Sxx, Q01 * Sxy), T01 = 0.5f * fmaf(Q00, Sxy, Q01 * Syy);
    const float T10 = 0.5f * fmaf(Q01, Sxx, Q11 * Sxy), T11 = 0.5f * fmaf(Q01, Sxy, Q11 * Syy);
    float P[2][3];
    {
        const float *b0 = G.B[0], *b1 = G.B[1], *n = G.n;
        const float c0[3] = {b1[1] * n[2] - b1[2] * n[1], b1[2] * n[0] - b1[0] * n[2], b1[0] * n[1] - b1[1] * n[0]};
        const float c1[3] = {n[1] * b0[2] - n[2] * b0[1], n[2] * b0[0] - n[0] * b0[2], n[0] * b0[1] - n[1] * b0[0]};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            P[0][k] = fmaf(dil, b0[k], c0[k]) * idet;
            P[1][k] = fmaf(dil, b1[k], c1[k]) * idet;
        }
    }
    float dB[2][3], da[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dB[0][k] = -2.0f * fmaf(T00, P[0][k], T01 * P[1][k]);
        dB[1][k] = -2.0f * fmaf(T10, P[0][k], T11 * P[1][k]);
        dsc[k] = fmaf(dB[0][k], G.ar[0][k], dB[1][k] * G.ar[1][k]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dR[3 * c + k] = s[k] * fmaf(dB[0][k], G.a[0][c], dB[1][k] * G.a[1][c]);
            da[0][c] = fmaf(dB[0][k] * s[k], Rq[3 * c + k], da[0][c]);
            da[1][c] = fmaf(dB[1][k] * s[k], Rq[3 * c + k], da[1][c]);
        }
    const float *W = V.R;
    const float dJ00 = da[0][0] * W[0] + da[0][1] * W[1] + da[0][2] * W[2];
    const float dJ02 = da[0][0] * W[6] + da[0][1] * W[7] + da[0][2] * W[8];
    const float dJ11 = da[1][0] * W[3] + da[1][1] * W[4] + da[1][2] * W[5];
    const float dJ12 = da[1][0] * W[6] + da[1][1] * W[7] + da[1][2] * W[8];
    const float jx = G.jx, jy = G.jy, u = G.u, v = G.v, iz = G.iz;
    const float dt0 = jx * fmaf(-dJ02, iz, dmx);
    const float dt1 = jy * fmaf(-dJ12, iz, dmy);
    const float dt2 = -jx * u * dmx - jy * v * dmy + jx * iz * fmaf(2.0f * u, dJ02, -dJ00) +
                      jy * iz * fmaf(2.0f * v, dJ12, -dJ11);
#pragma unroll
    for (int c = 0; c < 3; ++c) dm[c] = W[c] * dt0 + W[3 + c] * dt1 + W[6 + c] * dt2;
}

// One thread per Gaussian: it visits the Gaussian's item in every view, sums the parameter
// gradients in registers and writes them once (overwriting when `zero`, else adding), so no
// atomics are needed.  A warp owns 32 consecutive Gaussians: their SH rows are read, and their
// SH-gradient rows accumulated and written, through shared memory with coalesced instructions.
constexpr int kChainWarps = 2;

template <typename RT, typename ST, bool SPLAT, bool SH3>
__global__ void __launch_bounds__(32 * kChainWarps, 8)
k_chain(GaussIn g, const ViewInfo *__restrict__ views, int n_views, float *__restrict__ grad_acc, int zero,
        float *__restrict__ dmu, float *__restrict__ dscale, float *__restrict__ dquat, float *__restrict__ dkappa,
        float *__restrict__ dsh) {
    pdl_entry();
    // SH coefficients (as float) and the SH gradient being accumulated: kRowStride floats per row,
    // or (SH3: FP32 degree-3 rows and a 16-byte aligned dsh) kRow16 float4 per row
    constexpr int kStride = SH3 ? 4 * kRow16 : kRowStride;
    __shared__ __align__(16) float ssh[kChainWarps][32 * kStride];
    __shared__ __align__(16) float sdsh[kChainWarps][32 * kStride];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int K = (g.sh_degree + 1) * (g.sh_degree + 1), K3 = 3 * K;
    float *shrow = ssh[wi] + lane * kStride, *dshrow = sdsh[wi] + lane * kStride;
    const long long n_chunks = ((long long)g.n + 31) / 32;
    for (long long ch = (long long)blockIdx.x * kChainWarps + wi; ch < n_chunks; ch += (long long)gridDim.x * kChainWarps) {
        const long long gbase = ch * 32;
        const int nloc = (int)min(32LL, (long long)g.n - gbase);
        const long long gi = gbase + lane;
        if (SH3) {
            warp_load_sh3((const float *)g.sh + gbase * K3, nloc, reinterpret_cast<float4 *>(ssh[wi]), lane);
            if (zero) {
#pragma unroll
                for (int j = 0; j < kSh3Pieces; ++j)
                    reinterpret_cast<float4 *>(dshrow)[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            } else {
                warp_load_sh3(dsh + gbase * K3, nloc, reinterpret_cast<float4 *>(sdsh[wi]), lane);
            }
        } else {
            if (g.sh != nullptr) warp_load_rows<ST>((const ST *)g.sh + gbase * K3, nloc, K3, ssh[wi], lane);
            if (dsh != nullptr) {
                if (zero) {
                    for (int k = 0; k < K3; ++k) dshrow[k] = 0.0f;
                } else {
                    warp_load_rows<float>(dsh + gbase * K3, nloc, K3, sdsh[wi], lane);
                }
            }
        }
        // the parameters are requested before the wait, so that their round trip overlaps the SH
        // rows' copies
        float mu[3], s[3], q[4], kin;
        if (lane < nloc) {
            load_gauss<RT>(g, gi, mu, s, q, kin);
        }
        rows_wait();
        __syncwarp();
        if (lane < nloc) {
        float Sig[9], Rq[9], qn[4], smax;
        const Density dn = density_of(g, kin, s);
        const float kap = dn.kap;
        const bool valid = key_cov(mu, s, q, dn.kap_key, Sig, Rq, qn, smax);
        float am[3] = {0.0f, 0.0f, 0.0f}, asc[3] = {0.0f, 0.0f, 0.0f}, aq[4] = {0.0f, 0.0f, 0.0f, 0.0f}, ak = 0.0f;
        for (int v = 0; valid && v < n_views; ++v) {
        const long long it = (long long)v * g.n + gi;
        float4 *ga4 = (float4 *)(grad_acc + it * kGradN);
        float ga[kGradN];
        bool any = false;
#pragma unroll
        for (int k = 0; k < kGradN / 4; ++k) {
            const float4 t = ga4[k];
            ga[4 * k] = t.x;
            ga[4 * k + 1] = t.y;
            ga[4 * k + 2] = t.z;
            ga[4 * k + 3] = t.w;
            any |= (t.x != 0.0f) | (t.y != 0.0f) | (t.z != 0.0f) | (t.w != 0.0f);
        }
        if (!any) continue;
        // the accumulator is left zero for the next backward (no separate clearing pass)
#pragma unroll
        for (int k = 0; k < kGradN / 4; ++k) ga4[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const ViewInfo &V = views[v];
        float dR[9], dm[3], dsc[3];
        if constexpr (SPLAT) {
            splat_chain(V, mu, s, Rq, g.splat_dil, ga, dR, dm, dsc);
        } else {
        ItemGeom G;
        item_geom(V, mu, s, Rq, G);
        // dA_j = sum_k A_k Ma[k][j], dC_j = sum_k C_k Mq[k][j] with the symmetric moments
        // Ma = sum ga u u^T over u = (dx, dy, 1), stored as (xx, xy, x, yy, y, 1).
        float dA[9], dC[9];
        {
            const float Ma[9] = {ga[0], ga[1], ga[2], ga[1], ga[3], ga[4], ga[2], ga[4], ga[5]};
            const float Mq[9] = {ga[6], ga[7], ga[8], ga[7], ga[9], ga[10], ga[8], ga[10], ga[11]};
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    dA[3 * j + c] = G.A[c] * Ma[j] + G.A[3 + c] * Ma[3 + j] + G.A[6 + c] * Ma[6 + j];
                    dC[3 * j + c] = G.Cc[c] * Mq[j] + G.Cc[3 + c] * Mq[3 + j] + G.Cc[6 + c] * Mq[6 + j];
                }
        }
        // The record's C_k = o' x A_k with o' = -M mu_c.  Writing mu_c = t0 dc0 - v0 and
        // o' = Q2 - t0 A2 (t0 = camera depth of the mean, v0 and Q2 small), the two largest
        // terms of dL/dM, -t0 (dC2 x A2) (x) dc0 and -t0 (A2 x dC2) (x) dc0, cancel exactly and are
        // left out; what remains has no large cancelling parts:
        //   dL/dM = sum_k (dA_k + dC_k x Q2) (x) b_k - t0 [(dC0 x A2) (x) b_0 + (dC1 x A2) (x) b_1]
        //           - t0 (A0 x dC0 + A1 x dC1) (x) dc0 + dop (x) v0,   b = (e0/fx, e1/fy, dc0),
        //   dL/dmu_c = -M^T dop,  dop = sum_k A_k x dC_k.
        const float t0 = G.muc[2].hi;
        float Q2[3], v0[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Q2[i] = df_float(df_fma(G.opx[i], t0, G.A[6 + i]));
            v0[i] = df_float(df_fma(df_neg(G.muc[i]), t0, G.dc0[i]));
        }
        float dop[3] = {0.0f, 0.0f, 0.0f}, H[3] = {0.0f, 0.0f, 0.0f}, E[9] = {0.0f}, F[6] = {0.0f};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            cross_add(&G.A[3 * k], &dC[3 * k], dop);
#pragma unroll
            for (int i = 0; i < 3; ++i) E[3 * k + i] = dA[3 * k + i];
            cross_add(&dC[3 * k], Q2, &E[3 * k]);
        }
        cross_add(&G.A[0], &dC[0], H);
        cross_add(&G.A[3], &dC[3], H);
        cross_add(&dC[0], &G.A[6], &F[0]);
        cross_add(&dC[3], &G.A[6], &F[3]);
        float dM[9];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float base = E[6 + i] - t0 * H[i];
            dM[3 * i + 0] = (E[i] - t0 * F[i]) / V.fx + base * G.dc0[0] + dop[i] * v0[0];
            dM[3 * i + 1] = (E[3 + i] - t0 * F[3 + i]) / V.fy + base * G.dc0[1] + dop[i] * v0[1];
            dM[3 * i + 2] = base * G.dc0[2] + dop[i] * v0[2];
        }
        float dmuc[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) dmuc[j] = -(G.M[j] * dop[0] + G.M[3 + j] * dop[1] + G.M[6 + j] * dop[2]);
        // M[i][j] = B[j][i] / s_i
        float dB[9];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float is = 1.0f / s[i];
            dsc[i] = -(dM[3 * i] * G.M[3 * i] + dM[3 * i + 1] * G.M[3 * i + 1] + dM[3 * i + 2] * G.M[3 * i + 2]) * is;
#pragma unroll
            for (int j = 0; j < 3; ++j) dB[3 * j + i] = dM[3 * i + j] * is;
        }
        // B = Rc Rq  =>  dRq = Rc^T dB;  mu_c = Rc mu + t  =>  dmu = Rc^T dmu_c
        const float *Rc = V.R;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) dR[3 * a + b] = Rc[a] * dB[b] + Rc[3 + a] * dB[3 + b] + Rc[6 + a] * dB[6 + b];
            dm[a] = Rc[a] * dmuc[0] + Rc[3 + a] * dmuc[1] + Rc[6 + a] * dmuc[2];
        }
        }
        // rotation matrix of the unit quaternion (w, x, y, z), differentiated entry by entry
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

        // colour: rgb = max(sh . Y(dir) + 0.5, 0), dir = (mu - o)/|mu - o|
        if (g.sh != nullptr && (ga[13] != 0.0f || ga[14] != 0.0f || ga[15] != 0.0f)) {
            float dir[3], len;
            view_dir(V, mu, dir, len);
            float Y[16];
            sh_basis(g.sh_degree, dir[0], dir[1], dir[2], Y);
            float raw[3] = {0.5f, 0.5f, 0.5f};   // colour before the clamp (same order as eval_colour_row)
            float gc[3], w[16], gd[3];
            if constexpr (SH3) {
                const float4 *r4 = reinterpret_cast<const float4 *>(shrow);
                float4 *d4 = reinterpret_cast<float4 *>(dshrow);
#pragma unroll
                for (int qd = 0; qd < 4; ++qd) {   // 4 coefficients (three float4) at a time
                    const float4 a = r4[3 * qd], b = r4[3 * qd + 1], c = r4[3 * qd + 2];
                    const float v[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) raw[ch] = fmaf(v[3 * kk + ch], Y[4 * qd + kk], raw[ch]);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) gc[c] = ga[13 + c] * colour_act_grad(raw[c], g.softplus_beta);
#pragma unroll
                for (int qd = 0; qd < 4; ++qd) {
                    const float4 a = r4[3 * qd], b = r4[3 * qd + 1], c = r4[3 * qd + 2];
                    const float v[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
                    float4 e[3] = {d4[3 * qd], d4[3 * qd + 1], d4[3 * qd + 2]};
                    float *ev = reinterpret_cast<float *>(e);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const int k = 4 * qd + kk;
                        w[k] = 0.0f;
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) {
                            w[k] = fmaf(gc[ch], v[3 * kk + ch], w[k]);
                            ev[3 * kk + ch] += gc[ch] * Y[k];
                        }
                    }
                    d4[3 * qd] = e[0];
                    d4[3 * qd + 1] = e[1];
                    d4[3 * qd + 2] = e[2];
                }
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    if (k >= K) break;
#pragma unroll
                    for (int c = 0; c < 3; ++c) raw[c] = fmaf(shrow[3 * k + c], Y[k], raw[c]);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) gc[c] = ga[13 + c] * colour_act_grad(raw[c], g.softplus_beta);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    w[k] = 0.0f;
                    if (k >= K) continue;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        w[k] = fmaf(gc[c], shrow[3 * k + c], w[k]);
                        if (dsh != nullptr) dshrow[3 * k + c] += gc[c] * Y[k];
                    }
                }
            }
            sh_grad_dot(g.sh_degree, dir[0], dir[1], dir[2], w, gd);
            const float dd = gd[0] * dir[0] + gd[1] * dir[1] + gd[2] * dir[2];
            const float il = 1.0f / len;
#pragma unroll
            for (int c = 0; c < 3; ++c) dm[c] += (gd[c] - dir[c] * dd) * il;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            am[c] += dm[c];
            asc[c] += dsc[c];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) aq[c] += (dqn[c] - qn[c] * dot) / qnorm;
        ak += ga[12] / kap;
        }
        if (g.density_theta && valid) {   // Eq. 20: kappa(theta, s); ak = dL/dkappa becomes dL/dtheta
#pragma unroll
            for (int c = 0; c < 3; ++c) asc[c] -= ak * dn.lnv / (3.0f * s[c] * s[c]);
            ak = ak * 0.99f / (1.0f - 0.99f * kin) * dn.m;
        }
        if (zero) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dmu[3 * gi + c] = am[c];
                dscale[3 * gi + c] = asc[c];
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) dquat[4 * gi + c] = aq[c];
            dkappa[gi] = ak;
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dmu[3 * gi + c] += am[c];
                dscale[3 * gi + c] += asc[c];
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) dquat[4 * gi + c] += aq[c];
            dkappa[gi] += ak;
        }
        }
        __syncwarp();
        if (SH3)
            warp_store_sh3(dsh + gbase * K3, nloc, reinterpret_cast<const float4 *>(sdsh[wi]), lane);
        else if (dsh != nullptr)
            warp_store_rows(dsh + gbase * K3, nloc, K3, sdsh[wi], lane);
        __syncwarp();   // the buffers are reused by the next chunk
    }
}

template <typename RT, typename ST>
static cudaError_t launch_chain_t(const GaussIn &g, const ViewInfo *views_d, int n_views, float *grad_acc, int zero,
                                  float *dmu, float *dscale, float *dquat, float *dkappa, float *dsh, cudaStream_t st) {
    long long b = ((long long)g.n + 32 * kChainWarps - 1) / (32 * kChainWarps);
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    // FP32 degree-3 SH rows and a 16-byte aligned SH gradient: 16-byte pieces
    const bool sh3 = sh3_rows<ST>(g) && dsh != nullptr && ((uintptr_t)dsh & 15u) == 0;
#define VG_CHAIN_LAUNCH(SPL, S3)                                                                                     \
    pdl_launch(k_chain<RT, ST, SPL, S3>, (unsigned)b, 32 * kChainWarps, 0, st, g, views_d, n_views, grad_acc, zero, dmu, \
               dscale, dquat, dkappa, dsh)
    if (g.splat) {
        if (sh3)
            VG_CHAIN_LAUNCH(true, true);
        else
            VG_CHAIN_LAUNCH(true, false);
    } else {
        if (sh3)
            VG_CHAIN_LAUNCH(false, true);
        else
            VG_CHAIN_LAUNCH(false, false);
    }
#undef VG_CHAIN_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_chain(const GaussIn &g, const ViewInfo *views_d, int n_views, float *grad_acc, int zero,
                         float *dmu, float *dscale, float *dquat, float *dkappa, float *dsh, cudaStream_t st,
                         long long *launches) {
    if (g.n <= 0) return cudaSuccess;
    *launches += 1;
#define VG_CHAIN(RT, ST) launch_chain_t<RT, ST>(g, views_d, n_views, grad_acc, zero, dmu, dscale, dquat, dkappa, dsh, st)
    if (g.rec_dtype == VG_F32) {
        if (g.sh_dtype == VG_F16) return VG_CHAIN(float, __half);
        if (g.sh_dtype == VG_BF16) return VG_CHAIN(float, __nv_bfloat16);
        return VG_CHAIN(float, float);
    }
    if (g.rec_dtype == VG_BF16) {
        if (g.sh_dtype == VG_F16) return VG_CHAIN(__nv_bfloat16, __half);
        if (g.sh_dtype == VG_F32) return VG_CHAIN(__nv_bfloat16, float);
        return VG_CHAIN(__nv_bfloat16, __nv_bfloat16);
    }
    if (g.sh_dtype == VG_F32) return VG_CHAIN(__half, float);
    if (g.sh_dtype == VG_BF16) return VG_CHAIN(__half, __nv_bfloat16);
    return VG_CHAIN(__half, __half);
#undef VG_CHAIN
}

}  // namespace vg
