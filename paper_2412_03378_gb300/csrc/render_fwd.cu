// Front-to-back blend of the depth-sorted per-tile lists (Eq. 14 with the Eq. 19 alpha).
//
// One CTA per tile (16 x 16, 32 x 16 or 16 x 8 pixels), tiles taken longest list first; each of
// the tw th / P threads owns P pixels (P = 1, 2, 4).  Records of the tile's Gaussians are staged through shared memory in
// depth-ordered chunks (one record per thread); every record is read once per thread and
// serves its P pixels, which share the record's per-column inner terms (col_base: the pixels
// of a thread lie in one or two columns).  The closed form is evaluated in FP32 (FMA pipe + 3 MUFU ops per pair); the CTA
// leaves once all of its pixels have reached T < T_stop.  The per-pixel update is branch-free: a
// pixel that does not blend the visited Gaussian (finished, outside the image or the footprint,
// or below the skip threshold) takes tau = 0 (alpha = 0), which leaves its colour, T and S
// unchanged bit for bit (0.247 ms against 0.270 ms with per-pixel branches).  SPLAT selects the 3DGS comparison
// mode's alpha (Eq. 6) in the same loop.  No tensor cores: the work is not a
// dense contraction.
#include "blend.cuh"

namespace vg {


// One CTA of tw th / P threads per tile.  The register cap is that of 3 / 7 / 12 CTAs of a 16 x 16
// tile per SM for P = 1 / 2 / 4 (the occupancy measured fastest), whatever the tile shape.
template <int P, bool COUNT, bool PIXTEST, bool SPLAT, int CH>
__global__ void __maxnreg__(PixLayout<P>::kFwdRegs)
k_render_fwd(const ViewInfo *__restrict__ views, const int *__restrict__ tile_view, const int *__restrict__ tile_order,
             const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted_item, const float4 *__restrict__ rec,
             const short4 *__restrict__ prect, BlendParams bp, float *__restrict__ rgb, float *__restrict__ T_user, float *__restrict__ T_ws,
             float *__restrict__ S_out, uint32_t *__restrict__ nlast_out, uint32_t *__restrict__ tile_replay,
             unsigned long long *__restrict__ pair_count, L2Fused l2) {
    pdl_entry();
    using L = PixLayout<P>;
    constexpr int kChunk = CH;   // records per barrier
    __shared__ float4 srec[kChunk * kRecF4];
    __shared__ short4 srect[kChunk];
    __shared__ float4 scull[PIXTEST ? 1 : kChunk * kCullF4];   // Gram matrices for the opacity test
    // per record, contiguous for the opacity test: (px0, py0, log2 K, |A0|) and |A1|
    __shared__ float4 sref[PIXTEST ? 1 : kChunk];
    __shared__ float ssq1[PIXTEST ? 1 : kChunk];
    const int tile = tile_order ? tile_order[blockIdx.x] : (int)blockIdx.x;
    const ViewInfo &V = views[tile_view[tile]];
    const int local = tile - V.tile_base;
    const int tyi = local / V.tiles_x, txi = local - tyi * V.tiles_x;
    int ix, iy;
    L::origin(threadIdx.x, V.tw, ix, iy);
    const int x0 = txi * V.tw + ix, y0 = tyi * V.th + iy;
    float Lp[P], T[P], S[P], c0[P], c1[P], c2[P];
    uint32_t last[P];
    const uint2 rg = ranges[tile];
    unsigned live = 0;   // bit k: pixel k is inside the image and not finished
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const int x = x0 + L::ox(k), y = y0 + L::oy(k);
        Lp[k] = SPLAT ? 0.0f : pixel_ray(V, x, y).Lp;
        T[k] = 1.0f;
        S[k] = c0[k] = c1[k] = c2[k] = 0.0f;
        last[k] = rg.x;
        if (x < V.W && y < V.H) live |= 1u << k;
    }
    const float xf = (float)x0, yf = (float)y0;
    const WarpBox wb = warp_box<P>(x0, y0);
    const BoxCull bc = SPLAT ? box_cull_splat(wb, bp.alpha_min) : box_cull(V, wb, bp.tau_skip);
    const int lane = threadIdx.x & 31;
    unsigned long long pairs = 0, blended = 0;   // evaluated / blended pairs (COUNT only)
    for (uint32_t base = rg.x; base < rg.y; base += kChunk) {
        const uint32_t n = min((uint32_t)kChunk, rg.y - base);
        for (uint32_t r = threadIdx.x; r < n; r += blockDim.x) {
            const uint32_t item = sorted_item[base + r];
            const float4 *src = rec + (size_t)item * kRecF4;
            float4 q[kRecF4];
#pragma unroll
            for (int k = 0; k < kRecF4; ++k) {
                q[k] = __ldg(src + k);
                srec[r * kRecF4 + k] = q[k];
            }
            srect[r] = prect[item];
            if (!PIXTEST) {
                float4 c[kCullF4];
                cull_row(q[0], q[1], q[2], q[3], q[4], c);
#pragma unroll
                for (int k = 0; k < kCullF4; ++k) scull[r * kCullF4 + k] = c[k];
                sref[r] = make_float4(q[4].z, q[4].w, q[5].x, sqrtf(c[0].x));
                ssq1[r] = sqrtf(c[0].w);
            }
        }
        __syncthreads();
        // the warp ballots the records whose footprint touches its pixels (and, when pairs below
        // tau_skip are skipped, whose opacity can reach tau_skip there) and visits only those
        for (int w0 = 0; w0 < (int)n; w0 += 32) {
            if (!__any_sync(0xffffffffu, live != 0)) break;
            const int jl = w0 + lane;
            bool need = jl < (int)n && !box_misses(wb, srect[jl]);
            if (!PIXTEST && need) {   // skip records whose opacity stays below tau_skip on this warp
                const float4 *q = &scull[jl * kCullF4];
                const float4 rf = sref[jl];
                need = box_may_blend(q[0], q[1], q[2], rf.x, rf.y, rf.z, rf.w, ssq1[jl], bc);
            }
            unsigned m = __ballot_sync(0xffffffffu, need);
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int j = w0 + b;
                const float4 *r = &srec[j * kRecF4];
                const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3], r4 = r[4], r5 = r[5];
                short4 pr;
                if (PIXTEST) pr = srect[j];
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
                    bool valid = (live >> k) & 1u;
                    if (PIXTEST) valid = valid && !pixel_outside(x0 + L::ox(k), y0 + L::oy(k), pr);
                    float tau, e2, w;
                    if constexpr (SPLAT) {   // Eq. 6: alpha = min(o G'(p), alpha_max)
                        float dx, dy, q;
                        const float a_c =
                            fminf(splat_at(r3, r4, r5, sc[L::ox(k)], L::oy(k) ? yf + (float)L::oy(k) : yf, dx, dy, q), bp.alpha_max);
                        if (COUNT) pairs += valid;
                        valid = valid && a_c >= bp.alpha_min;
                        const float alpha = valid ? a_c : 0.0f;
                        e2 = __fsub_rn(1.0f, alpha);
                        tau = -log1pf(-alpha);
                        w = __fmul_rn(alpha, T[k]);
                    } else {
                        PairEval e;
                        pair_eval_col(r0, r1, r3, r4, r5, cb[L::ox(k)], L::oy(k) ? yf + (float)L::oy(k) : yf, Lp[k], e);
                        if (COUNT) pairs += valid;
                        const float t_c = fminf(e.tau, bp.tau_max);
                        valid = valid && t_c >= bp.tau_skip;
                        tau = valid ? t_c : 0.0f;
                        e2 = ex2_approx(__fmul_rn(-kLog2eF, tau));
                        w = __fmul_rn(__fsub_rn(1.0f, e2), T[k]);
                    }
                    if (COUNT) blended += valid;
                    c0[k] = fmaf(r5.y, w, c0[k]);
                    c1[k] = fmaf(r5.z, w, c1[k]);
                    c2[k] = fmaf(r5.w, w, c2[k]);
                    T[k] = __fmul_rn(T[k], e2);
                    S[k] = __fadd_rn(S[k], tau);
                    if (valid) last[k] = base + j + 1;
                    if (T[k] < bp.T_stop) live &= ~(1u << k);
                }
            }
        }
        if (__syncthreads_count(live != 0) == 0) break;
    }
    float l2acc = 0.0f;   // this thread's share of sum (rgb - target)^2 (fused loss only)
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const int x = x0 + L::ox(k), y = y0 + L::oy(k);
        if (x >= V.W || y >= V.H) continue;
        const long long pix = V.pix_base + (long long)y * V.W + x;
        if (rgb) {   // absent for the cone-beam projection, which needs T alone
            const float o[3] = {fmaf(T[k], bp.bg[0], c0[k]), fmaf(T[k], bp.bg[1], c1[k]), fmaf(T[k], bp.bg[2], c2[k])};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                rgb[3 * pix + c] = o[c];
                if (l2.target) {   // the operations of k_l2_loss: the same gradient bits
                    const float d = o[c] - l2.target[3 * pix + c];
                    l2.grad[3 * pix + c] = 2.0f * l2.scale * d;
                    l2acc = fmaf(d, d, l2acc);
                }
            }
        }
        T_ws[pix] = T[k];
        if (T_user) T_user[pix] = T[k];
        S_out[pix] = S[k];
        nlast_out[pix] = last[k];
    }
    if (l2.target) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l2acc += __shfl_xor_sync(0xffffffffu, l2acc, o);
        if (lane == 0 && l2acc != 0.0f) atomicAdd(l2.loss, l2acc * l2.scale);
    }
    if (tile_replay) {   // the backward's replay length of this tile: its largest last blended position
        uint32_t m = rg.x;
#pragma unroll
        for (int k = 0; k < P; ++k) m = max(m, last[k]);
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0 && m > rg.x) atomicMax(tile_replay + tile, m - rg.x);
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
static void launch_fwd_ptsc(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                            const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                            const BlendParams &bp, float *rgb, float *T_user, float *T_ws, float *S_out,
                            uint32_t *nlast_out, uint32_t *tile_replay, unsigned long long *pair_count,
                            const L2Fused &l2, cudaStream_t st) {
    const unsigned threads = (unsigned)(bp.tile_px / P);
    if (pair_count)
        pdl_launch(k_render_fwd<P, true, PIXTEST, SPLAT, CH>, (unsigned)n_tiles, threads, 0, st,
            views_d, tile_view, tile_order, ranges, sorted_item, rec, prect, bp, rgb, T_user, T_ws, S_out, nlast_out, tile_replay,
            pair_count, l2);
    else
        pdl_launch(k_render_fwd<P, false, PIXTEST, SPLAT, CH>, (unsigned)n_tiles, threads, 0, st,
            views_d, tile_view, tile_order, ranges, sorted_item, rec, prect, bp, rgb, T_user, T_ws, S_out, nlast_out, tile_replay,
            nullptr, l2);
}

template <int P, bool PIXTEST, bool SPLAT>
static void launch_fwd_pts(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                           const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                           const BlendParams &bp, float *rgb, float *T_user, float *T_ws, float *S_out,
                           uint32_t *nlast_out, uint32_t *tile_replay, unsigned long long *pair_count,
                           const L2Fused &l2, cudaStream_t st) {
    if (bp.chunk_fwd == 64)
        launch_fwd_ptsc<P, PIXTEST, SPLAT, 64>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect,
                                               bp, rgb, T_user, T_ws, S_out, nlast_out, tile_replay, pair_count, l2, st);
    else
        launch_fwd_ptsc<P, PIXTEST, SPLAT, 128>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect,
                                                bp, rgb, T_user, T_ws, S_out, nlast_out, tile_replay, pair_count, l2, st);
}

template <int P, bool PIXTEST>
static void launch_fwd_pt(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                          const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                          const BlendParams &bp, float *rgb, float *T_user, float *T_ws, float *S_out,
                          uint32_t *nlast_out, uint32_t *tile_replay, unsigned long long *pair_count,
                          const L2Fused &l2, cudaStream_t st) {
    if (bp.splat)
        launch_fwd_pts<P, PIXTEST, true>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp,
                                         rgb, T_user, T_ws, S_out, nlast_out, tile_replay, pair_count, l2, st);
    else
        launch_fwd_pts<P, PIXTEST, false>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp,
                                          rgb, T_user, T_ws, S_out, nlast_out, tile_replay, pair_count, l2, st);
}

template <int P>
static void launch_fwd_p(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                         const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                         const BlendParams &bp, float *rgb, float *T_user, float *T_ws, float *S_out,
                         uint32_t *nlast_out, uint32_t *tile_replay, unsigned long long *pair_count,
                         const L2Fused &l2, cudaStream_t st) {
    if (bp.pixel_test)
        launch_fwd_pt<P, true>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, rgb,
                               T_user, T_ws, S_out, nlast_out, tile_replay, pair_count, l2, st);
    else
        launch_fwd_pt<P, false>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, rgb,
                                T_user, T_ws, S_out, nlast_out, tile_replay, pair_count, l2, st);
}

cudaError_t launch_render_fwd(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                              const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                              const BlendParams &bp, int ppt, float *rgb, float *T_user, float *T_ws, float *S_out,
                              uint32_t *nlast_out, uint32_t *tile_replay, unsigned long long *pair_count,
                              const L2Fused &l2, cudaStream_t st, long long *launches) {
    if (n_tiles <= 0) return cudaSuccess;
    if (ppt == 1)
        launch_fwd_p<1>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, rgb, T_user, T_ws, S_out,
                        nlast_out, tile_replay, pair_count, l2, st);
    else if (ppt == 4)
        launch_fwd_p<4>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, rgb, T_user, T_ws, S_out,
                        nlast_out, tile_replay, pair_count, l2, st);
    else
        launch_fwd_p<2>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, rgb, T_user, T_ws, S_out,
                        nlast_out, tile_replay, pair_count, l2, st);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace vg
