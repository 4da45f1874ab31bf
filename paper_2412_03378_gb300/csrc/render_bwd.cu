// Backward of the blend (derived from Eq. 14 and Eq. 19 by the chain rule).
//
// k_render_bwd replays every pixel's list back to front from its stored blended count and
// log-transmittance S = sum tau (no per-pair state is kept by the forward):
//   T_i = exp(-(S_after - tau_i)),  dL/dc_i = g alpha_i T_i,
//   dL/dtau_i = g . (c_i T_{i+1} - R_i) - gT T_end,  R_i = sum_{j>i} c_j alpha_j T_j + T_end bg,
// then differentiates tau with respect to the record (A0..A2, C0..C2, ln kappa).  Per
// Gaussian the 22 partials are summed over the warp with shuffles, over the CTA in shared
// memory, and added to the per-item accumulator with one set of global atomics per
// (tile, Gaussian).  k_chain maps the accumulators to dmu, dscale, dquat, dkappa, dsh.
#include "blend.cuh"
#include "geometry.cuh"

namespace vg {

constexpr int kGradUsed = 22;

template <int P> struct BwdBounds;
template <> struct BwdBounds<1> { static constexpr int kMinBlocks = 2; };
template <> struct BwdBounds<2> { static constexpr int kMinBlocks = 4; };
template <> struct BwdBounds<4> { static constexpr int kMinBlocks = 8; };

// One CTA per tile (longest list first), 256/P threads owning P pixels each.  Per record the
// 22 partials are summed over the thread's pixels in registers, then over the warp by a
// reduce-scatter (lane k ends with partial k), over the CTA in shared memory, and finally
// added to the item's accumulator with one set of global atomics per (tile, Gaussian).
template <int P, bool COUNT, bool PIXTEST>
__global__ void __launch_bounds__(PixLayout<P>::kThreads, BwdBounds<P>::kMinBlocks)
k_render_bwd(const ViewInfo *__restrict__ views, const int *__restrict__ tile_view, const int *__restrict__ tile_order,
             const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted_item, const float4 *__restrict__ rec,
             const short4 *__restrict__ prect, BlendParams bp, const float *__restrict__ T_fin, const float *__restrict__ S_fin,
             const uint32_t *__restrict__ nlast, const float *__restrict__ dL_drgb, const float *__restrict__ dL_dT,
             float *__restrict__ grad_acc, unsigned long long *__restrict__ pair_count) {
    using L = PixLayout<P>;
    constexpr int kThreads = L::kThreads;
    constexpr int kChunk = kThreads < 128 ? kThreads : 128;   // records per shared-memory chunk
    __shared__ float4 srec[kChunk * kRecF4];
    __shared__ float sacc[kChunk * kGradUsed];
    __shared__ uint32_t sitem[kChunk];
    __shared__ short4 srect[kChunk];
    __shared__ uint32_t s_last;

    const int tile = tile_order ? tile_order[blockIdx.x] : (int)blockIdx.x;
    const ViewInfo &V = views[tile_view[tile]];
    const int local = tile - V.tile_base;
    const int tyi = local / V.tiles_x, txi = local - tyi * V.tiles_x;
    int ix, iy;
    L::origin(threadIdx.x, ix, iy);
    const int x0 = txi * kTile + ix, y0 = tyi * kTile + iy;
    const uint2 rg = ranges[tile];
    const int lane = threadIdx.x & 31;

    float Lp[P], S[P], Tafter[P], R0[P], R1[P], R2[P], g0[P], g1[P], g2[P], gTterm[P];
    uint32_t my_last[P];
    uint32_t thr_last = rg.x;
#pragma unroll
    for (int k = 0; k < P; ++k) {
        const int x = x0 + L::ox(k), y = y0 + L::oy(k);
        Lp[k] = pixel_ray(V, x, y).Lp;
        my_last[k] = rg.x;
        S[k] = 0.0f;
        float Tend = 1.0f;
        g0[k] = g1[k] = g2[k] = gTterm[k] = 0.0f;
        if (x < V.W && y < V.H) {
            const long long pix = V.pix_base + (long long)y * V.W + x;
            my_last[k] = nlast[pix];
            S[k] = S_fin[pix];
            Tend = T_fin[pix];
            g0[k] = dL_drgb[3 * pix];
            g1[k] = dL_drgb[3 * pix + 1];
            g2[k] = dL_drgb[3 * pix + 2];
            gTterm[k] = dL_dT ? -dL_dT[pix] * Tend : 0.0f;
        }
        Tafter[k] = ex2_approx(__fmul_rn(-kLog2eF, S[k]));
        R0[k] = Tend * bp.bg[0];
        R1[k] = Tend * bp.bg[1];
        R2[k] = Tend * bp.bg[2];
        thr_last = max(thr_last, my_last[k]);
    }
    if (threadIdx.x == 0) s_last = rg.x;
    __syncthreads();
    if (thr_last > rg.x) atomicMax(&s_last, thr_last);
    __syncthreads();
    const uint32_t tile_last = s_last;
    const uint32_t warp_last = __reduce_max_sync(0xffffffffu, thr_last);
    const WarpBox wb = warp_box<P>(x0, y0);
    const float xf = (float)x0, yf = (float)y0;
    unsigned long long pairs = 0;

    for (uint32_t end = tile_last; end > rg.x;) {
        const uint32_t start = (end - rg.x > (uint32_t)kChunk) ? end - kChunk : rg.x;
        const uint32_t n = end - start;
        if (threadIdx.x < n) {
            const uint32_t item = sorted_item[start + threadIdx.x];
            sitem[threadIdx.x] = item;
            const float4 *src = rec + (size_t)item * kRecF4;
#pragma unroll
            for (int k = 0; k < kRecF4; ++k) srec[threadIdx.x * kRecF4 + k] = __ldg(src + k);
            srect[threadIdx.x] = prect[item];
        }
        for (int k = threadIdx.x; k < kChunk * kGradUsed; k += kThreads) sacc[k] = 0.0f;
        __syncthreads();
        for (int j = (int)n - 1; j >= 0; --j) {
            const uint32_t idx = start + (uint32_t)j;
            const short4 pr = srect[j];
            // warp-uniform: nothing of this warp reached the record, or its footprint misses the warp
            if (idx >= warp_last || box_misses(wb, pr)) continue;
            float gv[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) gv[k] = 0.0f;
            bool any = false;
            if (idx < thr_last) {
                const float4 *r = &srec[j * kRecF4];
                const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3], r4 = r[4], r5 = r[5];
                QuadBase qb;
                quad_base(r0, r1, r2, r3, r4, xf, yf, qb);
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    if (idx >= my_last[k]) continue;
                    if (PIXTEST && pixel_outside(x0 + L::ox(k), y0 + L::oy(k), pr)) continue;
                    PairEval e;
                    pair_eval_at(r0, r1, r2, r3, r5, qb, L::ox(k) != 0, L::oy(k) != 0, Lp[k], e);
                    if (COUNT) ++pairs;
                    const bool clamped = e.tau > bp.tau_max;
                    const float tau = fminf(e.tau, bp.tau_max);
                    if (tau < bp.tau_skip) continue;
                    any = true;
                    const float e2 = ex2_approx(__fmul_rn(-kLog2eF, tau));
                    const float alpha = __fsub_rn(1.0f, e2);
                    const float Sb = S[k] - tau;
                    const float Tb = ex2_approx(-kLog2eF * Sb);
                    const float aT = alpha * Tb;
                    gv[19] = fmaf(g0[k], aT, gv[19]);
                    gv[20] = fmaf(g1[k], aT, gv[20]);
                    gv[21] = fmaf(g2[k], aT, gv[21]);
                    const float dtau = g0[k] * (r5.y * Tafter[k] - R0[k]) + g1[k] * (r5.z * Tafter[k] - R1[k]) +
                                       g2[k] * (r5.w * Tafter[k] - R2[k]) + gTterm[k];
                    R0[k] = fmaf(r5.y, aT, R0[k]);
                    R1[k] = fmaf(r5.z, aT, R1[k]);
                    R2[k] = fmaf(r5.w, aT, R2[k]);
                    S[k] = Sb;
                    Tafter[k] = Tb;
                    if (!clamped) {
                        const float G = dtau * tau;                // dL / d ln(tau)
                        const float r2s = e.rs * e.rs;
                        const float gda = G * r2s * (e.m2 - 1.0f);   // 2 dL/da
                        const float gdq = -G * r2s;                  // 2 dL/dq
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float a_ = gda * e.dp[c], q_ = gdq * e.cr[c];
                            gv[c] = fmaf(a_, e.dx, gv[c]);
                            gv[3 + c] = fmaf(a_, e.dy, gv[3 + c]);
                            gv[6 + c] += a_;
                            gv[9 + c] = fmaf(q_, e.dx, gv[9 + c]);
                            gv[12 + c] = fmaf(q_, e.dy, gv[12 + c]);
                            gv[15 + c] += q_;
                        }
                        gv[18] += G;
                    }
                }
            }
            if (__any_sync(0xffffffffu, any)) {
                const float mine = warp_reduce_scatter<kGradUsed>(gv, lane);
                if (lane < kGradUsed && mine != 0.0f) atomicAdd(&sacc[j * kGradUsed + lane], mine);
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < (int)n * kGradUsed; k += kThreads) {
            const int jj = k / kGradUsed, c = k - jj * kGradUsed;
            const float v = sacc[k];
            if (v != 0.0f) atomicAdd(&grad_acc[(size_t)sitem[jj] * kGradN + c], v);
        }
        __syncthreads();
        end = start;
    }
    if (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        if (lane == 0 && pairs) atomicAdd(pair_count, pairs);
    }
}

template <int P, bool PIXTEST>
static void launch_bwd_pt(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                          const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                          const BlendParams &bp, const float *T_fin, const float *S_fin, const uint32_t *nlast,
                          const float *dL_drgb, const float *dL_dT, float *grad_acc, unsigned long long *pair_count,
                          cudaStream_t st) {
    const unsigned threads = PixLayout<P>::kThreads;
    if (pair_count)
        k_render_bwd<P, true, PIXTEST><<<(unsigned)n_tiles, threads, 0, st>>>(
            views_d, tile_view, tile_order, ranges, sorted_item, rec, prect, bp, T_fin, S_fin, nlast, dL_drgb, dL_dT,
            grad_acc, pair_count);
    else
        k_render_bwd<P, false, PIXTEST><<<(unsigned)n_tiles, threads, 0, st>>>(
            views_d, tile_view, tile_order, ranges, sorted_item, rec, prect, bp, T_fin, S_fin, nlast, dL_drgb, dL_dT,
            grad_acc, nullptr);
}

template <int P>
static void launch_bwd_p(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                         const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                         const BlendParams &bp, const float *T_fin, const float *S_fin, const uint32_t *nlast,
                         const float *dL_drgb, const float *dL_dT, float *grad_acc, unsigned long long *pair_count,
                         cudaStream_t st) {
    if (bp.pixel_test)
        launch_bwd_pt<P, true>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, T_fin,
                               S_fin, nlast, dL_drgb, dL_dT, grad_acc, pair_count, st);
    else
        launch_bwd_pt<P, false>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, T_fin,
                                S_fin, nlast, dL_drgb, dL_dT, grad_acc, pair_count, st);
}

cudaError_t launch_render_bwd(const ViewInfo *views_d, const int *tile_view, const int *tile_order, long long n_tiles,
                              const uint2 *ranges, const uint32_t *sorted_item, const float4 *rec, const short4 *prect,
                              const BlendParams &bp, int ppt, const float *T_fin, const float *S_fin,
                              const uint32_t *nlast, const float *dL_drgb, const float *dL_dT, float *grad_acc,
                              unsigned long long *pair_count, cudaStream_t st, long long *launches) {
    if (n_tiles <= 0) return cudaSuccess;
    if (ppt == 1)
        launch_bwd_p<1>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, T_fin, S_fin, nlast,
                        dL_drgb, dL_dT, grad_acc, pair_count, st);
    else if (ppt == 4)
        launch_bwd_p<4>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, T_fin, S_fin, nlast,
                        dL_drgb, dL_dT, grad_acc, pair_count, st);
    else
        launch_bwd_p<2>(views_d, tile_view, tile_order, n_tiles, ranges, sorted_item, rec, prect, bp, T_fin, S_fin, nlast,
                        dL_drgb, dL_dT, grad_acc, pair_count, st);
    *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- chain
__device__ __forceinline__ void cross_add(const float a[3], const float b[3], float c[3]) {
    c[0] += a[1] * b[2] - a[2] * b[1];
    c[1] += a[2] * b[0] - a[0] * b[2];
    c[2] += a[0] * b[1] - a[1] * b[0];
}

template <typename RT, typename ST>
__global__ void __launch_bounds__(128)
k_chain(GaussIn g, const ViewInfo *__restrict__ views, int n_views, const float *__restrict__ grad_acc,
        float *__restrict__ dmu, float *__restrict__ dscale, float *__restrict__ dquat, float *__restrict__ dkappa,
        float *__restrict__ dsh) {
    const long long n_items = (long long)g.n * n_views;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < n_items;
         it += (long long)gridDim.x * blockDim.x) {
        const float4 *ga4 = (const float4 *)(grad_acc + it * kGradN);
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
        const int v = (int)(it / g.n);
        const long long gi = it - (long long)v * g.n;
        const ViewInfo &V = views[v];
        float mu[3], s[3], q[4], kap, Sig[9], Rq[9], qn[4], smax;
        load_gauss<RT>(g, gi, mu, s, q, kap);
        if (!key_cov(mu, s, q, kap, Sig, Rq, qn, smax)) continue;
        ItemGeom G;
        item_geom(V, mu, s, Rq, G);

        float dA[9], dC[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            dA[k] = ga[k];
            dC[k] = ga[9 + k];
        }
        // The record's C_k = o' x A_k with o' = -M mu_c.  Writing mu_c = t0 dc0 - v0 and
        // o' = Q2 - t0 A2 (t0 = camera depth of the mean, v0 and Q2 small), the two largest
        // terms of dL/dM, -t0 (dC2 x A2) (x) dc0 and -t0 (A2 x dC2) (x) dc0, cancel exactly and are
        // left out; what remains has no large cancelling parts:
        //   dL/dM = sum_k (dA_k + dC_k x Q2) (x) b_k - t0 [(dC0 x A2) (x) b_0 + (dC1 x A2) (x) b_1]
        //           - t0 (A0 x dC0 + A1 x dC1) (x) dc0 + dop (x) v0,   b = (e0/fx, e1/fy, dc0),
        //   dL/dmu_c = -M^T dop,  dop = sum_k A_k x dC_k.
        const float t0 = (float)G.muc[2];
        float Q2[3], v0[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double opd = -(G.M[3 * i] * G.muc[0] + G.M[3 * i + 1] * G.muc[1] + G.M[3 * i + 2] * G.muc[2]);
            Q2[i] = (float)(opd + (double)t0 * (double)G.A[6 + i]);
            v0[i] = (float)((double)t0 * (double)G.dc0[i] - G.muc[i]);
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
        float dsc[3], dB[9];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float is = 1.0f / s[i];
            dsc[i] = -(dM[3 * i] * G.M[3 * i] + dM[3 * i + 1] * G.M[3 * i + 1] + dM[3 * i + 2] * G.M[3 * i + 2]) * is;
#pragma unroll
            for (int j = 0; j < 3; ++j) dB[3 * j + i] = dM[3 * i + j] * is;
        }
        // B = Rc Rq  =>  dRq = Rc^T dB;  mu_c = Rc mu + t  =>  dmu = Rc^T dmu_c
        const float *Rc = V.R;
        float dR[9], dm[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) dR[3 * a + b] = Rc[a] * dB[b] + Rc[3 + a] * dB[3 + b] + Rc[6 + a] * dB[6 + b];
            dm[a] = Rc[a] * dmuc[0] + Rc[3 + a] * dmuc[1] + Rc[6 + a] * dmuc[2];
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
        if (g.sh != nullptr && (ga[19] != 0.0f || ga[20] != 0.0f || ga[21] != 0.0f)) {
            float dir[3], len, rgb[3], raw[3];
            view_dir(V, mu, dir, len);
            eval_colour<ST>(g, gi, dir, rgb, raw);
            float Y[16], dY[16][3];
            sh_basis(g.sh_degree, dir[0], dir[1], dir[2], Y);
            sh_basis_grad(g.sh_degree, dir[0], dir[1], dir[2], dY);
            const int K = (g.sh_degree + 1) * (g.sh_degree + 1);
            const ST *sh = (const ST *)g.sh + gi * K * 3;
            float gd[3] = {0.0f, 0.0f, 0.0f};
            for (int c = 0; c < 3; ++c) {
                if (!(raw[c] > 0.0f)) continue;
                const float gc = ga[19 + c];
                for (int k = 0; k < K; ++k) {
                    if (dsh) atomicAdd(&dsh[(gi * K + k) * 3 + c], gc * Y[k]);
                    const float sc = gc * ld_f<ST>(sh, 3 * k + c);
                    gd[0] = fmaf(sc, dY[k][0], gd[0]);
                    gd[1] = fmaf(sc, dY[k][1], gd[1]);
                    gd[2] = fmaf(sc, dY[k][2], gd[2]);
                }
            }
            const float dd = gd[0] * dir[0] + gd[1] * dir[1] + gd[2] * dir[2];
            const float il = 1.0f / len;
#pragma unroll
            for (int c = 0; c < 3; ++c) dm[c] += (gd[c] - dir[c] * dd) * il;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicAdd(&dmu[3 * gi + c], dm[c]);
            atomicAdd(&dscale[3 * gi + c], dsc[c]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) atomicAdd(&dquat[4 * gi + c], (dqn[c] - qn[c] * dot) / qnorm);
        atomicAdd(&dkappa[gi], ga[18] / kap);
    }
}

template <typename RT, typename ST>
static cudaError_t launch_chain_t(const GaussIn &g, const ViewInfo *views_d, int n_views, const float *grad_acc,
                                  float *dmu, float *dscale, float *dquat, float *dkappa, float *dsh, cudaStream_t st) {
    const long long n_items = (long long)g.n * n_views;
    long long b = (n_items + 127) / 128;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    k_chain<RT, ST><<<(unsigned)b, 128, 0, st>>>(g, views_d, n_views, grad_acc, dmu, dscale, dquat, dkappa, dsh);
    return cudaGetLastError();
}

cudaError_t launch_chain(const GaussIn &g, const ViewInfo *views_d, int n_views, const float *grad_acc, float *dmu,
                         float *dscale, float *dquat, float *dkappa, float *dsh, cudaStream_t st, long long *launches) {
    *launches += 1;
    if (g.rec_dtype == VG_F32) {
        if (g.sh_dtype == VG_F16)
            return launch_chain_t<float, __half>(g, views_d, n_views, grad_acc, dmu, dscale, dquat, dkappa, dsh, st);
        if (g.sh_dtype == VG_BF16)
            return launch_chain_t<float, __nv_bfloat16>(g, views_d, n_views, grad_acc, dmu, dscale, dquat, dkappa, dsh, st);
        return launch_chain_t<float, float>(g, views_d, n_views, grad_acc, dmu, dscale, dquat, dkappa, dsh, st);
    }
    if (g.rec_dtype == VG_BF16) {
        if (g.sh_dtype == VG_F16)
            return launch_chain_t<__nv_bfloat16, __half>(g, views_d, n_views, grad_acc, dmu, dscale, dquat, dkappa, dsh,
                                                         st);
        if (g.sh_dtype == VG_F32)
            return launch_chain_t<__nv_bfloat16, float>(g, views_d, n_views, grad_acc, dmu, dscale, dquat, dkappa, dsh,
                                                        st);
        return launch_chain_t<__nv_bfloat16, __nv_bfloat16>(g, views_d, n_views, grad_acc, dmu, dscale, dquat, dkappa,
                                                            dsh, st);
    }
    if (g.sh_dtype == VG_F32)
        return launch_chain_t<__half, float>(g, views_d, n_views, grad_acc, dmu, dscale, dquat, dkappa, dsh, st);
    if (g.sh_dtype == VG_BF16)
        return launch_chain_t<__half, __nv_bfloat16>(g, views_d, n_views, grad_acc, dmu, dscale, dquat, dkappa, dsh, st);
    return launch_chain_t<__half, __half>(g, views_d, n_views, grad_acc, dmu, dscale, dquat, dkappa, dsh, st);
}

}  // namespace vg
