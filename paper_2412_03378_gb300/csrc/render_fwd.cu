// Front-to-back blend of the depth-sorted per-tile lists (Eq. 14 with the Eq. 19 alpha).
//
// One CTA per 16x16 tile, one thread per pixel.  Records of the tile's Gaussians are staged
// through shared memory in chunks of 256 in depth order; every pixel evaluates the closed
// form in FP32 (FMA pipe + 3 MUFU ops per pair) and the CTA leaves as soon as all of its
// pixels have reached T < T_stop.  No tensor cores: the work is not a dense contraction.
#include "blend.cuh"

namespace vg {

template <bool COUNT>
__global__ void __launch_bounds__(kTilePix)
k_render_fwd(const ViewInfo *__restrict__ views, const int *__restrict__ tile_view, const uint2 *__restrict__ ranges,
             const uint32_t *__restrict__ sorted_item, const float4 *__restrict__ rec, BlendParams bp,
             float *__restrict__ rgb, float *__restrict__ T_user, float *__restrict__ T_ws, float *__restrict__ S_out,
             uint32_t *__restrict__ nlast_out, unsigned long long *__restrict__ pair_count) {
    __shared__ float4 srec[kTilePix * kRecF4];
    const int tile = blockIdx.x;
    const ViewInfo &V = views[tile_view[tile]];
    const int local = tile - V.tile_base;
    const int tyi = local / V.tiles_x, txi = local - tyi * V.tiles_x;
    const int x = txi * kTile + (threadIdx.x & (kTile - 1)), y = tyi * kTile + (threadIdx.x / kTile);
    const bool inside = x < V.W && y < V.H;
    const PixelRay pr = pixel_ray(V, x, y);
    const uint2 rg = ranges[tile];

    float T = 1.0f, S = 0.0f, c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
    uint32_t last = rg.x;
    bool done = !inside;
    unsigned long long pairs = 0;
    for (uint32_t base = rg.x; base < rg.y; base += kTilePix) {
        const uint32_t n = min((uint32_t)kTilePix, rg.y - base);
        if (threadIdx.x < n) {
            const float4 *src = rec + (size_t)sorted_item[base + threadIdx.x] * kRecF4;
#pragma unroll
            for (int k = 0; k < kRecF4; ++k) srec[threadIdx.x * kRecF4 + k] = __ldg(src + k);
        }
        __syncthreads();
        if (!done) {
            for (uint32_t j = 0; j < n; ++j) {
                const float4 *r = &srec[j * kRecF4];
                const float4 r5 = r[5];
                PairEval e;
                eval_pair(r[0], r[1], r[2], r[3], r[4], r5, pr, e);
                if (COUNT) ++pairs;
                const float tau = fminf(e.tau, bp.tau_max);
                if (tau < bp.tau_skip) continue;
                const float e2 = ex2_approx(__fmul_rn(-kLog2eF, tau));
                const float w = __fmul_rn(__fsub_rn(1.0f, e2), T);
                c0 = fmaf(r5.y, w, c0);
                c1 = fmaf(r5.z, w, c1);
                c2 = fmaf(r5.w, w, c2);
                T = __fmul_rn(T, e2);
                S = __fadd_rn(S, tau);
                last = base + j + 1;
                if (T < bp.T_stop) {
                    done = true;
                    break;
                }
            }
        }
        if (__syncthreads_count(!done) == 0) break;
    }
    if (inside) {
        const long long pix = V.pix_base + (long long)y * V.W + x;
        rgb[3 * pix + 0] = fmaf(T, bp.bg[0], c0);
        rgb[3 * pix + 1] = fmaf(T, bp.bg[1], c1);
        rgb[3 * pix + 2] = fmaf(T, bp.bg[2], c2);
        T_ws[pix] = T;
        if (T_user) T_user[pix] = T;
        S_out[pix] = S;
        nlast_out[pix] = last;
    }
    if (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        if ((threadIdx.x & 31) == 0 && pairs) atomicAdd(pair_count, pairs);
    }
}

cudaError_t launch_render_fwd(const ViewInfo *views_d, const int *tile_view, long long n_tiles, const uint2 *ranges,
                              const uint32_t *sorted_item, const float4 *rec, const BlendParams &bp, float *rgb,
                              float *T_user, float *T_ws, float *S_out, uint32_t *nlast_out,
                              unsigned long long *pair_count, cudaStream_t st, long long *launches) {
    if (n_tiles <= 0) return cudaSuccess;
    if (pair_count)
        k_render_fwd<true><<<(unsigned)n_tiles, kTilePix, 0, st>>>(views_d, tile_view, ranges, sorted_item, rec, bp,
                                                                  rgb, T_user, T_ws, S_out, nlast_out, pair_count);
    else
        k_render_fwd<false><<<(unsigned)n_tiles, kTilePix, 0, st>>>(views_d, tile_view, ranges, sorted_item, rec, bp,
                                                                   rgb, T_user, T_ws, S_out, nlast_out, nullptr);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace vg
