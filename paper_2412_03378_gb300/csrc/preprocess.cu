// Per-(view, Gaussian) preprocessing: key function (depth key + conservative tile
// rectangle), view-dependent colour and the blend record.  One thread per item, a warp per 32
// consecutive Gaussians of one view.  The SH rows come in through shared memory so that the HBM
// reads (the kernel's bound) are coalesced: FP32 degree-3 rows (SH3) as 16-byte pieces, other rows
// element by element.  Each visible item's 96-byte record goes out from registers as six 16-byte
// stores (records of culled items are never read and are not written).
#include "geometry.cuh"

namespace vg {

constexpr int kPreWarps = 4;   // warps per CTA; each owns 32 consecutive Gaussians of one view at a time

template <typename RT, typename ST, bool SH3>
__global__ void __launch_bounds__(32 * kPreWarps, 5)
k_preprocess(GaussIn g, const ViewInfo *__restrict__ views, int n_views, float z_near, float tau_cut,
             float4 *__restrict__ rec, uint32_t *__restrict__ depth, uint32_t *__restrict__ count,
             short4 *__restrict__ rect, short4 *__restrict__ prect, unsigned long long *__restrict__ n_visible) {
    pdl_entry();
    // SH rows: kRowStride floats per row, or (SH3) kRow16 float4
    __shared__ __align__(16) float sbuf[kPreWarps][32 * (SH3 ? 4 * kRow16 : kRowStride)];
    const int lane = threadIdx.x & 31;
    float *buf = sbuf[threadIdx.x >> 5];
    float *row = buf + lane * (SH3 ? 4 * kRow16 : kRowStride);
    const int K3 = 3 * (g.sh_degree + 1) * (g.sh_degree + 1);
    const long long per_view = ((long long)g.n + 31) / 32;
    const long long n_chunks = per_view * n_views;
    for (long long ch = (long long)blockIdx.x * kPreWarps + (threadIdx.x >> 5); ch < n_chunks;
         ch += (long long)gridDim.x * kPreWarps) {
        const int v = (int)(ch / per_view);
        const long long gbase = (ch - (long long)v * per_view) * 32;
        const int nloc = (int)min(32LL, (long long)g.n - gbase);
        const long long gi = gbase + lane;
        const long long it = (long long)v * g.n + gi;
        // the SH rows of the warp's Gaussians, coalesced, before (and independent of) the key; the
        // parameter loads are issued before the wait so that both round trips overlap
        if (SH3)
            warp_load_sh3((const float *)g.sh + gbase * K3, nloc, reinterpret_cast<float4 *>(buf), lane);
        else if (g.sh)
            warp_load_rows<ST>((const ST *)g.sh + gbase * K3, nloc, K3, buf, lane);
        float mu[3], s[3], q[4], kin;
        if (lane < nloc) load_gauss<RT>(g, gi, mu, s, q, kin);
        rows_wait();
        __syncwarp();
        const ViewInfo &V = views[v];
        int state = 0;
        uint32_t cnt = 0, dk = 0xFFFFFFFFu;
        short4 rc = make_short4(-1, -1, -1, -1), prc = rc;
        if (lane < nloc) {
            const Density dn = density_of(g, kin, s);
            float Sig[9], Rq[9], qn[4], smax, Zf;
            if (key_cov(mu, s, q, dn.kap_key, Sig, Rq, qn, smax)) {
                if (g.splat)
                    state = key_splat(V, mu, Sig, dn.kap_key, z_near, tau_cut, g.splat_dil, dk, rc, prc);
                else
                    state = key_persp(V, mu, Sig, smax, dn.kap_key, z_near, tau_cut, dk, rc, prc, Zf);
            }
            if (state == 2) {
                cnt = (uint32_t)(rc.z - rc.x + 1) * (uint32_t)(rc.w - rc.y + 1);
                float dir[3], len, rgb[3] = {0.0f, 0.0f, 0.0f}, raw[3];
                float rrow[4 * kRecF4];
                view_dir(V, mu, dir, len);
                if (SH3)
                    eval_colour_sh3(reinterpret_cast<const float4 *>(row), dir, rgb, raw, g.softplus_beta);
                else if (g.sh)
                    eval_colour_row(g.sh_degree, row, dir, rgb, raw, g.softplus_beta);   // else density only
                if (g.splat) {
                    SplatGeom SG;
                    if (splat_geom(V, mu, s, Rq, g.splat_dil, SG)) {
                        rrow[20] = splat_record(SG, dn.kap, rrow);
                    } else {   // degenerate 2D covariance: listed by the key, but alpha = 0
#pragma unroll
                        for (int k = 0; k < 20; ++k) rrow[k] = 0.0f;
                        rrow[20] = -INFINITY;
                    }
                } else {
                    ItemGeom G;
                    item_geom(V, mu, s, Rq, G);
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        rrow[k] = G.A[k];
                        rrow[9 + k] = G.Cc[k];
                    }
                    rrow[18] = G.px0;
                    rrow[19] = G.py0;
                    rrow[20] = log2f(dn.kap) + kLog2Sqrt2Pi;
                }
                rrow[21] = rgb[0];
                rrow[22] = rgb[1];
                rrow[23] = rgb[2];
                float4 *dst = rec + it * kRecF4;
#pragma unroll
                for (int k = 0; k < kRecF4; ++k)
                    dst[k] = make_float4(rrow[4 * k], rrow[4 * k + 1], rrow[4 * k + 2], rrow[4 * k + 3]);
            } else {
                rc = make_short4(-1, -1, -1, -1);
                prc = rc;
            }
            depth[it] = (state >= 1) ? dk : 0xFFFFFFFFu;
            count[it] = cnt;
            rect[it] = rc;
            prect[it] = prc;
        }
        const unsigned vis = __ballot_sync(0xffffffffu, state == 2);
        if (lane == 0 && vis) atomicAdd(n_visible, (unsigned long long)__popc(vis));
        __syncwarp();   // the buffer is reused by the next chunk
    }
}

template <typename RT, typename ST>
static cudaError_t launch_pre_t(const GaussIn &g, const ViewInfo *views_d, int n_views, float z_near, float tau_cut,
                                float4 *rec, uint32_t *depth, uint32_t *count, short4 *rect, short4 *prect,
                                unsigned long long *n_visible, cudaStream_t st) {
    const long long chunks = ((long long)g.n + 31) / 32 * n_views;
    long long blocks = (chunks + kPreWarps - 1) / kPreWarps;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    // FP32 degree-3 SH rows of a 16-byte aligned array: 16-byte copies
    if (sh3_rows<ST>(g))
        pdl_launch(k_preprocess<RT, ST, true>, (unsigned)blocks, 32 * kPreWarps, 0, st, g, views_d, n_views, z_near,
                   tau_cut, rec, depth, count, rect, prect, n_visible);
    else
        pdl_launch(k_preprocess<RT, ST, false>, (unsigned)blocks, 32 * kPreWarps, 0, st, g, views_d, n_views, z_near,
                   tau_cut, rec, depth, count, rect, prect, n_visible);
    return cudaGetLastError();
}

cudaError_t launch_preprocess(const GaussIn &g, const ViewInfo *views_d, int n_views, float z_near, float tau_cut,
                              float4 *rec, uint32_t *depth, uint32_t *count, short4 *rect, short4 *prect,
                              unsigned long long *n_visible, cudaStream_t st, long long *launches) {
    *launches += 1;
    if (g.rec_dtype == VG_F32) {
        if (g.sh_dtype == VG_F32)
            return launch_pre_t<float, float>(g, views_d, n_views, z_near, tau_cut, rec, depth, count, rect, prect, n_visible, st);
        if (g.sh_dtype == VG_F16)
            return launch_pre_t<float, __half>(g, views_d, n_views, z_near, tau_cut, rec, depth, count, rect, prect, n_visible, st);
        return launch_pre_t<float, __nv_bfloat16>(g, views_d, n_views, z_near, tau_cut, rec, depth, count, rect,
                                                  prect, n_visible, st);
    }
    if (g.rec_dtype == VG_BF16) {
        if (g.sh_dtype == VG_F16)
            return launch_pre_t<__nv_bfloat16, __half>(g, views_d, n_views, z_near, tau_cut, rec, depth, count, rect,
                                                       prect, n_visible, st);
        if (g.sh_dtype == VG_F32)
            return launch_pre_t<__nv_bfloat16, float>(g, views_d, n_views, z_near, tau_cut, rec, depth, count, rect,
                                                      prect, n_visible, st);
        return launch_pre_t<__nv_bfloat16, __nv_bfloat16>(g, views_d, n_views, z_near, tau_cut, rec, depth, count,
                                                          rect, prect, n_visible, st);
    }
    if (g.sh_dtype == VG_F16)
        return launch_pre_t<__half, __half>(g, views_d, n_views, z_near, tau_cut, rec, depth, count, rect, prect, n_visible, st);
    if (g.sh_dtype == VG_F32)
        return launch_pre_t<__half, float>(g, views_d, n_views, z_near, tau_cut, rec, depth, count, rect, prect, n_visible, st);
    return launch_pre_t<__half, __nv_bfloat16>(g, views_d, n_views, z_near, tau_cut, rec, depth, count, rect, prect,
                                               n_visible, st);
}

}  // namespace vg
