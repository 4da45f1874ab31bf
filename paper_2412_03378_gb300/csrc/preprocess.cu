// Per-(view, Gaussian) preprocessing: key function (depth key + conservative tile
// rectangle), view-dependent colour and the blend record.  One thread per item; the
// kernel is bound by the HBM traffic of the Gaussian parameters and the records.
#include "geometry.cuh"

namespace vg {

template <typename RT, typename ST>
__global__ void __launch_bounds__(256)
k_preprocess(GaussIn g, const ViewInfo *__restrict__ views, int n_views, float z_near, float tau_cut,
             float4 *__restrict__ rec, uint32_t *__restrict__ depth, uint32_t *__restrict__ count,
             short4 *__restrict__ rect, short4 *__restrict__ prect, unsigned long long *__restrict__ n_visible) {
    const long long n_items = (long long)g.n * n_views;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < n_items; it += stride) {
        const int v = (int)(it / g.n);
        const long long gi = it - (long long)v * g.n;
        const ViewInfo &V = views[v];
        float mu[3], s[3], q[4], kap;
        load_gauss<RT>(g, gi, mu, s, q, kap);
        float Sig[9], Rq[9], qn[4], smax, Zf;
        uint32_t dk = 0xFFFFFFFFu;
        short4 rc = make_short4(-1, -1, -1, -1), prc = make_short4(-1, -1, -1, -1);
        int state = 0;
        if (key_cov(mu, s, q, kap, Sig, Rq, qn, smax))
            state = key_persp(V, mu, Sig, smax, kap, z_near, tau_cut, dk, rc, prc, Zf);
        uint32_t cnt = 0;
        if (state == 2) {
            cnt = (uint32_t)(rc.z - rc.x + 1) * (uint32_t)(rc.w - rc.y + 1);
            ItemGeom G;
            item_geom(V, mu, s, Rq, G);
            float dir[3], len, rgb[3], raw[3];
            view_dir(V, mu, dir, len);
            eval_colour<ST>(g, gi, dir, rgb, raw);
            const float lnK2 = log2f(kap) + kLog2Sqrt2Pi;
            float4 *r = rec + it * kRecF4;
            r[0] = make_float4(G.A[0], G.A[1], G.A[2], G.A[3]);
            r[1] = make_float4(G.A[4], G.A[5], G.A[6], G.A[7]);
            r[2] = make_float4(G.A[8], G.Cc[0], G.Cc[1], G.Cc[2]);
            r[3] = make_float4(G.Cc[3], G.Cc[4], G.Cc[5], G.Cc[6]);
            r[4] = make_float4(G.Cc[7], G.Cc[8], G.px0, G.py0);
            r[5] = make_float4(lnK2, rgb[0], rgb[1], rgb[2]);
        } else {
            rc = make_short4(-1, -1, -1, -1);
            prc = rc;
        }
        depth[it] = (state >= 1) ? dk : 0xFFFFFFFFu;
        count[it] = cnt;
        rect[it] = rc;
        prect[it] = prc;
        const unsigned am = __activemask();
        const unsigned vis = __ballot_sync(am, state == 2);
        if ((int)(threadIdx.x & 31) == __ffs(am) - 1 && vis) atomicAdd(n_visible, (unsigned long long)__popc(vis));
    }
}

template <typename RT, typename ST>
static cudaError_t launch_pre_t(const GaussIn &g, const ViewInfo *views_d, int n_views, float z_near, float tau_cut,
                                float4 *rec, uint32_t *depth, uint32_t *count, short4 *rect, short4 *prect,
                                unsigned long long *n_visible, cudaStream_t st) {
    const long long n_items = (long long)g.n * n_views;
    long long blocks = (n_items + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    k_preprocess<RT, ST><<<(unsigned)blocks, 256, 0, st>>>(g, views_d, n_views, z_near, tau_cut, rec, depth, count,
                                                           rect, prect, n_visible);
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
