// Voxel density query: sigma(x) = sum_g kappa_g exp(-(x - mu)' P (x - mu) / 2) (Eq. 3-4) at the
// centres of a regular grid, for volumetric comparisons of a reconstruction.
//
// Each Gaussian is truncated to the voxel box of its ellipsoid (x - mu)' P (x - mu) <= k^2,
// k^2 = 2 ln 2 e with kappa / sigma_cut = m 2^e, computed in FP32 with a fixed operation order
// (the same rule as the key function).  Gaussians are binned into bricks of 8^3 voxels with the
// scan / radix sort / range kernels of the tile binning; one CTA per brick sums its list at its
// voxels (two per thread), so no atomics are needed and the sum is deterministic.
#include "geometry.cuh"

namespace vg {

constexpr int kBrick = 8;
constexpr int kVoxThreads = 256;              // 2 voxels per thread along z
constexpr int kVoxChunk = 128;                // records per shared-memory chunk
constexpr int kVoxRecF4 = 3;                  // (mu, log2 kappa), (P00 P01 P02 P11), (P12 P22 - -)

// Truncation box, record and brick count of every Gaussian.
template <typename RT>
__global__ void __launch_bounds__(256)
k_voxel_pre(GaussIn g, VoxelGrid grid, float sigma_cut, float4 *__restrict__ rec, short4 *__restrict__ box,
            uint32_t *__restrict__ count) {
    pdl_entry();
    for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < g.n;
         gi += (long long)gridDim.x * blockDim.x) {
        float mu[3], s[3], q[4], kin, Sig[9], Rq[9], qn[4], smax;
        load_gauss<RT>(g, gi, mu, s, q, kin);
        const Density dn = density_of(g, kin, s);
        short4 b0 = make_short4(-1, -1, -1, -1), b1 = make_short4(-1, -1, 0, 0);
        uint32_t cnt = 0;
        if (key_cov(mu, s, q, dn.kap_key, Sig, Rq, qn, smax)) {
            const float xr = VG_DIV(dn.kap_key, sigma_cut);
            if (xr > 1.0f) {
                const int e = (xr > FLT_MAX) ? 128 : (int)((__float_as_uint(xr) >> 23) & 0xFFu) - 126;
                const float k2 = VG_MUL((float)e, 1.3862944f);
                const float o[3] = {grid.ox, grid.oy, grid.oz}, v[3] = {grid.vx, grid.vy, grid.vz};
                const int n[3] = {grid.nx, grid.ny, grid.nz};
                int lo[3], hi[3];
                bool ok = true;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float h = VG_SQRT(VG_MUL(k2, Sig[4 * a]));
                    const float c = VG_SUB(mu[a], o[a]);
                    const float flo = VG_SUB(VG_DIV(VG_SUB(c, h), v[a]), 0.5f);
                    const float fhi = VG_SUB(VG_DIV(VG_ADD(c, h), v[a]), 0.5f);
                    pixel_span(flo, fhi, n[a], lo[a], hi[a]);
                    ok = ok && lo[a] <= hi[a];
                }
                if (ok) {
                    b0 = make_short4((short)lo[0], (short)lo[1], (short)lo[2], (short)hi[0]);
                    b1 = make_short4((short)hi[1], (short)hi[2], 0, 0);
                    cnt = (uint32_t)(hi[0] / kBrick - lo[0] / kBrick + 1) * (uint32_t)(hi[1] / kBrick - lo[1] / kBrick + 1) *
                          (uint32_t)(hi[2] / kBrick - lo[2] / kBrick + 1);
                    // precision P = Rq diag(1/s^2) Rq^T (columns of Rq are the principal axes)
                    float P[6];
                    const float w0 = 1.0f / (s[0] * s[0]), w1 = 1.0f / (s[1] * s[1]), w2 = 1.0f / (s[2] * s[2]);
                    const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        const int i = ij[k][0], j = ij[k][1];
                        P[k] = Rq[3 * i] * Rq[3 * j] * w0 + Rq[3 * i + 1] * Rq[3 * j + 1] * w1 +
                               Rq[3 * i + 2] * Rq[3 * j + 2] * w2;
                    }
                    float4 *r = rec + gi * kVoxRecF4;
                    r[0] = make_float4(mu[0], mu[1], mu[2], log2f(dn.kap));
                    r[1] = make_float4(P[0], P[1], P[2], P[3]);
                    r[2] = make_float4(P[4], P[5], 0.0f, 0.0f);
                }
            }
        }
        box[2 * gi] = b0;
        box[2 * gi + 1] = b1;
        count[gi] = cnt;
    }
}

// (brick, Gaussian) instances in Gaussian order; brick id = (bz * bricks_y + by) * bricks_x + bx.
__global__ void __launch_bounds__(256)
k_voxel_dup(const uint32_t *__restrict__ offsets, const short4 *__restrict__ box, VoxelGrid grid, long long n,
            uint32_t *__restrict__ inst_key, uint32_t *__restrict__ inst_val, long long capacity) {
    pdl_entry();
    for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < n;
         gi += (long long)gridDim.x * blockDim.x) {
        const uint32_t off = offsets[gi], end = offsets[gi + 1];
        if (end == off) continue;
        const short4 b0 = box[2 * gi], b1 = box[2 * gi + 1];
        long long o = off;
        for (int bz = b0.z / kBrick; bz <= b1.y / kBrick; ++bz)
            for (int by = b0.y / kBrick; by <= b1.x / kBrick; ++by)
                for (int bx = b0.x / kBrick; bx <= b0.w / kBrick; ++bx, ++o)
                    if (o < capacity) {
                        inst_key[o] = (uint32_t)((bz * grid.by + by) * grid.bx + bx);
                        inst_val[o] = (uint32_t)gi;
                    }
    }
}

// One CTA per brick: thread t owns voxels (x, y, z0) and (x, y, z0 + 1) of the brick with
// x = t % 8, y = (t / 8) % 8, z0 = 2 (t / 64); a warp owns an 8 x 4 x 2 box.
__global__ void __launch_bounds__(kVoxThreads)
k_voxel_eval(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted, const float4 *__restrict__ rec,
             const short4 *__restrict__ box, VoxelGrid grid, float *__restrict__ out) {
    pdl_entry();
    __shared__ float4 srec[kVoxChunk * kVoxRecF4];
    __shared__ short4 sbox[kVoxChunk * 2];
    const int brick = blockIdx.x;
    const int bxi = brick % grid.bx, byi = (brick / grid.bx) % grid.by, bzi = brick / (grid.bx * grid.by);
    const int t = threadIdx.x, lane = t & 31;
    const int i = bxi * kBrick + (t & 7), j = byi * kBrick + ((t >> 3) & 7), k0 = bzi * kBrick + 2 * (t >> 6);
    // the warp's box (voxel indices, inclusive)
    const int wx0 = bxi * kBrick, wx1 = wx0 + kBrick - 1;
    const int wy0 = byi * kBrick + 4 * ((t >> 5) & 1), wy1 = wy0 + 3;
    const int wz0 = bzi * kBrick + 2 * (t >> 6), wz1 = wz0 + 1;
    const float x = VG_ADD(grid.ox, VG_MUL((float)i + 0.5f, grid.vx));
    const float y = VG_ADD(grid.oy, VG_MUL((float)j + 0.5f, grid.vy));
    const float z[2] = {VG_ADD(grid.oz, VG_MUL((float)k0 + 0.5f, grid.vz)),
                        VG_ADD(grid.oz, VG_MUL((float)k0 + 1.5f, grid.vz))};
    float sum[2] = {0.0f, 0.0f};
    const uint2 rg = ranges[brick];
    for (uint32_t base = rg.x; base < rg.y; base += kVoxChunk) {
        const int n = (int)min((uint32_t)kVoxChunk, rg.y - base);
        __syncthreads();
        for (int r = t; r < n; r += kVoxThreads) {
            const uint32_t gi = sorted[base + r];
#pragma unroll
            for (int c = 0; c < kVoxRecF4; ++c) srec[r * kVoxRecF4 + c] = __ldg(rec + (size_t)gi * kVoxRecF4 + c);
            sbox[2 * r] = box[2 * gi];
            sbox[2 * r + 1] = box[2 * gi + 1];
        }
        __syncthreads();
        for (int w0 = 0; w0 < n; w0 += 32) {
            const int jl = w0 + lane;
            bool need = false;
            if (jl < n) {
                const short4 a = sbox[2 * jl], b = sbox[2 * jl + 1];
                need = !(a.w < wx0 || a.x > wx1 || b.x < wy0 || a.y > wy1 || b.y < wz0 || a.z > wz1);
            }
            unsigned m = __ballot_sync(0xffffffffu, need);
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                const int jj = w0 + bit;
                const short4 a = sbox[2 * jj], b = sbox[2 * jj + 1];
                const float4 r0 = srec[jj * kVoxRecF4], r1 = srec[jj * kVoxRecF4 + 1], r2 = srec[jj * kVoxRecF4 + 2];
                const bool inxy = i >= a.x && i <= a.w && j >= a.y && j <= b.x;
                const float dx = x - r0.x, dy = y - r0.y;
                const float pxy = fmaf(r1.x * dx, dx, fmaf(2.0f * r1.y * dx, dy, r1.w * dy * dy));
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int k = k0 + c;
                    const float dz = z[c] - r0.z;
                    const float m2 = pxy + dz * fmaf(2.0f * r1.z, dx, fmaf(2.0f * r2.x, dy, r2.y * dz));
                    const float val = ex2_approx(fmaf(m2, -0.72134752f, r0.w));
                    sum[c] += (inxy && k >= a.z && k <= b.y) ? val : 0.0f;
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int k = k0 + c;
        if (i < grid.nx && j < grid.ny && k < grid.nz) out[((size_t)k * grid.ny + j) * grid.nx + i] = sum[c];
    }
}

cudaError_t launch_voxel_pre(const GaussIn &g, const VoxelGrid &grid, float sigma_cut, float4 *rec, short4 *box,
                             uint32_t *count, cudaStream_t st, long long *launches) {
    if (g.n <= 0) return cudaSuccess;
    long long b = (g.n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (g.rec_dtype == VG_BF16)
        pdl_launch(k_voxel_pre<__nv_bfloat16>, (unsigned)b, 256, 0, st, g, grid, sigma_cut, rec, box, count);
    else if (g.rec_dtype == VG_F16)
        pdl_launch(k_voxel_pre<__half>, (unsigned)b, 256, 0, st, g, grid, sigma_cut, rec, box, count);
    else
        pdl_launch(k_voxel_pre<float>, (unsigned)b, 256, 0, st, g, grid, sigma_cut, rec, box, count);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_voxel_dup(const uint32_t *offsets, const short4 *box, const VoxelGrid &grid, long long n,
                             uint32_t *inst_key, uint32_t *inst_val, long long capacity, cudaStream_t st,
                             long long *launches) {
    if (n <= 0) return cudaSuccess;
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    pdl_launch(k_voxel_dup, (unsigned)b, 256, 0, st, offsets, box, grid, n, inst_key, inst_val, capacity);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_voxel_eval(const uint2 *ranges, const uint32_t *sorted, const float4 *rec, const short4 *box,
                              const VoxelGrid &grid, float *out, cudaStream_t st, long long *launches) {
    const long long bricks = (long long)grid.bx * grid.by * grid.bz;
    if (bricks <= 0) return cudaSuccess;
    pdl_launch(k_voxel_eval, (unsigned)bricks, kVoxThreads, 0, st, ranges, sorted, rec, box, grid, out);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace vg
