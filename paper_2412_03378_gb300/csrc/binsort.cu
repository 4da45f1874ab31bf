// Tile binning and sorting: device-wide exclusive scan, a stable LSD radix sort of
// (uint32 key, uint32 value) pairs, instance duplication and per-tile ranges.
//
// The per-tile front-to-back order (tile, depth, Gaussian index) is built in two stable
// steps: items are sorted by depth key (ties keep index order), their instances are
// emitted in that order, and a second stable sort on the tile id alone groups them by tile
// without disturbing the depth order inside each tile.
#include "vg_internal.cuh"

namespace vg {

// ---------------------------------------------------------------------------- scan
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

size_t scan_tmp_words(long long n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1024; }

__device__ __forceinline__ uint32_t load_count(const uint32_t *in, const uint32_t *perm, long long i) {
    return perm ? in[perm[i]] : in[i];
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t *__restrict__ in, const uint32_t *__restrict__ perm, long long n,
              uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t warp_sums[kScanThreads / 32];
    const long long base = (long long)blockIdx.x * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + k * kScanThreads + threadIdx.x;
        if (i < n) s += load_count(in, perm, i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t t = threadIdx.x < kScanThreads / 32 ? warp_sums[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) block_sums[blockIdx.x] = t;
    }
}

// Exclusive scan of the block sums by one block; writes the grand total to *total.
__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *__restrict__ sums, int nb, uint32_t *__restrict__ total) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        uint32_t v = i < nb ? sums[i] : 0;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t w = warp_tot[threadIdx.x];
            uint32_t xw = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, xw, o);
                if (threadIdx.x >= o) xw += y;
            }
            warp_tot[threadIdx.x] = xw - w;   // exclusive
        }
        __syncthreads();
        uint32_t excl = carry + warp_tot[threadIdx.x >> 5] + x - v;
        if (i < nb) sums[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_down(const uint32_t *__restrict__ in, const uint32_t *__restrict__ perm, long long n,
            const uint32_t *__restrict__ block_off, uint32_t *__restrict__ out) {
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + k;
        v[k] = i < n ? load_count(in, perm, i) : 0;
        s += v[k];
    }
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t w = threadIdx.x < kScanThreads / 32 ? warp_tot[threadIdx.x] : 0;
        uint32_t xw = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, xw, o);
            if (threadIdx.x >= o) xw += y;
        }
        if (threadIdx.x < kScanThreads / 32) warp_tot[threadIdx.x] = xw - w;
    }
    __syncthreads();
    uint32_t run = block_off[blockIdx.x] + warp_tot[threadIdx.x >> 5] + x - s;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
}

__global__ void k_write_total(const uint32_t *total, uint32_t *out, long long n) { out[n] = *total; }

cudaError_t launch_scan_gather(const uint32_t *count, const uint32_t *perm, uint32_t *out, long long n, uint32_t *tmp,
                               cudaStream_t st, long long *launches) {
    const long long nb = (n + kScanTile - 1) / kScanTile;
    uint32_t *sums = tmp, *total = tmp + nb;
    if (nb > 0) {
        k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(count, perm, n, sums);
        *launches += 1;
    }
    k_scan_top<<<1, 1024, 0, st>>>(sums, (int)nb, total);
    *launches += 1;
    if (nb > 0) {
        k_scan_down<<<(unsigned)nb, kScanThreads, 0, st>>>(count, perm, n, sums, out);
        *launches += 1;
    }
    k_write_total<<<1, 1, 0, st>>>(total, out, n);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t *in, uint32_t *out, long long n, uint32_t *tmp, cudaStream_t st,
                        long long *launches) {
    return launch_scan_gather(in, nullptr, out, n, tmp, st, launches);
}

// ---------------------------------------------------------------------------- radix sort
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 8;                         // per thread
constexpr int kRsTile = kRsThreads * kRsItems;      // 2048 keys per block
constexpr int kRsBins = 256;

size_t radix_hist_words(long long n) { return (size_t)kRsBins * (size_t)((n + kRsTile - 1) / kRsTile + 1); }

__global__ void __launch_bounds__(kRsThreads)
k_radix_hist(const uint32_t *__restrict__ keys, long long n, int shift, uint32_t mask, uint32_t *__restrict__ hist,
             int n_blocks) {
    __shared__ uint32_t cnt[kRsBins];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRsTile;
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
        long long i = base + k * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * n_blocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: warp w owns keys [w*256, (w+1)*256) of the block tile and ranks them in
// order, 32 at a time, with __match_any_sync; per-digit warp counts are then scanned
// across warps so every key gets its rank in the tile's original order.
__global__ void __launch_bounds__(kRsThreads)
k_radix_scatter(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals, uint32_t *__restrict__ ko,
                uint32_t *__restrict__ vo, long long n, int shift, uint32_t mask, const uint32_t *__restrict__ hist,
                int n_blocks) {
    __shared__ uint32_t warp_cnt[kRsWarps][kRsBins];
    __shared__ uint32_t digit_base[kRsBins];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRsWarps * kRsBins; i += kRsThreads) (&warp_cnt[0][0])[i] = 0;
    digit_base[threadIdx.x] = hist[(long long)threadIdx.x * n_blocks + blockIdx.x];
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRsTile + w * (kRsItems * 32);
    uint32_t k[kRsItems], v[kRsItems], r[kRsItems];
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        const long long i = base + it * 32 + lane;
        const bool valid = i < n;
        k[it] = valid ? keys[i] : 0u;
        v[it] = valid ? vals[i] : 0u;
        const uint32_t d = valid ? ((k[it] >> shift) & mask) : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t lower = peers & ((1u << lane) - 1u);
        const uint32_t prev = valid ? warp_cnt[w][d] : 0u;
        __syncwarp();
        if (valid && lower == 0u) warp_cnt[w][d] = prev + __popc(peers);
        __syncwarp();
        r[it] = prev + __popc(lower);
    }
    __syncthreads();
    {
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kRsWarps; ++ww) {
            uint32_t c = warp_cnt[ww][threadIdx.x];
            warp_cnt[ww][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        const long long i = base + it * 32 + lane;
        if (i < n) {
            const uint32_t d = (k[it] >> shift) & mask;
            const uint32_t pos = digit_base[d] + warp_cnt[w][d] + r[it];
            ko[pos] = k[it];
            vo[pos] = v[it];
        }
    }
}

cudaError_t launch_radix_sort(uint32_t *keys, uint32_t *vals, uint32_t *keys_tmp, uint32_t *vals_tmp, long long n,
                              int bits, uint32_t *hist, uint32_t *scan_tmp, uint32_t **keys_out, uint32_t **vals_out,
                              cudaStream_t st, long long *launches) {
    uint32_t *ka = keys, *va = vals, *kb = keys_tmp, *vb = vals_tmp;
    const int n_blocks = (int)((n + kRsTile - 1) / kRsTile);
    if (n > 0) {
        for (int shift = 0; shift < bits; shift += 8) {
            const int nbits = bits - shift < 8 ? bits - shift : 8;
            const uint32_t mask = (1u << nbits) - 1u;
            k_radix_hist<<<n_blocks, kRsThreads, 0, st>>>(ka, n, shift, mask, hist, n_blocks);
            *launches += 1;
            cudaError_t e = launch_scan(hist, hist, (long long)kRsBins * n_blocks, scan_tmp, st, launches);
            if (e != cudaSuccess) return e;
            k_radix_scatter<<<n_blocks, kRsThreads, 0, st>>>(ka, va, kb, vb, n, shift, mask, hist, n_blocks);
            *launches += 1;
            uint32_t *t = ka; ka = kb; kb = t;
            t = va; va = vb; vb = t;
        }
    }
    *keys_out = ka;
    *vals_out = va;
    return cudaGetLastError();
}

__global__ void k_iota(uint32_t *v, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = (uint32_t)i;
}

cudaError_t launch_iota(uint32_t *v, long long n, cudaStream_t st, long long *launches) {
    long long b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    k_iota<<<(unsigned)b, 256, 0, st>>>(v, n);
    *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- duplicate
__global__ void __launch_bounds__(256)
k_duplicate(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ offsets, const short4 *__restrict__ rect,
            const ViewInfo *__restrict__ views, long long n_items, int n_per_view, uint32_t *__restrict__ inst_key,
            uint32_t *__restrict__ inst_val, long long capacity) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_items;
         i += (long long)gridDim.x * blockDim.x) {
        const uint32_t off = offsets[i], end = offsets[i + 1];
        if (end == off) continue;
        const uint32_t item = perm ? perm[i] : (uint32_t)i;
        const short4 rc = rect[item];
        const int v = (int)(item / (uint32_t)n_per_view);
        const int tb = views[v].tile_base, tx = views[v].tiles_x;
        long long o = off;
        for (int y = rc.y; y <= rc.w; ++y)
            for (int x = rc.x; x <= rc.z; ++x, ++o)
                if (o < capacity) {
                    inst_key[o] = (uint32_t)(tb + y * tx + x);
                    inst_val[o] = item;
                }
    }
}

cudaError_t launch_duplicate(const uint32_t *perm, const uint32_t *offsets, const short4 *rect, const ViewInfo *views,
                             long long n_items, int n_per_view, uint32_t *inst_key, uint32_t *inst_val,
                             long long capacity, cudaStream_t st, long long *launches) {
    long long b = (n_items + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    k_duplicate<<<(unsigned)b, 256, 0, st>>>(perm, offsets, rect, views, n_items, n_per_view, inst_key, inst_val,
                                            capacity);
    *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- ranges
__global__ void k_ranges(const uint32_t *__restrict__ key, long long n, uint2 *__restrict__ ranges) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t t = key[i];
        if (i == 0 || key[i - 1] != t) ranges[t].x = (uint32_t)i;
        if (i == n - 1 || key[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
    }
}

cudaError_t launch_ranges(const uint32_t *sorted_key, long long n_inst, uint2 *ranges, long long n_tiles,
                          cudaStream_t st, long long *launches) {
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, st);
    if (e != cudaSuccess) return e;
    if (n_inst > 0) {
        long long b = (n_inst + 255) / 256;
        if (b > 152 * 64) b = 152 * 64;
        k_ranges<<<(unsigned)b, 256, 0, st>>>(sorted_key, n_inst, ranges);
        *launches += 1;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- tile order
// Longest-first scheduling of the blend kernels: tiles sorted by descending instance count
// (a stable 16-bit radix sort of 0xFFFF - min(count, 0xFFFF)).
__global__ void k_tile_keys(const uint2 *__restrict__ ranges, long long n, uint32_t *__restrict__ keys,
                            uint32_t *__restrict__ vals) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const uint2 r = ranges[t];
        const uint32_t c = r.y - r.x;
        keys[t] = 0xFFFFu - (c < 0xFFFFu ? c : 0xFFFFu);
        vals[t] = (uint32_t)t;
    }
}

cudaError_t launch_tile_order(const uint2 *ranges, long long n_tiles, uint32_t *keys, uint32_t *vals,
                              uint32_t *keys_tmp, uint32_t *vals_tmp, uint32_t *hist, uint32_t *scan_tmp,
                              uint32_t **order, cudaStream_t st, long long *launches) {
    if (n_tiles <= 0) {
        *order = vals;
        return cudaSuccess;
    }
    long long b = (n_tiles + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    k_tile_keys<<<(unsigned)b, 256, 0, st>>>(ranges, n_tiles, keys, vals);
    *launches += 1;
    uint32_t *ko = nullptr;
    return launch_radix_sort(keys, vals, keys_tmp, vals_tmp, n_tiles, 16, hist, scan_tmp, &ko, order, st, launches);
}

// ---------------------------------------------------------------------------- L2 loss
__global__ void k_l2_loss(const float *__restrict__ x, const float *__restrict__ y, long long n, float scale,
                          float *__restrict__ loss, float *__restrict__ grad) {
    float acc = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = x[i] - y[i];
        grad[i] = 2.0f * scale * d;
        acc = fmaf(d, d, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int k = 0; k < 8; ++k) t += ws[k];
        atomicAdd(loss, t * scale);
    }
}

cudaError_t launch_l2_loss(const float *x, const float *y, long long n, float scale, float *loss, float *grad,
                           cudaStream_t st, long long *launches) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    long long b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    k_l2_loss<<<(unsigned)b, 256, 0, st>>>(x, y, n, scale, loss, grad);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace vg
