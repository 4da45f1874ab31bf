// Tile binning and sorting: single-pass exclusive scan, a stable single-pass-per-digit LSD
// radix sort of (uint32 key, uint32 value) pairs, instance duplication and per-tile ranges.
//
// The per-tile front-to-back order (tile, depth, Gaussian index) is built in two stable
// steps: items are sorted by depth key (ties keep index order), their instances are
// emitted in that order, and a second stable sort on the tile id alone groups them by tile
// without disturbing the depth order inside each tile.
#include "vg_internal.cuh"

namespace vg {

// ---------------------------------------------------------------------------- look-back
// Single-pass prefix sums with decoupled look-back (Merrill, Garland: "Single-pass Parallel
// Prefix Scan with Decoupled Look-back", NVIDIA TR 2016): a CTA takes the next tile index
// from an atomic counter, publishes its tile's aggregate, then walks back over the tiles before
// it, adding aggregates until it meets an inclusive prefix, and publishes its own.  A CTA only
// ever waits for tiles handed out before its own, which belong to CTAs already running, so the
// walk always ends; the spin on each status word is bounded anyway and a timeout sets a sticky
// error flag that the host reads at its next synchronisation.  Flag bits: kErrTimeout (a
// look-back wait gave up), kErrCapacity (more instances than the fixed capacity).
constexpr int kSpinLimit = 1 << 21;
constexpr uint32_t kErrTimeout = kDevErrTimeout, kErrCapacity = kDevErrCapacity;

// 32-bit status: 2 flag bits + 30-bit count (radix sort, counts < 2^30)
constexpr uint32_t kFlagAgg = 1u << 30, kFlagPre = 2u << 30, kCountMask = (1u << 30) - 1u;
// 64-bit status: 2 flag bits + 62-bit sum (scan)
constexpr unsigned long long kFlagAgg64 = 1ull << 62, kFlagPre64 = 2ull << 62, kSumMask64 = (1ull << 62) - 1ull;

// The walk reads kLookWin status words at a time (all loads in flight together) and then
// consumes them nearest first; tile 0 always holds an inclusive prefix, so the walk ends there
// at the latest.
#ifndef VG_LOOK_WIN
#define VG_LOOK_WIN 8
#endif
constexpr int kLookWin = VG_LOOK_WIN;

__device__ __forceinline__ uint32_t lookback32(const uint32_t *status, long long tile, int stride, int col,
                                               uint32_t *err, int spin_limit = kSpinLimit) {
    uint32_t prefix = 0;
    for (long long t = tile - 1; t >= 0; t -= kLookWin) {
        uint32_t s[kLookWin];
#pragma unroll
        for (int k = 0; k < kLookWin; ++k) s[k] = (t - k >= 0) ? __ldcv(status + (t - k) * stride + col) : kFlagPre;
#pragma unroll
        for (int k = 0; k < kLookWin; ++k) {
            for (int spins = 0; (s[k] >> 30) == 0; ++spins) {
                if (spins >= spin_limit) {
                    atomicOr(err, kErrTimeout);
                    return prefix;
                }
                s[k] = __ldcv(status + (t - k) * stride + col);
            }
            prefix += s[k] & kCountMask;
            if ((s[k] & ~kCountMask) == kFlagPre) return prefix;
        }
    }
    return prefix;
}

// Warp-cooperative walk (all 32 lanes call it): lane l reads the status of tile t - l, so one
// round trip covers 32 predecessors; the walk stops at the nearest inclusive prefix once every
// tile up to it has published.
__device__ __forceinline__ unsigned long long warp_lookback64(const unsigned long long *status, long long tile,
                                                              uint32_t *err, int spin_limit = kSpinLimit) {
    const int lane = threadIdx.x & 31;
    unsigned long long prefix = 0;
    for (long long t = tile - 1; t >= 0; t -= 32) {
        const long long my = t - lane;
        unsigned long long s = my >= 0 ? __ldcv(status + my) : kFlagPre64;
        unsigned need = 0xffffffffu, pre = 0;
        for (int spins = 0;; ++spins) {
            pre = __ballot_sync(0xffffffffu, (s & ~kSumMask64) == kFlagPre64);
            need = pre ? ((pre & (0u - pre)) << 1) - 1u : 0xffffffffu;   // lanes up to the nearest prefix
            const unsigned waiting = __ballot_sync(0xffffffffu, (s >> 62) == 0) & need;
            if (waiting == 0) break;
            if (spins >= spin_limit) {
                if (lane == 0) atomicOr(err, kErrTimeout);
                break;
            }
            if ((s >> 62) == 0) s = __ldcv(status + my);
        }
        unsigned long long v = ((need >> lane) & 1u) ? (s & kSumMask64) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        prefix += v;
        if (pre) break;
    }
    return prefix;
}

// Exclusive scan over the threads of a CTA of NT threads (NT/32 warps); returns the exclusive
// prefix of x and the CTA total.  ws must hold NT/32 words; the CTA is synchronised on return.
template <int NT>
__device__ __forceinline__ unsigned long long cta_excl_scan(unsigned long long x, unsigned long long *ws,
                                                            unsigned long long &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    unsigned long long before = 0, all = 0;
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) {
        const unsigned long long v = ws[k];
        before += (k < w) ? v : 0ull;
        all += v;
    }
    __syncthreads();
    total = all;
    return before + incl - x;
}

// ---------------------------------------------------------------------------- scan
constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

size_t scan_tmp_words(long long n) {
    const long long tiles = (n + kScanTile - 1) / kScanTile;
    return (size_t)(2 * tiles + 4);   // u64 status per tile, tile counter
}

// Exclusive scan of count[perm[i]] (perm may be NULL); out[n] = total (low 32 bits) and
// total64 = the full sum.  tmp: tile counter in tmp[0], u64 status from tmp + 2.
__global__ void __launch_bounds__(kScanThreads)
k_scan_onepass(const uint32_t *__restrict__ in, const uint32_t *__restrict__ perm, long long n, uint32_t *__restrict__ out,
               uint32_t *tmp, unsigned long long *total64, unsigned long long cap, uint32_t *err) {
    pdl_entry();
    __shared__ unsigned long long ws[kScanThreads / 32];
    __shared__ unsigned long long s_prefix;
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(tmp, 1u);
    __syncthreads();
    const long long tile = s_tile;
    unsigned long long *status = (unsigned long long *)(tmp + 2);
    const long long i0 = tile * kScanTile + (long long)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    unsigned long long sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const long long i = i0 + k;
        v[k] = i < n ? (perm ? in[perm[i]] : in[i]) : 0u;
        sum += v[k];
    }
    unsigned long long agg;
    const unsigned long long excl = cta_excl_scan<kScanThreads>(sum, ws, agg);
    if (threadIdx.x < 32) {
        unsigned long long prefix = 0;
        if (tile == 0) {
            if (threadIdx.x == 0) atomicExch(status, kFlagPre64 | agg);
        } else {
            if (threadIdx.x == 0) atomicExch(status + tile, kFlagAgg64 | agg);
            prefix = warp_lookback64(status, tile, err);
            if (threadIdx.x == 0) atomicExch(status + tile, kFlagPre64 | (prefix + agg));
        }
        if (threadIdx.x == 0) {
            s_prefix = prefix;
            if ((tile + 1) * kScanTile >= n) {   // the last tile writes the total
                out[n] = (uint32_t)(prefix + agg);
                *total64 = prefix + agg;
                if (prefix + agg > cap) atomicOr(err, kErrCapacity);
            }
        }
    }
    __syncthreads();
    unsigned long long run = s_prefix + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const long long i = i0 + k;
        if (i < n) out[i] = (uint32_t)run;
        run += v[k];
    }
}

cudaError_t launch_scan_gather(const uint32_t *count, const uint32_t *perm, uint32_t *out, long long n, uint32_t *tmp,
                               unsigned long long *total64, unsigned long long cap, uint32_t *err, cudaStream_t st,
                               long long *launches) {
    const long long tiles = (n + kScanTile - 1) / kScanTile;
    cudaError_t e = cudaMemsetAsync(tmp, 0, scan_tmp_words(n) * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    if (tiles == 0) {
        e = cudaMemsetAsync(out, 0, sizeof(uint32_t), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(total64, 0, sizeof(unsigned long long), st);
        return e;
    }
    pdl_launch(k_scan_onepass, (unsigned)tiles, kScanThreads, 0, st, count, perm, n, out, tmp, total64, cap, err);
    *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- radix sort
// Stable LSD radix sort, one kernel per digit of at most 8 bits (Adinets, Merrill: "Onesweep: A Faster
// Least Significant Digit Radix Sort for GPUs", 2022): the digit totals of every pass come
// from one histogram kernel up front; per pass a CTA ranks its 2048-key tile stably in shared
// memory, finds each digit's offset from the tiles before it by decoupled look-back, and
// writes the tile digit by digit, so that stores land in consecutive runs.
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
#ifndef VG_RS_ITEMS
#define VG_RS_ITEMS 8
#endif
constexpr int kRsItems = VG_RS_ITEMS;                // keys per thread
constexpr int kRsTile = kRsThreads * kRsItems;      // keys per CTA tile
constexpr int kRsBins = 256;

static int rs_passes(int bits) { return (bits + 7) / 8; }

// Digit widths: the bits are shared out as evenly as the pass count allows, low digits first
// (13 bits: 7 + 6 rather than 8 + 5), so that no pass scatters a tile over all 256 buckets when
// fewer suffice: a wider low digit spreads each tile's keys over more, shorter output runs.
__host__ __device__ __forceinline__ int rs_width(int bits, int p) {
    const int passes = (bits + 7) / 8;
    return passes ? bits / passes + (p < bits % passes ? 1 : 0) : 0;
}
__host__ __device__ __forceinline__ int rs_shift(int bits, int p) {
    int s = 0;
    for (int q = 0; q < p; ++q) s += rs_width(bits, q);
    return s;
}

size_t radix_scratch_words(long long n, int bits) {
    const long long tiles = (n + kRsTile - 1) / kRsTile;
    const int p = rs_passes(bits);
    return (size_t)p * kRsBins + (size_t)p + 8 + (size_t)p * (size_t)tiles * kRsBins;
}

// digit totals of all passes: ghist[p * 256 + d]
__global__ void __launch_bounds__(kRsThreads)
k_digit_hist(const uint32_t *__restrict__ keys, long long n, const unsigned long long *__restrict__ n_dev, int bits,
             uint32_t *__restrict__ ghist) {
    pdl_entry();
    if (n_dev && (long long)*n_dev < n) n = (long long)*n_dev;
    __shared__ uint32_t h[4][kRsBins];
    const int passes = (bits + 7) / 8;
    for (int i = threadIdx.x; i < 4 * kRsBins; i += kRsThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    // each thread reads 4 consecutive keys at a time (16-byte loads; the key arrays are
    // allocation bases) and counts runs of equal digits in registers, flushing a run to the shared
    // histogram when its digit changes: a digit shared by most keys (the depth keys' exponent
    // byte) no longer serialises on one shared counter (depth sort 0.0835 -> 0.0806 ms)
    uint32_t run_d[4], run_c[4], dmask[4];
    int dshift[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        run_d[p] = 0u, run_c[p] = 0u;
        dshift[p] = rs_shift(bits, p);
        dmask[p] = (1u << rs_width(bits, p)) - 1u;
    }
    auto add = [&](uint32_t k) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            if (p < passes) {
                const uint32_t dg = (k >> dshift[p]) & dmask[p];
                if (dg != run_d[p]) {
                    if (run_c[p]) atomicAdd(&h[p][run_d[p]], run_c[p]);
                    run_d[p] = dg;
                    run_c[p] = 0u;
                }
                ++run_c[p];
            }
        }
    };
    const long long n4 = n / 4;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const uint4 q = reinterpret_cast<const uint4 *>(keys)[i];
        add(q.x);
        add(q.y);
        add(q.z);
        add(q.w);
    }
    for (long long i = 4 * n4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) add(keys[i]);
#pragma unroll
    for (int p = 0; p < 4; ++p)
        if (p < passes && run_c[p]) atomicAdd(&h[p][run_d[p]], run_c[p]);
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRsBins; i += kRsThreads) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&ghist[i], c);
    }
}

__global__ void __launch_bounds__(kRsThreads)
k_onesweep(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals, uint32_t *__restrict__ ko,
           uint32_t *__restrict__ vo, long long n, const unsigned long long *__restrict__ n_dev, int shift,
           uint32_t mask, const uint32_t *__restrict__ ghist, uint32_t *status, uint32_t *tile_ctr, uint32_t *err) {
    pdl_entry();
    __shared__ uint32_t wcnt[kRsWarps][kRsBins];    // per-warp digit counts, then exclusive over warps
    __shared__ uint32_t dig_local[kRsBins];          // first slot of each digit in the ranked tile
    __shared__ uint32_t dig_global[kRsBins];         // first output position of each digit's run
    __shared__ uint32_t sk[kRsTile], sv[kRsTile];
    __shared__ unsigned long long wsum[kRsWarps];
    __shared__ uint32_t s_tile;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, d = threadIdx.x;
    for (int i = threadIdx.x; i < kRsWarps * kRsBins; i += kRsThreads) (&wcnt[0][0])[i] = 0;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const long long tile = s_tile;
    if (n_dev && (long long)*n_dev < n) n = (long long)*n_dev;   // the count is known on the device only
    if (tile * kRsTile >= n) return;                             // the grid covers a larger capacity
    // a pass whose digit is the same for every key (the exponent byte of depth keys, often) is the
    // identity permutation: every CTA sees the same digit count and copies its tile instead
    if (ghist[(keys[tile * kRsTile] >> shift) & mask] == (uint32_t)n) {
        const long long t0 = tile * kRsTile, t1 = min(t0 + kRsTile, n);
        // 16-byte copies (tile starts are multiples of 2048 keys of allocation-based arrays)
        const long long q0 = t0 / 4, q1 = t1 / 4;
        for (long long q = q0 + threadIdx.x; q < q1; q += kRsThreads) {
            reinterpret_cast<uint4 *>(ko)[q] = reinterpret_cast<const uint4 *>(keys)[q];
            const uint32_t i = (uint32_t)(4 * q);
            reinterpret_cast<uint4 *>(vo)[q] = vals ? reinterpret_cast<const uint4 *>(vals)[q] : make_uint4(i, i + 1, i + 2, i + 3);
        }
        for (long long i = 4 * q1 + threadIdx.x; i < t1; i += kRsThreads) {
            ko[i] = keys[i];
            vo[i] = vals ? vals[i] : (uint32_t)i;
        }
        return;
    }
    // 1. stable rank inside the tile: warp w ranks keys [w*256, (w+1)*256) of the tile in order,
    //    32 at a time: the peers of every key first (__match_any_sync, independent of one another),
    //    then per key group the lowest lane adds the group's size to the warp's digit count with a
    //    shared-memory atomic, whose old value the group's lanes read by shuffle (a warp's atomics on
    //    one address take effect in program order, so the ranks stay stable; tile sort 0.088 ->
    //    0.085 ms against the previous load / store of the count between two __syncwarp)
    const long long base = tile * kRsTile + w * (kRsItems * 32);
    uint32_t k[kRsItems], v[kRsItems], r[kRsItems], pm[kRsItems];
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        const long long i = base + it * 32 + lane;
        const bool valid = i < n;
        k[it] = valid ? keys[i] : 0u;
        v[it] = valid ? (vals ? vals[i] : (uint32_t)i) : 0u;
    }
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        const bool valid = base + it * 32 + lane < n;
        const uint32_t dg = valid ? ((k[it] >> shift) & mask) : 0xFFFFFFFFu;
        pm[it] = __match_any_sync(0xffffffffu, dg);
    }
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        const bool valid = base + it * 32 + lane < n;
        const uint32_t dg = valid ? ((k[it] >> shift) & mask) : 0u;
        const uint32_t lower = pm[it] & ((1u << lane) - 1u);
        const int leader = __ffs(pm[it]) - 1;
        uint32_t prev = 0u;
        if (valid && lower == 0u) prev = atomicAdd(&wcnt[w][dg], (uint32_t)__popc(pm[it]));
        prev = __shfl_sync(0xffffffffu, prev, leader);
        r[it] = prev + __popc(lower);
    }
    __syncthreads();
    // 2. per digit (thread d): exclusive offsets over warps and the tile's count
    uint32_t cnt = 0;
#pragma unroll
    for (int ww = 0; ww < kRsWarps; ++ww) {
        const uint32_t c = wcnt[ww][d];
        wcnt[ww][d] = cnt;
        cnt += c;
    }
    if (tile == 0)
        atomicExch(status + d, kFlagPre | cnt);
    else
        atomicExch(status + tile * kRsBins + d, kFlagAgg | cnt);
    unsigned long long tot;
    const uint32_t local = (uint32_t)cta_excl_scan<kRsThreads>(cnt, wsum, tot);
    const uint32_t gbase = (uint32_t)cta_excl_scan<kRsThreads>(ghist[d], wsum, tot);
    uint32_t prefix = 0;
    if (tile > 0) {
        prefix = lookback32(status, tile, kRsBins, d, err);
        atomicExch(status + tile * kRsBins + d, kFlagPre | (prefix + cnt));
    }
    dig_local[d] = local;
    dig_global[d] = gbase + prefix;
    __syncthreads();
    // 3. place the keys in digit order in shared memory, then write each digit's run
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        const long long i = base + it * 32 + lane;
        if (i < n) {
            const uint32_t dg = (k[it] >> shift) & mask;
            const uint32_t p = dig_local[dg] + wcnt[w][dg] + r[it];
            sk[p] = k[it];
            sv[p] = v[it];
        }
    }
    __syncthreads();
    const long long rem = n - tile * kRsTile;
    const int tn = rem < kRsTile ? (int)rem : kRsTile;
    for (int i = threadIdx.x; i < tn; i += kRsThreads) {
        const uint32_t key = sk[i];
        const uint32_t dg = (key >> shift) & mask;
        const uint32_t pos = dig_global[dg] + (uint32_t)i - dig_local[dg];
        ko[pos] = key;
        vo[pos] = sv[i];
    }
}

cudaError_t launch_radix_sort(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *ka, uint32_t *va,
                              uint32_t *kb, uint32_t *vb, long long n, const unsigned long long *n_dev, int bits,
                              uint32_t *scratch, uint32_t *err, uint32_t **keys_out, uint32_t **vals_out,
                              cudaStream_t st, long long *launches) {
    const int passes = rs_passes(bits);
    *keys_out = const_cast<uint32_t *>(keys_in);
    *vals_out = const_cast<uint32_t *>(vals_in);
    if (n <= 0 || passes == 0) return cudaSuccess;
    if (n > (long long)kCountMask) return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(keys_in) & 15u) return cudaErrorMisalignedAddress;   // 16-byte key loads
    const long long tiles = (n + kRsTile - 1) / kRsTile;
    cudaError_t e = cudaMemsetAsync(scratch, 0, radix_scratch_words(n, bits) * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    uint32_t *ghist = scratch, *ctr = scratch + passes * kRsBins, *status = ctr + passes + 8;
    long long hb = (n + kRsThreads - 1) / kRsThreads;
    if (hb > 152 * 4) hb = 152 * 4;   // fewer CTAs: fewer same-address flushes of the digit totals
    pdl_launch(k_digit_hist, (unsigned)hb, kRsThreads, 0, st, keys_in, n, n_dev, bits, ghist);
    *launches += 1;
    const uint32_t *ki = keys_in, *vi = vals_in;
    for (int p = 0; p < passes; ++p) {
        uint32_t *kout = (p & 1) ? kb : ka, *vout = (p & 1) ? vb : va;
        const int nb = rs_width(bits, p);
        pdl_launch(k_onesweep, (unsigned)tiles, kRsThreads, 0, st, ki, vi, kout, vout, n, n_dev, rs_shift(bits, p),
                   (1u << nb) - 1u, ghist + p * kRsBins, status + (size_t)p * tiles * kRsBins, ctr + p, err);
        *launches += 1;
        ki = kout;
        vi = vout;
    }
    *keys_out = const_cast<uint32_t *>(ki);
    *vals_out = const_cast<uint32_t *>(vi);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- duplicate
// A warp takes 32 consecutive items: their instances fill one contiguous output range
// [offsets[first], offsets[last + 1]), which the lanes write together, position by position
// (coalesced stores).  The owner of position o is the last of the warp's items whose first
// instance is at or before o (items without instances share their successor's offset, so the
// last one wins); its instance r = o - offset is tile (x0 + r % w, y0 + r / w) of its rectangle,
// the row-major order of the rectangle.
constexpr int kDupWarps = 8;

__global__ void __launch_bounds__(32 * kDupWarps)
k_duplicate(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ offsets, const short4 *__restrict__ rect,
            const ViewInfo *__restrict__ views, long long n_items, int n_per_view, uint32_t *__restrict__ inst_key,
            uint32_t *__restrict__ inst_val, long long capacity) {
    pdl_entry();
    __shared__ uint32_t s_off[kDupWarps][32], s_item[kDupWarps][32];
    __shared__ short4 s_rc[kDupWarps][32];
    __shared__ int s_tb[kDupWarps][32], s_tx[kDupWarps][32];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const long long stride = (long long)gridDim.x * kDupWarps * 32;
    for (long long w0 = ((long long)blockIdx.x * kDupWarps + wi) * 32; w0 < n_items; w0 += stride) {
        const long long i = w0 + lane;
        const bool valid = i < n_items;
        uint32_t off = 0, end = 0, item = 0;
        short4 rc = make_short4(0, 0, -1, -1);
        int tb = 0, tx = 0;
        if (valid) {
            off = offsets[i];
            end = offsets[i + 1];
            item = perm ? perm[i] : (uint32_t)i;
            if (end > off) {
                rc = rect[item];
                const int v = (int)(item / (uint32_t)n_per_view);
                tb = views[v].tile_base;
                tx = views[v].tiles_x;
            }
        }
        const int last = (int)min(31LL, n_items - 1 - w0);
        const uint32_t r0 = __shfl_sync(0xffffffffu, off, 0), r1 = __shfl_sync(0xffffffffu, end, last);
        s_off[wi][lane] = valid ? off : r1;   // lanes past the end own nothing
        s_item[wi][lane] = item;
        s_rc[wi][lane] = rc;
        s_tb[wi][lane] = tb;
        s_tx[wi][lane] = tx;
        __syncwarp();
        for (uint32_t o = r0 + lane; o < r1; o += 32) {
            int l = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (s_off[wi][l + step] <= o) l += step;
            const short4 q = s_rc[wi][l];
            const uint32_t r = o - s_off[wi][l], w = (uint32_t)(q.z - q.x + 1);
            const uint32_t ry = r / w, rx = r - ry * w;
            if ((long long)o < capacity) {
                inst_key[o] = (uint32_t)(s_tb[wi][l] + ((int)q.y + (int)ry) * s_tx[wi][l] + (int)q.x + (int)rx);
                inst_val[o] = s_item[wi][l];
            }
        }
        __syncwarp();   // the staged items are reused by the warp's next 32
    }
}

cudaError_t launch_duplicate(const uint32_t *perm, const uint32_t *offsets, const short4 *rect, const ViewInfo *views,
                             long long n_items, int n_per_view, uint32_t *inst_key, uint32_t *inst_val,
                             long long capacity, cudaStream_t st, long long *launches) {
    long long b = (n_items + 32 * kDupWarps - 1) / (32 * kDupWarps);
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    pdl_launch(k_duplicate, (unsigned)b, 32 * kDupWarps, 0, st, perm, offsets, rect, views, n_items, n_per_view, inst_key, inst_val,
               capacity);
    *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- ranges
// Four consecutive sorted keys per thread (one 16-byte load plus the two neighbours): a tile's
// range starts where its key differs from the previous one and ends where the next differs.
__global__ void __launch_bounds__(256) k_ranges(const uint32_t *__restrict__ key, long long n,
                                                const unsigned long long *__restrict__ n_dev,
                                                uint2 *__restrict__ ranges) {
    pdl_entry();
    if (n_dev && (long long)*n_dev < n) n = (long long)*n_dev;
    const long long nq = (n + 3) / 4;
    for (long long qd = (long long)blockIdx.x * blockDim.x + threadIdx.x; qd < nq;
         qd += (long long)gridDim.x * blockDim.x) {
        const long long i0 = 4 * qd;
        uint32_t k[4];
        if (i0 + 4 <= n) {   // key is 16-byte aligned (a device allocation) and i0 a multiple of 4
            const uint4 v = *(const uint4 *)(key + i0);
            k[0] = v.x;
            k[1] = v.y;
            k[2] = v.z;
            k[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) k[j] = i0 + j < n ? key[i0 + j] : 0u;
        }
        const bool has_prev = i0 > 0, has_next = i0 + 4 < n;
        const uint32_t prev = has_prev ? key[i0 - 1] : 0u, next = has_next ? key[i0 + 4] : 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long i = i0 + j;
            if (i >= n) break;
            const uint32_t t = k[j];
            const bool first = j == 0 ? (!has_prev || prev != t) : k[j - 1] != t;
            const bool last = i + 1 == n || (j == 3 ? next != t : k[j + 1] != t);
            if (first) ranges[t].x = (uint32_t)i;
            if (last) ranges[t].y = (uint32_t)(i + 1);
        }
    }
}

cudaError_t launch_ranges(const uint32_t *sorted_key, long long n_inst, const unsigned long long *n_dev, uint2 *ranges,
                          long long n_tiles, cudaStream_t st, long long *launches) {
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, st);
    if (e != cudaSuccess) return e;
    if (n_inst > 0) {
        long long b = ((n_inst + 3) / 4 + 255) / 256;
        if (b > 152 * 64) b = 152 * 64;
        pdl_launch(k_ranges, (unsigned)b, 256, 0, st, sorted_key, n_inst, n_dev, ranges);
        *launches += 1;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- tile order
// Longest-first scheduling of the blend kernels: tiles in descending order of their instance
// count, bucketed at a third of an octave (64 buckets) by one CTA.  The order only decides
// which tile a CTA of the blend kernels takes; every order gives the same results.
constexpr int kOrderBuckets = 64;

__device__ __forceinline__ int order_bucket(uint32_t c) {
    if (c == 0) return 0;
    const int b = 1 + (int)(3.0f * __log2f((float)c));
    return b < kOrderBuckets - 1 ? b : kOrderBuckets - 1;
}

__device__ __forceinline__ uint32_t tile_len(const uint2 *ranges, const uint32_t *lens, long long t) {
    if (lens) return lens[t];
    const uint2 r = ranges[t];
    return r.y - r.x;
}

__global__ void __launch_bounds__(1024) k_tile_order(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ lens,
                                                     long long n, uint32_t *__restrict__ order) {
    pdl_entry();
    __shared__ uint32_t cnt[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (long long t = threadIdx.x; t < n; t += blockDim.x) atomicAdd(&cnt[order_bucket(tile_len(ranges, lens, t))], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {   // descending: largest bucket first
        uint32_t run = 0;
        for (int b = kOrderBuckets - 1; b >= 0; --b) {
            const uint32_t c = cnt[b];
            cnt[b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (long long t = threadIdx.x; t < n; t += blockDim.x)
        order[atomicAdd(&cnt[order_bucket(tile_len(ranges, lens, t))], 1u)] = (uint32_t)t;
}

cudaError_t launch_tile_order(const uint2 *ranges, const uint32_t *lens, long long n_tiles, uint32_t *order,
                              cudaStream_t st, long long *launches) {
    if (n_tiles <= 0) return cudaSuccess;
    pdl_launch(k_tile_order, 1, 1024, 0, st, ranges, lens, n_tiles, order);
    *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- L2 loss
__global__ void k_l2_loss(const float *__restrict__ x, const float *__restrict__ y, long long n, float scale,
                          float *__restrict__ loss, float *__restrict__ grad) {
    pdl_entry();
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
    return launch_l2_loss_acc(x, y, n, scale, loss, grad, st, launches);
}

cudaError_t launch_l2_loss_acc(const float *x, const float *y, long long n, float scale, float *loss, float *grad,
                               cudaStream_t st, long long *launches) {
    long long b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    pdl_launch(k_l2_loss, (unsigned)b, 256, 0, st, x, y, n, scale, loss, grad);
    *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- bounded-wait self-test
// One look-back of tile 1 over a status array whose tile 0 never publishes (all words zero), with
// a spin limit of `spin_limit` polls: the wait gives up, latches kErrTimeout in *err and returns.
// which = 0: the scan's warp-cooperative walk (64-bit status); 1: the radix pass's walk (32-bit).
__global__ void k_lookback_selftest(const unsigned long long *status64, const uint32_t *status32, int which,
                                    int spin_limit, uint32_t *err, unsigned long long *out) {
    pdl_entry();
    unsigned long long v;
    if (which == 0)
        v = warp_lookback64(status64, 1, err, spin_limit);
    else
        v = lookback32(status32, 1, 1, 0, err, spin_limit);
    if (threadIdx.x == 0) *out = v;
}

cudaError_t launch_lookback_selftest(void *status, int which, int spin_limit, uint32_t *err, unsigned long long *out,
                                     cudaStream_t st, long long *launches) {
    pdl_launch(k_lookback_selftest, 1, which == 0 ? 32 : 1, 0, st, (const unsigned long long *)status,
               (const uint32_t *)status, which, spin_limit, err, out);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace vg
