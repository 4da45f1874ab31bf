// Pipe-peak microbenchmarks: the measured denominators of the blend kernels' roofline.
//
// The blend and tomography kernels are bound by FP32 arithmetic (FMA pipe) and by the
// transcendental unit (ex2, rsqrt), not by memory.  These kernels measure what this GPU sustains
// on each pipe with no memory traffic: every thread runs kChains independent dependency chains
// (so that latency never limits issue), fully unrolled, on a grid of the occupancy limit per SM.
//   FMA: a <- fma(a, b, c)       one FFMA per step, 2 flop
//   EX2: x <- ex2.approx(-x)     one MUFU ex2 per step (x stays in (0, 1])
// The chains' final values feed a store that never happens (the compiler cannot drop them).
// Launched plainly (no programmatic dependent launch): nothing else runs beside a measurement.
// Also here: the self-test of the backward ring's bounded mbarrier wait.
#include "blend.cuh"

namespace vg {

constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;
constexpr int kPeakThreads = 256;

__device__ float g_peak_sink;   // external linkage: the store below cannot be dropped; never taken

__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(int iters, float b, float c) {
    float a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) a[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kPeakChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += a[k];
    if (s == -1.0f) g_peak_sink = s;   // the chains converge to c / (1 - b) > 0: never taken
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ex2(int iters) {
    float x[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kPeakChains; ++k) x[k] = ex2_approx(-x[k]);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += x[k];
    if (s == -1.0f) g_peak_sink = s;   // ex2 is positive: never taken
}

// Grid: the occupancy limit of the kernel on every SM.  Returns the operations one launch
// performs (FMA instructions or ex2 instructions, per lane) in *ops.
cudaError_t launch_pipe_peak(int pipe, int iters, double *ops, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (pipe == 0)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_fma, kPeakThreads, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_ex2, kPeakThreads, 0);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
    if (pipe == 0)
        k_peak_fma<<<blocks, kPeakThreads, 0, st>>>(iters, 0.999999f, 1e-7f);
    else
        k_peak_ex2<<<blocks, kPeakThreads, 0, st>>>(iters);
    *ops = (double)blocks * kPeakThreads * (double)iters * kPeakUnroll * kPeakChains;
    return cudaGetLastError();
}

// Failure-path check of the backward ring's bounded wait: one warp waits on a full barrier that
// no producer ever arrives on; the wait gives up after limit_ns, latches kDevErrTimeout and returns.
__global__ void k_ring_selftest(unsigned long long limit_ns, uint32_t *__restrict__ err) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        s_abort = 0;
    }
    __syncthreads();
    if (!mbar_wait(&bar, 0, limit_ns, &s_abort) && threadIdx.x == 0) atomicOr(err, kDevErrTimeout);
}

cudaError_t launch_ring_selftest(int limit_us, uint32_t *err, cudaStream_t st, long long *launches) {
    k_ring_selftest<<<1, 32, 0, st>>>((unsigned long long)limit_us * 1000ull, err);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace vg
