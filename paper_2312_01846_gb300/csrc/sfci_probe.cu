// Throughput probes of the SM pipes that bound the sigma kernels.
//
// The emit kernel multiplies every element by c_D in float64 (and sums the
// single-excitation elements in float64), the merge kernel adds 128-bit
// fixed-point integers with 64-bit shared-memory atomics.  These probes time
// each of those operations alone, with enough independent work per thread to
// fill the pipe, so that a kernel's counters can be read against the rate the
// chip actually delivers:
//   kind 0  float64 fused multiply-add   (8 independent chains per thread)
//   kind 1  float64 add
//   kind 2  float64 multiply
//   kind 3  float32 fused multiply-add
//   kind 4  64-bit integer multiply-add  (target-rank and hash arithmetic)
//   kind 5  64-bit integer atomic add on shared memory (distinct addresses per lane)
//   kind 6  32-bit integer atomic add on shared memory
//   kind 7  64-bit compare-and-swap on shared memory (always succeeding)
//   kind 8  float32 atomic add on shared memory
// One launch of 152 x 8 CTAs of 256 threads per measurement, timed with CUDA
// events on the given stream after one warm-up launch.  Result: operations
// (lane operations) per second.
#include "sfci_internal.cuh"

namespace sfci {
namespace {

constexpr int kPT = 256;
constexpr int kChains = 8;

template <int kKind>
__global__ void __launch_bounds__(kPT) probe_kernel(long long iters, double seed, unsigned long long *sink) {
    __shared__ unsigned long long sh64[kPT * 2];
    __shared__ unsigned sh32[kPT * 2];
    __shared__ float shf[kPT * 2];
    const int t = threadIdx.x;
    sh64[t] = sh64[t + kPT] = 0ull;
    sh32[t] = sh32[t + kPT] = 0u;
    shf[t] = shf[t + kPT] = 0.f;
    __syncthreads();
    double a[kChains];
    float f[kChains];
    unsigned long long u[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        a[k] = seed + 1e-3 * (k + t);
        f[k] = (float)a[k];
        u[k] = (unsigned long long)(t * 977 + k * 131 + 1);
    }
    const double x = 0.999999999, y = 1e-9;
    const unsigned long long m = 0x9E3779B97F4A7C15ull | (unsigned long long)seed;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            if constexpr (kKind == 0) a[k] = __fma_rn(a[k], x, y);
            if constexpr (kKind == 1) a[k] = __dadd_rn(a[k], y);
            if constexpr (kKind == 2) a[k] = __dmul_rn(a[k], x);
            if constexpr (kKind == 3) f[k] = __fmaf_rn(f[k], 0.9999f, 1e-7f);
            if constexpr (kKind == 4) u[k] = u[k] * m + (unsigned long long)k;
        }
        if constexpr (kKind == 5) {
            atomicAdd(&sh64[t], 1ull);
            atomicAdd(&sh64[t + kPT], 3ull);
        }
        if constexpr (kKind == 6) {
            atomicAdd(&sh32[t], 1u);
            atomicAdd(&sh32[t + kPT], 3u);
        }
        if constexpr (kKind == 8) {
            atomicAdd(&shf[t], 1.0f);
            atomicAdd(&shf[t + kPT], 3.0f);
        }
        if constexpr (kKind == 7) {
            const unsigned long long c0 = sh64[t];
            atomicCAS(&sh64[t], c0, c0 + 1ull);
            const unsigned long long c1 = sh64[t + kPT];
            atomicCAS(&sh64[t + kPT], c1, c1 + 1ull);
        }
    }
    unsigned long long r = sh64[t] + sh64[t + kPT] + sh32[t] + sh32[t + kPT] +
                           __float_as_uint(shf[t]) + __float_as_uint(shf[t + kPT]);
#pragma unroll
    for (int k = 0; k < kChains; ++k)
        r += (unsigned long long)__double_as_longlong(a[k]) + __float_as_uint(f[k]) + u[k];
    if (r == 0x1234567ull) *sink = r;  // keeps the work observable; never true in practice
}

template <int kKind>
cudaError_t run_probe(long long iters, int grid, cudaStream_t st, unsigned long long *sink, float *ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        count_launch();
        probe_kernel<kKind><<<grid, kPT, 0, st>>>(iters / 8 + 1, 1.0, sink);  // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        count_launch();
        probe_kernel<kKind><<<grid, kPT, 0, st>>>(iters, 1.0, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace
}  // namespace sfci

using namespace sfci;

extern "C" {

sfci_status sfci_debug_pipe_rate(int kind, int64_t iters, void *workspace, double *ops_per_s,
                                 void *stream) {
    if (kind < 0 || kind > 8 || iters < 1 || iters > (1ll << 30) || !workspace || !ops_per_s) {
        set_error("need kind in 0..8, 1 <= iters <= 2^30, a device workspace and a host result");
        return SFCI_E_INVALID;
    }
    int dev = 0, n_sm = 0;
    SFCI_CUDA(cudaGetDevice(&dev));
    SFCI_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = n_sm * 8;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long *sink = static_cast<unsigned long long *>(workspace);
    float ms = 0.f;
    cudaError_t e = cudaSuccess;
    switch (kind) {
        case 0: e = run_probe<0>(iters, grid, st, sink, &ms); break;
        case 1: e = run_probe<1>(iters, grid, st, sink, &ms); break;
        case 2: e = run_probe<2>(iters, grid, st, sink, &ms); break;
        case 3: e = run_probe<3>(iters, grid, st, sink, &ms); break;
        case 4: e = run_probe<4>(iters, grid, st, sink, &ms); break;
        case 5: e = run_probe<5>(iters, grid, st, sink, &ms); break;
        case 6: e = run_probe<6>(iters, grid, st, sink, &ms); break;
        case 7: e = run_probe<7>(iters, grid, st, sink, &ms); break;
        default: e = run_probe<8>(iters, grid, st, sink, &ms); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "pipe-rate probe");
    const double per_iter = kind <= 4 ? (double)kChains : 2.0;  // lane operations per thread and iteration
    *ops_per_s = (double)grid * kPT * per_iter * (double)iters / (ms * 1e-3);
    return SFCI_OK;
}

}  // extern "C"
