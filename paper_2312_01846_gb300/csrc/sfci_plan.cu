// Merge-bucket plan of the bucketed sigma (row mode), built on the device from
// the exact element count bound for each alpha string (the "bucket on the
// spin-up string" of Sec. 3, with rows too heavy for one bucket split).
//
// With W(r) = sum of the counts of the rows before r and windows of Q = P/2
// elements over W (P: elements per bucket):
//   - a light row (0 < w <= Q) joins the light bucket of the window
//     floor(W(r) / Q) it starts in; the rows of one light bucket are
//     consecutive and hold at most Q + Q = P elements;
//   - a heavy row (w > Q) gets ns = min(ceil(w / P), ceil(C / 1024)) buckets
//     of its own (C: beta strings), after the light bucket of the window it
//     starts in.  It spans more than a window, so the next row starts in a
//     later one: a window holds light rows, then at most one heavy row.
//     The split is by a hash of the beta index, so a bucket of a row with
//     ns = ceil(C / 1024) can hold no more distinct keys than the beta strings
//     hashed to it (about 1024, half the merge table): the rows that many sources reach (w > C, their
//     keys repeated many times) get fewer, larger buckets, which the merge
//     table still holds and whose regions overflow far less.
// Buckets are numbered window by window, so alpha rows and buckets are in the
// same order and every light bucket is a contiguous rank range.
#include <cstdint>

#include "sfci_internal.cuh"

namespace sfci {
namespace {

// distinct keys a bucket of a row split by the beta hash can hold at most,
// about: half the slots of the merge table (2048)
constexpr unsigned long long kKeysPerBucket = 1024;

__device__ __forceinline__ unsigned long long heavy_buckets(unsigned long long wr, unsigned long long P,
                                                         unsigned long long C) {
    const unsigned long long by_w = (wr + P - 1) / P, by_keys = (C + kKeysPerBucket - 1) / kKeysPerBucket;
    return by_w < by_keys ? by_w : by_keys;
}

__global__ void plan_windows_kernel(const unsigned long long *w, const unsigned long long *wpre,
                                    unsigned long long nrows, unsigned long long P, unsigned long long C,
                                    unsigned *tl, unsigned *th) {
    for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < nrows;
         r += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long wr = w[r];
        if (!wr) continue;
        const unsigned long long t = wpre[r] / (P / 2);
        if (wr > P / 2) th[t] = (unsigned)heavy_buckets(wr, P, C);
        else tl[t] = 1u;
    }
}

__global__ void plan_count_kernel(const unsigned *tl, const unsigned *th, unsigned long long T, unsigned *tc) {
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < T;
         t += (unsigned long long)gridDim.x * blockDim.x)
        tc[t] = tl[t] + th[t];
}

// row map entry (first bucket << 32 | bucket count) and bucket capacities:
// light buckets hold exactly their rows' counts; a heavy row's buckets get
// the mean plus four standard deviations plus 32 of its beta-hash split (the
// rest spills to the overflow list), a one-bucket heavy row exactly its count
// (rows must arrive in window order: P even, windows of P/2)
__global__ void plan_rows_kernel(const unsigned long long *w, const unsigned long long *wpre,
                                 unsigned long long nrows, unsigned long long P, unsigned long long C,
                                 const unsigned *tl, const unsigned long long *bstart,
                                 unsigned long long *rowmap, unsigned *cap) {
    for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < nrows;
         r += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long wr = w[r];
        if (!wr) {
            rowmap[r] = 0ull;
            continue;
        }
        const unsigned long long t = wpre[r] / (P / 2);
        if (wr > P / 2) {
            const unsigned long long ns = heavy_buckets(wr, P, C);
            const unsigned long long first = bstart[t] + tl[t];
            rowmap[r] = (first << 32) | ns;
            unsigned per;
            if (ns == 1) {
                per = (unsigned)wr;
            } else {
                const double mu = (double)wr / (double)ns;
                per = (unsigned)ceil(mu + 4.0 * sqrt(mu) + 32.0);
            }
            for (unsigned long long j = 0; j < ns; ++j) cap[first + j] = per;
        } else {
            const unsigned long long first = bstart[t];
            rowmap[r] = (first << 32) | 1ull;
            atomicAdd(&cap[first], (unsigned)wr);
        }
    }
}

// for each target: the first bucket b with boff[b] >= target (b <= nb), and boff there
__global__ void lower_bound_kernel(const unsigned long long *boff, unsigned long long nb,
                                   const unsigned long long *targets, int n, unsigned long long *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long x = targets[i];
    unsigned long long a = 0, e = nb;
    while (a < e) {
        const unsigned long long m = a + (e - a) / 2;
        if (boff[m] < x) a = m + 1;
        else e = m;
    }
    out[2 * i] = a;
    out[2 * i + 1] = boff[a];
}

// alpha rows that can hold buckets [lo, hi): rows after the last one whose
// buckets all lie below lo, up to the row before the first one whose buckets
// all lie at or above hi (rows without buckets between two passes count for both)
__global__ void pass_rows_kernel(const unsigned long long *rowmap, unsigned long long nrows, unsigned lo,
                                 unsigned hi, unsigned long long *lim) {
    for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < nrows;
         r += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long m = rowmap[r];
        const unsigned ns = (unsigned)m, first = (unsigned)(m >> 32);
        if (!ns) continue;
        if ((unsigned long long)first + ns <= lo) atomicMax(&lim[0], r + 1);
        if (first >= hi) atomicMin(&lim[1], r);
    }
}

__global__ void pass_offsets_kernel(const unsigned long long *boff, unsigned lo, unsigned hi, unsigned *start4) {
    const unsigned long long base = boff[lo];
    for (unsigned long long b = lo + blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; b <= hi;
         b += (unsigned long long)gridDim.x * blockDim.x)
        start4[b] = (unsigned)((boff[b] - base) >> 2);
}

__global__ void round_caps4_kernel(unsigned *cap, unsigned long long nb) {
    for (unsigned long long b = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; b < nb;
         b += (unsigned long long)gridDim.x * blockDim.x)
        cap[b] = (cap[b] + 3u) & ~3u;
}

unsigned grid_of(unsigned long long n) {
    const unsigned long long g = (n + 255) / 256;
    return (unsigned)(g < 16384 ? (g > 0 ? g : 1) : 16384);
}

}  // namespace

cudaError_t plan_windows(const unsigned long long *w, const unsigned long long *wpre, unsigned long long nrows,
                         unsigned long long P, unsigned long long C, unsigned long long T, unsigned *tl, unsigned *th,
                         unsigned *tc, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(tl, 0, size_t(T) * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(th, 0, size_t(T) * 4, st);
    if (e != cudaSuccess) return e;
    count_launch();
    plan_windows_kernel<<<grid_of(nrows), 256, 0, st>>>(w, wpre, nrows, P, C, tl, th);
    count_launch();
    plan_count_kernel<<<grid_of(T), 256, 0, st>>>(tl, th, T, tc);
    return cudaGetLastError();
}

cudaError_t plan_rows(const unsigned long long *w, const unsigned long long *wpre, unsigned long long nrows,
                      unsigned long long P, unsigned long long C, const unsigned *tl,
                      const unsigned long long *bstart, unsigned long long B, unsigned long long *rowmap,
                      unsigned *cap, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(cap, 0, size_t(B) * 4, st);
    if (e != cudaSuccess) return e;
    count_launch();
    plan_rows_kernel<<<grid_of(nrows), 256, 0, st>>>(w, wpre, nrows, P, C, tl, bstart, rowmap, cap);
    return cudaGetLastError();
}

cudaError_t boff_lower_bounds(const unsigned long long *boff, unsigned long long nb, const unsigned long long *targets,
                              int n, unsigned long long *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    lower_bound_kernel<<<(n + 127) / 128, 128, 0, st>>>(boff, nb, targets, n, out);
    return cudaGetLastError();
}

cudaError_t pass_rows(const unsigned long long *rowmap, unsigned long long nrows, unsigned lo, unsigned hi,
                      unsigned long long *lim, cudaStream_t st) {
    const unsigned long long init[2] = {0ull, nrows};
    cudaError_t e = cudaMemcpyAsync(lim, init, 16, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    count_launch();
    pass_rows_kernel<<<grid_of(nrows), 256, 0, st>>>(rowmap, nrows, lo, hi, lim);
    return cudaGetLastError();
}

cudaError_t pass_offsets(const unsigned long long *boff, unsigned lo, unsigned hi, unsigned *start4,
                         cudaStream_t st) {
    count_launch();
    pass_offsets_kernel<<<grid_of((unsigned long long)(hi - lo) + 1), 256, 0, st>>>(boff, lo, hi, start4);
    return cudaGetLastError();
}

cudaError_t round_caps4(unsigned *cap, unsigned long long nb, cudaStream_t st) {
    if (!nb) return cudaSuccess;
    count_launch();
    round_caps4_kernel<<<grid_of(nb), 256, 0, st>>>(cap, nb);
    return cudaGetLastError();
}

}  // namespace sfci
