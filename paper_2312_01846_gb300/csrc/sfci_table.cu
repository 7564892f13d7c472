// Operations on the merge table and on sparse vectors: clearing, the epsilon
// screen (Sec. 3), the Lanczos combination u = sigma - a w_i - b w_{i-1}
// (Eq. 10) as further adds into the table, extraction of the merged vector,
// and the dot products <w_j|sigma_i>, <w_j|w_i> that fill T and S (Sec. 2.1).
//
// All reductions here are deterministic: a fixed grid, a fixed per-thread
// stride, a fixed tree inside each block, and the block partials summed in
// order by one block.  HBM-bound: the table is streamed with 16-byte vector
// accesses, grids are multiples of the SM count.
#include "sfci_internal.cuh"

namespace sfci {
namespace {

constexpr int kThreads = 256;
constexpr int kRedBlocks = 304;  // 2 x 152 SMs, fixed for reproducible sums

__global__ void clear_kernel(Slot *slots, unsigned long long cap, int *status,
                             unsigned long long *count) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    ulonglong2 e;
    e.x = kEmpty;
    e.y = 0ull;  // +0.0
    ulonglong2 *p = reinterpret_cast<ulonglong2 *>(slots);
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
         i += stride)
        p[i] = e;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *status = 0;
        *count = 0;
    }
}

__global__ void screen_kernel(Slot *slots, unsigned long long cap, double eps,
                              unsigned long long *screened) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned c = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
         i += stride) {
        const ulonglong2 e = reinterpret_cast<const ulonglong2 *>(slots)[i];
        if (e.x != kEmpty && e.y != 0x8000000000000000ull &&
            fabs(__longlong_as_double((long long)e.y)) < eps) {
            slots[i].val = -0.0;
            ++c;
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(screened, (unsigned long long)c);
}

__global__ void validate_kernel(const unsigned long long *r, long long n, unsigned long long dim,
                                int *flag) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long x = r[i];
        if (x >= dim || (i + 1 < n && r[i + 1] <= x)) atomicOr(flag, 1);
    }
}

__global__ void axpy_kernel(Table t, const unsigned long long *rank, const double *coef,
                            long long m, const double *scale, double hscale, double sign) {
    const double s = scale ? *scale : hscale;
    unsigned ins = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (long long)gridDim.x * blockDim.x) {
        double v = __dmul_rn(s, coef[k]);
        if (sign < 0.0) v = -v;
        if (v != 0.0) table_add(t, rank[k], v, ins);
    }
    if (ins) atomicAdd(t.count, (unsigned long long)ins);
}

// live entry: key present, not screened (-0.0), and not below eps
__device__ __forceinline__ bool live(unsigned long long key, unsigned long long vbits, double eps) {
    if (key == kEmpty || vbits == 0x8000000000000000ull) return false;
    return !(fabs(__longlong_as_double((long long)vbits)) < eps);
}

__global__ void extract_kernel(const Slot *slots, unsigned long long cap, double eps,
                               unsigned long long *out_rank, double *out_val, long long out_cap,
                               unsigned long long *n_dev) {
    __shared__ unsigned warp_tot[kThreads / 32];
    __shared__ unsigned long long blk_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x; i0 < cap; i0 += stride) {
        const unsigned long long i = i0 + threadIdx.x;
        ulonglong2 e = make_ulonglong2(kEmpty, 0ull);
        if (i < cap) e = reinterpret_cast<const ulonglong2 *>(slots)[i];
        const bool ok = i < cap && live(e.x, e.y, eps);
        const unsigned bal = __ballot_sync(kFull, ok);
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned tot = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                unsigned c = warp_tot[w];
                warp_tot[w] = tot;
                tot += c;
            }
            blk_base = tot ? atomicAdd(n_dev, (unsigned long long)tot) : 0ull;
        }
        __syncthreads();
        if (ok) {
            const unsigned long long pos =
                blk_base + warp_tot[warp] + __popc(bal & ((1u << lane) - 1u));
            if ((long long)pos < out_cap) {
                out_rank[pos] = e.x;
                out_val[pos] = __longlong_as_double((long long)e.y);
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    __syncthreads();
    return r;  // valid in thread 0
}

struct VecPack {
    VecRef v[kMaxVec];
};

// partial[j * kRedBlocks + block] = sum over the block's entries of w_j * sigma
__global__ void dots_kernel(Table t, VecPack vp, double *partial) {
    __shared__ double sh[kThreads / 32];
    const int j = blockIdx.y;
    const VecRef w = vp.v[j];
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < w.n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long h = table_find(t, w.rank[k]);
        if (h >= 0) acc += w.coef[k] * __ldcg(&t.slots[h].val);
    }
    const double r = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[(size_t)j * gridDim.x + blockIdx.x] = r;
}

__device__ __forceinline__ long long bsearch_rank(const unsigned long long *r, long long n,
                                                  unsigned long long key) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        long long mid = lo + ((hi - lo) >> 1);
        if (r[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && r[lo] == key) ? lo : -1;
}

__global__ void overlap_kernel(VecPack vp, VecRef last, double *partial) {
    __shared__ double sh[kThreads / 32];
    const int j = blockIdx.y;
    const VecRef w = vp.v[j];
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < last.n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long p = bsearch_rank(w.rank, w.n, last.rank[k]);
        if (p >= 0) acc += w.coef[p] * last.coef[k];
    }
    const double r = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[(size_t)j * gridDim.x + blockIdx.x] = r;
}

__global__ void finish_kernel(const double *partial, int nparts, double *out) {
    __shared__ double sh[kThreads / 32];
    const int j = blockIdx.x;
    double acc = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) acc += partial[(size_t)j * nparts + k];
    const double r = block_sum(acc, sh);
    if (threadIdx.x == 0) out[j] = r;
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

unsigned stream_grid(unsigned long long work) {
    unsigned long long g = (work + kThreads - 1) / kThreads;
    unsigned long long cap = (unsigned long long)sm_count() * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

__global__ void finalize_exact_kernel(Table t) {
    const unsigned long long cap = t.mask + 1;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
         i += (unsigned long long)gridDim.x * blockDim.x)
        if (t.slots[i].key != kEmpty) t.slots[i].val = from_fixed(t.acc[2 * i], t.acc[2 * i + 1], t.fix_shift);
}

__global__ void max_abs_kernel(const double *x, long long n, unsigned long long *out) {
    unsigned long long m = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(x[k]) & 0x7fffffffffffffffull);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

}  // namespace

cudaError_t table_finalize_exact(Table t, cudaStream_t st) {
    count_launch();
    finalize_exact_kernel<<<stream_grid(t.mask + 1), kThreads, 0, st>>>(t);
    return cudaGetLastError();
}

cudaError_t max_abs_bits(const double *x, long long n, unsigned long long *out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, 8, st);
    if (e != cudaSuccess || n <= 0) return e;
    count_launch();
    max_abs_kernel<<<stream_grid((unsigned long long)n), kThreads, 0, st>>>(x, n, out);
    return cudaGetLastError();
}

cudaError_t table_clear(Table t, cudaStream_t st) {
    if (t.acc) {
        const cudaError_t e = cudaMemsetAsync(t.acc, 0, size_t(t.mask + 1) * 16, st);
        if (e != cudaSuccess) return e;
    }
    count_launch();
    clear_kernel<<<stream_grid(t.mask + 1), kThreads, 0, st>>>(t.slots, t.mask + 1, t.status, t.count);
    return cudaGetLastError();
}

cudaError_t table_screen(Table t, double eps, unsigned long long *screened_dev, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(screened_dev, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || !(eps > 0.0)) return e;
    count_launch();
    screen_kernel<<<stream_grid(t.mask + 1), kThreads, 0, st>>>(t.slots, t.mask + 1, eps,
                                                               screened_dev);
    return cudaGetLastError();
}

cudaError_t validate_sorted(const unsigned long long *rank, long long n, unsigned long long dim,
                            int *flag, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    count_launch();
    validate_kernel<<<stream_grid((unsigned long long)n), kThreads, 0, st>>>(rank, n, dim, flag);
    return cudaGetLastError();
}

cudaError_t table_axpy(Table t, const unsigned long long *rank, const double *coef, long long m,
                       const double *scale, double hscale, double sign, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    count_launch();
    axpy_kernel<<<stream_grid((unsigned long long)m), kThreads, 0, st>>>(t, rank, coef, m, scale,
                                                                        hscale, sign);
    return cudaGetLastError();
}

cudaError_t table_extract(Table t, double eps, unsigned long long *out_rank, double *out_val,
                          long long cap, unsigned long long *n_dev, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(n_dev, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    count_launch();
    extract_kernel<<<stream_grid(t.mask + 1), kThreads, 0, st>>>(t.slots, t.mask + 1, eps,
                                                                out_rank, out_val, cap, n_dev);
    return cudaGetLastError();
}

size_t dots_workspace_bytes(int nvec, long long) {
    return size_t(nvec > 0 ? nvec : 1) * kRedBlocks * sizeof(double);
}

cudaError_t table_dots(Table t, const VecRef *vecs, int nvec, double *out_dev, void *ws,
                       cudaStream_t st) {
    if (nvec <= 0) return cudaSuccess;
    if (nvec > kMaxVec) return cudaErrorInvalidValue;
    VecPack vp{};
    for (int j = 0; j < nvec; ++j) vp.v[j] = vecs[j];
    double *partial = static_cast<double *>(ws);
    count_launch();
    dots_kernel<<<dim3(kRedBlocks, nvec), kThreads, 0, st>>>(t, vp, partial);
    count_launch();
    finish_kernel<<<nvec, kThreads, 0, st>>>(partial, kRedBlocks, out_dev);
    return cudaGetLastError();
}

cudaError_t vec_overlaps(const VecRef *vecs, int nvec, VecRef last, double *out_dev, void *ws,
                         cudaStream_t st) {
    if (nvec <= 0) return cudaSuccess;
    if (nvec > kMaxVec) return cudaErrorInvalidValue;
    VecPack vp{};
    for (int j = 0; j < nvec; ++j) vp.v[j] = vecs[j];
    double *partial = static_cast<double *>(ws);
    count_launch();
    overlap_kernel<<<dim3(kRedBlocks, nvec), kThreads, 0, st>>>(vp, last, partial);
    count_launch();
    finish_kernel<<<nvec, kThreads, 0, st>>>(partial, kRedBlocks, out_dev);
    return cudaGetLastError();
}

}  // namespace sfci
