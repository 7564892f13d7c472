// Truncation of Eq. 11 and the ordering of sparse vectors.
//
// top-k: the k entries with the largest |c|, ties to the smaller rank, exact
// zeros excluded, decided exactly on bit patterns.  Each entry maps to a
// 127-bit composite X = (0x7fff...f - bits(|c|)) : rank, so the wanted entries
// are the k smallest X (for non-negative doubles the bit pattern orders like
// the value).  A radix select walks X from the top in 12-bit digits (the last
// digit has 7 bits): each pass histograms the digit of the entries whose
// higher digits equal the prefix found so far, and a one-block kernel picks
// the bin that holds the k-th smallest.  All state stays on the device; a pass
// that finds its bin exactly full ends the search early.  A last pass gathers
// every entry whose prefix is <= the threshold prefix.
//
// sort: stable LSD radix sort of (uint64 key, double val) pairs with 8-bit
// digits over the significant key bits only (ceil(log2(dim)) bits): per tile
// a digit histogram, one exclusive scan over (digit, tile), then a stable
// scatter ranked per warp with __match_any_sync.
#include "sfci_internal.cuh"

namespace sfci {
namespace {

constexpr int kT = 256;
constexpr int kBins = 4096;
constexpr int kPasses = 11;  // 10 x 12 bits + 7 bits = 127
constexpr int kRedBlocks = 304;

__host__ __device__ inline int pass_width(int p) { return p < 10 ? 12 : 7; }
__host__ __device__ inline int pass_low(int p) { return 127 - 12 * p - pass_width(p); }

struct SelState {
    unsigned long long pfx_hi, pfx_lo, mask_hi, mask_lo;
    unsigned long long need, total;
    int done, all, pass, pad;
    double sumsq;
};

struct SelLayout {
    size_t state, hist, n_gather, result, bytes;
};

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

SelLayout sel_layout() {
    SelLayout L{};
    size_t o = 0;
    L.state = o, o = a256(o + sizeof(SelState));
    L.hist = o, o = a256(o + sizeof(unsigned long long) * kBins);
    L.n_gather = o, o = a256(o + sizeof(unsigned long long));
    L.result = o, o = a256(o + sizeof(SplitResult));
    L.bytes = o;
    return L;
}

__device__ __forceinline__ bool item_valid(unsigned long long key, unsigned long long vbits) {
    return key != kEmpty && (vbits & 0x7fffffffffffffffull) != 0ull;
}

__device__ __forceinline__ unsigned digit_of(unsigned long long hi, unsigned long long lo, int p,
                                             int w) {
    unsigned long long v;
    if (p >= 64) v = hi >> (p - 64);
    else if (p + w <= 64) v = lo >> p;
    else v = (lo >> p) | (hi << (64 - p));
    return (unsigned)(v & ((1ull << w) - 1ull));
}

__global__ void sel_init_kernel(SelState *s, unsigned long long k, unsigned long long *hist,
                                unsigned long long *n_gather) {
    if (threadIdx.x == 0) {
        s->pfx_hi = s->pfx_lo = s->mask_hi = s->mask_lo = 0ull;
        s->need = k;
        s->total = 0;
        s->done = (k == 0);
        s->all = 0;
        s->pass = 0;
        s->sumsq = 0.0;
        *n_gather = 0;
    }
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) hist[b] = 0;
}

__global__ void sel_hist_kernel(Items it, SelState *s, unsigned long long *hist, int pass) {
    __shared__ unsigned sh[kBins];
    __shared__ double ssq[kT / 32];
    __shared__ unsigned long long scount[kT / 32];
    if (s->done) return;
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    const unsigned long long ph = s->pfx_hi, pl = s->pfx_lo, mh = s->mask_hi, ml = s->mask_lo;
    const int w = pass_width(pass), p = pass_low(pass);
    double sq = 0.0;
    unsigned long long cnt = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < it.n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = it.key[(size_t)i * it.stride];
        const unsigned long long vb = (unsigned long long)__double_as_longlong(it.val[(size_t)i * it.stride]);
        if (!item_valid(key, vb)) continue;
        const unsigned long long hi = 0x7fffffffffffffffull - (vb & 0x7fffffffffffffffull);
        if (pass == 0) {
            const double v = __longlong_as_double((long long)vb);
            sq += v * v;
            cnt += 1;
        }
        if ((hi & mh) != ph || (key & ml) != pl) continue;
        atomicAdd(&sh[digit_of(hi, key, p, w)], 1u);
    }
    if (pass == 0) {
        for (int o = 16; o > 0; o >>= 1) {
            sq += __shfl_xor_sync(kFull, sq, o);
            cnt += __shfl_xor_sync(kFull, cnt, o);
        }
        if ((threadIdx.x & 31) == 0) ssq[threadIdx.x >> 5] = sq, scount[threadIdx.x >> 5] = cnt;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], (unsigned long long)sh[b]);
    if (pass == 0 && threadIdx.x == 0) {
        double a = 0.0;
        unsigned long long c = 0;
        for (int q = 0; q < kT / 32; ++q) a += ssq[q], c += scount[q];
        atomicAdd(&s->sumsq, a);
        atomicAdd(&s->total, c);
    }
}

// one block of kT threads: choose the bin holding the need-th smallest
__global__ void sel_pick_kernel(SelState *s, unsigned long long *hist, int pass) {
    __shared__ unsigned long long tsum[kT];
    __shared__ int found_bin;
    __shared__ unsigned long long found_before;
    if (s->done) return;
    if (pass == 0 && s->total <= s->need) {
        __syncthreads();
        if (threadIdx.x == 0) s->all = 1, s->done = 1;
        return;
    }
    constexpr int per = kBins / kT;
    unsigned long long mine = 0;
    for (int q = 0; q < per; ++q) mine += hist[threadIdx.x * per + q];
    tsum[threadIdx.x] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        // exclusive scan (kT entries, sequential: tiny)
        unsigned long long run = 0;
        for (int t = 0; t < kT; ++t) {
            unsigned long long c = tsum[t];
            tsum[t] = run;
            run += c;
        }
        found_bin = -1;
    }
    __syncthreads();
    const unsigned long long need = s->need;
    const unsigned long long before = tsum[threadIdx.x];
    if (before < need && before + mine >= need) {
        unsigned long long run = before;
        for (int q = 0; q < per; ++q) {
            const unsigned long long c = hist[threadIdx.x * per + q];
            if (run + c >= need) {
                found_bin = threadIdx.x * per + q;
                found_before = run;
                break;
            }
            run += c;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int b = found_bin < 0 ? 0 : found_bin;
        const unsigned long long cnt = hist[b];
        const int w = pass_width(pass), p = pass_low(pass);
        const unsigned long long dm = (1ull << w) - 1ull;
        // set digit b at bits [p, p+w) of the composite prefix and mask
        if (p >= 64) {
            s->pfx_hi |= (unsigned long long)b << (p - 64);
            s->mask_hi |= dm << (p - 64);
        } else if (p + w <= 64) {
            s->pfx_lo |= (unsigned long long)b << p;
            s->mask_lo |= dm << p;
        } else {
            s->pfx_lo |= (unsigned long long)b << p;
            s->mask_lo |= dm << p;
            s->pfx_hi |= (unsigned long long)b >> (64 - p);
            s->mask_hi |= dm >> (64 - p);
        }
        s->need = need - found_before;
        // found_bin < 0 cannot happen for need <= total; stop instead of looping on
        if (found_bin < 0 || cnt == s->need || pass == kPasses - 1) s->done = 1;
        s->pass = pass + 1;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kBins; q += blockDim.x) hist[q] = 0;
}

__global__ void sel_gather_kernel(Items it, const SelState *s, unsigned long long *out_key,
                                  double *out_val, long long cap, unsigned long long *n_out) {
    __shared__ unsigned wt[kT / 32];
    __shared__ unsigned long long base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long ph = s->pfx_hi, pl = s->pfx_lo, mh = s->mask_hi, ml = s->mask_lo;
    const bool all = s->all;
    const bool none = (s->need == 0 && !all && mh == 0 && ml == 0);  // k == 0
    for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < it.n;
         i0 += (long long)gridDim.x * blockDim.x) {
        const long long i = i0 + threadIdx.x;
        bool ok = false;
        unsigned long long key = 0, vb = 0;
        if (i < it.n && !none) {
            key = it.key[(size_t)i * it.stride];
            vb = (unsigned long long)__double_as_longlong(it.val[(size_t)i * it.stride]);
            if (item_valid(key, vb)) {
                if (all) ok = true;
                else {
                    const unsigned long long hi = (0x7fffffffffffffffull - (vb & 0x7fffffffffffffffull)) & mh;
                    const unsigned long long lo = key & ml;
                    ok = (hi < ph) || (hi == ph && lo <= pl);
                }
            }
        }
        const unsigned bal = __ballot_sync(kFull, ok);
        if (lane == 0) wt[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned tot = 0;
            for (int w = 0; w < kT / 32; ++w) {
                unsigned c = wt[w];
                wt[w] = tot;
                tot += c;
            }
            base = tot ? atomicAdd(n_out, (unsigned long long)tot) : 0ull;
        }
        __syncthreads();
        if (ok) {
            const unsigned long long pos = base + wt[warp] + __popc(bal & ((1u << lane) - 1u));
            if ((long long)pos < cap) {
                out_key[pos] = key;
                out_val[pos] = __longlong_as_double((long long)vb);
            }
        }
        __syncthreads();
    }
}

__global__ void sel_stats_kernel(const SelState *s, double *sumsq_out, unsigned long long *total_out) {
    if (threadIdx.x == 0) {
        if (sumsq_out) *sumsq_out = s->sumsq;
        if (total_out) *total_out = s->total;
    }
}

// one pass: items of a smaller first digit than the picked bin -> out; of the
// picked bin -> cand (or out, when the bin is taken whole)
__global__ void sel_split_kernel(Items it, const SelState *s, unsigned long long *out_key,
                                 double *out_val, long long out_cap, unsigned long long *n_out,
                                 unsigned long long *cand_key, double *cand_val, long long cand_cap,
                                 unsigned long long *cand_n) {
    const int lane = threadIdx.x & 31;
    const bool all = s->all, done = s->done;
    const bool none = !all && s->mask_hi == 0;  // k == 0
    const unsigned b0 = (unsigned)(s->pfx_hi >> 51);
    for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < it.n;
         i0 += (long long)gridDim.x * blockDim.x) {
        const long long i = i0 + threadIdx.x;
        int dest = 0;  // 0 none, 1 out, 2 cand
        unsigned long long key = 0, vb = 0;
        if (i < it.n && !none) {
            key = it.key[(size_t)i * it.stride];
            vb = (unsigned long long)__double_as_longlong(it.val[(size_t)i * it.stride]);
            if (item_valid(key, vb)) {
                const unsigned d0 = (unsigned)((0x7fffffffffffffffull - (vb & 0x7fffffffffffffffull)) >> 51);
                if (all || d0 < b0 || (done && d0 == b0)) dest = 1;
                else if (d0 == b0) dest = 2;
            }
        }
        const unsigned bo = __ballot_sync(kFull, dest == 1), bc = __ballot_sync(kFull, dest == 2);
        unsigned long long base_o = 0, base_c = 0;
        if (lane == 0) {
            if (bo) base_o = atomicAdd(n_out, (unsigned long long)__popc(bo));
            if (bc) base_c = atomicAdd(cand_n, (unsigned long long)__popc(bc));
        }
        base_o = __shfl_sync(kFull, base_o, 0);
        base_c = __shfl_sync(kFull, base_c, 0);
        const unsigned lt = (1u << lane) - 1u;
        if (dest == 1) {
            const unsigned long long pos = base_o + __popc(bo & lt);
            if ((long long)pos < out_cap) out_key[pos] = key, out_val[pos] = __longlong_as_double((long long)vb);
        } else if (dest == 2) {
            const unsigned long long pos = base_c + __popc(bc & lt);
            if ((long long)pos < cand_cap) cand_key[pos] = key, cand_val[pos] = __longlong_as_double((long long)vb);
        }
    }
}

__global__ void sel_split_result_kernel(const SelState *s, const unsigned long long *n_out,
                                        const unsigned long long *cand_n, SplitResult *r) {
    if (threadIdx.x == 0) {
        r->n_out = *n_out;
        r->n_cand = *cand_n;
        r->need = s->need;
        r->total = s->total;
        r->all = s->all;
        r->done = s->done;
    }
}

int sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

unsigned grid_for(long long n, int per_sm) {
    long long g = (n + kT - 1) / kT;
    long long c = (long long)sms() * per_sm;
    if (g > c) g = c;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// ------------------------------------------------------------- radix sort

constexpr int kSortItems = 8;
constexpr int kTile = kT * kSortItems;  // 2048
constexpr int kRadix = 256;

__global__ void rs_hist_kernel(const unsigned long long *key, long long cap,
                               const unsigned long long *n_dev, int shift, unsigned *counts,
                               int ntiles) {
    __shared__ unsigned h[kRadix];
    for (int b = threadIdx.x; b < kRadix; b += blockDim.x) h[b] = 0;
    __syncthreads();
    long long n = (long long)*n_dev;
    if (n > cap) n = cap;
    const long long t0 = (long long)blockIdx.x * kTile;
    for (int q = 0; q < kSortItems; ++q) {
        const long long i = t0 + (long long)q * kT + threadIdx.x;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kRadix; b += blockDim.x) counts[(size_t)b * ntiles + blockIdx.x] = h[b];
}

// exclusive scan of m unsigned counters in place, one block of 1024 threads
__global__ void rs_scan_kernel(unsigned *c, long long m) {
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long b0 = 0; b0 < m; b0 += blockDim.x) {
        const long long i = b0 + threadIdx.x;
        unsigned long long v = i < m ? c[i] : 0;
        unsigned long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long s = wsum[lane];
            unsigned long long t = s;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(kFull, t, o);
                if (lane >= o) t += y;
            }
            wsum[lane] = t - s;  // exclusive over warps
        }
        __syncthreads();
        const unsigned long long excl = carry + wsum[warp] + x - v;
        if (i < m) c[i] = (unsigned)excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
}

__global__ void rs_scatter_kernel(const unsigned long long *kin, const double *vin,
                                  unsigned long long *kout, double *vout, long long cap,
                                  const unsigned long long *n_dev, int shift,
                                  const unsigned *offsets, int ntiles) {
    __shared__ unsigned wc[kT / 32][kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = threadIdx.x; b < (kT / 32) * kRadix; b += blockDim.x) (&wc[0][0])[b] = 0;
    __syncthreads();
    long long n = (long long)*n_dev;
    if (n > cap) n = cap;
    const long long w0 = (long long)blockIdx.x * kTile + (long long)warp * (32 * kSortItems);
    unsigned loc[kSortItems];
    unsigned dig[kSortItems];
    for (int q = 0; q < kSortItems; ++q) {
        const long long i = w0 + (long long)q * 32 + lane;
        const bool valid = i < n;
        const unsigned d = valid ? (unsigned)((kin[i] >> shift) & 0xff) : (0x1000u | lane);
        const unsigned peers = __match_any_sync(kFull, d);
        const unsigned before = __popc(peers & ((1u << lane) - 1u));
        unsigned base = valid ? wc[warp][d] : 0u;
        __syncwarp();
        if (valid && (peers >> lane) == 1u) wc[warp][d] = base + __popc(peers);  // highest peer
        __syncwarp();
        loc[q] = base + before;
        dig[q] = d;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
        unsigned run = 0;
        for (int w = 0; w < kT / 32; ++w) {
            unsigned c = wc[w][d];
            wc[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int q = 0; q < kSortItems; ++q) {
        const long long i = w0 + (long long)q * 32 + lane;
        if (i < n) {
            const unsigned d = dig[q];
            const unsigned long long pos =
                (unsigned long long)offsets[(size_t)d * ntiles + blockIdx.x] + wc[warp][d] + loc[q];
            kout[pos] = kin[i];
            vout[pos] = vin[i];
        }
    }
}

__global__ void copy_pairs_kernel(const unsigned long long *ks, const double *vs,
                                  unsigned long long *kd, double *vd, long long cap,
                                  const unsigned long long *n_dev) {
    long long n = (long long)*n_dev;
    if (n > cap) n = cap;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        kd[i] = ks[i];
        vd[i] = vs[i];
    }
}

// ------------------------------------------------------------- normalisation

__global__ void sumsq_kernel(const double *v, long long cap, const unsigned long long *n_dev,
                             double *partial) {
    __shared__ double sh[kT / 32];
    long long n = (long long)*n_dev;
    if (n > cap) n = cap;
    double a = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        a = __fma_rn(v[i], v[i], a);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < kT / 32; ++w) r += sh[w];
        partial[blockIdx.x] = r;
    }
}

__global__ void scale_kernel(double *v, long long cap, const unsigned long long *n_dev,
                             const double *partial, int nparts) {
    __shared__ double norm;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < nparts; ++k) s += partial[k];
        norm = sqrt(s);
    }
    __syncthreads();
    long long n = (long long)*n_dev;
    if (n > cap) n = cap;
    const double d = norm;
    if (!(d > 0.0)) return;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        v[i] = __ddiv_rn(v[i], d);
}

}  // namespace

size_t select_workspace_bytes(long long, long long) { return sel_layout().bytes; }

cudaError_t select_topk(Items it, long long k, unsigned long long *out_key, double *out_val,
                        unsigned long long *n_out_dev, double *sumsq_dev,
                        unsigned long long *total_dev, void *ws, size_t ws_bytes, cudaStream_t st) {
    const SelLayout L = sel_layout();
    if (ws_bytes < L.bytes) return cudaErrorInvalidValue;
    char *base = static_cast<char *>(ws);
    SelState *s = reinterpret_cast<SelState *>(base + L.state);
    unsigned long long *hist = reinterpret_cast<unsigned long long *>(base + L.hist);
    count_launch();
    sel_init_kernel<<<1, kT, 0, st>>>(s, (unsigned long long)(k < 0 ? 0 : k), hist, n_out_dev);
    const unsigned g = grid_for(it.n, 4);
    for (int p = 0; p < kPasses; ++p) {
        count_launch();
        sel_hist_kernel<<<g, kT, 0, st>>>(it, s, hist, p);
        count_launch();
        sel_pick_kernel<<<1, kT, 0, st>>>(s, hist, p);
    }
    count_launch();
    sel_gather_kernel<<<grid_for(it.n, 8), kT, 0, st>>>(it, s, out_key, out_val, k, n_out_dev);
    if (sumsq_dev || total_dev) {
        count_launch();
        sel_stats_kernel<<<1, 32, 0, st>>>(s, sumsq_dev, total_dev);
    }
    return cudaGetLastError();
}

cudaError_t select_split(Items it, long long k,
                         unsigned long long *out_key, double *out_val, unsigned long long *n_out_dev,
                         unsigned long long *cand_key, double *cand_val, long long cand_cap,
                         unsigned long long *cand_n, void *ws, size_t ws_bytes, SplitResult *res_host,
                         cudaStream_t st) {
    const SelLayout L = sel_layout();
    if (ws_bytes < L.bytes) return cudaErrorInvalidValue;
    char *base = static_cast<char *>(ws);
    SelState *s = reinterpret_cast<SelState *>(base + L.state);
    unsigned long long *hist = reinterpret_cast<unsigned long long *>(base + L.hist);
    SplitResult *r = reinterpret_cast<SplitResult *>(base + L.result);
    count_launch();
    sel_init_kernel<<<1, kT, 0, st>>>(s, (unsigned long long)(k < 0 ? 0 : k), hist, n_out_dev);
    cudaError_t e = cudaMemsetAsync(cand_n, 0, 8, st);
    if (e != cudaSuccess) return e;
    count_launch();
    sel_hist_kernel<<<grid_for(it.n, 4), kT, 0, st>>>(it, s, hist, 0);
    count_launch();
    sel_pick_kernel<<<1, kT, 0, st>>>(s, hist, 0);
    count_launch();
    sel_split_kernel<<<grid_for(it.n, 8), kT, 0, st>>>(it, s, out_key, out_val, k, n_out_dev,
                                                       cand_key, cand_val, cand_cap, cand_n);
    count_launch();
    sel_split_result_kernel<<<1, 32, 0, st>>>(s, n_out_dev, cand_n, r);
    e = cudaMemcpyAsync(res_host, r, sizeof(SplitResult), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

size_t sort_pairs_bytes(long long cap) {
    const long long ntiles = (cap + kTile - 1) / kTile;
    return a256(size_t(cap) * 8) * 2 + a256(size_t(ntiles > 0 ? ntiles : 1) * kRadix * 4);
}

size_t sort_workspace_bytes(long long n) { return sort_pairs_bytes(n); }

cudaError_t sort_pairs(unsigned long long *key, double *val, long long cap,
                       const unsigned long long *n_dev, int bits, void *ws, cudaStream_t st) {
    if (cap <= 0) return cudaSuccess;
    const int ntiles = (int)((cap + kTile - 1) / kTile);
    char *b = static_cast<char *>(ws);
    unsigned long long *k2 = reinterpret_cast<unsigned long long *>(b);
    double *v2 = reinterpret_cast<double *>(b + a256(size_t(cap) * 8));
    unsigned *counts = reinterpret_cast<unsigned *>(b + 2 * a256(size_t(cap) * 8));
    unsigned long long *ka = key, *kb = k2;
    double *va = val, *vb = v2;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        count_launch();
        rs_hist_kernel<<<ntiles, kT, 0, st>>>(ka, cap, n_dev, shift, counts, ntiles);
        count_launch();
        rs_scan_kernel<<<1, 1024, 0, st>>>(counts, (long long)ntiles * kRadix);
        count_launch();
        rs_scatter_kernel<<<ntiles, kT, 0, st>>>(ka, va, kb, vb, cap, n_dev, shift, counts, ntiles);
        unsigned long long *tk = ka;
        ka = kb, kb = tk;
        double *tv = va;
        va = vb, vb = tv;
        ++passes;
    }
    if (passes & 1) {
        count_launch();
        copy_pairs_kernel<<<grid_for(cap, 8), kT, 0, st>>>(ka, va, key, val, cap, n_dev);
    }
    return cudaGetLastError();
}

size_t normalize_ws_bytes(long long) { return a256(sizeof(double) * kRedBlocks); }

cudaError_t normalize_vec(double *val, long long cap, const unsigned long long *n_dev, void *ws,
                          cudaStream_t st) {
    double *partial = static_cast<double *>(ws);
    count_launch();
    sumsq_kernel<<<kRedBlocks, kT, 0, st>>>(val, cap, n_dev, partial);
    count_launch();
    scale_kernel<<<kRedBlocks, kT, 0, st>>>(val, cap, n_dev, partial, kRedBlocks);
    return cudaGetLastError();
}

}  // namespace sfci
