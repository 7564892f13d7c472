// Internal declarations shared by the translation units of libsfci.so.
//
// Data layout on the device (one GPU, HBM3e):
//  * a sparse vector is SoA: uint64 rank[m] ascending, double coef[m];
//  * sigma's intermediate elements are merged in an open-addressing hash table
//    of 16-byte slots {uint64 key, double val} (key = rank, kEmpty = free);
//    the key and the value share one 32-byte sector, so a hit costs one
//    sector;
//  * the integrals stay in HBM (g is n^4 doubles: 4.9 MB at n = 28, resident
//    in the 129 MB L2) and are read through the read-only path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/sfci.h"

namespace sfci {

constexpr unsigned long long kEmpty = ~0ull;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxProbe = 1 << 12;  // linear-probe bound; beyond it the table is "full"

struct Slot {
    unsigned long long key;
    double val;
};

// Exact sums (used by the bucket merge and by sfci_sigma's table).
// Each sigma entry is accumulated as a 128-bit two's-complement integer in
// units of 2^-S (S chosen by the host so that no sum leaves the range): an
// element v = m 2^e (m < 2^53) becomes m 2^(e+S), exactly unless e + S < 0
// (|v| below 2^(52-S), rounded to the nearest unit).  Integer atomics add
// them, so the sum is exact and independent of the order of the adds, and one
// correctly rounded conversion gives the entry's double.

struct Fix128 {
    unsigned long long lo, hi;
};

// 64-bit shifts whose amount may be 64 or more (the PTX shift instructions
// clamp the amount to the register width, so the result is 0)
__device__ __forceinline__ unsigned long long shl64(unsigned long long x, unsigned s) {
    unsigned long long r;
    asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
    return r;
}
__device__ __forceinline__ unsigned long long shr64(unsigned long long x, unsigned s) {
    unsigned long long r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
    return r;
}

// Without branches (lanes holding elements of different magnitudes do not
// diverge): both shift directions are formed and one is selected, and the
// two's-complement negation is a masked xor plus a carried one.
__device__ __forceinline__ Fix128 to_fixed(double v, int S, bool &range_ok) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((bits >> 52) & 0x7FF);
    const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (ex ? (1ull << 52) : 0ull);
    const int sh = (ex ? ex : 1) - 1075 + S;  // v = mant 2^(ex-1075): mant 2^sh units
    if (sh > 74 && mant) range_ok = false;      // would not fit in 127 bits
    const unsigned su = (unsigned)sh, r = (unsigned)(-sh);
    // sh >= 0: mant << sh as 128 bits; sh < 0: mant >> -sh, nearest, ties away from zero
    const unsigned long long lo_p = shl64(mant, su), hi_p = shr64(mant, 64u - su) | shl64(mant, su - 64u);
    const unsigned long long lo_n = shr64(mant, r) + (shr64(mant, r - 1u) & 1ull);
    unsigned long long lo = sh >= 0 ? lo_p : lo_n, hi = sh >= 0 ? hi_p : 0ull;
    const unsigned long long neg = (unsigned long long)((long long)bits >> 63);  // all ones if v < 0
    lo ^= neg, hi ^= neg;
    const unsigned long long one = neg & 1ull, lo2 = lo + one;
    hi += one & (lo2 == 0ull ? 1ull : 0ull);
    return Fix128{lo2, hi};
}

// the sum held in (lo, hi) as a double, rounded to nearest, ties to even
__device__ __forceinline__ double from_fixed(unsigned long long lo, unsigned long long hi, int S) {
    const bool neg = (long long)hi < 0;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    if (hi == 0ull && lo == 0ull) return 0.0;
    int p = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);  // leading bit
    unsigned long long m;
    if (p <= 52) {
        m = lo << (52 - p);
    } else {
        const int sh = p - 52;  // 1..74
        m = sh >= 64 ? hi >> (sh - 64) : (lo >> sh) | (hi << (64 - sh));
        const int g = sh - 1;   // guard bit position
        const unsigned long long gbit = g >= 64 ? (hi >> (g - 64)) & 1ull : (lo >> g) & 1ull;
        const bool sticky = g >= 64 ? (lo != 0ull || (hi & ((1ull << (g - 64)) - 1ull)) != 0ull)
                                    : (lo & ((1ull << g) - 1ull)) != 0ull;
        if (gbit && (sticky || (m & 1ull))) ++m;
        if (m >> 53) {
            m >>= 1;
            ++p;
        }
    }
    const unsigned long long bexp = (unsigned long long)(p - S + 1023);
    const unsigned long long bits = ((unsigned long long)neg << 63) | (bexp << 52) | (m & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)bits);
}


// The hash table as the kernels see it.
struct Table {
    Slot *slots;
    unsigned long long mask;  // capacity - 1 (capacity a power of two)
    int shift;                // 64 - log2(capacity)
    int *status;              // device: bit 0 = a probe ran past kMaxProbe; bit 1 = a value
                              // outside the fixed-point range
    unsigned long long *count;  // device: keys inserted
    unsigned long long *acc = nullptr;  // [2 x capacity] exact sums (lo, hi) of the emit's
                                        // table mode; nullptr: float64 adds into the slots
    int fix_shift = 0;                  // units 2^-fix_shift of acc
};

// Read-only description of a system for the kernels.
struct SysDev {
    int n, na, nb, va, vb;
    int ks;              // row stride of the binomial table: max(na, nb) + 3
    int sa, sb;          // singles per spin: na*va, nb*vb
    int po_a, pv_a, po_b, pv_b;  // pair counts C(na,2), C(va,2), C(nb,2), C(vb,2)
    int pair_off[4];     // offsets (in pairs) of the four pair lists
    int n_pairs;         // total pairs
    unsigned long long ca, cb, dim;
    long long n_conn;    // connected determinants per determinant
    double e_core;
    const double *h;     // n*n
    const double *g;     // n^4
    const unsigned long long *binom;  // [(n+1) * ks]: C(b, m)
    const unsigned char *pairs;       // 2 bytes per pair: (first, second) positions, first < second
    const float *hf;     // float32 copies of h and g (SFCI_FP32_ELEMENTS), else null
    const float *gf;
    // element bounds for the heat-bath style screen: bound_ab[a*n+i] >= |(ai|bj)|
    // for every (b, j); bound_ss[i*n+j] >= |(ai|bj) - (aj|bi)| for every (a, b)
    const double *bound_ab;
    const double *bound_ss;
    int ss_any;          // 1: some bound_ss entry is non-zero (else every same-spin double is zero)
    double hbound;       // |<D'|H|D>| <= hbound for every pair of determinants
};

}  // namespace sfci

struct sfci_system {
    sfci::SysDev d;
    void *dev_block;  // one allocation holding h, g, binom, pairs
    int *dev_status;  // scratch status words for rank/unrank
    int device;
};

namespace sfci {

// ------------------------------------------------------------- launch count
// every kernel launch of the library increments this host counter
void count_launch();
long long launch_count();

// ------------------------------------------------------------- shared memory
// Let `func` use up to the device's opt-in shared memory per block, less its
// static shared memory (need: this launch's dynamic bytes, checked against it).  The attribute belongs to the function,
// not to a launch: setting it to each launch's own size would race between
// host threads launching one kernel with different sizes, so it is always set
// to the device maximum.
template <typename F>
cudaError_t allow_max_smem(F func, size_t need) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    const int room = optin - (int)fa.sharedSizeBytes;  // opt-in limit less the static shared memory
    if (room < 0 || need > (size_t)room) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, room);
}

// ------------------------------------------------------------- error text
void set_error(const std::string &msg);
sfci_status cuda_fail(cudaError_t e, const char *what);
#define SFCI_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return sfci::cuda_fail(e_, #call); \
    } while (0)

// ------------------------------------------------------------- device helpers

__device__ __forceinline__ int parity64(unsigned long long x) { return __popcll(x) & 1; }

// bits strictly between orbitals x and y
__device__ __forceinline__ unsigned long long between_mask(int x, int y) {
    int lo = x < y ? x : y, hi = x < y ? y : x;
    return ((1ull << hi) - 1ull) & ~((2ull << lo) - 1ull);
}

// Eq. 12 on the device: h = sum over occupied orbitals b (0-based, ascending)
// of C(b, m), m the electron's 1-based position; bt = binomial table in smem.
__device__ __forceinline__ unsigned long long string_rank(unsigned long long s,
                                                          const unsigned long long *bt,
                                                          int ks) {
    unsigned long long h = 0;
    int m = 1;
    while (s) {
        int b = __ffsll((long long)s) - 1;
        h += bt[b * ks + m];
        ++m;
        s &= s - 1ull;
    }
    return h;
}

// Greedy inverse of Eq. 12, one warp: for i = m..1 the largest c <= top with
// C(c, i) <= r.  C(c, i) is non-decreasing in c, so the lanes testing
// c = lane and c = lane + 32 give a prefix; its last lane is c.
__device__ __forceinline__ unsigned long long string_unrank_warp(unsigned long long r, int n,
                                                                 int m,
                                                                 const unsigned long long *bt,
                                                                 int ks) {
    const int lane = threadIdx.x & 31;
    unsigned long long s = 0;
    int top = n - 1;
    for (int i = m; i >= 1; --i) {
        int c0 = lane, c1 = lane + 32;
        bool p0 = (c0 <= top) && bt[c0 * ks + i] <= r;
        bool p1 = (c1 <= top) && bt[c1 * ks + i] <= r;
        unsigned b0 = __ballot_sync(kFull, p0), b1 = __ballot_sync(kFull, p1);
        int c = b1 ? 63 - __clz(b1) : 31 - __clz(b0);
        s |= 1ull << c;
        r -= bt[c * ks + i];
        top = c - 1;
    }
    return s;
}

// Occupied / empty orbital lists (ascending) of two spin strings from warp
// ballots; every lane of the warp must call it.
__device__ __forceinline__ void build_lists(unsigned long long alpha, unsigned long long beta, int n,
                                            unsigned char *occA, unsigned char *virA,
                                            unsigned char *occB, unsigned char *virB) {
    const int lane = threadIdx.x & 31;
    int seen_oa = 0, seen_va = 0, seen_ob = 0, seen_vb = 0;
    const unsigned lt = (1u << lane) - 1u;
    for (int half = 0; half < 2; ++half) {
        const int p = lane + 32 * half;
        const bool in = p < n;
        const bool oa = in && ((alpha >> p) & 1ull), ob = in && ((beta >> p) & 1ull);
        const unsigned moa = __ballot_sync(kFull, oa), mva = __ballot_sync(kFull, in && !oa);
        const unsigned mob = __ballot_sync(kFull, ob), mvb = __ballot_sync(kFull, in && !ob);
        if (oa) occA[seen_oa + __popc(moa & lt)] = (unsigned char)p;
        else if (in) virA[seen_va + __popc(mva & lt)] = (unsigned char)p;
        if (ob) occB[seen_ob + __popc(mob & lt)] = (unsigned char)p;
        else if (in) virB[seen_vb + __popc(mvb & lt)] = (unsigned char)p;
        seen_oa += __popc(moa), seen_va += __popc(mva);
        seen_ob += __popc(mob), seen_vb += __popc(mvb);
    }
}

__device__ __forceinline__ unsigned long long hash_slot(unsigned long long key, int shift) {
    return (key * 0x9E3779B97F4A7C15ull) >> shift;
}

// Add v into the entry `key`, inserting the key if absent (linear probing).
__device__ __forceinline__ bool table_add(const Table &t, unsigned long long key, double v,
                                          unsigned &inserted) {
    unsigned long long h = hash_slot(key, t.shift);
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        // a table already marked full fails fast instead of probing on
        if ((probe & 255) == 255 && *(volatile int *)t.status) return false;
        Slot *s = t.slots + h;
        unsigned long long cur = __ldcg(&s->key);
        if (cur == key) {
            atomicAdd(&s->val, v);
            return true;
        }
        if (cur == kEmpty) {
            unsigned long long old = atomicCAS(&s->key, kEmpty, key);
            if (old == kEmpty || old == key) {
                inserted += (old == kEmpty);
                atomicAdd(&s->val, v);
                return true;
            }
        }
        h = (h + 1ull) & t.mask;
    }
    atomicOr(t.status, 1);
    return false;
}

// Add v exactly into the entry `key` (fixed-point sums in t.acc), inserting
// the key if absent: the sum does not depend on the order of the adds.
__device__ __forceinline__ bool table_add_exact(const Table &t, unsigned long long key, double v,
                                                unsigned &inserted) {
    bool ok = true;
    const Fix128 f = to_fixed(v, t.fix_shift, ok);
    if (!ok) atomicOr(t.status, 2);
    unsigned long long h = hash_slot(key, t.shift);
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        if ((probe & 255) == 255 && *(volatile int *)t.status) return false;
        Slot *s = t.slots + h;
        unsigned long long cur = __ldcg(&s->key);
        bool found = cur == key;
        if (!found && cur == kEmpty) {
            const unsigned long long old = atomicCAS(&s->key, kEmpty, key);
            if (old == kEmpty || old == key) {
                inserted += (old == kEmpty);
                found = true;
            }
        }
        if (found) {
            const unsigned long long old = atomicAdd(&t.acc[2 * h], f.lo);
            atomicAdd(&t.acc[2 * h + 1], f.hi + (old + f.lo < old ? 1ull : 0ull));
            return true;
        }
        h = (h + 1ull) & t.mask;
    }
    atomicOr(t.status, 1);
    return false;
}

// Find `key`; returns the slot index or -1.
__device__ __forceinline__ long long table_find(const Table &t, unsigned long long key) {
    unsigned long long h = hash_slot(key, t.shift);
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        unsigned long long cur = __ldcg(&t.slots[h].key);
        if (cur == key) return (long long)h;
        if (cur == kEmpty) return -1;
        h = (h + 1ull) & t.mask;
    }
    return -1;
}

// ------------------------------------------------------------- emit sinks
// Where the emit kernel sends each intermediate element.
enum EmitMode { kModeTable = 0, kModeDebug = 1, kModeBucket = 2 };

// How the intermediate elements are spread over merge buckets.  Row mode
// (rowmap set): the elements of one target alpha string ("row") go to that
// row's bucket; light rows share a bucket, a heavy row owns several and picks
// one by a hash of the beta index.  The emit then writes each group of
// elements bound for one row (e.g. the beta hops of one alpha hop) as one run.
// Hash mode (no rowmap, for spaces with too many alpha strings to map):
// bucket = mix64(rank) >> (64 - log2B).  Bucket b owns elements
// [boff[b], boff[b+1]) of the element buffer.
struct Buckets {
    int log2B;
    const unsigned long long *rowmap;  // [C(n, n_alpha)]: first bucket << 32 | count (0: none)
    unsigned long long cb;             // C(n, n_beta)
    const unsigned long long *boff;    // [B + 1]
};

struct BucketOut {
    Buckets bk;
    unsigned *count;          // [B] elements that arrived per bucket
    Slot *elem;               // regions of buckets [lo, hi), relative to boff[lo]
    unsigned long long base;  // boff[lo]
    const unsigned *start4;   // [B + 1]: (boff[b] - boff[lo]) / 4 for b in [lo, hi] (regions are
                              // multiples of 4 slots): the pass's offsets in half the bytes
    double eps_elem;          // elements with |<D'|H|D> c_D| < eps_elem are not generated (0: off)
    Slot *ovf;                // [ovf_cap]
    unsigned long long *ovf_n;
    long long ovf_cap;
    unsigned lo, hi;
    // alpha rows that can hold buckets [lo, hi) (row mode; rows without buckets
    // between two passes belong to both): a target outside needs no row-map load
    unsigned long long row_lo, row_hi;
    int *status;              // bit 1: overflow list full; bit 4: an element had no bucket
    int aa_runs;              // 1: alpha-alpha doubles by runs of sources sharing alpha (own kernel)
};

struct EmitOut {
    Table t;                  // kModeTable
    BucketOut b;              // kModeBucket
    long long *dsrc;          // kModeDebug
    unsigned long long *dtgt;
    double *delem;
};

__device__ __forceinline__ unsigned long long mix64(unsigned long long key) {
    return key * 0x9E3779B97F4A7C15ull;
}

constexpr unsigned kNoBucket = 0xffffffffu;

// bucket of the determinant (alpha index ha, beta index hb)
__device__ __forceinline__ unsigned bucket_ab(const Buckets &bk, unsigned long long ha,
                                              unsigned long long hb) {
    if (!bk.rowmap) {
        const unsigned long long key = ha * bk.cb + hb;
        return bk.log2B > 0 ? (unsigned)(mix64(key) >> (64 - bk.log2B)) : 0u;
    }
    const unsigned long long m = __ldg(&bk.rowmap[ha]);
    const unsigned ns = (unsigned)m, first = (unsigned)(m >> 32);
    if (ns <= 1) return ns ? first : kNoBucket;
    return first + (unsigned)(((mix64(hb) >> 32) * ns) >> 32);
}

__device__ __forceinline__ unsigned bucket_key(const Buckets &bk, unsigned long long key) {
    if (!bk.rowmap) return bk.log2B > 0 ? (unsigned)(mix64(key) >> (64 - bk.log2B)) : 0u;
    const unsigned long long ha = key / bk.cb;
    return bucket_ab(bk, ha, key - ha * bk.cb);
}

// ------------------------------------------------------------- launchers
// (defined in the .cu files; all enqueue on `st` and do not synchronise)

// sfci_emit.cu
size_t emit_smem_bytes(const SysDev &d, int warps);
cudaError_t launch_emit(const SysDev &d, const unsigned long long *in_rank,
                        const double *in_coef, long long n_in, Table t, cudaStream_t st);
cudaError_t launch_emit_buckets(const SysDev &d, const unsigned long long *in_rank,
                                const double *in_coef, long long n_in, const BucketOut &b,
                                cudaStream_t st, int warps = 0);
// weights[ha] += intermediate elements bound for alpha string ha (enumerated,
// zeros included), over all input determinants; *n_runs += the number of runs
// of consecutive inputs sharing alpha
cudaError_t launch_row_weights(const SysDev &d, const unsigned long long *in_rank,
                               const double *in_coef, long long n_in, double eps_elem,
                               unsigned long long *weights, unsigned long long *n_runs, cudaStream_t st);
cudaError_t launch_debug_excitations(const SysDev &d, const unsigned long long *in_rank,
                                     long long n_in, long long *src, unsigned long long *tgt,
                                     double *elem, cudaStream_t st);
cudaError_t launch_rank(const SysDev &d, const unsigned long long *a, const unsigned long long *b,
                        unsigned long long *r, long long count, int *status, cudaStream_t st);
cudaError_t launch_unrank(const SysDev &d, const unsigned long long *r, unsigned long long *a,
                          unsigned long long *b, long long count, int *status, cudaStream_t st);

// sfci_table.cu
cudaError_t table_clear(Table t, cudaStream_t st);
// slot values = the exact sums of t.acc rounded to float64 (occupied slots)
cudaError_t table_finalize_exact(Table t, cudaStream_t st);
// bits of max |x_k| (non-negative doubles order as integers) into *out (zeroed first)
cudaError_t max_abs_bits(const double *x, long long n, unsigned long long *out, cudaStream_t st);
// mark entries with |val| < eps as screened (-0.0)
cudaError_t table_screen(Table t, double eps, unsigned long long *screened_dev, cudaStream_t st);
// flag[0] |= 1 if rank is not strictly ascending or some rank >= dim
cudaError_t validate_sorted(const unsigned long long *rank, long long n, unsigned long long dim,
                            int *flag, cudaStream_t st);
// add sign * scale[0] * coef[k] into entry rank[k] (scale device pointer, or
// host constant when scale == nullptr: then value = sign * hscale * coef)
cudaError_t table_axpy(Table t, const unsigned long long *rank, const double *coef, long long m,
                       const double *scale, double hscale, double sign, cudaStream_t st);
// unordered extraction of live entries with !(|val| < eps) into out; count in *n_dev
cudaError_t table_extract(Table t, double eps, unsigned long long *out_rank, double *out_val,
                          long long cap, unsigned long long *n_dev, cudaStream_t st);
// dots: out[j] = sum_k w_j[k] * sigma[w_j.rank[k]] for j < nvec (partials workspace)
struct VecRef {
    const unsigned long long *rank;
    const double *coef;
    long long n;
};
constexpr int kMaxVec = 64;
size_t dots_workspace_bytes(int nvec, long long max_n);
cudaError_t table_dots(Table t, const VecRef *vecs_host, int nvec, double *out_dev,
                       void *ws, cudaStream_t st);
// S: out[j] = <w_j | w_last> by binary search of w_last entries in w_j
cudaError_t vec_overlaps(const VecRef *vecs_host, int nvec, VecRef last, double *out_dev,
                         void *ws, cudaStream_t st);

// sfci_merge.cu -- bucketed merge (see the file's header)
struct Probe {
    unsigned long long key;    // rank of a basis-vector entry
    unsigned long long where;  // vector index j << 40 | position in w_j
};
struct VecPackRef {
    VecRef v[kMaxVec];
};
struct SigPack {
    double *p[kMaxVec];
};
struct MergeArgs {
    unsigned lo, hi;
    Buckets bk;
    const unsigned *count;              // [B] elements per bucket
    const Slot *elem;                   // regions of the pass buckets, relative to boff[lo]
    const Slot *ovf_sorted;             // overflow elements sorted by bucket
    const unsigned long long *ovf_off;  // [hi - lo + 1]
    long long ovf_cap;                  // entries of ovf_sorted
    const Probe *probes;                // sorted by bucket
    const unsigned long long *probe_off;  // [B + 1]
    double *sigw[kMaxVec];              // sigma recorded at w_j's entries
    int ja, jb;                         // vectors whose entries stay out of the stream (w_i, w_{i-1}); -1 none
    double eps;                         // screen
    unsigned long long *out_key;
    double *out_val;
    long long out_cap;
    unsigned long long *out_n;
    // Stream threshold, raised while the merge runs: bit pattern of a
    // non-negative double (|u| >= it is streamed out); hist counts the streamed
    // entries by magnitude bin; when out_n passes *mark one CTA (holding *lock)
    // raises it to the highest bin edge that still has nkeep streamed entries
    // at or above it, and moves *mark halfway to out_cap.
    unsigned long long *tau_bits;
    unsigned long long *hist;           // [kHistBins]
    unsigned long long *mark;
    int *lock;
    long long nkeep;
    int fix_shift;                      // S: sigma entries are summed exactly in units of 2^-S
    double *sumsq;                      // sum of u^2 over the non-zero entries off w_i, w_{i-1}
    unsigned long long *n_live;         // entries that survive the screen
    unsigned long long *n_nonzero;      // non-zero entries off w_i, w_{i-1} (streamed or not)
    unsigned long long *n_read;         // intermediate elements merged (null: not counted)
    unsigned *queue;
    int *status;                        // bit 2: a bucket has too many distinct keys; bit 3: output full;
                                        // bit 5: an element outside the 2^-S fixed-point range
};
// magnitude bins of |u|: the top 14 bits of the IEEE bit pattern (11 exponent
// bits, 2 mantissa bits: quarter octaves) of a non-negative double
constexpr int kHistShift = 50;
constexpr int kHistBins = 1 << (63 - kHistShift);
size_t scan_ws_bytes(long long m);

// sfci_plan.cu: merge-bucket plan (row mode) from exact per-row element counts
// w[nrows] and their exclusive prefix wpre; P elements per bucket, C beta
// strings, T windows of P/2.  plan_windows: tl[t] = a light row starts in window t, tc[t] = tl[t] +
// buckets of the heavy row starting there (th may alias tc); then bstart =
// exclusive scan of tc, and plan_rows writes the row map and the capacities
// of B = bstart[T] buckets.
cudaError_t plan_windows(const unsigned long long *w, const unsigned long long *wpre, unsigned long long nrows,
                         unsigned long long P, unsigned long long C, unsigned long long T, unsigned *tl, unsigned *th,
                         unsigned *tc, cudaStream_t st);
cudaError_t plan_rows(const unsigned long long *w, const unsigned long long *wpre, unsigned long long nrows,
                      unsigned long long P, unsigned long long C, const unsigned *tl, const unsigned long long *bstart,
                      unsigned long long B, unsigned long long *rowmap, unsigned *cap, cudaStream_t st);
// out[2k] = first bucket b <= nb with boff[b] >= targets[k], out[2k+1] = boff[b]
cudaError_t boff_lower_bounds(const unsigned long long *boff, unsigned long long nb,
                              const unsigned long long *targets, int n, unsigned long long *out, cudaStream_t st);
// start4[b] = (boff[b] - boff[lo]) / 4 for b in [lo, hi]
cudaError_t pass_offsets(const unsigned long long *boff, unsigned lo, unsigned hi, unsigned *start4,
                         cudaStream_t st);
// cap[b] rounded up to a multiple of 4
cudaError_t round_caps4(unsigned *cap, unsigned long long nb, cudaStream_t st);
// lim[0] = first alpha row that can hold buckets [lo, hi), lim[1] = one past the last
cudaError_t pass_rows(const unsigned long long *rowmap, unsigned long long nrows, unsigned lo, unsigned hi,
                      unsigned long long *lim, cudaStream_t st);
cudaError_t exclusive_scan(const unsigned *in, long long m, unsigned long long *out, void *ws,
                           cudaStream_t st);
cudaError_t exclusive_scan(const unsigned long long *in, long long m, unsigned long long *out, void *ws,
                           cudaStream_t st);
cudaError_t sort_overflow(const Buckets &bk, const unsigned *count, unsigned lo, unsigned nb,
                          const Slot *ovf, const unsigned long long *ovf_n, long long ovf_cap,
                          unsigned *tmp_counts, unsigned long long *off, void *scan_ws, Slot *out,
                          cudaStream_t st);
// probes of rows that receive no element get sigma = 0 written at once
cudaError_t sort_probes(const Buckets &bk, unsigned long long nbuckets, const VecRef *vecs,
                        double *const *sigw, int nvec, unsigned *pcount, unsigned long long *poff,
                        void *scan_ws, Probe *out, cudaStream_t st);
// boff[b] = b * cap for the hash mode's uniform regions
cudaError_t uniform_offsets(unsigned long long *boff, unsigned long long nb, unsigned cap,
                            cudaStream_t st);
// slots: shared-memory table size (2048, 4096 or 8192 keys)
cudaError_t launch_merge(const MergeArgs &A, int slots, cudaStream_t st);
cudaError_t launch_u_entries(VecRef wi, const double *sig_i, VecRef wm, const double *sig_m,
                             double a, double b, unsigned long long *out_key, double *out_val,
                             unsigned long long base_n, long long out_cap, double *sumsq,
                             int *status, cudaStream_t st);
// *out = min |val[k]| over the first *n_dev entries (+inf when none)
cudaError_t min_abs(const double *val, const unsigned long long *n_dev, long long cap, double *out,
                    cudaStream_t st);
size_t aligned_dots_ws_bytes(int nvec);
cudaError_t aligned_dots(const VecRef *vecs, double *const *sig, int nvec, double *out_dev, void *ws,
                         cudaStream_t st);

// sfci_select.cu
size_t select_workspace_bytes(long long n_items, long long k);
// Generic source of (key, val) items: either SoA arrays (stride 1) or table
// slots (stride 2, keys == kEmpty skipped).
struct Items {
    const unsigned long long *key;
    const double *val;
    int stride;
    long long n;
};
// top-k by (|val| desc, key asc), non-zero only; writes up to k entries sorted
// (unordered) to out; count to *n_out_dev.  If sumsq_dev != nullptr it
// receives sum val^2 over all valid items, and total_dev their number.
cudaError_t select_topk(Items it, long long k, unsigned long long *out_key, double *out_val,
                        unsigned long long *n_out_dev, double *sumsq_dev,
                        unsigned long long *total_dev, void *ws, size_t ws_bytes, cudaStream_t st);
// Two-level top-k: one pass histograms the first digit (top 12 bits of the
// composite key, 4096 bins), the bin holding the k-th item is picked, and one
// more pass writes every item of a smaller bin to out and every item of the
// picked bin to cand.  *state_host receives {n_out, n_cand, need, all, done}; the caller
// finishes with select_topk over the candidates when !done.
struct SplitResult {
    unsigned long long n_out, n_cand, need, total;
    int all, done;
};
cudaError_t select_split(Items it, long long k,
                         unsigned long long *out_key, double *out_val, unsigned long long *n_out_dev,
                         unsigned long long *cand_key, double *cand_val, long long cand_cap,
                         unsigned long long *cand_n, void *ws, size_t ws_bytes, SplitResult *res_host,
                         cudaStream_t st);
size_t sort_workspace_bytes(long long n);
// stable LSD radix sort of (key, val) by key on the low `bits` bits; result in
// key/val (uses ws as ping-pong buffers); n read from the device when n_dev
size_t sort_pairs_bytes(long long cap);
cudaError_t sort_pairs(unsigned long long *key, double *val, long long cap,
                       const unsigned long long *n_dev, int bits, void *ws, cudaStream_t st);
// c[i] /= sqrt(sum c^2) over n (device count) entries, deterministic order
cudaError_t normalize_vec(double *val, long long cap, const unsigned long long *n_dev,
                          void *ws, cudaStream_t st);
size_t normalize_ws_bytes(long long cap);

}  // namespace sfci
