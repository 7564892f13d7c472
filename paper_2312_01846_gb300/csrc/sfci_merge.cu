// The merge of sigma's intermediate elements (Sec. 2.2, step 2), bucketed for
// GB300.
//
// The paper spreads intermediate elements over buckets by index range so that
// cores merge buckets independently (Sec. 2.2, Fig. 1).  Here the emit kernel
// appends every element to one of 2^log2B hash buckets (one L2 counter atomic
// and one 16-byte store per element; bucket tails stay in L2 until their
// sectors fill, so HBM sees full-sector writes).  Each bucket holds ~2k
// elements, so one CTA merges a bucket in a shared-memory hash table and
// streams the distinct entries out: sigma costs one sequential write and one
// sequential read of the elements instead of a random read-modify-write per
// element.  A bucket whose counter passes its capacity (one target reached
// from very many sources) spills into an overflow list that is sorted by
// bucket before the merge.  When the elements would not fit in memory, the
// bucket range is processed in passes, each re-enumerating the sources and
// keeping only its own buckets.
//
// The Lanczos quantities are folded into the merge so that sigma is never
// searched: "probes" (rank k, vector j, position) for every entry of the basis
// vectors w_0..w_i are sorted into the same buckets; the merge of a bucket looks
// each probe up in shared memory and records sigma_k next to w_j's entry.  The
// entries of w_i and w_{i-1} are left out of the streamed output; their
// u = sigma - a w_i - b w_{i-1} values are formed later from the recorded
// sigma_k (Eq. 10).  Only entries with |u| >= tau are streamed out (tau below
// the previous step's truncation cut; the caller checks afterwards that the
// N_d largest all cleared it, and otherwise redoes the step with tau = 0), so
// the truncation reads a few N_d entries instead of all of sigma.
#include "sfci_internal.cuh"

namespace sfci {
namespace {

#ifndef SFCI_MERGE_THREADS
#define SFCI_MERGE_THREADS 256
#endif
constexpr int kMT = SFCI_MERGE_THREADS;  // merge CTA threads
constexpr int kPre = 4;              // elements each thread loads before inserting (4: more unrolling
                                     // outgrows the instruction cache; measured)

// slot in the shared-memory table.  Hash mode: the mix64 bits just below
// those that chose the bucket.  Row mode: a split row's bucket was chosen by
// the top bits of mix64 of the beta index, so the keys of one bucket share
// those bits; the slot comes from an independent mix (xor-shift-multiply
// finaliser) instead, or the keys would crowd a few slots.
template <int kSlots>
__device__ __forceinline__ unsigned smem_slot(unsigned long long key, int log2B) {
    if (log2B > 0) return (unsigned)(mix64(key) >> (64 - log2B - 13)) & (kSlots - 1);
    key ^= key >> 31;
    key *= 0xD6E8FEB86659FD93ull;
    key ^= key >> 32;
    return (unsigned)key & (kSlots - 1);
}

__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// ------------------------------------------------------------- scan

// exclusive scan of unsigned 32- or 64-bit counts into 64-bit offsets, m
// entries, out[m] = total; three kernels (block sums, scan of sums, block scans)
template <typename T>
__global__ void scan_sums_kernel(const T *in, long long m, unsigned long long *bsum) {
    __shared__ unsigned long long w[32];
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    unsigned long long v = i < m ? in[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long x = w[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = x;
    }
}

__global__ void scan_top_kernel(unsigned long long *bsum, long long nb) {
    // one block: exclusive scan of nb block sums in place
    __shared__ unsigned long long carry, w[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (long long b0 = 0; b0 < nb; b0 += blockDim.x) {
        const long long i = b0 + threadIdx.x;
        const unsigned long long v = i < nb ? bsum[i] : 0;
        unsigned long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) w[wp] = x;
        __syncthreads();
        if (wp == 0) {
            const unsigned long long s = w[lane];
            unsigned long long t = s;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(kFull, t, o);
                if (lane >= o) t += y;
            }
            w[lane] = t - s;
        }
        __syncthreads();
        const unsigned long long ex = carry + w[wp] + x - v;
        if (i < nb) bsum[i] = ex;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = ex + v;
        __syncthreads();
    }
}

template <typename T>
__global__ void scan_block_kernel(const T *in, long long m, const unsigned long long *bsum,
                                  unsigned long long *out) {
    __shared__ unsigned long long w[32];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    const unsigned long long v = i < m ? in[i] : 0;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) w[wp] = x;
    __syncthreads();
    if (wp == 0) {
        const unsigned long long s = w[lane];
        unsigned long long t = s;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        w[lane] = t - s;
    }
    __syncthreads();
    const unsigned long long ex = bsum[blockIdx.x] + w[wp] + x - v;
    if (i < m) out[i] = ex;
    if (i == m - 1) out[m] = ex + v;
}

// ------------------------------------------------------------- overflow

// overflow elements per bucket of the pass = max(count - capacity, 0)
__global__ void ovf_counts_kernel(const unsigned long long *boff, const unsigned *count, unsigned lo,
                                  unsigned nb, unsigned *ovc) {
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        const unsigned c = count[lo + b];
        const unsigned cap = (unsigned)(boff[lo + b + 1] - boff[lo + b]);
        ovc[b] = c > cap ? c - cap : 0u;
    }
}

__global__ void ovf_scatter_kernel(Buckets bk, const Slot *ovf, const unsigned long long *ovf_n,
                                   long long ovf_cap, unsigned lo, const unsigned long long *off,
                                   unsigned *fill, Slot *out) {
    long long n = (long long)*ovf_n;
    if (n > ovf_cap) n = ovf_cap;
    const unsigned lane = threadIdx.x & 31;
    // whole warps iterate together so that the lanes sharing a bucket take
    // their places with one atomic
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
        const long long i = i0 + lane;
        bool act = i < n;
        ulonglong2 e = make_ulonglong2(0ull, 0ull);
        unsigned b = 0;
        if (act) {
            e = reinterpret_cast<const ulonglong2 *>(ovf)[i];
            act = e.x != kEmpty;  // a place the emitting warp left unused
            if (act) b = bucket_key(bk, e.x) - lo;
        }
        const unsigned peers = __match_any_sync(kFull, act ? b : (0x80000000u | lane));
        const int leader = __ffs(peers) - 1;
        unsigned f0 = 0;
        if (act && (int)lane == leader) f0 = atomicAdd(&fill[b], (unsigned)__popc(peers));
        f0 = __shfl_sync(kFull, f0, leader);
        if (!act) continue;
        const unsigned long long pos = off[b] + f0 + __popc(peers & ((1u << lane) - 1u));
        // offsets count every overflowing element; a truncated list (status
        // bit 1, the sigma is redone) must not write past its end
        if ((long long)pos < ovf_cap) reinterpret_cast<ulonglong2 *>(out)[pos] = e;
    }
}

// ------------------------------------------------------------- probes

__global__ void probe_count_kernel(Buckets bk, VecPackRef vp, SigPack sp, int nvec, unsigned *pcount) {
    for (int j = 0; j < nvec; ++j) {
        const VecRef w = vp.v[j];
        for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < w.n;
             k += (long long)gridDim.x * blockDim.x) {
            const unsigned b = bucket_key(bk, w.rank[k]);
            if (b == kNoBucket) sp.p[j][k] = 0.0;  // no element reaches this row
            else atomicAdd(&pcount[b], 1u);
        }
    }
}

__global__ void probe_scatter_kernel(Buckets bk, VecPackRef vp, int nvec, const unsigned long long *poff,
                                     unsigned *pfill, Probe *out) {
    for (int j = 0; j < nvec; ++j) {
        const VecRef w = vp.v[j];
        for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < w.n;
             k += (long long)gridDim.x * blockDim.x) {
            const unsigned long long key = w.rank[k];
            const unsigned b = bucket_key(bk, key);
            if (b == kNoBucket) continue;
            const unsigned long long pos = poff[b] + atomicAdd(&pfill[b], 1u);
            Probe p;
            p.key = key;
            p.where = ((unsigned long long)j << 40) | (unsigned long long)k;
            out[pos] = p;
        }
    }
}

__global__ void uniform_offsets_kernel(unsigned long long *boff, unsigned long long nb, unsigned cap) {
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; b <= nb;
         b += (unsigned long long)gridDim.x * blockDim.x)
        boff[b] = b * cap;
}

// ------------------------------------------------------------- merge

// One CTA merges one bucket at a time (dynamic queue) in a shared-memory hash
// table.  Every thread first loads up to kPre of the bucket's elements into
// registers (independent loads in flight together), then inserts them; slots
// taken for the first time are listed, so clearing and streaming out touch only
// the occupied slots.
// Called by every thread of the CTA that holds A.lock: the highest histogram
// bin b whose streamed entries at or above it number >= nkeep (counts read
// while other CTAs still add, so they only undercount: the threshold is never
// too high), then tau = max(tau, lower edge of b) and the next mark halfway
// between out_n and out_cap; releases the lock.
__device__ __noinline__ void raise_threshold(const MergeArgs &A, int tid, int *s_bin,
                                             unsigned long long *part) {
    constexpr int per = kHistBins / kMT;  // bins per thread, thread 0 owns the top ones
    unsigned long long sum = 0;
    const int top = kHistBins - 1 - tid * per;
    for (int q = 0; q < per; ++q) sum += *(volatile unsigned long long *)&A.hist[top - q];
    part[tid] = sum;
    __syncthreads();
    if (tid == 0) {  // exclusive prefix from the top (kMT values)
        unsigned long long run = 0;
        for (int t = 0; t < kMT; ++t) {
            const unsigned long long v = part[t];
            part[t] = run;
            run += v;
        }
    }
    __syncthreads();
    const unsigned long long need = (unsigned long long)(A.nkeep > 0 ? A.nkeep : 1);
    unsigned long long run = part[tid];
    if (run < need && run + sum >= need) {
        // re-read: counts only grow, so a bin found with fresher counts is still
        // one with >= nkeep streamed entries at or above it
        for (int q = 0; q < per; ++q) {
            run += *(volatile unsigned long long *)&A.hist[top - q];
            if (run >= need) {
                *s_bin = top - q;
                break;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        const int b = *s_bin;
        if (b > 0) atomicMax(A.tau_bits, (unsigned long long)b << kHistShift);
        const unsigned long long on = *(volatile unsigned long long *)A.out_n;
        const unsigned long long cap = (unsigned long long)(A.out_cap > 0 ? A.out_cap : 0);
        *(volatile unsigned long long *)A.mark = on < cap ? on + (cap - on) / 2 : cap;
        __threadfence();
        atomicExch(A.lock, 0);
    }
    __syncthreads();
}

template <int kSlots>
__global__ void __launch_bounds__(kMT, 4)
merge_kernel(MergeArgs A) {
    extern __shared__ __align__(16) unsigned char msm[];
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(msm);
    unsigned long long *acc_lo = keys + kSlots;  // exact sums, low and high words
    unsigned long long *acc_hi = acc_lo + kSlots;
    unsigned short *occ = reinterpret_cast<unsigned short *>(acc_hi + kSlots);
    unsigned char *flag = reinterpret_cast<unsigned char *>(occ + kSlots);
    __shared__ unsigned cur, n_occ;
    __shared__ unsigned long long s_tau;
    __shared__ int s_raise, s_bin;
    __shared__ unsigned long long s_nread;  // elements merged by this CTA (kept out of registers)
    const int tid = threadIdx.x, lane = tid & 31;
    const bool screen = A.eps > 0.0;
    // thresholds compared on bit patterns (|x| < t for t >= 0, NaN never below)
    const unsigned long long eps_bits = abs_bits(A.eps);
    for (int sl = tid; sl < kSlots; sl += kMT) keys[sl] = kEmpty, acc_lo[sl] = 0ull, acc_hi[sl] = 0ull, flag[sl] = 0;
    const int S = A.fix_shift;
    bool range_ok = true;
    if (tid == 0) n_occ = 0, s_nread = 0, cur = atomicAdd(A.queue, 1u), s_tau = *(volatile unsigned long long *)A.tau_bits;
    double sq = 0.0;
    unsigned long long n_live = 0, n_nonzero = 0;
    __syncthreads();
    for (;;) {
        const unsigned bi = cur;  // bucket index within the pass
        if (bi >= A.hi - A.lo) break;
        const unsigned long long tau_bits = s_tau;
        const unsigned b = A.lo + bi;
        const unsigned cnt = A.count[b];
        const unsigned long long r0 = A.bk.boff[b];
        const unsigned bcap = (unsigned)(A.bk.boff[b + 1] - r0);
        const unsigned n_main = cnt < bcap ? cnt : bcap;
        unsigned long long o0 = A.ovf_off[bi], o1 = A.ovf_off[bi + 1];
        if (o1 > (unsigned long long)A.ovf_cap) o1 = (unsigned long long)A.ovf_cap;  // truncated list
        if (o0 > o1) o0 = o1;
        const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(A.elem) + (r0 - A.bk.boff[A.lo]);
        const ulonglong2 *ovs = reinterpret_cast<const ulonglong2 *>(A.ovf_sorted) + o0;
        const unsigned total = n_main + (unsigned)(o1 - o0);
        if (tid == 0) s_nread += total;
        // keys repeat a lot in a bucket past its region or holding more than
        // four elements per table slot: there the lanes sharing a key are
        // summed first (one table update per key and round); elsewhere a
        // round of 32 records rarely repeats a key and the grouping costs more
        // than it saves (measured)
        const bool hot = o1 > o0 || total > 4u * (unsigned)kSlots;
        for (unsigned e0 = 0; e0 < total; e0 += kMT * kPre) {
            ulonglong2 x[kPre];
#pragma unroll
            for (int k = 0; k < kPre; ++k) {
                const unsigned e = e0 + k * kMT + tid;
                x[k] = make_ulonglong2(kEmpty, 0ull);
                if (e < total) x[k] = e < n_main ? __ldcs(src + e) : __ldcs(ovs + (e - n_main));  // read once
            }
            const unsigned lt = (1u << lane) - 1u;
#pragma unroll
            for (int k = 0; k < kPre; ++k) {
                if (e0 + (unsigned)k * kMT >= total) break;  // block-uniform: no elements left
                const unsigned long long key = x[k].x;
                // (a place left empty holds the value 0, which converts to 0)
                Fix128 f = to_fixed(__longlong_as_double((long long)x[k].y), S, range_ok);
                bool act = key != kEmpty;
                if (hot) {
                    // lanes holding the same key: the lowest one sums the group's
                    // values (exact integer adds) and alone touches the table, so
                    // a key that many elements share costs one atomic per round
                    const unsigned peers = __match_any_sync(kFull, key);
                    act = act && (peers & lt) == 0;
                    const Fix128 f0 = f;
                    unsigned todo = act ? peers & ~(1u << lane) : 0u;
                    while (__any_sync(kFull, todo != 0u)) {
                        const int src = todo ? __ffs(todo) - 1 : lane;
                        const unsigned long long olo = __shfl_sync(kFull, f0.lo, src);
                        const unsigned long long ohi = __shfl_sync(kFull, f0.hi, src);
                        if (todo) {
                            f.lo += olo;
                            f.hi += ohi + (f.lo < olo ? 1ull : 0ull);
                            todo &= todo - 1u;
                        }
                    }
                }
                unsigned h = 0;
                bool ins = false, found = false;
                if (act) {
                    h = smem_slot<kSlots>(key, A.bk.rowmap ? 0 : A.bk.log2B);
                    for (int probe = 0; probe < kSlots; ++probe) {
                        const unsigned long long c = keys[h];
                        if (c == key) {
                            found = true;
                            break;
                        }
                        if (c == kEmpty) {
                            const unsigned long long old = atomicCAS(&keys[h], kEmpty, key);
                            if (old == kEmpty || old == key) {
                                ins = old == kEmpty;
                                found = true;
                                break;
                            }
                        }
                        h = (h + (unsigned)probe + 1u) & (kSlots - 1);  // triangular steps: every slot once
                    }
                }
                // newly occupied slots: one list reservation per warp
                const unsigned bal = __ballot_sync(kFull, ins);
                if (bal) {
                    const int leader = __ffs(bal) - 1;
                    unsigned base = 0;
                    if (lane == leader) base = atomicAdd(&n_occ, (unsigned)__popc(bal));
                    base = __shfl_sync(kFull, base, leader);
                    if (ins) occ[base + __popc(bal & lt)] = (unsigned short)h;
                }
                if (act) {
                    if (found) {
                        // the 128-bit sum as four 32-bit limbs, each added with a native
                        // 32-bit shared-memory atomic and the carry passed up by hand
                        // (64-bit shared atomics run at a sixth of the 32-bit rate)
                        unsigned *l32 = reinterpret_cast<unsigned *>(acc_lo) + 2 * h;
                        unsigned *h32 = reinterpret_cast<unsigned *>(acc_hi) + 2 * h;
                        const unsigned w0 = (unsigned)f.lo, w1 = (unsigned)(f.lo >> 32);
                        const unsigned w2 = (unsigned)f.hi, w3 = (unsigned)(f.hi >> 32);
                        unsigned o = atomicAdd(l32, w0);
                        unsigned c = (o + w0) < o;
                        unsigned x = w1 + c, cx = c & (w1 == 0xFFFFFFFFu);  // w1 + c wrapped: carry out
                        o = atomicAdd(l32 + 1, x);
                        c = cx | ((o + x) < o);
                        x = w2 + c, cx = c & (w2 == 0xFFFFFFFFu);
                        o = atomicAdd(h32, x);
                        c = cx | ((o + x) < o);
                        atomicAdd(h32 + 1, w3 + c);
                    } else {
                        atomicOr(A.status, 4);
                    }
                }
            }
        }
        __syncthreads();
        // probes: record sigma at the basis-vector entries
        const unsigned long long p0 = A.probe_off[b], p1 = A.probe_off[b + 1];
        for (unsigned long long p = p0 + tid; p < p1; p += kMT) {
            const Probe pr = A.probes[p];
            unsigned h = smem_slot<kSlots>(pr.key, A.bk.rowmap ? 0 : A.bk.log2B);
            int found = -1;
            for (int q = 0; q < kSlots; ++q) {
                const unsigned long long c = keys[h];
                if (c == pr.key) {
                    found = (int)h;
                    break;
                }
                if (c == kEmpty) break;
                h = (h + (unsigned)q + 1u) & (kSlots - 1);
            }
            double sv = found >= 0 ? from_fixed(acc_lo[found], acc_hi[found], S) : 0.0;
            if (screen && abs_bits(sv) < eps_bits) sv = 0.0;  // screened entries count as absent
            const int j = (int)(pr.where >> 40);
            const long long k = (long long)(pr.where & ((1ull << 40) - 1));
            A.sigw[j][k] = sv;
            if (found >= 0 && (j == A.ja || j == A.jb)) flag[found] = 1;
        }
        __syncthreads();
        // stream the occupied slots with |u| >= tau out (u = sigma there) and
        // clear them for the next bucket
        const unsigned nocc = n_occ;
        for (unsigned t0 = 0; t0 < nocc; t0 += kMT) {
            const unsigned t = t0 + tid;
            unsigned long long key = kEmpty;
            double v = 0.0;
            bool live = false, w = false;
            unsigned hb = 0x80000000u | (unsigned)lane;
            if (t < nocc) {
                const unsigned sl = occ[t];
                key = keys[sl];
                v = from_fixed(acc_lo[sl], acc_hi[sl], S);
                const unsigned long long ab = abs_bits(v);
                live = !(screen && ab < eps_bits);
                const bool nz = live && !flag[sl] && ab != 0ull;
                if (nz) {
                    ++n_nonzero;
                    sq = __fma_rn(v, v, sq);
                }
                w = nz && !(ab < tau_bits);
                keys[sl] = kEmpty, acc_lo[sl] = 0ull, acc_hi[sl] = 0ull, flag[sl] = 0;
                if (w) hb = (unsigned)(ab >> kHistShift);
            }
            // histogram of the streamed entries (lanes sharing a bin add once)
            if (__any_sync(kFull, w)) {
                const unsigned peers = __match_any_sync(kFull, hb);
                if (w && (peers & ((1u << lane) - 1u)) == 0)
                    atomicAdd(&A.hist[hb], (unsigned long long)__popc(peers));
            }
            n_live += live;
            const unsigned bal = __ballot_sync(kFull, w);
            unsigned long long base = 0;
            if (lane == 0 && bal) base = atomicAdd(A.out_n, (unsigned long long)__popc(bal));
            base = __shfl_sync(kFull, base, 0);
            if (w) {
                const unsigned long long pos = base + __popc(bal & ((1u << lane) - 1u));
                if ((long long)pos < A.out_cap) {
                    A.out_key[pos] = key;
                    A.out_val[pos] = v;
                } else {
                    atomicOr(A.status, 8);
                }
            }
        }
        __syncthreads();
        // raise the threshold once the stream passes the mark (one CTA at a time)
        if (tid == 0) {
            s_raise = 0;
            s_bin = -1;
            const unsigned long long on = *(volatile unsigned long long *)A.out_n;
            if (on >= *(volatile unsigned long long *)A.mark && atomicCAS(A.lock, 0, 1) == 0) s_raise = 1;
        }
        __syncthreads();
        // (the bucket's occupied-slot list is spent: its shared memory holds the partial sums)
        if (s_raise) raise_threshold(A, tid, &s_bin, reinterpret_cast<unsigned long long *>(occ));
        if (tid == 0) n_occ = 0, cur = atomicAdd(A.queue, 1u), s_tau = *(volatile unsigned long long *)A.tau_bits;
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) {
        sq += __shfl_xor_sync(kFull, sq, o);
        n_live += __shfl_xor_sync(kFull, n_live, o);
        n_nonzero += __shfl_xor_sync(kFull, n_nonzero, o);
    }
    if (lane == 0) {
        atomicAdd(A.sumsq, sq);
        atomicAdd(A.n_live, n_live);
        atomicAdd(A.n_nonzero, n_nonzero);
    }
    if (tid == 0 && A.n_read) atomicAdd(A.n_read, s_nread);
    if (!range_ok) atomicOr(A.status, 32);
}

constexpr size_t merge_smem(int slots) { return size_t(slots) * (8 + 16 + 2 + 1); }

// ------------------------------------------------------------- u entries

// u on the support of w_i (and w_{i-1}): u_k = sigma_k - a w_i[k] - b w_{i-1}[k]
// (Eq. 10), appended after the streamed entries; entries of w_{i-1} that w_i
// also holds are written as empty keys.
__global__ void u_entries_kernel(VecRef wi, const double *sig_i, VecRef wm, const double *sig_m,
                                 double a, double b, unsigned long long *out_key, double *out_val,
                                 unsigned long long base_n, long long out_cap, double *sumsq,
                                 int *status) {
    double sq = 0.0;
    const long long total = wi.n + wm.n;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        unsigned long long key;
        double u;
        bool valid = true;
        if (t < wi.n) {
            key = wi.rank[t];
            u = __dsub_rn(sig_i[t], __dmul_rn(a, wi.coef[t]));
            // w_{i-1} entry with the same rank
            long long lo = 0, hi = wm.n;
            while (lo < hi) {
                const long long mid = lo + ((hi - lo) >> 1);
                if (wm.rank[mid] < key) lo = mid + 1;
                else hi = mid;
            }
            if (lo < wm.n && wm.rank[lo] == key) u = __dsub_rn(u, __dmul_rn(b, wm.coef[lo]));
        } else {
            const long long k = t - wi.n;
            key = wm.rank[k];
            long long lo = 0, hi = wi.n;
            while (lo < hi) {
                const long long mid = lo + ((hi - lo) >> 1);
                if (wi.rank[mid] < key) lo = mid + 1;
                else hi = mid;
            }
            if (lo < wi.n && wi.rank[lo] == key) valid = false;
            u = __dsub_rn(sig_m[k], __dmul_rn(b, wm.coef[k]));
        }
        const unsigned long long pos = base_n + (unsigned long long)t;
        if ((long long)pos >= out_cap) {
            atomicOr(status, 8);
            continue;
        }
        out_key[pos] = valid ? key : kEmpty;
        out_val[pos] = valid ? u : 0.0;
        if (valid && u != 0.0) sq = __fma_rn(u, u, sq);
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(kFull, sq, o);
    if ((threadIdx.x & 31) == 0 && sq != 0.0) atomicAdd(sumsq, sq);
}

// <w_j | sigma> from the recorded sigma at w_j's entries: fixed grid, fixed order
constexpr int kDotBlocks = 304;

__global__ void aligned_dots_kernel(VecPackRef vp, SigPack sp, double *partial) {
    __shared__ double sh[8];
    const int j = blockIdx.y;
    const VecRef w = vp.v[j];
    const double *sg = sp.p[j];
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < w.n;
         k += (long long)gridDim.x * blockDim.x)
        acc = __fma_rn(w.coef[k], sg[k], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r += sh[q];
        partial[(size_t)j * gridDim.x + blockIdx.x] = r;
    }
}

__global__ void aligned_finish_kernel(const double *partial, int np, double *out) {
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int k = 0; k < np; ++k) r += partial[(size_t)blockIdx.x * np + k];
        out[blockIdx.x] = r;
    }
}

__global__ void min_abs_kernel(const double *val, const unsigned long long *n_dev, long long cap,
                               double *out) {
    __shared__ double sh[32];
    long long n = (long long)*n_dev;
    if (n > cap) n = cap;
    double m = __longlong_as_double(0x7ff0000000000000ll);  // +inf
    for (long long i = threadIdx.x; i < n; i += blockDim.x) m = fmin(m, fabs(val[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = sh[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmin(r, sh[w]);
        *out = r;
    }
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

unsigned grid_for(long long work, int per_sm) {
    long long g = (work + 255) / 256;
    const long long c = (long long)sm_count() * per_sm;
    if (g > c) g = c;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

size_t scan_ws_bytes(long long m) {
    const long long nb = (m + 1023) / 1024;
    return size_t(nb > 0 ? nb : 1) * 8;
}

namespace {
template <typename T>
cudaError_t exclusive_scan_t(const T *in, long long m, unsigned long long *out, void *ws, cudaStream_t st) {
    if (m <= 0) return cudaMemsetAsync(out, 0, 8, st);
    const long long nb = (m + 1023) / 1024;
    unsigned long long *bsum = static_cast<unsigned long long *>(ws);
    count_launch();
    scan_sums_kernel<<<(unsigned)nb, 1024, 0, st>>>(in, m, bsum);
    count_launch();
    scan_top_kernel<<<1, 1024, 0, st>>>(bsum, nb);
    count_launch();
    scan_block_kernel<<<(unsigned)nb, 1024, 0, st>>>(in, m, bsum, out);
    return cudaGetLastError();
}
}  // namespace

cudaError_t exclusive_scan(const unsigned *in, long long m, unsigned long long *out, void *ws,
                           cudaStream_t st) {
    return exclusive_scan_t(in, m, out, ws, st);
}

cudaError_t exclusive_scan(const unsigned long long *in, long long m, unsigned long long *out, void *ws,
                           cudaStream_t st) {
    return exclusive_scan_t(in, m, out, ws, st);
}

cudaError_t sort_overflow(const Buckets &bk, const unsigned *count, unsigned lo, unsigned nb,
                          const Slot *ovf, const unsigned long long *ovf_n, long long ovf_cap,
                          unsigned *tmp_counts, unsigned long long *off, void *scan_ws, Slot *out,
                          cudaStream_t st) {
    count_launch();
    ovf_counts_kernel<<<grid_for(nb, 8), 256, 0, st>>>(bk.boff, count, lo, nb, tmp_counts);
    cudaError_t e = exclusive_scan(tmp_counts, nb, off, scan_ws, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(tmp_counts, 0, size_t(nb) * 4, st);
    if (e != cudaSuccess) return e;
    count_launch();
    ovf_scatter_kernel<<<grid_for(ovf_cap < (1 << 24) ? ovf_cap : (1 << 24), 8), 256, 0, st>>>(
        bk, ovf, ovf_n, ovf_cap, lo, off, tmp_counts, out);
    return cudaGetLastError();
}

cudaError_t sort_probes(const Buckets &bk, unsigned long long nbuckets, const VecRef *vecs,
                        double *const *sigw, int nvec, unsigned *pcount, unsigned long long *poff,
                        void *scan_ws, Probe *out, cudaStream_t st) {
    VecPackRef vp{};
    SigPack sp{};
    long long mx = 1;
    for (int j = 0; j < nvec; ++j) vp.v[j] = vecs[j], sp.p[j] = sigw[j], mx = vecs[j].n > mx ? vecs[j].n : mx;
    cudaError_t e = cudaMemsetAsync(pcount, 0, nbuckets * 4, st);
    if (e != cudaSuccess) return e;
    count_launch();
    probe_count_kernel<<<grid_for(mx, 8), 256, 0, st>>>(bk, vp, sp, nvec, pcount);
    e = exclusive_scan(pcount, (long long)nbuckets, poff, scan_ws, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(pcount, 0, nbuckets * 4, st);
    if (e != cudaSuccess) return e;
    count_launch();
    probe_scatter_kernel<<<grid_for(mx, 8), 256, 0, st>>>(bk, vp, nvec, poff, pcount, out);
    return cudaGetLastError();
}

cudaError_t uniform_offsets(unsigned long long *boff, unsigned long long nb, unsigned cap,
                            cudaStream_t st) {
    count_launch();
    uniform_offsets_kernel<<<grid_for((long long)nb + 1, 8), 256, 0, st>>>(boff, nb, cap);
    return cudaGetLastError();
}

template <int kSlots>
cudaError_t launch_merge_t(const MergeArgs &A, cudaStream_t st) {
    const size_t smem = merge_smem(kSlots);
    cudaError_t e = allow_max_smem(merge_kernel<kSlots>, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, merge_kernel<kSlots>, kMT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const long long nb = (long long)(A.hi - A.lo);
    long long grid = (long long)sm_count() * per_sm;
    if (grid > nb) grid = nb;
    if (grid < 1) return cudaSuccess;
    count_launch();
    merge_kernel<kSlots><<<(unsigned)grid, kMT, smem, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_merge(const MergeArgs &A, int slots, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(A.queue, 0, 4, st);
    if (e != cudaSuccess) return e;
    if (slots <= 1024) return launch_merge_t<1024>(A, st);
    if (slots <= 2048) return launch_merge_t<2048>(A, st);
    if (slots <= 4096) return launch_merge_t<4096>(A, st);
    return launch_merge_t<8192>(A, st);
}

cudaError_t launch_u_entries(VecRef wi, const double *sig_i, VecRef wm, const double *sig_m,
                             double a, double b, unsigned long long *out_key, double *out_val,
                             unsigned long long base_n, long long out_cap, double *sumsq,
                             int *status, cudaStream_t st) {
    const long long total = wi.n + wm.n;
    if (total <= 0) return cudaSuccess;
    count_launch();
    u_entries_kernel<<<grid_for(total, 8), 256, 0, st>>>(wi, sig_i, wm, sig_m, a, b, out_key, out_val,
                                                         base_n, out_cap, sumsq, status);
    return cudaGetLastError();
}

cudaError_t min_abs(const double *val, const unsigned long long *n_dev, long long cap, double *out,
                    cudaStream_t st) {
    count_launch();
    min_abs_kernel<<<1, 1024, 0, st>>>(val, n_dev, cap, out);
    return cudaGetLastError();
}

size_t aligned_dots_ws_bytes(int nvec) { return size_t(nvec > 0 ? nvec : 1) * kDotBlocks * 8; }

cudaError_t aligned_dots(const VecRef *vecs, double *const *sig, int nvec, double *out_dev, void *ws,
                         cudaStream_t st) {
    if (nvec <= 0) return cudaSuccess;
    VecPackRef vp{};
    SigPack sp{};
    for (int j = 0; j < nvec; ++j) vp.v[j] = vecs[j], sp.p[j] = sig[j];
    double *partial = static_cast<double *>(ws);
    count_launch();
    aligned_dots_kernel<<<dim3(kDotBlocks, nvec), 256, 0, st>>>(vp, sp, partial);
    count_launch();
    aligned_finish_kernel<<<nvec, 32, 0, st>>>(partial, kDotBlocks, out_dev);
    return cudaGetLastError();
}

}  // namespace sfci
