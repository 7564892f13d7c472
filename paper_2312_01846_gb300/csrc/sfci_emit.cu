// sigma = H psi, step 1 (Sec. 2.2): every input entry (D, c_D) generates its
// intermediate elements (rank(D'), <D'|H|D> c_D) for D' = D and all single and
// double excitations of D (Sec. 3; Sec. 4.3 notes that every single and
// double excitation is generated).  Where each element goes depends on the
// launch: in the solver's bucket mode it is appended as a 16-byte record
// (rank, value) to its target's merge-bucket region in HBM (past the region's
// end: to the overflow list), and the merge kernel reduces each bucket in
// shared memory (sfci_merge.cu); in table mode (the standalone sfci_sigma) it
// is added exactly into a device-wide hash table; the debug mode writes every
// element unscaled.
//
// One warp owns one input determinant at a time:
//   a1  rank -> (alpha, beta): division by C(n, n_beta), greedy inverse of Eq. 12
//       with one warp ballot per electron;
//   a2  occupied / empty orbital lists from warp ballots;
//       per-source tables of the alpha and beta single excitations (index of
//       the excited string by Eq. 12, signed single element, g row offset);
//   a3  fermionic signs from popc of the occupied bits strictly between the
//       two orbitals of each hop (hop 1, then hop 2 on the updated string);
//   a4  Slater-Condon elements: singles h_ai + sum_k (ai|kk) - sum_k' (ak'|k'i),
//       same-spin doubles (ai|bj) - (aj|bi), opposite-spin doubles (ai|bj),
//       the diagonal; terms summed in the same order as the oracle, with
//       explicit round-to-nearest intrinsics so no multiply-add is fused;
//   a5  target index: alpha-major rank = h(alpha') C(n, n_beta) + h(beta');
//       opposite-spin doubles combine two single-table entries (one IMAD);
//   a6  element * c_D, exact zeros dropped, then appended to the target's
//       bucket (warp-aggregated reservation, one atomic per bucket and round)
//       or added into the table.
// The lanes of the warp stride over the excitations of each class, one element
// per lane per round; the opposite-spin doubles of an alpha hop whose target
// row has at most kHopBins buckets reserve their places per bucket once for
// the whole hop, and reservations into a row split further compute its
// buckets' region offsets from the first one (equal regions).
//
// In bucket mode the alpha-alpha doubles can go by runs instead
// (emit_aa_kernel): the sources sharing an alpha string are consecutive, so a
// warp takes a window of 32 sources, computes each run's alpha-alpha
// excitations once and pairs the live ones with the run's beta strings.  The
// host picks that path when a pass leaves rows to others or the runs average
// two sources or more.
#include <algorithm>
#include <type_traits>

#include "sfci_internal.cuh"

namespace sfci {
namespace {

constexpr int kEmitThreads = 256;
constexpr int kEmitWarps = kEmitThreads / 32;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t block_smem(const SysDev &d) {
    return align16(size_t(d.n + 1) * d.ks * 8) + align16(size_t(d.n_pairs) * 2);
}

// Opposite-spin doubles of an alpha hop whose target row has at most this many
// buckets reserve their places per bucket once per hop (bins below).
constexpr int kHopBins = 32;

// per warp: overflow chunk cursor (2 u64), prefix sums (3 ks u64), rankA1,
// rankB1 (u32 when every string index fits 32 bits, else u64), offA1, offB1,
// mixB (u32), the hop's bins (4 x kHopBins u32), hopX (u16 per alpha hop), yoff
// (u16 per beta hop), occupation lists (256 B).  The 32-bit tables keep a CTA of
// eight warps small enough that four CTAs leave the SM 92 KB of L1 instead of
// 60 KB (the integral rows and the row map are read through it; measured).
__host__ __device__ inline size_t warp_smem(const SysDev &d, bool narrow = false) {
    const size_t r = narrow ? 4 : 8;
    return align16(16 + size_t(d.sa) * (r + 6) + size_t(d.sb) * (r + 10) + size_t(3 * d.ks) * 8 +
                   size_t(kHopBins) * 16 + 256);
}

// string indices below 2^32 on both spins: 32-bit single tables
__host__ __device__ inline bool narrow_ranks(const SysDev &d) { return (d.ca >> 32) == 0 && (d.cb >> 32) == 0; }

inline size_t emit_smem_bytes_w(const SysDev &d, int warps, bool narrow = false) {
    return block_smem(d) + size_t(warps) * warp_smem(d, narrow);
}

// single element h_ai + sum_{k occ alpha} (ai|kk) + sum_{k occ beta} (ai|kk)
//                 - sum_{k occ same spin} (ak|ki), source occupations
__device__ __forceinline__ double single_element(const SysDev &d, int i, int a,
                                                 const unsigned char *occA,
                                                 const unsigned char *occB,
                                                 const unsigned char *occS, int ns) {
    const int n = d.n;
    const size_t n2 = size_t(n) * n;
    const double *gai = d.g + size_t(a * n + i) * n2;
    double v = __ldg(&d.h[a * n + i]);
    for (int k = 0; k < d.na; ++k) {
        int o = occA[k];
        v = __dadd_rn(v, __ldg(&gai[o * n + o]));
    }
    for (int k = 0; k < d.nb; ++k) {
        int o = occB[k];
        v = __dadd_rn(v, __ldg(&gai[o * n + o]));
    }
    for (int k = 0; k < ns; ++k) {
        int o = occS[k];
        v = __dsub_rn(v, __ldg(&d.g[(size_t(a * n + o) * n + o) * n + i]));
    }
    return v;
}

// the same single element from the float32 integral copies, float32 sums in
// the same order (SFCI_FP32_ELEMENTS)
__device__ __forceinline__ double single_element_f32(const SysDev &d, int i, int a,
                                                     const unsigned char *occA,
                                                     const unsigned char *occB,
                                                     const unsigned char *occS, int ns) {
    const int n = d.n;
    const size_t n2 = size_t(n) * n;
    const float *gai = d.gf + size_t(a * n + i) * n2;
    float v = __ldg(&d.hf[a * n + i]);
    for (int k = 0; k < d.na; ++k) {
        int o = occA[k];
        v = __fadd_rn(v, __ldg(&gai[o * n + o]));
    }
    for (int k = 0; k < d.nb; ++k) {
        int o = occB[k];
        v = __fadd_rn(v, __ldg(&gai[o * n + o]));
    }
    for (int k = 0; k < ns; ++k) {
        int o = occS[k];
        v = __fsub_rn(v, __ldg(&d.gf[(size_t(a * n + o) * n + o) * n + i]));
    }
    return (double)v;
}

// <D|H|D> = e_core + sum_k h_kk + 1/2 sum_{k,l} (kk|ll) - 1/2 sum_{k,l same spin} (kl|lk)
__device__ double diagonal_element(const SysDev &d, const unsigned char *occA,
                                   const unsigned char *occB) {
    const int n = d.n;
    double one = 0.0, coul = 0.0, exch = 0.0;
    for (int k = 0; k < d.na; ++k) one = __dadd_rn(one, __ldg(&d.h[occA[k] * (n + 1)]));
    for (int k = 0; k < d.nb; ++k) one = __dadd_rn(one, __ldg(&d.h[occB[k] * (n + 1)]));
    const int m = d.na + d.nb;
    for (int k = 0; k < m; ++k) {
        int p = k < d.na ? occA[k] : occB[k - d.na];
        const double *gpp = d.g + size_t(p * n + p) * n * n;
        for (int l = 0; l < m; ++l) {
            int q = l < d.na ? occA[l] : occB[l - d.na];
            coul = __dadd_rn(coul, __ldg(&gpp[q * n + q]));
        }
    }
    for (int s = 0; s < 2; ++s) {
        const unsigned char *o = s ? occB : occA;
        int ms = s ? d.nb : d.na;
        for (int k = 0; k < ms; ++k)
            for (int l = 0; l < ms; ++l)
                exch = __dadd_rn(exch, __ldg(&d.g[(size_t(o[k] * n + o[l]) * n + o[l]) * n + o[k]]));
    }
    return __dsub_rn(__dadd_rn(__dadd_rn(d.e_core, one), __dmul_rn(0.5, coul)),
                     __dmul_rn(0.5, exch));
}

// flip the sign of x when s is 1 (bit operation, exact; keeps the FP64 pipe free)
__device__ __forceinline__ double flip(double x, unsigned s) {
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)s << 63));
}

__device__ __forceinline__ bool nonzero(double v) {
    return ((unsigned long long)__double_as_longlong(v) << 1) != 0ull;
}

constexpr int kU = 1;  // elements each lane carries per reservation round (2 and 3 measured slower)

__device__ __forceinline__ bool in_pass(const BucketOut &B, unsigned b) { return b >= B.lo && b < B.hi; }

// Elements past their bucket's region go to the overflow list.  Each warp
// takes the list in chunks of kOvfChunk places (one atomic on the list's
// counter per chunk; the counter is shared by every warp of the GPU) and fills
// them in order; the places a warp leaves unused are marked empty (key
// kEmpty), which the sort by bucket skips.  cur = {next place, chunk end} in
// the warp's shared memory.  Every lane calls it.
constexpr unsigned kOvfChunk = 256;

__device__ __forceinline__ void ovf_pad(const BucketOut &B, unsigned long long q, unsigned long long end) {
    for (q += threadIdx.x & 31; q < end; q += 32)
        if ((long long)q < B.ovf_cap) reinterpret_cast<ulonglong2 *>(B.ovf)[q] = make_ulonglong2(kEmpty, 0ull);
}

__device__ __forceinline__ void overflow_append(const BucketOut &B, bool of, const ulonglong2 &sl,
                                                unsigned long long *cur) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(kFull, of);
    if (!bal) return;
    const unsigned n = __popc(bal);
    unsigned long long pos = cur[0], end = cur[1];
    if (pos + n > end) {
        ovf_pad(B, pos, end);
        unsigned long long q0 = 0;
        if (lane == 0) q0 = atomicAdd(B.ovf_n, (unsigned long long)kOvfChunk);
        pos = __shfl_sync(kFull, q0, 0);
        end = pos + kOvfChunk;
    }
    __syncwarp();
    if (lane == 0) cur[0] = pos + n, cur[1] = end;
    __syncwarp();
    if (!of) return;
    const unsigned long long q = pos + __popc(bal & ((1u << lane) - 1u));
    if ((long long)q < B.ovf_cap) reinterpret_cast<ulonglong2 *>(B.ovf)[q] = sl;
    else atomicOr(B.status, 2);
}

// A row split into several buckets (a heavy row) gives them equal regions, so
// within one pass the region of its bucket b >= b0 starts at s0 + (b - b0) c4
// (units of 4 slots; b0 = the row's first bucket in the pass).  c4 == 0: not
// such a row (one bucket, or hash mode).  Only for rows with buckets in the pass.
struct RowRegion {
    unsigned b0, s0, c4;
};

// bucket of a target whose alpha row is known ahead (first bucket and bucket
// count of the row read once): ns == ~0 means hash mode (no row map)
struct RowCtx {
    unsigned first, ns;
};

__device__ __forceinline__ RowRegion row_region(const BucketOut &B, RowCtx rc) {
    if (rc.ns == 0xffffffffu || rc.ns < 2u) return RowRegion{0u, 0u, 0u};
    const unsigned b0 = rc.first > B.lo ? rc.first : B.lo;
    const unsigned s0 = __ldg(&B.start4[b0]);
    return RowRegion{b0, s0, __ldg(&B.start4[b0 + 1]) - s0};
}

// Up to kU elements per lane (ok[k]) are appended to their buckets: the lanes
// of the warp that share a bucket reserve their slots with one atomic, issued
// for all k before any result is used, and write one run.  With rr.c4 set,
// every element's bucket belongs to rr's row and its region is computed, not read.
__device__ __forceinline__ void warp_append(const BucketOut &B, const bool *ok, const unsigned *bk,
                                            const unsigned long long *tg, const double *v,
                                            unsigned long long *cur, RowRegion rr = RowRegion{0u, 0u, 0u}) {
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    unsigned peers[kU], base[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) peers[k] = __match_any_sync(kFull, ok[k] ? bk[k] : (0x80000000u | lane));
#pragma unroll
    for (int k = 0; k < kU; ++k) {
        base[k] = 0;
        if (ok[k] && (peers[k] & lt) == 0) base[k] = atomicAdd(&B.count[bk[k]], (unsigned)__popc(peers[k]));
    }
#pragma unroll
    for (int k = 0; k < kU; ++k) base[k] = __shfl_sync(kFull, base[k], __ffs(peers[k]) - 1);
#pragma unroll
    for (int k = 0; k < kU; ++k) {
        bool of = false;
        const ulonglong2 sl = make_ulonglong2(tg[k], (unsigned long long)__double_as_longlong(v[k]));
        if (ok[k]) {
            const unsigned pos = base[k] + __popc(peers[k] & lt);
            unsigned long long o0, room;
            if (rr.c4) {
                o0 = (unsigned long long)(rr.s0 + (bk[k] - rr.b0) * rr.c4) << 2;
                room = (unsigned long long)rr.c4 << 2;
            } else {
                o0 = (unsigned long long)__ldg(&B.start4[bk[k]]) << 2;
                room = ((unsigned long long)__ldg(&B.start4[bk[k] + 1]) << 2) - o0;
            }
            if (pos < room) __stcs(reinterpret_cast<ulonglong2 *>(B.elem) + o0 + pos, sl);  // streamed: read once by the merge
            else of = true;
        }
        overflow_append(B, of, sl, cur);
    }
}

__device__ __forceinline__ RowCtx row_ctx(const BucketOut &B, unsigned long long ha) {
    if (!B.bk.rowmap) return RowCtx{0u, 0xffffffffu};
    const unsigned long long m = __ldg(&B.bk.rowmap[ha]);
    return RowCtx{(unsigned)(m >> 32), (unsigned)m};
}

// same value as bucket_ab(bk, ha, hb) for the row of rc
__device__ __forceinline__ unsigned row_bucket(const Buckets &bk, RowCtx rc, unsigned long long ha,
                                               unsigned long long hb) {
    if (rc.ns == 0xffffffffu) {
        const unsigned long long key = ha * bk.cb + hb;
        return bk.log2B > 0 ? (unsigned)(mix64(key) >> (64 - bk.log2B)) : 0u;
    }
    if (rc.ns <= 1) return rc.ns ? rc.first : kNoBucket;
    return rc.first + (unsigned)(((mix64(hb) >> 32) * rc.ns) >> 32);
}

// can any bucket of the row be in this pass?  A row without buckets means
// the row weights missed it: status 16.
__device__ __forceinline__ bool ctx_in_pass(const BucketOut &B, RowCtx rc) {
    if (rc.ns == 0xffffffffu) return true;
    if (rc.ns == 0) {
        atomicOr(B.status, 16);
        return false;
    }
    return rc.first < B.hi && rc.first + rc.ns > B.lo;
}

// target in this launch?  (bucket mode: its bucket b is in the pass)
template <int kMode>
__device__ __forceinline__ bool wanted(const EmitOut &o, unsigned long long ha, unsigned long long hb,
                                       unsigned &b) {
    if (kMode != kModeBucket) return true;
    if (ha < o.b.row_lo || ha > o.b.row_hi) return false;
    b = bucket_ab(o.b.bk, ha, hb);
    if (b == kNoBucket) {
        atomicOr(o.b.status, 16);
        return false;
    }
    return in_pass(o.b, b);
}

template <int kMode>
__device__ __forceinline__ bool row_wanted(const EmitOut &o, RowCtx rc, unsigned long long ha,
                                           unsigned long long hb, unsigned &b) {
    if (kMode != kModeBucket) return true;
    b = row_bucket(o.b.bk, rc, ha, hb);
    return in_pass(o.b, b);
}

// A round whose elements all go to bucket b (a row with one bucket): one
// reservation for the whole warp, positions by ballot prefix.
__device__ __forceinline__ void single_append(const BucketOut &B, unsigned b, const bool *ok,
                                              const unsigned long long *tg, const double *v,
                                              unsigned long long *cur) {
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    unsigned pre[kU], tot = 0;
#pragma unroll
    for (int k = 0; k < kU; ++k) {
        const unsigned bal = __ballot_sync(kFull, ok[k]);
        pre[k] = tot + __popc(bal & lt);
        tot += __popc(bal);
    }
    if (tot == 0) return;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(&B.count[b], tot);
    base = __shfl_sync(kFull, base, 0);
    const unsigned long long o0 = (unsigned long long)__ldg(&B.start4[b]) << 2;
    const unsigned long long cap = ((unsigned long long)__ldg(&B.start4[b + 1]) << 2) - o0;
    ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(B.elem) + o0;
#pragma unroll
    for (int k = 0; k < kU; ++k) {
        bool of = false;
        const ulonglong2 sl = make_ulonglong2(tg[k], (unsigned long long)__double_as_longlong(v[k]));
        if (ok[k]) {
            const unsigned pos = base + pre[k];
            if (pos < cap) __stcs(dst + pos, sl);
            else of = true;
        }
        overflow_append(B, of, sl, cur);
    }
}

// the bucket of every wanted element of the round when they all share one,
// -2 when the round has none, else -1 (every lane calls it)
__device__ __forceinline__ long long round_single(const bool *want, const unsigned *bk) {
    unsigned mine = kNoBucket;
#pragma unroll
    for (int k = 0; k < kU; ++k)
        if (want[k] && mine == kNoBucket) mine = bk[k];
    const unsigned has = __ballot_sync(kFull, mine != kNoBucket);
    if (!has) return -2;
    const unsigned ref = __shfl_sync(kFull, mine, __ffs(has) - 1);
    bool diff = false;
#pragma unroll
    for (int k = 0; k < kU; ++k) diff |= want[k] && bk[k] != ref;
    return __any_sync(kFull, diff) ? -1 : (long long)ref;
}

// One round of the warp over up to kU elements per lane: element k of this
// lane targets (ha[k], hb[k]) in bucket bk[k] with unscaled value e[k] (only
// computed when want[k]); debug and table modes deliver lane by lane.  With
// single >= 0 every element of the round is in bucket `single`; -2: the
// round has no element.
template <int kMode>
__device__ __forceinline__ void emit_round(const EmitOut &o, const bool *want,
                                           const unsigned long long *ha, const unsigned long long *hb,
                                           const unsigned *bk, const double *e, const long long *di,
                                           long long s, double c, unsigned long long cb,
                                           unsigned &inserted, unsigned long long *cur,
                                           long long single = -1, RowRegion rr = RowRegion{0u, 0u, 0u}) {
    if constexpr (kMode == kModeDebug) {
#pragma unroll
        for (int k = 0; k < kU; ++k)
            if (want[k]) o.dsrc[di[k]] = s, o.dtgt[di[k]] = ha[k] * cb + hb[k], o.delem[di[k]] = e[k];
    } else if constexpr (kMode == kModeTable) {
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            if (!want[k]) continue;
            const double v = __dmul_rn(e[k], c);
            if (!nonzero(v)) continue;
            if (o.t.acc) table_add_exact(o.t, ha[k] * cb + hb[k], v, inserted);
            else table_add(o.t, ha[k] * cb + hb[k], v, inserted);
        }
    } else {
        if (single == -2) return;
        bool ok[kU];
        unsigned long long tg[kU];
        double v[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            ok[k] = false;
            tg[k] = 0;
            v[k] = 0.0;
            if (!want[k]) continue;
            v[k] = __dmul_rn(e[k], c);
            tg[k] = ha[k] * cb + hb[k];
            ok[k] = nonzero(v[k]);
        }
        if (o.b.eps_elem > 0.0) {  // heat-bath style screen (uniform branch: no FP64 compare when off)
#pragma unroll
            for (int k = 0; k < kU; ++k) ok[k] = ok[k] && !(fabs(v[k]) < o.b.eps_elem);
        }
        bool any = false;
#pragma unroll
        for (int k = 0; k < kU; ++k) any |= ok[k];
        if (!__any_sync(kFull, any)) return;  // nothing of this pass in the round
        if (single >= 0) single_append(o.b, (unsigned)single, ok, tg, v, cur);
        else warp_append(o.b, ok, bk, tg, v, cur, rr);
    }
}

// prefix sums A0 | A1 | A2 over the M - 2 electrons of str left after removing
// occupied positions io < jo:  A0[m] = sum_{t<=m} C(r_t, t), A1[m] = sum C(r_t, t+1),
// A2[m] = sum C(r_t, t+2) (every lane of the warp calls it)
__device__ __forceinline__ void pair_prefix(const unsigned char *occ, int M, int io, int jo,
                                            const unsigned long long *bt, int ks,
                                            unsigned long long *pre) {
    const int lane = threadIdx.x & 31;
    unsigned long long c0 = 0, c1 = 0, c2 = 0;
    if (lane < M - 2) {
        int t = lane;
        if (t >= io) ++t;
        if (t >= jo) ++t;
        const int e = occ[t];
        c0 = bt[e * ks + lane + 1];
        c1 = bt[e * ks + lane + 2];
        c2 = bt[e * ks + lane + 3];
    }
    for (int w = 1; w < 32; w <<= 1) {
        const unsigned long long y0 = __shfl_up_sync(kFull, c0, w);
        const unsigned long long y1 = __shfl_up_sync(kFull, c1, w);
        const unsigned long long y2 = __shfl_up_sync(kFull, c2, w);
        if (lane >= w) c0 += y0, c1 += y1, c2 += y2;
    }
    if (lane < M - 2) pre[lane + 1] = c0, pre[ks + lane + 1] = c1, pre[2 * ks + lane + 1] = c2;
    if (lane == 0) pre[0] = 0, pre[ks] = 0, pre[2 * ks] = 0;
    __syncwarp();
}

// Eq. 12 index of rem | a | b (a < b empty in rem) from the prefix sums: the
// spectators below a keep their position, those between a and b move up one,
// those above b move up two
__device__ __forceinline__ unsigned long long pair_rank(unsigned long long rem, int a, int b, int M,
                                                        const unsigned long long *pre,
                                                        const unsigned long long *bt, int ks) {
    const int q1 = __popcll(rem & ((1ull << a) - 1ull));
    const int q2 = __popcll(rem & ((1ull << b) - 1ull));
    return pre[q1] + bt[a * ks + q1 + 1] + pre[ks + q2] - pre[ks + q1] + bt[b * ks + q2 + 2] +
           pre[2 * ks + (M - 2)] - pre[2 * ks + q2];
}

template <int kMode, bool kNarrow = false>
__global__ void __launch_bounds__(kEmitThreads, 4)
emit_kernel(const SysDev d, const unsigned long long *__restrict__ in_rank,
            const double *__restrict__ in_coef, long long n_in, const EmitOut o) {
    using RankT = typename std::conditional<kNarrow, unsigned, unsigned long long>::type;
    extern __shared__ __align__(16) unsigned char sm[];
    const int n = d.n, ks = d.ks;
    unsigned long long *bt = reinterpret_cast<unsigned long long *>(sm);
    unsigned char *pairs = sm + align16(size_t(n + 1) * ks * 8);
    for (int i = threadIdx.x; i < (n + 1) * ks; i += blockDim.x) bt[i] = d.binom[i];
    for (int i = threadIdx.x; i < 2 * d.n_pairs; i += blockDim.x) pairs[i] = d.pairs[i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wb = sm + block_smem(d) + size_t(warp) * warp_smem(d, kNarrow);
    unsigned long long *ocur = reinterpret_cast<unsigned long long *>(wb);  // overflow chunk cursor
    unsigned long long *pre = ocur + 2;  // prefix sums A0 | A1 | A2, ks each
    RankT *rankA1 = reinterpret_cast<RankT *>(pre + 3 * ks);
    RankT *rankB1 = rankA1 + d.sa;
    unsigned *offA1 = reinterpret_cast<unsigned *>(rankB1 + d.sb);
    unsigned *offB1 = offA1 + d.sa;
    unsigned *mixB = offB1 + d.sb;  // top 32 bits of mix64 of each beta hop's index (its bucket in a split row)
    unsigned *hcnt = mixB + d.sb;   // per bucket of the current alpha hop's row: elements,
    unsigned *hbase = hcnt + kHopBins;  // first reserved place,
    unsigned *hs0 = hbase + kHopBins;   // region start (units of 4 slots), region capacity
    unsigned *hcap = hs0 + kHopBins;
    unsigned short *hopX = reinterpret_cast<unsigned short *>(hcap + kHopBins);  // kept alpha hops
    unsigned short *yoff = hopX + d.sa;  // place of each beta hop's element within its bucket's share
    unsigned char *occA = reinterpret_cast<unsigned char *>(yoff + d.sb);
    unsigned char *virA = occA + 64, *occB = occA + 128, *virB = occA + 192;
    const unsigned char *pOA = pairs + 2 * d.pair_off[0], *pVA = pairs + 2 * d.pair_off[1];
    const unsigned char *pOB = pairs + 2 * d.pair_off[2], *pVB = pairs + 2 * d.pair_off[3];
    const unsigned long long cb = d.cb;
    const double *__restrict__ g = d.g;
    const size_t n2 = size_t(n) * n;
    const bool f32 = d.gf != nullptr;  // SFCI_FP32_ELEMENTS: off-diagonal elements in float32

    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned inserted = 0;
    const long long per = d.n_conn + 1;
    if (lane == 0) ocur[0] = 0ull, ocur[1] = 0ull;
    __syncwarp();

    for (long long s = gw; s < n_in; s += nw) {
        const unsigned long long r = in_rank[s];
        const double c = kMode == kModeDebug ? 1.0 : in_coef[s];
        const unsigned long long hA = r / cb, hB = r - hA * cb;
        const unsigned long long alpha = string_unrank_warp(hA, n, d.na, bt, ks);
        const unsigned long long beta = string_unrank_warp(hB, n, d.nb, bt, ks);
        const long long base = s * per;

        build_lists(alpha, beta, n, occA, virA, occB, virB);
        __syncwarp();
        // single-excitation tables: Eq. 12 index of the excited string, g row
        // offset, hop sign (bit 31)
        for (int x = lane; x < d.sa; x += 32) {
            const int io = x / d.va, iv = x - io * d.va;
            const int i = occA[io], a = virA[iv];
            const unsigned sg = parity64(alpha & between_mask(i, a));
            rankA1[x] = (RankT)string_rank(alpha ^ (1ull << i) ^ (1ull << a), bt, ks);
            offA1[x] = unsigned((a * n + i) * n2) | (sg << 31);
        }
        for (int y = lane; y < d.sb; y += 32) {
            const int jo = y / d.vb, jv = y - jo * d.vb;
            const int j = occB[jo], b = virB[jv];
            const unsigned sg = parity64(beta & between_mask(j, b));
            rankB1[y] = (RankT)string_rank(beta ^ (1ull << j) ^ (1ull << b), bt, ks);
            offB1[y] = unsigned(b * n + j) | (sg << 31);
            if (kMode == kModeBucket) mixB[y] = (unsigned)(mix64((unsigned long long)rankB1[y]) >> 32);
        }
        __syncwarp();
        // alpha hops whose target row can hold buckets of this pass (every hop
        // outside bucket mode), compacted
        int m_hops = 0;
        for (int x0 = 0; x0 < d.sa; x0 += 32) {
            const int x = x0 + lane;
            bool keep = false;
            if (x < d.sa) {
                if (kMode == kModeBucket && rankA1[x] >= o.b.row_lo && rankA1[x] <= o.b.row_hi) {
                    const RowCtx rc = row_ctx(o.b, rankA1[x]);
                    keep = ctx_in_pass(o.b, rc);
                    // heat-bath style screen: no beta hop can lift |(ai|bj) c| to eps
                    if (keep && o.b.eps_elem > 0.0) {
                        const int io = x / d.va, iv = x - io * d.va;
                        keep = !(fabs(c) * __ldg(&d.bound_ab[virA[iv] * n + occA[io]]) < o.b.eps_elem);
                    }
                } else {
                    keep = kMode != kModeBucket;
                }
                // a hop whose integrals (ai|bj) are all exactly zero gives only zero
                // opposite-spin doubles, which are dropped anyway: skipped (exact;
                // e.g. the on-site interaction of a Hubbard model); the debug mode
                // lists every element
                if (keep && kMode != kModeDebug) {
                    const int io = x / d.va, iv = x - io * d.va;
                    keep = __double_as_longlong(__ldg(&d.bound_ab[virA[iv] * n + occA[io]])) != 0ll;
                }
            }
            const unsigned bal = __ballot_sync(kFull, keep);
            if (keep) hopX[m_hops + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)x;
            m_hops += __popc(bal);
        }
        __syncwarp();
        // the source's own row: first bucket and count read once
        const bool self_in = kMode != kModeBucket || (hA >= o.b.row_lo && hA <= o.b.row_hi);
        const RowCtx rs = kMode == kModeBucket && self_in ? row_ctx(o.b, hA) : RowCtx{0u, 0u};
        const bool self_row = kMode != kModeBucket || (self_in && ctx_in_pass(o.b, rs));
        const long long self_single = kMode == kModeBucket && rs.ns == 1 ? (long long)rs.first : -1;

        bool want[kU];
        unsigned long long ha[kU], hb[kU];
        unsigned bk[kU];
        double e[kU];
        long long di[kU];
#define SFCI_CLEAR()                                                                          \
    for (int k = 0; k < kU; ++k) want[k] = false, ha[k] = 0, hb[k] = 0, bk[k] = 0, e[k] = 0.0, di[k] = 0;

        // diagonal (lane 0, in the oracle's term order)
        unsigned dbk = 0;
        const bool dwant = self_row && row_wanted<kMode>(o, rs, hA, hB, dbk);
        const double ediag = dwant && lane == 0 ? diagonal_element(d, occA, occB) : 0.0;
        // diagonal and alpha singles
        for (int x0 = -1; x0 < d.sa; x0 += 32 * kU) {
            SFCI_CLEAR();
#pragma unroll
            for (int k = 0; k < kU; ++k) {
                const int x = x0 + 32 * k + lane;
                if (x == -1) {
                    if (!dwant) continue;
                    want[k] = true, ha[k] = hA, hb[k] = hB, bk[k] = dbk, di[k] = base;
                    e[k] = ediag;
                } else if (x >= 0 && x < d.sa) {
                    if (!wanted<kMode>(o, rankA1[x], hB, bk[k])) continue;
                    const int io = x / d.va, iv = x - io * d.va;
                    const double F = f32 ? single_element_f32(d, occA[io], virA[iv], occA, occB, occA, d.na)
                                         : single_element(d, occA[io], virA[iv], occA, occB, occA, d.na);
                    want[k] = true, ha[k] = rankA1[x], hb[k] = hB, di[k] = base + 1 + x;
                    e[k] = flip(F, offA1[x] >> 31);
                }
            }
            emit_round<kMode>(o, want, ha, hb, bk, e, di, s, c, cb, inserted, ocur);
        }
        long long off = base + 1 + d.sa;
        // beta singles (all in row hA)
        if (self_row) {
            for (int y0 = 0; y0 < d.sb; y0 += 32 * kU) {
                SFCI_CLEAR();
#pragma unroll
                for (int k = 0; k < kU; ++k) {
                    const int y = y0 + 32 * k + lane;
                    if (y >= d.sb || !row_wanted<kMode>(o, rs, hA, rankB1[y], bk[k])) continue;
                    const int jo = y / d.vb, jv = y - jo * d.vb;
                    const double F = f32 ? single_element_f32(d, occB[jo], virB[jv], occA, occB, occB, d.nb)
                                         : single_element(d, occB[jo], virB[jv], occA, occB, occB, d.nb);
                    want[k] = true, ha[k] = hA, hb[k] = rankB1[y], di[k] = off + y;
                    e[k] = flip(F, offB1[y] >> 31);
                }
                emit_round<kMode>(o, want, ha, hb, bk, e, di, s, c, cb, inserted, ocur, self_single,
                                  row_region(o.b, rs));  // (the own row is in this pass here)
            }
        }
        off += d.sb;
        // same-spin doubles (i<j) -> (a<b), i->a then j->b; the excited
        // string's index from the prefix sums (pair_rank)
        for (int spin = 0; spin < 2; ++spin) {
            const unsigned long long str = spin ? beta : alpha;
            const unsigned char *occ = spin ? occB : occA, *vir = spin ? virB : virA;
            const unsigned char *po = spin ? pOB : pOA, *pv = spin ? pVB : pVA;
            const int npo = spin ? d.po_b : d.po_a, npv = spin ? d.pv_b : d.pv_a;
            const int M = spin ? d.nb : d.na;
            // beta-beta doubles stay in row hA; alpha-alpha doubles go by runs of
            // sources sharing alpha (emit_aa_kernel) when o.b.aa_runs is set
            if ((spin == 1 && !self_row) || (spin == 0 && kMode == kModeBucket && o.b.aa_runs)) {
                off += (long long)npo * npv;
                continue;
            }
            for (int p = 0; p < npo; ++p) {
                const int io = po[2 * p], jo = po[2 * p + 1];
                const int i = occ[io], j = occ[jo];
                if (kMode == kModeBucket && o.b.eps_elem > 0.0 &&
                    fabs(c) * __ldg(&d.bound_ss[i * n + j]) < o.b.eps_elem)
                    continue;  // heat-bath style screen: no (a, b) of this pair survives
                if (kMode != kModeDebug && __double_as_longlong(__ldg(&d.bound_ss[i * n + j])) == 0ll)
                    continue;  // every (ai|bj) - (aj|bi) of this pair is exactly zero
                const unsigned long long rem = str ^ (1ull << i) ^ (1ull << j);
                pair_prefix(occ, M, io, jo, bt, ks, pre);
                for (int q0 = 0; q0 < npv; q0 += 32 * kU) {
                    SFCI_CLEAR();
#pragma unroll
                    for (int k = 0; k < kU; ++k) {
                        const int q = q0 + 32 * k + lane;
                        if (q >= npv) continue;
                        const int a = vir[pv[2 * q]], b = vir[pv[2 * q + 1]];
                        const unsigned long long h2 = pair_rank(rem, a, b, M, pre, bt, ks);
                        const unsigned long long ta = spin ? hA : h2, tb = spin ? h2 : hB;
                        if (spin ? !row_wanted<kMode>(o, rs, ta, tb, bk[k]) : !wanted<kMode>(o, ta, tb, bk[k]))
                            continue;
                        const int s1 = parity64(str & between_mask(i, a));
                        const unsigned long long s1s = str ^ (1ull << i) ^ (1ull << a);
                        const int s2 = parity64(s1s & between_mask(j, b));
                        want[k] = true, ha[k] = ta, hb[k] = tb, di[k] = off + (long long)p * npv + q;
                        const size_t x1 = (size_t(a * n + i) * n + b) * n + j;
                        const size_t x2 = (size_t(a * n + j) * n + b) * n + i;
                        const double gd = f32 ? (double)__fsub_rn(__ldg(&d.gf[x1]), __ldg(&d.gf[x2]))
                                              : __dsub_rn(__ldg(&g[x1]), __ldg(&g[x2]));
                        e[k] = flip(gd, unsigned(s1 ^ s2));
                    }
                    emit_round<kMode>(o, want, ha, hb, bk, e, di, s, c, cb, inserted, ocur, spin ? self_single : -1,
                                      spin ? row_region(o.b, rs) : RowRegion{0u, 0u, 0u});
                }
                __syncwarp();
            }
            off += (long long)npo * npv;
        }
        // opposite-spin doubles.  Bucket mode, one kept alpha hop at a time: when
        // the hop's target row has at most kHopBins buckets, its sb elements are
        // counted per bucket (shared-memory atomics), each bucket's places are
        // reserved with one atomic and its region read once, and every element
        // goes straight to its place (a zero product keeps its place as a
        // zero-valued element); rows split further take rounds with per-round
        // reservations.  Other modes: flattened over (kept alpha hop, beta hop)
        // pairs, lane t taking pairs t, t + 32, ... so every round is full.
        if (kMode == kModeBucket && d.sb > 0) {
            for (int cx = 0; cx < m_hops; ++cx) {
                const int x = hopX[cx];
                const unsigned long long ra = rankA1[x];
                const RowCtx rc = row_ctx(o.b, ra);
                const unsigned oa = offA1[x];
                const unsigned long long rbase = ra * cb;
                if (rc.ns != 0xffffffffu && rc.ns <= (unsigned)kHopBins) {
                    const unsigned ns = rc.ns, first = rc.first;
                    if ((unsigned)lane < ns) hcnt[lane] = 0u;
                    __syncwarp();
                    for (int y = lane; y < d.sb; y += 32) {
                        const unsigned bin = ns == 1u ? 0u : __umulhi(mixB[y], ns);
                        yoff[y] = in_pass(o.b, first + bin) ? (unsigned short)atomicAdd(&hcnt[bin], 1u)
                                                            : (unsigned short)0xffffu;
                    }
                    __syncwarp();
                    if ((unsigned)lane < ns) {
                        const unsigned cnt = hcnt[lane];
                        unsigned base = 0u, s0 = 0u, s1 = 0u;
                        if (cnt) {
                            const unsigned b = first + lane;
                            base = atomicAdd(&o.b.count[b], cnt);
                            s0 = __ldg(&o.b.start4[b]);
                            s1 = __ldg(&o.b.start4[b + 1]);
                        }
                        hbase[lane] = base, hs0[lane] = s0, hcap[lane] = (s1 - s0) << 2;
                    }
                    __syncwarp();
                    ulonglong2 *elem = reinterpret_cast<ulonglong2 *>(o.b.elem);
                    for (int y0 = 0; y0 < d.sb; y0 += 32) {
                        const int y = y0 + lane;
                        bool of = false;
                        ulonglong2 sl = make_ulonglong2(0ull, 0ull);
                        if (y < d.sb && yoff[y] != 0xffffu) {
                            const unsigned bin = ns == 1u ? 0u : __umulhi(mixB[y], ns);
                            const unsigned ob = offB1[y];
                            const unsigned gi = (oa & 0x7fffffffu) + (ob & 0x7fffffffu);
                            const double gv = f32 ? (double)__ldg(&d.gf[gi]) : __ldg(&g[gi]);
                            double v = __dmul_rn(flip(gv, (oa ^ ob) >> 31), c);
                            if (!nonzero(v) || (o.b.eps_elem > 0.0 && fabs(v) < o.b.eps_elem)) v = 0.0;
                            sl = make_ulonglong2(rbase + rankB1[y], (unsigned long long)__double_as_longlong(v));
                            const unsigned pos = hbase[bin] + yoff[y];
                            if (pos < hcap[bin]) __stcs(elem + ((unsigned long long)hs0[bin] << 2) + pos, sl);
                            else of = true;
                        }
                        overflow_append(o.b, of, sl, ocur);
                    }
                    __syncwarp();  // the bins are reused by the next hop
                } else {
                    // a row split more ways than there are bins (or hash mode): per
                    // round reservations, regions computed from the row's first one
                    const RowRegion rhop = row_region(o.b, rc);
                    for (int y0 = 0; y0 < d.sb; y0 += 32 * kU) {
                        SFCI_CLEAR();
#pragma unroll
                        for (int k = 0; k < kU; ++k) {
                            const int y = y0 + 32 * k + lane;
                            if (y >= d.sb) continue;
                            const unsigned long long hbv = rankB1[y];
                            if (!row_wanted<kMode>(o, rc, ra, hbv, bk[k])) continue;
                            const unsigned ob = offB1[y];
                            const unsigned gi = (oa & 0x7fffffffu) + (ob & 0x7fffffffu);
                            const double gv = f32 ? (double)__ldg(&d.gf[gi]) : __ldg(&g[gi]);
                            want[k] = true, ha[k] = ra, hb[k] = hbv;
                            e[k] = flip(gv, (oa ^ ob) >> 31);
                        }
                        emit_round<kMode>(o, want, ha, hb, bk, e, di, s, c, cb, inserted, ocur, -1, rhop);
                    }
                }
            }
        } else if (d.sb > 0 && m_hops > 0) {
            const long long nab = (long long)m_hops * d.sb;
            int cx = lane / d.sb;
            int cy = lane - cx * d.sb;
            for (long long t0 = 0; t0 < nab; t0 += 32 * kU) {
                SFCI_CLEAR();
#pragma unroll
                for (int k = 0; k < kU; ++k) {
                    if (t0 + 32 * k + lane < nab) {
                        const int x = hopX[cx];
                        const unsigned long long ra = rankA1[x], hbv = rankB1[cy];
                        const RowCtx rc{0u, 0u};  // not used outside bucket mode
                        if (row_wanted<kMode>(o, rc, ra, hbv, bk[k])) {
                            const unsigned oa = offA1[x], ob = offB1[cy];
                            const unsigned gi = (oa & 0x7fffffffu) + (ob & 0x7fffffffu);
                            const double gv = f32 ? (double)__ldg(&d.gf[gi]) : __ldg(&g[gi]);
                            want[k] = true, ha[k] = ra, hb[k] = hbv;
                            di[k] = off + (long long)x * d.sb + cy;
                            e[k] = flip(gv, (oa ^ ob) >> 31);
                        }
                    }
                    cy += 32;
                    while (cy >= d.sb) cy -= d.sb, ++cx;
                }
                emit_round<kMode>(o, want, ha, hb, bk, e, di, s, c, cb, inserted, ocur,
                                  kMode == kModeBucket ? round_single(want, bk) : -1);
            }
        }
#undef SFCI_CLEAR
        __syncwarp();
    }
    if constexpr (kMode == kModeBucket) {  // the unused rest of the warp's overflow chunk
        __syncwarp();
        ovf_pad(o.b, ocur[0], ocur[1]);
    }
    if (kMode == kModeTable) {
        for (int w = 16; w > 0; w >>= 1) inserted += __shfl_xor_sync(kFull, inserted, w);
        if (lane == 0 && inserted) atomicAdd(o.t.count, (unsigned long long)inserted);
    }
}

// Live alpha-alpha excitations of a run waiting for their elements: a ring
// of kAaQ entries per warp (target row, its first bucket and bucket count,
// unscaled element).
constexpr int kAaQ = 64;

// per warp: overflow chunk cursor (2 u64), prefix sums (3 ks u64), the queue
// (kAaQ x 24 B), occupation lists (256 B)
__host__ __device__ inline size_t aa_warp_smem(const SysDev &d) {
    return align16(16 + size_t(3 * d.ks) * 8 + size_t(kAaQ) * 24 + 256);
}

// Alpha-alpha doubles of bucket mode, by runs of sources sharing alpha.  The
// input is sorted by rank, alpha-major, so the determinants with one alpha
// string are consecutive; their alpha-alpha doubles reach the same target rows
// with the same integrals and signs and differ only in the beta column and the
// coefficient.  A work unit is a window of 32 consecutive sources and one of
// n_groups slices of the occupied pairs (i, j) (several slices when the
// windows alone are too few to fill the GPU); the warp splits the window into
// its runs.  For a run of length L, the warp first takes the excitations
// (i, j) -> (a, b) one per lane: target row, its buckets (one row-map read)
// and the element; those whose row can hold buckets of this pass and whose
// element is not zero join a queue.  Rounds of 32 (excitation,
// source) items then leave the queue (lane t: excitation t / L, source
// t mod L, in queue order), so a round is full whatever the share of rows in
// the pass, and the lanes of one excitation share a row and often a bucket
// (one reservation, one run of places).
__global__ void __launch_bounds__(kEmitThreads, 4)
emit_aa_kernel(const SysDev d, const unsigned long long *__restrict__ in_rank,
               const double *__restrict__ in_coef, long long n_in, int n_groups, const EmitOut o) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int n = d.n, ks = d.ks;
    unsigned long long *bt = reinterpret_cast<unsigned long long *>(sm);
    unsigned char *pairs = sm + align16(size_t(n + 1) * ks * 8);
    for (int i = threadIdx.x; i < (n + 1) * ks; i += blockDim.x) bt[i] = d.binom[i];
    for (int i = threadIdx.x; i < 2 * d.n_pairs; i += blockDim.x) pairs[i] = d.pairs[i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    unsigned char *wb = sm + block_smem(d) + size_t(warp) * aa_warp_smem(d);
    unsigned long long *ocur = reinterpret_cast<unsigned long long *>(wb);
    unsigned long long *pre = ocur + 2;
    unsigned long long *qh = pre + 3 * ks;  // queue: target row
    double *qe = reinterpret_cast<double *>(qh + kAaQ);  // unscaled element
    unsigned *qf = reinterpret_cast<unsigned *>(qe + kAaQ);  // first bucket of the row
    unsigned *qn = qf + kAaQ;  // bucket count of the row (~0: hash mode)
    unsigned char *occA = reinterpret_cast<unsigned char *>(qn + kAaQ);
    unsigned char *virA = occA + 64, *occB = occA + 128, *virB = occA + 192;
    const unsigned char *pOA = pairs + 2 * d.pair_off[0], *pVA = pairs + 2 * d.pair_off[1];
    const unsigned long long cb = d.cb;
    const double *__restrict__ g = d.g;
    const bool f32 = d.gf != nullptr;
    const int npo = d.po_a, npv = d.pv_a, M = d.na;

    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned inserted = 0;
    if (lane == 0) ocur[0] = 0ull, ocur[1] = 0ull;
    __syncwarp();

    const long long n_units = (n_in + 31) / 32 * n_groups;
    for (long long u = gw; u < n_units; u += nw) {
        const long long win = u / n_groups;
        const int grp = (int)(u - win * n_groups);
        const int p_lo = grp * npo / n_groups, p_hi = (grp + 1) * npo / n_groups;
        const long long sl = win * 32 + lane;
        const bool valid = sl < n_in;
        const unsigned long long r = valid ? in_rank[sl] : 0ull;
        const double cl = valid ? in_coef[sl] : 0.0;
        const unsigned long long hAl = r / cb, hBl = r - hAl * cb;
        const unsigned mixl = (unsigned)(mix64(hBl) >> 32);
        const unsigned long long hAu = __shfl_up_sync(kFull, hAl, 1);
        unsigned starts = __ballot_sync(kFull, valid && (lane == 0 || hAu != hAl));
        const int n_valid = __popc(__ballot_sync(kFull, valid));
        while (starts) {
            const int s0 = __ffs(starts) - 1;
            starts &= starts - 1u;
            const int L = (starts ? __ffs(starts) - 1 : n_valid) - s0;
            const unsigned long long hA = __shfl_sync(kFull, hAl, s0);
            double cmax = (lane >= s0 && lane < s0 + L) ? fabs(cl) : 0.0;  // the run's largest |c| (screen)
            for (int w = 16; w > 0; w >>= 1) cmax = fmax(cmax, __shfl_xor_sync(kFull, cmax, w));
            const unsigned long long alpha = string_unrank_warp(hA, n, d.na, bt, ks);
            build_lists(alpha, 0ull, n, occA, virA, occB, virB);
            __syncwarp();
            // queue state (warp-uniform): excitations pushed, items emitted; this
            // lane's item cur + lane is excitation k, source sr of the run
            const int dq = 32 / L, ds = 32 - dq * L;
            unsigned qhead = 0, cur = 0;
            int k = lane / L, sr = lane - (lane / L) * L;
            // one round: items cur .. cur + 31 (those below qhead * L exist)
            auto round = [&]() {
                bool want[kU] = {false};
                unsigned long long ha[kU] = {0ull}, hb[kU] = {0ull};
                unsigned bk[kU] = {0u};
                double e[kU] = {0.0};
                long long di[kU] = {0};
                const int src = s0 + sr;
                const unsigned long long hbs = __shfl_sync(kFull, hBl, src);
                const double cs = __shfl_sync(kFull, cl, src);
                const unsigned ms = __shfl_sync(kFull, mixl, src);
                if (cur + (unsigned)lane < qhead * (unsigned)L) {
                    const int qi = k & (kAaQ - 1);
                    const unsigned long long h2 = qh[qi];
                    const unsigned ns = qn[qi], first = qf[qi];
                    bk[0] = ns == 0xffffffffu ? bucket_ab(o.b.bk, h2, hbs)
                                              : (ns == 1u ? first : first + __umulhi(ms, ns));
                    want[0] = in_pass(o.b, bk[0]);
                    ha[0] = h2, hb[0] = hbs, e[0] = qe[qi];
                }
                emit_round<kModeBucket>(o, want, ha, hb, bk, e, di, 0, cs, cb, inserted, ocur,
                                        L == 32 ? round_single(want, bk) : -1);
                cur += 32u, k += dq, sr += ds;
                if (sr >= L) sr -= L, ++k;
            };
            for (int p = p_lo; p < p_hi; ++p) {
                const int io = pOA[2 * p], jo = pOA[2 * p + 1];
                const int i = occA[io], j = occA[jo];
                if (o.b.eps_elem > 0.0 && cmax * __ldg(&d.bound_ss[i * n + j]) < o.b.eps_elem)
                    continue;  // heat-bath style screen: no (a, b) of this pair survives for any source
                if (__double_as_longlong(__ldg(&d.bound_ss[i * n + j])) == 0ll)
                    continue;  // every (ai|bj) - (aj|bi) of this pair is exactly zero
                const unsigned long long rem = alpha ^ (1ull << i) ^ (1ull << j);
                pair_prefix(occA, M, io, jo, bt, ks, pre);
                for (int q0 = 0; q0 < npv; q0 += 32) {
                    const int q = q0 + lane;
                    bool live = false;
                    unsigned long long h2 = 0ull;
                    unsigned first = 0u, ns = 0u;
                    double ev = 0.0;
                    if (q < npv) {
                        const int a = virA[pVA[2 * q]], b = virA[pVA[2 * q + 1]];
                        h2 = pair_rank(rem, a, b, M, pre, bt, ks);
                        if (h2 >= o.b.row_lo && h2 <= o.b.row_hi) {
                            if (!o.b.bk.rowmap) {
                                ns = 0xffffffffu, live = true;
                            } else {
                                const RowCtx rc = row_ctx(o.b, h2);
                                first = rc.first, ns = rc.ns;
                                live = ctx_in_pass(o.b, rc);
                            }
                            if (live) {
                                const int s1 = parity64(alpha & between_mask(i, a));
                                const unsigned long long s1s = alpha ^ (1ull << i) ^ (1ull << a);
                                const int s2 = parity64(s1s & between_mask(j, b));
                                const size_t x1 = (size_t(a * n + i) * n + b) * n + j;
                                const size_t x2 = (size_t(a * n + j) * n + b) * n + i;
                                const double gd = f32 ? (double)__fsub_rn(__ldg(&d.gf[x1]), __ldg(&d.gf[x2]))
                                                      : __dsub_rn(__ldg(&g[x1]), __ldg(&g[x2]));
                                ev = flip(gd, unsigned(s1 ^ s2));
                                live = nonzero(ev);
                            }
                        }
                    }
                    // the ring holds fewer than 32 / L + 1 <= 32 unfinished
                    // excitations here, so 32 more fit; the last round's reads
                    // are done before any lane overwrites an entry
                    const unsigned bal = __ballot_sync(kFull, live);
                    __syncwarp();
                    if (live) {
                        const int qi = (qhead + __popc(bal & lt)) & (kAaQ - 1);
                        qh[qi] = h2, qe[qi] = ev, qf[qi] = first, qn[qi] = ns;
                    }
                    qhead += __popc(bal);
                    __syncwarp();
                    while (qhead * (unsigned)L - cur >= 32u) round();
                }
                __syncwarp();
            }
            while (cur < qhead * (unsigned)L) round();
            __syncwarp();
        }
    }
    __syncwarp();
    ovf_pad(o.b, ocur[0], ocur[1]);
}

// weights[ha] += elements bound for row ha: the source's own row gets the
// diagonal, its beta singles and beta-beta doubles; each alpha single's row
// gets the single plus one element per beta hop; each alpha-alpha double's row
// gets one element.  One warp per input determinant (per run of determinants
// sharing alpha when nothing is screened).  *n_runs += the number of such runs.
__global__ void __launch_bounds__(kEmitThreads)
row_weight_kernel(const SysDev d, const unsigned long long *__restrict__ in_rank,
                  const double *__restrict__ in_coef, long long n_in, double eps,
                  unsigned long long *__restrict__ weights, unsigned long long *__restrict__ n_runs) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int n = d.n, ks = d.ks;
    unsigned long long *bt = reinterpret_cast<unsigned long long *>(sm);
    unsigned char *pairs = sm + align16(size_t(n + 1) * ks * 8);
    for (int i = threadIdx.x; i < (n + 1) * ks; i += blockDim.x) bt[i] = d.binom[i];
    for (int i = threadIdx.x; i < 2 * d.n_pairs; i += blockDim.x) pairs[i] = d.pairs[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wb = sm + block_smem(d) + size_t(warp) * warp_smem(d);
    unsigned long long *pre = reinterpret_cast<unsigned long long *>(wb);
    unsigned char *occA = reinterpret_cast<unsigned char *>(pre + 3 * ks);
    unsigned char *virA = occA + 64, *occB = occA + 128, *virB = occA + 192;
    const unsigned char *pOA = pairs + 2 * d.pair_off[0], *pVA = pairs + 2 * d.pair_off[1];
    const unsigned long long cb = d.cb;
    const unsigned long long w_self = 1ull + d.sb + (unsigned long long)d.po_b * d.pv_b;
    const unsigned long long w_single = 1ull + d.sb;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned char *pOB = pairs + 2 * d.pair_off[2];
    unsigned long long runs = 0;
    for (long long s = gw; s < n_in; s += nw) {
        const unsigned long long r = in_rank[s];
        const unsigned long long hA = r / cb;
        const bool run_start = s == 0 || in_rank[s - 1] / cb != hA;
        runs += run_start;
        unsigned long long mult = 1;
        if (!(eps > 0.0)) {
            // without the screen the weights depend on alpha only: the first
            // source of each run of consecutive sources sharing alpha (the
            // input is sorted by rank, alpha-major) adds them times the run length
            if (!run_start) continue;
            long long e = s + 1;
            for (;;) {
                const long long q = e + lane;
                const unsigned bal = __ballot_sync(kFull, q < n_in && in_rank[q] / cb == hA);
                if (bal != kFull) {
                    e += __ffs(~bal) - 1;
                    break;
                }
                e += 32;
            }
            mult = (unsigned long long)(e - s);
        }
        const unsigned long long alpha = string_unrank_warp(hA, n, d.na, bt, ks);
        const double ac = eps > 0.0 ? fabs(in_coef[s]) : 0.0;
        unsigned long long beta = 0;
        if (eps > 0.0) beta = string_unrank_warp(r - hA * cb, n, d.nb, bt, ks);
        build_lists(alpha, beta, n, occA, virA, occB, virB);
        __syncwarp();
        if (lane == 0) {
            unsigned long long w = w_self;
            if (eps > 0.0) {  // beta-beta pairs the screen removes
                w = 1ull + d.sb;
                for (int p = 0; p < d.po_b; ++p)
                    if (!(ac * __ldg(&d.bound_ss[occB[pOB[2 * p]] * n + occB[pOB[2 * p + 1]]]) < eps))
                        w += (unsigned long long)d.pv_b;
            }
            atomicAdd(&weights[hA], w * mult);
        }
        for (int x = lane; x < d.sa; x += 32) {
            const int io = x / d.va, iv = x - io * d.va;
            const bool hops = !(eps > 0.0 && ac * __ldg(&d.bound_ab[virA[iv] * n + occA[io]]) < eps);
            atomicAdd(&weights[string_rank(alpha ^ (1ull << occA[io]) ^ (1ull << virA[iv]), bt, ks)],
                      (hops ? w_single : 1ull) * mult);
        }
        for (int p = 0; p < d.po_a; ++p) {
            const int io = pOA[2 * p], jo = pOA[2 * p + 1];
            if (eps > 0.0 && ac * __ldg(&d.bound_ss[occA[io] * n + occA[jo]]) < eps) continue;
            const unsigned long long rem = alpha ^ (1ull << occA[io]) ^ (1ull << occA[jo]);
            pair_prefix(occA, d.na, io, jo, bt, ks, pre);
            for (int q = lane; q < d.pv_a; q += 32)
                atomicAdd(&weights[pair_rank(rem, virA[pVA[2 * q]], virA[pVA[2 * q + 1]], d.na, pre, bt, ks)], mult);
            __syncwarp();
        }
    }
    if (lane == 0 && runs) atomicAdd(n_runs, runs);
}

__global__ void rank_kernel(const SysDev d, const unsigned long long *a, const unsigned long long *b,
                            unsigned long long *r, long long count, int *status) {
    extern __shared__ unsigned long long bt_s[];
    for (int i = threadIdx.x; i < (d.n + 1) * d.ks; i += blockDim.x) bt_s[i] = d.binom[i];
    __syncthreads();
    const unsigned long long high = d.n >= 64 ? 0ull : ~((1ull << d.n) - 1ull);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        const unsigned long long x = a[k], y = b[k];
        if (__popcll(x) != d.na || __popcll(y) != d.nb || (x & high) || (y & high)) {
            r[k] = ~0ull;
            atomicOr(status, 1);
            continue;
        }
        r[k] = string_rank(x, bt_s, d.ks) * d.cb + string_rank(y, bt_s, d.ks);
    }
}

__device__ unsigned long long unrank_thread(unsigned long long r, int n, int m,
                                            const unsigned long long *bt, int ks) {
    unsigned long long s = 0;
    int top = n - 1;
    for (int i = m; i >= 1; --i) {
        int c = top;
        while (c > 0 && bt[c * ks + i] > r) --c;
        s |= 1ull << c;
        r -= bt[c * ks + i];
        top = c - 1;
    }
    return s;
}

__global__ void unrank_kernel(const SysDev d, const unsigned long long *r, unsigned long long *a,
                              unsigned long long *b, long long count, int *status) {
    extern __shared__ unsigned long long bt_s[];
    for (int i = threadIdx.x; i < (d.n + 1) * d.ks; i += blockDim.x) bt_s[i] = d.binom[i];
    __syncthreads();
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        const unsigned long long x = r[k];
        if (x >= d.dim) {
            a[k] = 0, b[k] = 0;
            atomicOr(status, 1);
            continue;
        }
        const unsigned long long ha = x / d.cb, hb = x - ha * d.cb;
        a[k] = unrank_thread(ha, d.n, d.na, bt_s, d.ks);
        b[k] = unrank_thread(hb, d.n, d.nb, bt_s, d.ks);
    }
}

int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// warps per CTA: the requested count (0: 8), lowered until the CTA's shared
// memory fits the device's per-block limit
int emit_warps_for(const SysDev &d, int want, bool narrow = false) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int w = want > 0 && want < kEmitWarps ? want : kEmitWarps;
    while (w > 1 && emit_smem_bytes_w(d, w, narrow) > (size_t)optin) --w;
    return emit_smem_bytes_w(d, w, narrow) <= (size_t)optin ? w : 0;
}

template <int kMode, bool kNarrow>
cudaError_t launch_emit_k(const SysDev &d, const unsigned long long *in_rank,
                          const double *in_coef, long long n_in, const EmitOut &o,
                          cudaStream_t st, int want_warps) {
    const int warps = emit_warps_for(d, want_warps, kNarrow);
    if (warps < 1) return cudaErrorInvalidConfiguration;  // one warp's tables exceed shared memory
    const size_t smem = emit_smem_bytes_w(d, warps, kNarrow);
    auto kern = emit_kernel<kMode, kNarrow>;
    cudaError_t e = allow_max_smem(kern, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long want = (n_in + warps - 1) / warps;
    long long grid = (long long)device_sms() * per_sm;
    if (want < grid) grid = want;
    count_launch();
    kern<<<(unsigned)grid, warps * 32, smem, st>>>(d, in_rank, in_coef, n_in, o);
    return cudaGetLastError();
}

// bucket mode takes the 32-bit single tables when every string index fits
template <int kMode>
cudaError_t launch_emit_impl(const SysDev &d, const unsigned long long *in_rank,
                             const double *in_coef, long long n_in, const EmitOut &o,
                             cudaStream_t st, int want_warps = 0) {
    if (n_in <= 0) return cudaSuccess;
    if constexpr (kMode == kModeBucket) {
        if (narrow_ranks(d)) return launch_emit_k<kMode, true>(d, in_rank, in_coef, n_in, o, st, want_warps);
    }
    return launch_emit_k<kMode, false>(d, in_rank, in_coef, n_in, o, st, want_warps);
}

}  // namespace

size_t emit_smem_bytes(const SysDev &d, int warps) { return emit_smem_bytes_w(d, warps); }

cudaError_t launch_emit(const SysDev &d, const unsigned long long *in_rank, const double *in_coef,
                        long long n_in, Table t, cudaStream_t st) {
    EmitOut o{};
    o.t = t;
    return launch_emit_impl<kModeTable>(d, in_rank, in_coef, n_in, o, st);
}

cudaError_t launch_emit_buckets(const SysDev &d, const unsigned long long *in_rank,
                                const double *in_coef, long long n_in, const BucketOut &b,
                                cudaStream_t st, int warps) {
    EmitOut o{};
    o.b = b;
    cudaError_t e = launch_emit_impl<kModeBucket>(d, in_rank, in_coef, n_in, o, st, warps);
    // (no launch when every same-spin double is exactly zero, e.g. an on-site
    // interaction only: the main kernel skipped them as well)
    if (e != cudaSuccess || !b.aa_runs || !d.ss_any || n_in <= 0 || d.po_a == 0 || d.pv_a == 0) return e;
    // alpha-alpha doubles, by runs of sources sharing alpha
    const size_t smem = block_smem(d) + size_t(kEmitWarps) * aa_warp_smem(d);
    e = allow_max_smem(emit_aa_kernel, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, emit_aa_kernel, kEmitThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // about eight work units per resident warp: windows, split into slices of
    // the occupied pairs when they are too few
    const long long windows = (n_in + 31) / 32;
    const long long slots = (long long)device_sms() * per_sm * kEmitWarps;
    const int groups = (int)std::min<long long>(d.po_a, std::max<long long>(1, (8 * slots + windows - 1) / windows));
    const long long units = windows * groups;
    long long grid = (long long)device_sms() * per_sm;
    if ((units + kEmitWarps - 1) / kEmitWarps < grid) grid = (units + kEmitWarps - 1) / kEmitWarps;
    count_launch();
    emit_aa_kernel<<<(unsigned)grid, kEmitThreads, smem, st>>>(d, in_rank, in_coef, n_in, groups, o);
    return cudaGetLastError();
}

cudaError_t launch_row_weights(const SysDev &d, const unsigned long long *in_rank,
                               const double *in_coef, long long n_in, double eps_elem,
                               unsigned long long *weights, unsigned long long *n_runs, cudaStream_t st) {
    if (n_in <= 0) return cudaSuccess;
    const size_t smem = emit_smem_bytes(d, kEmitWarps);
    cudaError_t e = allow_max_smem(row_weight_kernel, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, row_weight_kernel, kEmitThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long want = (n_in + kEmitWarps - 1) / kEmitWarps;
    long long grid = (long long)device_sms() * per_sm;
    if (want < grid) grid = want;
    count_launch();
    row_weight_kernel<<<(unsigned)grid, kEmitThreads, smem, st>>>(d, in_rank, in_coef, n_in, eps_elem, weights,
                                                                   n_runs);
    return cudaGetLastError();
}

cudaError_t launch_debug_excitations(const SysDev &d, const unsigned long long *in_rank,
                                     long long n_in, long long *src, unsigned long long *tgt,
                                     double *elem, cudaStream_t st) {
    EmitOut o{};
    o.dsrc = src, o.dtgt = tgt, o.delem = elem;
    return launch_emit_impl<kModeDebug>(d, in_rank, nullptr, n_in, o, st);
}

cudaError_t launch_rank(const SysDev &d, const unsigned long long *a, const unsigned long long *b,
                        unsigned long long *r, long long count, int *status, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    long long grid = (count + 255) / 256;
    if (grid > 4096) grid = 4096;
    count_launch();
    rank_kernel<<<(unsigned)grid, 256, size_t(d.n + 1) * d.ks * 8, st>>>(d, a, b, r, count, status);
    return cudaGetLastError();
}

cudaError_t launch_unrank(const SysDev &d, const unsigned long long *r, unsigned long long *a,
                          unsigned long long *b, long long count, int *status, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    long long grid = (count + 255) / 256;
    if (grid > 4096) grid = 4096;
    count_launch();
    unrank_kernel<<<(unsigned)grid, 256, size_t(d.n + 1) * d.ks * 8, st>>>(d, r, a, b, count, status);
    return cudaGetLastError();
}

}  // namespace sfci
