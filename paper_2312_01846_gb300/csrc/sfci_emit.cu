// sigma = H psi, step 1 (Sec. 2.2): every input entry (D, c_D) generates its
// intermediate elements (rank(D'), <D'|H|D> c_D) for D' = D and all single and
// double excitations of D (Sec. 3 / Sec. 4 "all single and double
// excitations"), and adds them straight into the merge table, so the
// intermediate elements never travel through HBM.
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
//   a6  element * c_D, exact zeros dropped, hash-added (sfci_internal.cuh).
// The lanes of the warp stride over the excitations of each class, so a warp
// issues 32 independent table adds at a time.
#include "sfci_internal.cuh"

namespace sfci {
namespace {

constexpr int kEmitThreads = 256;
constexpr int kEmitWarps = kEmitThreads / 32;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t block_smem(const SysDev &d) {
    return align16(size_t(d.n + 1) * d.ks * 8) + align16(size_t(d.n_pairs) * 2);
}

__host__ __device__ inline size_t warp_smem(const SysDev &d) {
    return align16(size_t(d.sa + d.sb) * 20 + 256);
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

template <bool kDebug>
__global__ void __launch_bounds__(kEmitThreads)
emit_kernel(const SysDev d, const unsigned long long *__restrict__ in_rank,
            const double *__restrict__ in_coef, long long n_in, Table t,
            long long *__restrict__ dsrc, unsigned long long *__restrict__ dtgt,
            double *__restrict__ delem) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int n = d.n, ks = d.ks;
    unsigned long long *bt = reinterpret_cast<unsigned long long *>(sm);
    unsigned char *pairs = sm + align16(size_t(n + 1) * ks * 8);
    for (int i = threadIdx.x; i < (n + 1) * ks; i += blockDim.x) bt[i] = d.binom[i];
    for (int i = threadIdx.x; i < 2 * d.n_pairs; i += blockDim.x) pairs[i] = d.pairs[i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wb = sm + block_smem(d) + size_t(warp) * warp_smem(d);
    unsigned long long *rankA1 = reinterpret_cast<unsigned long long *>(wb);
    double *elemA1 = reinterpret_cast<double *>(rankA1 + d.sa);
    unsigned long long *rankB1 = reinterpret_cast<unsigned long long *>(elemA1 + d.sa);
    double *elemB1 = reinterpret_cast<double *>(rankB1 + d.sb);
    unsigned *offA1 = reinterpret_cast<unsigned *>(elemB1 + d.sb);
    unsigned *offB1 = offA1 + d.sa;
    unsigned char *occA = reinterpret_cast<unsigned char *>(offB1 + d.sb);
    unsigned char *virA = occA + 64, *occB = occA + 128, *virB = occA + 192;
    const unsigned char *pOA = pairs + 2 * d.pair_off[0], *pVA = pairs + 2 * d.pair_off[1];
    const unsigned char *pOB = pairs + 2 * d.pair_off[2], *pVB = pairs + 2 * d.pair_off[3];
    const unsigned long long cb = d.cb;
    const double *__restrict__ g = d.g;
    const size_t n2 = size_t(n) * n;

    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned inserted = 0;
    const long long per = d.n_conn + 1;

    for (long long s = gw; s < n_in; s += nw) {
        const unsigned long long r = in_rank[s];
        const double c = kDebug ? 1.0 : in_coef[s];
        const unsigned long long hA = r / cb, hB = r - hA * cb;
        const unsigned long long alpha = string_unrank_warp(hA, n, d.na, bt, ks);
        const unsigned long long beta = string_unrank_warp(hB, n, d.nb, bt, ks);
        const long long base = s * per;

        build_lists(alpha, beta, n, occA, virA, occB, virB);
        __syncwarp();
        // single-excitation tables
        for (int x = lane; x < d.sa; x += 32) {
            const int io = x / d.va, iv = x - io * d.va;
            const int i = occA[io], a = virA[iv];
            const int sg = parity64(alpha & between_mask(i, a));
            rankA1[x] = string_rank(alpha ^ (1ull << i) ^ (1ull << a), bt, ks);
            const double F = single_element(d, i, a, occA, occB, occA, d.na);
            elemA1[x] = sg ? -F : F;
            offA1[x] = unsigned((a * n + i) * n2) | (unsigned(sg) << 31);
        }
        for (int y = lane; y < d.sb; y += 32) {
            const int jo = y / d.vb, jv = y - jo * d.vb;
            const int j = occB[jo], b = virB[jv];
            const int sg = parity64(beta & between_mask(j, b));
            rankB1[y] = string_rank(beta ^ (1ull << j) ^ (1ull << b), bt, ks);
            const double F = single_element(d, j, b, occA, occB, occB, d.nb);
            elemB1[y] = sg ? -F : F;
            offB1[y] = unsigned(b * n + j) | (unsigned(sg) << 31);
        }
        __syncwarp();

        // diagonal
        if (lane == 0) {
            const double e = diagonal_element(d, occA, occB);
            if (kDebug) {
                dsrc[base] = s, dtgt[base] = r, delem[base] = e;
            } else {
                const double v = __dmul_rn(e, c);
                if (v != 0.0) table_add(t, r, v, inserted);
            }
        }
        // singles
        long long off = base + 1;
        for (int x = lane; x < d.sa; x += 32) {
            const unsigned long long tg = rankA1[x] * cb + hB;
            if (kDebug) {
                dsrc[off + x] = s, dtgt[off + x] = tg, delem[off + x] = elemA1[x];
            } else {
                const double v = __dmul_rn(elemA1[x], c);
                if (v != 0.0) table_add(t, tg, v, inserted);
            }
        }
        off += d.sa;
        for (int y = lane; y < d.sb; y += 32) {
            const unsigned long long tg = hA * cb + rankB1[y];
            if (kDebug) {
                dsrc[off + y] = s, dtgt[off + y] = tg, delem[off + y] = elemB1[y];
            } else {
                const double v = __dmul_rn(elemB1[y], c);
                if (v != 0.0) table_add(t, tg, v, inserted);
            }
        }
        off += d.sb;
        // same-spin doubles: (i<j) -> (a<b), i->a then j->b
        for (int spin = 0; spin < 2; ++spin) {
            const unsigned long long str = spin ? beta : alpha;
            const unsigned char *occ = spin ? occB : occA, *vir = spin ? virB : virA;
            const unsigned char *po = spin ? pOB : pOA, *pv = spin ? pVB : pVA;
            const int npo = spin ? d.po_b : d.po_a, npv = spin ? d.pv_b : d.pv_a;
            for (int p = 0; p < npo; ++p) {
                const int i = occ[po[2 * p]], j = occ[po[2 * p + 1]];
                for (int q = lane; q < npv; q += 32) {
                    const int a = vir[pv[2 * q]], b = vir[pv[2 * q + 1]];
                    const int s1 = parity64(str & between_mask(i, a));
                    const unsigned long long s1s = str ^ (1ull << i) ^ (1ull << a);
                    const int s2 = parity64(s1s & between_mask(j, b));
                    const unsigned long long s2s = s1s ^ (1ull << j) ^ (1ull << b);
                    double e = __dsub_rn(__ldg(&g[(size_t(a * n + i) * n + b) * n + j]),
                                         __ldg(&g[(size_t(a * n + j) * n + b) * n + i]));
                    if (s1 ^ s2) e = -e;
                    const unsigned long long h2 = string_rank(s2s, bt, ks);
                    const unsigned long long tg = spin ? hA * cb + h2 : h2 * cb + hB;
                    if (kDebug) {
                        const long long o = off + (long long)p * npv + q;
                        dsrc[o] = s, dtgt[o] = tg, delem[o] = e;
                    } else {
                        const double v = __dmul_rn(e, c);
                        if (v != 0.0) table_add(t, tg, v, inserted);
                    }
                }
            }
            off += (long long)npo * npv;
        }
        // opposite-spin doubles: alpha hop x, beta hop y
        for (int x = 0; x < d.sa; ++x) {
            const unsigned long long ra = rankA1[x] * cb;
            const unsigned oa = offA1[x];
            const double *gx = g + (oa & 0x7fffffffu);
            const unsigned sa = oa >> 31;
            for (int y = lane; y < d.sb; y += 32) {
                const unsigned ob = offB1[y];
                double e = __ldg(&gx[ob & 0x7fffffffu]);
                if (sa ^ (ob >> 31)) e = -e;
                const unsigned long long tg = ra + rankB1[y];
                if (kDebug) {
                    const long long o = off + (long long)x * d.sb + y;
                    dsrc[o] = s, dtgt[o] = tg, delem[o] = e;
                } else {
                    const double v = __dmul_rn(e, c);
                    if (v != 0.0) table_add(t, tg, v, inserted);
                }
            }
        }
        __syncwarp();
    }
    if (!kDebug) {
        for (int o = 16; o > 0; o >>= 1) inserted += __shfl_xor_sync(kFull, inserted, o);
        if (lane == 0 && inserted) atomicAdd(t.count, (unsigned long long)inserted);
    }
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

template <bool kDebug>
cudaError_t launch_emit_impl(const SysDev &d, const unsigned long long *in_rank,
                             const double *in_coef, long long n_in, Table t, long long *src,
                             unsigned long long *tgt, double *elem, cudaStream_t st) {
    if (n_in <= 0) return cudaSuccess;
    const size_t smem = emit_smem_bytes(d, kEmitWarps);
    auto kern = emit_kernel<kDebug>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kEmitThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long want = (n_in + kEmitWarps - 1) / kEmitWarps;
    long long grid = (long long)device_sms() * per_sm;
    if (want < grid) grid = want;
    count_launch();
    kern<<<(unsigned)grid, kEmitThreads, smem, st>>>(d, in_rank, in_coef, n_in, t, src, tgt, elem);
    return cudaGetLastError();
}

}  // namespace

size_t emit_smem_bytes(const SysDev &d, int warps) {
    return block_smem(d) + size_t(warps) * warp_smem(d);
}

cudaError_t launch_emit(const SysDev &d, const unsigned long long *in_rank, const double *in_coef,
                        long long n_in, Table t, cudaStream_t st) {
    return launch_emit_impl<false>(d, in_rank, in_coef, n_in, t, nullptr, nullptr, nullptr, st);
}

cudaError_t launch_debug_excitations(const SysDev &d, const unsigned long long *in_rank,
                                     long long n_in, long long *src, unsigned long long *tgt,
                                     double *elem, cudaStream_t st) {
    Table t{};
    return launch_emit_impl<true>(d, in_rank, nullptr, n_in, t, src, tgt, elem, st);
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
