// One- and two-particle density matrices of a sparse vector, produced by the
// same excitation generator as sigma (sfci_emit.cu): for every determinant D of
// psi and every D' in {D} and the single and double excitations of D, the
// coefficient c_D' is looked up in a hash table built from psi; each hit adds
// c_D' c_D <D'| a+_p a+_r a_s a_q |D> into the spin-summed
//   gamma[p,q]      = sum_s   <psi| a+_ps a_qs |psi>
//   Gamma[p,q,r,s]  = sum_st  <psi| a+_ps a+_rt a_st a_qs |psi>
// (not normalised).  The operator strings that connect D to D' are:
//   D' = D:        n_ps n_rt for distinct spin orbitals (p,s) != (r,t), minus the
//                  exchange n_ps n_rs (same spin) on Gamma[p,r,r,p];
//   single i->a:   gamma[a,i]; Gamma[a,i,k,k], Gamma[k,k,a,i] for every other
//                  occupied k, minus Gamma[a,k,k,i], Gamma[k,i,a,k] for k of the
//                  hop's spin;
//   double:        Gamma[a,i,b,j] + Gamma[b,j,a,i], and for same spin
//                  - Gamma[a,j,b,i] - Gamma[b,i,a,j]
// with the sign of the excitation (hop 1 then hop 2, as in sigma).  These give
// E = e_core <psi|psi> + sum h gamma + 1/2 sum (pq|rs) Gamma = <psi|H|psi>,
// so dE/dh = gamma / <psi|psi> and dE/d(pq|rs) = Gamma / (2 <psi|psi>) for a
// fixed psi.
#include "sfci_internal.cuh"

namespace sfci {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t rdm_block_smem(const SysDev &d) {
    return al16(size_t(d.n + 1) * d.ks * 8) + al16(size_t(d.n_pairs) * 2);
}

__host__ __device__ inline size_t rdm_warp_smem(const SysDev &d) {
    return al16(size_t(d.sa + d.sb) * 12 + 256);
}

__device__ __forceinline__ void acc(double *a, size_t i, double v) { atomicAdd(a + i, v); }

__global__ void __launch_bounds__(kThreads)
rdm_kernel(const SysDev d, const unsigned long long *__restrict__ rank,
           const double *__restrict__ coef, long long m, Table psi, double *__restrict__ g1,
           double *__restrict__ g2) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int n = d.n, ks = d.ks;
    unsigned long long *bt = reinterpret_cast<unsigned long long *>(sm);
    unsigned char *pairs = sm + al16(size_t(n + 1) * ks * 8);
    for (int i = threadIdx.x; i < (n + 1) * ks; i += blockDim.x) bt[i] = d.binom[i];
    for (int i = threadIdx.x; i < 2 * d.n_pairs; i += blockDim.x) pairs[i] = d.pairs[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wb = sm + rdm_block_smem(d) + size_t(warp) * rdm_warp_smem(d);
    unsigned long long *rankA1 = reinterpret_cast<unsigned long long *>(wb);
    unsigned long long *rankB1 = rankA1 + d.sa;
    unsigned *hopA = reinterpret_cast<unsigned *>(rankB1 + d.sb);  // i | a << 8 | sign << 16
    unsigned *hopB = hopA + d.sa;
    unsigned char *occA = reinterpret_cast<unsigned char *>(hopB + d.sb);
    unsigned char *virA = occA + 64, *occB = occA + 128, *virB = occA + 192;
    const unsigned char *pOA = pairs + 2 * d.pair_off[0], *pVA = pairs + 2 * d.pair_off[1];
    const unsigned char *pOB = pairs + 2 * d.pair_off[2], *pVB = pairs + 2 * d.pair_off[3];
    const unsigned long long cb = d.cb;
    const size_t N1 = size_t(n), N2 = N1 * n, N3 = N2 * n;
#define G2(p, q, r, s) (size_t(p) * N3 + size_t(q) * N2 + size_t(r) * N1 + size_t(s))

    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long s = gw; s < m; s += nw) {
        const unsigned long long r = rank[s];
        const double c = coef[s];
        const unsigned long long hA = r / cb, hB = r - hA * cb;
        const unsigned long long alpha = string_unrank_warp(hA, n, d.na, bt, ks);
        const unsigned long long beta = string_unrank_warp(hB, n, d.nb, bt, ks);
        build_lists(alpha, beta, n, occA, virA, occB, virB);
        __syncwarp();
        for (int x = lane; x < d.sa; x += 32) {
            const int io = x / d.va, iv = x - io * d.va;
            const int i = occA[io], a = virA[iv];
            rankA1[x] = string_rank(alpha ^ (1ull << i) ^ (1ull << a), bt, ks);
            hopA[x] = unsigned(i) | (unsigned(a) << 8) | (unsigned(parity64(alpha & between_mask(i, a))) << 16);
        }
        for (int y = lane; y < d.sb; y += 32) {
            const int jo = y / d.vb, jv = y - jo * d.vb;
            const int j = occB[jo], b = virB[jv];
            rankB1[y] = string_rank(beta ^ (1ull << j) ^ (1ull << b), bt, ks);
            hopB[y] = unsigned(j) | (unsigned(b) << 8) | (unsigned(parity64(beta & between_mask(j, b))) << 16);
        }
        __syncwarp();
        if (c == 0.0) continue;
        // D' = D
        {
            const double v = c * c;
            const int NE = d.na + d.nb;
            for (int k = lane; k < NE; k += 32) {
                const int p = k < d.na ? occA[k] : occB[k - d.na];
                acc(g1, size_t(p) * n + p, v);
            }
            for (int e = lane; e < NE * NE; e += 32) {
                const int k = e / NE, l = e - k * NE;
                if (k == l) continue;
                const int p = k < d.na ? occA[k] : occB[k - d.na];
                const int q = l < d.na ? occA[l] : occB[l - d.na];
                acc(g2, G2(p, p, q, q), v);
                if ((k < d.na) == (l < d.na)) acc(g2, G2(p, q, q, p), -v);
            }
        }
        // singles
        for (int spin = 0; spin < 2; ++spin) {
            const int ns = spin ? d.sb : d.sa;
            const unsigned long long *rk = spin ? rankB1 : rankA1;
            const unsigned *hop = spin ? hopB : hopA;
            const unsigned char *same = spin ? occB : occA, *other = spin ? occA : occB;
            const int nsame = spin ? d.nb : d.na, nother = spin ? d.na : d.nb;
            for (int x = lane; x < ns; x += 32) {
                const unsigned long long tg = spin ? hA * cb + rk[x] : rk[x] * cb + hB;
                const long long f = table_find(psi, tg);
                if (f < 0) continue;
                const unsigned hp = hop[x];
                const int i = hp & 0xff, a = (hp >> 8) & 0xff;
                double v = __ldcg(&psi.slots[f].val) * c;
                if (hp >> 16) v = -v;
                acc(g1, size_t(a) * n + i, v);
                for (int q = 0; q < nsame; ++q) {
                    const int k = same[q];
                    if (k == i) continue;
                    acc(g2, G2(a, i, k, k), v);
                    acc(g2, G2(k, k, a, i), v);
                    acc(g2, G2(a, k, k, i), -v);
                    acc(g2, G2(k, i, a, k), -v);
                }
                for (int q = 0; q < nother; ++q) {
                    const int k = other[q];
                    acc(g2, G2(a, i, k, k), v);
                    acc(g2, G2(k, k, a, i), v);
                }
            }
        }
        // same-spin doubles
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
                    const unsigned long long h2 = string_rank(s1s ^ (1ull << j) ^ (1ull << b), bt, ks);
                    const unsigned long long tg = spin ? hA * cb + h2 : h2 * cb + hB;
                    const long long f = table_find(psi, tg);
                    if (f < 0) continue;
                    double v = __ldcg(&psi.slots[f].val) * c;
                    if (s1 ^ s2) v = -v;
                    acc(g2, G2(a, i, b, j), v);
                    acc(g2, G2(b, j, a, i), v);
                    acc(g2, G2(a, j, b, i), -v);
                    acc(g2, G2(b, i, a, j), -v);
                }
            }
        }
        // opposite-spin doubles
        for (int x = 0; x < d.sa; ++x) {
            const unsigned long long ra = rankA1[x] * cb;
            const unsigned ha = hopA[x];
            const int i = ha & 0xff, a = (ha >> 8) & 0xff;
            for (int y = lane; y < d.sb; y += 32) {
                const long long f = table_find(psi, ra + rankB1[y]);
                if (f < 0) continue;
                const unsigned hb = hopB[y];
                const int j = hb & 0xff, b = (hb >> 8) & 0xff;
                double v = __ldcg(&psi.slots[f].val) * c;
                if ((ha >> 16) ^ (hb >> 16)) v = -v;
                acc(g2, G2(a, i, b, j), v);
                acc(g2, G2(b, j, a, i), v);
            }
        }
        __syncwarp();
    }
#undef G2
}

__global__ void norm2_kernel(const double *c, long long m, double *partial) {
    __shared__ double sh[kWarps];
    double a = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x)
        a = __fma_rn(c[i], c[i], a);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += sh[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void norm2_finish(const double *partial, int np, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < np; ++k) t += partial[k];
        *out = t;
    }
}

constexpr int kNormBlocks = 152;

// partial[b] = sum over block b's share of k of x[k] y[k] (x, y of length m),
// fixed grid and order; two launches (h.gamma, then g.Gamma) write disjoint halves
__global__ void contract_kernel(const double *x, const double *y, long long m, double *partial) {
    __shared__ double sh[kWarps];
    double a = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x)
        a = __fma_rn(x[i], y[i], a);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += sh[w];
        partial[blockIdx.x] = t;
    }
}

// E = e_core + (sum h gamma + 1/2 sum g Gamma) / norm2 from the two halves of partial
__global__ void energy_finish(const double *partial, int np, double e_core, double norm2, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double one = 0.0, two = 0.0;
        for (int k = 0; k < np; ++k) one += partial[k];
        for (int k = 0; k < np; ++k) two += partial[np + k];
        out[0] = e_core + (one + 0.5 * two) / norm2;
        out[1] = one;
        out[2] = two;
    }
}

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

unsigned long long rdm_slots(long long m) {
    unsigned long long want = 2ull * (unsigned long long)(m > 0 ? m : 1), p = 1024;
    while (p < want) p <<= 1;
    return p;
}

struct RdmLayout {
    unsigned long long slots;
    size_t table, status, count, partial, norm, bytes;
};

RdmLayout rdm_layout(long long m) {
    RdmLayout L{};
    L.slots = rdm_slots(m);
    size_t o = 0;
    L.table = o, o = a256(o + L.slots * sizeof(Slot));
    L.status = o, o = a256(o + sizeof(int));
    L.count = o, o = a256(o + 8);
    L.partial = o, o = a256(o + 8 * kNormBlocks);
    L.norm = o, o = a256(o + 8);
    L.bytes = o;
    return L;
}

int sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace
}  // namespace sfci

using namespace sfci;

extern "C" {

sfci_status sfci_rdm12_workspace_bytes(const sfci_system *s, int64_t n, size_t *bytes) {
    if (!s || !bytes || n < 0) {
        set_error("bad arguments");
        return SFCI_E_INVALID;
    }
    *bytes = rdm_layout(n).bytes;
    return SFCI_OK;
}

sfci_status sfci_rdm12(const sfci_system *s, const uint64_t *rank, const double *coef, int64_t n,
                       double *rdm1, double *rdm2, double *norm2, void *workspace,
                       size_t ws_bytes, void *stream) {
    if (!s || n < 0 || !rdm1 || !rdm2 || (n > 0 && (!rank || !coef))) {
        set_error("bad arguments");
        return SFCI_E_INVALID;
    }
    const RdmLayout L = rdm_layout(n);
    if (!workspace || ws_bytes < L.bytes) {
        set_error("workspace smaller than sfci_rdm12_workspace_bytes");
        return SFCI_E_CAPACITY;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const SysDev &d = s->d;
    const size_t n2 = size_t(d.n) * d.n;
    char *w = static_cast<char *>(workspace);
    SFCI_CUDA(cudaMemsetAsync(rdm1, 0, n2 * 8, st));
    SFCI_CUDA(cudaMemsetAsync(rdm2, 0, n2 * n2 * 8, st));
    Table t;
    t.slots = reinterpret_cast<Slot *>(w + L.table);
    t.mask = L.slots - 1;
    t.shift = 64 - __builtin_ctzll(L.slots);
    t.status = reinterpret_cast<int *>(w + L.status);
    t.count = reinterpret_cast<unsigned long long *>(w + L.count);
    const unsigned long long *r = reinterpret_cast<const unsigned long long *>(rank);
    int *flag = s->dev_status;
    SFCI_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    SFCI_CUDA(validate_sorted(r, n, d.dim, flag, st));
    SFCI_CUDA(table_clear(t, st));
    SFCI_CUDA(table_axpy(t, r, coef, n, nullptr, 1.0, 1.0, st));
    double *partial = reinterpret_cast<double *>(w + L.partial);
    double *nrm = reinterpret_cast<double *>(w + L.norm);
    count_launch();
    norm2_kernel<<<kNormBlocks, kThreads, 0, st>>>(coef, n, partial);
    count_launch();
    norm2_finish<<<1, 32, 0, st>>>(partial, kNormBlocks, nrm);
    if (n > 0) {
        const size_t smem = rdm_block_smem(d) + kWarps * rdm_warp_smem(d);
        SFCI_CUDA(allow_max_smem(rdm_kernel, smem));
        int per_sm = 0;
        SFCI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rdm_kernel, kThreads, smem));
        if (per_sm < 1) {
            set_error("rdm kernel does not fit on an SM for this system");
            return SFCI_E_CAPACITY;
        }
        long long grid = (long long)sms() * per_sm, want = (n + kWarps - 1) / kWarps;
        if (want < grid) grid = want;
        count_launch();
        rdm_kernel<<<(unsigned)grid, kThreads, smem, st>>>(d, r, coef, n, t, rdm1, rdm2);
        SFCI_CUDA(cudaGetLastError());
    }
    int hflag = 0;
    double hn = 0.0;
    SFCI_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaMemcpyAsync(&hn, nrm, 8, cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaStreamSynchronize(st));
    if (hflag) {
        set_error("input ranks must be strictly ascending and below dim");
        return SFCI_E_INVALID;
    }
    if (norm2) *norm2 = hn;
    return SFCI_OK;
}

sfci_status sfci_rdm_energy(int n_orb, const double *rdm1, const double *rdm2, double norm2,
                            const double *h, const double *g, double e_core, double *energy,
                            void *workspace, size_t ws_bytes, void *stream) {
    if (n_orb < 1 || n_orb > 64 || !rdm1 || !rdm2 || !h || !g || !energy || !(norm2 > 0.0)) {
        set_error("need 1 <= n_orb <= 64, device rdm1, rdm2, h, g, a host energy and norm2 > 0");
        return SFCI_E_INVALID;
    }
    if (!workspace || ws_bytes < size_t(2 * kNormBlocks + 3) * 8) {
        set_error("workspace below sfci_rdm_energy's 2456 bytes");
        return SFCI_E_CAPACITY;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *partial = static_cast<double *>(workspace);
    double *out = partial + 2 * kNormBlocks;
    const long long n2 = (long long)n_orb * n_orb;
    count_launch();
    contract_kernel<<<kNormBlocks, kThreads, 0, st>>>(h, rdm1, n2, partial);
    count_launch();
    contract_kernel<<<kNormBlocks, kThreads, 0, st>>>(g, rdm2, n2 * n2, partial + kNormBlocks);
    count_launch();
    energy_finish<<<1, 32, 0, st>>>(partial, kNormBlocks, e_core, norm2, out);
    SFCI_CUDA(cudaGetLastError());
    SFCI_CUDA(cudaMemcpyAsync(energy, out, 8, cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaStreamSynchronize(st));
    return SFCI_OK;
}

}  // extern "C"
