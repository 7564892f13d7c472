// The SFCI iterative solver of Sec. 2.1 on one GPU.
//
// Per step (one sigma application, one of the paper's N_I iterations):
//   sigma_i = H w_i into the merge table (sfci_emit.cu), screened (Sec. 3);
//   T_ji = <w_j|sigma_i> by table lookups, S_ji = <w_j|w_i> by binary search,
//   j <= i (the truncated w's are not orthogonal, so T is full and the
//   problem is T x = lambda S x);
//   u = sigma_i - a_i w_i - b_i w_{i-1} as two more rounds of adds into the same
//   table (Eq. 10), then w_{i+1} = top_{N_d}(u), normalised (Eq. 11);
//   at the last vector of a cycle: the lowest root of T x = lambda S x on the
//   host (N_L x N_L, FP64, canonical orthogonalisation + cyclic Jacobi),
//   Psi = sum_j x_j w_j accumulated in the table in ascending j, and the
//   restart vector w_0 = top_{N_d}(Psi), normalised; the halting test
//   compares successive lambda_min.
// The host sees only O(N_L) scalars per step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sfci_internal.cuh"

namespace sfci {
namespace {

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

unsigned long long next_pow2(unsigned long long x) {
    unsigned long long p = 1;
    while (p < x) p <<= 1;
    return p;
}

int key_bits(unsigned long long dim) {
    if (dim <= 1) return 8;
    return 64 - __builtin_clzll(dim - 1);
}

// Cyclic Jacobi for a symmetric n x n matrix (row-major).  Eigenvalues
// ascending in w, eigenvectors in the columns of V.
void jacobi_eigh(int n, std::vector<double> A, std::vector<double> &w, std::vector<double> &V) {
    V.assign(size_t(n) * n, 0.0);
    for (int i = 0; i < n; ++i) V[size_t(i) * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                const double a = A[size_t(p) * n + q];
                tot += a * a;
                if (p != q) off += a * a;
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[size_t(p) * n + q];
                if (apq == 0.0) continue;
                const double app = A[size_t(p) * n + p], aqq = A[size_t(q) * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = A[size_t(k) * n + p], akq = A[size_t(k) * n + q];
                    A[size_t(k) * n + p] = c * akp - s * akq;
                    A[size_t(k) * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = A[size_t(p) * n + k], aqk = A[size_t(q) * n + k];
                    A[size_t(p) * n + k] = c * apk - s * aqk;
                    A[size_t(q) * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[size_t(k) * n + p], vkq = V[size_t(k) * n + q];
                    V[size_t(k) * n + p] = c * vkp - s * vkq;
                    V[size_t(k) * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(),
              [&](int x, int y) { return A[size_t(x) * n + x] < A[size_t(y) * n + y]; });
    w.resize(n);
    std::vector<double> V2(size_t(n) * n);
    for (int j = 0; j < n; ++j) {
        w[j] = A[size_t(idx[j]) * n + idx[j]];
        for (int k = 0; k < n; ++k) V2[size_t(k) * n + j] = V[size_t(k) * n + idx[j]];
    }
    V.swap(V2);
}

// Lowest root of T x = lambda S x: eigendecompose S, drop eigenvalues below
// 1e-12 * max, solve the projected standard problem.
double gen_eig_lowest(int m, const std::vector<double> &T, const std::vector<double> &S,
                      std::vector<double> &x) {
    std::vector<double> s, U;
    jacobi_eigh(m, S, s, U);
    const double smax = s[m - 1];
    std::vector<int> keep;
    for (int k = 0; k < m; ++k)
        if (s[k] > 1e-12 * smax) keep.push_back(k);
    const int r = (int)keep.size();
    std::vector<double> X(size_t(m) * r);
    for (int c = 0; c < r; ++c) {
        const double f = 1.0 / std::sqrt(s[keep[c]]);
        for (int k = 0; k < m; ++k) X[size_t(k) * r + c] = U[size_t(k) * m + keep[c]] * f;
    }
    std::vector<double> TX(size_t(m) * r, 0.0), Tp(size_t(r) * r, 0.0);
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < r; ++c) {
            double acc = 0.0;
            for (int b = 0; b < m; ++b) acc += T[size_t(a) * m + b] * X[size_t(b) * r + c];
            TX[size_t(a) * r + c] = acc;
        }
    for (int c1 = 0; c1 < r; ++c1)
        for (int c2 = 0; c2 < r; ++c2) {
            double acc = 0.0;
            for (int a = 0; a < m; ++a) acc += X[size_t(a) * r + c1] * TX[size_t(a) * r + c2];
            Tp[size_t(c1) * r + c2] = acc;
        }
    for (int c1 = 0; c1 < r; ++c1)
        for (int c2 = c1 + 1; c2 < r; ++c2) {
            const double avg = 0.5 * (Tp[size_t(c1) * r + c2] + Tp[size_t(c2) * r + c1]);
            Tp[size_t(c1) * r + c2] = Tp[size_t(c2) * r + c1] = avg;
        }
    std::vector<double> lam, Y;
    jacobi_eigh(r, Tp, lam, Y);
    x.assign(m, 0.0);
    for (int a = 0; a < m; ++a) {
        double acc = 0.0;
        for (int c = 0; c < r; ++c) acc += X[size_t(a) * r + c] * Y[size_t(c) * r + 0];
        x[a] = acc;
    }
    return lam[0];
}

// NVTX range for the lifetime of a scope (a no-op unless a profiler attaches)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// One JSON line per step appended to the file named by SFCI_STEP_LOG (when set):
// the step's scalars, stage times and the sigma stage's rate.
std::mutex g_log_mu;

void log_step(const sfci_step_info &s) {
    const char *path = std::getenv("SFCI_STEP_LOG");
    if (!path || !*path) return;
    std::lock_guard<std::mutex> lk(g_log_mu);
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    const double gbs = s.ms_sigma > 0.0 ? 32.0 * (double)s.n_elements / (s.ms_sigma * 1e-3) / 1e9 : 0.0;
    std::fprintf(f,
                 "{\"iter\": %d, \"cycle\": %d, \"index\": %d, \"cycle_end\": %d, \"converged\": %d, "
                 "\"breakdown\": %d, \"lambda_min\": %.17g, \"a\": %.17g, \"b\": %.17g, \"u_norm\": %.17g, "
                 "\"n_in\": %lld, \"n_sigma\": %lld, \"n_kept\": %lld, \"n_elements\": %lld, "
                 "\"n_emitted\": %lld, \"n_psi\": %lld, \"ms_step\": %.4f, \"ms_sigma\": %.4f, "
                 "\"ms_emit\": %.4f, \"ms_merge\": %.4f, \"ms_plan\": %.4f, \"ms_topk\": %.4f, "
                 "\"n_passes\": %d, \"redo\": %d, \"bucket_redo\": %d, \"n_overflow\": %lld, "
                 "\"n_alpha_runs\": %lld, \"sigma_gbs_32B_per_element\": %.3f}\n",
                 s.iter, s.cycle, s.index, s.cycle_end, s.converged, s.breakdown, s.lambda_min, s.a, s.b,
                 s.u_norm, (long long)s.n_in, (long long)s.n_sigma, (long long)s.n_kept,
                 (long long)s.n_elements, (long long)s.n_emitted, (long long)s.n_psi, s.ms_step, s.ms_sigma,
                 s.ms_emit, s.ms_merge, s.ms_plan, s.ms_topk, s.n_passes, s.redo, s.bucket_redo,
                 (long long)s.n_overflow, (long long)s.n_alpha_runs, gbs);
    std::fclose(f);
}

}  // namespace
}  // namespace sfci

using namespace sfci;

struct sfci_lanczos {
    const sfci_system *sys = nullptr;
    sfci_params p{};
    cudaStream_t st = nullptr;
    int NL = 0;
    long long nkeep = 0;
    std::vector<unsigned long long *> wr;
    std::vector<double *> wc;
    std::vector<long long> wn;
    // merge table
    Slot *slots = nullptr;
    unsigned long long phys = 0;  // allocated slots
    unsigned long long budget = 0;  // max slots device memory allows
    // scratch
    char *scratch = nullptr;
    size_t off_sel = 0, off_sort = 0, off_norm = 0, off_dots = 0, off_small = 0;
    size_t sel_bytes = 0;
    // small device words
    int *tstatus = nullptr;
    unsigned long long *tcount = nullptr, *ndev = nullptr, *total = nullptr, *screened = nullptr;
    double *dT = nullptr, *dS = nullptr, *sumsq = nullptr;
    // host state
    std::vector<double> T, S;
    int idx = 0, cycle = 0, iter = 0;
    bool have_prev = false;
    double e_prev = 0.0;
    long long m_prev = 0, nin_prev = 0;
    long long ovf_used = 0;  // most overflow elements of a pass in the last sigma
    double elem_prev = 0.0;  // intermediate elements of the last sigma
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t evp[4] = {nullptr, nullptr, nullptr, nullptr};  // emit / merge timing
    // bucketed sigma (sfci_merge.cu); every buffer with its allocated bytes
    struct Buf {
        void *p = nullptr;
        size_t bytes = 0;
    };
    Buf bcount, belem, bovf, bovf_sorted, tmp_counts, ovf_off, probes, pcount, poff, scan_ws,
        sig_key, sig_val, cand_key, cand_val, weights, rowmap, boff,
        wpre, ptl, pth, pbstart, pcap, pq,  // device bucket plan (row mode)
        start4;                             // region offsets of the current pass
    long long sig_cap = 0, ovf_cap = 0, cand_cap = 0;
    double *sigw[kMaxVec] = {};
    char *words = nullptr;  // hist[kHistBins] | outn | mlive | ovf_n | cand_n | msumsq | queue | mstatus | nnz | dmin | tau | mark | lock
    unsigned long long *hist = nullptr, *outn = nullptr, *mlive = nullptr, *ovf_n = nullptr,
                       *cand_n = nullptr;
    double *msumsq = nullptr;
    unsigned *queue = nullptr;
    int *mstatus = nullptr;
    double ms_emit = 0, ms_merge = 0, ms_plan = 0, budget_gb = 0, regions_gb = 0, free_gb = 0, held_gb = 0,
           ms_alloc = 0;
    double tau_prev = 0.0;             // previous truncation cut in u (0: none)
    std::vector<double> cut_at;        // truncation cut at each basis index of the last cycle
    std::vector<long long> ovf_at;     // most overflow of a pass at each basis index of the last cycle
    int n_split = 0;                   // pass ranges split because their overflow outgrew the list
    double mult_prev = 0.0;            // elements per distinct sigma entry in the last sigma
    bool small_buckets = false;        // this sigma is being redone with 1024-element buckets
    double big_thresh = 1.5;           // mult_prev from which automatic mode tries 2048-element
                                       // buckets; raised above the level at which a try failed
    int bucket_redo = 0;               // sigmas of this step redone with 1024-element buckets
    std::vector<double> T_last, S_last;  // T and S solved at the last cycle end
    bool just_ended = false;           // the last step ended a cycle
    unsigned long long stream_prev = 0;  // entries streamed by the previous merge
    unsigned long long *nnz = nullptr;  // device word: non-zero entries off w_i, w_{i-1}
    unsigned long long *tau_w = nullptr, *mark_w = nullptr;  // stream threshold bits, raise mark
    int *lock_w = nullptr;
    unsigned long long *nread_w = nullptr;  // device word: intermediate elements merged
    long long n_emitted = 0;            // of the last sigma (host copy)
    unsigned long long alpha_runs = 0;  // runs of inputs sharing alpha (last sigma's plan)
    double *dmin = nullptr;             // device word: min |kept|
    int n_passes = 0, nb_log2 = 0;
};

namespace {

void destroy_lz(sfci_lanczos *z) {
    if (!z) return;
    for (auto p : z->wr) cudaFree(p);
    for (auto p : z->wc) cudaFree(p);
    cudaFree(z->slots);
    cudaFree(z->scratch);
    for (auto *b : {&z->bcount, &z->belem, &z->bovf, &z->bovf_sorted, &z->tmp_counts, &z->ovf_off,
                    &z->probes, &z->pcount, &z->poff, &z->scan_ws, &z->sig_key, &z->sig_val,
                    &z->cand_key, &z->cand_val, &z->weights, &z->rowmap, &z->boff, &z->wpre, &z->ptl,
                    &z->pth, &z->pbstart, &z->pcap, &z->pq, &z->start4})
        cudaFree(b->p);
    cudaFree(z->words);
    for (int j = 0; j < kMaxVec; ++j) cudaFree(z->sigw[j]);
    for (auto &e : z->ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : z->evp)
        if (e) cudaEventDestroy(e);
    delete z;
}

Table make_table(sfci_lanczos *z, unsigned long long cap) {
    Table t;
    t.slots = z->slots;
    t.mask = cap - 1;
    t.shift = 64 - __builtin_ctzll(cap);
    t.status = z->tstatus;
    t.count = z->tcount;
    return t;
}

sfci_status ensure_slots(sfci_lanczos *z, unsigned long long cap) {
    if (cap <= z->phys) return SFCI_OK;
    if (cap > z->budget) {
        set_error("sigma's merge table needs more device memory than is free");
        return SFCI_E_CAPACITY;
    }
    SFCI_CUDA(cudaStreamSynchronize(z->st));
    cudaFree(z->slots);
    z->slots = nullptr;
    z->phys = 0;
    cudaError_t e = cudaMalloc(&z->slots, cap * sizeof(Slot));
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc merge table: ") + cudaGetErrorString(e));
        return SFCI_E_NOMEM;
    }
    z->phys = cap;
    return SFCI_OK;
}

// top-k of the table into W[dst] (sorted by rank, normalised); host count
sfci_status table_topk(sfci_lanczos *z, unsigned long long cap, int dst, double *sumsq_host,
                       unsigned long long *total_host) {
    Items it{&z->slots[0].key, &z->slots[0].val, 2, (long long)cap};
    SFCI_CUDA(select_topk(it, z->nkeep, z->wr[dst], z->wc[dst], z->ndev, z->sumsq, z->total,
                          z->scratch + z->off_sel, z->sel_bytes, z->st));
    SFCI_CUDA(sort_pairs(z->wr[dst], z->wc[dst], z->nkeep, z->ndev, key_bits(z->sys->d.dim),
                         z->scratch + z->off_sort, z->st));
    SFCI_CUDA(normalize_vec(z->wc[dst], z->nkeep, z->ndev, z->scratch + z->off_norm, z->st));
    unsigned long long hn = 0;
    SFCI_CUDA(cudaMemcpyAsync(&hn, z->ndev, sizeof(hn), cudaMemcpyDeviceToHost, z->st));
    if (sumsq_host) SFCI_CUDA(cudaMemcpyAsync(sumsq_host, z->sumsq, 8, cudaMemcpyDeviceToHost, z->st));
    if (total_host) SFCI_CUDA(cudaMemcpyAsync(total_host, z->total, 8, cudaMemcpyDeviceToHost, z->st));
    SFCI_CUDA(cudaStreamSynchronize(z->st));
    z->wn[dst] = (long long)std::min<unsigned long long>(hn, (unsigned long long)z->nkeep);
    return SFCI_OK;
}

// make buffer b hold at least `want` bytes (contents are not kept); a buffer
// that has to grow gets `headroom` more, so a slowly growing need does not
// re-allocate every step
sfci_status ensure(sfci_lanczos::Buf &b, size_t want, cudaStream_t st, const char *what,
                   double headroom = 1.0) {
    if (b.p && b.bytes >= want) return SFCI_OK;
    SFCI_CUDA(cudaStreamSynchronize(st));
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (headroom > 1.0) {
        size_t free_b = 0, tot_b = 0;
        cudaMemGetInfo(&free_b, &tot_b);
        const size_t grown = size_t((double)want * headroom);
        if (grown < free_b / 10 * 9) want = grown;
    }
    cudaError_t e = cudaMalloc(&b.p, want > 0 ? want : 16);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc ") + what + ": " + cudaGetErrorString(e));
        return SFCI_E_NOMEM;
    }
    b.bytes = want;
    return SFCI_OK;
}

template <class T>
T *P(const sfci_lanczos::Buf &b) {
    return static_cast<T *>(b.p);
}

// Row mode is used when the alpha strings can be mapped densely.
constexpr unsigned long long kMaxRows = 1ull << 26;

// sigma_i = H w_i through the bucketed merge, with the probes of w_0..w_i.
// On return the streamed entries sit in sig_key/sig_val[0, *n_out) and sigma at
// every basis entry in sigw[j].
sfci_status bucketed_sigma(sfci_lanczos *z, int i, double *tau_io, unsigned long long *n_out,
                           unsigned long long *n_live, unsigned long long *n_nonzero, double *sumsq) {
    double tau = *tau_io;
    z->ms_alloc = 0.0;
    const SysDev &d = z->sys->d;
    const long long n_in = z->wn[i];
    const double E = (double)n_in * (double)(d.n_conn + 1);
    // elements per merge bucket: 1024 into 2048-slot tables; automatic mode takes
    // 2048 into the same tables when the previous sigma's entries repeated at
    // least 1.5 times on average, i.e. about 1400 distinct keys or fewer per
    // bucket (a bucket that still holds more distinct keys than slots is
    // reported by the merge, and sigma is redone with 1024)
    const double tau_entry = *tau_io;
    const bool force_big = (z->p.flags & SFCI_LZ_FALLBACK_STRESS) != 0;
    const bool big_auto = z->p.bucket_elems <= 0 && !z->small_buckets && (force_big || z->mult_prev >= z->big_thresh);
    const double per_bucket = z->p.bucket_elems > 0 ? (double)z->p.bucket_elems : (big_auto ? 2048.0 : 1024.0);
    const int slots = big_auto ? (force_big ? 1024 : 2048)
                               : (per_bucket <= 1024.0 ? 2048 : (per_bucket <= 2048.0 ? 4096 : 8192));
    const bool row_mode = d.ca <= kMaxRows;
    const auto t_plan0 = std::chrono::steady_clock::now();
    sfci_status r;
    Buckets bk{};
    bk.cb = d.cb;
    unsigned long long B = 0, runs = 0;
    unsigned hash_cap = 0;
    unsigned long long total_cap = 0;
    if (row_mode) {
        // exact element count per target alpha string, then the bucket plan on
        // the device: light rows packed into windows of half a bucket, heavy
        // rows split into buckets of their own (sfci_plan.cu)
        const unsigned long long nrows = d.ca;
        const unsigned long long Pb = std::max<unsigned long long>(2, (unsigned long long)per_bucket);
        const unsigned long long T = (unsigned long long)(E / (double)(Pb / 2)) + 2;  // windows
        if ((r = ensure(z->weights, (nrows + 1) * 8, z->st, "row weights", 1.5))) return r;
        if ((r = ensure(z->rowmap, nrows * 8, z->st, "row map", 1.5))) return r;
        if ((r = ensure(z->wpre, (nrows + 1) * 8, z->st, "row offsets", 1.5))) return r;
        if ((r = ensure(z->ptl, T * 4, z->st, "plan windows", 1.5))) return r;
        if ((r = ensure(z->pth, T * 4, z->st, "plan windows", 1.5))) return r;
        if ((r = ensure(z->pbstart, (T + 1) * 8, z->st, "plan window offsets", 1.5))) return r;
        if ((r = ensure(z->scan_ws, scan_ws_bytes((long long)std::max(T, nrows) + 1), z->st, "scan workspace", 1.5)))
            return r;
        // weights[nrows]: runs of inputs sharing alpha
        SFCI_CUDA(cudaMemsetAsync(z->weights.p, 0, (nrows + 1) * 8, z->st));
        SFCI_CUDA(launch_row_weights(d, z->wr[i], z->wc[i], n_in, z->p.eps_element,
                                     static_cast<unsigned long long *>(z->weights.p),
                                     static_cast<unsigned long long *>(z->weights.p) + nrows, z->st));
        auto *w = P<unsigned long long>(z->weights);
        SFCI_CUDA(exclusive_scan(static_cast<const unsigned long long *>(w), (long long)nrows,
                                 P<unsigned long long>(z->wpre), z->scan_ws.p, z->st));
        // windows: light flag in ptl, heavy bucket count in pth, their sum back in pth
        SFCI_CUDA(plan_windows(w, P<unsigned long long>(z->wpre), nrows, Pb, d.cb, T, P<unsigned>(z->ptl),
                               P<unsigned>(z->pth), P<unsigned>(z->pth), z->st));
        SFCI_CUDA(exclusive_scan(static_cast<const unsigned *>(P<unsigned>(z->pth)), (long long)T,
                                 P<unsigned long long>(z->pbstart), z->scan_ws.p, z->st));
        SFCI_CUDA(cudaMemcpyAsync(&B, P<unsigned long long>(z->pbstart) + T, 8, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaMemcpyAsync(&runs, w + nrows, 8, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaStreamSynchronize(z->st));
        if (B >= (1ull << 31)) {
            set_error("too many merge buckets");
            return SFCI_E_CAPACITY;
        }
        if ((r = ensure(z->pcap, std::max<unsigned long long>(B, 1) * 4, z->st, "bucket capacities", 1.5))) return r;
        if ((r = ensure(z->boff, (B + 1) * 8, z->st, "bucket offsets", 1.5))) return r;
        if ((r = ensure(z->scan_ws, scan_ws_bytes((long long)std::max({T, nrows, B}) + 1), z->st, "scan workspace",
                        1.5)))
            return r;
        SFCI_CUDA(plan_rows(w, P<unsigned long long>(z->wpre), nrows, Pb, d.cb, P<unsigned>(z->ptl),
                            P<unsigned long long>(z->pbstart), B, P<unsigned long long>(z->rowmap),
                            P<unsigned>(z->pcap), z->st));
        SFCI_CUDA(round_caps4(P<unsigned>(z->pcap), B, z->st));
        SFCI_CUDA(exclusive_scan(static_cast<const unsigned *>(P<unsigned>(z->pcap)), (long long)B,
                                 P<unsigned long long>(z->boff), z->scan_ws.p, z->st));
        SFCI_CUDA(cudaMemcpyAsync(&total_cap, P<unsigned long long>(z->boff) + B, 8, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaStreamSynchronize(z->st));
        bk.rowmap = static_cast<const unsigned long long *>(z->rowmap.p);
        bk.log2B = 0;
    } else {
        int log2B = 4;
        while (log2B < 30 && (double)(1ull << log2B) * per_bucket < E) ++log2B;
        B = 1ull << log2B;
        hash_cap = (unsigned)(std::ceil(1.125 * E / (double)B) + 128.0) & ~7u;
        if ((r = ensure(z->boff, (B + 1) * 8, z->st, "bucket offsets", 1.5))) return r;
        SFCI_CUDA(uniform_offsets(static_cast<unsigned long long *>(z->boff.p), B, hash_cap, z->st));
        bk.log2B = log2B;
        total_cap = B * (unsigned long long)hash_cap;
    }
    bk.boff = static_cast<const unsigned long long *>(z->boff.p);
    // bucket offsets on the host side: first bucket at or above each target
    // offset (and the offset there), and the offset of given buckets
    auto lower_bounds = [&](const std::vector<unsigned long long> &tg, std::vector<unsigned long long> &idx,
                            std::vector<unsigned long long> &at) -> cudaError_t {
        const size_t n = tg.size();
        idx.assign(n, 0ull);
        at.assign(n, 0ull);
        if (!n) return cudaSuccess;
        if (!row_mode) {
            for (size_t k = 0; k < n; ++k) {
                idx[k] = std::min<unsigned long long>(B, (tg[k] + hash_cap - 1) / hash_cap);
                at[k] = idx[k] * hash_cap;
            }
            return cudaSuccess;
        }
        cudaError_t e = cudaSuccess;
        if (z->pq.bytes < n * 24) {
            cudaFree(z->pq.p);
            z->pq.p = nullptr;
            z->pq.bytes = 0;
            e = cudaMalloc(&z->pq.p, n * 24 + 256);
            if (e != cudaSuccess) return e;
            z->pq.bytes = n * 24 + 256;
        }
        auto *dq = P<unsigned long long>(z->pq);
        e = cudaMemcpyAsync(dq, tg.data(), n * 8, cudaMemcpyHostToDevice, z->st);
        if (e == cudaSuccess) e = boff_lower_bounds(P<unsigned long long>(z->boff), B, dq, (int)n, dq + n, z->st);
        std::vector<unsigned long long> out(2 * n);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out.data(), dq + n, n * 16, cudaMemcpyDeviceToHost, z->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(z->st);
        for (size_t k = 0; k < n; ++k) idx[k] = out[2 * k], at[k] = out[2 * k + 1];
        return e;
    };
    auto boff_at = [&](unsigned long long b, unsigned long long &v) -> cudaError_t {
        if (!row_mode) {
            v = b * hash_cap;
            return cudaSuccess;
        }
        cudaError_t e = cudaMemcpyAsync(&v, P<unsigned long long>(z->boff) + b, 8, cudaMemcpyDeviceToHost, z->st);
        return e == cudaSuccess ? cudaStreamSynchronize(z->st) : e;
    };

    // streamed-output capacity: 16 N_d (the merge raises the threshold to keep
    // the stream within it) plus room for u's entries on w_i, w_{i-1}
    double sig_need = std::min(16.0 * (double)z->nkeep, E) + 2.0 * (double)z->nkeep + 1024.0;
    // overflow list per pass: 1.5 times the most any pass of the previous sigma
    // needed, grown by (element ratio)^0.75 when the input grew (a larger input
    // also runs more passes), at least 2^22 entries (warps take it in chunks of
    // 256 places); a pass that finds it short is split into pieces, or the
    // sigma is redone with a longer list
    // (and at least what this basis index needed one cycle earlier: a cycle's
    // first vector, the restart, concentrates sigma and overflows most)
    const double at_i = i < (int)z->ovf_at.size() ? (double)z->ovf_at[i] : 0.0;
    const long long ovf_lim = z->p.ovf_max_log2 > 0 ? 1ll << std::min(z->p.ovf_max_log2, 40)
                                                    : std::numeric_limits<long long>::max();
    long long ovf_cap = std::max<long long>(
        1 << 22, (long long)(1.5 * std::max(at_i, (double)z->ovf_used *
                                                std::pow(std::max(1.0, E / std::max(1.0, z->elem_prev)), 0.75))));
    ovf_cap = std::min(ovf_cap, ovf_lim);
    long long totp = 0;
    for (int j = 0; j <= i; ++j) totp += z->wn[j];
    // fixed-point unit of the exact sums: sigma entries are bounded by
    // (n_conn + 1) hbound max|c|, and the basis vectors are normalised (|c| <= 1)
    int fix_shift = (int)std::floor(125.0 - std::log2(std::max(1e-300, (double)(d.n_conn + 1) * d.hbound)));
    fix_shift = std::max(-900, std::min(1000, fix_shift));
    for (int attempt = 0; attempt < 8; ++attempt) {
        const double tau_start = tau;
        size_t free_b = 0, tot_b = 0;
        SFCI_CUDA(cudaMemGetInfo(&free_b, &tot_b));
        // memory the element regions may use: what is free plus what the big buffers hold
        const double held = (double)z->belem.bytes + (double)z->sig_key.bytes + (double)z->sig_val.bytes +
                            (double)z->bovf.bytes + (double)z->bovf_sorted.bytes;
        double avail = 0.85 * ((double)free_b + held);
        if (z->p.mem_budget > 0) avail = std::min(avail, (double)z->p.mem_budget);
        const double sig_bytes = 1.1 * sig_need * 16.0;
        // for the element regions (a pass's region offsets are 32-bit counts of 4 slots)
        const double budget = std::min(avail - sig_bytes - 2.0 * ovf_cap * 16.0, 4.0 * 4294967295.0 * sizeof(Slot));
        // passes: the fewest contiguous bucket ranges of about equal regions that
        // fit the budget (cut where the running region total crosses j/npass)
        const unsigned long long total_slots = total_cap;
        std::vector<unsigned long long> cuts, coff;  // pass boundaries (buckets) and their region offsets
        unsigned long long max_pass = 0;
        const int npass0 = std::max(1, (int)std::min(1e6, std::ceil((double)total_slots * sizeof(Slot) /
                                                                   std::max(budget, 1.0))));
        int npass = npass0;
        for (;; ++npass) {
            if (npass > (long long)B || budget <= 0.0 || npass > 4 * npass0 + 64) {
                set_error("not enough device memory for one merge bucket");
                return SFCI_E_CAPACITY;
            }
            std::vector<unsigned long long> tg, idx, at;
            for (int j = 1; j < npass; ++j) tg.push_back((unsigned long long)((double)total_slots * j / npass));
            SFCI_CUDA(lower_bounds(tg, idx, at));
            cuts.assign(1, 0ull);
            coff.assign(1, 0ull);
            for (int j = 1; j < npass; ++j) {
                unsigned long long c = std::max(idx[j - 1], cuts.back() + 1);
                c = std::min(c, B - (unsigned long long)(npass - j));
                unsigned long long o = at[j - 1];
                if (c != idx[j - 1]) SFCI_CUDA(boff_at(c, o));
                cuts.push_back(c);
                coff.push_back(o);
            }
            cuts.push_back(B);
            coff.push_back(total_slots);
            max_pass = 0;
            for (int j = 0; j < npass; ++j) max_pass = std::max(max_pass, coff[j + 1] - coff[j]);
            if ((double)max_pass * sizeof(Slot) <= budget) break;
        }
        const size_t need_elem = size_t(max_pass) * sizeof(Slot);
        size_t want_sig = size_t(sig_need) * 8;
        const auto t_alloc0 = std::chrono::steady_clock::now();
        const size_t need_ovf = size_t(ovf_cap) * sizeof(Slot);
        if (z->belem.bytes < need_elem || z->sig_key.bytes < want_sig || z->sig_val.bytes < want_sig ||
            z->bovf.bytes < need_ovf || z->bovf_sorted.bytes < need_ovf) {
            // the large buffers (elements, stream, overflow lists) are sized together
            // from one budget: free them all; the element regions get 5 % headroom,
            // the stream 10 %, and the overflow lists what is left (a longer list
            // saves splitting passes), up to a fifth of the elements each
            SFCI_CUDA(cudaStreamSynchronize(z->st));
            for (auto *bb : {&z->belem, &z->sig_key, &z->sig_val, &z->bovf, &z->bovf_sorted}) {
                cudaFree(bb->p);
                bb->p = nullptr;
                bb->bytes = 0;
            }
            want_sig = size_t(1.1 * sig_need) * 8;
            const size_t want_elem = size_t(std::min((double)need_elem * 1.05, budget));
            const double left = avail - sig_bytes - (double)want_elem;
            const double ovf_room = std::min({left / (2.0 * sizeof(Slot)), 0.2 * E + (double)(1 << 22),
                                              (double)ovf_lim});
            const size_t want_ovf = size_t(std::max((double)ovf_cap, ovf_room)) * sizeof(Slot);
            if ((r = ensure(z->sig_key, want_sig, z->st, "sigma keys"))) return r;
            if ((r = ensure(z->sig_val, want_sig, z->st, "sigma values"))) return r;
            if ((r = ensure(z->bovf, want_ovf, z->st, "overflow list"))) return r;
            if ((r = ensure(z->bovf_sorted, want_ovf, z->st, "sorted overflow"))) return r;
            if ((r = ensure(z->belem, want_elem, z->st, "element regions"))) return r;
        }
        z->sig_cap = (long long)(std::min(z->sig_key.bytes, z->sig_val.bytes) / 8);
        ovf_cap = std::min((long long)(std::min(z->bovf.bytes, z->bovf_sorted.bytes) / sizeof(Slot)), ovf_lim);
        z->ovf_cap = ovf_cap;
        if ((r = ensure(z->bcount, size_t(B) * 4, z->st, "bucket counters", 1.5))) return r;
        if ((r = ensure(z->start4, size_t(B + 1) * 4, z->st, "pass offsets", 1.5))) return r;
        if ((r = ensure(z->probes, size_t(std::max<long long>(totp, 1)) * sizeof(Probe), z->st, "probes"))) return r;
        if ((r = ensure(z->pcount, size_t(B) * 4, z->st, "probe counts", 1.5))) return r;
        if ((r = ensure(z->poff, size_t(B + 1) * 8, z->st, "probe offsets", 1.5))) return r;
        if ((r = ensure(z->tmp_counts, size_t(B + 1) * 4, z->st, "overflow counts", 1.5))) return r;
        if ((r = ensure(z->ovf_off, size_t(B + 1) * 8, z->st, "overflow offsets", 1.5))) return r;
        if ((r = ensure(z->scan_ws, scan_ws_bytes((long long)B + 1), z->st, "scan workspace", 1.5))) return r;
        for (int j = 0; j <= i; ++j)
            if (!z->sigw[j]) SFCI_CUDA(cudaMalloc(&z->sigw[j], size_t(z->nkeep) * 8));
        z->ms_alloc += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_alloc0).count();
        (void)total_cap;
        (void)hash_cap;

        // probes of w_0..w_i, bucketed once for all passes
        std::vector<VecRef> vr(i + 1);
        for (int j = 0; j <= i; ++j) vr[j] = VecRef{z->wr[j], z->wc[j], z->wn[j]};
        SFCI_CUDA(sort_probes(bk, B, vr.data(), z->sigw, i + 1, P<unsigned>(z->pcount),
                              P<unsigned long long>(z->poff), z->scan_ws.p, P<Probe>(z->probes), z->st));
        SFCI_CUDA(cudaMemsetAsync(z->bcount.p, 0, B * 4, z->st));
        SFCI_CUDA(cudaMemsetAsync(z->words, 0, kHistBins * 8 + 1024, z->st));
        // stream threshold (raised by the merge) and its first raise mark: half
        // of the room left for streamed entries once u's entries are set aside
        const long long u_room = 2 * z->nkeep + 1024;
        const long long out_cap = std::max<long long>(z->sig_cap - u_room, 0);
        unsigned long long tw[2];
        std::memcpy(&tw[0], &tau, 8);
        tw[1] = (unsigned long long)out_cap / 2;
        SFCI_CUDA(cudaMemcpyAsync(z->tau_w, tw, 16, cudaMemcpyHostToDevice, z->st));
        SFCI_CUDA(cudaStreamSynchronize(z->st));
        z->ms_plan = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_plan0).count();
        z->budget_gb = budget / 1e9;
        z->free_gb = (double)free_b / 1e9;
        z->held_gb = held / 1e9;
        z->regions_gb = (double)total_cap * sizeof(Slot) / 1e9;
        z->n_passes = npass;
        z->alpha_runs = runs;
        z->nb_log2 = 0;
        while ((1ull << z->nb_log2) < B) ++z->nb_log2;
        z->ms_emit = z->ms_merge = 0.0;
        unsigned long long max_ovf = 0;  // most overflow elements of any pass
        unsigned long long ovf_short = 0;  // a range's overflow that the list could not hold
        z->n_split = 0;
        // passes as bucket ranges; a range whose overflow outgrew the list is
        // split in two and emitted again (its merge has not run yet)
        struct Range {
            unsigned lo, hi;              // buckets
            unsigned long long olo, ohi;  // their region offsets
        };
        std::vector<Range> ranges;
        for (int pass = npass - 1; pass >= 0; --pass)
            ranges.push_back(Range{(unsigned)cuts[pass], (unsigned)cuts[pass + 1], coff[pass], coff[pass + 1]});
        while (!ranges.empty()) {
            const Range rg = ranges.back();
            const unsigned lo = rg.lo, hi = rg.hi;
            ranges.pop_back();
            SFCI_CUDA(cudaMemsetAsync(z->ovf_n, 0, 8, z->st));
            BucketOut bo;
            bo.bk = bk;
            bo.count = P<unsigned>(z->bcount);
            bo.elem = P<Slot>(z->belem);
            bo.base = rg.olo;
            SFCI_CUDA(pass_offsets(P<unsigned long long>(z->boff), lo, hi, P<unsigned>(z->start4), z->st));
            bo.start4 = P<unsigned>(z->start4);
            bo.eps_elem = z->p.eps_element > 0.0 ? z->p.eps_element : 0.0;
            bo.ovf = P<Slot>(z->bovf);
            bo.ovf_n = z->ovf_n;
            bo.ovf_cap = z->ovf_cap;
            bo.lo = lo, bo.hi = hi;
            bo.row_lo = 0, bo.row_hi = ~0ull;
            if (row_mode) {
                // rows are bucketed in order: the rows before the first one with a
                // bucket at or above lo, and from the first one with all its
                // buckets at or above hi on, hold no bucket of this pass
                if ((r = ensure(z->pq, 256, z->st, "plan queries"))) return r;
                unsigned long long lim[2];
                SFCI_CUDA(pass_rows(P<unsigned long long>(z->rowmap), d.ca, lo, hi, P<unsigned long long>(z->pq),
                                    z->st));
                SFCI_CUDA(cudaMemcpyAsync(lim, z->pq.p, 16, cudaMemcpyDeviceToHost, z->st));
                SFCI_CUDA(cudaStreamSynchronize(z->st));
                bo.row_lo = lim[0];
                bo.row_hi = lim[1] > 0 ? lim[1] - 1 : 0ull;
            }
            bo.status = z->mstatus;
            // alpha-alpha doubles by runs of sources sharing alpha when a pass
            // leaves rows for others (its queue skips them) or runs average two
            // sources or more (row reads and reservations shared); else inline
            bo.aa_runs = !(lo == 0 && (unsigned long long)hi >= B) || (runs > 0 && (unsigned long long)n_in >= 2 * runs);
            SFCI_CUDA(cudaEventRecord(z->evp[0], z->st));
            SFCI_CUDA(launch_emit_buckets(d, z->wr[i], z->wc[i], n_in, bo, z->st, z->p.emit_warps));
            SFCI_CUDA(cudaEventRecord(z->evp[1], z->st));
            unsigned long long on = 0;
            SFCI_CUDA(cudaMemcpyAsync(&on, z->ovf_n, 8, cudaMemcpyDeviceToHost, z->st));
            SFCI_CUDA(cudaStreamSynchronize(z->st));
            if ((long long)on > z->ovf_cap) {
                float a = 0.f;
                cudaEventElapsedTime(&a, z->evp[0], z->evp[1]);
                z->ms_emit += a;
                // the list was short for this range: split the range into pieces
                // the list can hold (each re-emits over all sources) when that is
                // cheaper than redoing sigma with a longer list
                // (when the list is at its limit, splitting is the only way on)
                const double k_need = std::ceil(1.25 * (double)on / (double)z->ovf_cap);
                const bool can_grow = z->ovf_cap < ovf_lim;
                const unsigned k = (unsigned)std::min<double>(hi - lo, k_need);
                if (hi - lo >= 2 && (k_need <= 3.0 || !can_grow) && z->n_split + (int)k - 1 <= (can_grow ? 6 : 256)) {
                    int hs2 = 0;
                    SFCI_CUDA(cudaMemcpyAsync(&hs2, z->mstatus, 4, cudaMemcpyDeviceToHost, z->st));
                    SFCI_CUDA(cudaStreamSynchronize(z->st));
                    hs2 &= ~2;  // the list's truncation bit: this range is emitted again in pieces
                    SFCI_CUDA(cudaMemcpyAsync(z->mstatus, &hs2, 4, cudaMemcpyHostToDevice, z->st));
                    SFCI_CUDA(cudaMemsetAsync(P<unsigned>(z->bcount) + lo, 0, size_t(hi - lo) * 4, z->st));
                    std::vector<unsigned long long> tg, idx, at;
                    for (unsigned j = 1; j < k; ++j) tg.push_back(rg.olo + (rg.ohi - rg.olo) * j / k);
                    SFCI_CUDA(lower_bounds(tg, idx, at));
                    std::vector<unsigned> cut{lo};
                    std::vector<unsigned long long> co{rg.olo};
                    for (unsigned j = 1; j < k; ++j) {
                        unsigned long long m = std::max<unsigned long long>(idx[j - 1], cut.back() + 1);
                        m = std::min<unsigned long long>(m, hi - (k - j));
                        unsigned long long o = at[j - 1];
                        if (m != idx[j - 1]) SFCI_CUDA(boff_at(m, o));
                        cut.push_back((unsigned)m);
                        co.push_back(o);
                    }
                    cut.push_back(hi);
                    co.push_back(rg.ohi);
                    for (unsigned j = k; j > 0; --j) ranges.push_back(Range{cut[j - 1], cut[j], co[j - 1], co[j]});
                    z->n_split += (int)k - 1;
                    continue;
                }
                ovf_short = std::max(ovf_short, on);
                break;
            }
            SFCI_CUDA(sort_overflow(bk, P<unsigned>(z->bcount), lo, hi - lo, P<Slot>(z->bovf), z->ovf_n,
                                    z->ovf_cap, P<unsigned>(z->tmp_counts), P<unsigned long long>(z->ovf_off),
                                    z->scan_ws.p, P<Slot>(z->bovf_sorted), z->st));
            MergeArgs A{};
            A.lo = lo, A.hi = hi;
            A.bk = bk;
            A.count = P<unsigned>(z->bcount);
            A.elem = P<Slot>(z->belem);
            A.ovf_sorted = P<Slot>(z->bovf_sorted);
            A.ovf_off = P<unsigned long long>(z->ovf_off);
            A.ovf_cap = z->ovf_cap;
            A.probes = P<Probe>(z->probes);
            A.probe_off = P<unsigned long long>(z->poff);
            for (int j = 0; j <= i; ++j) A.sigw[j] = z->sigw[j];
            A.ja = i;
            A.jb = i > 0 ? i - 1 : -1;
            A.eps = z->p.eps_screen > 0.0 ? z->p.eps_screen : 0.0;
            A.out_key = P<unsigned long long>(z->sig_key);
            A.out_val = P<double>(z->sig_val);
            A.out_cap = out_cap;
            A.out_n = z->outn;
            A.tau_bits = z->tau_w;
            A.hist = z->hist;
            A.mark = z->mark_w;
            A.lock = z->lock_w;
            A.nkeep = z->nkeep;
            A.fix_shift = fix_shift;
            A.sumsq = z->msumsq;
            A.n_live = z->mlive;
            A.n_nonzero = z->nnz;
            A.n_read = z->nread_w;
            A.queue = z->queue;
            A.status = z->mstatus;
            SFCI_CUDA(launch_merge(A, slots, z->st));
            SFCI_CUDA(cudaEventRecord(z->evp[2], z->st));
            unsigned long long ovf_here = 0;
            SFCI_CUDA(cudaMemcpyAsync(&ovf_here, z->ovf_n, 8, cudaMemcpyDeviceToHost, z->st));
            SFCI_CUDA(cudaEventSynchronize(z->evp[2]));
            SFCI_CUDA(cudaStreamSynchronize(z->st));
            max_ovf = std::max(max_ovf, ovf_here);
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, z->evp[0], z->evp[1]);
            cudaEventElapsedTime(&b, z->evp[1], z->evp[2]);
            z->ms_emit += a, z->ms_merge += b;
        }
        z->n_passes = npass + z->n_split;  // each split adds a pass
        int hs = 0;
        unsigned long long ho = 0, hl = 0, hz = 0;
        double hq = 0.0;
        SFCI_CUDA(cudaMemcpyAsync(&hs, z->mstatus, 4, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaMemcpyAsync(&ho, z->outn, 8, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaMemcpyAsync(&hl, z->mlive, 8, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaMemcpyAsync(&hz, z->nnz, 8, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaMemcpyAsync(&hq, z->msumsq, 8, cudaMemcpyDeviceToHost, z->st));
        unsigned long long tb = 0, hr = 0;
        SFCI_CUDA(cudaMemcpyAsync(&tb, z->tau_w, 8, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaMemcpyAsync(&hr, z->nread_w, 8, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaStreamSynchronize(z->st));
        std::memcpy(&tau, &tb, 8);  // as raised during the merge
        *tau_io = tau;
        if (hs == 0 && !ovf_short) {
            *n_out = ho, *n_live = hl, *n_nonzero = hz, *sumsq = hq;
            z->mult_prev = E / std::max(1.0, (double)hl);  // intermediate elements per sigma entry
            z->n_emitted = (long long)hr;
            z->stream_prev = ho;
            z->ovf_used = (long long)max_ovf;
            if ((int)z->ovf_at.size() <= i) z->ovf_at.resize(i + 1, 0);
            z->ovf_at[i] = (long long)max_ovf;
            z->elem_prev = E;
            return SFCI_OK;
        }
        if (hs & 16) {
            set_error("an intermediate element fell outside the row map");
            return SFCI_E_INVALID;
        }
        if (hs & 32) {  // an element beyond the fixed-point range (an input not normalised): coarser units
            fix_shift -= 16;
            tau = tau_start;
            *tau_io = tau;
            continue;
        }
        if (ovf_short) hs |= 2;  // passes left out: redo
        if (hs & 2) {  // the overflow list was cut short: the merge saw part of it, redo
            // (from the threshold this attempt started with)
            const long long grown = std::min(std::max(ovf_cap * 4, (long long)(1.5 * (double)ovf_short)), ovf_lim);
            if (grown <= ovf_cap) {
                set_error("the overflow list (elements past their merge bucket's region) needs more than its limit");
                return SFCI_E_CAPACITY;
            }
            ovf_cap = grown;
            tau = tau_start;
            *tau_io = tau;
            continue;
        }
        if (hs & 4) {
            if (big_auto) {  // the larger buckets did not fit the tables: this sigma with 1024
                // and no 2048-element try again until entries repeat clearly more
                // often than they did before this one
                if (!force_big) z->big_thresh = std::max(z->big_thresh, 1.25 * std::max(z->mult_prev, 1.5));
                z->bucket_redo += 1;
                z->small_buckets = true;
                *tau_io = tau_entry;
                const sfci_status r2 = bucketed_sigma(z, i, tau_io, n_out, n_live, n_nonzero, sumsq);
                z->small_buckets = false;
                return r2;
            }
            set_error("a merge bucket held more distinct entries than its table");
            return SFCI_E_CAPACITY;
        }
        // the stream outgrew its buffer before the raises caught up: redo from the
        // raised threshold (still at or below the N_d-th largest) with more room
        if (hs & 8) sig_need = std::max(sig_need * 2.0, (double)ho * 1.3 + 2.0 * z->nkeep);
    }
    set_error("bucketed sigma did not fit after 8 attempts");
    return SFCI_E_CAPACITY;
}

// w_0 = normalise(top_{N_d}(trial vector)); a new cycle begins
sfci_status load_vector(sfci_lanczos *z, const uint64_t *rank, const double *coef, long long n) {
    Items it{reinterpret_cast<const unsigned long long *>(rank), coef, 1, n};
    SFCI_CUDA(select_topk(it, z->nkeep, z->wr[0], z->wc[0], z->ndev, nullptr, nullptr,
                          z->scratch + z->off_sel, z->sel_bytes, z->st));
    SFCI_CUDA(sort_pairs(z->wr[0], z->wc[0], z->nkeep, z->ndev, 64, z->scratch + z->off_sort, z->st));
    SFCI_CUDA(normalize_vec(z->wc[0], z->nkeep, z->ndev, z->scratch + z->off_norm, z->st));
    unsigned long long hn = 0;
    SFCI_CUDA(cudaMemcpyAsync(&hn, z->ndev, 8, cudaMemcpyDeviceToHost, z->st));
    SFCI_CUDA(cudaStreamSynchronize(z->st));
    z->wn[0] = (long long)std::min<unsigned long long>(hn, (unsigned long long)z->nkeep);
    z->idx = 0;
    z->have_prev = false;
    z->just_ended = false;
    std::fill(z->T.begin(), z->T.end(), 0.0);
    std::fill(z->S.begin(), z->S.end(), 0.0);
    if (z->wn[0] == 0) {
        set_error("trial vector has no non-zero entry");
        return SFCI_E_INVALID;
    }
    return SFCI_OK;
}

}  // namespace

extern "C" {

sfci_status sfci_lanczos_load(sfci_lanczos *z, const uint64_t *rank, const double *coef,
                              int64_t n) {
    if (!z || n < 1 || !rank || !coef) {
        set_error("need a solver and a non-empty vector");
        return SFCI_E_INVALID;
    }
    return load_vector(z, rank, coef, n);
}

sfci_status sfci_lanczos_set_input(sfci_lanczos *z, const uint64_t *rank, const double *coef, int64_t n) {
    if (!z || n < 0 || (n > 0 && (!rank || !coef))) {
        set_error("need a solver and device vectors");
        return SFCI_E_INVALID;
    }
    if (n > z->nkeep) {
        set_error("the vector has more entries than n_keep");
        return SFCI_E_CAPACITY;
    }
    if (n == 0) {
        set_error("the input vector must not be empty");
        return SFCI_E_INVALID;
    }
    const int i = z->idx;
    SFCI_CUDA(cudaMemcpyAsync(z->wr[i], rank, size_t(n) * 8, cudaMemcpyDeviceToDevice, z->st));
    SFCI_CUDA(cudaMemcpyAsync(z->wc[i], coef, size_t(n) * 8, cudaMemcpyDeviceToDevice, z->st));
    SFCI_CUDA(cudaStreamSynchronize(z->st));
    z->wn[i] = n;
    return SFCI_OK;
}

sfci_status sfci_lanczos_create(sfci_lanczos **out, const sfci_system *sys,
                                const sfci_params *params, const uint64_t *init_rank,
                                const double *init_coef, int64_t n_init, void *stream) {
    if (!out || !sys || !params) {
        set_error("null argument");
        return SFCI_E_INVALID;
    }
    *out = nullptr;
    if (params->n_keep < 1 || params->n_lanczos < 1 || params->n_lanczos > kMaxVec || n_init < 1 ||
        !init_rank || !init_coef) {
        set_error("need n_keep >= 1, 1 <= n_lanczos <= 64 and a non-empty trial vector");
        return SFCI_E_INVALID;
    }
    if (params->emit_warps < 0 || params->emit_warps > 8 || params->mem_budget < 0 ||
        params->bucket_elems < 0 || !(params->eps_element >= 0.0) ||
        (params->flags & ~SFCI_LZ_FALLBACK_STRESS) != 0) {
        set_error("need 0 <= emit_warps <= 8, mem_budget, bucket_elems, eps_element >= 0, known flags");
        return SFCI_E_INVALID;
    }
    sfci_lanczos *z = new (std::nothrow) sfci_lanczos();
    if (!z) return SFCI_E_NOMEM;
    z->sys = sys;
    z->p = *params;
    z->st = static_cast<cudaStream_t>(stream);
    z->NL = params->n_lanczos;
    z->nkeep = params->n_keep;
    z->wr.assign(z->NL, nullptr);
    z->wc.assign(z->NL, nullptr);
    z->wn.assign(z->NL, 0);
    z->T.assign(size_t(z->NL) * z->NL, 0.0);
    z->S.assign(size_t(z->NL) * z->NL, 0.0);
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < z->NL && e == cudaSuccess; ++j) {
        e = cudaMalloc(&z->wr[j], size_t(z->nkeep) * 8);
        if (e == cudaSuccess) e = cudaMalloc(&z->wc[j], size_t(z->nkeep) * 8);
    }
    const long long sel_n = std::max<long long>(n_init, 1);
    z->sel_bytes = select_workspace_bytes(sel_n, z->nkeep);
    size_t o = 0;
    z->off_sel = o, o = a256(o + z->sel_bytes);
    z->off_sort = o, o = a256(o + sort_pairs_bytes(z->nkeep));
    z->off_norm = o, o = a256(o + normalize_ws_bytes(z->nkeep));
    z->off_dots = o, o = a256(o + dots_workspace_bytes(z->NL, z->nkeep));
    z->off_small = o, o = a256(o + 4096 + sizeof(double) * 2 * kMaxVec);
    if (e == cudaSuccess) e = cudaMalloc(&z->scratch, o);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&z->ev[k]);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&z->evp[k]);
    if (e == cudaSuccess) e = cudaMalloc(&z->words, kHistBins * 8 + 1024);
    if (e == cudaSuccess) {
        z->hist = reinterpret_cast<unsigned long long *>(z->words);
        char *w = z->words + kHistBins * 8;
        z->outn = reinterpret_cast<unsigned long long *>(w);
        z->mlive = reinterpret_cast<unsigned long long *>(w + 8);
        z->ovf_n = reinterpret_cast<unsigned long long *>(w + 16);
        z->cand_n = reinterpret_cast<unsigned long long *>(w + 24);
        z->msumsq = reinterpret_cast<double *>(w + 32);
        z->queue = reinterpret_cast<unsigned *>(w + 40);
        z->mstatus = reinterpret_cast<int *>(w + 44);
        z->nnz = reinterpret_cast<unsigned long long *>(w + 48);
        z->dmin = reinterpret_cast<double *>(w + 56);
        z->tau_w = reinterpret_cast<unsigned long long *>(w + 64);
        z->mark_w = reinterpret_cast<unsigned long long *>(w + 72);
        z->lock_w = reinterpret_cast<int *>(w + 80);
        z->nread_w = reinterpret_cast<unsigned long long *>(w + 88);
    }
    if (e != cudaSuccess) {
        destroy_lz(z);
        set_error(std::string("sfci_lanczos_create: ") + cudaGetErrorString(e));
        return SFCI_E_NOMEM;
    }
    char *sm = z->scratch + z->off_small;
    z->tstatus = reinterpret_cast<int *>(sm);
    z->tcount = reinterpret_cast<unsigned long long *>(sm + 256);
    z->ndev = reinterpret_cast<unsigned long long *>(sm + 512);
    z->total = reinterpret_cast<unsigned long long *>(sm + 768);
    z->screened = reinterpret_cast<unsigned long long *>(sm + 1024);
    z->sumsq = reinterpret_cast<double *>(sm + 1280);
    z->dT = reinterpret_cast<double *>(sm + 4096);
    z->dS = z->dT + kMaxVec;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    double table_bytes = 0.8 * (double)free_b;
    if (params->mem_budget > 0) table_bytes = std::min(table_bytes, 0.5 * (double)params->mem_budget);
    unsigned long long bud = (unsigned long long)table_bytes / sizeof(Slot);
    unsigned long long p2 = 1;
    while ((p2 << 1) <= bud) p2 <<= 1;
    z->budget = p2;
    if (params->table_capacity > 0) z->budget = std::min(z->budget, next_pow2(params->table_capacity));
    const sfci_status rs = load_vector(z, init_rank, init_coef, n_init);
    if (rs != SFCI_OK) {
        destroy_lz(z);
        return rs;
    }
    *out = z;
    return SFCI_OK;
}

sfci_status sfci_lanczos_step(sfci_lanczos *z, sfci_step_info *info) {
    if (!z || !info) {
        set_error("null argument");
        return SFCI_E_INVALID;
    }
    std::memset(info, 0, sizeof(*info));
    NvtxRange nv_step("sfci_lanczos_step");
    const SysDev &d = z->sys->d;
    const int i = z->idx, NL = z->NL;
    z->bucket_redo = 0;
    z->just_ended = false;
    const long long n_in = z->wn[i];
    SFCI_CUDA(cudaEventRecord(z->ev[0], z->st));

    bool last = (i == NL - 1) || (z->p.max_iter > 0 && z->iter + 1 >= z->p.max_iter);
    // Stream threshold tau: predicted from earlier cuts; nothing at a cycle's
    // last vector (u is not formed there).  Checked after the truncation and,
    // if the N_d largest did not all clear it, sigma is redone with the exact
    // threshold from this attempt's magnitude histogram.
    double tau = __builtin_inf();
    if (!last) {
        // a fraction of the cut at the same basis index one cycle earlier (else of
        // the previous cut); low on purpose, the merge raises it as it goes
        const double ci = i < (int)z->cut_at.size() ? z->cut_at[i] : 0.0;
        tau = (ci > 0.0 ? ci : z->tau_prev) * (i == 0 ? 1.0 / 32.0 : 0.125);
    }
    std::vector<VecRef> vr(i + 1);
    for (int j = 0; j <= i; ++j) vr[j] = VecRef{z->wr[j], z->wc[j], z->wn[j]};
    for (int attempt = 0;; ++attempt) {
        // ---- sigma_i = H w_i, bucketed merge with the probes of w_0..w_i
        unsigned long long n_stream = 0, n_live = 0, n_nz = 0;
        double sq = 0.0;
        {
            NvtxRange nv("sigma (plan, emit, merge)");
            const sfci_status rs = bucketed_sigma(z, i, &tau, &n_stream, &n_live, &n_nz, &sq);
            if (rs != SFCI_OK) return rs;
        }
        info->ms_sigma = z->ms_emit + z->ms_merge;
        info->ms_emit = z->ms_emit;
        info->ms_merge = z->ms_merge;
        info->ms_plan = z->ms_plan;
        info->n_passes = z->n_passes;
        info->pass_budget_gb = z->budget_gb;
        info->regions_gb = z->regions_gb;
        info->free_gb = z->free_gb + z->held_gb;
        info->n_overflow = z->ovf_used;
        info->n_alpha_runs = (long long)z->alpha_runs;
        info->ms_alloc = z->ms_alloc;
        info->n_buckets_log2 = z->nb_log2;
        info->n_elements = n_in * (d.n_conn + 1);
        info->n_sigma = (long long)n_live;
        info->bucket_redo = z->bucket_redo;
        info->n_emitted = z->n_emitted;
        z->m_prev = (long long)n_live;
        z->nin_prev = n_in;

        // ---- T_ji = <w_j|sigma_i> from sigma recorded at w_j's entries, S_ji = <w_j|w_i>
        SFCI_CUDA(aligned_dots(vr.data(), z->sigw, i + 1, z->dT, z->scratch + z->off_dots, z->st));
        SFCI_CUDA(vec_overlaps(vr.data(), i + 1, vr[i], z->dS, z->scratch + z->off_dots, z->st));
        std::vector<double> tcol(i + 1), scol(i + 1);
        SFCI_CUDA(cudaMemcpyAsync(tcol.data(), z->dT, 8 * (i + 1), cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaMemcpyAsync(scol.data(), z->dS, 8 * (i + 1), cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaStreamSynchronize(z->st));
        for (int j = 0; j <= i; ++j) {
            z->T[size_t(j) * NL + i] = tcol[j];
            z->S[size_t(j) * NL + i] = scol[j];
        }
        const double a = tcol[i], b = i > 0 ? tcol[i - 1] : 0.0;
        info->a = a;
        info->b = b;
        info->t00 = z->T[0];
        if (last) break;

        // u = sigma_i - a w_i - b w_{i-1} on the support of w_i and w_{i-1} (Eq. 10);
        // elsewhere u = sigma_i, streamed where |u| >= tau
        NvtxRange nv_trunc("u and truncation (Eq. 10-11)");
        SFCI_CUDA(cudaEventRecord(z->evp[3], z->st));
        const VecRef wi = vr[i];
        const VecRef wm = i > 0 ? vr[i - 1] : VecRef{nullptr, nullptr, 0};
        unsigned long long *skey = static_cast<unsigned long long *>(z->sig_key.p);
        double *sval = static_cast<double *>(z->sig_val.p);
        SFCI_CUDA(launch_u_entries(wi, z->sigw[i], wm, i > 0 ? z->sigw[i - 1] : nullptr, a, b, skey, sval,
                                   n_stream, z->sig_cap, z->msumsq, z->mstatus, z->st));
        const long long n_items = (long long)n_stream + wi.n + wm.n;
        // Eq. 11: top-N_d of u
        const long long cand_cap = std::max<long long>(4 * z->nkeep, 1 << 22);
        sfci_status rs;
        if ((rs = ensure(z->cand_key, size_t(cand_cap) * 8, z->st, "candidates"))) return rs;
        if ((rs = ensure(z->cand_val, size_t(cand_cap) * 8, z->st, "candidates"))) return rs;
        z->cand_cap = cand_cap;
        Items it{skey, sval, 1, n_items};
        SplitResult res{};
        SFCI_CUDA(select_split(it, z->nkeep, z->wr[i + 1], z->wc[i + 1], z->ndev,
                               static_cast<unsigned long long *>(z->cand_key.p),
                               static_cast<double *>(z->cand_val.p), cand_cap, z->cand_n,
                               z->scratch + z->off_sel, z->sel_bytes, &res, z->st));
        unsigned long long kept = std::min<unsigned long long>(res.n_out, (unsigned long long)z->nkeep);
        if (!res.done && !res.all) {
            unsigned long long n2 = 0;
            if ((long long)res.n_cand > cand_cap) {  // the picked bin is too crowded: exact select over all
                SFCI_CUDA(select_topk(it, z->nkeep, z->wr[i + 1], z->wc[i + 1], z->total, nullptr, nullptr,
                                      z->scratch + z->off_sel, z->sel_bytes, z->st));
                kept = 0;
            } else {
                Items ci{static_cast<const unsigned long long *>(z->cand_key.p),
                         static_cast<const double *>(z->cand_val.p), 1, (long long)res.n_cand};
                SFCI_CUDA(select_topk(ci, (long long)res.need, z->wr[i + 1] + kept, z->wc[i + 1] + kept,
                                      z->total, nullptr, nullptr, z->scratch + z->off_sel, z->sel_bytes,
                                      z->st));
            }
            SFCI_CUDA(cudaMemcpyAsync(&n2, z->total, 8, cudaMemcpyDeviceToHost, z->st));
            SFCI_CUDA(cudaStreamSynchronize(z->st));
            kept = std::min<unsigned long long>(kept + n2, (unsigned long long)z->nkeep);
        }
        double usq = 0.0, cut = 0.0;
        int hs = 0;
        SFCI_CUDA(cudaMemcpyAsync(z->ndev, &kept, 8, cudaMemcpyHostToDevice, z->st));
        SFCI_CUDA(min_abs(z->wc[i + 1], z->ndev, z->nkeep, z->dmin, z->st));
        SFCI_CUDA(cudaMemcpyAsync(&cut, z->dmin, 8, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaMemcpyAsync(&usq, z->msumsq, 8, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaMemcpyAsync(&hs, z->mstatus, 4, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaStreamSynchronize(z->st));
        if (hs & 8) {
            set_error("sigma output buffer overflowed while appending u");
            return SFCI_E_CAPACITY;
        }
        // were all of the N_d largest streamed?  (entries below tau were not)
        const bool complete = tau <= 0.0 || (kept == (unsigned long long)z->nkeep ? !(cut < tau)
                                                                                  : n_nz + wi.n + wm.n <= (unsigned long long)n_items);
        if (!complete) {
            // the predicted threshold hid part of the N_d largest: redo lower
            // (the merge raises it again as entries stream), last resort 0
            if (attempt >= 2) {
                set_error("truncation threshold check failed three times");
                return SFCI_E_CAPACITY;
            }
            tau = attempt == 0 ? tau / 64.0 : 0.0;
            info->redo += 1;
            continue;
        }
        z->tau_prev = kept == (unsigned long long)z->nkeep ? cut : 0.0;
        if ((int)z->cut_at.size() < NL) z->cut_at.assign(NL, 0.0);
        z->cut_at[i] = z->tau_prev;
        info->tau = tau;
        info->cut = z->tau_prev;
        SFCI_CUDA(sort_pairs(z->wr[i + 1], z->wc[i + 1], z->nkeep, z->ndev, key_bits(d.dim),
                             z->scratch + z->off_sort, z->st));
        SFCI_CUDA(normalize_vec(z->wc[i + 1], z->nkeep, z->ndev, z->scratch + z->off_norm, z->st));
        z->wn[i + 1] = (long long)kept;
        SFCI_CUDA(cudaEventRecord(z->evp[0], z->st));
        SFCI_CUDA(cudaEventSynchronize(z->evp[0]));
        {
            float tk = 0.f;
            cudaEventElapsedTime(&tk, z->evp[3], z->evp[0]);
            info->ms_topk = tk;
        }
        const double unorm = std::sqrt(usq);
        info->u_norm = unorm;
        if (unorm < 1e-14 * std::fabs(a) || res.total == 0) {
            last = true;
            info->breakdown = 1;
        } else {
            info->n_kept = z->wn[i + 1];
            z->idx = i + 1;
        }
        break;
    }
    z->iter += 1;
    info->iter = z->iter;
    info->cycle = z->cycle;
    info->index = i;
    info->n_in = n_in;
    if (last) {
        NvtxRange nv_end("cycle end (eigensolve, restart)");
        const int m = i + 1;
        std::vector<double> Tm(size_t(m) * m), Sm(size_t(m) * m);
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c) {
                const int lo = std::min(r, c), hi = std::max(r, c);
                Tm[size_t(r) * m + c] = z->T[size_t(lo) * NL + hi];
                Sm[size_t(r) * m + c] = z->S[size_t(lo) * NL + hi];
            }
        std::vector<double> x;
        const double lam = gen_eig_lowest(m, Tm, Sm, x);
        info->lambda_min = lam;
        info->cycle_end = 1;
        // Psi = sum_j x_j w_j, ascending j
        long long tot = 0;
        for (int j = 0; j < m; ++j) tot += z->wn[j];
        unsigned long long pcap = next_pow2((unsigned long long)std::max<long long>(65536, 2 * tot));
        if (pcap > z->budget) pcap = z->budget;
        sfci_status rs = ensure_slots(z, pcap);
        if (rs != SFCI_OK) return rs;
        Table tp = make_table(z, pcap);
        SFCI_CUDA(table_clear(tp, z->st));
        for (int j = 0; j < m; ++j)
            SFCI_CUDA(table_axpy(tp, z->wr[j], z->wc[j], z->wn[j], nullptr, x[j], 1.0, z->st));
        unsigned long long ptot = 0;
        rs = table_topk(z, pcap, 0, nullptr, &ptot);
        if (rs != SFCI_OK) return rs;
        info->n_psi = (long long)ptot;
        info->n_kept = z->wn[0];
        if (z->p.conv_tol > 0.0 && z->have_prev && z->e_prev - lam < z->p.conv_tol) info->converged = 1;
        z->e_prev = lam;
        z->have_prev = true;
        z->cycle += 1;
        z->idx = 0;
        z->T_last = z->T;
        z->S_last = z->S;
        z->just_ended = true;
        std::fill(z->T.begin(), z->T.end(), 0.0);
        std::fill(z->S.begin(), z->S.end(), 0.0);
    }
    SFCI_CUDA(cudaEventRecord(z->ev[3], z->st));
    SFCI_CUDA(cudaEventSynchronize(z->ev[3]));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, z->ev[0], z->ev[3]);
    info->ms_step = ms;
    log_step(*info);
    return SFCI_OK;
}

sfci_status sfci_lanczos_vector(const sfci_lanczos *z, uint64_t *rank, double *coef, int64_t cap,
                                int64_t *n) {
    if (!z || !n) {
        set_error("null argument");
        return SFCI_E_INVALID;
    }
    const long long m = z->wn[z->idx];
    *n = m;
    if (m > cap) {
        set_error("cap below the vector length");
        return SFCI_E_CAPACITY;
    }
    if (m == 0) return SFCI_OK;
    SFCI_CUDA(cudaMemcpyAsync(rank, z->wr[z->idx], m * 8, cudaMemcpyDeviceToDevice, z->st));
    SFCI_CUDA(cudaMemcpyAsync(coef, z->wc[z->idx], m * 8, cudaMemcpyDeviceToDevice, z->st));
    SFCI_CUDA(cudaStreamSynchronize(z->st));
    return SFCI_OK;
}

sfci_status sfci_lanczos_matrices(const sfci_lanczos *z, double *T, double *S) {
    if (!z || !T || !S) {
        set_error("null argument");
        return SFCI_E_INVALID;
    }
    const bool ended = z->just_ended && !z->T_last.empty();
    std::memcpy(T, (ended ? z->T_last : z->T).data(), z->T.size() * 8);
    std::memcpy(S, (ended ? z->S_last : z->S).data(), z->S.size() * 8);
    return SFCI_OK;
}

sfci_status sfci_lanczos_destroy(sfci_lanczos *z) {
    if (!z) return SFCI_OK;
    cudaStreamSynchronize(z->st);
    destroy_lz(z);
    return SFCI_OK;
}

}  // extern "C"
