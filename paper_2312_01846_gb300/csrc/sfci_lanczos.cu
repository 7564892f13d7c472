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
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

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
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

void destroy_lz(sfci_lanczos *z) {
    if (!z) return;
    for (auto p : z->wr) cudaFree(p);
    for (auto p : z->wc) cudaFree(p);
    cudaFree(z->slots);
    cudaFree(z->scratch);
    for (auto &e : z->ev)
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
    unsigned long long bud = (unsigned long long)(0.8 * (double)free_b) / sizeof(Slot);
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
    const SysDev &d = z->sys->d;
    const int i = z->idx, NL = z->NL;
    const long long n_in = z->wn[i];
    SFCI_CUDA(cudaEventRecord(z->ev[0], z->st));

    // ---- sigma_i = H w_i into the table, grown and redone if it overflows
    double est;
    if (z->m_prev > 0 && z->nin_prev > 0)
        est = 1.25 * (double)z->m_prev * std::max(1.0, (double)n_in / (double)z->nin_prev);
    else
        est = (double)n_in * (double)(d.n_conn + 1);
    est += 2.0 * (double)z->nkeep;
    double want = std::max(65536.0, 2.0 * est);
    unsigned long long cap = want >= (double)z->budget ? z->budget : next_pow2((unsigned long long)want);
    unsigned long long hcount = 0;
    for (;;) {
        sfci_status rs = ensure_slots(z, cap);
        if (rs != SFCI_OK) return rs;
        Table t = make_table(z, cap);
        SFCI_CUDA(table_clear(t, z->st));
        SFCI_CUDA(cudaEventRecord(z->ev[1], z->st));
        SFCI_CUDA(launch_emit(d, z->wr[i], z->wc[i], n_in, t, z->st));
        SFCI_CUDA(cudaEventRecord(z->ev[2], z->st));
        int hstatus = 0;
        SFCI_CUDA(cudaMemcpyAsync(&hstatus, z->tstatus, sizeof(int), cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaMemcpyAsync(&hcount, z->tcount, 8, cudaMemcpyDeviceToHost, z->st));
        SFCI_CUDA(cudaStreamSynchronize(z->st));
        const bool full = (hstatus & 1) ||
                          (double)hcount + 2.0 * (double)z->nkeep > 0.85 * (double)cap;
        if (!full) break;
        if (cap >= z->budget) {
            set_error("sigma's merge table needs more device memory than is free");
            return SFCI_E_CAPACITY;
        }
        cap = std::min(cap * 4, z->budget);
    }
    float ms_sigma = 0.f;
    cudaEventElapsedTime(&ms_sigma, z->ev[1], z->ev[2]);
    info->ms_sigma = ms_sigma;
    info->n_elements = n_in * (d.n_conn + 1);
    z->m_prev = (long long)hcount;
    z->nin_prev = n_in;
    Table t = make_table(z, cap);
    SFCI_CUDA(table_screen(t, z->p.eps_screen, z->screened, z->st));

    // ---- T_ji = <w_j|sigma_i>, S_ji = <w_j|w_i>, j <= i
    std::vector<VecRef> vr(i + 1);
    for (int j = 0; j <= i; ++j) vr[j] = VecRef{z->wr[j], z->wc[j], z->wn[j]};
    SFCI_CUDA(table_dots(t, vr.data(), i + 1, z->dT, z->scratch + z->off_dots, z->st));
    SFCI_CUDA(vec_overlaps(vr.data(), i + 1, vr[i], z->dS, z->scratch + z->off_dots, z->st));
    std::vector<double> tcol(i + 1), scol(i + 1);
    unsigned long long hscreened = 0;
    SFCI_CUDA(cudaMemcpyAsync(tcol.data(), z->dT, 8 * (i + 1), cudaMemcpyDeviceToHost, z->st));
    SFCI_CUDA(cudaMemcpyAsync(scol.data(), z->dS, 8 * (i + 1), cudaMemcpyDeviceToHost, z->st));
    SFCI_CUDA(cudaMemcpyAsync(&hscreened, z->screened, 8, cudaMemcpyDeviceToHost, z->st));
    SFCI_CUDA(cudaStreamSynchronize(z->st));
    for (int j = 0; j <= i; ++j) {
        z->T[size_t(j) * NL + i] = tcol[j];
        z->S[size_t(j) * NL + i] = scol[j];
    }
    z->iter += 1;
    info->iter = z->iter;
    info->cycle = z->cycle;
    info->index = i;
    info->n_in = n_in;
    info->n_sigma = (long long)(hcount - hscreened);
    const double a = tcol[i], b = i > 0 ? tcol[i - 1] : 0.0;
    info->a = a;
    info->b = b;
    info->t00 = z->T[0];

    bool last = (i == NL - 1) || (z->p.max_iter > 0 && z->iter >= z->p.max_iter);
    if (!last) {
        // u = sigma_i - a w_i - b w_{i-1}  (Eq. 10), then Eq. 11
        SFCI_CUDA(table_axpy(t, z->wr[i], z->wc[i], n_in, nullptr, a, -1.0, z->st));
        if (i > 0) SFCI_CUDA(table_axpy(t, z->wr[i - 1], z->wc[i - 1], z->wn[i - 1], nullptr, b, -1.0, z->st));
        double usq = 0.0;
        unsigned long long utot = 0;
        sfci_status rs = table_topk(z, cap, i + 1, &usq, &utot);
        if (rs != SFCI_OK) return rs;
        const double unorm = std::sqrt(usq);
        info->u_norm = unorm;
        if (unorm < 1e-14 * std::fabs(a) || utot == 0) {
            last = true;
            info->breakdown = 1;
        } else {
            info->n_kept = z->wn[i + 1];
            z->idx = i + 1;
        }
    }
    if (last) {
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
        std::fill(z->T.begin(), z->T.end(), 0.0);
        std::fill(z->S.begin(), z->S.end(), 0.0);
    }
    SFCI_CUDA(cudaEventRecord(z->ev[3], z->st));
    SFCI_CUDA(cudaEventSynchronize(z->ev[3]));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, z->ev[0], z->ev[3]);
    info->ms_step = ms;
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
    std::memcpy(T, z->T.data(), z->T.size() * 8);
    std::memcpy(S, z->S.data(), z->S.size() * 8);
    return SFCI_OK;
}

sfci_status sfci_lanczos_destroy(sfci_lanczos *z) {
    if (!z) return SFCI_OK;
    cudaStreamSynchronize(z->st);
    destroy_lz(z);
    return SFCI_OK;
}

}  // extern "C"
