// C ABI of libsfci.so: systems, Eq. 12 rank/unrank, sigma = H psi, the Eq. 11
// truncation and the element export.  Declarations and contracts: sfci.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sfci_internal.cuh"

namespace sfci {

namespace {
thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const std::string &msg) { g_last_error = msg; }

sfci_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return SFCI_E_CUDA;
}

namespace {

sfci_status invalid(const std::string &msg) {
    set_error(msg);
    return SFCI_E_INVALID;
}

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

unsigned long long next_pow2(unsigned long long x) {
    unsigned long long p = 1;
    while (p < x) p <<= 1;
    return p;
}

int key_bits(unsigned long long dim) {
    if (dim <= 1) return 8;
    int b = 64 - __builtin_clzll(dim - 1);
    return b;
}

// Layout of sfci_sigma's workspace.
struct SigmaLayout {
    unsigned long long slots;
    size_t table, acc, status, count, ndev, flag, screened, maxabs, sortws, bytes;
};

SigmaLayout sigma_layout(long long out_cap) {
    SigmaLayout L{};
    unsigned long long want = out_cap > 0 ? 2ull * (unsigned long long)out_cap : 1ull;
    L.slots = next_pow2(want < 1024 ? 1024 : want);
    size_t o = 0;
    L.table = o, o = a256(o + L.slots * sizeof(Slot));
    L.acc = o, o = a256(o + L.slots * 16);  // exact sums, 128 bits per slot
    L.status = o, o = a256(o + sizeof(int));
    L.count = o, o = a256(o + sizeof(unsigned long long));
    L.ndev = o, o = a256(o + sizeof(unsigned long long));
    L.flag = o, o = a256(o + sizeof(int));
    L.screened = o, o = a256(o + sizeof(unsigned long long));
    L.maxabs = o, o = a256(o + sizeof(unsigned long long));
    L.sortws = o, o = a256(o + sort_pairs_bytes(out_cap > 0 ? out_cap : 1));
    L.bytes = o;
    return L;
}

struct TopkLayout {
    size_t sel, sort, norm, ndev, bytes;
};

TopkLayout topk_layout(long long n, long long k) {
    TopkLayout L{};
    size_t o = 0;
    L.sel = o, o = a256(o + select_workspace_bytes(n, k));
    L.sort = o, o = a256(o + sort_pairs_bytes(k > 0 ? k : 1));
    L.norm = o, o = a256(o + normalize_ws_bytes(k));
    L.ndev = o, o = a256(o + sizeof(unsigned long long));
    L.bytes = o;
    return L;
}

sfci_status check_sys(const sfci_system *s) {
    if (!s) return invalid("null system");
    return SFCI_OK;
}

}  // namespace
}  // namespace sfci

using namespace sfci;

extern "C" {

const char *sfci_status_string(int status) {
    switch (status) {
    case SFCI_OK: return "ok";
    case SFCI_E_INVALID: return "invalid argument";
    case SFCI_E_CAPACITY: return "capacity exceeded";
    case SFCI_E_OVERFLOW: return "index overflow";
    case SFCI_E_CUDA: return "CUDA error";
    case SFCI_E_TIMEOUT: return "device wait timed out";
    case SFCI_E_NOMEM: return "out of memory";
    default: return "unknown status";
    }
}

const char *sfci_last_error(void) { return g_last_error.c_str(); }

int sfci_version(void) { return 100; }

int64_t sfci_kernel_launches(void) { return launch_count(); }

sfci_status sfci_system_create(sfci_system **out, int n, int na, int nb, const double *h_host,
                               const double *g_host, double e_core, uint32_t flags) {
    if (!out || !h_host || !g_host) return invalid("null argument");
    if (flags & ~SFCI_FP32_ELEMENTS) return invalid("unknown flag bits");
    const bool fp32 = (flags & SFCI_FP32_ELEMENTS) != 0;
    *out = nullptr;
    if (n < 1 || n > 64) {
        set_error("n_orb must be in [1, 64]");
        return SFCI_E_OVERFLOW;
    }
    if (na < 0 || nb < 0 || na > n || nb > n) return invalid("electron counts out of range");
    // binomials C(b, m), b <= 64 (built once; thread-safe static initialisation)
    struct Binomials {
        unsigned long long v[65][65];
        Binomials() {
            for (int a = 0; a <= 64; ++a) {
                for (int b = 0; b <= 64; ++b) v[a][b] = 0;
                v[a][0] = 1;
                for (int b = 1; b <= a; ++b) v[a][b] = v[a - 1][b - 1] + v[a - 1][b];
            }
        }
    };
    static const Binomials binomials;
    const auto &C = binomials.v;
    const unsigned long long ca = C[n][na], cb = C[n][nb];
    if (cb != 0 && ca > (~0ull - 1ull) / cb) {
        set_error("dim = C(n,na) C(n,nb) does not fit below 2^64 - 1");
        return SFCI_E_OVERFLOW;
    }
    SysDev d{};
    d.n = n, d.na = na, d.nb = nb, d.va = n - na, d.vb = n - nb;
    d.ks = (na > nb ? na : nb) + 3;
    d.sa = na * (n - na), d.sb = nb * (n - nb);
    d.po_a = int(C[na][2]), d.pv_a = int(C[n - na][2]);
    d.po_b = int(C[nb][2]), d.pv_b = int(C[n - nb][2]);
    d.pair_off[0] = 0;
    d.pair_off[1] = d.po_a;
    d.pair_off[2] = d.pair_off[1] + d.pv_a;
    d.pair_off[3] = d.pair_off[2] + d.po_b;
    d.n_pairs = d.pair_off[3] + d.pv_b;
    d.ca = ca, d.cb = cb, d.dim = ca * cb;
    d.n_conn = (long long)d.sa + d.sb + (long long)d.po_a * d.pv_a + (long long)d.po_b * d.pv_b +
               (long long)d.sa * d.sb;
    d.e_core = e_core;

    std::vector<unsigned long long> bt(size_t(n + 1) * d.ks, 0ull);
    for (int b = 0; b <= n; ++b)
        for (int m = 0; m < d.ks; ++m) bt[size_t(b) * d.ks + m] = (m <= 64) ? C[b][m] : 0ull;
    std::vector<unsigned char> pairs(size_t(d.n_pairs) * 2 + 2, 0);
    {
        size_t o = 0;
        const int ms[4] = {na, n - na, nb, n - nb};
        for (int l = 0; l < 4; ++l)
            for (int i = 0; i < ms[l]; ++i)
                for (int j = i + 1; j < ms[l]; ++j) pairs[o++] = (unsigned char)i, pairs[o++] = (unsigned char)j;
    }
    const size_t nh = size_t(n) * n, ng = nh * nh;
    size_t o = 0;
    const size_t off_h = o;
    o = a256(o + nh * 8);
    const size_t off_g = o;
    o = a256(o + ng * 8);
    const size_t off_bt = o;
    o = a256(o + bt.size() * 8);
    const size_t off_p = o;
    o = a256(o + pairs.size());
    // bounds for the heat-bath style screen (times 1 + 1e-6: float32 elements
    // may exceed the float64 values by a few units in the last place)
    std::vector<double> bab(nh, 0.0), bss(nh, 0.0);
    for (int a = 0; a < n; ++a)
        for (int i = 0; i < n; ++i) {
            // opposite-spin double with alpha hop i -> a: |(ai|bj)|, max over (b, j)
            double m = 0.0;
            for (size_t t = 0; t < nh; ++t) m = std::max(m, std::fabs(g_host[(size_t(a) * n + i) * nh + t]));
            bab[size_t(a) * n + i] = m * (1.0 + 1e-6);
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            // same-spin double (i, j) -> (a, b): |(ai|bj) - (aj|bi)|, max over (a, b)
            double m = 0.0;
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b) {
                    const double x = g_host[((size_t(a) * n + i) * n + b) * n + j];
                    const double y = g_host[((size_t(a) * n + j) * n + b) * n + i];
                    m = std::max(m, std::fabs(x - y));
                }
            bss[size_t(i) * n + j] = m * (1.0 + 1e-6);
        }
    const size_t off_bab = o;
    o = a256(o + nh * 8);
    const size_t off_bss = o;
    o = a256(o + nh * 8);
    const size_t off_hf = o;
    if (fp32) o = a256(o + nh * 4);
    const size_t off_gf = o;
    if (fp32) o = a256(o + ng * 4);
    std::vector<float> hf, gf;
    if (fp32) {
        hf.resize(nh), gf.resize(ng);
        for (size_t i = 0; i < nh; ++i) hf[i] = (float)h_host[i];
        for (size_t i = 0; i < ng; ++i) gf[i] = (float)g_host[i];
    }
    sfci_system *s = new (std::nothrow) sfci_system();
    if (!s) {
        set_error("host allocation failed");
        return SFCI_E_NOMEM;
    }
    cudaGetDevice(&s->device);
    char *blk = nullptr;
    cudaError_t e = cudaMalloc(&blk, o);
    if (e != cudaSuccess) {
        delete s;
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return SFCI_E_NOMEM;
    }
    e = cudaMalloc(&s->dev_status, 256);
    if (e == cudaSuccess) e = cudaMemcpy(blk + off_h, h_host, nh * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(blk + off_g, g_host, ng * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(blk + off_bt, bt.data(), bt.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(blk + off_p, pairs.data(), pairs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(blk + off_bab, bab.data(), nh * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(blk + off_bss, bss.data(), nh * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && fp32) e = cudaMemcpy(blk + off_hf, hf.data(), nh * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && fp32) e = cudaMemcpy(blk + off_gf, gf.data(), ng * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(blk);
        if (s->dev_status) cudaFree(s->dev_status);
        delete s;
        return cuda_fail(e, "sfci_system_create");
    }
    d.h = reinterpret_cast<const double *>(blk + off_h);
    d.g = reinterpret_cast<const double *>(blk + off_g);
    d.binom = reinterpret_cast<const unsigned long long *>(blk + off_bt);
    d.pairs = reinterpret_cast<const unsigned char *>(blk + off_p);
    d.hf = fp32 ? reinterpret_cast<const float *>(blk + off_hf) : nullptr;
    d.gf = fp32 ? reinterpret_cast<const float *>(blk + off_gf) : nullptr;
    {
        // |<D'|H|D>| <= |e_core| + N max|h| + N^2 max|g| (diagonal, singles and doubles)
        double mh = 0.0, mg = 0.0;
        for (size_t i = 0; i < nh; ++i) mh = std::max(mh, std::fabs(h_host[i]));
        for (size_t i = 0; i < ng; ++i) mg = std::max(mg, std::fabs(g_host[i]));
        const double N = (double)(na + nb);
        d.hbound = (std::fabs(e_core) + N * mh + N * N * mg) * (1.0 + 1e-6);
    }
    d.bound_ab = reinterpret_cast<const double *>(blk + off_bab);
    d.bound_ss = reinterpret_cast<const double *>(blk + off_bss);
    d.ss_any = std::any_of(bss.begin(), bss.end(), [](double x) { return x != 0.0; }) ? 1 : 0;
    s->d = d;
    s->dev_block = blk;
    *out = s;
    return SFCI_OK;
}

sfci_status sfci_system_destroy(sfci_system *s) {
    if (!s) return SFCI_OK;
    cudaFree(s->dev_block);
    cudaFree(s->dev_status);
    delete s;
    return SFCI_OK;
}

sfci_status sfci_dim(const sfci_system *s, uint64_t *dim) {
    if (check_sys(s) || !dim) return invalid("null argument");
    *dim = s->d.dim;
    return SFCI_OK;
}

sfci_status sfci_n_connected(const sfci_system *s, int64_t *n_conn) {
    if (check_sys(s) || !n_conn) return invalid("null argument");
    *n_conn = s->d.n_conn;
    return SFCI_OK;
}

sfci_status sfci_rank(const sfci_system *s, const uint64_t *alpha, const uint64_t *beta,
                      uint64_t *rank, int64_t count, void *stream) {
    if (check_sys(s)) return SFCI_E_INVALID;
    if (count < 0 || (count > 0 && (!alpha || !beta || !rank))) return invalid("bad arguments");
    if (count == 0) return SFCI_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SFCI_CUDA(cudaMemsetAsync(s->dev_status, 0, sizeof(int), st));
    SFCI_CUDA(launch_rank(s->d, reinterpret_cast<const unsigned long long *>(alpha),
                          reinterpret_cast<const unsigned long long *>(beta),
                          reinterpret_cast<unsigned long long *>(rank), count, s->dev_status, st));
    int flag = 0;
    SFCI_CUDA(cudaMemcpyAsync(&flag, s->dev_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaStreamSynchronize(st));
    if (flag) return invalid("a spin string has the wrong electron count or orbitals >= n");
    return SFCI_OK;
}

sfci_status sfci_unrank(const sfci_system *s, const uint64_t *rank, uint64_t *alpha,
                        uint64_t *beta, int64_t count, void *stream) {
    if (check_sys(s)) return SFCI_E_INVALID;
    if (count < 0 || (count > 0 && (!alpha || !beta || !rank))) return invalid("bad arguments");
    if (count == 0) return SFCI_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SFCI_CUDA(cudaMemsetAsync(s->dev_status, 0, sizeof(int), st));
    SFCI_CUDA(launch_unrank(s->d, reinterpret_cast<const unsigned long long *>(rank),
                            reinterpret_cast<unsigned long long *>(alpha),
                            reinterpret_cast<unsigned long long *>(beta), count, s->dev_status, st));
    int flag = 0;
    SFCI_CUDA(cudaMemcpyAsync(&flag, s->dev_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaStreamSynchronize(st));
    if (flag) return invalid("a rank is >= dim");
    return SFCI_OK;
}

sfci_status sfci_sigma_workspace_bytes(const sfci_system *s, int64_t n_in, int64_t out_cap,
                                       size_t *bytes) {
    (void)n_in;
    if (check_sys(s) || !bytes || out_cap < 0) return invalid("bad arguments");
    *bytes = sigma_layout(out_cap).bytes;
    return SFCI_OK;
}

sfci_status sfci_sigma(const sfci_system *s, const uint64_t *in_rank, const double *in_coef,
                       int64_t n_in, double eps_screen, uint64_t *out_rank, double *out_coef,
                       int64_t out_cap, int64_t *n_out, void *workspace, size_t ws_bytes,
                       void *stream) {
    if (check_sys(s)) return SFCI_E_INVALID;
    if (!n_out || n_in < 0 || out_cap < 0) return invalid("bad arguments");
    if (n_in > 0 && (!in_rank || !in_coef)) return invalid("null input vector");
    if (out_cap > 0 && (!out_rank || !out_coef)) return invalid("null output vector");
    const SigmaLayout L = sigma_layout(out_cap);
    if (!workspace || ws_bytes < L.bytes) {
        set_error("workspace smaller than sfci_sigma_workspace_bytes");
        *n_out = 0;
        return SFCI_E_CAPACITY;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(workspace);
    Table t;
    t.slots = reinterpret_cast<Slot *>(w + L.table);
    t.mask = L.slots - 1;
    t.shift = 64 - __builtin_ctzll(L.slots);
    t.status = reinterpret_cast<int *>(w + L.status);
    t.count = reinterpret_cast<unsigned long long *>(w + L.count);
    unsigned long long *ndev = reinterpret_cast<unsigned long long *>(w + L.ndev);
    int *flag = reinterpret_cast<int *>(w + L.flag);
    const unsigned long long *ir = reinterpret_cast<const unsigned long long *>(in_rank);
    SFCI_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    SFCI_CUDA(validate_sorted(ir, n_in, s->d.dim, flag, st));
    // exact sums: units 2^-S with no entry beyond (n_conn + 1) hbound max|c| < 2^125 units
    unsigned long long mbits = 0;
    SFCI_CUDA(max_abs_bits(in_coef, n_in, reinterpret_cast<unsigned long long *>(w + L.maxabs), st));
    SFCI_CUDA(cudaMemcpyAsync(&mbits, w + L.maxabs, 8, cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaStreamSynchronize(st));
    double cmax = 0.0;
    std::memcpy(&cmax, &mbits, 8);
    if (!std::isfinite(cmax)) return invalid("non-finite input coefficients");
    t.acc = reinterpret_cast<unsigned long long *>(w + L.acc);
    t.fix_shift = (int)std::floor(125.0 - std::log2(std::max(1e-300, (double)(s->d.n_conn + 1) * s->d.hbound *
                                                                         std::max(cmax, 1e-300))));
    t.fix_shift = std::max(-900, std::min(1000, t.fix_shift));
    SFCI_CUDA(table_clear(t, st));
    SFCI_CUDA(launch_emit(s->d, ir, in_coef, n_in, t, st));
    SFCI_CUDA(table_finalize_exact(t, st));
    SFCI_CUDA(table_extract(t, eps_screen > 0.0 ? eps_screen : 0.0,
                            reinterpret_cast<unsigned long long *>(out_rank), out_coef, out_cap,
                            ndev, st));
    SFCI_CUDA(sort_pairs(reinterpret_cast<unsigned long long *>(out_rank), out_coef, out_cap, ndev,
                         key_bits(s->d.dim), w + L.sortws, st));
    int hflag = 0, hstatus = 0;
    unsigned long long hn = 0, hcount = 0;
    SFCI_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaMemcpyAsync(&hstatus, t.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaMemcpyAsync(&hn, ndev, sizeof(hn), cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaMemcpyAsync(&hcount, t.count, sizeof(hcount), cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaStreamSynchronize(st));
    if (hflag) {
        *n_out = 0;
        return invalid("input ranks must be strictly ascending and below dim");
    }
    if (hstatus & 2) {
        *n_out = 0;
        return invalid("an element fell outside the fixed-point range of the exact sums");
    }
    if (hstatus & 1) {
        *n_out = (int64_t)(hcount + 1);
        set_error("sigma has more entries than the workspace table holds; raise out_cap");
        return SFCI_E_CAPACITY;
    }
    *n_out = (int64_t)hn;
    if ((long long)hn > out_cap) {
        set_error("sigma has more entries than out_cap");
        return SFCI_E_CAPACITY;
    }
    return SFCI_OK;
}

sfci_status sfci_truncate_topk_workspace_bytes(int64_t n, int64_t k, size_t *bytes) {
    if (!bytes || n < 0 || k < 0) return invalid("bad arguments");
    *bytes = topk_layout(n, k).bytes;
    return SFCI_OK;
}

sfci_status sfci_truncate_topk(const uint64_t *rank, const double *coef, int64_t n, int64_t k,
                               int normalize, uint64_t *out_rank, double *out_coef,
                               int64_t *n_out, void *workspace, size_t ws_bytes, void *stream) {
    if (!n_out || n < 0 || k < 0) return invalid("bad arguments");
    if (n > 0 && (!rank || !coef)) return invalid("null input vector");
    if (k > 0 && (!out_rank || !out_coef)) return invalid("null output vector");
    const TopkLayout L = topk_layout(n, k);
    if (!workspace || ws_bytes < L.bytes) {
        set_error("workspace smaller than sfci_truncate_topk_workspace_bytes");
        return SFCI_E_CAPACITY;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(workspace);
    unsigned long long *ndev = reinterpret_cast<unsigned long long *>(w + L.ndev);
    Items it{reinterpret_cast<const unsigned long long *>(rank), coef, 1, n};
    unsigned long long *ok = reinterpret_cast<unsigned long long *>(out_rank);
    SFCI_CUDA(select_topk(it, k, ok, out_coef, ndev, nullptr, nullptr, w + L.sel,
                          select_workspace_bytes(n, k), st));
    SFCI_CUDA(sort_pairs(ok, out_coef, k, ndev, 64, w + L.sort, st));
    if (normalize) SFCI_CUDA(normalize_vec(out_coef, k, ndev, w + L.norm, st));
    unsigned long long hn = 0;
    SFCI_CUDA(cudaMemcpyAsync(&hn, ndev, sizeof(hn), cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaStreamSynchronize(st));
    if ((long long)hn > k) {
        *n_out = k;
        return invalid("duplicate ranks in the input");
    }
    *n_out = (int64_t)hn;
    return SFCI_OK;
}

sfci_status sfci_debug_excitations(const sfci_system *s, const uint64_t *rank, int64_t n,
                                   int64_t *src, uint64_t *tgt, double *elem, int64_t cap,
                                   int64_t *n_out, void *stream) {
    if (check_sys(s)) return SFCI_E_INVALID;
    if (!n_out || n < 0) return invalid("bad arguments");
    const long long need = n * (s->d.n_conn + 1);
    *n_out = need;
    if (need > cap) {
        set_error("cap below n * (n_conn + 1)");
        return SFCI_E_CAPACITY;
    }
    if (n == 0) return SFCI_OK;
    if (!rank || !src || !tgt || !elem) return invalid("null pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *flag = s->dev_status;
    SFCI_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    SFCI_CUDA(validate_sorted(reinterpret_cast<const unsigned long long *>(rank), n, s->d.dim, flag, st));
    SFCI_CUDA(launch_debug_excitations(s->d, reinterpret_cast<const unsigned long long *>(rank), n,
                                       reinterpret_cast<long long *>(src),
                                       reinterpret_cast<unsigned long long *>(tgt), elem, st));
    int hflag = 0;
    SFCI_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaStreamSynchronize(st));
    if (hflag) return invalid("input ranks must be strictly ascending and below dim");
    return SFCI_OK;
}

}  // extern "C"
