// Eq. 11 truncation for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs while another
// framework owns every byte of the device through its own pool, a driver or
// plugin that is handed a fixed memory budget, or a loop that must not touch
// the allocator between steps.  They cannot size and pass the workspace that
// sfci_truncate_topk wants, so this entry point runs the same selection, sort
// and normalisation with its scratch in a fixed array of this file.
//
// The array is a file-scope __device__ variable: the CUDA runtime places it
// in device memory with the module, so neither this call nor the kernels it
// launches allocate.  Its address is looked up once per device, by the first
// call made with that device current, and cached.
#include <mutex>

#include "sfci_internal.cuh"

// scratch of the no-allocation top-k: 20 MiB, enough for k <= 2^20
static __device__ __align__(256) unsigned char sfci_topk_scratch[size_t(20) << 20];

namespace sfci {
namespace {

constexpr size_t kScratchBytes = size_t(20) << 20;
constexpr long long kMaxK = 1ll << 20;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
void *g_ptr[kMaxDevices];

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t sel, sel_bytes, sort, norm, ndev, bytes;
};

Layout layout(long long n, long long k) {
    Layout L{};
    size_t o = 0;
    L.sel = o, L.sel_bytes = select_workspace_bytes(n, k), o = a256(o + L.sel_bytes);
    L.sort = o, o = a256(o + sort_pairs_bytes(k > 0 ? k : 1));
    L.norm = o, o = a256(o + normalize_ws_bytes(k));
    L.ndev = o, o = a256(o + sizeof(unsigned long long));
    L.bytes = o;
    return L;
}

// device address of the scratch on the current device (first call per device
// looks it up)
sfci_status scratch_ptr(char **out) {
    int dev = -1;
    SFCI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal beyond the 64 devices the scratch table covers");
        return SFCI_E_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        SFCI_CUDA(cudaGetSymbolAddress(&p, sfci_topk_scratch));
        g_ptr[dev] = p;
    }
    *out = static_cast<char *>(g_ptr[dev]);
    return SFCI_OK;
}

}  // namespace
}  // namespace sfci

using namespace sfci;

extern "C" {

sfci_status sfci_truncate_topk_noalloc(const uint64_t *rank, const double *coef, int64_t n,
                                       int64_t k, int normalize, uint64_t *out_rank,
                                       double *out_coef, int64_t *n_out, void *stream) {
    if (!n_out || n < 0 || k < 0) {
        set_error("bad arguments");
        return SFCI_E_INVALID;
    }
    if ((n > 0 && (!rank || !coef)) || (k > 0 && (!out_rank || !out_coef))) {
        set_error("null vector");
        return SFCI_E_INVALID;
    }
    if (k > kMaxK) {
        set_error("k = " + std::to_string(k) + " is above 1048576, the most the fixed 20 MiB "
                  "scratch of sfci_truncate_topk_noalloc holds; use sfci_truncate_topk");
        return SFCI_E_CAPACITY;
    }
    const Layout L = layout(n, k);
    if (L.bytes > kScratchBytes) {
        set_error("scratch need exceeds the fixed 20 MiB");
        return SFCI_E_CAPACITY;
    }
    char *w = nullptr;
    const sfci_status s = scratch_ptr(&w);
    if (s != SFCI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the selection state, its histogram and the kept count start at zero
    SFCI_CUDA(cudaMemsetAsync(w + L.sel, 0, L.sel_bytes, st));
    SFCI_CUDA(cudaMemsetAsync(w + L.ndev, 0, sizeof(unsigned long long), st));
    unsigned long long *ndev = reinterpret_cast<unsigned long long *>(w + L.ndev);
    Items it{reinterpret_cast<const unsigned long long *>(rank), coef, 1, n};
    unsigned long long *ok = reinterpret_cast<unsigned long long *>(out_rank);
    SFCI_CUDA(select_topk(it, k, ok, out_coef, ndev, nullptr, nullptr, w + L.sel, L.sel_bytes, st));
    SFCI_CUDA(sort_pairs(ok, out_coef, k, ndev, 64, w + L.sort, st));
    if (normalize) SFCI_CUDA(normalize_vec(out_coef, k, ndev, w + L.norm, st));
    unsigned long long hn = 0;
    SFCI_CUDA(cudaMemcpyAsync(&hn, ndev, sizeof(hn), cudaMemcpyDeviceToHost, st));
    SFCI_CUDA(cudaStreamSynchronize(st));
    if ((long long)hn > k) {
        *n_out = k;
        set_error("duplicate ranks in the input");
        return SFCI_E_INVALID;
    }
    *n_out = (int64_t)hn;
    return SFCI_OK;
}

}  // extern "C"
