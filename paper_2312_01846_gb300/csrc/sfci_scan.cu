// Batched scan: many independent SFCI problems (a scan along a geometry-like
// parameter: uneven orbital counts, electron counts and N_d) advanced together.
//
// Each instance owns an sfci_lanczos solver on its own non-blocking stream.
// A step of the scan is one sfci_lanczos_step of every instance; a pool of
// host worker threads pulls instances from a shared queue, largest expected
// work first, so the kernels of different instances overlap on the GPU and the
// host-side planning of one instance hides behind the device work of others.
// Every instance gets a share of device memory for its sigma buffers in
// proportion to its expected intermediate elements per step.
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sfci_internal.cuh"

struct sfci_scan {
    int device = 0;
    int count = 0;
    std::vector<sfci_lanczos *> lz;
    std::vector<cudaStream_t> streams;
    std::vector<int> order;      // instances, largest expected work first
    std::vector<sfci_step_info> info;
    std::vector<sfci_status> status;
    std::vector<std::string> error;
    // worker pool
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_go, cv_done;
    long long generation = 0;   // bumped per step
    int running = 0;            // workers still busy in this step
    bool quit = false;
    std::atomic<int> next{0};   // position in `order`
};

namespace {

void worker_main(sfci_scan *s) {
    cudaSetDevice(s->device);
    long long seen = 0;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_go.wait(lk, [&] { return s->quit || s->generation != seen; });
            if (s->quit) return;
            seen = s->generation;
        }
        for (;;) {
            const int k = s->next.fetch_add(1);
            if (k >= s->count) break;
            const int i = s->order[k];
            s->status[i] = sfci_lanczos_step(s->lz[i], &s->info[i]);
            if (s->status[i] != SFCI_OK) s->error[i] = sfci_last_error();
        }
        std::lock_guard<std::mutex> lk(s->mu);
        if (--s->running == 0) s->cv_done.notify_all();
    }
}

void destroy_scan(sfci_scan *s) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->quit = true;
    }
    s->cv_go.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto *z : s->lz)
        if (z) sfci_lanczos_destroy(z);
    for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
    delete s;
}

}  // namespace

using namespace sfci;

extern "C" {

sfci_status sfci_scan_create(sfci_scan **out, int32_t count, const sfci_system *const *systems,
                             const sfci_params *params, const uint64_t *const *init_rank,
                             const double *const *init_coef, const int64_t *n_init,
                             int32_t workers) {
    if (!out || count < 1 || !systems || !params || !init_rank || !init_coef || !n_init) {
        set_error("null argument or count < 1");
        return SFCI_E_INVALID;
    }
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        if (!systems[i]) {
            set_error("null system in the scan");
            return SFCI_E_INVALID;
        }
        if (systems[i]->device != systems[0]->device) {
            set_error("all systems of a scan must live on one device");
            return SFCI_E_INVALID;
        }
    }
    sfci_scan *s = new (std::nothrow) sfci_scan();
    if (!s) return SFCI_E_NOMEM;
    s->device = systems[0]->device;
    s->count = count;
    s->lz.assign(count, nullptr);
    s->streams.assign(count, nullptr);
    s->info.assign(count, sfci_step_info{});
    s->status.assign(count, SFCI_OK);
    s->error.assign(count, std::string());
    const cudaError_t e0 = cudaSetDevice(s->device);
    if (e0 != cudaSuccess) {
        delete s;
        return cuda_fail(e0, "sfci_scan_create");
    }
    // expected intermediate elements per step: N_d (n_conn + 1)
    std::vector<double> work(count);
    double total = 0.0;
    for (int i = 0; i < count; ++i) {
        work[i] = (double)params[i].n_keep * (double)(systems[i]->d.n_conn + 1);
        total += work[i];
    }
    size_t free_b = 0, tot_b = 0;
    cudaMemGetInfo(&free_b, &tot_b);
    for (int i = 0; i < count; ++i) {
        sfci_params p = params[i];
        if (p.mem_budget == 0)  // a share of 80 % of what is free now
            p.mem_budget = (int64_t)(0.8 * (double)free_b * work[i] / total);
        cudaError_t e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            destroy_scan(s);
            return cuda_fail(e, "sfci_scan_create");
        }
        const sfci_status r = sfci_lanczos_create(&s->lz[i], systems[i], &p, init_rank[i], init_coef[i],
                                                  n_init[i], s->streams[i]);
        if (r != SFCI_OK) {
            const std::string msg = "instance " + std::to_string(i) + ": " + sfci_last_error();
            destroy_scan(s);
            set_error(msg);
            return r;
        }
    }
    s->order.resize(count);
    for (int i = 0; i < count; ++i) s->order[i] = i;
    std::stable_sort(s->order.begin(), s->order.end(), [&](int a, int b) { return work[a] > work[b]; });
    int nw = workers > 0 ? workers : std::min(count, 8);
    nw = std::max(1, std::min(nw, count));
    try {
        for (int w = 0; w < nw; ++w) s->workers.emplace_back(worker_main, s);
    } catch (...) {
        destroy_scan(s);
        set_error("could not start the worker threads");
        return SFCI_E_NOMEM;
    }
    *out = s;
    return SFCI_OK;
}

sfci_status sfci_scan_step(sfci_scan *s, sfci_step_info *infos) {
    if (!s || !infos) {
        set_error("null argument");
        return SFCI_E_INVALID;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->next.store(0);
        s->running = (int)s->workers.size();
        ++s->generation;
    }
    s->cv_go.notify_all();
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] { return s->running == 0; });
    }
    std::memcpy(infos, s->info.data(), sizeof(sfci_step_info) * s->count);
    for (int i = 0; i < s->count; ++i)
        if (s->status[i] != SFCI_OK) {
            set_error("instance " + std::to_string(i) + ": " + s->error[i]);
            return s->status[i];
        }
    return SFCI_OK;
}

sfci_status sfci_scan_solver(sfci_scan *s, int32_t i, sfci_lanczos **out) {
    if (!s || !out || i < 0 || i >= s->count) {
        set_error("bad scan index");
        return SFCI_E_INVALID;
    }
    *out = s->lz[i];
    return SFCI_OK;
}

sfci_status sfci_scan_destroy(sfci_scan *s) {
    if (!s) return SFCI_OK;
    destroy_scan(s);
    return SFCI_OK;
}

}  // extern "C"
