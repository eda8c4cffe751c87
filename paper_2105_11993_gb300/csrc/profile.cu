// Launch counting and optional CUDA-event timing of kernel classes.
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace thm {

std::atomic<long long> g_launches{0};

namespace {
struct ClassProf {
    int64_t launches = 0;
    double ms = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};
std::mutex g_mu;
unsigned g_mask = 0;
ClassProf g_cls[THM_K_NCLASSES];
std::vector<cudaEvent_t> g_pool;
thread_local cudaEvent_t t_start = nullptr;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    THM_CUDA(cudaEventCreate(&e));
    return e;
}

void drain(ClassProf& c) {
    for (auto& pr : c.pending) {
        THM_CUDA(cudaEventSynchronize(pr.second));
        float t = 0;
        THM_CUDA(cudaEventElapsedTime(&t, pr.first, pr.second));
        c.ms += t;
        g_pool.push_back(pr.first);
        g_pool.push_back(pr.second);
    }
    c.pending.clear();
}
}  // namespace

void prof_begin(int cls, cudaStream_t st) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!(g_mask & (1u << cls))) return;
    std::lock_guard<std::mutex> lk(g_mu);
    t_start = take_event();
    THM_CUDA(cudaEventRecord(t_start, st));
}

void prof_end(int cls, cudaStream_t st) {
    if (!(g_mask & (1u << cls)) || !t_start) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t e = take_event();
    THM_CUDA(cudaEventRecord(e, st));
    ClassProf& c = g_cls[cls];
    c.launches++;
    c.pending.emplace_back(t_start, e);
    t_start = nullptr;
    if (c.pending.size() > 4096) drain(c);
}

void prof_set(unsigned mask) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& c : g_cls) {
        drain(c);
        c.launches = 0;
        c.ms = 0;
    }
    g_mask = mask;
}

void prof_read(int cls, int64_t* launches, double* ms) {
    std::lock_guard<std::mutex> lk(g_mu);
    ClassProf& c = g_cls[cls];
    drain(c);
    if (launches) *launches = c.launches;
    if (ms) *ms = c.ms;
}

}  // namespace thm
