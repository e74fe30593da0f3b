// Every device and page-locked host allocation of the library goes through
// the wrappers below (dmalloc, dmalloc_async, hmalloc and their frees).  They
// keep a table of the live allocations, and a test hook can make the n-th
// next allocation fail as if the device were out of memory, so that a test
// can check that each entry point returns SBG_ERR_OOM and releases whatever
// it had allocated before the failure (the live table returns to where it
// was).  No fault is caused on the device: the failing call simply does not
// allocate.
#include <atomic>
#include <mutex>
#include <unordered_map>

#include "sbg_internal.cuh"

namespace sbg {

static std::atomic<int64_t> g_fail_countdown{0};  // > 0: allocations left until the failing one
static std::mutex g_live_mu;
static std::unordered_map<void *, size_t> g_live;  // live allocation -> bytes
static int64_t g_live_bytes = 0;

// true when this allocation is the one the hook makes fail
static bool take_fault() {
    int64_t c = g_fail_countdown.load();
    while (c > 0) {
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    }
    return false;
}

static void track(void *p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_live_mu);
    g_live[p] = bytes;
    g_live_bytes += (int64_t)bytes;
}

static void untrack(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_live_mu);
    auto it = g_live.find(p);
    if (it == g_live.end()) return;
    g_live_bytes -= (int64_t)it->second;
    g_live.erase(it);
}

cudaError_t dmalloc(void **p, size_t bytes) {
    if (take_fault()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) track(*p, bytes);
    return e;
}

cudaError_t dmalloc_async(void **p, size_t bytes, cudaStream_t s) {
    if (take_fault()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaSuccess) track(*p, bytes);
    return e;
}

cudaError_t hmalloc(void **p, size_t bytes) {
    if (take_fault()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) track(*p, bytes);
    return e;
}

cudaError_t dfree(void *p) {
    if (!p) return cudaSuccess;
    untrack(p);
    return cudaFree(p);
}

cudaError_t dfree_async(void *p, cudaStream_t s) {
    if (!p) return cudaSuccess;
    untrack(p);
    return cudaFreeAsync(p, s);
}

cudaError_t hfree(void *p) {
    if (!p) return cudaSuccess;
    untrack(p);
    return cudaFreeHost(p);
}

}  // namespace sbg

using namespace sbg;

extern "C" sbg_status sbg_debug_fail_alloc(int64_t n) {
    if (n < 0) return fail(SBG_ERR_INVALID_ARG, "sbg_debug_fail_alloc: n >= 0");
    g_fail_countdown.store(n);
    return SBG_OK;
}

extern "C" sbg_status sbg_debug_live_allocations(int64_t *count, int64_t *bytes) {
    std::lock_guard<std::mutex> lk(g_live_mu);
    if (count) *count = (int64_t)g_live.size();
    if (bytes) *bytes = g_live_bytes;
    return SBG_OK;
}
