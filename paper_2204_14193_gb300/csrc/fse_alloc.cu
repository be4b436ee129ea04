// fse_alloc.cu -- the library's allocation wrappers and their test hooks
// (fse_test_fail_allocation, fse_test_live_allocations in include/fse.h).
#include <atomic>

#include "fse.h"
#include "fse_alloc.cuh"

namespace {
std::atomic<int> g_countdown{0};         // > 0: the allocation that brings it to 0 fails
std::atomic<long long> g_live{0};        // allocations held (device + pinned host)

bool injected_failure() {
    int c = g_countdown.load();
    while (c > 0 && !g_countdown.compare_exchange_weak(c, c - 1)) {
    }
    return c == 1;
}
}  // namespace

namespace fse {

cudaError_t dev_malloc_raw(void **p, size_t n) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(p, n);
    if (e == cudaSuccess) ++g_live;
    return e;
}

cudaError_t dev_free(void *p) {
    if (!p) return cudaSuccess;
    const cudaError_t e = cudaFree(p);
    if (e == cudaSuccess) --g_live;
    return e;
}

cudaError_t host_malloc_raw(void **p, size_t n) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMallocHost(p, n);
    if (e == cudaSuccess) ++g_live;
    return e;
}

cudaError_t host_free(void *p) {
    if (!p) return cudaSuccess;
    const cudaError_t e = cudaFreeHost(p);
    if (e == cudaSuccess) --g_live;
    return e;
}

}  // namespace fse

extern "C" void fse_test_fail_allocation(int n) { g_countdown.store(n > 0 ? n : 0); }

extern "C" long long fse_test_live_allocations(void) { return g_live.load(); }
