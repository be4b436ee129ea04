// fse_alloc.cuh -- every device and pinned-host allocation of the library
// goes through these wrappers, so that tests can make one of them fail (as
// if memory were exhausted) and count what the library holds.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace fse {

cudaError_t dev_malloc_raw(void **p, size_t n);
cudaError_t dev_free(void *p);
cudaError_t host_malloc_raw(void **p, size_t n);
cudaError_t host_free(void *p);

template <typename T>
inline cudaError_t dev_malloc(T **p, size_t n) {
    return dev_malloc_raw(reinterpret_cast<void **>(p), n);
}
template <typename T>
inline cudaError_t host_malloc(T **p, size_t n) {
    return host_malloc_raw(reinterpret_cast<void **>(p), n);
}

}  // namespace fse
