// Device memory of the library's objects, drawn from the process-wide allocator of
// ml_set_allocator (default: cudaMallocAsync / cudaFreeAsync).  Every buffer remembers
// the allocator it came from, so it is returned to that one even if the process
// allocator has been replaced since.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "maxlink.h"

namespace ml {

struct DevBuf {
    void *p;
    size_t bytes;
    ml_free_fn fr;
    void *ctx;
};

// Allocate `bytes` of device memory (nothing for 0), zero it, wait for the zeroing, and
// record the buffer in `list`.  ML_ERR_OOM when the allocator refuses, ML_ERR_CUDA when
// the memory it returned is not 256-byte aligned device memory or cannot be zeroed.
ml_status dev_alloc(std::vector<DevBuf> &list, void **p, size_t bytes);

// Return one buffer of `list` to its allocator, after the device has finished all work,
// and drop it from the list.
void dev_release(std::vector<DevBuf> &list, void *p);

// Return every buffer of `list`, after the device has finished all work.
void dev_free_all(std::vector<DevBuf> &list);

// A list that frees its buffers when it goes out of scope.
struct DevList {
    std::vector<DevBuf> v;
    DevList() = default;
    DevList(const DevList &) = delete;
    DevList &operator=(const DevList &) = delete;
    ~DevList() { dev_free_all(v); }
};

}  // namespace ml
