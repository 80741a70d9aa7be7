// The process-wide device allocator of libmaxlink (ml_set_allocator) and the buffer
// lists of the library's objects.
#include <cstdint>
#include <mutex>
#include <string>

#include "devmem.cuh"
#include "grid.cuh"

namespace {

int default_alloc(void **p, size_t bytes, void *stream, void *) {
    if (cudaMallocAsync(p, bytes, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return 1;
    }
    return 0;
}

void default_free(void *p, size_t, void *stream, void *) { cudaFreeAsync(p, (cudaStream_t)stream); }

std::mutex g_mu;
ml_alloc_fn g_alloc = default_alloc;
ml_free_fn g_free = default_free;
void *g_ctx = nullptr;

}  // namespace

ml_status ml_set_allocator(ml_alloc_fn alloc, ml_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr))
        return ml::fail(ML_ERR_INVALID_ARG, "give both allocator functions or neither");
    std::lock_guard<std::mutex> lk(g_mu);
    g_alloc = alloc ? alloc : default_alloc;
    g_free = alloc ? free_fn : default_free;
    g_ctx = alloc ? ctx : nullptr;
    return ML_OK;
}

namespace ml {

ml_status dev_alloc(std::vector<DevBuf> &list, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return ML_OK;
    ml_alloc_fn al;
    ml_free_fn fr;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        al = g_alloc;
        fr = g_free;
        ctx = g_ctx;
    }
    void *q = nullptr;
    if (al(&q, bytes, nullptr, ctx) != 0 || q == nullptr)
        return fail(ML_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    if ((reinterpret_cast<uintptr_t>(q) & 255u) != 0) {
        fr(q, bytes, nullptr, ctx);
        return fail(ML_ERR_CUDA, "the allocator returned memory that is not 256-byte aligned");
    }
    list.push_back(DevBuf{q, bytes, fr, ctx});
    cudaError_t e = cudaMemsetAsync(q, 0, bytes, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ML_ERR_CUDA, std::string("zeroing new device memory: ") + cudaGetErrorString(e));
    }
    *p = q;
    return ML_OK;
}

void dev_release(std::vector<DevBuf> &list, void *p) {
    if (!p) return;
    for (size_t i = 0; i < list.size(); i++)
        if (list[i].p == p) {
            cudaDeviceSynchronize();
            list[i].fr(p, list[i].bytes, nullptr, list[i].ctx);
            list.erase(list.begin() + (long)i);
            return;
        }
}

void dev_free_all(std::vector<DevBuf> &list) {
    if (list.empty()) return;
    cudaDeviceSynchronize();
    for (auto &b : list) b.fr(b.p, b.bytes, nullptr, b.ctx);
    list.clear();
}

}  // namespace ml
