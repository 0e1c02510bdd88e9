// Process-wide choice of the allocator behind the handles' device buffers.

#include <mutex>

#include "alloc.h"
#include "internal.h"

namespace tvbx {
namespace {

std::mutex g_alloc_mutex;
DevAllocator g_alloc;

}  // namespace

DevAllocator current_allocator()
{
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    return g_alloc;
}

cudaError_t dev_alloc(void** p, size_t bytes, DevAllocator* used)
{
    const DevAllocator a = current_allocator();
    *used = a;
    *p = nullptr;
    if (!a.alloc) {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            *p = nullptr;
        }
        return e;
    }
    *p = a.alloc((uint64_t)bytes, a.ctx);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}

void dev_free(void* p, const DevAllocator& used)
{
    if (!p) return;
    if (!used.alloc) {
        cudaFree(p);
        return;
    }
    cudaDeviceSynchronize();
    used.free(p, used.ctx);
}

}  // namespace tvbx

using namespace tvbx;

extern "C" tvbx_status tvbx_set_allocator(tvbx_alloc_fn alloc, tvbx_free_fn free_fn, void* ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr))
        return report_error(TVBX_E_INVALID_ARG, "give both alloc and free, or neither");
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    g_alloc.alloc = alloc;
    g_alloc.free = free_fn;
    g_alloc.ctx = alloc ? ctx : nullptr;
    return TVBX_OK;
}
