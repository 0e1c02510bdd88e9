// Device memory of the engine's handles (sweeps, batches, surrogates): the
// default cudaMalloc / cudaFree, or a caller's pair installed with
// tvbx_set_allocator. Each buffer remembers the pair that allocated it and is
// released through that pair.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "tvbx.h"

namespace tvbx {

struct DevAllocator {
    tvbx_alloc_fn alloc = nullptr;   // nullptr: cudaMalloc / cudaFree
    tvbx_free_fn free = nullptr;
    void* ctx = nullptr;
};

// The pair in force now.
DevAllocator current_allocator();

// Allocate bytes (> 0) with the pair in force; *used receives that pair.
// cudaErrorMemoryAllocation when the caller's allocator returns NULL.
cudaError_t dev_alloc(void** p, size_t bytes, DevAllocator* used);

// Release p (nullable) through the pair that allocated it. With a caller's
// pair the device is synchronised first: a caching allocator may hand the
// block out again at once, while queued work could still be using it.
void dev_free(void* p, const DevAllocator& used);

}  // namespace tvbx
