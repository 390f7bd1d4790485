// Fixed-size device memory for callers that cannot allocate device memory.
//
// The array below is part of the library image: every GPU that loads
// libsmx.so holds it until the process exits.  Host code must not use the
// symbol's host-side name as a device address; noalloc_region() looks up the
// real device address once per device (with that device current) and caches it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/smx.h"

namespace smx {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SMX_NOALLOC_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_base[kMaxDevices] = {nullptr};
uint64_t g_owner[kMaxDevices] = {0};
}  // namespace

// Device address of the static array on the current device (looked up on the
// first call for that device) and the id of the context whose tables it holds.
int noalloc_region(void** base, uint64_t** owner) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SMX_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return SMX_EINVAL;
    std::lock_guard<std::mutex> guard(g_lock);
    if (g_base[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return SMX_ECUDA;
        g_base[dev] = p;
    }
    *base = g_base[dev];
    *owner = &g_owner[dev];
    return SMX_OK;
}

}  // namespace smx
