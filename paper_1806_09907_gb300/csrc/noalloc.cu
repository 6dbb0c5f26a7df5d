// al_similarity_noalloc: the similarity step (A3) for callers that cannot
// allocate device memory.
//
// Some hosts cannot hand this library a workspace: their device memory is
// owned by another allocator (a framework's caching pool that must see every
// allocation, or an embedded runtime that forbids allocation after start-up),
// or they are plain C programs with no device allocator of their own. For
// them this entry point takes its scratch from a fixed array that lives in
// the library's own device memory instead of a caller workspace. It calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// The array holds kNoAllocScratchBytes (4 MiB) on every GPU that loads the
// library, for the lifetime of the process. Every call on a device shares
// it, and a call leaves its contents behind: two calls whose kernels overlap
// on the GPU (different streams without ordering) race on it, so order them.
// The kernels overwrite every scratch word they read, so nothing needs to be
// cleared between calls.
//
// Host code may not use the array's name as a device address (in host code
// it is a host-side stand-in). The first call on each device looks up the
// device address with cudaGetSymbolAddress, with that device current, and
// caches it; make that first call before any stream capture.
#include <mutex>

#include "airgb.h"
#include "checks.h"
#include "launch.h"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)4 << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once).
al_status scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return AL_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices)
        return AL_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
            return AL_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return AL_OK;
}

}  // namespace

extern "C" {

size_t al_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

al_status al_similarity_noalloc(const al_grid *g, const al_sim_params *p, const float *fixed,
                                const float *warped, const uint8_t *mask, double *value_dev,
                                float *grad_warped, al_stream stream)
{
    const size_t need = al_similarity_workspace_bytes(g, p);
    if (need == 0) {
        // invalid grid or parameters: let the regular entry point report which
        return al_similarity(g, p, fixed, warped, mask, value_dev, grad_warped, nullptr, 0,
                             stream);
    }
    if (need > kNoAllocScratchBytes)
        return AL_ERR_SCRATCH_LIMIT;
    // the pointer checks of al_similarity, before the address lookup (which
    // is the first CUDA call)
    if (!fixed || !warped || !mask || !value_dev)
        return AL_ERR_INVALID_ARG;
    if (!airgb::aligned16(fixed) || !airgb::aligned16(warped) || !airgb::aligned16(mask) ||
        !airgb::aligned16(value_dev) || (grad_warped && !airgb::aligned16(grad_warped)))
        return AL_ERR_ALIGN;
    void *scratch = nullptr;
    const al_status st = scratch_address(&scratch);
    if (st != AL_OK)
        return st;
    return al_similarity(g, p, fixed, warped, mask, value_dev, grad_warped, scratch,
                         kNoAllocScratchBytes, stream);
}

}  // extern "C"
