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
// it is a host-side stand-in). The first call in each context of a device
// looks up the device address with cudaGetSymbolAddress, with that device
// current, and caches it together with the context's id: after a device
// reset (a new primary context, where the module and the array may move) the
// next call looks the address up again. Make the first call of a context
// before any stream capture.
#include <cuda.h>

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
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Id of the current context (driver entry points looked up once through the
// runtime); 0 when it cannot be read, which forces a fresh lookup.
unsigned long long current_ctx_id()
{
    using GetCur = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCur get_cur = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<GetCur>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(p);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx ||
        get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_noalloc_scratch in the current context of the current
// device (looked up once per context). A failed runtime call's error is
// cleared before returning, so later calls do not see it.
al_status scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return AL_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices)
        return AL_ERR_UNSUPPORTED;
    // 0 before the runtime has made a context current: then the lookup below
    // (which does) runs and the id is read after it
    const unsigned long long ctx = current_ctx_id();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            g_scratch_addr[dev] = nullptr;
            return AL_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx != 0 ? ctx : current_ctx_id();
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
