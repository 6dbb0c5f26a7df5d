// Per-kernel timing hooks (no-ops unless al_profile_enable(1) was called).
#pragma once

#include <cuda_runtime.h>

namespace airgb {

// Record a start event named `name` on stream s before a launch, and the
// matching stop event after it. Names must be string literals.
void prof_begin(cudaStream_t s, const char *name);
void prof_end(cudaStream_t s);

struct ProfScope {
    cudaStream_t s;
    ProfScope(cudaStream_t st, const char *name) : s(st) { prof_begin(st, name); }
    ~ProfScope() { prof_end(s); }
};

}  // namespace airgb
