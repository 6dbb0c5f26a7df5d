// Host-side argument checks shared by the entry points of libairgb.
#pragma once

#include <cuda_runtime.h>

#include "airgb.h"
#include "common.cuh"

namespace airgb {

bool aligned16(const void *p);
// Checks a grid and fills the kernel descriptor (out may be NULL).
al_status check_grid(const al_grid *g, Grid *out);
// Checks a B-spline transformation against its own grid; fills g and L.
al_status check_bspline(const al_bspline *bs, Grid *g, Lattice *L);
al_status check_sim(const al_sim_params *p, int ndim);
al_status launched(cudaError_t e);

}  // namespace airgb
