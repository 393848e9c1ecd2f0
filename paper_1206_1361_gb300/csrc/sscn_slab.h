// sscn_slab.h -- the fused x + y sweep over z-planes held in shared memory
// (sscn_slab.cu), as the host API calls it.
#pragma once

#include <cstddef>

#include "sscn_internal.h"

namespace gp {

// Shared memory one plane takes (ny rows of nx | 1 points), whether a plane
// fits one CTA, and the launch: calcnu (tables in x, y, z order) with the x
// sweep, then the y sweep, one CTA per plane, no norm partials.
// A plane larger than one CTA's shared memory is split over a 2-CTA cluster
// (split_bytes per CTA: half the rows, a halo row, two exchange rows).
size_t slab_bytes(int prec, int nx, int ny);
size_t split_bytes(int prec, int nx, int ny);
bool slab_split(int prec, int nx, int ny);
bool slab_fits(int prec, int nx, int ny);
cudaError_t launch_sweep_xy(int prec, int mode, void *psi, int nx, int ny, int nz,
                            const AxisTables &ax, const AxisTables &ay, const NonlinArgs &nl,
                            cudaStream_t st);

}  // namespace gp
