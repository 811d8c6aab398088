// Interval-mode count pass (internal): the screen-space overlap test of Sec. IV-B (Eq. 5-7).
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace mig {

// One tree level's counts in the interval mode (p.mode == MIG_MODE_INTERVAL): per owned unknown
// voxel, the union of the ancestors' overlap intervals of the candidate ray decides the exclusion.
// Same work items, counters and outputs as launch_count.
void launch_count_interval(const LevelParams &p, int grid, cudaStream_t s);
int count_interval_ctas_per_sm();

}  // namespace mig
