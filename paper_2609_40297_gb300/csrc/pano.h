// Panoramic-mode passes (internal): one 360-degree cast per node, then per-yaw window sums.
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace mig {

// Per-(node, column) absolute and marginal counts of one level into p.pano_cnt (work items from
// p.work[p.lvl]); then each yaw's window sums into p.cnt, ready for launch_select.
void launch_pano_count(const LevelParams &p, int grid, cudaStream_t s);
void launch_pano_window(const LevelParams &p, int grid, cudaStream_t s);
int pano_ctas_per_sm();  // also lifts the count kernel's dynamic shared-memory limit; call once

}  // namespace mig
