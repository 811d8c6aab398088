// Batched multi-tree engine (internal): one persistent kernel evaluates many trees, each on its
// own map and sensor, level by level with device-side dependencies (Sec. IV-C per tree).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kernels.h"
#include "mig_impl.h"

namespace mig {

// Per tree, in device memory: the tree's level parameters (pointers into the batch workspace)
// and the index of its level 0 in the per-(tree, level) counter arrays.
struct BatchTree {
    LevelParams p;
    int lvl_base;
    int n_levels;
};

// Work of one tree level is two segments: its count items (node, yaw, tile) and its render items
// (internal node, 32 pixels). Segment id = 2 * (lvl_base[tree] + level) + phase. A segment becomes
// ready (is "activated") when its dependencies are complete: the count segment of level d when
// level d-1 is complete, the render segment when the level's yaws are selected. Activation
// appends the segment to a log and gives it the next range of global item numbers; warps take
// item numbers from one counter and only ever receive ready work.
struct SegInfo {
    int tree;
    int level;
    int render;
    int items;
};

// Trees per persistent launch: their parameters travel in the kernel's parameter space (constant
// bank, up to 32 KB), indexed by the warp-uniform tree number. Larger batches use several launches.
constexpr int kBatchMaxTrees = 96;

struct BatchParams {
    const SegInfo *segs;        // by segment id
    int n_levels_total;
    long long total_items;      // of all segments of this launch
    unsigned long long *act;    // (log entries << 40) | activated items
    int2 *log;                  // per entry: (first item, segment id)
    int *log_valid;             // per entry: written (release flag)
    long long *work;            // global item counter
    int *count_left;            // per (tree, level): count items not finished
    int *render_left;           // per (tree, level): render items not finished
    int *status;                // [0] abort, [1] a wait timed out
    unsigned long long timeout_ns;
    unsigned long long *trace;  // NULL, or per segment (activated, completed) %globaltimer ns + kernel start
    int n_segs_total;
    int max_anc;                // ancestor records per warp: the deepest tree's depth (dynamic smem)
    BatchTree trees[kBatchMaxTrees];
};

void launch_batch(const BatchParams &bp, int grid, cudaStream_t s);
size_t batch_dyn_smem(int max_anc);
int batch_ctas_per_sm();

// Host-side description of one tree of a batch (or of a served request).
struct BatchItem {
    mig_map *map = nullptr;
    int n = 0;
    const int32_t *parent = nullptr;
    const float *pos = nullptr;
    mig_sensor sensor{};
    int mode = 0;
    int32_t *out_abs = nullptr, *out_marg = nullptr, *out_yaw = nullptr;  // host destinations
    HostPlan plan;
    const Camera *cam = nullptr;
    int level_lo = 0, level_hi = -1;  // levels evaluated by a launch
};

}  // namespace mig
