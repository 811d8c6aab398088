// Batched multi-tree engine (internal): one persistent kernel evaluates many trees, each on its
// own map and sensor, level by level with device-side dependencies (Sec. IV-C per tree).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kernels.h"
#include "mig_impl.h"

namespace mig {

// Per tree, in device memory: the tree's level parameters (pointers into the batch workspace; the
// step-count buffer of its chunks in p.steps).
struct BatchTree {
    LevelParams p;
};

// Work of one tree level is a chain of segments: for each chunk of whole nodes (as many as the
// tree's step-count buffer holds) a cast segment (items: (pair, 8x4 pixel tile)) and then a
// voxel segment (items: (node, slice, 32-row block), the per-node pass), and at the end of the
// level a render segment (items: (internal node, 32 pixels)). A segment becomes ready ("is
// activated") when its predecessor is complete: a voxel segment after its chunk's cast, the next
// chunk's cast after the voxel segment (they share the buffer), the render segment after the last
// voxel segment and the yaw selection of the level, and the next level's first cast after the
// render (the new depth buffers). Activation appends the segment to a log and gives it the next
// range of global item numbers; warps take item numbers from one counter and only ever receive
// ready work.
enum SegKind { kSegCast = 0, kSegVoxel = 1, kSegRender = 2 };
struct SegInfo {
    int tree;
    int level;
    int kind;      // SegKind
    int items;
    int q0, q1;    // cast / voxel: the chunk's (node, yaw) pairs [q0, q1) of the level (whole nodes)
    int next;      // the segment activated when this one completes (-1: the tree is done; the next
                   // waiting tree starts)
    int select;    // voxel segment of the level's last chunk: select the level's yaws first
};

// Trees per persistent launch: their parameters travel in the kernel's parameter space (constant
// bank, up to 32 KB), indexed by the warp-uniform tree number. Larger batches use several launches.
constexpr int kBatchMaxTrees = 96;
// 8x4-pixel cast tiles per work item of a cast segment (one item per warp takes one atomic).
#ifndef MIG_BATCH_CAST_TILES
#define MIG_BATCH_CAST_TILES 16
#endif
constexpr int kBatchCastTiles = MIG_BATCH_CAST_TILES;

struct BatchParams {
    const SegInfo *segs;        // by segment id
    long long total_items;      // of all segments of this launch
    unsigned long long *act;    // (log entries << 40) | activated items
    int2 *log;                  // per entry: (first item, segment id)
    int *log_valid;             // per entry: written (release flag)
    long long *work;            // global item counter
    int *seg_left;              // per segment: items not finished
    int *status;                // [0] abort, [1] a wait timed out
    unsigned long long timeout_ns;
    unsigned long long *trace;  // NULL, or per segment (activated, completed) %globaltimer ns + kernel start
    int n_segs_total;
    const int *pending;         // first segments of the trees not started at launch, in start order
    int *pending_next;          // next entry of `pending` to start
    int n_pending;
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
