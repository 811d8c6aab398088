// Device kernels of the marginal-gain path and their launch parameters (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace mig {

constexpr int kStatsCounters = 20;

struct GridView {
    const uint8_t *g;  // voxel codes in the traversal layout (x-fastest rows or 8x8x8 bricks)
    int nx, ny, nz;
    int nbx, nby;
};

// One tree level's work (Sec. IV-C): the nodes level_nodes[level_off[lvl] ..), the first
// level_int[lvl] of which have children and need their depth buffer rendered.
struct LevelParams {
    GridView grid;
    const int4 *body;        // H*W: body-frame ray (Q30) and camera z (Q30)
    const int32_t *yawtab;   // K*12: ck, sk, mu[3], mv[3], mz[3] (Q30, Q16)
    const float *yawf;       // K*9: mu, mv, mz as floats / 2^16 (estimates only)
    int W, H, K;
    int64_t Tq;              // range, Q16 voxel units
    int tile_w, tile_h, tiles_x, tiles;  // count-pass tile (rays per warp work item)
    const int32_t *level_off;   // device, levels + 1
    const int32_t *level_int;   // device, levels
    const int32_t *level_nodes; // device, n
    const int4 *node;           // device, n: Px, Py, Pz (Q16), arena slot
    const int2 *anc_range;      // device, n: (offset into anc, ancestor count = depth)
    const int32_t *anc;         // device: ancestors, parent first
    int32_t *sel_yaw;           // device, n (written by select)
    uint32_t *arena;            // device, slots * W * H depth buffers
    int32_t *cnt;               // device, n*K*2 (abs, excl) counts
    int32_t *work;              // device, levels: count-pass work counters (zeroed)
    int32_t *out_abs, *out_marg, *out_yaw;  // device, n
    int mode;                   // mig_mode
    int lvl;
    unsigned long long *stats;  // NULL, or kStatsCounters counters (instrumented pass)
    int max_anc;                // ancestor records per warp (>= the deepest node's depth, <= 64)
    // panoramic mode: A wedges ("columns") of `pano_step` per yaw bin, Wc columns per yaw window
    int pano_A, pano_Wc, pano_step;
    const int2 *pano_bc;        // A: wedge boundary cos, sin (Q30)
    const int4 *pano_dir;       // A*H: ray of cell (column, row) (Q30), pad
    const int4 *pano_row;       // A*2: strip rows (mv0 mv1 mv2 mz0) (mz1 mz2 - -) (Q16)
    int32_t *pano_cnt;          // n*A*2 (abs, excl) per column
    // checked builds (MIG_DEBUG_BOUNDS=1): out-of-buffer indices are or-ed into *bounds_err (NULL:
    // not recorded) and the access is skipped; arena_slots = depth buffers in the arena (0: unchecked)
    int32_t *bounds_err;
    int arena_slots;
    // owned-voxel count (voxcount.cu): per-ray DDA step counts of a chunk of (node, yaw) pairs
    // [q0, q1) of the level, steps_cap pairs of W * H each; NULL = the ray-by-ray count kernel
    uint16_t *steps;
    int32_t *vctr;  // work counter of the voxel pass (zeroed by the cast launch before it)
    int steps_cap;
    int q0, q1;
    // per-node voxel pass: the frustum's elevation band (tangents) and azimuth half-width
    float band_tlo, band_thi, az_half;
    int voxel_pass;  // MIG_COUNT_AUTO, MIG_COUNT_PAIRS or MIG_COUNT_NODES
};

void launch_count(const LevelParams &p, int grid, cudaStream_t s);
int count_ctas_per_sm();  // resident CTAs per SM of the count kernel
void launch_select(const LevelParams &p, int grid, cudaStream_t s);
void launch_render(const LevelParams &p, int grid, cudaStream_t s);
int render_tiles(int W, int H);  // 16x16 pixel tiles of the render pass
// Writes a box of voxel codes into a grid of nx * ny * nz and refreshes the brick occupancy bytes
// of the bricks it touches.
void launch_map_scatter(uint8_t *bricks, int nx, int ny, int nz, int nbx, int nby, const uint8_t *box, int x0, int y0,
                        int z0, int dx, int dy, int dz, cudaStream_t s);
// device bytes of an nx*ny*nz grid in the traversal layout (and its brick counts)
size_t map_layout_bytes(int nx, int ny, int nz, int *nbx, int *nby, int *nbz);
void launch_map_gather(const uint8_t *bricks, int nbx, int nby, uint8_t *lin, int nx, int ny, int nz, cudaStream_t s);

// Device planning (tree on the device): depth, levels, ancestors, slots, quantised positions.
struct DevPlanParams {
    int n, max_depth;
    const int32_t *parent;
    const float *pos;
    float ox, oy, oz, voxel;
    int nx, ny, nz;
    int32_t *depth;        // n
    int32_t *level_cnt;    // max_depth + 1 (zeroed)
    int32_t *level_icnt;   // max_depth + 1 (zeroed)
    int32_t *level_off;    // max_depth + 2
    int32_t *level_int;    // max_depth + 1
    int32_t *has_child;    // n (zeroed)
    int32_t *level_nodes;  // n
    int2 *anc_range;       // n: (n * max_depth, depth)
    int32_t *anc;          // n * max_depth
    int32_t *level_cur2;   // 2 * (max_depth + 1) (zeroed): internal / leaf scatter cursors
    int32_t *roots;        // 1 (zeroed)
    int4 *node;            // n
    int32_t *slot_cnt;     // 1 (zeroed)
    int32_t *err;          // device error word of this call
    int32_t *ctx_err;      // context error word (read by mig_ctx_sync)
    int32_t *out_abs, *out_marg, *out_yaw;
};
void launch_plan(const DevPlanParams &p, cudaStream_t s);

}  // namespace mig
