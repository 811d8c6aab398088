// Launchers of the owned-voxel count kernels (voxcount.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "kernels.h"

namespace mig {

// (node, yaw) pairs per chunk of the owned-voxel count: all `pairs` of a level, or as many as a
// step-count buffer of budget_bytes holds (W * H uint16 per pair), at least 1.
size_t steps_pairs(long long pairs, int W, int H, size_t budget_bytes);
// Device bytes of a step-count region for steps_cap pairs of W * H rays: the counts, then (256-byte
// aligned) the work counter of the voxel pass; steps_counter gives that counter's address.
inline size_t steps_region_bytes(int steps_cap, size_t WH) {
    return (((size_t)steps_cap * WH * sizeof(uint16_t) + 255) & ~(size_t)255) + 256;
}
inline int32_t *steps_counter(uint16_t *steps, int steps_cap, size_t WH) {
    return reinterpret_cast<int32_t *>(reinterpret_cast<char *>(steps) +
                                       (((size_t)steps_cap * WH * sizeof(uint16_t) + 255) & ~(size_t)255));
}
// Step-count buffer budget per evaluation (device bytes).
constexpr size_t kStepsBudget = (size_t)1 << 30;
// One level's count for the sample modes (marginal, single parent, absolute): for each chunk of
// p.steps_cap pairs of the first `pairs` (node, yaw) pairs, a cast launch and a voxel launch. The
// kernels read the level's true size from p.level_off and skip pairs beyond it, so `pairs` may be
// an upper bound.
// When every chunk holds whole nodes (all K yaws), the voxel pass runs once per node over all its
// yaws (node_kernel); otherwise once per (node, yaw) pair (voxel_kernel).
void launch_vox_level(const LevelParams &p, long long pairs, int num_sms, int vox_ctas, int node_ctas, cudaStream_t s);
// The launches of one chunk [c.q0, c.q1) (launch_vox_level runs them for every chunk).
void launch_cast_chunk(const LevelParams &c, int num_sms, cudaStream_t s);
void launch_voxel_chunk(const LevelParams &c, int num_sms, int vox_ctas, cudaStream_t s);
void launch_node_chunk(const LevelParams &c, int num_sms, int node_ctas, cudaStream_t s);
bool node_pass(const LevelParams &p);  // whole nodes per chunk and a frustum band: the per-node pass
int vox_chunk_pairs(const LevelParams &p);  // pairs per chunk (a multiple of K for the per-node pass)
int node_ctas_per_sm();
int vox_ctas_per_sm();
int cast_ctas_per_sm();
// Recomputes the brick occupancy bytes of the bricks overlapping a box of voxels.
void launch_bocc(uint8_t *grid, int nx, int ny, int nz, int x0, int y0, int z0, int dx, int dy, int dz, cudaStream_t s);

}  // namespace mig
