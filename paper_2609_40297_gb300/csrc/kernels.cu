// Device kernels: fused per-level count (3D DDA + owner test + ancestor depth test + integer
// reductions), yaw selection, depth-buffer render, map brick scatter/gather, device planning.
//
// All result-deciding arithmetic is integer (the fixed-point reading of Sec. IV-A..C):
// positions Q16 voxel units, ray directions Q30, projection rows Q16, depths Q16.16.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "dev_path.cuh"
#include "kernels.h"
#include "mig.h"
#include "voxcount.cuh"
#include "voxcount.h"

namespace mig {

namespace {

using namespace dev;

template <bool STATS>
__global__ void __launch_bounds__(kWarps * 32, MIG_COUNT_MINB) count_kernel(const LevelParams p) {
    // ancestor records: p.max_anc per warp, sized at launch from the tree's depth (dynamic shared
    // memory), so that the rest of the unified L1/shared storage serves the voxel gathers
    extern __shared__ AncRec s_anc_dyn[];
    __shared__ unsigned long long s_q[kWarps][kQueue];
    __shared__ int4 s_cam[kWarps][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int l0 = p.level_off[p.lvl];
    const int L = p.level_off[p.lvl + 1] - l0;
    const int chunks = L * p.K * p.tiles;
    for (;;) {
        int c = 0;
        if (lane == 0) c = atomicAdd(p.work + p.lvl, 1);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= chunks) break;
        count_chunk<STATS>(p, HotDirect{p}, l0, c, s_anc_dyn + warp * p.max_anc, s_q[warp], s_cam[warp], lane);
    }
}

// ------------------------------------------------------------------------------ select kernel
// Yaw selection (Sec. III-B): lowest k with the largest marginal count (absolute count in the
// absolute mode, where both counts are equal); g_abs = max over yaws of the absolute count.
__global__ void select_kernel(const LevelParams p) {
    const int l0 = p.level_off[p.lvl];
    const int L = p.level_off[p.lvl + 1] - l0;
    for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < L; li += gridDim.x * blockDim.x)
        select_node(p, p.level_nodes[l0 + li]);
}

// ------------------------------------------------------------------------------ render kernel
// Depth buffer of the selected yaw (Sec. IV-A): per pixel ray, camera z of the entry point of
// the first occupied voxel, else of the range endpoint. Only nodes with children (the level's
// first level_int nodes) are rendered; descendants read them in the ancestor test.
template <bool STATS>
__global__ void __launch_bounds__(256) render_kernel(const LevelParams p) {
    constexpr int RT = 16;  // render tile: 16 x 16 pixels, one ray per thread
    const int l0 = p.level_off[p.lvl];
    const int Li = p.level_int[p.lvl];
    const int rtx = (p.W + RT - 1) / RT;
    const int rtiles = rtx * ((p.H + RT - 1) / RT);
    const int items = Li * rtiles;
    const int tid = threadIdx.x;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int tile = item % rtiles;
        const int li = item / rtiles;
        const int n = p.level_nodes[l0 + li];
        const int4 nd = p.node[n];
        if (nd.w < 0) continue;
        const int ti = (tile % rtx) * RT + tid % RT;
        const int tj = (tile / rtx) * RT + tid / RT;
        if (ti >= p.W || tj >= p.H) continue;
        const uint32_t st_steps = render_pixel(p, n, nd, ti, tj);
        if constexpr (STATS) {
            atomicAdd(p.stats + 6, 1ull);
            atomicAdd(p.stats + 7, (unsigned long long)st_steps);
        }
    }
}

// ------------------------------------------------------------------------------- map kernels
__global__ void map_scatter_kernel(uint8_t *bricks, int nx, int ny, int nbx, int nby, const uint8_t *box, int x0,
                                   int y0, int z0, int dx, int dy, int dz) {
    const size_t total = (size_t)dx * dy * dz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % dx) + x0;
        const int y = (int)((i / dx) % dy) + y0;
        const int z = (int)(i / ((size_t)dx * dy)) + z0;
        const GridView G{nullptr, nx, ny, 0, nbx, nby};
        bricks[voxel_addr(G, x, y, z)] = box[i];
    }
}

__global__ void map_gather_kernel(const uint8_t *bricks, int nbx, int nby, uint8_t *lin, int nx, int ny, int nz) {
    // (the layout's address of voxel (x, y, z); identity for x-fastest rows)
    const size_t total = (size_t)nx * ny * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const int y = (int)((i / nx) % ny);
        const int z = (int)(i / ((size_t)nx * ny));
        const GridView G{nullptr, nx, ny, 0, nbx, nby};
        lin[i] = bricks[voxel_addr(G, x, y, z)];
    }
}

// ----------------------------------------------------------------------------- device plan
__global__ void plan_depth_kernel(const DevPlanParams p) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
        int d = 0, q = p.parent[i];
        bool bad = false;
        if (q == -1) atomicAdd(p.roots, 1);
        while (q != -1) {
            if (q < 0 || q >= p.n || d >= p.max_depth) {
                bad = true;
                break;
            }
            p.anc[(size_t)i * p.max_depth + d] = q;
            ++d;
            q = p.parent[q];
        }
        if (bad) {
            atomicOr(p.err, 1);
            d = 0;
        }
        p.depth[i] = d;
        p.anc_range[i] = make_int2(i * p.max_depth, d);
        const int pa = p.parent[i];
        if (!bad && pa >= 0) p.has_child[pa] = 1;
        // quantised position, round half to even (the same IEEE double steps as the host)
        const float pos3[3] = {p.pos[3 * (size_t)i], p.pos[3 * (size_t)i + 1], p.pos[3 * (size_t)i + 2]};
        const float org[3] = {p.ox, p.oy, p.oz};
        const int dims[3] = {p.nx, p.ny, p.nz};
        int P[3];
        for (int a = 0; a < 3; ++a) {
            const double qd = __dmul_rn(__ddiv_rn(__dsub_rn((double)pos3[a], (double)org[a]), (double)p.voxel), 65536.0);
            if (!(qd > -1.0 && qd < (double)dims[a] * 65536.0)) {
                atomicOr(p.err, 2);
                P[a] = 0;
                continue;
            }
            const long long v = __double2ll_rn(qd);
            if (v < 0 || v >= (long long)dims[a] * 65536) {
                atomicOr(p.err, 2);
                P[a] = 0;
            } else {
                P[a] = (int)v;
            }
        }
        p.node[i] = make_int4(P[0], P[1], P[2], -1);
        atomicAdd(p.level_cnt + d, 1);
    }
}

__global__ void plan_slot_kernel(const DevPlanParams p) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
        if (p.has_child[i]) {
            p.node[i].w = atomicAdd(p.slot_cnt, 1);
            atomicAdd(p.level_icnt + p.depth[i], 1);
        }
    }
}

__global__ void plan_scan_kernel(const DevPlanParams p) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (p.n > 0 && *p.roots != 1) atomicOr(p.err, 4);
    const bool bad = *p.err != 0;
    int acc = 0;
    for (int d = 0; d <= p.max_depth; ++d) {
        p.level_off[d] = bad ? 0 : acc;
        p.level_int[d] = bad ? 0 : p.level_icnt[d];
        acc += p.level_cnt[d];
    }
    p.level_off[p.max_depth + 1] = bad ? 0 : acc;
    if (bad) atomicOr(p.ctx_err, *p.err);
}

__global__ void plan_scatter_kernel(const DevPlanParams p) {
    const bool bad = *p.err != 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
        if (bad) {
            p.out_abs[i] = -1;
            p.out_marg[i] = -1;
            p.out_yaw[i] = -1;
            continue;
        }
        const int d = p.depth[i];
        int idx;
        if (p.has_child[i]) idx = p.level_off[d] + atomicAdd(p.level_cur2 + 2 * d, 1);
        else idx = p.level_off[d] + p.level_icnt[d] + atomicAdd(p.level_cur2 + 2 * d + 1, 1);
        p.level_nodes[idx] = i;
    }
}

}  // namespace

size_t count_dyn_smem(int max_anc) { return (size_t)kWarps * (size_t)std::max(1, max_anc) * sizeof(AncRec); }

void launch_count(const LevelParams &p, int grid, cudaStream_t s) {
    const size_t smem = count_dyn_smem(p.max_anc);
    if (p.stats) count_kernel<true><<<grid, kWarps * 32, smem, s>>>(p);
    else count_kernel<false><<<grid, kWarps * 32, smem, s>>>(p);
}

size_t map_layout_bytes(int nx, int ny, int nz, int *nbx, int *nby, int *nbz) {
    *nbx = (nx + 7) / 8;
    *nby = (ny + 7) / 8;
    *nbz = (nz + 7) / 8;
#if MIG_LAYOUT == 1
    // voxel codes, then (256-byte aligned) one occupancy byte per 8x8x8 brick and (256-byte aligned)
    // one per 32x32x32 super-brick
    return occ_summary_end(nx, ny, nz);
#else
    return (size_t)*nbx * *nby * *nbz * 512;
#endif
}

int count_ctas_per_sm() {
    int a = 0, b = 0;
    const size_t smem = count_dyn_smem(MIG_MAX_DEPTH);  // the worst case
    cudaFuncSetAttribute(count_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(count_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, count_kernel<false>, kWarps * 32, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, count_kernel<true>, kWarps * 32, smem);
    cudaGetLastError();
    return std::max(1, std::min(a, b));
}
void launch_select(const LevelParams &p, int grid, cudaStream_t s) { select_kernel<<<grid, 128, 0, s>>>(p); }
void launch_render(const LevelParams &p, int grid, cudaStream_t s) {
    if (p.stats) render_kernel<true><<<grid, 256, 0, s>>>(p);
    else render_kernel<false><<<grid, 256, 0, s>>>(p);
}

int render_tiles(int W, int H) { return ((W + 15) / 16) * ((H + 15) / 16); }
void launch_map_scatter(uint8_t *bricks, int nx, int ny, int nz, int nbx, int nby, const uint8_t *box, int x0, int y0,
                        int z0, int dx, int dy, int dz, cudaStream_t s) {
    const size_t total = (size_t)dx * dy * dz;
    const int grid = (int)std::min<size_t>((total + 255) / 256, 4096);
    map_scatter_kernel<<<grid, 256, 0, s>>>(bricks, nx, ny, nbx, nby, box, x0, y0, z0, dx, dy, dz);
#if MIG_LAYOUT == 1
    launch_bocc(bricks, nx, ny, nz, x0, y0, z0, dx, dy, dz, s);  // the occupancy bytes of the bricks it touched
#else
    (void)nz;
#endif
}
void launch_map_gather(const uint8_t *bricks, int nbx, int nby, uint8_t *lin, int nx, int ny, int nz, cudaStream_t s) {
    const size_t total = (size_t)nx * ny * nz;
    const int grid = (int)std::min<size_t>((total + 255) / 256, 4096);
    map_gather_kernel<<<grid, 256, 0, s>>>(bricks, nbx, nby, lin, nx, ny, nz);
}
void launch_plan(const DevPlanParams &p, cudaStream_t s) {
    const int grid = std::max(1, std::min((p.n + 255) / 256, 1024));
    plan_depth_kernel<<<grid, 256, 0, s>>>(p);
    plan_slot_kernel<<<grid, 256, 0, s>>>(p);
    plan_scan_kernel<<<1, 32, 0, s>>>(p);
    plan_scatter_kernel<<<grid, 256, 0, s>>>(p);
}

}  // namespace mig
