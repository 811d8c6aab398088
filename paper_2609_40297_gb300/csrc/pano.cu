// Panoramic mode: one 360-degree cast per node, per-column counts, per-yaw window sums.
//
// The yaw set of Sec. III-B is evaluated from shared rays: the horizon is cut into A azimuth
// wedges ("columns"), each a one-pixel-wide strip camera with the pinhole's rows. A voxel belongs
// to the cell (column, row) containing its centre: the column by the sign of its horizontal cross
// product with the wedge's two boundary vectors (Q30), the row by the strip's Eq. 5 projection
// (Q16 rows), all in integers. Owned unknown voxels are absolute gain of their column; each is
// tested against the ancestors' pinhole depth buffers (Sec. IV-B, the same voxel-centre test as
// the marginal mode) and otherwise counts as the column's marginal gain. Yaw k's counts are the
// sums over the Wc columns centred on its azimuth; yaw selection and the depth buffer of the
// selected yaw then run unchanged.
//
// Layout: one warp per work item (node, column); its lanes take the column's H rays, a new one
// as soon as their ray ends. Owned samples go to a per-warp queue and are tested against the
// ancestors 32 at a time, one per lane. Each (node, column) is written by exactly one warp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "dev_path.cuh"
#include "kernels.h"
#include "mig.h"
#include "pano.h"

namespace mig {

namespace {

using namespace dev;

template <bool STATS>
__global__ void __launch_bounds__(kWarps * 32, 4) pano_count_kernel(const LevelParams p) {
    extern __shared__ AncRec s_anc_dyn[];
    __shared__ unsigned long long s_q[kWarps][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    AncRec *anc = s_anc_dyn + warp * p.max_anc;
    unsigned long long *q = s_q[warp];
    const HotDirect hp{p};
    const int l0 = p.level_off[p.lvl];
    const int L = p.level_off[p.lvl + 1] - l0;
    const int A = p.pano_A, H = p.H;
    const int items = L * A;
    uint32_t st_rays = 0, st_steps = 0, st_unk = 0, st_anc = 0, st_reads = 0;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(p.work + p.lvl, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= items) break;
        const int li = item / A, col = item % A;
        const int n = p.level_nodes[l0 + li];
        const int4 nd = p.node[n];
        const int2 ar = p.anc_range[n];
        const int na = min(ar.y, p.max_anc);
        fill_anc_records(p, ar, na, anc, lane);
        const int2 b0 = p.pano_bc[col], b1 = p.pano_bc[col + 1 == A ? 0 : col + 1];
        const int4 m0 = p.pano_row[2 * col], m1 = p.pano_row[2 * col + 1];  // (mv0 mv1 mv2 mz0) (mz1 mz2 - -)
        int next = 0, j = 0, qn = 0, c_abs = 0, c_mrg = 0;
        bool have = false;
        RayIn r;
        uint32_t ne = 0, ade = 1;
        for (;;) {
            // lanes without a ray take the column's next rows in order
            const unsigned need = __ballot_sync(0xffffffffu, !have);
            if (need && next < H) {
                const int idx = next + __popc(need & lt_mask);
                next += __popc(need);
                if (!have && idx < H) {
                    j = idx;
                    const int4 d = p.pano_dir[(size_t)col * H + j];
                    ray_init(r, p.grid, nd.x, nd.y, nd.z, d.x, d.y, d.z, p.Tq);
                    have = true;
                    if constexpr (STATS) ++st_rays;
                }
            }
            if (!__any_sync(0xffffffffu, have)) {
                if (next >= H) break;
                continue;
            }
            bool owned = false;
            unsigned long long samp = 0;
            if (have) {
                const uint8_t code = load_code(p.grid.g, ray_addr(r, p.grid), p.grid, p.bounds_err);
                if constexpr (STATS) ++st_steps;
                if (code == kOcc) {
                    have = false;
                } else {
                    if (code == kUnknown) {
                        if constexpr (STATS) ++st_unk;
                        // owner test: the voxel centre lies in this column's wedge and this row
                        const int rx = voxel_offset(r.nx, r.sx), ry = voxel_offset(r.ny, r.sy),
                                  rz = voxel_offset(r.nz, r.sz);
                        const int64_t x0 = (int64_t)b0.x * ry - (int64_t)b0.y * rx;
                        const int64_t x1 = (int64_t)b1.x * ry - (int64_t)b1.y * rx;
                        if (x0 >= 0 && x1 < 0) {
                            const int64_t Z = (int64_t)m0.w * rx + (int64_t)m1.x * ry + (int64_t)m1.y * rz;
                            const int64_t V = (int64_t)m0.x * rx + (int64_t)m0.y * ry + (int64_t)m0.z * rz;
                            const int64_t jZ = (int64_t)j * Z;
                            owned = Z > 0 && V >= jZ && V < jZ + Z;
                            if (owned) samp = sample_key(rx, ry, rz, nd);
                        }
                    }
                    have = ray_step<false>(r, ne, ade);
                }
            }
            c_abs += owned;
            const unsigned bal = __ballot_sync(0xffffffffu, owned);
            if (bal) {
                if (owned) q[qn + __popc(bal & lt_mask)] = samp;
                qn += __popc(bal);
                if (qn >= 32) {  // a full batch: every lane tests one sample (Sec. IV-B)
                    __syncwarp();
                    const unsigned long long sm = q[lane];
                    c_mrg += !observed<STATS>(hp, anc, na, (int)(sm & 0xFFFF), (int)((sm >> 16) & 0xFFFF),
                                              (int)(sm >> 32), st_anc, st_reads);
                    __syncwarp();
                    if (lane < qn - 32) q[lane] = q[lane + 32];
                    __syncwarp();
                    qn -= 32;
                }
            }
        }
        __syncwarp();
        if (lane < qn) {
            const unsigned long long sm = q[lane];
            c_mrg += !observed<STATS>(hp, anc, na, (int)(sm & 0xFFFF), (int)((sm >> 16) & 0xFFFF), (int)(sm >> 32),
                                      st_anc, st_reads);
        }
        c_abs = __reduce_add_sync(0xffffffffu, c_abs);
        c_mrg = __reduce_add_sync(0xffffffffu, c_mrg);
        if (lane == 0) {
            p.pano_cnt[((size_t)n * A + col) * 2] = c_abs;
            p.pano_cnt[((size_t)n * A + col) * 2 + 1] = c_mrg;
            if constexpr (STATS) atomicAdd(p.stats + 3, (unsigned long long)(uint32_t)c_abs);
        }
        __syncwarp();
    }
    if constexpr (STATS) {
        st_rays = __reduce_add_sync(0xffffffffu, st_rays);
        st_steps = __reduce_add_sync(0xffffffffu, st_steps);
        st_unk = __reduce_add_sync(0xffffffffu, st_unk);
        st_anc = __reduce_add_sync(0xffffffffu, st_anc);
        st_reads = __reduce_add_sync(0xffffffffu, st_reads);
        if (lane == 0) {
            atomicAdd(p.stats + 0, (unsigned long long)st_rays);
            atomicAdd(p.stats + 1, (unsigned long long)st_steps);
            atomicAdd(p.stats + 2, (unsigned long long)st_unk);
            atomicAdd(p.stats + 4, (unsigned long long)st_anc);
            atomicAdd(p.stats + 5, (unsigned long long)st_reads);
        }
    }
}

// Yaw k's counts of each node of the level: sums over the Wc columns centred on its azimuth,
// starting at column k * step - Wc / 2 (mod A).
__global__ void pano_window_kernel(const LevelParams p) {
    const int l0 = p.level_off[p.lvl];
    const int L = p.level_off[p.lvl + 1] - l0;
    const int A = p.pano_A;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L * p.K; t += gridDim.x * blockDim.x) {
        const int li = t / p.K, k = t % p.K;
        const int n = p.level_nodes[l0 + li];
        const int s0 = k * p.pano_step - p.pano_Wc / 2;
        int c = ((s0 % A) + A) % A;
        const int32_t *pc = p.pano_cnt + (size_t)n * A * 2;
        int sa = 0, sm = 0;
        for (int i = 0; i < p.pano_Wc; ++i) {
            sa += pc[2 * c];
            sm += pc[2 * c + 1];
            if (++c == A) c = 0;
        }
        p.cnt[((size_t)n * p.K + k) * 2] = sa;
        p.cnt[((size_t)n * p.K + k) * 2 + 1] = sm;
    }
}

}  // namespace

void launch_pano_count(const LevelParams &p, int grid, cudaStream_t s) {
    const size_t smem = (size_t)kWarps * (size_t)std::max(1, p.max_anc) * sizeof(AncRec);
    if (p.stats) pano_count_kernel<true><<<grid, kWarps * 32, smem, s>>>(p);
    else pano_count_kernel<false><<<grid, kWarps * 32, smem, s>>>(p);
}

void launch_pano_window(const LevelParams &p, int grid, cudaStream_t s) {
    pano_window_kernel<<<grid, 256, 0, s>>>(p);
}

int pano_ctas_per_sm() {
    const size_t max_dyn = (size_t)kWarps * MIG_MAX_DEPTH * sizeof(AncRec);
    cudaFuncSetAttribute(pano_count_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dyn);
    cudaFuncSetAttribute(pano_count_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dyn);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pano_count_kernel<false>, kWarps * 32,
                                                  (size_t)kWarps * 16 * sizeof(AncRec));
    return std::max(1, n);
}

}  // namespace mig
