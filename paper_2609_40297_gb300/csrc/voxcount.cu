// Owned-voxel count of one tree level (Sec. IV-B, the counts of Eq. 1 and Eq. 2 by depth
// buffers), in two kernels per chunk of (node, yaw) pairs:
//   cast_kernel  - every pixel ray of every pair runs the DDA to its first occupied voxel within
//                  range and stores that voxel's step index (uint16 per ray; kNoHit if none);
//   voxel_kernel - for every pair, the voxels within range of the node are enumerated slice by
//                  slice (z), rows clipped to the camera frustum; each unknown voxel goes to the
//                  pixel that owns it (its centre's projection) and counts as absolute gain iff
//                  that pixel's DDA reaches it before the range and before its first occupied
//                  voxel; counted voxels are tested against the ancestors' depth buffers
//                  (marginal gain). Each test stage runs on full warps: the voxels that pass one
//                  stage wait in a per-warp queue until 32 of them are ready for the next.
// Results are identical to the ray-by-ray count kernel (and the CPU oracle) bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.h"
#include "mig.h"
#include "voxcount.h"
#include "voxitems.cuh"

namespace mig {

namespace {

using namespace dev;

constexpr int kCastWarps = 8;   // 256-thread CTAs, one ray per thread
constexpr int kVoxWarps = 8;

__device__ __forceinline__ int level_pairs(const LevelParams &p) {
    return (p.level_off[p.lvl + 1] - p.level_off[p.lvl]) * p.K;
}

// ------------------------------------------------------------------------------ cast kernel
// Warp work item = (pair q of the chunk, 8x4 pixel tile); one ray per lane.

template <bool STATS>
__global__ void __launch_bounds__(kCastWarps * 32) cast_kernel(const LevelParams p) {
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.vctr = 0;  // the voxel pass that follows hands out work from 0
    const int l0 = p.level_off[p.lvl];
    const int q1 = min(p.q1, level_pairs(p));
    if (p.q0 >= q1) return;
    const int tx = (p.W + kCastTileW - 1) / kCastTileW, ty = (p.H + kCastTileH - 1) / kCastTileH;
    const long long items = (long long)(q1 - p.q0) * tx * ty;
    const size_t WH = (size_t)p.W * p.H;
    const uint8_t *bocc = p.grid.g + bocc_offset(p.grid.nx, p.grid.ny, p.grid.nz);
    const uint8_t *sbocc = p.grid.g + sbocc_offset(p.grid.nx, p.grid.ny, p.grid.nz);
    uint32_t st_rays = 0, st_fine = 0, st_skip = 0;
    for (long long it = (long long)blockIdx.x * kCastWarps + (threadIdx.x >> 5); it < items;
         it += (long long)gridDim.x * kCastWarps) {
        const int tile = (int)(it % (tx * ty));
        const int ql = (int)(it / (tx * ty));
        cast_item<STATS>(p, bocc, sbocc, l0, p.q0 + ql, tile, tx, p.steps + (size_t)ql * WH, lane, st_rays, st_fine,
                         st_skip);
    }
    if constexpr (STATS) {
        st_rays = __reduce_add_sync(0xffffffffu, st_rays);
        st_fine = __reduce_add_sync(0xffffffffu, st_fine);
        st_skip = __reduce_add_sync(0xffffffffu, st_skip);
        if (lane == 0) {
            atomicAdd(p.stats + 8, (unsigned long long)st_rays);
            atomicAdd(p.stats + 9, (unsigned long long)st_fine);
            atomicAdd(p.stats + 10, (unsigned long long)st_skip);
        }
    }
}

// ----------------------------------------------------------------------------- voxel kernel
// Per-warp queues between the test stages: unknown voxels of the slice (x | y << 12), voxels whose
// owner pixel's ray may reach them (x | y << 12 | pixel << 24), counted samples (x | y << 16 |
// z << 32). Each holds fewer than 64 entries: a stage runs whenever 32 are waiting.
struct VoxQueues {
    unsigned long long unk[64], own[64], smp[64];
};


// Warp work item = (pair q of the chunk, slice z of the node's range ball). Lanes take 32 rows
// (y) of the slice at a time, clip each row to the frustum and the ball, and then load the rows'
// voxels 32 at a time (flattened over the rows with a warp prefix sum).
template <bool STATS>
__global__ void __launch_bounds__(kVoxWarps * 32, 3) voxel_kernel(const LevelParams p) {
    extern __shared__ AncRec s_anc_dyn[];
    __shared__ VoxQueues s_vq[kVoxWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    AncRec *anc = s_anc_dyn + warp * p.max_anc;
    VoxQueues &Q = s_vq[warp];
    const int l0 = p.level_off[p.lvl];
    const int q1 = min(p.q1, level_pairs(p));
    if (p.q0 >= q1) return;
    const int Rv = (int)(p.Tq >> 16) + 2;    // voxels: every visited voxel's centre is nearer than T + 1
    const int slices = 2 * Rv + 1;
    const int npairs = q1 - p.q0;
    const int items = npairs * slices;
    const float R = (float)p.Tq * (1.0f / 65536.0f) + 1.0f, R2 = R * R;
    const int gnx = p.grid.nx, gny = p.grid.ny, gnz = p.grid.nz;
    const size_t WH = (size_t)p.W * p.H;
    uint32_t st_cand = 0, st_unk = 0, st_visit = 0, st_anc = 0, st_reads = 0;
    int cur_node = -1, na = 0;
    // items are handed out one at a time from the launch's counter, in groups of pairs whose step
    // counts stay in L2 together; within a group every pair's slice at the node's own height first,
    // then outwards alternately above and below
    const int grp = (int)max((size_t)1, min((size_t)npairs, kStepsGroupBytes / (WH * sizeof(uint16_t))));
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(p.vctr, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= items) break;
        const int g = it / (grp * slices), r = it - g * grp * slices;
        const int gsz = min(grp, npairs - g * grp);
        const int rank = r / gsz, ql = g * grp + r % gsz;
        const int zi = Rv + ((rank & 1) ? (rank + 1) >> 1 : -(rank >> 1));
        const int qq = p.q0 + ql;
        const int n = p.level_nodes[l0 + qq / p.K], k = qq % p.K;
        const int4 nd = p.node[n];
        const int z = (nd.z >> 16) - Rv + zi;
        if (z < 0 || z >= gnz) continue;
        const float Pzf = (float)nd.z * (1.0f / 65536.0f) - 0.5f;  // centre of voxel z at offset z - Pzf
        const float rz = small_int_to_float(z) - Pzf;
        const float h2 = R2 - rz * rz;
        if (h2 < 0.f) continue;
        if (n != cur_node) {  // the node's ancestors (Sec. IV-B), parent first
            const int2 ar = p.anc_range[n];
            na = ar.y;
            if (p.mode == MIG_MODE_ABSOLUTE) na = 0;
            else if (p.mode == MIG_MODE_SINGLE_PARENT) na = min(na, 1);
            na = min(na, p.max_anc);
            fill_anc_records(p, ar, na, anc, lane);
            cur_node = n;
        }
        const int32_t *yk = p.yawtab + k * 12;
        const int ck = yk[0], sk = yk[1];
        const int mu0 = yk[2], mu1 = yk[3], mu2 = yk[4], mv0 = yk[5], mv1 = yk[6], mv2 = yk[7];
        const int mz0 = yk[8], mz1 = yk[9], mz2 = yk[10];
        const float s16 = 1.0f / 65536.0f;
        const float Pxf = (float)nd.x * s16 - 0.5f, Pyf = (float)nd.y * s16 - 0.5f;
        HalfSpace hs[5];
        frustum_half_spaces(mu0, mu1, mu2, mv0, mv1, mv2, mz0, mz1, mz2, p.W, p.H, hs);
        const uint16_t *steps = p.steps + (size_t)ql * WH;
        const int v0x = nd.x >> 16, v0y = nd.y >> 16, v0z = nd.z >> 16;
        const int zq = (z << 16) + 32768 - nd.z;
        int c_abs = 0, c_mrg = 0, nu = 0, no = 0, ns = 0;

        // stage 2: owner pixel of 32 unknown voxel centres (Eq. 5), and the cheap reach test: a voxel
        // is the (|x - x0| + |y - y0| + |z - z0|)-th of any ray that visits it, so it is reached only
        // if that index is below the owner ray's first occupied voxel
        auto owner_stage = [&](bool full) {
            const bool have = full || lane < nu;
            const unsigned long long e = full ? q_pop32(Q.unk, nu, lane) : Q.unk[lane];
            bool keep = false;
            int pix = 0;
            if (have) {
                const int x = (int)(e & 0xFFF), y = (int)((e >> 12) & 0xFFF);
                const int rx = (x << 16) + 32768 - nd.x, ry = (y << 16) + 32768 - nd.y;
                const int64_t Z = (int64_t)mz0 * rx + (int64_t)mz1 * ry + (int64_t)mz2 * zq;
                const int64_t U = (int64_t)mu0 * rx + (int64_t)mu1 * ry + (int64_t)mu2 * zq;
                const int64_t V = (int64_t)mv0 * rx + (int64_t)mv1 * ry + (int64_t)mv2 * zq;
                if (Z > 0) {
                    const float fxr = small_int_to_float(x) - Pxf, fyr = small_int_to_float(y) - Pyf;
                    const float zi_ = __fdividef(1.0f, fmaf(hs[0].a, fxr, fmaf(hs[0].b, fyr, hs[0].c * rz)));
                    const float uf = fmaf(hs[1].a, fxr, fmaf(hs[1].b, fyr, hs[1].c * rz)) * zi_;
                    const float vf = fmaf(hs[3].a, fxr, fmaf(hs[3].b, fyr, hs[3].c * rz)) * zi_;
                    int pu, pv;
                    if (pixel_in(U, Z, uf, p.W, pu) && pixel_in(V, Z, vf, p.H, pv)) {
                        pix = pv * p.W + pu;
                        const int man = abs(x - v0x) + abs(y - v0y) + abs(z - v0z);
                        keep = man < (int)__ldg(steps + pix);
                    }
                }
            }
            if (!full) nu = 0;
            q_push(Q.own, no, keep, (e & 0xFFFFFFull) | ((unsigned long long)pix << 24), lt_mask);
        };
        // stage 3: the exact visit test by the owner ray (event order of its DDA, range)
        auto visit_stage = [&](bool full) {
            const bool have = full || lane < no;
            const unsigned long long e = full ? q_pop32(Q.own, no, lane) : Q.own[lane];
            bool counted = false;
            int x = 0, y = 0;
            if (have) {
                if constexpr (STATS) ++st_visit;
                x = (int)(e & 0xFFF);
                y = (int)((e >> 12) & 0xFFF);
                const int pix = (int)(e >> 24);
                int dx, dy, dz;
                ray_dir(p.body[pix], ck, sk, dx, dy, dz);
                counted = visit_index(nd.x, nd.y, nd.z, dx, dy, dz, x, y, z, p.Tq) >= 0;
            }
            if (!full) no = 0;
            c_abs += counted;
            q_push(Q.smp, ns, counted,
                   (unsigned long long)x | ((unsigned long long)y << 16) | ((unsigned long long)z << 32), lt_mask);
        };
        // stage 4: the ancestor test of 32 counted samples (Sec. IV-B)
        auto ancestor_stage = [&](bool full) {
            const bool have = full || lane < ns;
            const unsigned long long sm = full ? q_pop32(Q.smp, ns, lane) : Q.smp[lane];
            if (have)
                c_mrg += !observed<STATS>(HotDirect{p}, anc, na, (int)(sm & 0xFFFF), (int)((sm >> 16) & 0xFFFF),
                                          (int)(sm >> 32), st_anc, st_reads);
            if (!full) ns = 0;
        };

        const float hy = sqrtf(h2);
        const int ylo = max(0, (int)floorf(Pyf - hy) - 1), yhi = min(gny - 1, (int)ceilf(Pyf + hy) + 1);
        for (int yb = ylo; yb <= yhi; yb += 32) {
            // this lane's row: x range of the centres inside the ball and the frustum
            const int y = yb + lane;
            int xa = 0, len = 0;
            if (y <= yhi) row_span(hs, Pxf, small_int_to_float(y) - Pyf, rz, h2, gnx, xa, len);
            int incl = len;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += v;
            }
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            for (int base = 0; base < tot; base += 32) {
                const int f = base + lane;
                // the row holding flat index f: the first lane whose inclusive sum exceeds f
                int r = 0;
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    const int cv = __shfl_sync(0xffffffffu, incl, r + s - 1);
                    if (cv <= f) r += s;
                }
                r = min(r, 31);
                const int rxa = __shfl_sync(0xffffffffu, xa, r);
                const int rstart = __shfl_sync(0xffffffffu, incl - len, r);
                bool unk = false;
                int x = 0;
                if (f < tot) {
                    x = rxa + (f - rstart);
                    if constexpr (STATS) ++st_cand;
                    const uint32_t addr = ((uint32_t)z * (uint32_t)gny + (uint32_t)(yb + r)) * (uint32_t)gnx + (uint32_t)x;
                    unk = load_code(p.grid.g, addr, p.grid, p.bounds_err) == kUnknown;
                    if constexpr (STATS) st_unk += unk;
                }
                q_push(Q.unk, nu, unk, (unsigned long long)x | ((unsigned long long)(yb + r) << 12), lt_mask);
                if (nu >= 32) {
                    owner_stage(true);
                    if (no >= 32) {
                        visit_stage(true);
                        if (ns >= 32) ancestor_stage(true);
                    }
                }
            }
        }
        // the slice's partial batches, stage by stage
        if (nu > 0) owner_stage(false);
        while (no >= 32) {
            visit_stage(true);
            if (ns >= 32) ancestor_stage(true);
        }
        if (no > 0) visit_stage(false);
        while (ns >= 32) ancestor_stage(true);
        if (ns > 0) ancestor_stage(false);
        c_abs = __reduce_add_sync(0xffffffffu, c_abs);
        c_mrg = __reduce_add_sync(0xffffffffu, c_mrg);
        if (lane == 0 && (c_abs | c_mrg)) {
            atomicAdd(p.cnt + ((size_t)n * p.K + k) * 2, c_abs);
            atomicAdd(p.cnt + ((size_t)n * p.K + k) * 2 + 1, c_mrg);
            if constexpr (STATS) atomicAdd(p.stats + 14, (unsigned long long)(uint32_t)c_abs);
        }
        __syncwarp();
    }
    if constexpr (STATS) {
        st_cand = __reduce_add_sync(0xffffffffu, st_cand);
        st_unk = __reduce_add_sync(0xffffffffu, st_unk);
        st_visit = __reduce_add_sync(0xffffffffu, st_visit);
        st_anc = __reduce_add_sync(0xffffffffu, st_anc);
        st_reads = __reduce_add_sync(0xffffffffu, st_reads);
        if (lane == 0) {
            atomicAdd(p.stats + 11, (unsigned long long)st_cand);
            atomicAdd(p.stats + 12, (unsigned long long)st_unk);
            atomicAdd(p.stats + 13, (unsigned long long)st_visit);
            atomicAdd(p.stats + 15, (unsigned long long)st_anc);
            atomicAdd(p.stats + 16, (unsigned long long)st_reads);
        }
    }
}

// ------------------------------------------------------------------------ per-node voxel kernel
// The same counts with each voxel taken once per node for all yaws: the ancestor test of Sec. IV-B
// does not depend on the node's own yaw, and a voxel lies in several yaws' frusta. Warp work item
// = (node of the chunk, slice z of its range ball, 32-row block of the slice), run by node_run
// (voxitems.cuh); the warp's per-yaw counters go to the level's counters when its node changes.
template <bool STATS>
__global__ void __launch_bounds__(kVoxWarps * 32, 4) node_kernel(const LevelParams p) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ NodeWarp s_nw[kVoxWarps];
    __shared__ int s_yi[kNodeMaxK * 12];    // yaw rows: ck sk mu mv mz -
    __shared__ float s_yf[kNodeMaxK * 9];   // mu mv mz / 2^16
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = p.K;
    AncRec *anc = reinterpret_cast<AncRec *>(s_dyn) + warp * p.max_anc;
    NodeWarp &Q = s_nw[warp];
    const int l0 = p.level_off[p.lvl];
    const int Ld = p.level_off[p.lvl + 1] - l0;
    const int nb0 = p.q0 / K, nb1 = min(p.q1 / K, Ld);
    if (nb0 >= nb1) return;
    for (int t = threadIdx.x; t < 12 * K; t += blockDim.x) s_yi[t] = p.yawtab[t];
    for (int t = threadIdx.x; t < 9 * K; t += blockDim.x) s_yf[t] = (float)p.yawtab[(t / 9) * 12 + 2 + t % 9] * (1.0f / 65536.0f);
    for (int t = lane; t < 2 * K; t += 32) Q.cnt[t] = 0;
    __syncthreads();
    const int slices = 2 * ((int)(p.Tq >> 16) + 2) + 1;
    const int nn = nb1 - nb0;
    const int yb_n = node_row_blocks(p.Tq);
    const int items = nn * slices * yb_n;
    const size_t WH = (size_t)p.W * p.H;
    NodeStats st;
    int cur_node = -1, na = 0;
    // items are handed out one at a time from the launch's counter, in groups of nodes whose step
    // counts stay in L2 together; within a group every node's slice at its own height first (the
    // fullest), then outwards alternately above and below, and within a slice the 32-row blocks from
    // the middle outwards. The warp's counters hold node cur_node's counts until the node changes.
    const int per_node = slices * yb_n;
    const int grp = (int)max((size_t)1, min((size_t)nn, kStepsGroupBytes / ((size_t)K * WH * sizeof(uint16_t))));
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(p.vctr, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= items) break;
        const int g = it / (grp * per_node), r = it - g * grp * per_node;
        const int gsz = min(grp, nn - g * grp);
        const int rzy = r / gsz, ln = g * grp + r % gsz;
        const int rank = rzy / yb_n, rb = rzy - rank * yb_n;
        const int n = p.level_nodes[l0 + nb0 + ln];
        NodeSlice S;
        if (!node_slice(p, n, rank, rb, yb_n, S)) continue;
        if (n != cur_node) {
            if (cur_node >= 0) node_flush(p, cur_node, Q, lane);
            na = node_ancestors(p, n, anc, lane);
            cur_node = n;
        }
        node_run<STATS>(p, S, s_yi, s_yf, p.steps + (size_t)ln * K * WH, Q, anc, na, lane, st);
    }
    if (cur_node >= 0) node_flush(p, cur_node, Q, lane);
    if constexpr (STATS) {
        st.cand = __reduce_add_sync(0xffffffffu, st.cand);
        st.unk = __reduce_add_sync(0xffffffffu, st.unk);
        st.visit = __reduce_add_sync(0xffffffffu, st.visit);
        st.anc = __reduce_add_sync(0xffffffffu, st.anc);
        st.reads = __reduce_add_sync(0xffffffffu, st.reads);
        st.smp = __reduce_add_sync(0xffffffffu, st.smp);
        if (lane == 0) {
            atomicAdd(p.stats + 11, (unsigned long long)st.cand);
            atomicAdd(p.stats + 12, (unsigned long long)st.unk);
            atomicAdd(p.stats + 13, (unsigned long long)st.visit);
            atomicAdd(p.stats + 14, (unsigned long long)st.smp);
            atomicAdd(p.stats + 15, (unsigned long long)st.anc);
            atomicAdd(p.stats + 16, (unsigned long long)st.reads);
        }
    }
}

// ------------------------------------------------------------------------- brick occupancy
// Recomputes the occupancy byte of every brick in [b0, b1) (brick coordinates).
__global__ void bocc_kernel(uint8_t *grid, int nx, int ny, int nz, int bx0, int by0, int bz0, int bx1, int by1,
                            int bz1) {
    const int nbx = (nx + 7) >> 3, nby = (ny + 7) >> 3;
    uint8_t *bocc = grid + bocc_offset(nx, ny, nz);
    const int wx = bx1 - bx0, wy = by1 - by0;
    const long long total = (long long)wx * wy * (bz1 - bz0);
    const int lane = threadIdx.x & 31;
    // one warp per brick: lane l checks rows (y, z) = (l & 7, l >> 3) and (l & 7, (l >> 3) + 4)
    for (long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < total;
         b += (long long)gridDim.x * (blockDim.x >> 5)) {
        const int bx = bx0 + (int)(b % wx), by = by0 + (int)((b / wx) % wy), bz = bz0 + (int)(b / ((long long)wx * wy));
        bool occ = false;
        for (int h = 0; h < 2; ++h) {
            const int y = (by << 3) + (lane & 7), z = (bz << 3) + (lane >> 3) + 4 * h;
            if (y >= ny || z >= nz) continue;
            const uint8_t *row = grid + ((size_t)z * ny + y) * nx;
            for (int x = bx << 3; x < min(nx, (bx << 3) + 8); ++x) occ |= row[x] == kOcc;
        }
        occ = __any_sync(0xffffffffu, occ);
        if (lane == 0) bocc[((size_t)bz * nby + by) * nbx + bx] = occ ? 1 : 0;
    }
}

// Recomputes the occupancy byte of every super-brick in [s0, s1) (super-brick coordinates) from its
// bricks' bytes.
__global__ void sbocc_kernel(uint8_t *grid, int nx, int ny, int nz, int sx0, int sy0, int sz0, int sx1, int sy1,
                             int sz1) {
    const int nbx = (nx + 7) >> 3, nby = (ny + 7) >> 3, nbz = (nz + 7) >> 3;
    const int nsx = (nx + 31) >> 5, nsy = (ny + 31) >> 5;
    const uint8_t *bocc = grid + bocc_offset(nx, ny, nz);
    uint8_t *sbocc = grid + sbocc_offset(nx, ny, nz);
    const int wx = sx1 - sx0, wy = sy1 - sy0;
    const long long total = (long long)wx * wy * (sz1 - sz0);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int sx = sx0 + (int)(i % wx), sy = sy0 + (int)((i / wx) % wy), sz = sz0 + (int)(i / ((long long)wx * wy));
        uint8_t occ = 0;
        for (int bz = 4 * sz; bz < min(4 * sz + 4, nbz); ++bz)
            for (int by = 4 * sy; by < min(4 * sy + 4, nby); ++by)
                for (int bx = 4 * sx; bx < min(4 * sx + 4, nbx); ++bx) occ |= bocc[((size_t)bz * nby + by) * nbx + bx];
        sbocc[((size_t)sz * nsy + sy) * nsx + sx] = occ ? 1 : 0;
    }
}

}  // namespace

size_t vox_dyn_smem(int max_anc) { return (size_t)kVoxWarps * (size_t)std::max(1, max_anc) * sizeof(AncRec); }

int vox_ctas_per_sm() {
    int a = 0, b = 0;
    const size_t smem = vox_dyn_smem(MIG_MAX_DEPTH);
    cudaFuncSetAttribute(voxel_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(voxel_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, voxel_kernel<false>, kVoxWarps * 32, vox_dyn_smem(16));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, voxel_kernel<true>, kVoxWarps * 32, vox_dyn_smem(16));
    cudaGetLastError();
    return std::max(1, std::min(a, b));
}

int cast_ctas_per_sm() {
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, cast_kernel<false>, kCastWarps * 32, 0);
    cudaGetLastError();
    return std::max(1, a);
}

size_t steps_pairs(long long pairs, int W, int H, size_t budget_bytes) {
    const size_t per = (size_t)W * H * sizeof(uint16_t);
    const size_t cap = std::max<size_t>(1, budget_bytes / per);
    return (size_t)std::max<long long>(1, std::min<long long>(pairs, (long long)cap));
}

void launch_cast_chunk(const LevelParams &c, int num_sms, cudaStream_t s) {
    const long long cast_warps =
        (long long)(c.q1 - c.q0) * ((c.W + kCastTileW - 1) / kCastTileW) * ((c.H + kCastTileH - 1) / kCastTileH);
    const int cg = (int)std::max<long long>(1, std::min<long long>((cast_warps + kCastWarps - 1) / kCastWarps,
                                                                    (long long)num_sms * 64));
    if (c.stats) cast_kernel<true><<<cg, kCastWarps * 32, 0, s>>>(c);
    else cast_kernel<false><<<cg, kCastWarps * 32, 0, s>>>(c);
}

void launch_voxel_chunk(const LevelParams &c, int num_sms, int vox_ctas, cudaStream_t s) {
    const long long vitems = (long long)(c.q1 - c.q0) * (2 * ((int)(c.Tq >> 16) + 2) + 1);
    const int vg = (int)std::max<long long>(1, std::min<long long>((vitems + kVoxWarps - 1) / kVoxWarps,
                                                                    (long long)num_sms * vox_ctas));
    const size_t smem = vox_dyn_smem(c.max_anc);
    if (c.stats) voxel_kernel<true><<<vg, kVoxWarps * 32, smem, s>>>(c);
    else voxel_kernel<false><<<vg, kVoxWarps * 32, smem, s>>>(c);
}

size_t node_dyn_smem(int max_anc) { return (size_t)kVoxWarps * std::max(1, max_anc) * sizeof(AncRec); }

int node_ctas_per_sm() {
    int a = 0, b = 0;
    const size_t smem = node_dyn_smem(MIG_MAX_DEPTH);
    cudaFuncSetAttribute(node_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(node_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, node_kernel<false>, kVoxWarps * 32, node_dyn_smem(16));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, node_kernel<true>, kVoxWarps * 32, node_dyn_smem(16));
    cudaGetLastError();
    return std::max(1, std::min(a, b));
}

// The per-node pass, when it applies: whole nodes in a chunk, at most kNodeMaxK yaws and a frustum
// band. By default it is taken when a voxel lies in at least 3 yaws' frusta on average (K times the
// azimuth half-width over pi; 4 at paper scale, 9 on the large workload, where it runs 1.2x and 1.3x
// faster than the per-pair pass).
bool node_pass(const LevelParams &p) {
    if (!(p.az_half > 0.f && p.K <= kNodeMaxK && p.steps_cap >= p.K) || p.voxel_pass == MIG_COUNT_PAIRS) return false;
    return p.voxel_pass == MIG_COUNT_NODES || (float)p.K * p.az_half >= 3.0f * 3.14159265f;
}

void launch_node_chunk(const LevelParams &c, int num_sms, int node_ctas, cudaStream_t s) {
    const int slices = 2 * ((int)(c.Tq >> 16) + 2) + 1;
    const long long items = (long long)((c.q1 - c.q0) / c.K) * slices * node_row_blocks(c.Tq);
    const int g = (int)std::max<long long>(1, std::min<long long>((items + kVoxWarps - 1) / kVoxWarps,
                                                                   (long long)num_sms * node_ctas));
    const size_t smem = node_dyn_smem(c.max_anc);
    if (c.stats) node_kernel<true><<<g, kVoxWarps * 32, smem, s>>>(c);
    else node_kernel<false><<<g, kVoxWarps * 32, smem, s>>>(c);
}

// Pairs per launch: within the step-count buffer, and few enough that the launch's work items
// (pairs x slices, or nodes x slices x row blocks) stay below 2^30 for the 32-bit work counter.
int vox_chunk_pairs(const LevelParams &p) {
    const long long slices = 2 * ((long long)(p.Tq >> 16) + 2) + 1;
    const long long lim = 1ll << 30;
    if (node_pass(p)) {
        const long long nodes = std::min<long long>(p.steps_cap / p.K, lim / (slices * node_row_blocks(p.Tq)));
        return (int)std::max<long long>(1, nodes) * p.K;
    }
    return (int)std::max<long long>(1, std::min<long long>(p.steps_cap, lim / slices));
}

void launch_vox_level(const LevelParams &p, long long pairs, int num_sms, int vox_ctas, int node_ctas, cudaStream_t s) {
    const int cap = vox_chunk_pairs(p);
    for (long long q0 = 0; q0 < pairs; q0 += cap) {
        LevelParams c = p;
        c.q0 = (int)q0;
        c.q1 = (int)std::min<long long>(pairs, q0 + cap);
        launch_cast_chunk(c, num_sms, s);
        if (node_pass(p)) launch_node_chunk(c, num_sms, node_ctas, s);
        else launch_voxel_chunk(c, num_sms, vox_ctas, s);
    }
}

void launch_bocc(uint8_t *grid, int nx, int ny, int nz, int x0, int y0, int z0, int dx, int dy, int dz, cudaStream_t s) {
    const int bx0 = x0 >> 3, by0 = y0 >> 3, bz0 = z0 >> 3;
    const int bx1 = (x0 + dx + 7) >> 3, by1 = (y0 + dy + 7) >> 3, bz1 = (z0 + dz + 7) >> 3;
    const long long total = (long long)(bx1 - bx0) * (by1 - by0) * (bz1 - bz0);
    const int grid_ = (int)std::max<long long>(1, std::min<long long>((total + 7) / 8, 4096));
    bocc_kernel<<<grid_, 256, 0, s>>>(grid, nx, ny, nz, bx0, by0, bz0, bx1, by1, bz1);
    // the super-bricks holding those bricks
    const int sx0 = bx0 >> 2, sy0 = by0 >> 2, sz0 = bz0 >> 2;
    const int sx1 = (bx1 + 3) >> 2, sy1 = (by1 + 3) >> 2, sz1 = (bz1 + 3) >> 2;
    const long long stotal = (long long)(sx1 - sx0) * (sy1 - sy0) * (sz1 - sz0);
    const int sgrid = (int)std::max<long long>(1, std::min<long long>((stotal + 255) / 256, 1024));
    sbocc_kernel<<<sgrid, 256, 0, s>>>(grid, nx, ny, nz, sx0, sy0, sz0, sx1, sy1, sz1);
}

}  // namespace mig
