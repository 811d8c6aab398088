// Work items of the owned-voxel count (the steps are described in voxcount.cuh), as device
// functions shared by the per-level kernels (voxcount.cu) and the persistent batch kernel
// (batch.cu): a cast item is one 8x4 pixel tile of one (node, yaw) pair; a per-node item is one
// 32-row block of one slice (z) of a node's range ball, tested against every yaw.
#pragma once

#include "voxcount.cuh"

namespace mig {
namespace dev {

// The voxel passes hand out their work in groups of (node, yaw) pairs or nodes whose step counts
// fit in this many bytes, so that the step counts the warps in flight read stay in L2.
#ifndef MIG_STEPS_GROUP_BYTES
#define MIG_STEPS_GROUP_BYTES (64u << 20)
#endif
constexpr size_t kStepsGroupBytes = MIG_STEPS_GROUP_BYTES;

constexpr int kCastTileW = 8, kCastTileH = 4;  // pixels of a cast item, one ray per lane

// Appends the lanes' `take` entries `val` to queue q holding n entries (in lane order).
__device__ __forceinline__ void q_push(unsigned long long *q, int &n, bool take, unsigned long long val,
                                       unsigned lt_mask) {
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    if (take) q[n + __popc(bal & lt_mask)] = val;
    n += __popc(bal);
    __syncwarp();
}
// Takes the first 32 entries of q (lane l gets entry l) and moves the rest to the front.
__device__ __forceinline__ unsigned long long q_pop32(unsigned long long *q, int &n, int lane) {
    const unsigned long long v = q[lane];
    const unsigned long long rest = lane + 32 < n ? q[lane + 32] : 0ull;
    __syncwarp();
    if (lane + 32 < n) q[lane] = rest;
    __syncwarp();
    n -= 32;
    return v;
}

constexpr int kNodeMaxK = 64;  // yaws of the per-node pass (one mask word, per-warp counters)

// Blocks of 32 rows covering one slice's rows of the range ball (at most 2 Rv + 3 rows, Rv = T + 2
// voxels): the per-node pass hands out (node, slice, row block) items.
__host__ __device__ inline int node_row_blocks(int64_t Tq) { return (2 * ((int)(Tq >> 16) + 2) + 3 + 31) / 32; }

// Per-warp state of the per-node pass: queues of unknown voxels in the band and of counted voxels
// with the mask of the yaws that count them, and the per-yaw (absolute, marginal) counters.
struct NodeWarp {
    unsigned long long unk[64];    // x | y << 12
    unsigned long long key[64];    // x | y << 12 | k_lo << 24 (first yaw of the mask)
    unsigned long long mask[64];   // yaws (from k_lo, cyclic) that count the voxel
    unsigned long long vm[32];     // stage B: mask of the yaws counting each of the 32 voxels
    unsigned long long xq[64];     // stage B: (voxel, yaw) pairs left to the exact visit test
    int cnt[2 * kNodeMaxK];
};

// Work counters of the per-node pass (statistics).
struct NodeStats {
    uint32_t cand = 0, unk = 0, visit = 0, anc = 0, reads = 0, smp = 0;
};

// Sec. IV-B's ancestor test of voxel (x, y, z) (observed iff some ancestor sees its centre at camera
// depth z <= D), deciding each ancestor's pixel and the depth comparison from the float rows where
// their proven error bounds do (pixel_fast), else with the exact integers of the per-ray test.
template <bool STATS>
__device__ __forceinline__ bool observed_fast(const LevelParams &p, const AncRec *anc, int na, int x, int y, int z,
                                              uint32_t &st_anc, uint32_t &st_reads) {
    for (int a = 0; a < na; ++a) {
        const AncRec &A = anc[a];
        const int ax = (x << 16) + 32768 - A.px, ay = (y << 16) + 32768 - A.py, az = (z << 16) + 32768 - A.pz;
        if constexpr (STATS) ++st_anc;
        const float ex = (float)ax * (1.0f / 65536.0f), ey = (float)ay * (1.0f / 65536.0f);
        const float ez = (float)az * (1.0f / 65536.0f);
        const float rinf = fmaxf(fabsf(ex), fmaxf(fabsf(ey), fabsf(ez)));
        int pu = 0, pv = 0;
        float zf, e_z;
        const int in = pixel_fast(A.m, ex, ey, ez, rinf, p.W, p.H, pu, pv, zf, e_z);
        if (in == 0) continue;
        const int4 *row = reinterpret_cast<const int4 *>(p.yawtab + A.yaw * 12);
        if (in > 0) {
            const uint32_t D = __ldg(A.D + pv * p.W + pu);
            if constexpr (STATS) ++st_reads;
            // z <= D  <=>  Z < (D + 1) / 2^16 (voxels); lim within relative 2^-23 of that
            const float lim = ((float)D + 1.0f) * (1.0f / 65536.0f);
            if (zf + e_z < lim * (1.0f - 2.4e-7f)) return true;
            if (zf - e_z >= lim * (1.0f + 2.4e-7f)) continue;
            const int4 r2 = __ldg(row + 2);
            const int64_t Za = (int64_t)r2.x * ax + (int64_t)r2.y * ay + (int64_t)r2.z * az;
            if (Za < (((int64_t)D + 1) << 16)) return true;
            continue;
        }
        // near a pixel boundary or Z = 0: the exact projection (Eq. 5)
        const int4 r0 = __ldg(row), r1 = __ldg(row + 1), r2 = __ldg(row + 2);  // ck sk mu0 mu1 | mu2 mv0 mv1 mv2 | mz0 mz1 mz2 -
        const int64_t Za = (int64_t)r2.x * ax + (int64_t)r2.y * ay + (int64_t)r2.z * az;
        if (Za <= 0) continue;
        const int64_t Ua = (int64_t)r0.z * ax + (int64_t)r0.w * ay + (int64_t)r1.x * az;
        const int64_t Va = (int64_t)r1.y * ax + (int64_t)r1.z * ay + (int64_t)r1.w * az;
        const float zi = __fdividef(1.0f, zf);
        const float uf = fmaf(A.m[0], ex, fmaf(A.m[1], ey, A.m[2] * ez)) * zi;
        const float vf = fmaf(A.m[3], ex, fmaf(A.m[4], ey, A.m[5] * ez)) * zi;
        if (!pixel_in(Ua, Za, uf, p.W, pu) || !pixel_in(Va, Za, vf, p.H, pv)) continue;
        const uint32_t D = __ldg(A.D + pv * p.W + pu);
        if constexpr (STATS) ++st_reads;
        if (Za < (((int64_t)D + 1) << 16)) return true;
    }
    return false;
}

// Stage C: the ancestor test of 32 (or the last n) counted voxels, then their per-yaw counts: every
// yaw of the voxel's mask gains an absolute count, and a marginal one unless an ancestor observes it.
template <bool STATS>
__device__ __forceinline__ void node_anc_stage(const LevelParams &p, NodeWarp &Q, int &nq, int lane,
                                               const AncRec *anc, int na, int z, int K, NodeStats &st, bool full) {
    const bool have = full || lane < nq;
    const unsigned long long key = Q.key[lane], mask0 = Q.mask[lane];
    if (full) {
        const unsigned long long rk = lane + 32 < nq ? Q.key[lane + 32] : 0ull;
        const unsigned long long rm = lane + 32 < nq ? Q.mask[lane + 32] : 0ull;
        __syncwarp();
        if (lane + 32 < nq) {
            Q.key[lane] = rk;
            Q.mask[lane] = rm;
        }
        __syncwarp();
        nq -= 32;
    } else {
        nq = 0;
    }
    if (have) {
        const int x = (int)(key & 0xFFF), y = (int)((key >> 12) & 0xFFF);
        const bool obs = observed_fast<STATS>(p, anc, na, x, y, z, st.anc, st.reads);
        const int k0 = (int)(key >> 24);
        unsigned long long mask = mask0;
        while (mask) {
            const int j = __ffsll((long long)mask) - 1;
            mask &= mask - 1;
            int kk = k0 + j;
            kk -= kk >= K ? K : 0;
            atomicAdd(Q.cnt + 2 * kk, 1);
            if (!obs) atomicAdd(Q.cnt + 2 * kk + 1, 1);
            if constexpr (STATS) ++st.smp;
        }
    }
    __syncwarp();
}


// One cast item: lane l's ray of the 8x4 tile `tile` (tx tiles per image row) of pair q of the
// level (node q / K, yaw q % K) runs the DDA to its first occupied voxel; its step index goes to
// `out` (the pair's step counts).
template <bool STATS>
__device__ __forceinline__ void cast_item(const LevelParams &p, const uint8_t *bocc, const uint8_t *sbocc, int l0, int q,
                                          int tile, int tx, uint16_t *out, int lane, uint32_t &st_rays,
                                          uint32_t &st_fine, uint32_t &st_skip) {
    const int i = (tile % tx) * kCastTileW + (lane % kCastTileW), j = (tile / tx) * kCastTileH + lane / kCastTileW;
    if (i >= p.W || j >= p.H) return;
    const int n = p.level_nodes[l0 + q / p.K];
    const int k = q % p.K;
    const int4 nd = p.node[n];
    const int4 b = p.body[j * p.W + i];
    const int32_t *yk = p.yawtab + k * 12;
    int dx, dy, dz;
    ray_dir(b, yk[0], yk[1], dx, dy, dz);
    const uint32_t m = cast_hit<STATS>(p.grid.g, bocc, sbocc, p.grid.nx, p.grid.ny, p.grid.nz, nd.x, nd.y, nd.z, dx, dy,
                                       dz, p.Tq, st_fine, st_skip);
    out[(size_t)j * p.W + i] = (uint16_t)m;
    if constexpr (STATS) ++st_rays;
}

// The per-node item's slice geometry: slice z (rank-th from the node's own height, alternately
// above and below) and its 32-row block (rb-th from the middle) of node n's range ball.
struct NodeSlice {
    int4 nd;
    int z, yb, yhi;
    float Pxf, Pyf, rz, h2;
};
// False when the item holds no voxel that can count: outside the grid or the ball, beyond the
// frustum's elevation band, or past the slice's last row.
__device__ __forceinline__ bool node_slice(const LevelParams &p, int n, int rank, int rb, int yb_n, NodeSlice &S) {
    const int Rv = (int)(p.Tq >> 16) + 2;
    const int zi = Rv + ((rank & 1) ? (rank + 1) >> 1 : -(rank >> 1));
    const int yblk = (yb_n - 1) / 2 + ((rb & 1) ? (rb + 1) >> 1 : -(rb >> 1));
    S.nd = p.node[n];
    const int4 nd = S.nd;
    S.z = (nd.z >> 16) - Rv + zi;
    if (S.z < 0 || S.z >= p.grid.nz) return false;
    const float s16 = 1.0f / 65536.0f;
    const float R = (float)p.Tq * s16 + 1.0f;
    S.Pxf = (float)nd.x * s16 - 0.5f;
    S.Pyf = (float)nd.y * s16 - 0.5f;
    const float Pzf = (float)nd.z * s16 - 0.5f;
    S.rz = small_int_to_float(S.z) - Pzf;
    S.h2 = R * R - S.rz * S.rz;
    if (S.h2 < 0.f) return false;
    // no voxel of this slice can be in the band: above the slice's plane every centre's elevation is
    // at least that of the outermost one, below it at most that of the outermost one
    const float rho_max = sqrtf(S.h2);
    const float eps = 0.01f * (rho_max + fabsf(S.rz)) + 0.05f;
    if ((S.rz > 0.f && p.band_thi < 1e29f && S.rz > p.band_thi * rho_max + eps) ||
        (S.rz < 0.f && p.band_tlo > -1e29f && S.rz < p.band_tlo * rho_max - eps))
        return false;
    const float hy = sqrtf(S.h2);
    const int ylo = max(0, (int)floorf(S.Pyf - hy) - 1);
    S.yhi = min(p.grid.ny - 1, (int)ceilf(S.Pyf + hy) + 1);
    S.yb = ylo + 32 * yblk;  // this item's rows: block yblk of the slice's rows [ylo, yhi]
    return S.yb <= S.yhi;
}

// The node's ancestors (Sec. IV-B), parent first, as the per-warp records of the ancestor test;
// returns how many the mode tests.
__device__ __forceinline__ int node_ancestors(const LevelParams &p, int n, AncRec *anc, int lane) {
    const int2 ar = p.anc_range[n];
    int na = ar.y;
    if (p.mode == MIG_MODE_ABSOLUTE) na = 0;
    else if (p.mode == MIG_MODE_SINGLE_PARENT) na = min(na, 1);
    na = min(na, p.max_anc);
    fill_anc_records(p, ar, na, anc, lane);
    return na;
}

// Adds the warp's per-yaw counters to node n's (abs, marginal) counters of the level and clears them.
__device__ __forceinline__ void node_flush(const LevelParams &p, int n, NodeWarp &Q, int lane) {
    for (int t = lane; t < 2 * p.K; t += 32) {
        const int v = Q.cnt[t];
        if (v) {
            atomicAdd(p.cnt + ((size_t)n * p.K + (t >> 1)) * 2 + (t & 1), v);
            Q.cnt[t] = 0;
        }
    }
    __syncwarp();
}

// One per-node item (its slice S): stage A enumerates the block's unknown voxels in the frustum's
// elevation band; stage B finds, per voxel, the yaws that count it; stage C tests the counted voxels
// against the ancestors' depth buffers once per voxel and adds the per-yaw counts to the warp's
// counters Q.cnt. s_yi / s_yf: the yaw rows (12 ints per yaw, as in the yaw table) and their
// projection rows as floats (9 per yaw, divided by 2^16); steps: the node's step counts (K images).
template <bool STATS>
__device__ __forceinline__ void node_run(const LevelParams &p, const NodeSlice &S, const int *s_yi, const float *s_yf,
                                         const uint16_t *steps, NodeWarp &Q, const AncRec *anc, int na, int lane,
                                         NodeStats &st) {
    const unsigned lt_mask = (1u << lane) - 1u;
    const int K = p.K;
    const int gnx = p.grid.nx, gny = p.grid.ny;
    const size_t WH = (size_t)p.W * p.H;
    const float yaw_scale = (float)K * 0.15915494309189535f;  // K / (2 pi)
    const float Tv = (float)p.Tq * (1.0f / 65536.0f);           // the range in voxels
    const int4 nd = S.nd;
    const int v0x = nd.x >> 16, v0y = nd.y >> 16, v0z = nd.z >> 16;
    const int z = S.z, yb = S.yb, yhi = S.yhi;
    const float Pxf = S.Pxf, Pyf = S.Pyf, rz = S.rz, h2 = S.h2;
    const int zq = (z << 16) + 32768 - nd.z;
    const float ez = (float)zq * (1.0f / 65536.0f);
    int nu = 0, nq = 0;

    // stage B: for 32 voxels (one per lane), the yaws that count them: every yaw whose frustum may
    // hold the voxel (azimuth window) in turn gets its owner pixel (Eq. 5) and the reach test by
    // step index; the visit test is decided by visit_surely where it can, else queued for the exact
    // test, which runs 32 pairs at a time
    auto yaw_stage = [&](bool full) {
        const bool have = full || lane < nu;
        const unsigned long long e = full ? q_pop32(Q.unk, nu, lane) : Q.unk[lane];
        if (!full) nu = 0;
        const int x = (int)(e & 0xFFF), y = (int)((e >> 12) & 0xFFF);
        // the yaws whose frustum may hold the centre: psi_k within az_half of its azimuth (every
        // yaw near the vertical axis)
        const float fxr = small_int_to_float(x) - Pxf, fyr = small_int_to_float(y) - Pyf;
        int klo = 0, nk = have ? K : 0;
        if (have && fxr * fxr + fyr * fyr >= 4.0f && p.az_half < 3.0f) {
            const float phi = atan2f(fyr, fxr);
            const int a0 = (int)ceilf((phi - p.az_half) * yaw_scale);
            const int a1 = (int)floorf((phi + p.az_half) * yaw_scale);
            nk = max(0, min(K, a1 - a0 + 1));
            klo = ((a0 % K) + K) % K;
        }
        Q.vm[lane] = 0ull;
        int nx = 0;  // (voxel, yaw) pairs queued in Q.xq for the exact visit test
        // exact visit test by the owner ray (event order of its DDA, range) of 32 queued pairs; the
        // pairs that pass set their bit in the voxel's mask word
        auto exact_stage = [&](bool xfull) {
            const bool xh = xfull || lane < nx;
            const unsigned long long q = xfull ? q_pop32(Q.xq, nx, lane) : Q.xq[lane];
            if (!xfull) nx = 0;
            if (xh) {
                const int qx = (int)(q & 0xFFF), qy = (int)((q >> 12) & 0xFFF);
                const int pix = (int)((q >> 24) & 0x3FFFFF), k = (int)((q >> 46) & 0x3F);
                const int j = (int)((q >> 52) & 0x3F), r = (int)(q >> 58);
                int dx, dy, dz;
                ray_dir(p.body[pix], s_yi[12 * k], s_yi[12 * k + 1], dx, dy, dz);
                if (visit_index(nd.x, nd.y, nd.z, dx, dy, dz, qx, qy, z, p.Tq) >= 0) atomicOr(Q.vm + r, 1ull << j);
            }
            __syncwarp();
        };
        __syncwarp();
        const int rxq = (x << 16) + 32768 - nd.x, ryq = (y << 16) + 32768 - nd.y;
        const int man = abs(x - v0x) + abs(y - v0y) + abs(z - v0z);
        // the centre's offset from the camera in voxels, from its exact Q16 value
        const float ex = (float)rxq * (1.0f / 65536.0f), ey = (float)ryq * (1.0f / 65536.0f);
        const float rinf = fmaxf(fabsf(ex), fmaxf(fabsf(ey), fabsf(ez)));
        unsigned long long mask = 0ull;
        const int nk_max = __reduce_max_sync(0xffffffffu, (unsigned)nk);
        for (int j = 0; j < nk_max; ++j) {
            bool exact = false;
            int pix = 0, k = 0;
            if (j < nk) {
                k = klo + j;
                k -= k >= K ? K : 0;
                const int *rw = s_yi + 12 * k;
                const float *fw = s_yf + 9 * k;
                // the owner pixel (Eq. 5): from the float rows where their error bound decides it,
                // else by the exact integer projection
                int pu = 0, pv = 0;
                float zf_, ez_;
                int in = pixel_fast(fw, ex, ey, ez, rinf, p.W, p.H, pu, pv, zf_, ez_);
                if (in < 0) {
                    in = 0;
                    const int64_t Z = (int64_t)rw[8] * rxq + (int64_t)rw[9] * ryq + (int64_t)rw[10] * zq;
                    if (Z > 0) {
                        const int64_t U = (int64_t)rw[2] * rxq + (int64_t)rw[3] * ryq + (int64_t)rw[4] * zq;
                        const int64_t V = (int64_t)rw[5] * rxq + (int64_t)rw[6] * ryq + (int64_t)rw[7] * zq;
                        const float zi_ = __fdividef(1.0f, fmaf(fw[6], ex, fmaf(fw[7], ey, fw[8] * ez)));
                        in = pixel_in(U, Z, fmaf(fw[0], ex, fmaf(fw[1], ey, fw[2] * ez)) * zi_, p.W, pu) &&
                             pixel_in(V, Z, fmaf(fw[3], ex, fmaf(fw[4], ey, fw[5] * ez)) * zi_, p.H, pv);
                    }
                }
                if (in) {
                    pix = pv * p.W + pu;
                    if (man < (int)__ldg(steps + (size_t)k * WH + pix)) {  // before the owner ray's hit
                        if constexpr (STATS) ++st.visit;
                        int dx, dy, dz;
                        ray_dir(p.body[pix], rw[0], rw[1], dx, dy, dz);
                        if (visit_surely(ex, ey, ez, dx, dy, dz, Tv)) mask |= 1ull << j;
                        else exact = true;
                    }
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, exact);
            if (exact)
                Q.xq[nx + __popc(bal & lt_mask)] = (unsigned long long)x | ((unsigned long long)y << 12) |
                                                   ((unsigned long long)pix << 24) | ((unsigned long long)k << 46) |
                                                   ((unsigned long long)j << 52) | ((unsigned long long)lane << 58);
            nx += __popc(bal);
            __syncwarp();
            if (nx >= 32) exact_stage(true);
        }
        if (nx > 0) exact_stage(false);
        mask |= Q.vm[lane];
        const bool put = have && mask != 0ull;
        const unsigned bal = __ballot_sync(0xffffffffu, put);
        if (put) {
            const int slot = nq + __popc(bal & lt_mask);
            Q.key[slot] = (unsigned long long)x | ((unsigned long long)y << 12) | ((unsigned long long)klo << 24);
            Q.mask[slot] = mask;
        }
        nq += __popc(bal);
        __syncwarp();
        if (nq >= 32) node_anc_stage<STATS>(p, Q, nq, lane, anc, na, z, K, st, true);
    };

    {
        const int y = yb + lane;
        int xa = 0, len = 0;
        if (y <= yhi) {
            const float ry = small_int_to_float(y) - Pyf;
            const float hx2 = h2 - ry * ry;
            if (hx2 >= 0.f) {
                const float hx = sqrtf(hx2);
                xa = max(0, (int)floorf(Pxf - hx) - 1);
                len = max(0, min(gnx - 1, (int)ceilf(Pxf + hx) + 1) - xa + 1);
            }
        }
        int incl = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += v;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        for (int base = 0; base < tot; base += 32) {
            const int f = base + lane;
            int r = 0;
#pragma unroll
            for (int sh = 16; sh >= 1; sh >>= 1) {
                const int cv = __shfl_sync(0xffffffffu, incl, r + sh - 1);
                if (cv <= f) r += sh;
            }
            r = min(r, 31);
            const int rxa = __shfl_sync(0xffffffffu, xa, r);
            const int rstart = __shfl_sync(0xffffffffu, incl - len, r);
            bool unk = false;
            int x = 0;
            if (f < tot) {
                x = rxa + (f - rstart);
                if constexpr (STATS) ++st.cand;
                const uint32_t addr = ((uint32_t)z * (uint32_t)gny + (uint32_t)(yb + r)) * (uint32_t)gnx + (uint32_t)x;
                if (load_code(p.grid.g, addr, p.grid, p.bounds_err) == kUnknown) {
                    // inside the frustum's elevation band (widened; exact tests follow)
                    const float fx = small_int_to_float(x) - Pxf, fy = small_int_to_float(yb + r) - Pyf;
                    const float rho = sqrtf(fx * fx + fy * fy);
                    const float eps = 0.01f * (rho + fabsf(rz)) + 0.05f;
                    unk = (p.band_thi >= 1e29f || rz <= p.band_thi * rho + eps) &&
                          (p.band_tlo <= -1e29f || rz >= p.band_tlo * rho - eps);
                }
                if constexpr (STATS) st.unk += unk;
            }
            q_push(Q.unk, nu, unk, (unsigned long long)x | ((unsigned long long)(yb + r) << 12), lt_mask);
            if (nu >= 32) yaw_stage(true);
        }
    }
    if (nu > 0) yaw_stage(false);
    while (nq >= 32) node_anc_stage<STATS>(p, Q, nq, lane, anc, na, z, K, st, true);
    if (nq > 0) node_anc_stage<STATS>(p, Q, nq, lane, anc, na, z, K, st, false);
}

}  // namespace dev
}  // namespace mig
