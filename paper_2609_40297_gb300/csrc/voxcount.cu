// Owned-voxel count of one tree level (Sec. IV-B, the counts of Eq. 1 and Eq. 2 by depth
// buffers), in two kernels per chunk of (node, yaw) pairs:
//   cast_kernel  - every pixel ray of every pair runs the DDA to its stopping point and stores
//                  the number of steps it takes (uint16 per ray);
//   voxel_kernel - for every pair, the voxels within range of the node are enumerated slice by
//                  slice (z), rows clipped to the camera frustum; each unknown voxel goes to the
//                  pixel that owns it (its centre's projection) and counts as absolute gain iff
//                  that pixel's DDA visits it within the stored step count; counted voxels are
//                  tested 32 at a time against the ancestors' depth buffers (marginal gain).
// Results are identical to the ray-by-ray count kernel (and the CPU oracle) bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.h"
#include "mig.h"
#include "voxcount.cuh"
#include "voxcount.h"

namespace mig {

namespace {

using namespace dev;

constexpr int kCastWarps = 8;   // 256-thread CTAs, one ray per thread
constexpr int kVoxWarps = 8;
constexpr int kVoxQueue = 64;   // per-warp queue of counted samples waiting for the ancestor test

__device__ __forceinline__ int level_pairs(const LevelParams &p) {
    return (p.level_off[p.lvl + 1] - p.level_off[p.lvl]) * p.K;
}

// ------------------------------------------------------------------------------ cast kernel
// Warp work item = (pair q of the chunk, 8x4 pixel tile); one ray per lane.
template <bool STATS>
__global__ void __launch_bounds__(kCastWarps * 32) cast_kernel(const LevelParams p) {
    const int lane = threadIdx.x & 31;
    const int l0 = p.level_off[p.lvl];
    const int q1 = min(p.q1, level_pairs(p));
    if (p.q0 >= q1) return;
    const int tx = (p.W + 7) >> 3, ty = (p.H + 3) >> 2;
    const long long items = (long long)(q1 - p.q0) * tx * ty;
    const size_t WH = (size_t)p.W * p.H;
    const uint8_t *bocc = p.grid.g + bocc_offset(p.grid.nx, p.grid.ny, p.grid.nz);
    uint32_t st_rays = 0, st_fine = 0, st_skip = 0;
    for (long long it = (long long)blockIdx.x * kCastWarps + (threadIdx.x >> 5); it < items;
         it += (long long)gridDim.x * kCastWarps) {
        const int tile = (int)(it % (tx * ty));
        const int ql = (int)(it / (tx * ty));
        const int q = p.q0 + ql;
        const int i = (tile % tx) * 8 + (lane & 7), j = (tile / tx) * 4 + (lane >> 3);
        if (i >= p.W || j >= p.H) continue;
        const int n = p.level_nodes[l0 + q / p.K];
        const int k = q % p.K;
        const int4 nd = p.node[n];
        const int4 b = p.body[j * p.W + i];
        const int32_t *yk = p.yawtab + k * 12;
        int dx, dy, dz;
        ray_dir(b, yk[0], yk[1], dx, dy, dz);
        const uint32_t m = cast_steps<STATS>(p.grid.g, bocc, p.grid.nx, p.grid.ny, p.grid.nz, nd.x, nd.y, nd.z, dx, dy,
                                             dz, p.Tq, st_fine, st_skip);
        p.steps[(size_t)ql * WH + (size_t)j * p.W + i] = (uint16_t)m;
        if constexpr (STATS) ++st_rays;
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
// Warp work item = (pair q of the chunk, slice z of the node's range ball). Lanes take 32 rows
// (y) of the slice at a time, clip each row to the frustum and the ball, and then walk the rows'
// voxels 32 at a time (flattened over the rows with a warp prefix sum).
template <bool STATS>
__global__ void __launch_bounds__(kVoxWarps * 32, 4) voxel_kernel(const LevelParams p) {
    extern __shared__ AncRec s_anc_dyn[];
    __shared__ unsigned long long s_q[kVoxWarps][kVoxQueue];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    AncRec *anc = s_anc_dyn + warp * p.max_anc;
    unsigned long long *q = s_q[warp];
    const int l0 = p.level_off[p.lvl];
    const int q1 = min(p.q1, level_pairs(p));
    if (p.q0 >= q1) return;
    const int Rv = (int)(p.Tq >> 16) + 2;    // voxels: every visited voxel's centre is nearer than T + 1
    const int slices = 2 * Rv + 1;
    const long long items = (long long)(q1 - p.q0) * slices;
    const float R = (float)p.Tq * (1.0f / 65536.0f) + 1.0f, R2 = R * R;
    const int gnx = p.grid.nx, gny = p.grid.ny, gnz = p.grid.nz;
    const size_t WH = (size_t)p.W * p.H;
    uint32_t st_cand = 0, st_unk = 0, st_visit = 0, st_anc = 0, st_reads = 0;
    int cur_node = -1, na = 0;
    for (long long it = (long long)blockIdx.x * kVoxWarps + warp; it < items; it += (long long)gridDim.x * kVoxWarps) {
        const int ql = (int)(it / slices), zi = (int)(it % slices);
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
        // the frustum of the owner rule as half-spaces of the centre offset: Z > 0, U >= 0,
        // W Z - U > 0, V >= 0, H Z - V > 0 (Eq. 5; W Z - U and H Z - V in exact integers)
        HalfSpace hs[5];
        frustum_half_spaces(mu0, mu1, mu2, mv0, mv1, mv2, mz0, mz1, mz2, p.W, p.H, hs);
        const HalfSpace &hz = hs[0], &hu = hs[1], &hv = hs[3];
        const float hy = sqrtf(h2);
        const int ylo = max(0, (int)floorf(Pyf - hy) - 1), yhi = min(gny - 1, (int)ceilf(Pyf + hy) + 1);
        int c_abs = 0, c_mrg = 0, qn = 0;
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
                bool counted = false;
                int x = 0, yy = 0;
                if (f < tot) {
                    x = rxa + (f - rstart);
                    yy = yb + r;
                    if constexpr (STATS) ++st_cand;
                    const uint32_t addr = ((uint32_t)z * (uint32_t)gny + (uint32_t)yy) * (uint32_t)gnx + (uint32_t)x;
                    if (load_code(p.grid.g, addr, p.grid, p.bounds_err) == kUnknown) {
                        if constexpr (STATS) ++st_unk;
                        // owner pixel of the centre (Eq. 5): floor(U / Z), floor(V / Z)
                        const int rx = (x << 16) + 32768 - nd.x, ryq = (yy << 16) + 32768 - nd.y,
                                  rzq = (z << 16) + 32768 - nd.z;
                        const int64_t Z = (int64_t)mz0 * rx + (int64_t)mz1 * ryq + (int64_t)mz2 * rzq;
                        const int64_t U = (int64_t)mu0 * rx + (int64_t)mu1 * ryq + (int64_t)mu2 * rzq;
                        const int64_t V = (int64_t)mv0 * rx + (int64_t)mv1 * ryq + (int64_t)mv2 * rzq;
                        if (Z > 0 && U >= 0 && U < (int64_t)p.W * Z && V >= 0 && V < (int64_t)p.H * Z) {
                            const float fxr = small_int_to_float(x) - Pxf, fyr = small_int_to_float(yy) - Pyf;
                            const float zi_ = __frcp_rn(fmaf(hz.a, fxr, fmaf(hz.b, fyr, hz.c * rz)));
                            const float uf = fmaf(hu.a, fxr, fmaf(hu.b, fyr, hu.c * rz)) * zi_;
                            const float vf = fmaf(hv.a, fxr, fmaf(hv.b, fyr, hv.c * rz)) * zi_;
                            const int pi = floor_div_from(U, Z, uf, p.W);
                            const int pj = floor_div_from(V, Z, vf, p.H);
                            const int man = abs(x - (nd.x >> 16)) + abs(yy - (nd.y >> 16)) + abs(z - (nd.z >> 16));
                            const int lim = p.steps[(size_t)ql * WH + (size_t)pj * p.W + pi];
                            if (man <= lim) {
                                if constexpr (STATS) ++st_visit;
                                int dx, dy, dz;
                                ray_dir(p.body[pj * p.W + pi], ck, sk, dx, dy, dz);
                                counted = visit_index(nd.x, nd.y, nd.z, dx, dy, dz, x, yy, z) >= 0;
                            }
                        }
                    }
                }
                // counted samples: absolute gain, then the ancestor test in batches of 32 (Sec. IV-B)
                c_abs += counted;
                const unsigned bal = __ballot_sync(0xffffffffu, counted);
                if (bal) {
                    if (counted)
                        q[qn + __popc(bal & lt_mask)] = (unsigned long long)x | ((unsigned long long)yy << 16) |
                                                        ((unsigned long long)z << 32);
                    qn += __popc(bal);
                    if (qn >= 32) {
                        __syncwarp();
                        const unsigned long long sm = q[lane];
                        c_mrg += !observed<STATS>(HotDirect{p}, anc, na, (int)(sm & 0xFFFF), (int)((sm >> 16) & 0xFFFF),
                                                  (int)(sm >> 32), st_anc, st_reads);
                        __syncwarp();
                        if (lane < qn - 32) q[lane] = q[lane + 32];
                        __syncwarp();
                        qn -= 32;
                    }
                }
            }
        }
        __syncwarp();
        if (lane < qn) {
            const unsigned long long sm = q[lane];
            c_mrg += !observed<STATS>(HotDirect{p}, anc, na, (int)(sm & 0xFFFF), (int)((sm >> 16) & 0xFFFF),
                                      (int)(sm >> 32), st_anc, st_reads);
        }
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
    const long long cast_warps = (long long)(c.q1 - c.q0) * ((c.W + 7) / 8) * ((c.H + 3) / 4);
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

void launch_vox_level(const LevelParams &p, long long pairs, int num_sms, int vox_ctas, cudaStream_t s) {
    for (long long q0 = 0; q0 < pairs; q0 += p.steps_cap) {
        LevelParams c = p;
        c.q0 = (int)q0;
        c.q1 = (int)std::min<long long>(pairs, q0 + p.steps_cap);
        launch_cast_chunk(c, num_sms, s);
        launch_voxel_chunk(c, num_sms, vox_ctas, s);
    }
}

void launch_bocc(uint8_t *grid, int nx, int ny, int nz, int x0, int y0, int z0, int dx, int dy, int dz, cudaStream_t s) {
    const int bx0 = x0 >> 3, by0 = y0 >> 3, bz0 = z0 >> 3;
    const int bx1 = (x0 + dx + 7) >> 3, by1 = (y0 + dy + 7) >> 3, bz1 = (z0 + dz + 7) >> 3;
    const long long total = (long long)(bx1 - bx0) * (by1 - by0) * (bz1 - bz0);
    const int grid_ = (int)std::max<long long>(1, std::min<long long>((total + 7) / 8, 4096));
    bocc_kernel<<<grid_, 256, 0, s>>>(grid, nx, ny, nz, bx0, by0, bz0, bx1, by1, bz1);
}

}  // namespace mig
