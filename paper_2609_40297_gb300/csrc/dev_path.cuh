// Device-side steps of the marginal-gain path, shared by the per-level kernels (kernels.cu)
// and the batched persistent kernel (batch.cu): the integer DDA (Sec. IV-B), the owner test
// (a voxel counts only for the ray of the pixel containing its centre's projection), the
// ancestor depth test (Sec. IV-B), yaw selection (Sec. III-B) and depth rendering (Sec. IV-A).
// All result-deciding arithmetic is integer: positions Q16 voxel units, ray directions Q30,
// projection rows Q16, depths Q16.16.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "mig.h"

// Voxel layout of the device grid: 0 = 8x8x8 bricks of 512 B (z-major inside a brick),
// 1 = x-fastest rows (the host order), stepped with an incremental address.
#ifndef MIG_LAYOUT
#define MIG_LAYOUT 1
#endif
// 1 = the chunk's own-camera constants (projection rows, yaw cos/sin, node position) are read
// from the warp's shared-memory slot at each use instead of being held in registers.
#ifndef MIG_CAM_SMEM
#define MIG_CAM_SMEM 1
#endif
// Count loop: each lane runs MIG_COUNT_BLOCK DDA steps of its ray between two warp-wide
// exchanges (ray refill, sample queue); 0 = one exchange per step.
#ifndef MIG_COUNT_BLOCK
#define MIG_COUNT_BLOCK 4
#endif
// Minimum resident count-kernel CTAs per SM requested from the register allocator.
#ifndef MIG_COUNT_MINB
#define MIG_COUNT_MINB 4
#endif

#ifndef MIG_DEBUG_BOUNDS
#define MIG_DEBUG_BOUNDS 0
#endif

namespace mig {
namespace dev {

constexpr int kOcc = 2;

// Checked builds (MIG_DEBUG_BOUNDS=1): an index outside its buffer sets `bit` in *err (when err is
// not NULL) and the access is skipped; other builds compile the check away.
constexpr int kBoundsVoxel = 1, kBoundsArena = 2, kBoundsDepth = 4;
__device__ __forceinline__ bool in_bounds(int32_t *err, bool ok, int bit) {
#if MIG_DEBUG_BOUNDS
    if (!ok && err) atomicOr(err, bit);
    return ok;
#else
    (void)err;
    (void)ok;
    (void)bit;
    return true;
#endif
}

__device__ __forceinline__ uint32_t grid_cells(int nx, int ny, int nz) {
#if MIG_LAYOUT == 1
    return (uint32_t)nx * (uint32_t)ny * (uint32_t)nz;
#else
    return (uint32_t)((nx + 7) >> 3) * (uint32_t)((ny + 7) >> 3) * (uint32_t)((nz + 7) >> 3) * 512u;
#endif
}

// The code of the ray's current voxel (an occupied code for a checked build's skipped access).
__device__ __forceinline__ uint8_t load_code(const uint8_t *g, uint32_t a, const GridView &G, int32_t *err) {
    if (!in_bounds(err, a < grid_cells(G.nx, G.ny, G.nz), kBoundsVoxel)) return (uint8_t)kOcc;
    return __ldg(g + a);
}

// Depth-buffer arena write of one pixel of the buffer in slot `slot`.
__device__ __forceinline__ void arena_store(uint32_t *arena, int slots, int slot, size_t texel, size_t WH, uint32_t v,
                                            int32_t *err) {
    if (!in_bounds(err, slot >= 0 && (slots == 0 || slot < slots) && texel < WH, kBoundsArena)) return;
    arena[(size_t)slot * WH + texel] = v;
}
constexpr int kUnknown = 0;
constexpr uint32_t kQ16 = 65536;

__device__ __forceinline__ uint32_t voxel_addr(const GridView &G, int x, int y, int z) {
#if MIG_LAYOUT == 1
    return ((uint32_t)z * (uint32_t)G.ny + (uint32_t)y) * (uint32_t)G.nx + (uint32_t)x;
#else
    const uint32_t b = ((uint32_t)(z >> 3) * (uint32_t)G.nby + (uint32_t)(y >> 3)) * (uint32_t)G.nbx + (uint32_t)(x >> 3);
    return (b << 9) | ((uint32_t)(z & 7) << 6) | ((uint32_t)(y & 7) << 3) | (uint32_t)(x & 7);
#endif
}

// Per-axis DDA set-up (Sec. IV-B, Amanatides-Woo). n = distance to the next face (Q16),
// ad = |d| (Q30), s = step sign, l = face limit: crossing k along this axis is at n + k 2^16 and
// is taken iff it stays inside the grid and starts before the range T (t = (n + k 2^16) / ad < T),
// i.e. iff the current n is below l. An axis with d = 0 is never stepped (l = n); it still gets
// s = 1 and n = distance to the upper face, so that s (n - 2^15) is the voxel-centre offset on
// every axis (see voxel_offset).
__device__ __forceinline__ void axis_init(int P, int d, int N, int64_t Tq, int &v, uint32_t &n, uint32_t &ad, int &s,
                                          uint32_t &l) {
    v = P >> 16;
    int grid_rem;
    if (d < 0) {
        s = -1;
        ad = (uint32_t)(-d);
        n = (uint32_t)(P - (v << 16));
        grid_rem = v;
    } else {
        s = 1;
        ad = (uint32_t)d;
        n = (uint32_t)(((v + 1) << 16) - P);
        grid_rem = N - 1 - v;
        if (d == 0) {
            l = n;
            return;
        }
    }
    const uint64_t lim = ((uint64_t)Tq * ad + ((1ull << 30) - 1)) >> 30;  // n >= lim  <=>  t >= T
    const int64_t range_rem = (n >= lim) ? 0 : (int64_t)((lim - n + (kQ16 - 1)) >> 16);
    l = n + ((uint32_t)min((int64_t)grid_rem, range_rem) << 16);
}

// DDA state of one ray. The current voxel is not stored: along an axis with step sign s, the
// centre of the current voxel lies s (n - 2^15) (Q16) from the ray origin, because n is the
// distance from the origin to the voxel's far face along the ray's direction of travel.
struct RayIn {
    uint32_t nx, ny, nz, adx, ady, adz, lx, ly, lz;
    int sx, sy, sz;
#if MIG_LAYOUT == 1
    uint32_t addr;
    int dax, day, daz;  // signed address strides of one step along each axis
#else
    int vx, vy, vz;
#endif
};

// Q16 offset, along one axis, of the current voxel's centre from the ray origin.
__device__ __forceinline__ int voxel_offset(uint32_t n, int s) { return s * (int)(n - 32768u); }

__device__ __forceinline__ void ray_init_dims(RayIn &r, int gnx, int gny, int gnz, const GridView &G, int Px, int Py,
                                              int Pz, int dx, int dy, int dz, int64_t Tq) {
    int vx, vy, vz;
    axis_init(Px, dx, gnx, Tq, vx, r.nx, r.adx, r.sx, r.lx);
    axis_init(Py, dy, gny, Tq, vy, r.ny, r.ady, r.sy, r.ly);
    axis_init(Pz, dz, gnz, Tq, vz, r.nz, r.adz, r.sz, r.lz);
#if MIG_LAYOUT == 1
    (void)G;
    r.addr = ((uint32_t)vz * (uint32_t)gny + (uint32_t)vy) * (uint32_t)gnx + (uint32_t)vx;
    r.dax = r.sx;
    r.day = r.sy * gnx;
    r.daz = r.sz * gnx * gny;
#else
    (void)gnx;
    (void)gny;
    r.vx = vx;
    r.vy = vy;
    r.vz = vz;
#endif
}

__device__ __forceinline__ void ray_init(RayIn &r, const GridView &G, int Px, int Py, int Pz, int dx, int dy, int dz,
                                         int64_t Tq) {
    ray_init_dims(r, G.nx, G.ny, G.nz, G, Px, Py, Pz, dx, dy, dz, Tq);
}

__device__ __forceinline__ uint32_t ray_addr(const RayIn &r, const GridView &G) {
#if MIG_LAYOUT == 1
    (void)G;
    return r.addr;
#else
    return voxel_addr(G, r.vx, r.vy, r.vz);
#endif
}

// World direction of (yaw k, pixel): yaw rotation of the body-frame ray, floored (Q30).
__device__ __forceinline__ void ray_dir(const int4 b, int ck, int sk, int &dx, int &dy, int &dz) {
    const int64_t bx = b.x, by = b.y;
    dx = (int)(((int64_t)ck * bx - (int64_t)sk * by) >> 30);
    dy = (int)(((int64_t)sk * bx + (int64_t)ck * by) >> 30);
    dz = b.z;
}

// One step of the DDA: picks the axis with the smallest next crossing (ties x, y, z), stops if
// that crossing leaves the grid or starts at t >= T. Returns false when the ray ends.
// DEPTH: also report that crossing's face distance / speed (ne / ade): the exit of the current
// voxel, which is the entry of the new one when the step is taken (reported on either return).
template <bool DEPTH>
__device__ __forceinline__ bool ray_step(RayIn &r, uint32_t &ne, uint32_t &ade) {
    // lexicographic minimum of (t, axis) in two comparisons: the earlier of x and y (ties x), then
    // that one against z (ties to it); t_a = n_a / ad_a compared by cross products
    const bool xly = (uint64_t)r.nx * r.ady <= (uint64_t)r.ny * r.adx;
    const uint32_t nw = xly ? r.nx : r.ny, aw = xly ? r.adx : r.ady, lw = xly ? r.lx : r.ly;
    const bool bz = !((uint64_t)nw * r.adz <= (uint64_t)r.nz * aw);
    const bool bx = !bz && xly;
    const bool by = !bz && !xly;
    const uint32_t nc = bz ? r.nz : nw;
    if constexpr (DEPTH) {
        ne = nc;
        ade = bz ? r.adz : aw;
    }
    if (nc >= (bz ? r.lz : lw)) return false;
    r.nx += bx ? kQ16 : 0u;
    r.ny += by ? kQ16 : 0u;
    r.nz += bz ? kQ16 : 0u;
#if MIG_LAYOUT == 1
    r.addr += bx ? r.dax : (by ? r.day : r.daz);
#else
    r.vx += bx ? r.sx : 0;
    r.vy += by ? r.sy : 0;
    r.vz += bz ? r.sz : 0;
#endif
    return true;
}

// Depth (Q16.16 voxel units, camera z) of the entry point t_e = ne / ade of the hit voxel, or
// of the range endpoint.
__device__ __forceinline__ uint32_t hit_depth(bool hit, uint32_t ne, uint32_t ade, int dzc, int64_t Tq) {
    if (hit) return (uint32_t)(((uint64_t)ne * (uint32_t)dzc) / ade);
    return (uint32_t)(((uint64_t)Tq * (uint32_t)dzc) >> 30);
}

__device__ __forceinline__ void decode_item(const LevelParams &p, int item, int &li, int &k, int &tile) {
    tile = item % p.tiles;
    const int rest = item / p.tiles;
    k = rest % p.K;
    li = rest / p.K;
}

// ------------------------------------------------------------------------------- count kernel
// Work item = (node of the level, yaw k, tile of tile_w x tile_h pixel rays), taken by one warp
// from the level's atomic work counter (no CTA barrier: warps never wait for each other). Lane l
// casts rays l, l+32, ... of the tile and starts its next ray as soon as the current one ends.
// Unknown voxels owned by the ray (the voxel centre projects into this pixel) count as
// absolute gain; their coordinates go to a per-warp queue, and each full batch of 32 samples is
// tested against the ancestors' depth buffers with all 32 lanes at once (Sec. IV-B), so the
// rare, long ancestor test never runs one lane at a time.
constexpr int kWarps = 8;
constexpr int kCountBlock = MIG_COUNT_BLOCK > 0 ? MIG_COUNT_BLOCK : 1;
// per-warp sample queue: the main queue (< 32 carried + 32 x kCountBlock appended at an exchange)
// followed by 32 x kCountBlock private slots (one column per lane)
constexpr int kQueueMain = 32 * (kCountBlock + 1);
constexpr int kQueue = kQueueMain + 32 * kCountBlock;

struct AncRec {
    int px, py, pz, yaw;
    float fx, fy, fz;  // P / 2^16 - 1/2 (voxel units): voxel centre offset for the float estimate
    float m[9];        // projection rows / 2^16 (float estimate of U, V, Z)
    const uint32_t *D;
};

__device__ __forceinline__ float small_int_to_float(int v) {  // exact for 0 <= v < 2^23
    return __int_as_float(0x4B000000 | v) - 8388608.0f;
}

// floor(U / Z) for 0 <= U < bound * Z, Z > 0, from a float estimate, corrected exactly.
__device__ __forceinline__ int floor_div_from(int64_t U, int64_t Z, float est, int bound) {
    int q = __float_as_int(est - 0.5f + 12582912.0f) - 0x4B400000;  // nearest of est - 1/2
    q = max(0, min(q, bound - 1));
    while (q > 0 && (int64_t)q * Z > U) --q;
    while (q < bound - 1 && (int64_t)(q + 1) * Z <= U) ++q;
    return q;
}

// The pixel coordinate floor(U / Z) (Eq. 5) for Z > 0, and whether it lies in [0, bound): from a
// float estimate of U / Z, moved by exact integer products until q Z <= U < (q + 1) Z. One product
// and two comparisons when the estimate is right (the estimate only sets the start).
__device__ __forceinline__ bool pixel_in(int64_t U, int64_t Z, float est, int bound, int &q) {
    int c = __float2int_rd(fminf(fmaxf(est, -1.0f), (float)bound));
    int64_t lo = (int64_t)c * Z;
    while (lo > U) {
        if (--c < 0) return false;
        lo -= Z;
    }
    while (U - lo >= Z) {
        if (++c >= bound) return false;
        lo += Z;
    }
    q = c;
    return c >= 0 && c < bound;
}

// Sec. IV-B: is the centre of voxel (x, y, z) observed by any ancestor (z <= stored depth)?
// (The depth texel index is inside the buffer by construction: both pixel coordinates are clamped.)
template <bool STATS, class HOT>
__device__ __forceinline__ bool observed(const HOT &p, const AncRec *anc, int na, int x, int y, int z,
                                         uint32_t &st_anc, uint32_t &st_reads) {
    const float xf = small_int_to_float(x), yf = small_int_to_float(y), zf = small_int_to_float(z);
    for (int a = 0; a < na; ++a) {
        const AncRec &A = anc[a];
        const int ax = (x << 16) + 32768 - A.px;
        const int ay = (y << 16) + 32768 - A.py;
        const int az = (z << 16) + 32768 - A.pz;
        const int4 *row = reinterpret_cast<const int4 *>(p.yawtab() + A.yaw * 12);
        const int4 r0 = __ldg(row), r1 = __ldg(row + 1), r2 = __ldg(row + 2);  // ck sk mu0 mu1 | mu2 mv0 mv1 mv2 | mz0 mz1 mz2 -
        const int64_t Za = (int64_t)r2.x * ax + (int64_t)r2.y * ay + (int64_t)r2.z * az;
        if constexpr (STATS) ++st_anc;
        if (Za <= 0) continue;
        const int64_t Ua = (int64_t)r0.z * ax + (int64_t)r0.w * ay + (int64_t)r1.x * az;
        const int64_t Va = (int64_t)r1.y * ax + (int64_t)r1.z * ay + (int64_t)r1.w * az;
        const float rx = xf - A.fx, ry = yf - A.fy, rz = zf - A.fz;
        const float zi = __fdividef(1.0f, fmaf(A.m[6], rx, fmaf(A.m[7], ry, A.m[8] * rz)));
        const float uf = fmaf(A.m[0], rx, fmaf(A.m[1], ry, A.m[2] * rz)) * zi;
        const float vf = fmaf(A.m[3], rx, fmaf(A.m[4], ry, A.m[5] * rz)) * zi;
        int pu, pv;
        if (!pixel_in(Ua, Za, uf, p.W(), pu) || !pixel_in(Va, Za, vf, p.H(), pv)) continue;
        const uint32_t D = __ldg(A.D + pv * p.W() + pu);
        if constexpr (STATS) ++st_reads;
        if (Za < (((int64_t)D + 1) << 16)) return true;  // z <= D
    }
    return false;
}

// One count work item (node of the level, yaw k, tile of rays) for one warp. l0 = offset of
// the level in level_nodes; c = item index inside the level. anc / q = the warp's shared-memory
// ancestor records and sample queue.
// Loop-live parameters of the count path. HotDirect reads the level parameters themselves (for a
// kernel argument the compiler keeps them in uniform registers); HotStaged re-reads them at every
// use from the warp's shared-memory copy, so that kernels whose tree changes per work item do not
// hold them in per-thread registers.
struct HotVals {
    const uint8_t *g;
    const int4 *body;
    const int32_t *yawtab;
    long long Tq;
    int nx, ny, nz, W, H, tile_w, pad0, pad1;
};

__device__ __forceinline__ int lds32v(const int *ptr) {
    int v;
    asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(ptr)));
    return v;
}
__device__ __forceinline__ long long lds64v(const long long *ptr) {
    long long v;
    asm volatile("ld.shared.s64 %0, [%1];" : "=l"(v) : "r"((unsigned)__cvta_generic_to_shared(ptr)));
    return v;
}

struct HotDirect {
    const LevelParams &p;
    __device__ __forceinline__ const uint8_t *g() const { return p.grid.g; }
    __device__ __forceinline__ const int4 *body() const { return p.body; }
    __device__ __forceinline__ const int32_t *yawtab() const { return p.yawtab; }
    __device__ __forceinline__ int64_t Tq() const { return p.Tq; }
    __device__ __forceinline__ int nx() const { return p.grid.nx; }
    __device__ __forceinline__ int ny() const { return p.grid.ny; }
    __device__ __forceinline__ int nz() const { return p.grid.nz; }
    __device__ __forceinline__ int W() const { return p.W; }
    __device__ __forceinline__ int H() const { return p.H; }
    __device__ __forceinline__ int tile_w() const { return p.tile_w; }
};

struct HotStaged {
    const HotVals *s;
    __device__ __forceinline__ const uint8_t *g() const { return (const uint8_t *)lds64v((const long long *)&s->g); }
    __device__ __forceinline__ const int4 *body() const { return (const int4 *)lds64v((const long long *)&s->body); }
    __device__ __forceinline__ const int32_t *yawtab() const {
        return (const int32_t *)lds64v((const long long *)&s->yawtab);
    }
    __device__ __forceinline__ int64_t Tq() const { return lds64v(&s->Tq); }
    __device__ __forceinline__ int nx() const { return lds32v(&s->nx); }
    __device__ __forceinline__ int ny() const { return lds32v(&s->ny); }
    __device__ __forceinline__ int nz() const { return lds32v(&s->nz); }
    __device__ __forceinline__ int W() const { return lds32v(&s->W); }
    __device__ __forceinline__ int H() const { return lds32v(&s->H); }
    __device__ __forceinline__ int tile_w() const { return lds32v(&s->tile_w); }
};

// 128-bit shared-memory load that the compiler may not hoist (keeps the value out of registers).
__device__ __forceinline__ int4 lds128(const int4 *ptr) {
    int4 v;
    asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"((unsigned)__cvta_generic_to_shared(ptr)));
    return v;
}

// The warp's ancestor records of a node (ancestor list ar = (offset, count), na of them, parent
// first), filled by the lanes together; a warp barrier before and after.
__device__ __forceinline__ void fill_anc_records(const LevelParams &p, int2 ar, int na, AncRec *anc, int lane) {
    __syncwarp();
    for (int t = lane; t < na; t += 32) {
        const int a = p.anc[ar.x + t];
        const int4 an = p.node[a];
        const int y = p.sel_yaw[a];
        const int32_t *yr = p.yawtab + y * 12;
        AncRec r;
        r.px = an.x;
        r.py = an.y;
        r.pz = an.z;
        r.yaw = y;
        r.fx = (float)an.x * (1.0f / 65536.0f) - 0.5f;
        r.fy = (float)an.y * (1.0f / 65536.0f) - 0.5f;
        r.fz = (float)an.z * (1.0f / 65536.0f) - 0.5f;
#pragma unroll
        for (int qq = 0; qq < 9; ++qq) r.m[qq] = (float)yr[2 + qq] * (1.0f / 65536.0f);
        r.D = p.arena + (size_t)an.w * p.W * p.H;
        anc[t] = r;
    }
    __syncwarp();
}

// Queue key of an owned sample: voxel coordinates (16 bits each) recovered from the voxel-centre
// offsets (Q16) and the ray origin o (Q16, o.x / o.y / o.z).
__device__ __forceinline__ unsigned long long sample_key(int rx, int ry, int rz, const int4 o) {
    const uint32_t x = (uint32_t)(rx + o.x - 32768) >> 16, y = (uint32_t)(ry + o.y - 32768) >> 16,
                   z = (uint32_t)(rz + o.z - 32768) >> 16;
    return (unsigned long long)x | ((unsigned long long)y << 16) | ((unsigned long long)z << 32);
}

// cam: the warp's 4 x int4 shared slot, (px py pz mz0) (mz1 mz2 mu0 mu1) (mu2 mv0 mv1 mv2) (ck sk - -)
template <bool STATS, class HOT>
__device__ __forceinline__ void count_chunk(const LevelParams &p, const HOT &hp, int l0, int c, AncRec *anc,
                                            unsigned long long *q, int4 *cam, int lane) {
    const unsigned lt_mask = (1u << lane) - 1u;
    int li, k, tile;
    decode_item(p, c, li, k, tile);
    const int n = p.level_nodes[l0 + li];
    const int4 nd = p.node[n];
    const int2 ar = p.anc_range[n];
    int na = ar.y;
    if (p.mode == MIG_MODE_ABSOLUTE) na = 0;
    else if (p.mode == MIG_MODE_SINGLE_PARENT) na = min(na, 1);
    na = min(na, p.max_anc);  // the plan bounds depth by max_anc; this keeps the records in bounds
    fill_anc_records(p, ar, na, anc, lane);
    const int32_t *yk = p.yawtab + k * 12;
#if MIG_CAM_SMEM
    if (lane == 0) {
        cam[0] = make_int4(nd.x, nd.y, nd.z, yk[8]);
        cam[1] = make_int4(yk[9], yk[10], yk[2], yk[3]);
        cam[2] = make_int4(yk[4], yk[5], yk[6], yk[7]);
        cam[3] = make_int4(yk[0], yk[1], 0, 0);
    }
    __syncwarp();
#else
    (void)cam;
    const int ck = yk[0], sk = yk[1];
    const int mu0 = yk[2], mu1 = yk[3], mu2 = yk[4];
    const int mv0 = yk[5], mv1 = yk[6], mv2 = yk[7];
    const int mz0 = yk[8], mz1 = yk[9], mz2 = yk[10];
#endif
    const int tx0 = (tile % p.tiles_x) * p.tile_w, ty0 = (tile / p.tiles_x) * p.tile_h;
    const int tile_rays = p.tile_w * p.tile_h;  // (chunk-start values read directly)
    int next = 0, ti = 0, tj = 0, qn = 0, c_abs = 0, c_mrg = 0;
    bool have = false;
    RayIn r;
    uint32_t ne = 0, ade = 1;
    uint32_t st_steps = 0, st_unk = 0, st_anc = 0, st_reads = 0, st_rays = 0;
#if MIG_COUNT_BLOCK > 0
    // Block-synchronous loop. Between two warp-wide exchanges every lane runs kCountBlock DDA steps
    // of its own ray with no vote; an owned sample goes to the lane's private slots of the queue
    // (pend[i * 32 + lane]). At the exchange, the warp refills ended rays, appends the pending
    // samples to the shared queue in lane order (prefix sum of the per-lane counts) and tests every
    // full batch of 32 against the ancestors.
    unsigned long long *pend = q + kQueueMain;
    for (;;) {
        const unsigned need = __ballot_sync(0xffffffffu, !have);
        if (need == 0xffffffffu && next >= tile_rays) break;
        if (need && next < tile_rays) {
            const int idx = next + __popc(need & lt_mask);
            next += __popc(need);
            if (!have && idx < tile_rays) {
                ti = tx0 + idx % hp.tile_w();
                tj = ty0 + idx / hp.tile_w();
                if (ti < hp.W() && tj < hp.H()) {
                    const int4 b = hp.body()[tj * hp.W() + ti];
                    int dx, dy, dz;
#if MIG_CAM_SMEM
                    const int4 c3 = lds128(cam + 3), c0 = lds128(cam);
                    ray_dir(b, c3.x, c3.y, dx, dy, dz);
                    ray_init_dims(r, hp.nx(), hp.ny(), hp.nz(), p.grid, c0.x, c0.y, c0.z, dx, dy, dz, hp.Tq());
#else
                    ray_dir(b, ck, sk, dx, dy, dz);
                    ray_init_dims(r, hp.nx(), hp.ny(), hp.nz(), p.grid, nd.x, nd.y, nd.z, dx, dy, dz, hp.Tq());
#endif
                    have = true;
                    if constexpr (STATS) ++st_rays;
                }
            }
        }
        int cnt = 0;
#pragma unroll
        for (int sidx = 0; sidx < kCountBlock; ++sidx) {
            if (have) {
                const uint8_t code = load_code(hp.g(), ray_addr(r, p.grid), p.grid, p.bounds_err);
                if constexpr (STATS) ++st_steps;
                if (code == kOcc) {
                    have = false;
                } else {
                    if (code == kUnknown) {
                        if constexpr (STATS) ++st_unk;
                        // owner test: centre of this voxel projects into pixel (ti, tj)
                        const int rx = voxel_offset(r.nx, r.sx);
                        const int ry = voxel_offset(r.ny, r.sy);
                        const int rz = voxel_offset(r.nz, r.sz);
#if MIG_CAM_SMEM
                        const int4 c0 = lds128(cam), c1 = lds128(cam + 1);
                        const int64_t Z = (int64_t)c0.w * rx + (int64_t)c1.x * ry + (int64_t)c1.y * rz;
                        const int64_t U = (int64_t)c1.z * rx + (int64_t)c1.w * ry + (int64_t)lds128(cam + 2).x * rz;
#else
                        const int64_t Z = (int64_t)mz0 * rx + (int64_t)mz1 * ry + (int64_t)mz2 * rz;
                        const int64_t U = (int64_t)mu0 * rx + (int64_t)mu1 * ry + (int64_t)mu2 * rz;
#endif
                        const int64_t iZ = (int64_t)ti * Z;
                        if (Z > 0 && U >= iZ && U < iZ + Z) {
#if MIG_CAM_SMEM
                            const int4 c2 = lds128(cam + 2);
                            const int64_t V = (int64_t)c2.y * rx + (int64_t)c2.z * ry + (int64_t)c2.w * rz;
#else
                            const int64_t V = (int64_t)mv0 * rx + (int64_t)mv1 * ry + (int64_t)mv2 * rz;
#endif
                            const int64_t jZ = (int64_t)tj * Z;
                            if (V >= jZ && V < jZ + Z) {
#if MIG_CAM_SMEM
                                const int4 o = lds128(cam);
#else
                                const int4 o = nd;
#endif
                                pend[cnt * 32 + lane] = sample_key(rx, ry, rz, o);
                                ++cnt;
                            }
                        }
                    }
                    have = ray_step<false>(r, ne, ade);
                }
            }
        }
        const int tot = __reduce_add_sync(0xffffffffu, (unsigned)cnt);
        if (tot) {
            c_abs += cnt;
            int off = cnt;  // inclusive prefix sum over the lanes, then exclusive
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, off, d);
                if (lane >= d) off += v;
            }
            off = qn + off - cnt;
            for (int i = 0; i < cnt; ++i) q[off + i] = pend[i * 32 + lane];
            qn += tot;
            if (qn >= 32) {  // full batches: every lane tests one sample (Sec. IV-B)
                __syncwarp();
                int base = 0;
                do {
                    const unsigned long long sm = q[base + lane];
                    const int sx = (int)(sm & 0xFFFF), sy = (int)((sm >> 16) & 0xFFFF), sz = (int)(sm >> 32);
                    c_mrg += !observed<STATS>(hp, anc, na, sx, sy, sz, st_anc, st_reads);
                    base += 32;
                } while (qn - base >= 32);
                const int left = qn - base;
                const unsigned long long keep = lane < left ? q[base + lane] : 0ull;
                __syncwarp();
                if (lane < left) q[lane] = keep;
                qn = left;
            }
        }
    }
#else
    for (;;) {
        // lanes without a ray take the chunk's next rays in order (neighbouring pixels)
        const unsigned need = __ballot_sync(0xffffffffu, !have);
        if (need && next < tile_rays) {
            const int idx = next + __popc(need & lt_mask);
            next += __popc(need);
            if (!have && idx < tile_rays) {
                ti = tx0 + idx % hp.tile_w();
                tj = ty0 + idx / hp.tile_w();
                if (ti < hp.W() && tj < hp.H()) {
                    const int4 b = hp.body()[tj * hp.W() + ti];
                    int dx, dy, dz;
#if MIG_CAM_SMEM
                    const int4 c3 = lds128(cam + 3), c0 = lds128(cam);
                    ray_dir(b, c3.x, c3.y, dx, dy, dz);
                    ray_init_dims(r, hp.nx(), hp.ny(), hp.nz(), p.grid, c0.x, c0.y, c0.z, dx, dy, dz, hp.Tq());
#else
                    ray_dir(b, ck, sk, dx, dy, dz);
                    ray_init_dims(r, hp.nx(), hp.ny(), hp.nz(), p.grid, nd.x, nd.y, nd.z, dx, dy, dz, hp.Tq());
#endif
                    have = true;
                    if constexpr (STATS) ++st_rays;
                }
            }
        }
        if (!__any_sync(0xffffffffu, have)) {
            if (next >= tile_rays) break;
            continue;
        }
        bool owned = false;
        unsigned long long samp = 0;
        if (have) {
            const uint8_t code = load_code(hp.g(), ray_addr(r, p.grid), p.grid, p.bounds_err);
            if constexpr (STATS) ++st_steps;
            if (code == kOcc) {
                have = false;
            } else {
                if (code == kUnknown) {
                    if constexpr (STATS) ++st_unk;
                    // owner test: centre of this voxel projects into pixel (ti, tj)
                    const int rx = voxel_offset(r.nx, r.sx);
                    const int ry = voxel_offset(r.ny, r.sy);
                    const int rz = voxel_offset(r.nz, r.sz);
#if MIG_CAM_SMEM
                    const int4 c0 = lds128(cam), c1 = lds128(cam + 1);
                    const int64_t Z = (int64_t)c0.w * rx + (int64_t)c1.x * ry + (int64_t)c1.y * rz;
                    const int64_t U = (int64_t)c1.z * rx + (int64_t)c1.w * ry + (int64_t)lds128(cam + 2).x * rz;
#else
                    const int64_t Z = (int64_t)mz0 * rx + (int64_t)mz1 * ry + (int64_t)mz2 * rz;
                    const int64_t U = (int64_t)mu0 * rx + (int64_t)mu1 * ry + (int64_t)mu2 * rz;
#endif
                    const int64_t iZ = (int64_t)ti * Z;
                    if (Z > 0 && U >= iZ && U < iZ + Z) {
#if MIG_CAM_SMEM
                        const int4 c2 = lds128(cam + 2);
                        const int64_t V = (int64_t)c2.y * rx + (int64_t)c2.z * ry + (int64_t)c2.w * rz;
#else
                        const int64_t V = (int64_t)mv0 * rx + (int64_t)mv1 * ry + (int64_t)mv2 * rz;
#endif
                        const int64_t jZ = (int64_t)tj * Z;
                        owned = V >= jZ && V < jZ + Z;
#if MIG_CAM_SMEM
                        samp = sample_key(rx, ry, rz, lds128(cam));
#else
                        samp = sample_key(rx, ry, rz, nd);
#endif
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
                const unsigned long long s = q[lane];
                const int sx = (int)(s & 0xFFFF), sy = (int)((s >> 16) & 0xFFFF), sz = (int)(s >> 32);
                c_mrg += !observed<STATS>(hp, anc, na, sx, sy, sz, st_anc, st_reads);
                __syncwarp();
                if (lane < qn - 32) q[lane] = q[lane + 32];
                __syncwarp();
                qn -= 32;
            }
        }
    }
#endif
    // the last, partial batch
    __syncwarp();
    if (lane < qn) {
        const unsigned long long s = q[lane];
        const int sx = (int)(s & 0xFFFF), sy = (int)((s >> 16) & 0xFFFF), sz = (int)(s >> 32);
        c_mrg += !observed<STATS>(hp, anc, na, sx, sy, sz, st_anc, st_reads);
    }
    c_abs = __reduce_add_sync(0xffffffffu, c_abs);
    c_mrg = __reduce_add_sync(0xffffffffu, c_mrg);
    if (lane == 0 && (c_abs | c_mrg)) {
        atomicAdd(p.cnt + ((size_t)n * p.K + k) * 2, c_abs);
        atomicAdd(p.cnt + ((size_t)n * p.K + k) * 2 + 1, c_mrg);
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
            atomicAdd(p.stats + 3, (unsigned long long)(uint32_t)c_abs);
            atomicAdd(p.stats + 4, (unsigned long long)st_anc);
            atomicAdd(p.stats + 5, (unsigned long long)st_reads);
        }
    }
}

// Yaw selection of node n (Sec. III-B): lowest k with the largest marginal count (absolute
// count in the absolute mode, where both counts are equal); g_abs = max over yaws of the
// absolute count.
__device__ __forceinline__ void select_node(const LevelParams &p, int n) {
    const int32_t *c = p.cnt + (size_t)n * p.K * 2;
    int best = 0, bm = c[1], amax = c[0];
    for (int k = 1; k < p.K; ++k) {
        const int m = c[2 * k + 1];
        if (m > bm) {
            bm = m;
            best = k;
        }
        amax = max(amax, c[2 * k]);
    }
    p.sel_yaw[n] = best;
    p.out_abs[n] = amax;
    p.out_marg[n] = bm;
    p.out_yaw[n] = best;
}

// Depth of pixel (ti, tj) of node n's selected yaw (Sec. IV-A): camera z of the entry point of
// the first occupied voxel, else of the range endpoint; returns the DDA steps taken.
__device__ __forceinline__ uint32_t render_pixel(const LevelParams &p, int n, const int4 nd, int ti, int tj) {
    const int32_t *yk = p.yawtab + p.sel_yaw[n] * 12;
    const int4 b = p.body[tj * p.W + ti];
    int dx, dy, dz;
    ray_dir(b, yk[0], yk[1], dx, dy, dz);
    RayIn r;
    ray_init(r, p.grid, nd.x, nd.y, nd.z, dx, dy, dz, p.Tq);
    uint32_t ne = 0, ade = 1, steps = 0;
    bool hit = false;
    for (;;) {
        const uint8_t code = load_code(p.grid.g, ray_addr(r, p.grid), p.grid, p.bounds_err);
        ++steps;
        if (code == kOcc) {
            hit = true;
            break;
        }
        if (!ray_step<true>(r, ne, ade)) break;
    }
    arena_store(p.arena, p.arena_slots, nd.w, (size_t)tj * p.W + ti, (size_t)p.W * p.H, hit_depth(hit, ne, ade, b.w, p.Tq),
                p.bounds_err);
    return steps;
}

// Render work item for one warp: the depth buffer of an 8 x 8 pixel tile of node n (Sec. IV-A).
// Lanes take the tile's next pixel as soon as their ray ends (ray lengths to the first hit vary).
__device__ __forceinline__ void render_chunk(const LevelParams &p, int n, int tile, int lane) {
    constexpr int RT = 8;
    const int4 nd = p.node[n];
    const int rtx = (p.W + RT - 1) / RT;
    const int tx0 = (tile % rtx) * RT, ty0 = (tile / rtx) * RT;
    const int32_t *yk = p.yawtab + p.sel_yaw[n] * 12;
    const int ck = yk[0], sk = yk[1];
    const unsigned lt_mask = (1u << lane) - 1u;
    int next = 0, ti = 0, tj = 0, dzc = 0;
    bool have = false;
    RayIn r;
    uint32_t ne = 0, ade = 1;
    for (;;) {
        const unsigned need = __ballot_sync(0xffffffffu, !have);
        if (need && next < RT * RT) {
            const int idx = next + __popc(need & lt_mask);
            next += __popc(need);
            if (!have && idx < RT * RT) {
                ti = tx0 + (idx & (RT - 1));
                tj = ty0 + idx / RT;
                if (ti < p.W && tj < p.H) {
                    const int4 b = p.body[tj * p.W + ti];
                    int dx, dy, dz;
                    ray_dir(b, ck, sk, dx, dy, dz);
                    ray_init(r, p.grid, nd.x, nd.y, nd.z, dx, dy, dz, p.Tq);
                    dzc = b.w;
                    ne = 0;
                    ade = 1;
                    have = true;
                }
            }
        }
        if (!__any_sync(0xffffffffu, have)) {
            if (next >= RT * RT) break;
            continue;
        }
        if (have) {
            const uint8_t code = load_code(p.grid.g, ray_addr(r, p.grid), p.grid, p.bounds_err);
            const bool hit = code == kOcc;
            if (hit || !ray_step<true>(r, ne, ade)) {
                arena_store(p.arena, p.arena_slots, nd.w, (size_t)tj * p.W + ti, (size_t)p.W * p.H,
                            hit_depth(hit, ne, ade, dzc, p.Tq), p.bounds_err);
                have = false;
            }
        }
    }
}

__device__ __forceinline__ int render_chunk_tiles(int W, int H) { return ((W + 7) / 8) * ((H + 7) / 8); }

}  // namespace dev
}  // namespace mig
