// Interval-mode count pass: the paper's screen-space overlap test (Sec. IV-B, Eq. 5-7).
//
// For every candidate ray the 3D DDA (Sec. IV-B) visits voxels exactly as in the sample mode;
// each owned unknown voxel (its centre projects into the ray's pixel) counts as absolute gain and
// becomes a sample at the midpoint of the ray's traversal of it. A sample is excluded from the
// marginal gain when it lies in the union of the ancestors' overlap intervals of the ray. For
// each ancestor the ray is
//   1. taken to the ancestor's camera as projective image coordinates (U, V, Z), exact integers
//      from the Q16 projection rows, then IEEE single precision in voxel units;
//   2. clipped to the valid depth range [Z_NEAR, range];
//   3. projected (Eq. 5) and clipped to the buffer [0, W] x [0, H] (Liang-Barsky);
//   4. walked pixel by pixel (2D DDA); each visited pixel holds one portion of the segment, whose
//      depth sample at the portion's midpoint (inverse depth linear in the screen parameter,
//      Eq. 6) is compared with the stored depth, "smaller or equal" => observed, in inverse depth
//      (w D >= 1); boundary crossings use one reciprocal of the segment's screen extent.
// A sample belongs to the first portion, in walk order, that contains its perspective-correct
// screen parameter. Every floating-point step is one correctly rounded single-precision
// operation (__fadd_rn and friends: no contraction), in a fixed order, so the counts are
// reproducible bit for bit.
//
// The walk is not stepped pixel by pixel here: its portion boundaries are a fixed function of the
// boundary index (the same rounded operations as the walk), non-decreasing along it, so the
// portion that contains a sample is found directly by counting the column and row crossings at or
// before the sample's screen parameter (seg_lookup). The result is the walk's, bit for bit.
//
// Layout: one warp per work item (node, yaw, tile of rays), taken from the level's atomic work
// counter; a lane takes the tile's next ray as soon as its ray ends. Owned samples go to a
// per-warp queue as the crossings that bound their voxel and their pixel; each full batch of 32 is
// tested against the ancestors with one sample per lane, which is also where each sample's ray
// fraction is computed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "dev_path.cuh"
#include "interval.h"
#include "kernels.h"
#include "mig.h"

namespace mig {

namespace {

using namespace dev;

// minimum resident interval-kernel CTAs per SM requested from the register allocator
#ifndef MIG_IV_MINB
#define MIG_IV_MINB 4
#endif

constexpr int kIvWarps = 8;
constexpr int kIvThreads = kIvWarps * 32;
constexpr float kZNear = 1.0f / 1024.0f;  // near end of the valid depth range, voxel units

// an ancestor as the interval walk needs it: position (Q16), selected yaw, depth buffer
struct IvAnc {
    int px, py, pz, yaw;
    const uint32_t *D;
};

struct Seg {
    float lo, hi;          // depth-clipped range of the ray fraction
    float Za, Zb;          // camera z at lo, hi (voxel units)
    float ua, va, ub, vb;  // projected clipped endpoints (pixels)
    float wa, wb;          // inverse depths at the endpoints
    float s0, s1;          // Liang-Barsky range of the screen parameter
    float ru, rv;          // reciprocals of the segment's screen extent (0 when it is 0)
};

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

// steps 1-3 for the candidate ray from P to its range endpoint E (Q16) and the ancestor at Pa
// with projection rows m (Q16: mu, mv, mz); false if nothing of the ray is in view, or if the
// sample's ray fraction lam lies outside the depth-clipped range (seg_param would then reject it,
// so the screen-space part is skipped with the same outcome)
__device__ bool seg_setup(const int32_t *m, const int3 Pa, const int64_t P[3], const int64_t E[3], float zf, int W,
                          int H, float lam, Seg &g) {
    const int64_t r0x = P[0] - Pa.x, r0y = P[1] - Pa.y, r0z = P[2] - Pa.z;
    const int64_t r1x = E[0] - Pa.x, r1y = E[1] - Pa.y, r1z = E[2] - Pa.z;
    const float sc = 2.3283064365386963e-10f;  // 2^-32: Q32 -> voxel units
    const float Z0 = fmul(__ll2float_rn((int64_t)m[6] * r0x + (int64_t)m[7] * r0y + (int64_t)m[8] * r0z), sc);
    const float Z1 = fmul(__ll2float_rn((int64_t)m[6] * r1x + (int64_t)m[7] * r1y + (int64_t)m[8] * r1z), sc);
    const float zn = kZNear;
    const float dZ = fsub(Z1, Z0);
    float lo = 0.0f, hi = 1.0f;
    if (Z0 < zn) {
        if (!(dZ > 0.0f)) return false;
        lo = fdiv(fsub(zn, Z0), dZ);
    }
    if (Z1 < zn) {
        if (!(dZ < 0.0f)) return false;
        hi = fdiv(fsub(zn, Z0), dZ);
    }
    if (Z0 > zf) {
        if (!(dZ < 0.0f)) return false;
        const float l = fdiv(fsub(zf, Z0), dZ);
        if (l > lo) lo = l;
    }
    if (Z1 > zf) {
        if (!(dZ > 0.0f)) return false;
        const float h = fdiv(fsub(zf, Z0), dZ);
        if (h < hi) hi = h;
    }
    if (!(lo < hi)) return false;
    if (!(lam >= lo && lam <= hi)) return false;
    const float U0 = fmul(__ll2float_rn((int64_t)m[0] * r0x + (int64_t)m[1] * r0y + (int64_t)m[2] * r0z), sc);
    const float V0 = fmul(__ll2float_rn((int64_t)m[3] * r0x + (int64_t)m[4] * r0y + (int64_t)m[5] * r0z), sc);
    const float U1 = fmul(__ll2float_rn((int64_t)m[0] * r1x + (int64_t)m[1] * r1y + (int64_t)m[2] * r1z), sc);
    const float V1 = fmul(__ll2float_rn((int64_t)m[3] * r1x + (int64_t)m[4] * r1y + (int64_t)m[5] * r1z), sc);
    const float dU = fsub(U1, U0), dV = fsub(V1, V0);
    const float Ua = fadd(U0, fmul(lo, dU)), Va = fadd(V0, fmul(lo, dV)), Za = fadd(Z0, fmul(lo, dZ));
    const float Ub = fadd(U0, fmul(hi, dU)), Vb = fadd(V0, fmul(hi, dV)), Zb = fadd(Z0, fmul(hi, dZ));
    if (!(Za > 0.0f && Zb > 0.0f)) return false;
    g.lo = lo;
    g.hi = hi;
    g.Za = Za;
    g.Zb = Zb;
    // Eq. 5 with the inverse depths of Eq. 6: u = U w, v = V w
    g.wa = fdiv(1.0f, Za);
    g.wb = fdiv(1.0f, Zb);
    g.ua = fmul(Ua, g.wa);
    g.va = fmul(Va, g.wa);
    g.ub = fmul(Ub, g.wb);
    g.vb = fmul(Vb, g.wb);
    // Liang-Barsky against 0 <= u <= W, 0 <= v <= H (edges in the order -u, +u, -v, +v); each
    // edge's crossing is q times the reciprocal of p
    const float du = fsub(g.ub, g.ua), dv = fsub(g.vb, g.va);
    g.ru = du != 0.0f ? fdiv(1.0f, du) : 0.0f;
    g.rv = dv != 0.0f ? fdiv(1.0f, dv) : 0.0f;
    const float pe[4] = {-du, du, -dv, dv};
    const float rp[4] = {-g.ru, g.ru, -g.rv, g.rv};
    const float qe[4] = {g.ua, fsub(__int2float_rn(W), g.ua), g.va, fsub(__int2float_rn(H), g.va)};
    float s0 = 0.0f, s1 = 1.0f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (pe[e] == 0.0f) {
            if (qe[e] < 0.0f) return false;
            continue;
        }
        const float r = fmul(qe[e], rp[e]);
        if (pe[e] < 0.0f) {
            if (r > s1) return false;
            if (r > s0) s0 = r;
        } else {
            if (r < s0) return false;
            if (r < s1) s1 = r;
        }
    }
    if (!(s0 < s1)) return false;
    g.s0 = s0;
    g.s1 = s1;
    return true;
}

// screen parameter of the ray fraction lam (perspective-correct); false outside the clip
__device__ __forceinline__ bool seg_param(const Seg &g, float lam, float &s) {
    if (!(lam >= g.lo && lam <= g.hi)) return false;
    const float mu = fdiv(fsub(lam, g.lo), fsub(g.hi, g.lo));
    const float num = fmul(mu, g.Zb);
    const float den = fadd(fmul(fsub(1.0f, mu), g.Za), num);
    s = fdiv(num, den);
    return s >= g.s0 && s < g.s1;
}

// a voxel's sample: midpoint of the ray's traversal of it (entry ne / ade, exit nx / adx capped at
// the range) as a fraction of the range T (= Tq / 2^30 in crossing units)
__device__ __forceinline__ float sample_lambda(uint32_t ne, uint32_t ade, uint32_t nx, uint32_t adx, float T) {
    const float lin = fdiv(fdiv(__uint2float_rn(ne), __uint2float_rn(ade)), T);
    float lout = fdiv(fdiv(__uint2float_rn(nx), __uint2float_rn(adx)), T);
    if (lout > 1.0f) lout = 1.0f;
    return fmul(fadd(lin, lout), 0.5f);
}

// Column (or row) crossings of the walk: boundary b_k = b0 + sgn k is crossed at screen parameter
// x(k) = (b_k - a0) * r, the walk's own formula, non-decreasing in k. Counts the crossings at or
// before s among k < kmax (crossing kmax leaves the buffer); lo / hi = the last crossing at or
// before s and the next one. The count starts from a float estimate and is corrected exactly.
__device__ __forceinline__ int count_crossings(float a0, float r, float d, int b0, int sgn, int kmax, float s,
                                               float &lo, float &hi) {
    const float est = (float)sgn * (s * d + a0 - (float)b0) + 1.0f;  // estimate only; corrected below
    int k = !(est > 0.0f) ? 0 : (est >= (float)kmax ? kmax : (int)est);
    auto x = [&](int kk) { return fmul(fsub(__int2float_rn(b0 + sgn * kk), a0), r); };
    while (k > 0 && x(k - 1) > s) --k;
    while (k < kmax && x(k) <= s) ++k;
    lo = k > 0 ? x(k - 1) : __int_as_float(0xff800000);
    hi = k < kmax ? x(k) : __int_as_float(0x7f800000);
    return k;
}

// Step 4 for one screen parameter s in [s0, s1): the walk's portion containing s, found directly.
// The walk crosses column and row boundaries in the order of their crossing parameters, so at s
// it is in column i0 + si * (column crossings <= s) and row j0 + sj * (row crossings <= s), in the
// portion from the latest crossing at or before s (s0 if none) to the next one (capped at s1).
// True if that portion is observed; false if not, or if the walk leaves the buffer before s.
__device__ bool seg_lookup(const Seg &g, int W, int H, const uint32_t *D, float s) {
    const float du = fsub(g.ub, g.ua), dv = fsub(g.vb, g.va);
    const float ru = g.ru, rv = g.rv;
    const float fi = floorf(fadd(g.ua, fmul(g.s0, du))), fj = floorf(fadd(g.va, fmul(g.s0, dv)));
    const int i0 = fi < 0.0f ? 0 : (fi > __int2float_rn(W - 1) ? W - 1 : __float2int_rz(fi));
    const int j0 = fj < 0.0f ? 0 : (fj > __int2float_rn(H - 1) ? H - 1 : __float2int_rz(fj));
    const int si = du > 0.0f ? 1 : (du < 0.0f ? -1 : 0), sj = dv > 0.0f ? 1 : (dv < 0.0f ? -1 : 0);
    float xlo = __int_as_float(0xff800000), xhi = __int_as_float(0x7f800000), ylo = xlo, yhi = xhi;
    int nx = 0, ny = 0;
    if (si) {
        const int kmax = si > 0 ? W - i0 : i0 + 1;
        nx = count_crossings(g.ua, ru, du, si > 0 ? i0 + 1 : i0, si, kmax, s, xlo, xhi);
        if (nx == kmax) return false;
    }
    if (sj) {
        const int kmax = sj > 0 ? H - j0 : j0 + 1;
        ny = count_crossings(g.va, rv, dv, sj > 0 ? j0 + 1 : j0, sj, kmax, s, ylo, yhi);
        if (ny == kmax) return false;
    }
    const int i = i0 + si * nx, j = j0 + sj * ny;
    const float s_in = (nx == 0 && ny == 0) ? g.s0 : (xlo > ylo ? xlo : ylo);
    float s_out = xhi < yhi ? xhi : yhi;
    if (g.s1 < s_out) s_out = g.s1;
    const float sm = fmul(fadd(s_in, s_out), 0.5f);
    const float wm = fadd(g.wa, fmul(sm, fsub(g.wb, g.wa)));
    const float Dv = fmul(__uint2float_rn(__ldg(D + (size_t)j * W + i)), 1.52587890625e-05f);
    return fmul(wm, Dv) >= 1.0f;  // z <= D in inverse depth
}

// A queued sample: the face distances of the crossings that enter and leave its voxel (Q16), and
// which of the ray's direction components |d_x|, |d_y|, |d_z| each is divided by (code 3: the
// ray's start, entry at t = 0 written as 0 / 1), with the pixel. The ray fraction is computed from
// it when the sample is tested, one sample per lane, not in the divergent DDA loop.
__device__ __forceinline__ uint32_t speed_code(uint32_t ad, const RayIn &r) {
    return ad == r.adx ? 0u : (ad == r.ady ? 1u : (ad == r.adz ? 2u : 3u));
}
__device__ __forceinline__ uint32_t speed_of(uint32_t code, uint32_t adx, uint32_t ady, uint32_t adz) {
    return code == 0u ? adx : (code == 1u ? ady : (code == 2u ? adz : 1u));
}

// Is the queued sample e (ray through pixel e.z >> 4, yaw ck / sk, origin P) inside an ancestor's
// observed portions? Ancestors parent first; the ray's set-up is rebuilt per sample.
template <bool STATS>
__device__ bool iv_observed(const LevelParams &p, const IvAnc *anc, int na, const int64_t P[3], int ck, int sk,
                            float zf, float T, const uint4 e, uint32_t &st_seg) {
    const int pix = (int)(e.z >> 4);
    const int4 b = p.body[pix];
    int dx, dy, dz;
    ray_dir(b, ck, sk, dx, dy, dz);
    const uint32_t adx = (uint32_t)(dx < 0 ? -dx : dx), ady = (uint32_t)(dy < 0 ? -dy : dy),
                   adz = (uint32_t)(dz < 0 ? -dz : dz);
    const float lam = sample_lambda(e.x, speed_of(e.z & 3u, adx, ady, adz), e.y, speed_of((e.z >> 2) & 3u, adx, ady, adz), T);
    const int64_t E[3] = {P[0] + (((int64_t)p.Tq * dx) >> 30), P[1] + (((int64_t)p.Tq * dy) >> 30),
                          P[2] + (((int64_t)p.Tq * dz) >> 30)};
    for (int a = 0; a < na; ++a) {
        const IvAnc &A = anc[a];
        Seg g;
        if constexpr (STATS) ++st_seg;
        if (!seg_setup(p.yawtab + A.yaw * 12 + 2, make_int3(A.px, A.py, A.pz), P, E, zf, p.W, p.H, lam, g)) continue;
        float s;
        if (seg_param(g, lam, s) && seg_lookup(g, p.W, p.H, A.D, s)) return true;
    }
    return false;
}

template <bool STATS>
__global__ void __launch_bounds__(kIvThreads, MIG_IV_MINB) interval_count_kernel(const LevelParams p) {
    extern __shared__ IvAnc s_iv_anc[];
    __shared__ uint4 s_q[kIvWarps][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    IvAnc *anc = s_iv_anc + warp * p.max_anc;
    uint4 *q = s_q[warp];
    const int l0 = p.level_off[p.lvl];
    const int L = p.level_off[p.lvl + 1] - l0;
    const int items = L * p.K * p.tiles;
    const float zf = fmul(__ll2float_rn(p.Tq), 1.52587890625e-05f);   // range, voxel units
    const float T = fmul(__ll2float_rn(p.Tq), 9.313225746154785e-10f);  // range, crossing units
    uint32_t st_rays = 0, st_steps = 0, st_unk = 0, st_seg = 0;
    for (;;) {
        int c = 0;
        if (lane == 0) c = atomicAdd(p.work + p.lvl, 1);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= items) break;
        int li, k, tile;
        decode_item(p, c, li, k, tile);
        const int n = p.level_nodes[l0 + li];
        const int4 nd = p.node[n];
        const int2 ar = p.anc_range[n];
        const int na = min(ar.y, p.max_anc);
        __syncwarp();
        for (int t = lane; t < na; t += 32) {
            const int a = p.anc[ar.x + t];
            const int4 an = p.node[a];
            IvAnc rec;
            rec.px = an.x;
            rec.py = an.y;
            rec.pz = an.z;
            rec.yaw = p.sel_yaw[a];
            rec.D = p.arena + (size_t)an.w * p.W * p.H;
            anc[t] = rec;
        }
        __syncwarp();
        const int32_t *yk = p.yawtab + k * 12;
        const int ck = yk[0], sk = yk[1];
        const int64_t P[3] = {nd.x, nd.y, nd.z};
        const int tx0 = (tile % p.tiles_x) * p.tile_w, ty0 = (tile / p.tiles_x) * p.tile_h;
        const int tile_rays = p.tile_w * p.tile_h;
        int next = 0, ti = 0, tj = 0, qn = 0, c_abs = 0, c_mrg = 0;
        bool have = false;
        RayIn r;
        uint32_t ne = 0, ade = 1;
        for (;;) {
            // lanes without a ray take the tile's next rays in order
            const unsigned need = __ballot_sync(0xffffffffu, !have);
            if (need && next < tile_rays) {
                const int idx = next + __popc(need & lt_mask);
                next += __popc(need);
                if (!have && idx < tile_rays) {
                    ti = tx0 + idx % p.tile_w;
                    tj = ty0 + idx / p.tile_w;
                    if (ti < p.W && tj < p.H) {
                        const int4 b = p.body[tj * p.W + ti];
                        int dx, dy, dz;
                        ray_dir(b, ck, sk, dx, dy, dz);
                        ray_init(r, p.grid, nd.x, nd.y, nd.z, dx, dy, dz, p.Tq);
                        ne = 0;
                        ade = 1;
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
            uint4 key = make_uint4(0u, 0u, 0u, 0u);
            if (have) {
                const uint8_t code = load_code(p.grid.g, ray_addr(r, p.grid), p.grid, p.bounds_err);
                if constexpr (STATS) ++st_steps;
                if (code == kOcc) {
                    have = false;
                } else {
                    if (code == kUnknown) {
                        if constexpr (STATS) ++st_unk;
                        // owner test: the voxel centre projects into pixel (ti, tj)
                        const int rx = voxel_offset(r.nx, r.sx), ry = voxel_offset(r.ny, r.sy),
                                  rz = voxel_offset(r.nz, r.sz);
                        const int64_t Z = (int64_t)yk[8] * rx + (int64_t)yk[9] * ry + (int64_t)yk[10] * rz;
                        const int64_t U = (int64_t)yk[2] * rx + (int64_t)yk[3] * ry + (int64_t)yk[4] * rz;
                        const int64_t iZ = (int64_t)ti * Z;
                        if (Z > 0 && U >= iZ && U < iZ + Z) {
                            const int64_t V = (int64_t)yk[5] * rx + (int64_t)yk[6] * ry + (int64_t)yk[7] * rz;
                            const int64_t jZ = (int64_t)tj * Z;
                            owned = V >= jZ && V < jZ + Z;
                        }
                    }
                    uint32_t nx = 0, adx = 1;
                    const bool more = ray_step<true>(r, nx, adx);  // nx / adx: this voxel's exit crossing
                    if (owned)
                        key = make_uint4(ne, nx, speed_code(ade, r) | (speed_code(adx, r) << 2) |
                                                     ((uint32_t)(tj * p.W + ti) << 4), 0u);
                    ne = nx;
                    ade = adx;
                    have = more;
                }
            }
            c_abs += owned;
            const unsigned bal = __ballot_sync(0xffffffffu, owned);
            if (bal) {
                if (owned) q[qn + __popc(bal & lt_mask)] = key;
                qn += __popc(bal);
                if (qn >= 32) {  // a full batch: every lane tests one sample against the ancestors
                    __syncwarp();
                    c_mrg += !iv_observed<STATS>(p, anc, na, P, ck, sk, zf, T, q[lane], st_seg);
                    __syncwarp();
                    if (lane < qn - 32) q[lane] = q[lane + 32];
                    __syncwarp();
                    qn -= 32;
                }
            }
        }
        __syncwarp();
        if (lane < qn) {
            c_mrg += !iv_observed<STATS>(p, anc, na, P, ck, sk, zf, T, q[lane], st_seg);
        }
        c_abs = __reduce_add_sync(0xffffffffu, c_abs);
        c_mrg = __reduce_add_sync(0xffffffffu, c_mrg);
        if (lane == 0 && (c_abs | c_mrg)) {
            atomicAdd(p.cnt + ((size_t)n * p.K + k) * 2, c_abs);
            atomicAdd(p.cnt + ((size_t)n * p.K + k) * 2 + 1, c_mrg);
        }
        if constexpr (STATS) {
            if (lane == 0) atomicAdd(p.stats + 3, (unsigned long long)(uint32_t)c_abs);
        }
        __syncwarp();
    }
    if constexpr (STATS) {
        st_rays = __reduce_add_sync(0xffffffffu, st_rays);
        st_steps = __reduce_add_sync(0xffffffffu, st_steps);
        st_unk = __reduce_add_sync(0xffffffffu, st_unk);
        st_seg = __reduce_add_sync(0xffffffffu, st_seg);
        if (lane == 0) {
            atomicAdd(p.stats + 0, (unsigned long long)st_rays);
            atomicAdd(p.stats + 1, (unsigned long long)st_steps);
            atomicAdd(p.stats + 2, (unsigned long long)st_unk);
            atomicAdd(p.stats + 4, (unsigned long long)st_seg);
        }
    }
}

}  // namespace

// dynamic shared memory: the warps' ancestor records, up to MIG_MAX_DEPTH each
constexpr size_t kIvMaxDyn = (size_t)kIvWarps * MIG_MAX_DEPTH * sizeof(IvAnc);

void launch_count_interval(const LevelParams &p, int grid, cudaStream_t s) {
    const size_t smem = (size_t)kIvWarps * (size_t)std::max(1, p.max_anc) * sizeof(IvAnc);
    if (p.stats) interval_count_kernel<true><<<grid, kIvThreads, smem, s>>>(p);
    else interval_count_kernel<false><<<grid, kIvThreads, smem, s>>>(p);
}

// Resident CTAs per SM (for the grid cap); also lifts the kernels' dynamic shared-memory limit to
// the deepest tree's ancestor records. Called once per context, before any launch.
int count_interval_ctas_per_sm() {
    cudaFuncSetAttribute(interval_count_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kIvMaxDyn);
    cudaFuncSetAttribute(interval_count_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kIvMaxDyn);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, interval_count_kernel<false>, kIvThreads,
                                                  (size_t)kIvWarps * 16 * sizeof(IvAnc));
    return std::max(1, n);
}

}  // namespace mig
