// Counting by owned voxels: device steps shared by the owned-voxel count kernels (voxcount.cu).
//
// The owner rule gives every unknown voxel at most one candidate ray: the ray of the pixel that
// contains the projection of its centre (Eq. 5). So instead of walking every ray through every
// voxel and rejecting the voxels that other pixels own, the count is taken in two passes per
// (node, yaw):
//   1. every pixel ray runs the integer DDA (Sec. IV-B) only to find where it stops, and keeps the
//      number of voxel-to-voxel steps it takes (bricks without an occupied voxel are crossed in one
//      exact jump);
//   2. the voxels in the camera's field of view and range are enumerated; each unknown one goes to
//      its owner pixel, and is counted iff that pixel's DDA visits it within its step budget.
// The DDA visits voxels in the order of its face-crossing events sorted by (t, axis) (ties x, y,
// z); the voxel k crossings along an axis from the start is visited iff its last entering event
// precedes its first leaving event in that order, and it is then the (sum of the per-axis
// crossings)-th voxel of the ray. Both tests are exact integer comparisons of t = n / |d|
// (cross-multiplied), so the counts equal those of the ray-by-ray walk bit for bit.
#pragma once

#include "dev_path.cuh"

namespace mig {
namespace dev {

// The integer steps below are plain functions of their arguments, callable from host code too.
#define MIG_HD __host__ __device__ __forceinline__

MIG_HD uint8_t ld_u8(const uint8_t *p) {
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

// Brick occupancy summary of a map: one byte per 8x8x8 brick (x-fastest), 1 iff the brick holds
// an occupied voxel. It sits after the voxel codes in the map's allocation (at a 256-byte aligned
// offset), so that every copy of a grid carries its summary.
constexpr int kOccBrickShift = 3;
MIG_HD size_t bocc_offset(int nx, int ny, int nz) {
    return ((size_t)nx * ny * nz + 255) & ~(size_t)255;
}

// Event order: (t1, axis1) < (t2, axis2) with t = n / ad, compared exactly by cross products.
MIG_HD bool ev_lt(uint32_t n1, uint32_t a1, int x1, uint32_t n2, uint32_t a2, int x2) {
    const uint64_t l = (uint64_t)n1 * a2, r = (uint64_t)n2 * a1;
    return l < r || (l == r && x1 < x2);
}

// Number of crossings j in [0, jmax] of an axis (face distances nb + j 2^16, speed adb, index b)
// that come before the event (NE / AE, e). The caller guarantees that crossing jmax does not, so
// the answer is at most jmax. tE = NE / AE in float gives a first guess; exact comparisons fix it.
MIG_HD int crossings_before(uint32_t nb, uint32_t adb, int b, int jmax, uint32_t NE, uint32_t AE,
                                                int e, float tE) {
    if (adb == 0 || jmax <= 0) return 0;
    int j = (int)ceilf((tE * (float)adb - (float)nb) * (1.0f / 65536.0f));
    j = max(0, min(j, jmax));
    while (j > 0 && !ev_lt(nb + ((uint32_t)(j - 1) << 16), adb, b, NE, AE, e)) --j;
    while (j < jmax && ev_lt(nb + ((uint32_t)j << 16), adb, b, NE, AE, e)) ++j;
    return j;
}

// Per-axis start of a ray: voxel v, step sign s, face distance n (Q16), speed ad (Q30), and the
// number of crossings `allowed` along this axis that stay inside the grid and start before the
// range (the same face limits as axis_init). An axis with d = 0 never crosses.
MIG_HD void cast_axis(int P, int d, int N, int64_t Tq, int &v, uint32_t &n, uint32_t &ad, int &s,
                                          int &allowed) {
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
            allowed = 0;
            return;
        }
    }
    const uint64_t lim = ((uint64_t)Tq * ad + ((1ull << 30) - 1)) >> 30;  // n >= lim  <=>  t >= T
    const int64_t range_rem = (n >= lim) ? 0 : (int64_t)((lim - n + (kQ16 - 1)) >> 16);
    allowed = (int)min((int64_t)grid_rem, range_rem);
}

// The first of three axis events (n_a / ad_a, a) in event order; axes with ad = 0 never win
// (t = n / 0 is infinite in the cross products), unless all three are 0, which a unit ray is not.
MIG_HD int ev_argmin3(uint32_t n0, uint32_t a0, uint32_t n1, uint32_t a1, uint32_t n2, uint32_t a2) {
    const bool xly = (uint64_t)n0 * a1 <= (uint64_t)n1 * a0;
    const uint32_t nw = xly ? n0 : n1, aw = xly ? a0 : a1;
    const bool bz = !((uint64_t)nw * a2 <= (uint64_t)n2 * aw);
    return bz ? 2 : (xly ? 0 : 1);
}

// DDA steps a ray takes before it stops: the index (0 = the start voxel) of the first occupied
// voxel it visits, else of the last voxel it visits before leaving the grid or reaching the range.
// `fine` and `skips` count voxel steps and brick jumps (statistics).
template <bool STATS>
MIG_HD uint32_t cast_steps(const uint8_t *g, const uint8_t *bocc, int gnx, int gny, int gnz,
                                               int Px, int Py, int Pz, int dx, int dy, int dz, int64_t Tq,
                                               uint32_t &fine, uint32_t &skips) {
    int vx, vy, vz, sx, sy, sz, cx, cy, cz;
    uint32_t nx, ny, nz, ax, ay, az;
    cast_axis(Px, dx, gnx, Tq, vx, nx, ax, sx, cx);
    cast_axis(Py, dy, gny, Tq, vy, ny, ay, sy, cy);
    cast_axis(Pz, dz, gnz, Tq, vz, nz, az, sz, cz);
    // the first disallowed crossing of each axis is at n + allowed 2^16; the earliest of them ends
    // the ray, after m_end allowed crossings
    uint32_t m_end;
    {
        const uint32_t Lx = nx + ((uint32_t)cx << 16), Ly = ny + ((uint32_t)cy << 16), Lz = nz + ((uint32_t)cz << 16);
        const int e = ev_argmin3(Lx, ax, Ly, ay, Lz, az);
        const uint32_t NE = e == 0 ? Lx : (e == 1 ? Ly : Lz), AE = e == 0 ? ax : (e == 1 ? ay : az);
        const float tE = (float)NE / (float)AE;
        m_end = (uint32_t)((e == 0 ? cx : crossings_before(nx, ax, 0, cx, NE, AE, e, tE)) +
                           (e == 1 ? cy : crossings_before(ny, ay, 1, cy, NE, AE, e, tE)) +
                           (e == 2 ? cz : crossings_before(nz, az, 2, cz, NE, AE, e, tE)));
    }
    const int nbx = (gnx + 7) >> 3, nby = (gny + 7) >> 3;
    const int dax = sx, day = sy * gnx, daz = sz * gnx * gny;
    uint32_t addr = ((uint32_t)vz * (uint32_t)gny + (uint32_t)vy) * (uint32_t)gnx + (uint32_t)vx;
    uint32_t m = 0;
    int cur = -1;
    bool occ = true;
    for (;;) {
        if (bocc) {
            const int bi = ((vz >> 3) * nby + (vy >> 3)) * nbx + (vx >> 3);
            if (bi != cur) {
                cur = bi;
                occ = ld_u8(bocc + bi) != 0;
            }
        }
        if (!occ) {
            // no occupied voxel in this brick: jump to the crossing that leaves it (exact)
            const int rx = ax == 0 ? 0 : (sx > 0 ? min(vx | 7, gnx - 1) - vx : vx & 7);
            const int ry = ay == 0 ? 0 : (sy > 0 ? min(vy | 7, gny - 1) - vy : vy & 7);
            const int rz = az == 0 ? 0 : (sz > 0 ? min(vz | 7, gnz - 1) - vz : vz & 7);
            const uint32_t Nx = nx + ((uint32_t)rx << 16), Ny = ny + ((uint32_t)ry << 16), Nz = nz + ((uint32_t)rz << 16);
            const int e = ev_argmin3(Nx, ax, Ny, ay, Nz, az);
            const uint32_t NX = e == 0 ? Nx : (e == 1 ? Ny : Nz), AX = e == 0 ? ax : (e == 1 ? ay : az);
            const float tX = (float)NX / (float)AX;
            const int kx = e == 0 ? rx + 1 : crossings_before(nx, ax, 0, rx, NX, AX, e, tX);
            const int ky = e == 1 ? ry + 1 : crossings_before(ny, ay, 1, ry, NX, AX, e, tX);
            const int kz = e == 2 ? rz + 1 : crossings_before(nz, az, 2, rz, NX, AX, e, tX);
            const uint32_t tot = (uint32_t)(kx + ky + kz);
            if constexpr (STATS) ++skips;
            if (m + tot >= m_end) return m_end;  // the ray ends inside this brick (or just after it)
            m += tot;
            nx += (uint32_t)kx << 16;
            ny += (uint32_t)ky << 16;
            nz += (uint32_t)kz << 16;
            vx += sx * kx;
            vy += sy * ky;
            vz += sz * kz;
            addr = ((uint32_t)vz * (uint32_t)gny + (uint32_t)vy) * (uint32_t)gnx + (uint32_t)vx;
            continue;
        }
        if constexpr (STATS) ++fine;
        if (ld_u8(g + addr) == kOcc) return m;
        if (m == m_end) return m;
        const int a = ev_argmin3(nx, ax, ny, ay, nz, az);
        nx += a == 0 ? kQ16 : 0u;
        ny += a == 1 ? kQ16 : 0u;
        nz += a == 2 ? kQ16 : 0u;
        vx += a == 0 ? sx : 0;
        vy += a == 1 ? sy : 0;
        vz += a == 2 ? sz : 0;
        addr += a == 0 ? dax : (a == 1 ? day : daz);
        ++m;
    }
}

// Does the DDA of the ray from P (Q16) along d (Q30) visit voxel (x, y, z), and after how many
// steps? The voxel lies c_a = s_a (v_a - v0_a) crossings from the start voxel along each axis; it
// is visited iff every c_a >= 0 (c_a = 0 where d_a = 0) and its last entering event precedes its
// first leaving event. Returns the step index (c_x + c_y + c_z), or -1 if never visited.
MIG_HD int visit_index(int Px, int Py, int Pz, int dx, int dy, int dz, int x, int y, int z) {
    uint32_t n[3], ad[3];
    int c[3];
    const int P[3] = {Px, Py, Pz}, d[3] = {dx, dy, dz}, v[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int v0 = P[a] >> 16;
        if (d[a] < 0) {
            ad[a] = (uint32_t)(-d[a]);
            n[a] = (uint32_t)(P[a] - (v0 << 16));
            c[a] = v0 - v[a];
        } else {
            ad[a] = (uint32_t)d[a];
            n[a] = (uint32_t)(((v0 + 1) << 16) - P[a]);
            c[a] = v[a] - v0;
        }
        if (c[a] < 0 || (ad[a] == 0 && c[a] != 0)) return -1;
    }
    // last entering event: crossing c_a - 1 of each axis with c_a >= 1
    int ea = -1;
    uint32_t en = 0, eA = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (c[a] >= 1) {
            const uint32_t na = n[a] + ((uint32_t)(c[a] - 1) << 16);
            if (ea < 0 || ev_lt(en, eA, ea, na, ad[a], a)) {
                ea = a;
                en = na;
                eA = ad[a];
            }
        }
    }
    if (ea < 0) return 0;  // the start voxel
    // first leaving event: crossing c_a of each axis that moves
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (ad[a] != 0 && !ev_lt(en, eA, ea, n[a] + ((uint32_t)c[a] << 16), ad[a], a)) return -1;
    }
    return c[0] + c[1] + c[2];
}

// One half-space a rx + b ry + c rz > 0 of the voxel-centre offsets r (voxel units, float),
// shifted outwards by one voxel (its L1 coefficient norm), narrows a row's [lo, hi] of rx. The
// shift covers the float rounding of the row terms, so no voxel inside the half-space is dropped;
// the exact tests decide every voxel kept.
struct HalfSpace {
    float a, b, c, nrm;
};
MIG_HD HalfSpace half_space(int64_t a, int64_t b, int64_t c) {
    const float s = 1.0f / 65536.0f;
    HalfSpace h{(float)a * s, (float)b * s, (float)c * s, 0.f};
    h.nrm = fabsf(h.a) + fabsf(h.b) + fabsf(h.c);
    return h;
}
// The owner rule's frustum (Eq. 5: Z > 0, U >= 0, V >= 0, W Z - U > 0, H Z - V > 0) from a yaw's
// projection rows (Q16), in the order Z, U, W Z - U, V, H Z - V; W Z - U and H Z - V are formed in
// exact integers before the conversion.
MIG_HD void frustum_half_spaces(int mu0, int mu1, int mu2, int mv0, int mv1, int mv2, int mz0, int mz1, int mz2, int W,
                                int H, HalfSpace hs[5]) {
    hs[0] = half_space(mz0, mz1, mz2);
    hs[1] = half_space(mu0, mu1, mu2);
    hs[2] = half_space((int64_t)W * mz0 - mu0, (int64_t)W * mz1 - mu1, (int64_t)W * mz2 - mu2);
    hs[3] = half_space(mv0, mv1, mv2);
    hs[4] = half_space((int64_t)H * mz0 - mv0, (int64_t)H * mz1 - mv1, (int64_t)H * mz2 - mv2);
}
MIG_HD void clip_row(const HalfSpace &h, float ry, float rz, float &lo, float &hi) {
    const float c = fmaf(h.b, ry, fmaf(h.c, rz, h.nrm));
    if (h.a > 0.f) lo = fmaxf(lo, -c / h.a);
    else if (h.a < 0.f) hi = fminf(hi, -c / h.a);
    else if (c < 0.f) hi = -1e30f;  // the row misses the half-space
}
// Voxels [xa, xa + len) of the row (ry, rz) (centre offsets from the node) that may lie in the
// ball h2 = R^2 - rz^2 and the frustum; Pxf = P_x / 2^16 - 1/2 places the row's x offsets.
MIG_HD void row_span(const HalfSpace hs[5], float Pxf, float ry, float rz, float h2, int gnx, int &xa, int &len) {
    xa = 0;
    len = 0;
    const float hx2 = h2 - ry * ry;
    if (hx2 < 0.f) return;
    const float hx = sqrtf(hx2);
    float lo = -hx, hi = hx;
    for (int i = 0; i < 5; ++i) clip_row(hs[i], ry, rz, lo, hi);
    if (hi < lo) return;
    xa = max(0, (int)floorf(Pxf + lo) - 1);
    const int xb = min(gnx - 1, (int)ceilf(Pxf + hi) + 1);
    len = max(0, xb - xa + 1);
}

}  // namespace dev
}  // namespace mig
