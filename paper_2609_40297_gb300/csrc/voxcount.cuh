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

// Occupancy summaries of a map: one byte per 8x8x8 brick (x-fastest), 1 iff the brick holds an
// occupied voxel, then one byte per 32x32x32 super-brick (4x4x4 bricks), 1 iff one of its bricks
// does. They sit after the voxel codes in the map's allocation (each at a 256-byte aligned offset),
// so that every copy of a grid carries its summaries.
constexpr int kOccBrickShift = 3;
constexpr int kOccSuperShift = 5;
MIG_HD size_t bocc_offset(int nx, int ny, int nz) {
    return ((size_t)nx * ny * nz + 255) & ~(size_t)255;
}
MIG_HD size_t sbocc_offset(int nx, int ny, int nz) {
    const size_t nb = (size_t)((nx + 7) >> 3) * (size_t)((ny + 7) >> 3) * (size_t)((nz + 7) >> 3);
    return bocc_offset(nx, ny, nz) + ((nb + 255) & ~(size_t)255);
}
MIG_HD size_t occ_summary_end(int nx, int ny, int nz) {
    return sbocc_offset(nx, ny, nz) +
           (size_t)((nx + 31) >> 5) * (size_t)((ny + 31) >> 5) * (size_t)((nz + 31) >> 5);
}

// Event order: (t1, axis1) < (t2, axis2) with t = n / ad, compared exactly by cross products.
MIG_HD bool ev_lt(uint32_t n1, uint32_t a1, int x1, uint32_t n2, uint32_t a2, int x2) {
    const uint64_t l = (uint64_t)n1 * a2, r = (uint64_t)n2 * a1;
    return l < r || (l == r && x1 < x2);
}

// a / b in float for a first guess (exact comparisons decide; the device uses the fast division).
MIG_HD float fast_div(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __fdividef((float)a, (float)b);
#else
    return (float)a / (float)b;
#endif
}

// a / b in float, approximately (the device's fast division; relative error about 1e-7).
MIG_HD float fast_divf(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
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

// "No occupied voxel within range": larger than every step index (at most 3 * 1027).
constexpr uint32_t kNoHit = 0xFFFF;

// Per-axis start of a ray from P (Q16) along d (Q30): voxel v0, step sign s, face distance n0 of the
// first crossing (Q16) and speed ad = |d| (Q30). An axis with d = 0 gets s = 1 and never crosses.
MIG_HD void ray_axis(int P, int d, int &v0, int &s, uint32_t &n0, uint32_t &ad) {
    v0 = P >> 16;
    if (d < 0) {
        s = -1;
        ad = (uint32_t)(-d);
        n0 = (uint32_t)(P - (v0 << 16));
    } else {
        s = 1;
        ad = (uint32_t)d;
        n0 = (uint32_t)(((v0 + 1) << 16) - P);
    }
}

// The first of three axis events (n_a / ad_a, a) in event order; axes with ad = 0 never win
// (t = n / 0 is infinite in the cross products), unless all three are 0, which a unit ray is not.
MIG_HD int ev_argmin3(uint32_t n0, uint32_t a0, uint32_t n1, uint32_t a1, uint32_t n2, uint32_t a2) {
    const bool xly = (uint64_t)n0 * a1 <= (uint64_t)n1 * a0;
    const uint32_t nw = xly ? n0 : n1, aw = xly ? a0 : a1;
    const bool bz = !((uint64_t)nw * a2 <= (uint64_t)n2 * aw);
    return bz ? 2 : (xly ? 0 : 1);
}

// Crossing index (from the start, 0-based) of the crossing that leaves the cell of 2^shift voxels
// (a brick or a super-brick) of voxel v along an axis with step s: the cell's last voxel in the
// direction of travel, or the grid's.
MIG_HD int cell_exit_crossing(int v, int v0, int s, int N, int shift) {
    const int m = (1 << shift) - 1;
    return s > 0 ? min(v | m, N - 1) - v0 : v0 - (v & ~m);
}
MIG_HD int brick_exit_crossing(int v, int v0, int s, int N) { return cell_exit_crossing(v, v0, s, N, kOccBrickShift); }

// Crossings an axis may take: those that stay inside the grid and start before the range T (the
// k-th crossing, k = 0, 1, ..., is at face distance n0 + k 2^16, i.e. at t = (n0 + k 2^16) / ad).
MIG_HD int allowed_crossings(int v0, int s, uint32_t n0, uint32_t ad, int N, int64_t Tq) {
    if (ad == 0) return 0;
    const int grid_rem = s > 0 ? N - 1 - v0 : v0;
    const uint64_t lim = ((uint64_t)Tq * ad + ((1ull << 30) - 1)) >> 30;  // n >= lim  <=>  t >= T
    const int64_t range_rem = (n0 >= lim) ? 0 : (int64_t)((lim - n0 + (kQ16 - 1)) >> 16);
    return (int)min((int64_t)grid_rem, range_rem);
}

// Step index of the first occupied voxel that the DDA (Sec. IV-B) visits, else kNoHit: the ray
// stops on that voxel and visits no voxel beyond it. A voxel is visited iff its entering crossing
// is allowed (inside the grid, before the range T); per axis the allowed crossings are a prefix
// of its crossings, so each step compares one crossing index (or face distance) with a limit
// fixed at the start. Cells without an occupied voxel are crossed by a cell-level walk whose
// crossings are exactly the cell faces of the voxel walk, in the same order: super-bricks
// (32 voxels a side) where `sbocc` marks them free, else bricks (8 a side) where `bocc` does. On
// entering a cell that holds an occupied voxel (or, from the brick walk, a free super-brick) the
// voxel state there is rebuilt exactly from the start (per axis, the crossings that precede the
// entering event) and the walk continues at the finer (or coarser) level. Null summaries disable
// their level. `fine` and `coarse` count voxel and cell steps (statistics).
template <bool STATS>
MIG_HD uint32_t cast_hit(const uint8_t *g, const uint8_t *bocc, const uint8_t *sbocc, int gnx, int gny, int gnz,
                         int Px, int Py, int Pz, int dx, int dy, int dz, int64_t Tq, uint32_t &fine,
                         uint32_t &coarse) {
    int v0x, v0y, v0z, sx, sy, sz;
    uint32_t n0x, n0y, n0z, ax, ay, az;
    ray_axis(Px, dx, v0x, sx, n0x, ax);
    ray_axis(Py, dy, v0y, sy, n0y, ay);
    ray_axis(Pz, dz, v0z, sz, n0z, az);
    const int kx = allowed_crossings(v0x, sx, n0x, ax, gnx, Tq), ky = allowed_crossings(v0y, sy, n0y, ay, gny, Tq),
              kz = allowed_crossings(v0z, sz, n0z, az, gnz, Tq);
    // face limits: a crossing at face distance n along an axis is allowed iff n < l
    const uint32_t lx = n0x + ((uint32_t)kx << 16), ly = n0y + ((uint32_t)ky << 16), lz = n0z + ((uint32_t)kz << 16);
    const int nbx = (gnx + 7) >> 3, nby = (gny + 7) >> 3;
    const int nsx = (gnx + 31) >> 5, nsy = (gny + 31) >> 5;
    const int dax = sx, day = sy * gnx, daz = sz * gnx * gny;
    // voxel state (valid in the voxel walk): current voxel, next crossing per axis, step index
    int vx = v0x, vy = v0y, vz = v0z;
    uint32_t nx = n0x, ny = n0y, nz = n0z, m = 0;
    // the voxel state after the event (NE / AE, e) that enters along e by crossing Ee, from the start;
    // ex, ey, ez: crossings of the other axes that come after that event
    auto enter = [&](uint32_t NE, uint32_t AE, int e, int Ee, int ex, int ey, int ez) {
        const float tE = fast_div(NE, AE);
        const int cx = e == 0 ? Ee + 1 : crossings_before(n0x, ax, 0, ex, NE, AE, e, tE);
        const int cy = e == 1 ? Ee + 1 : crossings_before(n0y, ay, 1, ey, NE, AE, e, tE);
        const int cz = e == 2 ? Ee + 1 : crossings_before(n0z, az, 2, ez, NE, AE, e, tE);
        vx = v0x + sx * cx;
        vy = v0y + sy * cy;
        vz = v0z + sz * cz;
        nx = n0x + ((uint32_t)cx << 16);
        ny = n0y + ((uint32_t)cy << 16);
        nz = n0z + ((uint32_t)cz << 16);
        m = (uint32_t)(cx + cy + cz);
    };
    for (;;) {
        if (sbocc && !ld_u8(sbocc + ((vz >> 5) * nsy + (vy >> 5)) * nsx + (vx >> 5))) {
            // super-brick walk: per axis the crossing index (from the start) that leaves the current
            // super-brick, until the ray enters one that holds an occupied voxel
            int ex = cell_exit_crossing(vx, v0x, sx, gnx, kOccSuperShift), ey = cell_exit_crossing(vy, v0y, sy, gny, kOccSuperShift),
                ez = cell_exit_crossing(vz, v0z, sz, gnz, kOccSuperShift);
            int bx = vx >> 5, by = vy >> 5, bz = vz >> 5;
            for (;;) {
                if constexpr (STATS) ++coarse;
                const uint32_t Nx = n0x + ((uint32_t)ex << 16), Ny = n0y + ((uint32_t)ey << 16), Nz = n0z + ((uint32_t)ez << 16);
                const int e = ev_argmin3(Nx, ax, Ny, ay, Nz, az);
                const int Ee = e == 0 ? ex : (e == 1 ? ey : ez);
                if (Ee >= (e == 0 ? kx : (e == 1 ? ky : kz))) return kNoHit;  // leaves the grid or the range
                const uint32_t NE = e == 0 ? Nx : (e == 1 ? Ny : Nz), AE = e == 0 ? ax : (e == 1 ? ay : az);
                const int s_e = e == 0 ? sx : (e == 1 ? sy : sz), v0e = e == 0 ? v0x : (e == 1 ? v0y : v0z);
                const int ue = v0e + s_e * (Ee + 1);
                const int nEe = cell_exit_crossing(ue, v0e, s_e, e == 0 ? gnx : (e == 1 ? gny : gnz), kOccSuperShift);
                bx = e == 0 ? ue >> 5 : bx;
                by = e == 1 ? ue >> 5 : by;
                bz = e == 2 ? ue >> 5 : bz;
                const int ox = ex, oy = ey, oz = ez;
                ex = e == 0 ? nEe : ex;
                ey = e == 1 ? nEe : ey;
                ez = e == 2 ? nEe : ez;
                if (ld_u8(sbocc + (bz * nsy + by) * nsx + bx)) {
                    enter(NE, AE, e, Ee, ox, oy, oz);
                    break;
                }
            }
            continue;
        }
        if (!bocc || ld_u8(bocc + ((vz >> 3) * nby + (vy >> 3)) * nbx + (vx >> 3))) {
            // voxel walk inside a brick that holds an occupied voxel, up to its faces: bnx.. = face
            // distance of the crossing that leaves the brick along each axis
            const uint32_t bnx = n0x + ((uint32_t)brick_exit_crossing(vx, v0x, sx, gnx) << 16);
            const uint32_t bny = n0y + ((uint32_t)brick_exit_crossing(vy, v0y, sy, gny) << 16);
            const uint32_t bnz = n0z + ((uint32_t)brick_exit_crossing(vz, v0z, sz, gnz) << 16);
            uint32_t addr = ((uint32_t)vz * (uint32_t)gny + (uint32_t)vy) * (uint32_t)gnx + (uint32_t)vx;
            for (;;) {
                if constexpr (STATS) ++fine;
                if (ld_u8(g + addr) == kOcc) return m;
                const int a = ev_argmin3(nx, ax, ny, ay, nz, az);
                const uint32_t na = a == 0 ? nx : (a == 1 ? ny : nz);
                if (na >= (a == 0 ? lx : (a == 1 ? ly : lz))) return kNoHit;  // leaves the grid or the range
                const bool leave = na == (a == 0 ? bnx : (a == 1 ? bny : bnz));
                nx += a == 0 ? kQ16 : 0u;
                ny += a == 1 ? kQ16 : 0u;
                nz += a == 2 ? kQ16 : 0u;
                vx += a == 0 ? sx : 0;
                vy += a == 1 ? sy : 0;
                vz += a == 2 ? sz : 0;
                addr += a == 0 ? dax : (a == 1 ? day : daz);
                ++m;
                if (leave) break;  // entered another brick
            }
            continue;
        }
        // brick walk: per axis the crossing index (from the start) that leaves the current brick,
        // until the ray enters a brick that holds an occupied voxel or a super-brick that holds none
        int ex = brick_exit_crossing(vx, v0x, sx, gnx), ey = brick_exit_crossing(vy, v0y, sy, gny),
            ez = brick_exit_crossing(vz, v0z, sz, gnz);
        int bx = vx >> 3, by = vy >> 3, bz = vz >> 3;
        for (;;) {
            if constexpr (STATS) ++coarse;
            const uint32_t Nx = n0x + ((uint32_t)ex << 16), Ny = n0y + ((uint32_t)ey << 16), Nz = n0z + ((uint32_t)ez << 16);
            const int e = ev_argmin3(Nx, ax, Ny, ay, Nz, az);
            const int Ee = e == 0 ? ex : (e == 1 ? ey : ez);
            if (Ee >= (e == 0 ? kx : (e == 1 ? ky : kz))) return kNoHit;  // leaves the grid or the range
            const uint32_t NE = e == 0 ? Nx : (e == 1 ? Ny : Nz), AE = e == 0 ? ax : (e == 1 ? ay : az);
            // the voxel that crossing enters along e, and the brick beyond
            const int s_e = e == 0 ? sx : (e == 1 ? sy : sz), v0e = e == 0 ? v0x : (e == 1 ? v0y : v0z);
            const int ue = v0e + s_e * (Ee + 1);
            const int nb = ue >> 3;
            const int nEe = brick_exit_crossing(ue, v0e, s_e, e == 0 ? gnx : (e == 1 ? gny : gnz));
            const bool new_super = (nb >> 2) != ((e == 0 ? bx : (e == 1 ? by : bz)) >> 2);
            bx = e == 0 ? nb : bx;
            by = e == 1 ? nb : by;
            bz = e == 2 ? nb : bz;
            const int ox = ex, oy = ey, oz = ez;
            ex = e == 0 ? nEe : ex;
            ey = e == 1 ? nEe : ey;
            ez = e == 2 ? nEe : ez;
            if (ld_u8(bocc + (bz * nby + by) * nbx + bx) ||
                (sbocc && new_super && !ld_u8(sbocc + ((bz >> 2) * nsy + (by >> 2)) * nsx + (bx >> 2)))) {
                enter(NE, AE, e, Ee, ox, oy, oz);
                break;
            }
        }
    }
}

// Does the DDA of the ray from P (Q16) along d (Q30) reach voxel (x, y, z) before the range T, and
// after how many steps? The voxel lies c_a = s_a (v_a - v0_a) crossings from the start voxel along
// each axis; it is on the ray iff every c_a >= 0 (c_a = 0 where d_a = 0) and its last entering
// event precedes its first leaving event, and it is reached iff that entering event starts before
// T. Returns the step index c_x + c_y + c_z, or -1. (The grid needs no test for a voxel inside it:
// the voxels between the start and it are inside too.)
MIG_HD int visit_index(int Px, int Py, int Pz, int dx, int dy, int dz, int x, int y, int z, int64_t Tq) {
    uint32_t n[3], ad[3];
    int c[3];
    const int P[3] = {Px, Py, Pz}, d[3] = {dx, dy, dz}, v[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int v0, s;
        ray_axis(P[a], d[a], v0, s, n[a], ad[a]);
        c[a] = s * (v[a] - v0);
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
    if (((uint64_t)en << 30) >= (uint64_t)Tq * eA) return -1;  // entered at t >= T
    // first leaving event: crossing c_a of each axis that moves
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (ad[a] != 0 && !ev_lt(en, eA, ea, n[a] + ((uint32_t)c[a] << 16), ad[a], a)) return -1;
    }
    return c[0] + c[1] + c[2];
}

// A sufficient condition for visit_index >= 0, in float: the point of the ray (origin P, direction
// d, Q30) nearest to the voxel's centre c (cx, cy, cz: c - P in voxels) lies inside the voxel, at
// least 0.01 voxel from every face, at a distance s along the ray with 0.01 <= s <= T - 0.01 (T in
// voxels). Then the ray crosses the voxel's interior there; between crossings the walk is in the
// voxel that holds the ray point, so it visits the voxel, before T, and inside the grid (a box,
// which holds the origin and the voxel). The float rounding of c (below 1e-3 voxel for grids up to
// 4096) and of the products and the quotient (relative 1e-6 of at most 1030 voxels) stays inside
// the 0.01 voxel margins. False says nothing.
MIG_HD bool visit_surely(float cx, float cy, float cz, int dx, int dy, int dz, float Tv) {
    const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
    const float dd = fx * fx + fy * fy + fz * fz;
    const float cd = cx * fx + cy * fy + cz * fz;
    const float lam = fast_divf(cd, dd);  // the nearest point is P + lam d
    const float ex = lam * fx - cx, ey = lam * fy - cy, ez = lam * fz - cz;
    const float s = cd * 1073741824.0f;  // distance along the ray times |d|^2 (|d| = 2^30)
    return fabsf(ex) < 0.49f && fabsf(ey) < 0.49f && fabsf(ez) < 0.49f && s >= 0.01f * dd &&
           s <= (Tv - 0.01f) * dd;
}

// Eq. 5's pixel of a voxel centre from float projection rows, with a proven error bound: returns 1
// when the exact test (Z > 0, pixel (floor(U/Z), floor(V/Z)) inside the image) surely passes with
// pixel (pu, pv), 0 when it surely fails, -1 when the float values are too close to a pixel boundary
// or to Z = 0 to tell (the caller runs the exact test). w: the yaw's rows mu, mv, mz as floats
// divided by 2^16 (each within relative 2^-24 of the exact row); ex, ey, ez: the centre's offset
// from the camera in voxels, converted from its exact Q16 value (within relative 2^-24). Each float
// sum of three products is then within 5 u S of the exact one (u = 2^-24, S = the row's L1 norm
// times the largest offset), so with eU, eV, eZ = norm * 6.5 u (rinf + 1):
//   |Z - Zf| <= eZ, and for Zf > 2 eZ, |U/Z - Uf/Zf| <= 2 (eU + |Uf/Zf| eZ) / Zf;
// the fast reciprocal and the product add at most 3.1e-7 |u|, covered by the 1e-6 terms.
// zf, e_z: the float camera depth (voxels) and its error bound, for a depth comparison that follows.
MIG_HD int pixel_fast(const float *w, float ex, float ey, float ez, float rinf, int W, int H, int &pu, int &pv,
                      float &zf, float &e_z) {
    const float c = 3.9e-7f * (rinf + 1.0f);  // 6.5 * 2^-24 * (rinf + 1)
    zf = fmaf(w[6], ex, fmaf(w[7], ey, w[8] * ez));
    e_z = (fabsf(w[6]) + fabsf(w[7]) + fabsf(w[8])) * c;
    if (!(zf > 2.0f * e_z)) return zf < -e_z ? 0 : -1;
    const float zi = fast_divf(1.0f, zf);
    const float u = fmaf(w[0], ex, fmaf(w[1], ey, w[2] * ez)) * zi;
    const float v = fmaf(w[3], ex, fmaf(w[4], ey, w[5] * ez)) * zi;
    const float e_u = 2.0f * zi * ((fabsf(w[0]) + fabsf(w[1]) + fabsf(w[2])) * c + fabsf(u) * e_z) + 1e-6f * fabsf(u) + 1e-6f;
    const float e_v = 2.0f * zi * ((fabsf(w[3]) + fabsf(w[4]) + fabsf(w[5])) * c + fabsf(v) * e_z) + 1e-6f * fabsf(v) + 1e-6f;
    if (u + e_u < 0.0f || u - e_u >= (float)W || v + e_v < 0.0f || v - e_v >= (float)H) return 0;
    const float fu = floorf(u - e_u), fv = floorf(v - e_v);
    if (fu < 0.0f || fv < 0.0f || floorf(u + e_u) != fu || floorf(v + e_v) != fv) return -1;
    pu = (int)fu;
    pv = (int)fv;
    return 1;
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
