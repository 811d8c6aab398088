/*
 * CPU ORACLE for path-dependent marginal information gain with depth buffers.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. It shares no code with the CUDA library and
 * includes none of its headers; it is a plain, slow, direct statement of the method:
 *
 *   - the depth-buffer method (Sec. IV-A..C), restated step by step over the tree in
 *     depth order, with integer readings of the paper's unstated details (all decisions are
 *     integer: quantised inputs, exact rational DDA, exact integer projection), in its modes:
 *     marginal with voxel-centre samples, single parent, absolute, the paper's screen-space
 *     interval overlap (Eq. 5-7, the literal per-ancestor pixel walk) and panoramic counting;
 *   - the visible-voxel sets I(n, psi) of Eq. 1, and the exact marginal gain of Eq. 2 by a
 *     depth-first walk with per-voxel reference counts (route 2 of the exact reference; the
 *     hash-set merge of Sec. I / Sec. IV-E is route 1, in oracle/exact.py).
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -shared -fPIC (no -ffast-math).
 * Parity: pinned by the tests in tests/test_oracle_*.py (brute-force DDA with exact
 * rationals, voxel-centric owner sets, closed-form depth and volume, invariants of Eq. 2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

#define ONE_Q16 ((i64)65536)
#define ONE_Q30 ((i64)1073741824)
#define OR_UNKNOWN 0
#define OR_FREE 1
#define OR_OCCUPIED 2
#define OR_MAX_DEPTH 64

enum { MODE_MARGINAL = 0, MODE_SINGLE_PARENT = 1, MODE_ABSOLUTE = 2, MODE_INTERVAL = 3, MODE_PANORAMIC = 4 };

/* Planted mistakes for the pin-strength tests (tests/test_oracle_mutants.py). The default
 * build defines none; each variant .so is built with -DORACLE_MUTANT=<m> and must fail at
 * least one pin. MUT(m) is 1 only in variant m. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUT(m) (ORACLE_MUTANT == (m))

/* floor(a / b) for b > 0, for any sign of a */
static i64 floor_div(i64 a, i64 b) {
    i64 q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

static int32_t q30(double x) { return (int32_t)llrint(x * 1073741824.0); }
static int32_t q16(double x) { return (int32_t)llrint(x * 65536.0); }

/* ------------------------------------------------------------------------------------
 * Camera model (Eq. 5): pinhole with principal point at the image centre, focal lengths
 * from the field of view, rays through pixel centres. Camera axes: x right, y down,
 * z forward; body forward = world +x at yaw 0; pitch positive = nose down; yaw bins
 * psi_k = 2 pi k / K counter-clockwise about world +z.
 * ------------------------------------------------------------------------------------ */
typedef struct {
    int W, H, K;
    double t_h, t_v, cp, sp;
    int32_t *bx, *by, *bz, *dzc; /* per pixel j*W+i: body-frame unit ray (Q30), camera z of it (Q30) */
    int32_t *ck, *sk;            /* per yaw: cos, sin (Q30) */
    int32_t *M;                  /* per yaw: rows mu, mv, mz (Q16): (u z, v z, z) = M r */
} cam_t;

static void cam_free(cam_t *c) {
    free(c->bx); free(c->by); free(c->bz); free(c->dzc);
    free(c->ck); free(c->sk); free(c->M);
}

static int cam_build(cam_t *c, float hfov_deg, float vfov_deg, int W, int H, int K, float pitch_deg) {
    memset(c, 0, sizeof(*c));
    if (W < 1 || H < 1 || W > 2048 || H > 2048 || K < 1 || K > 1024) return -1;
    if (!(hfov_deg > 0.0f && hfov_deg < 180.0f && vfov_deg > 0.0f && vfov_deg < 180.0f)) return -1;
    if (!(pitch_deg >= -90.0f && pitch_deg <= 90.0f)) return -1;
    c->W = W; c->H = H; c->K = K;
    c->t_h = tan(((double)hfov_deg * 0.5) * (M_PI / 180.0));
    c->t_v = tan(((double)vfov_deg * 0.5) * (M_PI / 180.0));
    double th = (double)pitch_deg * (M_PI / 180.0);
    c->cp = cos(th);
    c->sp = sin(th);
    size_t np = (size_t)W * H;
    c->bx = malloc(np * 4); c->by = malloc(np * 4); c->bz = malloc(np * 4); c->dzc = malloc(np * 4);
    c->ck = malloc((size_t)K * 4); c->sk = malloc((size_t)K * 4); c->M = malloc((size_t)K * 9 * 4);
    if (!c->bx || !c->by || !c->bz || !c->dzc || !c->ck || !c->sk || !c->M) { cam_free(c); return -2; }
    for (int j = 0; j < H; ++j) {
        for (int i = 0; i < W; ++i) {
            /* tangent-plane coordinates of the pixel centre: (i + 1/2 - c_x) / f_x */
            double a = ((double)(2 * i + (MUT(1) ? 0 : 1) - W) / (double)W) * c->t_h;
            double b = ((double)(2 * j + 1 - H) / (double)H) * c->t_v;
            double nrm = sqrt((a * a + b * b) + 1.0);
            double cx = a / nrm, cy = b / nrm, cz = 1.0 / nrm;
            size_t p = (size_t)j * W + i;
            c->bx[p] = q30(cz * c->cp - cy * c->sp);
            c->by[p] = q30(MUT(2) ? cx : -cx);
            c->bz[p] = q30(-(cy * c->cp + cz * c->sp));
            c->dzc[p] = q30(cz);
        }
    }
    double fx = ((double)W * 0.5) / c->t_h, fy = ((double)H * 0.5) / c->t_v;
    double cxp = (double)W * 0.5, cyp = (double)H * 0.5;
    for (int k = 0; k < K; ++k) {
        double ang = ((2.0 * M_PI) * (double)k) / (double)K;
        double cs = cos(ang), sn = sin(ang);
        c->ck[k] = q30(cs);
        c->sk[k] = q30(sn);
        double ex[3] = {sn, -cs, 0.0};
        double ey[3] = {-(c->sp * cs), -(c->sp * sn), -c->cp};
        double ez[3] = {c->cp * cs, c->cp * sn, -c->sp};
        for (int a = 0; a < 3; ++a) {
            double mu = fx * ex[a] + cxp * ez[a];
            double mv = fy * ey[a] + cyp * ez[a];
            if (fabs(mu) * 65536.0 >= 2147483647.0 || fabs(mv) * 65536.0 >= 2147483647.0) { cam_free(c); return -1; }
            c->M[k * 9 + a] = q16(mu);
            c->M[k * 9 + 3 + a] = q16(mv);
            c->M[k * 9 + 6 + a] = q16(ez[a]);
        }
    }
    return 0;
}

/* world direction of pixel p at yaw k (Q30): yaw rotation of the body-frame ray */
static void cam_dir(const cam_t *c, int k, size_t p, i64 d[3]) {
    i64 bx = c->bx[p], by = c->by[p];
    d[0] = floor_div((i64)c->ck[k] * bx - (i64)c->sk[k] * by, ONE_Q30);
    d[1] = floor_div((MUT(12) ? -1 : 1) * (i64)c->sk[k] * bx + (i64)c->ck[k] * by, ONE_Q30);
    d[2] = c->bz[p];
}

/* Eq. 5 in integers: project voxel centre v into the camera at P (Q16) with yaw k.
 * Returns 1 and the pixel when the centre is in front (z > 0); *Zq = z in Q32. */
static int project(const cam_t *c, int k, const i64 P[3], const int32_t v[3], i64 *pu, i64 *pv, i64 *Zq) {
    i64 r[3];
    for (int a = 0; a < 3; ++a) r[a] = (i64)v[a] * ONE_Q16 + ONE_Q16 / 2 - P[a];
    const int32_t *m = c->M + (size_t)k * 9;
    i64 U = (i64)m[0] * r[0] + (i64)m[1] * r[1] + (MUT(4) ? 0 : (i64)m[2] * r[2]);
    i64 V = (i64)m[3] * r[0] + (i64)m[4] * r[1] + (i64)m[5] * r[2];
    i64 Z = (i64)m[6] * r[0] + (i64)m[7] * r[1] + (i64)m[8] * r[2];
    *Zq = Z;
    if (Z <= 0) return 0;
    *pu = MUT(3) ? U / Z : floor_div(U, Z);
    *pv = MUT(3) ? V / Z : floor_div(V, Z);
    return 1;
}

/* ------------------------------------------------------------------------------------
 * Map
 * ------------------------------------------------------------------------------------ */
typedef struct {
    const uint8_t *g;
    int n[3];
} grid_t;

static uint8_t grid_at(const grid_t *G, const int32_t v[3]) {
    return G->g[((size_t)v[2] * G->n[1] + v[1]) * G->n[0] + v[0]];
}

/* ------------------------------------------------------------------------------------
 * 3D DDA (Amanatides-Woo, "Woo 1987", Sec. IV-B) on the quantised ray P + t d.
 * t is compared as an exact rational n/|d| per axis (n = distance to the next face in
 * Q16, |d| in Q30); the axis with the smallest next crossing steps, ties x, then y,
 * then z. A voxel is visited iff its entry t is < T (range); the ray ends on an
 * occupied voxel (visited, not counted), at the range, or on leaving the grid.
 * The visitor returns 0 to continue. Returns 1 on an occupied hit and the depth of the
 * hit's entry point in Q16 voxel units through *D (Sec. IV-A), else 0 and the range
 * endpoint's depth.
 * ------------------------------------------------------------------------------------ */
/* The visitor also receives the voxel's entry crossing te = (n, |d|) (t = n / |d|; (0, 1) for the
 * start voxel) and its exit crossing tx (the next crossing in the traversal order). */
typedef int (*visit_fn)(void *ctx, const int32_t v[3], uint8_t code, const i64 te[2], const i64 tx[2]);

static int dda(const grid_t *G, const i64 P[3], const i64 d[3], i64 Tq, i64 dzc, visit_fn fn, void *ctx,
               uint32_t *D) {
    int32_t v[3];
    int step[3];
    i64 nn[3], ad[3];
    for (int a = 0; a < 3; ++a) {
        v[a] = (int32_t)floor_div(P[a], ONE_Q16);
        if (d[a] > 0) { step[a] = 1; ad[a] = d[a]; nn[a] = ((i64)v[a] + 1) * ONE_Q16 - P[a]; }
        else if (d[a] < 0) { step[a] = -1; ad[a] = -d[a]; nn[a] = P[a] - (i64)v[a] * ONE_Q16; }
        else { step[a] = 0; ad[a] = 0; nn[a] = ONE_Q16; }
    }
    i64 ne = 0, ade = 1; /* entry t of the current voxel = ne / ade (scaled) */
    for (;;) {
        uint8_t code = grid_at(G, v);
        int best = -1;
        for (int a = 0; a < 3; ++a) {
            if (ad[a] == 0) continue;
            if (best < 0 || (MUT(5) ? nn[a] * ad[best] <= nn[best] * ad[a] : nn[a] * ad[best] < nn[best] * ad[a])) best = a;
        }
        if (fn) {
            const i64 te[2] = {ne, ade}, tx[2] = {nn[best], ad[best]};
            fn(ctx, v, code, te, tx);
        }
        if (code == OR_OCCUPIED) {
            if (D) *D = (uint32_t)floor_div((MUT(7) && ade > 1 ? ne + ONE_Q16 : ne) * dzc, ade);
            return 1;
        }
        /* next entry t = nn[best]/ad[best] (voxel units: nn * 2^14 / ad); stop if >= T */
        if (MUT(6) ? nn[best] * ONE_Q30 > Tq * ad[best] : nn[best] * ONE_Q30 >= Tq * ad[best]) break;
        v[best] += step[best];
        if (v[best] < 0 || v[best] >= G->n[best]) break;
        ne = nn[best];
        ade = ad[best];
        nn[best] += ONE_Q16;
    }
    if (D) *D = (uint32_t)floor_div(Tq * dzc, ONE_Q30);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Tree evaluation (Sec. IV-C): levels in increasing depth; per node and yaw, cast all
 * pixel rays, count owned unknown voxels (absolute, Eq. 1) and those no ancestor's depth
 * buffer observes (marginal, Eq. 2 by depth buffers, Sec. IV-B); argmax over yaw; keep
 * the depth buffer of the selected yaw (Sec. IV-A).
 * ------------------------------------------------------------------------------------ */
typedef struct {
    const cam_t *cam;
    const grid_t *G;
    int k;
    i64 pi, pj;
    const i64 *P;
    int n_anc;
    const i64 (*anc_P)[3];
    const int *anc_yaw;
    uint32_t *const *anc_D;
    i64 abs_count, marg_count;
} count_ctx;

static int owned(const cam_t *c, int k, const i64 P[3], const int32_t v[3], i64 pi, i64 pj) {
    i64 pu, pv, Z;
    if (!project(c, k, P, v, &pu, &pv, &Z)) return 0;
    return pu == pi && pv == pj;
}

static int observed_by(const cam_t *c, const i64 Pa[3], int ka, const uint32_t *Da, const int32_t v[3]) {
    i64 pu, pv, Z;
    if (!project(c, ka, Pa, v, &pu, &pv, &Z)) return 0;
    if (pu < 0 || pu >= c->W || pv < 0 || pv >= c->H) return 0;
    i64 Dq = Da[(size_t)pv * c->W + (size_t)pu];
    return MUT(10) ? Z < Dq * ONE_Q16 : Z < (Dq + 1) * ONE_Q16; /* floor(z in Q16) <= stored depth */
}

static int count_visit(void *vctx, const int32_t v[3], uint8_t code, const i64 te[2], const i64 tx[2]) {
    (void)te;
    (void)tx;
    count_ctx *x = (count_ctx *)vctx;
    if (code != OR_UNKNOWN) return 0;
    if (!MUT(8) && !owned(x->cam, x->k, x->P, v, x->pi, x->pj)) return 0;
    x->abs_count++;
    for (int a = 0; a < x->n_anc; ++a)
        if (observed_by(x->cam, x->anc_P[a], x->anc_yaw[a], x->anc_D[a], v)) return 0;
    x->marg_count++;
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Interval mode: the screen-space overlap of Sec. IV-B (Eq. 5-7), restated in the paper's
 * order. For a candidate ray r(t) = p_n + t d (0 <= t <= range) and each ancestor a:
 *   1. the ray's start and range endpoint in a's camera, as projective image coordinates
 *      (U, V, Z) = M_a (x - p_a) (exact integers, Q32, then IEEE float in voxel units);
 *      (U, V, Z) is linear in the ray fraction lambda = t / range;
 *   2. clip along camera z to the valid depth range [Z_NEAR, range] (Sec. IV-B: the
 *      "valid depth range"; depths beyond the range can never be <= a stored depth);
 *   3. project the clipped endpoints (Eq. 5), u = U / Z, v = V / Z, with inverse depths
 *      w = 1 / Z, and clip the 2D segment to the buffer [0, W] x [0, H] (Liang-Barsky);
 *   4. walk the pixels of the clipped segment with a 2D DDA ("Woo 1987"). Each visited pixel
 *      holds one portion [s_in, s_out) of the segment parameter s; its depth sample is taken
 *      at the portion's midpoint with w linear in s (Eq. 6), and the portion is observed iff
 *      its depth is <= D_a[pixel] ("smaller or equal"), compared in inverse depth as w D >= 1.
 *      Boundary crossings use one reciprocal of the segment's screen extent. The maximal runs of observed
 *      portions are the intervals S_a of Eq. 7.
 * Then the 3D DDA counts (Sec. IV-B, last paragraph): an owned unknown voxel is a sample at
 * the midpoint of the ray's traversal of it (lambda_s, the exit capped at the range); it is
 * observed iff it lies in the union of the S_a, i.e. iff for some ancestor its screen
 * parameter s (perspective-correct, from lambda_s) falls in an observed portion. Each sample
 * is classified by the first portion in walk order with s_in <= s < s_out.
 * All steps after the exact projective endpoints are IEEE single-precision operations in a
 * fixed order (no contraction): the decisions are reproducible bit for bit.
 * ------------------------------------------------------------------------------------ */
#define Z_NEAR (1.0f / 1024.0f) /* voxel units */

typedef struct {
    float lo, hi;         /* depth-clipped range of lambda */
    float Za, Zb;         /* camera z at lo, hi (voxel units) */
    float ua, va, ub, vb; /* projected clipped endpoints (pixels) */
    float wa, wb;         /* inverse depths at the endpoints */
    float s0, s1;         /* Liang-Barsky range of s over [0, 1] */
    float ru, rv;         /* reciprocals of the segment's screen extent (0 when it is 0) */
} seg2d_t;

typedef struct {
    float s_in, s_out;
    int obs;
    int i, j; /* the pixel */
} portion_t;

/* range endpoint of the ray, Q16: E = P + floor(T d / 2^30) */
static void ray_end(const i64 P[3], const i64 d[3], i64 Tq, i64 E[3]) {
    for (int a = 0; a < 3; ++a) E[a] = P[a] + floor_div(Tq * d[a], ONE_Q30);
}

/* steps 1-3; returns 0 if nothing of the ray is inside a's depth range and image */
static int seg_setup(const cam_t *c, int ka, const i64 Pa[3], const i64 P[3], const i64 E[3], i64 Tq, seg2d_t *g) {
    const int32_t *m = c->M + (size_t)ka * 9;
    i64 r0[3], r1[3];
    for (int a = 0; a < 3; ++a) { r0[a] = P[a] - Pa[a]; r1[a] = E[a] - Pa[a]; }
    const float sc = 1.0f / 4294967296.0f; /* Q32 -> voxel units (exact power of two) */
    float U0 = (float)(m[0] * r0[0] + m[1] * r0[1] + m[2] * r0[2]) * sc;
    float V0 = (float)(m[3] * r0[0] + m[4] * r0[1] + m[5] * r0[2]) * sc;
    float Z0 = (float)(m[6] * r0[0] + m[7] * r0[1] + m[8] * r0[2]) * sc;
    float U1 = (float)(m[0] * r1[0] + m[1] * r1[1] + m[2] * r1[2]) * sc;
    float V1 = (float)(m[3] * r1[0] + m[4] * r1[1] + m[5] * r1[2]) * sc;
    float Z1 = (float)(m[6] * r1[0] + m[7] * r1[1] + m[8] * r1[2]) * sc;
    const float zn = Z_NEAR, zf = (float)Tq * (1.0f / 65536.0f);
    float dZ = Z1 - Z0, lo = 0.0f, hi = 1.0f;
    if (Z0 < zn) { if (!(dZ > 0.0f)) return 0; lo = (zn - Z0) / dZ; }
    if (Z1 < zn) { if (!(dZ < 0.0f)) return 0; hi = (zn - Z0) / dZ; }
    if (Z0 > zf) { if (!(dZ < 0.0f)) return 0; float l = (zf - Z0) / dZ; if (l > lo) lo = l; }
    if (Z1 > zf) { if (!(dZ > 0.0f)) return 0; float h = (zf - Z0) / dZ; if (h < hi) hi = h; }
    if (!(lo < hi)) return 0;
    float dU = U1 - U0, dV = V1 - V0;
    float Ua = U0 + lo * dU, Va = V0 + lo * dV, Za = Z0 + lo * dZ;
    float Ub = U0 + hi * dU, Vb = V0 + hi * dV, Zb = Z0 + hi * dZ;
    if (!(Za > 0.0f && Zb > 0.0f)) return 0;
    g->lo = lo; g->hi = hi; g->Za = Za; g->Zb = Zb;
    /* Eq. 5 with the inverse depths of Eq. 6: u = U w, v = V w */
    g->wa = 1.0f / Za; g->wb = 1.0f / Zb;
    g->ua = Ua * g->wa; g->va = Va * g->wa; g->ub = Ub * g->wb; g->vb = Vb * g->wb;
    /* Liang-Barsky ("Liang 1984") against 0 <= u <= W, 0 <= v <= H; each edge's crossing is
     * q times the reciprocal of p (+-1/du or +-1/dv) */
    float du = g->ub - g->ua, dv = g->vb - g->va;
    g->ru = du != 0.0f ? 1.0f / du : 0.0f;
    g->rv = dv != 0.0f ? 1.0f / dv : 0.0f;
    float p[4] = {-du, du, -dv, dv};
    float rp[4] = {-g->ru, g->ru, -g->rv, g->rv};
    float q[4] = {g->ua, (float)c->W - g->ua, g->va, (float)c->H - g->va};
    float s0 = 0.0f, s1 = 1.0f;
    for (int e = 0; e < 4; ++e) {
        if (p[e] == 0.0f) { if (q[e] < 0.0f) return 0; continue; }
        float r = q[e] * rp[e];
        if (p[e] < 0.0f) { if (r > s1) return 0; if (r > s0) s0 = r; }
        else { if (r < s0) return 0; if (r < s1) s1 = r; }
    }
    if (!(s0 < s1)) return 0;
    g->s0 = s0; g->s1 = s1;
    return 1;
}

/* step 4: the 2D DDA over the clipped segment; writes the portions in walk order */
static int seg_walk(const seg2d_t *g, int W, int H, const uint32_t *D, portion_t *out) {
    float du = g->ub - g->ua, dv = g->vb - g->va;
    /* boundary crossings: (boundary - start) times the reciprocal of the segment's extent */
    float ru = g->ru, rv = g->rv;
    float s = g->s0;
    /* start pixel, clamped to the buffer in float (before any conversion to int) */
    float fi = floorf(g->ua + s * du), fj = floorf(g->va + s * dv);
    int i = fi < 0.0f ? 0 : (fi > (float)(W - 1) ? W - 1 : (int)fi);
    int j = fj < 0.0f ? 0 : (fj > (float)(H - 1) ? H - 1 : (int)fj);
    int si = du > 0.0f ? 1 : (du < 0.0f ? -1 : 0), sj = dv > 0.0f ? 1 : (dv < 0.0f ? -1 : 0);
    float sx = si ? ((float)(si > 0 ? i + 1 : i) - g->ua) * ru : INFINITY;
    float sy = sj ? ((float)(sj > 0 ? j + 1 : j) - g->va) * rv : INFINITY;
    int np = 0;
    for (;;) {
        float se = sx < sy ? sx : sy;
        if (g->s1 < se) se = g->s1;
        float sm = MUT(14) ? s : (s + se) * 0.5f;  /* Eq. 6 at the portion's midpoint */
        float wm = g->wa + sm * (g->wb - g->wa);
        float Dv = (float)D[(size_t)j * W + i] * (1.0f / 65536.0f);
        /* z <= D ("smaller or equal"), compared in inverse depth: w D >= 1 */
        float wD = wm * Dv;
        out[np].s_in = s;
        out[np].s_out = se;
        out[np].obs = MUT(16) ? wD > 1.0f : wD >= 1.0f;
        out[np].i = i;
        out[np].j = j;
        np++;
        if (!(se < g->s1)) break;
        if (sx <= sy) {
            i += si;
            if (i < 0 || i >= W) break;
            sx = ((float)(si > 0 ? i + 1 : i) - g->ua) * ru;
        } else {
            j += sj;
            if (j < 0 || j >= H) break;
            sy = ((float)(sj > 0 ? j + 1 : j) - g->va) * rv;
        }
        s = se;
    }
    return np;
}

/* screen parameter of the ray fraction lam (perspective-correct); 0 if outside the clip */
static int seg_param(const seg2d_t *g, float lam, float *s) {
    if (!(lam >= g->lo && lam <= g->hi)) return 0;
    float mu = (lam - g->lo) / (g->hi - g->lo);
    float num = mu * g->Zb;
    float den = (1.0f - mu) * g->Za + num;
    *s = MUT(15) ? mu : num / den;
    return *s >= g->s0 && *s < g->s1;
}

/* observed by one ancestor: the first portion (walk order) that contains s decides */
static int portions_observe(const portion_t *pt, int np, float s) {
    for (int q = 0; q < np; ++q)
        if (pt[q].s_in <= s && s < pt[q].s_out) return pt[q].obs;
    return 0;
}

/* the voxel's sample: midpoint of the ray's traversal of it, as a fraction of the range */
static float sample_lambda(const i64 te[2], const i64 tx[2], i64 Tq) {
    const float T = (float)Tq * (1.0f / 1073741824.0f);
    float lin = ((float)te[0] / (float)te[1]) / T;
    float lout = ((float)tx[0] / (float)tx[1]) / T;
    if (lout > 1.0f) lout = 1.0f;
    return MUT(17) ? lin : (lin + lout) * 0.5f;
}

typedef struct {
    const cam_t *cam;
    int k;
    i64 pi, pj;
    const i64 *P;
    i64 E[3]; /* the ray's range endpoint */
    i64 Tq;
    int n_anc;
    const i64 (*anc_P)[3];
    const int *anc_yaw;
    uint32_t *const *anc_D;
    int built;            /* the S_a of this ray are built (on its first sample) */
    seg2d_t *seg;         /* per ancestor */
    int *seg_ok, *n_por;  /* per ancestor */
    portion_t *por;       /* per ancestor, W + H + 2 each */
    i64 abs_count, marg_count;
} ival_ctx;

static void build_intervals(ival_ctx *x) {
    const int cap = x->cam->W + x->cam->H + 2;
    for (int a = 0; a < x->n_anc; ++a) {
        x->seg_ok[a] = seg_setup(x->cam, x->anc_yaw[a], x->anc_P[a], x->P, x->E, x->Tq, &x->seg[a]);
        x->n_por[a] = x->seg_ok[a] ? seg_walk(&x->seg[a], x->cam->W, x->cam->H, x->anc_D[a], x->por + (size_t)a * cap) : 0;
    }
    x->built = 1;
}

static int interval_visit(void *vctx, const int32_t v[3], uint8_t code, const i64 te[2], const i64 tx[2]) {
    ival_ctx *x = (ival_ctx *)vctx;
    if (code != OR_UNKNOWN) return 0;
    if (!owned(x->cam, x->k, x->P, v, x->pi, x->pj)) return 0;
    x->abs_count++;
    if (!x->built) build_intervals(x);
    const int cap = x->cam->W + x->cam->H + 2;
    float lam = sample_lambda(te, tx, x->Tq);
    for (int a = 0; a < x->n_anc; ++a) {
        float sp;
        if (!x->seg_ok[a] || !seg_param(&x->seg[a], lam, &sp)) continue;
        if (portions_observe(x->por + (size_t)a * cap, x->n_por[a], sp)) return 0;
    }
    x->marg_count++;
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Panoramic mode: one 360-degree cast per node, then a window sum per yaw bin (the yaw set of
 * Sec. III-B evaluated from shared rays). The horizon is cut into A azimuth wedges ("columns")
 * of width 2 pi / A, A = K * ceil(W 360 / (hfov K)) so that a yaw step is a whole number of
 * columns and a column is no wider than a pinhole pixel at the image centre. Column c holds
 * the directions with azimuth in [c, c + 1) * 2 pi / A (exact integer test against the wedge's
 * two boundary vectors, Q30). Each column is a one-pixel-wide strip camera looking along the
 * wedge's centre azimuth, with the pinhole's rows (Eq. 5's v, focal length and principal point
 * from the vertical field of view); its rays pass through the strip's row centres. A voxel is
 * owned by the cell (column, row) containing its centre (as a pinhole voxel is owned by the
 * pixel containing its centre's projection), counted as
 * absolute gain for the column, and as marginal gain unless an ancestor's (pinhole) depth
 * buffer observes it. Yaw k sums the Wc = round(A hfov / 360) columns centred on its azimuth.
 * Level camera only (pitch 0): wedges are vertical half-planes.
 * ------------------------------------------------------------------------------------ */
typedef struct {
    int A, Wc, step, H;
    int32_t *bc;   /* A: boundary (cos, sin) of azimuth c 2 pi / A, Q30 */
    int32_t *dir;  /* A*H*3: ray of cell (c, j), Q30 */
    int32_t *row;  /* A*6: strip projection rows mv (3), mz (3), Q16 */
} pano_t;

static void pano_free(pano_t *p) { free(p->bc); free(p->dir); free(p->row); }

static int pano_build(pano_t *p, float hfov, float vfov, int W, int H, int K, float pitch) {
    memset(p, 0, sizeof(*p));
    if (W < 1 || H < 1 || W > 2048 || H > 2048 || K < 1 || K > 1024) return -1;
    if (!(hfov > 0.0f && hfov < 180.0f && vfov > 0.0f && vfov < 180.0f)) return -1;
    if (pitch != 0.0f) return -1;
    int step = (int)ceil(((double)W * 360.0) / ((double)hfov * (double)K));
    if (step < 1) step = 1;
    int A = step * K;
    if (A > 65536) return -1;
    p->A = A; p->step = step; p->H = H;
    p->Wc = (int)llrint(((double)A * (double)hfov) / 360.0);
    if (p->Wc < 1) p->Wc = 1;
    p->bc = malloc((size_t)A * 2 * 4);
    p->dir = malloc((size_t)A * H * 3 * 4);
    p->row = malloc((size_t)A * 6 * 4);
    if (!p->bc || !p->dir || !p->row) { pano_free(p); return -2; }
    double t_v = tan(((double)vfov * 0.5) * (M_PI / 180.0));
    double fy = ((double)H * 0.5) / t_v, cyp = (double)H * 0.5;
    for (int c = 0; c < A; ++c) {
        double ang = ((2.0 * M_PI) * (double)c) / (double)A;
        p->bc[2 * c] = q30(cos(ang));
        p->bc[2 * c + 1] = q30(sin(ang));
        double th = ((2.0 * M_PI) * ((double)c + 0.5)) / (double)A;
        double cs = cos(th), sn = sin(th);
        /* strip camera at azimuth th: ez = (cs, sn, 0), ey = (0, 0, -1) */
        double mv[3] = {cyp * cs, cyp * sn, -fy};
        for (int a = 0; a < 3; ++a) if (fabs(mv[a]) * 65536.0 >= 2147483647.0) { pano_free(p); return -1; }
        p->row[6 * c] = q16(mv[0]); p->row[6 * c + 1] = q16(mv[1]); p->row[6 * c + 2] = q16(mv[2]);
        p->row[6 * c + 3] = q16(cs); p->row[6 * c + 4] = q16(sn); p->row[6 * c + 5] = 0;
        for (int j = 0; j < H; ++j) {
            double b = ((double)(2 * j + 1 - H) / (double)H) * t_v;
            double nrm = sqrt(b * b + 1.0);
            int32_t *o = p->dir + ((size_t)c * H + j) * 3;
            o[0] = q30(cs / nrm);
            o[1] = q30(sn / nrm);
            o[2] = q30(-b / nrm);
        }
    }
    return 0;
}

/* the cell (column, row) owning voxel v seen from P (Q16); 0 if none (on the vertical axis,
 * behind the strip or outside its rows) */
static int pano_cell(const pano_t *p, const i64 P[3], const int32_t v[3], int *cc, int *jj) {
    i64 r[3];
    for (int a = 0; a < 3; ++a) r[a] = (i64)v[a] * ONE_Q16 + ONE_Q16 / 2 - P[a];
    /* column: the wedge c with cross(b_c, r) >= 0 > cross(b_{c+1}, r) */
    int c = -1;
    for (int q = 0; q < p->A; ++q) {
        const int32_t *b0 = p->bc + 2 * q, *b1 = p->bc + 2 * ((q + 1) % p->A);
        i64 x0 = (i64)b0[0] * r[1] - (i64)b0[1] * r[0];
        i64 x1 = (i64)b1[0] * r[1] - (i64)b1[1] * r[0];
        if (x0 >= 0 && (MUT(18) ? x1 <= 0 : x1 < 0)) { c = q; break; }
    }
    if (c < 0) return 0;
    const int32_t *m = p->row + 6 * c;
    i64 V = (i64)m[0] * r[0] + (i64)m[1] * r[1] + (i64)m[2] * r[2];
    i64 Z = (i64)m[3] * r[0] + (i64)m[4] * r[1] + (i64)m[5] * r[2];
    if (Z <= 0) return 0;
    i64 j = floor_div(V, Z);
    if (j < 0 || j >= p->H) return 0;
    *cc = c;
    *jj = (int)j;
    return 1;
}

/* is voxel v (seen from P) in cell (c, j)? the wedge test against column c's two boundaries */
static int pano_owned(const pano_t *p, int c, int j, const i64 P[3], const int32_t v[3]) {
    i64 r[3];
    for (int a = 0; a < 3; ++a) r[a] = (i64)v[a] * ONE_Q16 + ONE_Q16 / 2 - P[a];
    const int32_t *b0 = p->bc + 2 * c, *b1 = p->bc + 2 * ((c + 1) % p->A);
    i64 x0 = (i64)b0[0] * r[1] - (i64)b0[1] * r[0];
    i64 x1 = (i64)b1[0] * r[1] - (i64)b1[1] * r[0];
    if (!(x0 >= 0 && (MUT(18) ? x1 <= 0 : x1 < 0))) return 0;
    const int32_t *m = p->row + 6 * c;
    i64 V = (i64)m[0] * r[0] + (i64)m[1] * r[1] + (i64)m[2] * r[2];
    i64 Z = (i64)m[3] * r[0] + (i64)m[4] * r[1] + (i64)m[5] * r[2];
    return Z > 0 && floor_div(V, Z) == j;
}

/* first column of yaw k's window */
static int pano_window_start(const pano_t *p, int k) {
    int s0 = k * p->step - p->Wc / 2 + (MUT(19) ? 1 : 0);
    return ((s0 % p->A) + p->A) % p->A;
}

typedef struct {
    const pano_t *pano;
    const cam_t *cam;
    int c, j;
    const i64 *P;
    int n_anc;
    const i64 (*anc_P)[3];
    const int *anc_yaw;
    uint32_t *const *anc_D;
    i64 abs_count, marg_count;
} pano_ctx;

static int pano_visit(void *vctx, const int32_t v[3], uint8_t code, const i64 te[2], const i64 tx[2]) {
    (void)te;
    (void)tx;
    pano_ctx *x = (pano_ctx *)vctx;
    if (code != OR_UNKNOWN) return 0;
    if (!pano_owned(x->pano, x->c, x->j, x->P, v)) return 0;
    x->abs_count++;
    for (int a = 0; a < x->n_anc; ++a)
        if (observed_by(x->cam, x->anc_P[a], x->anc_yaw[a], x->anc_D[a], v)) return 0;
    x->marg_count++;
    return 0;
}

/* per-column counts of one node: cast every cell's ray once */
static void pano_columns(const pano_t *pano, const cam_t *cam, const grid_t *G, const i64 P[3], i64 Tq, int na,
                         const i64 (*anc_P)[3], const int *anc_yaw, uint32_t *const *anc_D, i64 *col_abs,
                         i64 *col_marg) {
    pano_ctx x = {pano, cam, 0, 0, P, na, anc_P, anc_yaw, anc_D, 0, 0};
    for (int c = 0; c < pano->A; ++c) {
        x.abs_count = x.marg_count = 0;
        x.c = c;
        for (int j = 0; j < pano->H; ++j) {
            const int32_t *o = pano->dir + ((size_t)c * pano->H + j) * 3;
            i64 d[3] = {o[0], o[1], o[2]};
            x.j = j;
            dda(G, P, d, Tq, ONE_Q30, pano_visit, &x, NULL);
        }
        col_abs[c] = x.abs_count;
        col_marg[c] = x.marg_count;
    }
}

static int quantize_pos(const float *pos, const float origin[3], float voxel, const int dims[3], i64 P[3]) {
    for (int a = 0; a < 3; ++a) {
        double q = (((double)pos[a] - (double)origin[a]) / (double)voxel) * 65536.0;
        P[a] = llrint(q);
        if (P[a] < 0 || P[a] >= (i64)dims[a] * ONE_Q16) return -1;
    }
    return 0;
}

static int tree_depths(int n, const int32_t *parent, int32_t *depth) {
    int roots = 0;
    for (int i = 0; i < n; ++i) {
        if (parent[i] == -1) roots++;
        else if (parent[i] < 0 || parent[i] >= n || parent[i] == i) return -1;
    }
    if (n > 0 && roots != 1) return -1;
    for (int i = 0; i < n; ++i) {
        int d = 0, p = i;
        while (parent[p] != -1) {
            p = parent[p];
            if (++d > OR_MAX_DEPTH) return -1; /* cycle or too deep */
        }
        depth[i] = d;
    }
    return 0;
}

/* Returns 0, or a negative code on invalid input. Outputs per node: absolute gain
 * max_k abs[n][k], marginal gain marg[n][psi_n], psi_n = lowest k maximising the mode's
 * gain. Optional: per-(node, yaw) counts and every evaluated node's depth buffer. */
int oracle_eval_tree(const uint8_t *grid, int nx, int ny, int nz, float voxel, const float *origin,
                     int n, const int32_t *parent, const float *pos,
                     float hfov, float vfov, int W, int H, float range_m, int K, float pitch,
                     int mode, const uint8_t *node_mask,
                     int32_t *abs_out, int32_t *marg_out, int32_t *yaw_out,
                     int32_t *cnt_abs, int32_t *cnt_marg, uint32_t *depth_out, int n_threads) {
    if (n < 0 || nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096) return -1;
    if (!(voxel > 0.0f)) return -1;
    if (mode < 0 || mode > 4) return -1;
    if (n == 0) return 0;
    for (size_t i = 0, m = (size_t)nx * ny * nz; i < m; ++i)
        if (grid[i] > OR_OCCUPIED) return -1;
    cam_t cam;
    int rc = cam_build(&cam, hfov, vfov, W, H, K, pitch);
    if (rc) return rc;
    i64 Tq = llrint(((double)range_m / (double)voxel) * 65536.0);
    if (Tq < 1 || Tq > 1024 * ONE_Q16) { cam_free(&cam); return -1; }
    pano_t pano;
    memset(&pano, 0, sizeof(pano));
    if (mode == MODE_PANORAMIC && (rc = pano_build(&pano, hfov, vfov, W, H, K, pitch)) != 0) { cam_free(&cam); return rc; }
    grid_t G = {grid, {nx, ny, nz}};
    int dims[3] = {nx, ny, nz};
    int32_t *depth = malloc((size_t)n * 4);
    i64 (*P)[3] = malloc((size_t)n * sizeof(*P));
    int32_t *yaw = malloc((size_t)n * 4);
    uint32_t **Dn = calloc((size_t)n, sizeof(uint32_t *));
    int32_t *cabs = malloc((size_t)n * K * 4), *cmarg = malloc((size_t)n * K * 4);
    if (!depth || !P || !yaw || !Dn || !cabs || !cmarg) { rc = -2; goto done; }
    if (tree_depths(n, parent, depth)) { rc = -1; goto done; }
    for (int i = 0; i < n; ++i)
        if (quantize_pos(pos + 3 * (size_t)i, origin, voxel, dims, P[i])) { rc = -1; goto done; }
    if (node_mask) /* the evaluated subset must be closed under ancestors */
        for (int i = 0; i < n; ++i)
            if (node_mask[i] && parent[i] >= 0 && !node_mask[parent[i]]) { rc = -1; goto done; }
    int max_d = 0;
    for (int i = 0; i < n; ++i) if (depth[i] > max_d) max_d = depth[i];
    size_t WH = (size_t)W * H;
#ifdef _OPENMP
    omp_set_num_threads(n_threads > 0 ? n_threads : omp_get_num_procs());  /* 0 = every core */
#else
    (void)n_threads;
#endif
    int *lvl = malloc((size_t)n * sizeof(int));
    if (!lvl) { rc = -2; goto done; }
    for (int d = 0; d <= max_d && rc == 0; ++d) {
        int L = 0;
        for (int i = 0; i < n; ++i)
            if (depth[i] == d && (!node_mask || node_mask[i])) lvl[L++] = i;
        if (mode == MODE_PANORAMIC) {
            /* one 360-degree cast per node, per-column counts, then each yaw's window sum */
#pragma omp parallel for schedule(dynamic, 1)
            for (int li = 0; li < L; ++li) {
                int nd = lvl[li];
                i64 anc_P[OR_MAX_DEPTH][3];
                int anc_yaw[OR_MAX_DEPTH];
                uint32_t *anc_D[OR_MAX_DEPTH];
                int na = 0;
                for (int p = parent[nd]; p >= 0; p = parent[p]) {
                    memcpy(anc_P[na], P[p], sizeof(anc_P[na]));
                    anc_yaw[na] = yaw[p];
                    anc_D[na] = Dn[p];
                    na++;
                }
                i64 *ca = malloc((size_t)pano.A * 8), *cm = malloc((size_t)pano.A * 8);
                if (!ca || !cm) { rc = -2; free(ca); free(cm); continue; }
                pano_columns(&pano, &cam, &G, P[nd], Tq, na, (const i64(*)[3])anc_P, anc_yaw, anc_D, ca, cm);
                for (int k = 0; k < K; ++k) {
                    i64 sa = 0, sm = 0;
                    int c0 = pano_window_start(&pano, k);
                    for (int q = 0; q < pano.Wc; ++q) {
                        int c = (c0 + q) % pano.A;
                        sa += ca[c];
                        sm += cm[c];
                    }
                    cabs[(size_t)nd * K + k] = (int32_t)sa;
                    cmarg[(size_t)nd * K + k] = (int32_t)sm;
                }
                free(ca);
                free(cm);
            }
        } else
        /* counts for every (node of the level, yaw) */
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
        for (int li = 0; li < L; ++li) {
            for (int k = 0; k < K; ++k) {
                int nd = lvl[li];
                i64 anc_P[OR_MAX_DEPTH][3];
                int anc_yaw[OR_MAX_DEPTH];
                uint32_t *anc_D[OR_MAX_DEPTH];
                int na = 0;
                if (mode != MODE_ABSOLUTE) {
                    for (int p = parent[nd]; p >= 0; p = parent[p]) { /* parent first */
                        memcpy(anc_P[na], P[p], sizeof(anc_P[na]));
                        anc_yaw[na] = yaw[p];
                        anc_D[na] = Dn[p];
                        na++;
                        if (mode == MODE_SINGLE_PARENT || MUT(9)) break;
                    }
                }
                if (mode == MODE_INTERVAL) {
                    /* Sec. IV-B: per ray, the ancestors' overlap intervals, then the 3D DDA */
                    const size_t cap = (size_t)W + H + 2;
                    ival_ctx y;
                    memset(&y, 0, sizeof(y));
                    y.cam = &cam; y.k = k; y.P = P[nd]; y.Tq = Tq; y.n_anc = na;
                    y.anc_P = (const i64(*)[3])anc_P; y.anc_yaw = anc_yaw; y.anc_D = anc_D;
                    y.seg = malloc((size_t)(na > 0 ? na : 1) * sizeof(seg2d_t));
                    y.seg_ok = malloc((size_t)(na > 0 ? na : 1) * sizeof(int));
                    y.n_por = malloc((size_t)(na > 0 ? na : 1) * sizeof(int));
                    y.por = malloc((size_t)(na > 0 ? na : 1) * cap * sizeof(portion_t));
                    if (!y.seg || !y.seg_ok || !y.n_por || !y.por) {
                        rc = -2;
                    } else {
                        for (int j = 0; j < H; ++j) {
                            for (int i = 0; i < W; ++i) {
                                size_t p = (size_t)j * W + i;
                                i64 dvec[3];
                                cam_dir(&cam, k, p, dvec);
                                y.pi = i;
                                y.pj = j;
                                y.built = 0;
                                ray_end(P[nd], dvec, Tq, y.E);
                                dda(&G, P[nd], dvec, Tq, cam.dzc[p], interval_visit, &y, NULL);
                            }
                        }
                    }
                    free(y.seg); free(y.seg_ok); free(y.n_por); free(y.por);
                    cabs[(size_t)nd * K + k] = (int32_t)y.abs_count;
                    cmarg[(size_t)nd * K + k] = (int32_t)y.marg_count;
                    continue;
                }
                count_ctx x = {&cam, &G, k, 0, 0, P[nd], na, (const i64(*)[3])anc_P, anc_yaw, anc_D, 0, 0};
                for (int j = 0; j < H; ++j) {
                    for (int i = 0; i < W; ++i) {
                        size_t p = (size_t)j * W + i;
                        i64 dvec[3];
                        cam_dir(&cam, k, p, dvec);
                        x.pi = i;
                        x.pj = j;
                        dda(&G, P[nd], dvec, Tq, cam.dzc[p], count_visit, &x, NULL);
                    }
                }
                cabs[(size_t)nd * K + k] = (int32_t)x.abs_count;
                cmarg[(size_t)nd * K + k] = (int32_t)x.marg_count;
            }
        }
        /* yaw selection (Sec. III-B): lowest k with the largest gain of the mode */
        for (int li = 0; li < L; ++li) {
            int nd = lvl[li];
            const int32_t *sel = (mode == MODE_ABSOLUTE) ? cabs + (size_t)nd * K : cmarg + (size_t)nd * K;
            int kb = 0;
            int32_t amax = cabs[(size_t)nd * K];
            for (int k = 1; k < K; ++k) {
                if (MUT(11) ? sel[k] >= sel[kb] : sel[k] > sel[kb]) kb = k;
                if (cabs[(size_t)nd * K + k] > amax) amax = cabs[(size_t)nd * K + k];
            }
            yaw[nd] = kb;
            abs_out[nd] = amax;
            marg_out[nd] = cmarg[(size_t)nd * K + kb];
            yaw_out[nd] = kb;
            Dn[nd] = malloc(WH * 4);
            if (!Dn[nd]) rc = -2;
        }
        if (rc) break;
        /* depth buffer of the selected yaw (Sec. IV-A), kept for the descendants */
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
        for (int li = 0; li < L; ++li) {
            for (int j = 0; j < H; ++j) {
                int nd = lvl[li];
                for (int i = 0; i < W; ++i) {
                    size_t p = (size_t)j * W + i;
                    i64 dvec[3];
                    cam_dir(&cam, yaw[nd], p, dvec);
                    uint32_t Dv = 0;
                    dda(&G, P[nd], dvec, Tq, cam.dzc[p], NULL, NULL, &Dv);
                    Dn[nd][p] = Dv;
                }
            }
        }
    }
    free(lvl);
    if (rc == 0) {
        for (int i = 0; i < n; ++i) {
            if (node_mask && !node_mask[i]) continue;
            if (cnt_abs) memcpy(cnt_abs + (size_t)i * K, cabs + (size_t)i * K, (size_t)K * 4);
            if (cnt_marg) memcpy(cnt_marg + (size_t)i * K, cmarg + (size_t)i * K, (size_t)K * 4);
            if (depth_out) memcpy(depth_out + (size_t)i * WH, Dn[i], WH * 4);
        }
    }
done:
    if (Dn) for (int i = 0; i < n; ++i) free(Dn[i]);
    free(Dn); free(depth); free(P); free(yaw); free(cabs); free(cmarg);
    cam_free(&cam);
    pano_free(&pano);
    return rc;
}

/* ------------------------------------------------------------------------------------
 * Debug and pin entry points
 * ------------------------------------------------------------------------------------ */

/* camera tables as the oracle builds them (for pins against a float pinhole model) */
int oracle_camera_tables(float hfov, float vfov, int W, int H, int K, float pitch,
                         int32_t *body /* H*W*3 */, int32_t *dzc /* H*W */, int32_t *ck, int32_t *sk,
                         int32_t *M /* K*9 */, double *tv4 /* t_h, t_v, cp, sp */) {
    cam_t c;
    int rc = cam_build(&c, hfov, vfov, W, H, K, pitch);
    if (rc) return rc;
    size_t np = (size_t)W * H;
    for (size_t p = 0; p < np; ++p) {
        body[3 * p] = c.bx[p]; body[3 * p + 1] = c.by[p]; body[3 * p + 2] = c.bz[p];
        dzc[p] = c.dzc[p];
    }
    memcpy(ck, c.ck, (size_t)K * 4);
    memcpy(sk, c.sk, (size_t)K * 4);
    memcpy(M, c.M, (size_t)K * 9 * 4);
    tv4[0] = c.t_h; tv4[1] = c.t_v; tv4[2] = c.cp; tv4[3] = c.sp;
    cam_free(&c);
    return 0;
}

/* world ray directions of every (yaw, pixel): K*H*W*3 int64 (Q30) */
int oracle_ray_dirs(float hfov, float vfov, int W, int H, int K, float pitch, int64_t *out) {
    cam_t c;
    int rc = cam_build(&c, hfov, vfov, W, H, K, pitch);
    if (rc) return rc;
    for (int k = 0; k < K; ++k)
        for (size_t p = 0; p < (size_t)W * H; ++p) cam_dir(&c, k, p, out + 3 * ((size_t)k * W * H + p));
    cam_free(&c);
    return 0;
}

typedef struct {
    int32_t *out;
    uint8_t *codes;
    float *lam; /* interval-mode sample of each visited voxel (optional) */
    i64 Tq;
    int cap, count;
} trace_ctx;

static int trace_visit(void *vctx, const int32_t v[3], uint8_t code, const i64 te[2], const i64 tx[2]) {
    trace_ctx *t = (trace_ctx *)vctx;
    if (t->count < t->cap) {
        t->out[3 * t->count] = v[0]; t->out[3 * t->count + 1] = v[1]; t->out[3 * t->count + 2] = v[2];
        if (t->codes) t->codes[t->count] = code;
        if (t->lam) t->lam[t->count] = sample_lambda(te, tx, t->Tq);
    }
    t->count++;
    return 0;
}

/* One ray: P (Q16), d (Q30), T (Q16), dzc (Q30). Writes up to cap visited voxels; returns
 * the number visited (may exceed cap), *hit, *D. */
int oracle_trace(const uint8_t *grid, int nx, int ny, int nz, const int64_t *P, const int64_t *d, int64_t Tq,
                 int64_t dzc, int cap, int32_t *vox, uint8_t *codes, int32_t *hit, uint32_t *D, float *lam) {
    grid_t G = {grid, {nx, ny, nz}};
    for (int a = 0; a < 3; ++a)
        if (P[a] < 0 || P[a] >= (i64)G.n[a] * ONE_Q16) return -1;
    if (d[0] == 0 && d[1] == 0 && d[2] == 0) return -1;
    trace_ctx t = {vox, codes, lam, Tq, cap, 0};
    uint32_t Dv = 0;
    *hit = dda(&G, P, d, Tq, dzc, trace_visit, &t, &Dv);
    *D = Dv;
    return t.count;
}

/* Eq. 5 projection of voxel centres (for pins): out = (ok, pu, pv, Zq) per voxel */
int oracle_project(float hfov, float vfov, int W, int H, int K, float pitch, int k, const int64_t *P, int nv,
                   const int32_t *vox, int64_t *out) {
    cam_t c;
    int rc = cam_build(&c, hfov, vfov, W, H, K, pitch);
    if (rc) return rc;
    for (int i = 0; i < nv; ++i) {
        i64 pu = 0, pv = 0, Z = 0;
        int ok = project(&c, k, P, vox + 3 * (size_t)i, &pu, &pv, &Z);
        out[4 * (size_t)i] = ok; out[4 * (size_t)i + 1] = pu; out[4 * (size_t)i + 2] = pv; out[4 * (size_t)i + 3] = Z;
    }
    cam_free(&c);
    return 0;
}

/* the ancestor test of Sec. IV-B for one voxel against one depth buffer (for pins) */
int oracle_observed(float hfov, float vfov, int W, int H, int K, float pitch, int k, const int64_t *P,
                    const uint32_t *D, const int32_t *vox) {
    cam_t c;
    int rc = cam_build(&c, hfov, vfov, W, H, K, pitch);
    if (rc) return rc;
    int r = observed_by(&c, P, k, D, vox);
    cam_free(&c);
    return r;
}

/* The interval construction of one candidate ray against one ancestor (for pins):
 * seg_out[12] = lo, hi, Za, Zb, ua, va, ub, vb, wa, wb, s0, s1; portions (s_in, s_out, obs,
 * pixel i, j) in walk order; for each ray fraction lam[q]: its screen parameter and whether
 * the ancestor observes it (-1: outside the depth range or image). Returns the number of
 * portions (0 = nothing of the ray in the ancestor's view), or < 0 on bad input. */
int oracle_ray_intervals(float hfov, float vfov, int W, int H, int K, float pitch, int ka, const int64_t *Pa,
                         const uint32_t *D, const int64_t *P, const int64_t *d, int64_t Tq, int n_lam,
                         const float *lam, float *seg_out, int cap, float *por_out, int32_t *por_pix,
                         int32_t *lam_obs, float *lam_s) {
    cam_t c;
    int rc = cam_build(&c, hfov, vfov, W, H, K, pitch);
    if (rc) return rc;
    if (ka < 0 || ka >= K || cap < W + H + 2) { cam_free(&c); return -1; }
    i64 E[3];
    ray_end(P, d, Tq, E);
    seg2d_t g;
    memset(&g, 0, sizeof(g));
    int ok = seg_setup(&c, ka, Pa, P, E, Tq, &g);
    float gv[12] = {g.lo, g.hi, g.Za, g.Zb, g.ua, g.va, g.ub, g.vb, g.wa, g.wb, g.s0, g.s1};
    memcpy(seg_out, gv, sizeof(gv));
    int np = 0;
    portion_t *pt = malloc((size_t)cap * sizeof(portion_t));
    if (!pt) { cam_free(&c); return -2; }
    if (ok) np = seg_walk(&g, W, H, D, pt);
    for (int q = 0; q < np; ++q) {
        por_out[3 * q] = pt[q].s_in; por_out[3 * q + 1] = pt[q].s_out; por_out[3 * q + 2] = (float)pt[q].obs;
        por_pix[2 * q] = pt[q].i; por_pix[2 * q + 1] = pt[q].j;
    }
    for (int q = 0; q < n_lam; ++q) {
        float sp = 0.0f;
        int in = ok && seg_param(&g, lam[q], &sp);
        lam_s[q] = sp;
        lam_obs[q] = in ? portions_observe(pt, np, sp) : -1;
    }
    free(pt);
    cam_free(&c);
    return np;
}

/* the interval mode's sample of a voxel: traversal midpoint as a fraction of the range */
float oracle_sample_lambda(int64_t ne, int64_t ade, int64_t nx, int64_t adx, int64_t Tq) {
    const i64 te[2] = {ne, ade}, tx[2] = {nx, adx};
    return sample_lambda(te, tx, Tq);
}

/* panoramic tables (for pins): dims[3] = A, Wc, step; bc[A*2], dirs[A*H*3], rows[A*6],
 * wstart[K] = first column of each yaw's window */
int oracle_pano_tables(float hfov, float vfov, int W, int H, int K, float pitch, int32_t *dims, int32_t *bc,
                       int32_t *dirs, int32_t *rows, int32_t *wstart) {
    pano_t p;
    int rc = pano_build(&p, hfov, vfov, W, H, K, pitch);
    if (rc) return rc;
    dims[0] = p.A; dims[1] = p.Wc; dims[2] = p.step;
    if (bc) memcpy(bc, p.bc, (size_t)p.A * 2 * 4);
    if (dirs) memcpy(dirs, p.dir, (size_t)p.A * H * 3 * 4);
    if (rows) memcpy(rows, p.row, (size_t)p.A * 6 * 4);
    if (wstart) for (int k = 0; k < K; ++k) wstart[k] = pano_window_start(&p, k);
    pano_free(&p);
    return 0;
}

/* owning cell (c, j) of each voxel seen from P, by search over all wedges (-1, -1: none) */
int oracle_pano_cells(float hfov, float vfov, int W, int H, int K, float pitch, const int64_t *P, int nv,
                      const int32_t *vox, int32_t *out) {
    pano_t p;
    int rc = pano_build(&p, hfov, vfov, W, H, K, pitch);
    if (rc) return rc;
    for (int i = 0; i < nv; ++i) {
        int c = -1, j = -1;
        if (!pano_cell(&p, P, vox + 3 * (size_t)i, &c, &j)) c = j = -1;
        out[2 * (size_t)i] = c;
        out[2 * (size_t)i + 1] = j;
    }
    pano_free(&p);
    return 0;
}

/* per-column absolute counts of one node with no ancestors (for pins) */
int oracle_pano_node_columns(const uint8_t *grid, int nx, int ny, int nz, const int64_t *P, float hfov, float vfov,
                             int W, int H, int K, float pitch, int64_t Tq, int64_t *col_abs) {
    pano_t p;
    int rc = pano_build(&p, hfov, vfov, W, H, K, pitch);
    if (rc) return rc;
    cam_t c;
    if ((rc = cam_build(&c, hfov, vfov, W, H, K, pitch)) != 0) { pano_free(&p); return rc; }
    grid_t G = {grid, {nx, ny, nz}};
    i64 *cm = malloc((size_t)p.A * 8);
    if (!cm) { pano_free(&p); cam_free(&c); return -2; }
    pano_columns(&p, &c, &G, P, Tq, 0, NULL, NULL, NULL, col_abs, cm);
    free(cm);
    pano_free(&p);
    cam_free(&c);
    return 0;
}

int oracle_quantize(const float *pos, int n, const float *origin, float voxel, int nx, int ny, int nz, int64_t *P) {
    int dims[3] = {nx, ny, nz};
    for (int i = 0; i < n; ++i)
        if (quantize_pos(pos + 3 * (size_t)i, origin, voxel, dims, P + 3 * (size_t)i)) return -1;
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Exact part (Eq. 1 sets, Eq. 2 by reference counts)
 * ------------------------------------------------------------------------------------ */
typedef struct {
    const cam_t *cam;
    int k;
    i64 pi, pj;
    const i64 *P;
    int nx, ny;
    int32_t *ids;
    i64 count, cap;
} set_ctx;

static int set_visit(void *vctx, const int32_t v[3], uint8_t code, const i64 te[2], const i64 tx[2]) {
    (void)te;
    (void)tx;
    set_ctx *s = (set_ctx *)vctx;
    if (code != OR_UNKNOWN) return 0;
    if (!owned(s->cam, s->k, s->P, v, s->pi, s->pj)) return 0;
    if (s->ids && s->count < s->cap) s->ids[s->count] = (int32_t)(((i64)v[2] * s->ny + v[1]) * s->nx + v[0]);
    s->count++;
    return 0;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* I(n, yaw[n]) for every node: linear voxel ids (x fastest), sorted. Two calls: with
 * ids == NULL fills offsets[0..n] (sizes); then with ids of length offsets[n]. */
int oracle_visible_sets(const uint8_t *grid, int nx, int ny, int nz, float voxel, const float *origin,
                        int n, const float *pos, const int32_t *yaws,
                        float hfov, float vfov, int W, int H, float range_m, int K, float pitch,
                        const uint8_t *node_mask, int64_t *offsets, int32_t *ids, int n_threads) {
    cam_t cam;
    int rc = cam_build(&cam, hfov, vfov, W, H, K, pitch);
    if (rc) return rc;
    i64 Tq = llrint(((double)range_m / (double)voxel) * 65536.0);
    grid_t G = {grid, {nx, ny, nz}};
    int dims[3] = {nx, ny, nz};
    i64 (*P)[3] = malloc((size_t)(n > 0 ? n : 1) * sizeof(*P));
    for (int i = 0; i < n; ++i)
        if (quantize_pos(pos + 3 * (size_t)i, origin, voxel, dims, P[i])) { free(P); cam_free(&cam); return -1; }
#ifdef _OPENMP
    omp_set_num_threads(n_threads > 0 ? n_threads : omp_get_num_procs());  /* 0 = every core */
#else
    (void)n_threads;
#endif
    if (!ids) offsets[0] = 0;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int nd = 0; nd < n; ++nd) {
        if (node_mask && !node_mask[nd]) { if (!ids) offsets[nd + 1] = 0; continue; }
        if (yaws[nd] < 0 || yaws[nd] >= K) { bad = 1; continue; }
        set_ctx s = {&cam, yaws[nd], 0, 0, P[nd], nx, ny, NULL, 0, 0};
        if (ids) { s.ids = ids + offsets[nd]; s.cap = offsets[nd + 1] - offsets[nd]; }
        for (int j = 0; j < H; ++j)
            for (int i = 0; i < W; ++i) {
                size_t p = (size_t)j * W + i;
                i64 dvec[3];
                cam_dir(&cam, yaws[nd], p, dvec);
                s.pi = i; s.pj = j;
                dda(&G, P[nd], dvec, Tq, cam.dzc[p], set_visit, &s, NULL);
            }
        if (!ids) offsets[nd + 1] = s.count;
        else qsort(s.ids, (size_t)s.count, 4, cmp_i32);
    }
    if (!ids) for (int i = 0; i < n; ++i) offsets[i + 1] += offsets[i];
    free(P);
    cam_free(&cam);
    return bad ? -1 : 0;
}

/* The exact-yaw variant (Eq. 2 with the yaw chosen by the exact gain itself, Sec. III-B's
 * argmax over the yaw set): depth-first over the tree with a dense per-voxel reference count of
 * the sets on the current root path (as route 2); entering node n, every yaw's visible set
 * I(n, k) is built (the same owner-visible sets as Eq. 1), E_k = the number of its voxels whose
 * count is zero, psi = the lowest k maximising E_k, and I(n, psi) joins the path. Outputs psi and
 * E(n) = E_psi per node (nodes outside node_mask: -1). */
int oracle_exact_yaw(const uint8_t *grid, int nx, int ny, int nz, float voxel, const float *origin,
                     int n, const int32_t *parent, const float *pos,
                     float hfov, float vfov, int W, int H, float range_m, int K, float pitch,
                     const uint8_t *node_mask, int32_t *yaw_out, int32_t *E_out, int n_threads) {
    if (n == 0) return 0;
    cam_t cam;
    int rc = cam_build(&cam, hfov, vfov, W, H, K, pitch);
    if (rc) return rc;
    i64 Tq = llrint(((double)range_m / (double)voxel) * 65536.0);
    grid_t G = {grid, {nx, ny, nz}};
    int dims[3] = {nx, ny, nz};
    size_t nvox = (size_t)nx * ny * nz;
    i64 (*P)[3] = malloc((size_t)n * sizeof(*P));
    uint16_t *cnt = calloc(nvox, sizeof(uint16_t));
    int *head = malloc((size_t)n * sizeof(int)), *next = malloc((size_t)n * sizeof(int));
    int *stack = malloc((size_t)n * 2 * sizeof(int));
    int32_t **chosen = calloc((size_t)n, sizeof(int32_t *));
    i64 *chosen_n = calloc((size_t)n, sizeof(i64));
    int32_t **sets = calloc((size_t)K, sizeof(int32_t *));
    i64 *set_n = calloc((size_t)K, sizeof(i64)), *set_cap = calloc((size_t)K, sizeof(i64));
    if (!P || !cnt || !head || !next || !stack || !chosen || !chosen_n || !sets || !set_n || !set_cap) { rc = -2; goto done; }
    for (int i = 0; i < n; ++i)
        if (quantize_pos(pos + 3 * (size_t)i, origin, voxel, dims, P[i])) { rc = -1; goto done; }
#ifdef _OPENMP
    omp_set_num_threads(n_threads > 0 ? n_threads : omp_get_num_procs());  /* 0 = every core */
#else
    (void)n_threads;
#endif
    int root = -1;
    for (int i = 0; i < n; ++i) { head[i] = -1; yaw_out[i] = -1; E_out[i] = -1; }
    for (int i = n - 1; i >= 0; --i) {
        if (parent[i] < 0) root = i;
        else { next[i] = head[parent[i]]; head[parent[i]] = i; }
    }
    if (root < 0) { rc = -1; goto done; }
    int sp = 0;
    stack[sp++] = root; /* entries: node (enter) or ~node (leave) */
    while (sp > 0 && rc == 0) {
        int e = stack[--sp];
        if (e >= 0) {
            int nd = e;
            if (node_mask && !node_mask[nd]) continue;
            /* every yaw's visible set, in parallel over the yaws */
#pragma omp parallel for schedule(dynamic, 1)
            for (int k = 0; k < K; ++k) {
                set_ctx sc = {&cam, k, 0, 0, P[nd], nx, ny, NULL, 0, 0};
                for (int pass = 0; pass < 2; ++pass) { /* count, then fill */
                    sc.count = 0;
                    if (pass == 1) {
                        if (set_cap[k] < sc.cap) {
                            free(sets[k]);
                            sets[k] = malloc((size_t)(sc.cap > 0 ? sc.cap : 1) * 4);
                            set_cap[k] = sets[k] ? sc.cap : 0;
                        }
                        sc.ids = sets[k];
                    }
                    for (int j = 0; j < H; ++j)
                        for (int i = 0; i < W; ++i) {
                            size_t p = (size_t)j * W + i;
                            i64 dvec[3];
                            cam_dir(&cam, k, p, dvec);
                            sc.pi = i; sc.pj = j;
                            dda(&G, P[nd], dvec, Tq, cam.dzc[p], set_visit, &sc, NULL);
                        }
                    if (pass == 0) sc.cap = sc.count;
                }
                set_n[k] = sc.count;
            }
            int kb = 0;
            i64 eb = -1;
            for (int k = 0; k < K; ++k) {
                if (!sets[k] && set_n[k] > 0) { rc = -2; break; }
                i64 z = 0;
                for (i64 q = 0; q < set_n[k]; ++q) if (cnt[sets[k][q]] == 0) z++;
                if (MUT(20) ? z >= eb : z > eb) { eb = z; kb = k; }
            }
            if (rc) break;
            yaw_out[nd] = kb;
            E_out[nd] = (int32_t)eb;
            chosen[nd] = malloc((size_t)(set_n[kb] > 0 ? set_n[kb] : 1) * 4);
            if (!chosen[nd]) { rc = -2; break; }
            memcpy(chosen[nd], sets[kb], (size_t)set_n[kb] * 4);
            chosen_n[nd] = set_n[kb];
            for (i64 q = 0; q < chosen_n[nd]; ++q) cnt[chosen[nd][q]]++;
            stack[sp++] = ~nd;
            for (int c = head[nd]; c >= 0; c = next[c]) stack[sp++] = c;
        } else {
            int nd = ~e;
            for (i64 q = 0; q < chosen_n[nd]; ++q) cnt[chosen[nd][q]]--;
            free(chosen[nd]);
            chosen[nd] = NULL;
        }
    }
done:
    if (chosen) for (int i = 0; i < n; ++i) free(chosen[i]);
    if (sets) for (int k = 0; k < K; ++k) free(sets[k]);
    free(chosen); free(chosen_n); free(sets); free(set_n); free(set_cap);
    free(P); free(cnt); free(head); free(next); free(stack);
    cam_free(&cam);
    return rc;
}

/* Route 2 of the exact marginal gain (Eq. 2): depth-first over the tree with a dense
 * per-voxel reference count of the sets on the current root path. E(n) = number of
 * voxels of I(n) whose count is zero when n is entered. */
int oracle_exact_dfs(int n, const int32_t *parent, const int64_t *offsets, const int32_t *ids, int64_t nvox,
                     const uint8_t *node_mask, int32_t *E) {
    if (n == 0) return 0;
    uint16_t *cnt = calloc((size_t)nvox, sizeof(uint16_t));
    int *head = malloc((size_t)n * sizeof(int)), *next = malloc((size_t)n * sizeof(int));
    int *stack = malloc((size_t)n * 2 * sizeof(int));
    if (!cnt || !head || !next || !stack) { free(cnt); free(head); free(next); free(stack); return -2; }
    int root = -1;
    for (int i = 0; i < n; ++i) head[i] = -1;
    for (int i = n - 1; i >= 0; --i) {
        if (parent[i] < 0) root = i;
        else { next[i] = head[parent[i]]; head[parent[i]] = i; }
    }
    int sp = 0;
    stack[sp++] = root; /* entries: node (enter) or ~node (leave) */
    while (sp > 0) {
        int e = stack[--sp];
        if (e >= 0) {
            int nd = e;
            if (node_mask && !node_mask[nd]) continue;
            int32_t z = 0;
            for (i64 q = offsets[nd]; q < offsets[nd + 1]; ++q) if (cnt[ids[q]] == 0 || (MUT(13) && cnt[ids[q]] == 1)) z++;
            E[nd] = z;
            for (i64 q = offsets[nd]; q < offsets[nd + 1]; ++q) cnt[ids[q]]++;
            stack[sp++] = ~nd;
            for (int c = head[nd]; c >= 0; c = next[c]) stack[sp++] = c;
        } else {
            int nd = ~e;
            for (i64 q = offsets[nd]; q < offsets[nd + 1]; ++q) cnt[ids[q]]--;
        }
    }
    free(cnt); free(head); free(next); free(stack);
    return 0;
}
