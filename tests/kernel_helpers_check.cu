// Host checks of the owned-voxel count's integer and float helpers (csrc/voxcount.cuh, compiled for
// the host) against plain references written here:
//   cast   - cast_hit, with and without the brick and super-brick summaries, against a plain DDA
//            (Sec. IV-B: smallest crossing first, ties x, y, z; stop on an occupied voxel, at the
//            grid's edge or at the range);
//   visit  - visit_index against the voxels that plain DDA visits on an all-free grid;
//   surely - visit_surely (a sufficient condition) never claims a voxel that visit_index rejects;
//   pixel  - pixel_fast never disagrees with the exact integer pixel of Eq. 5 when it decides, and
//            its depth bound holds.
// Usage: kernel_helpers_check <seed> <scale>; prints one line of counts, exits 1 on any mismatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <tuple>
#include <vector>

#include "voxcount.cuh"

using namespace mig::dev;
typedef long long i64;

static i64 floor_div(i64 a, i64 b) {
    i64 q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

// Plain DDA: the visited voxels in order and the index of the first occupied one (-1 if none).
static int plain_dda(const std::vector<uint8_t> &g, const int N[3], const i64 P[3], const i64 d[3], i64 Tq,
                     std::vector<std::tuple<int, int, int>> *vis) {
    int v[3], step[3];
    i64 nn[3], ad[3];
    for (int a = 0; a < 3; ++a) {
        v[a] = (int)floor_div(P[a], 65536);
        if (d[a] > 0) { step[a] = 1; ad[a] = d[a]; nn[a] = ((i64)v[a] + 1) * 65536 - P[a]; }
        else if (d[a] < 0) { step[a] = -1; ad[a] = -d[a]; nn[a] = P[a] - (i64)v[a] * 65536; }
        else { step[a] = 0; ad[a] = 0; nn[a] = 65536; }
    }
    for (int m = 0;; ++m) {
        if (vis) vis->emplace_back(v[0], v[1], v[2]);
        if (g[((size_t)v[2] * N[1] + v[1]) * N[0] + v[0]] == 2) return m;
        int best = -1;
        for (int a = 0; a < 3; ++a) {
            if (ad[a] == 0) continue;
            if (best < 0 || nn[a] * ad[best] < nn[best] * ad[a]) best = a;
        }
        if (nn[best] * (i64(1) << 30) >= Tq * ad[best]) return -1;
        v[best] += step[best];
        if (v[best] < 0 || v[best] >= N[best]) return -1;
        nn[best] += 65536;
    }
}

static void random_dir(std::mt19937_64 &rng, i64 d[3]) {
    double dd[3];
    double nr = 0;
    do {
        for (int a = 0; a < 3; ++a) dd[a] = ((rng() % 2000001) / 1000000.0) - 1.0;
        const int m = rng() % 6;
        if (m == 0) dd[rng() % 3] = 0;
        if (m == 1) { dd[0] = dd[1] = 0.5; dd[2] = (rng() % 2) ? 0.5 : 0.0; }
        if (m == 2) { dd[0] = (rng() & 1) ? 1 : -1; dd[1] = 0; dd[2] = 0; }
        nr = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
    } while (nr < 1e-9);
    for (int a = 0; a < 3; ++a) d[a] = llrint(dd[a] / nr * 1073741824.0);
    if (rng() % 4 == 0)
        for (int a = 0; a < 3; ++a) d[a] = (d[a] / 1024) * 1024;  // exact ties
}

int main(int argc, char **argv) {
    std::mt19937_64 rng(argc > 1 ? atoi(argv[1]) : 1);
    const int scale = argc > 2 ? atoi(argv[2]) : 1;
    long long cast_rays = 0, cast_bad = 0, visit_checks = 0, visit_bad = 0;
    long long surely_tested = 0, surely_visits = 0, surely_yes = 0, surely_bad = 0;
    long long pix_n = 0, pix_dec = 0, pix_und = 0, pix_bad = 0;

    // ---- cast and visit
    for (int trial = 0; trial < 40 * scale; ++trial) {
        int N[3] = {int(rng() % 150) + 1, int(rng() % 150) + 1, int(rng() % 90) + 1};
        if (trial % 10 == 0) N[0] = 1 + rng() % 5;
        std::vector<uint8_t> g((size_t)N[0] * N[1] * N[2]);
        const double po = (trial % 4 == 0) ? 0.00002 : (trial % 4 == 1 ? 0.0002 : (trial % 4 == 2 ? 0.002 : 0.02));
        for (auto &c : g) {
            const double u = (rng() % 1000000) / 1000000.0;
            c = u < po ? 2 : (u < 0.6 ? 1 : 0);
        }
        for (int b = 0; b < (int)(rng() % 4); ++b) {  // blobs of occupied voxels
            const int cx = rng() % N[0], cy = rng() % N[1], cz = rng() % N[2], r = 1 + rng() % 6;
            for (int z = std::max(0, cz - r); z < std::min(N[2], cz + r); ++z)
                for (int y = std::max(0, cy - r); y < std::min(N[1], cy + r); ++y)
                    for (int x = std::max(0, cx - r); x < std::min(N[0], cx + r); ++x) g[((size_t)z * N[1] + y) * N[0] + x] = 2;
        }
        const int nbx = (N[0] + 7) / 8, nby = (N[1] + 7) / 8, nbz = (N[2] + 7) / 8;
        const int nsx = (N[0] + 31) / 32, nsy = (N[1] + 31) / 32, nsz = (N[2] + 31) / 32;
        std::vector<uint8_t> bocc((size_t)nbx * nby * nbz, 0), sbocc((size_t)nsx * nsy * nsz, 0);
        for (int z = 0; z < N[2]; ++z)
            for (int y = 0; y < N[1]; ++y)
                for (int x = 0; x < N[0]; ++x)
                    if (g[((size_t)z * N[1] + y) * N[0] + x] == 2) {
                        bocc[((size_t)(z >> 3) * nby + (y >> 3)) * nbx + (x >> 3)] = 1;
                        sbocc[((size_t)(z >> 5) * nsy + (y >> 5)) * nsx + (x >> 5)] = 1;
                    }
        for (int r = 0; r < 1500; ++r) {
            i64 P[3], d[3];
            for (int a = 0; a < 3; ++a) {
                const int mode = rng() % 5;
                if (mode == 0) P[a] = (i64)(rng() % N[a]) * 65536;
                else if (mode == 1) P[a] = (i64)(rng() % N[a]) * 65536 + 32768;
                else if (mode == 2) P[a] = (i64)(((rng() % ((N[a] + 31) / 32)) * 32) % N[a]) * 65536;
                else P[a] = (i64)(rng() % ((i64)N[a] * 65536));
            }
            random_dir(rng, d);
            const i64 Tq = (i64)(rng() % (200 * 65536)) + 1;
            const int hit = plain_dda(g, N, P, d, Tq, nullptr);
            const uint32_t want = hit < 0 ? kNoHit : (uint32_t)hit;
            uint32_t f = 0, c = 0;
            const uint32_t m1 = cast_hit<false>(g.data(), bocc.data(), sbocc.data(), N[0], N[1], N[2], (int)P[0], (int)P[1],
                                                (int)P[2], (int)d[0], (int)d[1], (int)d[2], Tq, f, c);
            const uint32_t m2 = cast_hit<false>(g.data(), bocc.data(), nullptr, N[0], N[1], N[2], (int)P[0], (int)P[1],
                                                (int)P[2], (int)d[0], (int)d[1], (int)d[2], Tq, f, c);
            const uint32_t m3 = cast_hit<false>(g.data(), nullptr, nullptr, N[0], N[1], N[2], (int)P[0], (int)P[1], (int)P[2],
                                                (int)d[0], (int)d[1], (int)d[2], Tq, f, c);
            ++cast_rays;
            if (m1 != want || m2 != want || m3 != want) {
                if (cast_bad < 5) printf("cast mismatch: plain %u got %u %u %u\n", want, m1, m2, m3);
                ++cast_bad;
            }
            if (r % 50 != 0 || N[0] * N[1] * N[2] > 200000) continue;
            // visit_index and visit_surely against the free-grid walk
            std::vector<uint8_t> free_g(g.size(), 1);
            std::vector<std::tuple<int, int, int>> vis;
            plain_dda(free_g, N, P, d, Tq, &vis);
            std::map<std::tuple<int, int, int>, int> idx;
            for (size_t i = 0; i < vis.size(); ++i) idx[vis[i]] = (int)i;
            const float Pxf = (float)P[0] * (1.0f / 65536.0f) - 0.5f, Pyf = (float)P[1] * (1.0f / 65536.0f) - 0.5f,
                        Pzf = (float)P[2] * (1.0f / 65536.0f) - 0.5f;
            for (int z = 0; z < N[2]; ++z)
                for (int y = 0; y < N[1]; ++y)
                    for (int x = 0; x < N[0]; ++x) {
                        const int want_i = idx.count({x, y, z}) ? idx[{x, y, z}] : -1;
                        const int got = visit_index((int)P[0], (int)P[1], (int)P[2], (int)d[0], (int)d[1], (int)d[2], x, y, z, Tq);
                        ++visit_checks;
                        if (want_i != got) {
                            if (visit_bad < 5) printf("visit mismatch at %d %d %d: plain %d got %d\n", x, y, z, want_i, got);
                            ++visit_bad;
                        }
                        const bool su = visit_surely((float)x - Pxf, (float)y - Pyf, (float)z - Pzf, (int)d[0], (int)d[1],
                                                     (int)d[2], (float)Tq * (1.0f / 65536.0f));
                        ++surely_tested;
                        surely_visits += want_i >= 0;
                        surely_yes += su;
                        if (su && want_i < 0) {
                            if (surely_bad < 5) printf("visit_surely claims an unvisited voxel %d %d %d\n", x, y, z);
                            ++surely_bad;
                        }
                    }
        }
    }

    // ---- pixel_fast against the exact pixel (Eq. 5) and depth
    for (int trial = 0; trial < 300 * scale; ++trial) {
        int W = 1 + rng() % 640, H = 1 + rng() % 480;
        if (trial % 7 == 0) { W = 1 + rng() % 4; H = 1 + rng() % 4; }
        if (trial % 11 == 0) { W = 2048; H = 2048; }
        const double hf = 5 + (rng() % 1700) / 10.0, vf = 5 + (rng() % 1700) / 10.0;
        const double pitch = (rng() % 1801) / 10.0 - 90.0;
        const int K = 1 + rng() % 64, k = rng() % K;
        const double t_h = tan(hf * 0.5 * M_PI / 180), t_v = tan(vf * 0.5 * M_PI / 180);
        const double th = pitch * M_PI / 180, cp = cos(th), sp = sin(th);
        const double fx = W * 0.5 / t_h, fy = H * 0.5 / t_v, cxp = W * 0.5, cyp = H * 0.5;
        if (fx * 65536.0 * 2 >= 2147483647.0 || fy * 65536.0 * 2 >= 2147483647.0) continue;
        const double ang = 2 * M_PI * k / K, cs = cos(ang), sn = sin(ang);
        const double exv[3] = {sn, -cs, 0}, eyv[3] = {-(sp * cs), -(sp * sn), -cp}, ezv[3] = {cp * cs, cp * sn, -sp};
        int mu[3], mv[3], mz[3];
        for (int a = 0; a < 3; ++a) {
            mu[a] = (int)llrint((fx * exv[a] + cxp * ezv[a]) * 65536.0);
            mv[a] = (int)llrint((fy * eyv[a] + cyp * ezv[a]) * 65536.0);
            mz[a] = (int)llrint(ezv[a] * 65536.0);
        }
        float w[9];
        for (int a = 0; a < 3; ++a) {
            w[a] = (float)mu[a] * (1.0f / 65536.0f);
            w[3 + a] = (float)mv[a] * (1.0f / 65536.0f);
            w[6 + a] = (float)mz[a] * (1.0f / 65536.0f);
        }
        const int R = (trial % 3 == 0) ? 1 + rng() % 200 : 1 + rng() % 1030;
        int P[3];
        for (int a = 0; a < 3; ++a) P[a] = (int)(rng() % (4096ll * 65536 - 1));
        for (int s = 0; s < 4000; ++s) {
            int v[3];
            for (int a = 0; a < 3; ++a) {
                const int v0 = P[a] >> 16;
                v[a] = (s % 5 == 0) ? v0 + (int)(rng() % 7) - 3 : v0 + (int)(rng() % (2 * R + 1)) - R;
            }
            i64 r[3];
            for (int a = 0; a < 3; ++a) r[a] = ((i64)v[a] << 16) + 32768 - P[a];
            const i64 Z = (i64)mz[0] * r[0] + (i64)mz[1] * r[1] + (i64)mz[2] * r[2];
            const i64 U = (i64)mu[0] * r[0] + (i64)mu[1] * r[1] + (i64)mu[2] * r[2];
            const i64 V = (i64)mv[0] * r[0] + (i64)mv[1] * r[1] + (i64)mv[2] * r[2];
            bool in = false;
            i64 qu = 0, qv = 0;
            if (Z > 0) {
                qu = floor_div(U, Z);
                qv = floor_div(V, Z);
                in = qu >= 0 && qu < W && qv >= 0 && qv < H;
            }
            const float ex = (float)(int)r[0] * (1.0f / 65536.0f), ey = (float)(int)r[1] * (1.0f / 65536.0f);
            const float ez = (float)(int)r[2] * (1.0f / 65536.0f);
            const float rinf = fmaxf(fabsf(ex), fmaxf(fabsf(ey), fabsf(ez)));
            int pu = -7, pv = -7;
            float zf = 0, e_z = 0;
            const int dcs = pixel_fast(w, ex, ey, ez, rinf, W, H, pu, pv, zf, e_z);
            ++pix_n;
            if (dcs < 0) { ++pix_und; continue; }
            ++pix_dec;
            const bool bad = (dcs == 1 && (!in || pu != qu || pv != qv)) || (dcs == 0 && in) ||
                             (dcs == 1 && fabs((double)Z / 4294967296.0 - (double)zf) > (double)e_z);
            if (bad) {
                if (pix_bad < 5) printf("pixel_fast disagrees: W %d H %d decision %d exact %d (%lld, %lld)\n", W, H, dcs, in, qu, qv);
                ++pix_bad;
            }
        }
    }
    printf("cast_rays %lld cast_bad %lld visit_checks %lld visit_bad %lld surely_tested %lld surely_visits %lld "
           "surely_yes %lld surely_bad %lld pixel %lld decided %lld undecided %lld pixel_bad %lld\n",
           cast_rays, cast_bad, visit_checks, visit_bad, surely_tested, surely_visits, surely_yes, surely_bad, pix_n,
           pix_dec, pix_und, pix_bad);
    return (cast_bad || visit_bad || surely_bad || pix_bad) ? 1 : 0;
}
