// Camera tables and sensor checks (host, IEEE double, compiled without FP contraction).
//
// Pinhole model of Eq. 5 with the principal point at the image centre, focal lengths from the
// field of view and rays through pixel centres. Camera axes x right, y down, z forward; body
// forward = world +x at yaw 0; pitch positive = nose down; yaw bin k at 2 pi k / K about +z.
// Every value that decides a result is quantised here once (rays Q30, projection rows Q16);
// all later steps run in integers on the device.
#include <algorithm>
#include <cmath>

#include "mig_impl.h"

namespace mig {

static int32_t q30(double x) { return (int32_t)std::llrint(x * 1073741824.0); }
static int32_t q16(double x) { return (int32_t)std::llrint(x * 65536.0); }

int64_t range_q16(float range_m, float voxel) {
    return (int64_t)std::llrint(((double)range_m / (double)voxel) * 65536.0);
}

mig_status sensor_check(const mig_sensor &s, float voxel) {
    if (s.width < 1 || s.height < 1 || s.width > MIG_MAX_IMAGE || s.height > MIG_MAX_IMAGE)
        return fail(MIG_EINVAL, "sensor: width/height outside [1, 2048]");
    if (s.yaw_bins < 1 || s.yaw_bins > MIG_MAX_YAW_BINS) return fail(MIG_EINVAL, "sensor: yaw_bins outside [1, 1024]");
    if (!(s.hfov_deg > 0.f && s.hfov_deg < 180.f && s.vfov_deg > 0.f && s.vfov_deg < 180.f))
        return fail(MIG_EINVAL, "sensor: field of view outside (0, 180) degrees");
    if (!(s.pitch_deg >= -90.f && s.pitch_deg <= 90.f)) return fail(MIG_EINVAL, "sensor: pitch outside [-90, 90]");
    if (!(voxel > 0.f)) return fail(MIG_EINVAL, "voxel size must be positive");
    if (!(s.range_m > 0.f)) return fail(MIG_EINVAL, "sensor: range must be positive");
    int64_t tq = range_q16(s.range_m, voxel);
    if (tq < 1 || tq > (int64_t)MIG_MAX_RANGE_VOXELS * kOneQ16)
        return fail(MIG_EINVAL, "sensor: range / voxel_size outside (0, 1024] voxels");
    return MIG_OK;
}

mig_status camera_build(const mig_sensor &s, Camera &c) {
    c.s = s;
    c.W = s.width;
    c.H = s.height;
    c.K = s.yaw_bins;
    const double t_h = std::tan(((double)s.hfov_deg * 0.5) * (M_PI / 180.0));
    const double t_v = std::tan(((double)s.vfov_deg * 0.5) * (M_PI / 180.0));
    const double th = (double)s.pitch_deg * (M_PI / 180.0);
    const double cp = std::cos(th), sp = std::sin(th);
    const int W = c.W, H = c.H, K = c.K;
    c.body.assign((size_t)W * H * 4, 0);
    for (int j = 0; j < H; ++j) {
        for (int i = 0; i < W; ++i) {
            // tangent-plane coordinates of the pixel centre, (i + 1/2 - c_x) / f_x
            const double a = ((double)(2 * i + 1 - W) / (double)W) * t_h;
            const double b = ((double)(2 * j + 1 - H) / (double)H) * t_v;
            const double nrm = std::sqrt((a * a + b * b) + 1.0);
            const double cx = a / nrm, cy = b / nrm, cz = 1.0 / nrm;
            int32_t *o = &c.body[((size_t)j * W + i) * 4];
            o[0] = q30(cz * cp - cy * sp);     // body forward
            o[1] = q30(-cx);                   // body left
            o[2] = q30(-(cy * cp + cz * sp));  // body up
            o[3] = q30(cz);                    // camera z of the unit ray
        }
    }
    // Elevation band and azimuth half-width of the frustum (culling bounds for the per-node voxel
    // pass): without a vertical direction inside the frustum, both extremes lie on the image
    // border, sampled densely here and widened by half a degree.
    {
        auto body_dir = [&](double a, double b, double out[3]) {
            const double nrm = std::sqrt((a * a + b * b) + 1.0);
            const double x = a / nrm, y = b / nrm, z = 1.0 / nrm;
            out[0] = z * cp - y * sp;
            out[1] = -x;
            out[2] = -(y * cp + z * sp);
        };
        double elo = 1e9, ehi = -1e9, az = 0.0;
        const int S = 4096;
        for (int e = 0; e < 4; ++e) {
            for (int t = 0; t <= S; ++t) {
                const double f = (double)t / S * 2.0 - 1.0;
                const double a = (e < 2 ? f : (e == 2 ? -1.0 : 1.0)) * t_h;
                const double b = (e < 2 ? (e == 0 ? -1.0 : 1.0) : f) * t_v;
                double d[3];
                body_dir(a, b, d);
                const double el = std::atan2(d[2], std::hypot(d[0], d[1]));
                elo = std::min(elo, el);
                ehi = std::max(ehi, el);
                az = std::max(az, std::fabs(std::atan2(d[1], d[0])));
            }
        }
        // the vertical directions in camera coordinates: up (0, -cp, -sp), down (0, cp, sp)
        const bool up_in = -sp > 0.0 && std::fabs(cp / sp) <= t_v;
        const bool down_in = sp > 0.0 && std::fabs(cp / sp) <= t_v;
        const double margin = 0.5 * M_PI / 180.0;
        elo -= margin;
        ehi += margin;
        c.band_thi = (up_in || ehi >= 89.5 * M_PI / 180.0) ? 1e30f : (float)std::tan(ehi);
        c.band_tlo = (down_in || elo <= -89.5 * M_PI / 180.0) ? -1e30f : (float)std::tan(elo);
        c.az_half = (up_in || down_in || az + margin >= M_PI) ? 3.2f : (float)(az + margin);
    }
    const double fx = ((double)W * 0.5) / t_h, fy = ((double)H * 0.5) / t_v;
    const double cxp = (double)W * 0.5, cyp = (double)H * 0.5;
    c.yaw.assign((size_t)K * kYawRec, 0);
    for (int k = 0; k < K; ++k) {
        const double ang = ((2.0 * M_PI) * (double)k) / (double)K;
        const double cs = std::cos(ang), sn = std::sin(ang);
        int32_t *o = &c.yaw[(size_t)k * kYawRec];
        o[0] = q30(cs);
        o[1] = q30(sn);
        const double ex[3] = {sn, -cs, 0.0};
        const double ey[3] = {-(sp * cs), -(sp * sn), -cp};
        const double ez[3] = {cp * cs, cp * sn, -sp};
        for (int a = 0; a < 3; ++a) {
            const double mu = fx * ex[a] + cxp * ez[a];
            const double mv = fy * ey[a] + cyp * ez[a];
            if (std::fabs(mu) * 65536.0 >= 2147483647.0 || std::fabs(mv) * 65536.0 >= 2147483647.0)
                return fail(MIG_EINVAL, "sensor: focal length too large for the Q16 projection rows");
            o[2 + a] = q16(mu);
            o[5 + a] = q16(mv);
            o[8 + a] = q16(ez[a]);
        }
    }
    return MIG_OK;
}

// Panoramic tables: one 360-degree cast per node. The horizon is cut into A = K * step azimuth
// wedges, step = ceil(W 360 / (hfov K)), so that a yaw step is a whole number of columns and a
// column is no wider than a pinhole pixel at the image centre; yaw k's window is the
// Wc = round(A hfov / 360) columns centred on its azimuth. Column c is a one-pixel-wide strip
// camera looking along the wedge's centre azimuth with the pinhole's rows.
mig_status pano_build(Camera &c) {
    const mig_sensor &s = c.s;
    if (s.pitch_deg != 0.0f) return fail(MIG_EINVAL, "panoramic mode: the camera must be level (pitch 0)");
    int step = (int)std::ceil(((double)s.width * 360.0) / ((double)s.hfov_deg * (double)s.yaw_bins));
    if (step < 1) step = 1;
    const int A = step * s.yaw_bins, H = s.height;
    if (A > MIG_MAX_PANO_COLUMNS) return fail(MIG_EINVAL, "panoramic mode: too many azimuth columns");
    int Wc = (int)std::llrint(((double)A * (double)s.hfov_deg) / 360.0);
    if (Wc < 1) Wc = 1;
    const double t_v = std::tan(((double)s.vfov_deg * 0.5) * (M_PI / 180.0));
    const double fy = ((double)H * 0.5) / t_v, cyp = (double)H * 0.5;
    c.pano_bc.assign((size_t)A * 2, 0);
    c.pano_dir.assign((size_t)A * H * 4, 0);
    c.pano_row.assign((size_t)A * 8, 0);
    for (int col = 0; col < A; ++col) {
        const double ang = ((2.0 * M_PI) * (double)col) / (double)A;
        c.pano_bc[2 * (size_t)col] = q30(std::cos(ang));
        c.pano_bc[2 * (size_t)col + 1] = q30(std::sin(ang));
        const double th = ((2.0 * M_PI) * ((double)col + 0.5)) / (double)A;
        const double cs = std::cos(th), sn = std::sin(th);
        const double mv[3] = {cyp * cs, cyp * sn, -fy};
        for (int a = 0; a < 3; ++a)
            if (std::fabs(mv[a]) * 65536.0 >= 2147483647.0)
                return fail(MIG_EINVAL, "sensor: focal length too large for the Q16 projection rows");
        int32_t *r = &c.pano_row[(size_t)col * 8];
        r[0] = q16(mv[0]);
        r[1] = q16(mv[1]);
        r[2] = q16(mv[2]);
        r[3] = q16(cs);
        r[4] = q16(sn);
        r[5] = 0;
        for (int j = 0; j < H; ++j) {
            const double b = ((double)(2 * j + 1 - H) / (double)H) * t_v;
            const double nrm = std::sqrt(b * b + 1.0);
            int32_t *o = &c.pano_dir[((size_t)col * H + j) * 4];
            o[0] = q30(cs / nrm);
            o[1] = q30(sn / nrm);
            o[2] = q30(-b / nrm);
        }
    }
    c.pano_A = A;
    c.pano_Wc = Wc;
    c.pano_step = step;
    return MIG_OK;
}

}  // namespace mig
