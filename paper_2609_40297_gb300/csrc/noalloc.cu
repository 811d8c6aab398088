// Tree evaluation that allocates nothing: every scratch buffer (camera tables, plan arrays,
// per-(node, yaw) counters, depth-buffer arena) lives in one file-scope device array of fixed
// size, loaded with the library and held on each GPU until the process exits.
//
// For callers that may not allocate device memory: a planner inside a real-time control loop
// whose policy forbids cudaMalloc after start-up (an allocation can stall or synchronise the
// device for an unbounded time), or a host framework that owns all device memory through its
// own pool and does not let third-party code call the CUDA allocator.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "kernels.h"
#include "mig_impl.h"

// The shared scratch. In host code this name is a host-side stand-in, not a device address:
// host code must pass the address obtained from cudaGetSymbolAddress (noalloc_scratch_ptr).
static __device__ __align__(256) unsigned char g_noalloc_scratch[MIG_NOALLOC_SCRATCH_BYTES];

namespace mig {
namespace {

// Per-pixel camera table on the device with the same IEEE double steps (explicit
// round-to-nearest intrinsics, no contraction) as the host build in camera.cpp.
__global__ void noalloc_camera_kernel(int4 *body, int W, int H, double t_h, double t_v, double cp, double sp) {
    const int total = W * H;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
        const int i = p % W, j = p / W;
        const double a = __dmul_rn(__ddiv_rn((double)(2 * i + 1 - W), (double)W), t_h);
        const double b = __dmul_rn(__ddiv_rn((double)(2 * j + 1 - H), (double)H), t_v);
        const double nrm = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), 1.0));
        const double cx = __ddiv_rn(a, nrm), cy = __ddiv_rn(b, nrm), cz = __ddiv_rn(1.0, nrm);
        const double q = 1073741824.0;
        body[p] = make_int4(__double2int_rn(__dmul_rn(__dsub_rn(__dmul_rn(cz, cp), __dmul_rn(cy, sp)), q)),
                            __double2int_rn(__dmul_rn(-cx, q)),
                            __double2int_rn(__dmul_rn(-__dadd_rn(__dmul_rn(cy, cp), __dmul_rn(cz, sp)), q)),
                            __double2int_rn(__dmul_rn(cz, q)));
    }
}

// Copies part of the per-yaw table into the scratch. The values travel in the kernel's parameters
// (captured by value at launch), so no host buffer has to outlive the call.
constexpr int kYawChunk = 1024;  // int32 per launch (4 KiB of parameters)
struct YawChunk {
    int32_t v[kYawChunk];
};
__global__ void noalloc_yaw_kernel(int32_t *dst, int count, const YawChunk chunk) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = chunk.v[i];
}

std::mutex g_setup_mu;
void *g_scratch_ptr[64] = {nullptr};

// Device address of the scratch on `device` (made current by the caller), looked up once per
// device. The first call on a device does this set-up.
mig_status noalloc_scratch_ptr(int device, unsigned char **out) {
    if (device < 0 || device >= 64) return fail(MIG_EINVAL, "tree_eval_device_noalloc: device index above 63");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(MIG_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[device] = p;
    }
    *out = (unsigned char *)g_scratch_ptr[device];
    return MIG_OK;
}

struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    }
};

}  // namespace
}  // namespace mig

using namespace mig;

extern "C" mig_status mig_tree_eval_device_noalloc(mig_map *m, int n, const int32_t *parent, const float *pos_m,
                                                   const mig_sensor *sensor, int max_depth, int32_t *abs_gain,
                                                   int32_t *marg_gain, int32_t *best_yaw) {
    if (!m || !sensor) return fail(MIG_EINVAL, "tree_eval_device_noalloc: map or sensor is NULL");
    if (n < 0) return fail(MIG_EINVAL, "tree_eval_device_noalloc: negative node count");
    if (max_depth < 0 || max_depth > MIG_MAX_DEPTH)
        return fail(MIG_EINVAL, "tree_eval_device_noalloc: max_depth outside [0, 64]");
    mig_status st = sensor_check(*sensor, m->voxel);
    if (st != MIG_OK) return st;
    if (n == 0) return MIG_OK;
    if (!parent || !pos_m || !abs_gain || !marg_gain || !best_yaw)
        return fail(MIG_EINVAL, "tree_eval_device_noalloc: NULL array");
    const int W = sensor->width, H = sensor->height, K = sensor->yaw_bins, L = max_depth + 1;
    const size_t WH = (size_t)W * H;
    // scratch layout: zeroed region first, then the rest
    Carve cv;
    const size_t o_lcnt = cv.take(4 * (size_t)L), o_licnt = cv.take(4 * (size_t)L), o_cur2 = cv.take(8 * (size_t)L);
    const size_t o_hasc = cv.take(4 * (size_t)n), o_slot = cv.take(4), o_roots = cv.take(4), o_err = cv.take(4);
    const size_t o_cnt = cv.take(8 * (size_t)n * K);
    const size_t o_work = cv.take(4 * (size_t)L);
    const size_t zero_bytes = cv.off;
    const size_t o_depth = cv.take(4 * (size_t)n), o_loff = cv.take(4 * (size_t)(L + 1)), o_lint = cv.take(4 * (size_t)L);
    const size_t o_lnodes = cv.take(4 * (size_t)n), o_ar = cv.take(8 * (size_t)n);
    const size_t o_anc = cv.take(4 * std::max<size_t>(1, (size_t)n * max_depth)), o_node = cv.take(16 * (size_t)n);
    const size_t o_sel = cv.take(4 * (size_t)n), o_body = cv.take(16 * WH), o_yaw = cv.take(4 * (size_t)K * kYawRec);
    const size_t o_arena = cv.take(4 * (size_t)n * WH);
    if (cv.off > (size_t)MIG_NOALLOC_SCRATCH_BYTES)
        return fail(MIG_EINVAL, "tree_eval_device_noalloc: needs " + std::to_string(cv.off) + " bytes of scratch, above the " +
                                    std::to_string((size_t)MIG_NOALLOC_SCRATCH_BYTES) +
                                    "-byte maximum (about nodes * width * height * 4 bytes of depth buffers)");
    // per-yaw rotation and projection rows from the host's libm, on the stack (no allocation); they
    // reach the device as kernel parameters
    const double t_h = std::tan(((double)sensor->hfov_deg * 0.5) * (M_PI / 180.0));
    const double t_v = std::tan(((double)sensor->vfov_deg * 0.5) * (M_PI / 180.0));
    const double th = (double)sensor->pitch_deg * (M_PI / 180.0);
    const double cp = std::cos(th), sp = std::sin(th);
    int32_t yaw_tab[MIG_MAX_YAW_BINS * kYawRec];
    {
        const double fx = ((double)W * 0.5) / t_h, fy = ((double)H * 0.5) / t_v;
        const double cxp = (double)W * 0.5, cyp = (double)H * 0.5;
        for (int k = 0; k < K; ++k) {
            const double ang = ((2.0 * M_PI) * (double)k) / (double)K;
            const double cs = std::cos(ang), sn = std::sin(ang);
            int32_t *o = yaw_tab + (size_t)k * kYawRec;
            o[0] = (int32_t)std::llrint(cs * 1073741824.0);
            o[1] = (int32_t)std::llrint(sn * 1073741824.0);
            const double ex[3] = {sn, -cs, 0.0};
            const double ey[3] = {-(sp * cs), -(sp * sn), -cp};
            const double ez[3] = {cp * cs, cp * sn, -sp};
            for (int a = 0; a < 3; ++a) {
                const double mu = fx * ex[a] + cxp * ez[a];
                const double mv = fy * ey[a] + cyp * ez[a];
                if (std::fabs(mu) * 65536.0 >= 2147483647.0 || std::fabs(mv) * 65536.0 >= 2147483647.0)
                    return fail(MIG_EINVAL, "sensor: focal length too large for the Q16 projection rows");
                o[2 + a] = (int32_t)std::llrint(mu * 65536.0);
                o[5 + a] = (int32_t)std::llrint(mv * 65536.0);
                o[8 + a] = (int32_t)std::llrint(ez[a] * 65536.0);
            }
            o[11] = 0;
        }
    }
    mig_ctx *ctx = m->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaSetDevice(ctx->device));
    unsigned char *dev = nullptr;
    st = noalloc_scratch_ptr(ctx->device, &dev);
    if (st != MIG_OK) return st;
    cudaStream_t s = ctx->stream;
    // the scratch keeps the previous call's contents: clear what must start at zero
    MIG_CUDA_TRY(cudaMemsetAsync(dev, 0, zero_bytes, s));
    for (int i0 = 0; i0 < K * kYawRec; i0 += kYawChunk) {
        YawChunk c;
        const int cnt = std::min(kYawChunk, K * kYawRec - i0);
        std::memcpy(c.v, yaw_tab + i0, (size_t)cnt * 4);
        noalloc_yaw_kernel<<<1, 256, 0, s>>>((int32_t *)(dev + o_yaw) + i0, cnt, c);
    }
    noalloc_camera_kernel<<<(int)std::min<size_t>((WH + 255) / 256, 1024), 256, 0, s>>>((int4 *)(dev + o_body), W, H,
                                                                                      t_h, t_v, cp, sp);
    DevPlanParams dp{};
    dp.n = n;
    dp.max_depth = max_depth;
    dp.parent = parent;
    dp.pos = pos_m;
    dp.ox = m->origin[0];
    dp.oy = m->origin[1];
    dp.oz = m->origin[2];
    dp.voxel = m->voxel;
    dp.nx = m->nx;
    dp.ny = m->ny;
    dp.nz = m->nz;
    dp.depth = (int32_t *)(dev + o_depth);
    dp.level_cnt = (int32_t *)(dev + o_lcnt);
    dp.level_icnt = (int32_t *)(dev + o_licnt);
    dp.level_off = (int32_t *)(dev + o_loff);
    dp.level_int = (int32_t *)(dev + o_lint);
    dp.has_child = (int32_t *)(dev + o_hasc);
    dp.level_nodes = (int32_t *)(dev + o_lnodes);
    dp.anc_range = (int2 *)(dev + o_ar);
    dp.anc = (int32_t *)(dev + o_anc);
    dp.level_cur2 = (int32_t *)(dev + o_cur2);
    dp.roots = (int32_t *)(dev + o_roots);
    dp.node = (int4 *)(dev + o_node);
    dp.slot_cnt = (int32_t *)(dev + o_slot);
    dp.err = (int32_t *)(dev + o_err);
    dp.ctx_err = ctx->d_err;
    dp.out_abs = abs_gain;
    dp.out_marg = marg_gain;
    dp.out_yaw = best_yaw;
    launch_plan(dp, s);
    LevelParams p{};
    p.grid = GridView{m->d_grid, m->nx, m->ny, m->nz, m->nbx, m->nby};
    p.body = (const int4 *)(dev + o_body);
    p.yawtab = (const int32_t *)(dev + o_yaw);
    p.W = W;
    p.H = H;
    p.K = K;
    p.Tq = range_q16(sensor->range_m, m->voxel);
    p.tile_w = ctx->tiles.tile_w;
    p.tile_h = ctx->tiles.tile_h;
    p.tiles_x = (W + p.tile_w - 1) / p.tile_w;
    p.tiles = p.tiles_x * ((H + p.tile_h - 1) / p.tile_h);
    p.level_off = dp.level_off;
    p.level_int = dp.level_int;
    p.level_nodes = dp.level_nodes;
    p.node = dp.node;
    p.anc_range = dp.anc_range;
    p.anc = dp.anc;
    p.sel_yaw = (int32_t *)(dev + o_sel);
    p.out_abs = abs_gain;
    p.out_marg = marg_gain;
    p.out_yaw = best_yaw;
    p.cnt = (int32_t *)(dev + o_cnt);
    p.work = (int32_t *)(dev + o_work);
    p.arena = (uint32_t *)(dev + o_arena);
    p.mode = MIG_MODE_MARGINAL;
    p.stats = nullptr;
    p.max_anc = std::max(1, max_depth);
    const int cap = ctx->num_sms * 16;
    const int count_cap = ctx->num_sms * std::min(ctx->count_ctas, std::max(1, (int)ctx->tiles.ctas_per_sm));
    const int sel_grid = std::max(1, std::min((n + 127) / 128, 1024));
    for (int d = 0; d < L; ++d) {
        p.lvl = d;
        timed_launch(ctx, kProfCount, [&] { launch_count(p, count_cap, s); });
        timed_launch(ctx, kProfSelect, [&] { launch_select(p, sel_grid, s); });
        timed_launch(ctx, kProfRender, [&] { launch_render(p, cap, s); });
    }
    MIG_CUDA_TRY(cudaGetLastError());
    return MIG_OK;
}
