// C ABI of the marginal-gain library: contexts, maps, and tree evaluation in depth order
// (Sec. IV-C) with one count / select / render launch triple per level on the context stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "interval.h"
#include "kernels.h"
#include "mig_impl.h"
#include "pano.h"
#include "voxcount.h"

namespace mig {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
mig_status fail(mig_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

void *DeviceAllocator::alloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 256;
    if (has_user) return user.alloc(bytes, (void *)s, user.user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void DeviceAllocator::free(void *p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (has_user) user.free(p, bytes, (void *)s, user.user);
    else cudaFreeAsync(p, s);
}

extern "C" void mig_batch_drop_graphs(mig_ctx *ctx);  // batch.cu

mig_status ctx_workspace(mig_ctx *ctx, size_t bytes, void **out) {
    if (ctx->ws.bytes < bytes) {
        const size_t want = std::max(bytes, ctx->ws.bytes + ctx->ws.bytes / 2);
        if (ctx->ws.ptr) mig_batch_drop_graphs(ctx);  // captured graphs copy into the old buffer
        ctx->alloc.free(ctx->ws.ptr, ctx->ws.bytes, ctx->stream);
        ctx->ws.ptr = nullptr;
        ctx->ws.bytes = 0;
        void *p = ctx->alloc.alloc(want, ctx->stream);
        if (!p) {
            p = ctx->alloc.alloc(bytes, ctx->stream);
            if (!p) return fail(MIG_ENOMEM, "device workspace allocation of " + std::to_string(bytes) + " bytes failed");
            ctx->ws.bytes = bytes;
        } else {
            ctx->ws.bytes = want;
        }
        ctx->ws.ptr = p;
    }
    *out = ctx->ws.ptr;
    return MIG_OK;
}

mig_status ctx_pinned(mig_ctx *ctx, size_t bytes, void **out) {
    if (ctx->pinned_bytes < bytes) {
        const size_t want = std::max({bytes, (size_t)1 << 20, 2 * ctx->pinned_bytes});
        if (ctx->pinned) {
            mig_batch_drop_graphs(ctx);  // captured graphs copy from and to the old buffer
            cudaStreamSynchronize(ctx->stream);
            cudaFreeHost(ctx->pinned);
        }
        ctx->pinned = nullptr;
        ctx->pinned_bytes = 0;
        if (cudaHostAlloc(&ctx->pinned, want, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            ctx->pinned = nullptr;
            return fail(MIG_ENOMEM, "pinned host staging allocation failed");
        }
        ctx->pinned_bytes = want;
    }
    *out = ctx->pinned;
    return MIG_OK;
}

mig_status ctx_camera(mig_ctx *ctx, const mig_sensor &s, const Camera **out) {
    for (auto &c : ctx->cameras) {
        if (std::memcmp(&c->s, &s, sizeof(mig_sensor)) == 0) {
            *out = c.get();
            return MIG_OK;
        }
    }
    auto cam = std::make_unique<Camera>();
    mig_status st = camera_build(s, *cam);
    if (st != MIG_OK) return st;
    cam->yawf.resize((size_t)cam->K * 9);
    for (int k = 0; k < cam->K; ++k)
        for (int t = 0; t < 9; ++t) cam->yawf[(size_t)k * 9 + t] = (float)cam->yaw[(size_t)k * kYawRec + 2 + t] * (1.0f / 65536.0f);
    const size_t bb = cam->body.size() * 4, yb = (cam->yaw.size() + cam->yawf.size()) * 4;
    cam->d_body = (int32_t *)ctx->alloc.alloc(bb, ctx->stream);
    cam->d_yaw = (int32_t *)ctx->alloc.alloc(yb, ctx->stream);
    if (!cam->d_body || !cam->d_yaw) {
        ctx->alloc.free(cam->d_body, bb, ctx->stream);
        ctx->alloc.free(cam->d_yaw, yb, ctx->stream);
        return fail(MIG_ENOMEM, "camera table allocation failed");
    }
    MIG_CUDA_TRY(cudaMemcpyAsync(cam->d_body, cam->body.data(), bb, cudaMemcpyHostToDevice, ctx->stream));
    cam->d_yawf = reinterpret_cast<const float *>(cam->d_yaw + cam->yaw.size());
    MIG_CUDA_TRY(cudaMemcpyAsync(cam->d_yaw, cam->yaw.data(), cam->yaw.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    MIG_CUDA_TRY(cudaMemcpyAsync(const_cast<float *>(cam->d_yawf), cam->yawf.data(), cam->yawf.size() * 4,
                                 cudaMemcpyHostToDevice, ctx->stream));
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));  // host tables may move with the vector
    *out = cam.get();
    ctx->cameras.push_back(std::move(cam));
    return MIG_OK;
}

// The panoramic tables of a context's camera, built and uploaded on first use.
mig_status ctx_pano(mig_ctx *ctx, const Camera *ccam) {
    Camera *cam = nullptr;
    for (auto &c : ctx->cameras)
        if (c.get() == ccam) cam = c.get();
    if (!cam) return fail(MIG_EINVAL, "panoramic mode: unknown camera");
    if (cam->d_pano_dir) return MIG_OK;
    mig_status st = pano_build(*cam);
    if (st != MIG_OK) return st;
    const size_t bb = cam->pano_bc.size() * 4, db = cam->pano_dir.size() * 4, rb = cam->pano_row.size() * 4;
    int32_t *b = (int32_t *)ctx->alloc.alloc(bb, ctx->stream), *d = (int32_t *)ctx->alloc.alloc(db, ctx->stream),
            *r = (int32_t *)ctx->alloc.alloc(rb, ctx->stream);
    if (!b || !d || !r) {
        ctx->alloc.free(b, bb, ctx->stream);
        ctx->alloc.free(d, db, ctx->stream);
        ctx->alloc.free(r, rb, ctx->stream);
        return fail(MIG_ENOMEM, "panoramic table allocation failed");
    }
    MIG_CUDA_TRY(cudaMemcpyAsync(b, cam->pano_bc.data(), bb, cudaMemcpyHostToDevice, ctx->stream));
    MIG_CUDA_TRY(cudaMemcpyAsync(d, cam->pano_dir.data(), db, cudaMemcpyHostToDevice, ctx->stream));
    MIG_CUDA_TRY(cudaMemcpyAsync(r, cam->pano_row.data(), rb, cudaMemcpyHostToDevice, ctx->stream));
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    cam->d_pano_bc = b;
    cam->d_pano_dir = d;
    cam->d_pano_row = r;
    return MIG_OK;
}

void set_band(LevelParams &p, const Camera *cam) {
    p.band_tlo = cam->band_tlo;
    p.band_thi = cam->band_thi;
    p.az_half = cam->az_half;
}

void set_pano_params(LevelParams &p, const Camera *cam, int32_t *pcnt) {
    p.pano_A = cam->pano_A;
    p.pano_Wc = cam->pano_Wc;
    p.pano_step = cam->pano_step;
    p.pano_bc = (const int2 *)cam->d_pano_bc;
    p.pano_dir = (const int4 *)cam->d_pano_dir;
    p.pano_row = (const int4 *)cam->d_pano_row;
    p.pano_cnt = pcnt;
}

void launch_level_count(const mig_ctx *ctx, const LevelParams &p, int Ld, int count_cap, cudaStream_t s) {
    const int items = Ld * p.K * p.tiles;
    if (p.mode == MIG_MODE_INTERVAL) {
        launch_count_interval(p, std::max(1, std::min((items + 7) / 8, ctx->num_sms * ctx->interval_ctas)), s);
    } else if (p.mode == MIG_MODE_PANORAMIC) {
        const int pitems = Ld * p.pano_A;
        launch_pano_count(p, std::max(1, std::min((pitems + 7) / 8, ctx->num_sms * ctx->pano_ctas)), s);
        launch_pano_window(p, std::max(1, std::min((Ld * p.K + 255) / 256, 1024)), s);
    } else if (p.steps) {
        launch_vox_level(p, (long long)Ld * p.K, ctx->num_sms, ctx->vox_ctas, ctx->node_ctas, s);
    } else {
        launch_count(p, std::max(1, std::min((items + 7) / 8, count_cap)), s);
    }
}

void launch_level_count_timed(mig_ctx *ctx, const LevelParams &p, int Ld, int count_cap) {
    if (!p.steps || p.mode == MIG_MODE_INTERVAL || p.mode == MIG_MODE_PANORAMIC) {
        timed_launch(ctx, kProfCount, [&] { launch_level_count(ctx, p, Ld, count_cap, ctx->stream); });
        return;
    }
    const long long pairs = (long long)Ld * p.K;
    const int cap = vox_chunk_pairs(p);
    for (long long q0 = 0; q0 < pairs; q0 += cap) {
        LevelParams c = p;
        c.q0 = (int)q0;
        c.q1 = (int)std::min<long long>(pairs, q0 + cap);
        timed_launch(ctx, kProfCast, [&] { launch_cast_chunk(c, ctx->num_sms, ctx->stream); });
        timed_launch(ctx, kProfVoxel, [&] {
            if (node_pass(c)) launch_node_chunk(c, ctx->num_sms, ctx->node_ctas, ctx->stream);
            else launch_voxel_chunk(c, ctx->num_sms, ctx->vox_ctas, ctx->stream);
        });
    }
}

int steps_cap_for(const mig_ctx *ctx, int Lmax, int K, int W, int H, int mode) {
    if (ctx->ray_count || mode == MIG_MODE_INTERVAL || mode == MIG_MODE_PANORAMIC) return 0;
    return (int)steps_pairs((long long)std::max(1, Lmax) * K, W, H, ctx->steps_budget);
}

void prof_begin(mig_ctx *ctx, int kind, cudaEvent_t *a) {
    (void)kind;
    *a = nullptr;
    if (!ctx->prof.on) return;
    cudaEvent_t e = nullptr;
    if (!ctx->prof.pool.empty()) {
        e = ctx->prof.pool.back();
        ctx->prof.pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(e, ctx->stream);
    *a = e;
}

void prof_end(mig_ctx *ctx, int kind, cudaEvent_t a) {
    if (!ctx->prof.on || !a) return;
    cudaEvent_t b = nullptr;
    if (!ctx->prof.pool.empty()) {
        b = ctx->prof.pool.back();
        ctx->prof.pool.pop_back();
    } else if (cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        ctx->prof.pool.push_back(a);
        return;
    }
    cudaEventRecord(b, ctx->stream);
    ctx->prof.pending.push_back({kind, a, b});
}

static void prof_collect(mig_ctx *ctx) {
    for (auto &pr : ctx->prof.pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pr.a, pr.b) == cudaSuccess) {
            ctx->prof.ms[pr.kind] += ms;
            ctx->prof.launches[pr.kind] += 1;
        } else {
            cudaGetLastError();
        }
        ctx->prof.pool.push_back(pr.a);
        ctx->prof.pool.push_back(pr.b);
    }
    ctx->prof.pending.clear();
}

// Carves 256-byte aligned regions out of one allocation.
struct Carver {
    size_t off = 0;
    template <class T>
    size_t take(size_t count) {
        const size_t o = off;
        off += (count * sizeof(T) + 255) & ~(size_t)255;
        return o;
    }
};

static mig_status check_codes(const uint8_t *v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (v[i] > 2) return fail(MIG_EINVAL, "map: voxel code " + std::to_string(v[i]) + " at index " + std::to_string(i) + " (codes are 0, 1, 2)");
    return MIG_OK;
}

static LevelParams level_params(const mig_map *m, const Camera *cam, const mig_ctx *ctx) {
    LevelParams p{};
    p.grid = GridView{m->d_grid, m->nx, m->ny, m->nz, m->nbx, m->nby};
    p.body = (const int4 *)cam->d_body;
    p.yawtab = cam->d_yaw;
    p.yawf = cam->d_yawf;
    p.W = cam->W;
    p.H = cam->H;
    p.K = cam->K;
    p.Tq = range_q16(cam->s.range_m, m->voxel);
    p.tile_w = ctx->tiles.tile_w;
    p.tile_h = ctx->tiles.tile_h;
    p.tiles_x = (p.W + p.tile_w - 1) / p.tile_w;
    p.tiles = p.tiles_x * ((p.H + p.tile_h - 1) / p.tile_h);
    set_band(p, cam);
    p.voxel_pass = ctx->voxel_pass;
    return p;
}

}  // namespace mig

using namespace mig;

extern "C" {

const char *mig_last_error(void) { return g_last_error.c_str(); }

int mig_build_flags(void) {
#if defined(MIG_DEBUG_BOUNDS) && MIG_DEBUG_BOUNDS
    return MIG_BUILD_CHECKED;
#else
    return 0;
#endif
}

mig_status mig_ctx_create(int device, void *stream, const mig_allocator *allocator, mig_ctx **out) {
    if (!out) return fail(MIG_EINVAL, "ctx_create: out is NULL");
    *out = nullptr;
    int count = 0;
    MIG_CUDA_TRY(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return fail(MIG_EINVAL, "ctx_create: no such device");
    MIG_CUDA_TRY(cudaSetDevice(device));
    auto ctx = std::make_unique<mig_ctx>();
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    if (allocator) {
        if (!allocator->alloc || !allocator->free) return fail(MIG_EINVAL, "ctx_create: allocator callbacks are NULL");
        ctx->alloc.user = *allocator;
        ctx->alloc.has_user = true;
    }
    MIG_CUDA_TRY(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
    ctx->count_ctas = count_ctas_per_sm();
    ctx->interval_ctas = count_interval_ctas_per_sm();
    ctx->pano_ctas = pano_ctas_per_sm();
    ctx->vox_ctas = vox_ctas_per_sm();
    ctx->node_ctas = node_ctas_per_sm();
    ctx->steps_budget = kStepsBudget;
    ctx->d_err = (int32_t *)ctx->alloc.alloc(256, ctx->stream);
    if (!ctx->d_err) return fail(MIG_ENOMEM, "ctx_create: allocation failed");
    MIG_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, 256, ctx->stream));
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    *out = ctx.release();
    return MIG_OK;
}

void mig_batch_release(mig_ctx *ctx);  // batch.cu

void mig_ctx_destroy(mig_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    mig_batch_release(ctx);
    for (auto &c : ctx->cameras) {
        ctx->alloc.free(c->d_body, c->body.size() * 4, ctx->stream);
        ctx->alloc.free(c->d_yaw, (c->yaw.size() + c->yawf.size()) * 4, ctx->stream);
        ctx->alloc.free(c->d_pano_bc, c->pano_bc.size() * 4, ctx->stream);
        ctx->alloc.free(c->d_pano_dir, c->pano_dir.size() * 4, ctx->stream);
        ctx->alloc.free(c->d_pano_row, c->pano_row.size() * 4, ctx->stream);
    }
    ctx->alloc.free(ctx->ws.ptr, ctx->ws.bytes, ctx->stream);
    ctx->alloc.free(ctx->d_err, 256, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    for (auto &pr : ctx->prof.pending) {
        cudaEventDestroy(pr.a);
        cudaEventDestroy(pr.b);
    }
    for (auto e : ctx->prof.pool) cudaEventDestroy(e);
    delete ctx;
}

mig_status mig_ctx_set_stream(mig_ctx *ctx, void *stream) {
    if (!ctx) return fail(MIG_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    ctx->stream = (cudaStream_t)stream;
    return MIG_OK;
}

mig_status mig_ctx_sync(mig_ctx *ctx) {
    if (!ctx) return fail(MIG_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaSetDevice(ctx->device));
    int32_t err = 0;
    MIG_CUDA_TRY(cudaMemcpyAsync(&err, ctx->d_err, 4, cudaMemcpyDeviceToHost, ctx->stream));
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (err) {
        MIG_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, 4, ctx->stream));
        MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        return fail(MIG_EINVAL, "device-side tree check failed (code " + std::to_string(err) +
                                    ": 1 = bad parent/cycle/too deep, 2 = position outside the grid, 4 = not exactly one root)");
    }
    return MIG_OK;
}

mig_status mig_ctx_set_count_kernel(mig_ctx *ctx, int kernel, uint64_t steps_budget_bytes) {
    if (!ctx) return fail(MIG_EINVAL, "ctx is NULL");
    if (kernel < MIG_COUNT_AUTO || kernel > MIG_COUNT_NODES) return fail(MIG_EINVAL, "set_count_kernel: unknown kernel");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->ray_count = kernel == MIG_COUNT_RAYS;
    ctx->voxel_pass = kernel == MIG_COUNT_RAYS ? MIG_COUNT_AUTO : kernel;
    ctx->steps_budget = steps_budget_bytes ? (size_t)steps_budget_bytes : kStepsBudget;
    return MIG_OK;
}

mig_status mig_ctx_profile(mig_ctx *ctx, int enable) {
    if (!ctx) return fail(MIG_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaSetDevice(ctx->device));
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    prof_collect(ctx);
    for (int k = 0; k < kProfKinds; ++k) {
        ctx->prof.ms[k] = 0;
        ctx->prof.launches[k] = 0;
    }
    ctx->prof.on = enable != 0;
    return MIG_OK;
}

mig_status mig_ctx_profile_read(mig_ctx *ctx, mig_kernel_times *out) {
    if (!ctx || !out) return fail(MIG_EINVAL, "profile_read: NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaSetDevice(ctx->device));
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    prof_collect(ctx);
    out->count_ms = ctx->prof.ms[kProfCount];
    out->select_ms = ctx->prof.ms[kProfSelect];
    out->render_ms = ctx->prof.ms[kProfRender];
    out->plan_ms = ctx->prof.ms[kProfPlan];
    out->batch_ms = ctx->prof.ms[kProfBatch];
    out->count_launches = ctx->prof.launches[kProfCount];
    out->select_launches = ctx->prof.launches[kProfSelect];
    out->render_launches = ctx->prof.launches[kProfRender];
    out->plan_launches = ctx->prof.launches[kProfPlan];
    out->batch_launches = ctx->prof.launches[kProfBatch];
    out->cast_ms = ctx->prof.ms[kProfCast];
    out->voxel_ms = ctx->prof.ms[kProfVoxel];
    out->cast_launches = ctx->prof.launches[kProfCast];
    out->voxel_launches = ctx->prof.launches[kProfVoxel];
    for (int k = 0; k < kProfKinds; ++k) {
        ctx->prof.ms[k] = 0;
        ctx->prof.launches[k] = 0;
    }
    return MIG_OK;
}

// ------------------------------------------------------------------------------------ maps
mig_status mig_map_create(mig_ctx *ctx, int nx, int ny, int nz, float voxel_size_m, const float origin_m[3],
                          const uint8_t *host_voxels, mig_map **out) {
    if (!ctx || !out) return fail(MIG_EINVAL, "map_create: ctx or out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || nx > MIG_MAX_DIM || ny > MIG_MAX_DIM || nz > MIG_MAX_DIM)
        return fail(MIG_EINVAL, "map_create: dimensions outside [1, 4096]");
    if (!(voxel_size_m > 0.f) || !std::isfinite(voxel_size_m)) return fail(MIG_EINVAL, "map_create: voxel size must be positive");
    auto m = std::make_unique<mig_map>();
    m->ctx = ctx;
    m->nx = nx;
    m->ny = ny;
    m->nz = nz;
    m->grid_bytes = map_layout_bytes(nx, ny, nz, &m->nbx, &m->nby, &m->nbz);
    if (m->grid_bytes >= ((size_t)1 << 32)) return fail(MIG_EINVAL, "map_create: padded grid above 2^32 voxels");
    m->voxel = voxel_size_m;
    for (int a = 0; a < 3; ++a) m->origin[a] = origin_m ? origin_m[a] : 0.f;
    const size_t nvox = (size_t)nx * ny * nz;
    if (host_voxels) {
        mig_status st = check_codes(host_voxels, nvox);
        if (st != MIG_OK) return st;
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaSetDevice(ctx->device));
    m->d_grid = (uint8_t *)ctx->alloc.alloc(m->grid_bytes, ctx->stream);
    if (!m->d_grid) return fail(MIG_ENOMEM, "map_create: grid allocation failed");
    MIG_CUDA_TRY(cudaMemsetAsync(m->d_grid, 0, m->grid_bytes, ctx->stream));
    if (host_voxels) {
        uint8_t *tmp = (uint8_t *)ctx->alloc.alloc(nvox, ctx->stream);
        if (!tmp) {
            ctx->alloc.free(m->d_grid, m->grid_bytes, ctx->stream);
            return fail(MIG_ENOMEM, "map_create: staging allocation failed");
        }
        MIG_CUDA_TRY(cudaMemcpyAsync(tmp, host_voxels, nvox, cudaMemcpyHostToDevice, ctx->stream));
        launch_map_scatter(m->d_grid, m->nx, m->ny, m->nz, m->nbx, m->nby, tmp, 0, 0, 0, nx, ny, nz, ctx->stream);
        MIG_CUDA_TRY(cudaGetLastError());
        ctx->alloc.free(tmp, nvox, ctx->stream);
    }
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    *out = m.release();
    return MIG_OK;
}

mig_status mig_map_update(mig_map *m, int x0, int y0, int z0, int dx, int dy, int dz, const uint8_t *host_voxels) {
    if (!m || !host_voxels) return fail(MIG_EINVAL, "map_update: map or voxels NULL");
    if (dx < 1 || dy < 1 || dz < 1 || x0 < 0 || y0 < 0 || z0 < 0 || x0 + dx > m->nx || y0 + dy > m->ny || z0 + dz > m->nz)
        return fail(MIG_EINVAL, "map_update: box outside the grid or empty");
    const size_t nvox = (size_t)dx * dy * dz;
    mig_status st = check_codes(host_voxels, nvox);
    if (st != MIG_OK) return st;
    mig_ctx *ctx = m->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaSetDevice(ctx->device));
    uint8_t *tmp = (uint8_t *)ctx->alloc.alloc(nvox, ctx->stream);
    if (!tmp) return fail(MIG_ENOMEM, "map_update: staging allocation failed");
    MIG_CUDA_TRY(cudaMemcpyAsync(tmp, host_voxels, nvox, cudaMemcpyHostToDevice, ctx->stream));
    launch_map_scatter(m->d_grid, m->nx, m->ny, m->nz, m->nbx, m->nby, tmp, x0, y0, z0, dx, dy, dz, ctx->stream);
    MIG_CUDA_TRY(cudaGetLastError());
    ctx->alloc.free(tmp, nvox, ctx->stream);
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));  // the host buffer may be reused on return
    m->version++;
    return MIG_OK;
}

mig_status mig_map_read(mig_map *m, uint8_t *host_out) {
    if (!m || !host_out) return fail(MIG_EINVAL, "map_read: NULL argument");
    mig_ctx *ctx = m->ctx;
    const size_t nvox = (size_t)m->nx * m->ny * m->nz;
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaSetDevice(ctx->device));
    uint8_t *tmp = (uint8_t *)ctx->alloc.alloc(nvox, ctx->stream);
    if (!tmp) return fail(MIG_ENOMEM, "map_read: staging allocation failed");
    launch_map_gather(m->d_grid, m->nbx, m->nby, tmp, m->nx, m->ny, m->nz, ctx->stream);
    MIG_CUDA_TRY(cudaGetLastError());
    MIG_CUDA_TRY(cudaMemcpyAsync(host_out, tmp, nvox, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->alloc.free(tmp, nvox, ctx->stream);
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return MIG_OK;
}

void mig_map_destroy(mig_map *m) {
    if (!m) return;
    mig_ctx *ctx = m->ctx;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        ctx->alloc.free(m->d_grid, m->grid_bytes, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
    }
    delete m;
}

// ----------------------------------------------------------------------------- host helpers
mig_status mig_default_resolution(const mig_sensor *s, float voxel_size_m, int32_t *w, int32_t *h) {
    if (!s || !w || !h) return fail(MIG_EINVAL, "default_resolution: NULL argument");
    if (!(voxel_size_m > 0.f) || !(s->range_m > 0.f) || !(s->hfov_deg > 0.f && s->hfov_deg < 180.f) ||
        !(s->vfov_deg > 0.f && s->vfov_deg < 180.f))
        return fail(MIG_EINVAL, "default_resolution: invalid sensor or voxel size");
    // Sec. IV-A: W_D = ceil(2 d_max tan(theta_h / 2) / v_size), H_D likewise
    const double W = std::ceil(2.0 * s->range_m * std::tan(s->hfov_deg * M_PI / 360.0) / voxel_size_m);
    const double H = std::ceil(2.0 * s->range_m * std::tan(s->vfov_deg * M_PI / 360.0) / voxel_size_m);
    if (W < 1 || H < 1 || W > MIG_MAX_IMAGE || H > MIG_MAX_IMAGE) return fail(MIG_EINVAL, "default_resolution: image too large");
    *w = (int32_t)W;
    *h = (int32_t)H;
    return MIG_OK;
}

mig_status mig_tree_check(int n, const int32_t *parent, int32_t *depth_out, int32_t *max_depth_out) {
    return tree_check(n, parent, depth_out, max_depth_out);
}

// ------------------------------------------------------------------------- tree evaluation
static mig_status eval_host(mig_map *m, int n, const int32_t *parent, const float *pos_m, const mig_sensor *sensor,
                            const mig_eval_opts *opts, mig_eval_stats *stats, int32_t *abs_gain, int32_t *marg_gain,
                            int32_t *best_yaw) {
    NvtxRange range("mig_tree_eval");
    if (!m || !sensor) return fail(MIG_EINVAL, "tree_eval: map or sensor is NULL");
    if (n < 0) return fail(MIG_EINVAL, "tree_eval: negative node count");
    if (n > 0 && (!abs_gain || !marg_gain || !best_yaw)) return fail(MIG_EINVAL, "tree_eval: output array is NULL");
    const int mode = opts ? opts->mode : MIG_MODE_MARGINAL;
    if (mode < 0 || mode > MIG_MODE_PANORAMIC) return fail(MIG_EINVAL, "tree_eval: unknown mode");
    mig_status st = sensor_check(*sensor, m->voxel);
    if (st != MIG_OK) return st;
    if (n == 0) return MIG_OK;
    const int dims[3] = {m->nx, m->ny, m->nz};
    HostPlan plan;
    st = plan_build(n, parent, pos_m, m->origin, m->voxel, dims, plan);
    if (st != MIG_OK) return st;
    const bool want_depth = opts && opts->depth_buffers;
    if (want_depth) {  // every node gets a depth buffer (diagnostics)
        for (int i = 0; i < n; ++i) plan.node[(size_t)i * 4 + 3] = i;
        for (size_t d = 0; d < plan.level_int.size(); ++d) plan.level_int[d] = plan.level_off[d + 1] - plan.level_off[d];
        plan.n_internal = n;
    }
    mig_ctx *ctx = m->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaSetDevice(ctx->device));
    const Camera *cam = nullptr;
    st = ctx_camera(ctx, *sensor, &cam);
    if (st != MIG_OK) return st;
    const bool pano = mode == MIG_MODE_PANORAMIC;
    if (pano) {
        st = ctx_pano(ctx, cam);
        if (st != MIG_OK) return st;
    }
    const int K = cam->K, L = plan.max_depth + 1;
    const size_t WH = (size_t)cam->W * cam->H;
    // device layout: [upload prefix | sel_yaw | out | cnt | arena]
    Carver cv;
    const size_t o_node = cv.take<int4>(n), o_ar = cv.take<int2>(n), o_anc = cv.take<int32_t>(std::max(1, plan.total_anc));
    const size_t o_loff = cv.take<int32_t>(L + 1), o_lint = cv.take<int32_t>(L), o_lnodes = cv.take<int32_t>(n);
    const size_t up_bytes = cv.off;
    const size_t o_sel = cv.take<int32_t>(n), o_out = cv.take<int32_t>(3 * (size_t)n);
    const size_t o_cnt = cv.take<int32_t>((size_t)n * K * 2);
    const size_t o_work = cv.take<int32_t>(L);
    const size_t o_arena = cv.take<uint32_t>((size_t)std::max(1, plan.n_internal) * WH);
    const size_t o_stats = cv.take<unsigned long long>(kStatsCounters);
    const size_t o_pcnt = cv.take<int32_t>(pano ? (size_t)n * cam->pano_A * 2 : 1);
    int Lmax = 1;
    for (int d = 0; d < L; ++d) Lmax = std::max(Lmax, plan.level_off[d + 1] - plan.level_off[d]);
    const int steps_cap = steps_cap_for(ctx, Lmax, K, cam->W, cam->H, mode);
    const size_t o_steps = cv.take<char>(steps_region_bytes(steps_cap, WH));
    // instrumented pass: the ray-by-ray count kernel is re-run into scratch counters afterwards,
    // for the method's own work counts (rays, DDA steps, owner tests) and as a cross-check
    const bool rerun = stats && steps_cap > 0;
    const size_t o_cnt2 = cv.take<int32_t>(rerun ? (size_t)n * K * 2 + L : 1);
    char *dev = nullptr;
    st = ctx_workspace(ctx, cv.off, (void **)&dev);
    if (st != MIG_OK) return st;
    char *host = nullptr;
    st = ctx_pinned(ctx, std::max(up_bytes, 3 * (size_t)n * 4), (void **)&host);
    if (st != MIG_OK) return st;
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));  // staging may still feed an earlier copy
    {
        int32_t *nodep = (int32_t *)(host + o_node);
        std::memcpy(nodep, plan.node.data(), (size_t)n * 16);
        int2 *arp = (int2 *)(host + o_ar);
        for (int i = 0; i < n; ++i) arp[i] = make_int2(plan.anc_off[i], plan.depth[i]);
        if (plan.total_anc) std::memcpy(host + o_anc, plan.anc.data(), (size_t)plan.total_anc * 4);
        std::memcpy(host + o_loff, plan.level_off.data(), (size_t)(L + 1) * 4);
        std::memcpy(host + o_lint, plan.level_int.data(), (size_t)L * 4);
        std::memcpy(host + o_lnodes, plan.level_nodes.data(), (size_t)n * 4);
    }
    MIG_CUDA_TRY(cudaMemcpyAsync(dev, host, up_bytes, cudaMemcpyHostToDevice, ctx->stream));
    MIG_CUDA_TRY(cudaMemsetAsync(dev + o_cnt, 0, o_arena - o_cnt, ctx->stream));  // counters + work counters
    LevelParams p = level_params(m, cam, ctx);
    p.level_off = (const int32_t *)(dev + o_loff);
    p.level_int = (const int32_t *)(dev + o_lint);
    p.level_nodes = (const int32_t *)(dev + o_lnodes);
    p.node = (const int4 *)(dev + o_node);
    p.anc_range = (const int2 *)(dev + o_ar);
    p.anc = (const int32_t *)(dev + o_anc);
    p.sel_yaw = (int32_t *)(dev + o_sel);
    p.out_abs = (int32_t *)(dev + o_out);
    p.out_marg = p.out_abs + n;
    p.out_yaw = p.out_abs + 2 * (size_t)n;
    p.cnt = (int32_t *)(dev + o_cnt);
    p.work = (int32_t *)(dev + o_work);
    p.arena = (uint32_t *)(dev + o_arena);
    p.mode = mode;
    p.max_anc = std::max(1, plan.max_depth);
    p.arena_slots = std::max(1, plan.n_internal);
    if (pano) set_pano_params(p, cam, (int32_t *)(dev + o_pcnt));
#if defined(MIG_DEBUG_BOUNDS) && MIG_DEBUG_BOUNDS
    p.bounds_err = ctx->d_err + 16;  // checked build: out-of-buffer indices are recorded here
    MIG_CUDA_TRY(cudaMemsetAsync(p.bounds_err, 0, 4, ctx->stream));
#endif
    p.steps = steps_cap ? (uint16_t *)(dev + o_steps) : nullptr;
    p.vctr = steps_counter((uint16_t *)(dev + o_steps), steps_cap, WH);
    p.steps_cap = steps_cap;
    if (stats) {
        p.stats = (unsigned long long *)(dev + o_stats);
        MIG_CUDA_TRY(cudaMemsetAsync(p.stats, 0, kStatsCounters * sizeof(unsigned long long), ctx->stream));
    }
    const int cap = ctx->num_sms * 16;
    const int count_cap = ctx->num_sms * std::min(ctx->count_ctas, std::max(1, (int)ctx->tiles.ctas_per_sm));
    uint64_t n_count = 0, n_render = 0;
    for (int d = 0; d < L; ++d) {
        p.lvl = d;
        const int Ld = plan.level_off[d + 1] - plan.level_off[d];
        launch_level_count_timed(ctx, p, Ld, count_cap);
        timed_launch(ctx, kProfSelect,
                     [&] { launch_select(p, std::max(1, std::min((Ld + 127) / 128, 1024)), ctx->stream); });
        const int ritems = plan.level_int[d] * render_tiles(p.W, p.H);
        if (ritems > 0) timed_launch(ctx, kProfRender, [&] { launch_render(p, std::min(ritems, cap), ctx->stream); });
        n_count++;
        n_render += ritems > 0;
    }
    std::vector<int32_t> cnt_rerun;
    if (rerun) {
        LevelParams r = p;
        r.steps = nullptr;
        r.cnt = (int32_t *)(dev + o_cnt2);
        r.work = r.cnt + (size_t)n * K * 2;
        MIG_CUDA_TRY(cudaMemsetAsync(r.cnt, 0, ((size_t)n * K * 2 + L) * 4, ctx->stream));
        for (int d = 0; d < L; ++d) {
            r.lvl = d;
            launch_level_count(ctx, r, plan.level_off[d + 1] - plan.level_off[d], count_cap, ctx->stream);
        }
        cnt_rerun.resize((size_t)n * K * 2);
        MIG_CUDA_TRY(cudaMemcpyAsync(cnt_rerun.data(), r.cnt, cnt_rerun.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    }
    unsigned long long st8[kStatsCounters] = {};
    if (stats)
        MIG_CUDA_TRY(cudaMemcpyAsync(st8, p.stats, sizeof(st8), cudaMemcpyDeviceToHost, ctx->stream));
    MIG_CUDA_TRY(cudaGetLastError());
    MIG_CUDA_TRY(cudaMemcpyAsync(host, p.out_abs, 3 * (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<int32_t> cnt_h;
    if (rerun) cnt_h.resize((size_t)n * K * 2);
    if (rerun || (opts && (opts->counts_abs || opts->counts_marg))) {
        cnt_h.resize((size_t)n * K * 2);
        MIG_CUDA_TRY(cudaMemcpyAsync(cnt_h.data(), p.cnt, cnt_h.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (want_depth)
        MIG_CUDA_TRY(cudaMemcpyAsync(opts->depth_buffers, p.arena, (size_t)n * WH * 4, cudaMemcpyDeviceToHost, ctx->stream));
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
#if defined(MIG_DEBUG_BOUNDS) && MIG_DEBUG_BOUNDS
    int32_t berr = 0;
    MIG_CUDA_TRY(cudaMemcpy(&berr, p.bounds_err, 4, cudaMemcpyDeviceToHost));
    if (berr) return fail(MIG_ECUDA, "bounds check: an index left its buffer (kinds " + std::to_string(berr) + ")");
#endif
    std::memcpy(abs_gain, host, (size_t)n * 4);
    std::memcpy(marg_gain, host + (size_t)n * 4, (size_t)n * 4);
    std::memcpy(best_yaw, host + (size_t)n * 8, (size_t)n * 4);
    if (rerun && cnt_h != cnt_rerun)
        return fail(MIG_ECUDA, "instrumented pass: the owned-voxel and ray-by-ray counts differ");
    if (!cnt_h.empty() && opts) {
        for (size_t i = 0; i < (size_t)n * K; ++i) {
            if (opts->counts_abs) opts->counts_abs[i] = cnt_h[2 * i];
            if (opts->counts_marg) opts->counts_marg[i] = cnt_h[2 * i + 1];
        }
    }
    if (stats) {
        stats->rays = st8[0];
        stats->dda_steps = st8[1];
        stats->unknown_visits = st8[2];
        stats->samples = st8[3];
        stats->ancestor_tests = st8[4];
        stats->depth_reads = st8[5];
        stats->render_rays = st8[6];
        stats->render_steps = st8[7];
        stats->count_launches = n_count;
        stats->render_launches = n_render;
        stats->cast_rays = st8[8];
        stats->cast_steps = st8[9];
        stats->cast_jumps = st8[10];
        stats->voxel_candidates = st8[11];
        stats->voxel_unknown = st8[12];
        stats->visit_tests = st8[13];
        stats->owned_samples = st8[14];
        stats->voxel_ancestor_tests = st8[15];
        stats->voxel_depth_reads = st8[16];
        stats->voxel_pass = !p.steps ? MIG_COUNT_RAYS : (node_pass(p) ? MIG_COUNT_NODES : MIG_COUNT_PAIRS);
    }
    return MIG_OK;
}

mig_status mig_tree_eval_ex(mig_map *m, int n, const int32_t *parent, const float *pos_m, const mig_sensor *sensor,
                            const mig_eval_opts *opts, int32_t *abs_gain, int32_t *marg_gain, int32_t *best_yaw) {
    return eval_host(m, n, parent, pos_m, sensor, opts, nullptr, abs_gain, marg_gain, best_yaw);
}

mig_status mig_tree_eval_stats(mig_map *m, int n, const int32_t *parent, const float *pos_m, const mig_sensor *sensor,
                               mig_eval_stats *stats, int32_t *abs_gain, int32_t *marg_gain, int32_t *best_yaw) {
    if (!stats) return fail(MIG_EINVAL, "tree_eval_stats: stats is NULL");
    std::memset(stats, 0, sizeof(*stats));
    return eval_host(m, n, parent, pos_m, sensor, nullptr, stats, abs_gain, marg_gain, best_yaw);
}

mig_status mig_tree_eval(mig_map *m, int n, const int32_t *parent, const float *pos_m, const mig_sensor *sensor,
                         int32_t *abs_gain, int32_t *marg_gain, int32_t *best_yaw) {
    return mig_tree_eval_ex(m, n, parent, pos_m, sensor, nullptr, abs_gain, marg_gain, best_yaw);
}

mig_status mig_tree_eval_device(mig_map *m, int n, const int32_t *parent, const float *pos_m, const mig_sensor *sensor,
                                int max_depth, int32_t *abs_gain, int32_t *marg_gain, int32_t *best_yaw) {
    NvtxRange range("mig_tree_eval_device");
    if (!m || !sensor) return fail(MIG_EINVAL, "tree_eval_device: map or sensor is NULL");
    if (n < 0) return fail(MIG_EINVAL, "tree_eval_device: negative node count");
    if (max_depth < 0 || max_depth > MIG_MAX_DEPTH) return fail(MIG_EINVAL, "tree_eval_device: max_depth outside [0, 64]");
    mig_status st = sensor_check(*sensor, m->voxel);
    if (st != MIG_OK) return st;
    if (n == 0) return MIG_OK;
    if (!parent || !pos_m || !abs_gain || !marg_gain || !best_yaw) return fail(MIG_EINVAL, "tree_eval_device: NULL array");
    mig_ctx *ctx = m->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaSetDevice(ctx->device));
    const Camera *cam = nullptr;
    st = ctx_camera(ctx, *sensor, &cam);
    if (st != MIG_OK) return st;
    const int K = cam->K, L = max_depth + 1;
    const size_t WH = (size_t)cam->W * cam->H;
    Carver cv;
    // zero-initialised region first
    const size_t o_lcnt = cv.take<int32_t>(L), o_licnt = cv.take<int32_t>(L), o_cur2 = cv.take<int32_t>(2 * L);
    const size_t o_hasc = cv.take<int32_t>(n), o_slot = cv.take<int32_t>(1), o_roots = cv.take<int32_t>(1);
    const size_t o_err = cv.take<int32_t>(1), o_cnt = cv.take<int32_t>((size_t)n * K * 2);
    const size_t o_work = cv.take<int32_t>(L);
    const size_t zero_bytes = cv.off;
    const size_t o_depth = cv.take<int32_t>(n), o_loff = cv.take<int32_t>(L + 1), o_lint = cv.take<int32_t>(L);
    const size_t o_lnodes = cv.take<int32_t>(n), o_ar = cv.take<int2>(n);
    const size_t o_anc = cv.take<int32_t>(std::max<size_t>(1, (size_t)n * max_depth)), o_node = cv.take<int4>(n);
    const size_t o_sel = cv.take<int32_t>(n);
    const size_t o_arena = cv.take<uint32_t>((size_t)n * WH);
    // level sizes are known on the device only: the step-count buffer is sized for n nodes (its
    // chunks beyond a level's pairs return at once)
    const int steps_cap = steps_cap_for(ctx, n, K, cam->W, cam->H, MIG_MODE_MARGINAL);
    const size_t o_steps = cv.take<char>(steps_region_bytes(steps_cap, WH));
    char *dev = nullptr;
    st = ctx_workspace(ctx, cv.off, (void **)&dev);
    if (st != MIG_OK) return st;
    MIG_CUDA_TRY(cudaMemsetAsync(dev, 0, zero_bytes, ctx->stream));
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
    timed_launch(ctx, kProfPlan, [&] { launch_plan(dp, ctx->stream); });
    LevelParams p = level_params(m, cam, ctx);
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
    p.max_anc = std::max(1, max_depth);
    p.steps = steps_cap ? (uint16_t *)(dev + o_steps) : nullptr;
    p.vctr = steps_counter((uint16_t *)(dev + o_steps), steps_cap, WH);
    p.steps_cap = steps_cap;
    const int cap = ctx->num_sms * 16;
    const int count_cap = ctx->num_sms * std::min(ctx->count_ctas, std::max(1, (int)ctx->tiles.ctas_per_sm));
    const int sel_grid = std::max(1, std::min((n + 127) / 128, 1024));
    for (int d = 0; d < L; ++d) {
        p.lvl = d;
        launch_level_count_timed(ctx, p, n, count_cap);
        timed_launch(ctx, kProfSelect, [&] { launch_select(p, sel_grid, ctx->stream); });
        timed_launch(ctx, kProfRender, [&] { launch_render(p, cap, ctx->stream); });
    }
    MIG_CUDA_TRY(cudaGetLastError());
    return MIG_OK;
}

}  // extern "C"
