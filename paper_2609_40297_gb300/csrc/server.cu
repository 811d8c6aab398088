// Serving loop: continuous batching of replanning requests on one GPU.
//
// Requests (a tree, a map, a sensor) are submitted from any thread and wait in a FIFO queue. A
// worker thread admits queued requests while the number in flight and their device memory
// (plan, counts, depth-buffer arena) fit the limits, then runs steps: in one step every request
// in flight evaluates one tree level (Sec. IV-C: count, yaw select, depth render), each on its own
// stream of a pool, all forked from and joined into the context stream, so the levels of many
// requests run on the device together. A request that has finished its deepest level copies its
// results out and leaves; new requests join at the next step.
//
// Map updates go through the same queue: an update is applied when it reaches the front, i.e.
// after every earlier request was admitted. If a request in flight still reads the map's grid,
// the update goes to a copy (copy-on-write), so every request sees the map exactly as it was when
// it was submitted and its results equal a lone mig_tree_eval on that map.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>

#include "kernels.h"
#include "voxcount.h"
#include "mig_impl.h"

using namespace mig;
using Clock = std::chrono::steady_clock;

namespace {

struct Grid {  // one device grid buffer of a map, shared by the requests that read it
    mig_map *map = nullptr;
    uint8_t *ptr = nullptr;
    size_t bytes = 0;
    int users = 0;       // requests in flight reading this buffer
    bool retired = false;  // replaced by a newer version: free when users reach 0
};

struct Request {
    uint64_t ticket = 0;
    mig_map *map = nullptr;
    mig_sensor sensor{};
    int mode = 0;
    HostPlan plan;
    int steps_cap = 0;  // owned-voxel count: (node, yaw) pairs per chunk (0 = ray by ray)
    int32_t *out_abs = nullptr, *out_marg = nullptr, *out_yaw = nullptr;
    const Camera *cam = nullptr;
    // device state while in flight
    char *dev = nullptr;
    size_t dev_bytes = 0;
    LevelParams p{};
    std::shared_ptr<Grid> grid;
    int level = 0;
    // timing (since submit)
    Clock::time_point t_submit, t_admit, t_start, t_done;
    mig_status status = MIG_EBUSY;
};

struct Update {
    mig_map *map;
    int x0, y0, z0, dx, dy, dz;
    std::vector<uint8_t> voxels;
};

struct Entry {  // queue entry: a request or a map update
    std::unique_ptr<Request> req;
    std::unique_ptr<Update> upd;
};

struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    }
};

}  // namespace

struct mig_server {
    mig_ctx *ctx = nullptr;
    size_t budget = 0, in_use = 0;
    // device bytes of superseded map grids that requests in flight still read (copy-on-write
    // snapshots), and the largest in_use + snapshot bytes seen; written by the worker only
    std::atomic<size_t> snap_bytes{0}, peak_bytes{0};
    int max_inflight = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Entry> queue;
    std::vector<std::unique_ptr<Request>> inflight;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> done;
    std::map<mig_map *, std::shared_ptr<Grid>> grids;  // current grid buffer of each map
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    char *pinned = nullptr;
    size_t pinned_bytes = 0;
    std::string fatal;
};

namespace {

size_t request_bytes(const Request &r) {
    const HostPlan &pl = r.plan;
    const size_t n = pl.n, L = pl.max_depth + 1, K = r.sensor.yaw_bins;
    const size_t WH = (size_t)r.sensor.width * r.sensor.height;
    Carve cv;
    cv.take(16 * n);
    cv.take(8 * n);
    cv.take(4 * std::max(1, pl.total_anc));
    cv.take(4 * (L + 1));
    cv.take(4 * L);
    cv.take(4 * n);
    cv.take(8 * n * K);
    cv.take(4 * L);
    cv.take(12 * n);
    cv.take(4 * n);
    cv.take(4 * std::max(1, pl.n_internal) * WH);
    cv.take(steps_region_bytes(r.steps_cap, WH));
    return cv.off;
}

std::shared_ptr<Grid> current_grid(mig_server *s, mig_map *m) {
    auto it = s->grids.find(m);
    if (it != s->grids.end() && it->second->ptr == m->d_grid) return it->second;
    auto g = std::make_shared<Grid>();
    g->map = m;
    g->ptr = m->d_grid;
    g->bytes = m->grid_bytes;
    s->grids[m] = g;
    return g;
}

// Admission (worker thread, ctx->mu held): device region, plan upload, zeroed counters.
mig_status admit(mig_server *s, Request &r) {
    mig_ctx *ctx = s->ctx;
    const HostPlan &pl = r.plan;
    const int n = pl.n, L = pl.max_depth + 1, K = r.sensor.yaw_bins;
    const size_t WH = (size_t)r.sensor.width * r.sensor.height;
    mig_status st = ctx_camera(ctx, r.sensor, &r.cam);
    if (st != MIG_OK) return st;
    const bool pano = r.mode == MIG_MODE_PANORAMIC;
    if (pano && (st = ctx_pano(ctx, r.cam)) != MIG_OK) return st;
    Carve cv;
    const size_t o_node = cv.take(16 * (size_t)n), o_ar = cv.take(8 * (size_t)n);
    const size_t o_anc = cv.take(4 * (size_t)std::max(1, pl.total_anc)), o_loff = cv.take(4 * (size_t)(L + 1));
    const size_t o_lint = cv.take(4 * (size_t)L), o_lnodes = cv.take(4 * (size_t)n);
    const size_t up = cv.off;
    const size_t o_cnt = cv.take(8 * (size_t)n * K), o_work = cv.take(4 * (size_t)L);
    const size_t zero_end = cv.off;
    const size_t o_out = cv.take(12 * (size_t)n), o_sel = cv.take(4 * (size_t)n);
    const size_t o_arena = cv.take(4 * (size_t)std::max(1, pl.n_internal) * WH);
    const size_t o_pcnt = pano ? cv.take(8 * (size_t)n * r.cam->pano_A) : 0;
    const size_t o_steps = cv.take(steps_region_bytes(r.steps_cap, WH));
    r.dev_bytes = cv.off;
    r.dev = (char *)ctx->alloc.alloc(r.dev_bytes, ctx->stream);
    if (!r.dev) return fail(MIG_ENOMEM, "server: request allocation failed");
    if (s->pinned_bytes < up) {
        if (s->pinned) {
            cudaStreamSynchronize(ctx->stream);
            cudaFreeHost(s->pinned);
        }
        s->pinned = nullptr;
        s->pinned_bytes = 0;
        if (cudaHostAlloc((void **)&s->pinned, std::max(up, (size_t)1 << 20), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return fail(MIG_ENOMEM, "server: pinned staging allocation failed");
        }
        s->pinned_bytes = std::max(up, (size_t)1 << 20);
    }
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));  // the staging buffer may feed an earlier copy
    char *h = s->pinned;
    std::memcpy(h + o_node, pl.node.data(), 16 * (size_t)n);
    int2 *ar = (int2 *)(h + o_ar);
    for (int i = 0; i < n; ++i) ar[i] = make_int2(pl.anc_off[i], pl.depth[i]);
    if (pl.total_anc) std::memcpy(h + o_anc, pl.anc.data(), 4 * (size_t)pl.total_anc);
    std::memcpy(h + o_loff, pl.level_off.data(), 4 * (size_t)(L + 1));
    std::memcpy(h + o_lint, pl.level_int.data(), 4 * (size_t)L);
    std::memcpy(h + o_lnodes, pl.level_nodes.data(), 4 * (size_t)n);
    MIG_CUDA_TRY(cudaMemcpyAsync(r.dev, h, up, cudaMemcpyHostToDevice, ctx->stream));
    MIG_CUDA_TRY(cudaMemsetAsync(r.dev + up, 0, zero_end - up, ctx->stream));
    r.grid = current_grid(s, r.map);
    r.grid->users++;
    LevelParams &p = r.p;
    mig_map *m = r.map;
    p.grid = GridView{r.grid->ptr, m->nx, m->ny, m->nz, m->nbx, m->nby};
    p.body = (const int4 *)r.cam->d_body;
    p.yawtab = r.cam->d_yaw;
    p.yawf = r.cam->d_yawf;
    set_band(p, r.cam);
    p.W = r.cam->W;
    p.H = r.cam->H;
    p.K = r.cam->K;
    p.Tq = range_q16(r.sensor.range_m, m->voxel);
    p.tile_w = ctx->tiles.tile_w;
    p.tile_h = ctx->tiles.tile_h;
    p.tiles_x = (p.W + p.tile_w - 1) / p.tile_w;
    p.tiles = p.tiles_x * ((p.H + p.tile_h - 1) / p.tile_h);
    p.level_off = (const int32_t *)(r.dev + o_loff);
    p.level_int = (const int32_t *)(r.dev + o_lint);
    p.level_nodes = (const int32_t *)(r.dev + o_lnodes);
    p.node = (const int4 *)(r.dev + o_node);
    p.anc_range = (const int2 *)(r.dev + o_ar);
    p.anc = (const int32_t *)(r.dev + o_anc);
    p.sel_yaw = (int32_t *)(r.dev + o_sel);
    p.arena = (uint32_t *)(r.dev + o_arena);
    p.cnt = (int32_t *)(r.dev + o_cnt);
    p.work = (int32_t *)(r.dev + o_work);
    p.out_abs = (int32_t *)(r.dev + o_out);
    p.out_marg = p.out_abs + n;
    p.out_yaw = p.out_abs + 2 * (size_t)n;
    p.mode = r.mode;
    p.stats = nullptr;
    p.max_anc = std::max(1, pl.max_depth);
    if (pano) set_pano_params(p, r.cam, (int32_t *)(r.dev + o_pcnt));
    p.steps = r.steps_cap ? (uint16_t *)(r.dev + o_steps) : nullptr;
    p.vctr = steps_counter((uint16_t *)(r.dev + o_steps), r.steps_cap, WH);
    p.voxel_pass = ctx->voxel_pass;
    p.steps_cap = r.steps_cap;
    r.level = 0;
    return MIG_OK;
}

void note_peak(mig_server *s) {
    const size_t now = s->in_use + s->snap_bytes.load();
    if (now > s->peak_bytes.load()) s->peak_bytes.store(now);
}

void release_grid(mig_server *s, Request &r) {
    if (!r.grid) return;
    r.grid->users--;
    if (r.grid->retired && r.grid->users == 0) {
        s->ctx->alloc.free(r.grid->ptr, r.grid->bytes, s->ctx->stream);
        r.grid->ptr = nullptr;
        s->snap_bytes -= r.grid->bytes;
    }
    r.grid.reset();
}

// Would applying an update to map m now copy its grid (requests in flight still read it)?
bool update_needs_copy(mig_server *s, mig_map *m) {
    auto it = s->grids.find(m);
    return it != s->grids.end() && it->second->ptr == m->d_grid && it->second->users > 0;
}

// Applies a map update (worker thread, ctx->mu held): copy-on-write if requests read the grid.
mig_status apply_update(mig_server *s, Update &u) {
    mig_ctx *ctx = s->ctx;
    mig_map *m = u.map;
    auto g = current_grid(s, m);
    if (g->users > 0) {
        uint8_t *fresh = (uint8_t *)ctx->alloc.alloc(m->grid_bytes, ctx->stream);
        if (!fresh) return fail(MIG_ENOMEM, "server: map copy allocation failed");
        MIG_CUDA_TRY(cudaMemcpyAsync(fresh, m->d_grid, m->grid_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        g->retired = true;  // freed by the last request that reads it
        s->snap_bytes += g->bytes;
        m->d_grid = fresh;
        current_grid(s, m);
    }
    const size_t nv = u.voxels.size();
    uint8_t *tmp = (uint8_t *)ctx->alloc.alloc(nv, ctx->stream);
    if (!tmp) return fail(MIG_ENOMEM, "server: update staging allocation failed");
    MIG_CUDA_TRY(cudaMemcpyAsync(tmp, u.voxels.data(), nv, cudaMemcpyHostToDevice, ctx->stream));
    launch_map_scatter(m->d_grid, m->nx, m->ny, m->nz, m->nbx, m->nby, tmp, u.x0, u.y0, u.z0, u.dx, u.dy, u.dz, ctx->stream);
    MIG_CUDA_TRY(cudaGetLastError());
    ctx->alloc.free(tmp, nv, ctx->stream);
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));  // the host voxels are freed with the update
    m->version++;
    return MIG_OK;
}

// One step: every request in flight evaluates its current level.
mig_status run_step(mig_server *s) {
    mig_ctx *ctx = s->ctx;
    const int R = (int)s->inflight.size();
    const int S = std::min<int>(R, (int)s->pool.size());
    cudaStream_t s0 = ctx->stream;
    MIG_CUDA_TRY(cudaEventRecord(s->fork, s0));
    for (int i = 0; i < S; ++i) MIG_CUDA_TRY(cudaStreamWaitEvent(s->pool[i], s->fork, 0));
    const int cap = ctx->num_sms * 16, count_cap = ctx->num_sms * ctx->count_ctas;
    const Clock::time_point now = Clock::now();
    for (int i = 0; i < R; ++i) {
        Request &r = *s->inflight[i];
        if (r.level == 0) r.t_start = now;
        cudaStream_t st = s->pool[i % S];
        LevelParams p = r.p;
        p.lvl = r.level;
        const HostPlan &pl = r.plan;
        const int d = r.level;
        const int Ld = pl.level_off[d + 1] - pl.level_off[d];
        launch_level_count(ctx, p, Ld, count_cap, st);
        launch_select(p, std::max(1, std::min((Ld + 127) / 128, 1024)), st);
        if (pl.level_int[d] > 0 && d < pl.max_depth) launch_render(p, std::min(pl.level_int[d] * render_tiles(p.W, p.H), cap), st);
    }
    MIG_CUDA_TRY(cudaGetLastError());
    for (int i = 0; i < S; ++i) {
        MIG_CUDA_TRY(cudaEventRecord(s->join[i], s->pool[i]));
        MIG_CUDA_TRY(cudaStreamWaitEvent(s0, s->join[i], 0));
    }
    MIG_CUDA_TRY(cudaStreamSynchronize(s0));
    return MIG_OK;
}

void worker_main(mig_server *s) {
    mig_ctx *ctx = s->ctx;
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // admission: FIFO; updates apply when they reach the front
        while (!s->queue.empty()) {
            Entry &e = s->queue.front();
            if (e.upd) {
                // a copy-on-write snapshot counts against the budget too: while it would not fit,
                // the update (and every entry behind it) waits for requests in flight to finish
                if (!s->inflight.empty() && update_needs_copy(s, e.upd->map) &&
                    s->in_use + s->snap_bytes.load() + e.upd->map->grid_bytes > s->budget)
                    break;
                lk.unlock();
                mig_status st;
                {
                    std::lock_guard<std::mutex> cl(ctx->mu);
                    st = apply_update(s, *e.upd);
                }
                lk.lock();
                if (st != MIG_OK) s->fatal = mig_last_error();
                note_peak(s);
                s->queue.pop_front();
                continue;
            }
            Request &r = *e.req;
            const size_t need = request_bytes(r);
            if ((int)s->inflight.size() >= s->max_inflight) break;
            // map snapshots held for requests in flight count against the budget; a lone request
            // always runs
            if (!s->inflight.empty() && s->in_use + s->snap_bytes.load() + need > s->budget) break;
            std::unique_ptr<Request> rq = std::move(e.req);
            s->queue.pop_front();
            lk.unlock();
            mig_status st;
            {
                std::lock_guard<std::mutex> cl(ctx->mu);
                st = admit(s, *rq);
            }
            lk.lock();
            rq->t_admit = Clock::now();
            if (st != MIG_OK) {
                rq->status = st;
                if (rq->dev) ctx->alloc.free(rq->dev, rq->dev_bytes, ctx->stream);
                rq->dev = nullptr;
                s->done[rq->ticket] = std::move(rq);
                s->cv_done.notify_all();
                continue;
            }
            s->in_use += rq->dev_bytes;
            note_peak(s);
            s->inflight.push_back(std::move(rq));
        }
        if (s->inflight.empty()) {
            if (s->stop && s->queue.empty()) break;
            s->cv_work.wait(lk);
            continue;
        }
        lk.unlock();
        mig_status st;
        std::vector<std::unique_ptr<Request>> finished;
        {
            std::lock_guard<std::mutex> cl(ctx->mu);
            st = run_step(s);
            // requests past their deepest level: results out, device state freed
            for (auto &rp : s->inflight) {
                Request &r = *rp;
                if (st == MIG_OK && r.level < r.plan.max_depth) {
                    r.level++;
                    continue;
                }
                if (st == MIG_OK) {
                    const int n = r.plan.n;
                    std::vector<int32_t> out(3 * (size_t)n);
                    if (cudaMemcpy(out.data(), r.p.out_abs, 12 * (size_t)n, cudaMemcpyDeviceToHost) == cudaSuccess) {
                        std::memcpy(r.out_abs, out.data(), 4 * (size_t)n);
                        std::memcpy(r.out_marg, out.data() + n, 4 * (size_t)n);
                        std::memcpy(r.out_yaw, out.data() + 2 * (size_t)n, 4 * (size_t)n);
                        r.status = MIG_OK;
                    } else {
                        cudaGetLastError();
                        r.status = MIG_ECUDA;
                    }
                } else {
                    r.status = st;
                }
                ctx->alloc.free(r.dev, r.dev_bytes, ctx->stream);
                r.dev = nullptr;
                release_grid(s, r);
                r.t_done = Clock::now();
                rp->level = -1;
            }
        }
        lk.lock();
        for (auto &rp : s->inflight) {
            if (rp->level != -1) continue;
            s->in_use -= rp->dev_bytes;
            s->done[rp->ticket] = std::move(rp);
        }
        s->inflight.erase(std::remove_if(s->inflight.begin(), s->inflight.end(),
                                         [](const std::unique_ptr<Request> &p) { return !p; }),
                          s->inflight.end());
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" mig_status mig_server_create(mig_ctx *ctx, size_t arena_budget_bytes, int max_inflight, mig_server **out) {
    if (!ctx || !out || max_inflight < 1 || max_inflight > 4096) return fail(MIG_EINVAL, "server_create: invalid argument");
    *out = nullptr;
    auto s = std::make_unique<mig_server>();
    s->ctx = ctx;
    s->budget = arena_budget_bytes;
    s->max_inflight = max_inflight;
    {
        std::lock_guard<std::mutex> cl(ctx->mu);
        MIG_CUDA_TRY(cudaSetDevice(ctx->device));
        const int S = std::min(max_inflight, 16);
        for (int i = 0; i < S; ++i) {
            cudaStream_t st = nullptr;
            cudaEvent_t e = nullptr;
            MIG_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            MIG_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            s->pool.push_back(st);
            s->join.push_back(e);
        }
        MIG_CUDA_TRY(cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming));
    }
    mig_server *raw = s.release();
    raw->worker = std::thread(worker_main, raw);
    *out = raw;
    return MIG_OK;
}

extern "C" mig_status mig_server_submit(mig_server *s, const mig_tree_desc *d, uint64_t *ticket) {
    if (!s || !d || !ticket) return fail(MIG_EINVAL, "server_submit: NULL argument");
    if (!d->map || d->map->ctx != s->ctx) return fail(MIG_EINVAL, "server_submit: map of another context");
    if (d->mode < 0 || d->mode > MIG_MODE_PANORAMIC) return fail(MIG_EINVAL, "server_submit: unknown mode");
    if (d->mode == MIG_MODE_PANORAMIC && d->sensor.pitch_deg != 0.0f)
        return fail(MIG_EINVAL, "panoramic mode: the camera must be level (pitch 0)");
    if (d->n_nodes < 1) return fail(MIG_EINVAL, "server_submit: a request needs at least one node");
    if (!d->abs_gain || !d->marg_gain || !d->best_yaw) return fail(MIG_EINVAL, "server_submit: output array is NULL");
    mig_status st = sensor_check(d->sensor, d->map->voxel);
    if (st != MIG_OK) return st;
    auto r = std::make_unique<Request>();
    const int dims[3] = {d->map->nx, d->map->ny, d->map->nz};
    st = plan_build(d->n_nodes, d->parent, d->pos_m, d->map->origin, d->map->voxel, dims, r->plan);
    if (st != MIG_OK) return st;
    r->map = d->map;
    r->sensor = d->sensor;
    r->mode = d->mode;
    {
        int Lmax = 1;
        for (int lv = 0; lv <= r->plan.max_depth; ++lv)
            Lmax = std::max(Lmax, r->plan.level_off[lv + 1] - r->plan.level_off[lv]);
        r->steps_cap = steps_cap_for(s->ctx, Lmax, d->sensor.yaw_bins, d->sensor.width, d->sensor.height, d->mode);
    }
    r->out_abs = d->abs_gain;
    r->out_marg = d->marg_gain;
    r->out_yaw = d->best_yaw;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(MIG_EINVAL, "server_submit: server is shutting down");
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    Entry e;
    e.req = std::move(r);
    s->queue.push_back(std::move(e));
    s->cv_work.notify_one();
    return MIG_OK;
}

extern "C" mig_status mig_server_map_update(mig_server *s, mig_map *m, int x0, int y0, int z0, int dx, int dy, int dz,
                                            const uint8_t *host_voxels) {
    if (!s || !m || !host_voxels || m->ctx != s->ctx) return fail(MIG_EINVAL, "server_map_update: invalid argument");
    if (dx < 1 || dy < 1 || dz < 1 || x0 < 0 || y0 < 0 || z0 < 0 || x0 + dx > m->nx || y0 + dy > m->ny || z0 + dz > m->nz)
        return fail(MIG_EINVAL, "server_map_update: box outside the grid or empty");
    auto u = std::make_unique<Update>();
    u->map = m;
    u->x0 = x0;
    u->y0 = y0;
    u->z0 = z0;
    u->dx = dx;
    u->dy = dy;
    u->dz = dz;
    u->voxels.assign(host_voxels, host_voxels + (size_t)dx * dy * dz);
    for (uint8_t c : u->voxels)
        if (c > 2) return fail(MIG_EINVAL, "server_map_update: voxel code above 2");
    std::lock_guard<std::mutex> lk(s->mu);
    Entry e;
    e.upd = std::move(u);
    s->queue.push_back(std::move(e));
    s->cv_work.notify_one();
    return MIG_OK;
}

extern "C" mig_status mig_server_poll(mig_server *s, uint64_t ticket, int64_t timeout_us) {
    if (!s) return fail(MIG_EINVAL, "server_poll: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = Clock::now() + std::chrono::microseconds(std::max<int64_t>(0, timeout_us));
    for (;;) {
        auto it = s->done.find(ticket);
        if (it != s->done.end()) {
            const mig_status st = it->second->status;
            if (st != MIG_OK) return fail(st, "server: request failed");
            return MIG_OK;
        }
        if (ticket == 0 || ticket >= s->next_ticket) return fail(MIG_ENOTFOUND, "server_poll: unknown ticket");
        if (timeout_us <= 0) return MIG_EBUSY;
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && Clock::now() >= deadline) {
            if (s->done.count(ticket)) continue;
            return fail(MIG_ETIMEOUT, "server_poll: not finished within the timeout");
        }
    }
}

extern "C" mig_status mig_server_timing(mig_server *s, uint64_t ticket, double *admit_us, double *start_us,
                                        double *done_us) {
    if (!s) return fail(MIG_EINVAL, "server_timing: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) return fail(MIG_ENOTFOUND, "server_timing: ticket not finished or unknown");
    const Request &r = *it->second;
    auto us = [&](Clock::time_point t) { return std::chrono::duration<double, std::micro>(t - r.t_submit).count(); };
    if (admit_us) *admit_us = us(r.t_admit);
    if (start_us) *start_us = us(r.t_start);
    if (done_us) *done_us = us(r.t_done);
    return MIG_OK;
}

extern "C" mig_status mig_server_memory(mig_server *s, uint64_t *in_use, uint64_t *snapshots, uint64_t *peak) {
    if (!s) return fail(MIG_EINVAL, "server_memory: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (in_use) *in_use = s->in_use;
    if (snapshots) *snapshots = s->snap_bytes.load();
    if (peak) *peak = s->peak_bytes.load();
    return MIG_OK;
}

extern "C" void mig_server_destroy(mig_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();  // drains the queue and the requests in flight
    mig_ctx *ctx = s->ctx;
    {
        std::lock_guard<std::mutex> cl(ctx->mu);
        cudaSetDevice(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        for (auto &kv : s->grids)
            if (kv.second->retired && kv.second->ptr) ctx->alloc.free(kv.second->ptr, kv.second->bytes, ctx->stream);
        for (auto st : s->pool) cudaStreamDestroy(st);
        for (auto e : s->join) cudaEventDestroy(e);
        if (s->fork) cudaEventDestroy(s->fork);
        if (s->pinned) cudaFreeHost(s->pinned);
    }
    delete s;
}
