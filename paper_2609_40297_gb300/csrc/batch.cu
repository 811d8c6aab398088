// Batched evaluation of many independent trees in one persistent launch (Sec. IV-C per tree).
//
// Each tree level is a chain of segments (batch.h): per chunk of whole nodes a cast segment and a
// per-node voxel segment (the owned-voxel count, voxitems.cuh), then a render segment. Warps take
// item numbers from one atomic counter; a segment's items are numbered only once it is ready (its
// predecessor complete), so warps only ever receive ready work. The warp that finishes a segment's
// last item activates its successor; the one that finishes a level's last voxel segment first
// selects the level's yaws. Every wait is bounded by a time limit; a wait that runs out sets an
// abort flag, all warps leave, and the host returns MIG_ETIMEOUT.
//
// The host packs the plans of all trees into one upload, launches the persistent kernel and
// downloads all outputs; the sequence is captured once into a CUDA graph and replayed while the
// batch keeps the same shape.
#include <cuda/atomic>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <memory>

#include "batch.h"
#include "dev_path.cuh"
#include "kernels.h"
#include "voxcount.h"
#include "voxitems.cuh"

namespace mig {
namespace {

using namespace dev;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}


__device__ __forceinline__ int load_relaxed_i(const int *p) {
    return cuda::atomic_ref<const int, cuda::thread_scope_device>(*p).load(cuda::memory_order_relaxed);
}

__device__ __forceinline__ unsigned long long load_relaxed_u64(const unsigned long long *p) {
    return cuda::atomic_ref<const unsigned long long, cuda::thread_scope_device>(*p).load(cuda::memory_order_relaxed);
}

__device__ __forceinline__ void store_release(int *p, int v) {
    cuda::atomic_ref<int, cuda::thread_scope_device>(*p).store(v, cuda::memory_order_release);
}

constexpr unsigned long long kActItemsMask = (1ull << 40) - 1;

// Appends a ready segment to the activation log and gives it the next item numbers.
__device__ void activate(const BatchParams &bp, int seg) {
    const int items = bp.segs[seg].items;
    if (bp.trace) bp.trace[2 * (size_t)seg] = global_ns();
    const unsigned long long old = atomicAdd(bp.act, (1ull << 40) | (unsigned long long)items);
    const int pos = (int)(old >> 40);
    bp.log[pos] = make_int2((int)(old & kActItemsMask), seg);
    __threadfence();
    store_release(bp.log_valid + pos, 1);
}

__device__ __forceinline__ bool timed_out(const BatchParams &bp, unsigned long long &deadline) {
    if (deadline == 0) deadline = global_ns() + bp.timeout_ns;
    if (global_ns() > deadline) {
        atomicExch(bp.status + 1, 1);
        atomicExch(bp.status, 1);
        return true;
    }
    return false;
}

constexpr int kBatchWarps = 8;

#ifndef MIG_BATCH_MINB
#define MIG_BATCH_MINB 3
#endif
// Dynamic shared memory per warp: a copy of the current tree's yaw rows (the per-node items read
// them for every voxel; 12 ints and 9 floats per yaw), then bp.max_anc ancestor records.
constexpr size_t kBatchYawBytes = (size_t)kNodeMaxK * (12 * sizeof(int) + 9 * sizeof(float));
__global__ void __launch_bounds__(kBatchWarps * 32, MIG_BATCH_MINB) batch_kernel(const BatchParams bp) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ NodeWarp s_nw[kBatchWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *s_yi = reinterpret_cast<int *>(s_dyn + warp * kBatchYawBytes);
    float *s_yf = reinterpret_cast<float *>(s_dyn + warp * kBatchYawBytes + (size_t)kNodeMaxK * 12 * sizeof(int));
    int yaw_tree = -1;  // whose yaw rows the warp's copies hold
    AncRec *anc = reinterpret_cast<AncRec *>(s_dyn + kBatchWarps * kBatchYawBytes) + warp * bp.max_anc;
    NodeWarp &Q = s_nw[warp];
    for (int t = lane; t < 2 * kNodeMaxK; t += 32) Q.cnt[t] = 0;
    __syncwarp();
    if (bp.trace && blockIdx.x == 0 && threadIdx.x == 0) bp.trace[2 * (size_t)bp.n_segs_total] = global_ns();
    int pos = 0;                       // (lane 0) activation-log entry of this warp's previous item
    int anc_tree = -1, anc_node = -1;  // whose ancestor records `anc` holds
    int na = 0;
    NodeStats nst;
    uint32_t st_rays = 0, st_fine = 0, st_skip = 0;
    for (;;) {
        // lane 0 takes the next item number, waits (bounded) until it is activated, finds its
        // activation-log entry with relaxed loads, then one acquire fence orders this warp's
        // reads after the dependencies' writes; the result is broadcast to the warp
        int seg = -1, local = 0;
        if (lane == 0) {
            const long long g = load_relaxed_i(bp.status) ? LLONG_MAX
                                                          : (long long)atomicAdd((unsigned long long *)bp.work, 1ull);
            if (g < bp.total_items) {
                unsigned long long deadline = 0, a = 0;
                bool ok = true;
                unsigned nap = 128;  // exponential backoff keeps idle warps off the memory system
                for (;;) {
                    a = load_relaxed_u64(bp.act);
                    if ((long long)(a & kActItemsMask) > g) break;
                    if (load_relaxed_i(bp.status) || timed_out(bp, deadline)) {
                        ok = false;
                        break;
                    }
                    __nanosleep(nap);
                    nap = min(nap * 2, 8192u);
                }
                int lo = pos, hi = (int)(a >> 40) - 1;
                while (ok && lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    while (!load_relaxed_i(bp.log_valid + mid))
                        if (load_relaxed_i(bp.status) || timed_out(bp, deadline)) {
                            ok = false;
                            break;
                        }
                    if (ok) {
                        if ((long long)load_relaxed_i(&bp.log[mid].x) <= g) lo = mid;
                        else hi = mid - 1;
                    }
                }
                while (ok && !load_relaxed_i(bp.log_valid + lo))
                    if (load_relaxed_i(bp.status) || timed_out(bp, deadline)) ok = false;
                if (ok) {
                    cuda::atomic_thread_fence(cuda::memory_order_acquire, cuda::thread_scope_device);
                    pos = lo;
                    seg = load_relaxed_i(&bp.log[lo].y);
                    local = (int)(g - load_relaxed_i(&bp.log[lo].x));
                } else {
                    seg = -2;
                }
            }
        }
        seg = __shfl_sync(0xffffffffu, seg, 0);
        local = __shfl_sync(0xffffffffu, local, 0);
        __syncwarp();
        if (seg < 0) break;
        const SegInfo sg = bp.segs[seg];
        const LevelParams &p = bp.trees[sg.tree].p;
        const int l0 = p.level_off[sg.level];
        const size_t WH = (size_t)p.W * p.H;
        if (sg.kind == kSegCast) {  // kBatchCastTiles consecutive tiles of one pair
            const int tx = (p.W + kCastTileW - 1) / kCastTileW, tiles = tx * ((p.H + kCastTileH - 1) / kCastTileH);
            const int ipp = (tiles + kBatchCastTiles - 1) / kBatchCastTiles;
            const int ql = local / ipp, t0 = (local - ql * ipp) * kBatchCastTiles;
            const uint8_t *bocc = p.grid.g + bocc_offset(p.grid.nx, p.grid.ny, p.grid.nz);
            const uint8_t *sbocc = p.grid.g + sbocc_offset(p.grid.nx, p.grid.ny, p.grid.nz);
            for (int tile = t0; tile < min(tiles, t0 + kBatchCastTiles); ++tile)
                cast_item<false>(p, bocc, sbocc, l0, sg.q0 + ql, tile, tx, p.steps + (size_t)ql * WH, lane, st_rays,
                                 st_fine, st_skip);
        } else if (sg.kind == kSegVoxel) {
            // the per-node item of the chunk's nodes, numbered as in the per-level kernel: groups of
            // nodes whose step counts fit in L2 together, each node's slices and row blocks
            const int K = p.K;
            const int nb0 = sg.q0 / K, nn = (sg.q1 - sg.q0) / K;
            const int yb_n = node_row_blocks(p.Tq);
            const int per_node = (2 * ((int)(p.Tq >> 16) + 2) + 1) * yb_n;
            const int grp = (int)max((size_t)1, min((size_t)nn, kStepsGroupBytes / ((size_t)K * WH * sizeof(uint16_t))));
            const int g = local / (grp * per_node), r = local - g * grp * per_node;
            const int gsz = min(grp, nn - g * grp);
            const int rzy = r / gsz, ln = g * grp + r % gsz;
            const int rank = rzy / yb_n, rb = rzy - rank * yb_n;
            const int n = p.level_nodes[l0 + nb0 + ln];
            NodeSlice S;
            if (node_slice(p, n, rank, rb, yb_n, S)) {
                if (sg.tree != anc_tree || n != anc_node) {
                    na = node_ancestors(p, n, anc, lane);
                    anc_tree = sg.tree;
                    anc_node = n;
                }
                if (sg.tree != yaw_tree) {
                    __syncwarp();
                    for (int t = lane; t < 12 * K; t += 32) s_yi[t] = p.yawtab[t];
                    for (int t = lane; t < 9 * K; t += 32) s_yf[t] = p.yawf[t];
                    __syncwarp();
                    yaw_tree = sg.tree;
                }
                node_run<false>(p, S, s_yi, s_yf, p.steps + (size_t)ln * K * WH, Q, anc, na, lane, nst);
                node_flush(p, n, Q, lane);  // before the item counts as done
            }
        } else {
            const int groups = (int)((WH + 31) >> 5);
            const int li = local / groups;
            const int pix = (local - li * groups) * 32 + lane;
            if (pix < (int)WH) {
                const int n = p.level_nodes[l0 + li];
                render_pixel(p, n, p.node[n], pix % p.W, pix / p.W);
            }
        }
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence();
            last = atomicSub(bp.seg_left + seg, 1) == 1;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {  // every item of the segment is done
            if (bp.trace && lane == 0) bp.trace[2 * (size_t)seg + 1] = global_ns();
            __threadfence();
            if (sg.select) {  // the level's last voxel segment: select its yaws
                const int L = p.level_off[sg.level + 1] - l0;
                for (int i = lane; i < L; i += 32) select_node(p, p.level_nodes[l0 + i]);
                __threadfence();
                __syncwarp();
            }
            if (lane == 0) {
                if (sg.next >= 0) {
                    activate(bp, sg.next);
                } else {  // the tree is done: the next waiting tree starts
                    const int i = atomicAdd(bp.pending_next, 1);
                    if (i < bp.n_pending) activate(bp, bp.pending[i]);
                }
            }
        }
    }
}

}  // namespace

size_t batch_dyn_smem(int max_anc) {
    return (size_t)kBatchWarps * (kBatchYawBytes + (size_t)std::max(1, max_anc) * sizeof(AncRec));
}

void launch_batch(const BatchParams &bp, int grid, cudaStream_t s) {
    batch_kernel<<<grid, kBatchWarps * 32, batch_dyn_smem(bp.max_anc), s>>>(bp);
}

int batch_ctas_per_sm() {
    int a = 0;
    const size_t smem = batch_dyn_smem(MIG_MAX_DEPTH);  // the worst case
    cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, batch_kernel, kBatchWarps * 32, batch_dyn_smem(16));
    cudaGetLastError();
    return std::max(1, a);
}

}  // namespace mig

using namespace mig;

namespace {
struct GraphKey {
    BatchParams bp;
    void *host;
    size_t up, zero_start, zero, down_start, down, status;
    int grid;
};
}  // namespace

struct mig_ctx::Batch {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    GraphKey key;  // shape of the captured graph
    int ctas = 0;
    uint64_t replays = 0, captures = 0;
    std::vector<mig_trace_rec> trace;  // last traced launch
    // stream-chain engine: stream pool, fork/join events, its own captured graph
    static constexpr size_t kPool = 16;
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t sexec = nullptr;
    cudaGraph_t sgraph = nullptr;
    std::vector<char> skey;
    Batch() { std::memset(&key, 0, sizeof(key)); }
};

namespace {

// Step-count buffer of each tree of a persistent launch: its largest level's (one cast and one voxel
// segment per level keep every tree's chain of segments short), at most 1 GiB per tree and, scaled
// down evenly, 24 GiB per launch; smaller buffers split levels into chunks that run one after another.
#ifndef MIG_BATCH_TREE_STEPS
#define MIG_BATCH_TREE_STEPS (1ull << 30)
#endif
constexpr size_t kBatchTreeStepsBytes = MIG_BATCH_TREE_STEPS;
constexpr size_t kBatchStepsBytes = (size_t)24 << 30;
// Trees in flight at once: the others wait, in order of decreasing work, until one finishes (fewer
// trees interleave their items, so each tree's level chain waits less behind the others').
#ifndef MIG_BATCH_IN_FLIGHT
#define MIG_BATCH_IN_FLIGHT 16
#endif
constexpr int kBatchInFlight = MIG_BATCH_IN_FLIGHT;

struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    }
};

mig_status batch_run(mig_ctx *ctx, std::vector<BatchItem> &items) {
    const int T = (int)items.size();
    if (T > kBatchMaxTrees) return fail(MIG_EINVAL, "batch_run: too many trees for one launch");
    // ---- per tree: whole nodes per chunk, as many as its step-count buffer holds (at least one)
    std::vector<int> chunk_nodes(T);
    for (int t = 0; t < T; ++t) {
        const BatchItem &it = items[t];
        int Lmax = 1;
        for (int d = it.level_lo; d <= it.level_hi; ++d)
            Lmax = std::max(Lmax, it.plan.level_off[d + 1] - it.plan.level_off[d]);
        const size_t node_bytes = (size_t)it.cam->K * it.cam->W * it.cam->H * sizeof(uint16_t);
        chunk_nodes[t] = (int)std::max<size_t>(1, std::min<size_t>((size_t)Lmax, kBatchTreeStepsBytes / node_bytes));
    }
    {
        size_t total_steps = 0;
        for (int t = 0; t < T; ++t)
            total_steps += (size_t)chunk_nodes[t] * items[t].cam->K * items[t].cam->W * items[t].cam->H * sizeof(uint16_t);
        if (total_steps > kBatchStepsBytes) {
            const double f = (double)kBatchStepsBytes / (double)total_steps;
            for (int t = 0; t < T; ++t) chunk_nodes[t] = std::max(1, (int)(chunk_nodes[t] * f));
        }
    }
    // ---- segments, tree by tree in level order: per chunk a cast and a voxel segment, then the
    // level's render segment (if it has internal nodes); each segment's successor is the next one
    // of its tree (the last voxel segment of a level selects the yaws first)
    std::vector<SegInfo> segs;
    std::vector<int> first_seg(T, -1);
    long long total = 0;
    for (int t = 0; t < T; ++t) {
        const BatchItem &it = items[t];
        const int K = it.cam->K, W = it.cam->W, H = it.cam->H;
        const int cast_tiles = ((W + kCastTileW - 1) / kCastTileW) * ((H + kCastTileH - 1) / kCastTileH);
        const int cast_ipp = (cast_tiles + kBatchCastTiles - 1) / kBatchCastTiles;  // cast items per pair
        const int per_node = (2 * ((int)(range_q16(it.sensor.range_m, it.map->voxel) >> 16) + 2) + 1) *
                             node_row_blocks(range_q16(it.sensor.range_m, it.map->voxel));
        const int groups = (W * H + 31) / 32;  // 32-pixel render items
        for (int d = it.level_lo; d <= it.level_hi; ++d) {
            const int Ld = it.plan.level_off[d + 1] - it.plan.level_off[d];
            if (first_seg[t] < 0) first_seg[t] = (int)segs.size();
            for (int n0 = 0; n0 < Ld; n0 += chunk_nodes[t]) {
                const int nc = std::min(chunk_nodes[t], Ld - n0);
                const int q0 = n0 * K, q1 = (n0 + nc) * K;
                segs.push_back(SegInfo{t, d, kSegCast, (q1 - q0) * cast_ipp, q0, q1, (int)segs.size() + 1, 0});
                segs.push_back(SegInfo{t, d, kSegVoxel, nc * per_node, q0, q1, (int)segs.size() + 1, n0 + nc == Ld});
            }
            if (it.plan.level_int[d] > 0)
                segs.push_back(SegInfo{t, d, kSegRender, it.plan.level_int[d] * groups, 0, 0, (int)segs.size() + 1, 0});
        }
        if (first_seg[t] >= 0) segs.back().next = -1;
    }
    std::vector<int> seg_left(segs.size());
    for (size_t e = 0; e < segs.size(); ++e) {
        seg_left[e] = segs[e].items;
        total += segs[e].items;
    }
    if (ctx->batch_debug_stall) {
        // test hook: one segment can never complete, so the waits behind it must run out
        for (int t = 0; t < T; ++t)
            if (first_seg[t] >= 0 && segs[first_seg[t]].next >= 0) {
                seg_left[first_seg[t]] += 1;
                break;
            }
    }
    // the first segment of each tree is ready from the start; the trees with the most work first
    std::vector<int2> log0;
    long long act_items = 0;
    std::vector<int> by_work(T);
    for (int t = 0; t < T; ++t) by_work[t] = t;
    std::stable_sort(by_work.begin(), by_work.end(), [&](int a, int b) {
        return (long long)items[a].plan.n * items[a].cam->K * items[a].cam->W * items[a].cam->H >
               (long long)items[b].plan.n * items[b].cam->K * items[b].cam->W * items[b].cam->H;
    });
    std::vector<int> pending;
    for (int t : by_work) {
        if (first_seg[t] < 0) continue;
        if ((int)log0.size() >= kBatchInFlight) {
            pending.push_back(first_seg[t]);
            continue;
        }
        log0.push_back(make_int2((int)act_items, first_seg[t]));
        act_items += segs[first_seg[t]].items;
    }
    if (total >= ((long long)1 << 31)) return fail(MIG_EINVAL, "tree_eval_batch: more than 2^31 work items in one batch");
    const int log_cap = std::max<int>(1, (int)segs.size());
    Carve cv;
    const size_t o_segs = cv.take(sizeof(SegInfo) * std::max<size_t>(1, segs.size()));
    const size_t o_left = cv.take(4 * std::max<size_t>(1, segs.size()));
    const size_t o_pend = cv.take(4 * std::max<size_t>(1, pending.size())), o_pnext = cv.take(4);
    const size_t o_act = cv.take(8), o_work = cv.take(8);
    const size_t o_log = cv.take(8 * (size_t)log_cap), o_valid = cv.take(4 * (size_t)log_cap);
    struct TreeOff {
        size_t node, ar, anc, loff, lint, lnodes, cnt, sel, out, arena, steps;
    };
    std::vector<TreeOff> to(T);
    for (int t = 0; t < T; ++t) {
        const HostPlan &pl = items[t].plan;
        const int n = pl.n, L = pl.max_depth + 1;
        to[t].node = cv.take(16 * (size_t)n);
        to[t].ar = cv.take(8 * (size_t)n);
        to[t].anc = cv.take(4 * (size_t)std::max(1, pl.total_anc));
        to[t].loff = cv.take(4 * (size_t)(L + 1));
        to[t].lint = cv.take(4 * (size_t)L);
        to[t].lnodes = cv.take(4 * (size_t)n);
    }
    const size_t up_bytes = cv.off;
    const size_t zero_start = cv.off;
    for (int t = 0; t < T; ++t) to[t].cnt = cv.take(8 * (size_t)items[t].plan.n * items[t].cam->K);
    const size_t zero_bytes = cv.off - zero_start;
    const size_t down_start = cv.off;
    const size_t o_status = cv.take(64);
    const bool tracing = ctx->batch_trace;
    const size_t o_trace = cv.take(8 * (2 * segs.size() + 1));
    for (int t = 0; t < T; ++t) to[t].out = cv.take(12 * (size_t)items[t].plan.n);
    const size_t down_bytes = cv.off - down_start;
    for (int t = 0; t < T; ++t) {
        to[t].sel = cv.take(4 * (size_t)items[t].plan.n);
        to[t].arena = cv.take(4 * (size_t)std::max(1, items[t].plan.n_internal) * items[t].cam->W * items[t].cam->H);
        to[t].steps = cv.take((size_t)chunk_nodes[t] * items[t].cam->K * items[t].cam->W * items[t].cam->H * sizeof(uint16_t));
    }
    char *dev = nullptr;
    mig_status st = ctx_workspace(ctx, cv.off, (void **)&dev);
    if (st != MIG_OK) return st;
    char *host = nullptr;
    st = ctx_pinned(ctx, std::max(up_bytes, down_bytes) + 256, (void **)&host);
    if (st != MIG_OK) return st;
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    // ---- host image of the upload region
    std::memset(host, 0, up_bytes);
    std::unique_ptr<BatchParams> bpp(new BatchParams());
    std::memset(bpp.get(), 0, sizeof(BatchParams));
    BatchParams &bp = *bpp;
    BatchTree *bt = bp.trees;
    for (int t = 0; t < T; ++t) {
        const BatchItem &it = items[t];
        const HostPlan &pl = it.plan;
        const int n = pl.n, L = pl.max_depth + 1;
        std::memcpy(host + to[t].node, pl.node.data(), 16 * (size_t)n);
        int2 *ar = (int2 *)(host + to[t].ar);
        for (int i = 0; i < n; ++i) ar[i] = make_int2(pl.anc_off[i], pl.depth[i]);
        if (pl.total_anc) std::memcpy(host + to[t].anc, pl.anc.data(), 4 * (size_t)pl.total_anc);
        std::memcpy(host + to[t].loff, pl.level_off.data(), 4 * (size_t)(L + 1));
        std::memcpy(host + to[t].lint, pl.level_int.data(), 4 * (size_t)L);
        std::memcpy(host + to[t].lnodes, pl.level_nodes.data(), 4 * (size_t)n);
        LevelParams p{};
        mig_map *m = it.map;
        p.grid = GridView{m->d_grid, m->nx, m->ny, m->nz, m->nbx, m->nby};
        p.body = (const int4 *)it.cam->d_body;
        p.yawtab = it.cam->d_yaw;
        p.yawf = it.cam->d_yawf;
        set_band(p, it.cam);
        p.W = it.cam->W;
        p.H = it.cam->H;
        p.K = it.cam->K;
        p.Tq = range_q16(it.sensor.range_m, m->voxel);
        p.level_off = (const int32_t *)(dev + to[t].loff);
        p.level_int = (const int32_t *)(dev + to[t].lint);
        p.level_nodes = (const int32_t *)(dev + to[t].lnodes);
        p.node = (const int4 *)(dev + to[t].node);
        p.anc_range = (const int2 *)(dev + to[t].ar);
        p.anc = (const int32_t *)(dev + to[t].anc);
        p.sel_yaw = (int32_t *)(dev + to[t].sel);
        p.arena = (uint32_t *)(dev + to[t].arena);
        p.cnt = (int32_t *)(dev + to[t].cnt);
        p.work = nullptr;
        p.out_abs = (int32_t *)(dev + to[t].out);
        p.out_marg = p.out_abs + n;
        p.out_yaw = p.out_abs + 2 * (size_t)n;
        p.mode = it.mode;
        p.lvl = 0;
        p.stats = nullptr;
        p.max_anc = std::max(1, pl.max_depth);
        p.steps = (uint16_t *)(dev + to[t].steps);
        p.steps_cap = chunk_nodes[t] * p.K;
        bt[t].p = p;
    }
    if (!segs.empty()) {
        std::memcpy(host + o_segs, segs.data(), sizeof(SegInfo) * segs.size());
        std::memcpy(host + o_left, seg_left.data(), 4 * segs.size());
    }
    if (!pending.empty()) std::memcpy(host + o_pend, pending.data(), 4 * pending.size());
    *(int *)(host + o_pnext) = 0;
    *(unsigned long long *)(host + o_act) = ((unsigned long long)log0.size() << 40) | (unsigned long long)act_items;
    *(long long *)(host + o_work) = 0;
    if (!log0.empty()) std::memcpy(host + o_log, log0.data(), 8 * log0.size());
    for (size_t e = 0; e < log0.size(); ++e) ((int *)(host + o_valid))[e] = 1;
    bp.segs = (const SegInfo *)(dev + o_segs);
    bp.total_items = total;
    bp.act = (unsigned long long *)(dev + o_act);
    bp.log = (int2 *)(dev + o_log);
    bp.log_valid = (int *)(dev + o_valid);
    bp.work = (long long *)(dev + o_work);
    bp.seg_left = (int *)(dev + o_left);
    bp.pending = (const int *)(dev + o_pend);
    bp.pending_next = (int *)(dev + o_pnext);
    bp.n_pending = (int)pending.size();
    bp.status = (int *)(dev + o_status);
    bp.trace = tracing ? (unsigned long long *)(dev + o_trace) : nullptr;
    bp.n_segs_total = (int)segs.size();
    bp.max_anc = 1;
    for (int t = 0; t < T; ++t) bp.max_anc = std::max(bp.max_anc, items[t].plan.max_depth);
    bp.timeout_ns = (unsigned long long)ctx->batch_timeout_ns;
    if (!ctx->batch) ctx->batch = new mig_ctx::Batch();
    mig_ctx::Batch *B = ctx->batch;
    if (!B->ctas) B->ctas = batch_ctas_per_sm();
    const int grid = ctx->num_sms * std::min(B->ctas, std::max(1, (int)ctx->tiles.ctas_per_sm));
    // ---- graph: upload, zero counts and status, persistent kernel, download. The captured
    // graph bakes in the kernel parameters and the copy sizes: replay only while all match.
    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.bp = bp;
    key.host = host;
    key.up = up_bytes;
    key.zero_start = zero_start;
    key.zero = zero_bytes;
    key.down_start = down_start;
    key.down = down_bytes;
    key.status = o_status;
    key.grid = grid;
    cudaStream_t s = ctx->stream;
    auto enqueue = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dev, host, up_bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && zero_bytes) e = cudaMemsetAsync(dev + zero_start, 0, zero_bytes, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(dev + o_status, 0, 64, s);
        if (e != cudaSuccess) return e;
        timed_launch(ctx, kProfBatch, [&] { launch_batch(bp, grid, s); });
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(host, dev + down_start, down_bytes, cudaMemcpyDeviceToHost, s);
        return e;
    };
    const bool same = B->exec && std::memcmp(&B->key, &key, sizeof(key)) == 0 && !ctx->prof.on && !tracing;
    if (same) {
        // the kernel's parameters (bp) are baked into the graph; they depend only on the key
        MIG_CUDA_TRY(cudaGraphLaunch(B->exec, s));
        B->replays++;
    } else if (!ctx->prof.on && !tracing && s != nullptr) {
        if (B->exec) {
            cudaGraphExecDestroy(B->exec);
            cudaGraphDestroy(B->graph);
            B->exec = nullptr;
            B->graph = nullptr;
        }
        MIG_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue();
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(MIG_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        MIG_CUDA_TRY(cudaGraphInstantiate(&B->exec, g, 0));
        B->graph = g;
        std::memcpy(&B->key, &key, sizeof(key));
        B->captures++;
        MIG_CUDA_TRY(cudaGraphLaunch(B->exec, s));
    } else {
        // profiling or the legacy default stream (which cannot be captured): plain launches
        cudaError_t e = enqueue();
        if (e != cudaSuccess) return fail(MIG_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    }
    if (tracing) {
        std::vector<unsigned long long> tr(2 * segs.size() + 1);
        MIG_CUDA_TRY(cudaMemcpyAsync(tr.data(), dev + o_trace, 8 * tr.size(), cudaMemcpyDeviceToHost, s));
        MIG_CUDA_TRY(cudaStreamSynchronize(s));
        const unsigned long long t0 = tr[2 * segs.size()];
        B->trace.clear();
        for (size_t i = 0; i < segs.size(); ++i) {
            if (!segs[i].items) continue;
            mig_trace_rec rec{};
            rec.tree = segs[i].tree;
            rec.level = segs[i].level;
            rec.phase = segs[i].kind;
            rec.items = segs[i].items;
            rec.activated_us = tr[2 * i] ? (double)(long long)(tr[2 * i] - t0) * 1e-3 : 0.0;
            rec.done_us = tr[2 * i + 1] ? (double)(long long)(tr[2 * i + 1] - t0) * 1e-3 : -1.0;
            B->trace.push_back(rec);
        }
    }
    MIG_CUDA_TRY(cudaStreamSynchronize(s));
    const int *status = (const int *)host;
    if (status[1]) return fail(MIG_ETIMEOUT, "batch: a device-side dependency wait ran out (no output is valid)");
    if (status[0]) return fail(MIG_ECUDA, "batch: aborted");
    for (int t = 0; t < T; ++t) {
        const int n = items[t].plan.n;
        const int32_t *o = (const int32_t *)(host + (to[t].out - down_start));
        if (items[t].out_abs) std::memcpy(items[t].out_abs, o, 4 * (size_t)n);
        if (items[t].out_marg) std::memcpy(items[t].out_marg, o + n, 4 * (size_t)n);
        if (items[t].out_yaw) std::memcpy(items[t].out_yaw, o + 2 * (size_t)n, 4 * (size_t)n);
    }
    return MIG_OK;
}

// Alternative engine: each tree's chain of per-level kernels (count, select, render per level,
// Sec. IV-C) on its own stream of a pool, forked from and joined back into the context stream,
// captured into one CUDA graph. Kernels of different trees run concurrently and fill each
// other's level tails and launch gaps, while every kernel keeps its parameters in the constant
// bank (the per-level kernels' code).
mig_status batch_run_streams(mig_ctx *ctx, std::vector<BatchItem> &items) {
    const int T = (int)items.size();
    const mig_tile_config tc = ctx->tiles;
    Carve cv;
    struct TreeOff {
        size_t node, ar, anc, loff, lint, lnodes, cnt, work, sel, out, arena, pcnt;
    };
    std::vector<TreeOff> to(T);
    for (int t = 0; t < T; ++t) {
        const HostPlan &pl = items[t].plan;
        const int n = pl.n, L = pl.max_depth + 1;
        to[t].node = cv.take(16 * (size_t)n);
        to[t].ar = cv.take(8 * (size_t)n);
        to[t].anc = cv.take(4 * (size_t)std::max(1, pl.total_anc));
        to[t].loff = cv.take(4 * (size_t)(L + 1));
        to[t].lint = cv.take(4 * (size_t)L);
        to[t].lnodes = cv.take(4 * (size_t)n);
    }
    const size_t up_bytes = cv.off, zero_start = cv.off;
    for (int t = 0; t < T; ++t) {
        to[t].cnt = cv.take(8 * (size_t)items[t].plan.n * items[t].cam->K);
        to[t].work = cv.take(4 * (size_t)(items[t].plan.max_depth + 1));
    }
    const size_t zero_bytes = cv.off - zero_start, down_start = cv.off;
    for (int t = 0; t < T; ++t) to[t].out = cv.take(12 * (size_t)items[t].plan.n);
    const size_t down_bytes = cv.off - down_start;
    for (int t = 0; t < T; ++t) {
        to[t].sel = cv.take(4 * (size_t)items[t].plan.n);
        to[t].arena = cv.take(4 * (size_t)std::max(1, items[t].plan.n_internal) * items[t].cam->W * items[t].cam->H);
        to[t].pcnt = items[t].mode == MIG_MODE_PANORAMIC ? cv.take(8 * (size_t)items[t].plan.n * items[t].cam->pano_A) : 0;
    }
    // longest trees first, round-robin over the stream pool; the trees of one stream run one after
    // another, so each stream has one step-count buffer for the owned-voxel count
    const int S = std::min(T, (int)mig_ctx::Batch::kPool);
    std::vector<int> order(T);
    for (int t = 0; t < T; ++t) order[t] = t;
    std::sort(order.begin(), order.end(), [&](int a, int c) { return items[a].plan.n > items[c].plan.n; });
    std::vector<int> steps_cap(T, 0);
    std::vector<size_t> stream_steps(S, 0);
    for (int oi = 0; oi < T; ++oi) {
        const int t = order[oi];
        const HostPlan &pl = items[t].plan;
        int Lmax = 1;
        for (int d = 0; d <= pl.max_depth; ++d) Lmax = std::max(Lmax, pl.level_off[d + 1] - pl.level_off[d]);
        steps_cap[t] = steps_cap_for(ctx, Lmax, items[t].cam->K, items[t].cam->W, items[t].cam->H, items[t].mode);
        stream_steps[oi % S] = std::max(stream_steps[oi % S],
                                        steps_region_bytes(steps_cap[t], (size_t)items[t].cam->W * items[t].cam->H));
    }
    std::vector<size_t> o_steps(S);
    for (int i = 0; i < S; ++i) o_steps[i] = cv.take(std::max<size_t>(stream_steps[i], 1));
    char *dev = nullptr;
    mig_status st = ctx_workspace(ctx, cv.off, (void **)&dev);
    if (st != MIG_OK) return st;
    char *host = nullptr;
    st = ctx_pinned(ctx, std::max(up_bytes, down_bytes) + 256, (void **)&host);
    if (st != MIG_OK) return st;
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    std::memset(host, 0, up_bytes);
    std::vector<LevelParams> lp(T);
    for (int t = 0; t < T; ++t) {
        const BatchItem &it = items[t];
        const HostPlan &pl = it.plan;
        const int n = pl.n, L = pl.max_depth + 1;
        std::memcpy(host + to[t].node, pl.node.data(), 16 * (size_t)n);
        int2 *ar = (int2 *)(host + to[t].ar);
        for (int i = 0; i < n; ++i) ar[i] = make_int2(pl.anc_off[i], pl.depth[i]);
        if (pl.total_anc) std::memcpy(host + to[t].anc, pl.anc.data(), 4 * (size_t)pl.total_anc);
        std::memcpy(host + to[t].loff, pl.level_off.data(), 4 * (size_t)(L + 1));
        std::memcpy(host + to[t].lint, pl.level_int.data(), 4 * (size_t)L);
        std::memcpy(host + to[t].lnodes, pl.level_nodes.data(), 4 * (size_t)n);
        LevelParams p{};
        mig_map *m = it.map;
        p.grid = GridView{m->d_grid, m->nx, m->ny, m->nz, m->nbx, m->nby};
        p.body = (const int4 *)it.cam->d_body;
        p.yawtab = it.cam->d_yaw;
        p.yawf = it.cam->d_yawf;
        set_band(p, it.cam);
        p.W = it.cam->W;
        p.H = it.cam->H;
        p.K = it.cam->K;
        p.Tq = range_q16(it.sensor.range_m, m->voxel);
        p.tile_w = tc.tile_w;
        p.tile_h = tc.tile_h;
        p.tiles_x = (p.W + tc.tile_w - 1) / tc.tile_w;
        p.tiles = p.tiles_x * ((p.H + tc.tile_h - 1) / tc.tile_h);
        p.level_off = (const int32_t *)(dev + to[t].loff);
        p.level_int = (const int32_t *)(dev + to[t].lint);
        p.level_nodes = (const int32_t *)(dev + to[t].lnodes);
        p.node = (const int4 *)(dev + to[t].node);
        p.anc_range = (const int2 *)(dev + to[t].ar);
        p.anc = (const int32_t *)(dev + to[t].anc);
        p.sel_yaw = (int32_t *)(dev + to[t].sel);
        p.arena = (uint32_t *)(dev + to[t].arena);
        p.cnt = (int32_t *)(dev + to[t].cnt);
        p.work = (int32_t *)(dev + to[t].work);
        p.out_abs = (int32_t *)(dev + to[t].out);
        p.out_marg = p.out_abs + n;
        p.out_yaw = p.out_abs + 2 * (size_t)n;
        p.mode = it.mode;
        p.max_anc = std::max(1, pl.max_depth);
        if (it.mode == MIG_MODE_PANORAMIC) set_pano_params(p, it.cam, (int32_t *)(dev + to[t].pcnt));
        lp[t] = p;
    }
    for (int oi = 0; oi < T; ++oi) {
        const int t = order[oi];
        lp[t].steps = steps_cap[t] ? (uint16_t *)(dev + o_steps[oi % S]) : nullptr;
        lp[t].voxel_pass = ctx->voxel_pass;
        lp[t].vctr = steps_counter((uint16_t *)(dev + o_steps[oi % S]), steps_cap[t],
                                   (size_t)items[t].cam->W * items[t].cam->H);
        lp[t].steps_cap = steps_cap[t];
    }
    if (!ctx->batch) ctx->batch = new mig_ctx::Batch();
    mig_ctx::Batch *B = ctx->batch;
    for (int i = (int)B->pool.size(); i < S; ++i) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        MIG_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        MIG_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        B->pool.push_back(s);
        B->join.push_back(e);
    }
    if (!B->fork) MIG_CUDA_TRY(cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming));
    cudaStream_t s0 = ctx->stream;
    const int cap = ctx->num_sms * 16;
    const int count_cap = ctx->num_sms * std::min(ctx->count_ctas, std::max(1, (int)ctx->tiles.ctas_per_sm));
    auto enqueue = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dev, host, up_bytes, cudaMemcpyHostToDevice, s0);
        if (e == cudaSuccess && zero_bytes) e = cudaMemsetAsync(dev + zero_start, 0, zero_bytes, s0);
        if (e == cudaSuccess) e = cudaEventRecord(B->fork, s0);
        for (int i = 0; i < S && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(B->pool[i], B->fork, 0);
        for (int oi = 0; oi < T && e == cudaSuccess; ++oi) {
            const int t = order[oi];
            cudaStream_t s = B->pool[oi % S];
            LevelParams p = lp[t];
            const HostPlan &pl = items[t].plan;
            const int rt = render_tiles(p.W, p.H);
            for (int d = 0; d <= pl.max_depth; ++d) {
                p.lvl = d;
                const int Ld = pl.level_off[d + 1] - pl.level_off[d];
                launch_level_count(ctx, p, Ld, count_cap, s);
                launch_select(p, std::max(1, std::min((Ld + 127) / 128, 1024)), s);
                if (pl.level_int[d] > 0) launch_render(p, std::min(pl.level_int[d] * rt, cap), s);
            }
            e = cudaGetLastError();
        }
        for (int i = 0; i < S && e == cudaSuccess; ++i) e = cudaEventRecord(B->join[i], B->pool[i]);
        for (int i = 0; i < S && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(s0, B->join[i], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(host, dev + down_start, down_bytes, cudaMemcpyDeviceToHost, s0);
        return e;
    };
    // graph key: every kernel parameter and copy is fixed by the trees' parameters and sizes
    std::vector<char> key(sizeof(LevelParams) * T + 64 + 8 * T);
    std::memcpy(key.data(), lp.data(), sizeof(LevelParams) * T);
    size_t extra[8] = {(size_t)host, up_bytes, zero_bytes, down_bytes, (size_t)S, (size_t)count_cap, 0, 0};
    std::memcpy(key.data() + sizeof(LevelParams) * T, extra, sizeof(extra));
    for (int t = 0; t < T; ++t) {
        const long long md = items[t].plan.max_depth;
        std::memcpy(key.data() + sizeof(LevelParams) * T + 64 + 8 * t, &md, 8);
    }
    const bool same = B->sexec && B->skey == key && !ctx->prof.on;
    if (same) {
        MIG_CUDA_TRY(cudaGraphLaunch(B->sexec, s0));
        B->replays++;
    } else if (!ctx->prof.on && s0 != nullptr) {
        if (B->sexec) {
            cudaGraphExecDestroy(B->sexec);
            cudaGraphDestroy(B->sgraph);
            B->sexec = nullptr;
            B->sgraph = nullptr;
        }
        MIG_CUDA_TRY(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue();
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(s0, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(MIG_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        MIG_CUDA_TRY(cudaGraphInstantiate(&B->sexec, g, 0));
        B->sgraph = g;
        B->skey = key;
        B->captures++;
        MIG_CUDA_TRY(cudaGraphLaunch(B->sexec, s0));
    } else {
        cudaError_t e = enqueue();
        if (e != cudaSuccess) return fail(MIG_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    }
    MIG_CUDA_TRY(cudaStreamSynchronize(s0));
    for (int t = 0; t < T; ++t) {
        const int n = items[t].plan.n;
        const int32_t *o = (const int32_t *)(host + (to[t].out - down_start));
        if (items[t].out_abs) std::memcpy(items[t].out_abs, o, 4 * (size_t)n);
        if (items[t].out_marg) std::memcpy(items[t].out_marg, o + n, 4 * (size_t)n);
        if (items[t].out_yaw) std::memcpy(items[t].out_yaw, o + 2 * (size_t)n, 4 * (size_t)n);
    }
    return MIG_OK;
}

}  // namespace

// Destroys the captured batch graphs of both engines. Called before the context frees a buffer
// that their copy nodes reference (the device workspace, the pinned staging buffer): a graph must
// not outlive memory it copies to or from, even when a later allocation returns the same address
// and the replay key would match again.
extern "C" void mig_batch_drop_graphs(mig_ctx *ctx) {
    if (!ctx || !ctx->batch) return;
    mig_ctx::Batch *B = ctx->batch;
    if (!B->exec && !B->sexec) return;
    cudaStreamSynchronize(ctx->stream);  // every batch launch is on the context stream
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->sexec) cudaGraphExecDestroy(B->sexec);
    if (B->sgraph) cudaGraphDestroy(B->sgraph);
    B->exec = B->sexec = nullptr;
    B->graph = B->sgraph = nullptr;
    std::memset(&B->key, 0, sizeof(B->key));
    B->skey.clear();
}

extern "C" void mig_batch_release(mig_ctx *ctx) {
    if (!ctx || !ctx->batch) return;
    if (ctx->batch->exec) cudaGraphExecDestroy(ctx->batch->exec);
    if (ctx->batch->graph) cudaGraphDestroy(ctx->batch->graph);
    if (ctx->batch->sexec) cudaGraphExecDestroy(ctx->batch->sexec);
    if (ctx->batch->sgraph) cudaGraphDestroy(ctx->batch->sgraph);
    for (auto s : ctx->batch->pool) cudaStreamDestroy(s);
    for (auto e : ctx->batch->join) cudaEventDestroy(e);
    if (ctx->batch->fork) cudaEventDestroy(ctx->batch->fork);
    delete ctx->batch;
    ctx->batch = nullptr;
}

extern "C" mig_status mig_tree_eval_batch(mig_ctx *ctx, int n_trees, const mig_tree_desc *trees) {
    NvtxRange range("mig_tree_eval_batch");
    if (!ctx || n_trees < 0 || (n_trees > 0 && !trees)) return fail(MIG_EINVAL, "tree_eval_batch: invalid argument");
    std::vector<BatchItem> items;
    items.reserve(n_trees);
    for (int t = 0; t < n_trees; ++t) {
        const mig_tree_desc &d = trees[t];
        if (!d.map || d.map->ctx != ctx) return fail(MIG_EINVAL, "tree_eval_batch: tree " + std::to_string(t) + " has no map of this context");
        if (d.mode < 0 || d.mode > MIG_MODE_PANORAMIC) return fail(MIG_EINVAL, "tree_eval_batch: unknown mode");
        if (d.n_nodes < 0) return fail(MIG_EINVAL, "tree_eval_batch: negative node count");
        if (d.n_nodes > 0 && (!d.abs_gain || !d.marg_gain || !d.best_yaw))
            return fail(MIG_EINVAL, "tree_eval_batch: output array is NULL");
        mig_status st = sensor_check(d.sensor, d.map->voxel);
        if (st != MIG_OK) return st;
        if (d.n_nodes == 0) continue;
        BatchItem it;
        it.map = d.map;
        it.n = d.n_nodes;
        it.parent = d.parent;
        it.pos = d.pos_m;
        it.sensor = d.sensor;
        it.mode = d.mode;
        it.out_abs = d.abs_gain;
        it.out_marg = d.marg_gain;
        it.out_yaw = d.best_yaw;
        const int dims[3] = {d.map->nx, d.map->ny, d.map->nz};
        st = plan_build(d.n_nodes, d.parent, d.pos_m, d.map->origin, d.map->voxel, dims, it.plan);
        if (st != MIG_OK) return st;
        it.level_lo = 0;
        it.level_hi = it.plan.max_depth;
        items.push_back(std::move(it));
    }
    if (items.empty()) return MIG_OK;
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaSetDevice(ctx->device));
    // the persistent kernel runs the per-node owned-voxel pass of the sample modes; batches holding an
    // interval or panoramic tree, a sensor outside the per-node pass (more than kNodeMaxK yaws, a
    // frustum without an azimuth window) or a context counting ray by ray run on the stream chains
    bool per_level_kernels = ctx->ray_count;
    for (auto &it : items) {
        mig_status st = ctx_camera(ctx, it.sensor, &it.cam);
        if (st != MIG_OK) return st;
        if (it.mode == MIG_MODE_PANORAMIC && (st = ctx_pano(ctx, it.cam)) != MIG_OK) return st;
        per_level_kernels |= it.mode == MIG_MODE_INTERVAL || it.mode == MIG_MODE_PANORAMIC;
        per_level_kernels |= !(it.cam->az_half > 0.f && it.cam->K <= kNodeMaxK);
    }
    if (ctx->tiles.engine == 1 || per_level_kernels) return batch_run_streams(ctx, items);
    if ((int)items.size() <= kBatchMaxTrees) return batch_run(ctx, items);
    for (size_t s = 0; s < items.size(); s += kBatchMaxTrees) {  // one persistent launch per group
        std::vector<BatchItem> part(std::make_move_iterator(items.begin() + s),
                                    std::make_move_iterator(items.begin() + std::min(items.size(), s + kBatchMaxTrees)));
        mig_status st = batch_run(ctx, part);
        if (st != MIG_OK) return st;
    }
    return MIG_OK;
}

extern "C" mig_status mig_batch_set_tiles(mig_ctx *ctx, const mig_tile_config *cfg) {
    if (!ctx || !cfg) return fail(MIG_EINVAL, "batch_set_tiles: NULL argument");
    if (cfg->tile_w < 1 || cfg->tile_h < 1 || cfg->tile_w * cfg->tile_h > 4096 || (cfg->tile_w * cfg->tile_h) % 32 != 0 ||
        cfg->ctas_per_sm < 1 || cfg->ctas_per_sm > 32 || cfg->engine < 0 || cfg->engine > 1)
        return fail(MIG_EINVAL, "batch_set_tiles: a tile holds a multiple of 32 rays, at most 4096; engine 0 or 1");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->tiles = *cfg;
    return MIG_OK;
}

extern "C" mig_status mig_batch_get_tiles(mig_ctx *ctx, mig_tile_config *cfg) {
    if (!ctx || !cfg) return fail(MIG_EINVAL, "batch_get_tiles: NULL argument");
    *cfg = ctx->tiles;
    return MIG_OK;
}

extern "C" mig_status mig_batch_set_timeout(mig_ctx *ctx, int64_t timeout_us, int debug_stall) {
    if (!ctx || timeout_us < 1) return fail(MIG_EINVAL, "batch_set_timeout: invalid argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->batch_timeout_ns = timeout_us * 1000;
    ctx->batch_debug_stall = debug_stall != 0;
    return MIG_OK;
}

extern "C" mig_status mig_batch_graph_stats(mig_ctx *ctx, uint64_t *captures, uint64_t *replays) {
    if (!ctx) return fail(MIG_EINVAL, "batch_graph_stats: NULL argument");
    if (captures) *captures = ctx->batch ? ctx->batch->captures : 0;
    if (replays) *replays = ctx->batch ? ctx->batch->replays : 0;
    return MIG_OK;
}

extern "C" mig_status mig_batch_trace(mig_ctx *ctx, int enable) {
    if (!ctx) return fail(MIG_EINVAL, "batch_trace: NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->batch_trace = enable != 0;
    return MIG_OK;
}

extern "C" mig_status mig_batch_trace_read(mig_ctx *ctx, mig_trace_rec *out, int cap, int *n) {
    if (!ctx || !n || (cap > 0 && !out)) return fail(MIG_EINVAL, "batch_trace_read: NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    const int m = ctx->batch ? (int)ctx->batch->trace.size() : 0;
    *n = m;
    for (int i = 0; i < std::min(m, cap); ++i) out[i] = ctx->batch->trace[i];
    return MIG_OK;
}

// Autotuner: times each candidate configuration on a sample batch (wall clock around the
// synchronous batch call, best of `reps` after one warm-up), checks that every candidate gives
// the same results, and leaves the fastest configuration set on the context.
extern "C" mig_status mig_autotune(mig_ctx *ctx, int n_trees, const mig_tree_desc *sample, int n_cands,
                                   const mig_tile_config *cands, int reps, mig_tile_config *best, double *ms_out) {
    if (!ctx || n_trees < 1 || !sample || n_cands < 1 || !cands || reps < 1)
        return fail(MIG_EINVAL, "autotune: invalid argument");
    const mig_tile_config keep = ctx->tiles;
    std::vector<std::vector<int32_t>> ref;
    std::vector<mig_tree_desc> d(sample, sample + n_trees);
    std::vector<std::vector<int32_t>> buf(n_trees);
    for (int t = 0; t < n_trees; ++t) {
        buf[t].assign(3 * (size_t)std::max(0, d[t].n_nodes), 0);
        d[t].abs_gain = buf[t].data();
        d[t].marg_gain = buf[t].data() + d[t].n_nodes;
        d[t].best_yaw = buf[t].data() + 2 * (size_t)d[t].n_nodes;
    }
    int best_i = -1;
    double best_ms = 1e300;
    for (int c = 0; c < n_cands; ++c) {
        mig_status st = mig_batch_set_tiles(ctx, &cands[c]);
        if (st != MIG_OK) {
            ctx->tiles = keep;
            return st;
        }
        st = mig_tree_eval_batch(ctx, n_trees, d.data());  // warm-up (camera tables, graph capture)
        if (st != MIG_OK) {
            ctx->tiles = keep;
            return st;
        }
        double ms = 1e300;
        for (int r = 0; r < reps; ++r) {
            const auto t0 = std::chrono::steady_clock::now();
            st = mig_tree_eval_batch(ctx, n_trees, d.data());
            const auto t1 = std::chrono::steady_clock::now();
            if (st != MIG_OK) {
                ctx->tiles = keep;
                return st;
            }
            ms = std::min(ms, std::chrono::duration<double, std::milli>(t1 - t0).count());
        }
        if (ref.empty()) {
            ref = buf;
        } else if (ref != buf) {
            ctx->tiles = keep;
            return fail(MIG_ECUDA, "autotune: candidate " + std::to_string(c) + " changed the results");
        }
        if (ms_out) ms_out[c] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best_i = c;
        }
    }
    ctx->tiles = cands[best_i];
    if (best) *best = cands[best_i];
    return MIG_OK;
}
