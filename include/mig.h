/*
 * mig.h — path-dependent marginal information gain over an RRT planning tree, on one GPU.
 *
 * The method: each tree node n is a candidate viewpoint (position p_n, yaw psi_n) in a voxel
 * map of free / occupied / unknown voxels (Sec. III-A). Its absolute gain counts the unknown
 * voxels visible from it (Eq. 1); its marginal gain counts those that no ancestor on its
 * path already observes (Eq. 2). Previous observations are depth buffers: each node keeps
 * the depth buffer of its selected yaw (Sec. IV-A), and every unknown-voxel sample of a
 * candidate ray is projected into its ancestors' buffers (Eq. 5) and dropped when its depth
 * is smaller than or equal to the stored one (Sec. IV-B). Nodes are evaluated level by level
 * in depth order, nodes and rays of a level in parallel (Sec. IV-C).
 *
 * Conventions (all calls):
 *  - Status codes are returned, never abort. mig_last_error() gives a thread-local message.
 *  - Host pointers are caller-owned and only read/written during the call unless stated.
 *  - Maps, contexts and servers are library-owned objects, destroyed by their _destroy call.
 *  - Gains are integer voxel counts; the volume of Eq. 1 is count * voxel_size^3.
 *  - Depth buffers hold the camera z in Q16.16 voxel units (uint32).
 *  - Grids are x-fastest: index = (z * ny + y) * nx + x, codes 0 unknown, 1 free, 2 occupied.
 *  - World frame z-up; yaw bin k is psi_k = 2 pi k / K counter-clockwise from +x; camera
 *    x right, y down, z forward; pitch positive = nose down; pinhole with principal point at
 *    the image centre and rays through pixel centres (Eq. 5).
 *  - Every result-deciding step is exact integer arithmetic (positions quantised to Q16 voxel
 *    units, ray directions Q30, projection rows Q16, the DDA's crossings compared as exact
 *    rationals), except the interval mode's fixed sequence of correctly rounded single-precision
 *    operations: results are deterministic and identical on every run.
 */
#ifndef MIG_H
#define MIG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MIG_ABI_VERSION 1
#define MIG_MAX_DEPTH 64        /* deepest node (root = 0) */
#define MIG_MAX_DIM 4096        /* voxels per grid axis */
#define MIG_MAX_IMAGE 2048      /* rays (pixels) per image axis */
#define MIG_MAX_YAW_BINS 1024
#define MIG_MAX_RANGE_VOXELS 1024
#define MIG_MAX_PANO_COLUMNS 65536 /* azimuth columns of the panoramic mode */

typedef enum {
    MIG_OK = 0,
    MIG_EINVAL = 1,   /* invalid argument: bad code, tree, sensor, size or position */
    MIG_ENOMEM = 2,   /* device or host allocation failed; nothing leaked */
    MIG_ECUDA = 3,    /* a CUDA call failed (message in mig_last_error) */
    MIG_ETIMEOUT = 4, /* a bounded wait (device queue or poll) ran out */
    MIG_EBUSY = 5,    /* not finished yet (server poll) or object in use */
    MIG_ENOTFOUND = 6 /* unknown ticket */
} mig_status;

typedef struct mig_ctx mig_ctx;
typedef struct mig_map mig_map;
typedef struct mig_server mig_server;

/* Device memory provider. alloc returns device memory of `bytes` usable on `stream`
 * (NULL on failure); free releases it (stream-ordered). NULL allocator = cudaMallocAsync. */
typedef struct mig_allocator {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} mig_allocator;

/* Depth camera (Sec. IV-A, Sec. V): field of view, ray grid = depth-buffer size W x H,
 * maximum range d_max, number of candidate yaws K, and camera pitch. Limits: 0 < fov < 180,
 * 1 <= W, H <= MIG_MAX_IMAGE, 1 <= K <= MIG_MAX_YAW_BINS, -90 <= pitch <= 90,
 * 0 < range / voxel_size <= MIG_MAX_RANGE_VOXELS, focal lengths W/2/tan(hfov/2) < 2^15 - W. */
typedef struct mig_sensor {
    float hfov_deg, vfov_deg;
    int32_t width, height;
    float range_m;
    int32_t yaw_bins;
    float pitch_deg;
} mig_sensor;

/* Gain formulation (Sec. III-B, Sec. V-A): marginal over all ancestors (Eq. 2, the default),
 * single-parent exclusion g_sp, or absolute gain (Eq. 1, no exclusion; yaw = argmax abs).
 * MIG_MODE_INTERVAL is the marginal gain with the paper's screen-space overlap test (Sec. IV-B,
 * Eq. 5-7) in place of the voxel-centre test: per ancestor, the candidate ray is clipped to the
 * valid depth range, projected, clipped to the buffer (Liang-Barsky) and walked pixel by pixel
 * (2D DDA), one inverse-depth sample per visited pixel (Eq. 6); an owned unknown voxel, sampled
 * at the midpoint of the ray's traversal of it, is excluded when it falls in an observed
 * portion of any ancestor.
 * MIG_MODE_PANORAMIC evaluates the yaw set from one 360-degree cast per node instead of one
 * pinhole cast per yaw: A = K * ceil(W 360 / (hfov K)) azimuth wedges ("columns"), each a
 * one-pixel-wide strip camera with the pinhole's H rows; owned unknown voxels are counted per
 * column (owner = the cell containing the voxel centre), excluded by the ancestors' pinhole
 * depth buffers as in the marginal mode, and yaw k's gain is the sum over the
 * round(A hfov / 360) columns centred on its azimuth. The selected yaw's pinhole depth buffer is
 * rendered for the descendants. Its gains differ from the pinhole modes (different ray geometry).
 * Needs pitch 0 and at most MIG_MAX_PANO_COLUMNS columns (else MIG_EINVAL).
 * The mode is chosen per call by mig_tree_eval_ex, and per tree by mig_tree_eval_batch and
 * mig_server_submit (a batch holding an interval or panoramic tree runs on the stream-chain
 * engine); the device-resident entry points and mig_tree_eval_stats evaluate the marginal mode. */
typedef enum {
    MIG_MODE_MARGINAL = 0,
    MIG_MODE_SINGLE_PARENT = 1,
    MIG_MODE_ABSOLUTE = 2,
    MIG_MODE_INTERVAL = 3,
    MIG_MODE_PANORAMIC = 4
} mig_mode;

/* ---------------------------------------------------------------------------------------
 * Context: one GPU, one CUDA stream, one allocator. `stream` is a cudaStream_t (NULL = the
 * legacy default stream). Thread-compatible: one thread at a time per context.
 * Errors: MIG_EINVAL (bad device), MIG_ECUDA, MIG_ENOMEM.
 * --------------------------------------------------------------------------------------- */
mig_status mig_ctx_create(int device, void *stream, const mig_allocator *allocator, mig_ctx **out);
void mig_ctx_destroy(mig_ctx *ctx);
mig_status mig_ctx_set_stream(mig_ctx *ctx, void *stream);
/* Waits for all work on the context's stream; returns MIG_EINVAL if a device-side check of an
 * earlier asynchronous call (mig_tree_eval_device) failed since the last sync. */
mig_status mig_ctx_sync(mig_ctx *ctx);

/* ---------------------------------------------------------------------------------------
 * Voxel map (Sec. III-A): nx*ny*nz voxels of edge voxel_size_m, voxel (0,0,0)'s low corner
 * at origin_m. host_voxels: x-fastest codes, copied to the device (NULL = all unknown).
 * The device copy is library-owned, kept resident until mig_map_destroy.
 * Errors: MIG_EINVAL (dims outside [1, MIG_MAX_DIM], voxel_size <= 0, a code > 2).
 * --------------------------------------------------------------------------------------- */
mig_status mig_map_create(mig_ctx *ctx, int nx, int ny, int nz, float voxel_size_m, const float origin_m[3],
                          const uint8_t *host_voxels, mig_map **out);
/* Overwrites the box [x0,x0+dx) x [y0,y0+dy) x [z0,z0+dz) from host_voxels (x-fastest, dx*dy*dz).
 * Ordered on the context stream after earlier evaluations (they see the old contents).
 * Errors: MIG_EINVAL (box outside the grid, empty box, a code > 2). */
mig_status mig_map_update(mig_map *map, int x0, int y0, int z0, int dx, int dy, int dz,
                          const uint8_t *host_voxels);
/* Reads the whole grid back (x-fastest, nx*ny*nz bytes). */
mig_status mig_map_read(mig_map *map, uint8_t *host_out);
void mig_map_destroy(mig_map *map);

/* Depth-buffer resolution rule of Sec. IV-A: W = ceil(2 d_max tan(hfov/2) / v),
 * H = ceil(2 d_max tan(vfov/2) / v), so that one pixel at range is one voxel. Host only. */
mig_status mig_default_resolution(const mig_sensor *sensor, float voxel_size_m, int32_t *width, int32_t *height);

/* Tree check and depth (Sec. III-B, Sec. IV-C): exactly one root (parent -1), parents in
 * [0, n), no cycles, depth <= MIG_MAX_DEPTH. depth_out (nullable, n) receives each node's
 * depth, max_depth_out (nullable) the largest. Host only, no GPU needed. MIG_EINVAL if invalid. */
mig_status mig_tree_check(int n, const int32_t *parent, int32_t *depth_out, int32_t *max_depth_out);

/* ---------------------------------------------------------------------------------------
 * Tree evaluation, host arrays (Sec. IV-C). parent[n] (-1 = root), pos_m[n*3] world metres.
 * Outputs (host, n each): abs_gain = max over yaws of the absolute count (Eq. 1),
 * marg_gain = marginal count at the selected yaw (Eq. 2), best_yaw = lowest k maximising the
 * marginal count. Synchronous: returns when the outputs are written. Each position must lie
 * inside the grid box. n = 0 is a no-op.
 * Errors: MIG_EINVAL (tree, sensor, positions), MIG_ENOMEM, MIG_ECUDA.
 * --------------------------------------------------------------------------------------- */
mig_status mig_tree_eval(mig_map *map, int n, const int32_t *parent, const float *pos_m, const mig_sensor *sensor,
                         int32_t *abs_gain, int32_t *marg_gain, int32_t *best_yaw);

/* Extended evaluation: a gain mode and optional diagnostic outputs (host, nullable):
 * per-(node, yaw) counts [n][K] and every node's selected depth buffer [n][H][W]. */
typedef struct mig_eval_opts {
    int32_t mode;           /* mig_mode */
    int32_t *counts_abs;    /* n*K or NULL */
    int32_t *counts_marg;   /* n*K or NULL (the mode's exclusion count) */
    uint32_t *depth_buffers;/* n*H*W or NULL: D_n at best_yaw, Q16.16 voxel units */
} mig_eval_opts;
mig_status mig_tree_eval_ex(mig_map *map, int n, const int32_t *parent, const float *pos_m, const mig_sensor *sensor,
                            const mig_eval_opts *opts, int32_t *abs_gain, int32_t *marg_gain, int32_t *best_yaw);

/* Device-resident evaluation: parent, pos_m and the three outputs are DEVICE pointers; the
 * tree is planned on the device; the call only enqueues work on the context stream and
 * returns. max_depth bounds the tree's depth (levels launched = max_depth + 1; a deeper node,
 * a cycle, a second root or an out-of-grid position is flagged on the device, all outputs
 * are then -1 and the next mig_ctx_sync returns MIG_EINVAL).
 * Errors at call time: MIG_EINVAL (sensor, n, max_depth), MIG_ENOMEM, MIG_ECUDA. */
mig_status mig_tree_eval_device(mig_map *map, int n, const int32_t *parent, const float *pos_m,
                                const mig_sensor *sensor, int max_depth, int32_t *abs_gain, int32_t *marg_gain,
                                int32_t *best_yaw);

/* ---------------------------------------------------------------------------------------
 * Path scoring (Sec. III-C): traversal cost c(n) = c(Pa) + ||p_n - p_Pa|| (Eq. 3), objective
 * o(n) = o(Pa) + g(n) exp(-lambda c(n)) (Eq. 4) with g(n) = gain_counts[n] * voxel_size^3 (m^3),
 * and best_node = the lowest index with the largest objective (the branch the planner follows).
 * Double precision. mig_tree_score takes host arrays and returns when done; the _device variant
 * takes device arrays (gain_counts e.g. the marg_gain output of mig_tree_eval_device) and only
 * enqueues on the context stream (a bad parent chain gives best_node = -1 and MIG_EINVAL at the
 * next mig_ctx_sync). Errors: MIG_EINVAL (tree, voxel_size <= 0, lambda < 0), MIG_ENOMEM.
 * --------------------------------------------------------------------------------------- */
mig_status mig_tree_score(mig_ctx *ctx, int n, const int32_t *parent, const float *pos_m, const int32_t *gain_counts,
                          double voxel_size_m, double lambda, double *cost, double *objective, int32_t *best_node);
mig_status mig_tree_score_device(mig_ctx *ctx, int n, const int32_t *parent, const float *pos_m,
                                 const int32_t *gain_counts, double voxel_size_m, double lambda, double *cost,
                                 double *objective, int32_t *best_node);

/* ---------------------------------------------------------------------------------------
 * Allocation-free evaluation. The paper has no counterpart; this entry point serves callers
 * that may not allocate device memory: a planner in a real-time control loop whose policy
 * forbids cudaMalloc after start-up (an allocation can stall or synchronise the device for an
 * unbounded time), or a host framework that owns all device memory through its own pool.
 * Same arguments, device pointers, asynchrony and device-side checks as mig_tree_eval_device,
 * and the same results. It calls no cudaMalloc, cudaFree or other allocating routine: all
 * scratch (camera tables, plan, counters, depth buffers) lives in one static device array of
 * MIG_NOALLOC_SCRATCH_BYTES, held by every GPU that loads the library until the process exits.
 * A tree needs about n * width * height * 4 bytes plus n * (K * 8 + 64 + 4 * max_depth) bytes;
 * a larger request returns MIG_EINVAL with the size in mig_last_error. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and keeps it for the life
 * of the process; do not call cudaDeviceReset on that device afterwards (the array may move).
 * The yaw table travels in kernel parameters, not by a copy from host memory. Every call shares the one
 * array: calls whose work overlaps on the GPU (other streams, other contexts on the same
 * device) race and corrupt each other. It counts with the ray-by-ray kernel (identical results).
 * --------------------------------------------------------------------------------------- */
#define MIG_NOALLOC_SCRATCH_BYTES (64u << 20)
mig_status mig_tree_eval_device_noalloc(mig_map *map, int n, const int32_t *parent, const float *pos_m,
                                        const mig_sensor *sensor, int max_depth, int32_t *abs_gain,
                                        int32_t *marg_gain, int32_t *best_yaw);

/* ---------------------------------------------------------------------------------------
 * Batched evaluation: many independent trees (each on its own map and sensor) in one
 * persistent launch with per-level device work queues, replayed from a captured CUDA graph
 * when the batch's shape repeats. Host arrays as in mig_tree_eval; results are identical to
 * n_trees separate mig_tree_eval calls. Synchronous.
 * Errors: as mig_tree_eval (the first failing tree's status), MIG_ETIMEOUT (a device-side
 * dependency wait ran out; no output is then valid).
 * --------------------------------------------------------------------------------------- */
typedef struct mig_tree_desc {
    mig_map *map;
    int32_t n_nodes;
    const int32_t *parent; /* host, n_nodes */
    const float *pos_m;    /* host, n_nodes*3 */
    mig_sensor sensor;
    int32_t mode;          /* mig_mode */
    int32_t *abs_gain;     /* host outputs, n_nodes each */
    int32_t *marg_gain;
    int32_t *best_yaw;
} mig_tree_desc;
mig_status mig_tree_eval_batch(mig_ctx *ctx, int n_trees, const mig_tree_desc *trees);

/* Tile shape of the batched kernel (chosen by the autotuner; exposed for the tuner and tests). */
typedef struct mig_tile_config {
    int32_t tile_w, tile_h;   /* count pass: pixel rays per warp work item (a multiple of 32, <= 4096) */
    int32_t ctas_per_sm;      /* persistent CTAs per SM */
    int32_t engine;           /* batches: 0 = one persistent dataflow kernel (the sample modes with at
                                 most 64 yaws; other batches use engine 1), 1 = per-tree launch
                                 chains on concurrent streams in one graph */
} mig_tile_config;
mig_status mig_batch_set_tiles(mig_ctx *ctx, const mig_tile_config *cfg);
mig_status mig_batch_get_tiles(mig_ctx *ctx, mig_tile_config *cfg);
/* Autotuner: times each of the n_cands configurations on the sample batch (wall clock around the
 * synchronous call, best of reps after a warm-up), fails with MIG_ECUDA if any candidate changes a
 * result, and leaves the fastest configuration set on the context (also returned in *best;
 * ms_out, nullable, receives n_cands times). The sample's output pointers are not used. */
mig_status mig_autotune(mig_ctx *ctx, int n_trees, const mig_tree_desc *sample, int n_cands,
                        const mig_tile_config *cands, int reps, mig_tile_config *best, double *ms_out);
/* Time limit of every device-side dependency wait of the batched kernel (default 5 s); after
 * it the launch stops and returns MIG_ETIMEOUT, leaving the context usable. debug_stall != 0 is
 * a test hook that makes one level of the next batches never complete, so that the waits
 * behind it run out. */
mig_status mig_batch_set_timeout(mig_ctx *ctx, int64_t timeout_us, int debug_stall);
/* Number of CUDA-graph captures and replays of batched launches so far (a batch of the same
 * shape as the previous one replays the captured graph; the legacy default stream and
 * profiling use plain launches). */
mig_status mig_batch_graph_stats(mig_ctx *ctx, uint64_t *captures, uint64_t *replays);
/* Device-side trace of batched launches: with tracing on, every segment (the cast or the voxel count
 * of one chunk of a tree level's nodes, or the level's render work) records when it became ready and
 * when its last item finished (microseconds from the kernel start, %globaltimer).
 * mig_batch_trace_read copies the records of the last traced launch (n = number available).
 * Traced launches do not use the graph. */
typedef struct mig_trace_rec {
    int32_t tree, level, phase, items; /* phase 0 = cast, 1 = voxel count, 2 = render */
    double activated_us, done_us;
} mig_trace_rec;
mig_status mig_batch_trace(mig_ctx *ctx, int enable);
mig_status mig_batch_trace_read(mig_ctx *ctx, mig_trace_rec *out, int cap, int *n);


/* ---------------------------------------------------------------------------------------
 * Serving: continuous batching of replanning requests. Submitted trees wait in an admission
 * queue until their device bytes (depth-buffer arena nodes * W * H * 4, counters, step counts) plus
 * the bytes already held (requests in flight and map snapshots) fit the budget, then
 * join the device work of the requests already running; each request's results are the same
 * as a lone mig_tree_eval on the map contents at submission time. The descriptor's host arrays
 * are copied at submit; outputs are written when the request completes. A worker thread
 * drives the device; submit and poll are thread-safe.
 * mig_server_poll: MIG_OK = done (outputs written), MIG_EBUSY = not yet (timeout_us = 0),
 * MIG_ETIMEOUT = still running after timeout_us, MIG_ENOTFOUND = unknown ticket.
 * --------------------------------------------------------------------------------------- */
mig_status mig_server_create(mig_ctx *ctx, size_t arena_budget_bytes, int max_inflight, mig_server **out);
/* (a request whose bytes alone exceed the budget still runs when nothing else is in flight) */
mig_status mig_server_submit(mig_server *srv, const mig_tree_desc *tree, uint64_t *ticket);
mig_status mig_server_poll(mig_server *srv, uint64_t ticket, int64_t timeout_us);
/* Map update routed through the server: applied after every request submitted before it and
 * before every request submitted after it (requests keep their map snapshot). */
mig_status mig_server_map_update(mig_server *srv, mig_map *map, int x0, int y0, int z0, int dx, int dy, int dz,
                                 const uint8_t *host_voxels);
/* Device bytes the server holds: requests in flight (plans, counters, step counts, depth-buffer
 * arenas) and map snapshots (a map updated while requests still read it keeps its previous grid
 * until they finish; those copies count against the budget as well, and an update whose copy would
 * not fit waits for requests to finish); peak = the largest sum of the two so far. */
mig_status mig_server_memory(mig_server *srv, uint64_t *in_use, uint64_t *snapshots, uint64_t *peak);
/* Per-request timing (microseconds since submit): admitted, started on device, completed. */
mig_status mig_server_timing(mig_server *srv, uint64_t ticket, double *admit_us, double *start_us, double *done_us);
void mig_server_destroy(mig_server *srv);

/* ---------------------------------------------------------------------------------------
 * Measurement (no counterpart in the paper; used by the benchmark's roofline figures).
 * mig_ctx_profile(ctx, 1) starts recording a CUDA event pair around every kernel the
 * library launches on the context stream (0 stops); mig_ctx_profile_read synchronises and
 * returns the summed device time and launch count per kernel kind since the last read.
 * mig_tree_eval_stats runs mig_tree_eval with an instrumented count pass and returns the
 * algorithmic work: rays cast, DDA steps (1-byte voxel gathers), owner tests, samples,
 * ancestor projections and depth texels read (4 B each). Results are identical to
 * mig_tree_eval; the instrumented pass is slower and is not meant to be timed.
 * --------------------------------------------------------------------------------------- */
typedef struct mig_kernel_times {
    double count_ms, select_ms, render_ms, plan_ms, batch_ms;
    uint64_t count_launches, select_launches, render_launches, plan_launches, batch_launches;
    /* the owned-voxel count's two kernels (count_ms then covers the ray-by-ray, interval and
     * panoramic count kernels only) */
    double cast_ms, voxel_ms;
    uint64_t cast_launches, voxel_launches;
} mig_kernel_times;
/* Count kernels of the sample modes (marginal, single parent, absolute; no counterpart in the
 * paper; all give identical results). Owned-voxel counting casts each pixel ray once to its first
 * occupied voxel, then tests every unknown voxel of the frustum against the ray of the pixel that
 * owns it (its centre's projection): MIG_COUNT_PAIRS enumerates each (node, yaw) frustum,
 * MIG_COUNT_NODES each node's voxels once for all yaws (at most 64 yaws; its ancestor test runs
 * once per voxel), MIG_COUNT_AUTO (the default) takes the per-node pass when a voxel lies in at least
 * 3 yaws' frusta on average. MIG_COUNT_RAYS walks every ray through every voxel it crosses and
 * owner-tests the unknown ones. The owned-voxel kernels keep one uint16 step count per (node, yaw,
 * pixel) of a level in a buffer of at most steps_budget_bytes (0 = the default, 1 GiB); a level
 * that does not fit is counted in chunks. Errors: MIG_EINVAL (ctx NULL, unknown kernel). */
#define MIG_COUNT_AUTO 0
#define MIG_COUNT_RAYS 1
#define MIG_COUNT_PAIRS 2
#define MIG_COUNT_NODES 3
mig_status mig_ctx_set_count_kernel(mig_ctx *ctx, int kernel, uint64_t steps_budget_bytes);
mig_status mig_ctx_profile(mig_ctx *ctx, int enable);
mig_status mig_ctx_profile_read(mig_ctx *ctx, mig_kernel_times *out);

/* Random-gather probe: the rate (loads per second) at which the device serves independent loads
 * of elem_bytes (1 or 4) from pseudo-random positions of a buffer of buffer_bytes (rounded down to
 * a power-of-two element count; 4 KiB .. 4 GiB), L1 bypassed, so that each load is one sector
 * request: L2-served when the buffer fits in L2, HBM-served otherwise. The ceiling for the count
 * pass's scattered voxel (1 B) and depth-texel (4 B) gathers. Allocates and frees its buffer on the
 * context; synchronous. Errors: MIG_EINVAL, MIG_ENOMEM, MIG_ECUDA. */
mig_status mig_probe_gather(mig_ctx *ctx, uint64_t buffer_bytes, int elem_bytes, double *loads_per_s);

typedef struct mig_eval_stats {
    uint64_t rays, dda_steps, unknown_visits, samples, ancestor_tests, depth_reads;
    uint64_t render_rays, render_steps;
    uint64_t count_launches, render_launches;
    /* the owned-voxel count's own work (zero when the context counts ray by ray): rays cast to
     * their stopping point, voxel steps and brick jumps of those casts, voxels enumerated in the
     * frusta, unknown ones among them, exact visit tests, counted samples (== samples), and the
     * ancestor tests and depth reads of those samples */
    uint64_t cast_rays, cast_steps, cast_jumps, voxel_candidates, voxel_unknown, visit_tests, owned_samples;
    uint64_t voxel_ancestor_tests, voxel_depth_reads;
    /* the voxel pass that ran: MIG_COUNT_PAIRS or MIG_COUNT_NODES (MIG_COUNT_RAYS when counting ray by ray) */
    uint64_t voxel_pass;
} mig_eval_stats;
mig_status mig_tree_eval_stats(mig_map *map, int n, const int32_t *parent, const float *pos_m,
                               const mig_sensor *sensor, mig_eval_stats *stats, int32_t *abs_gain,
                               int32_t *marg_gain, int32_t *best_yaw);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *mig_last_error(void);

/* Build of this library (no counterpart in the paper). MIG_BUILD_CHECKED: built with
 * MIG_DEBUG_BOUNDS=1, where every voxel load and depth-buffer write checks its index; an index
 * outside its buffer skips the access and makes the host-array evaluation calls return MIG_ECUDA
 * ("bounds check") instead of touching memory outside the buffer. Slower; for testing. */
#define MIG_BUILD_CHECKED 1
int mig_build_flags(void);

#ifdef __cplusplus
}
#endif
#endif /* MIG_H */
