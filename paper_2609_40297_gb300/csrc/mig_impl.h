// Internal declarations of the marginal-gain library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "mig.h"

namespace mig {

constexpr int64_t kOneQ16 = 65536;
constexpr int64_t kOneQ30 = int64_t(1) << 30;
constexpr int kBrickShift = 3;  // 8x8x8 bricks of uint8 codes, 512 B each
constexpr int kBrick = 1 << kBrickShift;
constexpr int kYawRec = 12;  // per yaw: ck, sk, mu[3], mv[3], mz[3], pad

// ---------------------------------------------------------------------------------- errors
void set_error(const std::string &msg);
mig_status fail(mig_status st, const std::string &msg);
#define MIG_CUDA_TRY(call)                                                                        \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return ::mig::fail(MIG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

// ------------------------------------------------------------------------------ allocation
struct DeviceAllocator {
    mig_allocator user{};
    bool has_user = false;
    void *alloc(size_t bytes, cudaStream_t s);
    void free(void *p, size_t bytes, cudaStream_t s);
};

// Grow-only device buffer owned by a context.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// ---------------------------------------------------------------------------- camera tables
// Per sensor: per-pixel body-frame unit rays + camera z (Q30), per-yaw rotation and projection
// rows. Built on the host in IEEE double (no contraction), uploaded once per context.
struct Camera {
    mig_sensor s{};
    int W = 0, H = 0, K = 0;
    std::vector<int32_t> body;  // H*W*4: bx, by, bz, dzc
    std::vector<int32_t> yaw;   // K*kYawRec
    std::vector<float> yawf;    // K*9: each yaw's projection rows mu, mv, mz as floats (/ 2^16)
    int32_t *d_body = nullptr;
    int32_t *d_yaw = nullptr;   // the yaw table, then (same allocation) the float rows
    const float *d_yawf = nullptr;
    // the frustum's extent about its yaw axis, for enumerating voxels once per node over all yaws
    // (conservative culling bounds, not result-deciding): tangents of the lowest and highest
    // elevation of a voxel centre that can project into the image, and the largest azimuth offset
    // from the yaw direction (pi when the frustum holds the vertical)
    float band_tlo = -1e30f, band_thi = 1e30f, az_half = 3.2f;
    // panoramic mode (built on first use; level camera only): A azimuth wedges of a yaw step's
    // `pano_step` columns each, Wc columns per yaw window
    int pano_A = 0, pano_Wc = 0, pano_step = 0;
    std::vector<int32_t> pano_bc;   // A*2: wedge boundary cos, sin (Q30)
    std::vector<int32_t> pano_dir;  // A*H*4: ray of cell (c, j) (Q30), pad
    std::vector<int32_t> pano_row;  // A*8: strip rows mv[3], mz[3] (Q16), pad[2]
    int32_t *d_pano_bc = nullptr, *d_pano_dir = nullptr, *d_pano_row = nullptr;
};
mig_status camera_build(const mig_sensor &s, Camera &out);
mig_status pano_build(Camera &c);  // fills the pano_* host tables (MIG_EINVAL unless pitch is 0)
mig_status sensor_check(const mig_sensor &s, float voxel);
int64_t range_q16(float range_m, float voxel);

// ------------------------------------------------------------------------------------- plan
struct HostPlan {
    int n = 0, max_depth = 0, n_internal = 0, total_anc = 0;
    std::vector<int32_t> depth;       // n
    std::vector<int32_t> level_off;   // max_depth + 2
    std::vector<int32_t> level_int;   // max_depth + 1: internal nodes leading each level
    std::vector<int32_t> level_nodes; // n (internal nodes first within a level)
    std::vector<int32_t> anc_off;     // n + 1
    std::vector<int32_t> anc;         // ancestors, parent first
    std::vector<int32_t> node;        // n*4: Px, Py, Pz (Q16), slot (-1 = leaf)
};
mig_status tree_check(int n, const int32_t *parent, int32_t *depth, int32_t *max_depth);
mig_status plan_build(int n, const int32_t *parent, const float *pos, const float origin[3], float voxel,
                      const int dims[3], HostPlan &p);

// CUDA-event timing of the library's own launches (mig_ctx_profile).
enum ProfKind { kProfCount = 0, kProfSelect, kProfRender, kProfPlan, kProfBatch, kProfCast, kProfVoxel, kProfKinds };
struct Profiler {
    bool on = false;
    struct Pair {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Pair> pending;
    std::vector<cudaEvent_t> pool;
    double ms[kProfKinds] = {};
    uint64_t launches[kProfKinds] = {};
};

}  // namespace mig

// ----------------------------------------------------------------------------- public objects
struct mig_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    mig::DeviceAllocator alloc;
    int num_sms = 0;
    int count_ctas = 1;        // resident count-kernel CTAs per SM
    int interval_ctas = 1;     // resident interval-mode count CTAs per SM
    int pano_ctas = 1;         // resident panoramic count CTAs per SM
    int vox_ctas = 1;          // resident owned-voxel count CTAs per SM
    int node_ctas = 1;         // resident per-node voxel-pass CTAs per SM
    bool ray_count = false;    // count with the ray-by-ray kernel instead of the owned-voxel kernels
    int voxel_pass = MIG_COUNT_AUTO;  // owned-voxel pass: per (node, yaw) pair, per node, or chosen
    size_t steps_budget = 0;   // owned-voxel step-count buffer per evaluation (bytes; set at creation)
    std::vector<std::unique_ptr<mig::Camera>> cameras;
    mig::DevBuf ws;          // per-call workspace (plan, counters, outputs, arena)
    void *pinned = nullptr;  // pinned host staging
    size_t pinned_bytes = 0;
    int32_t *d_err = nullptr;  // device-side check word (device planning)
    mig_tile_config tiles{4, 16, 4, 1};  // 64-ray count tiles; batches on stream chains
    mig::Profiler prof;
    int64_t batch_timeout_ns = 5000000000LL;  // bound of every device-side wait of the batch kernel
    bool batch_debug_stall = false;           // test hook: one level never completes
    bool batch_trace = false;                 // record per-segment device timestamps
    struct Batch;            // batched engine state (batch.cu)
    Batch *batch = nullptr;
    std::mutex mu;           // serialises calls that share the workspace
};

struct mig_map {
    mig_ctx *ctx = nullptr;
    int nx = 0, ny = 0, nz = 0;
    int nbx = 0, nby = 0, nbz = 0;  // bricks per axis
    float voxel = 0.f;
    float origin[3] = {0.f, 0.f, 0.f};
    uint8_t *d_grid = nullptr;       // bricked codes, nbx*nby*nbz*512 bytes
    size_t grid_bytes = 0;
    uint64_t version = 0;
};

namespace mig {
// workspace / staging helpers (api.cu)
mig_status ctx_workspace(mig_ctx *ctx, size_t bytes, void **out);
mig_status ctx_pinned(mig_ctx *ctx, size_t bytes, void **out);
mig_status ctx_camera(mig_ctx *ctx, const mig_sensor &s, const Camera **out);
// The panoramic tables of a context camera, built and uploaded on first use (ctx->mu held).
mig_status ctx_pano(mig_ctx *ctx, const Camera *cam);
// The frustum band of the per-node voxel pass, from the camera.
void set_band(LevelParams &p, const Camera *cam);
// Panoramic level parameters from the camera's tables; pcnt = n * A * 2 int32 of workspace.
void set_pano_params(LevelParams &p, const Camera *cam, int32_t *pcnt);
// One level's count pass for p.mode: the sample, interval or panoramic kernels (Ld = nodes of
// the level, or an upper bound of it for the sample modes' owned-voxel kernels, which read the
// level's size on the device). The sample modes use the owned-voxel kernels when p.steps is set,
// else the ray-by-ray count kernel. The panoramic mode also runs its window sums, so
// launch_select may follow.
void launch_level_count(const mig_ctx *ctx, const LevelParams &p, int Ld, int count_cap, cudaStream_t s);
// The same on the context stream, each launch timed under its own kind (mig_ctx_profile).
void launch_level_count_timed(mig_ctx *ctx, const LevelParams &p, int Ld, int count_cap);
// (node, yaw) pairs per owned-voxel chunk for a tree whose widest level has Lmax nodes (0 when the
// context counts ray by ray); the step-count buffer holds steps_cap * W * H uint16.
int steps_cap_for(const mig_ctx *ctx, int Lmax, int K, int W, int H, int mode);
// records an event pair around launch() on the context stream when profiling is on
void prof_begin(mig_ctx *ctx, int kind, cudaEvent_t *a);
void prof_end(mig_ctx *ctx, int kind, cudaEvent_t a);
// NVTX range on the host thread (visible to ncu --nvtx and to timeline profilers; a no-op
// when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

template <class F>
inline void timed_launch(mig_ctx *ctx, int kind, F &&launch) {
    static const char *const kNames[kProfKinds] = {"mig count", "mig select", "mig render", "mig plan",
                                                   "mig batch", "mig cast",   "mig voxel"};
    NvtxRange range(kNames[kind]);
    cudaEvent_t a = nullptr;
    prof_begin(ctx, kind, &a);
    launch();
    prof_end(ctx, kind, a);
}
}  // namespace mig
