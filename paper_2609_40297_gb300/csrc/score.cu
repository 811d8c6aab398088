// Path scoring after gain evaluation: traversal cost (Eq. 3), exponential objective (Eq. 4) and
// the best node, on the device. One thread per node walks its root path (depth <= 64) and sums in
// IEEE double with explicit round-to-nearest operations; the best node is the lowest index with
// the largest objective (two passes over the nodes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "mig_impl.h"

namespace mig {
namespace {

__device__ __forceinline__ unsigned long long order_key(double x) {  // monotone map of doubles
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | (1ull << 63));
}

__global__ void score_kernel(int n, const int32_t *parent, const float *pos, const int32_t *gain, double v3,
                             double lam, double *cost, double *obj, unsigned long long *best_key, int *err) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int path[MIG_MAX_DEPTH + 1];
        int len = 0, q = i;
        bool bad = false;
        while (q >= 0) {
            if (q >= n || len > MIG_MAX_DEPTH) {
                bad = true;
                break;
            }
            path[len++] = q;
            q = parent[q];
        }
        if (bad) {
            atomicOr(err, 1);
            cost[i] = obj[i] = 0.0;
            continue;
        }
        double c = 0.0, o = 0.0;
        for (int k = len - 1; k >= 0; --k) {  // root first
            const int a = path[k];
            if (k < len - 1) {
                const int b = path[k + 1];
                const double dx = __dsub_rn((double)pos[3 * (size_t)a], (double)pos[3 * (size_t)b]);
                const double dy = __dsub_rn((double)pos[3 * (size_t)a + 1], (double)pos[3 * (size_t)b + 1]);
                const double dz = __dsub_rn((double)pos[3 * (size_t)a + 2], (double)pos[3 * (size_t)b + 2]);
                c = __dadd_rn(c, __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz))));
            }
            o = __dadd_rn(o, __dmul_rn(__dmul_rn((double)gain[a], v3), exp(__dmul_rn(-lam, c))));
        }
        cost[i] = c;
        obj[i] = o;
        atomicMax(best_key, order_key(o));
    }
}

__global__ void best_kernel(int n, const double *obj, const unsigned long long *best_key, int *best) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (order_key(obj[i]) == *best_key) atomicMin(best, i);
}

__global__ void score_init_kernel(unsigned long long *best_key, int *best, int *err, int n) {
    *best_key = 0;
    *best = n;
    *err = 0;
}

__global__ void score_finish_kernel(int *best, const int *err, int32_t *best_out, int32_t *ctx_err) {
    *best_out = *err ? -1 : *best;
    if (*err) atomicOr(ctx_err, 1);
}

}  // namespace
}  // namespace mig

using namespace mig;

extern "C" mig_status mig_tree_score_device(mig_ctx *ctx, int n, const int32_t *parent, const float *pos_m,
                                            const int32_t *gain_counts, double voxel_size_m, double lambda,
                                            double *cost, double *objective, int32_t *best_node) {
    if (!ctx || n < 0) return fail(MIG_EINVAL, "tree_score: invalid argument");
    if (!(voxel_size_m > 0.0) || !(lambda >= 0.0)) return fail(MIG_EINVAL, "tree_score: voxel size > 0, lambda >= 0");
    if (n == 0) return MIG_OK;
    if (!parent || !pos_m || !gain_counts || !cost || !objective || !best_node) return fail(MIG_EINVAL, "tree_score: NULL array");
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaSetDevice(ctx->device));
    // small scratch: best key, best index, error word
    char *scr = (char *)ctx->alloc.alloc(256, ctx->stream);
    if (!scr) return fail(MIG_ENOMEM, "tree_score: scratch allocation failed");
    unsigned long long *key = (unsigned long long *)scr;
    int *best = (int *)(scr + 8), *err = (int *)(scr + 12);
    const double v3 = voxel_size_m * voxel_size_m * voxel_size_m;
    const int grid = std::max(1, std::min((n + 127) / 128, 4096));
    score_init_kernel<<<1, 1, 0, ctx->stream>>>(key, best, err, n);
    score_kernel<<<grid, 128, 0, ctx->stream>>>(n, parent, pos_m, gain_counts, v3, lambda, cost, objective, key, err);
    best_kernel<<<grid, 128, 0, ctx->stream>>>(n, objective, key, best);
    score_finish_kernel<<<1, 1, 0, ctx->stream>>>(best, err, best_node, ctx->d_err);
    MIG_CUDA_TRY(cudaGetLastError());
    ctx->alloc.free(scr, 256, ctx->stream);
    return MIG_OK;
}

extern "C" mig_status mig_tree_score(mig_ctx *ctx, int n, const int32_t *parent, const float *pos_m,
                                     const int32_t *gain_counts, double voxel_size_m, double lambda, double *cost,
                                     double *objective, int32_t *best_node) {
    if (!ctx || n < 0) return fail(MIG_EINVAL, "tree_score: invalid argument");
    if (n == 0) {
        if (best_node) *best_node = -1;
        return MIG_OK;
    }
    if (!parent || !pos_m || !gain_counts || !cost || !objective || !best_node) return fail(MIG_EINVAL, "tree_score: NULL array");
    mig_status st = tree_check(n, parent, nullptr, nullptr);
    if (st != MIG_OK) return st;
    const size_t bytes = (size_t)n * (4 + 12 + 4 + 8 + 8) + 4 + 1024;
    char *dev = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        MIG_CUDA_TRY(cudaSetDevice(ctx->device));
        dev = (char *)ctx->alloc.alloc(bytes, ctx->stream);
        if (!dev) return fail(MIG_ENOMEM, "tree_score: allocation failed");
        MIG_CUDA_TRY(cudaMemcpyAsync(dev, parent, 4 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
        MIG_CUDA_TRY(cudaMemcpyAsync(dev + 4 * (size_t)n, pos_m, 12 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
        MIG_CUDA_TRY(cudaMemcpyAsync(dev + 16 * (size_t)n, gain_counts, 4 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
    }
    double *dcost = (double *)(dev + ((20 * (size_t)n + 255) & ~(size_t)255));
    double *dobj = dcost + n;
    int32_t *dbest = (int32_t *)(dobj + n);
    st = mig_tree_score_device(ctx, n, (const int32_t *)dev, (const float *)(dev + 4 * (size_t)n),
                               (const int32_t *)(dev + 16 * (size_t)n), voxel_size_m, lambda, dcost, dobj, dbest);
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (st == MIG_OK) {
        MIG_CUDA_TRY(cudaMemcpyAsync(cost, dcost, 8 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
        MIG_CUDA_TRY(cudaMemcpyAsync(objective, dobj, 8 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
        MIG_CUDA_TRY(cudaMemcpyAsync(best_node, dbest, 4, cudaMemcpyDeviceToHost, ctx->stream));
    }
    ctx->alloc.free(dev, bytes, ctx->stream);
    MIG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return st;
}
