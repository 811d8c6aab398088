// Measurement probe (no counterpart in the paper): the random-gather ceiling of the memory system
// for the count pass's access pattern. Every thread issues independent loads of `elem_bytes` from
// pseudo-random positions of a device buffer; with L1 bypassed (ld.global.cg) each load is one
// sector request to L2 (or HBM when the buffer does not fit in L2), so loads per second is the
// rate at which a kernel can gather scattered voxels or depth texels. The result is or-ed into one
// word per thread so that no load is dead code.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "mig_impl.h"

namespace mig {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeUnroll = 8;

__device__ __forceinline__ uint32_t mix32(uint32_t x) {  // an integer hash (xorshift-multiply)
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ uint32_t ld_cg_u8(const uint8_t *p) {
    uint32_t v;
    asm volatile("ld.global.cg.u8 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_cg_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Positions from a per-thread linear congruential sequence (its high bits index a power-of-two
// buffer), so that the address arithmetic stays a few instructions per load.
template <int ELEM>
__global__ void __launch_bounds__(kProbeThreads) gather_probe_kernel(const uint8_t *buf, int shift, int rounds,
                                                                     uint32_t seed, uint32_t *sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0, h = mix32(tid ^ seed);
    for (int r = 0; r < rounds; ++r) {
        uint32_t v[kProbeUnroll];
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
            h = h * 1664525u + 1013904223u;
            const uint32_t i = h >> shift;
            if constexpr (ELEM == 1) v[u] = ld_cg_u8(buf + i);
            else v[u] = ld_cg_u32(reinterpret_cast<const uint32_t *>(buf) + i);
        }
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) acc ^= v[u];
    }
    sink[tid] = acc;
}

}  // namespace

}  // namespace mig

using namespace mig;

extern "C" mig_status mig_probe_gather(mig_ctx *ctx, uint64_t buffer_bytes, int elem_bytes, double *loads_per_s) {
    if (!ctx || !loads_per_s || (elem_bytes != 1 && elem_bytes != 4) || buffer_bytes < 4096 ||
        buffer_bytes > ((uint64_t)1 << 32))
        return fail(MIG_EINVAL, "probe_gather: buffer 4 KiB .. 4 GiB, elements of 1 or 4 bytes");
    int log2n = 0;  // the largest power-of-two element count that fits the buffer
    while (((uint64_t)2 << log2n) * (uint64_t)elem_bytes <= buffer_bytes && log2n < 31) ++log2n;
    buffer_bytes = ((uint64_t)1 << log2n) * (uint64_t)elem_bytes;
    std::lock_guard<std::mutex> lk(ctx->mu);
    MIG_CUDA_TRY(cudaSetDevice(ctx->device));
    const int blocks = ctx->num_sms * 8, rounds = 64;
    const size_t threads = (size_t)blocks * kProbeThreads;
    uint8_t *buf = (uint8_t *)ctx->alloc.alloc((size_t)buffer_bytes, ctx->stream);
    uint32_t *sink = (uint32_t *)ctx->alloc.alloc(threads * 4, ctx->stream);
    cudaEvent_t a = nullptr, b = nullptr;
    mig_status st = MIG_OK;
    if (!buf || !sink) st = fail(MIG_ENOMEM, "probe_gather: allocation failed");
    if (st == MIG_OK && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess))
        st = fail(MIG_ECUDA, "probe_gather: event creation failed");
    double best_ms = 1e30;
    if (st == MIG_OK) {
        cudaMemsetAsync(buf, 1, (size_t)buffer_bytes, ctx->stream);
        const int shift = 32 - log2n;
        for (int rep = 0; rep < 6; ++rep) {  // the first launches warm L2 with the buffer
            cudaEventRecord(a, ctx->stream);
            if (elem_bytes == 1)
                gather_probe_kernel<1><<<blocks, kProbeThreads, 0, ctx->stream>>>(buf, shift, rounds, 0x9e3779b9u * rep, sink);
            else
                gather_probe_kernel<4><<<blocks, kProbeThreads, 0, ctx->stream>>>(buf, shift, rounds, 0x9e3779b9u * rep, sink);
            cudaEventRecord(b, ctx->stream);
            if (cudaEventSynchronize(b) != cudaSuccess) {
                st = fail(MIG_ECUDA, "probe_gather: kernel failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (rep >= 2) best_ms = std::min(best_ms, (double)ms);
        }
        if (st == MIG_OK && cudaGetLastError() != cudaSuccess) st = fail(MIG_ECUDA, "probe_gather: launch failed");
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    ctx->alloc.free(buf, (size_t)buffer_bytes, ctx->stream);
    ctx->alloc.free(sink, threads * 4, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    if (st != MIG_OK) return st;
    *loads_per_s = (double)threads * rounds * kProbeUnroll / (best_ms * 1e-3);
    return MIG_OK;
}
