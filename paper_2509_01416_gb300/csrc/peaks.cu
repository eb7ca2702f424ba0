// Measured arithmetic ceilings of the sweep kernels (a microbenchmark of the
// two instruction kinds the diamond-difference update is built from).
//
// The slab sweep's cell-angle update needs one reciprocal of (2|mu|/dx +
// Sigma_t) and a few fused multiply-adds; its roofline is therefore the
// device's rate of the special-function reciprocal (rcp.approx.ftz.f32, the
// instruction rcp_dd issues) and of FP32 FMA.  Both kernels below run 8
// independent dependency chains per thread over a grid of 8 blocks of 256
// threads per SM, so the pipes, not latency, set the rate; events on the
// context stream time them.
#include <algorithm>

#include "nop_internal.cuh"

namespace nop {
namespace {

constexpr int PK_CHAINS = 8;

__global__ void rcp_rate_kernel(int iters, float seed, float c, float* sink) {
    float x[PK_CHAINS];
#pragma unroll
    for (int j = 0; j < PK_CHAINS; ++j) x[j] = seed + 0.125f * j + 1e-6f * threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) {
            // x <- 1 / (x + c): a contraction to a fixed point that no
            // compiler can fold (c is a run-time value); one add per
            // reciprocal, on a pipe eight times wider than the reciprocal's
            const float d = x[j] + c;
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(x[j]) : "f"(d));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PK_CHAINS; ++j) s += x[j];
    if (s == 12345.678f) sink[0] = s;   // keeps the chains live
}

__global__ void fma_rate_kernel(int iters, float seed, float* sink) {
    float x[PK_CHAINS];
#pragma unroll
    for (int j = 0; j < PK_CHAINS; ++j) x[j] = seed + 0.125f * j + 1e-6f * threadIdx.x;
    const float a = 0.999f, b = 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < PK_CHAINS; ++j) x[j] = fmaf(x[j], a, b);   // bounded fixed point
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PK_CHAINS; ++j) s += x[j];
    if (s == 12345.678f) sink[0] = s;
}

}  // namespace
}  // namespace nop

extern "C" int nop_measure_alu_peaks(nop_ctx* ctx, double* rcp_per_s, double* fma_per_s) {
    if (!ctx || !rcp_per_s || !fma_per_s) return NOP_EINVAL;
    void* p;
    NOP_TRY(ctx->scratch("pk_sink", sizeof(float), &p));
    float* sink = (float*)p;
    const int blocks = 8 * ctx->sm_count, threads = 256, iters = 4096;
    const double ops = (double)blocks * threads * iters * nop::PK_CHAINS;
    cudaEvent_t e0, e1;
    NOP_CUDA_TRY(ctx, cudaEventCreate(&e0));
    NOP_CUDA_TRY(ctx, cudaEventCreate(&e1));
    double best[2] = {0.0, 0.0};
    for (int kind = 0; kind < 2; ++kind) {
        for (int rep = 0; rep < 4; ++rep) {   // the first run warms up; the best counts
            NOP_CUDA_TRY(ctx, cudaEventRecord(e0, ctx->stream));
            if (kind == 0)
                nop::rcp_rate_kernel<<<blocks, threads, 0, ctx->stream>>>(iters, 1.5f, 0.75f, sink);
            else
                nop::fma_rate_kernel<<<blocks, threads, 0, ctx->stream>>>(iters, 1.5f, sink);
            NOP_CUDA_TRY(ctx, cudaGetLastError());
            NOP_CUDA_TRY(ctx, cudaEventRecord(e1, ctx->stream));
            NOP_CUDA_TRY(ctx, cudaEventSynchronize(e1));
            float ms = 0.f;
            NOP_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0 && ms > 0.f) best[kind] = std::max(best[kind], ops / (ms * 1e-3));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *rcp_per_s = best[0];
    *fma_per_s = best[1];
    return NOP_OK;
}
