// Final DeepONet flux at every cell centre on the 5th-generation tensor
// cores: phi_c = <beta_b, t(x_c)> for the 128-wide, depth-4 trunk (Sec. 4.1
// Eq. 11), t = W4 relu(W3 relu(W2 relu(w1 x + b1) + b2) + b3) + b4.
//
// The trunk depends on the cell centre x = (i + 0.5) / I only, so instances
// with the same cell count share it: the kernel walks the distinct points
// (CSR groups of instances with equal I) and writes the inner product for
// every instance of the group.
//
// One persistent CTA per SM with two warpgroups on different 128-point tiles
// (one group's epilogue overlaps the other's products); thread t of a
// warpgroup owns point t of its tile and TMEM lane t of its 256 columns.
// W2..W4 sit in shared memory as BF16 in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix,
// K-adjacent matrices 128 B apart, row groups 2048 B apart).  Per layer one
// thread issues eight tcgen05.mma (M = N = 128, K = 16, FP32 accumulator in
// 128 TMEM columns) and commits them to an mbarrier; every thread then reads
// its row back with tcgen05.ld, adds the bias, applies ReLU, rounds to BF16
// and stores the row as the next layer's A operand.  The inner products with
// the coefficients are one more product (N = 32 instances per chunk).  Waits
// are bounded (TC_SPIN polls, or the context's nop_set_wait_limit): on a
// timeout the kernel records an error and stops issuing work; a warpgroup
// whose wait gave up then waits (bounded by TC_SPIN) for the products it
// already committed, so no product still writes TMEM when the block frees it
// and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "nop_internal.cuh"

namespace nop {
namespace {

constexpr int TC_W = 128, TC_M = 128;
constexpr int TC_MAT = TC_W * TC_W;                               // elements per matrix
constexpr int TC_NB = 32;                                        // coefficient columns per MMA
constexpr size_t TC_SMEM = sizeof(__nv_bfloat16) * (3 * TC_MAT + 2 * (TC_MAT + TC_NB * TC_W))
                           + 1024;   // W2-W4, per warpgroup H and beta; alignment slack
constexpr long long TC_SPIN = 1ll << 26;                          // mbarrier poll limit

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// element offset of (row r, column k) in a 128 x 128 core-matrix tile
__device__ __forceinline__ int cm(int r, int k) {
    return (r >> 3) * 1024 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// shared-memory matrix descriptor: no swizzle, K-major; LBO = 128 B between
// K-adjacent core matrices, SBO = 2048 B between row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(2048u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 128, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) |
                              ((128u >> 4) << 24);
// the same with N = 32: the inner products with up to 32 coefficient vectors
constexpr uint32_t TC_IDESC_B = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) |
                                ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc,
                                         uint32_t idesc = TC_IDESC) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// 32 consecutive columns of the thread's TMEM lane (no wait)
__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(addr));
}

// waits for the phase of the mbarrier; false after `limit` polls (none when
// limit is 0)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(phase));
        if (done) return true;
    }
    return false;
}

// 64 consecutive columns of the thread's TMEM lane (no wait)
__device__ __forceinline__ void tmem_ld64(uint32_t addr, uint32_t (&r)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]),
          "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]),
          "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
          "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]),
          "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]),
          "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(addr));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *(const uint32_t*)&h;
}

// Two warpgroups per CTA work on different tiles, so one group's epilogue
// overlaps the other's tensor-core products.
__device__ __forceinline__ void wg_sync(int wg) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + wg), "r"(TC_M));
}

// tinfo[tile] = {first group, last group, first and end instance index} of
// the tile's points, prepared on the host.
__global__ void __launch_bounds__(2 * TC_M, 1) trunk_tc_kernel(
    long long P, const int4* tinfo, const long long* grp_pt_off, const int* grp_I,
    const int* grp_inst_off, const int* inst_list, const long long* cell_off, const float* W1,
    const float* b1, const float* W2, const float* b2, const float* W3, const float* b3,
    const float* W4, const float* b4, const float* beta_keep, const int* status, double* phi,
    int* err, long long spin) {
    extern __shared__ unsigned char tc_raw[];
    // 1024-byte aligned operand area: W2-W4, then per warpgroup H and B
    __nv_bfloat16* base = (__nv_bfloat16*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    __nv_bfloat16* Ws = base;
    __shared__ float bs[4][TC_W], w1s[TC_W];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag[2];
    // per warpgroup: the tile's groups (at most one per point) and one chunk
    // of instances
    __shared__ long long s_gpt[2][TC_M + 1], s_off[2][TC_NB];
    __shared__ int s_gI[2][TC_M], s_gio[2][TC_M + 1], s_b[2][TC_NB], s_st[2][TC_NB];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int wg = tid / TC_M, t = tid % TC_M;
    __nv_bfloat16* H = base + 3 * TC_MAT + wg * (TC_MAT + TC_NB * TC_W);   // A operand
    __nv_bfloat16* Bq = H + TC_MAT;                                         // coefficients

    for (int e = tid; e < TC_MAT; e += 2 * TC_M) {
        const int n = e / TC_W, k = e % TC_W;
        Ws[0 * TC_MAT + cm(n, k)] = __float2bfloat16_rn(W2[e]);
        Ws[1 * TC_MAT + cm(n, k)] = __float2bfloat16_rn(W3[e]);
        Ws[2 * TC_MAT + cm(n, k)] = __float2bfloat16_rn(W4[e]);
    }
    for (int n = tid; n < TC_W; n += 2 * TC_M) {
        // the trunk input weights are rounded to BF16 like any GEMM operand
        w1s[n] = __bfloat162float(__float2bfloat16_rn(W1[n]));
        bs[0][n] = b1[n];
        bs[1][n] = b2[n];
        bs[2][n] = b3[n];
        bs[3][n] = b4[n];
    }
    if (tid < 2) {
        abort_flag[tid] = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[tid])));
    }
    if (warp == 0) {
        // per warpgroup 256 columns: 0-127 the layer accumulator, 128-159
        // the inner products
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
            smem_addr(&tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot + (uint32_t)(wg * 256);
    const uint32_t row_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t bar = smem_addr(&mbar[wg]);
    const uint32_t h_addr = smem_addr(H);
    uint32_t phase = 0;
    int* abort_wg = &abort_flag[wg];
    // the phase of a commit whose wait gave up (products possibly in flight)
    bool stuck = false;
    uint32_t stuck_phase = 0;

    for (long long t0 = ((long long)blockIdx.x * 2 + wg) * TC_M; t0 < P;
         t0 += (long long)gridDim.x * 2 * TC_M) {
        // this thread's point: group, index within the instance, coordinate,
        // from the tile's group bounds staged in shared memory
        const int4 ti = tinfo[t0 / TC_M];
        const int ngt = ti.y - ti.x + 1, k_lo = ti.z, k_hi = ti.w;
        wg_sync(wg);   // the previous tile is done with the staged arrays
        if (t <= ngt) {
            s_gpt[wg][t] = grp_pt_off[ti.x + t];
            s_gio[wg][t] = grp_inst_off[ti.x + t];
            if (t < ngt) s_gI[wg][t] = grp_I[ti.x + t];
        }
        wg_sync(wg);
        const long long c = t0 + t;
        int gl = -1, i = 0;
        float x = 0.f;
        if (c < P) {
            gl = 0;
            while (gl + 1 < ngt && s_gpt[wg][gl + 1] <= c) ++gl;
            i = (int)(c - s_gpt[wg][gl]);
            x = (float)((i + 0.5) / s_gI[wg][gl]);
        }
        // layer 1 (one input): h = relu(x w1 + b1), BF16, into the A tile
        const float xb = __bfloat162float(__float2bfloat16_rn(x));
#pragma unroll 4
        for (int kb = 0; kb < TC_W / 8; ++kb) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = fmaxf(xb * w1s[kb * 8 + j] + bs[0][kb * 8 + j], 0.f);
            uint4 q;
            q.x = pack_bf16(v[0], v[1]);
            q.y = pack_bf16(v[2], v[3]);
            q.z = pack_bf16(v[4], v[5]);
            q.w = pack_bf16(v[6], v[7]);
            *(uint4*)&H[cm(t, kb * 8)] = q;
        }
        // layers 2-4 on the tensor cores
        for (int l = 0; l < 3; ++l) {
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            wg_sync(wg);
            if (*abort_wg) break;
            if (t == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t w_addr = smem_addr(Ws + l * TC_MAT);
#pragma unroll
                for (int kk = 0; kk < TC_W / 16; ++kk)   // K = 16: two core matrices
                    mma_bf16(tmem, smem_desc(h_addr + kk * 256), smem_desc(w_addr + kk * 256),
                             kk > 0 ? 1u : 0u);
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        bar));
            }
            const bool ok = mbar_wait(bar, phase, spin);
            if (!ok) {
                atomicExch(err, 1);
                *abort_wg = 1;
                stuck = true;
                stuck_phase = phase;
            }
            phase ^= 1u;
            wg_sync(wg);
            if (*abort_wg) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            // epilogue: row t of the accumulator (two 64-column loads, one
            // wait), + bias, ReLU except after the output layer, rounded to
            // BF16 into the row of H
            uint32_t r0[64], r1[64];
            tmem_ld64(row_addr, r0);
            tmem_ld64(row_addr + 64u, r1);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int kb = 0; kb < TC_W / 8; ++kb) {
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int col = kb * 8 + j;
                    const float a = __uint_as_float(kb < 8 ? r0[col] : r1[col - 64]) + bs[l + 1][col];
                    v[j] = l < 2 ? fmaxf(a, 0.f) : a;
                }
                uint4 q;
                q.x = pack_bf16(v[0], v[1]);
                q.y = pack_bf16(v[2], v[3]);
                q.z = pack_bf16(v[4], v[5]);
                q.w = pack_bf16(v[6], v[7]);
                *(uint4*)&H[cm(t, kb * 8)] = q;
            }
        }
        if (*abort_wg) break;
        // inner products with the coefficients of the tile's instances, as
        // one more tensor-core product: [128 points x 128] . [128 x 32 beta]
        // per chunk of 32 instances (BF16 operands, FP32 accumulation)
        const int kb_g = gl >= 0 ? s_gio[wg][gl] : 0, ke_g = gl >= 0 ? s_gio[wg][gl + 1] : 0;
        for (int kc = k_lo; kc < k_hi; kc += TC_NB) {
            const int nb = min(TC_NB, k_hi - kc);
            wg_sync(wg);   // the previous chunk is done with s_b and Bq
            if (t < nb) {
                const int b = inst_list[kc + t];
                s_b[wg][t] = b;
                s_off[wg][t] = cell_off[b];
                s_st[wg][t] = status ? status[b] : 0;
            }
            wg_sync(wg);
            for (int e = t; e < TC_NB * TC_W; e += TC_M) {
                const int r = e / TC_W, k = e % TC_W;
                const float v = r < nb ? beta_keep[(long long)s_b[wg][r] * TC_W + k] : 0.f;
                Bq[cm(r, k)] = __float2bfloat16_rn(v);
            }
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            wg_sync(wg);
            if (t == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t b_addr = smem_addr(Bq);
#pragma unroll
                for (int kk = 0; kk < TC_W / 16; ++kk)
                    mma_bf16(tmem + 128u, smem_desc(h_addr + kk * 256),
                             smem_desc(b_addr + kk * 256), kk > 0 ? 1u : 0u, TC_IDESC_B);
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        bar));
            }
            const bool ok = mbar_wait(bar, phase, spin);
            if (!ok) {
                atomicExch(err, 1);
                *abort_wg = 1;
                stuck = true;
                stuck_phase = phase;
            }
            phase ^= 1u;
            wg_sync(wg);
            if (*abort_wg) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            uint32_t rv[32];
            tmem_ld32(row_addr + 128u, rv);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            // this point's instances inside the chunk
            const int lo = max(kb_g, kc), hi = min(ke_g, kc + nb);
#pragma unroll
            for (int j = 0; j < TC_NB; ++j) {
                const int k = kc + j;
                if (k >= lo && k < hi)
                    phi[s_off[wg][j] + i] = s_st[wg][j] == 3 ? 0.0 : (double)__uint_as_float(rv[j]);
            }
            // the next chunk reuses Bq and the TMEM columns
            asm volatile("tcgen05.fence::before_thread_sync;");
        }
        if (*abort_wg) break;
    }
    // a wait that gave up left products in flight: let them finish (bounded)
    // before the TMEM they write is freed
    if (stuck) mbar_wait(bar, stuck_phase, TC_SPIN);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tslot));
}

}  // namespace

size_t trunk_tc_smem() { return TC_SMEM; }

int trunk_tc_launch(nop_ctx* ctx, long long P, const int4* tinfo, const long long* gpt,
                    const int* gI, const int* ginst, const int* list, const long long* cell_off,
                    const float* const W[4], const float* const b[4], const float* beta_keep,
                    const int* status, double* phi, int* err) {
    NOP_CUDA_TRY(ctx, cudaFuncSetAttribute(trunk_tc_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)TC_SMEM));
    const int grid = (int)std::max<long long>(
        1, std::min<long long>((P + 2 * TC_M - 1) / (2 * TC_M), ctx->sm_count));
    trunk_tc_kernel<<<grid, 2 * TC_M, TC_SMEM, ctx->stream>>>(
        P, tinfo, gpt, gI, ginst, list, cell_off, W[0], b[0], W[1], b[1], W[2], b[2], W[3], b[3],
        beta_keep, status, phi, err, ctx->wait_limit >= 0 ? ctx->wait_limit : TC_SPIN);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    return NOP_OK;
}

}  // namespace nop
