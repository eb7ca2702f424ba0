// BF16 tensor-core GEMM (mma.sync m16n8k16, FP32 accumulation) and the
// elementwise kernels of neural-operator training.
#include <cuda_bf16.h>

#include <algorithm>

#include "nn_kernels.cuh"

namespace nop {

namespace {

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8, GEMM_THREADS = 128;

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Block tile 64 x 64, K step 32; 4 warps in 2 x 2, each a 32 x 32 sub-tile of
// 2 x 4 mma tiles.  Shared tiles hold As[m][k] and Bs[n][k] (k contiguous) as
// BF16 so that fragment loads are 32-bit words.
__global__ void __launch_bounds__(GEMM_THREADS) gemm_kernel(GemmArgs g) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (blockIdx.z > 0) {
        g.A += blockIdx.z * g.sA;
        g.B += blockIdx.z * g.sB;
        g.C += blockIdx.z * g.sC;
    }
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

    for (int k0 = 0; k0 < g.K; k0 += BK) {
        // stage A (64 x 32) and B (32 x 64) as BF16
        for (int e = tid; e < BM * BK; e += GEMM_THREADS) {
            int r, c;
            if (!g.transA) {
                r = e / BK;
                c = e % BK;
            } else {
                c = e / BM;
                r = e % BM;
            }
            const int m = m0 + r, k = k0 + c;
            float v = 0.f;
            if (m < g.M && k < g.K)
                v = g.transA ? g.A[(long long)k * g.lda + m] : g.A[(long long)m * g.lda + k];
            As[r][c] = __float2bfloat16_rn(v);
        }
        for (int e = tid; e < BN * BK; e += GEMM_THREADS) {
            int r, c;   // r: n, c: k
            if (g.transB) {
                r = e / BK;
                c = e % BK;
            } else {
                c = e / BN;
                r = e % BN;
            }
            const int n = n0 + r, k = k0 + c;
            float v = 0.f;
            if (n < g.N && k < g.K)
                v = g.transB ? g.B[(long long)n * g.ldb + k] : g.B[(long long)k * g.ldb + n];
            Bs[r][c] = __float2bfloat16_rn(v);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = wm * 32 + mt * 16 + gq;
                af[mt][0] = *(const uint32_t*)&As[r][kk + 2 * tq];
                af[mt][1] = *(const uint32_t*)&As[r + 8][kk + 2 * tq];
                af[mt][2] = *(const uint32_t*)&As[r][kk + 2 * tq + 8];
                af[mt][3] = *(const uint32_t*)&As[r + 8][kk + 2 * tq + 8];
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int n = wn * 32 + nt * 8 + gq;
                bfr[nt][0] = *(const uint32_t*)&Bs[n][kk + 2 * tq];
                bfr[nt][1] = *(const uint32_t*)&Bs[n][kk + 2 * tq + 8];
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bfr[nt]);
        }
        __syncthreads();
    }
    // epilogue: rows gq, gq + 8; columns 2 tq, 2 tq + 1 of every mma tile
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int m = m0 + wm * 32 + mt * 16 + gq + 8 * h;
                    const int n = n0 + wn * 32 + nt * 8 + 2 * tq + cc;
                    if (m >= g.M || n >= g.N) continue;
                    float v = g.alpha * acc[mt][nt][2 * h + cc];
                    const long long o = (long long)m * g.ldc + n;
                    if (g.accumulate) v += g.C[o];
                    if (g.bias) v += g.bias[n];
                    if (g.Z) g.Z[o] = v;
                    if (g.relu) v = fmaxf(v, 0.f);
                    g.C[o] = v;
                }
}

__global__ void relu_backward_kernel(long long n, const float* dA, const float* Z, float* dZ) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dZ[i] = Z[i] > 0.f ? dA[i] : 0.f;
}

// one block per 32 columns; threads stride over rows, partial sums in FP64
__global__ void colsum_kernel(int M, int N, const float* dZ, float* db, int accumulate) {
    __shared__ double part[8][33];
    const int col = blockIdx.x * 32 + (threadIdx.x & 31);
    const int ry = threadIdx.x >> 5;
    double s = 0.0;
    if (col < N)
        for (int m = ry; m < M; m += 8) s += dZ[(long long)m * N + col];
    part[ry][threadIdx.x & 31] = s;
    __syncthreads();
    if (ry == 0 && col < N) {
        double t = 0.0;
        for (int r = 0; r < 8; ++r) t += part[r][threadIdx.x & 31];
        db[col] = accumulate ? db[col] + (float)t : (float)t;
    }
}

__global__ void mse_kernel(long long n, const float* out, const float* y, float* d,
                           double* loss, double count) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float e = out[i] - y[i];
        d[i] = (float)(2.0 * e / count);
        s += (double)e * e;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, s / count);
}

__global__ void adam_kernel(long long n, float* p, const float* g, float* m, float* v, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

int grid_for(long long n, int threads, int sm) {
    return (int)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, 32LL * sm));
}

}  // namespace

int gemm(nop_ctx* ctx, const GemmArgs& g) {
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return NOP_OK;
    // grid.y is limited to 65535 row tiles: taller problems run in row chunks
    const int max_rows = 65535 * BM;
    if (g.M > max_rows) {
        if (g.batch > 1) {
            ctx->set_error("batched GEMM too tall");
            return NOP_EINVAL;
        }
        for (int m0 = 0; m0 < g.M; m0 += max_rows) {
            GemmArgs c = g;
            c.M = std::min(max_rows, g.M - m0);
            c.A = g.transA ? g.A + m0 : g.A + (long long)m0 * g.lda;
            c.C = g.C + (long long)m0 * g.ldc;
            if (g.Z) c.Z = g.Z + (long long)m0 * g.ldc;
            NOP_TRY(gemm(ctx, c));
        }
        return NOP_OK;
    }
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch > 1 ? g.batch : 1);
    const int mk = ctx->phase_begin(1);
    gemm_kernel<<<grid, GEMM_THREADS, 0, ctx->stream>>>(g);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->phase_end(mk);
    ctx->count_launch(false);
    return NOP_OK;
}

int linear(nop_ctx* ctx, int M, int in, int out, const float* X, const float* W,
           const float* b, float* Y, float* Z, bool relu) {
    GemmArgs g{};
    g.M = M;
    g.N = out;
    g.K = in;
    g.A = X;
    g.lda = in;
    g.transA = 0;
    g.B = W;
    g.ldb = in;
    g.transB = 1;
    g.C = Y;
    g.ldc = out;
    g.bias = b;
    g.relu = relu ? 1 : 0;
    g.Z = Z;
    g.alpha = 1.f;
    g.accumulate = 0;
    return gemm(ctx, g);
}

int relu_backward(nop_ctx* ctx, long long n, const float* dA, const float* Z, float* dZ) {
    relu_backward_kernel<<<grid_for(n, 256, ctx->sm_count), 256, 0, ctx->stream>>>(n, dA, Z, dZ);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    return NOP_OK;
}

int colsum(nop_ctx* ctx, int M, int N, const float* dZ, float* db, bool accumulate) {
    colsum_kernel<<<(N + 31) / 32, 256, 0, ctx->stream>>>(M, N, dZ, db, accumulate ? 1 : 0);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    return NOP_OK;
}

int mse_grad(nop_ctx* ctx, long long n, const float* out, const float* y, float* d,
             double* loss, double count) {
    mse_kernel<<<grid_for(n, 256, ctx->sm_count), 256, 0, ctx->stream>>>(n, out, y, d, loss,
                                                                          count);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    return NOP_OK;
}

int adam(nop_ctx* ctx, long long n, float* p, const float* g, float* m, float* v, int t,
         float lr, float b1, float b2, float eps) {
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<grid_for(n, 256, ctx->sm_count), 256, 0, ctx->stream>>>(n, p, g, m, v, lr, b1,
                                                                           b2, eps, c1, c2);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    return NOP_OK;
}

}  // namespace nop
