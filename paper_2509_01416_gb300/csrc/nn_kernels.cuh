// Dense building blocks of the neural operators: a BF16 tensor-core GEMM with
// FP32 accumulation and a fused bias/ReLU epilogue, and the elementwise
// kernels of training (ReLU masks, bias gradients, MSE, Adam).
#pragma once
#include <cuda_bf16.h>

#include "nop_internal.cuh"

namespace nop {

// C[M x N] = act(alpha * op(A) op(B) + bias) (+ C when accumulate).
//   op(A) is M x K: transA = 0 -> A[m * lda + k], 1 -> A[k * lda + m]
//   op(B) is K x N: transB = 0 -> B[k * ldb + n], 1 -> B[n * ldb + k]
// Operands are FP32 in memory and rounded to BF16 (nearest even) when staged;
// products accumulate in FP32.  Z (optional) receives the pre-activation.
// batch > 1 runs that many problems with operand offsets sA, sB, sC (Z and
// bias are not batched).
struct GemmArgs {
    int M, N, K;
    const float* A;
    int lda, transA;
    const float* B;
    int ldb, transB;
    float* C;
    int ldc;
    const float* bias;
    int relu;
    float* Z;
    float alpha;
    int accumulate;
    // strided batch (blockIdx.z): element offsets between consecutive problems
    int batch;
    long long sA, sB, sC;
};

int gemm(nop_ctx* ctx, const GemmArgs& g);

// Y = X W^T + b with optional ReLU (W is [out][in] row-major): the layer of an MLP.
int linear(nop_ctx* ctx, int M, int in, int out, const float* X, const float* W,
           const float* b, float* Y, float* Z, bool relu);

// dZ = dA * (Z > 0)
int relu_backward(nop_ctx* ctx, long long n, const float* dA, const float* Z, float* dZ);
// db[n] (+)= sum_m dZ[m * N + n]
int colsum(nop_ctx* ctx, int M, int N, const float* dZ, float* db, bool accumulate);
// d = 2 (out - y) / count; loss += sum (out - y)^2 / count (FP64, device scalar)
int mse_grad(nop_ctx* ctx, long long n, const float* out, const float* y, float* d,
             double* loss, double count);
// Adam (Kingma & Ba) on n parameters, step t (1-based).
int adam(nop_ctx* ctx, long long n, float* p, const float* g, float* m, float* v, int t,
         float lr, float b1, float b2, float eps);

}  // namespace nop
