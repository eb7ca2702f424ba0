// The whole recast iteration (Sec. 5.1 Eq. 24) in one launch for the
// DeepONet of 128 sensors, four 128-wide branch layers and 128 basis
// functions.  Every iteration of an instance: split of the recast source into
// unit-integral parts, the branch MLP on both parts, the coefficients beta =
// sigma+ N[+] - sigma- N[-], the operator-grid flux u = T_ref beta and the
// convergence bookkeeping.  Instances are independent, so a CTA iterates its
// tile of 16 instances until all of them are frozen (converged, diverged) or
// the cap is reached, with no grid-wide step in between.
//
// A persistent CTA per SM keeps the four branch weight matrices and T_ref in
// shared memory as BF16 (the operand precision of the GEMM path), staged once
// per launch, and walks tiles of 16 instances (32 rows: the positive and
// negative part of each); the products run on mma.sync BF16 tensor-core
// instructions with FP32 accumulation, bias and ReLU in FP32.
#include <cuda_bf16.h>

#include <algorithm>

#include "nop_internal.cuh"

namespace nop {
namespace {

constexpr int RF_W = 128, RF_LD = RF_W + 8, RF_NI = 16, RF_ROWS = 2 * RF_NI, RF_THREADS = 256;
constexpr size_t RF_SMEM = sizeof(__nv_bfloat16) * (5 * RF_W * RF_LD + 2 * RF_ROWS * RF_LD) +
                           sizeof(float) * (RF_ROWS * (RF_W + 4) + 4 * RF_W + 2 * RF_NI) +
                           sizeof(int) * RF_NI;

struct RfArgs {
    int B;
    float h;
    double tol;
    int diverge_run;
    const float* PS;
    const float* PD;
    const float* PL;            // off-diagonal mismatch bands (diffusion), or null
    const float* PU;
    float* u;
    const __nv_bfloat16* Wbf;   // [5][128][128]: branch layers 1-4 ([out][in]), T_ref ([m][k])
    const float* bias[4];
    float* beta;
    float* beta_keep;
    int* status;
    int* iters;
    double* prev;
    int* run;
    int itmax;                  // recast iterations at most
};

__device__ __forceinline__ void rf_mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                       uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// acc[MT x 16 rows][16 columns from n0] = A[rows][128] . Wt[n][128]^T
template <int MT>
__device__ __forceinline__ void rf_tile(const __nv_bfloat16 (*A)[RF_LD],
                                        const __nv_bfloat16 (*Wt)[RF_LD], int n0, int lane,
                                        float (&acc)[MT][2][4]) {
    const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[mt][nt][c] = 0.f;
#pragma unroll
    for (int kk = 0; kk < RF_W; kk += 16) {
        uint32_t af[MT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const int r = mt * 16 + gq;
            af[mt][0] = *(const uint32_t*)&A[r][kk + 2 * tq];
            af[mt][1] = *(const uint32_t*)&A[r + 8][kk + 2 * tq];
            af[mt][2] = *(const uint32_t*)&A[r][kk + 2 * tq + 8];
            af[mt][3] = *(const uint32_t*)&A[r + 8][kk + 2 * tq + 8];
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int n = n0 + nt * 8 + gq;
            const uint32_t b0 = *(const uint32_t*)&Wt[n][kk + 2 * tq];
            const uint32_t b1 = *(const uint32_t*)&Wt[n][kk + 2 * tq + 8];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) rf_mma(acc[mt][nt], af[mt], b0, b1);
        }
    }
}

__device__ __forceinline__ float warp_sumf(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sumd(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(RF_THREADS, 1) recast_fused_kernel(RfArgs a) {
    extern __shared__ __align__(16) unsigned char rf_smem[];
    __nv_bfloat16(*W)[RF_W][RF_LD] = (__nv_bfloat16(*)[RF_W][RF_LD])rf_smem;
    __nv_bfloat16(*Ha)[RF_LD] =
        (__nv_bfloat16(*)[RF_LD])(rf_smem + sizeof(__nv_bfloat16) * 5 * RF_W * RF_LD);
    __nv_bfloat16(*Hb)[RF_LD] = Ha + RF_ROWS;
    float(*O)[RF_W + 4] = (float(*)[RF_W + 4])(Hb + RF_ROWS);
    float(*bs)[RF_W] = (float(*)[RF_W])(O + RF_ROWS);
    float* spv = (float*)(bs + 4);
    float* snv = spv + RF_NI;
    int* flv = (int*)(snv + RF_NI);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // stage the five BF16 matrices with 16-byte copies into padded rows
    for (int e = tid; e < 5 * RF_W * (RF_W / 8); e += RF_THREADS) {
        const int mtx = e / (RF_W * (RF_W / 8));
        const int r = (e / (RF_W / 8)) % RF_W, c8 = e % (RF_W / 8);
        *(uint4*)&W[mtx][r][c8 * 8] = ((const uint4*)a.Wbf)[e];
    }
    for (int e = tid; e < 4 * RF_W; e += RF_THREADS) bs[e / RF_W][e % RF_W] = a.bias[e / RF_W][e % RF_W];
    __syncthreads();

    const int gq = lane >> 2, tq = lane & 3, n0 = 16 * warp;
    const int ntiles = (a.B + RF_NI - 1) / RF_NI;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    for (int it = 0; it < a.itmax; ++it) {
        // a tile whose instances are all frozen (converged or diverged) is
        // done
        {
            const int b = tile * RF_NI + (tid & (RF_NI - 1));
            const int running = tid < RF_NI && b < a.B && a.status[b] == 0;
            if (!__syncthreads_or(running)) break;
        }
        // 1. recast source S + D u of two instances per warp, split into parts
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = 2 * warp + q, b = tile * RF_NI + i;
            float s[4];
            float ap = 0.f, an = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int m = lane + 32 * j;
                const long long e = (long long)b * RF_W + m;
                s[j] = 0.f;
                if (b < a.B) {
                    s[j] = a.PS[e] + a.PD[e] * a.u[e];
                    if (a.PL && m > 0) s[j] += a.PL[e] * a.u[e - 1];
                    if (a.PU && m < RF_W - 1) s[j] += a.PU[e] * a.u[e + 1];
                }
                if (s[j] > 0.f) ap += s[j];
                else an -= s[j];
            }
            const float sp = warp_sumf(ap) * a.h, sn = warp_sumf(an) * a.h;
            const float ip = sp > 0.f ? 1.f / sp : 0.f, in = sn > 0.f ? 1.f / sn : 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int m = lane + 32 * j;
                Ha[2 * i][m] = __float2bfloat16_rn(fmaxf(s[j], 0.f) * ip);
                Ha[2 * i + 1][m] = __float2bfloat16_rn(fmaxf(-s[j], 0.f) * in);
            }
            if (lane == 0) {
                spv[i] = sp;
                snv[i] = sn;
                flv[i] = (sp > 0.f ? 1 : 0) | (sn > 0.f ? 2 : 0);
            }
        }
        __syncthreads();
        // 2. branch MLP on the 32 rows: Ha -> Hb -> Ha -> Hb -> O
        __nv_bfloat16(*src)[RF_LD] = Ha;
        __nv_bfloat16(*dst)[RF_LD] = Hb;
        for (int l = 0; l < 4; ++l) {
            float acc[2][2][4];
            rf_tile<2>(src, W[l], n0, lane, acc);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh)
#pragma unroll
                        for (int cc = 0; cc < 2; ++cc) {
                            const int row = mt * 16 + gq + 8 * hh, col = n0 + nt * 8 + 2 * tq + cc;
                            const float v = acc[mt][nt][2 * hh + cc] + bs[l][col];
                            if (l < 3) dst[row][col] = __float2bfloat16_rn(fmaxf(v, 0.f));
                            else O[row][col] = v;
                        }
            __syncthreads();
            __nv_bfloat16(*t)[RF_LD] = src;
            src = dst;
            dst = t;
        }
        // 3. beta = sigma+ N[+] - sigma- N[-] (rows 2i, 2i+1), BF16 copy in Ha
        for (int e = tid; e < RF_NI * RF_W; e += RF_THREADS) {
            const int i = e / RF_W, n = e % RF_W, f = flv[i];
            float v = 0.f;
            if (f & 1) v += spv[i] * O[2 * i][n];
            if (f & 2) v -= snv[i] * O[2 * i + 1][n];
            Ha[i][n] = __float2bfloat16_rn(v);
            const int b = tile * RF_NI + i;
            if (b < a.B) a.beta[(long long)b * RF_W + n] = v;
        }
        __syncthreads();
        // 4. u = T_ref beta on the 128 bins (16 rows)
        {
            float acc[1][2][4];
            rf_tile<1>(Ha, W[4], n0, lane, acc);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int hh = 0; hh < 2; ++hh)
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc)
                        O[gq + 8 * hh][n0 + nt * 8 + 2 * tq + cc] = acc[0][nt][2 * hh + cc];
        }
        __syncthreads();
        // 5. convergence bookkeeping, two instances per warp
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = 2 * warp + q, b = tile * RF_NI + i;
            if (b >= a.B || a.status[b] != 0) continue;
            float d2 = 0.f, n2 = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int m = lane + 32 * j;
                const long long e = (long long)b * RF_W + m;
                const float nv = O[i][m], d = nv - a.u[e];
                d2 += d * d;
                n2 += nv * nv;
                a.u[e] = nv;
                a.beta_keep[e] = a.beta[e];
            }
            const double D = warp_sumd((double)d2), Nn = warp_sumd((double)n2);
            if (lane == 0) {
                a.iters[b] += 1;
                const double ab = sqrt(D);
                const double ch = Nn > 0 ? ab / sqrt(Nn) : 0.0;
                int st = 0;
                if (!isfinite(ch) || !isfinite(Nn)) {
                    st = 3;
                } else if (ch <= a.tol) {
                    st = 1;
                } else {
                    a.run[b] = ab >= a.prev[b] ? a.run[b] + 1 : 0;
                    a.prev[b] = ab;
                    if (a.run[b] >= a.diverge_run) st = 3;
                }
                a.status[b] = st;
            }
        }
        __syncthreads();
    }
}

__global__ void to_bf16_kernel(int n, const float* x, __nv_bfloat16* y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

}  // namespace

bool recast_fused_supported(const nop_no_config& c) {
    return c.kind == NOP_NO_DEEPONET && c.sensors == RF_W && c.width == RF_W &&
           c.basis == RF_W && c.depth == 4;
}

// The recast loop on the fused kernel (one launch).  active2: unused device
// counters kept for the generic path's signature.  *its: the iteration cap.
int recast_fused_run(nop_ctx* ctx, int B, double h, double tol, int itmax, const float* PS,
                     const float* PD, const float* PL, const float* PU, float* u,
                     const float* const W[4], const float* const b[4],
                     const float* Tref, float* beta, float* beta_keep, int* status, int* iters,
                     double* prev, int* run, int* active2, int* its) {
    void* p;
    NOP_TRY(ctx->scratch("rf_wbf", sizeof(__nv_bfloat16) * 5 * RF_W * RF_W, &p));
    __nv_bfloat16* Wbf = (__nv_bfloat16*)p;
    const int nm = RF_W * RF_W;
    for (int l = 0; l < 5; ++l) {
        to_bf16_kernel<<<(nm + 255) / 256, 256, 0, ctx->stream>>>(nm, l < 4 ? W[l] : Tref,
                                                                  Wbf + (size_t)l * nm);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        ctx->count_launch(false);
    }
    NOP_CUDA_TRY(ctx, cudaFuncSetAttribute(recast_fused_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)RF_SMEM));
    RfArgs a;
    a.B = B;
    a.h = (float)h;
    a.tol = tol;
    a.diverge_run = 5;
    a.PS = PS;
    a.PD = PD;
    a.PL = PL;
    a.PU = PU;
    a.u = u;
    a.Wbf = Wbf;
    for (int l = 0; l < 4; ++l) a.bias[l] = b[l];
    a.beta = beta;
    a.beta_keep = beta_keep;
    a.status = status;
    a.iters = iters;
    a.prev = prev;
    a.run = run;
    a.itmax = itmax;
    const int ntiles = (B + RF_NI - 1) / RF_NI;
    const int grid = std::max(1, std::min(ntiles, ctx->sm_count));
    recast_fused_kernel<<<grid, RF_THREADS, RF_SMEM, ctx->stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) {
        ctx->set_error("fused recast iteration failed");
        return NOP_ECUDA;
    }
    ctx->count_launch(false);
    *its = itmax;
    return NOP_OK;
}

}  // namespace nop
