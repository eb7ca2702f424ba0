// DeepONet solution operator (Sec. 4.1, Eq. 11) and the equation-recast
// iteration around it (Sec. 3.1 Eq. 7, Sec. 3.2 Eq. 8, Sec. 5.1 Eq. 24).
//
// Network: branch MLP on `sensors` source values, trunk MLP on x/length,
// output <branch, trunk>; ReLU after hidden layers.  Matrix products run on
// BF16 tensor cores with FP32 accumulation: the GEMM of nn_kernels.cu in
// general, the fused recast step (recast_fused.cu) and the tcgen05 trunk
// evaluation (trunk_tc.cu) for the 128-sensor, 4 x 128, p = 128 network.
//
// Recast on a batch of slabs: the operator lives on its own grid of M bins
// over [0, L]; each instance's source S and mismatch
// delta = (Sigma_s - Sigma_s*) - (Sigma_t - Sigma_t*) are averaged onto the
// bins (overlap weights) once, then every iteration applies the operator to
// src = P S + (P delta) u through the linear scaling
// sigma+ N[src+/sigma+] - sigma- N[src-/sigma-] (each signed part at unit
// integral, sigma+- = h sum max(+-src, 0)), giving branch
// coefficients beta and u_new = T_ref beta with T_ref the trunk at the bin
// centres.  Converged instances freeze.  The final flux at the instance's own
// cell centres is beta . trunk(x_c), with the trunk evaluated once per
// distinct cell centre of the batch.
#include <algorithm>
#include <numeric>
#include <cmath>
#include <cstdio>
#include <vector>

#include <cuda_bf16.h>

#include "nn_kernels.cuh"

namespace nop {

int no_layout(const nop_no_config* c, std::vector<long long>* off, std::vector<long long>* len,
              long long* total) {
    off->clear();
    len->clear();
    long long o = 0;
    auto push = [&](long long n) {
        off->push_back(o);
        len->push_back(n);
        o += n;
    };
    if (c->width < 1 || c->depth < 1) return NOP_EINVAL;
    if (c->kind == NOP_NO_DEEPONET) {
        if (c->sensors < 1 || c->basis < 1 || c->depth < 2) return NOP_EINVAL;
        for (int net = 0; net < 2; ++net)
            for (int l = 0; l < c->depth; ++l) {
                const int in = l == 0 ? (net == 0 ? c->sensors : 1) : c->width;
                const int out = l == c->depth - 1 ? c->basis : c->width;
                push((long long)out * in);
                push(out);
            }
    } else if (c->kind == NOP_NO_FNO1D || c->kind == NOP_NO_FNO2D) {
        if (c->modes < 1 || c->proj < 1) return NOP_EINVAL;
        const int W = c->width, in_ch = c->kind == NOP_NO_FNO1D ? 2 : 3;
        push((long long)W * in_ch);
        push(W);
        for (int l = 0; l < c->depth; ++l) {
            const long long spec = c->kind == NOP_NO_FNO1D
                                       ? (long long)c->modes * W * W
                                       : (long long)c->modes * c->modes * W * W;
            const int nspec = c->kind == NOP_NO_FNO1D ? 2 : 4;
            for (int k = 0; k < nspec; ++k) push(spec);
            push((long long)W * W);
            push(W);
        }
        push((long long)c->proj * W);
        push(c->proj);
        push(c->proj);
        push(1);
    } else {
        return NOP_EINVAL;
    }
    *total = o;
    return NOP_OK;
}

namespace {

// tensor index of layer l of net (0 branch, 1 trunk): W at 2*(net*depth+l), b at +1
inline const float* Wp(nop_ctx* ctx, int net, int l) {
    return ctx->no.params + ctx->no.off[2 * (net * ctx->no.cfg.depth + l)];
}
inline const float* Bp(nop_ctx* ctx, int net, int l) {
    return ctx->no.params + ctx->no.off[2 * (net * ctx->no.cfg.depth + l) + 1];
}
inline float* dWp(nop_ctx* ctx, int net, int l) {
    return ctx->no.grad + ctx->no.off[2 * (net * ctx->no.cfg.depth + l)];
}
inline float* dBp(nop_ctx* ctx, int net, int l) {
    return ctx->no.grad + ctx->no.off[2 * (net * ctx->no.cfg.depth + l) + 1];
}
inline int dim_in(const nop_no_config& c, int net, int l) {
    return l == 0 ? (net == 0 ? c.sensors : 1) : c.width;
}
inline int dim_out(const nop_no_config& c, int l) { return l == c.depth - 1 ? c.basis : c.width; }

// activation buffers of one net: A[l], Z[l] of rows x width (max)
int acts(nop_ctx* ctx, int net, int rows, std::vector<float*>* A, std::vector<float*>* Z) {
    const nop_no_config& c = ctx->no.cfg;
    const int wmax = c.width > c.basis ? c.width : c.basis;
    A->resize(c.depth);
    Z->resize(c.depth);
    for (int l = 0; l < c.depth; ++l) {
        char na[32], nz[32];
        snprintf(na, sizeof na, "don_A%d_%d", net, l);
        snprintf(nz, sizeof nz, "don_Z%d_%d", net, l);
        void* p;
        NOP_TRY(ctx->scratch(na, sizeof(float) * (size_t)rows * wmax, &p));
        (*A)[l] = (float*)p;
        NOP_TRY(ctx->scratch(nz, sizeof(float) * (size_t)rows * wmax, &p));
        (*Z)[l] = (float*)p;
    }
    return NOP_OK;
}

int mlp_forward(nop_ctx* ctx, int net, int rows, const float* X, float** out, bool keep) {
    const nop_no_config& c = ctx->no.cfg;
    std::vector<float*> A, Z;
    NOP_TRY(acts(ctx, net, rows, &A, &Z));
    const float* h = X;
    for (int l = 0; l < c.depth; ++l) {
        const bool relu = l < c.depth - 1;
        NOP_TRY(linear(ctx, rows, dim_in(c, net, l), dim_out(c, l), h, Wp(ctx, net, l),
                       Bp(ctx, net, l), A[l], keep ? Z[l] : nullptr, relu));
        h = A[l];
    }
    *out = A[c.depth - 1];
    return NOP_OK;
}

int mlp_backward(nop_ctx* ctx, int net, int rows, const float* X, const float* dout) {
    const nop_no_config& c = ctx->no.cfg;
    std::vector<float*> A, Z;
    NOP_TRY(acts(ctx, net, rows, &A, &Z));
    void* p;
    const int wmax = c.width > c.basis ? c.width : c.basis;
    NOP_TRY(ctx->scratch(net ? "don_gT0" : "don_gB0", sizeof(float) * (size_t)rows * wmax, &p));
    float* g0 = (float*)p;
    NOP_TRY(ctx->scratch(net ? "don_gT1" : "don_gB1", sizeof(float) * (size_t)rows * wmax, &p));
    float* g1 = (float*)p;
    const float* g = dout;
    for (int l = c.depth - 1; l >= 0; --l) {
        const int in = dim_in(c, net, l), out = dim_out(c, l);
        const float* dZ = g;
        if (l < c.depth - 1) {
            float* t = (g == g0) ? g1 : g0;
            NOP_TRY(relu_backward(ctx, (long long)rows * out, g, Z[l], t));
            dZ = t;
        }
        const float* hin = l == 0 ? X : A[l - 1];
        GemmArgs w{};
        w.M = out;
        w.N = in;
        w.K = rows;
        w.A = dZ;
        w.lda = out;
        w.transA = 1;
        w.B = hin;
        w.ldb = in;
        w.transB = 0;
        w.C = dWp(ctx, net, l);
        w.ldc = in;
        w.alpha = 1.f;
        NOP_TRY(gemm(ctx, w));
        NOP_TRY(colsum(ctx, rows, out, dZ, dBp(ctx, net, l), false));
        if (l > 0) {
            float* t = (dZ == g0) ? g1 : g0;
            GemmArgs d{};
            d.M = rows;
            d.N = in;
            d.K = out;
            d.A = dZ;
            d.lda = out;
            d.B = Wp(ctx, net, l);
            d.ldb = in;
            d.transB = 0;
            d.C = t;
            d.ldc = in;
            d.alpha = 1.f;
            NOP_TRY(gemm(ctx, d));
            g = t;
        }
    }
    return NOP_OK;
}

// ------------------------------------------------------------ recast kernels
// Overlap-weighted bin averages of cell fields: bins of width h = L/M, cells
// of width dx = L/I of instance b, one thread per bin.  out0 receives the
// average of `field` (when given), out1 (when given) that of the recast
// mismatch (Sigma_s - Sigma_s*) - (Sigma_t - Sigma_t*), both from one pass
// over the bin's cells.  The cell edges are taken relative to the bin's left
// edge (found in FP64 once per bin), so the overlaps and sums run in FP32
// without the rounding of positions far from the origin.
__global__ void project_kernel(int B, int M, const long long* cell_off, const int* ncell,
                               const double* width, const double* field, const double* sigt,
                               const double* sigs, double st_star, double ss_star, float* out0,
                               float* out1) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)B * M) return;
    const int b = (int)(e / M), m = (int)(e % M);
    const int I = ncell[b];
    const double L = width[b], h = L / M, dx = L / I;
    const double lo = m * h;
    int i0 = (int)floor(lo / dx);
    int i1 = (int)floor((m + 1) * h / dx);
    i0 = max(0, min(I - 1, i0));
    i1 = max(0, min(I - 1, i1));
    const float hf = (float)h, dxf = (float)dx;
    const float left0 = (float)(i0 * dx - lo);   // edge of cell i0 from the bin's edge
    const float sts = (float)st_star, sss = (float)ss_star;
    const long long c0 = cell_off[b];
    float a0 = 0.f, a1 = 0.f;
    for (int i = i0; i <= i1; ++i) {
        const float l = left0 + (float)(i - i0) * dxf;
        const float ov = fminf(hf, l + dxf) - fmaxf(0.f, l);
        if (ov <= 0.f) continue;
        const long long c = c0 + i;
        if (out0) a0 = fmaf(ov, (float)field[c], a0);
        if (out1) a1 = fmaf(ov, ((float)sigs[c] - sss) - ((float)sigt[c] - sts), a1);
    }
    const float ih = 1.0f / hf;
    if (out0) out0[e] = a0 * ih;
    if (out1) out1[e] = a1 * ih;
}

// recast source of bin m: PS + PD u_m (+ PL u_{m-1} + PU u_{m+1} with the
// off-diagonal mismatch bands of a diffusion batch)
__device__ __forceinline__ float recast_src(const float* PS, const float* PD, const float* PL,
                                            const float* PU, const float* u, long long e, int m,
                                            int M) {
    float s = PS[e] + PD[e] * u[e];
    if (PL && m > 0) s += PL[e] * u[e - 1];
    if (PU && m < M - 1) s += PU[e] * u[e + 1];
    return s;
}

// Split and scale the bin sources of every instance (one block per instance):
// src = PS + PD * u (+ off-diagonal terms);  sigma+- = h sum max(+-src, 0);
// rows 2b / 2b+1 of U are src+/sigma+ and src-/sigma- (each part at unit
// integral, as in training).
__global__ void split_kernel(int M, double h, const float* PS, const float* PD, const float* PL,
                             const float* PU, const float* u, float* U, float* sig, int* flags) {
    __shared__ double red[2][32];
    const int b = blockIdx.x;
    // FP32 partial sums per thread, FP64 across threads
    float apf = 0.f, anf = 0.f;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float s = recast_src(PS, PD, PL, PU, u, (long long)b * M + m, m, M);
        if (s > 0.f) apf += s;
        else anf -= s;
    }
    double ap = apf, an = anf;
    for (int o = 16; o > 0; o >>= 1) {
        ap += __shfl_xor_sync(0xffffffffu, ap, o);
        an += __shfl_xor_sync(0xffffffffu, an, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = ap;
        red[1][threadIdx.x >> 5] = an;
    }
    __syncthreads();
    double sp = 0.0, sn = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        sp += red[0][w];
        sn += red[1][w];
    }
    sp *= h;
    sn *= h;
    const float ip = sp > 0 ? (float)(1.0 / sp) : 0.f, in = sn > 0 ? (float)(1.0 / sn) : 0.f;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float s = recast_src(PS, PD, PL, PU, u, (long long)b * M + m, m, M);
        U[(2LL * b) * M + m] = fmaxf(s, 0.f) * ip;
        U[(2LL * b + 1) * M + m] = fmaxf(-s, 0.f) * in;
    }
    if (threadIdx.x == 0) {
        sig[2 * b] = (float)sp;
        sig[2 * b + 1] = (float)sn;
        flags[b] = (sp > 0 ? 1 : 0) | (sn > 0 ? 2 : 0);
    }
}

// beta_b = sigma+ N[+] - sigma- N[-] from the branch outputs of rows 2b, 2b+1
__global__ void beta_kernel(int B, int p, const float* Bn, const float* sig, const int* flags,
                            float* beta) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)B * p) return;
    const int b = (int)(e / p), k = (int)(e % p);
    const int f = flags[b];
    float v = 0.f;
    if (f & 1) v += sig[2 * b] * Bn[(2LL * b) * p + k];
    if (f & 2) v -= sig[2 * b + 1] * Bn[(2LL * b + 1) * p + k];
    beta[e] = v;
}

// Convergence bookkeeping of one recast iteration (one block per instance).
// status: 0 running, 1 converged, 2 not converged (cap), 3 diverged.
__global__ void recast_update_kernel(int M, int p, double tol, int diverge_run, const float* unew,
                                     float* u, const float* beta, float* beta_keep, int* status,
                                     int* iters, double* prev, int* run, int* active) {
    __shared__ double red[2][32];
    const int b = blockIdx.x;
    if (status[b] != 0) return;
    float d2f = 0.f, n2f = 0.f;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const float a = unew[(long long)b * M + m], o = u[(long long)b * M + m];
        d2f += (a - o) * (a - o);
        n2f += a * a;
    }
    double d2 = d2f, n2 = n2f;
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = d2;
        red[1][threadIdx.x >> 5] = n2;
    }
    __syncthreads();
    double D = 0.0, Nn = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        D += red[0][w];
        Nn += red[1][w];
    }
    for (int m = threadIdx.x; m < M; m += blockDim.x) u[(long long)b * M + m] = unew[(long long)b * M + m];
    for (int k = threadIdx.x; k < p; k += blockDim.x)
        beta_keep[(long long)b * p + k] = beta[(long long)b * p + k];
    if (threadIdx.x == 0) {
        iters[b] += 1;
        const double ab = sqrt(D);
        const double ch = Nn > 0 ? ab / sqrt(Nn) : 0.0;
        int st = 0;
        if (!isfinite(ch) || !isfinite(Nn)) {
            st = 3;
        } else if (ch <= tol) {
            st = 1;
        } else {
            run[b] = ab >= prev[b] ? run[b] + 1 : 0;
            prev[b] = ab;
            if (run[b] >= diverge_run) st = 3;
        }
        status[b] = st;
        if (st == 0) atomicAdd(active, 1);
    }
}

// Trunk input column and owning instance of global cells [c0, c0 + n).
__global__ void cell_points_kernel(long long c0, int n, int B, const long long* cell_off,
                                   const int* ncell, float* X, int* inst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long c = c0 + k;
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cell_off[mid] <= c) lo = mid;
        else hi = mid - 1;
    }
    const int i = (int)(c - cell_off[lo]);
    X[k] = (float)((i + 0.5) / ncell[lo]);
    inst[k] = lo;
}

// phi_c = beta_inst(c) . t(x_c), operands rounded to BF16 like the GEMMs
__global__ void trunk_dot_kernel(long long c0, int n, int p, const float* Tn, const int* inst,
                                 const float* beta_keep, const int* status, double* phi) {
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= n) return;
    const int b = inst[k];
    float acc = 0.f;
    if (!status || status[b] != 3)
        for (int j = lane; j < p; j += 32)
            acc += __bfloat162float(__float2bfloat16_rn(beta_keep[(long long)b * p + j])) *
                   __bfloat162float(__float2bfloat16_rn(Tn[(long long)k * p + j]));
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) phi[c0 + k] = acc;
}

// ---- fused trunk evaluation at cell centres (width = basis = 128, depth 4)
// One persistent block of 8 warps holds the three 128 x 128 trunk matrices as
// BF16 in shared memory; each warp owns 16 points of a 128-point tile and runs
// layer 1 (elementwise, K = 1), layers 2-4 on mma.sync (BF16 operands, FP32
// accumulation, activations rounded to BF16 between layers like the generic
// GEMM), then the inner product with its instance's coefficients.
constexpr int FT_W = 128;

__global__ void bin_centres_kernel(int M, float* X) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) X[m] = (float)((m + 0.5) / M);
}

}  // namespace

int deeponet_forward_raw(nop_ctx* ctx, int n, const float* U, int P, const float* X,
                         float* out, bool keep) {
    float *Bn, *Tn;
    NOP_TRY(mlp_forward(ctx, 0, n, U, &Bn, keep));
    NOP_TRY(mlp_forward(ctx, 1, P, X, &Tn, keep));
    GemmArgs g{};
    g.M = n;
    g.N = P;
    g.K = ctx->no.cfg.basis;
    g.A = Bn;
    g.lda = ctx->no.cfg.basis;
    g.B = Tn;
    g.ldb = ctx->no.cfg.basis;
    g.transB = 1;
    g.C = out;
    g.ldc = P;
    g.alpha = 1.f;
    return gemm(ctx, g);
}

// Backward of the last deeponet_forward_raw(keep = true) for dL/dout (n x P).
int deeponet_backward(nop_ctx* ctx, int n, int P, const float* dout, const float* U,
                      const float* X) {
    const nop_no_config& c = ctx->no.cfg;
    std::vector<float*> Ab, Zb, At, Zt;
    NOP_TRY(acts(ctx, 0, n, &Ab, &Zb));
    NOP_TRY(acts(ctx, 1, P, &At, &Zt));
    const float* Bn = Ab[c.depth - 1];
    const float* Tn = At[c.depth - 1];
    void* p;
    NOP_TRY(ctx->scratch("don_dBn", sizeof(float) * (size_t)n * c.basis, &p));
    float* dBn = (float*)p;
    NOP_TRY(ctx->scratch("don_dTn", sizeof(float) * (size_t)P * c.basis, &p));
    float* dTn = (float*)p;
    GemmArgs g{};
    g.M = n;
    g.N = c.basis;
    g.K = P;
    g.A = dout;
    g.lda = P;
    g.B = Tn;
    g.ldb = c.basis;
    g.transB = 0;
    g.C = dBn;
    g.ldc = c.basis;
    g.alpha = 1.f;
    NOP_TRY(gemm(ctx, g));
    GemmArgs h{};
    h.M = P;
    h.N = c.basis;
    h.K = n;
    h.A = dout;
    h.lda = P;
    h.transA = 1;
    h.B = Bn;
    h.ldb = c.basis;
    h.C = dTn;
    h.ldc = c.basis;
    h.alpha = 1.f;
    NOP_TRY(gemm(ctx, h));
    NOP_TRY(mlp_backward(ctx, 0, n, U, dBn));
    NOP_TRY(mlp_backward(ctx, 1, P, X, dTn));
    return NOP_OK;
}

// Operator input map of a host cell field: bin averages per instance.
int deeponet_project(nop_ctx* ctx, const double* field_host, float* out_host) {
    SlabDev& s = ctx->slab;
    const int B = s.n_inst, M = ctx->no.cfg.sensors;
    void* q;
    NOP_TRY(ctx->scratch("pj_field", sizeof(double) * (size_t)s.C, &q));
    double* f = (double*)q;
    NOP_TRY(ctx->scratch("pj_out", sizeof(float) * (size_t)B * M, &q));
    float* o = (float*)q;
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(f, field_host, sizeof(double) * (size_t)s.C,
                                      cudaMemcpyHostToDevice, ctx->stream));
    const long long BM_ = (long long)B * M;
    project_kernel<<<(int)((BM_ + 255) / 256), 256, 0, ctx->stream>>>(
        B, M, s.cell_off_d, s.ncell_d, s.width_d, f, nullptr, nullptr, 0.0, 0.0, o, nullptr);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(out_host, o, sizeof(float) * BM_, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return NOP_OK;
}

// Batched recast (predict_only: one operator application to src_d instead).
// phi_d: device [C] doubles.  status_d / iters_d: device [B] (may be null).
int deeponet_recast(nop_ctx* ctx, double tol, int itmax, double* phi_d, int* status_d,
                    int* iters_d, bool predict_only, const double* src_d) {
    const nop_no_config& c = ctx->no.cfg;
    SlabDev& s = ctx->slab;
    const int B = s.n_inst, M = c.sensors, p = c.basis;
    const double h = c.length / M;
    void* q;
    NOP_TRY(ctx->scratch("rc_PS", sizeof(float) * (size_t)B * M, &q));
    float* PS = (float*)q;
    NOP_TRY(ctx->scratch("rc_PD", sizeof(float) * (size_t)B * M, &q));
    float* PD = (float*)q;
    // off-diagonal bands of the mismatch (diffusion batches; null for transport)
    float *PL = nullptr, *PU = nullptr;
    if (ctx->diffusion) {
        NOP_TRY(ctx->scratch("rc_PLU", sizeof(float) * 2 * (size_t)B * M, &q));
        PL = (float*)q;
        PU = PL + (size_t)B * M;
    }
    NOP_TRY(ctx->scratch("rc_u", sizeof(float) * (size_t)B * M, &q));
    float* u = (float*)q;
    NOP_TRY(ctx->scratch("rc_unew", sizeof(float) * (size_t)B * M, &q));
    float* unew = (float*)q;
    NOP_TRY(ctx->scratch("rc_U", sizeof(float) * (size_t)2 * B * M, &q));
    float* Usp = (float*)q;
    NOP_TRY(ctx->scratch("rc_sig", sizeof(float) * 2 * (size_t)B, &q));
    float* sig = (float*)q;
    NOP_TRY(ctx->scratch("rc_beta", sizeof(float) * (size_t)B * p, &q));
    float* beta = (float*)q;
    NOP_TRY(ctx->scratch("rc_betak", sizeof(float) * (size_t)B * p, &q));
    float* beta_keep = (float*)q;
    NOP_TRY(ctx->scratch("rc_int", sizeof(int) * (size_t)(4 * B + 4), &q));
    int* flags = (int*)q;
    int* status = flags + B;
    int* iters = flags + 2 * B;
    int* run = flags + 3 * B;
    int* active = flags + 4 * B;
    NOP_TRY(ctx->scratch("rc_prev", sizeof(double) * (size_t)B, &q));
    double* prev = (double*)q;
    NOP_TRY(ctx->scratch("rc_Xb", sizeof(float) * (size_t)M, &q));
    float* Xb = (float*)q;
    NOP_TRY(ctx->scratch("rc_Tref", sizeof(float) * (size_t)M * p, &q));
    float* Tref = (float*)q;

    const int mk = ctx->phase_begin(1);
    const long long BM_ = (long long)B * M;
    // the source on the bins, and (transport) the mismatch from the same pass
    project_kernel<<<(int)((BM_ + 255) / 256), 256, 0, ctx->stream>>>(
        B, M, s.cell_off_d, s.ncell_d, s.width_d, predict_only ? src_d : ctx->src_d,
        ctx->sigt_d, ctx->sigs_d, c.sigma_t_star, c.sigma_s_star, PS,
        ctx->diffusion ? nullptr : PD);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    if (ctx->diffusion) {
        // Table 1: -dL of -(D u')' + Sigma_a u on the bins; the operator's p*
        // is (D*, Sigma_a*) = (sigma_t_star, sigma_s_star) of its configuration
        NOP_TRY(diffusion_bands(ctx, M, c.sigma_t_star, c.sigma_s_star, PL, PD, PU));
    }
    if (predict_only) {
        NOP_CUDA_TRY(ctx, cudaMemsetAsync(PD, 0, sizeof(float) * BM_, ctx->stream));
        PL = PU = nullptr;
    }
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(u, 0, sizeof(float) * BM_, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)(4 * B + 4), ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(prev, 0x7f, sizeof(double) * (size_t)B, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(beta_keep, 0, sizeof(float) * (size_t)B * p, ctx->stream));
    // trunk at the bin centres
    bin_centres_kernel<<<(M + 127) / 128, 128, 0, ctx->stream>>>(M, Xb);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    float* Tn;
    NOP_TRY(mlp_forward(ctx, 1, M, Xb, &Tn, false));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(Tref, Tn, sizeof(float) * (size_t)M * p,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    const int imax = predict_only ? 1 : itmax;
    int it = 0;
    int rc = NOP_OK;
    if (recast_fused_supported(c)) {
        const float* const Wl[4] = {Wp(ctx, 0, 0), Wp(ctx, 0, 1), Wp(ctx, 0, 2), Wp(ctx, 0, 3)};
        const float* const bl[4] = {Bp(ctx, 0, 0), Bp(ctx, 0, 1), Bp(ctx, 0, 2), Bp(ctx, 0, 3)};
        rc = recast_fused_run(ctx, B, h, predict_only ? 1e300 : tol, imax, PS, PD, PL, PU, u, Wl,
                              bl, Tref, beta, beta_keep, status, iters, prev, run, active, &it);
        if (rc != NOP_OK) return rc;
        it = imax + 1;   // skip the generic loop
    }
    int* active_h = nullptr;
    NOP_TRY(ctx->pinned("rc_active", sizeof(int), &q));
    active_h = (int*)q;
    for (it = it == 0 ? 1 : it; it <= imax; ++it) {
        split_kernel<<<B, 128, 0, ctx->stream>>>(M, h, PS, PD, PL, PU, u, Usp, sig, flags);
        if (cudaGetLastError() != cudaSuccess) { rc = NOP_ECUDA; break; }
        ctx->count_launch(false);
        float* Bn;
        if ((rc = mlp_forward(ctx, 0, 2 * B, Usp, &Bn, false)) != NOP_OK) break;
        beta_kernel<<<(int)(((long long)B * p + 255) / 256), 256, 0, ctx->stream>>>(B, p, Bn, sig,
                                                                                  flags, beta);
        if (cudaGetLastError() != cudaSuccess) { rc = NOP_ECUDA; break; }
        ctx->count_launch(false);
        GemmArgs g{};
        g.M = B;
        g.N = M;
        g.K = p;
        g.A = beta;
        g.lda = p;
        g.B = Tref;
        g.ldb = p;
        g.transB = 1;
        g.C = unew;
        g.ldc = M;
        g.alpha = 1.f;
        if ((rc = gemm(ctx, g)) != NOP_OK) break;
        if (cudaMemsetAsync(active, 0, sizeof(int), ctx->stream) != cudaSuccess) { rc = NOP_ECUDA; break; }
        recast_update_kernel<<<B, 128, 0, ctx->stream>>>(M, p, predict_only ? 1e300 : tol, 5, unew,
                                                        u, beta, beta_keep, status, iters, prev,
                                                        run, active);
        if (cudaGetLastError() != cudaSuccess) { rc = NOP_ECUDA; break; }
        ctx->count_launch(false);
        // converged instances are frozen, so the host checks for completion
        // only every few iterations
        if (it % 4 != 0 && it != imax) continue;
        if (cudaMemcpyAsync(active_h, active, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            rc = NOP_ECUDA;
            break;
        }
        if (*active_h == 0) break;
    }
    if (rc != NOP_OK) {
        ctx->set_error("recast iteration failed");
        return rc;
    }
    // final flux at every cell centre
    const long long C = s.C;
    if (c.width == FT_W && c.basis == FT_W && c.depth == 4) {
        // instances grouped by cell count (CSR): distinct points once; the
        // grouping depends on the batch layout only, so it is built and
        // uploaded once per problem
        NOP_TRY(ctx->scratch("ft_gpt", sizeof(long long) * (B + 1), &q));
        long long* gpt_d = (long long*)q;
        NOP_TRY(ctx->scratch("ft_gint", sizeof(int) * (3 * (size_t)B + 1), &q));
        int* gI_d = (int*)q;
        if (s.ft_version != s.layout_version) {
            std::vector<int> order(B);
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(),
                             [&](int x, int y) { return s.ncell[x] < s.ncell[y]; });
            std::vector<long long> gpt(1, 0);
            std::vector<int> gI, ginst(1, 0);
            for (int k = 0; k < B; ++k) {
                const int I = s.ncell[order[k]];
                if (gI.empty() || gI.back() != I) {
                    if (!gI.empty()) ginst.push_back(k);
                    gI.push_back(I);
                    gpt.push_back(gpt.back() + I);
                }
            }
            ginst.push_back(B);
            const int NG = (int)gI.size();
            const long long P = gpt.back();
            std::vector<int> ints(gI);
            ints.insert(ints.end(), ginst.begin(), ginst.end());
            ints.insert(ints.end(), order.begin(), order.end());
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(gpt_d, gpt.data(), sizeof(long long) * (NG + 1),
                                              cudaMemcpyHostToDevice, ctx->stream));
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(gI_d, ints.data(), sizeof(int) * ints.size(),
                                              cudaMemcpyHostToDevice, ctx->stream));
            // per 128-point tile: first and last group, instance range
            const long long ntile = (P + 127) / 128;
            std::vector<int4> tinfo((size_t)ntile);
            int gg = 0;
            for (long long tt = 0; tt < ntile; ++tt) {
                const long long p0 = tt * 128, p1 = std::min(P, p0 + 128) - 1;
                while (gpt[gg + 1] <= p0) ++gg;
                int gl = gg;
                while (gpt[gl + 1] <= p1) ++gl;
                tinfo[(size_t)tt] = make_int4(gg, gl, ginst[gg], ginst[gl + 1]);
            }
            NOP_TRY(ctx->scratch("ft_tinfo", sizeof(int4) * (size_t)ntile, &q));
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(q, tinfo.data(), sizeof(int4) * (size_t)ntile,
                                              cudaMemcpyHostToDevice, ctx->stream));
            // the host vectors go out of scope: let the copies finish (once
            // per problem)
            NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            s.ft_groups = NG;
            s.ft_points = P;
            s.ft_version = s.layout_version;
        }
        const int NG = s.ft_groups;
        const long long P = s.ft_points;
        int* ginst_d = gI_d + NG;
        int* list_d = ginst_d + NG + 1;
        NOP_TRY(ctx->scratch("ft_tinfo", sizeof(int4) * (size_t)((P + 127) / 128), &q));
        int4* tinfo_d = (int4*)q;
        NOP_TRY(ctx->scratch("tc_err", sizeof(int), &q));
        int* err_d = (int*)q;
        NOP_CUDA_TRY(ctx, cudaMemsetAsync(err_d, 0, sizeof(int), ctx->stream));
        const float* const TW[4] = {Wp(ctx, 1, 0), Wp(ctx, 1, 1), Wp(ctx, 1, 2), Wp(ctx, 1, 3)};
        const float* const TB[4] = {Bp(ctx, 1, 0), Bp(ctx, 1, 1), Bp(ctx, 1, 2), Bp(ctx, 1, 3)};
        NOP_TRY(trunk_tc_launch(ctx, P, tinfo_d, gpt_d, gI_d, ginst_d, list_d, s.cell_off_d, TW,
                                TB, beta_keep, status, phi_d, err_d));
        ctx->phase_end(mk);
        NOP_TRY(ctx->pinned("tc_err", sizeof(int), &q));
        int* herr = (int*)q;
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(herr, err_d, sizeof(int), cudaMemcpyDeviceToHost,
                                          ctx->stream));
        if (ctx->defer_tc_check) {
            // the caller reads the flag after its own final synchronisation
            ctx->tc_err_pending = herr;
        } else {
            NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            if (*herr) {
                ctx->set_error("trunk evaluation: tensor-core completion wait timed out");
                return NOP_ETIMEOUT;
            }
        }
        if (status_d)
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(status_d, status, sizeof(int) * B,
                                              cudaMemcpyDeviceToDevice, ctx->stream));
        if (iters_d)
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(iters_d, iters, sizeof(int) * B,
                                              cudaMemcpyDeviceToDevice, ctx->stream));
        return NOP_OK;
    }
    const int CH = 1 << 16;
    NOP_TRY(ctx->scratch("rc_Xc", sizeof(float) * CH, &q));
    float* Xc = (float*)q;
    NOP_TRY(ctx->scratch("rc_inst", sizeof(int) * CH, &q));
    int* inst = (int*)q;
    for (long long c0 = 0; c0 < C; c0 += CH) {
        const int n = (int)std::min<long long>(CH, C - c0);
        cell_points_kernel<<<(n + 255) / 256, 256, 0, ctx->stream>>>(c0, n, B, s.cell_off_d,
                                                                    s.ncell_d, Xc, inst);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        ctx->count_launch(false);
        float* Tc;
        NOP_TRY(mlp_forward(ctx, 1, n, Xc, &Tc, false));
        trunk_dot_kernel<<<(n + 7) / 8, 256, 0, ctx->stream>>>(c0, n, p, Tc, inst, beta_keep,
                                                               status, phi_d);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        ctx->count_launch(false);
    }
    ctx->phase_end(mk);
    if (status_d)
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(status_d, status, sizeof(int) * B,
                                          cudaMemcpyDeviceToDevice, ctx->stream));
    if (iters_d)
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(iters_d, iters, sizeof(int) * B,
                                          cudaMemcpyDeviceToDevice, ctx->stream));
    return NOP_OK;
}


// Steps of the recast iteration shared with the FNO (operator grid of M points).
int recast_split(nop_ctx* ctx, int B, int M, double h, const float* PS, const float* PD,
                 const float* u, float* U, float* sig, int* flags) {
    split_kernel<<<B, 128, 0, ctx->stream>>>(M, h, PS, PD, nullptr, nullptr, u, U, sig, flags);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    return NOP_OK;
}

int recast_combine(nop_ctx* ctx, int B, int M, const float* out, const float* sig,
                   const int* flags, float* res) {
    beta_kernel<<<(int)(((long long)B * M + 255) / 256), 256, 0, ctx->stream>>>(B, M, out, sig,
                                                                              flags, res);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    return NOP_OK;
}

int recast_update(nop_ctx* ctx, int B, int M, double tol, const float* unew, float* u,
                  int* status, int* iters, double* prev, int* run, int* active) {
    recast_update_kernel<<<B, 128, 0, ctx->stream>>>(M, 0, tol, 5, unew, u, nullptr, nullptr,
                                                    status, iters, prev, run, active);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    return NOP_OK;
}

}  // namespace nop
