// Fourier neural operator (Sec. 4.2; App. A1): lift, Fourier layers
// v <- relu(SpectralConv(v) + W v + b), projection W -> proj -> 1.
//
// Activations are stored point-major, act[p][b][c] (p the grid point, x-major
// in 2D: p = x * ny + y), so every pointwise layer is one GEMM over rows
// (p, b) and the truncated transforms are GEMMs over p:
//   1D:  Vhat [2K x (B W)] = F [2K x n] v,      u = E [n x 2K] What,
//        F rows: cos(2 pi k x/n) then -sin(...); E columns c_k/n cos, -c_k/n sin
//        (c_0 = 1, else 2), the inverse of the truncated real spectrum.
//   2D:  along x, Xh [2m x (ny B W)] = Fx v with rows (k_x re, k_x im)
//        interleaved; along y for every k_x (strided batch) the complex
//        product as one real block GEMM, [Vr; Vi] = [[Fr, -Fi], [Fi, Fr]] [Xr; Xi]
//        over k_y in {0..m-1} U {ny-m..ny-1}; the inverse mirrors both steps.
// Per mode the channel mixing What = Vhat R (complex, C_in x C_out) is a small
// kernel.  All GEMMs are the BF16 tensor-core GEMM with FP32 accumulation;
// the mixing rounds its operands to BF16 the same way.  Backward passes are
// the adjoint GEMMs and the transposed mixing.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "nn_kernels.cuh"

namespace nop {
namespace {

struct FnoShape {
    bool two_d;
    int n1, n2;      // 1D: n1 = 1, n2 = n;  2D: n1 = ny, n2 = nx
    int P;           // grid points
    int W, K, L, proj;
    int nmode;       // mixing modes: 1D K; 2D 2m * m
};

FnoShape shape_of(const nop_no_config& c, int n1, int n2) {
    FnoShape s;
    s.two_d = c.kind == NOP_NO_FNO2D;
    s.n1 = n1;
    s.n2 = n2;
    s.P = n1 * n2;
    s.W = c.width;
    s.K = c.modes;
    s.L = c.depth;
    s.proj = c.proj;
    s.nmode = s.two_d ? 2 * c.modes * c.modes : c.modes;
    return s;
}

// parameter tensor indices
inline int t_lift_W() { return 0; }
inline int t_lift_b() { return 1; }
inline int t_spec(const FnoShape& s, int l, int k) { return 2 + l * (s.two_d ? 6 : 4) + k; }
inline int t_pw_W(const FnoShape& s, int l) { return 2 + l * (s.two_d ? 6 : 4) + (s.two_d ? 4 : 2); }
inline int t_pw_b(const FnoShape& s, int l) { return t_pw_W(s, l) + 1; }
inline int t_proj(const FnoShape& s, int k) { return 2 + s.L * (s.two_d ? 6 : 4) + k; }

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---------------------------------------------------------------- matrices
// 1D: F [2K x n], E [n x 2K]
__global__ void dft1d_kernel(int n, int K, float* F, float* E) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)K * n) return;
    const int k = (int)(e / n), x = (int)(e % n);
    double sv, cv;
    sincospi(2.0 * k * x / n, &sv, &cv);
    F[(long long)k * n + x] = (float)cv;
    F[(long long)(K + k) * n + x] = (float)(-sv);
    const double ck = (k == 0 ? 1.0 : 2.0) / n;
    E[(long long)x * 2 * K + k] = (float)(ck * cv);
    E[(long long)x * 2 * K + K + k] = (float)(-ck * sv);
}

// 2D x-step matrices: Fx [2m x nx] (rows 2k re, 2k+1 im), Ex [nx x 2m]
__global__ void dft2d_x_kernel(int nx, int m, float* Fx, float* Ex) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)m * nx) return;
    const int k = (int)(e / nx), x = (int)(e % nx);
    double sv, cv;
    sincospi(2.0 * k * x / nx, &sv, &cv);
    Fx[(long long)(2 * k) * nx + x] = (float)cv;
    Fx[(long long)(2 * k + 1) * nx + x] = (float)(-sv);
    const double ck = (k == 0 ? 1.0 : 2.0) / nx;
    Ex[(long long)x * 2 * m + 2 * k] = (float)(ck * cv);
    Ex[(long long)x * 2 * m + 2 * k + 1] = (float)(-ck * sv);
}

// 2D y-step block matrices: Gy [4m x 2ny] = [[Fr, -Fi], [Fi, Fr]] with
// F = exp(-2 pi i k y/ny); Ey [2ny x 4m] = [[Er, -Ei], [Ei, Er]] with
// E = exp(+2 pi i k y/ny)/ny; k over {0..m-1} U {ny-m..ny-1}.
__global__ void dft2d_y_kernel(int ny, int m, float* Gy, float* Ey) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)2 * m * ny) return;
    const int kf = (int)(e / ny), y = (int)(e % ny);
    const int k = kf < m ? kf : ny - 2 * m + kf;
    double sv, cv;
    sincospi(2.0 * k * y / ny, &sv, &cv);
    const float Fr = (float)cv, Fi = (float)(-sv);
    const int R = 2 * m, Cg = 2 * ny;
    Gy[(long long)kf * Cg + y] = Fr;
    Gy[(long long)kf * Cg + ny + y] = -Fi;
    Gy[(long long)(R + kf) * Cg + y] = Fi;
    Gy[(long long)(R + kf) * Cg + ny + y] = Fr;
    const float Er = (float)(cv / ny), Ei = (float)(sv / ny);
    const int Ce = 4 * m;
    Ey[(long long)y * Ce + kf] = Er;
    Ey[(long long)y * Ce + R + kf] = -Ei;
    Ey[(long long)(ny + y) * Ce + kf] = Ei;
    Ey[(long long)(ny + y) * Ce + R + kf] = Er;
}

// ------------------------------------------------------------ lift / output
// v0[p][b][c] = W[c] . (S_b(p), coords(p)) + b[c]; operands rounded to BF16.
// inputs are [B][points] in the problem's order (2D row-major j*nx + i).
__global__ void lift_kernel(int B, int n1, int n2, int W, bool two_d, const float* in,
                            const float* Wl, const float* bl, float* v) {
    const long long P = (long long)n1 * n2;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= P * B * W) return;
    const int c = (int)(e % W);
    const int b = (int)((e / W) % B);
    const long long p = e / ((long long)W * B);
    long long q;   // point in the problem order
    float x, y = 0.f;
    if (two_d) {
        const int ny = n1, nx = n2;
        const int xi = (int)(p / ny), yj = (int)(p % ny);
        q = (long long)yj * nx + xi;
        x = (float)((xi + 0.5) / nx);
        y = (float)((yj + 0.5) / ny);
    } else {
        q = p;
        x = (float)((p + 0.5) / n2);
    }
    const int in_ch = two_d ? 3 : 2;
    float acc = bfr(in[(long long)b * P + q]) * bfr(Wl[c * in_ch + 0]) + bfr(x) * bfr(Wl[c * in_ch + 1]);
    if (two_d) acc += bfr(y) * bfr(Wl[c * in_ch + 2]);
    v[e] = acc + bl[c];
}

// lift backward: dW[c][j] = sum_{p,b} dv[p][b][c] inp_j, db[c] = sum dv (one block per c)
__global__ void lift_backward_kernel(int B, int n1, int n2, int W, bool two_d, const float* in,
                                     const float* dv, float* dW, float* db) {
    const int c = blockIdx.x;
    const long long P = (long long)n1 * n2;
    double a0 = 0, a1 = 0, a2 = 0, ab = 0;
    for (long long r = threadIdx.x; r < P * B; r += blockDim.x) {
        const int b = (int)(r % B);
        const long long p = r / B;
        long long q;
        float x, y = 0.f;
        if (two_d) {
            const int ny = n1, nx = n2;
            const int xi = (int)(p / ny), yj = (int)(p % ny);
            q = (long long)yj * nx + xi;
            x = (float)((xi + 0.5) / nx);
            y = (float)((yj + 0.5) / ny);
        } else {
            q = p;
            x = (float)((p + 0.5) / n2);
        }
        const float g = dv[r * W + c];
        a0 += (double)bfr(g) * bfr(in[(long long)b * P + q]);
        a1 += (double)bfr(g) * bfr(x);
        a2 += (double)bfr(g) * bfr(y);
        ab += g;
    }
    __shared__ double red[4][32];
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        ab += __shfl_xor_sync(0xffffffffu, ab, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a0;
        red[1][threadIdx.x >> 5] = a1;
        red[2][threadIdx.x >> 5] = a2;
        red[3][threadIdx.x >> 5] = ab;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0, s2 = 0, sb = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
            s2 += red[2][w];
            sb += red[3][w];
        }
        const int in_ch = two_d ? 3 : 2;
        dW[c * in_ch + 0] = (float)s0;
        dW[c * in_ch + 1] = (float)s1;
        if (two_d) dW[c * in_ch + 2] = (float)s2;
        db[c] = (float)sb;
    }
}

// out[b][q] <- o[p][b]  (and the reverse for gradients)
__global__ void to_user_kernel(int B, int n1, int n2, bool two_d, const float* o, float* out,
                               bool reverse) {
    const long long P = (long long)n1 * n2;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= P * B) return;
    const int b = (int)(e % B);
    const long long p = e / B;
    long long q = p;
    if (two_d) {
        const int ny = n1, nx = n2;
        q = (long long)(p % ny) * nx + p / ny;
    }
    if (reverse) out[e] = o[(long long)b * P + q];   // out: [p][b], o: [b][q]
    else out[(long long)b * P + q] = o[e];
}

// ------------------------------------------------------------------ mixing
// V, Wout: [mode-block][B][C] with real rows then imaginary rows (layout
// helpers below); R: real and imaginary [mode][Cin][Cout].
struct MixLayout {
    // element offset of (mode, part, b, c) in the spectrum buffer
    bool two_d;
    int K, m, B, C;
    __device__ __forceinline__ long long at(int mode, int part, int b, int c) const {
        const long long BC = (long long)B * C;
        if (!two_d) return ((long long)(part * K + mode)) * BC + (long long)b * C + c;
        const int kf = mode / m, kx = mode % m;   // kf in [0, 2m)
        return ((long long)kx * 4 * m + part * 2 * m + kf) * BC + (long long)b * C + c;
    }
    __device__ __forceinline__ long long rat(int mode, int c, int o) const {
        // R tensors: 1D [K][C][C]; 2D blocks [m][m][C][C] for kf < m and kf >= m
        if (!two_d) return ((long long)mode * C + c) * C + o;
        const int kf = mode / m, kx = mode % m;
        const int ky = kf < m ? kf : kf - m;
        return (((long long)ky * m + kx) * C + c) * C + o;
    }
};

__device__ __forceinline__ void rsel(const MixLayout& L, int mode, const float* r1, const float* i1,
                                     const float* r2, const float* i2, const float*& rr,
                                     const float*& ri) {
    if (!L.two_d || mode / L.m < L.m) {
        rr = r1;
        ri = i1;
    } else {
        rr = r2;
        ri = i2;
    }
}

__global__ void mix_kernel(MixLayout L, int nmode, const float* V, const float* r1, const float* i1,
                           const float* r2, const float* i2, float* Wo) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)nmode * L.B * L.C) return;
    const int o = (int)(e % L.C);
    const int b = (int)((e / L.C) % L.B);
    const int mode = (int)(e / ((long long)L.C * L.B));
    const float *rr, *ri;
    rsel(L, mode, r1, i1, r2, i2, rr, ri);
    float ar = 0.f, ai = 0.f;
    for (int c = 0; c < L.C; ++c) {
        const float vr = bfr(V[L.at(mode, 0, b, c)]), vi = bfr(V[L.at(mode, 1, b, c)]);
        const long long ro = L.rat(mode, c, o);
        const float Rr = bfr(rr[ro]), Ri = bfr(ri[ro]);
        ar += vr * Rr - vi * Ri;
        ai += vr * Ri + vi * Rr;
    }
    Wo[L.at(mode, 0, b, o)] = ar;
    Wo[L.at(mode, 1, b, o)] = ai;
}

// dV[mode][b][c] = sum_o dW (x) conj(R); the incoming gradient stays FP32
__global__ void mix_dv_kernel(MixLayout L, int nmode, const float* dWs, const float* r1,
                              const float* i1, const float* r2, const float* i2, float* dV) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)nmode * L.B * L.C) return;
    const int c = (int)(e % L.C);
    const int b = (int)((e / L.C) % L.B);
    const int mode = (int)(e / ((long long)L.C * L.B));
    const float *rr, *ri;
    rsel(L, mode, r1, i1, r2, i2, rr, ri);
    float ar = 0.f, ai = 0.f;
    for (int o = 0; o < L.C; ++o) {
        const float gr = dWs[L.at(mode, 0, b, o)], gi = dWs[L.at(mode, 1, b, o)];
        const long long ro = L.rat(mode, c, o);
        const float Rr = bfr(rr[ro]), Ri = bfr(ri[ro]);
        ar += gr * Rr + gi * Ri;
        ai += gi * Rr - gr * Ri;
    }
    dV[L.at(mode, 0, b, c)] = ar;
    dV[L.at(mode, 1, b, c)] = ai;
}

// dR[mode][c][o] = sum_b conj(V) (x) dW, written into the gradient tensors
__global__ void mix_dr_kernel(MixLayout L, int nmode, const float* V, const float* dWs, float* gr1,
                              float* gi1, float* gr2, float* gi2) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)nmode * L.C * L.C) return;
    const int o = (int)(e % L.C);
    const int c = (int)((e / L.C) % L.C);
    const int mode = (int)(e / ((long long)L.C * L.C));
    double ar = 0, ai = 0;
    for (int b = 0; b < L.B; ++b) {
        const float vr = bfr(V[L.at(mode, 0, b, c)]), vi = bfr(V[L.at(mode, 1, b, c)]);
        const float gr = dWs[L.at(mode, 0, b, o)], gi = dWs[L.at(mode, 1, b, o)];
        ar += (double)vr * gr + (double)vi * gi;
        ai += (double)vr * gi - (double)vi * gr;
    }
    const long long ro = L.rat(mode, c, o);
    if (!L.two_d || mode / L.m < L.m) {
        gr1[ro] = (float)ar;
        gi1[ro] = (float)ai;
    } else {
        gr2[ro] = (float)ar;
        gi2[ro] = (float)ai;
    }
}

int launch_grid(long long n) { return (int)std::max<long long>(1, (n + 255) / 256); }

// operator-grid source and mismatch coefficient (Eq. 24) of a one-group problem
__global__ void recast_fields_kernel(long long C, const double* src, const double* sigt,
                                     const double* sigs, double st_star, double ss_star,
                                     int with_delta, float* PS, float* PD) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= C) return;
    PS[c] = (float)src[c];
    PD[c] = with_delta ? (float)((sigs[c] - ss_star) - (sigt[c] - st_star)) : 0.f;
}

// final flux; a diverged instance gets zero
__global__ void recast_out_kernel(int B, int M, const float* u, const int* status, double* phi) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)B * M) return;
    phi[e] = status[e / M] == 3 ? 0.0 : (double)u[e];
}

}  // namespace

// ----------------------------------------------------------------------------
// state of one forward pass kept for the backward pass
namespace {

struct FnoBufs {
    std::vector<float*> v;   // L+1 activations [P][B][W]
    std::vector<float*> z;   // L pre-activations
    std::vector<float*> vh;  // L spectra
    float *h, *hz, *o, *in;  // projection hidden, its pre-activation, output [P][B], inputs
    float *tmpA, *tmpB, *spec2;
    float *F, *E, *Gy, *Ey;  // transform matrices
};

int fno_bufs(nop_ctx* ctx, const FnoShape& s, int B, FnoBufs* f) {
    const long long PBW = (long long)s.P * B * s.W;
    const long long spec = s.two_d ? (long long)s.K * 4 * s.K * B * s.W : 2LL * s.K * B * s.W;
    const long long xh = s.two_d ? 2LL * s.K * s.n1 * B * s.W : 0;
    void* p;
    f->v.resize(s.L + 1);
    f->z.resize(s.L);
    f->vh.resize(s.L);
    for (int l = 0; l <= s.L; ++l) {
        char nm[32];
        snprintf(nm, sizeof nm, "fno_v%d", l);
        NOP_TRY(ctx->scratch(nm, sizeof(float) * PBW, &p));
        f->v[l] = (float*)p;
        if (l < s.L) {
            snprintf(nm, sizeof nm, "fno_z%d", l);
            NOP_TRY(ctx->scratch(nm, sizeof(float) * PBW, &p));
            f->z[l] = (float*)p;
            snprintf(nm, sizeof nm, "fno_vh%d", l);
            NOP_TRY(ctx->scratch(nm, sizeof(float) * spec, &p));
            f->vh[l] = (float*)p;
        }
    }
    NOP_TRY(ctx->scratch("fno_h", sizeof(float) * (size_t)s.P * B * s.proj, &p));
    f->h = (float*)p;
    NOP_TRY(ctx->scratch("fno_hz", sizeof(float) * (size_t)s.P * B * s.proj, &p));
    f->hz = (float*)p;
    NOP_TRY(ctx->scratch("fno_o", sizeof(float) * (size_t)s.P * B, &p));
    f->o = (float*)p;
    NOP_TRY(ctx->scratch("fno_tA", sizeof(float) * std::max(PBW, (long long)s.P * B * s.proj), &p));
    f->tmpA = (float*)p;
    NOP_TRY(ctx->scratch("fno_tB", sizeof(float) * std::max(PBW, std::max(spec, xh)), &p));
    f->tmpB = (float*)p;
    NOP_TRY(ctx->scratch("fno_s2", sizeof(float) * std::max(spec, xh + 1), &p));
    f->spec2 = (float*)p;
    // transform matrices for this grid (rebuilt every call: cheap)
    if (!s.two_d) {
        NOP_TRY(ctx->scratch("fno_F", sizeof(float) * 2 * s.K * s.n2, &p));
        f->F = (float*)p;
        NOP_TRY(ctx->scratch("fno_E", sizeof(float) * 2 * s.K * s.n2, &p));
        f->E = (float*)p;
        dft1d_kernel<<<launch_grid((long long)s.K * s.n2), 256, 0, ctx->stream>>>(s.n2, s.K, f->F, f->E);
        f->Gy = f->Ey = nullptr;
    } else {
        const int nx = s.n2, ny = s.n1, m = s.K;
        NOP_TRY(ctx->scratch("fno_F", sizeof(float) * 2 * m * nx, &p));
        f->F = (float*)p;
        NOP_TRY(ctx->scratch("fno_E", sizeof(float) * 2 * m * nx, &p));
        f->E = (float*)p;
        NOP_TRY(ctx->scratch("fno_Gy", sizeof(float) * 8 * m * ny, &p));
        f->Gy = (float*)p;
        NOP_TRY(ctx->scratch("fno_Ey", sizeof(float) * 8 * m * ny, &p));
        f->Ey = (float*)p;
        dft2d_x_kernel<<<launch_grid((long long)m * nx), 256, 0, ctx->stream>>>(nx, m, f->F, f->E);
        dft2d_y_kernel<<<launch_grid(2LL * m * ny), 256, 0, ctx->stream>>>(ny, m, f->Gy, f->Ey);
    }
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    return NOP_OK;
}

GemmArgs G(int M, int N, int K, const float* A, int lda, int tA, const float* B, int ldb, int tB,
           float* C, int ldc) {
    GemmArgs g{};
    g.M = M;
    g.N = N;
    g.K = K;
    g.A = A;
    g.lda = lda;
    g.transA = tA;
    g.B = B;
    g.ldb = ldb;
    g.transB = tB;
    g.C = C;
    g.ldc = ldc;
    g.alpha = 1.f;
    return g;
}

// forward transform: v [P][BW] -> spectrum (layout of MixLayout)
int spectral_fwd(nop_ctx* ctx, const FnoShape& s, const FnoBufs& f, int BW, const float* v, float* vh) {
    if (!s.two_d) return gemm(ctx, G(2 * s.K, BW, s.n2, f.F, s.n2, 0, v, BW, 0, vh, BW));
    const int nx = s.n2, ny = s.n1, m = s.K;
    NOP_TRY(gemm(ctx, G(2 * m, ny * BW, nx, f.F, nx, 0, v, ny * BW, 0, f.tmpB, ny * BW)));
    GemmArgs g = G(4 * m, BW, 2 * ny, f.Gy, 2 * ny, 0, f.tmpB, BW, 0, vh, BW);
    g.batch = m;
    g.sA = 0;
    g.sB = 2LL * ny * BW;
    g.sC = 4LL * m * BW;
    return gemm(ctx, g);
}

// inverse transform: spectrum -> u [P][BW] (written or accumulated into u)
int spectral_inv(nop_ctx* ctx, const FnoShape& s, const FnoBufs& f, int BW, const float* wh, float* u) {
    if (!s.two_d) return gemm(ctx, G(s.n2, BW, 2 * s.K, f.E, 2 * s.K, 0, wh, BW, 0, u, BW));
    const int nx = s.n2, ny = s.n1, m = s.K;
    GemmArgs g = G(2 * ny, BW, 4 * m, f.Ey, 4 * m, 0, wh, BW, 0, f.tmpB, BW);
    g.batch = m;
    g.sA = 0;
    g.sB = 4LL * m * BW;
    g.sC = 2LL * ny * BW;
    NOP_TRY(gemm(ctx, g));
    return gemm(ctx, G(nx, ny * BW, 2 * m, f.E, 2 * m, 0, f.tmpB, ny * BW, 0, u, ny * BW));
}

// adjoint of spectral_inv: du [P][BW] -> dWh (spectrum layout)
int spectral_inv_T(nop_ctx* ctx, const FnoShape& s, const FnoBufs& f, int BW, const float* du,
                   float* dwh) {
    if (!s.two_d) return gemm(ctx, G(2 * s.K, BW, s.n2, f.E, 2 * s.K, 1, du, BW, 0, dwh, BW));
    const int nx = s.n2, ny = s.n1, m = s.K;
    NOP_TRY(gemm(ctx, G(2 * m, ny * BW, nx, f.E, 2 * m, 1, du, ny * BW, 0, f.tmpB, ny * BW)));
    GemmArgs g = G(4 * m, BW, 2 * ny, f.Ey, 4 * m, 1, f.tmpB, BW, 0, dwh, BW);
    g.batch = m;
    g.sA = 0;
    g.sB = 2LL * ny * BW;
    g.sC = 4LL * m * BW;
    return gemm(ctx, g);
}

// adjoint of spectral_fwd: dVh -> dv [P][BW] (accumulated into dv)
int spectral_fwd_T(nop_ctx* ctx, const FnoShape& s, const FnoBufs& f, int BW, const float* dvh,
                   float* dv) {
    if (!s.two_d) {
        GemmArgs g = G(s.n2, BW, 2 * s.K, f.F, s.n2, 1, dvh, BW, 0, dv, BW);
        g.accumulate = 1;
        return gemm(ctx, g);
    }
    const int nx = s.n2, ny = s.n1, m = s.K;
    GemmArgs g = G(2 * ny, BW, 4 * m, f.Gy, 2 * ny, 1, dvh, BW, 0, f.tmpB, BW);
    g.batch = m;
    g.sA = 0;
    g.sB = 4LL * m * BW;
    g.sC = 2LL * ny * BW;
    NOP_TRY(gemm(ctx, g));
    GemmArgs h = G(nx, ny * BW, 2 * m, f.F, nx, 1, f.tmpB, ny * BW, 0, dv, ny * BW);
    h.accumulate = 1;
    return gemm(ctx, h);
}

MixLayout mix_layout(const FnoShape& s, int B) {
    MixLayout L;
    L.two_d = s.two_d;
    L.K = s.K;
    L.m = s.K;
    L.B = B;
    L.C = s.W;
    return L;
}

const float* P_(nop_ctx* ctx, int t) { return ctx->no.params + ctx->no.off[t]; }
float* G_(nop_ctx* ctx, int t) { return ctx->no.grad + ctx->no.off[t]; }

}  // namespace

// Forward of B samples; inputs [B][points] (device), out [B][points] (device).
int fno_forward_raw(nop_ctx* ctx, int B, const float* in, int n1, int n2, float* out, bool keep) {
    (void)keep;
    const FnoShape s = shape_of(ctx->no.cfg, n1, n2);
    if (s.two_d ? (2 * s.K > n1 || s.K > n2 / 2) : (s.K > n2 / 2)) {
        ctx->set_error("FNO modes exceed the grid");
        return NOP_EINVAL;
    }
    FnoBufs f;
    NOP_TRY(fno_bufs(ctx, s, B, &f));
    const int BW = B * s.W;
    const long long PBW = (long long)s.P * BW;
    lift_kernel<<<launch_grid(PBW), 256, 0, ctx->stream>>>(B, n1, n2, s.W, s.two_d, in,
                                                          P_(ctx, t_lift_W()), P_(ctx, t_lift_b()),
                                                          f.v[0]);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    const MixLayout ML = mix_layout(s, B);
    for (int l = 0; l < s.L; ++l) {
        NOP_TRY(spectral_fwd(ctx, s, f, BW, f.v[l], f.vh[l]));
        const float* r1 = P_(ctx, t_spec(s, l, 0));
        const float* i1 = P_(ctx, t_spec(s, l, 1));
        const float* r2 = s.two_d ? P_(ctx, t_spec(s, l, 2)) : r1;
        const float* i2 = s.two_d ? P_(ctx, t_spec(s, l, 3)) : i1;
        mix_kernel<<<launch_grid((long long)s.nmode * B * s.W), 256, 0, ctx->stream>>>(
            ML, s.nmode, f.vh[l], r1, i1, r2, i2, f.spec2);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        NOP_TRY(spectral_inv(ctx, s, f, BW, f.spec2, f.v[l + 1]));
        // z = u + v W^T + b ; v_{l+1} = relu(z)
        GemmArgs g = G(s.P * B, s.W, s.W, f.v[l], s.W, 0, P_(ctx, t_pw_W(s, l)), s.W, 1, f.v[l + 1], s.W);
        g.accumulate = 1;
        g.bias = P_(ctx, t_pw_b(s, l));
        g.Z = f.z[l];
        g.relu = 1;
        NOP_TRY(gemm(ctx, g));
    }
    NOP_TRY(linear(ctx, s.P * B, s.W, s.proj, f.v[s.L], P_(ctx, t_proj(s, 0)), P_(ctx, t_proj(s, 1)),
                   f.h, f.hz, true));
    NOP_TRY(linear(ctx, s.P * B, s.proj, 1, f.h, P_(ctx, t_proj(s, 2)), P_(ctx, t_proj(s, 3)), f.o,
                   nullptr, false));
    to_user_kernel<<<launch_grid((long long)s.P * B), 256, 0, ctx->stream>>>(B, n1, n2, s.two_d, f.o,
                                                                            out, false);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    // keep the inputs for the lift gradient
    void* p;
    NOP_TRY(ctx->scratch("fno_in", sizeof(float) * (size_t)B * s.P, &p));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(p, in, sizeof(float) * (size_t)B * s.P,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    return NOP_OK;
}

// Backward of the last fno_forward_raw for dL/dout [B][points] (device).
int fno_backward(nop_ctx* ctx, int B, int n1, int n2, const float* dout) {
    const FnoShape s = shape_of(ctx->no.cfg, n1, n2);
    FnoBufs f;
    NOP_TRY(fno_bufs(ctx, s, B, &f));
    const int BW = B * s.W;
    void* p;
    NOP_TRY(ctx->scratch("fno_in", sizeof(float) * (size_t)B * s.P, &p));
    const float* in = (const float*)p;
    NOP_TRY(ctx->scratch("fno_do", sizeof(float) * (size_t)B * s.P, &p));
    float* d_o = (float*)p;
    NOP_TRY(ctx->scratch("fno_dv", sizeof(float) * (size_t)s.P * BW, &p));
    float* dv = (float*)p;
    NOP_TRY(ctx->scratch("fno_dz", sizeof(float) * (size_t)s.P * B * std::max(s.W, s.proj), &p));
    float* dz = (float*)p;
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(ctx->no.grad, 0, sizeof(float) * ctx->no.n_params, ctx->stream));
    to_user_kernel<<<launch_grid((long long)s.P * B), 256, 0, ctx->stream>>>(B, n1, n2, s.two_d, dout,
                                                                            d_o, true);
    // projection layers
    NOP_TRY(gemm(ctx, G(1, s.proj, s.P * B, d_o, 1, 1, f.h, s.proj, 0, G_(ctx, t_proj(s, 2)), s.proj)));
    NOP_TRY(colsum(ctx, s.P * B, 1, d_o, G_(ctx, t_proj(s, 3)), false));
    NOP_TRY(gemm(ctx, G(s.P * B, s.proj, 1, d_o, 1, 0, P_(ctx, t_proj(s, 2)), s.proj, 0, f.tmpA, s.proj)));
    NOP_TRY(relu_backward(ctx, (long long)s.P * B * s.proj, f.tmpA, f.hz, dz));
    NOP_TRY(gemm(ctx, G(s.proj, s.W, s.P * B, dz, s.proj, 1, f.v[s.L], s.W, 0, G_(ctx, t_proj(s, 0)), s.W)));
    NOP_TRY(colsum(ctx, s.P * B, s.proj, dz, G_(ctx, t_proj(s, 1)), false));
    NOP_TRY(gemm(ctx, G(s.P * B, s.W, s.proj, dz, s.proj, 0, P_(ctx, t_proj(s, 0)), s.W, 0, dv, s.W)));
    const MixLayout ML = mix_layout(s, B);
    for (int l = s.L - 1; l >= 0; --l) {
        NOP_TRY(relu_backward(ctx, (long long)s.P * BW, dv, f.z[l], dz));
        // pointwise path
        NOP_TRY(gemm(ctx, G(s.W, s.W, s.P * B, dz, s.W, 1, f.v[l], s.W, 0, G_(ctx, t_pw_W(s, l)), s.W)));
        NOP_TRY(colsum(ctx, s.P * B, s.W, dz, G_(ctx, t_pw_b(s, l)), false));
        NOP_TRY(gemm(ctx, G(s.P * B, s.W, s.W, dz, s.W, 0, P_(ctx, t_pw_W(s, l)), s.W, 0, dv, s.W)));
        // spectral path: dWh = inv^T dz; dR, dVh from the mixing; dv += fwd^T dVh
        NOP_TRY(spectral_inv_T(ctx, s, f, BW, dz, f.spec2));
        const float* r1 = P_(ctx, t_spec(s, l, 0));
        const float* i1 = P_(ctx, t_spec(s, l, 1));
        const float* r2 = s.two_d ? P_(ctx, t_spec(s, l, 2)) : r1;
        const float* i2 = s.two_d ? P_(ctx, t_spec(s, l, 3)) : i1;
        float* g1 = G_(ctx, t_spec(s, l, 0));
        float* gi1 = G_(ctx, t_spec(s, l, 1));
        float* g2 = s.two_d ? G_(ctx, t_spec(s, l, 2)) : g1;
        float* gi2 = s.two_d ? G_(ctx, t_spec(s, l, 3)) : gi1;
        mix_dr_kernel<<<launch_grid((long long)s.nmode * s.W * s.W), 256, 0, ctx->stream>>>(
            ML, s.nmode, f.vh[l], f.spec2, g1, gi1, g2, gi2);
        // dVh into tmpA (spectrum layout), then dv += F^T dVh
        mix_dv_kernel<<<launch_grid((long long)s.nmode * B * s.W), 256, 0, ctx->stream>>>(
            ML, s.nmode, f.spec2, r1, i1, r2, i2, f.tmpA);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        NOP_TRY(spectral_fwd_T(ctx, s, f, BW, f.tmpA, dv));
    }
    lift_backward_kernel<<<s.W, 256, 0, ctx->stream>>>(B, n1, n2, s.W, s.two_d, in, dv,
                                                       G_(ctx, t_lift_W()), G_(ctx, t_lift_b()));
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    return NOP_OK;
}

// Eq. 24 with an FNO: phi <- N[S + ((Sigma_s - Sigma_s*) - (Sigma_t - Sigma_t*)) phi]
// from phi = 0 on the instance grid (FNO-1D: every slab of the batch has the
// same cell count; FNO-2D: the x-y rectangle).  Sources are applied part by
// part at unit integral (Eq. 13), cell size from the operator's domain length.
int fno_recast(nop_ctx* ctx, double tol, int itmax, double* phi_d, int* status_d, int* iters_d,
               bool predict_only, const double* src_d) {
    const nop_no_config& c = ctx->no.cfg;
    int B, n1, n2;
    double h;
    if (c.kind == NOP_NO_FNO1D) {
        if (ctx->geometry != NOP_GEOM_SLAB) {
            ctx->set_error("FNO-1D operates on slab problems");
            return NOP_EINVAL;
        }
        const SlabDev& sl = ctx->slab;
        for (int b = 1; b < sl.n_inst; ++b)
            if (sl.ncell[b] != sl.ncell[0]) {
                ctx->set_error("FNO-1D recast needs instances with equal cell counts");
                return NOP_EINVAL;
            }
        B = sl.n_inst;
        n1 = 1;
        n2 = sl.ncell[0];
        h = c.length / n2;
    } else {
        if (ctx->geometry != NOP_GEOM_XY) {
            ctx->set_error("FNO-2D operates on x-y problems");
            return NOP_EINVAL;
        }
        B = 1;
        n1 = ctx->xy.ny;
        n2 = ctx->xy.nx;
        h = (c.length / n2) * (c.length / n1);
    }
    const int M = n1 * n2;
    const long long BM = (long long)B * M;
    void* q;
    NOP_TRY(ctx->scratch("fr_PS", sizeof(float) * BM, &q));
    float* PS = (float*)q;
    NOP_TRY(ctx->scratch("fr_PD", sizeof(float) * BM, &q));
    float* PD = (float*)q;
    NOP_TRY(ctx->scratch("fr_u", sizeof(float) * BM, &q));
    float* u = (float*)q;
    NOP_TRY(ctx->scratch("fr_unew", sizeof(float) * BM, &q));
    float* unew = (float*)q;
    NOP_TRY(ctx->scratch("fr_U", sizeof(float) * 2 * BM, &q));
    float* U = (float*)q;
    NOP_TRY(ctx->scratch("fr_out", sizeof(float) * 2 * BM, &q));
    float* out = (float*)q;
    NOP_TRY(ctx->scratch("fr_sig", sizeof(float) * 2 * (size_t)B, &q));
    float* sig = (float*)q;
    NOP_TRY(ctx->scratch("fr_int", sizeof(int) * (size_t)(4 * B + 4), &q));
    int* flags = (int*)q;
    int* status = flags + B;
    int* iters = flags + 2 * B;
    int* run = flags + 3 * B;
    int* active = flags + 4 * B;
    NOP_TRY(ctx->scratch("fr_prev", sizeof(double) * (size_t)B, &q));
    double* prev = (double*)q;

    const int mk = ctx->phase_begin(1);
    recast_fields_kernel<<<launch_grid(BM), 256, 0, ctx->stream>>>(
        BM, predict_only ? src_d : ctx->src_d, ctx->sigt_d, ctx->sigs_d, c.sigma_t_star,
        c.sigma_s_star, predict_only ? 0 : 1, PS, PD);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(u, 0, sizeof(float) * BM, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)(4 * B + 4), ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(prev, 0x7f, sizeof(double) * (size_t)B, ctx->stream));
    int* active_h = nullptr;
    {
        void* ph;
        NOP_TRY(ctx->pinned("fno_active", sizeof(int), &ph));
        active_h = (int*)ph;
    }
    const int imax = predict_only ? 1 : itmax;
    int rc = NOP_OK;
    for (int it = 1; it <= imax; ++it) {
        if ((rc = recast_split(ctx, B, M, h, PS, PD, u, U, sig, flags)) != NOP_OK) break;
        if ((rc = fno_forward_raw(ctx, 2 * B, U, n1, n2, out, false)) != NOP_OK) break;
        // rows 2b and 2b+1 of the output are N[+] and N[-] of instance b
        if ((rc = recast_combine(ctx, B, M, out, sig, flags, unew)) != NOP_OK) break;
        if (cudaMemsetAsync(active, 0, sizeof(int), ctx->stream) != cudaSuccess) {
            rc = NOP_ECUDA;
            break;
        }
        if ((rc = recast_update(ctx, B, M, predict_only ? 1e300 : tol, unew, u, status, iters,
                                prev, run, active)) != NOP_OK)
            break;
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
        if (ctx->err.empty()) ctx->set_error("FNO recast iteration failed");
        return rc;
    }
    recast_out_kernel<<<launch_grid(BM), 256, 0, ctx->stream>>>(B, M, u, status, phi_d);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    ctx->phase_end(mk);
    if (status_d)
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(status_d, status, sizeof(int) * B,
                                          cudaMemcpyDeviceToDevice, ctx->stream));
    if (iters_d)
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(iters_d, iters, sizeof(int) * B,
                                          cudaMemcpyDeviceToDevice, ctx->stream));
    return NOP_OK;
}

}  // namespace nop
