// 2D x-y S_N solver: level-symmetric S8, diamond difference, source iteration
// and power iteration (the paper's method in two dimensions, Sec. 6;
// multigroup coupling of Sec. 5.3 Eq. 27-29 with upscatter allowed; the k
// update of App. A2 Eq. A2-A4).
//
// Layout.  Every field is stored column-major inside a group, [g][i][j] with
// the y index j fastest, so that the threads of a sweep, which own rows j,
// touch consecutive addresses at every step.  Inputs and outputs cross in the
// row-major [g][j][i] of the C ABI and are transposed at set-up and finish.
//
// Sweep kernel.  One CTA sweeps one group, one quadrant and a pack of ND
// directions of that quadrant over the whole mesh: thread t owns row t in
// sweep order and, at wavefront step s, processes column s - t for its ND
// directions (independent dependency chains).  The x-edge fluxes stay in
// registers along the row; the y-edge flux of a column passes from row t to
// row t + 1 by a warp shuffle, and across a warp boundary through a
// double-buffered shared-memory slot (one barrier per step).  The angle sum
// of the pack goes to its own partial array (no atomics, so FP32 results are
// deterministic), and a combine kernel adds the partials of all packs and
// quadrants into the group's flux.  Diamond difference in increment form,
// with c_x = 2|mu|/dx, c_y = 2|eta|/dy, D = sigma_t + c_x + c_y:
//     psi_c - psi_x = (q + c_y psi_y - (sigma_t + c_y) psi_x) / D,
//     psi_x' = psi_x + 2 (psi_c - psi_x),   psi_y' = psi_y + 2 (psi_c - psi_y),
// the edge fluxes carried with compensated sums in FP32.
//
// Iteration.  Default: Jacobi in energy with the reflected inflow of the
// previous iteration -- every group and quadrant of an iteration is swept in
// one launch (8 groups x 4 quadrants x 5 packs of 2 directions = 160 CTAs on
// the 8-group workload); the fixed point is the transport solution, as for
// any source iteration, and only the path to it differs.  NOP_GAUSS_SEIDEL:
// groups in order with the newest fluxes, quadrants in the order (-,-);
// (+,-) and (-,+); (+,+) with the newest reflected flux (the oracle's
// iteration, Sec. 5.3).  A one-thread control kernel closes every iteration
// on the device (change norm, stopping test, iteration count), and the
// kernels of an iteration enqueued after convergence return at once, so the
// host reads the state back only every few iterations.
#include <algorithm>
#include <cmath>

#include "nop_internal.cuh"

namespace nop {
namespace {

constexpr int MAXN = 1024;   // rows per mesh (threads per sweep CTA)
constexpr int XY_ND = 2;     // directions per thread
constexpr int XY_NP = 10 / XY_ND;   // direction packs per quadrant
constexpr int XY_BATCH = 8;  // iterations enqueued between host checks

// device control block of the inner iteration
struct XYCtl {
    int done;      // stopping test met (or cap, or non-finite change)
    int its;       // iterations completed
    int status;    // NOP_OK, NOP_ENOCONV (cap), NOP_ENAN
    int pad;
    double change; // relative change of the last iteration
    double acc[2]; // sum (phi_new - phi_old)^2, sum phi_new^2 of the running iteration
};

template <typename T>
struct XYArgs {
    int nx, ny;
    long long C;
    double dx, dy;
    const double* mu;
    const double* eta;
    const double* w;
    const int* mir_x;
    const int* mir_y;
    const T* sigt;       // [G][nx][ny] column-major
    const T* q;          // [G][nx][ny] emission
    T* part;             // [G][4][XY_NP][nx][ny] partial angle sums
    const T* in_x;       // [G][40][ny] outgoing flux through the x-face a direction leaves (read)
    const T* in_y;       // [G][40][nx]
    T* out_x;            // the same, written
    T* out_y;
    int g0, q0;          // first group and quadrant of the launch
    int bc_x0, bc_xL, bc_y0, bc_yL;
    const XYCtl* ctl;
};

template <typename T>
__device__ __forceinline__ T rcp_xy(T d) {
    return T(1) / d;
}
// FP32: the special-function reciprocal refined by one Newton step
template <>
__device__ __forceinline__ float rcp_xy<float>(float d) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return fmaf(r, fmaf(-d, r, 1.0f), r);
}

template <typename T>
__global__ void __launch_bounds__(MAXN) xy_sweep_kernel(XYArgs<T> a) {
    if (a.ctl->done) return;
    __shared__ T ybh[2][MAXN / 32][XY_ND], ybl[2][MAXN / 32][XY_ND];
    const int g = a.g0 + blockIdx.z, qd = a.q0 + blockIdx.y, pk = blockIdx.x;
    const int d0 = qd * 10 + pk * XY_ND;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nx = a.nx, ny = a.ny;
    const bool xp = a.mu[d0] > 0, yp = a.eta[d0] > 0;
    const bool rx = xp ? a.bc_x0 : a.bc_xL;   // reflective face the x-inflow enters through
    const bool ry = yp ? a.bc_y0 : a.bc_yL;
    T cx[XY_ND], cy[XY_ND], wd[XY_ND], sxy[XY_ND];
    int mx[XY_ND], my[XY_ND];
#pragma unroll
    for (int k = 0; k < XY_ND; ++k) {
        const int d = d0 + k;
        cx[k] = (T)(2.0 * fabs(a.mu[d]) / a.dx);
        cy[k] = (T)(2.0 * fabs(a.eta[d]) / a.dy);
        sxy[k] = cx[k] + cy[k];
        wd[k] = (T)a.w[d];
        mx[k] = a.mir_x[d];
        my[k] = a.mir_y[d];
    }
    const int jp = t < ny ? (yp ? t : ny - 1 - t) : 0;
    const long long gC = (long long)g * a.C;
    const long long gx = (long long)g * 40;
    // x-edge flux of every direction along the row (compensated)
    T xh[XY_ND], xl[XY_ND];
#pragma unroll
    for (int k = 0; k < XY_ND; ++k) {
        xh[k] = (t < ny && rx) ? a.in_x[(gx + mx[k]) * ny + jp] : T(0);
        xl[k] = T(0);
    }
    // y-edge flux entering this row at the current column (from row t - 1)
    T yh[XY_ND], yl[XY_ND];
#pragma unroll
    for (int k = 0; k < XY_ND; ++k) yh[k] = yl[k] = T(0);
    T* part = a.part + ((long long)(g * 4 + qd) * XY_NP + pk) * a.C;
    const T* st = a.sigt + gC;
    const T* qq = a.q + gC;
    // operands of step s (and, for row 0, the reflected y-inflow of its
    // column) are loaded PF steps ahead
    constexpr int PF = 4;
    T sgr[PF], qr[PF], yir[PF][XY_ND];
    auto fetch = [&](int s, int p) {
        const int i = s - t;
        if (t < ny && i >= 0 && i < nx) {
            const int ipf = xp ? i : nx - 1 - i;
            const long long c = (long long)ipf * ny + jp;
            sgr[p] = st[c];
            qr[p] = qq[c];
            if (t == 0)
#pragma unroll
                for (int k = 0; k < XY_ND; ++k)
                    yir[p][k] = ry ? a.in_y[(gx + my[k]) * nx + ipf] : T(0);
        }
    };
#pragma unroll
    for (int p = 0; p < PF; ++p) {
        sgr[p] = T(1);
        qr[p] = T(0);
#pragma unroll
        for (int k = 0; k < XY_ND; ++k) yir[p][k] = T(0);
        fetch(p, p);
    }
    const int S = nx + ny - 1;
    for (int s0 = 0; s0 < S; s0 += PF)
#pragma unroll
        for (int p = 0; p < PF; ++p) {
            const int s = s0 + p;
            if (s >= S) break;   // uniform over the block
            const T sg = sgr[p], qv = qr[p];
            // the inflow of the first row comes from the y-face
            if (t == 0)
#pragma unroll
                for (int k = 0; k < XY_ND; ++k) {
                    yh[k] = yir[p][k];
                    yl[k] = T(0);
                }
            fetch(s + PF, p);
            const int i = s - t;   // column in sweep order
            const bool active = t < ny && i >= 0 && i < nx;
            const int ip = xp ? i : nx - 1 - i;
            T oh[XY_ND], ol[XY_ND];
            if (active) {
                T phi = T(0);
#pragma unroll
                for (int k = 0; k < XY_ND; ++k) {
                    const T r = rcp_xy<T>(sg + sxy[k]);
                    const T dxs = (qv + cy[k] * yh[k] - (sg + cy[k]) * xh[k]) * r;   // psi_c - psi_x
                    const T dys = (qv + cx[k] * xh[k] - (sg + cx[k]) * yh[k]) * r;   // psi_c - psi_y
                    phi += wd[k] * (xh[k] + (dxs + xl[k]));
                    {
                        const T u = (dxs + dxs) + xl[k];
                        const T tt = xh[k] + u;
                        xl[k] = u - (tt - xh[k]);
                        xh[k] = tt;
                    }
                    {
                        const T u = (dys + dys) + yl[k];
                        const T tt = yh[k] + u;
                        ol[k] = u - (tt - yh[k]);
                        oh[k] = tt;
                    }
                }
                const long long c = (long long)ip * ny + jp;
                part[c] = phi;
                if (i == nx - 1)
#pragma unroll
                    for (int k = 0; k < XY_ND; ++k) a.out_x[(gx + d0 + k) * ny + jp] = xh[k] + xl[k];
                if (t == ny - 1)
#pragma unroll
                    for (int k = 0; k < XY_ND; ++k) a.out_y[(gx + d0 + k) * nx + ip] = oh[k] + ol[k];
            } else {
#pragma unroll
                for (int k = 0; k < XY_ND; ++k) oh[k] = ol[k] = T(0);
            }
            // hand the outgoing y-flux to the next row for the next step
#pragma unroll
            for (int k = 0; k < XY_ND; ++k) {
                const T h = __shfl_up_sync(0xffffffffu, oh[k], 1);
                const T l = __shfl_up_sync(0xffffffffu, ol[k], 1);
                if (lane == 31) {
                    ybh[s & 1][warp][k] = oh[k];
                    ybl[s & 1][warp][k] = ol[k];
                }
                yh[k] = h;
                yl[k] = l;
            }
            __syncthreads();
            if (lane == 0 && warp > 0)
#pragma unroll
                for (int k = 0; k < XY_ND; ++k) {
                    yh[k] = ybh[s & 1][warp - 1][k];
                    yl[k] = ybl[s & 1][warp - 1][k];
                }
        }
}

// emission of groups [g0, g0 + ng): q = sum_g' Sigma_s(g'->g) phi_g' + ext_g
template <typename T>
__global__ void xy_emission_kernel(long long C, int G, int g0, int ng, const T* sigs,
                                   const T* phi, const T* ext, T* q, const XYCtl* ctl) {
    if (ctl->done) return;
    const long long n = (long long)ng * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int g = g0 + (int)(e / C);
        const long long c = e % C;
        T s = ext[(long long)g * C + c];
        for (int gp = 0; gp < G; ++gp)
            s += sigs[((long long)gp * G + g) * C + c] * phi[(long long)gp * C + c];
        q[(long long)g * C + c] = s;
    }
}

// new flux of groups [g0, g0 + ng) from the partial sums; change norms
template <typename T>
__global__ void xy_combine_kernel(long long C, int g0, int ng, const T* part, T* phi,
                                  XYCtl* ctl) {
    if (ctl->done) return;
    double d2 = 0.0, n2 = 0.0;
    const long long n = (long long)ng * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int g = g0 + (int)(e / C);
        const long long c = e % C;
        const T* pg = part + (long long)g * 4 * XY_NP * C + c;
        T v = T(0);
        for (int p = 0; p < 4 * XY_NP; ++p) v += pg[(long long)p * C];
        const T old = phi[(long long)g * C + c];
        const double df = (double)v - (double)old;
        d2 += df * df;
        n2 += (double)v * (double)v;
        phi[(long long)g * C + c] = v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&ctl->acc[0], d2);
        atomicAdd(&ctl->acc[1], n2);
    }
}

// closes an iteration: relative change, stopping test, iteration count
__global__ void xy_control_kernel(XYCtl* ctl, double tol, int itmax) {
    if (ctl->done) return;
    const double d2 = ctl->acc[0], n2 = ctl->acc[1];
    const double ch = n2 > 0 ? sqrt(d2 / n2) : (d2 > 0 ? INFINITY : 0.0);
    ctl->acc[0] = ctl->acc[1] = 0.0;
    ctl->its += 1;
    ctl->change = ch;
    if (!isfinite(ch)) {
        ctl->status = NOP_ENAN;
        ctl->done = 1;
    } else if (ch <= tol) {
        ctl->done = 1;
    } else if (ctl->its >= itmax) {
        ctl->status = NOP_ENOCONV;
        ctl->done = 1;
    }
}

__global__ void xy_ctl_reset_kernel(XYCtl* ctl) {
    ctl->done = 0;
    ctl->its = 0;
    ctl->status = NOP_OK;
    ctl->change = 0.0;
    ctl->acc[0] = ctl->acc[1] = 0.0;
}

// row-major [g][j][i] FP64 -> column-major [g][i][j] T
template <typename T>
__global__ void xy_prepare_kernel(int nx, int ny, int G, const double* sigt, const double* sigs,
                                  const double* src, const double* nsf, const double* phi0,
                                  int flat, T* sigtT, T* sigsT, T* ext, T* nsfT, T* phi) {
    const long long C = (long long)nx * ny, GC = (long long)G * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < GC;
         e += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(e / C);
        const long long r = e - (long long)g * C;   // row-major cell j * nx + i
        const int j = (int)(r / nx), i = (int)(r % nx);
        const long long t = (long long)g * C + (long long)i * ny + j;
        sigtT[t] = (T)sigt[e];
        ext[t] = src ? (T)src[e] : T(0);
        if (nsf) nsfT[t] = (T)nsf[e];
        phi[t] = phi0 ? (T)phi0[e] : (flat ? T(1) : T(0));
        for (int gp = 0; gp < G; ++gp)
            sigsT[((long long)gp * G + g) * C + (long long)i * ny + j] =
                (T)sigs[((long long)gp * G + g) * C + r];
    }
}

template <typename T>
__global__ void xy_finish_kernel(int nx, int ny, long long GC, const T* phi, double* out) {
    const long long C = (long long)nx * ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < GC;
         e += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(e / C);
        const long long r = e - (long long)g * C;
        const int j = (int)(r / nx), i = (int)(r % nx);
        out[e] = (double)phi[(long long)g * C + (long long)i * ny + j];
    }
}

// production sum nsf phi (FP64) into acc[0]
template <typename T>
__global__ void xy_production_kernel(long long GC, const T* nsf, const T* phi, double* acc) {
    double s = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < GC;
         e += (long long)gridDim.x * blockDim.x)
        s += (double)nsf[e] * (double)phi[e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

// outer-iteration step: phi *= 1/P, change vs previous into acc[0..1]
template <typename T>
__global__ void xy_normalize_kernel(long long GC, T sc, T* phi, const T* prev, double* acc) {
    double d2 = 0.0, n2 = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < GC;
         e += (long long)gridDim.x * blockDim.x) {
        const T v = phi[e] * sc;
        phi[e] = v;
        const double df = (double)v - (double)prev[e];
        d2 += df * df;
        n2 += (double)v * (double)v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, d2);
        atomicAdd(acc + 1, n2);
    }
}

// frozen fission source ext_g = chi_g F / k and the previous flux
template <typename T>
__global__ void xy_fission_kernel(long long C, int G, double inv_k, const double* chi, const T* nsf,
                                  const T* phi, T* ext, T* prev) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        double F = 0.0;
        for (int g = 0; g < G; ++g) {
            F += (double)nsf[(long long)g * C + c] * (double)phi[(long long)g * C + c];
            prev[(long long)g * C + c] = phi[(long long)g * C + c];
        }
        for (int g = 0; g < G; ++g) ext[(long long)g * C + c] = (T)(chi[g] * F * inv_k);
    }
}

template <typename T>
__global__ void xy_scale_kernel(long long n, T sc, T* x) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        x[e] *= sc;
}

__global__ void mirror_kernel(const double* mu, const double* eta, int* mx, int* my) {
    const int d = threadIdx.x;
    if (d >= 40) return;
    int bx = 0, by = 0;
    double ex = 1e300, ey = 1e300;
    for (int e = 0; e < 40; ++e) {
        const double fx = fabs(mu[e] + mu[d]) + fabs(eta[e] - eta[d]);
        const double fy = fabs(mu[e] - mu[d]) + fabs(eta[e] + eta[d]);
        if (fx < ex) { ex = fx; bx = e; }
        if (fy < ey) { ey = fy; by = e; }
    }
    mx[d] = bx;
    my[d] = by;
}

int grid_of(long long n, int sm) {
    return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8LL * sm));
}

template <typename T>
int run(nop_ctx* ctx, const nop_solve_opts* o, bool eigen, const double* phi0, double k0,
        double* phi_out, bool out_dev, double* k_out, nop_stats* st) {
    XYDev& xy = ctx->xy;
    const int G = ctx->G, nx = xy.nx, ny = xy.ny;
    const long long C = (long long)nx * ny, GC = (long long)G * C;
    if (ny > MAXN) {
        ctx->set_error("x-y meshes are limited to 1024 rows");
        return NOP_EINVAL;
    }
    const bool gs = (o->flags & NOP_GAUSS_SEIDEL) != 0;
    void* p;
    NOP_TRY(ctx->scratch("xy_sigt", sizeof(T) * GC, &p));
    T* sigt = (T*)p;
    NOP_TRY(ctx->scratch("xy_sigs", sizeof(T) * G * GC, &p));
    T* sigs = (T*)p;
    NOP_TRY(ctx->scratch("xy_ext", sizeof(T) * GC, &p));
    T* ext = (T*)p;
    NOP_TRY(ctx->scratch("xy_nsf", sizeof(T) * (eigen ? GC : 1), &p));
    T* nsf = (T*)p;
    NOP_TRY(ctx->scratch("xy_phi", sizeof(T) * GC, &p));
    T* phi = (T*)p;
    NOP_TRY(ctx->scratch("xy_prev", sizeof(T) * (eigen ? GC : 1), &p));
    T* prev = (T*)p;
    NOP_TRY(ctx->scratch("xy_q", sizeof(T) * GC, &p));
    T* q = (T*)p;
    NOP_TRY(ctx->scratch("xy_part", sizeof(T) * (size_t)GC * 4 * XY_NP, &p));
    T* part = (T*)p;
    // boundary outflows: two buffers (the Jacobi iteration reads the previous
    // iteration's and writes the other); Gauss-Seidel uses buffer 0 alone
    const size_t nbx = (size_t)G * 40 * ny, nby = (size_t)G * 40 * nx;
    NOP_TRY(ctx->scratch("xy_outx", sizeof(T) * 2 * nbx, &p));
    T* outx = (T*)p;
    NOP_TRY(ctx->scratch("xy_outy", sizeof(T) * 2 * nby, &p));
    T* outy = (T*)p;
    NOP_TRY(ctx->scratch("xy_mir", sizeof(int) * 80, &p));
    int* mir = (int*)p;
    NOP_TRY(ctx->scratch("xy_ctl", sizeof(XYCtl) + 4 * sizeof(double), &p));
    XYCtl* ctl = (XYCtl*)p;
    double* acc = (double*)(ctl + 1);
    NOP_TRY(ctx->pinned("xy_ctl_h", sizeof(XYCtl) + 4 * sizeof(double), &p));
    XYCtl* ctl_h = (XYCtl*)p;
    double* acc_h = (double*)(ctl_h + 1);
    const double* phi0_d = nullptr;
    if (phi0) {
        if (o->flags & NOP_PHI0_DEVICE) {
            phi0_d = phi0;
        } else {
            NOP_TRY(ctx->scratch("xy_phi0", sizeof(double) * GC, &p));
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(p, phi0, sizeof(double) * GC, cudaMemcpyHostToDevice,
                                              ctx->stream));
            phi0_d = (const double*)p;
        }
    }
    const int gb = grid_of(GC, ctx->sm_count);
    int mk = ctx->phase_begin(2);
    xy_prepare_kernel<T><<<gb, 256, 0, ctx->stream>>>(nx, ny, G, ctx->sigt_d, ctx->sigs_d,
                                                      eigen ? nullptr : ctx->src_d,
                                                      eigen ? ctx->nsf_d : nullptr, phi0_d,
                                                      (eigen && !phi0_d) ? 1 : 0, sigt, sigs, ext,
                                                      nsf, phi);
    mirror_kernel<<<1, 64, 0, ctx->stream>>>(xy.mu_d, xy.eta_d, mir, mir + 40);
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(outx, 0, sizeof(T) * 2 * nbx, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(outy, 0, sizeof(T) * 2 * nby, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->phase_end(mk);
    ctx->count_launch(false);
    ctx->count_launch(false);

    XYArgs<T> a;
    a.nx = nx;
    a.ny = ny;
    a.C = C;
    a.dx = xy.lx / nx;
    a.dy = xy.ly / ny;
    a.mu = xy.mu_d;
    a.eta = xy.eta_d;
    a.w = xy.w_d;
    a.mir_x = mir;
    a.mir_y = mir + 40;
    a.sigt = sigt;
    a.q = q;
    a.part = part;
    a.bc_x0 = ctx->bc[0];
    a.bc_xL = ctx->bc[1];
    a.bc_y0 = ctx->bc[2];
    a.bc_yL = ctx->bc[3];
    a.ctl = ctl;
    const int threads = ((ny + 31) / 32) * 32;
    const int gc = grid_of(GC, ctx->sm_count);

    // one source iteration enqueued (parity: the boundary buffer it writes)
    auto enqueue_si = [&](int parity) -> int {
        if (gs) {
            a.in_x = a.out_x = outx;
            a.in_y = a.out_y = outy;
            for (int g = 0; g < G; ++g) {
                xy_emission_kernel<T><<<grid_of(C, ctx->sm_count), 256, 0, ctx->stream>>>(
                    C, G, g, 1, sigs, phi, ext, q, ctl);
                ctx->count_launch(false);
                a.g0 = g;
                const int mks = ctx->phase_begin(0);
                // quadrants (-,-) | (+,-) and (-,+) | (+,+), newest reflected flux
                a.q0 = 0;
                xy_sweep_kernel<T><<<dim3(XY_NP, 1, 1), threads, 0, ctx->stream>>>(a);
                a.q0 = 1;
                xy_sweep_kernel<T><<<dim3(XY_NP, 2, 1), threads, 0, ctx->stream>>>(a);
                a.q0 = 3;
                xy_sweep_kernel<T><<<dim3(XY_NP, 1, 1), threads, 0, ctx->stream>>>(a);
                ctx->phase_end(mks);
                for (int k = 0; k < 3; ++k) ctx->count_launch(true);
                xy_combine_kernel<T><<<grid_of(C, ctx->sm_count), 256, 0, ctx->stream>>>(
                    C, g, 1, part, phi, ctl);
                ctx->count_launch(false);
            }
        } else {
            a.in_x = outx + (size_t)(parity ^ 1) * nbx;
            a.out_x = outx + (size_t)parity * nbx;
            a.in_y = outy + (size_t)(parity ^ 1) * nby;
            a.out_y = outy + (size_t)parity * nby;
            xy_emission_kernel<T><<<gc, 256, 0, ctx->stream>>>(C, G, 0, G, sigs, phi, ext, q, ctl);
            ctx->count_launch(false);
            a.g0 = 0;
            a.q0 = 0;
            const int mks = ctx->phase_begin(0);
            xy_sweep_kernel<T><<<dim3(XY_NP, 4, G), threads, 0, ctx->stream>>>(a);
            ctx->phase_end(mks);
            ctx->count_launch(true);
            xy_combine_kernel<T><<<gc, 256, 0, ctx->stream>>>(C, 0, G, part, phi, ctl);
            ctx->count_launch(false);
        }
        return NOP_OK;
    };
    int issued = 0;   // iterations enqueued so far in this solve (boundary parity)
    // inner source iteration to `tol`, at most `itmax` iterations; returns the
    // control block (iterations, status, last change) in ctl_h
    auto inner = [&](double tol, int itmax) -> int {
        const int start = issued;
        xy_ctl_reset_kernel<<<1, 1, 0, ctx->stream>>>(ctl);
        ctx->count_launch(false);
        for (;;) {
            for (int b = 0; b < XY_BATCH; ++b) {
                NOP_TRY(enqueue_si(issued & 1));
                ++issued;
                xy_control_kernel<<<1, 1, 0, ctx->stream>>>(ctl, tol, itmax);
                ctx->count_launch(false);
            }
            NOP_CUDA_TRY(ctx, cudaGetLastError());
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(ctl_h, ctl, sizeof(XYCtl), cudaMemcpyDeviceToHost,
                                              ctx->stream));
            NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            if (ctl_h->done) break;
        }
        if (ctx->timing) ctx->cell_angle_updates += (double)C * 40 * G * ctl_h->its;
        // iterations enqueued after the stop did nothing: the next executed
        // iteration reads the boundary buffer of the last executed one
        issued = start + ctl_h->its;
        return NOP_OK;
    };

    int status = NOP_OK, its = 0, n = 0;
    double k = k0 > 0 ? k0 : 1.0, dphi = 0.0;
    if (!eigen) {
        NOP_TRY(inner(o->tol, o->itmax));
        its = ctl_h->its;
        status = ctl_h->status;
        dphi = ctl_h->change;
    } else {
        // normalise the initial flux to unit production (cell area dx dy)
        const double area = a.dx * a.dy;
        auto prod = [&](double* P) -> int {
            NOP_CUDA_TRY(ctx, cudaMemsetAsync(acc, 0, sizeof(double), ctx->stream));
            xy_production_kernel<T><<<gb, 256, 0, ctx->stream>>>(GC, nsf, phi, acc);
            ctx->count_launch(false);
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(acc_h, acc, sizeof(double), cudaMemcpyDeviceToHost,
                                              ctx->stream));
            NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            *P = acc_h[0] * area;
            return NOP_OK;
        };
        double P;
        NOP_TRY(prod(&P));
        if (!(P > 0) || !std::isfinite(P)) return NOP_ENAN;
        xy_scale_kernel<T><<<gb, 256, 0, ctx->stream>>>(GC, (T)(1.0 / P), phi);
        ctx->count_launch(false);
        double dk = INFINITY;
        for (n = 1; n <= o->itmax; ++n) {
            xy_fission_kernel<T><<<grid_of(C, ctx->sm_count), 256, 0, ctx->stream>>>(
                C, G, 1.0 / k, ctx->chi_d, nsf, phi, ext, prev);
            ctx->count_launch(false);
            NOP_TRY(inner(o->tol_inner, o->itmax_inner));
            its += ctl_h->its;
            if (ctl_h->status == NOP_ENAN) {
                status = NOP_ENAN;
                break;
            }
            NOP_TRY(prod(&P));
            if (!(P > 0) || !std::isfinite(P)) {
                status = NOP_ENAN;
                break;
            }
            const double kn = k * P;
            NOP_CUDA_TRY(ctx, cudaMemsetAsync(acc + 1, 0, sizeof(double) * 2, ctx->stream));
            xy_normalize_kernel<T><<<gb, 256, 0, ctx->stream>>>(GC, (T)(1.0 / P), phi, prev, acc + 1);
            xy_scale_kernel<T><<<grid_of(2 * (long long)nbx, ctx->sm_count), 256, 0, ctx->stream>>>(
                2 * (long long)nbx, (T)(1.0 / P), outx);
            xy_scale_kernel<T><<<grid_of(2 * (long long)nby, ctx->sm_count), 256, 0, ctx->stream>>>(
                2 * (long long)nby, (T)(1.0 / P), outy);
            ctx->count_launch(false);
            ctx->count_launch(false);
            ctx->count_launch(false);
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(acc_h + 1, acc + 1, sizeof(double) * 2,
                                              cudaMemcpyDeviceToHost, ctx->stream));
            NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            dphi = acc_h[2] > 0 ? std::sqrt(acc_h[1] / acc_h[2]) : 0.0;
            dk = std::fabs(kn - k) / std::fabs(kn);
            k = kn;
            if (dk <= o->tol_k && dphi <= o->tol) break;
        }
        if (status == NOP_OK && n > o->itmax) {
            n = o->itmax;
            status = NOP_ENOCONV;
        }
    }
    mk = ctx->phase_begin(2);
    double* dst = phi_out;
    if (!out_dev) {
        NOP_TRY(ctx->scratch("xy_out", sizeof(double) * GC, &p));
        dst = (double*)p;
    }
    xy_finish_kernel<T><<<gb, 256, 0, ctx->stream>>>(nx, ny, GC, phi, dst);
    ctx->count_launch(false);
    ctx->phase_end(mk);
    if (!out_dev)
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(phi_out, dst, sizeof(double) * GC, cudaMemcpyDeviceToHost,
                                          ctx->stream));
    if (eigen && k_out) {
        if (out_dev) {
            NOP_TRY(ctx->pinned("xy_k", sizeof(double), &p));
            *(double*)p = k;
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(k_out, p, sizeof(double), cudaMemcpyHostToDevice,
                                              ctx->stream));
        } else {
            *k_out = k;
        }
    }
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (st) {
        st->status = status;
        st->max_iterations = its;
        st->sum_iterations = its;
        st->max_outer = eigen ? n : 0;
        st->max_change = dphi;
        if (st->inst_iterations) st->inst_iterations[0] = its;
        if (st->inst_status) st->inst_status[0] = status;
    }
    return status;
}

}  // namespace

int xy_solve(nop_ctx* ctx, const nop_solve_opts* o, bool eigen, const double* phi0, double k0,
             double* phi_out, bool out_dev, double* k_out, nop_stats* st) {
    if (o->precision == NOP_PREC_F64)
        return run<double>(ctx, o, eigen, phi0, k0, phi_out, out_dev, k_out, st);
    return run<float>(ctx, o, eigen, phi0, k0, phi_out, out_dev, k_out, st);
}

}  // namespace nop
