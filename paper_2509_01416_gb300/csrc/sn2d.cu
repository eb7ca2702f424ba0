// 2D x-y S_N solver: level-symmetric S8, diamond difference, source iteration
// with Gauss-Seidel over groups and power iteration (the paper's method in two
// dimensions, Sec. 6; multigroup coupling of Sec. 5.3 Eq. 27-29 with
// upscatter allowed; the k update of App. A2 Eq. A2-A4).
//
// Sweep: one CTA per direction walks the anti-diagonals of the mesh in the
// direction's sweep order; thread t owns row t (in sweep order) and processes
// cell (s - t, t) at step s, carrying the x-edge flux in registers and handing
// the y-edge flux of column i to row t + 1 through shared memory.  Directions
// of one quadrant are independent; quadrants follow the oracle's order with
// the newest reflected flux: (-,-); then (+,-) and (-,+) together (each reads
// only (-,-) of this iteration and (+,+) of the previous one); then (+,+).
// Diamond difference in increment form, with c_x = 2|mu|/dx, c_y = 2|eta|/dy,
// D = sigma_t + c_x + c_y:
//     psi_c - psi_x = (q + c_y psi_y - (sigma_t + c_y) psi_x) / D,
//     psi_x' = psi_x + 2 (psi_c - psi_x),   psi_y' = psi_y + 2 (psi_c - psi_y),
// the edge fluxes carried with compensated sums in FP32.  The angle sum
// phi = sum_d w_d psi_c is accumulated with atomic adds per cell.
#include <algorithm>
#include <cmath>

#include "nop_internal.cuh"

namespace nop {
namespace {

constexpr int MAXN = 1024;   // rows per mesh (threads per sweep CTA)

template <typename T>
struct XYArgs {
    int nx, ny, G;
    double dx, dy;
    const double* mu;
    const double* eta;
    const double* w;
    const int* mir_x;
    const int* mir_y;
    const T* sigt;       // [G][ny][nx]
    const T* q;          // [ny][nx] emission of the group being swept
    T* phi;              // [ny][nx] angle sum (accumulated)
    T* out_x;            // [G][40][ny] outgoing through the x-face the direction leaves
    T* out_y;            // [G][40][nx]
    int g;
    int d0;              // first direction of the phase
    int bc_x0, bc_xL, bc_y0, bc_yL;
};

template <typename T>
__device__ __forceinline__ T rcp2(T d) {
    return T(1) / d;
}

template <typename T>
__global__ void __launch_bounds__(MAXN) xy_sweep_kernel(XYArgs<T> a) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* yhi = (T*)sm_raw;
    T* ylo = yhi + a.nx;
    const int d = a.d0 + blockIdx.x;
    const int t = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const double mud = a.mu[d], etd = a.eta[d];
    const bool xp = mud > 0, yp = etd > 0;
    const T cx = (T)(2.0 * fabs(mud) / a.dx), cy = (T)(2.0 * fabs(etd) / a.dy);
    const T wd = (T)a.w[d];
    const long long gx = (long long)a.g * 40;
    // incoming edge fluxes: vacuum 0, reflective = mirror's latest outgoing
    const bool rx = xp ? a.bc_x0 : a.bc_xL;
    const bool ry = yp ? a.bc_y0 : a.bc_yL;
    for (int i = t; i < nx; i += blockDim.x) {
        // column i in sweep order = physical column of the first row
        const int ip = xp ? i : nx - 1 - i;
        yhi[i] = ry ? a.out_y[(gx + a.mir_y[d]) * nx + ip] : T(0);
        ylo[i] = T(0);
    }
    const int jp = t < ny ? (yp ? t : ny - 1 - t) : 0;
    T xh = T(0), xl = T(0);
    if (t < ny && rx) xh = a.out_x[(gx + a.mir_x[d]) * ny + jp];
    __syncthreads();
    const T* st = a.sigt + (long long)a.g * nx * ny;
    // The cell operands (sigma_t, q) of step s are loaded PF steps ahead, so
    // their latency hides behind the steps in between instead of stalling
    // every step of the wavefront.
    constexpr int PF = 4;
    const int S = nx + ny - 1;
    T sgr[PF], qr[PF];
    auto fetch = [&](int s, T& sg, T& qq) {
        const int i = s - t;
        if (t < ny && i >= 0 && i < nx) {
            const long long c = (long long)jp * nx + (xp ? i : nx - 1 - i);
            sg = st[c];
            qq = a.q[c];
        }
    };
#pragma unroll
    for (int p = 0; p < PF; ++p) {
        sgr[p] = T(1);
        qr[p] = T(0);
        fetch(p, sgr[p], qr[p]);
    }
    for (int s0 = 0; s0 < S; s0 += PF)
#pragma unroll
    for (int p = 0; p < PF; ++p) {
        const int s = s0 + p;
        if (s >= S) break;     // uniform over the block
        const T sg = sgr[p], qq = qr[p];
        fetch(s + PF, sgr[p], qr[p]);
        const int i = s - t;   // column in sweep order
        if (t < ny && i >= 0 && i < nx) {
            const int ip = xp ? i : nx - 1 - i;
            const long long c = (long long)jp * nx + ip;
            const T yh = yhi[i], yl = ylo[i];
            const T r = rcp2(sg + cx + cy);
            const T dxs = (qq + cy * yh - (sg + cy) * xh) * r;   // psi_c - psi_x
            const T dys = (qq + cx * xh - (sg + cx) * yh) * r;   // psi_c - psi_y
            atomicAdd(&a.phi[c], wd * (xh + (dxs + xl)));
            // compensated edge updates
            {
                const T u = (dxs + dxs) + xl;
                const T tt = xh + u;
                xl = u - (tt - xh);
                xh = tt;
            }
            {
                const T u = (dys + dys) + yl;
                const T tt = yh + u;
                ylo[i] = u - (tt - yh);
                yhi[i] = tt;
            }
            if (i == nx - 1) a.out_x[(gx + d) * ny + jp] = xh + xl;
        }
        __syncthreads();
    }
    for (int i = t; i < nx; i += blockDim.x) {
        const int ip = xp ? i : nx - 1 - i;
        a.out_y[(gx + d) * nx + ip] = yhi[i] + ylo[i];
    }
}

// emission of group g: q = sum_g' Sigma_s(g'->g) phi_g' + ext_g (newest fluxes)
template <typename T>
__global__ void xy_source_kernel(long long C, int G, int g, const T* sigs, const T* phi,
                                 const T* ext, T* q, T* phinew) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        T s = ext[(long long)g * C + c];
        for (int gp = 0; gp < G; ++gp) s += sigs[((long long)gp * G + g) * C + c] * phi[(long long)gp * C + c];
        q[c] = s;
        phinew[c] = T(0);
    }
}

// phi_g <- phinew; accumulate |change|^2 and |phi|^2 (FP32 per thread, FP64 sums)
template <typename T>
__global__ void xy_update_kernel(long long C, int g, const T* phinew, T* phi, double* acc) {
    double d2 = 0.0, n2 = 0.0;
    T pd = T(0), pn = T(0);
    int k = 0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        const T v = phinew[c];
        const T df = v - phi[(long long)g * C + c];
        pd += df * df;
        pn += v * v;
        phi[(long long)g * C + c] = v;
        if (++k == 64) {
            d2 += (double)pd;
            n2 += (double)pn;
            pd = pn = T(0);
            k = 0;
        }
    }
    d2 += (double)pd;
    n2 += (double)pn;
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, d2);
        atomicAdd(acc + 1, n2);
    }
}

template <typename T>
__global__ void xy_prepare_kernel(long long C, int G, const double* sigt, const double* sigs,
                                  const double* src, const double* nsf, const double* phi0,
                                  int flat, T* sigtT, T* sigsT, T* ext, T* nsfT, T* phi) {
    const long long GC = (long long)G * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < GC;
         e += (long long)gridDim.x * blockDim.x) {
        sigtT[e] = (T)sigt[e];
        ext[e] = src ? (T)src[e] : T(0);
        if (nsf) nsfT[e] = (T)nsf[e];
        phi[e] = phi0 ? (T)phi0[e] : (flat ? T(1) : T(0));
        const int g = (int)(e / C);
        const long long c = e - (long long)g * C;
        for (int gp = 0; gp < G; ++gp)
            sigsT[((long long)gp * G + g) * C + c] = (T)sigs[((long long)gp * G + g) * C + c];
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

// outer-iteration step: phi *= 1/P, change vs previous, boundary fluxes scaled;
// then the frozen fission source ext_g = chi_g F / k (k already updated)
template <typename T>
__global__ void xy_normalize_kernel(long long C, int G, T sc, T* phi, T* prev, double* acc) {
    double d2 = 0.0, n2 = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)G * C;
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

template <typename T>
__global__ void xy_finish_kernel(long long n, const T* phi, double* out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        out[e] = (double)phi[e];
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
    NOP_TRY(ctx->scratch("xy_q", sizeof(T) * C, &p));
    T* q = (T*)p;
    NOP_TRY(ctx->scratch("xy_phinew", sizeof(T) * C, &p));
    T* phinew = (T*)p;
    NOP_TRY(ctx->scratch("xy_outx", sizeof(T) * (size_t)G * 40 * ny, &p));
    T* outx = (T*)p;
    NOP_TRY(ctx->scratch("xy_outy", sizeof(T) * (size_t)G * 40 * nx, &p));
    T* outy = (T*)p;
    NOP_TRY(ctx->scratch("xy_mir", sizeof(int) * 80, &p));
    int* mir = (int*)p;
    NOP_TRY(ctx->scratch("xy_acc", sizeof(double) * 4, &p));
    double* acc = (double*)p;
    double* acc_h = nullptr;
    NOP_CUDA_TRY(ctx, cudaMallocHost(&acc_h, sizeof(double) * 4));
    auto fail = [&](int rc) {
        cudaFreeHost(acc_h);
        return rc;
    };
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
    xy_prepare_kernel<T><<<gb, 256, 0, ctx->stream>>>(C, G, ctx->sigt_d, ctx->sigs_d,
                                                      eigen ? nullptr : ctx->src_d,
                                                      eigen ? ctx->nsf_d : nullptr, phi0_d,
                                                      (eigen && !phi0_d) ? 1 : 0, sigt, sigs, ext,
                                                      nsf, phi);
    mirror_kernel<<<1, 64, 0, ctx->stream>>>(xy.mu_d, xy.eta_d, mir, mir + 40);
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(outx, 0, sizeof(T) * (size_t)G * 40 * ny, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(outy, 0, sizeof(T) * (size_t)G * 40 * nx, ctx->stream));
    if (cudaGetLastError() != cudaSuccess) return fail(NOP_ECUDA);
    ctx->phase_end(mk);
    ctx->count_launch(false);
    ctx->count_launch(false);

    XYArgs<T> a;
    a.nx = nx;
    a.ny = ny;
    a.G = G;
    a.dx = xy.lx / nx;
    a.dy = xy.ly / ny;
    a.mu = xy.mu_d;
    a.eta = xy.eta_d;
    a.w = xy.w_d;
    a.mir_x = mir;
    a.mir_y = mir + 40;
    a.sigt = sigt;
    a.q = q;
    a.phi = phinew;
    a.out_x = outx;
    a.out_y = outy;
    a.bc_x0 = ctx->bc[0];
    a.bc_xL = ctx->bc[1];
    a.bc_y0 = ctx->bc[2];
    a.bc_yL = ctx->bc[3];
    const int threads = ((ny + 31) / 32) * 32;
    const size_t smem = 2 * sizeof(T) * nx;
    if (smem > 48 * 1024)
        NOP_CUDA_TRY(ctx, cudaFuncSetAttribute(xy_sweep_kernel<T>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem));

    // one source iteration over all groups; returns the relative change
    auto si = [&](double* change) -> int {
        if (cudaMemsetAsync(acc, 0, sizeof(double) * 2, ctx->stream) != cudaSuccess) return NOP_ECUDA;
        for (int g = 0; g < G; ++g) {
            xy_source_kernel<T><<<grid_of(C, ctx->sm_count), 256, 0, ctx->stream>>>(
                C, G, g, sigs, phi, ext, q, phinew);
            ctx->count_launch(false);
            a.g = g;
            const int mks = ctx->phase_begin(0);
            // quadrants: (-,-) | (+,-) and (-,+) | (+,+)
            a.d0 = 0;
            xy_sweep_kernel<T><<<10, threads, smem, ctx->stream>>>(a);
            a.d0 = 10;
            xy_sweep_kernel<T><<<20, threads, smem, ctx->stream>>>(a);
            a.d0 = 30;
            xy_sweep_kernel<T><<<10, threads, smem, ctx->stream>>>(a);
            ctx->phase_end(mks);
            for (int k = 0; k < 3; ++k) ctx->count_launch(true);
            xy_update_kernel<T><<<grid_of(C, ctx->sm_count), 256, 0, ctx->stream>>>(C, g, phinew,
                                                                                   phi, acc);
            ctx->count_launch(false);
        }
        if (cudaGetLastError() != cudaSuccess) return NOP_ECUDA;
        if (cudaMemcpyAsync(acc_h, acc, sizeof(double) * 2, cudaMemcpyDeviceToHost, ctx->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess)
            return NOP_ECUDA;
        *change = acc_h[1] > 0 ? std::sqrt(acc_h[0] / acc_h[1]) : (acc_h[0] > 0 ? INFINITY : 0.0);
        return NOP_OK;
    };
    if (ctx->timing) ctx->cell_angle_updates += 0;   // counted per iteration below

    int status = NOP_OK, its = 0, n = 0;
    double change = 0.0, k = k0 > 0 ? k0 : 1.0, dphi = 0.0;
    if (!eigen) {
        for (its = 1; its <= o->itmax; ++its) {
            const int rc = si(&change);
            if (rc != NOP_OK) return fail(rc);
            if (ctx->timing) ctx->cell_angle_updates += (double)C * 40 * G;
            if (!std::isfinite(change)) {
                status = NOP_ENAN;
                break;
            }
            if (change <= o->tol) break;
        }
        if (its > o->itmax) {
            its = o->itmax;
            status = NOP_ENOCONV;
        }
        dphi = change;
    } else {
        // normalise the initial flux to unit production (cell area dx dy)
        const double area = a.dx * a.dy;
        auto prod = [&](double* P) -> int {
            if (cudaMemsetAsync(acc + 2, 0, sizeof(double), ctx->stream) != cudaSuccess) return NOP_ECUDA;
            xy_production_kernel<T><<<gb, 256, 0, ctx->stream>>>(GC, nsf, phi, acc + 2);
            ctx->count_launch(false);
            if (cudaMemcpyAsync(acc_h + 2, acc + 2, sizeof(double), cudaMemcpyDeviceToHost,
                                ctx->stream) != cudaSuccess ||
                cudaStreamSynchronize(ctx->stream) != cudaSuccess)
                return NOP_ECUDA;
            *P = acc_h[2] * area;
            return NOP_OK;
        };
        double P;
        int rc = prod(&P);
        if (rc != NOP_OK) return fail(rc);
        if (!(P > 0) || !std::isfinite(P)) return fail(NOP_ENAN);
        xy_scale_kernel<T><<<gb, 256, 0, ctx->stream>>>(GC, (T)(1.0 / P), phi);
        ctx->count_launch(false);
        double dk = INFINITY;
        for (n = 1; n <= o->itmax; ++n) {
            xy_fission_kernel<T><<<grid_of(C, ctx->sm_count), 256, 0, ctx->stream>>>(
                C, G, 1.0 / k, ctx->chi_d, nsf, phi, ext, prev);
            ctx->count_launch(false);
            int it;
            for (it = 1; it <= o->itmax_inner; ++it) {
                rc = si(&change);
                if (rc != NOP_OK) return fail(rc);
                if (ctx->timing) ctx->cell_angle_updates += (double)C * 40 * G;
                if (!std::isfinite(change)) {
                    status = NOP_ENAN;
                    break;
                }
                if (change <= o->tol_inner) break;
            }
            its += std::min(it, o->itmax_inner);
            if (status != NOP_OK) break;
            rc = prod(&P);
            if (rc != NOP_OK) return fail(rc);
            if (!(P > 0) || !std::isfinite(P)) {
                status = NOP_ENAN;
                break;
            }
            const double kn = k * P;
            if (cudaMemsetAsync(acc, 0, sizeof(double) * 2, ctx->stream) != cudaSuccess)
                return fail(NOP_ECUDA);
            xy_normalize_kernel<T><<<gb, 256, 0, ctx->stream>>>(C, G, (T)(1.0 / P), phi, prev, acc);
            xy_scale_kernel<T><<<grid_of((long long)G * 40 * ny, ctx->sm_count), 256, 0, ctx->stream>>>(
                (long long)G * 40 * ny, (T)(1.0 / P), outx);
            xy_scale_kernel<T><<<grid_of((long long)G * 40 * nx, ctx->sm_count), 256, 0, ctx->stream>>>(
                (long long)G * 40 * nx, (T)(1.0 / P), outy);
            ctx->count_launch(false);
            ctx->count_launch(false);
            ctx->count_launch(false);
            if (cudaMemcpyAsync(acc_h, acc, sizeof(double) * 2, cudaMemcpyDeviceToHost, ctx->stream) !=
                    cudaSuccess ||
                cudaStreamSynchronize(ctx->stream) != cudaSuccess)
                return fail(NOP_ECUDA);
            dphi = acc_h[1] > 0 ? std::sqrt(acc_h[0] / acc_h[1]) : 0.0;
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
    xy_finish_kernel<T><<<gb, 256, 0, ctx->stream>>>(GC, phi, dst);
    ctx->count_launch(false);
    ctx->phase_end(mk);
    if (!out_dev)
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(phi_out, dst, sizeof(double) * GC, cudaMemcpyDeviceToHost,
                                          ctx->stream));
    if (eigen && k_out) {
        if (out_dev)
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(k_out, &k, sizeof(double), cudaMemcpyHostToDevice,
                                              ctx->stream));
        else
            *k_out = k;
    }
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFreeHost(acc_h);
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
