// Simple-preconditioning eigen warm start (App. A2, Eq. A5): a power
// iteration whose inner solve is one application of the neural operator per
// group and outer step, on the recast source of that group,
//   phi_g <- N[ chi_g F / k + sum_{g' != g} Sigma_s^{g'->g} phi_g' + delta_g phi_g ],
//   delta_g = (Sigma_s^{g->g} - Sigma_s*) - (Sigma_t,g - Sigma_t*),
// groups in order with the newest fluxes of the groups already visited, then
// k <- k P and phi <- phi / P with P the production integral (Eq. A6 seeds the
// model-based power iteration with the result).  Every instance of a slab
// batch iterates on its own (k, phi) and is frozen once
// |dk|/k <= tol and ||dphi||/||phi|| <= tol.
#include <algorithm>
#include <cmath>
#include <vector>

#include "nop_internal.cuh"

namespace nop {
namespace {

int grid_of(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 1 << 20)); }

__global__ void inst_of_kernel(long long C, int B, const long long* cell_off, int* inst) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cell_off[mid] <= c) lo = mid;
            else hi = mid - 1;
        }
        inst[c] = lo;
    }
}

__global__ void fill_kernel(long long n, double v, double* x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        x[i] = v;
}

// F_c = sum_g nu Sigma_f,g phi_g
__global__ void fission_kernel(int G, long long C, const double* nsf, const double* phi, double* F) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        double f = 0.0;
        for (int g = 0; g < G; ++g) f += nsf[(long long)g * C + c] * phi[(long long)g * C + c];
        F[c] = f;
    }
}

// recast source of group g (Eq. A5 with the mismatch of Eq. 24)
__global__ void group_source_kernel(int g, int G, long long C, const int* inst, const double* chi,
                                    const double* F, const double* k, const double* sigt,
                                    const double* sigs, double st_star, double ss_star,
                                    const double* nw, const double* phi, double* src) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        double s = chi[g] * F[c] / k[inst[c]];
        for (int gp = 0; gp < G; ++gp)
            if (gp != g) s += sigs[((long long)gp * G + g) * C + c] * nw[(long long)gp * C + c];
        const double d = (sigs[((long long)g * G + g) * C + c] - ss_star) -
                         (sigt[(long long)g * C + c] - st_star);
        src[c] = s + d * phi[(long long)g * C + c];
    }
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

// production integral of each instance (one block per instance)
__global__ void production_kernel(int G, long long C, const long long* cell_off, const int* ncell,
                                  const double* vol, const double* nsf, const double* phi,
                                  double* P) {
    __shared__ double red[32];
    const int b = blockIdx.x;
    const long long off = cell_off ? cell_off[b] : 0;
    const long long I = ncell ? ncell[b] : C;
    double s = 0.0;
    for (int g = 0; g < G; ++g)
        for (long long i = threadIdx.x; i < I; i += blockDim.x)
            s += nsf[(long long)g * C + off + i] * phi[(long long)g * C + off + i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) P[b] = s * vol[b];
}

// phi <- phi / P of its instance (one block per instance)
__global__ void scale_kernel(int G, long long C, const long long* cell_off, const int* ncell,
                             const double* P, double* phi) {
    const int b = blockIdx.x;
    const long long off = cell_off ? cell_off[b] : 0;
    const long long I = ncell ? ncell[b] : C;
    const double inv = 1.0 / P[b];
    for (int g = 0; g < G; ++g)
        for (long long i = threadIdx.x; i < I; i += blockDim.x) phi[(long long)g * C + off + i] *= inv;
}

// status: 0 running, 1 converged, 3 diverged
__global__ void sp_update_kernel(int G, long long C, const long long* cell_off, const int* ncell,
                                 double tol, const double* P, const double* nw, double* phi,
                                 double* k, int* status, int* iters, int* active) {
    __shared__ double red[32];
    const int b = blockIdx.x;
    if (status[b] != 0) return;
    const long long off = cell_off ? cell_off[b] : 0;
    const long long I = ncell ? ncell[b] : C;
    const double Pn = P[b];
    const double inv = 1.0 / Pn;
    double d2 = 0.0, n2 = 0.0;
    for (int g = 0; g < G; ++g)
        for (long long i = threadIdx.x; i < I; i += blockDim.x) {
            const long long e = (long long)g * C + off + i;
            const double a = nw[e] * inv, o = phi[e];
            d2 += (a - o) * (a - o);
            n2 += a * a;
        }
    d2 = block_sum(d2, red);
    n2 = block_sum(n2, red);
    const bool bad = !isfinite(Pn) || !(Pn != 0.0) || !isfinite(d2) || !isfinite(n2) || !(n2 > 0);
    if (!bad)
        for (int g = 0; g < G; ++g)
            for (long long i = threadIdx.x; i < I; i += blockDim.x) {
                const long long e = (long long)g * C + off + i;
                phi[e] = nw[e] * inv;
            }
    if (threadIdx.x == 0) {
        iters[b] += 1;
        if (bad) {
            status[b] = 3;
            return;
        }
        const double kn = k[b] * Pn;
        const double dk = fabs(kn - k[b]) / fabs(kn);
        const double dphi = sqrt(d2 / n2);
        k[b] = kn;
        if (dk <= tol && dphi <= tol) status[b] = 1;
        else atomicAdd(active, 1);
    }
}

// fission source of the refinement step: chi_g F_c / k of the cell's instance
__global__ void fission_source_kernel(int G, long long C, const int* inst, const double* chi,
                                      const double* F, const double* k, double* src) {
    const long long n = (long long)G * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(e / C);
        const long long c = e - (long long)g * C;
        src[e] = chi[g] * F[c] / k[inst[c]];
    }
}

// diverged instances restart from the plain guess (flat flux, k = 1)
__global__ void fallback_kernel(int G, long long C, const int* inst, const int* status, double* phi,
                                double* k) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        const int b = inst[c];
        if (status[b] != 3) continue;
        for (int g = 0; g < G; ++g) phi[(long long)g * C + c] = 1.0;
        if (c == 0 || inst[c - 1] != b) k[b] = 1.0;
    }
}

}  // namespace

namespace {

// Eq. A8: one model-based source iteration from u (device [G*C]) with the
// fixed source src (device [G*C]) into out; the solver's own schedule cache
// is left as it was.
int refine_once(nop_ctx* ctx, const double* u, const double* src, double* out) {
    nop_solve_opts o{};
    o.tol = 1e-300;
    o.itmax = 1;
    o.precision = NOP_PREC_F32;
    // one model source iteration of the reference order (Gauss-Seidel over
    // groups), as Eq. A7-A8 apply it
    o.flags = NOP_PHI0_DEVICE | NOP_OUT_DEVICE | NOP_GAUSS_SEIDEL;
    double* keep_src = ctx->src_d;
    ctx->src_d = const_cast<double*>(src);
    std::vector<int> keep_iters = ctx->slab.last_iters;
    int rc;
    if (ctx->geometry == NOP_GEOM_SLAB)
        rc = sn1d_solve(ctx, &o, false, u, true, nullptr, out, true, nullptr, nullptr);
    else
        rc = xy_solve(ctx, &o, false, u, 0.0, out, true, nullptr, nullptr);
    ctx->src_d = keep_src;
    ctx->slab.last_iters = keep_iters;
    return rc == NOP_ENOCONV ? NOP_OK : rc;   // one iteration is the cap by design
}

}  // namespace

int sp_eigen(nop_ctx* ctx, double tol, int itmax, double* phi_d, std::vector<double>* k_h,
             std::vector<int>* status_h, std::vector<int>* iters_h, bool constrained) {
    if (!ctx->no.loaded) {
        ctx->set_error("the eigen warm start needs a neural operator");
        return NOP_ESTATE;
    }
    if (!ctx->has_fission) {
        ctx->set_error("the eigen warm start needs a problem with nu_sigma_f and chi");
        return NOP_ESTATE;
    }
    const bool slab = ctx->geometry == NOP_GEOM_SLAB;
    if (constrained)
        for (int f = 0; f < (slab ? 2 : 4); ++f)
            if (ctx->bc[f] != NOP_BC_VACUUM) {
                ctx->set_error("the constrained eigen warm start needs vacuum faces");
                return NOP_EINVAL;
            }
    const int B = slab ? ctx->slab.n_inst : 1;
    const int G = ctx->G;
    const long long C = ctx->C, GC = (long long)G * C;
    void* p;
    NOP_TRY(ctx->scratch("sp_new", sizeof(double) * GC, &p));
    double* nw = (double*)p;
    NOP_TRY(ctx->scratch("sp_F", sizeof(double) * C, &p));
    double* F = (double*)p;
    NOP_TRY(ctx->scratch("sp_src", sizeof(double) * C, &p));
    double* src = (double*)p;
    NOP_TRY(ctx->scratch("sp_inst", sizeof(int) * C, &p));
    int* inst = (int*)p;
    double *cp_src = nullptr, *cp_half = nullptr;
    if (constrained) {
        NOP_TRY(ctx->scratch("cp_src", sizeof(double) * GC, &p));
        cp_src = (double*)p;
        NOP_TRY(ctx->scratch("cp_half", sizeof(double) * GC, &p));
        cp_half = (double*)p;
    }
    NOP_TRY(ctx->scratch("sp_dbl", sizeof(double) * 3 * (size_t)B, &p));
    double* k = (double*)p;
    double* P = k + B;
    double* vol = k + 2 * B;
    NOP_TRY(ctx->scratch("sp_int", sizeof(int) * (2 * (size_t)B + 1), &p));
    int* status = (int*)p;
    int* iters = status + B;
    int* active = status + 2 * B;
    const long long* cell_off = slab ? ctx->slab.cell_off_d : nullptr;
    const int* ncell = slab ? ctx->slab.ncell_d : nullptr;

    std::vector<double> volh(B);
    for (int b = 0; b < B; ++b)
        volh[b] = slab ? ctx->slab.width[b] / ctx->slab.ncell[b]
                       : (ctx->xy.lx / ctx->xy.nx) * (ctx->xy.ly / ctx->xy.ny);
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(vol, volh.data(), sizeof(double) * B, cudaMemcpyHostToDevice,
                                      ctx->stream));
    if (slab) {
        inst_of_kernel<<<grid_of(C), 256, 0, ctx->stream>>>(C, B, cell_off, inst);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
    } else {
        NOP_CUDA_TRY(ctx, cudaMemsetAsync(inst, 0, sizeof(int) * C, ctx->stream));
    }
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(status, 0, sizeof(int) * (2 * (size_t)B + 1), ctx->stream));
    fill_kernel<<<grid_of(GC), 256, 0, ctx->stream>>>(GC, 1.0, phi_d);
    fill_kernel<<<grid_of(B), 256, 0, ctx->stream>>>(B, 1.0, k);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    // unit production start: phi <- phi / P (k stays 1)
    production_kernel<<<B, 256, 0, ctx->stream>>>(G, C, cell_off, ncell, vol, ctx->nsf_d, phi_d, P);
    scale_kernel<<<B, 256, 0, ctx->stream>>>(G, C, cell_off, ncell, P, phi_d);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    const nop_no_config& c = ctx->no.cfg;
    const bool fno = c.kind == NOP_NO_FNO1D || c.kind == NOP_NO_FNO2D;
    int* active_h = nullptr;
    {
        void* ph;
        NOP_TRY(ctx->pinned("sp_active", sizeof(int), &ph));
        active_h = (int*)ph;
    }
    int rc = NOP_OK;
    const int mk = ctx->phase_begin(1);
    for (int it = 1; it <= itmax && rc == NOP_OK; ++it) {
        fission_kernel<<<grid_of(C), 256, 0, ctx->stream>>>(G, C, ctx->nsf_d, phi_d, F);
        if (cudaMemcpyAsync(nw, phi_d, sizeof(double) * GC, cudaMemcpyDeviceToDevice,
                            ctx->stream) != cudaSuccess) {
            rc = NOP_ECUDA;
            break;
        }
        for (int g = 0; g < G && rc == NOP_OK; ++g) {
            group_source_kernel<<<grid_of(C), 256, 0, ctx->stream>>>(
                g, G, C, inst, ctx->chi_d, F, k, ctx->sigt_d, ctx->sigs_d, c.sigma_t_star,
                c.sigma_s_star, nw, phi_d, src);
            if (cudaGetLastError() != cudaSuccess) {
                rc = NOP_ECUDA;
                break;
            }
            rc = fno ? fno_recast(ctx, 0, 1, nw + (long long)g * C, nullptr, nullptr, true, src)
                     : deeponet_recast(ctx, 0, 1, nw + (long long)g * C, nullptr, nullptr, true,
                                       src);
        }
        if (rc != NOP_OK) break;
        const double* upd = nw;
        if (constrained) {
            // Eq. A8: one source iteration from the prediction, its own
            // fission source with the current k
            fission_kernel<<<grid_of(C), 256, 0, ctx->stream>>>(G, C, ctx->nsf_d, nw, F);
            fission_source_kernel<<<grid_of(GC), 256, 0, ctx->stream>>>(G, C, inst, ctx->chi_d, F,
                                                                        k, cp_src);
            if (cudaGetLastError() != cudaSuccess) {
                rc = NOP_ECUDA;
                break;
            }
            if ((rc = refine_once(ctx, nw, cp_src, cp_half)) != NOP_OK) break;
            upd = cp_half;
        }
        production_kernel<<<B, 256, 0, ctx->stream>>>(G, C, cell_off, ncell, vol, ctx->nsf_d, upd, P);
        if (cudaMemsetAsync(active, 0, sizeof(int), ctx->stream) != cudaSuccess) {
            rc = NOP_ECUDA;
            break;
        }
        sp_update_kernel<<<B, 256, 0, ctx->stream>>>(G, C, cell_off, ncell, tol, P, upd, phi_d, k,
                                                     status, iters, active);
        if (cudaGetLastError() != cudaSuccess) {
            rc = NOP_ECUDA;
            break;
        }
        if (it % 4 != 0 && it != itmax) continue;
        if (cudaMemcpyAsync(active_h, active, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            rc = NOP_ECUDA;
            break;
        }
        if (*active_h == 0) break;
    }
    if (rc != NOP_OK) {
        if (ctx->err.empty()) ctx->set_error("eigen warm start failed");
        return rc;
    }
    fallback_kernel<<<grid_of(C), 256, 0, ctx->stream>>>(G, C, inst, status, phi_d, k);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->phase_end(mk);
    k_h->assign(B, 0.0);
    status_h->assign(B, 0);
    iters_h->assign(B, 0);
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(k_h->data(), k, sizeof(double) * B, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(status_h->data(), status, sizeof(int) * B,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(iters_h->data(), iters, sizeof(int) * B,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return NOP_OK;
}

}  // namespace nop
