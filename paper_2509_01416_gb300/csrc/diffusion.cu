// Diffusion problems on the recast driver (Sec. 3.1, Table 1): a batch of 1D
// slabs with -(D u')' + Sigma_a u = S and u = 0 at both faces, on cell-centred
// finite volumes (harmonic face coefficients; a boundary face half a cell
// from its centre).  Table 1's diffusion row is Sigma_a = 0 with p = D(x); its
// Helmholtz row is D = 1, Sigma_a = -k^2.
//
// diffusion_solve_kernel: the model-based solver, the tridiagonal system of
// every instance solved by elimination in FP64 (one thread per instance).
// diffusion_bands_kernel: the recast mismatch on the operator's M-bin grid,
// -dL = -(L(D, Sigma_a) - L(D*, Sigma_a*)) with D and Sigma_a averaged onto
// the bins (overlap-weighted, like every field the operator sees), as three
// bands: the recast source of bin m is PS_m + PL_m u_{m-1} + PD_m u_m +
// PU_m u_{m+1}.
#include <cmath>

#include "nop_internal.cuh"

namespace nop {
namespace {

// face coefficient D_{i-1/2} / h^2 of a row, i = 0..I (boundary faces: 2 D)
__device__ __forceinline__ double face_coef(const double* D, int I, int i, double h) {
    if (i == 0) return 2.0 * D[0] / (h * h);
    if (i == I) return 2.0 * D[I - 1] / (h * h);
    return 2.0 * D[i - 1] * D[i] / (D[i - 1] + D[i]) / (h * h);
}

__global__ void diffusion_solve_kernel(int B, const long long* cell_off, const int* ncell,
                                       const double* width, const double* D, const double* siga,
                                       const double* S, double* u, double* cp) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int I = ncell[b];
    const long long o = cell_off[b];
    const double h = width[b] / I;
    const double* Db = D + o;
    // forward elimination: c'_i = upper_i / m_i, d'_i = (S_i - lower_i d'_{i-1}) / m_i
    double cprev = 0.0, dprev = 0.0;
    for (int i = 0; i < I; ++i) {
        const double aw = face_coef(Db, I, i, h), ae = face_coef(Db, I, i + 1, h);
        const double lower = i > 0 ? -aw : 0.0, upper = i < I - 1 ? -ae : 0.0;
        const double m = aw + ae + siga[o + i] - lower * cprev;
        cprev = upper / m;
        dprev = (S[o + i] - lower * dprev) / m;
        cp[o + i] = cprev;
        u[o + i] = dprev;
    }
    // back substitution
    for (int i = I - 2; i >= 0; --i) u[o + i] -= cp[o + i] * u[o + i + 1];
}

// overlap-weighted average of a cell field over bin m of instance b
__device__ double bin_avg(const double* f, long long o, int I, double L, int M, int m) {
    const double h = L / M, dx = L / I;
    const double lo = m * h, hi = (m + 1) * h;
    const int i0 = max(0, min(I - 1, (int)floor(lo / dx)));
    const int i1 = max(0, min(I - 1, (int)floor(hi / dx)));
    double acc = 0.0;
    for (int i = i0; i <= i1; ++i) {
        const double ov = fmin(hi, (i + 1) * dx) - fmax(lo, i * dx);
        if (ov > 0.0) acc += ov * f[o + i];
    }
    return acc / h;
}

__global__ void diffusion_bands_kernel(int B, int M, const long long* cell_off, const int* ncell,
                                       const double* width, const double* D, const double* siga,
                                       double d_star, double siga_star, float* PL, float* PD,
                                       float* PU) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)B * M) return;
    const int b = (int)(e / M), m = (int)(e % M);
    const int I = ncell[b];
    const long long o = cell_off[b];
    const double L = width[b], h = L / M, h2 = h * h;
    const double Dm = bin_avg(D, o, I, L, M, m);
    const double Sm = bin_avg(siga, o, I, L, M, m);
    // face coefficients of the bin grid for p and p*
    double aw, ae;
    if (m == 0) {
        aw = 2.0 * Dm;
    } else {
        const double Dl = bin_avg(D, o, I, L, M, m - 1);
        aw = 2.0 * Dl * Dm / (Dl + Dm);
    }
    if (m == M - 1) {
        ae = 2.0 * Dm;
    } else {
        const double Dr = bin_avg(D, o, I, L, M, m + 1);
        ae = 2.0 * Dm * Dr / (Dm + Dr);
    }
    const double aws = m == 0 ? 2.0 * d_star : d_star, aes = m == M - 1 ? 2.0 * d_star : d_star;
    // -dL: lower = -aw / h^2 (p) minus -aws / h^2 (p*), negated; likewise
    PL[e] = m > 0 ? (float)((aw - aws) / h2) : 0.f;
    PU[e] = m < M - 1 ? (float)((ae - aes) / h2) : 0.f;
    PD[e] = (float)(-((aw + ae) - (aws + aes)) / h2 - (Sm - siga_star));
}

}  // namespace

int diffusion_bands(nop_ctx* ctx, int M, double d_star, double siga_star, float* PL, float* PD,
                    float* PU) {
    SlabDev& s = ctx->slab;
    const long long n = (long long)s.n_inst * M;
    diffusion_bands_kernel<<<(int)((n + 255) / 256), 256, 0, ctx->stream>>>(
        s.n_inst, M, s.cell_off_d, s.ncell_d, s.width_d, ctx->sigt_d, ctx->sigs_d, d_star,
        siga_star, PL, PD, PU);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    return NOP_OK;
}

}  // namespace nop

extern "C" {

int nop_set_diffusion(nop_ctx* ctx, int n_inst, const int* n_cells, const double* width,
                      const double* diffusion, const double* absorption, const double* source) {
    if (!ctx) return NOP_EINVAL;
    if (n_inst < 1 || !n_cells || !width || !diffusion || !source) {
        ctx->set_error("diffusion batch needs n_inst >= 1, n_cells, width, diffusion, source");
        return NOP_EINVAL;
    }
    long long C = 0;
    for (int b = 0; b < n_inst; ++b) {
        if (n_cells[b] < 1) {
            ctx->set_error("diffusion instance " + std::to_string(b) + ": n_cells < 1");
            return NOP_EINVAL;
        }
        C += n_cells[b];
    }
    // the slab batch machinery carries the fields: D in the total cross
    // section's place (checked positive), Sigma_a in the in-group scattering's
    // (any finite value: Helmholtz has Sigma_a = -k^2)
    std::vector<int> order(n_inst, 2);
    std::vector<double> zero;
    if (!absorption) zero.assign((size_t)C, 0.0);
    nop_problem p{};
    p.geometry = NOP_GEOM_SLAB;
    p.n_inst = n_inst;
    p.n_cells = n_cells;
    p.width = width;
    p.order = order.data();
    p.n_groups = 1;
    p.sigma_t = diffusion;
    p.sigma_s = absorption ? absorption : zero.data();
    p.source = source;
    const int rc = nop_set_problem(ctx, &p);
    if (rc != NOP_OK) return rc;
    ctx->diffusion = true;
    return NOP_OK;
}

int nop_diffusion_solve(nop_ctx* ctx, double* u_out) {
    if (!ctx || !u_out) return NOP_EINVAL;
    if (!ctx->has_problem || !ctx->diffusion) {
        ctx->set_error("nop_diffusion_solve needs a problem from nop_set_diffusion");
        return NOP_ESTATE;
    }
    NOP_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    nop::SlabDev& s = ctx->slab;
    void* p;
    NOP_TRY(ctx->scratch("df_u", sizeof(double) * s.C, &p));
    double* u = (double*)p;
    NOP_TRY(ctx->scratch("df_cp", sizeof(double) * s.C, &p));
    double* cp = (double*)p;
    nop::diffusion_solve_kernel<<<(s.n_inst + 127) / 128, 128, 0, ctx->stream>>>(
        s.n_inst, s.cell_off_d, s.ncell_d, s.width_d, ctx->sigt_d, ctx->sigs_d, ctx->src_d, u, cp);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    ctx->count_launch(false);
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(u_out, u, sizeof(double) * s.C, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return NOP_OK;
}

}  // extern "C"
