// Dispatch of the batched 1D slab solver (kernels in sn1d_impl.cuh, compiled
// once per precision in sn1d_f32.cu / sn1d_f64.cu) and its lane-split model.
#include <algorithm>
#include <cmath>

#include "nop_internal.cuh"

namespace nop {

template <typename T>
int sn1d_run(nop_ctx* ctx, const nop_solve_opts* o, bool eigen, const double* phi0,
             const double* k0, double* phi_out, bool out_dev, double* k_out, nop_stats* st);
extern template int sn1d_run<float>(nop_ctx*, const nop_solve_opts*, bool, const double*,
                                    const double*, double*, bool, double*, nop_stats*);
extern template int sn1d_run<double>(nop_ctx*, const nop_solve_opts*, bool, const double*,
                                     const double*, double*, bool, double*, nop_stats*);

// Cost model of one sweep of I cells with N angles for a lane split: a warp
// instruction of the reciprocal takes 8 cycles of the SM sub-partition's
// special-function unit, so a cell step costs max(8 A, issue slots); chunked
// splits add the map-composition pass.
void sn1d_pick_config(int I, int N, int* lg_out, int* A_out) {
    const int h = N / 2;
    double best = 1e300;
    int bl = 5, bA = (h + 31) / 32;
    for (int lg = 0; lg <= 5; ++lg) {
        const int ng = 1 << lg, nt = 32 >> lg;
        const int A = (h + ng - 1) / ng;
        if (A > 8) continue;
        const int m = (I + nt - 1) / nt;
        const double passB = std::max(8.0 * A, 6.0 * A + 2.0 * lg + 8.0);
        const double passA = nt > 1 ? std::max(8.0 * A, 6.0 * A + 4.0) : 0.0;
        const double scan = nt > 1 ? 4.0 * A * std::log2((double)nt) * 4.0 : 0.0;
        const double cost = m * (passB + passA) + scan;
        if (cost < best) {
            best = cost;
            bl = lg;
            bA = A;
        }
    }
    *lg_out = bl;
    *A_out = bA;
}

int sn1d_solve(nop_ctx* ctx, const nop_solve_opts* o, bool eigen, const double* phi0,
               bool phi0_dev, const double* k0, double* phi_out, bool out_dev,
               double* k_out, nop_stats* st) {
    const double* phi0_d = nullptr;
    if (phi0) {
        if (phi0_dev) {
            phi0_d = phi0;
        } else {
            void* p;
            NOP_TRY(ctx->scratch("sn1d_phi0", sizeof(double) * ctx->G * ctx->slab.C, &p));
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(p, phi0, sizeof(double) * ctx->G * ctx->slab.C,
                                              cudaMemcpyHostToDevice, ctx->stream));
            phi0_d = (const double*)p;
        }
    }
    if (o->precision == NOP_PREC_F64)
        return sn1d_run<double>(ctx, o, eigen, phi0_d, k0, phi_out, out_dev, k_out, st);
    return sn1d_run<float>(ctx, o, eigen, phi0_d, k0, phi_out, out_dev, k_out, st);
}

}  // namespace nop
