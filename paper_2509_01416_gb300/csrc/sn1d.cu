// Dispatch of the batched 1D slab solver (kernels in sn1d_impl.cuh, compiled
// once per precision in sn1d_f32.cu / sn1d_f64.cu).
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

// Lane-split model for one sweep of I cells with N angles: issue slots per
// cell step of a warp (per-cell loads and ownership ~12, the xor reduction 2
// per level, ~13 FP32 pipe instructions per angle in the compensated update),
// bounded below by the reciprocal unit (8 cycles per warp instruction).
// Chunked splits add the map-composition pass and a scan.  A lane carries
// A in {1, 2, 4} angles (the compiled variants; wider lanes would raise the
// kernel's register count and cut its occupancy).
void sn1d_pick_config(int I, int N, int* lg_out, int* A_out, bool pow2, double* cost_out) {
    // A angles per lane: any count up to 6 (powers of two only when asked),
    // so that ng x A covers the half-angle set with few idle slots
    const int h = N / 2;
    double best = 1e300;
    int bl = 5, bA = 4;
    for (int lg = 0; lg <= 5; ++lg) {
        const int ng = 1 << lg, nt = 32 >> lg;
        const int need = (h + ng - 1) / ng;
        int A = need;
        if (pow2) {
            A = 1;
            while (A < need) A <<= 1;
        }
        if (A > (pow2 ? 4 : 6)) continue;
        const double m = (double)((I + nt - 1) / nt);
        const double mufu = 8.0 * A;
        const double passB = std::max(mufu, 12.0 + 2.0 * lg + 13.0 * A);
        const double passA = nt > 1 ? std::max(mufu, 8.0 + 12.0 * A) : 0.0;
        const double scan = nt > 1 ? 20.0 * A * std::log2((double)nt) : 0.0;
        const double cost = m * (passB + passA) + scan;
        if (cost < best) {
            best = cost;
            bl = lg;
            bA = A;
        }
    }
    *lg_out = bl;
    *A_out = bA;
    if (cost_out) *cost_out = best;
}

// Team selection of the slab batch scheduler (host arithmetic).  lat_w[b]:
// latency of instance b on one warp; lat_t[b]: on a team of `width` warps
// (< 0: no team possible).  mode 0: the instances that can have a team are
// taken in decreasing warp latency and given one while their warp latency
// exceeds the expected span S = (warp latencies of the warp instances +
// width x team latencies of the team instances) / warps, S updated after
// each; so the fewest, longest instances get teams and no instance left on a
// warp (that could have a team) outlasts S.  mode 1: every instance that can;
// mode 2: none.  Returns the final S in *span.
int sn1d_select_teams(int n, const double* lat_w, const double* lat_t, int warps, int width,
                      int mode, double margin, std::vector<char>& team, double* span) {
    if (n < 0 || warps < 1 || width < 1 || !(margin >= 1.0) || (n > 0 && (!lat_w || !lat_t)))
        return NOP_EINVAL;
    team.assign(n, 0);
    double work = 0.0;
    for (int b = 0; b < n; ++b) work += lat_w[b];
    if (mode == 1) {
        for (int b = 0; b < n; ++b)
            if (lat_t[b] >= 0.0) {
                team[b] = 1;
                work += width * lat_t[b] - lat_w[b];
            }
    } else if (mode == 0) {
        std::vector<int> cand;
        for (int b = 0; b < n; ++b)
            if (lat_t[b] >= 0.0) cand.push_back(b);
        std::stable_sort(cand.begin(), cand.end(),
                         [&](int x, int y) { return lat_w[x] > lat_w[y]; });
        for (int b : cand) {
            if (!(margin * lat_w[b] > work / warps)) break;
            team[b] = 1;
            work += width * lat_t[b] - lat_w[b];
        }
    }
    if (span) *span = work / warps;
    return NOP_OK;
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
