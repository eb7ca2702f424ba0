// Internal declarations of the GB300 S_N / MD-PNOP library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/nop.h"

namespace nop {

// Status of one CUDA call; records the message on the context and returns.
#define NOP_CUDA_TRY(ctx, call)                                                   \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            (ctx)->set_error(std::string(#call) + ": " + cudaGetErrorString(e_)); \
            return NOP_ECUDA;                                                     \
        }                                                                         \
    } while (0)

#define NOP_TRY(expr)              \
    do {                           \
        int r_ = (expr);           \
        if (r_ != NOP_OK) return r_; \
    } while (0)

// A device allocation that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Installed neural operator: FP32 master parameters, gradient, Adam moments.
struct NoState {
    bool loaded = false;
    nop_no_config cfg{};
    long long n_params = 0;
    float* params = nullptr;
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int adam_t = 0;
    // offsets of every tensor in the flat parameter array
    std::vector<long long> off;
    std::vector<long long> len;
};

// Problem state of a 1D slab batch (device side unless noted).
struct SlabDev {
    int n_inst = 0;
    long long C = 0;                 // total cells
    std::vector<int> ncell, order;   // host copies
    std::vector<double> width;
    std::vector<double> rho;         // host: estimated contraction of source iteration
    std::vector<double> siga_mean;   // host: mean absorption of the group that sets rho
    std::vector<double> rho_si;      // host: diffusion estimate of the source iteration's
                                     // spectral radius (largest over groups)
    std::vector<int> gl_orders, gl_offs;   // host: the orders whose Gauss-Legendre sets
                                           // are built, and where each set starts
    std::vector<int> last_iters;     // host: iterations of each instance in the last solve
    // the last slab schedule and the hash of what it was computed from
    std::vector<int> plan_small, plan_big, plan_cfg;
    int plan_big_blocks = 0, plan_smem_cells = 1, plan_direct = 0;
    unsigned long long plan_key = 0;
    long long version = 0;           // bumped by every nop_set_problem
    long long layout_version = 0;    // bumped when the cell counts or orders change
    long long ft_version = -1;       // layout version of the trunk point grouping
    int ft_groups = 0;
    long long ft_points = 0;
    std::vector<int> last_iters_dsa; // the same for solves with the diffusion correction
                                     // of this batch layout (0 = unknown); the scheduler's cost
    std::vector<long long> cell_off; // host prefix sums
    long long* cell_off_d = nullptr;
    int* ncell_d = nullptr;
    int* nang_d = nullptr;
    double* dx_d = nullptr;
    double* width_d = nullptr;
    int* qoff_d = nullptr;           // offset of the instance's nodes in mu_d/w_d
    long long* boff_d = nullptr;     // offset of the instance's boundary fluxes
    long long bnd_total = 0;
    double* mu_d = nullptr;          // Gauss-Legendre nodes, one block per distinct order
    double* w_d = nullptr;
    std::vector<int> qoff_h;
};

struct XYDev {
    int nx = 0, ny = 0;
    double lx = 0, ly = 0;
    double* mu_d = nullptr;          // 40 directions
    double* eta_d = nullptr;
    double* w_d = nullptr;
};

}  // namespace nop

struct nop_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    std::string err;

    // problem
    bool has_problem = false;
    bool diffusion = false;   // a diffusion batch (nop_set_diffusion), not transport
    int geometry = 0;
    int G = 0;
    bool has_source = false, has_fission = false;
    int bc[4] = {0, 0, 0, 0};
    nop::SlabDev slab;
    nop::XYDev xy;
    long long C = 0;
    nop::NoState no;
    // FP64 originals
    double *sigt_d = nullptr, *sigs_d = nullptr, *src_d = nullptr, *nsf_d = nullptr,
           *chi_d = nullptr, *sigs1_d = nullptr;

    // slab autotuner: per precision, bucket key -> measured microseconds of
    // one source iteration per cell of {direct warp, chunked warp, direct
    // team, chunked team} (-1: not measured); kept for the context's life
    std::map<long long, std::array<double, 4>> sn1d_tune[2];
    double last_tune_ms = 0.0;   // calibration time of the last slab solve
    int last_direct = 0;         // instances of the last slab solve on direct lanes
    // mbarrier poll limit of the tensor-core kernels (nop_set_wait_limit);
    // negative: the library default
    long long wait_limit = -1;
    // phase timing (nop_set_timing)
    bool timing = false;
    struct Mark {
        int phase;                 // 0 sweep, 1 operator, 2 setup
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;
    int phase_depth = 0;
    std::vector<cudaEvent_t> event_pool;
    long long launches = 0, sweep_launches = 0;
    double cell_angle_updates = 0;
    // per-instance trace summary of the last slab solve (timing on)
    double trace_span_ms = 0, trace_max_ms = 0, trace_mean_ms = 0;
    int trace_big = 0;
    std::vector<double> trace_inst;   // per instance: start ms, duration ms, block path
    // Open a timed phase on the stream; returns the mark index or -1.
    int phase_begin(int phase);
    void phase_end(int mark);
    void count_launch(bool sweep) {
        if (timing) {
            ++launches;
            if (sweep) ++sweep_launches;
        }
    }

    // scratch owned by the solvers (named buffers)
    std::vector<std::pair<std::string, nop::DevBuf>> bufs;
    // pinned host buffers (named) that per-call host <-> device copies go
    // through, so that the copies stay asynchronous; every call that fills
    // one ends with a stream synchronisation before the next call reuses it
    std::vector<std::pair<std::string, nop::DevBuf>> pins;
    // a tensor-core kernel's wait-limit flag whose check is deferred to the
    // caller's final synchronisation (pinned host int), or null
    const int* tc_err_pending = nullptr;
    bool defer_tc_check = false;   // set by a solve whose warm start ends in its sync

    void set_error(const std::string& m) { err = m; }
    // Device buffer `name` with at least `bytes` bytes (grows, contents kept undefined).
    int scratch(const char* name, size_t bytes, void** out);
    // Pinned host buffer `name` with at least `bytes` bytes (grows after a
    // stream synchronisation, contents kept undefined).
    int pinned(const char* name, size_t bytes, void** out);
    // After the stream was synchronised: NOP_ETIMEOUT if a deferred
    // tensor-core wait-limit flag is set (and clears the pending check).
    int check_deferred();
};

namespace nop {
// Quadrature builders (quadrature.cu)
int build_gauss_legendre(nop_ctx* ctx);
int build_level_symmetric_s8(nop_ctx* ctx);

// 1D slab solvers (sn1d.cu)
int sn1d_solve(nop_ctx* ctx, const nop_solve_opts* o, bool eigen, const double* phi0,
               bool phi0_dev, const double* k0, double* phi_out, bool out_dev,
               double* k_out, nop_stats* st);

// Neural operators (deeponet.cu, fno.cu)
int no_layout(const nop_no_config* cfg, std::vector<long long>* off,
              std::vector<long long>* len, long long* total);
int deeponet_forward_raw(nop_ctx* ctx, int n, const float* U, int P, const float* X,
                         float* out, bool keep);
int deeponet_backward(nop_ctx* ctx, int n, int P, const float* dout, const float* U,
                      const float* X);
int deeponet_project(nop_ctx* ctx, const double* field_host, float* out_host);
// Recast mismatch bands of a diffusion batch on the operator's M-bin grid
// (diffusion.cu): PL, PD, PU of -dL.
int diffusion_bands(nop_ctx* ctx, int M, double d_star, double siga_star, float* PL, float* PD,
                    float* PU);
// The recast iteration (Eq. 24) enqueued without synchronising (no_capi.cu):
// statistics land in a pinned buffer *stat_h, read by recast_collect after the
// stream was synchronised.
int recast_enqueue(nop_ctx* ctx, double tol, int itmax, double* pd, const int** stat_h);
void recast_collect(nop_ctx* ctx, const int* stat_h, nop_stats* st, bool per_instance);
int deeponet_recast(nop_ctx* ctx, double tol, int itmax, double* phi_d, int* status_d,
                    int* iters_d, bool predict_only, const double* src_d);
int fno_forward_raw(nop_ctx* ctx, int n, const float* in, int n1, int n2, float* out, bool keep);
int fno_backward(nop_ctx* ctx, int n, int n1, int n2, const float* dout);
int fno_recast(nop_ctx* ctx, double tol, int itmax, double* phi_d, int* status_d, int* iters_d,
               bool predict_only, const double* src_d);
// Recast steps on an operator grid of M points, B instances (deeponet.cu):
// split the source S + D u into unit-integral parts U [2B][M] (cell size h),
// combine the operator outputs as sigma+ N[+] - sigma- N[-], and the
// convergence bookkeeping (status 0 running, 1 converged, 3 diverged).
int recast_split(nop_ctx* ctx, int B, int M, double h, const float* PS, const float* PD,
                 const float* u, float* U, float* sig, int* flags);
int recast_combine(nop_ctx* ctx, int B, int M, const float* out, const float* sig,
                   const int* flags, float* res);
int recast_update(nop_ctx* ctx, int B, int M, double tol, const float* unew, float* u,
                  int* status, int* iters, double* prev, int* run, int* active);

// Simple-preconditioning eigen warm start (sp_eigen.cu): phi_d [G*C] device
// out (unit production), k/status/iterations per instance on the host.
// status: 0 cap reached, 1 converged, 3 diverged (phi flat, k = 1).
// constrained: refine each prediction by one model-based source iteration
// (App. A2 Eq. A7-A8).
int sp_eigen(nop_ctx* ctx, double tol, int itmax, double* phi_d, std::vector<double>* k_h,
             std::vector<int>* status_h, std::vector<int>* iters_h, bool constrained = false);

// Fused recast iteration for the 128-sensor, 4 x 128, p = 128 DeepONet
// (recast_fused.cu); active2 points at two device counters.
bool recast_fused_supported(const nop_no_config& c);
int recast_fused_run(nop_ctx* ctx, int B, double h, double tol, int itmax, const float* PS,
                     const float* PD, const float* PL, const float* PU, float* u,
                     const float* const W[4], const float* const b[4],
                     const float* Tref, float* beta, float* beta_keep, int* status, int* iters,
                     double* prev, int* run, int* active2, int* its);

// Final DeepONet flux of the 128-wide depth-4 trunk on tcgen05 tensor cores
// (trunk_tc.cu): distinct points in CSR groups of instances with equal cell
// counts; err (device int) is set if a completion wait timed out.
// tinfo: per 128-point tile {first group, last group, first and end index
// into the instance list}.
int trunk_tc_launch(nop_ctx* ctx, long long P, const int4* tinfo, const long long* gpt,
                    const int* gI, const int* ginst, const int* list, const long long* cell_off,
                    const float* const W[4], const float* const b[4], const float* beta_keep,
                    const int* status, double* phi, int* err);

// 2D x-y solver (sn2d.cu)
int xy_solve(nop_ctx* ctx, const nop_solve_opts* o, bool eigen, const double* phi0, double k0,
             double* phi_out, bool out_dev, double* k_out, nop_stats* st);

// Lane split of the 1D sweep (log2 lanes per angle group, angles per lane).
// team selection of the slab batch scheduler (sn1d.cu)
int sn1d_select_teams(int n, const double* lat_w, const double* lat_t, int warps, int width,
                      int mode, double margin, std::vector<char>& team, double* span);

// lane split of the chunked layout for I cells and order N; cost_out: the
// model's issue slots of one direction half per iteration
void sn1d_pick_config(int cells, int order, int* lg_ng, int* A, bool pow2 = false,
                      double* cost_out = nullptr);
}  // namespace nop
