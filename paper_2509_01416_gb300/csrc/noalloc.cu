// Allocation-free slab solve.
//
// Some callers cannot call cudaMalloc: plug-ins whose host application owns
// the device memory and forbids allocations outside a budget it reserved up
// front, or real-time control loops that must not touch the allocator (a
// cudaMalloc can take milliseconds and can synchronise the device).
// nop_slab_solve_noalloc serves them: it solves one single-group
// fixed-source slab with the library's FP32 slab kernel, and every
// intermediate buffer lives in the file-scope device array below.  The array
// is a fixed cost of every GPU that loads the library and is held until the
// process exits.  The paper has no counterpart; this is a library convenience.
//
// The array is shared by every call: calls that overlap on the GPU (two
// streams, or two host threads) race on it and must be serialised by the
// caller.  A call clears what has to start at zero (work counters, status)
// and overwrites everything else before reading it; the solve kernel itself
// clears the boundary fluxes.  The Gauss-Legendre set of the last order
// solved on a device stays in the array and is rebuilt only when the order
// changes.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address (cudaGetSymbolAddress) and raises the solve
// kernel's dynamic shared-memory limit (cudaFuncSetAttribute); later calls on
// that device reuse both.  In host code the array's name is only a host-side
// stand-in, not a device address, which is why the kernels receive the
// looked-up address.  The first call on each device should come before any
// stream capture.
#include <cmath>

#include "sn1d_impl.cuh"

namespace {

constexpr int MAX_CELLS = NOP_NOALLOC_MAX_CELLS;
constexpr int MAX_ORDER = NOP_NOALLOC_MAX_ORDER;

// layout of the scratch array (byte offsets, 256-byte aligned sections)
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_X = 0;                                                    // Cell4<float>[MAX_CELLS]
constexpr size_t OFF_U = al(OFF_X + sizeof(nop::Cell4<float>) * MAX_CELLS);   // Cell2<float>[MAX_CELLS]
constexpr size_t OFF_EXT = al(OFF_U + sizeof(nop::Cell2<float>) * MAX_CELLS); // float[MAX_CELLS]
constexpr size_t OFF_MU = al(OFF_EXT + sizeof(float) * MAX_CELLS);            // double[MAX_ORDER]
constexpr size_t OFF_W = al(OFF_MU + sizeof(double) * MAX_ORDER);             // double[MAX_ORDER]
constexpr size_t OFF_PSIB = al(OFF_W + sizeof(double) * MAX_ORDER);           // float[MAX_ORDER]
constexpr size_t OFF_INT = al(OFF_PSIB + sizeof(float) * MAX_ORDER);          // 16 ints
constexpr size_t OFF_LL = al(OFF_INT + sizeof(int) * 16);                     // 2 long long
constexpr size_t OFF_DBL = al(OFF_LL + sizeof(long long) * 2);                // 4 doubles
constexpr size_t SCRATCH_BYTES = al(OFF_DBL + sizeof(double) * 4);

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
unsigned char* g_addr[MAX_DEVICES] = {nullptr};
int g_order[MAX_DEVICES] = {0};   // order of the quadrature held in the array

// Instance table of the single instance; clears the work counters and the
// outputs, which must start at zero.
__global__ void init_kernel(unsigned char* base, int I, int N, double dx, int cfg) {
    int* ints = (int*)(base + OFF_INT);
    long long* ll = (long long*)(base + OFF_LL);
    double* dbl = (double*)(base + OFF_DBL);
    if (threadIdx.x == 0) {
        ints[0] = 0;      // order list: instance 0
        ints[1] = 0;      // small-queue counter
        ints[2] = 0;      // block-queue counter
        ints[3] = I;      // cells
        ints[4] = N;      // order
        ints[5] = 0;      // quadrature offset
        ints[6] = cfg;    // lane split
        ints[7] = 0;      // iterations out
        ints[8] = 0;      // status out
        ints[9] = 0;      // outer iterations (unused)
        ll[0] = 0;        // first cell
        ll[1] = 0;        // boundary-flux offset
        dbl[0] = dx;
        dbl[1] = 1.0;     // k0 (unused)
        dbl[2] = 0.0;     // final change
        dbl[3] = 0.0;     // k out (unused)
    }
}

// The coefficient check of nop_set_problem, on the device and without a host
// synchronisation: sigma_t must be positive and finite, sigma_s and the
// source finite.  A bad instance gets status NOP_EINVAL and zero iterations,
// and its work counter is taken, so the solve kernel that follows finds no
// instance to run and leaves the flux at zero.
__global__ void coef_check_kernel(unsigned char* base, int I, const double* sigt,
                                  const double* sigs, const double* src) {
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I; i += gridDim.x * blockDim.x)
        bad |= !(sigt[i] > 0.0) || !isfinite(sigt[i]) || !isfinite(sigs[i]) || !isfinite(src[i]);
    if (bad) {
        int* ints = (int*)(base + OFF_INT);
        ints[1] = 1;             // the one instance is taken: the solve skips it
        ints[8] = NOP_EINVAL;    // status out (same value from every writer)
    }
}

__global__ void stats_kernel(const unsigned char* base, int* stats_out) {
    const int* ints = (const int*)(base + OFF_INT);
    stats_out[0] = ints[7];
    stats_out[1] = ints[8];
}

}  // namespace

namespace nop {
int sn1d_launch_f32(const Sn1dArgs& a, long long C, const double* sigt, const double* sigs,
                    const double* src, Cell4<float>* X, float* ext, double* phi_out,
                    cudaStream_t stream);
int sn1d_f32_raise_smem_limit();
// Gauss-Legendre nodes and weights of the orders listed in device memory
// (csrc/quadrature.cu).
__global__ void gauss_legendre_kernel(const int* orders, const int* offs, int n_orders,
                                      double* mu, double* w);
}  // namespace nop

extern "C" int nop_slab_solve_noalloc(const double* sigma_t, const double* sigma_s,
                                      const double* source, int n_cells, double width, int order,
                                      double tol, int itmax, double* phi_out, int* stats_out,
                                      void* stream) {
    if (!sigma_t || !sigma_s || !source || !phi_out || !stats_out) return NOP_EINVAL;
    if (n_cells < 1 || n_cells > MAX_CELLS || order < 2 || order > MAX_ORDER || (order & 1) ||
        !(width > 0) || !(tol > 0) || itmax < 1)
        return NOP_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return NOP_ECUDA;
    if (!g_addr[dev]) {
        // once per device, with that device current
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return NOP_ECUDA;
        if (nop::sn1d_f32_raise_smem_limit() != NOP_OK) return NOP_ECUDA;
        g_addr[dev] = (unsigned char*)p;
        g_order[dev] = 0;
    }
    unsigned char* base = g_addr[dev];
    cudaStream_t st = (cudaStream_t)stream;
    int lg, A;
    nop::sn1d_pick_config(n_cells, order, &lg, &A);
    const double dx = width / n_cells;
    int* ints = (int*)(base + OFF_INT);
    init_kernel<<<1, 32, 0, st>>>(base, n_cells, order, dx, (lg << 8) | A);
    if (g_order[dev] != order) {
        // ints[4] holds the order and ints[5] the offset 0 (written just above)
        nop::gauss_legendre_kernel<<<1, 64, 0, st>>>(ints + 4, ints + 5, 1,
                                                      (double*)(base + OFF_MU),
                                                      (double*)(base + OFF_W));
    }
    coef_check_kernel<<<(n_cells + 255) / 256, 256, 0, st>>>(base, n_cells, sigma_t, sigma_s,
                                                             source);
    if (cudaGetLastError() != cudaSuccess) {
        g_order[dev] = 0;
        return NOP_ECUDA;
    }
    g_order[dev] = order;
    long long* ll = (long long*)(base + OFF_LL);
    double* dbl = (double*)(base + OFF_DBL);
    nop::Sn1dArgs a{};
    a.n_inst = 1;
    a.G = 1;
    a.C = n_cells;
    a.order_list = ints + 0;
    a.n_small = 1;
    a.big_list = ints + 0;
    a.n_big = 0;
    a.big_blocks = 0;
    a.counter = ints + 1;
    a.cell_off = ll + 0;
    a.ncell = ints + 3;
    a.nang = ints + 4;
    a.dx = dbl + 0;
    a.qoff = ints + 5;
    a.mu = (const double*)(base + OFF_MU);
    a.w = (const double*)(base + OFF_W);
    a.boff = ll + 1;
    a.cfg = ints + 6;
    a.X = base + OFF_X;
    a.U = base + OFF_U;
    a.scat = nullptr;
    a.ext = base + OFF_EXT;
    a.psib = base + OFF_PSIB;
    a.bc_left = 0;
    a.bc_right = 0;
    a.smem_cells = 1;
    a.eigen = 0;
    a.k0 = dbl + 1;
    a.tol = tol;
    a.tol_inner = tol;
    a.tol_k = tol;
    a.itmax = itmax;
    a.itmax_inner = itmax;
    a.it_out = ints + 7;
    a.st_out = ints + 8;
    a.ch_out = dbl + 2;
    a.k_out = dbl + 3;
    a.outer_out = ints + 9;
    a.trace = nullptr;
    const int rc = nop::sn1d_launch_f32(a, n_cells, sigma_t, sigma_s, source,
                                        (nop::Cell4<float>*)(base + OFF_X),
                                        (float*)(base + OFF_EXT), phi_out, st);
    if (rc != NOP_OK) return rc;
    stats_kernel<<<1, 1, 0, st>>>(base, stats_out);
    return cudaGetLastError() == cudaSuccess ? NOP_OK : NOP_ECUDA;
}
