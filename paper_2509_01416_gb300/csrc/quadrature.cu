// Angular quadratures built on the device (FP64).
//
// 1D: Gauss-Legendre S_N, the slab quadrature of the S_N method (Sec. 5.1;
// the paper's benchmark solver uses N = 32).  Nodes are the roots of P_N found
// by Newton's method from the Tricomi initial guess, weights
// 2 / ((1 - x^2) P_N'(x)^2); nodes ascending, weights summing to 2 so that
// phi = sum w psi integrates over mu in [-1, 1] (Eq. 17).
//
// 2D: level-symmetric S8 for the x-y extension (Sec. 6 notes that the method
// carries over to higher dimensions).  Squared direction cosines take the
// levels l_i = t + (i - 1)(1 - 3t)/3, i = 1..4; the octant points are the
// triples (i, j, k) with i + j + k = 6, grouped into the permutation classes
// (1,1,4), (1,2,3), (2,2,2) with one weight each.  For a trial t the three
// weights solve <1> = 1, <mu^4> = 1/5, <mu^6> = 1/7 over the octant (Cramer's
// rule); t is the root of <mu^8> - 1/9 found by bisection.  The folded x-y set
// keeps the xi > 0 hemisphere with weights w_class / 4 (sum 1 over the 40
// directions).  Direction order: quadrants (mu<0, eta<0), (mu>0, eta<0),
// (mu<0, eta>0), (mu>0, eta>0); inside a quadrant the points in lexicographic
// (i, j) order.
#include <cmath>
#include <map>

#include "nop_internal.cuh"

namespace nop {

__global__ void gauss_legendre_kernel(const int* orders, const int* offs, int n_orders,
                                      double* mu, double* w) {
    int blk = blockIdx.x;
    if (blk >= n_orders) return;
    int N = orders[blk];
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        // ascending: the n-th root counted from -1
        double x = -cos(M_PI * (n + 0.75) / (N + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 1; k < N; ++k) {
                double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = N * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        // final derivative at the converged root
        double p0 = 1.0, p1 = x;
        for (int k = 1; k < N; ++k) {
            double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
            p0 = p1;
            p1 = p2;
        }
        dp = N * (x * p1 - p0) / (x * x - 1.0);
        mu[offs[blk] + n] = x;
        w[offs[blk] + n] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

int build_gauss_legendre(nop_ctx* ctx) {
    SlabDev& s = ctx->slab;
    std::map<int, int> off;
    int total = 0;
    for (int N : s.order)
        if (!off.count(N)) {
            off[N] = total;
            total += N;
        }
    std::vector<int> ords, offs;
    for (auto& kv : off) {
        ords.push_back(kv.first);
        offs.push_back(kv.second);
    }
    s.qoff_h.resize(s.n_inst);
    for (int b = 0; b < s.n_inst; ++b) s.qoff_h[b] = off[s.order[b]];
    int *ords_d, *offs_d;
    void* p;
    NOP_TRY(ctx->scratch("gl_orders", ords.size() * sizeof(int), &p));
    ords_d = (int*)p;
    NOP_TRY(ctx->scratch("gl_offs", offs.size() * sizeof(int), &p));
    offs_d = (int*)p;
    NOP_TRY(ctx->scratch("gl_mu", total * sizeof(double), &p));
    s.mu_d = (double*)p;
    NOP_TRY(ctx->scratch("gl_w", total * sizeof(double), &p));
    s.w_d = (double*)p;
    NOP_TRY(ctx->scratch("gl_qoff", s.n_inst * sizeof(int), &p));
    s.qoff_d = (int*)p;
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(s.qoff_d, s.qoff_h.data(), s.n_inst * sizeof(int),
                                      cudaMemcpyHostToDevice, ctx->stream));
    // the sets depend on the orders and their offsets (the order in which the
    // orders first appear in the batch): a new problem with both unchanged
    // keeps the sets already built
    if (ords != s.gl_orders || offs != s.gl_offs) {
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(ords_d, ords.data(), ords.size() * sizeof(int),
                                          cudaMemcpyHostToDevice, ctx->stream));
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(offs_d, offs.data(), offs.size() * sizeof(int),
                                          cudaMemcpyHostToDevice, ctx->stream));
        gauss_legendre_kernel<<<(int)ords.size(), 64, 0, ctx->stream>>>(ords_d, offs_d,
                                                                       (int)ords.size(), s.mu_d,
                                                                       s.w_d);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        s.gl_orders = ords;
        s.gl_offs = offs;
    }
    // host copies of the orders must stay valid until the copies above complete
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return NOP_OK;
}

// ----------------------------------------------------------------- LS S8
__device__ void ls8_weights(double t, double wc[3], double lev2[4]) {
    double d = (1.0 - 3.0 * t) / 3.0;
    for (int i = 0; i < 4; ++i) lev2[i] = t + i * d;
    // rows: moment 0, 4, 6 ; columns: classes (1,1,4), (1,2,3), (2,2,2)
    double M[3][3];
    const double* l = lev2;
    for (int r = 0; r < 3; ++r) {
        int p = (r == 0) ? 0 : (r == 1 ? 2 : 3);   // powers of the squared cosine
        M[r][0] = 2.0 * pow(l[0], p) + pow(l[3], p);
        M[r][1] = 2.0 * (pow(l[0], p) + pow(l[1], p) + pow(l[2], p));
        M[r][2] = pow(l[1], p);
    }
    double rhs[3] = {1.0, 1.0 / 5.0, 1.0 / 7.0};
    auto det3 = [](double a[3][3]) {
        return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
               a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
               a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    };
    double D = det3(M);
    for (int c = 0; c < 3; ++c) {
        double Mc[3][3];
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) Mc[r][q] = (q == c) ? rhs[r] : M[r][q];
        wc[c] = det3(Mc) / D;
    }
}

__device__ double ls8_m8(double t) {
    double wc[3], l[4];
    ls8_weights(t, wc, l);
    double m = wc[0] * (2.0 * pow(l[0], 4) + pow(l[3], 4)) +
               wc[1] * 2.0 * (pow(l[0], 4) + pow(l[1], 4) + pow(l[2], 4)) +
               wc[2] * pow(l[1], 4);
    return m - 1.0 / 9.0;
}

__global__ void ls8_kernel(double* mu, double* eta, double* w) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo = 0.03, hi = 0.06, flo = ls8_m8(lo);
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi), fm = ls8_m8(mid);
        if ((fm > 0) == (flo > 0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
    }
    double wc[3], l[4];
    ls8_weights(0.5 * (lo + hi), wc, l);
    const int sx[4] = {-1, 1, -1, 1}, sy[4] = {-1, -1, 1, 1};
    int d = 0;
    for (int q = 0; q < 4; ++q)
        for (int i = 1; i <= 4; ++i)
            for (int j = 1; j <= 4; ++j) {
                int k = 6 - i - j;
                if (k < 1 || k > 4) continue;
                int a = i, b = j, c = k;
                // sort the triple to find its permutation class
                if (a > b) { int t = a; a = b; b = t; }
                if (b > c) { int t = b; b = c; c = t; }
                if (a > b) { int t = a; a = b; b = t; }
                int cls = (a == 1 && b == 1) ? 0 : (a == 2 ? 2 : 1);
                mu[d] = sx[q] * sqrt(l[i - 1]);
                eta[d] = sy[q] * sqrt(l[j - 1]);
                w[d] = wc[cls] / 4.0;
                ++d;
            }
}

int build_level_symmetric_s8(nop_ctx* ctx) {
    void* p;
    NOP_TRY(ctx->scratch("ls8_mu", 40 * sizeof(double), &p));
    ctx->xy.mu_d = (double*)p;
    NOP_TRY(ctx->scratch("ls8_eta", 40 * sizeof(double), &p));
    ctx->xy.eta_d = (double*)p;
    NOP_TRY(ctx->scratch("ls8_w", 40 * sizeof(double), &p));
    ctx->xy.w_d = (double*)p;
    ls8_kernel<<<1, 32, 0, ctx->stream>>>(ctx->xy.mu_d, ctx->xy.eta_d, ctx->xy.w_d);
    NOP_CUDA_TRY(ctx, cudaGetLastError());
    return NOP_OK;
}

}  // namespace nop
