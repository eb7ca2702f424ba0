/*
 * oracle/sn_sweep.c -- FP64 reference transport sweeps (TEST INFRASTRUCTURE ONLY).
 *
 * This file is part of the CPU oracle.  Only tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the CUDA library never links it.
 *
 * What it computes (paper Sec. 5.1, Eq. 12, and the S_N method named there):
 * one transport sweep of the discrete-ordinates equations with the diamond-
 * difference (DD) spatial closure, for a given emission density q (the whole
 * right-hand side of the streaming-collision equation, already including any
 * angular normalisation factor).  A sweep solves, for every direction, the
 * streaming + collision operator exactly on the DD mesh and returns the
 * scalar flux phi = sum_d w_d psi_d (cell averages) and the outgoing
 * boundary angular fluxes.
 *
 * 1D slab, one direction mu != 0, cell i of width dx_i:
 *     mu (psi_{i+1/2} - psi_{i-1/2}) / dx_i + sigt_i psi_i = q_i
 *     psi_i = (psi_{i+1/2} + psi_{i-1/2}) / 2              (diamond difference)
 * hence, with a = |mu|/dx_i and psi_in the upwind edge value,
 *     psi_i   = (q_i + 2 a psi_in) / (sigt_i + 2 a)
 *     psi_out = 2 psi_i - psi_in.
 *
 * 2D x-y, one direction (mu, eta), cell (i, j) of size dx x dy:
 *     mu (psi_R - psi_L)/dx + eta (psi_T - psi_B)/dy + sigt psi_c = q
 *     psi_c = (psi_L + psi_R)/2 = (psi_B + psi_T)/2
 * hence psi_c = (q + 2a psi_xin + 2b psi_yin) / (sigt + 2a + 2b),
 *       a = |mu|/dx, b = |eta|/dy, and each outgoing edge = 2 psi_c - incoming.
 *
 * No negative-flux fix-up is applied: the plain DD answer is the definition.
 * Plain loops in the order the definition states; nothing is blocked or fused.
 */
#include <stddef.h>

/* 1D sweep.
 *   I                cells; dx[I], sigt[I], q[I]
 *   N                directions; mu[N] (nonzero), w[N]
 *   in_left[n]       incoming psi at x = 0 for directions with mu[n] > 0
 *   in_right[n]      incoming psi at x = L for directions with mu[n] < 0
 *   phi[I]           out: sum_n w[n] psi_n,i
 *   out_left[n]      out: psi at x = 0 for mu[n] < 0 (left untouched for mu > 0)
 *   out_right[n]     out: psi at x = L for mu[n] > 0 (left untouched for mu < 0)
 */
void ora_sweep1d(int I, const double *dx, const double *sigt, const double *q,
                 int N, const double *mu, const double *w,
                 const double *in_left, const double *in_right,
                 double *phi, double *out_left, double *out_right)
{
    for (int i = 0; i < I; ++i) phi[i] = 0.0;
    for (int n = 0; n < N; ++n) {
        double m = mu[n];
        if (m > 0.0) {
            double psi_in = in_left[n];
            for (int i = 0; i < I; ++i) {
                double a = m / dx[i];
                double psi_c = (q[i] + 2.0 * a * psi_in) / (sigt[i] + 2.0 * a);
                phi[i] += w[n] * psi_c;
                psi_in = 2.0 * psi_c - psi_in;
            }
            out_right[n] = psi_in;
        } else {
            double psi_in = in_right[n];
            for (int i = I - 1; i >= 0; --i) {
                double a = -m / dx[i];
                double psi_c = (q[i] + 2.0 * a * psi_in) / (sigt[i] + 2.0 * a);
                phi[i] += w[n] * psi_c;
                psi_in = 2.0 * psi_c - psi_in;
            }
            out_left[n] = psi_in;
        }
    }
}

/* 1D sweep with a linearly anisotropic emission (Sec. 5.1 Eq. 25): the
 * emission of direction n in cell i is q0[i] + mu[n] q1[i].  Same arguments
 * as ora_sweep1d plus
 *   cur[I]           out: sum_n w[n] mu[n] psi_n,i (the current)
 */
void ora_sweep1d_p1(int I, const double *dx, const double *sigt, const double *q0,
                    const double *q1, int N, const double *mu, const double *w,
                    const double *in_left, const double *in_right,
                    double *phi, double *cur, double *out_left, double *out_right)
{
    for (int i = 0; i < I; ++i) {
        phi[i] = 0.0;
        cur[i] = 0.0;
    }
    for (int n = 0; n < N; ++n) {
        double m = mu[n];
        if (m > 0.0) {
            double psi_in = in_left[n];
            for (int i = 0; i < I; ++i) {
                double a = m / dx[i];
                double q = q0[i] + m * q1[i];
                double psi_c = (q + 2.0 * a * psi_in) / (sigt[i] + 2.0 * a);
                phi[i] += w[n] * psi_c;
                cur[i] += w[n] * m * psi_c;
                psi_in = 2.0 * psi_c - psi_in;
            }
            out_right[n] = psi_in;
        } else {
            double psi_in = in_right[n];
            for (int i = I - 1; i >= 0; --i) {
                double a = -m / dx[i];
                double q = q0[i] + m * q1[i];
                double psi_c = (q + 2.0 * a * psi_in) / (sigt[i] + 2.0 * a);
                phi[i] += w[n] * psi_c;
                cur[i] += w[n] * m * psi_c;
                psi_in = 2.0 * psi_c - psi_in;
            }
            out_left[n] = psi_in;
        }
    }
}

/* 2D x-y sweep on a uniform nx x ny mesh, cell (i, j) stored at [j*nx + i].
 *   sigt, q          [ny*nx]
 *   M                directions; mu[M], eta[M] (both nonzero), w[M]
 *   in_x[d*ny + j]   incoming psi on the x-face the direction enters
 *                    (x = 0 if mu > 0, x = Lx if mu < 0), row j
 *   in_y[d*nx + i]   incoming psi on the y-face it enters (y = 0 if eta > 0)
 *   phi              out: sum_d w[d] psi_d  [ny*nx]
 *   out_x[d*ny + j]  out: psi leaving through the opposite x-face, row j
 *   out_y[d*nx + i]  out: psi leaving through the opposite y-face, column i
 *   ybuf             scratch of nx doubles (the running y-edge fluxes)
 */
void ora_sweep2d(int nx, int ny, double dx, double dy,
                 const double *sigt, const double *q,
                 int M, const double *mu, const double *eta, const double *w,
                 const double *in_x, const double *in_y,
                 double *phi, double *out_x, double *out_y, double *ybuf)
{
    for (int c = 0; c < nx * ny; ++c) phi[c] = 0.0;
    for (int d = 0; d < M; ++d) {
        double a = (mu[d] > 0 ? mu[d] : -mu[d]) / dx;
        double b = (eta[d] > 0 ? eta[d] : -eta[d]) / dy;
        int i0 = mu[d] > 0 ? 0 : nx - 1, di = mu[d] > 0 ? 1 : -1;
        int j0 = eta[d] > 0 ? 0 : ny - 1, dj = eta[d] > 0 ? 1 : -1;
        for (int i = 0; i < nx; ++i) ybuf[i] = in_y[(size_t)d * nx + i];
        for (int jj = 0, j = j0; jj < ny; ++jj, j += dj) {
            double psi_x = in_x[(size_t)d * ny + j];
            for (int ii = 0, i = i0; ii < nx; ++ii, i += di) {
                size_t c = (size_t)j * nx + i;
                double psi_c = (q[c] + 2.0 * a * psi_x + 2.0 * b * ybuf[i]) /
                               (sigt[c] + 2.0 * a + 2.0 * b);
                phi[c] += w[d] * psi_c;
                psi_x = 2.0 * psi_c - psi_x;
                ybuf[i] = 2.0 * psi_c - ybuf[i];
            }
            out_x[(size_t)d * ny + j] = psi_x;
        }
        for (int i = 0; i < nx; ++i) out_y[(size_t)d * nx + i] = ybuf[i];
    }
}
