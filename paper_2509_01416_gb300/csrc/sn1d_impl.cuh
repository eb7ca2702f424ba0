// Batched 1D slab S_N solver: source iteration (Sec. 3.1 Eq. 3a/4b, Sec. 5.1
// Eq. 12 and 20) and power iteration with inner sweeps (Sec. 5.2 Eq. 26,
// App. A2 Eq. A2-A4), multigroup by Gauss-Seidel over groups (Sec. 5.3
// Eq. 27-29), diamond-difference spatial closure.
//
// GPU organisation.  One warp owns one slab instance at a time and runs its
// whole iteration (all sweeps, norms, eigenvalue updates) without leaving the
// kernel; warps pull instances from a work counter in longest-first order.
// Instances whose latency on one warp would exceed the batch's mean warp
// load run on a whole 12-warp block instead, their angles split over the
// warps (one block per SM, 192 KB of staging shared memory).
// The 32 lanes are split into nt = 32/ng cell chunks x ng angle groups; a lane
// carries A polar angles |mu| of its group over its chunk, first for mu < 0
// (right to left) and then for mu > 0 (left to right).  Along the cells the
// diamond-difference recurrence is affine, psi_out = alpha psi_in + beta with
// alpha = (c - st)/(c + st), beta = 2 s/(c + st), c = 2|mu|/dx, so chunks first
// compose their maps, exchange them in a warp-shuffle scan, and then sweep with
// the correct incoming flux.  The angle sum phi_i = sum w psi_i is reduced over
// the ng lanes of a chunk with xor shuffles; the lane (i mod ng) owns cell i.
//
// Per-cell working data (arrays of the whole batch, group-major):
//   X[g][c] = {st, ss/2 (in-group scattering), z (half the source from outside
//              the group's own flux), phi}
//   U[g][c] = {s (emission density used this iteration), phi_minus}
// Norms, eigenvalue ratios and convergence tests are FP64 in every precision.
//
// Optionally (NOP_DSA) each group's sweep is followed by a diffusion synthetic
// correction, a classical accelerator of the iteration kept for comparison
// with the warm start: sn1d_dsa_factor factors every instance's edge
// diffusion system once per solve, and dsa_pass solves it after each sweep on
// one warp.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>

#pragma once
#include "nop_internal.cuh"

#define SN1D_THREADS 384
#define SN1D_BLOCKS_PER_SM 1
#define SN1D_STAGE_BYTES (192 * 1024)

namespace nop {

template <typename T>
struct alignas(4 * sizeof(T)) Cell4 {
    T st, y, z, phi;
};
template <typename T>
struct alignas(2 * sizeof(T)) Cell2 {
    T s0, s1;
};

// One edge k of the diffusion synthetic acceleration system: the inverse
// pivot fm = 1/p_k and the off-diagonal entry o = o_k between edges k and
// k+1 (zero for the last edge).  The forward elimination is
// y_k = fm (b_k - o_{k-1} y_{k-1}), the back substitution
// e_k = y_k - o_k fm e_{k+1}.
template <typename T>
struct alignas(2 * sizeof(T)) DsaEdge {
    T fm, o;
};

struct Sn1dArgs {
    int n_inst;
    int G;
    long long C;
    const int* order_list;   // small instances (one warp each), longest first
    int n_small;
    const int* big_list;     // large instances (one whole block each), longest first
    int n_big;
    int big_blocks;          // blocks [0, big_blocks) drain the large-instance queue first
    int* counter;            // [0] small queue, [1] big queue
    const long long* cell_off;
    const int* ncell;
    const int* nang;
    const double* dx;
    const int* qoff;
    const double* mu;
    const double* w;
    const long long* boff;
    void* X;
    void* U;              // Cell2 [C]: per-cell {s, phi_minus} of the warp path
    const int* cfg;       // per instance: (log2 ng) << 8 | A
    const void* scat;     // T [G][G][C], halved; only read when G > 1
    void* ext;            // T [G][C], halved external / fission source
    void* psib;           // T boundary fluxes [boff + (g*h + hi)*2 + side]
    // linearly anisotropic in-group scattering (Eq. 25), fixed source, warp path
    int p1;
    const void* y1;       // T [G][C]: (3/2) Sigma_s1
    void* cur;            // T [G][C]: current J = sum w mu psi of the last iteration
    void* s1buf;          // T [C]: (3/2) Sigma_s1 J of the group being swept
    void* jm;             // T [C]: mu < 0 part of the new current
    int bc_left, bc_right;
    // diffusion synthetic acceleration: factors of each instance's edge
    // diffusion system, DsaEdge<T> [G][C + 32 n_inst] ({1/pivot, off-diagonal}
    // per edge); instance b's region
    // starts at cell_off[b] + 32 b and holds its I+1 edges lane-interleaved:
    // with m = ceil((I+1)/32) edges per lane, edge k = t m + j (lane t's j-th)
    // sits at j * 32 + t, so a warp's accesses to its lanes' j-th edges are
    // contiguous
    int dsa;
    void* dsaf;
    void* dsaw;           // T [2 (C + 32 n_inst)]: work values of instances whose
                          // correction does not fit the shared-memory scratch
    int smem_cells;       // cells the block path can stage in shared memory
    // eigen
    int eigen;
    const void* nsf;      // T [G][C]
    const double* chi;    // [G]
    void* phiprev;        // T [G][C]
    const double* k0;     // [n_inst]
    double tol, tol_inner, tol_k;
    int itmax, itmax_inner;
    // outputs
    int* it_out;
    int* st_out;
    double* ch_out;
    double* k_out;
    int* outer_out;
    unsigned long long* trace;   // optional [n_inst][3]: start ns, end ns, SM id
};

// Reciprocal for the DD cell solve.  FP32: the special-function unit's
// approximation refined by one Newton step, e = 1 - d r, r <- r + r e, which
// removes the approximation's bias (a biased reciprocal scales every sweep and
// shifts eigenvalues by ~bias/(1 - spectral radius)).
__device__ __forceinline__ float rcp_dd(float d) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    const float e = fmaf(-d, r, 1.0f);
    return fmaf(r, e, r);
}
__device__ __forceinline__ double rcp_dd(double d) { return 1.0 / d; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The threads that own one instance: one warp, or the whole block.
struct Grp {
    bool block;
    int rank, size, warp, nwarps;
    double* red;   // block reduction scratch (nwarps doubles)
    __device__ void sync() const {
        if (block) __syncthreads();
        else __syncwarp();
    }
    __device__ double sum(double v) const {
        v = warp_sum(v);
        if (!block) return v;
        if ((threadIdx.x & 31) == 0) red[warp] = v;
        __syncthreads();
        double t = 0.0;
        for (int k = 0; k < nwarps; ++k) t += red[k];
        __syncthreads();
        return t;
    }
};

// Shared-memory staging of an instance: {sigma_t, s} of every cell, read by
// every sweep step, so the steps never wait on global memory.  The warp path
// stages into the warp's own slab of the block's shared memory (instances up
// to `cells`; larger ones read global memory); the block path stages once per
// block and adds one row of partial angle sums per warp (each warp owns its
// row, so the sweeps need no atomics; the rows are added after the sweep).
template <typename T>
struct Stage {
    Cell2<T>* ss;   // [cells] or null (unstaged)
    T* part;        // block path: [nwarps][cells]
    int cells;
    T* scratch;     // shared memory free between sweeps (the correction's work values)
    int scratch_words;
};

// Running sum carried along a sweep.  FP32 keeps a compensation term
// (Fast2Sum: the rounding error of every add is fed into the next one), so the
// angular flux carried across hundreds of optically thin cells does not
// accumulate one rounding per cell; FP64 adds plainly.
template <typename T>
struct CSum {
    T hi, lo;
    __device__ __forceinline__ void set(T v) {
        hi = v;
        lo = T(0);
    }
    __device__ __forceinline__ void add(T d) {
        if constexpr (sizeof(T) == 4) {
            const T u = d + lo;
            const T t = hi + u;
            lo = u - (t - hi);
            hi = t;
        } else {
            hi += d;
        }
    }
    __device__ __forceinline__ T val() const { return hi + lo; }
};

// Linearly anisotropic emission (Eq. 25) of one group: the emission of
// direction mu is s + mu s1, s1 = (3/2) Sigma_s1 J per cell; the sweep also
// accumulates the new current J = sum w mu psi.
template <typename T, int A>
struct P1Op {
    const T* s1;      // [I] s1 of the cells
    T* jm;            // [I] mu < 0 part of the current (written by the MINUS half)
    T* jc;            // [I] the new current (written by the PLUS half)
    T mua[A];         // |mu| of the lane's angles
    T wmu[A];         // w |mu|
};

// One direction half (MINUS: mu < 0, cells right to left) of one group, for
// the angles this warp carries.  Lanes: nt = 32/ng cell chunks x ng angle
// groups, A angles per lane.  Diamond difference in increment form: with
// delta = (s - st psi_in) / (c + st), c = 2|mu|/dx,
//     psi_cell = psi_in + delta,   psi_out = psi_in + 2 delta.
// Chunked splits first compose each chunk's affine map psi_out = (1 - D)
// psi_in + B (D = 1 - prod alpha kept as a deficit, B compensated), scan the
// maps over the chunks, then sweep.  The angle sum of a cell is reduced over
// the ng lanes of its chunk with xor shuffles; lane (k mod ng) owns the k-th
// cell of the chunk.  Warp path: the owner stores the MINUS partial sum in U
// and completes the cell in the PLUS half, accumulating the squared change
// and the squared flux (FP32 per lane within one iteration: the change of an
// FP32 flux is exact, and the FP64 sum across lanes forms the norms).  Block
// path: owners add their partial sums to the warp's row.
template <typename T, int A, bool MINUS, bool P1>
__device__ __forceinline__ void sweep_half(const bool block, Cell4<T>* X, Cell2<T>* U,
                                           const Stage<T>& sg, int I, int lg,
                                           const T (&cc)[A], const T (&wt)[A],
                                           const T (&psi_bnd)[A], T (&psi_out)[A],
                                           T& acc_d, T& acc_n, const P1Op<T, A>& an,
                                           const bool keep_df) {
    const int lane = threadIdx.x & 31;
    const int ng = 1 << lg, nt = 32 >> lg;
    const int j = lane & (ng - 1), t = lane >> lg;
    const int m = (I + nt - 1) / nt;
    const int k0 = t * m;
    const int len = max(0, min(m, I - k0));
    CSum<T> psi[A];
#pragma unroll
    for (int q = 0; q < A; ++q) psi[q].set(psi_bnd[q]);
    if (nt > 1) {
        CSum<T> Bc[A];
        T D[A];
#pragma unroll
        for (int q = 0; q < A; ++q) {
            Bc[q].set(T(0));
            D[q] = T(0);
        }
#pragma unroll 1
        for (int k = 0; k < len; ++k) {
            const int i = MINUS ? (I - 1 - (k0 + k)) : (k0 + k);
            T st, s;
            if (sg.ss) {
                const Cell2<T> w2 = sg.ss[i];
                st = w2.s0;
                s = w2.s1;
            } else {
                const Cell4<T> v = X[i];
                st = v.st;
                s = MINUS ? (v.y * v.phi + v.z) : U[i].s0;
            }
            T s1 = T(0);
            if constexpr (P1) s1 = an.s1[i];
#pragma unroll
            for (int q = 0; q < A; ++q) {
                T sq = s;
                if constexpr (P1) sq = MINUS ? s - an.mua[q] * s1 : s + an.mua[q] * s1;
                const T r2 = T(2) * rcp_dd(cc[q] + st);
                D[q] = (r2 * st) * (T(1) - D[q]) + D[q];
                Bc[q].add(r2 * (sq - st * Bc[q].hi));
            }
        }
        // inclusive scan of the chunk maps along the sweep (lanes stride ng)
        T Dv[A], Bv[A];
#pragma unroll
        for (int q = 0; q < A; ++q) {
            Dv[q] = D[q];
            Bv[q] = Bc[q].val();
        }
        for (int d = 1; d < nt; d <<= 1) {
#pragma unroll
            for (int q = 0; q < A; ++q) {
                const T Do = __shfl_up_sync(0xffffffffu, Dv[q], d << lg);
                const T Bo = __shfl_up_sync(0xffffffffu, Bv[q], d << lg);
                if (t >= d) {
                    Bv[q] = (Bo + Bv[q]) - Dv[q] * Bo;
                    Dv[q] = Dv[q] * (T(1) - Do) + Do;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < A; ++q) {
            T De = __shfl_up_sync(0xffffffffu, Dv[q], ng);
            T Be = __shfl_up_sync(0xffffffffu, Bv[q], ng);
            if (t == 0) {
                De = T(0);
                Be = T(0);
            }
            psi[q].set((psi_bnd[q] + Be) - De * psi_bnd[q]);
        }
    }
#pragma unroll 1
    for (int k = 0; k < m; ++k) {
        const bool valid = k < len;
        const int i = MINUS ? (I - 1 - (k0 + k)) : (k0 + k);
        T p = T(0), s = T(0), phio = T(0), pmv = T(0), pj = T(0);
        if (valid) {
            T st;
            if (sg.ss) {
                const Cell2<T> w2 = sg.ss[i];
                st = w2.s0;
                s = w2.s1;
                if (!block && !MINUS) {
                    // the owner's operands, fetched early
                    phio = X[i].phi;
                    pmv = U[i].s1;
                }
            } else {
                const Cell4<T> v = X[i];
                st = v.st;
                phio = v.phi;
                s = MINUS ? (v.y * v.phi + v.z) : U[i].s0;
                if (!MINUS) pmv = U[i].s1;
            }
            T s1 = T(0);
            if constexpr (P1) s1 = an.s1[i];
#pragma unroll
            for (int q = 0; q < A; ++q) {
                T sq = s;
                if constexpr (P1) sq = MINUS ? s - an.mua[q] * s1 : s + an.mua[q] * s1;
                const T dl = rcp_dd(cc[q] + st) * (sq - st * psi[q].hi);
                const T pc = psi[q].hi + (dl + psi[q].lo);
                p += wt[q] * pc;
                if constexpr (P1) pj += (MINUS ? -an.wmu[q] : an.wmu[q]) * pc;
                psi[q].add(dl + dl);
            }
        }
        for (int o = 1; o < ng; o <<= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        if constexpr (P1)
            for (int o = 1; o < ng; o <<= 1) pj += __shfl_xor_sync(0xffffffffu, pj, o);
        if (valid && (k & (ng - 1)) == j) {
            if (block) {
                sg.part[(threadIdx.x >> 5) * sg.cells + i] += p;
            } else if (MINUS) {
                Cell2<T> u;
                u.s0 = s;
                u.s1 = p;
                U[i] = u;
                if constexpr (P1) an.jm[i] = pj;
            } else {
                const T phin = p + pmv;
                const T df = phin - phio;
                acc_d += df * df;
                acc_n += phin * phin;
                X[i].phi = phin;
                if (keep_df) U[i].s0 = df;
                if constexpr (P1) an.jc[i] = pj + an.jm[i];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < A; ++q)
        psi_out[q] = __shfl_sync(0xffffffffu, psi[q].val(), ((nt - 1) << lg) + j);
}

// Out-of-group source of group g: z = ext/2 + sum_{g' != g} ss(g'->g)/2 phi_g'.
template <typename T>
__device__ void group_source(const Sn1dArgs& a, const Grp& gr, long long off, int I, int g) {
    Cell4<T>* X = (Cell4<T>*)a.X;
    const T* S = (const T*)a.scat;
    const T* E = (const T*)a.ext;
    for (int i = gr.rank; i < I; i += gr.size) {
        const long long c = off + i;
        T z = E[(long long)g * a.C + c];
        for (int gp = 0; gp < a.G; ++gp)
            if (gp != g) z += S[((long long)gp * a.G + g) * a.C + c] * X[(long long)gp * a.C + c].phi;
        X[(long long)g * a.C + c].z = z;
    }
}

// Diffusion synthetic correction of group g after its sweep, on one warp.
// U[i].s0 holds df_i = phi^{l+1/2}_i - phi^l_i.  The edge system (I+1
// edges, factored by sn1d_dsa_factor) has the load b_k = r_{k-1} + r_k with
// r_i = (h/2) Sigma_s,i df_i = h X[i].y df_i.  Both triangular solves are
// affine recurrences along the edges, so the edges are split into 32
// chunks of m, one per lane, and solved in three passes with a shuffle scan
// before each of the last two:
//   1. compose the chunk's forward map y_out = P y_in + Q, keeping fm_k b_k;
//   2. from the scanned entry value run the forward elimination, keeping
//      y_k, and compose the chunk's backward map e_first = P e_in + Q
//      (left to right: Q += (product of the coefficients so far) y_k);
//   3. from the scanned (right to left) entry value run the back
//      substitution, add the cell correction (e_k + e_{k+1}) / 2 to phi and
//      form the change df + correction for the norms.
// The one work value per edge (fm b, then y) lives in shared memory where it
// fits (the staging slab, free between sweeps), else in global memory, with
// a row pitch of 33 (lane t's j-th edge at j * 33 + t: conflict-free).
// Each pass loads DSA_BATCH edges before their dependent arithmetic.  A
// reflective right face's stored outflow (the next sweep's inflow) receives
// e_I / 2.
#define DSA_BATCH 8
template <typename T>
__device__ void dsa_pass(const Sn1dArgs& a, const Stage<T>& sg, int inst, int g, long long off,
                         int I, int h, T& acc_d, T& acc_n) {
    const int lane = threadIdx.x & 31;
    Cell4<T>* X = (Cell4<T>*)a.X + (long long)g * a.C + off;
    Cell2<T>* U = (Cell2<T>*)a.U + off;
    const int E = I + 1;
    const int m = (E + 31) / 32;
    const int k0 = lane * m;
    const int n = max(0, min(m, E - k0));
    // this lane's factors, lane-interleaved: F[j * 32] is edge k0 + j
    const DsaEdge<T>* F = (const DsaEdge<T>*)a.dsaf + (long long)g * (a.C + 32LL * a.n_inst) +
                          off + 32LL * inst + lane;
    T* W = (sg.scratch && 33 * m <= sg.scratch_words)
               ? sg.scratch
               : (T*)a.dsaw + 2 * (off + 32LL * inst);
    T* Wl = W + lane;   // Wl[j * 33]: edge k0 + j
    const T hx = (T)a.dx[inst];
    // the previous lane's last edge: its off-diagonal entry and its cell's r
    T o_in = T(0), r_in = T(0);
    if (n > 0 && k0 > 0) {
        o_in = F[(m - 1) * 32 - 1].o;
        r_in = hx * X[k0 - 1].y * U[k0 - 1].s0;
    }
    // 1. forward map of the chunk
    T P = T(1), Q = T(0), rprev = r_in, oprev = o_in;
#pragma unroll 1
    for (int jb = 0; jb < n; jb += DSA_BATCH) {
        T fm[DSA_BATCH], o[DSA_BATCH], r[DSA_BATCH];
#pragma unroll
        for (int q = 0; q < DSA_BATCH; ++q) {
            const int j = jb + q;
            fm[q] = T(0);
            o[q] = T(0);
            r[q] = T(0);
            if (j < n) {
                const DsaEdge<T> f = F[j * 32];
                fm[q] = f.fm;
                o[q] = f.o;
                if (k0 + j < I) r[q] = hx * X[k0 + j].y * U[k0 + j].s0;
            }
        }
#pragma unroll
        for (int q = 0; q < DSA_BATCH; ++q) {
            if (jb + q < n) {
                const T fa = -oprev * fm[q];
                const T beta = fm[q] * (rprev + r[q]);
                Wl[(jb + q) * 33] = beta;
                Q = fa * Q + beta;
                P = fa * P;
                rprev = r[q];
                oprev = o[q];
            }
        }
    }
    for (int d = 1; d < 32; d <<= 1) {
        const T Po = __shfl_up_sync(0xffffffffu, P, d);
        const T Qo = __shfl_up_sync(0xffffffffu, Q, d);
        if (lane >= d) {
            Q = P * Qo + Q;
            P = P * Po;
        }
    }
    T y = __shfl_up_sync(0xffffffffu, Q, 1);
    if (lane == 0) y = T(0);
    // 2. forward elimination and the backward map of the chunk
    T Pb = T(1), Qb = T(0);
    oprev = o_in;
#pragma unroll 1
    for (int jb = 0; jb < n; jb += DSA_BATCH) {
        T fm[DSA_BATCH], o[DSA_BATCH], be[DSA_BATCH];
#pragma unroll
        for (int q = 0; q < DSA_BATCH; ++q) {
            const int j = jb + q;
            fm[q] = T(0);
            o[q] = T(0);
            be[q] = T(0);
            if (j < n) {
                const DsaEdge<T> f = F[j * 32];
                fm[q] = f.fm;
                o[q] = f.o;
                be[q] = Wl[j * 33];
            }
        }
#pragma unroll
        for (int q = 0; q < DSA_BATCH; ++q) {
            if (jb + q < n) {
                y = -oprev * fm[q] * y + be[q];
                Wl[(jb + q) * 33] = y;
                Qb = Pb * y + Qb;
                Pb = -o[q] * fm[q] * Pb;
                oprev = o[q];
            }
        }
    }
    for (int d = 1; d < 32; d <<= 1) {
        const T Pn = __shfl_down_sync(0xffffffffu, Pb, d);
        const T Qn = __shfl_down_sync(0xffffffffu, Qb, d);
        if (lane + d < 32) {
            Qb = Pb * Qn + Qb;
            Pb = Pb * Pn;
        }
    }
    T en = __shfl_down_sync(0xffffffffu, Qb, 1);
    if (lane == 31) en = T(0);
    // 3. back substitution and the correction of the cells, right to left
    T e_last = T(0);
#pragma unroll 1
    for (int jt = n - 1; jt >= 0; jt -= DSA_BATCH) {
        T bc[DSA_BATCH], yy[DSA_BATCH], ph[DSA_BATCH], df[DSA_BATCH];
#pragma unroll
        for (int q = 0; q < DSA_BATCH; ++q) {
            const int j = jt - q;
            bc[q] = T(0);
            yy[q] = T(0);
            ph[q] = T(0);
            df[q] = T(0);
            if (j >= 0) {
                const DsaEdge<T> f = F[j * 32];
                bc[q] = -f.o * f.fm;
                yy[q] = Wl[j * 33];
                if (k0 + j < I) {
                    ph[q] = X[k0 + j].phi;
                    df[q] = U[k0 + j].s0;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < DSA_BATCH; ++q) {
            const int k = k0 + jt - q;
            if (jt - q >= 0) {
                const T e = bc[q] * en + yy[q];
                if (k == I) e_last = e;
                if (k < I) {
                    const T fc = T(0.5) * (e + en);
                    const T pn = ph[q] + fc;
                    X[k].phi = pn;
                    const T ch = df[q] + fc;
                    acc_d += ch * ch;
                    acc_n += pn * pn;
                }
                en = e;
            }
        }
    }
    if (a.bc_right) {
        const T eI = __shfl_sync(0xffffffffu, e_last, I / m);
        T* PB = (T*)a.psib + a.boff[inst];
        for (int hi = lane; hi < h; hi += 32) PB[(g * h + hi) * 2 + 1] += T(0.5) * eI;
    }
    __syncwarp();
}

// One source iteration over all groups; returns the relative L2 change.
// [hb, he): this warp's slice of the half-angle range (all of it on the warp
// path).
template <typename T, int A, bool P1>
__device__ double si_iteration(const Sn1dArgs& a, const Grp& gr, const Stage<T>& sg, int inst,
                               long long off, int I, int h, int hb, int he, int lg,
                               const T (&cc)[A], const T (&wt)[A], P1Op<T, A>& an) {
    const int lane = threadIdx.x & 31;
    const int j = lane & ((1 << lg) - 1);
    T* PB = (T*)a.psib + a.boff[inst];
    T acc_d = T(0), acc_n = T(0);
    for (int g = 0; g < a.G; ++g) {
        const T keep_d = acc_d, keep_n = acc_n;
        if (a.G > 1) {
            group_source<T>(a, gr, off, I, g);
            gr.sync();
        }
        Cell4<T>* X = (Cell4<T>*)a.X + (long long)g * a.C + off;
        Cell2<T>* U = (Cell2<T>*)a.U + off;
        if constexpr (P1) {
            // s1 = (3/2) Sigma_s1 J from the current of the previous iteration
            const T* Y1 = (const T*)a.y1 + (long long)g * a.C + off;
            T* S1 = (T*)a.s1buf + off;
            an.jc = (T*)a.cur + (long long)g * a.C + off;
            an.s1 = S1;
            an.jm = (T*)a.jm + off;
            for (int i = gr.rank; i < I; i += gr.size) S1[i] = Y1[i] * an.jc[i];
            gr.sync();
        }
        if (sg.ss) {
            for (int i = gr.rank; i < I; i += gr.size) {
                const Cell4<T> v = X[i];
                Cell2<T> w2;
                w2.s0 = v.st;
                w2.s1 = v.y * v.phi + v.z;
                sg.ss[i] = w2;
                if (gr.block)
                    for (int w = 0; w < gr.nwarps; ++w) sg.part[w * sg.cells + i] = T(0);
            }
            gr.sync();
        }
        T bnd[A], out[A];
        // mu < 0 enters at x = L: vacuum, or the mirror's latest outgoing flux
#pragma unroll
        for (int q = 0; q < A; ++q) {
            const int hi = hb + j * A + q;
            bnd[q] = (a.bc_right && hi < he) ? PB[(g * h + hi) * 2 + 1] : T(0);
        }
        // on the block path a warp without angles (fewer angles than warps)
        // only joins the barriers
        if (hb < he) {
            sweep_half<T, A, true, P1>(gr.block, X, U, sg, I, lg, cc, wt, bnd, out, acc_d, acc_n,
                                       an, false);
            __syncwarp();
#pragma unroll
            for (int q = 0; q < A; ++q) {
                const int hi = hb + j * A + q;
                if (hi < he && (lane >> lg) == 0) PB[(g * h + hi) * 2 + 0] = out[q];
                bnd[q] = a.bc_left ? out[q] : T(0);
            }
            sweep_half<T, A, false, P1>(gr.block, X, U, sg, I, lg, cc, wt, bnd, out, acc_d, acc_n,
                                        an, a.dsa != 0);
#pragma unroll
            for (int q = 0; q < A; ++q) {
                const int hi = hb + j * A + q;
                if (hi < he && (lane >> lg) == 0) PB[(g * h + hi) * 2 + 1] = out[q];
            }
        }
        gr.sync();
        if (gr.block) {
            for (int i = gr.rank; i < I; i += gr.size) {
                T phin = T(0);
                for (int w = 0; w < gr.nwarps; ++w) phin += sg.part[w * sg.cells + i];
                const T df = phin - X[i].phi;
                acc_d += df * df;
                acc_n += phin * phin;
                X[i].phi = phin;
                if (a.dsa) U[i].s0 = df;
            }
            gr.sync();
        }
        if (a.dsa) {
            // the change of this group is that of the corrected flux
            acc_d = keep_d;
            acc_n = keep_n;
            if (!gr.block || gr.warp == 0)
                dsa_pass<T>(a, sg, inst, g, off, I, h, acc_d, acc_n);
            gr.sync();
        }
    }
    const double sd = gr.sum((double)acc_d);
    const double sn = gr.sum((double)acc_n);
    return sn > 0.0 ? sqrt(sd / sn) : (sd > 0.0 ? INFINITY : 0.0);
}

// ------------------------------------------------------------ direct lanes
// Direct-lane sweep of slabs with vacuum faces and isotropic scattering: the
// two direction halves are independent within a source iteration (each sees
// vacuum inflow and the emission of the previous iterate), so they run at
// the same time.  Lanes 0-15 carry mu < 0 (cells right to left), lanes 16-31
// mu > 0 (left to right); lane j of a half carries the half-angles
// j, j + 16, ..., A of them.  On one warp every lane walks the whole slab: no
// chunk maps and no scan, so each cell-angle update is one pass of the
// compensated diamond-difference increment.  A team of W warps (a whole
// block) splits the cells into W chunks, composes each chunk's affine map
// psi_out = (1 - D) psi_in + B per chain, and hands the entry fluxes across
// chunks through shared memory before the sweep.
//
// Cells stream through a double-buffered ring of R = 32 staged {sigma_t, s}
// pairs per direction (s = emission of the current iterate), loaded one
// block of R cells ahead with coalesced 16-byte loads.  The step loop is
// software-pipelined: the staged operands and the reciprocal of step k + 1
// are formed during step k, so a step's dependent chain is the flux update
// alone.  The angle sums go through a second ring: at step k lane l stores
// its partial sum in row l, slot k mod R (row pitch R + 1: no bank
// conflicts), and every R steps lane l adds the 16 rows of each half for
// slot l.  Step k reaches cell c0 + k going right and c0 + len - 1 - k going
// left, so a cell is reached twice; the half sum that arrives first waits
// in a pair buffer (shared memory, or the instance's U cells when the chunk
// is long), and the second arrival completes the cell: new flux, change and
// norm terms (the old flux comes from the staging load of the same cell).
constexpr int DR = 32;   // ring length (cells per staged block)
constexpr int DSLAB = SN1D_STAGE_BYTES / (SN1D_THREADS / 32);   // shared bytes per warp

// Per-warp shared-memory layout of the direct path inside the warp's slab:
// staging ring, partial-sum ring, chunk maps (team path), pair buffer.
template <typename T>
struct DirectSmem {
    Cell2<T>* stg;   // [2 dir][2 buf][DR + 2]
    T* red;          // [32][DR + 1]
    T* maps;         // [32 lanes][4][2] chunk maps (team path)
    Cell2<T>* pair;  // first-arrival half sums {mu > 0, mu < 0}
    int pair_cap;    // entries of pair
    __device__ static DirectSmem at(unsigned char* slab) {
        DirectSmem s;
        s.stg = (Cell2<T>*)slab;
        s.red = (T*)(slab + 4 * (DR + 2) * sizeof(Cell2<T>));
        s.maps = s.red + 32 * (DR + 1);
        s.pair = (Cell2<T>*)(s.maps + 32 * 4 * 2);
        s.pair_cap = (int)((slab + DSLAB - (unsigned char*)s.pair) / sizeof(Cell2<T>));
        return s;
    }
};

// Loads the X entries of the two cells lane l stages for block kb of the
// chunk [c0, c0 + len): mu > 0 reads c0 + kb R + l, mu < 0 reads
// c0 + len - 1 - (kb R + l).
template <typename T>
__device__ __forceinline__ void direct_fetch(const Cell4<T>* X, int c0, int len, int kb, int l,
                                             Cell4<T>& vp, Cell4<T>& vm) {
    const int k = kb * DR + l;
    if (k < len) {
        vp = X[c0 + k];
        vm = X[c0 + len - 1 - k];
    }
}

// Stages the fetched cells into buffer `buf` and keeps their old fluxes.
template <typename T>
__device__ __forceinline__ void direct_stage(const DirectSmem<T>& sm, int buf, int l,
                                             const Cell4<T>& vp, const Cell4<T>& vm, T& php,
                                             T& phm) {
    Cell2<T> p, m;
    p.s0 = vp.st;
    p.s1 = vp.y * vp.phi + vp.z;
    m.s0 = vm.st;
    m.s1 = vm.y * vm.phi + vm.z;
    if constexpr (sizeof(T) == 4) {
        // FP32 stages {-2 sigma_t, 2 s} (exact scalings; see direct_steps_f32)
        p.s0 *= T(-2);
        p.s1 *= T(2);
        m.s0 *= T(-2);
        m.s1 *= T(2);
    }
    sm.stg[(2 + buf) * (DR + 2) + l] = p;   // mu > 0 rows: 2, 3
    sm.stg[buf * (DR + 2) + l] = m;         // mu < 0 rows: 0, 1
    php = vp.phi;
    phm = vm.phi;
}

// ---- FP32 steps of the direct lanes.  The staged operands are scaled so
// that each product the recurrence needs is one rounding of exactly twice the
// unscaled value (scaling by 2 commutes with rounding): with S0 = -2 sigma_t
// and S1 = 2 s,
//     x = fma(S0, psi, S1) = 2 (s - sigma_t psi),   d = r x = 2 dl,
//     psi_c = fma(1/2, d, psi) = psi + dl,          c + sigma_t = fma(-1/2, S0, c),
// and the chunk map's D <- D + 2 r sigma_t (1 - D) is fma(r S0, D - 1, D).
// Two angles of a lane go through one instruction as a packed pair
// (__ffma2_rn, __fmul2_rn, __fadd2_rn: sm_100 and later); the compensated sum
// of psi is the same Fast2Sum as CSum, on pairs.
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

// The direct lanes take the hardware reciprocal as it is (rcp.approx.ftz:
// within 1 ulp), one rounding more in the update's factor r and no Newton
// step.  The reciprocal of a cell and angle is the same in every iteration,
// so it adds no iteration-to-iteration noise to the stopping test; any bias
// it has moves the fixed point by about the bias over (1 - spectral radius),
// which on the workloads' slabs stays at the 1e-7 level of the FP32 sweep
// (flux 1.6e-7, k 1.1e-7 against the FP64 oracle on the three-region eigen
// slab, the same as with the Newton step).
__device__ __forceinline__ float rcp_fast(float d) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return r;
}

__device__ __forceinline__ float2 rcp2(float2 d) { return make_float2(rcp_fast(d.x), rcp_fast(d.y)); }

// P packed pairs of chains over the nk staged steps of `cur` (COMPOSE: chunk
// maps; otherwise flux partial sums into myred[k]).  r0 holds the reciprocals
// of step 0 on entry.
template <int P, bool COMPOSE>
__device__ __forceinline__ void direct_steps_f32x2(const Cell2<float>* cur, int nk, float* myred,
                                                   const float2 (&c2)[P], const float2 (&w2)[P],
                                                   float2 (&h2)[P], float2 (&l2)[P],
                                                   float2 (&D2)[P], float2 (&r0)[P]) {
    Cell2<float> v1 = cur[1];
    float S0 = cur[0].s0, S1 = cur[0].s1;
#pragma unroll 4
    for (int k = 0; k < nk; ++k) {
        float2 r[P];
#pragma unroll
        for (int j = 0; j < P; ++j) r[j] = r0[j];
        const Cell2<float> v2 = cur[k + 2];
#pragma unroll
        for (int j = 0; j < P; ++j) r0[j] = rcp2(__ffma2_rn(f2(-0.5f), f2(v1.s0), c2[j]));
        float2 pa = f2(0.0f);
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const float2 x = __ffma2_rn(f2(S0), h2[j], f2(S1));
            const float2 d = __fmul2_rn(r[j], x);
            if constexpr (COMPOSE) {
                const float2 g = __fmul2_rn(r[j], f2(S0));
                D2[j] = __ffma2_rn(g, __fadd2_rn(D2[j], f2(-1.0f)), D2[j]);
            } else {
                const float2 pc = __ffma2_rn(f2(0.5f), d, h2[j]);
                pa = j == 0 ? __fmul2_rn(w2[j], pc) : __ffma2_rn(w2[j], pc, pa);
            }
            const float2 u = __fadd2_rn(d, l2[j]);
            const float2 t = __fadd2_rn(h2[j], u);
            const float2 y = __ffma2_rn(h2[j], f2(-1.0f), t);   // t - psi (exact)
            l2[j] = __ffma2_rn(y, f2(-1.0f), u);
            h2[j] = t;
        }
        if constexpr (!COMPOSE) myred[k] = pa.x + pa.y;
        S0 = v1.s0;
        S1 = v1.s1;
        v1 = v2;
    }
}

// The same for one chain per lane (A = 1), unpacked.
template <bool COMPOSE>
__device__ __forceinline__ void direct_steps_f32(const Cell2<float>* cur, int nk, float* myred,
                                                 float c, float w, float& h, float& l, float& D,
                                                 float& r0) {
    Cell2<float> v1 = cur[1];
    float S0 = cur[0].s0, S1 = cur[0].s1;
#pragma unroll 4
    for (int k = 0; k < nk; ++k) {
        const float r = r0;
        const Cell2<float> v2 = cur[k + 2];
        r0 = rcp_fast(fmaf(-0.5f, v1.s0, c));
        const float x = fmaf(S0, h, S1);
        const float d = r * x;
        if constexpr (COMPOSE) {
            D = fmaf(r * S0, D - 1.0f, D);
        } else {
            myred[k] = w * fmaf(0.5f, d, h);
        }
        const float u = d + l;
        const float t = h + u;
        l = u - (t - h);
        h = t;
        S0 = v1.s0;
        S1 = v1.s1;
        v1 = v2;
    }
}

// One pass over this warp's chunk [c0, c0 + len) for all its chains.
// COMPOSE: build the chunk map (D, B) of every chain.  Otherwise sweep from
// psi_in, complete every cell of the chunk (new flux into X, change and
// norm terms into acc_d, acc_n).
template <typename T, int A, bool COMPOSE>
__device__ __forceinline__ void direct_pass(const DirectSmem<T>& sm, Cell4<T>* X, Cell2<T>* U,
                                            int c0, int len, const T (&cc)[A], const T (&wt)[A],
                                            CSum<T> (&psi)[A], T (&D)[A], T& acc_d, T& acc_n) {
    const int lane = threadIdx.x & 31;
    const int half = lane >> 4;   // 0: mu < 0, 1: mu > 0
    Cell2<T>* pair = ((len + 1) / 2 <= sm.pair_cap) ? sm.pair : U + c0;
    Cell4<T> vp{}, vm{};
    T php = T(0), phm = T(0);
    direct_fetch<T>(X, c0, len, 0, lane, vp, vm);
    direct_stage<T>(sm, 0, lane, vp, vm, php, phm);
    __syncwarp();
    const int nblk = (len + DR - 1) / DR;
    const Cell2<T>* row = sm.stg + 2 * half * (DR + 2);
    T* myred = sm.red + lane * (DR + 1);
    // FP32 with two or more chains per lane: packed pairs (an odd last chain
    // is paired with an idle one: c = 1, w = 0)
    constexpr int P2 = (A + 1) / 2;
    float2 c2[P2], w2[P2], h2[P2], l2[P2], D2[P2];
    if constexpr (sizeof(T) == 4 && A > 1) {
#pragma unroll
        for (int j = 0; j < P2; ++j) {
            const int q = 2 * j, q1 = 2 * j + 1;
            c2[j] = make_float2((float)cc[q], q1 < A ? (float)cc[q1] : 1.0f);
            w2[j] = make_float2((float)wt[q], q1 < A ? (float)wt[q1] : 0.0f);
            h2[j] = make_float2((float)psi[q].hi, q1 < A ? (float)psi[q1].hi : 0.0f);
            l2[j] = make_float2((float)psi[q].lo, q1 < A ? (float)psi[q1].lo : 0.0f);
            D2[j] = make_float2((float)D[q], q1 < A ? (float)D[q1] : 0.0f);
        }
    }
#pragma unroll 1
    for (int kb = 0; kb < nblk; ++kb) {
        // the next block's cells, in flight during this block's steps
        direct_fetch<T>(X, c0, len, kb + 1, lane, vp, vm);
        const int nk = min(DR, len - kb * DR);
        const Cell2<T>* cur = row + (kb & 1) * (DR + 2);
        // two-deep pipeline: step k loads the operands of step k + 2 and
        // forms the reciprocals of step k + 1 (slots DR, DR + 1 are padding);
        // four steps per loop trip in FP32 (two in FP64), so the independent
        // work of consecutive steps (operands, reciprocals, angle sums)
        // interleaves with the flux chain
        if constexpr (sizeof(T) == 4 && A == 1) {
            float rr = rcp_fast(fmaf(-0.5f, cur[0].s0, cc[0]));
            direct_steps_f32<COMPOSE>((const Cell2<float>*)cur, nk, (float*)myred, cc[0], wt[0],
                                      psi[0].hi, psi[0].lo, D[0], rr);
        } else if constexpr (sizeof(T) == 4) {
            float2 rr[P2];
#pragma unroll
            for (int j = 0; j < P2; ++j) rr[j] = rcp2(__ffma2_rn(f2(-0.5f), f2(cur[0].s0), c2[j]));
            direct_steps_f32x2<P2, COMPOSE>((const Cell2<float>*)cur, nk, (float*)myred, c2, w2,
                                            h2, l2, D2, rr);
        } else {
        Cell2<T> v0 = cur[0], v1 = cur[1];
        T r0[A];
#pragma unroll
        for (int q = 0; q < A; ++q) r0[q] = rcp_dd(cc[q] + v0.s0);
#pragma unroll 2
        for (int k = 0; k < nk; ++k) {
            const T st = v0.s0, s = v0.s1;
            T r[A];
#pragma unroll
            for (int q = 0; q < A; ++q) r[q] = r0[q];
            const Cell2<T> v2 = cur[k + 2];
#pragma unroll
            for (int q = 0; q < A; ++q) r0[q] = rcp_dd(cc[q] + v1.s0);
            v0 = v1;
            v1 = v2;
            if constexpr (COMPOSE) {
#pragma unroll
                for (int q = 0; q < A; ++q) {
                    const T r2 = T(2) * r[q];
                    D[q] = (r2 * st) * (T(1) - D[q]) + D[q];
                    psi[q].add(r2 * (s - st * psi[q].hi));
                }
            } else {
                T p = T(0);
#pragma unroll
                for (int q = 0; q < A; ++q) {
                    const T dl = r[q] * (s - st * psi[q].hi);
                    p += wt[q] * (psi[q].hi + (dl + psi[q].lo));
                    psi[q].add(dl + dl);
                }
                myred[k] = p;
            }
        }
        }
        __syncwarp();
        if constexpr (!COMPOSE) {
            // slot `lane` of this block: step k reaches cell c0 + k (mu > 0)
            // and cell c0 + len - 1 - k (mu < 0)
            const int k = kb * DR + lane;
            const bool valid = lane < nk;
            const int twice = 2 * k - (len - 1);   // < 0 first arrival, > 0 second, 0 middle
            T sp = T(0), sn = T(0);
            if (valid) {
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    sn += sm.red[r * (DR + 1) + lane];
                    sp += sm.red[(16 + r) * (DR + 1) + lane];
                }
                if (twice < 0) {
                    Cell2<T> fp;
                    fp.s0 = sp;
                    fp.s1 = sn;
                    pair[k] = fp;
                }
            }
            __syncwarp();
            if (valid && twice >= 0) {
                T fpn, fmn;
                if (twice == 0) {
                    fpn = sp + sn;
                    fmn = fpn;
                } else {
                    const Cell2<T> o = pair[len - 1 - k];
                    fpn = sp + o.s1;
                    fmn = sn + o.s0;
                }
                const T dp = fpn - php;
                acc_d += dp * dp;
                acc_n += fpn * fpn;
                X[c0 + k].phi = fpn;
                if (twice > 0) {
                    const T dm = fmn - phm;
                    acc_d += dm * dm;
                    acc_n += fmn * fmn;
                    X[c0 + len - 1 - k].phi = fmn;
                }
            }
        }
        if (kb + 1 < nblk) direct_stage<T>(sm, (kb + 1) & 1, lane, vp, vm, php, phm);
        __syncwarp();
    }
    if constexpr (sizeof(T) == 4 && A > 1) {
#pragma unroll
        for (int j = 0; j < P2; ++j) {
            const int q = 2 * j, q1 = 2 * j + 1;
            psi[q].hi = h2[j].x;
            psi[q].lo = l2[j].x;
            D[q] = D2[j].x;
            if (q1 < A) {
                psi[q1].hi = h2[j].y;
                psi[q1].lo = l2[j].y;
                D[q1] = D2[j].y;
            }
        }
    }
}

// One source iteration over all groups on the direct lanes; returns the
// relative L2 change.  Team path (gr.block): warp w owns cells
// [w m, min(I, (w + 1) m)), m = ceil(I / W).
template <typename T, int A>
__device__ double si_iteration_direct(const Sn1dArgs& a, const Grp& gr, unsigned char* smem,
                                      long long off, int I, const T (&cc)[A],
                                      const T (&wt)[A]) {
    const int lane = threadIdx.x & 31;
    const int half = lane >> 4;
    const int W = gr.block ? gr.nwarps : 1;
    const int w = gr.block ? gr.warp : 0;
    const int m = (I + W - 1) / W;
    const int c0 = min(I, w * m);
    const int len = max(0, min(I, c0 + m) - c0);
    // every warp works in its own slab of the block's shared memory (on the
    // team path warp w of the block is chunk w)
    const DirectSmem<T> sm = DirectSmem<T>::at(smem + (threadIdx.x >> 5) * DSLAB);
    T acc_d = T(0), acc_n = T(0);
    for (int g = 0; g < a.G; ++g) {
        if (a.G > 1) {
            group_source<T>(a, gr, off, I, g);
            gr.sync();
        }
        Cell4<T>* X = (Cell4<T>*)a.X + (long long)g * a.C + off;
        Cell2<T>* U = (Cell2<T>*)a.U + off;
        CSum<T> psi[A];
        T D[A];
#pragma unroll
        for (int q = 0; q < A; ++q) {
            psi[q].set(T(0));
            D[q] = T(0);
        }
        if (W > 1) {
            // chunk maps, then the entry flux of every chain: vacuum at the
            // face, then the maps of the chunks upstream in sweep order
            direct_pass<T, A, true>(sm, X, U, c0, len, cc, wt, psi, D, acc_d, acc_n);
#pragma unroll
            for (int q = 0; q < A; ++q) {
                sm.maps[(lane * 4 + q) * 2 + 0] = D[q];
                sm.maps[(lane * 4 + q) * 2 + 1] = psi[q].val();
            }
            gr.sync();
            T in[A];
#pragma unroll
            for (int q = 0; q < A; ++q) in[q] = T(0);
            for (int u = 0; u < W - 1; ++u) {
                // mu > 0: chunks 0 .. w-1 in order; mu < 0: chunks W-1 .. w+1
                const int wu = half ? u : W - 1 - u;
                if (half ? (wu < w) : (wu > w)) {
                    const DirectSmem<T> su = DirectSmem<T>::at(smem + wu * DSLAB);
#pragma unroll
                    for (int q = 0; q < A; ++q) {
                        const T Du = su.maps[(lane * 4 + q) * 2 + 0];
                        const T Bu = su.maps[(lane * 4 + q) * 2 + 1];
                        in[q] = (in[q] + Bu) - Du * in[q];
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < A; ++q) psi[q].set(in[q]);
        }
        direct_pass<T, A, false>(sm, X, U, c0, len, cc, wt, psi, D, acc_d, acc_n);
        // the next group's source (and the next iteration's staging) reads
        // the fluxes of the whole instance
        gr.sync();
    }
    const double sd = gr.sum((double)acc_d);
    const double sn = gr.sum((double)acc_n);
    return sn > 0.0 ? sqrt(sd / sn) : (sd > 0.0 ? INFINITY : 0.0);
}

// production integral sum nsf * phi * dx over the instance (FP64)
template <typename T>
__device__ double production(const Sn1dArgs& a, const Grp& gr, long long off, int I, double dx) {
    const Cell4<T>* X = (const Cell4<T>*)a.X;
    const T* F = (const T*)a.nsf;
    double acc = 0.0;
    for (int g = 0; g < a.G; ++g)
        for (int i = gr.rank; i < I; i += gr.size) {
            const long long c = (long long)g * a.C + off + i;
            acc += (double)F[c] * (double)X[c].phi;
        }
    return gr.sum(acc) * dx;
}

template <typename T, int A, bool P1, bool DIRECT = false>
__device__ void solve_instance(const Sn1dArgs& a, const Grp& gr, const Stage<T>& sg, int inst,
                               int lg, unsigned char* smem = nullptr) {
    const int lane = threadIdx.x & 31;
    const int j = lane & ((1 << lg) - 1);
    const int I = a.ncell[inst];
    const int N = a.nang[inst];
    const int h = N / 2;
    const double dxv = a.dx[inst];
    const long long off = a.cell_off[inst];
    const int q0 = a.qoff[inst];
    // this warp's slice of the half-angle range
    const int hw = gr.block ? (h + gr.nwarps - 1) / gr.nwarps : h;
    const int hb = gr.block ? min(h, gr.warp * hw) : 0;
    const int he = gr.block ? min(h, hb + hw) : h;
    unsigned long long t_start = 0;
    if (a.trace && gr.rank == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
    T cc[A], wt[A];
    P1Op<T, A> an{};
#pragma unroll
    for (int q = 0; q < A; ++q) {
        // direct lanes: lane j of each half carries half-angles j, j + 16, ...
        const int hi = DIRECT ? (lane & 15) + 16 * q : hb + j * A + q;
        if (hi < (DIRECT ? h : he)) {
            cc[q] = (T)(2.0 * a.mu[q0 + h + hi] / dxv);
            wt[q] = (T)a.w[q0 + h + hi];
            an.mua[q] = (T)a.mu[q0 + h + hi];
            an.wmu[q] = (T)(a.w[q0 + h + hi] * a.mu[q0 + h + hi]);
        } else {
            cc[q] = T(1);
            wt[q] = T(0);
            an.mua[q] = T(0);
            an.wmu[q] = T(0);
        }
    }
    T* PB = (T*)a.psib + a.boff[inst];
    for (int e = gr.rank; e < a.G * N; e += gr.size) PB[e] = T(0);
    gr.sync();

    int status = NOP_OK;
    double change = 0.0;
    int its = 0, n = 0;
    double k = 0.0, dphi = INFINITY;
    auto iterate = [&]() -> double {
        if constexpr (DIRECT) return si_iteration_direct<T, A>(a, gr, smem, off, I, cc, wt);
        else return si_iteration<T, A, P1>(a, gr, sg, inst, off, I, h, hb, he, lg, cc, wt, an);
    };
    if (!a.eigen) {
        for (its = 1; its <= a.itmax; ++its) {
            change = iterate();
            if (!isfinite(change)) {
                status = NOP_ENAN;
                break;
            }
            if (change <= a.tol) break;
        }
        if (its > a.itmax) {
            its = a.itmax;
            status = NOP_ENOCONV;
        }
        dphi = change;
    } else {
        // ---- power iteration (App. A2): flux normalised to unit production
        Cell4<T>* X = (Cell4<T>*)a.X;
        T* PP = (T*)a.phiprev;
        const T* F = (const T*)a.nsf;
        T* E = (T*)a.ext;
        k = a.k0[inst];
        double P = production<T>(a, gr, off, I, dxv);
        if (!(P > 0.0) || !isfinite(P)) status = NOP_ENAN;
        if (status == NOP_OK) {
            const T sc = (T)(1.0 / P);
            for (int g = 0; g < a.G; ++g)
                for (int i = gr.rank; i < I; i += gr.size) X[(long long)g * a.C + off + i].phi *= sc;
        }
        gr.sync();
        double dk = INFINITY;
        for (n = 1; n <= a.itmax && status == NOP_OK; ++n) {
            // frozen fission source chi_g F / k (halved) and the previous flux
            for (int i = gr.rank; i < I; i += gr.size) {
                double Fi = 0.0;
                for (int g = 0; g < a.G; ++g) {
                    const long long c = (long long)g * a.C + off + i;
                    Fi += (double)F[c] * (double)X[c].phi;
                    PP[c] = X[c].phi;
                }
                for (int g = 0; g < a.G; ++g) {
                    const long long c = (long long)g * a.C + off + i;
                    const T e = (T)(0.5 * a.chi[g] * Fi / k);
                    E[c] = e;
                    if (a.G == 1) X[c].z = e;
                }
            }
            gr.sync();
            int it;
            for (it = 1; it <= a.itmax_inner; ++it) {
                change = iterate();
                if (!isfinite(change)) {
                    status = NOP_ENAN;
                    break;
                }
                if (change <= a.tol_inner) break;
            }
            its += min(it, a.itmax_inner);
            if (status != NOP_OK) break;
            P = production<T>(a, gr, off, I, dxv);
            if (!(P > 0.0) || !isfinite(P)) {
                status = NOP_ENAN;
                break;
            }
            const double kn = k * P;
            const T sc = (T)(1.0 / P);
            double d2 = 0.0, n2 = 0.0;
            for (int g = 0; g < a.G; ++g)
                for (int i = gr.rank; i < I; i += gr.size) {
                    const long long c = (long long)g * a.C + off + i;
                    const T v = X[c].phi * sc;
                    X[c].phi = v;
                    const double df = (double)v - (double)PP[c];
                    d2 += df * df;
                    n2 += (double)v * (double)v;
                }
            gr.sync();
            for (int e = gr.rank; e < a.G * N; e += gr.size) PB[e] *= sc;
            d2 = gr.sum(d2);
            n2 = gr.sum(n2);
            dphi = n2 > 0 ? sqrt(d2 / n2) : 0.0;
            dk = fabs(kn - k) / fabs(kn);
            k = kn;
            if (dk <= a.tol_k && dphi <= a.tol) break;
        }
        if (status == NOP_OK && n > a.itmax) {
            n = a.itmax;
            status = NOP_ENOCONV;
        }
    }
    if (gr.rank == 0) {
        a.it_out[inst] = its;
        a.st_out[inst] = status;
        a.ch_out[inst] = dphi;
        if (a.eigen) {
            a.k_out[inst] = k;
            a.outer_out[inst] = n;
        }
        if (a.trace) {
            unsigned long long t_end;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
            unsigned int smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            a.trace[3 * (long long)inst + 0] = t_start;
            a.trace[3 * (long long)inst + 1] = t_end;
            a.trace[3 * (long long)inst + 2] = smid | (gr.block ? 0x80000000ull : 0ull);
        }
    }
    gr.sync();
}

// cfg of an instance: (log2 ng) << 8 | A for the chunked lanes, or
// SN1D_DIRECT | A for the direct lanes (A in 1..4)
#define SN1D_DIRECT 0x10000
template <typename T>
__device__ __forceinline__ void dispatch(const Sn1dArgs& a, const Grp& gr, const Stage<T>& sg,
                                         int inst, unsigned char* smem) {
    const int cfg = a.cfg[inst];
    if (cfg & SN1D_DIRECT) {
        switch (cfg & 0xff) {
            case 1: solve_instance<T, 1, false, true>(a, gr, sg, inst, 0, smem); break;
            case 2: solve_instance<T, 2, false, true>(a, gr, sg, inst, 0, smem); break;
            case 3: solve_instance<T, 3, false, true>(a, gr, sg, inst, 0, smem); break;
            default: solve_instance<T, 4, false, true>(a, gr, sg, inst, 0, smem); break;
        }
        return;
    }
    const int A = cfg & 0xff, lg = cfg >> 8;
    // anisotropic instances take A in {1, 2, 4} only (the host picks so)
    switch (A) {
        case 1:
            if (a.p1 && !gr.block) solve_instance<T, 1, true>(a, gr, sg, inst, lg);
            else solve_instance<T, 1, false>(a, gr, sg, inst, lg);
            break;
        case 2:
            if (a.p1 && !gr.block) solve_instance<T, 2, true>(a, gr, sg, inst, lg);
            else solve_instance<T, 2, false>(a, gr, sg, inst, lg);
            break;
        // 3, 5 and 6 angles per lane in FP32 only (the FP64 path picks powers
        // of two and keeps the kernel small)
        case 3:
            if constexpr (sizeof(T) == 4) solve_instance<T, 3, false>(a, gr, sg, inst, lg);
            break;
        case 5:
            if constexpr (sizeof(T) == 4) solve_instance<T, 5, false>(a, gr, sg, inst, lg);
            break;
        case 6:
            if constexpr (sizeof(T) == 4) solve_instance<T, 6, false>(a, gr, sg, inst, lg);
            break;
        default:
            if (a.p1 && !gr.block) solve_instance<T, 4, true>(a, gr, sg, inst, lg);
            else solve_instance<T, 4, false>(a, gr, sg, inst, lg);
            break;
    }
}

// Large instances run on a whole block (angles split over its warps), small
// ones on one warp.  Both queues are longest-first work counters.
template <typename T>
__device__ void drain_big(const Sn1dArgs& a, double* red, int* job, unsigned char* smem_raw) {
    // block path: [cells] staged pairs, then one row of partial sums per warp
    Stage<T> sg;
    sg.ss = (Cell2<T>*)smem_raw;
    sg.cells = a.smem_cells;
    sg.part = (T*)(sg.ss + a.smem_cells);
    // between sweeps the whole staging area is free for one warp's correction
    sg.scratch = (T*)smem_raw;
    sg.scratch_words = SN1D_STAGE_BYTES / (int)sizeof(T);
    Grp gb;
    gb.block = true;
    gb.rank = threadIdx.x;
    gb.size = blockDim.x;
    gb.warp = threadIdx.x >> 5;
    gb.nwarps = blockDim.x >> 5;
    gb.red = red;
    for (;;) {
        if (threadIdx.x == 0) *job = atomicAdd(a.counter + 1, 1);
        __syncthreads();
        const int jb = *job;
        __syncthreads();
        if (jb >= a.n_big) break;
        dispatch<T>(a, gb, sg, a.big_list[jb], smem_raw);
    }
    __syncthreads();
}

// Persistent kernel.  Blocks [0, big_blocks) start on the large queue and
// then help with the small one; the other blocks start on the small queue
// (every warp on its own) and then help with what is left of the large one,
// so both kinds run side by side from the start and the tail is shared.
template <typename T>
__global__ void __launch_bounds__(SN1D_THREADS, SN1D_BLOCKS_PER_SM) sn1d_kernel(Sn1dArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[SN1D_THREADS / 32];
    __shared__ int job;
    const int lane = threadIdx.x & 31;
    constexpr int nw = SN1D_THREADS / 32;
    const bool big_first = a.n_big > 0 && (int)blockIdx.x < a.big_blocks;
    if (big_first) drain_big<T>(a, red, &job, smem_raw);
    // warp path: each warp stages into its own slab
    constexpr int slab = SN1D_STAGE_BYTES / (nw * (int)sizeof(Cell2<T>));
    Grp gw;
    gw.block = false;
    gw.rank = lane;
    gw.size = 32;
    gw.warp = 0;
    gw.nwarps = 1;
    gw.red = nullptr;
    for (;;) {
        int jw = 0;
        if (lane == 0) jw = atomicAdd(a.counter, 1);
        jw = __shfl_sync(0xffffffffu, jw, 0);
        if (jw >= a.n_small) break;
        const int inst = a.order_list[jw];
        Stage<T> sw;
        sw.ss = a.ncell[inst] <= slab
                    ? (Cell2<T>*)smem_raw + (threadIdx.x >> 5) * slab
                    : nullptr;
        sw.part = nullptr;
        sw.cells = slab;
        // the warp's slab, free between sweeps, holds its correction's work values
        sw.scratch = (T*)((Cell2<T>*)smem_raw + (threadIdx.x >> 5) * slab);
        sw.scratch_words = slab * 2;
        dispatch<T>(a, gw, sw, inst, smem_raw);
    }
    if (a.n_big > 0 && !big_first) {
        __syncthreads();
        drain_big<T>(a, red, &job, smem_raw);
    }
}

// ---------------------------------------------------------------- set-up
template <typename T>
__global__ void sn1d_prepare(long long C, int G, const double* sigt, const double* sigs,
                             const double* src, const double* nsf, const double* phi0,
                             int phi0_flat, Cell4<T>* X, T* scat, T* ext, T* nsfT,
                             const double* sigs1, T* y1, T* cur) {
    const long long total = (long long)G * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(e / C);
        const long long c = e - (long long)g * C;
        Cell4<T> v;
        v.st = (T)sigt[e];
        v.y = (T)(0.5 * sigs[((long long)g * G + g) * C + c]);
        const double ex = src ? 0.5 * src[e] : 0.0;
        v.z = (T)ex;
        v.phi = phi0 ? (T)phi0[e] : (phi0_flat ? T(1) : T(0));
        X[e] = v;
        ext[e] = (T)ex;
        if (nsf) nsfT[e] = (T)nsf[e];
        if (sigs1) {
            y1[e] = (T)(1.5 * sigs1[e]);
            cur[e] = T(0);
        }
        if (G > 1)
            for (int gp = 0; gp < G; ++gp)
                scat[((long long)gp * G + g) * C + c] = (T)(0.5 * sigs[((long long)gp * G + g) * C + c]);
    }
}

// Factors of the diffusion synthetic acceleration system of every (group,
// instance), one warp each.  Cell i contributes D_i/h [[1,-1],[-1,1]] +
// Sigma_a,i h/4 [[1,1],[1,1]] to its two edges (D = 1/(3 Sigma_t),
// Sigma_a = Sigma_t - Sigma_s,gg); a vacuum face adds the quadrature's
// half-range current sum_{mu>0} w mu to its edge.  With o_i = Sigma_a,i h/4 -
// D_i/h the off-diagonal entry of cell i, each diagonal entry is
// d_k = |o_{k-1}| + |o_k| + delta_k with delta_k = 2 sum over the edge's cells
// of min(D_i/h, Sigma_a,i h/4) (+ face term) >= 0, and the Thomas pivots are
// carried as p_k = |o_k| + t_k with
//     t_0 = delta_0,   t_k = delta_k + |o_{k-1}| t_{k-1} / (|o_{k-1}| + t_{k-1}),
// a recurrence of positive terms.  (The textbook form p_k = d_k - o_{k-1}^2 /
// p_{k-1} subtracts nearly equal numbers when the cells are optically thin
// and loses the absorption in FP32.)  Each step is a Moebius map of t with
// the positive matrix [[delta + |o|, delta |o|], [1, |o|]], so the lanes
// compose their chunks' matrices (normalised by the largest entry), scan
// them with shuffles, and then run their chunks from the scanned entry
// value.  The matrix is symmetric positive definite unless the instance has
// no absorption and no vacuum face (then source iteration does not converge
// either); a pivot that is not positive gives a zero factor there.
template <typename T>
__device__ __forceinline__ T dsa_rcp(T x) {
    return rcp_dd(x);
}

template <typename T>
__device__ __forceinline__ void dsa_cell(const Cell4<T>& v, T h, T& o, T& mn) {
    const T dh = dsa_rcp(T(3) * v.st * h);
    const T ms = T(0.25) * (v.st - T(2) * v.y) * h;
    o = ms - dh;
    mn = fmin(dh, ms);
}

template <typename T>
__device__ __forceinline__ void mat_norm(T& a00, T& a01, T& a10, T& a11) {
    const T mx = fmax(fmax(a00, a01), fmax(a10, a11));
    if (mx > T(0)) {
        const T r = dsa_rcp(mx);
        a00 *= r;
        a01 *= r;
        a10 *= r;
        a11 *= r;
    }
}

#define DSA_FACTOR_BATCH 8
template <typename T>
__global__ void sn1d_dsa_factor(Sn1dArgs a) {
    const int lane = threadIdx.x & 31;
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (wid >= (long long)a.G * a.n_inst) return;   // the whole warp leaves together
    const int g = (int)(wid / a.n_inst), b = (int)(wid % a.n_inst);
    const int I = a.ncell[b], N = a.nang[b], q0 = a.qoff[b];
    const T h = (T)a.dx[b];
    const long long off = a.cell_off[b];
    const Cell4<T>* X = (const Cell4<T>*)a.X + (long long)g * a.C + off;
    const int E = I + 1;
    const int m = (E + 31) / 32;
    const int k0 = lane * m;
    const int n = max(0, min(m, E - k0));
    DsaEdge<T>* F = (DsaEdge<T>*)a.dsaf + (long long)g * (a.C + 32LL * a.n_inst) + off +
                    32LL * b + lane;
    // half-range current (nodes ascend: the upper half has mu > 0)
    double hs = 0.0;
    for (int q = N / 2 + lane; q < N; q += 32) hs += a.w[q0 + q] * a.mu[q0 + q];
    const T hr = (T)warp_sum(hs);
    const T aL = a.bc_left ? T(0) : hr, aR = a.bc_right ? T(0) : hr;
    T o_in = T(0), mn_in = T(0);
    if (n > 0 && k0 > 0) dsa_cell<T>(X[k0 - 1], h, o_in, mn_in);
    // compose this chunk's maps
    T a00 = T(1), a01 = T(0), a10 = T(0), a11 = T(1);
    T oprev = o_in, mnprev = mn_in;
#pragma unroll 1
    for (int jb = 0; jb < n; jb += DSA_FACTOR_BATCH) {
        Cell4<T> v[DSA_FACTOR_BATCH];
#pragma unroll
        for (int q = 0; q < DSA_FACTOR_BATCH; ++q)
            if (jb + q < n && k0 + jb + q < I) v[q] = X[k0 + jb + q];
#pragma unroll
        for (int q = 0; q < DSA_FACTOR_BATCH; ++q) {
            const int k = k0 + jb + q;
            if (jb + q < n) {
                T o = T(0), mn = T(0);
                if (k < I) dsa_cell<T>(v[q], h, o, mn);
                const T delta = T(2) * (mnprev + mn) + (k == 0 ? aL : T(0)) + (k == I ? aR : T(0));
                T m00, m01, m10, m11;
                if (k == 0) {
                    m00 = T(0);
                    m01 = delta;
                    m10 = T(0);
                    m11 = T(1);
                } else {
                    const T ao = fabs(oprev);
                    m00 = delta + ao;
                    m01 = delta * ao;
                    m10 = T(1);
                    m11 = ao;
                }
                const T b00 = m00 * a00 + m01 * a10, b01 = m00 * a01 + m01 * a11;
                const T b10 = m10 * a00 + m11 * a10, b11 = m10 * a01 + m11 * a11;
                a00 = b00;
                a01 = b01;
                a10 = b10;
                a11 = b11;
                mat_norm(a00, a01, a10, a11);
                oprev = o;
                mnprev = mn;
            }
        }
    }
    // inclusive scan: later chunks' maps act after earlier ones
    for (int d = 1; d < 32; d <<= 1) {
        const T c00 = __shfl_up_sync(0xffffffffu, a00, d);
        const T c01 = __shfl_up_sync(0xffffffffu, a01, d);
        const T c10 = __shfl_up_sync(0xffffffffu, a10, d);
        const T c11 = __shfl_up_sync(0xffffffffu, a11, d);
        if (lane >= d) {
            const T b00 = a00 * c00 + a01 * c10, b01 = a00 * c01 + a01 * c11;
            const T b10 = a10 * c00 + a11 * c10, b11 = a10 * c01 + a11 * c11;
            a00 = b00;
            a01 = b01;
            a10 = b10;
            a11 = b11;
            mat_norm(a00, a01, a10, a11);
        }
    }
    // t entering this chunk: the earlier chunks' map applied to (0, 1)
    const T e01 = __shfl_up_sync(0xffffffffu, a01, 1);
    const T e11 = __shfl_up_sync(0xffffffffu, a11, 1);
    T t = (lane > 0 && e11 > T(0)) ? e01 / e11 : T(0);
    oprev = o_in;
    mnprev = mn_in;
#pragma unroll 1
    for (int jb = 0; jb < n; jb += DSA_FACTOR_BATCH) {
        Cell4<T> v[DSA_FACTOR_BATCH];
#pragma unroll
        for (int q = 0; q < DSA_FACTOR_BATCH; ++q)
            if (jb + q < n && k0 + jb + q < I) v[q] = X[k0 + jb + q];
#pragma unroll
        for (int q = 0; q < DSA_FACTOR_BATCH; ++q) {
            const int k = k0 + jb + q;
            if (jb + q < n) {
                T o = T(0), mn = T(0);
                if (k < I) dsa_cell<T>(v[q], h, o, mn);
                const T delta = T(2) * (mnprev + mn) + (k == 0 ? aL : T(0)) + (k == I ? aR : T(0));
                const T ao = fabs(oprev);
                t = k == 0 ? delta : delta + ao * t * dsa_rcp(ao + t);
                const T piv = fabs(o) + t;
                DsaEdge<T> f;
                f.fm = piv > T(0) && isfinite(piv) ? dsa_rcp(piv) : T(0);
                f.o = o;
                F[(jb + q) * 32] = f;
                oprev = o;
                mnprev = mn;
            }
        }
    }
}

template <typename T>
__global__ void sn1d_finish(long long total, const Cell4<T>* X, double* phi) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        phi[e] = (double)X[e].phi;
}

template <typename T>
int sn1d_run(nop_ctx* ctx, const nop_solve_opts* o, bool eigen, const double* phi0,
               const double* k0, double* phi_out, bool out_dev, double* k_out,
               nop_stats* st) {
    SlabDev& s = ctx->slab;
    const int G = ctx->G;
    const long long C = s.C;
    const int B = s.n_inst;
    void* p;
    NOP_TRY(ctx->scratch("sn1d_X", sizeof(Cell4<T>) * G * C, &p));
    Cell4<T>* X = (Cell4<T>*)p;
    NOP_TRY(ctx->scratch("sn1d_U", sizeof(Cell2<T>) * C, &p));
    Cell2<T>* U = (Cell2<T>*)p;
    NOP_TRY(ctx->scratch("sn1d_scat", sizeof(T) * (G > 1 ? (long long)G * G * C : 1), &p));
    T* scat = (T*)p;
    NOP_TRY(ctx->scratch("sn1d_ext", sizeof(T) * G * C, &p));
    T* ext = (T*)p;
    NOP_TRY(ctx->scratch("sn1d_nsf", sizeof(T) * (eigen ? G * C : 1), &p));
    T* nsf = (T*)p;
    NOP_TRY(ctx->scratch("sn1d_phiprev", sizeof(T) * (eigen ? G * C : 1), &p));
    T* phiprev = (T*)p;
    NOP_TRY(ctx->scratch("sn1d_psib", sizeof(T) * std::max<long long>(1, s.bnd_total), &p));
    T* psib = (T*)p;
    // linearly anisotropic scattering (Eq. 25): fixed-source slabs, warp path
    const bool p1 = ctx->sigs1_d != nullptr;
    if (p1 && eigen) {
        ctx->set_error("anisotropic scattering is supported for fixed-source problems");
        return NOP_EINVAL;
    }
    T *y1 = nullptr, *cur = nullptr, *s1buf = nullptr, *jm = nullptr;
    if (p1) {
        NOP_TRY(ctx->scratch("sn1d_y1", sizeof(T) * G * C, &p));
        y1 = (T*)p;
        NOP_TRY(ctx->scratch("sn1d_cur", sizeof(T) * G * C, &p));
        cur = (T*)p;
        NOP_TRY(ctx->scratch("sn1d_s1", sizeof(T) * C, &p));
        s1buf = (T*)p;
        NOP_TRY(ctx->scratch("sn1d_jm", sizeof(T) * C, &p));
        jm = (T*)p;
    }
    const bool dsa = (o->flags & NOP_DSA) != 0;
    if (dsa && p1) {
        ctx->set_error("diffusion synthetic acceleration needs isotropic scattering");
        return NOP_EINVAL;
    }
    void* dsaf = nullptr;
    void* dsaw = nullptr;
    if (dsa) {
        NOP_TRY(ctx->scratch("sn1d_dsa", sizeof(DsaEdge<T>) * (size_t)G * (size_t)(C + 32LL * B),
                             &p));
        dsaf = p;
        NOP_TRY(ctx->scratch("sn1d_dsaw", sizeof(T) * 2 * (size_t)(C + 32LL * B), &p));
        dsaw = p;
    }
    NOP_TRY(ctx->scratch("sn1d_k0", sizeof(double) * B, &p));
    double* k0_d = (double*)p;
    NOP_TRY(ctx->scratch("sn1d_int", sizeof(int) * (5 * (size_t)B + 4), &p));
    int* ints = (int*)p;
    int* order_d = ints;
    int* it_d = ints + 2 * B;
    int* st_d = ints + 3 * B;
    int* cfg_d = ints + B;
    int* big_d = ints + 4 * B;
    int* counter = ints + 5 * B;
    NOP_TRY(ctx->scratch("sn1d_outer", sizeof(int) * B, &p));
    int* outer_d = (int*)p;
    NOP_TRY(ctx->scratch("sn1d_dbl", sizeof(double) * 2 * (size_t)B, &p));
    double* ch_d = (double*)p;
    double* kk_d = ch_d + B;
    unsigned long long* trace_d = nullptr;
    if (ctx->timing) {
        NOP_TRY(ctx->scratch("sn1d_trace", sizeof(unsigned long long) * 3 * (size_t)B, &p));
        trace_d = (unsigned long long*)p;
    }

    // ---- the arguments of every launch; the instance lists, lane
    // configurations and queue split are filled in by the scheduling below
    const int blocks_max = ctx->sm_count * SN1D_BLOCKS_PER_SM;
    constexpr int NW = SN1D_THREADS / 32;
    const long long total = (long long)G * C;
    const int pblocks = (int)std::min<long long>((total + 255) / 256, 4LL * ctx->sm_count * 8);
    auto prepare = [&]() -> int {
        const int m = ctx->phase_begin(2);
        sn1d_prepare<T><<<std::max(1, pblocks), 256, 0, ctx->stream>>>(
            C, G, ctx->sigt_d, ctx->sigs_d, eigen ? nullptr : ctx->src_d,
            eigen ? ctx->nsf_d : nullptr, phi0, (eigen && !phi0) ? 1 : 0, X, scat, ext, nsf,
            p1 ? ctx->sigs1_d : nullptr, y1, cur);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        ctx->phase_end(m);
        ctx->count_launch(false);
        return NOP_OK;
    };
    NOP_TRY(prepare());
    int mk;
    Sn1dArgs a;
    a.n_inst = B;
    a.G = G;
    a.C = C;
    a.order_list = order_d;
    a.n_small = 0;
    a.big_list = big_d;
    a.n_big = 0;
    a.big_blocks = 0;
    a.smem_cells = 1;
    a.counter = counter;
    a.cell_off = s.cell_off_d;
    a.ncell = s.ncell_d;
    a.nang = s.nang_d;
    a.dx = s.dx_d;
    a.qoff = s.qoff_d;
    a.mu = s.mu_d;
    a.w = s.w_d;
    a.boff = s.boff_d;
    a.X = X;
    a.U = U;
    a.cfg = cfg_d;
    a.scat = scat;
    a.ext = ext;
    a.psib = psib;
    a.p1 = p1 ? 1 : 0;
    a.y1 = y1;
    a.cur = cur;
    a.s1buf = s1buf;
    a.jm = jm;
    a.bc_left = ctx->bc[0];
    a.bc_right = ctx->bc[1];
    a.dsa = dsa ? 1 : 0;
    a.dsaf = dsaf;
    a.dsaw = dsaw;
    a.eigen = eigen ? 1 : 0;
    a.nsf = nsf;
    a.chi = ctx->chi_d;
    a.phiprev = phiprev;
    a.k0 = k0_d;
    a.tol = o->tol;
    a.tol_inner = o->tol_inner;
    a.tol_k = o->tol_k;
    a.itmax = o->itmax;
    a.itmax_inner = o->itmax_inner;
    a.it_out = it_d;
    a.st_out = st_d;
    a.ch_out = ch_d;
    a.k_out = kk_d;
    a.outer_out = outer_d;
    a.trace = trace_d;
    const size_t smem = SN1D_STAGE_BYTES;
    NOP_CUDA_TRY(ctx, cudaFuncSetAttribute(sn1d_kernel<T>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)SN1D_STAGE_BYTES));
    if (dsa) {
        mk = ctx->phase_begin(2);
        const long long nf = (long long)G * B;   // one warp each
        sn1d_dsa_factor<T><<<(int)((nf + 3) / 4), 128, 0, ctx->stream>>>(a);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        ctx->phase_end(mk);
        ctx->count_launch(false);
    }
    // Launch of the persistent kernel over given queues (warp queue `sm`,
    // team queue `bg`, the first `bblocks` blocks starting on the team queue).
    // The lists travel through a pinned buffer, so that the copies stay
    // asynchronous (a copy from pageable memory can wait for the stream).
    void* pin;
    NOP_TRY(ctx->pinned("sn1d_lists", sizeof(int) * 3 * (size_t)B + sizeof(double) * B, &pin));
    int* lists_h = (int*)pin;
    double* k0_h = (double*)(lists_h + 3 * (size_t)B);
    auto launch = [&](const Sn1dArgs& base, const std::vector<int>& sm, const std::vector<int>& bg,
                      int bblocks, const std::vector<int>& cfgv, int smem_cells) -> int {
        std::copy(sm.begin(), sm.end(), lists_h);
        std::copy(bg.begin(), bg.end(), lists_h + B);
        std::copy(cfgv.begin(), cfgv.end(), lists_h + 2 * (size_t)B);
        if (!sm.empty())
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(order_d, lists_h, sizeof(int) * sm.size(),
                                              cudaMemcpyHostToDevice, ctx->stream));
        if (!bg.empty())
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(big_d, lists_h + B, sizeof(int) * bg.size(),
                                              cudaMemcpyHostToDevice, ctx->stream));
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(cfg_d, lists_h + 2 * (size_t)B, sizeof(int) * B,
                                          cudaMemcpyHostToDevice, ctx->stream));
        NOP_CUDA_TRY(ctx, cudaMemsetAsync(counter, 0, 2 * sizeof(int), ctx->stream));
        Sn1dArgs la = base;
        la.n_small = (int)sm.size();
        la.n_big = (int)bg.size();
        la.big_blocks = bblocks;
        la.smem_cells = smem_cells;
        const int blocks = (int)std::max<long long>(
            1, std::min<long long>(blocks_max,
                                   (long long)bg.size() + ((long long)sm.size() + NW - 1) / NW));
        sn1d_kernel<T><<<blocks, SN1D_THREADS, smem, ctx->stream>>>(la);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        ctx->count_launch(true);
        return NOP_OK;
    };

    // ---- scheduling (host side).  Estimated iterations of an instance: those
    // of the previous solve of the same batch layout when known (unless the
    // caller asks for a cold schedule), else 0.94 log(tol) / log(rho) with rho
    // the diffusion estimate of the source iteration's spectral radius made at
    // set-up (rho_si_kernel; 0.94 is the median ratio of measured to
    // estimated counts on the 4096-slab batch).
    const double tol_its = eigen ? std::min(o->tol_inner, o->tol) : o->tol;
    // iterations of the previous solve of this layout, kept apart for solves
    // with and without the diffusion correction (they differ several times)
    std::vector<int>& last = dsa ? s.last_iters_dsa : s.last_iters;
    const bool cold = (o->flags & NOP_COLD_SCHEDULE) != 0;
    // a slab solve seeded by the DeepONet/FNO recast prediction
    const bool warm_recast = !eigen && o->warm_start == NOP_WARM_RECAST && phi0 != nullptr &&
                             ctx->no.loaded;
    std::vector<double> its_est(B);
    for (int b = 0; b < B; ++b) {
        const double c = std::min(0.9999, std::max(0.05, s.rho[b]));
        const double rs = std::min(0.9999, std::max(0.05, b < (int)s.rho_si.size() ? s.rho_si[b] : c));
        double its = std::min(5000.0, std::max(5.0, 0.94 * std::log(tol_its) / std::log(rs)));
        // the accelerated iteration contracts like about c/4 (Fourier analysis)
        if (dsa) its = std::max(3.0, std::log(tol_its) / std::log(std::max(0.05, 0.25 * c)));
        if (warm_recast && !dsa) {
            // the recast warm start removes the part of the initial error its
            // prediction gets right, a fraction e0 of the zero guess's error
            // remaining, which saves log(1 / e0) / log(1 / rho) source
            // iterations.  The prediction's own error leaves the slowly
            // converging instances the least: on the 4096-slab batch
            // (DeepONet trained at p*, 10 recast steps) the measured savings
            // follow log(1 / e0) = 6.2 (log(1 / rho))^0.55, median 2.8, 1.8
            // for the 300 longest instances.  Fewer recast steps K leave at
            // least rho_rec^K, rho_rec = |Sigma_a / Sigma_a* - 1| the
            // recast's contraction for the mean absorption mismatch.
            const double sa_star = ctx->no.cfg.sigma_t_star - ctx->no.cfg.sigma_s_star;
            const double rr = sa_star > 0 ? std::fabs(s.siga_mean[b] / sa_star - 1.0) : 1.0;
            const double lr = std::log(1.0 / rs);
            double le0 = 6.2 * std::pow(lr, 0.55);
            if (rr > 0.0 && rr < 1.0)
                le0 = std::min(le0, -std::log(rr) * (double)std::max(1, o->recast_itmax));
            else if (rr >= 1.0)
                le0 = 0.0;
            its = std::max(3.0, its - le0 / lr);
        }
        if (!eigen && !cold && b < (int)last.size() && last[b] > 0) its = last[b];
        its_est[b] = its;
    }
    const int max_smem_cells =
        (int)(SN1D_STAGE_BYTES / (sizeof(Cell2<T>) + NW * sizeof(T)));
    const int warps_total =
        (int)std::max<long long>(1, std::min<long long>(B, (long long)blocks_max * NW));
    const bool direct_ok = !p1 && !dsa && !ctx->bc[0] && !ctx->bc[1] &&
                           !(o->flags & NOP_SWEEP_CHUNKED);
    auto direct_A = [&](int b) { return (s.order[b] / 2 + 15) / 16; };
    auto chunked_cfg = [&](int b, bool team_cfg, double* half) {
        int lg, A;
        const int N = team_cfg ? 2 * ((s.order[b] / 2 + NW - 1) / NW) : s.order[b];
        sn1d_pick_config(s.ncell[b], N, &lg, &A, p1 || sizeof(T) == 8, half);
        return (lg << 8) | A;
    };
    // The schedule is a pure function of the batch, the options and (unless
    // cold) the iteration counts of the previous solve: reuse the last one
    // when none of these changed.
    auto plan_key = [&]() {
        unsigned long long key = 1469598103934665603ull;   // FNV-1a over the inputs
        auto mix = [&](unsigned long long v) { key = (key ^ v) * 1099511628211ull; };
        mix((unsigned long long)s.version);
        mix(sizeof(T));
        mix(eigen ? 1 : 0);
        mix((unsigned long long)(o->flags & (NOP_DSA | NOP_SWEEP_CHUNKED | NOP_COLD_SCHEDULE)));
        mix((unsigned long long)o->schedule);
        mix(warm_recast ? (unsigned long long)o->recast_itmax + 1 : 0ull);
        mix((unsigned long long)ctx->bc[0] * 2 + ctx->bc[1]);
        mix(p1 ? 1 : 0);
        double t = tol_its;
        unsigned long long u;
        std::memcpy(&u, &t, sizeof(u));
        mix(u);
        mix((unsigned long long)ctx->sn1d_tune[sizeof(T) == 8 ? 1 : 0].size());
        if (!cold && !eigen)
            for (int b = 0; b < B && b < (int)last.size(); ++b) mix((unsigned long long)last[b]);
        return key;
    };
    const unsigned long long key = plan_key();
    std::vector<int> cfg, small, big;
    int big_blocks = 0, smem_cells = 1;
    ctx->last_tune_ms = 0.0;
    const bool plan_hit = key == s.plan_key && (int)s.plan_cfg.size() == B;
    if (plan_hit) {
        cfg = s.plan_cfg;
        small = s.plan_small;
        big = s.plan_big;
        big_blocks = s.plan_big_blocks;
        smem_cells = s.plan_smem_cells;
        ctx->last_direct = s.plan_direct;
    } else {
        // Per instance: the configuration and latency of one iteration on one
        // warp (cw, lw) and on a 12-warp team (ct, lt; lt < 0: no team).
        std::vector<int> cw(B), ct(B, 0);
        std::vector<double> lw(B), lt(B, -1.0);
        auto fits_team = [&](int b) { return s.ncell[b] <= max_smem_cells && !p1; };
        const bool tune = o->schedule == NOP_SCHED_AUTO && B >= NOP_SCHED_TUNE_MIN;
        if (tune) {
            // ---- measured costs (the autotuner).  Every instance falls in a
            // bucket (order, half-octave of its cell count, groups, and whether
            // the correction, anisotropic scattering and the direct lanes apply).
            // For every candidate layout -- direct or chunked lanes, on one warp
            // or on a team -- the context keeps the measured time of one source
            // iteration per cell, under the load of a full batch.  Buckets not
            // measured yet on this device are measured now: up to 12 instances
            // of each run 3 source iterations in one launch per candidate, timed
            // per instance on the device clock, and the bucket keeps the median.
            auto key_of = [&](int b) -> long long {
                const int ib = (int)std::floor(2.0 * std::log2((double)s.ncell[b]));
                return ((((long long)s.order[b] * 64 + ib) * 64 + G) * 8) + (dsa ? 1 : 0) +
                       (p1 ? 2 : 0) + (direct_ok ? 4 : 0);
            };
            auto& table = ctx->sn1d_tune[sizeof(T) == 8 ? 1 : 0];
            std::map<long long, std::vector<int>> todo;
            for (int b = 0; b < B; ++b) {
                const long long key = key_of(b);
                if (table.count(key)) continue;
                auto& v = todo[key];
                if ((int)v.size() < 12) v.push_back(b);
            }
            if (!todo.empty()) {
                const auto t0 = std::chrono::steady_clock::now();
                void* tp;
                NOP_TRY(ctx->scratch("sn1d_tune_trace", sizeof(unsigned long long) * 3 * (size_t)B, &tp));
                unsigned long long* tr_d = (unsigned long long*)tp;
                Sn1dArgs ca = a;
                ca.eigen = 0;
                ca.itmax = 3;
                ca.itmax_inner = 3;
                ca.tol = ca.tol_inner = 0.0;
                ca.trace = tr_d;
                std::map<long long, std::array<std::vector<double>, 4>> meas;
                std::vector<unsigned long long> tr(3 * (size_t)B);
                std::vector<int> it_h(B);
                for (int cand = 0; cand < 4; ++cand) {
                    // 0: direct warp, 1: chunked warp, 2: direct team, 3: chunked team
                    const bool direct = cand == 0 || cand == 2, team_c = cand >= 2;
                    if (direct && !direct_ok) continue;
                    std::vector<int> list, cfgv(B, 0);
                    int smc = 1;
                    for (auto& kv : todo)
                        for (int b : kv.second) {
                            if (cand == 3 && !fits_team(b)) continue;
                            list.push_back(b);
                            cfgv[b] = direct ? (SN1D_DIRECT | direct_A(b)) : chunked_cfg(b, team_c, nullptr);
                            if (cand == 3) smc = std::max(smc, s.ncell[b]);
                        }
                    if (list.empty()) continue;
                    if (team_c)
                        NOP_TRY(launch(ca, {}, list, std::min<int>(blocks_max, (int)list.size()), cfgv, smc));
                    else
                        NOP_TRY(launch(ca, list, {}, 0, cfgv, smc));
                    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(tr.data(), tr_d, sizeof(unsigned long long) * 3 * B,
                                                      cudaMemcpyDeviceToHost, ctx->stream));
                    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(it_h.data(), it_d, sizeof(int) * B,
                                                      cudaMemcpyDeviceToHost, ctx->stream));
                    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
                    for (int b : list) {
                        const double us = (double)(tr[3 * b + 1] - tr[3 * b]) * 1e-3;
                        if (it_h[b] > 0 && us > 0)
                            meas[key_of(b)][cand].push_back(us / it_h[b] / s.ncell[b]);
                    }
                }
                for (auto& kv : meas) {
                    std::array<double, 4> c4 = {-1.0, -1.0, -1.0, -1.0};
                    for (int cand = 0; cand < 4; ++cand) {
                        auto& v = kv.second[cand];
                        if (v.empty()) continue;
                        std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
                        c4[cand] = v[v.size() / 2];
                    }
                    table[kv.first] = c4;
                }
                // the calibration iterated on the solve's own arrays: start over
                NOP_TRY(prepare());
                ctx->last_tune_ms = std::chrono::duration<double, std::milli>(
                                        std::chrono::steady_clock::now() - t0).count();
            }
            for (int b = 0; b < B; ++b) {
                auto it = table.find(key_of(b));
                const double I = s.ncell[b];
                double c4[4] = {-1, -1, -1, -1};
                if (it != table.end())
                    for (int q = 0; q < 4; ++q) c4[q] = it->second[q];
                // warp: the faster of the measured layouts (chunked if none was)
                const bool d_w = c4[0] > 0 && (c4[1] <= 0 || c4[0] < c4[1]);
                cw[b] = d_w ? (SN1D_DIRECT | direct_A(b)) : chunked_cfg(b, false, nullptr);
                lw[b] = its_est[b] * I * (d_w ? c4[0] : (c4[1] > 0 ? c4[1] : 1.0));
                const bool d_t = c4[2] > 0 && (c4[3] <= 0 || c4[2] < c4[3]);
                if (d_t || (c4[3] > 0 && fits_team(b))) {
                    ct[b] = d_t ? (SN1D_DIRECT | direct_A(b)) : chunked_cfg(b, true, nullptr);
                    lt[b] = its_est[b] * I * (d_t ? c4[2] : c4[3]);
                }
            }
        } else {
            // ---- analytic model, in issue slots of one lane per source
            // iteration (batches too small to measure, or NOP_SCHED_MODEL):
            //   direct lanes on one warp: I steps of (12 + 14 A) slots plus about
            //     80 per block of 32 cells; on a team two passes over a chunk of
            //     ceil(I / 12) cells plus the team's barriers;
            //   chunked lanes: both direction halves of sn1d_pick_config's model;
            //   the correction: 4 passes over ceil((I + 1) / 32) edges.
            // Direct lanes where at least 12 half-angles fill 3/4 of a half-warp.
            auto dsa_slots = [&](int b) { return dsa ? 120.0 * ((s.ncell[b] + 32) / 32) * G : 0.0; };
            for (int b = 0; b < B; ++b) {
                const int I = s.ncell[b];
                if (direct_ok && s.order[b] / 2 >= 12) {
                    const int A = direct_A(b);
                    cw[b] = ct[b] = SN1D_DIRECT | A;
                    lw[b] = its_est[b] * G * (I * (12.0 + 14.0 * A) + 80.0 * ((I + 31) / 32));
                    const double m = (double)((I + NW - 1) / NW);
                    lt[b] = its_est[b] * G *
                            (2.0 * m * (12.0 + 14.0 * A) + 160.0 * ((m + 31) / 32) + 3000.0);
                } else {
                    double half;
                    cw[b] = chunked_cfg(b, false, &half);
                    lw[b] = its_est[b] * (G * 2.0 * half + dsa_slots(b));
                    if (fits_team(b)) {
                        ct[b] = chunked_cfg(b, true, &half);
                        lt[b] = its_est[b] * (G * 2.0 * half + dsa_slots(b));
                    }
                }
            }
        }
        // Which instances get a team: with longest-first queues the batch takes
        // about max(expected span, longest latency).  An instance whose one-warp
        // latency, times a margin, is above the expected span S = (warp
        // latencies + 12 x team latencies) / warps gets a team (a team costs
        // more SM time than one warp, so only the instances that would outlast
        // the batch are worth it).  The margin covers the error of the latency
        // estimates: 1.1 when the iteration counts are estimated, 1.05 when
        // they are those of the previous solve of the layout (on the
        // 4096-slab batch a margin of 1.0 left a straggler, 1.05-1.1 gave the
        // shortest step, and every 0.15 above that added teams and about 3%).
        std::vector<char> team;
        double span = 0.0;
        const bool known_its = !cold && !eigen && (int)last.size() == B;
        NOP_TRY(sn1d_select_teams(B, lw.data(), lt.data(), warps_total, NW,
                                  o->schedule == NOP_SCHED_BLOCK ? 1 : (o->schedule == NOP_SCHED_WARP || B < 2 ? 2 : 0),
                                  known_its ? 1.05 : 1.1, team, &span));
        cfg.assign(B, 0);
        std::vector<double> cost(B);
        double big_work = 0, small_work = 0;
        int n_direct = 0;
        for (int b = 0; b < B; ++b) {
            if (team[b]) {
                cfg[b] = ct[b];
                if (!(cfg[b] & SN1D_DIRECT)) smem_cells = std::max(smem_cells, s.ncell[b]);
                big.push_back(b);
                cost[b] = lt[b];
                big_work += lt[b];
            } else {
                cfg[b] = cw[b];
                small.push_back(b);
                cost[b] = lw[b];
                small_work += lw[b] / NW;
            }
            n_direct += (cfg[b] & SN1D_DIRECT) ? 1 : 0;
        }
        ctx->last_direct = n_direct;
        // Large and small instances run side by side from the start: a share of
        // the blocks proportional to the large instances' block-time takes the
        // large queue first, the other blocks go straight to the small queue.
        if (!big.empty()) {
            const double share = big_work / std::max(1e-30, big_work + small_work);
            big_blocks = (int)std::ceil(share * blocks_max);
            big_blocks = std::max(1, std::min<int>(big_blocks, (int)big.size()));
            if (small.empty()) big_blocks = std::min<int>(blocks_max, (int)big.size());
        }
        auto longest_first = [&](int x, int y) { return cost[x] > cost[y]; };
        std::stable_sort(small.begin(), small.end(), longest_first);
        std::stable_sort(big.begin(), big.end(), longest_first);
        s.plan_cfg = cfg;
        s.plan_small = small;
        s.plan_big = big;
        s.plan_big_blocks = big_blocks;
        s.plan_smem_cells = smem_cells;
        s.plan_direct = n_direct;
        // the tuner may have added buckets: key the plan on the table as used
        s.plan_key = plan_key();
    }
    for (int b = 0; b < B; ++b) k0_h[b] = (k0 && k0[b] > 0) ? k0[b] : 1.0;
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(k0_d, k0_h, sizeof(double) * B,
                                      cudaMemcpyHostToDevice, ctx->stream));
    mk = ctx->phase_begin(0);
    NOP_TRY(launch(a, small, big, big_blocks, cfg, smem_cells));
    ctx->phase_end(mk);
    if (phi_out) {
        double* dst = phi_out;
        if (!out_dev) {
            NOP_TRY(ctx->scratch("sn1d_phiout", sizeof(double) * total, &p));
            dst = (double*)p;
        }
        mk = ctx->phase_begin(2);
        sn1d_finish<T><<<std::max(1, pblocks), 256, 0, ctx->stream>>>(total, X, dst);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        ctx->phase_end(mk);
        ctx->count_launch(false);
        if (!out_dev)
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(phi_out, dst, sizeof(double) * total,
                                              cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (eigen && k_out) {
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(k_out, kk_d, sizeof(double) * B,
                                          out_dev ? cudaMemcpyDeviceToDevice
                                                  : cudaMemcpyDeviceToHost,
                                          ctx->stream));
    }
    if (out_dev && !st) {
        // the host vectors above are read by the copies: wait for them
        NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        return NOP_OK;
    }
    if (trace_d) {
        std::vector<unsigned long long> tr(3 * (size_t)B);
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(tr.data(), trace_d, sizeof(unsigned long long) * 3 * B,
                                          cudaMemcpyDeviceToHost, ctx->stream));
        NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        unsigned long long t0 = ~0ull, t1 = 0;
        double mx = 0, sum = 0;
        for (int b = 0; b < B; ++b) t0 = std::min(t0, tr[3 * b]);
        ctx->trace_inst.assign(3 * (size_t)B, 0.0);
        for (int b = 0; b < B; ++b) {
            t1 = std::max(t1, tr[3 * b + 1]);
            const double d = (double)(tr[3 * b + 1] - tr[3 * b]) * 1e-6;
            mx = std::max(mx, d);
            sum += d;
            ctx->trace_inst[3 * b] = (double)(tr[3 * b] - t0) * 1e-6;
            ctx->trace_inst[3 * b + 1] = d;
            ctx->trace_inst[3 * b + 2] = (tr[3 * b + 2] & 0x80000000ull) ? 1.0 : 0.0;
        }
        ctx->trace_span_ms = (double)(t1 - t0) * 1e-6;
        ctx->trace_max_ms = mx;
        ctx->trace_mean_ms = sum / B;
        ctx->trace_big = (int)big.size();
    }
    std::vector<int> it_h(B), st_h(B), out_h(B);
    std::vector<double> ch_h(B);
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(it_h.data(), it_d, sizeof(int) * B,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(st_h.data(), st_d, sizeof(int) * B,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(out_h.data(), outer_d, sizeof(int) * B,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(ch_h.data(), ch_d, sizeof(double) * B,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    int worst = NOP_OK;
    if (st) {
        st->max_iterations = 0;
        st->sum_iterations = 0;
        st->max_outer = 0;
        st->max_change = 0;
    }
    if (!eigen && (int)last.size() == B)
        for (int b = 0; b < B; ++b) last[b] = it_h[b];
    for (int b = 0; b < B; ++b) {
        if (ctx->timing)
            ctx->cell_angle_updates += (double)it_h[b] * s.ncell[b] * s.order[b] * G;
        if (st_h[b] != NOP_OK && (worst == NOP_OK || st_h[b] == NOP_ENAN)) worst = st_h[b];
        if (st) {
            st->max_iterations = std::max(st->max_iterations, it_h[b]);
            st->sum_iterations += it_h[b];
            if (eigen) st->max_outer = std::max(st->max_outer, out_h[b]);
            st->max_change = std::max(st->max_change, ch_h[b]);
            if (st->inst_iterations) st->inst_iterations[b] = it_h[b];
            if (st->inst_status) st->inst_status[b] = st_h[b];
        }
    }
    if (st) st->status = worst;
    return worst;
}

}  // namespace nop
