"""Pins for the FP64 transport oracle against what the physics and the paper fix.

Each test checks the oracle against something other than itself: closed forms,
invariants, dense linear-algebra solves of the discrete system, and the
eigenvalues the paper prints (Tables 7 and 10).
"""
import os

import numpy as np
import pytest
from scipy.special import expn

from oracle import quadrature as Qd
from oracle import transport as T
from oracle import native

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            vals[k] = np.array([float(t) for t in v])
    return vals


# ----------------------------------------------------------------- quadrature
@pytest.mark.parametrize("N", [2, 8, 16, 32, 64])
def test_gauss_legendre_integrates_polynomials(N):
    mu, w = Qd.gauss_legendre(N)
    for k in range(0, 2 * N):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * mu ** k) - exact) < 1e-13
    assert np.all(w > 0) and np.all(np.abs(mu) < 1)


def test_level_symmetric_s8_moments():
    mu, eta, w = Qd.level_symmetric_s8()
    xi = Qd.xi_of(mu, eta)
    assert len(mu) == 40 and np.all(w > 0)
    assert abs(w.sum() - 1) < 1e-14
    for a in (mu, eta, xi):
        assert abs(np.sum(w * a * a) - 1 / 3) < 1e-13
        assert abs(np.sum(w * a ** 4) - 1 / 5) < 1e-13
    assert abs(np.sum(w * mu) ) < 1e-14 and abs(np.sum(w * eta)) < 1e-14
    assert abs(np.sum(w * mu ** 3 * eta)) < 1e-14
    # not imposed in the derivation: the mixed sixth moment of the sphere
    assert abs(np.sum(w * mu ** 2 * eta ** 2 * xi ** 2) - 1 / 105) < 1e-12
    # the levels are equally spaced in mu^2 (level-symmetric structure)
    lev = np.unique(np.round(np.abs(mu), 12))
    assert len(lev) == 4
    assert np.allclose(np.diff(lev ** 2), np.diff(lev ** 2)[0], atol=1e-12)
    # S8's first level: mu_1^2 = 1/21 follows from the 8th-moment condition
    assert abs(lev[0] ** 2 - 1 / 21) < 1e-10


# --------------------------------------------------------------- 1D physics
def test_infinite_medium_reflective_flat_flux():
    # reflective on both faces: the flat flux Q / Sigma_a solves the DD equations
    P = T.uniform_slab(40, 10.0, 1.3, 0.9, Q=2.0, bc_left=T.REFLECTIVE,
                       bc_right=T.REFLECTIVE)
    r = T.source_iteration(P, Qd.gauss_legendre(8), tol=1e-14)
    assert np.max(np.abs(r.phi[0] - 2.0 / 0.4)) < 1e-10


def test_pure_absorber_dd_geometric_closed_form():
    # with Sigma_s = 0 one sweep is exact; per direction the DD recurrence
    # psi_out = alpha psi_in + beta has the closed form beta (1 - alpha^i)/(1 - alpha)
    I, L, st, Q = 30, 6.0, 0.7, 1.5
    mu, w = Qd.gauss_legendre(8)
    P = T.uniform_slab(I, L, st, 0.0, Q=Q)
    r = T.source_iteration(P, (mu, w), tol=1e-15)
    dx = L / I
    phi = np.zeros(I)
    for m, wt in zip(mu, w):
        a = abs(m) / dx
        alpha = (2 * a - st) / (2 * a + st)
        beta = Q / (2 * a + st)                 # 2 q / (2a + st), q = Q/2
        edge = lambda i: beta * (1 - alpha ** i) / (1 - alpha)
        idx = np.arange(I) if m > 0 else np.arange(I)[::-1]
        for step, i in enumerate(idx):
            phi[i] += wt * 0.5 * (edge(step) + edge(step + 1))
    assert np.max(np.abs(r.phi[0] - phi)) < 1e-12


def test_pure_absorber_converges_to_exponential_integral():
    # continuum solution of Eq. 12 with Sigma_s = 0, uniform Q, vacuum:
    # phi(x) = Q/st [1 - (E2(st x) + E2(st (L - x)))/2]; DD converges O(dx^2)
    # away from the boundary layer
    from scipy.integrate import quad
    L, st, Q = 4.0, 1.0, 1.0
    f = lambda x: Q / st * (1 - 0.5 * (expn(2, st * x) + expn(2, st * (L - x))))
    errs = []
    for I in (50, 100, 200):
        P = T.uniform_slab(I, L, st, 0.0, Q=Q)
        phi = T.source_iteration(P, Qd.gauss_legendre(64), tol=1e-15).phi[0]
        dx = L / I
        exact = np.array([quad(f, i * dx, (i + 1) * dx, limit=200)[0] / dx
                          for i in range(I)])
        errs.append(np.max(np.abs(phi - exact)[I // 4: 3 * I // 4]))
    assert errs[-1] < 1e-5
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4


def test_particle_balance_and_symmetry():
    P = T.uniform_slab(80, 10.0, 1.0, 0.8, Q=1.0)
    quad = Qd.gauss_legendre(16)
    r = T.source_iteration(P, quad, tol=1e-14)
    src, absn, leak = T.balance_1d(P, quad, r.phi, r.sweeper)
    assert abs(src - absn - leak) < 1e-10 * src
    assert np.max(np.abs(r.phi[0] - r.phi[0][::-1])) < 1e-11


def _dense_dd_1d(dx, sigt, sigs, Q, mu, w, bcl, bcr, G=None):
    """Assemble the DD edge-flux system of a 1-group slab and solve it densely."""
    I, N = len(dx), len(mu)
    E = I + 1
    idx = lambda n, j: n * E + j
    A = np.zeros((N * E, N * E))
    b = np.zeros(N * E)
    row = 0
    for n in range(N):
        for i in range(I):
            A[row, idx(n, i + 1)] += mu[n] / dx[i] + sigt[i] / 2
            A[row, idx(n, i)] += -mu[n] / dx[i] + sigt[i] / 2
            for m in range(N):
                A[row, idx(m, i)] -= 0.5 * sigs[i] * w[m] / 2
                A[row, idx(m, i + 1)] -= 0.5 * sigs[i] * w[m] / 2
            b[row] = 0.5 * Q[i]
            row += 1
    for n in range(N):
        mirror = int(np.argmin(np.abs(mu + mu[n])))
        if mu[n] > 0:
            A[row, idx(n, 0)] = 1.0
            if bcl:
                A[row, idx(mirror, 0)] -= 1.0
        else:
            A[row, idx(n, I)] = 1.0
            if bcr:
                A[row, idx(mirror, I)] -= 1.0
        row += 1
    e = np.linalg.solve(A, b).reshape(N, E)
    return np.sum(w[:, None] * 0.5 * (e[:, :-1] + e[:, 1:]), axis=0)


@pytest.mark.parametrize("bcl,bcr", [(0, 0), (1, 0), (0, 1)])
def test_source_iteration_matches_dense_dd_system(bcl, bcr):
    rng = np.random.default_rng(7)
    I = 7
    dx = rng.uniform(0.2, 0.9, I)
    sigt = rng.uniform(0.5, 2.0, I)
    sigs = sigt * rng.uniform(0.2, 0.9, I)
    Q = rng.uniform(0, 2, I)
    mu, w = Qd.gauss_legendre(6)
    P = T.Slab(dx=dx, sigt=sigt[None], sigs=sigs[None, None], Q=Q[None],
               bc_left=T.REFLECTIVE if bcl else T.VACUUM,
               bc_right=T.REFLECTIVE if bcr else T.VACUUM)
    r = T.source_iteration(P, (mu, w), tol=1e-15, itmax=100000)
    ref = _dense_dd_1d(dx, sigt, sigs, Q, mu, w, bcl, bcr)
    assert np.max(np.abs(r.phi[0] - ref)) < 1e-11 * np.max(ref)


def test_multigroup_upscatter_matches_dense_system():
    # two groups with down- and upscatter: Gauss-Seidel SI vs block dense solve
    rng = np.random.default_rng(11)
    I, G = 5, 2
    dx = np.full(I, 0.5)
    sigt = rng.uniform(0.8, 1.6, (G, I))
    S = np.zeros((G, G, I))
    S[0, 0], S[0, 1] = 0.3 * sigt[0], 0.3 * sigt[0]
    S[1, 1], S[1, 0] = 0.5 * sigt[1], 0.2 * sigt[1]
    Q = rng.uniform(0, 1, (G, I))
    mu, w = Qd.gauss_legendre(4)
    P = T.Slab(dx=dx, sigt=sigt, sigs=S, Q=Q)
    r = T.source_iteration(P, (mu, w), tol=1e-15)
    # dense: unknown edge fluxes for both groups
    N, E = len(mu), I + 1
    nu = N * E
    A = np.zeros((G * nu, G * nu))
    b = np.zeros(G * nu)
    ix = lambda g, n, j: g * nu + n * E + j
    row = 0
    for g in range(G):
        for n in range(N):
            for i in range(I):
                A[row, ix(g, n, i + 1)] += mu[n] / dx[i] + sigt[g, i] / 2
                A[row, ix(g, n, i)] += -mu[n] / dx[i] + sigt[g, i] / 2
                for gp in range(G):
                    for m in range(N):
                        for j in (i, i + 1):
                            A[row, ix(gp, m, j)] -= 0.5 * S[gp, g, i] * w[m] / 2
                b[row] = 0.5 * Q[g, i]
                row += 1
        for n in range(N):
            A[row, ix(g, n, 0 if mu[n] > 0 else I)] = 1.0
            row += 1
    e = np.linalg.solve(A, b).reshape(G, N, E)
    ref = np.sum(w[None, :, None] * 0.5 * (e[:, :, :-1] + e[:, :, 1:]), axis=1)
    assert np.max(np.abs(r.phi - ref)) < 1e-11 * np.max(ref)


# ------------------------------------------------------------------ eigen
def test_reflective_homogeneous_k_is_production_over_absorption():
    P = T.uniform_slab(30, 5.0, 1.0, 0.6, nusigf=0.5, bc_left=T.REFLECTIVE,
                       bc_right=T.REFLECTIVE)
    e = T.power_iteration(P, Qd.gauss_legendre(8), tol_k=1e-13, tol_phi=1e-11,
                          tol_inner=1e-13)
    assert abs(e.k - 0.5 / 0.4) < 1e-10


def test_multigroup_infinite_medium_k():
    g = _golden("table10_multigroup_k.txt")
    S = np.stack([g["sigma_s_row_from_g1"], g["sigma_s_row_from_g2"],
                  g["sigma_s_row_from_g3"]])
    st, nsf, chi = g["sigma_t"], g["nu"] * g["sigma_f"], g["chi"]
    # k_inf = dominant eigenvalue of (diag(st) - S^T)^-1 chi nsf^T
    Mop = np.linalg.solve(np.diag(st) - S.T, np.outer(chi, nsf))
    kinf = max(np.linalg.eigvals(Mop).real)
    I = 10
    P = T.Slab(dx=np.full(I, 0.5), sigt=st[:, None] * np.ones(I),
               sigs=S[:, :, None] * np.ones(I), nusigf=nsf[:, None] * np.ones(I),
               chi=chi, bc_left=T.REFLECTIVE, bc_right=T.REFLECTIVE)
    e = T.power_iteration(P, Qd.gauss_legendre(4), tol_k=1e-13, tol_phi=1e-11,
                          tol_inner=1e-13)
    assert abs(e.k - kinf) < 1e-9
    assert abs(kinf - 1.72) < 0.01         # hand elimination of Tables 8-9


def test_table10_three_group_k():
    g = _golden("table10_multigroup_k.txt")
    S = np.stack([g["sigma_s_row_from_g1"], g["sigma_s_row_from_g2"],
                  g["sigma_s_row_from_g3"]])
    I = 100
    P = T.Slab(dx=np.full(I, 0.1), sigt=g["sigma_t"][:, None] * np.ones(I),
               sigs=S[:, :, None] * np.ones(I),
               nusigf=(g["nu"] * g["sigma_f"])[:, None] * np.ones(I), chi=g["chi"])
    e = T.power_iteration(P, Qd.gauss_legendre(32), tol_k=1e-11, tol_phi=1e-9,
                          tol_inner=1e-11)
    assert abs(e.k - g["k_model"][0]) <= 5e-6


def test_table7_case1_k_loose():
    g = _golden("table7_case1_k.txt")
    P = T.uniform_slab(100, 10.0, g["sigma_t"][0], g["sigma_s"][0],
                       nusigf=g["nu_reading"][0] * g["sigma_f"][0])
    e = T.power_iteration(P, Qd.gauss_legendre(32), tol_k=1e-10, tol_phi=1e-8,
                          tol_inner=1e-10)
    assert abs(e.k - g["k_model"][0]) < 1e-3


def test_power_iteration_matches_dense_generalised_eigenproblem():
    rng = np.random.default_rng(3)
    I = 6
    dx = np.full(I, 0.8)
    sigt = rng.uniform(0.8, 1.5, I)
    sigs = 0.5 * sigt
    nsf = rng.uniform(0.2, 0.6, I)
    mu, w = Qd.gauss_legendre(4)
    N, E = len(mu), I + 1
    A = np.zeros((N * E, N * E))
    B = np.zeros((N * E, N * E))
    ix = lambda n, j: n * E + j
    row = 0
    for n in range(N):
        for i in range(I):
            A[row, ix(n, i + 1)] += mu[n] / dx[i] + sigt[i] / 2
            A[row, ix(n, i)] += -mu[n] / dx[i] + sigt[i] / 2
            for m in range(N):
                for j in (i, i + 1):
                    A[row, ix(m, j)] -= 0.5 * sigs[i] * w[m] / 2
                    B[row, ix(m, j)] += 0.5 * nsf[i] * w[m] / 2
            row += 1
    for n in range(N):
        A[row, ix(n, 0 if mu[n] > 0 else I)] = 1.0
        row += 1
    ev = np.linalg.eigvals(np.linalg.solve(A, B))
    kd = max(ev.real)
    P = T.Slab(dx=dx, sigt=sigt[None], sigs=sigs[None, None], nusigf=nsf[None],
               chi=np.ones(1))
    e = T.power_iteration(P, (mu, w), tol_k=1e-14, tol_phi=1e-12, tol_inner=1e-14)
    assert abs(e.k - kd) < 1e-10


# ---------------------------------------------------------------------- 2D
def _xy(nx, ny, dx, dy, sigt, sigs, Q, bc):
    G = 1
    return T.XY(dx=dx, dy=dy, sigt=np.full((G, ny, nx), sigt) if np.isscalar(sigt) else sigt,
                sigs=np.full((G, G, ny, nx), sigs) if np.isscalar(sigs) else sigs,
                Q=np.full((G, ny, nx), Q) if np.isscalar(Q) else Q, bc=bc)


def test_2d_infinite_medium_flat_flux():
    bc = {f: T.REFLECTIVE for f in ("x0", "xL", "y0", "yL")}
    P = _xy(6, 5, 0.4, 0.3, 1.2, 0.7, 1.0, bc)
    r = T.source_iteration(P, Qd.level_symmetric_s8(), tol=1e-14)
    assert np.max(np.abs(r.phi - 1.0 / 0.5)) < 1e-10


def test_2d_y_homogeneous_reduces_to_slab():
    # reflective y-faces and y-independent data: the 2D solution equals the
    # 1D slab solution with the 2D set's x-cosines and weights (x2, so sum 2)
    mu, eta, w = Qd.level_symmetric_s8()
    nx, ny = 12, 3
    rng = np.random.default_rng(5)
    st = rng.uniform(0.5, 2.0, nx)
    ss = st * rng.uniform(0.3, 0.9, nx)
    Q = rng.uniform(0.0, 1.0, nx)
    bc = {"x0": T.VACUUM, "xL": T.REFLECTIVE, "y0": T.REFLECTIVE, "yL": T.REFLECTIVE}
    P = _xy(nx, ny, 0.5, 0.7, np.tile(st, (1, ny, 1)), np.tile(ss, (1, 1, ny, 1)),
            np.tile(Q, (1, ny, 1)), bc)
    r2 = T.source_iteration(P, (mu, eta, w), tol=1e-14)
    P1 = T.Slab(dx=np.full(nx, 0.5), sigt=st[None], sigs=ss[None, None], Q=Q[None],
                bc_right=T.REFLECTIVE)
    r1 = T.source_iteration(P1, (mu, 2 * w), tol=1e-14)
    for j in range(ny):
        assert np.max(np.abs(r2.phi[0, j] - r1.phi[0])) < 1e-10


def test_2d_diagonal_symmetry():
    mu, eta, w = Qd.level_symmetric_s8()
    n = 7
    rng = np.random.default_rng(1)
    A = rng.uniform(0.5, 1.5, (n, n))
    st = (A + A.T)[None]
    bc = {"x0": T.REFLECTIVE, "xL": T.VACUUM, "y0": T.REFLECTIVE, "yL": T.VACUUM}
    P = _xy(n, n, 0.3, 0.3, st, 0.6 * st[None], np.ones((1, n, n)), bc)
    r = T.source_iteration(P, (mu, eta, w), tol=1e-14)
    assert np.max(np.abs(r.phi[0] - r.phi[0].T)) < 1e-11


def test_2d_matches_dense_dd_system():
    mu, eta, w = Qd.level_symmetric_s8()
    M = len(mu)
    nx, ny, dx, dy = 3, 2, 0.6, 0.4
    rng = np.random.default_rng(9)
    st = rng.uniform(0.6, 1.4, (ny, nx))
    ss = 0.5 * st
    Q = rng.uniform(0.2, 1.0, (ny, nx))
    bc = {"x0": T.REFLECTIVE, "xL": T.VACUUM, "y0": T.VACUUM, "yL": T.REFLECTIVE}
    # unknowns per direction: x-edges X[j, e] (e = 0..nx), y-edges Y[e, i] (e = 0..ny)
    nX, nY = ny * (nx + 1), (ny + 1) * nx
    per = nX + nY
    iX = lambda d, j, e: d * per + j * (nx + 1) + e
    iY = lambda d, e, i: d * per + nX + e * nx + i
    A = np.zeros((M * per, M * per))
    b = np.zeros(M * per)
    row = 0
    mx = [int(np.argmin(np.abs(mu + mu[d]) + np.abs(eta - eta[d]))) for d in range(M)]
    my = [int(np.argmin(np.abs(mu - mu[d]) + np.abs(eta + eta[d]))) for d in range(M)]
    for d in range(M):
        for j in range(ny):
            for i in range(nx):
                # balance with psi_c = (X_L + X_R)/2 and scattering of all directions
                A[row, iX(d, j, i + 1)] += mu[d] / dx + st[j, i] / 2
                A[row, iX(d, j, i)] += -mu[d] / dx + st[j, i] / 2
                A[row, iY(d, j + 1, i)] += eta[d] / dy
                A[row, iY(d, j, i)] += -eta[d] / dy
                for m in range(M):
                    A[row, iX(m, j, i)] -= ss[j, i] * w[m] / 2
                    A[row, iX(m, j, i + 1)] -= ss[j, i] * w[m] / 2
                b[row] = Q[j, i]
                row += 1
                # diamond consistency X_L + X_R = Y_B + Y_T
                A[row, iX(d, j, i)] += 1
                A[row, iX(d, j, i + 1)] += 1
                A[row, iY(d, j, i)] -= 1
                A[row, iY(d, j + 1, i)] -= 1
                row += 1
        for j in range(ny):
            e = 0 if mu[d] > 0 else nx
            A[row, iX(d, j, e)] = 1
            if bc["x0" if mu[d] > 0 else "xL"] == T.REFLECTIVE:
                A[row, iX(mx[d], j, e)] -= 1
            row += 1
        for i in range(nx):
            e = 0 if eta[d] > 0 else ny
            A[row, iY(d, e, i)] = 1
            if bc["y0" if eta[d] > 0 else "yL"] == T.REFLECTIVE:
                A[row, iY(my[d], e, i)] -= 1
            row += 1
    sol = np.linalg.solve(A, b)
    phi = np.zeros((ny, nx))
    for d in range(M):
        for j in range(ny):
            for i in range(nx):
                phi[j, i] += w[d] * 0.5 * (sol[iX(d, j, i)] + sol[iX(d, j, i + 1)])
    P = _xy(nx, ny, dx, dy, st[None], ss[None, None], Q[None], bc)
    r = T.source_iteration(P, (mu, eta, w), tol=1e-15)
    assert np.max(np.abs(r.phi[0] - phi)) < 1e-11 * np.max(phi)


def test_2d_reflective_homogeneous_k():
    # all faces reflective, uniform data: k = nu Sigma_f / Sigma_a exactly
    n = 5
    bc = {f: T.REFLECTIVE for f in ("x0", "xL", "y0", "yL")}
    P = T.XY(dx=0.4, dy=0.6, sigt=np.full((1, n, n), 1.1), sigs=np.full((1, 1, n, n), 0.6),
             nusigf=np.full((1, n, n), 0.55), chi=np.ones(1), bc=bc)
    e = T.power_iteration(P, Qd.level_symmetric_s8(), tol_k=1e-13, tol_phi=1e-11,
                          tol_inner=1e-13)
    assert abs(e.k - 0.55 / 0.5) < 1e-10


def test_2d_multigroup_infinite_medium_k():
    g = _golden("table10_multigroup_k.txt")
    S = np.stack([g["sigma_s_row_from_g1"], g["sigma_s_row_from_g2"],
                  g["sigma_s_row_from_g3"]])
    st, nsf, chi = g["sigma_t"], g["nu"] * g["sigma_f"], g["chi"]
    kinf = max(np.linalg.eigvals(np.linalg.solve(np.diag(st) - S.T, np.outer(chi, nsf))).real)
    n = 4
    bc = {f: T.REFLECTIVE for f in ("x0", "xL", "y0", "yL")}
    one = np.ones((n, n))
    P = T.XY(dx=0.5, dy=0.5, sigt=st[:, None, None] * one, sigs=S[:, :, None, None] * one,
             nusigf=nsf[:, None, None] * one, chi=chi, bc=bc)
    e = T.power_iteration(P, Qd.level_symmetric_s8(), tol_k=1e-13, tol_phi=1e-11,
                          tol_inner=1e-13)
    assert abs(e.k - kinf) < 1e-9


def test_native_sweep_loads():
    assert os.path.exists(native.build())


# ------------------------------------------------- anisotropic scattering (Eq. 25)
def _dense_dd_p1(dx, sigt, sigs, sigs1, Q, mu, w):
    """DD edge-flux system of a 1-group vacuum slab with the emission
    1/2 Sigma_s0 phi + 3/2 Sigma_s1 mu J + 1/2 Q, solved densely."""
    I, N = len(dx), len(mu)
    E = I + 1
    idx = lambda n, j: n * E + j
    A = np.zeros((N * E, N * E))
    b = np.zeros(N * E)
    row = 0
    for n in range(N):
        for i in range(I):
            A[row, idx(n, i + 1)] += mu[n] / dx[i] + sigt[i] / 2
            A[row, idx(n, i)] += -mu[n] / dx[i] + sigt[i] / 2
            for m in range(N):
                coef = 0.5 * sigs[i] * w[m] + 1.5 * sigs1[i] * mu[n] * w[m] * mu[m]
                A[row, idx(m, i)] -= coef / 2
                A[row, idx(m, i + 1)] -= coef / 2
            b[row] = 0.5 * Q[i]
            row += 1
    for n in range(N):
        A[row, idx(n, 0) if mu[n] > 0 else idx(n, I)] = 1.0
        row += 1
    e = np.linalg.solve(A, b).reshape(N, E)
    c = 0.5 * (e[:, :-1] + e[:, 1:])
    return np.sum(w[:, None] * c, axis=0), np.sum((w * mu)[:, None] * c, axis=0)


def test_anisotropic_source_iteration_matches_dense_system():
    rng = np.random.default_rng(17)
    I = 8
    dx = rng.uniform(0.2, 0.9, I)
    sigt = rng.uniform(0.6, 2.0, I)
    sigs = sigt * rng.uniform(0.2, 0.8, I)
    sigs1 = sigs * rng.uniform(-0.3, 0.6, I)
    Q = rng.uniform(0, 2, I)
    mu, w = Qd.gauss_legendre(6)
    P = T.Slab(dx=dx, sigt=sigt[None], sigs=sigs[None, None], Q=Q[None], sigs1=sigs1[None])
    r = T.source_iteration(P, (mu, w), tol=1e-15, itmax=100000)
    ref, cur = _dense_dd_p1(dx, sigt, sigs, sigs1, Q, mu, w)
    assert np.max(np.abs(r.phi[0] - ref)) < 1e-11 * np.max(ref)
    # and the anisotropic term matters here
    iso = T.source_iteration(T.Slab(dx=dx, sigt=sigt[None], sigs=sigs[None, None], Q=Q[None]),
                             (mu, w), tol=1e-15)
    assert np.max(np.abs(iso.phi[0] - ref)) > 1e-4 * np.max(ref)


def test_anisotropic_balance_and_symmetry():
    # the anisotropic emission has zero angular integral, so the particle
    # balance of the isotropic problem still holds; a symmetric slab keeps a
    # symmetric flux
    I, L = 60, 6.0
    x = (np.arange(I) + 0.5) * L / I
    sigt = 1.0 + 0.4 * np.cos(2 * np.pi * (x - L / 2) / L)
    P = T.uniform_slab(I, L, sigt, 0.7 * sigt, Q=1.0 + 0.0 * x, sigs1=0.3)
    quad = Qd.gauss_legendre(16)
    r = T.source_iteration(P, quad, tol=1e-14, itmax=200000)
    src, absorbed, leak = T.balance_1d(P, quad, r.phi, r.sweeper)
    assert abs(src - absorbed - leak) < 1e-10 * src
    assert np.max(np.abs(r.phi[0] - r.phi[0][::-1])) < 1e-11 * np.max(r.phi)
