"""Pins of the diffusion-recast oracle (oracle/diffusion.py; Sec. 3.1 Table 1)
against what the mathematics fixes, not against itself."""
import numpy as np
import pytest

import workloads as W
from oracle import diffusion as DF
from oracle import neural as NN
from oracle import recast as R


def _err(I, D, siga, S_of, u_of, L=10.0):
    h = L / I
    x = (np.arange(I) + 0.5) * h
    u = DF.solve(h, D * np.ones(I), siga, S_of(x))
    return np.max(np.abs(u - u_of(x))) / np.max(np.abs(u_of(x)))


def test_uniform_pure_diffusion_parabola_second_order():
    # -D u'' = 1, u(0) = u(L) = 0:  u = x (L - x) / (2 D)
    L, D = 10.0, 1.7
    e = [_err(I, D, 0.0, lambda x: np.ones_like(x), lambda x: x * (L - x) / (2 * D))
         for I in (50, 100, 200)]
    assert e[0] < 1e-2
    assert 3.6 < e[0] / e[1] < 4.4 and 3.6 < e[1] / e[2] < 4.4


def test_absorbing_sine_mode_second_order():
    # -D u'' + Sa u = (D pi^2 / L^2 + Sa) sin(pi x / L):  u = sin(pi x / L)
    L, D, Sa = 10.0, 0.8, 0.3
    k2 = (np.pi / L) ** 2
    e = [_err(I, D, Sa, lambda x: (D * k2 + Sa) * np.sin(np.pi * x / L),
              lambda x: np.sin(np.pi * x / L)) for I in (40, 80, 160)]
    assert e[0] < 1e-3
    assert 3.6 < e[0] / e[1] < 4.4 and 3.6 < e[1] / e[2] < 4.4


def test_helmholtz_row_sine_mode():
    # Table 1 Helmholtz: -u'' - k^2 u = S with D = 1, Sigma_a = -k^2 (k^2 below
    # the first Dirichlet eigenvalue, so the operator stays positive definite)
    L, kk = 10.0, 0.05
    k2 = (np.pi / L) ** 2
    e = [_err(I, 1.0, -kk, lambda x: (k2 - kk) * np.sin(np.pi * x / L),
              lambda x: np.sin(np.pi * x / L)) for I in (40, 80)]
    assert e[0] < 2e-3 and 3.6 < e[0] / e[1] < 4.4


def test_banded_system_is_the_face_flux_assembly():
    # an independent dense assembly face by face: a face between cells i and
    # i+1 carries the flux D_f (u_i - u_{i+1}) / h with D_f the harmonic mean;
    # a boundary face carries 2 D u / h (the face value is 0, half a cell away)
    rng = np.random.default_rng(1)
    I, h = 9, 0.37
    D = rng.uniform(0.2, 3.0, I)
    Sa = rng.uniform(-0.1, 0.5, I)
    A = np.diag(Sa * h)
    for i in range(I - 1):
        df = 2 * D[i] * D[i + 1] / (D[i] + D[i + 1]) / h
        A[i, i] += df
        A[i + 1, i + 1] += df
        A[i, i + 1] -= df
        A[i + 1, i] -= df
    A[0, 0] += 2 * D[0] / h
    A[-1, -1] += 2 * D[-1] / h
    S = rng.uniform(0, 1, I)
    ref = np.linalg.solve(A, S * h)
    assert np.allclose(DF.solve(h, D, Sa, S), ref, rtol=1e-12, atol=1e-14)


def test_particle_balance():
    # integrating over the slab: source = absorption + leakage through both faces
    rng = np.random.default_rng(2)
    I, L = 120, 10.0
    h = L / I
    D = rng.uniform(0.5, 2.0, I)
    Sa = rng.uniform(0.0, 0.4, I)
    S = rng.uniform(0.0, 2.0, I)
    u = DF.solve(h, D, Sa, S)
    leak = 2 * D[0] * u[0] / h + 2 * D[-1] * u[-1] / h
    assert abs(np.sum(S) * h - (np.sum(Sa * u) * h + leak)) < 1e-11 * np.sum(S) * h


def test_recast_with_the_exact_operator_is_the_exact_solution():
    # Eq. 7 with N = exact solve at p*: the fixed point solves L(p) u = S
    # exactly, because dL is the difference of the discrete operators
    x = W.cell_centres(200)
    D = 1.0 + 0.5 * np.sin(2 * np.pi * 3 * x / 10.0)
    Sa = 0.05 + 0.04 * np.cos(2 * np.pi * x / 10.0)
    S = W.fourier_source(np.random.default_rng(3), x)
    h = 10.0 / 200
    u, it = DF.recast_exact(h, D, Sa, S, (1.0, 0.05), tol=1e-13)
    ref = DF.solve(h, D, Sa, S)
    assert it > 3 and np.max(np.abs(u - ref)) < 1e-10 * np.max(np.abs(ref))


def test_mismatch_vanishes_at_p_star_and_the_recast_is_one_application():
    # D = D*, Sigma_a = Sigma_a*: dL = 0, and the DeepONet recast is N[S]
    P = W.deeponet_init(4, m=32, width=16, p=8)
    op = R.DeepONetOp(P, 10.0, 32)
    I = 64
    S = W.fourier_source(np.random.default_rng(5), W.cell_centres(I))
    lo, di, up = DF.mismatch_bands(10.0 / 32, np.full(32, 1.3), 0.2, 1.3, 0.2)
    assert np.all(lo == 0) and np.all(di == 0) and np.all(up == 0)
    u, it, st, beta = DF.recast_deeponet(op, 10.0, np.full(I, 1.3), np.full(I, 0.2), S,
                                         (1.3, 0.2), tol=1e-12, itmax=5)
    edges = np.linspace(0, 10.0, I + 1)
    ref = op.coef((R.projection_matrix(edges, 32, 10.0) @ S)[None])[0]
    assert it == 2 and np.allclose(beta, ref, rtol=1e-13, atol=1e-15)
