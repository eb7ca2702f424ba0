"""Pins for the equation-recast oracle (Eq. 7/8, Eq. 24, App. A2 Eq. A5).

The recast loop is checked with the exact S_N solve at p* as the operator, so
its fixed point is known in closed form: Eq. 24 solves the transport problem
whose total cross section is Sigma_t* and whose scattering is
Sigma_s - Sigma_t + Sigma_t* (same absorption).  A sign error or dropped term
in the recast source moves that fixed point and fails the test.
"""
import numpy as np
import pytest

from oracle import quadrature as Qd
from oracle import recast as R
from oracle import transport as T
from workloads import P_STAR


def _exact_star_apply(I, L, quad):
    def factory(s):
        return T.uniform_slab(I, L, P_STAR[0], P_STAR[1], Q=s)
    return R.recast_exact_operator(factory, quad)


def test_recast_limit_is_the_equal_absorption_problem():
    I, L = 40, 10.0
    quad = Qd.gauss_legendre(8)
    rng = np.random.default_rng(1)
    x = (np.arange(I) + 0.5) * L / I
    sigt = 1.0 + 0.3 * np.sin(2 * np.pi * x / L)
    sigs = 0.6 * sigt
    S = rng.uniform(0.2, 1.0, I)
    delta = (sigs - P_STAR[1]) - (sigt - P_STAR[0])
    phi, it, st = R.recast_grid(_exact_star_apply(I, L, quad), S, delta, tol=1e-12,
                                itmax=500)
    assert st == R.OK
    eq = T.uniform_slab(I, L, P_STAR[0], sigs - sigt + P_STAR[0], Q=S)
    ref = T.source_iteration(eq, quad, tol=1e-14).phi[0]
    assert np.max(np.abs(phi - ref)) < 1e-9 * np.max(ref)
    # ... which is not the true solution: the isotropic approximation (Eq. 23)
    true = T.source_iteration(T.uniform_slab(I, L, sigt, sigs, Q=S), quad, tol=1e-14).phi[0]
    assert np.max(np.abs(true - ref)) > 1e-4 * np.max(ref)


def test_recast_at_p_star_is_one_operator_application():
    I, L = 20, 10.0
    quad = Qd.gauss_legendre(8)
    S = np.linspace(0.1, 1.0, I)
    apply = _exact_star_apply(I, L, quad)
    phi, it, st = R.recast_grid(apply, S, np.zeros(I), tol=1e-12)
    assert st == R.OK and it == 2
    assert np.max(np.abs(phi - apply(S[None])[0])) < 1e-14


def test_split_scaling_is_exact_for_a_linear_operator():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((9, 9))
    lin = lambda U: U @ A.T
    s = rng.standard_normal((4, 9))
    s[1] = np.abs(s[1])
    s[2] = -np.abs(s[2])
    s[3] = 0.0
    out = R._split_apply(lin, s, 0.3)
    assert np.max(np.abs(out - s @ A.T)) < 1e-12


def test_projection_preserves_integrals():
    rng = np.random.default_rng(4)
    for I in (64, 100, 128, 333, 2048):
        edges = np.linspace(0, 10.0, I + 1)
        P = R.projection_matrix(edges, 128, 10.0)
        assert np.allclose(P.sum(axis=1), 1.0)
        f = rng.uniform(0, 1, I)
        assert abs(np.sum(P @ f) * 10.0 / 128 - np.sum(f * np.diff(edges))) < 1e-12


def test_recast_detects_divergence():
    # an operator with gain 2: the recast change grows and the loop gives up
    apply = lambda U: 2.0 * U
    phi, it, st = R.recast_grid(apply, np.ones(5), np.ones(5), tol=1e-8, itmax=200)
    assert st == R.DIVERGED and it < 20


def test_warm_start_does_not_change_the_answer():
    I, L = 50, 10.0
    quad = Qd.gauss_legendre(16)
    rng = np.random.default_rng(5)
    x = (np.arange(I) + 0.5) * L / I
    sigt = 1.0 + 0.4 * np.sin(2 * np.pi * 2 * x / L)
    P = T.uniform_slab(I, L, sigt, 0.8 * sigt, Q=rng.uniform(0, 1, I))
    delta = (P.sigs[0, 0] - P_STAR[1]) - (P.sigt[0] - P_STAR[0])
    phi_no, _, st = R.recast_grid(_exact_star_apply(I, L, quad), P.Q[0], delta,
                                  tol=1e-6)
    cold = T.source_iteration(P, quad, tol=1e-12)
    warm = T.source_iteration(P, quad, phi0=phi_no[None], tol=1e-12)
    assert warm.iterations < cold.iterations
    assert np.max(np.abs(warm.phi - cold.phi)) < 1e-9 * np.max(cold.phi)


def test_sp_eigen_with_exact_operator_at_p_star():
    # at p = p* the exact operator makes SP an ordinary power iteration with
    # fully converged inner solves, so it reaches the model-based k
    I, L = 40, 10.0
    quad = Qd.gauss_legendre(8)
    P = T.uniform_slab(I, L, P_STAR[0], P_STAR[1], nusigf=0.7)
    k, phi, n, st = R.sp_eigen(P, _exact_star_apply(I, L, quad), P_STAR,
                               tol_k=1e-11, tol_phi=1e-9)
    e = T.power_iteration(P, quad, tol_k=1e-12, tol_phi=1e-10, tol_inner=1e-13)
    assert st == R.OK
    assert abs(k - e.k) < 1e-9
    assert np.max(np.abs(phi - e.phi)) < 1e-7 * np.max(e.phi)


def test_cp_eigen_with_exact_operator_at_p_star():
    # App. A2 Eq. A7-A8: with the exact operator at p = p* the true eigenpair
    # is a fixed point of the constrained step (the prediction reproduces it
    # and one source iteration leaves it unchanged), so CP reaches the
    # model-based k and flux
    I, L = 40, 10.0
    quad = Qd.gauss_legendre(8)
    x = (np.arange(I) + 0.5) * L / I
    nsf = 0.5 + 0.4 * np.sin(np.pi * x / L)
    P = T.uniform_slab(I, L, P_STAR[0], P_STAR[1], nusigf=nsf)
    k, phi, n, st = R.cp_eigen(P, _exact_star_apply(I, L, quad), P_STAR, quad,
                               tol_k=1e-11, tol_phi=1e-9)
    e = T.power_iteration(P, quad, tol_k=1e-12, tol_phi=1e-10, tol_inner=1e-13)
    assert st == R.OK
    assert abs(k - e.k) < 1e-9
    assert np.max(np.abs(phi - e.phi)) < 1e-7 * np.max(e.phi)


def test_cp_refinement_is_one_model_iteration():
    # with an operator that returns its input unchanged the prediction is the
    # recast source itself; the constrained step must then equal one source
    # iteration from that prediction with its own fission source.  A CP step
    # that skipped the refinement, or refined from phi^n instead, fails.
    I, L = 30, 10.0
    quad = Qd.gauss_legendre(8)
    x = (np.arange(I) + 0.5) * L / I
    P = T.uniform_slab(I, L, 1.0 + 0.2 * np.cos(x), 0.4 + 0.1 * np.sin(x), nusigf=0.6)
    ident = lambda S: np.array(S, float)
    k1, phi1, n, st = R.cp_eigen(P, ident, P_STAR, quad, tol_k=0.0, tol_phi=0.0, itmax=1)
    phi0 = np.ones((1, I)) / T.production(P, np.ones((1, I)))
    delta = (P.sigs[0, 0] - P_STAR[1]) - (P.sigt[0] - P_STAR[0])
    quarter = (P.nusigf[0] * phi0[0] * 1.0 + delta * phi0[0])[None]
    src = P.nusigf * quarter
    half = T.source_iteration(P, quad, src=src, phi0=quarter, tol=0.0, itmax=1).phi
    Pn = T.production(P, half)
    assert abs(k1 - Pn) < 1e-12
    assert np.max(np.abs(phi1 - half / Pn)) < 1e-12 * np.max(np.abs(half / Pn))
