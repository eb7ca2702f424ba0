"""FP64 oracle of the diffusion recast (Sec. 3.1 Eq. 6a-8, Table 1): a second
PDE on the same recast driver as the transport solve.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Problem.  -(D u')' + Sigma_a u = S on (0, L) with u = 0 at both faces.  Table
1's diffusion row is Sigma_a = 0 with parameter p = D(x); its Helmholtz row,
-u'' - k^2 u = S with p = k^2, is D = 1 and Sigma_a = -k^2.  Table 1 writes
the diffusion mismatch as grad(D - D*) . grad u + (D - D*) lap u, i.e.
((D - D*) u')'; both rows are the operator difference
dL = L(p) - L(p*) moved to the source side (Eq. 6b-7a).

Readings where the paper is silent (the CUDA side does the same):
  * discretisation: cell-centred finite volumes on uniform cells; the face
    coefficient is the harmonic mean D_{i+1/2} = 2 D_i D_{i+1} / (D_i +
    D_{i+1}) (continuous flux across a face), and a boundary face sits half a
    cell from its centre (flux 2 D_0 u_0 / h at x = 0).  Row i of the system:
        (a_w + a_e + Sigma_a,i) u_i - a_w u_{i-1} - a_e u_{i+1} = S_i,
    a_w = D_{i-1/2} / h^2 (2 D_0 / h^2 at the left face), a_e likewise.
  * the operator difference is taken between the discrete operators (direct
    subtraction, the case Table 1's discussion names), so the recast with the
    exact p* solve as its operator converges to the exact discrete solution
    of L(p) u = S (no approximation as in Sec. 5.1 Eq. 23 for transport).
  * the DeepONet recast runs on the operator's M-bin grid like the transport
    one (oracle/recast.py): D, Sigma_a and S reach the bins by the
    overlap-weighted average, the bin-grid operators of p and p* are built
    with the same finite-volume formulas, and the recast source is
    s - dL_bins u on the bins; stopping, divergence test, split scaling and
    the final evaluation at cell centres are those of the transport recast.
"""
import numpy as np
from scipy.linalg import solve_banded

from . import recast as R
from . import transport as T


def fv_bands(h, D, siga):
    """(lower, diag, upper) of the finite-volume operator on cells of width h:
    row i reads lower[i] u_{i-1} + diag[i] u_i + upper[i] u_{i+1}."""
    D = np.asarray(D, float)
    siga = np.broadcast_to(np.asarray(siga, float), D.shape)
    I = D.size
    face = np.empty(I + 1)                       # face coefficients D_{i-1/2}, i = 0..I
    face[0] = 2.0 * D[0]
    face[I] = 2.0 * D[-1]
    face[1:I] = 2.0 * D[:-1] * D[1:] / (D[:-1] + D[1:])
    aw, ae = face[:-1] / h ** 2, face[1:] / h ** 2
    lower = -aw.copy()
    upper = -ae.copy()
    lower[0] = 0.0
    upper[-1] = 0.0
    return lower, aw + ae + siga, upper


def apply_bands(bands, u):
    lower, diag, upper = bands
    out = diag * u
    out[1:] += lower[1:] * u[:-1]
    out[:-1] += upper[:-1] * u[1:]
    return out


def solve(h, D, siga, S):
    """The discrete solution of -(D u')' + Sigma_a u = S, u = 0 at the faces."""
    lower, diag, upper = fv_bands(h, D, siga)
    ab = np.zeros((3, diag.size))
    ab[0, 1:] = upper[:-1]
    ab[1] = diag
    ab[2, :-1] = lower[1:]
    return solve_banded((1, 1), ab, np.asarray(S, float))


def mismatch_bands(h, D, siga, d_star, siga_star):
    """Bands of dL = L(D, Sigma_a) - L(D*, Sigma_a*) (constant p*)."""
    lo, di, up = fv_bands(h, D, siga)
    one = np.ones_like(np.asarray(D, float))
    ls, ds, us = fv_bands(h, d_star * one, siga_star)
    return lo - ls, di - ds, up - us


def recast_exact(h, D, siga, S, p_star, tol=1e-13, itmax=10000):
    """Eq. 7 with the exact p* solve as the operator: u <- L*^{-1}[S - dL u].
    Returns (u, iterations)."""
    d_star, siga_star = p_star
    dl = mismatch_bands(h, D, siga, d_star, siga_star)
    one = np.ones_like(np.asarray(D, float))
    u = np.zeros_like(one)
    it = 0
    for it in range(1, itmax + 1):
        u_new = solve(h, d_star * one, siga_star, np.asarray(S, float) - apply_bands(dl, u))
        ch = T.rel_change(u_new, u)
        u = u_new
        if ch <= tol:
            break
    return u, it


def recast_deeponet(op, L, D, siga, S, p_star, tol=1e-4, itmax=200):
    """Eq. 8 for one diffusion slab with a DeepONet operator trained at p*.

    D, siga, S are cell values on uniform cells over [0, L].  Returns (u_NO on
    the cells, iterations, status, beta)."""
    I = len(D)
    edges = np.linspace(0.0, L, I + 1)
    P = R.projection_matrix(edges, op.M, L)
    hb = L / op.M
    s = P @ np.asarray(S, float)
    dl = mismatch_bands(hb, P @ np.asarray(D, float), P @ np.broadcast_to(siga, (I,)),
                        *p_star)
    Tref = op.trunk(op.xb)
    u = np.zeros(op.M)
    beta = np.zeros(Tref.shape[1])
    status, it = R.NOCONV, 0
    prev, run = np.inf, 0
    for it in range(1, itmax + 1):
        src = s - apply_bands(dl, u)
        beta = op.coef(src[None])[0]
        u_new = op.quant(beta) @ op.quant(Tref).T
        if not np.all(np.isfinite(u_new)):
            status = R.DIVERGED
            break
        ch = T.rel_change(u_new, u)
        ab = float(np.sqrt(np.sum((u_new - u) ** 2)))
        u = u_new
        if ch <= tol:
            status = R.OK
            break
        run = run + 1 if ab >= prev else 0
        prev = ab
        if run >= R.DIVERGE_RUN:
            status = R.DIVERGED
            break
    xc = (edges[:-1] + edges[1:]) / 2 / L
    return op.eval(beta[None], xc)[0], it, status, beta
