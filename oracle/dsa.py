"""Diffusion synthetic acceleration of slab source iteration, FP64 (TEST
INFRASTRUCTURE ONLY, see oracle/__init__.py).

Not part of the paper's method.  The paper accelerates the unchanged
iteration operator M of Sec. 3.1 (Eq. 3a/4b) with a better first iterate and
contrasts this with schemes that change the iteration itself (Sec. 3.3).
Diffusion synthetic acceleration is the classical scheme of that second kind
for the one-group slab equation of Sec. 5.1 (Eq. 12); it is here so that both
can be compared on the same workloads.

After the sweep of group g has turned phi^l into phi^{l+1/2}, the error of
phi^{l+1/2} obeys the transport equation with the source
R = Sigma_s,gg (phi^{l+1/2} - phi^l).  It is approximated by the P1
equations written with the same diamond-difference closure as the sweep:
with psi = (phi + 3 mu J) / 2 inserted into the DD cell equations, the
zeroth and first angular moments over cell i (width h_i) read

    J_{i+1/2} - J_{i-1/2} + Sigma_a,i h_i phi_i = h_i R_i
    (phi_{i+1/2} - phi_{i-1/2}) / 3 + Sigma_t,i h_i J_i = 0
    phi_i = (phi_{i-1/2} + phi_{i+1/2}) / 2,   J_i = (J_{i-1/2} + J_{i+1/2}) / 2

(Sigma_a = Sigma_t - Sigma_s,gg, the in-group removal).  Eliminating the
currents leaves one symmetric equation per edge: the sum over the (at most
two) cells touching the edge of the cell matrices

    K_i = D_i / h_i [[1, -1], [-1, 1]] + Sigma_a,i h_i / 4 [[1, 1], [1, 1]],
    D_i = 1 / (3 Sigma_t,i),

acting on the cell's two edge values, equal to h_i R_i / 2 from each cell.
Faces: a vacuum face has no incoming flux; its half-range current moment
with the P1 flux gives J = -/+ a phi with a = sum_{mu_n > 0} w_n mu_n (the
quadrature's own half-range current, 1/2 in the limit), which adds a to the
face edge's diagonal; a reflective face has J = 0 and adds nothing.  The cell
correction is f_i = (e_{i-1/2} + e_{i+1/2}) / 2 and phi^{l+1} = phi^{l+1/2}
+ f.  The stored outgoing angular flux of a reflective face, which the next
sweep reads as its incoming flux, receives the isotropic part e_face / 2 of
the correction.

Once the iterates stop changing, R = 0 and the corrections vanish: the
converged flux is the source-iteration answer.

A reflective right face is lagged by the sweep order (the mu < 0 sweep
enters with the mu > 0 outflow of the previous iteration); the error that
this lag carries is not a P1 shape, and the correction leaves it to the
sweeps, so such slabs converge somewhat slower than the Fourier-analysis
rate of an unbounded medium.
"""
import numpy as np
from scipy.linalg import solve_banded

from . import transport as T


def half_range_current(mu, w):
    """a = sum over mu_n > 0 of w_n mu_n (weights summing to 2)."""
    mu, w = np.asarray(mu, float), np.asarray(w, float)
    return float(np.sum(w[mu > 0] * mu[mu > 0]))


def edge_matrix(dx, sigt, siga, a_left, a_right):
    """Banded (upper, diagonal, lower) form of the (I+1)-edge system.

    a_left / a_right: the face terms added to the first / last diagonal entry
    (the half-range current a for a vacuum face, 0 for a reflective one).
    """
    dx, sigt, siga = (np.asarray(v, float) for v in (dx, sigt, siga))
    I = len(dx)
    diff = 1.0 / (3.0 * sigt * dx)          # D_i / h_i
    mass = siga * dx / 4.0
    diag = np.zeros(I + 1)
    off = np.zeros(I)                        # entry (i, i+1) = entry (i+1, i)
    for i in range(I):
        diag[i] += diff[i] + mass[i]
        diag[i + 1] += diff[i] + mass[i]
        off[i] += -diff[i] + mass[i]
    diag[0] += a_left
    diag[I] += a_right
    ab = np.zeros((3, I + 1))
    ab[0, 1:] = off
    ab[1] = diag
    ab[2, :-1] = off
    return ab


def edge_load(dx, R):
    """Right-hand side: h_i R_i / 2 to each of the two edges of cell i."""
    dx, R = np.asarray(dx, float), np.asarray(R, float)
    b = np.zeros(len(dx) + 1)
    b[:-1] += 0.5 * dx * R
    b[1:] += 0.5 * dx * R
    return b


def edge_correction(prob, g, R, quad):
    """Edge corrections e (I+1 values) of group g for the residual source R."""
    mu, w = quad
    a = half_range_current(mu, w)
    aL = a if prob.bc_left == T.VACUUM else 0.0
    aR = a if prob.bc_right == T.VACUUM else 0.0
    siga = prob.sigt[g] - prob.sigs[g, g]
    ab = edge_matrix(prob.dx, prob.sigt[g], siga, aL, aR)
    return solve_banded((1, 1), ab, edge_load(prob.dx, R))


def correct(prob, g, phi_half, phi_old, quad, sweeper):
    """One DSA correction of group g; returns phi^{l+1} and updates the
    stored reflective-face angular fluxes of `sweeper` in place."""
    R = prob.sigs[g, g] * (phi_half - phi_old)
    e = edge_correction(prob, g, R, quad)
    if prob.bc_left == T.REFLECTIVE:
        sweeper.out_left[g][sweeper.neg] += 0.5 * e[0]
    if prob.bc_right == T.REFLECTIVE:
        sweeper.out_right[g][sweeper.pos] += 0.5 * e[-1]
    return phi_half + 0.5 * (e[:-1] + e[1:])
