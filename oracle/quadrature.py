"""Angular quadratures for the oracle (TEST INFRASTRUCTURE ONLY).

1D: Gauss-Legendre S_N (the slab quadrature of the S_N method, Sec. 5.1; N=32
in the paper's benchmark solver).  Weights sum to 2 so that phi = sum w psi is
the integral of psi over mu in [-1, 1], matching Eq. 17.

2D: level-symmetric S8 on the x-y plane (the paper's Sec. 6 remark that the
method extends to higher dimensions; the 2D workload uses S8).  The set is
derived here from its definition, not copied from a table:
  * levels: mu_i^2 = mu_1^2 + (i-1) * 2 (1 - 3 mu_1^2) / (N - 2), i = 1..N/2;
  * points in an octant: (mu_i, mu_j, mu_k) with i + j + k = N/2 + 2;
  * one weight per permutation class, fixed by the even-moment conditions
    <1> = 1, <mu^4> = 1/5, <mu^6> = 1/7 over the octant (odd moments vanish by
    symmetry and <mu^2> = 1/3 follows from mu^2 + eta^2 + xi^2 = 1);
  * mu_1 is the root that also makes <mu^8> = 1/9 exact.
The 2D set keeps the upper hemisphere (xi > 0) with weights doubled (the
lower hemisphere mirrors it in x-y geometry), normalised so that the 40
weights sum to 1: phi = sum_d w_d psi_d and the isotropic emission density is
(Sigma_s phi + Q), the 2D counterpart of the 1D (1/2)(Sigma_s phi + Q) with
sum w = 2.
Direction order: quadrants (mu<0, eta<0), (mu>0, eta<0), (mu<0, eta>0),
(mu>0, eta>0); inside a quadrant, octant points in lexicographic (i, j) order.
"""
import numpy as np


def gauss_legendre(N):
    """Gauss-Legendre nodes (ascending) and weights on [-1, 1]; sum(w) == 2."""
    if N < 2 or N % 2:
        raise ValueError("S_N order must be even and >= 2")
    mu, w = np.polynomial.legendre.leggauss(N)
    return mu, w


def _ls_octant(mu1sq, N):
    delta = 2.0 * (1.0 - 3.0 * mu1sq) / (N - 2)
    levels = np.sqrt(mu1sq + delta * np.arange(N // 2))
    pts = [(i, j, k) for i in range(1, N // 2 + 1) for j in range(1, N // 2 + 1)
           for k in range(1, N // 2 + 1) if i + j + k == N // 2 + 2]
    classes = sorted(set(tuple(sorted(p)) for p in pts))
    return levels, pts, classes


def _ls_weights(mu1sq, N):
    levels, pts, classes = _ls_octant(mu1sq, N)
    A = np.zeros((3, len(classes)))
    rhs = np.array([1.0, 1.0 / 5.0, 1.0 / 7.0])
    for r, p in enumerate((0, 4, 6)):
        for c, cl in enumerate(classes):
            A[r, c] = sum(levels[t[0] - 1] ** p for t in pts if tuple(sorted(t)) == cl)
    wc = np.linalg.solve(A, rhs)
    w = np.array([wc[classes.index(tuple(sorted(t)))] for t in pts])
    return levels, pts, w


def _ls_m8(mu1sq, N):
    levels, pts, w = _ls_weights(mu1sq, N)
    return sum(wi * levels[t[0] - 1] ** 8 for wi, t in zip(w, pts)) - 1.0 / 9.0


def level_symmetric_s8():
    """Return (mu, eta, w), 40 directions of the folded 2D S8 set, sum(w) == 1."""
    N = 8
    # bisection for <mu^8> = 1/9 on the bracket where all weights stay positive
    lo, hi = 0.03, 0.06
    flo = _ls_m8(lo, N)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        fm = _ls_m8(mid, N)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    mu1sq = 0.5 * (lo + hi)
    levels, pts, w_oct = _ls_weights(mu1sq, N)
    mus, etas, ws = [], [], []
    for sx, sy in ((-1, -1), (1, -1), (-1, 1), (1, 1)):
        for (i, j, k), wo in zip(pts, w_oct):
            mus.append(sx * levels[i - 1])
            etas.append(sy * levels[j - 1])
            # sphere weight wo/8 per direction, doubled for the folded hemisphere
            ws.append(wo / 4.0)
    return np.array(mus), np.array(etas), np.array(ws)


def xi_of(mu, eta):
    """Polar cosine of each 2D direction (the folded z component)."""
    return np.sqrt(np.maximum(0.0, 1.0 - mu * mu - eta * eta))
