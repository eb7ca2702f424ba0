"""FP64 S_N transport oracle: source iteration and power iteration.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows the paper's model-based solver:
  * fixed source, Sec. 5.1 Eq. 12 (1D slab, isotropic scattering, isotropic
    source S entering as S/2) solved by source iteration, the iteration
    operator M of Eq. 3a/4b (Sec. 3.1) and Eq. 20;
  * k-eigenvalue, Sec. 5.2 Eq. 26 and App. A2 Eq. A2-A4: an inner source
    iteration M with the fission source frozen, and an outer update P that
    recomputes k from the production rate and renormalises the flux;
  * multigroup, Sec. 5.3 Eq. 27-29: group-to-group scattering and the
    chi-weighted fission source enter each group's equation as sources;
  * linearly anisotropic in-group scattering, Sec. 5.1 Eq. 25 (1D fixed
    source): the emission of direction mu adds (3/2) Sigma_s1 mu J, with the
    current J = sum w mu psi of the previous source iteration (zero at first).

Readings where the paper is silent (identical on the CUDA side):
  * spatial scheme: diamond difference, no negative-flux fix-up;
  * one source iteration visits groups 0..G-1 in order and each group's
    scattering source uses the newest flux of every group (Gauss-Seidel in
    energy); with one group this is plain source iteration;
  * boundary conditions: vacuum (no incoming flux) or reflective (incoming
    flux = outgoing flux of the mirror direction on that face, taken from the
    most recent sweep of the mirror direction).  Directions are swept in a
    fixed order: 1D mu<0 then mu>0; 2D quadrants (-,-), (+,-), (-,+), (+,+);
  * convergence: ||phi_new - phi_old||_2 / ||phi_new||_2 over all cells and
    groups (relative L2 change between successive iterates);
  * eigen: flux normalised so that the production integral
    sum_{g,i} nuSigma_f phi vol = 1; k_{n+1} = k_n * production(phi_{n+1/2});
    boundary angular fluxes are rescaled with the flux; the inner iteration
    starts from the current normalised flux and runs to its own tolerance.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import native

VACUUM, REFLECTIVE = "vacuum", "reflective"


@dataclass
class Slab:
    """1D slab problem.  Arrays are group-major: sigt[g, i]."""
    dx: np.ndarray                 # (I,) cell widths
    sigt: np.ndarray               # (G, I)
    sigs: np.ndarray               # (G, G, I): sigs[gp, g, i] scatters gp -> g
    Q: Optional[np.ndarray] = None       # (G, I) isotropic external source S
    nusigf: Optional[np.ndarray] = None  # (G, I) production nu*Sigma_f
    chi: Optional[np.ndarray] = None     # (G,) fission spectrum
    bc_left: str = VACUUM
    bc_right: str = VACUUM
    # (G, I) first Legendre moment of the in-group scattering, Sec. 5.1 Eq. 25
    # (linearly anisotropic emission); None: isotropic scattering
    sigs1: Optional[np.ndarray] = None

    @property
    def G(self):
        return self.sigt.shape[0]

    @property
    def vol(self):
        return self.dx


@dataclass
class XY:
    """2D x-y problem on a uniform nx-by-ny mesh.  Arrays are [g, j, i]."""
    dx: float
    dy: float
    sigt: np.ndarray               # (G, ny, nx)
    sigs: np.ndarray               # (G, G, ny, nx)
    Q: Optional[np.ndarray] = None
    nusigf: Optional[np.ndarray] = None
    chi: Optional[np.ndarray] = None
    bc: dict = field(default_factory=lambda: {"x0": VACUUM, "xL": VACUUM,
                                              "y0": VACUUM, "yL": VACUUM})

    @property
    def G(self):
        return self.sigt.shape[0]

    @property
    def vol(self):
        return np.full(self.sigt.shape[1:], self.dx * self.dy)


def uniform_slab(I, L, sigt, sigs, Q=None, nusigf=None, chi=None,
                 bc_left=VACUUM, bc_right=VACUUM, sigs1=None):
    """Slab of I equal cells over width L; scalar or per-cell coefficients, 1 group."""
    one = np.ones(I)
    P = Slab(dx=np.full(I, L / I),
             sigt=(np.asarray(sigt, float) * one)[None, :],
             sigs=(np.asarray(sigs, float) * one)[None, None, :],
             bc_left=bc_left, bc_right=bc_right)
    if sigs1 is not None:
        P.sigs1 = (np.asarray(sigs1, float) * one)[None, :]
    if Q is not None:
        P.Q = (np.asarray(Q, float) * one)[None, :]
    if nusigf is not None:
        P.nusigf = (np.asarray(nusigf, float) * one)[None, :]
        P.chi = np.ones(1) if chi is None else np.asarray(chi, float)
    return P


def _mirror(a):
    """Index of the direction with the opposite sign of a[n] (symmetric sets)."""
    idx = np.empty(len(a), dtype=int)
    for n in range(len(a)):
        m = int(np.argmin(np.abs(a + a[n])))
        if abs(a[m] + a[n]) > 1e-12 * max(1.0, abs(a[n])):
            raise ValueError("quadrature set is not symmetric")
        idx[n] = m
    return idx


class _Sweeper1D:
    """One group's transport sweep with the boundary state of Sec. 5 slabs."""

    def __init__(self, prob, mu, w):
        self.p, self.mu, self.w = prob, np.asarray(mu, float), np.asarray(w, float)
        self.neg = np.where(self.mu < 0)[0]
        self.pos = np.where(self.mu > 0)[0]
        self.mir = _mirror(self.mu)
        G, N = prob.G, len(self.mu)
        self.out_left = np.zeros((G, N))    # valid for mu < 0
        self.out_right = np.zeros((G, N))   # valid for mu > 0

    def emission(self, scat_plus_src):
        return 0.5 * scat_plus_src          # Eq. 12: (1/2)(Sigma_s phi + S)

    def sweep(self, g, q):
        p, mu, w = self.p, self.mu, self.w
        neg, pos, mir = self.neg, self.pos, self.mir
        in_r = np.zeros(len(neg))
        if p.bc_right == REFLECTIVE:
            in_r = self.out_right[g][mir[neg]]
        phi_n, out_l, _ = native.sweep1d(p.dx, p.sigt[g], q, mu[neg], w[neg],
                                         np.zeros(len(neg)), in_r)
        self.out_left[g][neg] = out_l
        in_l = np.zeros(len(pos))
        if p.bc_left == REFLECTIVE:
            in_l = self.out_left[g][mir[pos]]
        phi_p, _, out_r = native.sweep1d(p.dx, p.sigt[g], q, mu[pos], w[pos],
                                         in_l, np.zeros(len(pos)))
        self.out_right[g][pos] = out_r
        return phi_n + phi_p

    def sweep_p1(self, g, q0, q1):
        """Sweep with the emission q0 + mu q1 of Eq. 25; returns (phi, current)."""
        p, mu, w = self.p, self.mu, self.w
        neg, pos, mir = self.neg, self.pos, self.mir
        in_r = np.zeros(len(neg))
        if p.bc_right == REFLECTIVE:
            in_r = self.out_right[g][mir[neg]]
        phi_n, cur_n, out_l, _ = native.sweep1d_p1(p.dx, p.sigt[g], q0, q1, mu[neg], w[neg],
                                                   np.zeros(len(neg)), in_r)
        self.out_left[g][neg] = out_l
        in_l = np.zeros(len(pos))
        if p.bc_left == REFLECTIVE:
            in_l = self.out_left[g][mir[pos]]
        phi_p, cur_p, _, out_r = native.sweep1d_p1(p.dx, p.sigt[g], q0, q1, mu[pos], w[pos],
                                                   in_l, np.zeros(len(pos)))
        self.out_right[g][pos] = out_r
        return phi_n + phi_p, cur_n + cur_p

    def scale(self, s):
        self.out_left *= s
        self.out_right *= s


class _SweeperXY:
    QUADRANTS = ((-1, -1), (1, -1), (-1, 1), (1, 1))

    def __init__(self, prob, mu, eta, w):
        self.p = prob
        self.mu, self.eta, self.w = (np.asarray(a, float) for a in (mu, eta, w))
        G, (ny, nx), M = prob.G, prob.sigt.shape[1:], len(self.mu)
        # mirror across an x-face flips mu, across a y-face flips eta
        self.mir_x = np.array([self._find(-self.mu[d], self.eta[d]) for d in range(M)])
        self.mir_y = np.array([self._find(self.mu[d], -self.eta[d]) for d in range(M)])
        self.out_x = np.zeros((G, M, ny))
        self.out_y = np.zeros((G, M, nx))

    def _find(self, m, e):
        d = int(np.argmin(np.abs(self.mu - m) + np.abs(self.eta - e)))
        if abs(self.mu[d] - m) + abs(self.eta[d] - e) > 1e-12:
            raise ValueError("2D quadrature set is not reflection-symmetric")
        return d

    def emission(self, scat_plus_src):
        return scat_plus_src               # sum w = 1 over the 2D set

    def sweep(self, g, q):
        p = self.p
        ny, nx = p.sigt.shape[1:]
        phi = np.zeros((ny, nx))
        for sx, sy in self.QUADRANTS:
            ds = np.where((np.sign(self.mu) == sx) & (np.sign(self.eta) == sy))[0]
            in_x = np.zeros((len(ds), ny))
            in_y = np.zeros((len(ds), nx))
            xface = "x0" if sx > 0 else "xL"
            yface = "y0" if sy > 0 else "yL"
            if p.bc[xface] == REFLECTIVE:
                in_x = self.out_x[g][self.mir_x[ds]]
            if p.bc[yface] == REFLECTIVE:
                in_y = self.out_y[g][self.mir_y[ds]]
            ph, ox, oy = native.sweep2d(p.dx, p.dy, p.sigt[g], q, self.mu[ds],
                                        self.eta[ds], self.w[ds], in_x, in_y)
            self.out_x[g][ds] = ox
            self.out_y[g][ds] = oy
            phi += ph
        return phi

    def scale(self, s):
        self.out_x *= s
        self.out_y *= s


def make_sweeper(prob, quad):
    if isinstance(prob, Slab):
        return _Sweeper1D(prob, *quad)
    return _SweeperXY(prob, *quad)


@dataclass
class SIResult:
    phi: np.ndarray
    iterations: int
    change: float
    history: list
    sweeper: object = None


def rel_change(new, old):
    nn = np.sqrt(np.sum(new * new))
    return np.sqrt(np.sum((new - old) ** 2)) / nn if nn > 0 else 0.0


def source_iteration(prob, quad, src=None, phi0=None, tol=1e-10, itmax=100000,
                     sweeper=None, history=False, dsa=False):
    """Source iteration (the operator M of Eq. 3a/4b, Eq. 20) to ||dphi||/||phi|| <= tol.

    ``src`` is the isotropic source S per group (default prob.Q); ``phi0`` the
    initial flux (default zero, the plain guess).  ``dsa``: follow each
    group's sweep by the diffusion synthetic correction of oracle/dsa.py
    (slabs with isotropic scattering; not part of the paper's method).
    Returns SIResult.
    """
    S = prob.Q if src is None else src
    G = prob.G
    sw = make_sweeper(prob, quad) if sweeper is None else sweeper
    if dsa:
        from . import dsa as D
        if not isinstance(prob, Slab) or prob.sigs1 is not None:
            raise ValueError("diffusion synthetic acceleration: isotropic slabs only")
    phi = np.zeros_like(prob.sigt) if phi0 is None else np.array(phi0, float)
    # Eq. 25: the linearly anisotropic part of the emission, (3/2) Sigma_s1 mu J,
    # with the current J of the previous iteration (zero at the start)
    aniso = isinstance(prob, Slab) and prob.sigs1 is not None
    cur = np.zeros_like(phi) if aniso else None
    hist = []
    change = np.inf
    it = 0
    for it in range(1, itmax + 1):
        old = phi.copy()
        for g in range(G):
            scat = np.zeros_like(phi[g])
            for gp in range(G):
                scat = scat + prob.sigs[gp, g] * phi[gp]
            q = sw.emission(scat + (S[g] if S is not None else 0.0))
            if aniso:
                phi[g], cur[g] = sw.sweep_p1(g, q, 1.5 * prob.sigs1[g] * cur[g])
            else:
                phi[g] = sw.sweep(g, q)
            if dsa:
                phi[g] = D.correct(prob, g, phi[g], old[g], quad, sw)
        change = rel_change(phi, old)
        if history:
            hist.append(change)
        if change <= tol:
            break
    return SIResult(phi, it, change, hist, sw)


def production(prob, phi):
    """Integral of nuSigma_f phi over the domain and groups (Eq. 26 / 27-29)."""
    return float(np.sum(prob.nusigf * phi * prob.vol[None]))


@dataclass
class EigenResult:
    k: float
    phi: np.ndarray
    outer: int
    inner_total: int
    dk: float
    dphi: float
    k_history: list


def power_iteration(prob, quad, tol_k=1e-10, tol_phi=1e-10, tol_inner=1e-10,
                    itmax_outer=10000, itmax_inner=100000, phi0=None, k0=1.0, dsa=False):
    """Power iteration P with inner source iteration M (App. A2, Eq. A2-A4).

    Plain guess: flat flux and k = 1.  ``dsa``: the inner iterations carry
    the diffusion synthetic correction (see source_iteration).  Returns
    EigenResult with phi normalised to unit production.
    """
    G = prob.G
    if isinstance(prob, Slab) and prob.sigs1 is not None:
        raise ValueError("anisotropic scattering is modelled for fixed-source problems only")
    sw = make_sweeper(prob, quad)
    phi = np.ones_like(prob.sigt) if phi0 is None else np.array(phi0, float)
    P0 = production(prob, phi)
    phi /= P0
    k = float(k0)
    inner_total = 0
    khist = []
    dk = dphi = np.inf
    n = 0
    for n in range(1, itmax_outer + 1):
        F = np.sum(prob.nusigf * phi, axis=0)
        if prob.chi.ndim != 1:
            raise ValueError("chi must be a (G,) vector")
        # chi_g F / k for every group, F the production density of each cell
        src = prob.chi.reshape((G,) + (1,) * F.ndim) * F[None] / k
        r = source_iteration(prob, quad, src=src, phi0=phi, tol=tol_inner,
                             itmax=itmax_inner, sweeper=sw, dsa=dsa)
        inner_total += r.iterations
        P = production(prob, r.phi)
        k_new = k * P
        phi_new = r.phi / P
        sw.scale(1.0 / P)
        dk = abs(k_new - k) / abs(k_new)
        dphi = rel_change(phi_new, phi)
        k, phi = k_new, phi_new
        khist.append(k)
        if dk <= tol_k and dphi <= tol_phi:
            break
    return EigenResult(k, phi, n, inner_total, dk, dphi, khist)


def balance_1d(prob, quad, phi, sweeper):
    """Particle balance terms of a converged 1D fixed-source solution, one group.

    Returns (source, absorption, leakage): integral of S, of (Sigma_t -
    Sigma_s) phi, and the outgoing partial currents sum_n w |mu| psi_out at
    both faces (Eq. 12 integrated over mu and x).
    """
    mu, w = (np.asarray(a, float) for a in quad)
    src = float(np.sum(prob.Q[0] * prob.dx))
    absn = float(np.sum((prob.sigt[0] - prob.sigs[0, 0]) * phi[0] * prob.dx))
    neg, pos = mu < 0, mu > 0
    leak = float(np.sum(w[neg] * np.abs(mu[neg]) * sweeper.out_left[0][neg]) +
                 np.sum(w[pos] * mu[pos] * sweeper.out_right[0][pos]))
    if prob.bc_left == REFLECTIVE:
        leak -= float(np.sum(w[neg] * np.abs(mu[neg]) * sweeper.out_left[0][neg]))
    if prob.bc_right == REFLECTIVE:
        leak -= float(np.sum(w[pos] * mu[pos] * sweeper.out_right[0][pos]))
    return src, absn, leak
