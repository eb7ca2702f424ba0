"""Equation-recast neural-operator iteration and warm starts (FP64 oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3.1 Eq. 6a-7 and Sec. 3.2 Eq. 8: with p = p* + dp the operator
difference moves to the source side and a solution operator N trained at p*
is iterated, u_{k+1} = N[S - dL(dp) u_k].  For the transport equation,
Sec. 5.1 Eq. 21-24 with the isotropic approximation of Eq. 23, this is

    phi_{k+1} = N[ S + ((Sigma_s - Sigma_s*) - (Sigma_t - Sigma_t*)) phi_k ],

started from phi_0 = 0 (so phi_1 = N[S]).  The result seeds the model-based
solver (Eq. 9a/10b, Eq. 20).  For eigenproblems the simple preconditioning of
App. A2 (Eq. A5) replaces the inner solve by one recast operator application
per outer iteration, and its (k, phi) seed the model-based power iteration
(Eq. A6); the constrained preconditioning (Eq. A7-A8) follows every operator
prediction by one model-based source iteration.

Readings where the paper is silent (the CUDA side does the same):
  * the operator acts on its own grid.  DeepONet: M uniform bins over the
    slab; an instance's cell fields reach the bins by the overlap-weighted
    cell average P, and the recast loop runs on the bins with u = T_ref beta
    (trunk evaluated at bin centres); only the final flux is evaluated at the
    instance's cell centres.  FNO: the operator grid is the instance grid.
  * linear scaling: the trained operator saw sources normalised to unit
    integral (Eq. 13), and the exact solution operator is linear.  A source s
    is applied part by part, each part normalised to unit integral:
        sigma+ N[s+ / sigma+] - sigma- N[s- / sigma-],
    s+ = max(s, 0), s- = max(-s, 0), sigma+- = integral of s+-; a part with
    zero integral contributes nothing (a ReLU network maps 0 to a nonzero
    constant, so it is never evaluated on an empty part).
  * stopping: ||u_{k+1} - u_k||_2 / ||u_{k+1}||_2 <= tol or k = itmax;
    divergence: a non-finite iterate, or the absolute change ||u_{k+1} - u_k||_2
    failing to shrink for DIVERGE_RUN consecutive iterations (a fixed-point
    map that does not contract).
"""
import numpy as np

from . import neural
from . import transport as T

DIVERGE_RUN = 5
OK, NOCONV, DIVERGED = 0, 1, 2


def projection_matrix(edges, M, L):
    """P[m, i] = |cell_i ∩ bin_m| / |bin_m| for cell edges ``edges`` (I+1,)."""
    I = len(edges) - 1
    h = L / M
    P = np.zeros((M, I))
    for m in range(M):
        lo, hi = m * h, (m + 1) * h
        for i in range(I):
            ov = min(hi, edges[i + 1]) - max(lo, edges[i])
            if ov > 0:
                P[m, i] = ov / h
    return P


def _split_apply(apply_unit, s, cellsize):
    """sigma+ N[s+/sigma+] - sigma- N[s-/sigma-] over a batch s (B, ...)."""
    axes = tuple(range(1, s.ndim))
    res = []
    for b in range(s.shape[0]):
        pos = np.maximum(s[b], 0)
        neg = np.maximum(-s[b], 0)
        sp = float(np.sum(pos) * cellsize)
        sn = float(np.sum(neg) * cellsize)
        acc = None
        if sp > 0:
            acc = sp * apply_unit((pos / sp)[None])[0]
        if sn > 0:
            t = sn * apply_unit((neg / sn)[None])[0]
            acc = -t if acc is None else acc - t
        res.append(acc)
    shape = None
    for r in res:
        if r is not None:
            shape = np.shape(r)
    if shape is None:
        return None
    return np.stack([np.zeros(shape) if r is None else r for r in res])


class DeepONetOp:
    """DeepONet solution operator N at p* on an M-bin sensor grid over [0, L]."""

    def __init__(self, params, L, M, quant=neural._id):
        self.p, self.L, self.M, self.quant = params, float(L), int(M), quant
        self.xb = ((np.arange(M) + 0.5) / M)[:, None]      # bin centres / L

    def _branch(self, U):
        nb = sum(1 for k in self.p if k.startswith("b") and k.endswith(".W"))
        out, _ = neural.mlp_forward(neural.deeponet_layers(self.p, "b", nb), U, self.quant)
        return out

    def trunk(self, xn):
        nt = sum(1 for k in self.p if k.startswith("t") and k.endswith(".W"))
        out, _ = neural.mlp_forward(neural.deeponet_layers(self.p, "t", nt), xn, self.quant)
        return out

    def coef(self, s):
        """Branch coefficients beta (B, p) of the scaled/split source s (B, M)."""
        h = self.L / self.M
        r = _split_apply(self._branch, s, h)
        if r is None:
            nb = sum(1 for k in self.p if k.startswith("b") and k.endswith(".W"))
            return np.zeros((s.shape[0], self.p["b%d.b" % (nb - 1)].shape[0]))
        return r

    def eval(self, beta, xn):
        """phi at normalised coordinates xn (P,) for coefficients beta (B, p)."""
        return self.quant(beta) @ self.quant(self.trunk(np.asarray(xn, float)[:, None])).T


def recast_deeponet(op, prob, p_star, tol=1e-4, itmax=200):
    """Eq. 24 for one single-group 1D slab with a DeepONet operator.

    Returns (phi_NO on the instance cells, iterations, status, beta).
    """
    L = float(np.sum(prob.dx))
    edges = np.concatenate([[0.0], np.cumsum(prob.dx)])
    P = projection_matrix(edges, op.M, L)
    sigt_s, sigs_s = p_star
    delta = (prob.sigs[0, 0] - sigs_s) - (prob.sigt[0] - sigt_s)
    s = P @ prob.Q[0]
    d = P @ delta
    Tref = op.trunk(op.xb)
    u = np.zeros(op.M)
    beta = np.zeros(Tref.shape[1])
    status, it = NOCONV, 0
    prev, run = np.inf, 0
    for it in range(1, itmax + 1):
        src = s + d * u
        beta = op.coef(src[None])[0]
        u_new = op.quant(beta) @ op.quant(Tref).T
        if not np.all(np.isfinite(u_new)):
            status = DIVERGED
            break
        ch = T.rel_change(u_new, u)
        ab = float(np.sqrt(np.sum((u_new - u) ** 2)))
        u = u_new
        if ch <= tol:
            status = OK
            break
        run = run + 1 if ab >= prev else 0
        prev = ab
        if run >= DIVERGE_RUN:
            status = DIVERGED
            break
    xc = (edges[:-1] + edges[1:]) / 2 / L
    phi = op.eval(beta[None], xc)[0]
    return phi, it, status, beta


class FNOOp1D:
    """FNO-1D solution operator N at p* on the instance grid (uniform cells)."""

    def __init__(self, params, L, quant=neural._id):
        self.p, self.L, self.quant = params, float(L), quant

    def __call__(self, S):
        n = S.shape[-1]
        xc = (np.arange(n) + 0.5) / n
        f = lambda U: neural.fno1d_forward(self.p, U, xc, self.quant)[0]
        r = _split_apply(f, S, self.L / n)
        return np.zeros_like(S) if r is None else r


class FNOOp2D:
    """FNO-2D solution operator N at p* on the instance grid (ny, nx)."""

    def __init__(self, params, Lx, Ly, quant=neural._id):
        self.p, self.Lx, self.Ly, self.quant = params, float(Lx), float(Ly), quant

    def __call__(self, S):
        ny, nx = S.shape[-2:]
        yc = (np.arange(ny) + 0.5) / ny
        xc = (np.arange(nx) + 0.5) / nx
        f = lambda U: neural.fno2d_forward(self.p, U, yc, xc, self.quant)[0]
        r = _split_apply(f, S, (self.Lx / nx) * (self.Ly / ny))
        return np.zeros_like(S) if r is None else r


def recast_grid(apply, S, delta, tol=1e-4, itmax=200):
    """Eq. 24 on the operator's own grid: phi <- N[S + delta * phi], phi_0 = 0.

    ``apply`` maps a batch (1, ...) of sources to fluxes.  Returns
    (phi, iterations, status).
    """
    phi = np.zeros_like(S)
    status, it = NOCONV, 0
    prev, run = np.inf, 0
    for it in range(1, itmax + 1):
        new = apply((S + delta * phi)[None])[0]
        if not np.all(np.isfinite(new)):
            status = DIVERGED
            break
        ch = T.rel_change(new, phi)
        ab = float(np.sqrt(np.sum((new - phi) ** 2)))
        phi = new
        if ch <= tol:
            status = OK
            break
        run = run + 1 if ab >= prev else 0
        prev = ab
        if run >= DIVERGE_RUN:
            status = DIVERGED
            break
    return phi, it, status


def recast_exact_operator(prob_star_factory, quad, tol=1e-13):
    """N = the exact S_N fixed-source solve at p* (for the recast-limit identity)."""
    def apply(S):
        out = []
        for s in S:
            P = prob_star_factory(s)
            out.append(T.source_iteration(P, quad, tol=tol).phi[0])
        return np.stack(out)
    return apply


def sp_eigen(prob, apply_group, p_star, tol_k=1e-6, tol_phi=1e-6, itmax=2000):
    """Simple preconditioning, App. A2 Eq. A5: power iteration whose inner solve
    is one recast operator application per group and outer step.

    ``apply_group(S)`` maps a (1, cells...) source to a flux.  Groups are
    visited in order; group g's source is chi_g F/k + sum_{g' != g}
    Sigma_s^{g'->g} phi_g' (newest) + delta_g phi_g with delta_g =
    (Sigma_s^{g->g} - Sigma_s*) - (Sigma_t,g - Sigma_t*).  Returns
    (k, phi normalised to unit production, outer iterations, status).
    """
    sigt_s, sigs_s = p_star
    G = prob.G
    phi = np.ones_like(prob.sigt)
    phi /= T.production(prob, phi)
    k = 1.0
    status = NOCONV
    n = 0
    for n in range(1, itmax + 1):
        F = np.sum(prob.nusigf * phi, axis=0)
        new = phi.copy()
        for g in range(G):
            src = prob.chi[g] * F / k
            for gp in range(G):
                if gp != g:
                    src = src + prob.sigs[gp, g] * new[gp]
            delta = (prob.sigs[g, g] - sigs_s) - (prob.sigt[g] - sigt_s)
            new[g] = apply_group((src + delta * phi[g])[None])[0]
        if not np.all(np.isfinite(new)):
            status = DIVERGED
            break
        Pn = T.production(prob, new)
        k_new = k * Pn
        new /= Pn
        dk = abs(k_new - k) / abs(k_new)
        dphi = T.rel_change(new, phi)
        k, phi = k_new, new
        if dk <= tol_k and dphi <= tol_phi:
            status = OK
            break
    return k, phi, n, status


def cp_eigen(prob, apply_group, p_star, quad, tol_k=1e-6, tol_phi=1e-6, itmax=2000):
    """Constrained preconditioning, App. A2 Eq. A7-A8.

    Every outer step first predicts with the operator exactly as the simple
    preconditioning does (Eq. A7: groups in order, newest in-scatter, recast
    mismatch delta_g phi_g), then refines the prediction with one application
    of the model-based iteration operator M (Eq. A8): one source iteration
    (a transport sweep per group, Gauss-Seidel over groups) started from the
    prediction, whose fission source chi F / k is built from the prediction
    with the current k.  The outer update P then sets k <- k P and scales the
    flux to unit production.  Returns (k, phi, outer iterations, status).
    """
    sigt_s, sigs_s = p_star
    G = prob.G
    sw = T.make_sweeper(prob, quad)
    phi = np.ones_like(prob.sigt)
    phi /= T.production(prob, phi)
    k = 1.0
    status = NOCONV
    n = 0
    shape = (G,) + (1,) * (prob.sigt.ndim - 1)
    for n in range(1, itmax + 1):
        # Eq. A7: the operator's prediction u^(n+1/4)
        F = np.sum(prob.nusigf * phi, axis=0)
        quarter = phi.copy()
        for g in range(G):
            src = prob.chi[g] * F / k
            for gp in range(G):
                if gp != g:
                    src = src + prob.sigs[gp, g] * quarter[gp]
            delta = (prob.sigs[g, g] - sigs_s) - (prob.sigt[g] - sigt_s)
            quarter[g] = apply_group((src + delta * phi[g])[None])[0]
        if not np.all(np.isfinite(quarter)):
            status = DIVERGED
            break
        # Eq. A8: one model-based source iteration from the prediction
        Fq = np.sum(prob.nusigf * quarter, axis=0)
        srcq = prob.chi.reshape(shape) * Fq[None] / k
        half = T.source_iteration(prob, quad, src=srcq, phi0=quarter, tol=0.0, itmax=1,
                                  sweeper=sw).phi
        Pn = T.production(prob, half)
        if not np.isfinite(Pn) or Pn == 0:
            status = DIVERGED
            break
        k_new = k * Pn
        half = half / Pn
        sw.scale(1.0 / Pn)
        dk = abs(k_new - k) / abs(k_new)
        dphi = T.rel_change(half, phi)
        k, phi = k_new, half
        if dk <= tol_k and dphi <= tol_phi:
            status = OK
            break
    return k, phi, n, status
