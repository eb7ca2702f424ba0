"""Seeded synthetic inputs shaped like the paper's transport problems.

This module holds input recipes only (random coefficients, sources, network
initial weights); none of the method's arithmetic lives here.  Both the CUDA
path and the oracle draw their inputs from it.  All randomness comes from
``numpy.random.default_rng(seed)``.

Recipes (the paper's own samples are not published; these stand in for them):
  * GRF source (App. A1): Gaussian random field on the cell centres with
    squared-exponential covariance var * exp(-(x-x')^2 / (2 ell^2)), mean 0.07,
    var 3e-4, ell 1.2, drawn by Cholesky factorisation (jitter 1e-10), clipped
    at zero, then scaled to unit integral (Eq. 13).
  * Fourier source: max(0, 1 + sum_{j=1..16} a_j cos(2 pi j x/L) + b_j sin(...)),
    a_j, b_j ~ N(0, (0.6/j)^2).
  * sinusoidal total cross section: 1 + 0.5 sin(2 pi k x / L), k ~ U{1..4}.
  * piecewise regions: R region boundaries drawn uniformly in (0, L), sorted.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

L_SLAB = 10.0
P_STAR = (1.0, 0.5)           # (Sigma_t*, Sigma_s*), Sec. 5.1


def cell_centres(I, L=L_SLAB):
    return (np.arange(I) + 0.5) * (L / I)


def grf(rng, x, n, mean=0.07, var=3e-4, ell=1.2):
    """n GRF samples on points x, clipped at 0 and scaled to unit integral."""
    d = x[:, None] - x[None, :]
    C = var * np.exp(-d * d / (2 * ell * ell)) + 1e-10 * np.eye(len(x))
    Lc = np.linalg.cholesky(C)
    z = rng.standard_normal((n, len(x)))
    s = np.maximum(mean + z @ Lc.T, 0.0)
    h = (x[-1] - x[0]) / (len(x) - 1) if len(x) > 1 else 1.0
    return s / (s.sum(axis=1, keepdims=True) * h)


def fourier_source(rng, x, L=L_SLAB, terms=16, amp=0.6):
    j = np.arange(1, terms + 1)
    a = rng.standard_normal(terms) * amp / j
    b = rng.standard_normal(terms) * amp / j
    arg = 2 * np.pi * np.outer(x, j) / L
    return np.maximum(0.0, 1.0 + np.cos(arg) @ a + np.sin(arg) @ b)


def regions(rng, x, R, L=L_SLAB):
    """Region index of each point for R random regions over (0, L)."""
    cuts = np.sort(rng.uniform(0, L, R - 1))
    return np.searchsorted(cuts, x)


@dataclass
class Slab1G:
    """One single-group 1D slab instance (uniform cells over [0, L])."""
    I: int
    N: int
    sigt: np.ndarray
    sigs: np.ndarray
    Q: Optional[np.ndarray] = None
    nusigf: Optional[np.ndarray] = None
    L: float = L_SLAB
    bc_left: int = 0          # 0 vacuum, 1 reflective
    bc_right: int = 0
    sigs1: Optional[np.ndarray] = None   # first Legendre moment (Eq. 25), or None


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------
def uniform_slab_s16():
    """200 cells, width 10, Sigma_t 1.0, Sigma_s 0.9, Q = 1, vacuum, S16."""
    I = 200
    return Slab1G(I=I, N=16, sigt=np.full(I, 1.0), sigs=np.full(I, 0.9), Q=np.ones(I))


def hetero_slab_s32(seed=2):
    """512 cells, S32, sinusoidal Sigma_t, piecewise scattering ratio, Fourier Q."""
    rng = np.random.default_rng(seed)
    I = 512
    x = cell_centres(I)
    k = rng.integers(1, 5)
    sigt = 1.0 + 0.5 * np.sin(2 * np.pi * k * x / L_SLAB)
    R = int(rng.integers(4, 9))
    c = rng.uniform(0.5, 0.99, R)[regions(rng, x, R)]
    Q = fourier_source(rng, x)
    return Slab1G(I=I, N=32, sigt=sigt, sigs=c * sigt, Q=Q)


def _bare_slab_nonleakage(sigt, sigs, L):
    """Diffusion-theory non-leakage estimate used only to place k near 1."""
    st = float(np.mean(sigt))
    D = 1.0 / (3.0 * st)
    B = np.pi / (L + 2 * 0.7104 / st)
    sa = float(np.mean(sigt - sigs))
    return sa / (sa + D * B * B)


def eigen_slab_s32(seed=3):
    """1000 cells, S32, 3 regions, Sigma_t in [0.8, 1.5], c in [0.6, 0.9],
    production scaled so that k lands near [0.9, 1.1], vacuum."""
    rng = np.random.default_rng(seed)
    I = 1000
    x = cell_centres(I)
    reg = regions(rng, x, 3)
    st_r = rng.uniform(0.8, 1.5, 3)
    c_r = rng.uniform(0.6, 0.9, 3)
    f_r = rng.uniform(0.5, 1.5, 3)
    sigt, sigs = st_r[reg], (c_r * st_r)[reg]
    shape = (f_r * st_r * (1 - c_r))[reg]
    target = rng.uniform(0.9, 1.1)
    kinf = float(np.sum(shape)) / float(np.sum(sigt - sigs))
    nusigf = shape * target / (kinf * _bare_slab_nonleakage(sigt, sigs, L_SLAB))
    inst = Slab1G(I=I, N=32, sigt=sigt, sigs=sigs, nusigf=nusigf)
    # the eigenvalue this instance is meant to have; a caller that solved it
    # once (eigenvalue lam) lands exactly there by scaling nusigf by target/lam
    inst.k_target = float(target)
    return inst


@dataclass
class XYMG:
    """2D x-y multigroup problem on a uniform mesh (arrays [g, j, i])."""
    nx: int
    ny: int
    Lx: float
    Ly: float
    sigt: np.ndarray          # (G, ny, nx)
    sigs: np.ndarray          # (G, G, ny, nx) from g' to g
    nusigf: np.ndarray        # (G, ny, nx)
    chi: np.ndarray           # (G,)
    bc: dict = field(default_factory=dict)   # faces x0, xL, y0, yL -> 0/1


KINF_8G = 1.3


def base_table_8g():
    """An 8-group base table: downscatter to the next two groups, upscatter
    from group 8 into 7 and within the last two groups, fission in groups 1 and
    5-8, chi in groups 1-3.  Values are a synthetic stand-in, not data."""
    G = 8
    sigt = np.array([0.22, 0.30, 0.42, 0.55, 0.70, 0.90, 1.20, 1.45])
    S = np.zeros((G, G))
    for g in range(G):
        S[g, g] = 0.55 * sigt[g]
        if g + 1 < G:
            S[g, g + 1] = 0.12 * sigt[g]
        if g + 2 < G:
            S[g, g + 2] = 0.04 * sigt[g]
    S[7, 6] = 0.10 * sigt[7]          # upscatter 8 -> 7
    nsf = np.array([0.020, 0.0, 0.0, 0.0, 0.010, 0.030, 0.110, 0.160])
    chi = np.array([0.70, 0.25, 0.05, 0, 0, 0, 0, 0])
    # scale production so that the infinite-medium multiplication of the base
    # table is KINF_8G (leakage from the 10 cm domain then brings k near 1)
    kinf = max(np.linalg.eigvals(np.linalg.solve(np.diag(sigt) - S.T, np.outer(chi, nsf))).real)
    return sigt, S, nsf * (KINF_8G / kinf), chi


def checkerboard_xy_8g(seed=4, n=256, L=10.0):
    """256x256, 8 groups, 4x4 checkerboard of 16 material sets drawn +-30%
    around the base table; reflective x=0 and y=0, vacuum x=L and y=L."""
    rng = np.random.default_rng(seed)
    st0, S0, nsf0, chi = base_table_8g()
    G = len(st0)
    mats = []
    for _ in range(16):
        f = rng.uniform(0.7, 1.3, size=(3, G))
        st = st0 * f[0]
        S = S0 * f[1][:, None]
        S = S * np.minimum(1.0, 0.95 * st / np.maximum(S.sum(axis=1), 1e-30))[:, None]
        mats.append((st, S, nsf0 * f[2]))
    blk = n // 4
    ii = np.minimum(np.arange(n) // blk, 3)
    mid = ii[:, None] * 4 + ii[None, :]            # [j, i]
    sigt = np.zeros((G, n, n))
    sigs = np.zeros((G, G, n, n))
    nsf = np.zeros((G, n, n))
    for m, (st, S, nf) in enumerate(mats):
        msk = mid == m
        sigt[:, msk] = st[:, None]
        sigs[:, :, msk] = S[:, :, None]
        nsf[:, msk] = nf[:, None]
    return XYMG(nx=n, ny=n, Lx=L, Ly=L, sigt=sigt, sigs=sigs, nusigf=nsf, chi=chi,
                bc={"x0": 1, "xL": 0, "y0": 1, "yL": 0})


def aniso_slab(seed=25, I=100, N=32, sigt=1.2, sigs0=0.8, sigs1=0.3):
    """The fixed-source slab with linearly anisotropic scattering of Sec. 5.1
    Eq. 25 (Sigma_t 1.2, Sigma_s0 0.8, Sigma_s1 0.3, 10 cm, dL = 0.1 cm, S32),
    with a GRF source of unit integral drawn from the seed."""
    rng = np.random.default_rng(seed)
    x = cell_centres(I)
    one = np.ones(I)
    return Slab1G(I=I, N=N, sigt=sigt * one, sigs=sigs0 * one, Q=grf(rng, x, 1)[0],
                  sigs1=sigs1 * one)


D_STAR = (1.0, 0.0)            # (D*, Sigma_a*) of the diffusion operator


def diffusion_slab(rng, I, L=L_SLAB, helmholtz=False):
    """One diffusion slab of the recast's second PDE (Table 1): diffusion row,
    D(x) = 1 + a sin(2 pi k x / L + ph) (a ~ U[0.2, 0.6], k ~ U{1..4}) with
    Sigma_a = 0, or (helmholtz) the Helmholtz row, D = 1 with
    Sigma_a = -k^2(x) = -(0.02 + 0.03 U[0,1]) below the first Dirichlet mode;
    source a clipped Fourier series.  Returns (D, Sigma_a, S) on I cells."""
    x = cell_centres(I, L)
    if helmholtz:
        D = np.ones(I)
        siga = -(0.02 + 0.03 * rng.uniform(0, 1, I))
    else:
        a, k, ph = rng.uniform(0.2, 0.6), rng.integers(1, 5), rng.uniform(0, 2 * np.pi)
        D = 1.0 + a * np.sin(2 * np.pi * k * x / L + ph)
        siga = np.zeros(I)
    return D, siga, fourier_source(rng, x, L)


def slab_instance(rng, I, N):
    """One instance of the slab batch: sinusoidal or piecewise coefficients, Fourier Q."""
    x = cell_centres(I)
    if rng.uniform() < 0.5:
        k = rng.integers(1, 5)
        ph = rng.uniform(0, 2 * np.pi)
        sigt = 1.0 + 0.5 * np.sin(2 * np.pi * k * x / L_SLAB + ph)
        c = 0.5 + 0.49 * (0.5 + 0.5 * np.sin(2 * np.pi * rng.integers(1, 4) * x / L_SLAB))
    else:
        R = int(rng.integers(4, 9))
        reg = regions(rng, x, R)
        sigt = rng.uniform(0.5, 1.5, R)[reg]
        c = rng.uniform(0.5, 0.99, R)[reg]
    return Slab1G(I=I, N=N, sigt=sigt, sigs=c * sigt, Q=fourier_source(rng, x))


def slab_batch(seed=5, n_inst=4096, I_range=(64, 2048), N_range=(8, 64)):
    """4096 independent slabs, I ~ U{64..2048}, N even ~ U{8..64}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        I = int(rng.integers(I_range[0], I_range[1] + 1))
        N = 2 * int(rng.integers(N_range[0] // 2, N_range[1] // 2 + 1))
        out.append(slab_instance(np.random.default_rng(rng.integers(1 << 62)), I, N))
    return out


def training_sources(seed, n_samples, I, L=L_SLAB):
    """GRF training sources on I cell centres (App. A1 recipe), unit integral."""
    rng = np.random.default_rng(seed)
    return grf(rng, cell_centres(I, L), n_samples)


def training_sources_2d(seed, n_samples, n, L=10.0, ell=1.2, var=3e-4, mean=0.07):
    """Separable-kernel 2D GRF sources on an n x n grid, unit integral."""
    rng = np.random.default_rng(seed)
    x = cell_centres(n, L)
    d = x[:, None] - x[None, :]
    C = np.exp(-d * d / (2 * ell * ell)) + 1e-10 * np.eye(n)
    Lc = np.linalg.cholesky(C)
    z = rng.standard_normal((n_samples, n, n))
    f = np.sqrt(var) * np.matmul(np.matmul(Lc, z), Lc.T)   # Lc z Lc^T per sample
    s = np.maximum(mean + f, 0.0)
    h = L / n
    return s / (s.sum(axis=(1, 2), keepdims=True) * h * h)


def slab_batch_arrays(insts):
    """Pack single-group slab instances into the flat arrays of the C ABI's
    slab batch: (n_cells, width, order, sigma_t, sigma_s, source, nu_sigma_f),
    cells of all instances concatenated in instance order (None for a field
    the instances do not carry)."""
    n = np.array([s.I for s in insts], dtype=np.int32)
    wdt = np.array([s.L for s in insts])
    order = np.array([s.N for s in insts], dtype=np.int32)
    sigt = np.concatenate([s.sigt for s in insts])
    sigs = np.concatenate([s.sigs for s in insts])
    src = None if insts[0].Q is None else np.concatenate([s.Q for s in insts])
    nsf = None if insts[0].nusigf is None else np.concatenate([s.nusigf for s in insts])
    return n, wdt, order, sigt, sigs, src, nsf


# ---------------------------------------------------------------------------
# neural-operator initial weights (Kaiming-uniform style), as plain arrays
# ---------------------------------------------------------------------------
def _lin(rng, o, i):
    bound = 1.0 / np.sqrt(i)
    return rng.uniform(-bound, bound, (o, i)), rng.uniform(-bound, bound, o)


def deeponet_init(seed, m=128, width=128, p=128, depth=4, d_trunk=1):
    rng = np.random.default_rng(seed)
    P = {}
    dims_b = [m] + [width] * (depth - 1) + [p]
    dims_t = [d_trunk] + [width] * (depth - 1) + [p]
    for net, dims in (("b", dims_b), ("t", dims_t)):
        for l in range(depth):
            P["%s%d.W" % (net, l)], P["%s%d.b" % (net, l)] = _lin(rng, dims[l + 1], dims[l])
    return P


def fno1d_init(seed, width=64, modes=32, layers=4, proj=128, in_ch=2):
    rng = np.random.default_rng(seed)
    P = {}
    P["lift.W"], P["lift.b"] = _lin(rng, width, in_ch)
    sc = 1.0 / (width * width)
    for l in range(layers):
        P["spec%d.re" % l] = sc * rng.uniform(0, 1, (modes, width, width))
        P["spec%d.im" % l] = sc * rng.uniform(0, 1, (modes, width, width))
        P["pw%d.W" % l], P["pw%d.b" % l] = _lin(rng, width, width)
    P["proj1.W"], P["proj1.b"] = _lin(rng, proj, width)
    P["proj2.W"], P["proj2.b"] = _lin(rng, 1, proj)
    return P


def fno2d_init(seed, width=32, modes=16, layers=4, proj=128, in_ch=3):
    rng = np.random.default_rng(seed)
    P = {}
    P["lift.W"], P["lift.b"] = _lin(rng, width, in_ch)
    sc = 1.0 / (width * width)
    for l in range(layers):
        for k in ("re1", "im1", "re2", "im2"):
            P["spec%d.%s" % (l, k)] = sc * rng.uniform(0, 1, (modes, modes, width, width))
        P["pw%d.W" % l], P["pw%d.b" % l] = _lin(rng, width, width)
    P["proj1.W"], P["proj1.b"] = _lin(rng, proj, width)
    P["proj2.W"], P["proj2.b"] = _lin(rng, 1, proj)
    return P
