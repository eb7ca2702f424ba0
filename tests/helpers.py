"""Shared test plumbing: oracle problems for workload instances, comparisons."""
import numpy as np

from oracle import transport as T
from workloads import slab_batch_arrays  # noqa: F401  (re-exported for the tests)


def oracle_slab(s, bc=(0, 0)):
    P = T.uniform_slab(s.I, s.L, s.sigt, s.sigs, Q=s.Q, nusigf=s.nusigf,
                       bc_left=T.REFLECTIVE if bc[0] else T.VACUUM,
                       bc_right=T.REFLECTIVE if bc[1] else T.VACUUM,
                       sigs1=getattr(s, "sigs1", None))
    return P


def split(phi, insts):
    out, o = [], 0
    for s in insts:
        out.append(phi[o:o + s.I])
        o += s.I
    return out


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


_CFG3 = {}


def eigen_slab_config3(seed=3):
    """The three-region 1000-cell S32 eigen slab with its production scaled so
    that its dominant eigenvalue is the recipe's target in [0.9, 1.1]: one
    converged plain FP64 oracle solve gives lam, and nusigf is multiplied by
    target / lam (k scales linearly with the production coefficient)."""
    if seed not in _CFG3:
        from oracle import quadrature as Qd
        import workloads as W
        c = W.eigen_slab_s32(seed)
        e = T.power_iteration(oracle_slab(c), Qd.gauss_legendre(c.N), tol_k=1e-12,
                              tol_phi=1e-10, tol_inner=1e-12)
        c.nusigf = c.nusigf * (c.k_target / e.k)
        _CFG3[seed] = c
    return _CFG3[seed]


def xy_golden():
    """tests/golden/xy_checkerboard_8g.txt (written by make_xy_golden.py with
    the FP64 oracle): k, and flux samples (g, j, i, phi) of the unit-production
    eigenvector of the 256 x 256 8-group checkerboard."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "xy_checkerboard_8g.txt")
    k, rows, gint = None, [], {}
    with open(path) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "k":
                k = float(t[1])
            elif t[0] == "group_integral":
                gint[int(t[1])] = float(t[2])
            elif len(t) == 4:
                rows.append((int(t[0]), int(t[1]), int(t[2]), float(t[3])))
    a = np.array(rows)
    return k, a[:, 0].astype(int), a[:, 1].astype(int), a[:, 2].astype(int), a[:, 3], gint
