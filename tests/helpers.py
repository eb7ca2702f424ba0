"""Shared test plumbing: turn workload instances into C-ABI arrays and oracle problems."""
import numpy as np

from oracle import transport as T


def slab_batch_arrays(insts):
    """Single-group slab instances -> (n_cells, width, order, sigt, sigs, src, nsf)."""
    n = np.array([s.I for s in insts], dtype=np.int32)
    wdt = np.array([s.L for s in insts])
    order = np.array([s.N for s in insts], dtype=np.int32)
    sigt = np.concatenate([s.sigt for s in insts])
    sigs = np.concatenate([s.sigs for s in insts])
    src = None if insts[0].Q is None else np.concatenate([s.Q for s in insts])
    nsf = None if insts[0].nusigf is None else np.concatenate([s.nusigf for s in insts])
    return n, wdt, order, sigt, sigs, src, nsf


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
