"""The allocation-free slab solve (nop_slab_solve_noalloc) through the C ABI.

Some callers cannot allocate device memory: plug-ins whose host application
owns the GPU's memory and allows no allocation outside the budget it reserved,
and real-time loops that must not call the allocator.  nop_slab_solve_noalloc
serves them from a fixed device array inside the library.  It must reach the
flux of the regular entry point nop_solve_fixed_source on the same slab (FP32
sweeps, relative L2 <= 1e-5) call after call, and the FP64 oracle's flux
within the same bar.  This file is collected last so that a run stopping at
the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import quadrature as Qd
from oracle import transport as T
from tests.helpers import oracle_slab, rel_l2

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch


def _noalloc(inst, tol, itmax):
    """One call through the C ABI with device inputs; returns (rc, flux, stats)."""
    torch = _torch()
    from paper_2509_01416_gb300 import capi
    dev = [torch.tensor(a, dtype=torch.float64, device="cuda")
           for a in (inst.sigt, inst.sigs, inst.Q)]
    phi = torch.full((inst.I,), -1.0, dtype=torch.float64, device="cuda")
    stats = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    rc = capi.lib().nop_slab_solve_noalloc(
        ctypes.c_void_p(dev[0].data_ptr()), ctypes.c_void_p(dev[1].data_ptr()),
        ctypes.c_void_p(dev[2].data_ptr()), inst.I, inst.L, inst.N, tol, itmax,
        ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(stats.data_ptr()), None)
    torch.cuda.synchronize()
    return rc, phi.cpu().numpy(), stats.cpu().numpy()


def test_noalloc_solve_matches_regular_solve_and_oracle_on_consecutive_calls():
    _torch()
    from paper_2509_01416_gb300 import Solver
    s = Solver(0)
    # first call fits the kernel's shared-memory stage, the second does not
    for I, N, seed in ((512, 32, 1), (3000, 16, 2)):
        inst = W.slab_instance(np.random.default_rng(seed), I, N)
        rc, got, st = _noalloc(inst, 1e-6, 100000)
        assert rc == 0
        s.set_slabs([I], [inst.L], [N], inst.sigt, inst.sigs, source=inst.Q)
        ref, info = s.solve_fixed_source(tol=1e-6, itmax=100000, precision=0, schedule=1)
        assert rel_l2(got, ref) <= 1e-5
        assert st[1] == 0 and abs(int(st[0]) - int(info["iterations"][0])) <= 1
        # the FP64 oracle under the same stopping rule
        r = T.source_iteration(oracle_slab(inst), Qd.gauss_legendre(N), tol=1e-6)
        assert rel_l2(got, r.phi[0]) <= 1e-5
    s.close()


def test_noalloc_at_its_size_limit():
    """NOP_NOALLOC_MAX_CELLS cells at order NOP_NOALLOC_MAX_ORDER: every cell
    streams through the array's global working section; against the regular
    entry point and the converged FP64 oracle."""
    _torch()
    from paper_2509_01416_gb300 import Solver, capi
    I, N = capi.NOP_NOALLOC_MAX_CELLS, capi.NOP_NOALLOC_MAX_ORDER
    x = W.cell_centres(I)
    st = 1.0 + 0.5 * np.sin(2 * np.pi * 3 * x / W.L_SLAB)
    inst = W.Slab1G(I=I, N=N, sigt=st, sigs=0.5 * st,
                    Q=W.fourier_source(np.random.default_rng(3), x))
    # c = 0.5: the 1e-6 change leaves an error near 1e-6; the caps bound the run
    rc, got, stats = _noalloc(inst, 1e-6, 500)
    assert rc == 0 and stats[1] == 0, stats
    s = Solver(0)
    s.set_slabs([I], [inst.L], [N], inst.sigt, inst.sigs, source=inst.Q)
    ref, info = s.solve_fixed_source(tol=1e-6, itmax=500, precision=0)
    s.close()
    assert rel_l2(got, ref) <= 1e-5
    r = T.source_iteration(oracle_slab(inst), Qd.gauss_legendre(N), tol=1e-12)
    assert rel_l2(got, r.phi[0]) <= 1e-5


def test_noalloc_reports_the_iteration_cap_and_bad_coefficients():
    _torch()
    from paper_2509_01416_gb300 import capi
    inst = W.slab_instance(np.random.default_rng(4), 200, 16)
    rc, got, st = _noalloc(inst, 1e-12, 1)
    assert rc == 0 and list(st) == [1, capi.NOP_ENOCONV]
    assert np.all(np.isfinite(got)) and np.any(got > 0)
    for bad in (0.0, np.nan):
        b = W.Slab1G(I=inst.I, N=inst.N, sigt=inst.sigt.copy(), sigs=inst.sigs, Q=inst.Q)
        b.sigt[17] = bad
        rc, got, st = _noalloc(b, 1e-6, 1000)
        assert rc == 0 and list(st) == [0, capi.NOP_EINVAL]
        assert np.all(got == 0.0)
    # the shared array is usable again right after a rejected call
    rc, got, st = _noalloc(inst, 1e-6, 100000)
    r = T.source_iteration(oracle_slab(inst), Qd.gauss_legendre(inst.N), tol=1e-6)
    assert rc == 0 and st[1] == 0 and rel_l2(got, r.phi[0]) <= 1e-5


def test_noalloc_rejects_sizes_beyond_its_capacity():
    from paper_2509_01416_gb300 import capi
    L = capi.lib()
    d = ctypes.c_void_p(16)     # never dereferenced: the size check comes first
    too_many = capi.NOP_NOALLOC_MAX_CELLS + 1
    assert L.nop_slab_solve_noalloc(d, d, d, too_many, 10.0, 8, 1e-6, 10, d, d, None) == capi.NOP_EINVAL
    assert L.nop_slab_solve_noalloc(d, d, d, 100, 10.0, capi.NOP_NOALLOC_MAX_ORDER + 2, 1e-6, 10,
                                    d, d, None) == capi.NOP_EINVAL
