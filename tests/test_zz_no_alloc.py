"""The allocation-free slab solve against the regular fixed-source solve.

Some callers cannot allocate device memory: code running while a stream is
captured into a graph, or hosts that forbid device allocations outside a
reserved budget.  nop_slab_solve_noalloc serves them from a fixed device
array inside the library; it must reach the same flux as
nop_solve_fixed_source on the same slab (FP32 sweeps, relative L2 <= 1e-5),
call after call.  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


def test_noalloc_solve_matches_regular_solve_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2509_01416_gb300 import Solver, capi
    L = capi.lib()
    s = Solver(0)
    # first call fits the kernel's shared-memory stage, the second does not
    for I, N, seed in ((512, 32, 1), (3000, 16, 2)):
        inst = W.slab_instance(np.random.default_rng(seed), I, N)
        dev = [torch.tensor(a, dtype=torch.float64, device="cuda")
               for a in (inst.sigt, inst.sigs, inst.Q)]
        phi = torch.full((I,), -1.0, dtype=torch.float64, device="cuda")
        stats = torch.full((2,), -7, dtype=torch.int32, device="cuda")
        rc = L.nop_slab_solve_noalloc(ctypes.c_void_p(dev[0].data_ptr()),
                                      ctypes.c_void_p(dev[1].data_ptr()),
                                      ctypes.c_void_p(dev[2].data_ptr()), I, inst.L, N, 1e-6,
                                      100000, ctypes.c_void_p(phi.data_ptr()),
                                      ctypes.c_void_p(stats.data_ptr()), None)
        torch.cuda.synchronize()
        assert rc == 0
        s.set_slabs([I], [inst.L], [N], inst.sigt, inst.sigs, source=inst.Q)
        ref, info = s.solve_fixed_source(tol=1e-6, itmax=100000, precision=0, schedule=1)
        got = phi.cpu().numpy()
        assert rel_l2(got, ref) <= 1e-5
        st = stats.cpu().numpy()
        assert st[1] == 0 and abs(int(st[0]) - int(info["iterations"][0])) <= 1
    s.close()


def test_noalloc_rejects_sizes_beyond_its_capacity():
    from paper_2509_01416_gb300 import capi
    L = capi.lib()
    d = ctypes.c_void_p(16)     # never dereferenced: the size check comes first
    too_many = capi.NOP_NOALLOC_MAX_CELLS + 1
    assert L.nop_slab_solve_noalloc(d, d, d, too_many, 10.0, 8, 1e-6, 10, d, d, None) == capi.NOP_EINVAL
    assert L.nop_slab_solve_noalloc(d, d, d, 100, 10.0, capi.NOP_NOALLOC_MAX_ORDER + 2, 1e-6, 10,
                                    d, d, None) == capi.NOP_EINVAL
