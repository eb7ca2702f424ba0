"""Edge cases of the slab solver and the warm start on the GPU, against the
FP64 oracle: the smallest instances (one cell, S2), the largest order (S128),
a long slab beyond the staging capacity of one warp, a pure absorber (one
source iteration), a zero source (zero flux, zero change), a scattering
ratio near one, zero-size and malformed batches, and a recast whose source
is zero everywhere.
"""
import numpy as np
import pytest

import workloads as W
from oracle import quadrature as Qd
from oracle import transport as T
from tests.helpers import oracle_slab, rel_l2, slab_batch_arrays, split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2509_01416_gb300 import Solver
    s = Solver(0)
    yield s
    s.close()


def _set(s, insts):
    n, wdt, order, sigt, sigs, src, _ = slab_batch_arrays(insts)
    s.set_slabs(n, wdt, order, sigt, sigs, source=src)


def _oracle(s, tol):
    return T.source_iteration(oracle_slab(s), Qd.gauss_legendre(s.N), tol=tol, itmax=1000000)


def test_extreme_shapes_fp64(solver):
    rng = np.random.default_rng(1)
    insts = []
    for I, N in [(1, 2), (1, 128), (2, 2), (3, 128), (5000, 8), (700, 128)]:
        x = W.cell_centres(I)
        st = rng.uniform(0.5, 1.5, I)
        insts.append(W.Slab1G(I=I, N=N, sigt=st, sigs=0.7 * st, Q=W.fourier_source(rng, x)))
    _set(solver, insts)
    phi, info = solver.solve_fixed_source(tol=1e-12, itmax=100000, precision=1)
    for s, g in zip(insts, split(phi, insts)):
        assert rel_l2(g, _oracle(s, 1e-12).phi[0]) < 1e-9, (s.I, s.N)


def test_extreme_shapes_fp32_same_rule(solver):
    rng = np.random.default_rng(2)
    insts = []
    for I, N in [(1, 2), (1, 64), (4, 2), (5000, 8), (3000, 64), (2048, 128)]:
        x = W.cell_centres(I)
        st = rng.uniform(0.5, 1.5, I)
        insts.append(W.Slab1G(I=I, N=N, sigt=st, sigs=0.8 * st, Q=W.fourier_source(rng, x)))
    _set(solver, insts)
    phi, info = solver.solve_fixed_source(tol=1e-6, itmax=100000, precision=0)
    for b, (s, g) in enumerate(zip(insts, split(phi, insts))):
        r = _oracle(s, 1e-6)
        assert abs(int(info["iterations"][b]) - r.iterations) <= 1, (s.I, s.N)
        assert rel_l2(g, r.phi[0]) < 1e-5, (s.I, s.N)


def test_pure_absorber_converges_in_two_iterations(solver):
    # no scattering: the first sweep is the answer, the second sees no change
    I = 300
    s = W.Slab1G(I=I, N=16, sigt=np.full(I, 1.3), sigs=np.zeros(I), Q=np.ones(I))
    _set(solver, [s])
    phi, info = solver.solve_fixed_source(tol=1e-12, itmax=100, precision=1)
    assert int(info["iterations"][0]) == 2
    assert rel_l2(phi, _oracle(s, 1e-14).phi[0]) < 1e-12


def test_zero_source_gives_zero_flux(solver):
    insts = [W.Slab1G(I=50, N=8, sigt=np.ones(50), sigs=np.full(50, 0.5), Q=np.zeros(50)),
             W.slab_instance(np.random.default_rng(3), 80, 16)]
    _set(solver, insts)
    for prec in (0, 1):
        # FP32 need not reach a 1e-8 change: the cap (NOP_ENOCONV) is accepted there
        phi, info = solver.solve_fixed_source(tol=1e-8, itmax=1000, precision=prec,
                                              allow_noconv=prec == 0)
        z, other = split(phi, insts)
        assert np.all(z == 0.0) and info["status"][0] == 0
        assert rel_l2(other, _oracle(insts[1], 1e-8).phi[0]) < 1e-5


def test_scattering_ratio_near_one(solver):
    # c = 0.999 in a thick slab: a slowly converging source iteration
    I = 400
    s = W.Slab1G(I=I, N=16, sigt=np.full(I, 2.0), sigs=np.full(I, 1.998), Q=np.ones(I))
    _set(solver, [s])
    phi, info = solver.solve_fixed_source(tol=1e-10, itmax=200000, precision=1)
    r = _oracle(s, 1e-10)
    assert abs(int(info["iterations"][0]) - r.iterations) <= 1
    assert rel_l2(phi, r.phi[0]) < 1e-8


def test_malformed_batches_are_rejected(solver):
    from paper_2509_01416_gb300 import NopError
    with pytest.raises(NopError):            # no instance
        solver.set_slabs(np.zeros(0, np.int32), np.zeros(0), np.zeros(0, np.int32),
                         np.zeros(0), np.zeros(0), source=np.zeros(0))
    with pytest.raises(NopError):            # zero cells
        solver.set_slabs([0], [1.0], [4], np.zeros(0), np.zeros(0), source=np.zeros(0))
    with pytest.raises(NopError):            # order above 128
        solver.set_slabs([5], [1.0], [130], np.ones(5), np.zeros(5), source=np.ones(5))
    with pytest.raises(NopError):            # non-finite coefficient
        solver.set_slabs([3], [1.0], [4], np.array([1.0, np.nan, 1.0]), np.zeros(3),
                         source=np.ones(3))


def test_recast_of_a_zero_source_is_zero(solver):
    # every recast part is empty: the operator is never applied and the
    # prediction is zero, after which the solve is the plain one
    from paper_2509_01416_gb300 import NOP_NO_DEEPONET, no_config
    insts = [W.Slab1G(I=64, N=8, sigt=np.ones(64), sigs=np.full(64, 0.5), Q=np.zeros(64))]
    _set(solver, insts)
    solver.no_set(no_config(NOP_NO_DEEPONET, sensors=128, width=128, basis=128),
                  W.deeponet_init(5))
    phi, info = solver.recast_iterate(tol=1e-4, itmax=10)
    assert np.all(phi == 0.0)
    warm, wi = solver.solve_fixed_source(tol=1e-8, itmax=100, precision=1, warm_start=1)
    assert np.all(warm == 0.0)
