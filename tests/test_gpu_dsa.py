"""GPU parity of diffusion synthetic acceleration (NOP_DSA) against the FP64
oracle's accelerated source iteration (oracle/dsa.py).

FP64: iterate for iterate (same stopping rule, iteration counts within one,
flux to 1e-9).  FP32: flux relative L2 <= 1e-5 at the same stopping rule.
Covers the warp path (staged and unstaged instances, chunk boundaries of the
edge scan, one and two cells), the block path, reflective faces, two
groups, the inner iterations of eigen solves, the full 4096-slab batch and
the combination with the recast warm start.
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


def _set(s, insts, bc=(0, 0)):
    n, wdt, order, sigt, sigs, src, nsf = slab_batch_arrays(insts)
    s.set_slabs(n, wdt, order, sigt, sigs, source=src, nu_sigma_f=nsf,
                chi=None if nsf is None else [1.0], bc=bc)


def _oracle(s, tol, bc=(0, 0)):
    return T.source_iteration(oracle_slab(s, bc), Qd.gauss_legendre(s.N), tol=tol,
                              itmax=100000, dsa=True)


def _instances(seed, shapes, cmin=0.5, cmax=0.999):
    rng = np.random.default_rng(seed)
    out = []
    for I, N in shapes:
        x = W.cell_centres(I)
        st = rng.uniform(0.5, 2.0, I)
        out.append(W.Slab1G(I=I, N=N, sigt=st, sigs=st * rng.uniform(cmin, cmax, I),
                            Q=W.fourier_source(rng, x)))
    return out


# shapes around the edge-scan chunking (I+1 edges over 32 lanes), staged and
# unstaged warp-path instances
SHAPES = [(1, 2), (2, 4), (31, 8), (32, 16), (63, 8), (64, 32), (95, 6), (500, 16),
          (2048, 32), (2100, 8), (5000, 16)]


def test_fp64_matches_oracle_iteration_for_iteration(solver):
    insts = _instances(1, SHAPES)
    _set(solver, insts)
    phi, info = solver.solve_fixed_source(tol=1e-10, itmax=1000, precision=1, dsa=True,
                                          schedule=1)
    assert np.all(info["status"] == 0)
    for b, (s, g) in enumerate(zip(insts, split(phi, insts))):
        r = _oracle(s, 1e-10)
        assert abs(int(info["iterations"][b]) - r.iterations) <= 1, (s.I, s.N)
        assert rel_l2(g, r.phi[0]) < 1e-9, (s.I, s.N)


def test_block_path_fp64(solver):
    # a whole block per instance: angles over 12 warps, the correction on one
    insts = _instances(2, [(700, 64), (1500, 128), (33, 48)])
    _set(solver, insts)
    phi, info = solver.solve_fixed_source(tol=1e-10, itmax=1000, precision=1, dsa=True,
                                          schedule=2)
    for b, (s, g) in enumerate(zip(insts, split(phi, insts))):
        r = _oracle(s, 1e-10)
        assert abs(int(info["iterations"][b]) - r.iterations) <= 1, (s.I, s.N)
        assert rel_l2(g, r.phi[0]) < 1e-9, (s.I, s.N)


@pytest.mark.parametrize("bc", [(1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("schedule", [1, 2])
def test_reflective_faces_fp64(solver, bc, schedule):
    insts = _instances(3 + bc[0] + 2 * bc[1], [(120, 16), (77, 24)], cmax=0.99)
    _set(solver, insts, bc=bc)
    phi, info = solver.solve_fixed_source(tol=1e-10, itmax=1000, precision=1, dsa=True,
                                          schedule=schedule)
    for b, (s, g) in enumerate(zip(insts, split(phi, insts))):
        r = _oracle(s, 1e-10, bc)
        assert abs(int(info["iterations"][b]) - r.iterations) <= 1, (bc, s.I)
        assert rel_l2(g, r.phi[0]) < 1e-9, (bc, s.I)


def test_fp32_same_rule(solver):
    insts = _instances(4, SHAPES)
    _set(solver, insts)
    phi, info = solver.solve_fixed_source(tol=1e-6, itmax=1000, precision=0, dsa=True)
    for b, (s, g) in enumerate(zip(insts, split(phi, insts))):
        r = _oracle(s, 1e-6)
        assert abs(int(info["iterations"][b]) - r.iterations) <= 1, (s.I, s.N)
        assert rel_l2(g, r.phi[0]) <= 1e-5, (s.I, s.N)


def test_full_4096_slab_batch_sampled(solver):
    insts = W.slab_batch()
    _set(solver, insts)
    _, plain = solver.solve_fixed_source(tol=1e-6, itmax=50000, precision=0)
    phi, info = solver.solve_fixed_source(tol=1e-6, itmax=50000, precision=0, dsa=True)
    assert np.all(info["status"] == 0)
    # the correction removes most of the slowly converging iterations
    assert info["iterations"].mean() * 3 < plain["iterations"].mean()
    parts = split(phi, insts)
    for b in np.random.default_rng(1).choice(len(insts), 6, replace=False):
        s = insts[b]
        r = _oracle(s, 1e-6)
        assert rel_l2(parts[b], r.phi[0]) <= 1e-5, (b, s.I, s.N)
        assert abs(int(info["iterations"][b]) - r.iterations) <= 1


def test_two_groups_and_eigen_fp64(solver):
    rng = np.random.default_rng(11)
    I, G = 60, 2
    sigt = np.stack([rng.uniform(0.8, 1.2, I), rng.uniform(1.5, 2.5, I)])
    S = np.zeros((G, G, I))
    S[0, 0], S[0, 1] = 0.6 * sigt[0], 0.2 * sigt[0]
    S[1, 1], S[1, 0] = 0.9 * sigt[1], 0.05 * sigt[1]
    Q = np.stack([np.ones(I), np.zeros(I)])
    solver.set_slabs([I], [6.0], [8], sigt.reshape(-1), S.reshape(-1), source=Q.reshape(-1))
    phi, info = solver.solve_fixed_source(tol=1e-11, itmax=1000, precision=1, dsa=True)
    P = T.Slab(dx=np.full(I, 0.1), sigt=sigt, sigs=S, Q=Q)
    r = T.source_iteration(P, Qd.gauss_legendre(8), tol=1e-11, dsa=True)
    assert abs(int(info["iterations"][0]) - r.iterations) <= 1
    assert rel_l2(phi, r.phi.reshape(-1)) < 1e-9
    # eigen: the inner iterations carry the correction
    insts = []
    for b, (I, N) in enumerate([(40, 8), (75, 16), (120, 32)]):
        st = np.full(I, 1.0 + 0.1 * b)
        insts.append(W.Slab1G(I=I, N=N, sigt=st, sigs=0.7 * st,
                              nusigf=np.full(I, 0.45 + 0.05 * b)))
    _set(solver, insts)
    k, phi, info = solver.solve_eigen(tol=1e-9, tol_k=1e-11, tol_inner=1e-11, itmax=5000,
                                      precision=1, dsa=True)
    k0, _, info0 = solver.solve_eigen(tol=1e-9, tol_k=1e-11, tol_inner=1e-11, itmax=5000,
                                      precision=1)
    for b, s in enumerate(insts):
        e = T.power_iteration(oracle_slab(s), Qd.gauss_legendre(s.N), tol_k=1e-11,
                              tol_phi=1e-9, tol_inner=1e-11, dsa=True)
        assert abs(k[b] - e.k) < 1e-9
        assert abs(int(info["inner"][b]) - e.inner_total) <= 2 * e.outer
    assert np.all(info["inner"] * 2 < info0["inner"])
    assert np.max(np.abs(k - k0)) < 1e-8


def test_warm_start_with_dsa_keeps_the_answer(solver):
    from paper_2509_01416_gb300 import NOP_NO_DEEPONET, no_config
    insts = _instances(6, [(256, 16), (512, 32), (100, 8)])
    _set(solver, insts)
    solver.no_set(no_config(NOP_NO_DEEPONET, sensors=128, width=128, basis=128),
                  W.deeponet_init(5))
    base, _ = solver.solve_fixed_source(tol=1e-8, itmax=1000, precision=1, dsa=True)
    warm, info = solver.solve_fixed_source(tol=1e-8, itmax=1000, precision=1, dsa=True,
                                           warm_start=1)
    assert np.all(info["status"] == 0)
    assert rel_l2(warm, base) < 1e-6


def test_dsa_needs_isotropic_slabs(solver):
    from paper_2509_01416_gb300 import NopError
    I = 20
    solver.set_slabs([I], [2.0], [8], np.ones(I), np.full(I, 0.5), source=np.ones(I),
                     sigma_s1=np.full(I, 0.1))
    with pytest.raises(NopError):
        solver.solve_fixed_source(tol=1e-6, itmax=100, dsa=True)
    n = 8
    solver.set_xy(n, n, 1.0, 1.0, np.ones(n * n), np.full(n * n, 0.5), source=np.ones(n * n))
    with pytest.raises(NopError):
        solver.solve_fixed_source(tol=1e-6, itmax=100, dsa=True)


def test_near_critical_thick_slab_converges_fast(solver):
    # c = 0.999 over 200 mean free paths: plain source iteration needs
    # thousands of sweeps, the corrected iteration a handful
    I = 400
    s = W.Slab1G(I=I, N=16, sigt=np.full(I, 2.0), sigs=np.full(I, 1.998), Q=np.ones(I), L=100.0)
    _set(solver, [s])
    phi, info = solver.solve_fixed_source(tol=1e-8, itmax=1000, precision=1, dsa=True)
    assert int(info["iterations"][0]) < 30
    r = _oracle(s, 1e-13)
    assert rel_l2(phi, r.phi[0]) < 1e-7
