"""GPU parity of the 1D slab solver (C ABI) against the FP64 oracle.

Tolerances: FP64 sweeps agree with the oracle to rounding (1e-9 relative or
tighter).  FP32 sweeps: scalar flux relative L2 <= 1e-5 and |dk| <= 1e-6
against the oracle, the bar the workloads state.  Where both sides stop at
the same relative-change tolerance they are compared iterate to iterate;
where the GPU answer is compared with a fully converged oracle, the GPU runs
to a tolerance tight enough that its truncation error is below the bar.
"""
import numpy as np
import pytest

import workloads as W
from oracle import quadrature as Qd
from oracle import transport as T
from tests.helpers import eigen_slab_config3, oracle_slab, rel_l2, slab_batch_arrays, split

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


def test_gauss_legendre_on_device_matches_oracle(solver):
    orders = [2, 4, 8, 16, 32, 64, 128, 10, 26]
    insts = [W.Slab1G(I=3, N=N, sigt=np.ones(3), sigs=np.zeros(3), Q=np.ones(3)) for N in orders]
    _set(solver, insts)
    for b, N in enumerate(orders):
        mu, _, w = solver.quadrature(b)
        m0, w0 = Qd.gauss_legendre(N)
        assert np.max(np.abs(mu - m0)) < 1e-14 and np.max(np.abs(w - w0)) < 1e-14


def test_uniform_slab_fp64_matches_oracle_iteration_for_iteration(solver):
    c = W.uniform_slab_s16()
    _set(solver, [c])
    phi, info = solver.solve_fixed_source(tol=1e-8, itmax=10000, precision=1)
    r = T.source_iteration(oracle_slab(c), Qd.gauss_legendre(c.N), tol=1e-8)
    assert abs(int(info["iterations"][0]) - r.iterations) <= 1
    assert rel_l2(phi, r.phi[0]) < 1e-10
    assert info["status"][0] == 0


def test_heterogeneous_slab_fp32_within_workload_tolerance(solver):
    c = W.hetero_slab_s32()
    _set(solver, [c])
    quad = Qd.gauss_legendre(c.N)
    phi, info = solver.solve_fixed_source(tol=1e-6, itmax=20000, precision=0)
    same_rule = T.source_iteration(oracle_slab(c), quad, tol=1e-6)
    assert rel_l2(phi, same_rule.phi[0]) <= 1e-5
    assert abs(int(info["iterations"][0]) - same_rule.iterations) <= 2
    conv = T.source_iteration(oracle_slab(c), quad, tol=1e-13)
    tight, info2 = solver.solve_fixed_source(tol=2e-7, itmax=40000, precision=0)
    assert rel_l2(tight, conv.phi[0]) <= 1e-5, info2


def test_three_region_eigen_fp32(solver):
    c = eigen_slab_config3()
    _set(solver, [c])
    quad = Qd.gauss_legendre(c.N)
    # same stopping rule on both sides (tol 1e-6 flux, 1e-7 in k, inner 1e-6)
    k, phi, info = solver.solve_eigen(tol=1e-6, tol_k=1e-7, tol_inner=1e-6, itmax=2000,
                                      precision=0)
    same = T.power_iteration(oracle_slab(c), quad, tol_k=1e-7, tol_phi=1e-6, tol_inner=1e-6)
    assert abs(k[0] - same.k) <= 1e-6, (k[0], same.k, info)
    assert rel_l2(phi, same.phi[0]) <= 1e-5
    # run to a tolerance whose truncation error is below the bar: converged oracle
    e = T.power_iteration(oracle_slab(c), quad, tol_k=1e-12, tol_phi=1e-10, tol_inner=1e-12)
    assert 0.9 <= e.k <= 1.1 and abs(e.k - c.k_target) < 1e-9
    k2, phi2, info2 = solver.solve_eigen(tol=1e-7, tol_k=1e-9, tol_inner=1e-7, itmax=5000,
                                         itmax_inner=2000, precision=0, check=False)
    assert abs(k2[0] - e.k) <= 1e-6, (k2[0], e.k, info2)
    assert rel_l2(phi2, e.phi[0]) <= 1e-5


def _table10():
    S = np.array([[0.024, 0.171, 0.033], [0.0, 0.6, 0.275], [0.0, 0.0, 2.0]])
    nu = np.array([3.0, 2.5, 2.0])
    st = np.array([0.24, 0.975, 3.0])
    sf = np.array([0.006, 0.06, 0.9])
    chi = np.array([0.96, 0.04, 0.0])
    return S, nu * sf, st, chi


@pytest.mark.parametrize("precision", [1, 0])
def test_table10_three_group_eigenvalue_on_gpu(solver, precision):
    S, nsf, st, chi = _table10()
    I = 100
    solver.set_slabs([I], [10.0], [32], np.repeat(st, I), np.repeat(S.reshape(-1), I),
                     nu_sigma_f=np.repeat(nsf, I), chi=chi)
    P = T.Slab(dx=np.full(I, 0.1), sigt=st[:, None] * np.ones(I), sigs=S[:, :, None] * np.ones(I),
               nusigf=nsf[:, None] * np.ones(I), chi=chi)
    quad = Qd.gauss_legendre(32)
    if precision == 1:
        # FP64: same stopping rule, compared iterate to iterate
        k, phi, info = solver.solve_eigen(tol=1e-7, tol_k=1e-9, tol_inner=1e-8, itmax=500,
                                          precision=1)
        e = T.power_iteration(P, quad, tol_k=1e-9, tol_phi=1e-7, tol_inner=1e-8)
        assert abs(k[0] - e.k) <= 1e-10, (k[0], e.k)
        assert rel_l2(phi, e.phi.reshape(-1)) <= 1e-9
    else:
        k, phi, info = solver.solve_eigen(tol=1e-7, tol_k=1e-9, tol_inner=1e-7, itmax=500,
                                          itmax_inner=3000, precision=0, check=False)
        e = T.power_iteration(P, quad, tol_k=1e-12, tol_phi=1e-10, tol_inner=1e-12)
        assert abs(k[0] - e.k) <= 1e-6, (k[0], e.k, info)
        assert rel_l2(phi, e.phi.reshape(-1)) <= 1e-5
    # the paper's printed value (Table 10)
    assert abs(k[0] - 1.30621) <= 5e-6, (k, info)


@pytest.mark.parametrize("bc", [(1, 1), (1, 0), (0, 1)])
def test_reflective_boundaries(solver, bc):
    rng = np.random.default_rng(sum(bc) * 7 + bc[0])
    I = 37
    st = rng.uniform(0.5, 1.5, I)
    inst = W.Slab1G(I=I, N=12, sigt=st, sigs=st * rng.uniform(0.3, 0.95, I),
                    Q=rng.uniform(0, 1, I), L=6.0)
    _set(solver, [inst], bc=bc)
    phi, info = solver.solve_fixed_source(tol=1e-13, itmax=200000, precision=1)
    r = T.source_iteration(oracle_slab(inst, bc), Qd.gauss_legendre(12), tol=1e-13,
                           itmax=200000)
    assert rel_l2(phi, r.phi[0]) < 1e-9
    if bc == (1, 1):
        flat = W.Slab1G(I=20, N=8, sigt=np.full(20, 1.3), sigs=np.full(20, 0.9), Q=np.full(20, 2.0))
        _set(solver, [flat], bc=bc)
        for prec, tol in ((1, 1e-10), (0, 1e-5)):
            phi, _ = solver.solve_fixed_source(tol=1e-12 if prec else 1e-7, itmax=200000,
                                               precision=prec, check=False)
            assert np.max(np.abs(phi - 5.0)) / 5.0 < tol


def test_ragged_batch_fp64_every_instance(solver):
    rng = np.random.default_rng(21)
    insts = []
    for b in range(40):
        I = int(rng.integers(1, 300)) if b > 1 else (1 if b == 0 else 2)
        N = 2 * int(rng.integers(1, 17)) if b > 1 else 2
        insts.append(W.slab_instance(np.random.default_rng(b), I, N))
    _set(solver, insts)
    phi, info = solver.solve_fixed_source(tol=1e-12, itmax=200000, precision=1)
    for s, ph in zip(insts, split(phi, insts)):
        r = T.source_iteration(oracle_slab(s), Qd.gauss_legendre(s.N), tol=1e-12, itmax=200000)
        assert rel_l2(ph, r.phi[0]) < 1e-9, (s.I, s.N)
    assert np.all(info["status"] == 0)


def test_ragged_batch_fp32_same_rule(solver):
    rng = np.random.default_rng(22)
    insts = [W.slab_instance(np.random.default_rng(100 + b), int(rng.integers(20, 400)),
                             2 * int(rng.integers(4, 33))) for b in range(64)]
    _set(solver, insts)
    phi, info = solver.solve_fixed_source(tol=1e-6, itmax=50000, precision=0)
    for b, (s, ph) in enumerate(zip(insts, split(phi, insts))):
        if b % 4:
            continue
        r = T.source_iteration(oracle_slab(s), Qd.gauss_legendre(s.N), tol=1e-6)
        assert rel_l2(ph, r.phi[0]) <= 1e-5, (s.I, s.N)


def test_full_4096_slab_batch_sampled(solver):
    insts = W.slab_batch()
    _set(solver, insts)
    phi, info = solver.solve_fixed_source(tol=1e-6, itmax=50000, precision=0)
    assert np.all(info["status"] == 0)
    parts = split(phi, insts)
    for b in np.random.default_rng(0).choice(len(insts), 6, replace=False):
        s = insts[b]
        r = T.source_iteration(oracle_slab(s), Qd.gauss_legendre(s.N), tol=1e-6)
        assert rel_l2(parts[b], r.phi[0]) <= 1e-5, (b, s.I, s.N)
        assert abs(int(info["iterations"][b]) - r.iterations) <= 2


def test_multigroup_upscatter_fixed_source_fp64(solver):
    rng = np.random.default_rng(11)
    I, G = 30, 2
    sigt = rng.uniform(0.8, 1.6, (G, I))
    S = np.zeros((G, G, I))
    S[0, 0], S[0, 1] = 0.3 * sigt[0], 0.3 * sigt[0]
    S[1, 1], S[1, 0] = 0.5 * sigt[1], 0.2 * sigt[1]
    Q = rng.uniform(0, 1, (G, I))
    solver.set_slabs([I], [7.0], [8], sigt.reshape(-1), S.reshape(-1), source=Q.reshape(-1))
    phi, info = solver.solve_fixed_source(tol=1e-13, itmax=100000, precision=1)
    P = T.Slab(dx=np.full(I, 7.0 / I), sigt=sigt, sigs=S, Q=Q)
    r = T.source_iteration(P, Qd.gauss_legendre(8), tol=1e-13)
    assert rel_l2(phi, r.phi.reshape(-1)) < 1e-10


def test_eigen_batch_of_different_shapes(solver):
    insts = []
    for b, (I, N) in enumerate([(40, 8), (75, 16), (120, 32), (9, 4)]):
        st = np.full(I, 1.0 + 0.1 * b)
        insts.append(W.Slab1G(I=I, N=N, sigt=st, sigs=0.5 * st, nusigf=np.full(I, 0.7 + 0.05 * b)))
    _set(solver, insts)
    k, phi, info = solver.solve_eigen(tol=1e-10, tol_k=1e-12, tol_inner=1e-12, itmax=5000,
                                      precision=1)
    for b, s in enumerate(insts):
        e = T.power_iteration(oracle_slab(s), Qd.gauss_legendre(s.N), tol_k=1e-13,
                              tol_phi=1e-11, tol_inner=1e-13)
        assert abs(k[b] - e.k) < 1e-9


def test_errors_and_caps(solver):
    from paper_2509_01416_gb300 import NopError
    with pytest.raises(NopError):
        solver.set_slabs([5], [1.0], [3], np.ones(5), np.zeros(5), source=np.ones(5))
    with pytest.raises(NopError):
        solver.set_slabs([5], [1.0], [4], -np.ones(5), np.zeros(5), source=np.ones(5))
    c = W.uniform_slab_s16()
    _set(solver, [c])
    phi, info = solver.solve_fixed_source(tol=1e-12, itmax=3, precision=0, check=False)
    assert info["rc"] == -4 and info["status"][0] == -4 and info["iterations"][0] == 3
    with pytest.raises(NopError):
        solver.solve_eigen(tol=1e-6)         # no production cross section


# ------------------------------------------------- anisotropic scattering (Eq. 25)
def _set_aniso(s, insts, bc=(0, 0)):
    n, wdt, order, sigt, sigs, src, _ = slab_batch_arrays(insts)
    s1 = np.concatenate([i.sigs1 if i.sigs1 is not None else np.zeros(i.I) for i in insts])
    s.set_slabs(n, wdt, order, sigt, sigs, source=src, bc=bc, sigma_s1=s1)


def _aniso_batch():
    out = []
    for b, (I, N, a1) in enumerate([(40, 4, 0.3), (75, 8, -0.2), (120, 16, 0.5), (33, 32, 0.0),
                                    (64, 10, 0.25)]):
        rng = np.random.default_rng(50 + b)
        x = W.cell_centres(I)
        st = 1.0 + 0.4 * np.sin(2 * np.pi * x / W.L_SLAB + b)
        c = rng.uniform(0.5, 0.9, I)
        out.append(W.Slab1G(I=I, N=N, sigt=st, sigs=c * st, Q=W.fourier_source(rng, x),
                            sigs1=a1 * c * st))
    return out


@pytest.mark.parametrize("bc", [(0, 0), (1, 0), (0, 1)])
def test_anisotropic_fp64_matches_oracle(solver, bc):
    insts = _aniso_batch()
    _set_aniso(solver, insts, bc=bc)
    phi, info = solver.solve_fixed_source(tol=1e-12, itmax=100000, precision=1)
    for s, g in zip(insts, split(phi, insts)):
        r = T.source_iteration(oracle_slab(s, bc=bc), Qd.gauss_legendre(s.N), tol=1e-12,
                               itmax=100000)
        assert rel_l2(g, r.phi[0]) < 1e-9


def test_anisotropic_case_fp32_within_tolerance(solver):
    # Sec. 5.1 case with Sigma_s1 = 0.3: FP32 sweeps, same stopping rule
    s = W.aniso_slab()
    _set_aniso(solver, [s])
    phi, info = solver.solve_fixed_source(tol=1e-6, itmax=100000, precision=0)
    r = T.source_iteration(oracle_slab(s), Qd.gauss_legendre(s.N), tol=1e-6, itmax=100000)
    assert abs(int(info["iterations"][0]) - r.iterations) <= 1
    assert rel_l2(phi, r.phi[0]) < 1e-5
    # the anisotropic term is not negligible in this case
    iso = T.source_iteration(T.uniform_slab(s.I, s.L, s.sigt, s.sigs, Q=s.Q),
                             Qd.gauss_legendre(s.N), tol=1e-10)
    assert rel_l2(iso.phi[0], r.phi[0]) > 1e-3


def test_anisotropic_warm_start_keeps_the_answer(solver):
    # the recast warm start ignores Sigma_s1 (the operator knows isotropic
    # scattering only); the model solve restores the anisotropic answer
    from paper_2509_01416_gb300 import NOP_NO_DEEPONET, no_config
    insts = [W.aniso_slab(seed=30 + b) for b in range(3)]
    _set_aniso(solver, insts)
    P = W.deeponet_init(4, m=128, width=64, p=32)
    P["b3.W"] *= 2e-3
    P["b3.b"] *= 2e-3
    solver.no_set(no_config(NOP_NO_DEEPONET, sensors=128, width=64, basis=32), P)
    plain, _ = solver.solve_fixed_source(tol=1e-10, itmax=100000, precision=1)
    warm, wi = solver.solve_fixed_source(tol=1e-10, itmax=100000, precision=1, warm_start=1)
    assert wi["recast_iterations"] > 0
    assert rel_l2(warm, plain) < 1e-8


def test_anisotropic_rejected_outside_fixed_source_slabs(solver):
    from paper_2509_01416_gb300 import NopError
    s = W.aniso_slab()
    n, wdt, order, sigt, sigs, src, _ = slab_batch_arrays([s])
    with pytest.raises(NopError):
        solver.set_slabs(n, wdt, order, sigt, sigs, nu_sigma_f=0.5 * sigt, chi=[1.0],
                         sigma_s1=s.sigs1)


# ------------------------------------------------------------ lane layouts
def _direct_batch(seed=70):
    """Vacuum slabs whose orders take the direct lanes (N >= 24): cell counts
    from 1 to 5000 (ragged ring blocks of 32, chunks of 12 warps shorter than
    one block), orders up to 128 (4 angles per lane)."""
    rng = np.random.default_rng(seed)
    shapes = [(1, 24), (31, 32), (32, 40), (33, 64), (97, 26), (300, 128), (2047, 48),
              (5000, 30), (11, 64), (640, 56)]
    return [W.slab_instance(np.random.default_rng(int(rng.integers(1 << 30))), I, N)
            for I, N in shapes]


@pytest.mark.parametrize("schedule", [1, 2])
def test_direct_lanes_fp64_iterate_for_iterate(solver, schedule):
    """One warp per instance (schedule 1) and a 12-warp team per instance
    (schedule 2, chunk maps handed across warps): every source iterate equals
    the oracle's to rounding, so the iteration counts agree too."""
    insts = _direct_batch()
    _set(solver, insts)
    phi, info = solver.solve_fixed_source(tol=1e-9, itmax=100000, precision=1,
                                          schedule=schedule)
    for b, (s, ph) in enumerate(zip(insts, split(phi, insts))):
        r = T.source_iteration(oracle_slab(s), Qd.gauss_legendre(s.N), tol=1e-9, itmax=100000)
        assert abs(int(info["iterations"][b]) - r.iterations) <= 1, (s.I, s.N)
        assert rel_l2(ph, r.phi[0]) < 1e-10, (s.I, s.N)


def test_direct_and_chunked_layouts_agree_fp32(solver):
    """The same FP32 batch on the direct lanes and on the chunked lanes: both
    meet the workload bar against the oracle under the same stopping rule."""
    insts = _direct_batch(71)
    _set(solver, insts)
    d, di = solver.solve_fixed_source(tol=1e-6, itmax=100000, precision=0)
    c, ci = solver.solve_fixed_source(tol=1e-6, itmax=100000, precision=0, chunked=True)
    for b, (s, pd, pc) in enumerate(zip(insts, split(d, insts), split(c, insts))):
        r = T.source_iteration(oracle_slab(s), Qd.gauss_legendre(s.N), tol=1e-6, itmax=100000)
        assert rel_l2(pd, r.phi[0]) <= 1e-5, (s.I, s.N)
        assert rel_l2(pc, r.phi[0]) <= 1e-5, (s.I, s.N)
        assert abs(int(di["iterations"][b]) - r.iterations) <= 1, (s.I, s.N)


@pytest.mark.parametrize("schedule", [1, 2])
def test_direct_lanes_multigroup_eigen_fp64(solver, schedule):
    """Two groups with up- and down-scatter, power iteration, on the direct
    lanes (S32, vacuum) against the oracle."""
    rng = np.random.default_rng(72)
    I, G = 150, 2
    sigt = rng.uniform(0.8, 1.6, (G, I))
    S = np.zeros((G, G, I))
    S[0, 0], S[0, 1] = 0.4 * sigt[0], 0.2 * sigt[0]
    S[1, 1], S[1, 0] = 0.6 * sigt[1], 0.1 * sigt[1]
    nsf = np.stack([0.05 * np.ones(I), 0.3 * np.ones(I)])
    chi = np.array([0.9, 0.1])
    solver.set_slabs([I], [8.0], [32], sigt.reshape(-1), S.reshape(-1),
                     nu_sigma_f=nsf.reshape(-1), chi=chi)
    k, phi, info = solver.solve_eigen(tol=1e-10, tol_k=1e-12, tol_inner=1e-12, itmax=5000,
                                      precision=1, schedule=schedule)
    P = T.Slab(dx=np.full(I, 8.0 / I), sigt=sigt, sigs=S, nusigf=nsf, chi=chi)
    e = T.power_iteration(P, Qd.gauss_legendre(32), tol_k=1e-13, tol_phi=1e-11,
                          tol_inner=1e-13)
    assert abs(k[0] - e.k) < 1e-9
    assert rel_l2(phi, e.phi.reshape(-1)) < 1e-8
