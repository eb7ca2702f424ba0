"""The diffusion recast (Sec. 3.1, Table 1) on the GPU against the FP64
oracle (oracle/diffusion.py): the model-based solve, the recast iteration
through nop_recast_iterate with the fused 128-wide DeepONet kernel and with
the GEMM path, and a trained operator's recast approaching the true solution
of a new D(x).  The operator computes in BF16 with FP32 accumulation, so the
recast is compared with the oracle run with BF16 operand rounding."""
import numpy as np
import pytest

import workloads as W
from oracle import diffusion as DF
from oracle import neural as NN
from oracle import recast as R
from tests.helpers import rel_l2, split

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


def _batch(seed, shapes, helmholtz=False):
    rng = np.random.default_rng(seed)
    out = [W.diffusion_slab(np.random.default_rng(int(rng.integers(1 << 30))), I,
                            helmholtz=helmholtz) for I in shapes]
    return out


def _set(solver, insts, L=10.0):
    n = np.array([len(d) for d, _, _ in insts], dtype=np.int32)
    solver.set_diffusion(n, np.full(len(n), L), np.concatenate([d for d, _, _ in insts]),
                         np.concatenate([s for _, _, s in insts]),
                         absorption=np.concatenate([a for _, a, _ in insts]))
    return n


@pytest.mark.parametrize("helmholtz", [False, True])
def test_model_solve_matches_oracle(solver, helmholtz):
    insts = _batch(1, [1, 2, 37, 300, 2048], helmholtz)
    n = _set(solver, insts)
    u = solver.diffusion_solve()
    for (D, a, S), g in zip(insts, split(u, [type("I", (), {"I": int(k)}) for k in n])):
        ref = DF.solve(10.0 / len(D), D, a, S)
        assert rel_l2(g, ref) < 1e-12


def _deeponet(solver, width, p, seed, scale_last):
    from paper_2509_01416_gb300 import NOP_NO_DEEPONET, no_config
    P = W.deeponet_init(seed, m=128, width=width, p=p)
    P["b3.W"] *= scale_last
    P["b3.b"] *= scale_last
    cfg = no_config(NOP_NO_DEEPONET, sensors=128, width=width, basis=p, depth=4,
                    sigma_t_star=W.D_STAR[0], sigma_s_star=W.D_STAR[1], length=10.0)
    solver.no_set(cfg, P)
    return P


@pytest.mark.parametrize("width,p", [(64, 32), (128, 128)])
def test_recast_matches_oracle(solver, width, p):
    # 128 x 128 x depth 4 runs the one-launch fused recast, other shapes the
    # GEMM chain; a small last layer makes the recast map a contraction
    insts = _batch(2, [120, 64, 300, 511] + [200] * 13)
    n = _set(solver, insts)
    P = _deeponet(solver, width, p, 11, 2e-3)
    phi, info = solver.recast_iterate(tol=1e-5, itmax=100)
    op = R.DeepONetOp(P, 10.0, 128, quant=NN.bf16_round)
    parts = split(phi, [type("I", (), {"I": int(k)}) for k in n])
    for b, ((D, a, S), g) in enumerate(zip(insts, parts)):
        ref, it, st, _ = DF.recast_deeponet(op, 10.0, D, a, S, W.D_STAR, tol=1e-5, itmax=100)
        assert st == R.OK and info["status"][b] == 0
        assert abs(int(info["iterations"][b]) - it) <= 1, (b, it, info["iterations"][b])
        assert rel_l2(g, ref) < 1e-2


def test_trained_operator_recast_approaches_the_new_solution(solver):
    """A DeepONet trained on p* = (D* = 1, Sigma_a* = 0) solutions only (GRF
    sources, solved by nop_diffusion_solve) recasts Table 1's Helmholtz row,
    -u'' - k^2(x) u = S: the recast answer is closer to the true solution
    than the operator applied once at p* (the recast's point, Eq. 7).  (The
    diffusion row's mismatch -((D - D*) u')' takes second differences of the
    operator's own output, which amplify its error by 1/h^2; with a trained
    operator that recast does not improve on one application -- the caveat
    Sec. 3.1 attaches to approximated operator differences.  Its machinery
    is checked above with a contracting operator.)"""
    from paper_2509_01416_gb300 import train as TR
    _deeponet(solver, 128, 128, 21, 1.0)
    cfg = solver.no_cfg
    U, X, Y = TR.diffusion_training_set(solver, cfg, W.training_sources(22, 1000, 128))
    hist = TR.train(solver, U, X, Y, steps=6000, batch=100, seed=23, lr=1e-3)
    assert hist[-50:].mean() < 0.05 * hist[:50].mean()
    insts = _batch(3, [256] * 8, helmholtz=True)
    n = _set(solver, insts)
    # stop at the operator's own accuracy (BF16 operands), as the warm starts do
    rec, info = solver.recast_iterate(tol=1e-3, itmax=50)
    one, _ = solver.recast_iterate(tol=1e300, itmax=1)     # N[S] at p*
    true = solver.diffusion_solve()
    print("\nHelmholtz recast: error %.3g after %s iterations (status %s); one application %.3g"
          % (rel_l2(rec, true), list(info["iterations"]), list(info["status"]), rel_l2(one, true)))
    assert np.all(info["status"] == 0)
    assert rel_l2(rec, true) < 0.5 * rel_l2(one, true), (rel_l2(rec, true), rel_l2(one, true))
