"""GPU parity of the DeepONet kernels (C ABI) against the FP64 oracle.

The kernels compute in BF16 operands with FP32 accumulation.  The oracle is
run twice: with BF16 rounding at the same operand points (the tight bar,
limited by FP32 accumulation order and rare double roundings) and in plain
FP64 (a looser bar set by BF16 operand rounding, 2^-9 relative per operand).
"""
import numpy as np
import pytest

import workloads as W
from oracle import neural as NN
from oracle import recast as R
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


def _cfg(**kw):
    from paper_2509_01416_gb300 import NOP_NO_DEEPONET, no_config
    return no_config(NOP_NO_DEEPONET, **kw)


def _small(solver, seed=1, m=32, width=48, p=40, depth=4, scale_last=1.0):
    P = W.deeponet_init(seed, m=m, width=width, p=p, depth=depth)
    P["b%d.W" % (depth - 1)] *= scale_last
    P["b%d.b" % (depth - 1)] *= scale_last
    cfg = _cfg(sensors=m, width=width, basis=p, depth=depth)
    solver.no_set(cfg, P)
    return cfg, P


def test_forward_matches_oracle(solver):
    cfg, P = _small(solver)
    rng = np.random.default_rng(3)
    U = rng.standard_normal((37, 32))
    X = rng.uniform(0, 1, (29, 1))
    gpu = solver.no_forward(U, X[:, 0])
    q, _ = NN.deeponet_forward(P, U, X, quant=NN.bf16_round)
    f, _ = NN.deeponet_forward(P, U, X)
    assert rel_l2(gpu, q) < 2e-3
    assert rel_l2(gpu, f) < 3e-2


def test_gradients_match_oracle(solver):
    cfg, P = _small(solver, seed=2)
    rng = np.random.default_rng(4)
    U = rng.standard_normal((21, 32))
    X = rng.uniform(0, 1, (17, 1))
    Y = rng.standard_normal((21, 17))
    loss, g = solver.no_loss_grad(U, Y, X[:, 0])
    out, cache = NN.deeponet_forward(P, U, X, quant=NN.bf16_round)
    l0, dout = NN.mse(out, Y)
    g0 = NN.deeponet_backward(P, cache, dout, quant=NN.bf16_round)
    assert abs(loss - l0) < 1e-3 * l0
    for k in g0:
        assert rel_l2(g[k], g0[k]) < 2e-2, k


def test_adam_step_on_device(solver):
    cfg, P = _small(solver, seed=5)
    rng = np.random.default_rng(6)
    U = rng.standard_normal((16, 32))
    X = rng.uniform(0, 1, 9)
    Y = rng.standard_normal((16, 9))
    p0 = solver.no_get()
    _, g = solver.no_loss_grad(U, Y, X)
    solver.no_train(U, Y, X, steps=1, batch=16, lr=1e-3, order=np.arange(16))
    p1 = solver.no_get()
    for k in p0:
        gk = g[k].astype(np.float32)
        expect = p0[k] - 1e-3 * gk / (np.abs(gk) + 1e-8)
        assert np.max(np.abs(p1[k] - expect)) < 2e-6, k


def test_three_adam_steps_match_oracle(solver):
    """Three consecutive Adam steps (the moments and the step count persist
    across nop_no_train calls) against oracle.neural.adam_step fed with the
    device's own gradient of each step, moments carried in FP64."""
    cfg, P = _small(solver, seed=8)
    rng = np.random.default_rng(9)
    U = rng.standard_normal((16, 32))
    X = rng.uniform(0, 1, 9)
    Y = rng.standard_normal((16, 9))
    p = solver.no_get()
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v2 = {k: np.zeros_like(v) for k, v in p.items()}
    for t in (1, 2, 3):
        _, g = solver.no_loss_grad(U, Y, X)
        g = {k: a.astype(np.float32).astype(np.float64) for k, a in g.items()}
        expect = {k: a.copy() for k, a in p.items()}
        NN.adam_step(expect, g, m, v2, t, lr=1e-3)
        solver.no_train(U, Y, X, steps=1, batch=16, lr=1e-3, order=np.arange(16))
        p = solver.no_get()
        for k in p:
            assert np.max(np.abs(p[k] - expect[k])) < 2e-6, (t, k)
        # continue from the device's parameters (FP32) so the steps stay comparable
        p = {k: a.astype(np.float64) for k, a in p.items()}


def test_input_map_matches_oracle_projection(solver):
    rng = np.random.default_rng(7)
    insts = [W.slab_instance(np.random.default_rng(b), I, 8) for b, I in
             enumerate([64, 100, 128, 333, 1000])]
    n, wdt, order, sigt, sigs, src, _ = slab_batch_arrays(insts)
    solver.set_slabs(n, wdt, order, sigt, sigs, source=src)
    _small(solver, m=128, width=32, p=16)
    field = rng.uniform(-1, 2, int(n.sum()))
    got = solver.no_sensors(field)
    for b, f in enumerate(split(field, insts)):
        edges = np.linspace(0, 10.0, insts[b].I + 1)
        ref = R.projection_matrix(edges, 128, 10.0) @ f
        assert np.max(np.abs(got[b] - ref)) < 1e-5 * (1 + np.max(np.abs(ref)))


def _setup_instances(solver, Is, seed=0):
    insts = [W.slab_instance(np.random.default_rng(seed + b), I, 8) for b, I in enumerate(Is)]
    n, wdt, order, sigt, sigs, src, _ = slab_batch_arrays(insts)
    solver.set_slabs(n, wdt, order, sigt, sigs, source=src)
    return insts


@pytest.mark.parametrize("width,p", [(64, 32), (128, 128)])
def test_predict_matches_oracle(solver, width, p):
    # 128 x 128 x depth 4 takes the fused trunk kernel, other shapes the GEMM chain
    insts = _setup_instances(solver, [100, 256, 77])
    cfg, P = _small(solver, m=128, width=width, p=p, seed=9)
    rng = np.random.default_rng(8)
    srcs = [rng.uniform(-0.5, 1.0, s.I) for s in insts]
    got = split(solver.no_predict(np.concatenate(srcs)), insts)
    op = R.DeepONetOp(P, 10.0, 128, quant=NN.bf16_round)
    for s, src, g in zip(insts, srcs, got):
        edges = np.linspace(0, 10.0, s.I + 1)
        beta = op.coef((R.projection_matrix(edges, 128, 10.0) @ src)[None])
        ref = op.eval(beta, (np.arange(s.I) + 0.5) / s.I)[0]
        assert rel_l2(g, ref) < 5e-3


def test_tensor_core_wait_limit_reports_timeout_and_recovers(solver):
    """Failure detection without a fault: with the completion-wait bound at 0
    the fused trunk kernel gives up at its first wait, lets the committed
    products finish, frees its tensor memory and returns; the call reports
    NOP_ETIMEOUT, and the same context then reproduces the normal result."""
    from paper_2509_01416_gb300 import NopError, capi
    insts = _setup_instances(solver, [100, 256, 77])
    _small(solver, m=128, width=128, p=128, seed=9)
    rng = np.random.default_rng(8)
    src = np.concatenate([rng.uniform(-0.5, 1.0, s.I) for s in insts])
    good = solver.no_predict(src)
    solver.set_wait_limit(0)
    try:
        with pytest.raises(NopError) as e:
            solver.no_predict(src)
        assert e.value.code == capi.NOP_ETIMEOUT
    finally:
        solver.set_wait_limit(-1)
    assert np.array_equal(solver.no_predict(src), good)


@pytest.mark.parametrize("width,p", [(64, 32), (128, 128)])
def test_recast_matches_oracle(solver, width, p):
    # small last-layer weights make the recast map a contraction for random
    # nets; 128 x 128 x depth 4 runs the fused one-launch iteration
    insts = _setup_instances(solver, [120, 64, 300, 511] + [200] * 17, seed=20)
    cfg, P = _small(solver, m=128, width=width, p=p, seed=11, scale_last=2e-3)
    phi, info = solver.recast_iterate(tol=1e-5, itmax=100)
    op = R.DeepONetOp(P, 10.0, 128, quant=NN.bf16_round)
    for b, (s, g) in enumerate(zip(insts, split(phi, insts))):
        ref, it, st, _ = R.recast_deeponet(op, oracle_slab(s), W.P_STAR, tol=1e-5, itmax=100)
        assert st == R.OK and info["status"][b] == 0
        assert abs(int(info["iterations"][b]) - it) <= 1
        assert rel_l2(g, ref) < 1e-2


@pytest.mark.parametrize("width,p", [(64, 32), (128, 128)])
def test_recast_divergence_falls_back(solver, width, p):
    # an operator with a large output scale makes the recast map expand
    insts = _setup_instances(solver, [100], seed=30)
    cfg, P = _small(solver, m=128, width=width, p=p, seed=12, scale_last=50.0)
    phi, info = solver.recast_iterate(tol=1e-8, itmax=200)
    if info["status"][0] == -5:          # diverged: the prediction is the plain zero guess
        assert np.all(phi == 0)
    # the warm-started solve still reaches the plain solution
    plain, _ = solver.solve_fixed_source(tol=1e-6, precision=0)
    warm, wi = solver.solve_fixed_source(tol=1e-6, precision=0, warm_start=1)
    assert rel_l2(warm, plain) < 2e-5


def test_trained_operator_cuts_iterations(solver):
    """Train at p* on solver-generated GRF solutions (App. A1 recipe, fewer
    samples and steps), then warm-start the heterogeneous 512-cell slab: the
    recast warm start must cut source iterations and leave the answer alone."""
    from paper_2509_01416_gb300 import train as TR
    cfg = _cfg(sensors=128, width=128, basis=128, depth=4)
    solver.no_set(cfg, W.deeponet_init(0))
    src = W.training_sources(1, 500, 512)
    U, X, Y, _ = TR.deeponet_training_set(solver, cfg, src, order=32)
    hist = TR.train(solver, U, X, Y, steps=1500, batch=100, seed=2)
    assert hist[-50:].mean() < 0.2 * hist[:50].mean()
    c = W.hetero_slab_s32()
    n, wdt, order, sigt, sigs, s2, _ = slab_batch_arrays([c])
    solver.set_slabs(n, wdt, order, sigt, sigs, source=s2)
    plain, pi = solver.solve_fixed_source(tol=1e-6, precision=0)
    warm, wi = solver.solve_fixed_source(tol=1e-6, precision=0, warm_start=1, recast_tol=1e-3)
    assert wi["recast_status"] in (0, -4)
    assert int(wi["iterations"][0]) < int(pi["iterations"][0])
    assert rel_l2(warm, plain) <= 2e-5
