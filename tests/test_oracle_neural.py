"""Pins for the FP64 neural-operator oracle (DeepONet, FNO, MSE, Adam).

Independent checks: the paper's printed parameter counts (App. A1), central
finite differences of the loss for every backward pass, numpy's FFT for the
truncated spectral transforms, torch's bfloat16 rounding for the precision
model, and Adam's closed-form first step.
"""
import numpy as np
import pytest

from oracle import neural as NN
from workloads import deeponet_init, fno1d_init, fno2d_init


def _dense_mlp(rng, dims):
    return [(rng.standard_normal((dims[i + 1], dims[i])), rng.standard_normal(dims[i + 1]))
            for i in range(len(dims) - 1)]


def test_paper_deeponet_parameter_count():
    # App. A1: BN [100,200,200,100], TN [1,200,200,100] -> 141,200 parameters
    rng = np.random.default_rng(0)
    P = {}
    for net, dims in (("b", [100, 200, 200, 100]), ("t", [1, 200, 200, 100])):
        for l, (W, b) in enumerate(_dense_mlp(rng, dims)):
            P["%s%d.W" % (net, l)], P["%s%d.b" % (net, l)] = W, b
    assert NN.param_count(P) == 141200


def test_paper_fno_parameter_count():
    # App. A1: lifting width 64, 4 Fourier layers, 16 modes -> 549,569
    P = fno1d_init(0, width=64, modes=16, layers=4, proj=128)
    assert NN.param_count(P) == 549569


def _fd_check(loss_fn, params, grads, keys, n_probe=6, eps=1e-6, rtol=1e-6):
    rng = np.random.default_rng(42)
    for k in keys:
        flat = params[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(n_probe, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = loss_fn()
            flat[idx] = old - eps
            lm = loss_fn()
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = grads[k].reshape(-1)[idx]
            assert abs(fd - an) <= rtol * max(1.0, abs(fd)) + 1e-9, (k, idx, fd, an)


def test_deeponet_backward_matches_finite_differences():
    P = deeponet_init(1, m=12, width=10, p=8, depth=4)
    rng = np.random.default_rng(2)
    U = rng.standard_normal((5, 12))
    X = rng.uniform(0, 1, (7, 1))
    Y = rng.standard_normal((5, 7))

    def loss():
        return NN.mse(NN.deeponet_forward(P, U, X)[0], Y)[0]

    out, cache = NN.deeponet_forward(P, U, X)
    _, dout = NN.mse(out, Y)
    grads = NN.deeponet_backward(P, cache, dout)
    _fd_check(loss, P, grads, sorted(P))


def test_fno1d_backward_matches_finite_differences():
    P = fno1d_init(3, width=6, modes=4, layers=2, proj=8)
    rng = np.random.default_rng(4)
    n = 16
    S = rng.standard_normal((3, n))
    xc = (np.arange(n) + 0.5) / n
    Y = rng.standard_normal((3, n))

    def loss():
        return NN.mse(NN.fno1d_forward(P, S, xc, n_layers=2)[0], Y)[0]

    out, cache = NN.fno1d_forward(P, S, xc, n_layers=2)
    _, dout = NN.mse(out, Y)
    grads = NN.fno1d_backward(P, cache, dout, n_layers=2)
    _fd_check(loss, P, grads, sorted(P))


def test_fno2d_backward_matches_finite_differences():
    P = fno2d_init(5, width=4, modes=3, layers=2, proj=6)
    rng = np.random.default_rng(6)
    ny, nx = 8, 10
    S = rng.standard_normal((2, ny, nx))
    yc, xc = (np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx
    Y = rng.standard_normal((2, ny, nx))

    def loss():
        return NN.mse(NN.fno2d_forward(P, S, yc, xc, n_layers=2)[0], Y)[0]

    out, cache = NN.fno2d_forward(P, S, yc, xc, n_layers=2)
    _, dout = NN.mse(out, Y)
    grads = NN.fno2d_backward(P, cache, dout, n_layers=2)
    _fd_check(loss, P, grads, sorted(P))


def test_spectral1d_matches_numpy_fft():
    rng = np.random.default_rng(8)
    B, n, C, O, K = 2, 24, 3, 4, 5
    v = rng.standard_normal((B, n, C))
    Rr, Ri = rng.standard_normal((K, C, O)), rng.standard_normal((K, C, O))
    u, _ = NN.spectral1d_forward(v, Rr, Ri)
    vh = np.fft.rfft(v, axis=1)[:, :K]
    wh = np.einsum("bkc,kco->bko", vh, Rr + 1j * Ri)
    full = np.zeros((B, n // 2 + 1, O), complex)
    full[:, :K] = wh
    ref = np.fft.irfft(full, n=n, axis=1)
    assert np.max(np.abs(u - ref)) < 1e-12


def test_spectral2d_matches_numpy_fft():
    rng = np.random.default_rng(9)
    B, ny, nx, C, O, m1, m2 = 2, 12, 10, 2, 3, 3, 4
    v = rng.standard_normal((B, ny, nx, C))
    R = [rng.standard_normal((m1, m2, C, O)) for _ in range(4)]
    u, _ = NN.spectral2d_forward(v, *R)
    vh = np.fft.rfft2(v, axes=(1, 2))
    full = np.zeros((B, ny, nx // 2 + 1, O), complex)
    full[:, :m1, :m2] = np.einsum("bklc,klco->bklo", vh[:, :m1, :m2], R[0] + 1j * R[1])
    full[:, -m1:, :m2] = np.einsum("bklc,klco->bklo", vh[:, -m1:, :m2], R[2] + 1j * R[3])
    ref = np.fft.irfft2(full, s=(ny, nx), axes=(1, 2))
    assert np.max(np.abs(u - ref)) < 1e-12


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(10)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(NN.bf16_round(x), ref)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(11)
    P = {"w": rng.standard_normal(50)}
    g = {"w": rng.standard_normal(50)}
    m, v = {"w": np.zeros(50)}, {"w": np.zeros(50)}
    w0 = P["w"].copy()
    NN.adam_step(P, g, m, v, 1, lr=1e-3)
    # bias-corrected first step: m_hat = g, v_hat = g^2
    assert np.allclose(P["w"], w0 - 1e-3 * g["w"] / (np.abs(g["w"]) + 1e-8), atol=1e-15)


def test_adam_second_step_closed_form():
    """Two steps written out by hand for scalars (Kingma & Ba): with zero
    initial moments, m_hat_2 = (b1 g1 + g2)/(1 + b1) and v_hat_2 =
    (b2 g1^2 + g2^2)/(1 + b2); a wrong beta2, a missing bias correction or a
    bias exponent off by one moves the second step."""
    b1, b2, lr, eps = 0.9, 0.999, 1e-3, 1e-8
    g1 = np.array([0.3, -2.0, 1e-3, 5.0])
    g2 = np.array([-0.5, -1.0, 4e-3, 5.0])
    P = {"w": np.array([1.0, -0.25, 0.0, 3.0])}
    w0 = P["w"].copy()
    m, v = {"w": np.zeros(4)}, {"w": np.zeros(4)}
    NN.adam_step(P, {"w": g1}, m, v, 1, lr=lr, b1=b1, b2=b2, eps=eps)
    NN.adam_step(P, {"w": g2}, m, v, 2, lr=lr, b1=b1, b2=b2, eps=eps)
    step1 = g1 / (np.abs(g1) + eps)
    mh = (b1 * g1 + g2) / (1 + b1)
    vh = (b2 * g1 * g1 + g2 * g2) / (1 + b2)
    expect = w0 - lr * step1 - lr * mh / (np.sqrt(vh) + eps)
    assert np.allclose(P["w"], expect, rtol=0, atol=1e-15)
    # first entry by hand: step 1 is 0.3/(0.3 + eps), then m_hat = -0.23/1.9,
    # v_hat = 0.33991/1.999
    by_hand = (1.0 - 1e-3 * 0.3 / (0.3 + eps)
               - 1e-3 * (-0.23 / 1.9) / (np.sqrt(0.33991 / 1.999) + eps))
    assert abs(P["w"][0] - by_hand) < 1e-13


def test_mse_gradient():
    rng = np.random.default_rng(12)
    a, b = rng.standard_normal((3, 4)), rng.standard_normal((3, 4))
    l, g = NN.mse(a, b)
    assert abs(l - np.sum((a - b) ** 2) / 12) < 1e-15
    assert np.allclose(g, 2 * (a - b) / 12)
