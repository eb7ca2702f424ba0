"""Operator files on the GPU: an operator saved from one context and loaded
into another gives bit-identical parameters and forward outputs."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solvers():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2509_01416_gb300 import Solver
    a, b = Solver(0), Solver(0)
    yield a, b
    a.close()
    b.close()


def test_deeponet_round_trip(solvers, tmp_path):
    from paper_2509_01416_gb300 import NOP_NO_DEEPONET, no_config
    a, b = solvers
    cfg = no_config(NOP_NO_DEEPONET, sensors=128, width=128, basis=128)
    P = W.deeponet_init(7)
    a.no_set(cfg, P)
    path = tmp_path / "don.bin"
    a.no_save(path)
    b.no_load(path, like=P)
    pa, pb = a.no_get(), b.no_get()
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
    rng = np.random.default_rng(1)
    U = rng.uniform(0, 1, (5, 128)).astype(np.float32)
    X = np.linspace(0.0, 1.0, 37).astype(np.float32)
    assert np.array_equal(a.no_forward(U, X), b.no_forward(U, X))


def test_fno1d_round_trip(solvers, tmp_path):
    from paper_2509_01416_gb300 import NOP_NO_FNO1D, no_config
    a, b = solvers
    cfg = no_config(NOP_NO_FNO1D, width=64, modes=16, depth=4, proj=128, length=10.0)
    P = W.fno1d_init(3, width=64, modes=16, proj=128)
    a.no_set(cfg, P)
    path = tmp_path / "fno.bin"
    a.no_save(path)
    b.no_load(path)
    S = np.random.default_rng(2).uniform(0, 1, (3, 100)).astype(np.float32)
    assert np.array_equal(a.no_forward(S, coords=np.zeros(100)),
                          b.no_forward(S, coords=np.zeros(100)))


def test_save_without_operator_is_refused(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2509_01416_gb300 import NopError, Solver, capi
    s = Solver(0)
    try:
        with pytest.raises(NopError) as e:
            s.no_save(tmp_path / "none.bin")
        assert e.value.code == capi.NOP_ESTATE
        with pytest.raises(NopError) as e:
            s.no_load(tmp_path / "missing.bin")
        assert e.value.code == capi.NOP_EIO
    finally:
        s.close()
