"""Operator files (nop_no_write_file / nop_no_read_file): host-only, no GPU.

The byte layout is checked against the format include/nop.h states, read
back independently with the struct module; round trips are bit-exact; each
kind of malformed file is rejected.
"""
import struct

import numpy as np
import pytest

from paper_2509_01416_gb300 import (NOP_NO_DEEPONET, NOP_NO_FNO1D, NOP_NO_FNO2D, NopError,
                                    capi, no_config, no_read_file, no_write_file)
from paper_2509_01416_gb300 import build as B

CONFIGS = [
    dict(kind=NOP_NO_DEEPONET, sensors=128, width=128, basis=128, depth=4),
    dict(kind=NOP_NO_FNO1D, width=64, modes=32, depth=4, proj=128, sigma_t_star=1.0,
         sigma_s_star=0.5, length=10.0),
    dict(kind=NOP_NO_FNO2D, width=32, modes=16, depth=4, proj=128, length=10.0),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()


def _count(cfg):
    import ctypes as C
    n = C.c_longlong()
    assert capi.lib().nop_no_param_count(C.byref(cfg), C.byref(n)) == 0
    return n.value


@pytest.mark.parametrize("kw", CONFIGS)
def test_layout_matches_the_stated_format(tmp_path, kw):
    cfg = no_config(**kw)
    n = _count(cfg)
    p = np.random.default_rng(n).standard_normal(n).astype(np.float32)
    f = tmp_path / "op.bin"
    no_write_file(f, cfg, p)
    raw = f.read_bytes()
    assert len(raw) == 68 + 4 * n
    assert raw[:8] == b"NOPNET01"
    ints = struct.unpack_from("<7i", raw, 8)
    assert ints == (cfg.kind, cfg.sensors, cfg.width, cfg.basis, cfg.depth, cfg.modes, cfg.proj)
    assert struct.unpack_from("<3d", raw, 36) == (cfg.sigma_t_star, cfg.sigma_s_star, cfg.length)
    assert struct.unpack_from("<q", raw, 60)[0] == n
    assert np.array_equal(np.frombuffer(raw, dtype="<f4", offset=68), p)
    cfg2, q = no_read_file(f)
    assert np.array_equal(q.view(np.uint32), p.view(np.uint32))
    for k, _ in cfg._fields_:
        assert getattr(cfg2, k) == getattr(cfg, k)


def test_special_values_survive(tmp_path):
    cfg = no_config(NOP_NO_DEEPONET, sensors=8, width=8, basis=8, depth=2)
    n = _count(cfg)
    p = np.zeros(n, dtype=np.float32)
    p[:5] = [np.float32(-0.0), np.inf, -np.inf, np.float32(1e-45), np.nan]
    f = tmp_path / "op.bin"
    no_write_file(f, cfg, p)
    _, q = no_read_file(f)
    assert np.array_equal(q.view(np.uint32), p.view(np.uint32))


def _err(path):
    with pytest.raises(NopError) as e:
        no_read_file(path)
    return e.value.code


def test_malformed_files_are_rejected(tmp_path):
    cfg = no_config(NOP_NO_DEEPONET, sensors=16, width=16, basis=16, depth=3)
    n = _count(cfg)
    good = tmp_path / "good.bin"
    no_write_file(good, cfg, np.ones(n, dtype=np.float32))
    raw = good.read_bytes()
    cases = {
        "magic": b"NOPNET02" + raw[8:],
        "short": raw[:-1],
        "trailing": raw + b"\0",
        "header only": raw[:40],
        "count": raw[:60] + struct.pack("<q", n + 1) + raw[68:],
        "config": raw[:8] + struct.pack("<i", 99) + raw[12:],
    }
    for name, data in cases.items():
        f = tmp_path / (name.replace(" ", "_") + ".bin")
        f.write_bytes(data)
        assert _err(f) == capi.NOP_EIO, name
    assert _err(tmp_path / "missing.bin") == capi.NOP_EIO


def test_capacity_and_invalid_config(tmp_path):
    import ctypes as C
    cfg = no_config(NOP_NO_DEEPONET, sensors=16, width=16, basis=16, depth=3)
    n = _count(cfg)
    f = tmp_path / "op.bin"
    no_write_file(f, cfg, np.ones(n, dtype=np.float32))
    L = capi.lib()
    out = np.zeros(n - 1, dtype=np.float32)
    cap = C.c_longlong(n - 1)
    c2 = capi.nop_no_config()
    assert L.nop_no_read_file(str(f).encode(), C.byref(c2), capi._ptr(out, capi._fp),
                              C.byref(cap)) == capi.NOP_EINVAL
    bad = no_config(NOP_NO_DEEPONET, sensors=0, width=16, basis=16, depth=3)
    with pytest.raises(NopError) as e:
        no_write_file(tmp_path / "bad.bin", bad, np.ones(4, dtype=np.float32))
    assert e.value.code == capi.NOP_EINVAL
