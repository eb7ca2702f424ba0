"""Build and load the oracle's plain-C sweeps (TEST INFRASTRUCTURE ONLY)."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sn_sweep.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libsn_oracle.so")

_lib = None


def build(force=False):
    """Compile sn_sweep.c into oracle/_build/libsn_oracle.so with gcc -O2."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99",
                           "-o", tmp, _SRC])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        L.ora_sweep1d.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, dp, dp,
                                  dp, dp, dp, dp, dp]
        L.ora_sweep1d.restype = None
        L.ora_sweep1d_p1.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_int, dp, dp,
                                     dp, dp, dp, dp, dp, dp]
        L.ora_sweep1d_p1.restype = None
        L.ora_sweep2d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, dp, dp, ctypes.c_int, dp, dp, dp,
                                  dp, dp, dp, dp, dp, dp]
        L.ora_sweep2d.restype = None
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def sweep1d(dx, sigt, q, mu, w, in_left, in_right):
    """One DD sweep of a 1D slab for one group.  Returns (phi, out_left, out_right).

    ``out_left[n]`` is meaningful for mu[n] < 0 and ``out_right[n]`` for
    mu[n] > 0; the other entries are zero.
    """
    dx, sigt, q, mu, w = map(_f64, (dx, sigt, q, mu, w))
    in_left, in_right = _f64(in_left), _f64(in_right)
    I, N = sigt.shape[0], mu.shape[0]
    phi = np.zeros(I)
    out_l = np.zeros(N)
    out_r = np.zeros(N)
    lib().ora_sweep1d(I, _p(dx), _p(sigt), _p(q), N, _p(mu), _p(w),
                      _p(in_left), _p(in_right), _p(phi), _p(out_l), _p(out_r))
    return phi, out_l, out_r


def sweep1d_p1(dx, sigt, q0, q1, mu, w, in_left, in_right):
    """DD sweep with emission q0 + mu q1 per direction (Eq. 25).  Returns
    (phi, current, out_left, out_right)."""
    dx, sigt, q0, q1, mu, w = map(_f64, (dx, sigt, q0, q1, mu, w))
    in_left, in_right = _f64(in_left), _f64(in_right)
    I, N = sigt.shape[0], mu.shape[0]
    phi = np.zeros(I)
    cur = np.zeros(I)
    out_l = np.zeros(N)
    out_r = np.zeros(N)
    lib().ora_sweep1d_p1(I, _p(dx), _p(sigt), _p(q0), _p(q1), N, _p(mu), _p(w),
                         _p(in_left), _p(in_right), _p(phi), _p(cur), _p(out_l), _p(out_r))
    return phi, cur, out_l, out_r


def sweep2d(dx, dy, sigt, q, mu, eta, w, in_x, in_y):
    """One DD sweep of a 2D x-y mesh for one group.  Returns (phi, out_x, out_y).

    ``sigt`` and ``q`` are [ny, nx]; ``in_x``/``out_x`` are [M, ny] and
    ``in_y``/``out_y`` are [M, nx] (see sn_sweep.c for which face each means).
    """
    sigt, q, mu, eta, w = map(_f64, (sigt, q, mu, eta, w))
    in_x, in_y = _f64(in_x), _f64(in_y)
    ny, nx = sigt.shape
    M = mu.shape[0]
    phi = np.zeros((ny, nx))
    out_x = np.zeros((M, ny))
    out_y = np.zeros((M, nx))
    ybuf = np.zeros(nx)
    lib().ora_sweep2d(nx, ny, float(dx), float(dy), _p(sigt), _p(q), M, _p(mu),
                      _p(eta), _p(w), _p(in_x), _p(in_y), _p(phi), _p(out_x),
                      _p(out_y), _p(ybuf))
    return phi, out_x, out_y
