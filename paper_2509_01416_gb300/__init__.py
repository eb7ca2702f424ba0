"""GB300-native S_N transport solver with equation-recast neural-operator warm start.

The compute lives in libnop.so (hand-written sm_103a CUDA behind the C ABI of
include/nop.h).  ``capi`` is the ctypes binding under the C names; ``Solver``
below marshals numpy arrays into those calls and adds nothing else.
"""
import ctypes as C

import numpy as np

from . import capi
from .capi import (NOP_BC_REFLECTIVE, NOP_BC_VACUUM, NOP_GEOM_SLAB, NOP_GEOM_XY,
                   NOP_NO_DEEPONET, NOP_NO_FNO1D, NOP_NO_FNO2D, NOP_PREC_F32, NOP_PREC_F64,
                   NOP_WARM_NONE, NOP_WARM_RECAST, NopError)



def no_config(kind, sensors=128, width=128, basis=128, depth=4, modes=16, proj=128,
              sigma_t_star=1.0, sigma_s_star=0.5, length=10.0):
    c = capi.nop_no_config()
    c.kind, c.sensors, c.width, c.basis, c.depth = kind, sensors, width, basis, depth
    c.modes, c.proj = modes, proj
    c.sigma_t_star, c.sigma_s_star, c.length = sigma_t_star, sigma_s_star, length
    return c


def no_param_names(cfg):
    """Tensor names in the flat parameter order of include/nop.h."""
    names = []
    if cfg.kind == NOP_NO_DEEPONET:
        for net in ("b", "t"):
            for l in range(cfg.depth):
                names += ["%s%d.W" % (net, l), "%s%d.b" % (net, l)]
    else:
        names += ["lift.W", "lift.b"]
        spec = ["re", "im"] if cfg.kind == NOP_NO_FNO1D else ["re1", "im1", "re2", "im2"]
        for l in range(cfg.depth):
            names += ["spec%d.%s" % (l, k) for k in spec] + ["pw%d.W" % l, "pw%d.b" % l]
        names += ["proj1.W", "proj1.b", "proj2.W", "proj2.b"]
    return names


def flatten_params(cfg, params):
    return np.concatenate([np.asarray(params[k], dtype=np.float32).reshape(-1)
                           for k in no_param_names(cfg)])


def unflatten_params(cfg, flat, like):
    out, o = {}, 0
    for k in no_param_names(cfg):
        n = np.asarray(like[k]).size
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(np.shape(like[k]))
        o += n
    return out

def no_write_file(path, cfg, params):
    """Write an operator file (format in include/nop.h); params: dict or flat FP32."""
    flat = (np.ascontiguousarray(params, dtype=np.float32) if not isinstance(params, dict)
            else flatten_params(cfg, params))
    rc = capi.lib().nop_no_write_file(str(path).encode(), C.byref(cfg), capi._ptr(flat, capi._fp))
    if rc != 0:
        raise NopError(rc, "nop_no_write_file %s" % path)


def no_read_file(path):
    """Read an operator file: (nop_no_config, flat FP32 parameters)."""
    cfg = capi.nop_no_config()
    n = C.c_longlong(0)
    L = capi.lib()
    rc = L.nop_no_read_file(str(path).encode(), C.byref(cfg), None, C.byref(n))
    if rc == 0:
        flat = np.zeros(n.value, dtype=np.float32)
        rc = L.nop_no_read_file(str(path).encode(), C.byref(cfg), capi._ptr(flat, capi._fp),
                                C.byref(n))
    if rc != 0:
        raise NopError(rc, "nop_no_read_file %s" % path)
    return cfg, flat


__all__ = ["Solver", "NopError", "capi", "no_write_file", "no_read_file"]


def _opts(tol=1e-6, itmax=10000, precision=NOP_PREC_F32, tol_k=1e-7, tol_inner=None,
          itmax_inner=10000, warm_start=NOP_WARM_NONE, recast_tol=1e-4, recast_itmax=200,
          flags=0, schedule=0, dsa=False, chunked=False, cold=False, gauss_seidel=False):
    o = capi.nop_solve_opts()
    if gauss_seidel:
        flags |= capi.NOP_GAUSS_SEIDEL
    if cold:
        flags |= capi.NOP_COLD_SCHEDULE
    if dsa:
        flags |= capi.NOP_DSA
    if chunked:
        flags |= capi.NOP_SWEEP_CHUNKED
    o.tol, o.tol_k = tol, tol_k
    o.tol_inner = tol if tol_inner is None else tol_inner
    o.itmax, o.itmax_inner, o.precision = itmax, itmax_inner, precision
    o.warm_start, o.recast_tol, o.recast_itmax, o.flags = warm_start, recast_tol, recast_itmax, flags
    o.schedule = schedule
    return o


class Solver:
    """One nop_ctx on one CUDA device."""

    def __init__(self, device=0):
        self._L = capi.lib()
        h = C.c_void_p()
        rc = self._L.nop_create(C.byref(h), device)
        if rc != 0:
            raise NopError(rc, "nop_create(device=%d)" % device)
        self.h = h
        self._keep = []
        self.n_inst = 0
        self.G = 0
        self.C = 0

    def close(self):
        if self.h:
            self._L.nop_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != 0:
            raise NopError(rc, "%s: %s" % (what, self._L.nop_last_error(self.h).decode()))
        return rc

    def set_stream(self, stream_handle):
        self._check(self._L.nop_set_stream(self.h, C.c_void_p(stream_handle)), "nop_set_stream")

    def set_wait_limit(self, polls=-1):
        """Bound of the tensor-core kernels' completion waits (nop_set_wait_limit);
        -1 restores the default."""
        self._check(self._L.nop_set_wait_limit(self.h, int(polls)), "nop_set_wait_limit")

    def measure_alu_peaks(self):
        """(reciprocal/s, FP32 FMA/s) measured on this device (nop_measure_alu_peaks)."""
        r, f = C.c_double(), C.c_double()
        self._check(self._L.nop_measure_alu_peaks(self.h, C.byref(r), C.byref(f)),
                    "nop_measure_alu_peaks")
        return r.value, f.value

    def set_timing(self, enable=True):
        self._check(self._L.nop_set_timing(self.h, 1 if enable else 0), "nop_set_timing")

    def timing(self):
        t = capi.nop_timings()
        self._check(self._L.nop_get_timing(self.h, C.byref(t)), "nop_get_timing")
        return {k: getattr(t, k) for k, _ in t._fields_}

    # ---------------------------------------------------- neural operator
    def trace(self):
        """Per-instance (start ms, duration ms, block path) of the last timed slab solve."""
        t0, d = np.zeros(self.n_inst), np.zeros(self.n_inst)
        bp = np.zeros(self.n_inst, dtype=np.int32)
        self._check(self._L.nop_get_trace(self.h, self.n_inst, t0.ctypes.data, d.ctypes.data,
                                          bp.ctypes.data), "nop_get_trace")
        return t0, d, bp

    def no_set(self, cfg, params):
        """Install an operator; params: dict of arrays (names of no_param_names)."""
        flat = flatten_params(cfg, params)
        n = C.c_longlong()
        self._check(self._L.nop_no_param_count(C.byref(cfg), C.byref(n)), "nop_no_param_count")
        if n.value != flat.size:
            raise ValueError("parameter count %d != %d" % (flat.size, n.value))
        self._check(self._L.nop_no_set(self.h, C.byref(cfg), capi._ptr(flat, capi._fp)),
                    "nop_no_set")
        self.no_cfg, self.no_like = cfg, {k: np.asarray(v) for k, v in params.items()}

    def no_save(self, path):
        self._check(self._L.nop_no_save(self.h, str(path).encode()), "nop_no_save")

    def no_load(self, path, like=None):
        """Install the operator of a file; like: optional dict of arrays whose
        shapes no_get() then uses."""
        self._check(self._L.nop_no_load(self.h, str(path).encode()), "nop_no_load")
        self.no_cfg, _ = no_read_file(path)
        self.no_like = like

    def no_get(self):
        n = C.c_longlong()
        self._L.nop_no_param_count(C.byref(self.no_cfg), C.byref(n))
        flat = np.zeros(n.value, dtype=np.float32)
        self._check(self._L.nop_no_get(self.h, capi._ptr(flat, capi._fp)), "nop_no_get")
        return unflatten_params(self.no_cfg, flat, self.no_like)

    @staticmethod
    def _f32(a):
        return np.ascontiguousarray(a, dtype=np.float32)

    def no_forward(self, inputs, coords=None, out_width=None):
        U = self._f32(inputs)
        X = None if coords is None else self._f32(coords)
        n = U.shape[0]
        nc = 0 if X is None else X.size
        ow = out_width if out_width is not None else (nc if self.no_cfg.kind == NOP_NO_DEEPONET else U.shape[1])
        out = np.zeros((n, ow), dtype=np.float32)
        self._check(self._L.nop_no_forward(self.h, n, capi._ptr(U, capi._fp),
                                           None if X is None else capi._ptr(X, capi._fp), nc,
                                           capi._ptr(out, capi._fp)), "nop_no_forward")
        return out

    def no_loss_grad(self, inputs, targets, coords=None):
        U, Y = self._f32(inputs), self._f32(targets)
        X = None if coords is None else self._f32(coords)
        nc = 0 if X is None else X.size
        loss = C.c_double()
        n = C.c_longlong()
        self._L.nop_no_param_count(C.byref(self.no_cfg), C.byref(n))
        g = np.zeros(n.value, dtype=np.float32)
        self._check(self._L.nop_no_loss_grad(self.h, U.shape[0], capi._ptr(U, capi._fp),
                                             None if X is None else capi._ptr(X, capi._fp), nc,
                                             capi._ptr(Y, capi._fp), C.byref(loss),
                                             capi._ptr(g, capi._fp)), "nop_no_loss_grad")
        return loss.value, unflatten_params(self.no_cfg, g, self.no_like)

    def no_train(self, inputs, targets, coords=None, steps=1000, batch=100, lr=1e-3,
                 beta1=0.9, beta2=0.999, eps=1e-8, order=None):
        U, Y = self._f32(inputs), self._f32(targets)
        X = None if coords is None else self._f32(coords)
        nc = 0 if X is None else X.size
        tc = capi.nop_train_config()
        tc.steps, tc.batch, tc.lr, tc.beta1, tc.beta2, tc.eps = steps, batch, lr, beta1, beta2, eps
        ordr = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
        tc.order = None if ordr is None else capi._ptr(ordr, capi._ip)
        hist = np.zeros(steps)
        self._check(self._L.nop_no_train(self.h, C.byref(tc), U.shape[0], capi._ptr(U, capi._fp),
                                         None if X is None else capi._ptr(X, capi._fp), nc,
                                         capi._ptr(Y, capi._fp), capi._ptr(hist)), "nop_no_train")
        return hist

    def no_sensors(self, field):
        f = capi._f64(field)
        out = np.zeros((self.n_inst, self.no_cfg.sensors), dtype=np.float32)
        self._check(self._L.nop_no_sensors(self.h, capi._ptr(f), capi._ptr(out, capi._fp)),
                    "nop_no_sensors")
        return out

    def no_predict(self, src):
        s = capi._f64(src)
        out = np.zeros(self.G * self.C)
        self._check(self._L.nop_no_predict(self.h, capi._ptr(s), capi._ptr(out)), "nop_no_predict")
        return out

    def recast_iterate(self, tol=1e-4, itmax=200):
        out = np.zeros(self.G * self.C)
        st, it, ss = self._stats()
        self._check(self._L.nop_recast_iterate(self.h, tol, itmax, 0, out.ctypes.data,
                                               C.byref(st)), "nop_recast_iterate")
        return out, {"iterations": it, "status": ss, "max_iterations": st.recast_iterations,
                     "recast_status": st.recast_status}

    # ---------------------------------------------------------- problems
    def set_slabs(self, n_cells, width, order, sigma_t, sigma_s, source=None,
                  nu_sigma_f=None, chi=None, bc=(0, 0), sigma_s1=None):
        """Batch of slabs; arrays group-major over all cells (see nop.h).
        sigma_s1: in-group first Legendre moment (fixed source only)."""
        n_cells = np.ascontiguousarray(n_cells, dtype=np.int32)
        order = np.ascontiguousarray(order, dtype=np.int32)
        width = capi._f64(width)
        total = int(n_cells.sum())
        # an empty batch reaches the library, which rejects it
        G = int(np.asarray(sigma_t).size // total) if total > 0 else 1
        arrs = [capi._f64(sigma_t), capi._f64(sigma_s),
                None if source is None else capi._f64(source),
                None if nu_sigma_f is None else capi._f64(nu_sigma_f),
                None if chi is None else capi._f64(chi)]
        p = capi.nop_problem()
        p.geometry, p.n_inst = NOP_GEOM_SLAB, len(n_cells)
        p.n_cells, p.width, p.order = capi._ptr(n_cells, capi._ip), capi._ptr(width), capi._ptr(order, capi._ip)
        p.n_groups = G
        p.sigma_t, p.sigma_s, p.source, p.nu_sigma_f, p.chi = [capi._ptr(a) for a in arrs]
        p.bc[0], p.bc[1] = int(bc[0]), int(bc[1])
        s1 = None if sigma_s1 is None else capi._f64(sigma_s1)
        p.sigma_s1 = capi._ptr(s1)
        self._check(self._L.nop_set_problem(self.h, C.byref(p)), "nop_set_problem")
        self.n_inst, self.G, self.C = len(n_cells), G, int(n_cells.sum())

    def set_diffusion(self, n_cells, width, diffusion, source, absorption=None):
        """Batch of 1D diffusion slabs (Table 1): -(D u')' + Sigma_a u = S, u = 0
        at the faces; cell arrays concatenated over the instances."""
        n_cells = np.ascontiguousarray(n_cells, dtype=np.int32)
        width = capi._f64(width)
        d, s = capi._f64(diffusion), capi._f64(source)
        a = None if absorption is None else capi._f64(absorption)
        self._check(self._L.nop_set_diffusion(self.h, len(n_cells), capi._ptr(n_cells, capi._ip),
                                              capi._ptr(width), capi._ptr(d), capi._ptr(a),
                                              capi._ptr(s)), "nop_set_diffusion")
        self.n_inst, self.G, self.C = len(n_cells), 1, int(n_cells.sum())

    def diffusion_solve(self):
        """The model-based solution of the diffusion batch (FP64)."""
        out = np.zeros(self.C)
        self._check(self._L.nop_diffusion_solve(self.h, capi._ptr(out)), "nop_diffusion_solve")
        return out

    def set_xy(self, nx, ny, lx, ly, sigma_t, sigma_s, source=None, nu_sigma_f=None,
               chi=None, bc=(0, 0, 0, 0)):
        G = int(np.asarray(sigma_t).size // (nx * ny))
        arrs = [capi._f64(sigma_t), capi._f64(sigma_s),
                None if source is None else capi._f64(source),
                None if nu_sigma_f is None else capi._f64(nu_sigma_f),
                None if chi is None else capi._f64(chi)]
        order = np.array([8], dtype=np.int32)
        p = capi.nop_problem()
        p.geometry, p.n_inst, p.order = NOP_GEOM_XY, 1, capi._ptr(order, capi._ip)
        p.nx, p.ny, p.lx, p.ly, p.n_groups = nx, ny, lx, ly, G
        p.sigma_t, p.sigma_s, p.source, p.nu_sigma_f, p.chi = [capi._ptr(a) for a in arrs]
        for f in range(4):
            p.bc[f] = int(bc[f])
        self._check(self._L.nop_set_problem(self.h, C.byref(p)), "nop_set_problem")
        self.n_inst, self.G, self.C = 1, G, nx * ny

    def quadrature(self, inst=0):
        mu, eta, w = np.zeros(128), np.zeros(128), np.zeros(128)
        n = C.c_int()
        self._check(self._L.nop_get_quadrature(self.h, inst, capi._ptr(mu), capi._ptr(eta),
                                               capi._ptr(w), C.byref(n)), "nop_get_quadrature")
        k = n.value
        return mu[:k], eta[:k], w[:k]

    # ------------------------------------------------------------ solves
    def _out(self, out):
        if out is None:
            return np.zeros(self.G * self.C)
        if (not isinstance(out, np.ndarray) or out.dtype != np.float64 or
                not out.flags.c_contiguous or out.size != self.G * self.C):
            raise ValueError("out must be a contiguous float64 array of %d entries"
                             % (self.G * self.C))
        return out

    def _stats(self):
        st = capi.nop_stats()
        it = np.zeros(self.n_inst, dtype=np.int32)
        ss = np.zeros(self.n_inst, dtype=np.int32)
        st.inst_iterations, st.inst_status = capi._ptr(it, capi._ip), capi._ptr(ss, capi._ip)
        return st, it, ss

    def _rc(self, rc, check, allow_noconv, what):
        """Raise on a failed call.  NOP_ENOCONV (an iteration cap reached; the
        outputs hold the last iterate) raises too unless allow_noconv."""
        if check and rc != 0 and not (allow_noconv and rc == capi.NOP_ENOCONV):
            self._check(rc, what)

    def solve_fixed_source(self, phi0=None, check=True, out=None, allow_noconv=False, **kw):
        """Fixed-source solve; out: optional float64 host array of G*C entries
        (for instance a pinned buffer) that receives the flux.  Raises NopError
        on any failure, including an instance that reached the iteration cap,
        unless check=False or (for the cap alone) allow_noconv=True."""
        o = _opts(**kw)
        phi = self._out(out)
        p0 = None if phi0 is None else capi._f64(phi0)
        st, it, ss = self._stats()
        rc = self._L.nop_solve_fixed_source(self.h, C.byref(o),
                                            None if p0 is None else p0.ctypes.data,
                                            phi.ctypes.data, C.byref(st))
        self._rc(rc, check, allow_noconv, "nop_solve_fixed_source")
        return phi, {"rc": rc, "iterations": it, "status": ss, "max_change": st.max_change,
                     "recast_iterations": st.recast_iterations,
                     "recast_status": st.recast_status}

    def solve_fixed_source_dev(self, phi_out_ptr, phi0_ptr=None, check=True, allow_noconv=False,
                               **kw):
        """Device-resident variant: phi_out_ptr (and phi0_ptr) are device pointers
        to FP64 arrays of G*C entries; per-instance statistics come back to the
        host.  Failures raise as in solve_fixed_source."""
        flags = capi.NOP_OUT_DEVICE | (capi.NOP_PHI0_DEVICE if phi0_ptr else 0)
        o = _opts(flags=flags, **kw)
        st, it, ss = self._stats()
        rc = self._L.nop_solve_fixed_source(self.h, C.byref(o), phi0_ptr, phi_out_ptr,
                                            C.byref(st))
        self._rc(rc, check, allow_noconv, "nop_solve_fixed_source")
        return {"rc": rc, "iterations": it, "status": ss,
                "recast_iterations": st.recast_iterations, "recast_status": st.recast_status}

    def solve_eigen(self, phi0=None, k0=0.0, check=True, out=None, allow_noconv=False, **kw):
        """Eigen solve: (k per instance, phi, info).  Failures raise as in
        solve_fixed_source (an outer iteration cap is NOP_ENOCONV)."""
        o = _opts(**kw)
        phi = self._out(out)
        k = np.zeros(self.n_inst)
        p0 = None if phi0 is None else capi._f64(phi0)
        st, it, ss = self._stats()
        rc = self._L.nop_solve_eigen(self.h, C.byref(o), None if p0 is None else p0.ctypes.data,
                                     float(k0), phi.ctypes.data, k.ctypes.data, C.byref(st))
        self._rc(rc, check, allow_noconv, "nop_solve_eigen")
        return k, phi, {"rc": rc, "inner": it, "status": ss, "outer": st.max_outer,
                        "max_change": st.max_change,
                        "recast_iterations": st.recast_iterations,
                        "recast_status": st.recast_status}

    def sp_eigen(self, tol=1e-4, itmax=200, constrained=False):
        """Eigen warm start alone (simple preconditioning, or the constrained
        variant): (k per instance, phi, info)."""
        phi = np.zeros(self.G * self.C)
        k = np.zeros(self.n_inst)
        st, it, ss = self._stats()
        flags = capi.NOP_SP_CONSTRAINED if constrained else 0
        self._check(self._L.nop_sp_eigen(self.h, tol, itmax, flags, phi.ctypes.data,
                                         k.ctypes.data, C.byref(st)), "nop_sp_eigen")
        return k, phi, {"iterations": it, "status": ss, "max_iterations": st.recast_iterations,
                        "recast_status": st.recast_status}
