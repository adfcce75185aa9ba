"""Python face of the library's continuum solver (``lbm_fem_*``): Q1 finite
elements for the advection-diffusion equation stepped on the GPU.
Argument marshalling only; assembly is done once by the library and every
time step runs in its CUDA kernels."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import FemParams, check
from .lbm import _in_ptr, _out_ptr, current_stream_handle


class FEM:
    """Q1 mesh of nex x ney elements on [x0, x0 + nex hx] x [y0, y0 + ney hy]
    (Sec. 3; trapezoidal rule of Sec. 6.1.1).  ``elem_active`` [ney, nex]
    switches elements off; ``dirichlet`` lists the node ids (j (nex+1) + i)
    whose values ``step`` prescribes, in that order; other boundaries are
    zero-flux."""

    def __init__(self, nex, ney, x0, y0, hx, hy, D, v=(0.0, 0.0), theta=0.5, dt=1.0,
                 supg=False, elem_active=None, dirichlet=(), d0=None, tol=1e-12,
                 max_iter=1000, stream=None):
        self._lib = _lib.load()
        p = FemParams()
        p.nex, p.ney = int(nex), int(ney)
        p.x0, p.y0, p.hx, p.hy = float(x0), float(y0), float(hx), float(hy)
        p.D, p.vx, p.vy = float(D), float(v[0]), float(v[1])
        p.theta, p.dt, p.supg = float(theta), float(dt), int(bool(supg))
        p.tol, p.max_iter = float(tol), int(max_iter)
        self.params = p
        self.nex, self.ney = p.nex, p.ney
        self.n = (p.nex + 1) * (p.ney + 1)
        keep = []
        act = None if elem_active is None else _in_ptr(elem_active, "u8", p.nex * p.ney, keep)
        dn = np.ascontiguousarray(np.asarray(dirichlet, dtype=np.int32).reshape(-1))
        self.n_dir = int(dn.size)
        keep.append(dn)
        d0p = _in_ptr(d0, "f64", self.n, keep)
        if stream is None:
            stream = current_stream_handle()
        h = ctypes.c_void_p()
        check(self._lib.lbm_fem_init(ctypes.byref(h), ctypes.byref(p), act, self.n_dir,
                                     dn.ctypes.data if dn.size else None, d0p, stream))
        self._h = h

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.lbm_fem_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, dir_values=None):
        """One time step with the Dirichlet nodes at ``dir_values`` (t^{n+1})."""
        keep = []
        ptr = _in_ptr(dir_values, "f64", self.n_dir, keep) if self.n_dir else None
        check(self._lib.lbm_fem_step(self._h, ptr))

    def interpolate(self, xy, out=None):
        """Element interpolant of d at points xy [npts, 2]."""
        keep = []
        npts = (xy.numel() if hasattr(xy, "numel") else np.asarray(xy).size) // 2
        ptr = _in_ptr(xy, "f64", 2 * npts, keep)
        if out is None:
            out = np.empty(npts)
        check(self._lib.lbm_fem_interpolate(self._h, int(npts), ptr, _out_ptr(out, "f64", npts)))
        return out

    def get(self, out=None):
        if out is None:
            out = np.empty(self.n)
        check(self._lib.lbm_fem_get(self._h, _out_ptr(out, "f64", self.n)))
        return out

    def set(self, d):
        keep = []
        check(self._lib.lbm_fem_set(self._h, _in_ptr(d, "f64", self.n, keep)))

    def solver_info(self):
        it, res = ctypes.c_int(), ctypes.c_double()
        check(self._lib.lbm_fem_solver_info(self._h, ctypes.byref(it), ctypes.byref(res)))
        return it.value, res.value
