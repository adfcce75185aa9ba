"""The one-dimensional hybrid of Sec. 7.1 on the GPU: the library's D1Q2
lattice (``lbm1d_*``) on the fine subdomain (1/2 - L/2, 1) and its
continuum solver on the coarse one (0, 1/2 + L/2), coupled by Algorithm 1
with multi-time-stepping (Eq. "MTS") and Schwarz iterations.

The continuum solver is the library's Q1 one with a single row of elements
and zero flux on its top and bottom: for data that do not vary across the
row the bilinear system reduces exactly to the two-node linear elements of
the section (the across-row factor of every element matrix is the same row
sum), so its nodes along the bottom carry the 1-D solution.  Argument
marshalling and call sequencing only; every step runs in the library.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _lib
from ._lib import check
from .fem import FEM
from .lbm import _in_ptr, current_stream_handle

DIRICHLET, NEUMANN = 1, 2


class LBM1D:
    """D1Q2 lattice of n nodes (lbm1d_*): relaxation time tau, lattice
    velocity vl = v dt / h, end kinds (DIRICHLET or NEUMANN), initial u0."""

    def __init__(self, n, tau, vl, u0=None, left=DIRICHLET, right=NEUMANN, stream=None):
        self._lib = _lib.load()
        self.n = int(n)
        keep = []
        if stream is None:
            stream = current_stream_handle()
        h = ctypes.c_void_p()
        check(self._lib.lbm1d_init(ctypes.byref(h), self.n, float(tau), float(vl), int(left),
                                   int(right), _in_ptr(u0, "f64", self.n, keep), stream))
        self._h = h

    def substeps(self, n, eta, ends_t0=(0.0, 0.0), ends_t1=None, q=(0.0, 0.0)):
        keep = []
        a = _in_ptr(np.asarray(ends_t0, float), "f64", 2, keep)
        b = None if ends_t1 is None else _in_ptr(np.asarray(ends_t1, float), "f64", 2, keep)
        qq = _in_ptr(np.asarray(q, float), "f64", 2, keep)
        check(self._lib.lbm1d_substeps(self._h, int(n), int(eta), a, b, qq))

    def u(self):
        out = np.empty(self.n)
        check(self._lib.lbm1d_get(self._h, out.ctypes.data))
        return out

    def save(self):
        nb = ctypes.c_size_t()
        check(self._lib.lbm1d_state_bytes(self._h, ctypes.byref(nb)))
        buf = np.empty(nb.value, dtype=np.uint8)
        check(self._lib.lbm1d_save(self._h, buf.ctypes.data, nb.value))
        return buf

    def restore(self, buf):
        check(self._lib.lbm1d_restore(self._h, buf.ctypes.data, buf.size))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lbm1d_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gaussian(x, t, phi=0.1, sigma0=0.01, x0=0.3, v=1.0, D=1e-2):
    """The section's Gaussian hill in free space (initial data at t = 0)."""
    s2 = sigma0 ** 2 + 2 * D * t
    return phi / math.sqrt(2 * math.pi * s2) * np.exp(-(np.asarray(x) - x0 - v * t) ** 2 / (2 * s2))


class Hybrid1D:
    """The coupled run of Sec. 7.1 for one parameter set: element size h_c,
    lattice spacing h_f (dt_f = h_f^2 / 2D, so tau = 1), eta lattice steps per
    coarse step, overlap length L, max_iter Schwarz iterations; v = 1,
    D = 1e-2, the Gaussian hill of the section initially.  ``init(x)``
    replaces the initial data; ``right``/``right_value(t)`` make the
    lattice's far end a Dirichlet end with those data (the section's end is
    zero-flux)."""

    def __init__(self, h_c, h_f, eta, overlap, max_iter, D=1e-2, v=1.0, theta=0.5, init=None,
                 right=NEUMANN, right_value=None):
        self.h_c, self.h_f, self.eta, self.max_iter = h_c, h_f, int(eta), int(max_iter)
        self.lc = 0.5 + overlap / 2.0
        self.xf0 = 0.5 - overlap / 2.0
        self.n_el = int(round(self.lc / h_c))
        self.nf = int(round((1.0 - self.xf0) / h_f)) + 1
        self.j_trace = int(round(overlap / h_f))  # the lattice node at x = lc
        self.dt_f = h_f * h_f / (2.0 * D)
        self.dt_c = self.eta * self.dt_f
        tau = 0.5 + D * self.dt_f / (h_f * h_f)
        self.x_c = np.arange(self.n_el + 1) * h_c
        self.x_f = self.xf0 + np.arange(self.nf) * h_f
        self.D, self.v = D, v
        f0 = init if init is not None else (lambda x: gaussian(x, 0.0, D=D, v=v))
        self.right_value = right_value
        nxn = self.n_el + 1
        d0 = np.tile(f0(self.x_c), 2)  # both rows of nodes
        self.fem = FEM(self.n_el, 1, 0.0, 0.0, h_c, h_c, D, (v, 0.0), theta, self.dt_c,
                       dirichlet=[nxn - 1, 2 * nxn - 1], d0=d0, tol=1e-14)
        self.lat = LBM1D(self.nf, tau, v * self.dt_f / h_f, f0(self.x_f), right=right)
        self._pt = np.array([[self.xf0, 0.0]])
        self.t = 0.0

    def coarse_step(self):
        fem, lat = self.fem, self.lat
        d_n = fem.get()
        snap = lat.save()
        trace = lat.u()[self.j_trace]
        a_left = fem.interpolate(self._pt)[0]
        rv = self.right_value
        ra, rb = (rv(self.t), rv(self.t + self.dt_c)) if rv else (0.0, 0.0)
        for it in range(self.max_iter):
            if it > 0:
                fem.set(d_n)
                lat.restore(snap)
            fem.step([trace, trace])
            b_left = fem.interpolate(self._pt)[0]
            lat.substeps(self.eta, self.eta, (a_left, ra), (b_left, rb))
            trace = lat.u()[self.j_trace]
        self.t += self.dt_c

    def run(self, T=0.4):
        n = int(round(T / self.dt_c))
        for _ in range(n):
            self.coarse_step()
        return n

    def coarse(self):
        return self.fem.get()[:self.n_el + 1]

    def fine(self):
        return self.lat.u()

    def errors(self):
        """(E_c, E_f): max errors against the free-space solution at the
        current time, on the coarse and fine nodes (Eq. "Error1D")."""
        ex = lambda x: gaussian(x, self.t, D=self.D, v=self.v)
        return (float(np.abs(self.coarse() - ex(self.x_c)).max()),
                float(np.abs(self.fine() - ex(self.x_f)).max()))

    def close(self):
        self.fem.close()
        self.lat.close()
