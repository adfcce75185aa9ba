"""FP64 CPU oracle of the pore-scale LBM hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the product path
(``paper_1601_02708_gb300``) never imports it and fails loudly when its CUDA
library is missing instead of falling back here.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, no fast-math); this
module only compiles it and marshals numpy arrays through ctypes.  Each C
function cites the passage of the paper it follows (Sec. 4.1, 4.1.1, 6.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

EDGE_PERIODIC, EDGE_DIRICHLET, EDGE_NEUMANN = 0, 1, 2
REACT_NONE, REACT_SURFACE, REACT_BULK = 0, 1, 2
WALLS = {"bounce": 0, "maxent": 1}  # pore walls: halfway bounce-back or zero-flux max-entropy

# D2Q9 velocities and weights, typed here for the tests' own use (this list
# is not shared with the CUDA library, which carries its own copy).
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
WT = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, OpenMP over rows)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        D = ctypes.c_double
        I = ctypes.c_int
        lib.or_lbm_new.restype = P
        lib.or_lbm_new.argtypes = [I, I, P, D, I, D, P, I, P, P, P, P]
        lib.or_lbm_free.argtypes = [P]
        lib.or_lbm_substeps.argtypes = [P, I, I, P, P, P]
        for name in ("or_lbm_get_u", "or_lbm_get_f", "or_lbm_get_solid",
                     "or_lbm_get_mineral", "or_lbm_get_fpost", "or_lbm_diag",
                     "or_lbm_get_flip_steps"):
            getattr(lib, name).argtypes = [P, P]
        lib.or_lbm_H.restype = D
        lib.or_lbm_H.argtypes = [P]
        lib.or_trace_point.restype = D
        lib.or_trace_point.argtypes = [P, D, D]
        lib.or_maxent_dirichlet.restype = I
        lib.or_maxent_dirichlet.argtypes = [P, P, D]
        lib.or_lbm_clone.restype = P
        lib.or_lbm_clone.argtypes = [P]
        lib.or_lbm_assign.argtypes = [P, P]
        lib.or_lbm_adjoint.restype = I
        lib.or_lbm_adjoint.argtypes = [P, I, I, P, P, P, P, P, P, P, P]
        lib.or_maxent_neumann.restype = I
        lib.or_maxent_neumann.argtypes = [P, P, D, D, D, P, P]
        lib.or_lbm_set_wall_mode.argtypes = [P, I]
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class LBMOracle:
    """D2Q9 ADE-LBM state advanced by the plain C oracle (FP64).

    Arguments mirror the problem statement of Sec. 6 (Eq. "CouplingPDE"):
    ``solid`` [ny, nx] (nonzero = solid), ``vel`` [2, ny, nx] advection
    velocity in lattice units, ``tau`` relaxation time, ``edges`` the kinds of
    the W, E, S, N sides, ``u0`` the initial concentration, and the reaction
    (``react_mode``, ``k``/``k_field``, ``dissolution``, ``mineral``).
    ``walls`` treats the pore walls by halfway bounce-back ("bounce") or as
    zero-flux boundaries of the maximum-entropy kind (Sec. 4.1.1 (b), "maxent").
    """

    def __init__(self, nx, ny, tau, edges=(0, 0, 0, 0), solid=None, vel=None,
                 u0=None, react_mode=REACT_NONE, k=0.0, k_field=None,
                 dissolution=False, mineral=None, walls="bounce"):
        lib = _load()
        if walls not in WALLS:
            raise ValueError(f"walls must be one of {sorted(WALLS)}")
        if (edges[0] == EDGE_PERIODIC) != (edges[1] == EDGE_PERIODIC):
            raise ValueError("W and E must both be periodic or both not")
        if (edges[2] == EDGE_PERIODIC) != (edges[3] == EDGE_PERIODIC):
            raise ValueError("S and N must both be periodic or both not")
        self.nx, self.ny = int(nx), int(ny)
        N = self.nx * self.ny
        self._edges = np.ascontiguousarray(edges, dtype=np.int32)
        self._solid = None if solid is None else np.ascontiguousarray(
            np.asarray(solid).reshape(N) != 0, dtype=np.uint8)
        self._vel = _f64(vel, (2 * N,))
        self._k = _f64(k_field, (N,))
        self._min = _f64(mineral, (N,))
        self._u0 = _f64(u0, (N,))
        self._h = lib.or_lbm_new(
            self.nx, self.ny, _ptr(self._edges), float(tau), int(react_mode),
            float(k), _ptr(self._k), int(bool(dissolution)), _ptr(self._solid),
            _ptr(self._vel), _ptr(self._min), _ptr(self._u0))
        if not self._h:
            raise MemoryError("oracle allocation failed")
        self._lib = lib
        lib.or_lbm_set_wall_mode(self._h, WALLS[walls])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_lbm_free(h)
            self._h = None

    @property
    def n_edge(self):
        return 2 * (self.nx + self.ny)

    def substeps(self, n, eta=1, u_dir_t0=None, u_dir_t1=None, q_neu=None):
        """Substeps j = 1..n of ratio eta; Dirichlet data interpolated in time
        between ``u_dir_t0`` and ``u_dir_t1`` (Eq. "MTS"); arrays use the edge
        layout [W: ny][E: ny][S: nx][N: nx]."""
        a = _f64(u_dir_t0, (self.n_edge,))
        b = _f64(u_dir_t1 if u_dir_t1 is not None else u_dir_t0, (self.n_edge,))
        q = _f64(q_neu, (self.n_edge,))
        self._lib.or_lbm_substeps(self._h, int(n), int(eta), _ptr(a), _ptr(b), _ptr(q))

    def snapshot(self):
        """Deep copy of the evolving state (for the Schwarz rollback)."""
        snap = LBMOracle.__new__(LBMOracle)
        snap.__dict__.update(self.__dict__)
        snap._h = self._lib.or_lbm_clone(self._h)
        if not snap._h:
            raise MemoryError("oracle allocation failed")
        return snap

    def rollback(self, snap):
        """Restore the state saved by ``snapshot``."""
        self._lib.or_lbm_assign(self._h, snap._h)

    def adjoint(self, n, eta=1, u_dir_t0=None, u_dir_t1=None, q_neu=None):
        """Advance n substeps (as ``substeps``) and return the outlet
        breakthrough J = sum of the east-edge fluid concentrations over the n
        substeps with its gradients: dict(J, k [ny, nx] with respect to the
        rate of every node, ua / ub with respect to the Dirichlet data at the
        start / end of the coarse step, q with respect to the Neumann data;
        the last three in the edge layout).  Fixed mask only."""
        a = _f64(u_dir_t0, (self.n_edge,))
        b = _f64(u_dir_t1 if u_dir_t1 is not None else u_dir_t0, (self.n_edge,))
        q = _f64(q_neu, (self.n_edge,))
        J = ctypes.c_double()
        gk = np.zeros((self.ny, self.nx))
        ga, gb, gq = (np.zeros(self.n_edge) for _ in range(3))
        rc = self._lib.or_lbm_adjoint(self._h, int(n), int(eta), _ptr(a), _ptr(b), _ptr(q),
                                      ctypes.byref(J), _ptr(gk), _ptr(ga), _ptr(gb), _ptr(gq))
        if rc != 0:
            raise ValueError({-1: "the adjoint needs a fixed mask (dissolution off)",
                              -2: "two Neumann sides meet at a corner",
                              -4: "the adjoint covers bounce-back walls only",
                              -3: "out of memory"}.get(rc, f"error {rc}"))
        return dict(J=J.value, k=gk, ua=ga, ub=gb, q=gq)

    def u(self):
        out = np.empty((self.ny, self.nx))
        self._lib.or_lbm_get_u(self._h, _ptr(out))
        return out

    def f(self):
        out = np.empty((9, self.ny, self.nx))
        self._lib.or_lbm_get_f(self._h, _ptr(out))
        return out

    def fpost(self):
        out = np.empty((9, self.ny, self.nx))
        self._lib.or_lbm_get_fpost(self._h, _ptr(out))
        return out

    def solid(self):
        out = np.empty((self.ny, self.nx), dtype=np.uint8)
        self._lib.or_lbm_get_solid(self._h, _ptr(out))
        return out

    def mineral(self):
        out = np.empty((self.ny, self.nx))
        self._lib.or_lbm_get_mineral(self._h, _ptr(out))
        return out

    def flip_steps(self):
        """[ny, nx] int32: steps after which each node was first fluid by
        dissolution (-1 for nodes never turned fluid) -- the integer record
        behind the exact-mask comparison (reading c16)."""
        out = np.empty((self.ny, self.nx), dtype=np.int32)
        self._lib.or_lbm_get_flip_steps(self._h, _ptr(out))
        return out

    def diag(self):
        d = np.empty(8)
        self._lib.or_lbm_diag(self._h, _ptr(d))
        keys = ("mass", "J", "reacted", "bc_infeasible", "flips",
                "newton_iters", "newton_fail", "steps")
        return dict(zip(keys, d.tolist()))

    def H(self):
        return float(self._lib.or_lbm_H(self._h))

    def trace(self, xy):
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        return np.array([self._lib.or_trace_point(self._h, float(p[0]), float(p[1]))
                         for p in xy])


def maxent_dirichlet(f, unknown, up):
    """Single-node max-entropy Dirichlet solution (Sec. 4.1.1 (a))."""
    lib = _load()
    f = np.array(f, dtype=np.float64)
    unk = np.ascontiguousarray(unknown, dtype=np.int32)
    bad = lib.or_maxent_dirichlet(_ptr(f), _ptr(unk), float(up))
    return f, bool(bad)


def maxent_neumann(f, unknown, normal, q):
    """Single-node max-entropy Neumann solution (Sec. 4.1.1 (b)); unknowns
    with e_i.n >= 0 must already be filled by the caller."""
    lib = _load()
    f = np.array(f, dtype=np.float64)
    unk = np.ascontiguousarray(unknown, dtype=np.int32)
    iters = ctypes.c_longlong(0)
    fail = ctypes.c_int(0)
    bad = lib.or_maxent_neumann(_ptr(f), _ptr(unk), float(normal[0]),
                                float(normal[1]), float(q),
                                ctypes.byref(iters), ctypes.byref(fail))
    return f, bool(bad), int(iters.value), bool(fail.value)
