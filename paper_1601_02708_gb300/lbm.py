"""Python face of liblbmade.so: one D2Q9 ADE-LBM lattice on one GPU.

Argument marshalling only; every step of the method runs in the CUDA
library.  Arrays may be numpy arrays (host) or torch tensors (host or CUDA);
device tensors are passed to the library by pointer, host arrays are copied
by the library.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import Diag, LBMError, Params, check

PERIODIC, DIRICHLET, NEUMANN = 0, 1, 2
REACT_NONE, REACT_SURFACE, REACT_BULK = 0, 1, 2
# lbm_wall_mode: halfway bounce-back; zero-flux maximum entropy with the
# Newton solve in FP64 ("maxent") or in the lattice's own precision
# ("maxent_lattice", FP32 on an FP32 lattice)
WALLS = {"bounce": 0, "maxent": 1, "maxent_lattice": 2}


def _torch():
    import torch
    return torch


def _is_tensor(a):
    try:
        return isinstance(a, _torch().Tensor)
    except ImportError:  # pragma: no cover
        return False


_NP = {"f64": np.float64, "f32": np.float32, "u8": np.uint8}


def _in_ptr(a, kind, count, keep):
    """Pointer to a contiguous copy of `a` (dtype `kind`, `count` elements)."""
    if a is None:
        return None
    if _is_tensor(a):
        torch = _torch()
        td = {"f64": torch.float64, "f32": torch.float32, "u8": torch.uint8}[kind]
        t = a.detach()
        if t.dtype != td:
            t = (t != 0).to(td) if kind == "u8" else t.to(td)
        t = t.contiguous()
        if t.numel() != count:
            raise ValueError(f"expected {count} elements, got {t.numel()}")
        keep.append(t)
        return t.data_ptr()
    arr = np.asarray(a)
    if kind == "u8":
        arr = (arr != 0).astype(np.uint8)
    arr = np.ascontiguousarray(arr, dtype=_NP[kind]).reshape(-1)
    if arr.size != count:
        raise ValueError(f"expected {count} elements, got {arr.size}")
    keep.append(arr)
    return arr.ctypes.data


def _out_ptr(out, kind, count):
    if _is_tensor(out):
        torch = _torch()
        td = {"f64": torch.float64, "f32": torch.float32, "u8": torch.uint8}[kind]
        if out.dtype != td or not out.is_contiguous() or out.numel() != count:
            raise ValueError("output tensor has the wrong dtype, size or layout")
        return out.data_ptr()
    if not (isinstance(out, np.ndarray) and out.dtype == _NP[kind]
            and out.flags["C_CONTIGUOUS"] and out.size == count):
        raise ValueError("output array has the wrong dtype, size or layout")
    return out.ctypes.data


def current_stream_handle():
    """cudaStream_t of torch's current stream (None without CUDA)."""
    torch = _torch()
    if not torch.cuda.is_available():
        return None
    return torch.cuda.current_stream().cuda_stream


class LBM:
    """A D2Q9 lattice for the advection-diffusion(-reaction) equation.

    Parameters follow the problem statement of the pore-scale subdomain
    (Sec. 6, Eq. "CouplingPDE"): lattice size, relaxation time ``tau``
    (D = (tau - 1/2) / 3 in lattice units), side kinds ``edges`` for W, E, S, N
    (PERIODIC, DIRICHLET or NEUMANN), solid mask, advection velocity
    [2, ny, nx], initial concentration, and the first-order reaction
    (``react_mode``, ``k`` or ``k_field``, ``dissolution``, ``mineral``).
    ``precision`` 32 runs FP32 populations with FP64 boundary solves and
    sums; 64 runs FP64 throughout.  ``walls`` treats the pore walls by
    halfway bounce-back ("bounce") or as zero-flux boundaries of the
    maximum-entropy kind (Sec. 4.1.1 (b)) with the Lagrange multiplier's
    Newton solve in FP64 ("maxent") or in the lattice's precision
    ("maxent_lattice").
    """

    def __init__(self, nx, ny, tau, edges=(PERIODIC,) * 4, precision=32,
                 solid=None, vel=None, u0=None, react_mode=REACT_NONE, k=0.0,
                 k_field=None, dissolution=False, mineral=None, stream=None, walls="bounce"):
        self._lib = _lib.load()
        self.nx, self.ny = int(nx), int(ny)
        self.ny_whole = self.ny  # rows of the inputs (a slab's lattice has more)
        self.precision = int(precision)
        p = Params()
        p.nx, p.ny, p.precision = self.nx, self.ny, self.precision
        for i, e in enumerate(edges):
            p.edge[i] = int(e)
        p.tau = float(tau)
        p.react_mode = int(react_mode)
        p.k_scalar = float(k)
        p.dissolution = int(bool(dissolution))
        self.params = p
        self.edges = tuple(int(e) for e in edges)
        N = self.nx * self.ny_whole
        keep = []
        args = (_in_ptr(solid, "u8", N, keep), _in_ptr(vel, "f64", 2 * N, keep),
                _in_ptr(k_field, "f64", N, keep), _in_ptr(mineral, "f64", N, keep),
                _in_ptr(u0, "f64", N, keep))
        if stream is None:
            stream = current_stream_handle()
        self._stream = stream
        self._h = self._create(p, args, stream)
        self.set_walls(walls)

    def _create(self, p, args, stream):
        h = ctypes.c_void_p()
        check(self._lib.lbm_init(ctypes.byref(h), ctypes.byref(p), *args, stream))
        return h

    def set_walls(self, walls):
        """Pore walls from the next step on: "bounce" (halfway bounce-back),
        "maxent" or "maxent_lattice" (zero-flux maximum-entropy condition,
        lbm_set_wall_mode)."""
        if walls not in WALLS:
            raise ValueError(f"walls must be one of {sorted(WALLS)}")
        check(self._lib.lbm_set_wall_mode(self.handle, WALLS[walls]))
        self.walls = walls

    # -- lifetime --------------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.lbm_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        if self._h is None:
            raise LBMError(-5, "context is closed")
        return self._h

    @property
    def n_edge(self):
        return 2 * (self.nx + self.ny)

    # -- stepping --------------------------------------------------------------
    def substeps(self, n, eta=1, u_dir_t0=None, u_dir_t1=None, q_neu=None):
        """Advance n steps (substeps j = 1..n of ratio eta); edge arrays in
        the layout [W: ny][E: ny][S: nx][N: nx]."""
        keep = []
        m = self.n_edge
        a = _in_ptr(u_dir_t0, "f64", m, keep)
        b = _in_ptr(u_dir_t1, "f64", m, keep)
        q = _in_ptr(q_neu, "f64", m, keep)
        check(self._lib.lbm_substeps(self.handle, int(n), int(eta), a, b, q))
        self._keep = keep  # device inputs stay referenced until the next call

    def set_rate_field(self, k_field):
        """Replace the per-node rate k(x) [ny, nx] (the context must have
        been created with a ``k_field``)."""
        keep = []
        check(self._lib.lbm_set_rate_field(
            self.handle, _in_ptr(k_field, "f64", self.nx * self.ny, keep)))
        self.synchronize()

    def adjoint(self, n, eta=1, u_dir_t0=None, u_dir_t1=None, q_neu=None, stride=0):
        """Advance n substeps as ``substeps`` does and return the outlet
        breakthrough J (sum over the substeps of the fluid concentrations on
        the east edge) with its gradients, computed by the library's reverse
        sweep with sqrt(n) checkpoints: dict(J, k [ny, nx] = dJ/dk(x),
        ua / ub [n_edge] = dJ/d(Dirichlet data at the start / end),
        q [n_edge] = dJ/d(Neumann data), side [4] = dJ/d(one Dirichlet
        value held on the whole W, E, S, N side)).  Fixed mask only."""
        keep = []
        m = self.n_edge
        a = _in_ptr(u_dir_t0, "f64", m, keep)
        b = _in_ptr(u_dir_t1, "f64", m, keep)
        q = _in_ptr(q_neu, "f64", m, keep)
        J = ctypes.c_double()
        gk = np.empty((self.ny, self.nx))
        ga, gb, gq = (np.empty(m) for _ in range(3))
        gs = np.empty(4)
        check(self._lib.lbm_adjoint(self.handle, int(n), int(eta), int(stride), a, b, q,
                                    ctypes.byref(J), gk.ctypes.data, ga.ctypes.data,
                                    gb.ctypes.data, gq.ctypes.data, gs.ctypes.data))
        return dict(J=J.value, k=gk, ua=ga, ub=gb, q=gq, side=gs)

    KERNELS = {"auto": 0, "generic": 1, "tma": 2}

    def set_kernel(self, variant="auto"):
        """Step kernel: "auto", "generic" (thread per node) or "tma" (FP32
        tile pipeline); every variant computes the same update."""
        check(self._lib.lbm_set_kernel(self.handle, self.KERNELS[variant]))

    def kernel(self):
        """The step kernel the lattice runs now: "generic" or "tma"."""
        v = ctypes.c_int()
        check(self._lib.lbm_get_kernel(self.handle, ctypes.byref(v)))
        return {1: "generic", 2: "tma"}[v.value]

    def kernel_timing(self, enable=True):
        """Record CUDA events around every step and dissolution launch."""
        check(self._lib.lbm_kernel_timing(self.handle, int(bool(enable))))

    def kernel_times(self):
        """(step_ms_total, step_launches, dissolve_ms_total, dissolve_launches)."""
        a, c = ctypes.c_double(), ctypes.c_double()
        b, d = ctypes.c_longlong(), ctypes.c_longlong()
        check(self._lib.lbm_kernel_times_read(self.handle, ctypes.byref(a), ctypes.byref(b),
                                              ctypes.byref(c), ctypes.byref(d)))
        return a.value, b.value, c.value, d.value

    def synchronize(self):
        """Wait for the context's stream; returns 1 (LBM_WARN_BC_INFEASIBLE)
        when boundary solves since the last report met data with no
        non-negative solution, else 0."""
        return check(self._lib.lbm_synchronize(self.handle))

    # -- read-out --------------------------------------------------------------
    def concentration(self, out=None, precision=64):
        """u = sum_i f_i at the current time, [ny, nx] (numpy unless `out`
        is given)."""
        kind = "f64" if precision == 64 else "f32"
        if out is None:
            out = np.empty((self.ny, self.nx), dtype=_NP[kind])
        check(self._lib.lbm_get_concentration(
            self.handle, _out_ptr(out, kind, self.nx * self.ny), int(precision)))
        return out

    def min_population(self):
        """Smallest stored population over the fluid nodes (FP64)."""
        v = ctypes.c_double()
        check(self._lib.lbm_min_population(self.handle, ctypes.byref(v)))
        return v.value

    def populations(self, out=None):
        """Stored post-collision populations [9, ny, nx] (FP64)."""
        if out is None:
            out = np.empty((9, self.ny, self.nx))
        check(self._lib.lbm_get_populations(self.handle, _out_ptr(out, "f64", 9 * self.nx * self.ny)))
        return out

    def solid(self, out=None):
        if out is None:
            out = np.empty((self.ny, self.nx), dtype=np.uint8)
        check(self._lib.lbm_get_solid(self.handle, _out_ptr(out, "u8", self.nx * self.ny)))
        return out

    def flip_steps(self, out=None):
        """Dissolution record [ny, nx] (int32): the number of steps after
        which each node was first fluid, -1 for nodes never turned fluid."""
        if out is None:
            out = np.empty((self.ny, self.nx), dtype=np.int32)
        if not (isinstance(out, np.ndarray) and out.dtype == np.int32 and out.size == self.nx * self.ny) \
                and not _is_tensor(out):
            raise ValueError("output must be an int32 array of ny * nx elements")
        ptr = out.data_ptr() if _is_tensor(out) else out.ctypes.data
        check(self._lib.lbm_get_flip_steps(self.handle, ptr))
        return out

    def mineral(self, out=None):
        if out is None:
            out = np.empty((self.ny, self.nx))
        check(self._lib.lbm_get_mineral(self.handle, _out_ptr(out, "f64", self.nx * self.ny)))
        return out

    def diagnostics(self):
        """FP64 reductions and counters (lbm_diag).  The counts of boundary
        solves without a non-negative solution and of wall solves short of
        the Newton tolerance are reported here, not raised."""
        d = Diag()
        st = self._lib.lbm_diagnostics(self.handle, ctypes.byref(d))
        if st != _lib.LBM_ERR_NEWTON:
            check(st)
        return {k: getattr(d, k) for k, _ in Diag._fields_}

    def trace(self, xy, out=None):
        """LBM -> FEM transfer (Sec. 6.2 (ii)) at points xy [npts, 2] in
        lattice coordinates."""
        keep = []
        if _is_tensor(xy):
            npts = xy.numel() // 2
        else:
            xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
            npts = xy.shape[0]
        ptr = _in_ptr(xy, "f64", 2 * npts, keep)
        if out is None:
            out = np.empty(npts)
        check(self._lib.lbm_interface_trace(self.handle, int(npts), ptr,
                                            _out_ptr(out, "f64", npts)))
        return out

    # -- Schwarz rollback ------------------------------------------------------
    def state_bytes(self):
        n = ctypes.c_size_t()
        check(self._lib.lbm_state_bytes(self.handle, ctypes.byref(n)))
        return n.value

    def save(self, buf=None):
        """Save the full state into `buf` (a uint8 torch tensor, CUDA or
        host, or a numpy array) allocated here if not given."""
        nb = self.state_bytes()
        if buf is None:
            torch = _torch()
            buf = torch.empty(nb, dtype=torch.uint8,
                              device="cuda" if torch.cuda.is_available() else "cpu")
        check(self._lib.lbm_save(self.handle, _out_ptr(buf, "u8", buf.numel() if _is_tensor(buf) else buf.size), nb))
        return buf

    def restore(self, buf):
        nb = buf.numel() if _is_tensor(buf) else buf.size
        ptr = buf.data_ptr() if _is_tensor(buf) else buf.ctypes.data
        check(self._lib.lbm_restore(self.handle, ptr, nb))


class LBMPair:
    """Two lattices of one geometry stepped together (lbm_pair_*): one kernel
    launch a substep reads the shared velocity and link words once and
    updates both fields, each exactly as its own ``substeps`` would.  Both
    must be FP32, of one size, sides, mask, velocity, stream and step count,
    with bounce-back walls and no dissolution; ``LBMError`` otherwise.  The
    lattices stay usable on their own for read-outs; close the pair first."""

    def __init__(self, a, b):
        self._lib = _lib.load()
        self.a, self.b = a, b
        h = ctypes.c_void_p()
        check(self._lib.lbm_pair_create(ctypes.byref(h), a.handle, b.handle))
        self._h = h

    def substeps(self, n, eta=1, a_dir=(None, None), b_dir=(None, None), a_q=None, b_q=None):
        """n substeps of both; Dirichlet data per lattice as (at the start,
        at the end of the coarse step), Neumann data likewise, each in the
        edge layout of ``LBM.substeps``."""
        if self._h is None:
            raise LBMError(-5, "pair is closed")
        keep = []
        m = self.a.n_edge
        ptrs = [_in_ptr(x, "f64", m, keep) for x in (a_dir[0], a_dir[1], a_q,
                                                     b_dir[0], b_dir[1], b_q)]
        check(self._lib.lbm_pair_substeps(self._h, int(n), int(eta), *ptrs))
        self._keep = keep

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.lbm_pair_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def outlet_breakthrough(lbm, k_field, c_in, n, start_state, stride=0):
    """J(k, c_in): the outlet breakthrough of ``lbm`` over n substeps from
    ``start_state`` (a blob of ``lbm.save()``), with the rate field
    ``k_field`` [ny, nx] and a uniform inlet value ``c_in`` on the west side
    (zero-flux Neumann data elsewhere), as a differentiable torch function:
    its backward returns dJ/dk and dJ/dc_in from the library's adjoint.  The
    reverse sweep runs with the forward (one call computes both), so the
    backward only scales the stored gradients.  ``lbm`` is left after the n
    substeps."""
    return _Breakthrough.apply(k_field, c_in, lbm, int(n), start_state, int(stride))


def _breakthrough_class():
    torch = _torch()

    class Breakthrough(torch.autograd.Function):
        @staticmethod
        def forward(ctx, k_field, c_in, lbm, n, start_state, stride):
            lbm.restore(start_state)
            lbm.set_rate_field(k_field.detach().to(torch.float64).reshape(lbm.ny, lbm.nx))
            cin = float(c_in.detach().reshape(()).item()) if torch.is_tensor(c_in) else float(c_in)
            ud = np.zeros(lbm.n_edge)
            if lbm.edges[0] == DIRICHLET:
                ud[:lbm.ny] = cin
            r = lbm.adjoint(n, 1, ud, ud, None, stride)
            dev = k_field.device if torch.is_tensor(k_field) else "cpu"
            gk = torch.as_tensor(r["k"], device=dev).to(k_field.dtype).reshape(k_field.shape)
            gc = float(r["side"][0])  # dJ/dc_in of the west side, from the library
            ctx.save_for_backward(gk)
            ctx.gc = gc
            ctx.cin_like = c_in if torch.is_tensor(c_in) else None
            return torch.tensor(r["J"], dtype=torch.float64, device=dev)

        @staticmethod
        def backward(ctx, gJ):
            (gk,) = ctx.saved_tensors
            gc = None
            if ctx.cin_like is not None:
                gc = (gJ * ctx.gc).to(ctx.cin_like.dtype).reshape(ctx.cin_like.shape)
            return (gJ * gk).to(gk.dtype), gc, None, None, None, None

    return Breakthrough


class _LazyFunction:
    _cls = None

    def apply(self, *args):
        if _LazyFunction._cls is None:
            _LazyFunction._cls = _breakthrough_class()
        return _LazyFunction._cls.apply(*args)


_Breakthrough = _LazyFunction()


class LBMBatch:
    """Several lattices advanced together (Sec. 6.3, Algorithm 2 runs many
    pore-scale subdomains): every time step of the whole batch is one
    persistent step launch over all members' tiles plus one dissolution
    launch, replayed from a recorded CUDA graph.  Members are LBM objects
    sharing precision and a created stream (``LBM(..., stream=s)`` with
    ``s = torch.cuda.Stream().cuda_stream``); they stay usable for read-out.
    """

    def __init__(self, members):
        self._lib = _lib.load()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m.handle.value for m in self.members])
        h = ctypes.c_void_p()
        _lib.check_batch(self._lib.lbm_batch_create(ctypes.byref(h), len(self.members), arr))
        self._h = h
        sh = ctypes.c_int()
        _lib.check_batch(self._lib.lbm_batch_get_shape(self._h, ctypes.byref(sh)))
        self.shape = sh.value

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.lbm_batch_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptr_array(self, arrays, keep):
        if arrays is None:
            return None
        ptrs = []
        for m, a in zip(self.members, arrays):
            ptrs.append(_in_ptr(a, "f64", m.n_edge, keep) if a is not None else None)
        return (ctypes.c_void_p * len(ptrs))(*ptrs)

    def substeps(self, n, eta=1, u_dir_t0=None, u_dir_t1=None, q_neu=None):
        """n steps of every member; each edge argument is a list with one
        array (or None) per member."""
        keep = []
        a = self._ptr_array(u_dir_t0, keep)
        b = self._ptr_array(u_dir_t1, keep)
        q = self._ptr_array(q_neu, keep)
        _lib.check_batch(self._lib.lbm_batch_substeps(self._h, int(n), int(eta), a, b, q))

    @staticmethod
    def shapes():
        """Step-kernel shapes as (tile width, tile height, threads per
        block, pipelined)."""
        out = []
        lib = _lib.load()
        while True:
            v = [ctypes.c_int() for _ in range(4)]
            if lib.lbm_batch_shape_info(len(out), *[ctypes.byref(x) for x in v]) != 0:
                return out
            out.append((v[0].value, v[1].value, v[2].value, bool(v[3].value)))

    def set_shape(self, shape):
        _lib.check_batch(self._lib.lbm_batch_set_shape(self._h, int(shape)))
        self.shape = int(shape)

    def time_steps(self, n):
        """Device milliseconds of n steps (advances the state)."""
        ms = ctypes.c_float()
        _lib.check_batch(self._lib.lbm_batch_time_steps(self._h, int(n), ctypes.byref(ms)))
        return ms.value

    def autotune(self, trial_steps=20, repeats=2):
        """Pick the fastest tile shape by timing trial steps of the real
        batch; every member's state is saved before and restored after, so
        the batch ends where it started.  Returns {shape: ms}."""
        blobs = [m.save() for m in self.members]
        times = {}
        for s in range(len(self.shapes())):
            try:
                self.set_shape(s)
            except LBMError:  # the pipelined shape needs FP32 members
                continue
            self.time_steps(trial_steps)  # records the graph
            best = min(self.time_steps(trial_steps) for _ in range(repeats))
            times[s] = best
            for m, bl in zip(self.members, blobs):
                m.restore(bl)
        self.set_shape(min(times, key=times.get))
        for m, bl in zip(self.members, blobs):
            m.restore(bl)
        return times


__all__ = ["LBM", "LBMBatch", "LBMError", "outlet_breakthrough", "PERIODIC", "DIRICHLET", "NEUMANN",
           "REACT_NONE", "REACT_SURFACE", "REACT_BULK"]
