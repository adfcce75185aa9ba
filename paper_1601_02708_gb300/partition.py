"""One lattice split into row slabs with a one-row halo exchange.

Sec. 5 couples subdomains that overlap and exchange data on their
interfaces; the lattice Boltzmann step (Eq. "LBE") reaches one node, so a
lattice split by rows needs one row of overlap, which each slab keeps in the
ghost row beyond a shared side.  Every step of the method runs in the
library: ``lbm_step_stream`` and ``lbm_step_dissolve`` are the two halves of
a time step, ``lbm_halo_pack`` / ``lbm_halo_unpack`` build and apply the two
messages each shared side carries per step (phase 0 after the fused step:
the populations that stream across and the reaction shares; phase 1 after
the dissolution pass: the boundary row's solid flags).  This module only
sequences the calls and moves the messages: between slabs held by one
process (``LocalExchange``, device-to-device copies -- several slabs on one
GPU), or between processes, one slab per rank (``DistExchange``,
torch.distributed point-to-point operations: NCCL between GPUs, gloo between
CPU processes).  The split lattice computes bit for bit what the whole one
does.

The exchange logic is written against a small protocol -- ``halo_bytes``,
``pack``, ``unpack``, ``stream``, ``dissolve`` -- so that it can be driven
with stand-in slabs on the CPU (the library's kernels need a GPU).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import check
from .lbm import LBM, PERIODIC, _in_ptr

SIDE_S, SIDE_N = 2, 3
EXCHANGE = 3  # lbm_edge_kind of a shared side


def slab_bounds(ny, parts):
    """Row ranges [(y0, y1), ...] of `parts` slabs covering ny rows, as even
    as possible (the first ny % parts slabs one row taller)."""
    parts = int(parts)
    if parts < 1 or ny < 2 * parts:
        raise ValueError("need at least two rows per slab")
    base, extra = divmod(int(ny), parts)
    out, y = [], 0
    for k in range(parts):
        h = base + (1 if k < extra else 0)
        out.append((y, y + h))
        y += h
    return out


def slice_edges(arr, nx, ny, y0, y1):
    """The slab's edge array [W: y1-y0][E: y1-y0][S: nx][N: nx] from the
    whole lattice's [W: ny][E: ny][S: nx][N: nx] (None stays None); the S and
    N parts only matter on a slab that holds that side of the lattice."""
    if arr is None:
        return None
    a = np.asarray(arr, dtype=np.float64)
    if hasattr(arr, "device") and not isinstance(arr, np.ndarray):  # a torch tensor
        import torch
        a = arr.to(torch.float64)
        return torch.cat([a[y0:y1], a[ny + y0:ny + y1], a[2 * ny:2 * ny + nx],
                          a[2 * ny + nx:2 * ny + 2 * nx]])
    return np.concatenate([a[y0:y1], a[ny + y0:ny + y1], a[2 * ny:2 * ny + nx],
                           a[2 * ny + nx:2 * ny + 2 * nx]])


class Slab(LBM):
    """Rows y0 .. y1 - 1 of a lattice (lbm_init_slab).  Inputs are the whole
    lattice's arrays; read-outs (concentration, populations, ...) are the
    slab's rows.  Sides shared with neighbouring slabs are `shared`."""

    def __init__(self, nx, ny, tau, y0, y1, **kw):
        self.y0, self.y1 = int(y0), int(y1)
        super().__init__(nx, ny, tau, **kw)
        self.ny = self.y1 - self.y0
        per_y = self.edges[2] == PERIODIC
        whole = self.y0 == 0 and self.y1 == self.ny_whole
        self.shared = [] if (whole and per_y) else \
            [s for s, cond in ((SIDE_S, self.y0 > 0 or per_y), (SIDE_N, self.y1 < self.ny_whole or per_y))
             if cond]
        self._bufs = {}

    def _create(self, p, args, stream):
        h = ctypes.c_void_p()
        check(self._lib.lbm_init_slab(ctypes.byref(h), ctypes.byref(p), self.y0, self.y1,
                                      *args, stream))
        return h

    # -- the exchange protocol ------------------------------------------------
    def halo_bytes(self, phase):
        n = ctypes.c_size_t()
        check(self._lib.lbm_halo_bytes(self.handle, int(phase), ctypes.byref(n)))
        return n.value

    def buffer(self, key, phase):
        """A device message buffer of this slab, kept between steps."""
        import torch
        b = self._bufs.get((key, phase))
        if b is None:
            b = torch.empty(self.halo_bytes(phase), dtype=torch.uint8, device="cuda")
            self._bufs[(key, phase)] = b
        return b

    def pack(self, side, phase):
        buf = self.buffer(("out", side), phase)
        check(self._lib.lbm_halo_pack(self.handle, int(side), int(phase), buf.data_ptr()))
        return buf

    def unpack(self, side, phase, buf):
        check(self._lib.lbm_halo_unpack(self.handle, int(side), int(phase), buf.data_ptr()))

    def inbox(self, side, phase):
        """The buffer a message arriving across `side` is received into."""
        return self.buffer(("in", side), phase)

    def stage_edges(self, u_dir_t0=None, u_dir_t1=None, q_neu=None):
        keep = []
        m = self.n_edge
        check(self._lib.lbm_stage_edges(self.handle, _in_ptr(u_dir_t0, "f64", m, keep),
                                        _in_ptr(u_dir_t1, "f64", m, keep),
                                        _in_ptr(q_neu, "f64", m, keep)))
        self._keep = keep

    def stream(self, j, eta, final):
        check(self._lib.lbm_step_stream(self.handle, int(j), int(eta), int(bool(final))))

    def dissolve(self):
        check(self._lib.lbm_step_dissolve(self.handle))


def _neighbour(k, side, parts, periodic):
    """Index of the slab across `side` of slab k (None at a lattice side)."""
    j = k - 1 if side == SIDE_S else k + 1
    if 0 <= j < parts:
        return j
    return j % parts if periodic else None


class LocalExchange:
    """Every slab in this process: a shared side's message goes straight to
    its neighbour (device-to-device, on the slabs' common stream)."""

    def __init__(self, slabs, periodic):
        self.slabs = slabs
        self.periodic = periodic

    def exchange(self, phase):
        P = len(self.slabs)
        sent = {}
        for k, s in enumerate(self.slabs):  # every pack before any unpack
            for side in s.shared:
                sent[(k, side)] = s.pack(side, phase)
        for k, s in enumerate(self.slabs):
            for side in s.shared:
                j = _neighbour(k, side, P, self.periodic)
                opposite = SIDE_N if side == SIDE_S else SIDE_S
                s.unpack(side, phase, sent[(j, opposite)])


class DistExchange:
    """One slab per rank of a torch.distributed group (rank k holds slab k):
    each shared side sends its message to the neighbouring rank and receives
    the neighbour's, in one batch of point-to-point operations (NCCL between
    GPUs, gloo between CPU processes).  With two ranks on a periodic lattice
    both sides face the same rank; the batch posts the sends and receives of
    each pair of ranks in the same order on both, so they match up."""

    def __init__(self, slab, rank, world, periodic, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.slab = slab
        self.rank, self.world = rank, world
        self.periodic = periodic
        self.group = group

    def exchange(self, phase):
        dist = self.dist
        s = self.slab
        ops = []
        outs = {side: s.pack(side, phase) for side in s.shared}
        # order: messages travelling up (N side out, S side in) first, then
        # those travelling down -- the same order on every rank
        for side in (SIDE_N, SIDE_S):
            if side in s.shared:
                peer = _neighbour(self.rank, side, self.world, self.periodic)
                ops.append(dist.P2POp(dist.isend, outs[side], peer, group=self.group))
            back = SIDE_S if side == SIDE_N else SIDE_N
            if back in s.shared:
                peer = _neighbour(self.rank, back, self.world, self.periodic)
                ops.append(dist.P2POp(dist.irecv, s.inbox(back, phase), peer, group=self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for side in s.shared:
            s.unpack(side, phase, s.inbox(side, phase))


def run_steps(slabs, exchange, n, eta, first=False):
    """n time steps of a split lattice: for each, the fused step of every
    slab, the phase-0 exchange, the dissolution pass, the phase-1 exchange.
    `first`: before the first step after initialisation, the first
    dissolution pass between the two exchanges."""
    if first:
        exchange.exchange(0)
        for s in slabs:
            s.dissolve()
        exchange.exchange(1)
    for j in range(1, int(n) + 1):
        for s in slabs:
            s.stream(j, eta, j == n)
        exchange.exchange(0)
        for s in slabs:
            s.dissolve()
        exchange.exchange(1)


class SlabLattice:
    """A lattice of nx x ny nodes split into row slabs.

    ``parts``: number of slabs (all in this process, ``LocalExchange``);
    or ``rank``/``world`` with a torch.distributed process group initialised
    (this process holds slab ``rank`` of ``world``, ``DistExchange``).  The
    other arguments are those of ``LBM`` and describe the whole lattice
    (whole-lattice input arrays, whole-lattice edge data in ``substeps``).
    """

    def __init__(self, nx, ny, tau, parts=None, rank=None, world=None, group=None, **kw):
        self.nx, self.ny = int(nx), int(ny)
        edges = tuple(int(e) for e in kw.get("edges", (PERIODIC,) * 4))
        self.periodic = edges[2] == PERIODIC
        if rank is None:
            self.bounds = slab_bounds(self.ny, parts or 1)
            self.slabs = [Slab(nx, ny, tau, y0, y1, **kw) for y0, y1 in self.bounds]
            self.exchange = LocalExchange(self.slabs, self.periodic)
        else:
            self.bounds = slab_bounds(self.ny, world)
            y0, y1 = self.bounds[rank]
            self.slabs = [Slab(nx, ny, tau, y0, y1, **kw)]
            self.exchange = DistExchange(self.slabs[0], rank, world, self.periodic, group)
        self._first = True

    def substeps(self, n, eta=1, u_dir_t0=None, u_dir_t1=None, q_neu=None):
        """n time steps (substeps j = 1..n of ratio eta) with whole-lattice
        edge arrays, as ``LBM.substeps``."""
        for s in self.slabs:
            s.stage_edges(*(slice_edges(a, self.nx, self.ny, s.y0, s.y1)
                            for a in (u_dir_t0, u_dir_t1, q_neu)))
        run_steps(self.slabs, self.exchange, n, eta, first=self._first)
        self._first = False

    def _gather(self, fn, dtype=np.float64):
        return np.concatenate([fn(s) for s in self.slabs], axis=-2)

    def concentration(self):
        """u [rows, nx] of the slabs this process holds, stacked in row order
        (the whole lattice with ``parts``)."""
        return self._gather(lambda s: s.concentration())

    def populations(self):
        return self._gather(lambda s: s.populations())

    def solid(self):
        return self._gather(lambda s: s.solid())

    def mineral(self):
        return self._gather(lambda s: s.mineral())

    def flip_steps(self):
        return self._gather(lambda s: s.flip_steps())

    def diagnostics(self):
        """Sums and counts over the slabs this process holds (FP64 sums in
        slab order)."""
        ds = [s.diagnostics() for s in self.slabs]
        out = {k: sum(d[k] for d in ds) for k in ("mass", "outlet_J", "outlet_flux",
                                                  "bc_infeasible", "newton_fail", "flips",
                                                  "n_solid")}
        out["steps"] = ds[0]["steps"]
        out["min_f"] = min(d["min_f"] for d in ds)
        return out

    def close(self):
        for s in self.slabs:
            s.close()


__all__ = ["SlabLattice", "Slab", "LocalExchange", "DistExchange", "run_steps", "slab_bounds",
           "slice_edges", "SIDE_S", "SIDE_N"]
