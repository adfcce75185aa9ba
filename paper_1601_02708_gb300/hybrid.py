"""Host driver of the hybrid method: the multi-time-step coupling of
Algorithm 1 (Sec. 6.2) between the library's Q1 continuum solver (``FEM``)
and its lattice (``LBM``), with overlapping Schwarz iterations -- and, with
several lattices embedded in one continuum, the many-subdomain form of
Algorithm 2, whose lattices advance together as one batch (``LBMBatch``).

Per coarse step t_n -> t_{n+1} = t_n + eta dt_f:
  1. keep d^n and every lattice's state (the rollback point of every
     iteration);
  2. coarse-to-fine data at t_n: the element interpolant of d^n at every
     lattice's Gamma_c->f nodes (Sec. 5.1; Sec. 6.2 (iii));
  3. fine-to-coarse data: each lattice's bilinear trace at the continuum's
     Gamma_f->c nodes in it (Sec. 6.2 (ii)), from the lattices at t_n;
  4. for each of max_iter Schwarz iterations (restarting every solver from
     t_n after the first): a coarse step with the traces as Dirichlet data,
     the interpolant of d^{n+1} at every Gamma_c->f, eta lattice substeps
     whose Dirichlet data move linearly from the t_n to the t_{n+1} values
     (Eq. "MTS"), then the new traces for the next iteration.
Every array stays in device memory: each trace is written straight into its
slice of the continuum's Dirichlet vector and each interpolant straight into
its lattice's edge arrays, all on one CUDA stream; the host only sequences
the calls.
"""
from __future__ import annotations

import numpy as np

from .fem import FEM
from .lbm import LBM, LBMBatch


class Hybrid:
    """A hybrid run built from a layout on the current CUDA device: one
    lattice (``inputs.hybrid_plain_layout``, ``inputs.hybrid_block_layout``:
    keys ``lbm``, ``gamma_lattice_xy``, ``lbm_points``, ``lbm_slots``) or
    several (``inputs.hybrid_multiblock_layout``: ``lbms`` and lists of the
    others)."""

    def __init__(self, layout, precision=32, stream=None):
        import torch
        self.torch = torch
        self.layout = layout
        self.eta = int(layout["eta"])
        self.max_iter = int(layout["max_iter"])
        many = "lbms" in layout
        lbm_args = layout["lbms"] if many else [layout["lbm"]]
        gammas = layout["gamma_lattice_xy"] if many else [layout["gamma_lattice_xy"]]
        points = layout["lbm_points"] if many else [layout["lbm_points"]]
        slots = layout["lbm_slots"] if many else [layout["lbm_slots"]]
        if stream is None:
            if many:  # a batch records CUDA graphs: it needs a created stream
                self._stream = torch.cuda.Stream()
                stream = self._stream.cuda_stream
            else:
                stream = torch.cuda.current_stream().cuda_stream
        dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()
        self.lbms = [LBM(precision=precision, stream=stream, **a) for a in lbm_args]
        self.lbm = self.lbms[0]
        self.batch = LBMBatch(self.lbms) if many else None
        self.fem = FEM(stream=stream, **layout["fem"])
        nf = len(layout["fixed_values"])
        self.nf = nf
        self.dir_values = torch.zeros(self.fem.n_dir, dtype=torch.float64, device="cuda")
        self.dir_values[:nf] = dev(layout["fixed_values"])
        self.gammas, self.trace_out = [], []
        off = nf
        for g in gammas:
            self.gammas.append(dev(g))
            self.trace_out.append(self.dir_values[off:off + len(g)])
            off += len(g)
        assert off == self.fem.n_dir, "Dirichlet list does not match the traces"
        self.points = [dev(p) for p in points]
        self.ua, self.ub, self.ua_out, self.ub_out = [], [], [], []
        for lat, (s0, s1) in zip(self.lbms, slots):
            ua = torch.zeros(lat.n_edge, dtype=torch.float64, device="cuda")
            ub = torch.zeros(lat.n_edge, dtype=torch.float64, device="cuda")
            self.ua.append(ua)
            self.ub.append(ub)
            self.ua_out.append(ua[int(s0):int(s1)])
            self.ub_out.append(ub[int(s0):int(s1)])
        q = layout.get("q_neu")
        self.q = None if q is None else dev(q)
        self.d_n = torch.empty(self.fem.n, dtype=torch.float64, device="cuda")
        self.snaps = [None] * len(self.lbms)
        self.coarse_steps = 0
        self.solver_iters = []

    def _substeps(self):
        if self.batch is not None:
            qs = None if self.q is None else [self.q] * len(self.lbms)
            self.batch.substeps(self.eta, self.eta, self.ua, self.ub, qs)
        else:
            self.lbm.substeps(self.eta, self.eta, self.ua[0], self.ub[0], self.q)

    def _trace(self):
        for lat, g, out in zip(self.lbms, self.gammas, self.trace_out):
            lat.trace(g, out=out)

    def coarse_step(self):
        """One coarse step of Algorithm 1 / 2 (max_iter Schwarz iterations)."""
        fem = self.fem
        fem.get(self.d_n)
        for k, lat in enumerate(self.lbms):
            self.snaps[k] = lat.save(self.snaps[k])
            fem.interpolate(self.points[k], out=self.ua_out[k])
        self._trace()
        for it in range(self.max_iter):
            if it > 0:
                fem.set(self.d_n)
            # the continuum solve waits for its outcome, so the lattices'
            # restores (which wait to read their blob headers) come after it
            # and find the stream drained
            fem.step(self.dir_values)
            self.solver_iters.append(fem.solver_info()[0])
            if it > 0:
                for lat, snap in zip(self.lbms, self.snaps):
                    lat.restore(snap)
            for k in range(len(self.lbms)):
                fem.interpolate(self.points[k], out=self.ub_out[k])
            self._substeps()
            self._trace()
        self.coarse_steps += 1

    def run(self, n_coarse=None):
        for _ in range(int(self.layout["n_coarse"] if n_coarse is None else n_coarse)):
            self.coarse_step()

    def continuum(self):
        return self.fem.get()

    def close(self):
        if self.batch is not None:
            self.batch.close()
        for lat in self.lbms:
            lat.close()
        self.fem.close()
