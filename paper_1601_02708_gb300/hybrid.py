"""Host driver of the two-subdomain hybrid method: the multi-time-step
coupling of Algorithm 1 (Sec. 6.2) between the library's Q1 continuum solver
(``FEM``) and its lattice (``LBM``), with overlapping Schwarz iterations.

Per coarse step t_n -> t_{n+1} = t_n + eta dt_f:
  1. keep d^n and the lattice state (the rollback point of every iteration);
  2. coarse-to-fine data at t_n: the element interpolant of d^n at the
     lattice's Gamma_c->f nodes (Sec. 5.1; Sec. 6.2 (iii));
  3. fine-to-coarse data: the lattice's bilinear trace at the continuum's
     Gamma_f->c nodes (Sec. 6.2 (ii)), from the lattice at t_n;
  4. for each of max_iter Schwarz iterations (restarting both solvers from
     t_n after the first): a coarse step with the trace as Dirichlet data,
     the interpolant of d^{n+1} at Gamma_c->f, eta lattice substeps whose
     Dirichlet data move linearly from the t_n to the t_{n+1} values
     (Eq. "MTS"), then the new trace for the next iteration.
Every array stays in device memory: the trace is written straight into the
continuum's Dirichlet vector and the interpolant straight into the lattice's
edge arrays, all on one CUDA stream; the host only sequences the calls.
"""
from __future__ import annotations

import numpy as np

from .fem import FEM
from .lbm import LBM


class Hybrid:
    """A hybrid run built from a layout (see ``inputs.hybrid_plain_layout``
    and ``inputs.hybrid_block_layout``) on the current CUDA device."""

    def __init__(self, layout, precision=32, stream=None):
        import torch
        self.torch = torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.layout = layout
        self.eta = int(layout["eta"])
        self.max_iter = int(layout["max_iter"])
        dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()
        self.lbm = LBM(precision=precision, stream=stream, **layout["lbm"])
        self.fem = FEM(stream=stream, **layout["fem"])
        nf = len(layout["fixed_values"])
        self.nf = nf
        self.dir_values = torch.zeros(self.fem.n_dir, dtype=torch.float64, device="cuda")
        self.dir_values[:nf] = dev(layout["fixed_values"])
        self.gamma_xy = dev(layout["gamma_lattice_xy"])
        self.points = dev(layout["lbm_points"])
        s0, s1 = layout["lbm_slots"]
        self.s0, self.s1 = int(s0), int(s1)
        ne = self.lbm.n_edge
        self.ua = torch.zeros(ne, dtype=torch.float64, device="cuda")
        self.ub = torch.zeros(ne, dtype=torch.float64, device="cuda")
        q = layout.get("q_neu")
        self.q = None if q is None else dev(q)
        self.d_n = torch.empty(self.fem.n, dtype=torch.float64, device="cuda")
        self.snap = None
        self.coarse_steps = 0
        self.solver_iters = []

    def coarse_step(self):
        """One coarse step of Algorithm 1 (max_iter Schwarz iterations)."""
        lbm, fem = self.lbm, self.fem
        fem.get(self.d_n)
        self.snap = lbm.save(self.snap)
        fem.interpolate(self.points, out=self.ua[self.s0:self.s1])
        lbm.trace(self.gamma_xy, out=self.dir_values[self.nf:])
        for it in range(self.max_iter):
            if it > 0:
                fem.set(self.d_n)
                lbm.restore(self.snap)
            fem.step(self.dir_values)
            self.solver_iters.append(fem.solver_info()[0])
            fem.interpolate(self.points, out=self.ub[self.s0:self.s1])
            lbm.substeps(self.eta, self.eta, self.ua, self.ub, self.q)
            lbm.trace(self.gamma_xy, out=self.dir_values[self.nf:])
        self.coarse_steps += 1

    def run(self, n_coarse=None):
        for _ in range(int(self.layout["n_coarse"] if n_coarse is None else n_coarse)):
            self.coarse_step()

    def continuum(self):
        return self.fem.get()

    def close(self):
        self.lbm.close()
        self.fem.close()
