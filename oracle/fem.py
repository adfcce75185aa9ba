"""Q1 finite elements for the continuum advection-diffusion equation, and
the two-subdomain hybrid coupling loop (Algorithm 1).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` may use this module; the product path never imports it.

Continuum model (Sec. 3, Eq. "ADE"): dc/dt + v.grad c - D lap c = 0 on a
rectangle meshed by nex x ney bilinear (Q1) elements, some of which may be
switched off (a hole where the pore-scale subdomain lives).  Weak forms:
 - Galerkin (Sec. 3.1.1): M_ab = int N_a N_b,
   K_ab = int N_a v.grad N_b + D grad N_a . grad N_b;
 - SUPG (Sec. 3.1.2, Eq. "SUPG", "SUPG_tau"): the test function gains
   tau_e v.grad N_a applied to the whole residual; inside a bilinear element
   lap c = 0, so M gains tau int (v.grad N_a) N_b and K gains
   tau int (v.grad N_a)(v.grad N_b), with tau_e = h/(2|v|) (coth Pe - 1/Pe),
   Pe = |v| h / (2 D), h = 2 / sum_a |v^.grad N_a| at the element centre
   (the element length along the flow).
Integrals use 2 x 2 Gauss points, exact for these bilinear products.
Time stepping, the generalized trapezoidal rule of Sec. 6.1.1 (Eq.
"FEM_discrete"): (M + theta dt K) d^{n+1} = (M - (1 - theta) dt K) d^n, the
Dirichlet nodes taking their prescribed values at t^{n+1}; sides that are not
Dirichlet are zero-flux (natural).  The linear system is solved by a sparse
direct factorisation (a library primitive).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_G = 1.0 / math.sqrt(3.0)
# local node order: (0,0), (1,0), (1,1), (0,1) in element coordinates
_LOC = ((0, 0), (1, 0), (1, 1), (0, 1))


def _shape(xi, eta):
    """Bilinear shape functions on [0,1]^2 and their xi, eta derivatives."""
    N = np.array([(1 - xi) * (1 - eta), xi * (1 - eta), xi * eta, (1 - xi) * eta])
    dxi = np.array([-(1 - eta), (1 - eta), eta, -eta])
    deta = np.array([-(1 - xi), -xi, xi, (1 - xi)])
    return N, dxi, deta


def supg_tau(hx, hy, D, v):
    """tau_e of Eq. "SUPG_tau" for a uniform velocity v on an hx x hy element."""
    vx, vy = v
    speed = math.hypot(vx, vy)
    if speed == 0.0:
        return 0.0
    _, dxi, deta = _shape(0.5, 0.5)
    s = np.abs((vx * dxi / hx + vy * deta / hy) / speed).sum()
    h = 2.0 / s
    pe = speed * h / (2.0 * D) if D > 0 else math.inf
    xi = 1.0 if math.isinf(pe) else (1.0 / math.tanh(pe) - 1.0 / pe)
    return h / (2.0 * speed) * xi


def element_matrices(hx, hy, D, v=(0.0, 0.0), tau=0.0):
    """(M, K) of one hx x hy element with uniform D, v and SUPG weight tau."""
    vx, vy = v
    M = np.zeros((4, 4))
    K = np.zeros((4, 4))
    w = hx * hy / 4.0  # Gauss weights 1/2 x 1/2 on [0,1]^2 times the Jacobian
    for gx in (0.5 - 0.5 * _G, 0.5 + 0.5 * _G):
        for gy in (0.5 - 0.5 * _G, 0.5 + 0.5 * _G):
            N, dxi, deta = _shape(gx, gy)
            Nx, Ny = dxi / hx, deta / hy
            adv = vx * Nx + vy * Ny  # v.grad N
            test = N + tau * adv     # SUPG test function
            M += w * np.outer(test, N)
            K += w * (np.outer(test, adv) + D * (np.outer(Nx, Nx) + np.outer(Ny, Ny)))
    return M, K


class Q1FEM:
    """Structured Q1 mesh on [x0, x0 + nex hx] x [y0, y0 + ney hy].

    ``elem_active`` [ney, nex] (bool, default all), ``dirichlet`` a list of
    node ids whose values are prescribed at every step (the others on the
    mesh boundary are zero-flux), node id = j (nex + 1) + i.
    """

    def __init__(self, nex, ney, x0, y0, hx, hy, D, v=(0.0, 0.0), theta=0.5, dt=1.0,
                 supg=False, elem_active=None, dirichlet=(), d0=None):
        self.nex, self.ney = int(nex), int(ney)
        self.x0, self.y0, self.hx, self.hy = float(x0), float(y0), float(hx), float(hy)
        nxn, nyn = self.nex + 1, self.ney + 1
        self.n = nxn * nyn
        act = np.ones((self.ney, self.nex), bool) if elem_active is None else \
            np.asarray(elem_active, bool)
        self.elem_active = act
        tau = supg_tau(hx, hy, D, v) if supg else 0.0
        Me, Ke = element_matrices(hx, hy, D, v, tau)
        rows, cols, mv, kv = [], [], [], []
        touched = np.zeros(self.n, bool)
        for j in range(self.ney):
            for i in range(self.nex):
                if not act[j, i]:
                    continue
                ids = [(j + b) * nxn + (i + a) for a, b in _LOC]
                touched[ids] = True
                for p in range(4):
                    for q in range(4):
                        rows.append(ids[p])
                        cols.append(ids[q])
                        mv.append(Me[p, q])
                        kv.append(Ke[p, q])
        M = sp.csr_matrix((mv, (rows, cols)), shape=(self.n, self.n))
        K = sp.csr_matrix((kv, (rows, cols)), shape=(self.n, self.n))
        self.M, self.K = M, K
        self.active_nodes = touched
        self.dirichlet = np.asarray(dirichlet, dtype=np.int64)
        fixed = np.zeros(self.n, bool)
        fixed[self.dirichlet] = True
        self.free = np.flatnonzero(touched & ~fixed)
        self.theta, self.dt = float(theta), float(dt)
        A = (M + self.theta * self.dt * K).tocsc()
        self._B = (M - (1.0 - self.theta) * self.dt * K).tocsr()
        self._A_ff = A[self.free][:, self.free].tocsc()
        self._A_fd = A[self.free][:, self.dirichlet].tocsc()
        self._lu = spla.splu(self._A_ff)
        self.d = np.zeros(self.n) if d0 is None else np.array(d0, dtype=np.float64).reshape(-1)
        self.d[~touched] = 0.0

    def node_xy(self):
        nxn = self.nex + 1
        ids = np.arange(self.n)
        return np.stack([self.x0 + (ids % nxn) * self.hx, self.y0 + (ids // nxn) * self.hy], 1)

    def step(self, dir_values=()):
        """Advance one dt with the Dirichlet nodes at the given values."""
        vals = np.asarray(dir_values, dtype=np.float64).reshape(-1)
        rhs = (self._B @ self.d)[self.free]
        if self.dirichlet.size:
            rhs -= self._A_fd @ vals
        new = np.zeros(self.n)
        new[self.free] = self._lu.solve(rhs)
        if self.dirichlet.size:
            new[self.dirichlet] = vals
        self.d = new

    def interpolate(self, xy):
        """Finite-element (bilinear) value of d at points xy [n, 2] inside
        the mesh (Sec. 5.1: coarse-to-fine transfer by the element's own
        interpolant)."""
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        nxn = self.nex + 1
        out = np.empty(len(xy))
        for k, (x, y) in enumerate(xy):
            i = min(max(int(math.floor((x - self.x0) / self.hx)), 0), self.nex - 1)
            j = min(max(int(math.floor((y - self.y0) / self.hy)), 0), self.ney - 1)
            xi = (x - self.x0) / self.hx - i
            eta = (y - self.y0) / self.hy - j
            N, _, _ = _shape(xi, eta)
            ids = [(j + b) * nxn + (i + a) for a, b in _LOC]
            out[k] = N @ self.d[ids]
        return out

    def mass(self):
        """int c = 1^T M d."""
        return float(np.ones(self.n) @ (self.M @ self.d))


def schwarz_step(fem, lbm, eta, max_iter, fem_fixed_values, fem_gamma_lattice_xy,
                 lbm_gamma_points, lbm_gamma_slots, q_neu=None):
    """One coarse step of Algorithm 1 (two subdomains, multi-time-step).

    fem: Q1FEM whose Dirichlet list is [fixed nodes..., Gamma_f->c nodes...];
    lbm: the fine solver (LBMOracle) with snapshot/rollback;
    fem_fixed_values: values of the fixed Dirichlet nodes;
    fem_gamma_lattice_xy: lattice coordinates of the Gamma_f->c FEM nodes
      (where the fine solution is traced, Sec. 6.2 (ii));
    lbm_gamma_points: physical coordinates of the lattice Gamma_c->f edge
      nodes, lbm_gamma_slots their slots in the lattice edge layout.
    Every Schwarz iteration restarts both solvers from t_n; iteration 1
    takes the fine trace at t_n, later ones the trace at t_{n+1} of the
    previous iteration; the lattice Dirichlet data are interpolated in time
    between the FEM solutions at t_n and t_{n+1} (Eq. "MTS").
    """
    d_n = fem.d.copy()
    snap = lbm.snapshot()
    trace = lbm.trace(fem_gamma_lattice_xy)
    n_edge = lbm.n_edge
    for it in range(max_iter):
        fem.d = d_n.copy()
        fem.step(np.concatenate([np.asarray(fem_fixed_values, float), trace]))
        ua = np.zeros(n_edge)
        ub = np.zeros(n_edge)
        fem_new = fem.d
        fem.d = d_n
        ua[lbm_gamma_slots] = fem.interpolate(lbm_gamma_points)
        fem.d = fem_new
        ub[lbm_gamma_slots] = fem.interpolate(lbm_gamma_points)
        if it > 0:
            lbm.rollback(snap)
        lbm.substeps(eta, eta, ua, ub, q_neu)
        trace = lbm.trace(fem_gamma_lattice_xy)
    return trace


def schwarz_step_many(fem, lbms, eta, max_iter, fem_fixed_values, fem_gamma_lattice_xy,
                      lbm_gamma_points, lbm_gamma_slots, q_neu=None):
    """One coarse step of Algorithm 2 with one continuum subdomain and several
    fine ones: the continuum's Dirichlet list is [fixed nodes..., Gamma_f->c
    nodes of lattice 0..., of lattice 1..., ...]; the per-lattice arguments
    are lists.  Each Schwarz iteration advances the continuum with the traces
    of every lattice, then every lattice with the continuum's interpolants at
    t_n and t_{n+1}; all restart from t_n after the first iteration."""
    d_n = fem.d.copy()
    snaps = [l.snapshot() for l in lbms]
    traces = [l.trace(g) for l, g in zip(lbms, fem_gamma_lattice_xy)]
    ua_all = []
    for l, p, s in zip(lbms, lbm_gamma_points, lbm_gamma_slots):
        ua = np.zeros(l.n_edge)
        ua[s] = fem.interpolate(p)
        ua_all.append(ua)
    for it in range(max_iter):
        fem.d = d_n.copy()
        fem.step(np.concatenate([np.asarray(fem_fixed_values, float)] + traces))
        for k, (l, p, s) in enumerate(zip(lbms, lbm_gamma_points, lbm_gamma_slots)):
            ub = np.zeros(l.n_edge)
            ub[s] = fem.interpolate(p)
            if it > 0:
                l.rollback(snaps[k])
            l.substeps(eta, eta, ua_all[k], ub, q_neu)
        traces = [l.trace(g) for l, g in zip(lbms, fem_gamma_lattice_xy)]
    return traces
