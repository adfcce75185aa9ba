"""The one-dimensional hybrid of Sec. 7.1 (advection and diffusion of a
Gaussian hill): a D1Q2 lattice Boltzmann solver on the fine subdomain,
two-node linear finite elements (Galerkin) on the coarse one, coupled by
Algorithm 1 with multi-time-stepping (Eq. "MTS") and Schwarz iterations.

TEST INFRASTRUCTURE ONLY: the tests may use this module; the product path
never imports it.

Readings (the paper is silent or garbled on these):
 - D1Q2 (Sec. 4.1, "the standard DnQm lattices"): velocities +-c with
   c = h / dt, weights 1/2, c_s^2 = c^2; in lattice units c = 1, so
   D dt / h^2 = tau - 1/2 and the equilibrium is f_+- = (u/2)(1 +- v dt/h)
   (Eq. "LBM_feq" for D1Q2).  The section's dt_f = h_f^2 / (2D) gives tau = 1.
 - Step order as in the 2-D oracle: collide, stream (push), boundary
   conditions, moments.
 - Boundary conditions of Sec. 4.1.1 on D1Q2: each end has one unknown
   population.  Dirichlet u^p: the unknown takes the missing mass,
   f = u^p - (the known one).  Neumann q^p (first moment, outward): the
   unknown's e.n = -1, so f = (the known one) - q^p; zero flux is bounce-back
   (the paper notes the reduction for D1Q2).
 - Continuum: linear elements of length h on [0, Lc], M_e = h/6 [2 1; 1 2],
   K_e = D/h [1 -1; -1 1] + v/2 [-1 1; -1 1] (Galerkin, Sec. 3.1.1), the
   trapezoidal rule with theta = 1/2 (Eq. "FEM_discrete"); x = 0 natural
   (zero diffusive flux), x = Lc Dirichlet (the lattice's trace).
 - Transfers: the lattice's left node takes the element interpolant of the
   continuum; the continuum's right node takes the lattice value at that
   point (a lattice node: L_overlap is a multiple of h_f).
 - Algorithm 1 as in oracle.fem.schwarz_step: exactly max_iter iterations,
   each restarting both solvers from t_n; iteration 1 uses the lattice
   value at t_n, later ones that of the previous iteration at t_{n+1}.
 - T = 0.4: the text prints T = 4e-2, at which the hill (x0 = 0.3, v = 1)
   has not reached the overlap at x = 0.5 - L/2; the tables' errors and
   their floor at fine spacing (the free-space solution at x = 1, t = 0.4 is
   1.7e-3, the zero-flux wall's departure from it) fix T = 0.4.
 - The exact solution is the free-space Gaussian,
   u = phi / sqrt(2 pi s^2) exp(-(x - x0 - v t)^2 / (2 s^2)), s^2 = sigma0^2 + 2 D t.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_banded

DIRICHLET, NEUMANN = 1, 2


class D1Q2:
    """D1Q2 BGK lattice on nodes x0 + j h, j = 0 .. n-1 (lattice units in the
    update; tau and the lattice velocity vl = v dt / h fix the physics)."""

    def __init__(self, n, tau, vl, u0, left=DIRICHLET, right=NEUMANN):
        self.n, self.tau, self.vl = int(n), float(tau), float(vl)
        self.left, self.right = left, right
        u0 = np.asarray(u0, dtype=np.float64)
        self.f = np.stack([0.5 * u0 * (1 + self.vl), 0.5 * u0 * (1 - self.vl)])  # f_+, f_-
        self.u = u0.copy()

    def feq(self, u):
        return np.stack([0.5 * u * (1 + self.vl), 0.5 * u * (1 - self.vl)])

    def substeps(self, n, eta, a, b, q=(0.0, 0.0)):
        """n steps j = 1..n; end data (left, right) at step j interpolated as
        (1 - j/eta) a + (j/eta) b (Eq. "MTS"); q: Neumann data (left, right)."""
        for j in range(1, int(n) + 1):
            frac = j / eta
            data = [(1 - frac) * a[s] + frac * b[s] for s in (0, 1)]
            post = self.f - (self.f - self.feq(self.u)) / self.tau  # collide
            new = np.empty_like(post)
            new[0, 1:] = post[0, :-1]   # f_+ moves right
            new[1, :-1] = post[1, 1:]   # f_- moves left
            # left end: f_+ unknown; right end: f_- unknown
            if self.left == DIRICHLET:
                new[0, 0] = data[0] - new[1, 0]
            else:
                new[0, 0] = new[1, 0] - q[0]
            if self.right == DIRICHLET:
                new[1, -1] = data[1] - new[0, -1]
            else:
                new[1, -1] = new[0, -1] - q[1]
            self.f = new
            self.u = new[0] + new[1]

    def snapshot(self):
        return self.f.copy(), self.u.copy()

    def rollback(self, snap):
        self.f, self.u = snap[0].copy(), snap[1].copy()


class Linear1DFEM:
    """Two-node linear elements of length h on [0, n_el h]; the last node is
    a Dirichlet node, the first a natural (zero diffusive flux) one."""

    def __init__(self, n_el, h, D, v, dt, theta=0.5, d0=None):
        self.n = int(n_el) + 1
        self.h, self.dt, self.theta = float(h), float(dt), float(theta)
        Me = h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
        Ke = D / h * np.array([[1.0, -1.0], [-1.0, 1.0]]) + v / 2.0 * np.array([[-1.0, 1.0],
                                                                                [-1.0, 1.0]])
        M = np.zeros((self.n, self.n))
        K = np.zeros((self.n, self.n))
        for e in range(int(n_el)):
            M[e:e + 2, e:e + 2] += Me
            K[e:e + 2, e:e + 2] += Ke
        self.M, self.K = M, K
        self.A = M + self.theta * self.dt * K
        self.B = M - (1.0 - self.theta) * self.dt * K
        # banded form of the free block (all nodes but the last) for the solve
        Af = self.A[:-1, :-1]
        m = self.n - 1
        self._ab = np.zeros((3, m))
        self._ab[0, 1:] = np.diag(Af, 1)
        self._ab[1] = np.diag(Af)
        self._ab[2, :-1] = np.diag(Af, -1)
        self._a_fd = self.A[:-1, -1]
        self.d = np.zeros(self.n) if d0 is None else np.array(d0, dtype=np.float64)

    def step(self, right_value):
        rhs = (self.B @ self.d)[:-1] - self._a_fd * right_value
        new = np.empty(self.n)
        new[:-1] = solve_banded((1, 1), self._ab, rhs)
        new[-1] = right_value
        self.d = new

    def interpolate(self, x):
        i = min(max(int(math.floor(x / self.h)), 0), self.n - 2)
        xi = x / self.h - i
        return (1 - xi) * self.d[i] + xi * self.d[i + 1]


def gaussian(x, t, phi=0.1, sigma0=0.01, x0=0.3, v=1.0, D=1e-2):
    s2 = sigma0 ** 2 + 2 * D * t
    return phi / math.sqrt(2 * math.pi * s2) * np.exp(-(np.asarray(x) - x0 - v * t) ** 2 / (2 * s2))


def setup(h_c, h_f, eta, overlap, D=1e-2, v=1.0):
    """Geometry and step sizes of one table row: dt_f = h_f^2 / (2D),
    dt_c = eta dt_f (the tables' dt_c = h_c^2 / (2D) where eta matches)."""
    lc = 0.5 + overlap / 2.0
    xf0 = 0.5 - overlap / 2.0
    n_el = int(round(lc / h_c))
    nf = int(round((1.0 - xf0) / h_f)) + 1
    j_trace = int(round(overlap / h_f))  # the lattice node at x = lc
    dt_f = h_f * h_f / (2.0 * D)
    return dict(lc=lc, xf0=xf0, n_el=n_el, nf=nf, j_trace=j_trace, dt_f=dt_f, dt_c=eta * dt_f,
                tau=0.5 + D * dt_f / (h_f * h_f), vl=v * dt_f / h_f, h_c=h_c, h_f=h_f,
                eta=int(eta), D=D, v=v)


def run(h_c, h_f, eta, overlap, max_iter, T=0.4, theta=0.5, D=1e-2, v=1.0, init=None,
        right=NEUMANN, right_value=None, n_coarse=None):
    """The coupled run of Sec. 7.1 to time T (or n_coarse coarse steps);
    returns dict(E_c, E_f, u_c, u_f, x_c, x_f, n_coarse, t) with the errors
    against the free-space Gaussian.  ``init(x)`` replaces the Gaussian
    initial data; ``right``/``right_value(t)`` make the lattice's far end a
    Dirichlet end with the given data (the section's is zero-flux)."""
    g = setup(h_c, h_f, eta, overlap, D=D, v=v)
    x_c = np.arange(g["n_el"] + 1) * h_c
    x_f = g["xf0"] + np.arange(g["nf"]) * h_f
    f0 = init if init is not None else (lambda x: gaussian(x, 0.0, D=D, v=v))
    fem = Linear1DFEM(g["n_el"], h_c, D, v, g["dt_c"], theta, d0=f0(x_c))
    lat = D1Q2(g["nf"], g["tau"], g["vl"], f0(x_f), right=right)
    if n_coarse is None:
        n_coarse = int(round(T / g["dt_c"]))
    t = 0.0
    for _ in range(n_coarse):
        d_n = fem.d.copy()
        snap = lat.snapshot()
        trace = lat.u[g["j_trace"]]
        a_left = fem.interpolate(g["xf0"])
        ra = right_value(t) if right_value else 0.0
        rb = right_value(t + g["dt_c"]) if right_value else 0.0
        for it in range(max_iter):
            fem.d = d_n.copy()
            fem.step(trace)
            b_left = fem.interpolate(g["xf0"])
            if it > 0:
                lat.rollback(snap)
            lat.substeps(eta, eta, (a_left, ra), (b_left, rb))
            trace = lat.u[g["j_trace"]]
        t += g["dt_c"]
    return dict(E_c=float(np.abs(fem.d - gaussian(x_c, t, D=D, v=v)).max()),
                E_f=float(np.abs(lat.u - gaussian(x_f, t, D=D, v=v)).max()),
                u_c=fem.d.copy(), u_f=lat.u.copy(), x_c=x_c, x_f=x_f, n_coarse=n_coarse, t=t)
