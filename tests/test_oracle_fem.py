"""Pins of the oracle's Q1 finite elements (Sec. 3, Sec. 6.1) and of its
hybrid coupling loop (Algorithm 1), all on the CPU: element matrices against
the textbook closed forms (tensor products of the 1-D linear-element
matrices), exactness for linear steady states, nodal exactness of SUPG with
the optimal tau for steady 1-D advection-diffusion, conservation, the
second-order convergence of the trapezoidal rule on a diffusing Gaussian,
exactness of the element interpolant, and the coupled steady linear profile
across both subdomains."""
import math

import numpy as np
import pytest


def _fem():
    from oracle import fem
    return fem


def _m1(h):
    return h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])


def _k1(h):
    return 1.0 / h * np.array([[1.0, -1.0], [-1.0, 1.0]])


def _c1():  # int phi_a phi_b' on one linear element
    return 0.5 * np.array([[-1.0, 1.0], [-1.0, 1.0]])


def _tensor(ax, ay):
    """4 x 4 element matrix from 1-D matrices along x and y, local node order
    (0,0), (1,0), (1,1), (0,1)."""
    loc = ((0, 0), (1, 0), (1, 1), (0, 1))
    return np.array([[ax[a[0], b[0]] * ay[a[1], b[1]] for b in loc] for a in loc])


def test_element_matrices_closed_forms():
    fem = _fem()
    hx, hy, D, v = 0.3, 0.7, 0.11, (0.4, -0.25)
    M, K = fem.element_matrices(hx, hy, D, v)
    assert np.allclose(M, _tensor(_m1(hx), _m1(hy)), rtol=0, atol=1e-15)
    K_ref = D * (_tensor(_k1(hx), _m1(hy)) + _tensor(_m1(hx), _k1(hy))) + \
        v[0] * _tensor(_c1(), _m1(hy)) + v[1] * _tensor(_m1(hx), _c1())
    assert np.allclose(K, K_ref, rtol=0, atol=1e-14)
    # the textbook mass matrix of a rectangle
    assert np.allclose(M * 36 / (hx * hy), [[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2],
                                            [2, 1, 2, 4]], atol=1e-12)
    # SUPG terms: tau int (v.grad N_a) N_b and tau int (v.grad N_a)(v.grad N_b)
    tau = 0.05
    Ms, Ks = fem.element_matrices(hx, hy, D, v, tau)
    G = v[0] * _tensor(_c1(), _m1(hy)) + v[1] * _tensor(_m1(hx), _c1())   # N_a v.grad N_b
    VV = v[0] ** 2 * _tensor(_k1(hx), _m1(hy)) + v[1] ** 2 * _tensor(_m1(hx), _k1(hy)) + \
        v[0] * v[1] * (_tensor(_c1().T, _c1()) + _tensor(_c1(), _c1().T))
    assert np.allclose(Ms - M, tau * G.T, atol=1e-15)
    assert np.allclose(Ks - K, tau * VV, atol=1e-15)


def test_supg_tau_formula():
    fem = _fem()
    hx, hy, D = 0.02, 0.05, 1e-3
    for v in ((0.3, 0.0), (0.0, 0.2)):
        h = hx if v[1] == 0 else hy
        speed = math.hypot(*v)
        pe = speed * h / (2 * D)
        ref = h / (2 * speed) * (1 / math.tanh(pe) - 1 / pe)
        assert fem.supg_tau(hx, hy, D, v) == pytest.approx(ref, rel=1e-14)
    assert fem.supg_tau(hx, hy, D, (0.0, 0.0)) == 0.0


def _x_sides(nex, ney):
    nxn = nex + 1
    west = [j * nxn for j in range(ney + 1)]
    east = [j * nxn + nex for j in range(ney + 1)]
    return west, east


def test_steady_linear_diffusion_is_exact():
    fem = _fem()
    nex, ney = 12, 4
    west, east = _x_sides(nex, ney)
    f = fem.Q1FEM(nex, ney, 0.0, 0.0, 0.1, 0.2, D=0.3, theta=1.0, dt=1e14,
                  dirichlet=west + east)
    f.step([1.0] * len(west) + [2.0] * len(east))
    x = f.node_xy()[:, 0]
    assert np.abs(f.d - (1.0 + x / 1.2)).max() <= 1e-12


@pytest.mark.parametrize("nex", [10, 24])
def test_supg_nodally_exact_steady_advection_diffusion(nex):
    fem = _fem()
    L, D, vx = 1.0, 0.02, 1.0
    west, east = _x_sides(nex, 2)
    kw = dict(D=D, v=(vx, 0.0), theta=1.0, dt=1e14, dirichlet=west + east)
    vals = [0.0] * len(west) + [1.0] * len(east)
    f = fem.Q1FEM(nex, 2, 0.0, 0.0, L / nex, 0.1, supg=True, **kw)
    f.step(vals)
    x = f.node_xy()[:, 0]
    exact = np.expm1(vx * x / D) / np.expm1(vx * L / D)
    assert np.abs(f.d - exact).max() <= 1e-10
    g = fem.Q1FEM(nex, 2, 0.0, 0.0, L / nex, 0.1, supg=False, **kw)
    g.step(vals)
    assert np.abs(g.d - exact).max() > 1e-3  # plain Galerkin is not


def test_galerkin_conserves_mass_with_zero_flux():
    fem = _fem()
    rng = np.random.default_rng(3)
    f = fem.Q1FEM(9, 7, 0.0, 0.0, 0.1, 0.1, D=0.05, dt=0.3,
                  d0=rng.uniform(0, 1, 80))
    m0 = f.mass()
    for _ in range(20):
        f.step()
    assert f.mass() == pytest.approx(m0, rel=1e-13)


def test_trapezoid_gaussian_second_order():
    """Diffusing Gaussian (y-invariant, zero flux far from the pulse):
    halving h and dt together quarters the error."""
    fem = _fem()
    D, T, s0 = 1e-2, 0.5, 0.01

    def err(nex):
        h = 1.0 / nex
        x = np.arange(nex + 1) * h
        c0 = sum(np.exp(-(x - 0.5 - m) ** 2 / (2 * s0)) for m in range(-4, 5))
        d0 = np.tile(c0, 3)
        nsteps = nex // 4
        f = fem.Q1FEM(nex, 2, 0.0, 0.0, h, 0.1, D=D, dt=T / nsteps, d0=d0)
        for _ in range(nsteps):
            f.step()
        s = s0 + 2 * D * T
        # zero flux at x = 0 and 1: images of the pulse at every half-integer
        exact = sum(math.sqrt(s0 / s) * np.exp(-(x - 0.5 - m) ** 2 / (2 * s))
                    for m in range(-4, 5))
        return np.abs(f.d[: nex + 1] - exact).max()

    e1, e2, e3 = err(40), err(80), err(160)
    assert 3.5 < e1 / e2 < 4.5 and 3.5 < e2 / e3 < 4.5


def test_interpolation_exact_for_bilinear_fields():
    fem = _fem()
    f = fem.Q1FEM(5, 4, -0.2, 0.1, 0.25, 0.3, D=1.0)
    xy = f.node_xy()
    g = lambda x, y: 1.5 - 0.7 * x + 0.4 * y + 0.9 * x * y
    f.d = g(xy[:, 0], xy[:, 1])
    rng = np.random.default_rng(1)
    pts = np.stack([rng.uniform(-0.2, 1.05, 50), rng.uniform(0.1, 1.3, 50)], 1)
    assert np.abs(f.interpolate(pts) - g(pts[:, 0], pts[:, 1])).max() <= 1e-13


def test_inactive_elements_form_a_hole():
    fem = _fem()
    act = np.ones((6, 8), bool)
    act[2:4, 3:5] = False
    f = fem.Q1FEM(8, 6, 0.0, 0.0, 0.1, 0.1, D=0.1, elem_active=act, d0=np.ones(63))
    inner = 3 * 9 + 4  # node (4, 3): every element around it is off
    assert not f.active_nodes[inner] and f.d[inner] == 0.0
    m0 = f.mass()
    for _ in range(5):
        f.step()
    assert f.mass() == pytest.approx(m0, rel=1e-13)  # the hole's edge is zero-flux


def test_coupled_steady_linear_profile(oracle_mod):
    """Pure diffusion across both subdomains with c = 1 at the FEM inlet and
    c = 2 at the lattice outlet (Dirichlet): the steady state is the straight
    line, which the FEM (Q1 holds linears), the lattice (max-ent Dirichlet is
    exact for a linear state) and both transfers reproduce, so Algorithm 1
    must converge to it."""
    fem = _fem()
    from oracle import LBMOracle
    nfx = 16
    h = 0.5 / nfx                      # lattice on [0.5, 1.0], nfx + 1 columns
    ny_f = 4                           # periodic in y, period ny_f h
    nex, ney = 12, 2                   # FEM on [0, 0.6], height ny_f h
    hy = ny_f * h / ney
    tau = 1.5
    lbm = LBMOracle(nfx + 1, ny_f, tau, edges=(1, 1, 0, 0))
    D = (tau - 0.5) / 3.0 * h * h      # lattice units: dt_f = 1
    eta = 10                           # 1700 coarse steps: 5.5 diffusion times
    west, east = _x_sides(nex, ney)
    f = fem.Q1FEM(nex, ney, 0.0, 0.0, 0.6 / nex, hy, D=D, dt=eta,
                  dirichlet=west + east)
    gamma_fc = np.array([[(0.6 - 0.5) / h, (j * hy) / h] for j in range(ney + 1)])
    pts = np.array([[0.5, y * h] for y in range(ny_f)])
    slots = np.arange(ny_f)                        # the lattice W side
    n_edge = lbm.n_edge
    east_data = np.zeros(n_edge)
    east_data[ny_f:2 * ny_f] = 2.0
    for _ in range(1700):
        d_n = f.d.copy()
        snap = lbm.snapshot()
        trace = lbm.trace(gamma_fc)
        for it in range(2):
            f.d = d_n.copy()
            f.step(np.concatenate([[1.0] * len(west), trace]))
            fem_new = f.d
            f.d = d_n
            ua = east_data.copy()
            ua[slots] = f.interpolate(pts)
            f.d = fem_new
            ub = east_data.copy()
            ub[slots] = f.interpolate(pts)
            if it:
                lbm.rollback(snap)
            lbm.substeps(eta, eta, ua, ub)
            trace = lbm.trace(gamma_fc)
    x_fem = f.node_xy()[:, 0]
    assert np.abs(f.d - (1.0 + x_fem)).max() <= 1e-9
    x_lat = 0.5 + np.arange(nfx + 1) * h
    assert np.abs(lbm.u() - (1.0 + x_lat)[None, :]).max() <= 1e-9


def _coupled_gaussian(level, T=0.02, D=0.05):
    """A Gaussian pulse centred in the overlap diffuses across both
    subdomains (pure diffusion, y-invariant data): FEM on [0, 0.6], lattice
    on [0.5, 1.0], eta = 4 substeps per coarse step, 3 Schwarz iterations,
    both grids refined together with a diffusive time step.  Returns the
    max errors against the free-space solution at T in each subdomain."""
    from oracle import LBMOracle
    fem = _fem()
    nfx = 32 * 2 ** level
    h = 0.5 / nfx
    tau = 1.0
    dt_f = (tau - 0.5) / 3.0 * h * h / D      # physical time of one lattice step
    eta = 4
    nex = 12 * 2 ** level
    hx = 0.6 / nex
    ny_f = 4
    x0, s0 = 0.55, 0.03 ** 2

    def exact(x, t):
        return math.sqrt(s0 / (s0 + 2 * D * t)) * np.exp(-(x - x0) ** 2 / (2 * (s0 + 2 * D * t)))

    xl = 0.5 + np.arange(nfx + 1) * h
    lbm = LBMOracle(nfx + 1, ny_f, tau, edges=(1, 2, 0, 0), u0=np.tile(exact(xl, 0), (ny_f, 1)))
    nxn = nex + 1
    west, east = _x_sides(nex, 1)
    xf = (np.arange(2 * nxn) % nxn) * hx
    f = fem.Q1FEM(nex, 1, 0.0, 0.0, hx, ny_f * h, D=D, dt=eta * dt_f, dirichlet=west + east,
                  d0=exact(xf, 0))
    gamma = np.array([[(0.6 - 0.5) / h, 0.0]] * 2)
    pts = np.array([[0.5, y * h] for y in range(ny_f)])
    slots = np.arange(ny_f)
    ncoarse = int(round(T / (eta * dt_f)))
    for _ in range(ncoarse):
        fem.schwarz_step(f, lbm, eta, 3, [0.0, 0.0], gamma, pts, slots)
    t = ncoarse * eta * dt_f
    ec = np.abs(f.d[:nxn] - exact(xf[:nxn], t)).max()
    ef = np.abs(lbm.u()[0] - exact(xl, t)).max()
    return ec, ef


def test_coupled_gaussian_converges_to_the_exact_solution(oracle_mod):
    """The transient coupled solution (Algorithm 1 with the multi-time-step
    interpolation) approaches the continuum solution in both subdomains as
    both grids are refined together."""
    errs = [_coupled_gaussian(level) for level in range(3)]
    (c0, f0), (c1, f1), (c2, f2) = errs
    assert c2 <= 4e-3 and f2 <= 1.2e-3
    assert c0 / c1 >= 2.0 and c1 / c2 >= 2.0
    assert f0 / f1 >= 1.8 and f1 / f2 >= 1.8
