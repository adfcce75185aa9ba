"""Pins of the oracle's one-dimensional hybrid (oracle/hybrid1d.py, Sec. 7.1):
the D1Q2 lattice alone (its Neumann ends carry their flux datum, second
order on a diffusing Gaussian), the coupled loop on a closed form it must
reproduce to rounding (u = a + b t + (b / 2D) x^2 at tau = 1, v = 0: exact
for the D1Q2 step, for linear Crank-Nicolson elements with the natural end
at x = 0, and for the time interpolation of Eq. "MTS" -- data one substep
late or held at t_n miss it), second-order convergence of the coupled run to
the free-space solution away from the zero-flux wall, and the printed tables
of the section as upper bounds (our reading is far more accurate than the
tables, whose fine-scale errors fall like max|du/dx| h_f: first order)."""
import math
import os

import numpy as np
import pytest

from oracle import hybrid1d as h1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "e5_1d_hybrid_tables.txt")


def _rows():
    rows = []
    for ln in open(GOLDEN):
        if ln.strip() and not ln.startswith("#"):
            t, hc, hf, eta, L, it, ec, ef = ln.split()
            snap = lambda v: 1e-2 * 2.0 ** -round(math.log2(1e-2 / float(v)))  # 3.13e-4 -> 3.125e-4
            rows.append((int(t), snap(hc), snap(hf), int(eta), float(L), int(it), float(ec),
                         float(ef)))
    return rows


def test_d1q2_neumann_ends_carry_the_flux_datum():
    """Sec. 4.1.1 (b) on D1Q2: after each step the first moment through a
    Neumann end, outward positive, equals its datum (f_- - f_+ at the left
    end, f_+ - f_- at the right end); zero data make the unknown the known
    population (bounce-back)."""
    n = 50
    rng = np.random.default_rng(1)
    lat = h1.D1Q2(n, 0.8, 0.3, rng.uniform(0.5, 1.5, n), left=h1.NEUMANN, right=h1.NEUMANN)
    q = (0.02, -0.01)
    for _ in range(3):
        lat.substeps(1, 1, (0.0, 0.0), (0.0, 0.0), q)
        assert abs((lat.f[1, 0] - lat.f[0, 0]) - q[0]) <= 1e-15
        assert abs((lat.f[0, -1] - lat.f[1, -1]) - q[1]) <= 1e-15
    lat.substeps(1, 1, (0.0, 0.0), (0.0, 0.0), (0.0, 0.0))
    assert lat.f[1, -1] == lat.f[0, -1] and lat.f[0, 0] == lat.f[1, 0]


def test_d1q2_gaussian_converges_at_second_order():
    """The lattice alone, a Gaussian far from both (Dirichlet) ends: the
    error against the free-space solution falls by 4 per halving of h."""
    errs = []
    for h in (4e-3, 2e-3, 1e-3):
        g = h1.setup(h, h, 1, 0.0)  # dt = h^2 / 2D, tau = 1
        x = np.arange(0.0, 1.0 + h / 2, h)
        lat = h1.D1Q2(len(x), g["tau"], g["vl"], h1.gaussian(x, 0.0))
        n = int(round(0.2 / g["dt_f"]))
        for j in range(n):
            t0, t1 = j * g["dt_f"], (j + 1) * g["dt_f"]
            lat.substeps(1, 1, (h1.gaussian(0.0, t0), h1.gaussian(1.0, t0)),
                         (h1.gaussian(0.0, t1), h1.gaussian(1.0, t1)))
        errs.append(np.abs(lat.u - h1.gaussian(x, n * g["dt_f"])).max())
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4


D, BETA = 1e-2, 0.3


def _exact(x, t):
    return 1.0 + BETA * t + BETA / (2 * D) * np.asarray(x) ** 2


def _exact_run(eta, max_iter=3, n_coarse=40):
    return h1.run(1e-2, 5e-3, eta, 0.1, max_iter, D=D, v=0.0, init=lambda x: _exact(x, 0.0),
                  right=h1.DIRICHLET, right_value=lambda t: _exact(1.0, t), n_coarse=n_coarse)


@pytest.mark.parametrize("eta", [1, 4, 7])
def test_coupled_loop_reproduces_the_quadratic_closed_form(eta):
    out = _exact_run(eta)
    t = out["t"]
    assert np.abs(out["u_c"] - _exact(out["x_c"], t)).max() <= 1e-12
    assert np.abs(out["u_f"] - _exact(out["x_f"], t)).max() <= 1e-12


def test_closed_form_catches_late_or_frozen_interface_data(monkeypatch):
    """Planted in the oracle: the lattice's end data one substep late, or
    held at the coarse level t_n through the substeps; each leaves the
    closed form by O(b dt_f)."""
    orig = h1.D1Q2.substeps

    def late(self, n, eta, a, b, q=(0.0, 0.0)):
        for j in range(1, int(n) + 1):
            lag = [a[s] + (b[s] - a[s]) * (j - 1) / eta for s in (0, 1)]
            orig(self, 1, eta, lag, lag, q)

    def frozen(self, n, eta, a, b, q=(0.0, 0.0)):
        orig(self, n, eta, a, a, q)

    g = h1.setup(1e-2, 5e-3, 4, 0.1, D=D, v=0.0)
    for bad in (late, frozen):
        monkeypatch.setattr(h1.D1Q2, "substeps", bad)
        out = _exact_run(4)
        err = np.abs(out["u_f"] - _exact(out["x_f"], out["t"])).max()
        assert err > 0.1 * BETA * g["dt_f"], bad.__name__
        monkeypatch.setattr(h1.D1Q2, "substeps", orig)


def test_coupled_run_converges_at_second_order_away_from_the_wall():
    """Joint refinement of h_c and h_f (eta = 4, L = 0.1, MaxIter 4): the
    errors against the free-space Gaussian on the coarse nodes and on the
    fine nodes with x <= 0.8 (the zero-flux wall at x = 1 bends the solution
    near it) fall by about 4 per level."""
    ec, ef = [], []
    for hc, hf in ((1e-2, 5e-3), (5e-3, 2.5e-3), (2.5e-3, 1.25e-3)):
        out = h1.run(hc, hf, 4, 0.1, 4)
        t = out["t"]
        ec.append(np.abs(out["u_c"] - h1.gaussian(out["x_c"], t)).max())
        m = out["x_f"] <= 0.8
        ef.append(np.abs(out["u_f"][m] - h1.gaussian(out["x_f"][m], t)).max())
    for e in (ec, ef):
        assert 3.5 < e[0] / e[1] < 4.8 and 3.7 < e[1] / e[2] < 4.4


@pytest.mark.parametrize("row", [r for r in _rows() if r[1] >= 2.5e-3 and r[2] >= 1.25e-3])
def test_printed_tables_bound_the_errors(row):
    _, hc, hf, eta, L, it, ec, ef = row
    out = h1.run(hc, hf, eta, L, it)
    assert out["E_c"] <= ec and out["E_f"] <= ef
