"""Pins of the oracle's discrete adjoint (the reverse mode of its own
substep with a fixed mask): central finite differences of the oracle's
forward objective with respect to every rate, every Dirichlet value (start
and end of the coarse step) and every Neumann value, on small lattices that
exercise bounce-back, periodic wrap, Dirichlet corners, the Neumann root and
its zero limit; and the homogeneity of J in the inlet value."""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def _case(seed, nx, ny, edges, react_mode, solid_cells, q_scale=0.02):
    from oracle import LBMOracle
    rng = np.random.default_rng(seed)
    solid = np.zeros((ny, nx), np.uint8)
    for (y, x) in solid_cells:
        solid[y, x] = 1
    vel = 0.04 * rng.standard_normal((2, ny, nx))
    vel[:, solid != 0] = 0
    kf = 2e-2 * (1 + 0.2 * rng.uniform(-1, 1, (ny, nx)))
    u0 = rng.uniform(0, 1, (ny, nx))
    u0[solid != 0] = 0
    ne = 2 * (nx + ny)
    ua = rng.uniform(0.5, 1.5, ne)
    ub = rng.uniform(0.5, 1.5, ne)
    q = q_scale * rng.uniform(-1, 1, ne)

    def make(k):
        return LBMOracle(nx, ny, 0.8, edges=edges, solid=solid, vel=vel, u0=u0,
                         react_mode=react_mode, k_field=k)
    return make, kf, ua, ub, q


def _fd_check(make, kf, ua, ub, q, n, eta, hk=1e-6, he=1e-3):
    r = make(kf).adjoint(n, eta, ua, ub, q)

    def J(k=kf, a=ua, b=ub, qq=q):
        o = make(k)
        o.substeps(n, eta, a, b, qq)
        return o.diag()["J"]

    assert r["J"] == pytest.approx(J(), rel=1e-14)
    ny, nx = kf.shape
    fd_k = np.zeros_like(kf)
    for y in range(ny):
        for x in range(nx):
            kp, km = kf.copy(), kf.copy()
            kp[y, x] += hk
            km[y, x] -= hk
            fd_k[y, x] = (J(k=kp) - J(k=km)) / (2 * hk)
    scale = np.abs(fd_k).max()
    assert scale > 0
    assert np.abs(fd_k - r["k"]).max() <= 1e-6 * scale
    for key, arr in (("ua", ua), ("ub", ub), ("q", q)):
        fd = np.zeros_like(arr)
        for e in range(arr.size):
            d = np.zeros_like(arr)
            d[e] = he
            kw = {"ua": "a", "ub": "b", "q": "qq"}[key]
            fd[e] = (J(**{kw: arr + d}) - J(**{kw: arr - d})) / (2 * he)
        # J is affine in the edge data while no Neumann branch switches
        assert np.abs(fd - r[key]).max() <= 1e-7 * max(np.abs(fd).max(), 1.0), key
    return r


def test_adjoint_matches_fd_inlet_outlet_periodic_bulk(oracle_mod):
    make, kf, ua, ub, q = _case(1, 7, 6, (1, 2, 0, 0), 2, [(2, 3), (3, 3), (5, 1)])
    r = _fd_check(make, kf, ua, ub, q, n=25, eta=6)
    assert np.abs(r["q"][6:12]).max() > 0 and np.abs(r["ua"][:6]).max() > 0


def test_adjoint_matches_fd_neumann_zero_limit(oracle_mod):
    # large positive q on part of the outlet: no root there (zero limit), so
    # those unknowns do not depend on the data and the q gradient vanishes
    make, kf, ua, ub, q = _case(2, 6, 5, (1, 2, 0, 0), 2, [(1, 2)])
    q[5:8] = 5.0
    r = _fd_check(make, kf, ua, ub, q, n=20, eta=4)
    assert np.all(r["q"][5:8] == 0.0) and np.abs(r["q"][8:10]).max() > 0


def test_adjoint_matches_fd_dirichlet_box_surface_reaction(oracle_mod):
    # Dirichlet west, south and north, Neumann east: corners with five
    # unknowns (Dirichlet wins where it meets the Neumann side); surface
    # reaction (only fluid nodes next to a solid react)
    make, kf, ua, ub, q = _case(3, 7, 6, (1, 2, 1, 1), 1, [(2, 2), (3, 3), (1, 5)])
    r = _fd_check(make, kf, ua, ub, q, n=18, eta=5)
    assert r["k"][4, 0] == 0.0  # not next to a solid: no reaction there
    assert np.abs(r["ua"][2 * 6 + 7:]).max() > 0  # the north side's data count


def test_adjoint_neumann_sides_on_x_and_dirichlet_on_y(oracle_mod):
    # Neumann west and east, Dirichlet south and north: every corner is
    # Dirichlet (it wins), so the map stays affine
    make, kf, ua, ub, q = _case(4, 6, 5, (2, 2, 1, 1), 2, [(2, 2)])
    _fd_check(make, kf, ua, ub, q, n=15, eta=3)


def test_adjoint_inlet_homogeneity(oracle_mod):
    """With c0 = 0 and zero-flux outlet, every state scales with the inlet
    value, so J = c_in dJ/dc_in exactly (dJ/dc_in = the sum of the W-side
    gradients with respect to the start and end data)."""
    from oracle import LBMOracle
    rng = np.random.default_rng(5)
    nx, ny = 10, 8
    solid = np.zeros((ny, nx), np.uint8)
    solid[3:5, 4:6] = 1
    vel = 0.04 * rng.standard_normal((2, ny, nx))
    vel[:, solid != 0] = 0
    kf = 1e-2 * (1 + 0.2 * rng.uniform(-1, 1, (ny, nx)))
    o = LBMOracle(nx, ny, 0.7, edges=(1, 2, 0, 0), solid=solid, vel=vel,
                  react_mode=2, k_field=kf)
    ne = 2 * (nx + ny)
    c_in = 1.7
    ud = np.zeros(ne)
    ud[:ny] = c_in
    r = o.adjoint(60, 1, ud, ud, np.zeros(ne))
    dj = r["ua"][:ny].sum() + r["ub"][:ny].sum()
    assert r["J"] > 0
    assert c_in * dj == pytest.approx(r["J"], rel=1e-12)


def test_adjoint_rejects_what_is_not_affine(oracle_mod):
    from oracle import LBMOracle
    o = LBMOracle(6, 6, 0.8, edges=(2, 2, 2, 2))
    with pytest.raises(ValueError):
        o.adjoint(3)
    o = LBMOracle(6, 6, 0.8, edges=(1, 2, 0, 0), react_mode=1, k=1e-3,
                  dissolution=True, solid=np.eye(6, dtype=np.uint8))
    with pytest.raises(ValueError):
        o.adjoint(3)
