"""Pins of the oracle's maximum-entropy pore walls (Sec. 4.1.1 (b) with zero
flux at fluid nodes beside solid ones), checked against the condition's own
definition: unknowns are the populations whose source is solid, the normal
is the lattice-weighted direction to the solid neighbours, unknowns with
e_i . n >= 0 take halfway bounce-back, and the rest are w_i exp(-1 - gamma
e_i . n) with one gamma that makes the normal flux sum_i f_i e_i . n zero.
The lattice constants are typed out here, apart from the oracle's."""
import numpy as np
import pytest

from paper_1601_02708_gb300 import inputs

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
REV = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])


def _pair(oracle_mod, nx, ny, solid, seed, steps=1, tau=0.8):
    """A bounce-back and a max-entropy-wall oracle from the same state, after
    `steps` steps (all sides periodic: every fluid node is off the open
    sides)."""
    rng = np.random.default_rng(seed)
    vel = inputs.streamfunction_velocity(nx, ny, seed + 1, solid=solid)
    u0 = np.where(solid != 0, 0.0, rng.uniform(0.2, 1.0, (ny, nx)))
    runs = []
    for walls in ("bounce", "maxent"):
        o = oracle_mod.LBMOracle(nx, ny, tau, solid=solid, vel=vel, u0=u0, walls=walls)
        o.substeps(steps)
        runs.append(o)
    return runs


def _wall_geometry(solid, x, y):
    """Unknown directions (source x - e_i solid), the normal of node (x, y)
    and the unknowns tangent to it or pointing into the wall; the latter are
    decided on the normal scaled by 36 (integers: exact)."""
    ny, nx = solid.shape
    unk = [i for i in range(1, 9) if solid[(y - CY[i]) % ny, (x - CX[i]) % nx]]
    m = np.zeros(2, dtype=np.int64)
    for i in unk:  # the solid neighbour lies along -e_i
        m -= int(round(36 * W[i])) * np.array([CX[i], CY[i]])
    ln = np.hypot(*m)
    n = m / ln if ln > 0 else np.zeros(2)
    bounce = [i for i in unk if CX[i] * m[0] + CY[i] * m[1] >= 0]
    return unk, n, bounce


def test_flat_walls_split_the_incoming_flux_by_weight(oracle_mod):
    """A channel between two solid rows: at the nodes next to the bottom wall
    the unknowns N, NE, NW are 2/3, 1/6, 1/6 of f_S + f_SW + f_SE (the axis
    closed form), mirrored at the top wall; the known populations are those
    of a bounce-back run from the same state."""
    nx, ny = 23, 12
    solid = np.zeros((ny, nx), np.uint8)
    solid[0], solid[-1] = 1, 1
    bb, me = _pair(oracle_mod, nx, ny, solid, seed=4)
    f, fb = me.f(), bb.f()
    for y, unk, inc in ((1, (2, 5, 6), (4, 7, 8)), (ny - 2, (4, 7, 8), (2, 5, 6))):
        s = f[list(inc), y].sum(axis=0)
        np.testing.assert_allclose(f[list(inc), y], fb[list(inc), y], rtol=0, atol=1e-15)
        np.testing.assert_allclose(f[unk[0], y], 2 / 3 * s, rtol=1e-14)
        np.testing.assert_allclose(f[unk[1], y], s / 6, rtol=1e-14)
        np.testing.assert_allclose(f[unk[2], y], s / 6, rtol=1e-14)
    # away from the walls both runs agree after one step
    np.testing.assert_allclose(f[:, 2:ny - 2], fb[:, 2:ny - 2], rtol=0, atol=1e-15)


def test_single_solid_node_has_one_unknown_per_neighbour(oracle_mod):
    """Around one solid node every fluid neighbour has exactly one unknown,
    pointing away from the solid (e . n < 0), so the zero-flux constraint
    alone fixes it: f_u = -sum_{j != u} (e_j . n) f_j / (e_u . n)."""
    nx, ny = 15, 13
    solid = np.zeros((ny, nx), np.uint8)
    sx, sy = 7, 6
    solid[sy, sx] = 1
    _, me = _pair(oracle_mod, nx, ny, solid, seed=8, steps=3)
    f = me.f()
    for k in range(1, 9):
        x, y = sx + CX[k], sy + CY[k]
        unk, n, bounce = _wall_geometry(solid, x, y)
        assert unk == [k] and not bounce
        a = CX * n[0] + CY * n[1]
        assert a[k] < 0
        others = sum(a[j] * f[j, y, x] for j in range(9) if j != k)
        assert f[k, y, x] == pytest.approx(-others / a[k], rel=1e-13)
    assert me.diag()["bc_infeasible"] == 0


@pytest.mark.parametrize("seed,steps", [(11, 1), (12, 25)])
def test_porous_walls_have_zero_normal_flux(oracle_mod, seed, steps):
    """Every wall node of a disk packing: unknowns along or into the wall
    equal halfway bounce-back, the others share one gamma in the form
    w_i exp(-1 - gamma e_i . n), are non-negative, and the normal flux is
    zero (nodes with infeasible data are counted by the oracle instead)."""
    nx, ny = 48, 40
    solid = inputs.disk_packing(nx, ny, 0.6, seed, rmin=2, rmax=6)
    _, me = _pair(oracle_mod, nx, ny, solid, seed=seed, steps=steps - 1)
    fp = me.fpost()  # what the last step streams (and bounces back)
    me.substeps(1)
    f = me.f()
    checked = zeroed = 0
    for y in range(ny):
        for x in range(nx):
            if solid[y, x]:
                continue
            unk, n, bounce = _wall_geometry(solid, x, y)
            if not unk:
                continue
            a = CX * n[0] + CY * n[1]
            neg = [i for i in unk if i not in bounce]
            for i in bounce:
                assert f[i, y, x] == fp[REV[i], y, x]
            assert all(f[i, y, x] >= 0 for i in neg)
            if not neg:
                continue
            if any(f[i, y, x] == 0 for i in neg):
                zeroed += 1
                continue
            gam = [-(np.log(f[i, y, x] / W[i]) + 1) / a[i] for i in neg]
            assert np.ptp(gam) <= 1e-10 * max(1.0, abs(gam[0]))
            flux = float(np.dot(a, f[:, y, x]))
            assert abs(flux) <= 1e-13 * np.abs(f[:, y, x]).sum()
            checked += 1
    assert checked > 100
    assert zeroed <= me.diag()["bc_infeasible"]  # counted over all steps
    assert me.diag()["newton_fail"] == 0
