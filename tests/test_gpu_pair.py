"""The fused two-field step (lbm_pair_*): two lattices of one geometry
stepped by one kernel a substep.  Each field's populations must be the
ones its own lbm_substeps computes, bit for bit (the per-node arithmetic is
the same; only the tiling differs), its mass partials equal to rounding, and
both fields within the FP32 bound of the oracle; lattices that do not share
a geometry are refused."""
import numpy as np
import pytest

from paper_1601_02708_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02708_gb300 import build
    build.build()
    import paper_1601_02708_gb300 as pkg
    return pkg


def _case(nx, ny, seed):
    solid = inputs.disk_packing(nx, ny, 0.65, seed, rmin=3, rmax=9)
    vel = inputs.streamfunction_velocity(nx, ny, seed + 1, solid=solid)
    rng = np.random.default_rng(seed)
    u0 = np.where(solid != 0, 0.0, rng.uniform(0.0, 1.0, (ny, nx)))
    v0 = np.where(solid != 0, 0.0, rng.uniform(0.0, 0.5, (ny, nx)))
    return solid, vel, u0, v0


# sizes spanning several 96 x 4 tiles with ragged tails in x and y; the last
# one leaves the grid fewer tiles than SMs
@pytest.mark.parametrize("nx,ny,edges", [(200, 131, (1, 2, 0, 0)), (96, 64, (1, 1, 2, 2)),
                                         (301, 45, (0, 0, 0, 0)), (37, 5, (1, 2, 2, 1))])
def test_pair_equals_two_single_lattices(gb, nx, ny, edges):
    solid, vel, u0, v0 = _case(nx, ny, nx + ny)
    kw = dict(edges=edges, solid=solid, vel=vel, precision=32)
    singles = [gb.LBM(nx, ny, 0.8, u0=u0, **kw), gb.LBM(nx, ny, 0.62, u0=v0, **kw)]
    paired = [gb.LBM(nx, ny, 0.8, u0=u0, **kw), gb.LBM(nx, ny, 0.62, u0=v0, **kw)]
    pair = gb.LBMPair(*paired)
    ne = 2 * (nx + ny)
    rng = np.random.default_rng(5)
    d = [rng.uniform(0.2, 1.0, (2, ne)) for _ in range(2)]
    q = [rng.uniform(-0.01, 0.01, ne) for _ in range(2)]
    for n, eta in ((7, 7), (1, 3), (12, 12)):
        for s, dd, qq in zip(singles, d, q):
            s.substeps(n, eta, dd[0], dd[1], qq)
        pair.substeps(n, eta, (d[0][0], d[0][1]), (d[1][0], d[1][1]), q[0], q[1])
    for s, p in zip(singles, paired):
        assert np.array_equal(s.populations(), p.populations())
        assert np.array_equal(s.concentration(), p.concentration())
        ms, mp = s.diagnostics()["mass"], p.diagnostics()["mass"]
        assert abs(ms - mp) <= 1e-13 * abs(ms)
    pair.close()
    for x in singles + paired:
        x.close()


def test_pair_matches_the_oracle(gb, oracle_mod):
    nx, ny, steps = 150, 77, 60
    solid, vel, u0, v0 = _case(nx, ny, 9)
    edges = (1, 2, 0, 0)
    ud = inputs.edge_array(nx, ny, W=1.0)
    a = gb.LBM(nx, ny, 0.9, u0=u0, edges=edges, solid=solid, vel=vel)
    b = gb.LBM(nx, ny, 0.7, u0=v0, edges=edges, solid=solid, vel=vel)
    pair = gb.LBMPair(a, b)
    pair.substeps(steps, 1, (ud, ud), (0.5 * ud, 0.5 * ud))
    for lat, tau, u, scale in ((a, 0.9, u0, 1.0), (b, 0.7, v0, 0.5)):
        ref = oracle_mod.LBMOracle(nx, ny, tau, edges=edges, solid=solid, vel=vel, u0=u)
        ref.substeps(steps, 1, scale * ud, scale * ud)
        want = ref.u()
        assert np.abs(lat.concentration() - want).max() <= 1e-5 * np.abs(want).max()
    pair.close()
    a.close()
    b.close()


def test_pair_refusals(gb):
    nx, ny = 64, 40
    solid, vel, u0, _ = _case(nx, ny, 3)
    kw = dict(edges=(1, 2, 0, 0), solid=solid, vel=vel)
    a = gb.LBM(nx, ny, 0.8, u0=u0, **kw)
    other = [
        gb.LBM(nx, ny, 0.8, u0=u0, precision=64, **kw),                 # FP64
        gb.LBM(nx + 1, ny, 0.8, edges=(1, 2, 0, 0)),                      # size
        gb.LBM(nx, ny, 0.8, u0=u0, edges=(1, 1, 0, 0), solid=solid, vel=vel),  # sides
        gb.LBM(nx, ny, 0.8, u0=u0, edges=(1, 2, 0, 0), solid=solid, vel=0.5 * vel),  # flow
        gb.LBM(nx, ny, 0.8, u0=u0, edges=(1, 2, 0, 0), solid=np.zeros_like(solid), vel=vel),
        gb.LBM(nx, ny, 0.8, u0=u0, walls="maxent", **kw),                # wall treatment
    ]
    for o in other:
        with pytest.raises(gb.LBMError):
            gb.LBMPair(a, o)
    with pytest.raises(gb.LBMError):
        gb.LBMPair(a, a)
    b = gb.LBM(nx, ny, 0.8, u0=u0, **kw)
    pair = gb.LBMPair(a, b)
    pair.substeps(0)
    a.substeps(1)  # stepped apart: the pair's lattices are out of step
    with pytest.raises(gb.LBMError):
        pair.substeps(1)
    pair.close()
    for x in [a, b] + other:
        x.close()


def test_calcite_transport_fused_and_separate_agree(gb, oracle_mod):
    """Calcite (Sec. 7.4) on a porous lattice: psi1, psi2 carried by the
    fused pair and by two separate lattices agree bit for bit, match the
    oracle's lattices within the FP32 bound, and the species satisfy the
    equilibrium."""
    from oracle import chemistry
    nx, ny, steps, ksp = 120, 72, 80, 0.05
    solid, vel, _, _ = _case(nx, ny, 21)
    fluid = solid == 0
    u1 = np.where(fluid, 0.8, 0.0)
    u2 = np.where(fluid, 0.1, 0.0)
    u3 = np.where(fluid, 0.3, 0.0)
    edges = (1, 2, 0, 0)
    ud1 = inputs.edge_array(nx, ny, W=0.2)  # psi1 at the inlet
    ud2 = inputs.edge_array(nx, ny, W=0.6)  # psi2 at the inlet
    runs = [gb.Calcite(nx, ny, 0.8, ksp, u1, u2, u3, fused=f, edges=edges, solid=solid, vel=vel)
            for f in (True, False)]
    assert runs[0].pair is not None and runs[1].pair is None
    for r in runs:
        r.substeps(steps, 1, (ud1, ud1), (ud2, ud2))
    for x, y in zip(runs[0].invariants(), runs[1].invariants()):
        assert np.array_equal(x, y)
    p0 = chemistry.calcite_invariants(u1, u2, u3)
    refs = []
    for p, ud in zip(p0, (ud1, ud2)):
        o = oracle_mod.LBMOracle(nx, ny, 0.8, edges=edges, solid=solid, vel=vel, u0=p)
        o.substeps(steps, 1, ud, ud)
        refs.append(o.u())
    for got, want in zip(runs[0].invariants(), refs):
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    s1, s2, s3 = runs[0].species()
    lhs, rhs = s2 * s3, ksp * s1
    assert np.all(np.abs(lhs - rhs) <= 1e-14 * np.maximum(lhs, rhs) + 1e-300)
    for r in runs:
        r.close()
