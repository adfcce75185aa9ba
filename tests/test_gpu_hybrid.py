"""The library's Q1 continuum solver and the hybrid driver (Algorithm 1)
against the oracle's: the continuum alone (Galerkin and SUPG, a hole,
Dirichlet data that change every step, the element interpolant), the plain
hybrid at full size (40 x 10 elements coupled to a 256 x 64 lattice, 100
coarse steps of 3 Schwarz iterations and 10 substeps), the pore-block hybrid
on a small mesh, and one coarse step of the pore-block hybrid at full size
(400 x 100 elements around a 2048 x 2048 lattice)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02708_gb300 import build
    build.build()
    import paper_1601_02708_gb300 as p
    return p


def _oracle_run(layout, n_coarse):
    from oracle import LBMOracle
    from oracle.fem import Q1FEM, schwarz_step
    lbm = LBMOracle(**layout["lbm"])
    fem = Q1FEM(**layout["fem"])
    s0, s1 = layout["lbm_slots"]
    for _ in range(n_coarse):
        schwarz_step(fem, lbm, layout["eta"], layout["max_iter"], layout["fixed_values"],
                     layout["gamma_lattice_xy"], layout["lbm_points"], np.arange(s0, s1),
                     layout["q_neu"])
    return fem, lbm


# 38 x 12 nodes are solved by one block, 98 x 54 (above 4096 nodes) by the
# cooperative launch over several blocks
@pytest.mark.parametrize("nex,ney", [(37, 11), (97, 53)])
@pytest.mark.parametrize("supg,hole", [(True, False), (False, True)])
def test_fem_matches_oracle(pkg, oracle_mod, supg, hole, nex, ney):
    from oracle.fem import Q1FEM
    from paper_1601_02708_gb300.fem import FEM
    rng = np.random.default_rng(7)
    act = None
    if hole:
        act = np.ones((ney, nex), np.uint8)
        act[3:8, 10:20] = 0
    nxn = nex + 1
    dirichlet = [j * nxn for j in range(ney + 1)] + [3 * nxn + 25, 9 * nxn + 30]
    kw = dict(nex=nex, ney=ney, x0=-0.3, y0=0.2, hx=0.02, hy=0.03, D=1e-3,
              v=(0.4, -0.15) if supg else (0.0, 0.0), theta=0.5, dt=0.01, supg=supg,
              elem_active=act, dirichlet=dirichlet, d0=rng.uniform(0, 1, nxn * (ney + 1)))
    g = FEM(**kw)
    o = Q1FEM(**kw)
    for step in range(15):
        vals = rng.uniform(0, 2, len(dirichlet))
        g.step(vals)
        o.step(vals)
    d = g.get()
    assert np.abs(d - o.d).max() <= 1e-10 * np.abs(o.d).max()
    it, res = g.solver_info()
    assert 0 < it < 1000 and res <= 1e-12
    pts = np.stack([rng.uniform(-0.3, 0.44, 40), rng.uniform(0.2, 0.53, 40)], 1)
    assert np.abs(g.interpolate(pts) - o.interpolate(pts)).max() <= 1e-10


@pytest.mark.parametrize("nex,ney", [(37, 11), (97, 53)])
def test_fem_reports_a_solve_cut_short(pkg, nex, ney):
    """Both solve paths (one block up to 2048 nodes, the cooperative launch
    above) report a solve stopped by max_iter before the tolerance as an
    error, with the iterations it ran; the same system then converges with
    the default limit."""
    from paper_1601_02708_gb300.fem import FEM
    rng = np.random.default_rng(3)
    nxn = nex + 1
    kw = dict(nex=nex, ney=ney, x0=0.0, y0=0.0, hx=0.02, hy=0.03, D=1e-3, v=(0.4, -0.15),
              theta=0.5, dt=0.01, supg=True, dirichlet=[j * nxn for j in range(ney + 1)],
              d0=rng.uniform(0, 1, nxn * (ney + 1)), tol=1e-14)
    vals = rng.uniform(0, 2, ney + 1)
    cut = FEM(max_iter=1, **kw)
    with pytest.raises(pkg.LBMError):
        cut.step(vals)
    assert cut.solver_info()[0] == 1
    full = FEM(**kw)
    full.step(vals)
    it, res = full.solver_info()
    assert 1 < it < 1000 and res <= 1e-14
    cut.close()
    full.close()


def test_fem_rejects_bad_input(pkg):
    from paper_1601_02708_gb300.fem import FEM
    with pytest.raises(pkg.LBMError):
        FEM(4, 4, 0, 0, 0.1, 0.1, D=1.0, dirichlet=[0, 0])   # repeated node
    with pytest.raises(pkg.LBMError):
        FEM(4, 4, 0, 0, 0.1, 0.1, D=1.0, dirichlet=[25])      # out of range
    with pytest.raises(pkg.LBMError):
        FEM(4, 4, 0, 0, -0.1, 0.1, D=1.0)                     # bad spacing


@pytest.mark.parametrize("prec", [64, 32])
def test_plain_hybrid_full_size(pkg, oracle_mod, prec):
    from paper_1601_02708_gb300 import inputs
    from paper_1601_02708_gb300.hybrid import Hybrid
    layout = inputs.hybrid_plain_layout()
    run = Hybrid(layout, precision=prec)
    run.run()
    fem, lbm = _oracle_run(layout, layout["n_coarse"])
    tol = 1e-9 if prec == 64 else 1e-5
    d = run.continuum()
    assert np.abs(d - fem.d).max() <= tol * np.abs(fem.d).max()
    u = run.lbm.concentration()
    assert np.abs(u - lbm.u()).max() <= tol * np.abs(fem.d).max()
    assert run.lbm.diagnostics()["steps"] == 100 * 3 * 10 - 100 * 2 * 10  # rollbacks
    assert lbm.u().max() > 1e-6  # the pulse has entered the lattice


@pytest.mark.parametrize("prec,k", [(64, 5e-3), (32, 5e-4)])
def test_block_hybrid_small(pkg, oracle_mod, prec, k):
    """FP64 with a rate that dissolves dozens of nodes (exact masks); FP32
    with the configuration's rate, under which no node flips in these steps
    (an FP32 flip can land one step from the FP64 one)."""
    from paper_1601_02708_gb300 import inputs
    from paper_1601_02708_gb300.hybrid import Hybrid
    layout = inputs.hybrid_block_layout(nex=40, ney=10, hole=(17, 23, 2, 8), n_f=96,
                                        k=k, eta=20, max_iter=3, n_coarse=4,
                                        rmin=3, rmax=8)
    run = Hybrid(layout, precision=prec)
    run.run()
    fem, lbm = _oracle_run(layout, 4)
    tol = 1e-9 if prec == 64 else 1e-5
    assert np.abs(run.continuum() - fem.d).max() <= tol
    u = run.lbm.concentration()
    assert np.abs(u - lbm.u()).max() <= tol
    assert np.array_equal(run.lbm.solid(), lbm.solid())
    fluid = lbm.solid() == 0
    assert u[fluid].min() < 0.99  # the surface reaction has drawn the block down
    if prec == 64:
        assert lbm.diag()["flips"] > 0


def test_block_hybrid_full_size_one_coarse_step(pkg, oracle_mod):
    """400 x 100 elements around a 2048 x 2048 lattice: one coarse step
    (5 Schwarz iterations of 50 substeps) against the oracle, FP32 lattice."""
    from paper_1601_02708_gb300 import inputs
    from paper_1601_02708_gb300.hybrid import Hybrid
    layout = inputs.hybrid_block_layout(n_coarse=1)
    run = Hybrid(layout, precision=32)
    run.run()
    fem, lbm = _oracle_run(layout, 1)
    assert np.abs(run.continuum() - fem.d).max() <= 1e-5
    u = run.lbm.concentration()
    assert np.abs(u - lbm.u()).max() <= 1e-5


def _gaussian_layout(level=1, T=0.02, D=0.05):
    """Pure diffusion of a Gaussian centred in the overlap (the oracle's
    transient coupling pin), as a layout for the library's driver."""
    import math
    nfx, ny_f, eta, tau = 32 * 2 ** level, 4, 4, 1.0
    h = 0.5 / nfx
    dt_f = (tau - 0.5) / 3.0 * h * h / D
    nex = 12 * 2 ** level
    hx = 0.6 / nex
    x0, s0 = 0.55, 0.03 ** 2

    def exact(x, t):
        return math.sqrt(s0 / (s0 + 2 * D * t)) * np.exp(-(x - x0) ** 2 / (2 * (s0 + 2 * D * t)))

    xl = 0.5 + np.arange(nfx + 1) * h
    nxn = nex + 1
    xf = (np.arange(2 * nxn) % nxn) * hx
    ncoarse = int(round(T / (eta * dt_f)))
    layout = dict(
        lbm=dict(nx=nfx + 1, ny=ny_f, tau=tau, edges=(1, 2, 0, 0),
                 u0=np.tile(exact(xl, 0), (ny_f, 1))),
        fem=dict(nex=nex, ney=1, x0=0.0, y0=0.0, hx=hx, hy=ny_f * h, D=D, v=(0.0, 0.0),
                 theta=0.5, dt=eta * dt_f, supg=False, elem_active=None,
                 dirichlet=[0, nxn, nex, nxn + nex], d0=exact(xf, 0)),
        fixed_values=np.zeros(2), gamma_lattice_xy=np.array([[(0.6 - 0.5) / h, 0.0]] * 2),
        lbm_points=np.array([[0.5, y * h] for y in range(ny_f)]), lbm_slots=(0, ny_f),
        q_neu=None, eta=eta, max_iter=3, n_coarse=ncoarse, h=h)
    return layout, exact, xl, xf[:nxn], ncoarse * eta * dt_f


@pytest.mark.parametrize("prec", [64, 32])
def test_coupled_gaussian_against_oracle_and_exact(pkg, oracle_mod, prec):
    from paper_1601_02708_gb300.hybrid import Hybrid
    layout, exact, xl, xf, t = _gaussian_layout()
    run = Hybrid(layout, precision=prec)
    run.run()
    fem, lbm = _oracle_run(layout, layout["n_coarse"])
    tol = 1e-9 if prec == 64 else 1e-5
    d = run.continuum()
    u = run.lbm.concentration()
    assert np.abs(d - fem.d).max() <= tol
    assert np.abs(u - lbm.u()).max() <= tol
    nxn = len(xf)
    assert np.abs(d[:nxn] - exact(xf, t)).max() <= 1.2e-2   # level-1 errors of the pin
    assert np.abs(u[0] - exact(xl, t)).max() <= 3.5e-3


@pytest.mark.parametrize("prec,k", [(64, 5e-2), (32, 5e-4)])
def test_many_blocks_in_one_continuum(pkg, oracle_mod, prec, k):
    """Algorithm 2 with one continuum and two pore blocks of different
    spacing, stepped together as a batch, against the oracle's
    many-subdomain step."""
    from oracle import LBMOracle
    from oracle.fem import Q1FEM, schwarz_step_many
    from paper_1601_02708_gb300 import inputs
    from paper_1601_02708_gb300.hybrid import Hybrid
    layout = inputs.hybrid_multiblock_layout(nex=40, ney=10, holes=((5, 9, 2, 6), (20, 26, 3, 7)),
                                             n_f=(64, 72), k=k, eta=10, max_iter=3,
                                             n_coarse=3, rmin=2, rmax=5)
    run = Hybrid(layout, precision=prec)
    run.run()
    fem = Q1FEM(**layout["fem"])
    lbms = [LBMOracle(**a) for a in layout["lbms"]]
    slots = [np.arange(a, b) for a, b in layout["lbm_slots"]]
    for _ in range(3):
        schwarz_step_many(fem, lbms, layout["eta"], layout["max_iter"], layout["fixed_values"],
                          layout["gamma_lattice_xy"], layout["lbm_points"], slots)
    tol = 1e-9 if prec == 64 else 1e-5
    assert np.abs(run.continuum() - fem.d).max() <= tol
    flips = 0
    for lat, ref in zip(run.lbms, lbms):
        assert np.abs(lat.concentration() - ref.u()).max() <= tol
        assert np.array_equal(lat.solid(), ref.solid())
        flips += ref.diag()["flips"]
    assert flips > 0 or prec == 32
    assert fem.d[fem.free].min() < 1.0 - 1e-9  # the blocks draw the continuum down
