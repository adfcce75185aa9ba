"""Pore walls of the maximum-entropy kind (zero flux, Sec. 4.1.1 (b)) through
the C ABI against the FP64 oracle, element by element: both FP32 step
kernels and FP64, ragged shapes, with and without dissolution, batch
members, and the refusals.  Tolerances as in test_gpu_parity: FP64 1e-12,
FP32 1e-5 relative to max|u|; masks bit for bit."""
import numpy as np
import pytest

from paper_1601_02708_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}


@pytest.fixture(scope="module")
def gb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02708_gb300 import build
    build.build()
    import paper_1601_02708_gb300 as pkg
    return pkg


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _case(nx, ny, seed, dissolution, k=0.05, mineral=0.03):
    solid = inputs.disk_packing(nx, ny, 0.6, seed, rmin=2, rmax=7)
    vel = inputs.streamfunction_velocity(nx, ny, seed + 1, solid=solid)
    kw = dict(edges=(1, 2, 0, 0), solid=solid, vel=vel, u0=np.zeros((ny, nx)))
    if dissolution:
        kw.update(react_mode=1, k=k, dissolution=True, mineral=np.full((ny, nx), mineral))
    return kw


@pytest.mark.parametrize("prec,kernel", [(64, "auto"), (32, "tma"), (32, "generic")])
@pytest.mark.parametrize("shape,dissolution", [((97, 61), False), ((300, 37), True),
                                               ((33, 9), True)])
def test_maxent_walls_match_oracle(gb, oracle_mod, prec, kernel, shape, dissolution):
    """Dirichlet inlet, Neumann outlet, periodic y: interior wall nodes take
    the maximum-entropy solve, wall nodes on the open sides bounce-back."""
    nx, ny = shape
    steps = 120
    kw = _case(nx, ny, nx * 5 + ny, dissolution)
    ud = inputs.edge_array(nx, ny, W=1.0)
    ref = oracle_mod.LBMOracle(nx, ny, 0.7, walls="maxent", **kw)
    ref.substeps(steps, 1, ud, ud)
    lat = gb.LBM(nx, ny, 0.7, precision=prec, walls="maxent", **kw)
    lat.set_kernel(kernel)
    lat.substeps(steps, 1, ud, ud)
    assert _relerr(lat.concentration(), ref.u()) <= TOL[prec]
    assert _relerr(lat.populations(), ref.fpost()) <= TOL[prec]
    assert np.array_equal(lat.solid(), ref.solid())
    d, dr = lat.diagnostics(), ref.diag()
    assert abs(d["mass"] - dr["mass"]) <= TOL[prec] * dr["mass"]
    if prec == 64:
        assert d["bc_infeasible"] == dr["bc_infeasible"]
    # the walls change the answer: the bounce-back run differs
    bb = oracle_mod.LBMOracle(nx, ny, 0.7, **kw)
    bb.substeps(steps, 1, ud, ud)
    assert _relerr(ref.u(), bb.u()) > 1e-4
    ref.substeps(1, 1, ud, ud)  # the library decides a flip one step ahead
    if dissolution and shape == (300, 37):
        assert ref.diag()["flips"] > 0
    assert d["flips"] == ref.diag()["flips"]


def test_batch_members_with_either_wall(gb, oracle_mod):
    """A batch whose members use bounce-back and maximum-entropy walls."""
    import torch
    s = torch.cuda.Stream()
    cases = inputs.batch_cases(n_inst=4, seed=9, smin=40, smax=160)
    keys = ("edges", "solid", "vel", "u0", "react_mode", "k", "dissolution", "mineral")
    walls = ["maxent", "bounce", "maxent", "maxent"]
    mem = [gb.LBM(c["nx"], c["ny"], c["tau"], precision=32, stream=s.cuda_stream,
                  walls=w, **{k: c[k] for k in keys}) for c, w in zip(cases, walls)]
    b = gb.LBMBatch(mem)
    ud = [c["u_dir"] for c in cases]
    b.substeps(60, 1, ud, ud)
    for c, w, m in zip(cases, walls, mem):
        ref = oracle_mod.LBMOracle(c["nx"], c["ny"], c["tau"], walls=w,
                                   **{k: c[k] for k in keys})
        ref.substeps(60, 1, c["u_dir"], c["u_dir"])
        assert _relerr(m.concentration(), ref.u()) <= TOL[32]
        assert np.array_equal(m.solid(), ref.solid())


def test_refusals(gb):
    nx, ny = 40, 24
    kw = _case(nx, ny, 3, False)
    lat = gb.LBM(nx, ny, 0.8, precision=64, walls="maxent", **kw)
    ud = inputs.edge_array(nx, ny, W=1.0)
    with pytest.raises(gb.LBMError):  # the adjoint covers bounce-back walls only
        lat.adjoint(10, 1, ud, ud)
    with pytest.raises(gb.LBMError):  # an unknown mode
        gb._lib.check(lat._lib.lbm_set_wall_mode(lat.handle, 7))
    lat.set_walls("bounce")
    lat.adjoint(10, 1, ud, ud)  # bounce-back again: the adjoint runs
