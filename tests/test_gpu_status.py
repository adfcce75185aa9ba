"""Status codes and read-outs of the C ABI: the infeasible-data warning, the
diagnostics fields (outlet flux, smallest population, Newton failures)
against the oracle, the per-side gradient of lbm_adjoint, and the refusal
of a batch whose members' buffers went out of step."""
import math

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


def test_infeasible_dirichlet_data_warn_once(gb, oracle_mod):
    """Sec. 4.1.1 (a): zero Dirichlet data beside positive known
    populations have no non-negative solution; they are applied literally,
    counted like the oracle counts them, and reported once as
    LBM_WARN_BC_INFEASIBLE (status 1) by the next call that waits."""
    n = 26
    X, Y = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n))
    u0 = np.sin(math.pi * Y) * np.cos(math.pi * X / 2)
    lat = gb.LBM(n, n, 1.0, edges=(2, 1, 1, 1), precision=64, u0=u0)
    ref = oracle_mod.LBMOracle(n, n, 1.0, edges=(2, 1, 1, 1), u0=u0)
    lat.substeps(20)
    ref.substeps(20)
    assert lat.synchronize() == 1
    assert lat.synchronize() == 0  # nothing new since the last report
    d = lat.diagnostics()
    assert d["bc_infeasible"] == ref.diag()["bc_infeasible"] > 0
    lat.substeps(3)
    st = lat._lib.lbm_synchronize(lat.handle)
    assert st == 1 and b"no non-negative" in lat._lib.lbm_last_error()


@pytest.mark.parametrize("prec", [64, 32])
def test_diagnostics_fields_against_oracle(gb, oracle_mod, prec):
    """outlet_flux is the first moment sum_i f_i e_ix over the east-edge
    fluid nodes after the boundary conditions of the last step; min_f the
    smallest stored population; newton_fail stays 0 with FP64 wall solves."""
    nx, ny, steps = 90, 52, 120
    solid = inputs.disk_packing(nx, ny, 0.7, 8, rmin=3, rmax=6)
    vel = inputs.streamfunction_velocity(nx, ny, 9, solid=solid)
    vel[0][solid == 0] += 0.03
    kw = dict(edges=(1, 1, 0, 0), solid=solid, vel=vel, u0=np.zeros((ny, nx)),
              react_mode=1, k=2e-3)
    ud = inputs.edge_array(nx, ny, W=1.0, E=0.25)
    ref = oracle_mod.LBMOracle(nx, ny, 0.8, walls="maxent", **kw)
    lat = gb.LBM(nx, ny, 0.8, precision=prec, walls="maxent", **kw)
    ref.substeps(steps, 1, ud, ud)
    lat.substeps(steps, 1, ud, ud)
    f = ref.f()  # state after the boundary conditions
    east = solid[:, -1] == 0
    qx = (f[1] + f[5] + f[8] - f[3] - f[6] - f[7])[:, -1]
    want = qx[east].sum()
    d = lat.diagnostics()
    tol = 1e-12 if prec == 64 else 1e-5
    scale = np.abs(f[:, :, -1]).sum()
    assert abs(d["outlet_flux"] - want) <= tol * scale
    assert d["min_f"] == lat.min_population()
    assert d["newton_fail"] == 0 and ref.diag()["newton_fail"] == 0


def test_adjoint_side_gradient(gb):
    """grad_side of lbm_adjoint: dJ/d(one value held on a whole Dirichlet
    side) is the sum of that side's start and end gradients, zero for a
    side that is not Dirichlet, and J's homogeneity in the inlet value
    (c0 = 0, zero-flux outlet) makes it J / c_in."""
    nx, ny = 80, 40
    solid = inputs.disk_packing(nx, ny, 0.75, 4, rmin=2, rmax=5)
    vel = inputs.streamfunction_velocity(nx, ny, 5, umax=0.04, solid=solid)
    vel[0][solid == 0] += 0.1
    kf = 1e-3 * np.ones((ny, nx))
    lat = gb.LBM(nx, ny, 0.8, edges=(1, 2, 0, 0), precision=64, solid=solid, vel=vel,
                 react_mode=2, k_field=kf)
    ud = inputs.edge_array(nx, ny, W=0.7)
    r = lat.adjoint(400, 1, ud, ud, None)
    want = r["ua"][:ny].sum() + r["ub"][:ny].sum()
    assert r["side"][0] == pytest.approx(want, rel=1e-13)
    assert r["side"][1] == 0.0 and r["side"][2] == 0.0 and r["side"][3] == 0.0
    assert r["J"] > 0 and r["side"][0] == pytest.approx(r["J"] / 0.7, rel=1e-10)


def test_batch_refuses_members_out_of_step(gb):
    """A member stepped on its own by an odd number of steps no longer
    matches the buffer parity the batch's graphs were recorded with: the
    batch refuses to run (LBM_ERR_STATE) instead of reading the wrong
    buffer."""
    import torch
    s = torch.cuda.Stream()
    members = [gb.LBM(40, 24, 0.8, precision=32, stream=s.cuda_stream,
                      u0=np.ones((24, 40))) for _ in range(2)]
    batch = gb.LBMBatch(members)
    batch.substeps(2)
    members[1].substeps(1)
    with pytest.raises(gb.LBMError) as e:
        batch.substeps(2)
    assert e.value.status == -5
    members[0].substeps(1)  # back in step
    batch.substeps(2)
    batch.close()


def test_status_numbering(gb):
    with pytest.raises(gb.LBMError) as e:
        gb.LBM(8, 8, 0.5)
    assert e.value.status == -1
    lat = gb.LBM(8, 8, 0.8, precision=32)
    lat.close()
    with pytest.raises(gb.LBMError) as e:
        lat.substeps(1)
    assert e.value.status == -5
    with pytest.raises(gb.LBMError) as e:
        gb.LBM(8, 8, 0.8, precision=32).flip_steps()  # no dissolution
    assert e.value.status == -5


def test_kernel_choice(gb):
    """LBM_KERNEL_AUTO: the tile pipeline below 8 M nodes or with
    maximum-entropy walls, the plain kernel for larger bounce-back lattices;
    an explicit choice survives a change of wall treatment; FP64 runs the
    plain kernel."""
    small = gb.LBM(64, 64, 0.8)
    assert small.kernel() == "tma"
    big = gb.LBM(2900, 2900, 0.8)  # 8.4 M nodes
    assert big.kernel() == "generic"
    big.set_walls("maxent_lattice")
    assert big.kernel() == "tma"
    big.set_walls("bounce")
    assert big.kernel() == "generic"
    big.set_kernel("tma")
    big.set_walls("maxent")
    big.set_walls("bounce")
    assert big.kernel() == "tma"
    big.set_kernel("auto")
    assert big.kernel() == "generic"
    assert gb.LBM(64, 64, 0.8, precision=64).kernel() == "generic"
    small.close()
    big.close()
