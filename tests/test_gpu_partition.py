"""One lattice split into row slabs (lbm_init_slab, the halo exchange of
lbm_halo_pack / lbm_halo_unpack between the two halves of each step) on one
GPU, against the same lattice unsplit: bit for bit in FP64 and FP32 --
concentration, stored populations, solid mask, mineral and flip record --
with dissolution flipping nodes next to the cuts, periodic and
non-periodic y, Dirichlet corners, maximum-entropy walls, several calls with
time-interpolated edge data, and ragged slab heights."""
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


def _case(nx, ny, seed, edges, walls="bounce"):
    solid = inputs.disk_packing(nx, ny, 0.6, seed, rmin=3, rmax=9)
    vel = inputs.streamfunction_velocity(nx, ny, seed + 1, solid=solid)
    return dict(edges=edges, solid=solid, vel=vel, u0=np.where(solid != 0, 0.0, 0.3), react_mode=1,
                k=0.05, dissolution=True, mineral=np.full((ny, nx), 0.03), walls=walls)


def _run_both(gb, nx, ny, parts, prec, kw, calls, eta):
    from paper_1601_02708_gb300.partition import SlabLattice
    whole = gb.LBM(nx, ny, 0.7, precision=prec, **kw)
    split = SlabLattice(nx, ny, 0.7, parts=parts, precision=prec, **kw)
    rng = np.random.default_rng(nx + ny + parts)
    ne = 2 * (nx + ny)
    ua = rng.uniform(0.5, 1.5, ne)
    for _ in range(calls):
        ub = rng.uniform(0.5, 1.5, ne)
        whole.substeps(eta, eta, ua, ub)
        split.substeps(eta, eta, ua, ub)
        ua = ub
    return whole, split


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("parts,edges", [(2, (1, 2, 0, 0)), (3, (1, 2, 0, 0)),
                                         (4, (1, 2, 1, 2)), (3, (0, 0, 1, 1))])
def test_split_lattice_is_bit_identical(gb, prec, parts, edges):
    nx, ny = 211, 157  # ragged: several tiles, slab heights that differ
    from paper_1601_02708_gb300.partition import slab_bounds
    kw = _case(nx, ny, 17 * parts + edges[2], edges)
    for y0, _ in slab_bounds(ny, parts):  # little mineral on both sides of every cut
        for y in (y0 - 2, y0 - 1, y0, y0 + 1):
            kw["mineral"][y % ny] = 0.002
    whole, split = _run_both(gb, nx, ny, parts, prec, kw, calls=6, eta=25)
    assert np.array_equal(split.concentration(), whole.concentration())
    assert np.array_equal(split.populations(), whole.populations())
    assert np.array_equal(split.solid(), whole.solid())
    assert np.array_equal(split.mineral(), whole.mineral())
    assert np.array_equal(split.flip_steps(), whole.flip_steps())
    d, dw = split.diagnostics(), whole.diagnostics()
    assert d["flips"] == dw["flips"] > 0  # nodes flipped, some next to the cuts
    assert d["steps"] == dw["steps"] == 150
    assert abs(d["mass"] - dw["mass"]) <= 1e-12 * dw["mass"]
    assert abs(d["outlet_J"] - dw["outlet_J"]) <= 1e-12 * max(dw["outlet_J"], 1.0)
    # flips next to a cut: the exchange of flags and shares was exercised
    fs = whole.flip_steps()
    cuts = [y0 for y0, _ in split.bounds[1:]]
    near = np.zeros(ny, bool)
    for y in cuts:
        near[max(0, y - 1):y + 1] = True
    assert (fs[near] >= 0).any()
    split.close()
    whole.close()


def test_split_with_maxent_walls(gb):
    nx, ny = 160, 96
    kw = _case(nx, ny, 5, (1, 2, 0, 0), walls="maxent")
    kw["dissolution"] = False
    kw.pop("mineral")
    whole, split = _run_both(gb, nx, ny, 3, 32, kw, calls=4, eta=20)
    assert np.array_equal(split.concentration(), whole.concentration())
    assert np.array_equal(split.populations(), whole.populations())


def test_slab_refusals(gb):
    from paper_1601_02708_gb300.partition import Slab
    import torch
    s = Slab(40, 30, 0.8, 10, 20, precision=32)
    with pytest.raises(gb.LBMError):  # a slab steps with its halo exchange
        s.substeps(1)
    buf = torch.empty(s.halo_bytes(0), dtype=torch.uint8, device="cuda")
    with pytest.raises(gb.LBMError):  # W is not a shared side
        gb._lib.check(s._lib.lbm_halo_pack(s.handle, 0, 0, buf.data_ptr()))
    host = np.zeros(s.halo_bytes(0), dtype=np.uint8)
    with pytest.raises(gb.LBMError):  # message buffers are device memory
        gb._lib.check(s._lib.lbm_halo_pack(s.handle, 2, 0, host.ctypes.data))
    with pytest.raises(gb.LBMError):
        Slab(40, 30, 0.8, 25, 26, precision=32)  # one row
