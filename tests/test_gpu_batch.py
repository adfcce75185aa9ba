"""Batches of lattices advanced together (one persistent step launch over
every member's tiles, one dissolution launch, replayed from a CUDA graph):
each member against its own oracle run, independence of the tile shape, and
the autotuner leaving the state where it found it."""
import numpy as np
import pytest

from paper_1601_02708_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {64: 1e-12, 32: 1e-5}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02708_gb300 import build
    build.build()
    import paper_1601_02708_gb300 as pkg
    return torch, pkg


def _members(pkg, stream, prec, cases):
    keys = ("edges", "solid", "vel", "u0", "react_mode", "k", "dissolution", "mineral")
    return [pkg.LBM(c["nx"], c["ny"], c["tau"], precision=prec, stream=stream,
                    **{k: c[k] for k in keys}) for c in cases]


def _small_cases():
    cases = inputs.batch_cases(n_inst=6, seed=11, smin=20, smax=140, k=0.05, rmin=2, rmax=6)
    for c in cases:
        c["mineral"] = np.full((c["ny"], c["nx"]), 0.05)
    return cases


@pytest.mark.parametrize("prec,dissolution", [(64, True), (32, False)])
def test_members_match_the_oracle(env, oracle_mod, prec, dissolution):
    """FP64 with dissolution (exact masks through many flips); FP32 without
    (an FP32 flip can land one step from the FP64 one, so FP32 dissolution
    is checked against individually stepped contexts below)."""
    torch, pkg = env
    s = torch.cuda.Stream()
    cases = _small_cases()
    for c in cases:
        c["dissolution"] = dissolution
    members = _members(pkg, s.cuda_stream, prec, cases)
    batch = pkg.LBMBatch(members)
    ud = [c["u_dir"] for c in cases]
    q = [c["q_neu"] for c in cases]
    keys = ("edges", "solid", "vel", "u0", "react_mode", "k", "dissolution", "mineral")
    refs = [oracle_mod.LBMOracle(c["nx"], c["ny"], c["tau"], **{k: c[k] for k in keys})
            for c in cases]
    for n in (1, 40, 59):  # odd counts exercise both buffer parities
        batch.substeps(n, 1, ud, ud, q)
        for r, c in zip(refs, cases):
            r.substeps(n, 1, c["u_dir"], c["u_dir"], c["q_neu"])
    flips = 0
    for m, r in zip(members, refs):
        u, ur = m.concentration(), r.u()
        assert np.abs(u - ur).max() <= TOL[prec] * np.abs(ur).max()
        assert np.array_equal(m.solid(), r.solid())
        d = m.diagnostics()
        assert d["steps"] == 100
        assert abs(d["mass"] - r.diag()["mass"]) <= TOL[prec] * r.diag()["mass"]
        flips += r.diag()["flips"]
    assert flips > 0 or not dissolution


def _same_diag(x, y):
    dx, dy = x.diagnostics(), y.diagnostics()
    mass_x, mass_y = dx.pop("mass"), dy.pop("mass")
    assert dx == dy
    # the mass sum folds per-tile partials, whose grouping follows the tiling
    assert abs(mass_x - mass_y) <= 1e-13 * abs(mass_y)


@pytest.mark.parametrize("prec,shape", [(64, 0), (64, 4), (32, 0), (32, 5), (32, 6)])
def test_batch_equals_members_stepped_alone(env, prec, shape):
    """A batch gives bit-identical states to the same contexts stepped one
    by one with the kernel of the same kind (one thread per node for the
    plain shapes, the TMA pipeline for the pipelined one), with dissolution,
    over calls of several lengths (both buffer parities)."""
    torch, pkg = env
    s = torch.cuda.Stream()
    cases = _small_cases()
    a = _members(pkg, s.cuda_stream, prec, cases)
    b = _members(pkg, s.cuda_stream, prec, cases)
    pipelined = pkg.LBMBatch.shapes()[shape][3]
    for m in b:
        m.set_kernel("tma" if pipelined else "generic")
    batch = pkg.LBMBatch(a)
    batch.set_shape(shape)
    ud = [c["u_dir"] for c in cases]
    for n in (1, 40, 59):
        batch.substeps(n, 1, ud, ud)
        for m, c in zip(b, cases):
            m.substeps(n, 1, c["u_dir"], c["u_dir"])
    for x, y in zip(a, b):
        assert np.array_equal(x.concentration(), y.concentration())
        assert np.array_equal(x.solid(), y.solid())
        assert np.array_equal(x.mineral(), y.mineral())
        _same_diag(x, y)


def test_shapes_agree_and_autotune_restores_state(env):
    torch, pkg = env
    s = torch.cuda.Stream()
    cases = inputs.batch_cases(n_inst=5, seed=5, smin=64, smax=300)
    ud = [c["u_dir"] for c in cases]
    shapes = pkg.LBMBatch.shapes()
    assert shapes[-1] == (96, 8, 832, True)
    results = []
    for shape in range(len(shapes)):
        members = _members(pkg, s.cuda_stream, 32, cases)
        batch = pkg.LBMBatch(members)
        batch.set_shape(shape)
        batch.substeps(30, 1, ud, ud)
        results.append([m.concentration() for m in members])
    for shape, other in enumerate(results[1:], start=1):
        for a, b in zip(results[0], other):
            if shapes[shape][3]:  # another kernel: same arithmetic, own compilation
                assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max()
            else:
                assert np.array_equal(a, b)
    members = _members(pkg, s.cuda_stream, 32, cases)
    batch = pkg.LBMBatch(members)
    assert batch.shape == len(shapes) - 1  # the pipelined shape by default in FP32
    batch.substeps(10, 1, ud, ud)
    before = [m.concentration() for m in members]
    times = batch.autotune(trial_steps=5, repeats=1)
    assert len(times) == len(shapes) and batch.shape in times
    after = [m.concentration() for m in members]
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    batch.substeps(5, 1, ud, ud)
    assert members[0].diagnostics()["steps"] == 15


def test_batch_argument_errors(env):
    torch, pkg = env
    a = pkg.LBM(16, 16, 0.8, precision=32)  # legacy default stream
    with pytest.raises(pkg.LBMError):
        pkg.LBMBatch([a])
    s = torch.cuda.Stream()
    b = pkg.LBM(16, 16, 0.8, precision=32, stream=s.cuda_stream)
    c = pkg.LBM(16, 16, 0.8, precision=64, stream=s.cuda_stream)
    with pytest.raises(pkg.LBMError):
        pkg.LBMBatch([b, c])  # mixed precision
    with pytest.raises(pkg.LBMError):
        pkg.LBMBatch([b, b])
    d = pkg.LBM(16, 16, 0.8, precision=64, stream=s.cuda_stream)
    bd = pkg.LBMBatch([c, d])
    assert bd.shape == 0
    with pytest.raises(pkg.LBMError):
        bd.set_shape(len(pkg.LBMBatch.shapes()) - 1)  # the pipeline is FP32 only
    with pytest.raises(pkg.LBMError):
        bd.set_shape(len(pkg.LBMBatch.shapes()))
