"""The instantaneous bimolecular reaction (Sec. 7.2) on the GPU against the
oracle: the species step of the library bit for bit (host arrays and device
tensors), and two transported invariants with their species on a porous
lattice (FP64 1e-12, FP32 1e-5 relative to the largest value)."""
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


@pytest.mark.parametrize("coeffs", [(1.0, 2.0, 1.0), (2.0, 3.0, 5.0)])
def test_species_step_is_exact(gb, coeffs):
    import torch
    from oracle import chemistry
    rng = np.random.default_rng(7)
    alpha, beta = rng.uniform(0, 1, (2, 37, 53))
    want = chemistry.species(alpha, beta, *coeffs)
    got = gb.species_from_invariants(alpha, beta, coeffs)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    dev = [torch.from_numpy(x).cuda() for x in (alpha, beta)]
    got_dev = gb.species_from_invariants(dev[0], dev[1], coeffs)
    torch.cuda.synchronize()
    for g, w in zip(got_dev, want):
        assert g.is_cuda and np.array_equal(g.cpu().numpy(), w)
    inv = gb.invariants_from_species(*want, coeffs)
    for g, w in zip(inv, chemistry.invariants(*want, *coeffs)):
        assert np.array_equal(g, w)


def test_species_step_refuses_bad_input(gb):
    a = np.ones(4)
    with pytest.raises(gb.LBMError):
        gb.species_from_invariants(a, a, (1.0, 0.0, 1.0))
    with pytest.raises(gb.LBMError):
        gb.species_from_invariants(a, a, (1.0, float("nan"), 1.0))
    empty = np.zeros(0)
    assert all(x.size == 0 for x in gb.species_from_invariants(empty, empty, (1, 2, 1)))


@pytest.mark.parametrize("prec", [64, 32])
def test_transported_invariants_and_species(gb, oracle_mod, prec):
    """A and B released on either side of a pore space (bounce-back walls,
    zero-flux sides, a stream-function flow): both invariants against two
    oracle lattices, then the species."""
    from oracle import chemistry
    nx, ny, tau, steps = 96, 64, 0.8, 150
    coeffs = (1.0, 2.0, 1.0)
    solid = inputs.disk_packing(nx, ny, 0.7, 31, rmin=3, rmax=7)
    vel = inputs.streamfunction_velocity(nx, ny, 32, solid=solid)
    X = np.arange(nx)[None, :].repeat(ny, 0)
    uA0 = np.where(solid != 0, 0.0, np.exp(-((X - 0.3 * nx) / 12.0) ** 2))
    uB0 = np.where(solid != 0, 0.0, 0.5 * np.exp(-((X - 0.7 * nx) / 12.0) ** 2))
    edges = (2, 2, 0, 0)
    bm = gb.Bimolecular(nx, ny, tau, coeffs, uA0, uB0, precision=prec, edges=edges,
                        solid=solid, vel=vel)
    bm.substeps(steps)
    a0, b0 = chemistry.invariants(uA0, uB0, np.zeros_like(uA0), *coeffs)
    refs = []
    for u0 in (a0, b0):
        r = oracle_mod.LBMOracle(nx, ny, tau, edges=edges, solid=solid, vel=vel, u0=u0)
        r.substeps(steps)
        refs.append(r.u())
    tol = 1e-12 if prec == 64 else 1e-5
    for got, ref in zip(bm.invariants(), refs):
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    want = chemistry.species(refs[0], refs[1], *coeffs)
    scale = max(np.abs(w).max() for w in want)
    for got, w in zip(bm.species(), want):
        assert np.abs(got - w).max() <= 2 * tol * scale
    uA, uB, uC = bm.species()
    assert uC.max() > 1e-3  # the fronts have met and reacted
    assert np.abs(np.minimum(uA, uB)).max() <= 2 * tol * scale
    bm.close()
