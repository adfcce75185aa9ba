"""The calcite equilibrium read-out (Sec. 7.4, lbm_calcite_species /
lbm_calcite_invariants) on the GPU against the oracle.

The oracle evaluates the printed root in exact rational arithmetic and
rounds once, so it is the root to half an ulp.  The library evaluates the same root in
FP64 in a form without cancellation (2 K_sp psi1 / ((psi2 + K_sp) + r) where
psi2 + K_sp > 0, (r - (psi2 + K_sp)) / 2 otherwise, r the square root of the
discriminant): a handful of correctly rounded operations on terms of one
sign, so u2 is within 4 eps of the root relative to it (about 2 eps seen
when the same operations are carried out in numpy); u1 = psi1 - u2 and
u3 = psi2 + u2 add one rounding to that error, within 3 eps (|psi| + |u2|)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
KSP = 3.36e-9


@pytest.fixture(scope="module")
def gb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02708_gb300 import build
    build.build()
    import paper_1601_02708_gb300 as pkg
    return pkg


def _invariants(n, seed):
    """Invariants of non-negative species over several decades, a few with
    psi2 + K_sp <= 0 (carbonate below calcium) and a few exact zeros."""
    rng = np.random.default_rng(seed)
    u = 10.0 ** rng.uniform(-9, 0, (3, n))
    u[:, :7] = 0.0
    p1 = u[0] + u[1]
    p2 = u[2] - u[1]
    return p1, p2


def _check(got, want, p1, p2):
    g1, g2, g3 = (np.asarray(x) for x in got)
    w1, w2, w3 = want
    assert np.all(np.abs(g2 - w2) <= 4 * EPS * np.abs(w2))
    assert np.all(np.abs(g1 - w1) <= 3 * EPS * (np.abs(p1) + np.abs(w2)))
    assert np.all(np.abs(g3 - w3) <= 3 * EPS * (np.abs(p2) + np.abs(w2)))


@pytest.mark.parametrize("ksp", [KSP, 1e-4, 0.3, 40.0])
@pytest.mark.parametrize("n", [1, 1000, 4099])
def test_species_match_the_oracle(gb, ksp, n):
    from oracle import chemistry
    p1, p2 = _invariants(n, n + int(ksp * 1e9) % 97)
    want = chemistry.calcite_species(p1, p2, ksp)
    _check(gb.calcite_species(p1, p2, ksp), want, p1, p2)


def test_device_tensors_and_invariants(gb):
    import torch
    from oracle import chemistry
    p1, p2 = _invariants(3000, 1)
    want = chemistry.calcite_species(p1, p2, KSP)
    d1, d2 = (torch.from_numpy(x).cuda() for x in (p1, p2))
    got = gb.calcite_species(d1, d2, KSP)
    torch.cuda.synchronize()
    assert all(g.is_cuda for g in got)
    _check([g.cpu().numpy() for g in got], want, p1, p2)
    # the inverse map is exact arithmetic of the definition: bit for bit
    inv = gb.calcite_invariants(*want)
    for g, w in zip(inv, chemistry.calcite_invariants(*want)):
        assert np.array_equal(g, w)
    inv_dev = gb.calcite_invariants(*[torch.from_numpy(w).cuda() for w in want])
    for g, w in zip(inv_dev, chemistry.calcite_invariants(*want)):
        assert np.array_equal(g.cpu().numpy(), w)


def test_refusals_and_empty(gb):
    a = np.ones(3)
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(gb.LBMError):
            gb.calcite_species(a, a, bad)
    e = np.zeros(0)
    assert all(x.size == 0 for x in gb.calcite_species(e, e, KSP))
    assert all(x.size == 0 for x in gb.calcite_invariants(e, e, e))
