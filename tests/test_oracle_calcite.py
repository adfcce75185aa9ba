"""Pins of the oracle's calcite algebra (Sec. 7.4) on facts derived apart
from the printed root: the equilibrium K_sp = u2 u3 / u1 itself, the
invariants' conservation under the reaction (which fixes the reading
psi1 = u1 + u2), a root found by bisection in exact rational arithmetic, and
the special cases where the root is known in closed form."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import chemistry

KSP = 3.36e-9  # the section's solubility product at room temperature


def _states(rng, n):
    """Non-negative species at equilibrium-free random values."""
    return rng.uniform(0.0, 1.0, (3, n))


@pytest.mark.parametrize("ksp", [KSP, 1e-3, 0.7, 25.0])
def test_species_satisfy_the_equilibrium(ksp):
    """u2 u3 = K_sp u1 (Eq. "Hybrid_Ksp") to rounding, all species
    non-negative, for invariants of non-negative species."""
    rng = np.random.default_rng(11)
    u1, u2, u3 = _states(rng, 400)
    p1, p2 = chemistry.calcite_invariants(u1, u2, u3)
    s1, s2, s3 = chemistry.calcite_species(p1, p2, ksp)
    assert min(s1.min(), s2.min(), s3.min()) >= 0.0
    lhs, rhs = s2 * s3, ksp * s1
    assert np.all(np.abs(lhs - rhs) <= 8e-16 * np.maximum(np.abs(lhs), np.abs(rhs)) + 1e-300)
    q1, q2 = chemistry.calcite_invariants(s1, s2, s3)
    assert np.all(np.abs(q1 - p1) <= 4e-16 * (np.abs(p1) + 1))
    assert np.all(np.abs(q2 - p2) <= 4e-16 * (np.abs(p2) + 1))


def test_reaction_conserves_psi1_as_u1_plus_u2():
    """Dissolving d of CaCO3 (u1 - d, u2 + d, u3 + d) leaves u1 + u2 and
    u3 - u2 unchanged, and changes the printed u1 - u2 by -2d: only the sum
    is an invariant, and only it leads to the printed root."""
    rng = np.random.default_rng(12)
    u1, u2, u3 = _states(rng, 50)
    d = rng.uniform(0, 1, 50) * u1
    before = chemistry.calcite_invariants(u1, u2, u3)
    after = chemistry.calcite_invariants(u1 - d, u2 + d, u3 + d)
    for x, y in zip(before, after):
        np.testing.assert_allclose(x, y, atol=1e-15)
    np.testing.assert_allclose((u1 - d) - (u2 + d) - (u1 - u2), -2 * d, atol=1e-15)
    # any state reached by the reaction relaxes to the same equilibrium
    e0 = chemistry.calcite_species(*before, 0.1)
    e1 = chemistry.calcite_species(*after, 0.1)
    for x, y in zip(e0, e1):
        np.testing.assert_allclose(x, y, atol=1e-15)


def _bisect(psi1, psi2, ksp, iters=200):
    """The root in [max(0, -psi2), psi1] of u2 (psi2 + u2) - ksp (psi1 - u2)
    (equilibrium with u1 = psi1 - u2, u3 = psi2 + u2), in rational arithmetic."""
    a, b, k = Fraction(psi1), Fraction(psi2), Fraction(ksp)
    g = lambda x: x * (b + x) - k * (a - x)
    lo, hi = max(Fraction(0), -b), a
    assert g(lo) <= 0 <= g(hi)
    for _ in range(iters):
        mid = (lo + hi) / 2
        if g(mid) <= 0:
            lo = mid
        else:
            hi = mid
    return float(lo)


@pytest.mark.parametrize("psi1,psi2,ksp", [(1.0, 1.0, KSP), (0.4, -0.3, KSP), (0.7, 0.0, 0.2),
                                           (1e-6, 2.0, KSP), (2.0, -1.9, 1e-4), (0.3, 0.5, 3.0)])
def test_root_matches_exact_bisection(psi1, psi2, ksp):
    _, u2, _ = chemistry.calcite_species(np.array([psi1]), np.array([psi2]), ksp)
    want = _bisect(psi1, psi2, ksp)
    assert abs(u2[0] - want) <= 2e-16 * abs(want)


def test_closed_form_special_cases():
    """psi1 = 0 (no calcium at all) leaves u2 = 0 when psi2 + K_sp > 0;
    psi2 = -K_sp gives u2 = sqrt(K_sp psi1); K_sp large against the
    invariants dissolves nearly all: u2 -> psi1."""
    z = chemistry.calcite_species(np.array([0.0]), np.array([0.5]), KSP)
    assert z[1][0] == 0.0 and z[0][0] == 0.0 and z[2][0] == 0.5
    k = 0.04
    m = chemistry.calcite_species(np.array([0.25]), np.array([-k]), k)
    assert abs(m[1][0] - np.sqrt(k * 0.25)) <= 1e-16
    big = chemistry.calcite_species(np.array([0.3]), np.array([0.2]), 1e12)
    assert abs(big[1][0] - 0.3) <= 1e-12


def test_planted_sign_error_fails_the_equilibrium(monkeypatch):
    """Planted in the oracle: the root of the printed psi1 = u1 - u2 reading
    (u2^2 + (psi2 - K_sp) u2 - K_sp psi1 = 0, species from u1 = psi1 + u2)
    leaves u2 u3 != K_sp u1 for the species the invariants came from."""
    rng = np.random.default_rng(13)
    u1, u2, u3 = _states(rng, 20)
    p1, p2 = chemistry.calcite_invariants(u1, u2, u3)
    ksp = 0.05

    def wrong(psi1, psi2, k):
        s = psi2 - k
        c = 0.5 * (-s + np.sqrt(s * s + 4 * k * psi1))
        return psi1 - c, c, psi2 + c

    monkeypatch.setattr(chemistry, "calcite_species", wrong)
    s1, s2, s3 = chemistry.calcite_species(p1, p2, ksp)
    assert np.abs(s2 * s3 - ksp * s1).max() > 1e-3
