"""Pins of the oracle's bimolecular algebra (Sec. 7.2) against the reaction
extent, derived apart from the paper's formulas: an unreacted mixture u_A,
u_B, u_C reacts by the extent xi = min(u_A / n_A, u_B / n_B), leaving
u_A - n_A xi, u_B - n_B xi, u_C + n_C xi."""
import numpy as np
import pytest

from oracle import chemistry


@pytest.mark.parametrize("coeffs", [(1.0, 2.0, 1.0), (2.0, 3.0, 5.0), (1.0, 1.0, 1.0)])
def test_species_follow_the_reaction_extent(coeffs):
    nA, nB, nC = coeffs
    rng = np.random.default_rng(4)
    uA, uB, uC = rng.uniform(0, 1, (3, 500))
    xi = np.minimum(uA / nA, uB / nB)
    a, b = chemistry.invariants(uA, uB, uC, *coeffs)
    sA, sB, sC = chemistry.species(a, b, *coeffs)
    np.testing.assert_allclose(sA, uA - nA * xi, atol=1e-14)
    np.testing.assert_allclose(sB, uB - nB * xi, atol=1e-14)
    np.testing.assert_allclose(sC, uC + nC * xi, atol=1e-14)
    assert np.all(np.minimum(sA, sB) <= 1e-14)  # the limiting reagent is used up


def test_reacted_states_are_fixed_points():
    """States with u_A u_B = 0 are what the instantaneous reaction leaves:
    species(invariants(s)) = s."""
    nA, nB, nC = 1.0, 2.0, 1.0
    rng = np.random.default_rng(5)
    uA, uB, uC = rng.uniform(0, 1, (3, 400))
    uA[:200] = 0.0
    uB[200:] = 0.0
    s = chemistry.species(*chemistry.invariants(uA, uB, uC, nA, nB, nC), nA, nB, nC)
    for got, want in zip(s, (uA, uB, uC)):
        np.testing.assert_allclose(got, want, atol=1e-15)


def test_invariants_are_linear_and_conserved_by_the_reaction():
    """Reacting by any extent leaves alpha and beta unchanged."""
    nA, nB, nC = 2.0, 3.0, 5.0
    rng = np.random.default_rng(6)
    uA, uB, uC = rng.uniform(0, 1, (3, 100))
    xi = rng.uniform(0, 1, 100) * np.minimum(uA / nA, uB / nB)
    before = chemistry.invariants(uA, uB, uC, nA, nB, nC)
    after = chemistry.invariants(uA - nA * xi, uB - nB * xi, uC + nC * xi, nA, nB, nC)
    for x, y in zip(before, after):
        np.testing.assert_allclose(x, y, atol=1e-15)
