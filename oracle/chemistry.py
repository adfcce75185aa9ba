"""FP64 restatement of the algebra of an instantaneous bimolecular reaction
n_A A + n_B B -> n_C C (Sec. 7.2).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU baseline may use it; the product path never imports it.

The invariants alpha = u_A + (n_A / n_C) u_C and beta = u_B + (n_B / n_C) u_C
are what the lattices transport; the species are recovered as the paper
states them (u_A and u_B from the positive parts, u_C from alpha)."""
import math
from fractions import Fraction

import numpy as np


def invariants(uA, uB, uC, nA, nB, nC):
    """(alpha, beta) of species concentrations."""
    return uA + (nA / nC) * uC, uB + (nB / nC) * uC


def species(alpha, beta, nA, nB, nC):
    """(u_A, u_B, u_C) of the invariants, Sec. 7.2."""
    uA = np.maximum(alpha - (nA / nB) * beta, 0.0)
    uB = (nB / nA) * np.maximum(-alpha + (nA / nB) * beta, 0.0)
    uC = (nC / nA) * (alpha - uA)
    return uA, uB, uC


# ---- calcite, Sec. 7.4: CaCO3 <-> Ca2+ + CO3^2- at equilibrium ---------------
# u1, u2, u3: CaCO3, Ca2+, CO3^2-; Eq. "Hybrid_Ksp": K_sp = u2 u3 / u1.
# Reading: the first invariant is psi1 = u1 + u2.  The printed psi1 = u1 - u2
# changes under the reaction (by -2 per unit that dissolves) and does not
# lead to the printed root; u1 + u2 is conserved and, with psi2 = u3 - u2
# (Eq. "Carbonate_uncoupled"), gives u2^2 + (psi2 + K_sp) u2 - K_sp psi1 = 0,
# whose non-negative root is the printed one.


def calcite_invariants(u1, u2, u3):
    """(psi1, psi2) of the species: psi1 = u1 + u2, psi2 = u3 - u2."""
    return u1 + u2, u3 - u2


def _sqrt_dyadic(x, bits):
    """floor(sqrt(x) 2^bits) / 2^bits for a non-negative rational x whose
    denominator divides 2^(2 bits): exact when sqrt(x) has at most `bits`
    binary fraction digits, within 2^-bits otherwise."""
    m = x * (1 << (2 * bits))
    assert m.denominator == 1
    return Fraction(math.isqrt(m.numerator), 1 << bits)


def calcite_species(psi1, psi2, ksp):
    """(u1, u2, u3) from the invariants, Sec. 7.4: the printed root
    u2 = (-(psi2 + K_sp) + sqrt((psi2 + K_sp)^2 + 4 K_sp psi1)) / 2, then
    u1 = psi1 - u2 and u3 = psi2 + u2.

    The formula is evaluated as printed in exact rational arithmetic (FP64
    inputs are dyadic rationals; the square root is taken to 2^-B with B
    above 1200 bits, exact when the discriminant is a square), and each
    result rounded once to FP64.  In FP64 alone the printed form would lose
    about eight digits of u2 at K_sp = 3.36e-9, the section's value, where it
    subtracts two nearly equal numbers.  Non-physical invariants with a
    negative discriminant give NaN."""
    p1 = np.asarray(psi1, dtype=np.float64)
    p2 = np.asarray(psi2, dtype=np.float64)
    p1, p2 = np.broadcast_arrays(p1, p2)
    out = np.empty((3,) + p1.shape)
    k = Fraction(float(ksp))
    for idx in np.ndindex(p1.shape):
        a, b = Fraction(float(p1[idx])), Fraction(float(p2[idx]))
        s = b + k
        disc = s * s + 4 * k * a
        if disc < 0:
            out[(slice(None),) + idx] = np.nan
            continue
        bits = max(1200, (disc.denominator.bit_length() + 1) // 2 + 64)
        u2 = (-s + _sqrt_dyadic(disc, bits)) / 2
        out[0][idx] = float(a - u2)
        out[1][idx] = float(u2)
        out[2][idx] = float(b + u2)
    return out[0], out[1], out[2]
