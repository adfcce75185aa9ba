"""FP64 restatement of the algebra of an instantaneous bimolecular reaction
n_A A + n_B B -> n_C C (Sec. 7.2).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU baseline may use it; the product path never imports it.

The invariants alpha = u_A + (n_A / n_C) u_C and beta = u_B + (n_B / n_C) u_C
are what the lattices transport; the species are recovered as the paper
states them (u_A and u_B from the positive parts, u_C from alpha)."""
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
