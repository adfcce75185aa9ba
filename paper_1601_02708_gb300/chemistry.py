"""Instantaneous bimolecular reactions n_A A + n_B B -> n_C C (Sec. 7.2) on
the GPU lattices.

The invariants alpha = u_A + (n_A / n_C) u_C and beta = u_B + (n_B / n_C) u_C
are unchanged by the reaction, so two lattices of one geometry transport
them like any concentration (no sink); the species follow node by node in
the library (lbm_species_from_invariants), as the paper recovers them from
the transported invariants."""
from __future__ import annotations

import numpy as np

from ._lib import check, load
from .lbm import LBM, _in_ptr, _is_tensor, _out_ptr, current_stream_handle


def _empty_like(a, shape):
    if _is_tensor(a):
        import torch
        return torch.empty(shape, dtype=torch.float64, device=a.device)
    return np.empty(shape, dtype=np.float64)


def _count(a):
    return int(a.numel()) if _is_tensor(a) else int(np.asarray(a).size)


def _shape(a):
    return tuple(a.shape)


def species_from_invariants(alpha, beta, coeffs, stream=None, out=None):
    """(u_A, u_B, u_C) from the invariants; numpy arrays or torch tensors
    (the outputs follow the type and device of ``alpha``, or are the three
    arrays given as ``out``)."""
    lib = load()
    nA, nB, nC = (float(c) for c in coeffs)
    n = _count(alpha)
    keep = []
    pa, pb = _in_ptr(alpha, "f64", n, keep), _in_ptr(beta, "f64", n, keep)
    out = list(out) if out is not None else [_empty_like(alpha, _shape(alpha)) for _ in range(3)]
    check(lib.lbm_species_from_invariants(n, nA, nB, nC, pa, pb,
                                          *[_out_ptr(o, "f64", n) for o in out],
                                          current_stream_handle() if stream is None else stream))
    return tuple(out)


def invariants_from_species(uA, uB, uC, coeffs, stream=None):
    """(alpha, beta) of given species concentrations."""
    lib = load()
    nA, nB, nC = (float(c) for c in coeffs)
    n = _count(uA)
    keep = []
    ptrs = [_in_ptr(u, "f64", n, keep) for u in (uA, uB, uC)]
    out = [_empty_like(uA, _shape(uA)) for _ in range(2)]
    check(lib.lbm_invariants_from_species(n, nA, nB, nC, *ptrs,
                                          *[_out_ptr(o, "f64", n) for o in out],
                                          current_stream_handle() if stream is None else stream))
    return tuple(out)


class Bimolecular:
    """Two lattices of one geometry carrying alpha and beta.

    ``coeffs`` = (n_A, n_B, n_C); ``uA0``, ``uB0``, ``uC0`` the initial
    species [ny, nx] (uC0 None: zero); the other keyword arguments are those
    of ``LBM`` except the reaction ones (the invariants carry no sink)."""

    def __init__(self, nx, ny, tau, coeffs, uA0, uB0, uC0=None, **lattice):
        for k in ("react_mode", "k", "k_field", "dissolution", "mineral", "u0"):
            if k in lattice:
                raise ValueError(f"{k} does not apply: the invariants carry no reaction")
        self.coeffs = tuple(float(c) for c in coeffs)
        uA0 = np.asarray(uA0, dtype=np.float64).reshape(ny, nx)
        uB0 = np.asarray(uB0, dtype=np.float64).reshape(ny, nx)
        uC0 = np.zeros((ny, nx)) if uC0 is None else np.asarray(uC0, np.float64).reshape(ny, nx)
        a0, b0 = invariants_from_species(uA0, uB0, uC0, self.coeffs)
        self.alpha = LBM(nx, ny, tau, u0=a0, **lattice)
        self.beta = LBM(nx, ny, tau, u0=b0, **lattice)

    def substeps(self, n, eta=1, alpha_dir=(None, None), beta_dir=(None, None),
                 alpha_q=None, beta_q=None):
        """n substeps of both lattices; Dirichlet data per invariant as
        (at the start, at the end of the coarse step), Neumann data likewise
        (Eq. "MTS" and the edge layout of ``LBM.substeps``)."""
        self.alpha.substeps(n, eta, alpha_dir[0], alpha_dir[1], alpha_q)
        self.beta.substeps(n, eta, beta_dir[0], beta_dir[1], beta_q)

    def invariants(self):
        return self.alpha.concentration(), self.beta.concentration()

    def species(self):
        """(u_A, u_B, u_C) [ny, nx] at the current time."""
        a, b = self.invariants()
        return species_from_invariants(a, b, self.coeffs)

    def close(self):
        self.alpha.close()
        self.beta.close()
