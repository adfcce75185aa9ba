"""Fast reactions carried by their invariants on the GPU lattices: the
instantaneous bimolecular reaction n_A A + n_B B -> n_C C (Sec. 7.2) and
calcite at equilibrium, CaCO3 <-> Ca2+ + CO3^2- (Sec. 7.4).

The invariants (alpha = u_A + (n_A / n_C) u_C, beta = u_B + (n_B / n_C) u_C;
psi1 = u1 + u2, psi2 = u3 - u2) are unchanged by the reaction, so two
lattices of one geometry transport them like any concentration (no sink),
stepped together by the library's fused two-field kernel where they qualify
(lbm_pair_*); the species follow node by node in the library
(lbm_species_from_invariants, lbm_calcite_species), as the paper recovers
them from the transported invariants."""
from __future__ import annotations

import numpy as np

from ._lib import check, load
from .lbm import LBM, LBMPair, _in_ptr, _is_tensor, _out_ptr, current_stream_handle


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


def calcite_species(psi1, psi2, ksp, stream=None, out=None):
    """(u1, u2, u3) = (CaCO3, Ca2+, CO3^2-) at equilibrium K_sp = u2 u3 / u1
    from the invariants psi1 = u1 + u2, psi2 = u3 - u2 (lbm_calcite_species);
    numpy arrays or torch tensors, as ``species_from_invariants``."""
    lib = load()
    n = _count(psi1)
    keep = []
    p1, p2 = _in_ptr(psi1, "f64", n, keep), _in_ptr(psi2, "f64", n, keep)
    out = list(out) if out is not None else [_empty_like(psi1, _shape(psi1)) for _ in range(3)]
    check(lib.lbm_calcite_species(n, float(ksp), p1, p2, *[_out_ptr(o, "f64", n) for o in out],
                                  current_stream_handle() if stream is None else stream))
    return tuple(out)


def calcite_invariants(u1, u2, u3, stream=None):
    """(psi1, psi2) = (u1 + u2, u3 - u2) of given species."""
    lib = load()
    n = _count(u1)
    keep = []
    ptrs = [_in_ptr(u, "f64", n, keep) for u in (u1, u2, u3)]
    out = [_empty_like(u1, _shape(u1)) for _ in range(2)]
    check(lib.lbm_calcite_invariants(n, *ptrs, *[_out_ptr(o, "f64", n) for o in out],
                                     current_stream_handle() if stream is None else stream))
    return tuple(out)


def _pair(a, b, fused):
    """The fused stepper of two lattices, or None for two separate calls
    (fused False; or None and the lattices do not qualify, or run the
    one-thread-per-node kernel, which on the large lattices it is chosen for
    steps two fields faster than the fused tile pipeline)."""
    if fused is False:
        return None
    if fused is None and a.kernel() != "tma":
        return None
    try:
        return LBMPair(a, b)
    except Exception:
        if fused:
            raise
        return None


class _TwoFields:
    """Two lattices of one geometry carrying two invariants."""

    @staticmethod
    def _no_reaction(lattice):
        for k in ("react_mode", "k", "k_field", "dissolution", "mineral", "u0"):
            if k in lattice:
                raise ValueError(f"{k} does not apply: the invariants carry no reaction")

    def _lattices(self, nx, ny, tau, f0, g0, fused, lattice):
        self.first = LBM(nx, ny, tau, u0=f0, **lattice)
        self.second = LBM(nx, ny, tau, u0=g0, **lattice)
        self.pair = _pair(self.first, self.second, fused)

    def _step(self, n, eta, d0, d1, q0, q1):
        if self.pair is not None:
            self.pair.substeps(n, eta, d0, d1, q0, q1)
        else:
            self.first.substeps(n, eta, d0[0], d0[1], q0)
            self.second.substeps(n, eta, d1[0], d1[1], q1)

    def invariants(self):
        return self.first.concentration(), self.second.concentration()

    def close(self):
        if self.pair is not None:
            self.pair.close()
        self.first.close()
        self.second.close()


class Calcite(_TwoFields):
    """Calcite at equilibrium (Sec. 7.4): lattices carrying psi1 = u1 + u2
    and psi2 = u3 - u2, the species recovered with K_sp = u2 u3 / u1.

    ``u10``, ``u20``, ``u30`` the initial CaCO3, Ca2+, CO3^2- [ny, nx];
    ``fused`` True steps both lattices with one kernel (lbm_pair_*; an error
    where they do not qualify), False with two, None (default) fused where
    they qualify and run the tile pipeline; the other keyword arguments are those of ``LBM`` except
    the reaction ones."""

    def __init__(self, nx, ny, tau, ksp, u10, u20, u30, fused=None, **lattice):
        self._no_reaction(lattice)
        self.ksp = float(ksp)
        sh = lambda u: np.asarray(u, dtype=np.float64).reshape(ny, nx)
        p1, p2 = calcite_invariants(sh(u10), sh(u20), sh(u30))
        self._lattices(nx, ny, tau, p1, p2, fused, lattice)
        self.psi1, self.psi2 = self.first, self.second

    def substeps(self, n, eta=1, psi1_dir=(None, None), psi2_dir=(None, None), psi1_q=None,
                 psi2_q=None):
        """n substeps of both lattices; edge data as ``Bimolecular.substeps``."""
        self._step(n, eta, psi1_dir, psi2_dir, psi1_q, psi2_q)

    def species(self):
        """(u1, u2, u3) [ny, nx] at the current time."""
        a, b = self.invariants()
        return calcite_species(a, b, self.ksp)


class Bimolecular(_TwoFields):
    """Two lattices of one geometry carrying alpha and beta.

    ``coeffs`` = (n_A, n_B, n_C); ``uA0``, ``uB0``, ``uC0`` the initial
    species [ny, nx] (uC0 None: zero); ``fused`` as for ``Calcite``; the
    other keyword arguments are those of ``LBM`` except the reaction ones
    (the invariants carry no sink)."""

    def __init__(self, nx, ny, tau, coeffs, uA0, uB0, uC0=None, fused=None, **lattice):
        self._no_reaction(lattice)
        self.coeffs = tuple(float(c) for c in coeffs)
        uA0 = np.asarray(uA0, dtype=np.float64).reshape(ny, nx)
        uB0 = np.asarray(uB0, dtype=np.float64).reshape(ny, nx)
        uC0 = np.zeros((ny, nx)) if uC0 is None else np.asarray(uC0, np.float64).reshape(ny, nx)
        a0, b0 = invariants_from_species(uA0, uB0, uC0, self.coeffs)
        self._lattices(nx, ny, tau, a0, b0, fused, lattice)
        self.alpha, self.beta = self.first, self.second

    def substeps(self, n, eta=1, alpha_dir=(None, None), beta_dir=(None, None),
                 alpha_q=None, beta_q=None):
        """n substeps of both lattices; Dirichlet data per invariant as
        (at the start, at the end of the coarse step), Neumann data likewise
        (Eq. "MTS" and the edge layout of ``LBM.substeps``)."""
        self._step(n, eta, alpha_dir, beta_dir, alpha_q, beta_q)

    def species(self):
        """(u_A, u_B, u_C) [ny, nx] at the current time."""
        a, b = self.invariants()
        return species_from_invariants(a, b, self.coeffs)
