"""Sensitivity of the pore block's outlet breakthrough to the continuum's
inlet value, computed with the oracle (FP64).

TEST INFRASTRUCTURE / ANALYSIS ONLY: nothing on the product path imports it.

With the solid mask held fixed (no dissolution during the derivative, the
reading the adjoint takes) every operation of the coupled scheme is linear
in its data: the Crank-Nicolson continuum step of Sec. 6.1.1 (Eq.
"FEM_discrete", a sparse direct solve), the lattice step with its
Dirichlet closed form (Sec. 4.1.1 (a)), the transfers of Sec. 6.2 and the
Schwarz iterations of Algorithm 1.  The breakthrough J (the sum over all
substeps of the lattice's east-edge fluid concentrations) is then affine in
the inlet value c_in, and its slope dJ/dc_in is J itself computed from
homogeneous data: zero initial state in both subdomains and c_in = 1.  Every
number of that run is of the size of its derivative, so FP64 resolves it
(no cancellation against the O(1) forward values).

``continuum_only`` is the continuum part alone (the hole's ring held at 0):
the inlet's reach at the block's sides over the run.  ``coupled`` runs the
whole scheme on the homogeneous data and reports dJ/dc_in.

Usage: python -m oracle.inlet_sensitivity [continuum|coupled] [n_coarse]
"""
from __future__ import annotations

import sys
import time

import numpy as np


def _layout():
    from paper_1601_02708_gb300 import inputs  # seeded input generators only
    return inputs.hybrid_block_layout()


def _fem(L, fem_mod):
    F = L["fem"]
    return fem_mod.Q1FEM(F["nex"], F["ney"], F["x0"], F["y0"], F["hx"], F["hy"], F["D"], F["v"],
                         F["theta"], F["dt"], supg=F["supg"], elem_active=F["elem_active"],
                         dirichlet=F["dirichlet"], d0=np.zeros_like(F["d0"]))


def _side_points(L):
    """The lattice's edge nodes in continuum coordinates."""
    F = L["fem"]
    hc, h = F["hx"], L["h"]
    ring = np.asarray(F["dirichlet"][len(L["fixed_values"]):])
    nxn = F["nex"] + 1
    bx0 = (ring % nxn).min() * hc - 2 * hc
    by0 = (ring // nxn).min() * hc - 2 * hc
    p = L["lbm_points"]
    return np.stack([bx0 + p[:, 0] * h, by0 + p[:, 1] * h], 1)


def continuum_only(n_coarse=None):
    """max over the block's side points of |d| after each coarse step of the
    continuum driven by c_in = 1 from zero, the ring held at zero."""
    from oracle import fem as fem_mod
    L = _layout()
    n_coarse = L["n_coarse"] if n_coarse is None else int(n_coarse)
    q = _fem(L, fem_mod)
    nin = len(L["fixed_values"])
    nring = len(L["fem"]["dirichlet"]) - nin
    xy = _side_points(L)
    out = []
    for _ in range(n_coarse):
        q.step(np.concatenate([np.ones(nin), np.zeros(nring)]))
        out.append(float(np.abs(q.interpolate(xy)).max()))
    return np.array(out)


def coupled(n_coarse=None, log=print):
    """dJ/dc_in of the whole scheme (fixed mask), with per-step magnitudes."""
    import oracle
    from oracle import fem as fem_mod
    L = _layout()
    n_coarse = L["n_coarse"] if n_coarse is None else int(n_coarse)
    lb = dict(L["lbm"])
    lb["u0"] = np.zeros_like(lb["u0"])
    lb["dissolution"] = False
    lb.pop("mineral")
    lat = oracle.LBMOracle(**lb)
    q = _fem(L, fem_mod)
    ones = np.ones(len(L["fixed_values"]))
    slots = np.arange(*L["lbm_slots"])
    xy = _side_points(L)
    t0 = time.time()
    rows = []
    for n in range(n_coarse):
        fem_mod.schwarz_step(q, lat, L["eta"], L["max_iter"], ones, L["gamma_lattice_xy"],
                             L["lbm_points"], slots, L["q_neu"])
        J = lat.diag()["J"]
        row = (n + 1, J, float(np.abs(lat.u()).max()), float(np.abs(q.interpolate(xy)).max()))
        rows.append(row)
        log("step %d  dJ/dc_in %.6e  max|u_lattice| %.3e  max|d| at the sides %.3e  (%.0f s)"
            % (row + (time.time() - t0,)))
    return rows


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "continuum"
    n = int(sys.argv[2]) if len(sys.argv) > 2 else None
    if what == "continuum":
        m = continuum_only(n)
        print("max over %d coarse steps of |d| at the block's sides: %.6e" % (len(m), m.max()))
    else:
        coupled(n, log=lambda s: print(s, flush=True))
