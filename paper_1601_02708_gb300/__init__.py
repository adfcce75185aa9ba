"""GB300-native D2Q9 lattice Boltzmann advection-diffusion-reaction library
for the pore-scale subdomain of the hybrid FEM/LBM multi-time-step method
(Karimi & Nakshatrala, arXiv 1601.02708).

The compute path is the CUDA library liblbmade.so (C ABI in
include/lbm_ade.h); `LBM` wraps it.  Nothing here falls back to a CPU
implementation: without the built library, constructing `LBM` raises.
"""
from .chemistry import (Bimolecular, Calcite, calcite_invariants, calcite_species,
                        invariants_from_species, species_from_invariants)
from .fem import FEM
from .hybrid import Hybrid
from .lbm import (DIRICHLET, LBM, LBMBatch, LBMError, LBMPair, NEUMANN, PERIODIC, REACT_BULK,
                  REACT_NONE, REACT_SURFACE, outlet_breakthrough)

__all__ = ["LBM", "LBMBatch", "LBMError", "FEM", "Hybrid", "outlet_breakthrough", "PERIODIC", "DIRICHLET", "NEUMANN",
           "REACT_NONE", "REACT_SURFACE", "REACT_BULK", "Bimolecular", "species_from_invariants",
           "invariants_from_species", "Calcite", "calcite_species", "calcite_invariants",
           "LBMPair"]
