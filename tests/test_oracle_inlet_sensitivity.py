"""The pore-block hybrid's inlet sensitivity (oracle/inlet_sensitivity.py):
the continuum alone, driven from zero by a unit inlet value with the hole's
ring held at zero, over the 200 coarse steps of the configuration.  The
implicit step couples the inlet to every node, so the values at the block's
sides are not zero, but the consistent-mass Crank-Nicolson step damps them
by about 2 - sqrt(3) per element over the 168 elements from the inlet: they
stay near 1e-97, which bounds what the inlet can pass to the lattice."""
import numpy as np

from oracle import inlet_sensitivity


def test_inlet_reach_at_the_block_is_below_fp64_resolution():
    m = inlet_sensitivity.continuum_only()
    assert len(m) == 200
    assert np.all(m > 0.0)          # coupled by the implicit solve: not zero
    assert m.max() <= 1e-95         # ... but 95 orders below the data
