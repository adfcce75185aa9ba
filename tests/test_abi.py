"""The C-ABI library builds, loads without a GPU and exports every entry
point declared in include/lbm_ade.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lbm_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1601_02708_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lbm_init", "lbm_substeps", "lbm_interface_trace"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_abi_version(lib):
    lib.lbm_abi_version.restype = ctypes.c_int
    text = open(os.path.join(ROOT, "include", "lbm_ade.h")).read()
    want = int(re.search(r"#define LBM_ADE_ABI_VERSION (\d+)", text).group(1))
    assert lib.lbm_abi_version() == want


def test_init_refuses_bad_sizes_before_touching_the_device(lib):
    """Size checks come first in lbm_init: rows above 65535 (the y block
    index of the row launches) and sides under two nodes are LBM_ERR_ARG,
    with no CUDA call made (this runs without a GPU)."""
    from paper_1601_02708_gb300._lib import Params
    for nx, ny in ((64, 65536), (1, 64), (64, 1)):
        p = Params()
        p.nx, p.ny, p.precision, p.tau = nx, ny, 32, 0.8
        for s in range(4):
            p.edge[s] = 0
        h = ctypes.c_void_p()
        lib.lbm_init.restype = ctypes.c_int
        st = lib.lbm_init(ctypes.byref(h), ctypes.byref(p), None, None, None, None, None, None)
        assert st == -1 and not h.value


def test_product_path_has_no_oracle_dependency():
    """The package never imports or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_1601_02708_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lbm_oracle" not in text, f


def test_bimolecular_refuses_reaction_arguments():
    """The invariants carry no reaction: a sink or dissolution is refused
    before any lattice is made (host logic, no GPU needed)."""
    import numpy as np
    import pytest
    from paper_1601_02708_gb300 import Bimolecular
    z = np.zeros((4, 5))
    for kw in ({"k": 1e-3}, {"dissolution": True}, {"react_mode": 1}, {"u0": z}):
        with pytest.raises(ValueError):
            Bimolecular(5, 4, 0.8, (1, 2, 1), z, z, **kw)


def test_calcite_refuses_reaction_arguments():
    """Calcite's invariants carry no sink either: refused before any lattice
    is made (host logic, no GPU needed)."""
    import numpy as np
    import pytest
    from paper_1601_02708_gb300 import Calcite
    z = np.zeros((4, 5))
    for kw in ({"k": 1e-3}, {"dissolution": True}, {"react_mode": 1}, {"k_field": z},
               {"mineral": z}):
        with pytest.raises(ValueError):
            Calcite(5, 4, 0.8, 3.36e-9, z, z, z, **kw)


def test_chemistry_pairs_only_when_asked_or_possible():
    """fused=False never makes a pair; fused=None makes none for lattices
    on the one-thread-per-node kernel and falls back to two separate
    lattices when the pair is refused; fused=True passes the refusal on
    (stand-in lattices and pair constructor, no GPU)."""
    import pytest
    from paper_1601_02708_gb300 import chemistry

    class Refused(Exception):
        pass

    class Lat:
        def __init__(self, kernel):
            self._k = kernel

        def kernel(self):
            return self._k

    calls = []

    def refuse(a, b):
        calls.append((a, b))
        raise Refused()

    tma, plain = Lat("tma"), Lat("generic")
    orig = chemistry.LBMPair
    chemistry.LBMPair = refuse
    try:
        assert chemistry._pair(tma, tma, False) is None and not calls
        assert chemistry._pair(plain, plain, None) is None and not calls
        assert chemistry._pair(tma, tma, None) is None and len(calls) == 1
        with pytest.raises(Refused):
            chemistry._pair(plain, plain, True)
    finally:
        chemistry.LBMPair = orig
