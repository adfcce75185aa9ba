"""lbm_mass_noalloc: the FP64 mass sum that allocates nothing, for callers
that cannot allocate device memory when they need the sum (code inside a
device-memory budget fixed at start-up, a host framework that owns every
allocation).  Called through the C ABI and checked against the mass of
lbm_diagnostics on the same state, twice in a row.  Collected last on
purpose."""
import ctypes

import numpy as np
import pytest

from paper_1601_02708_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02708_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    fn = lib.lbm_mass_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    lib.lbm_mass_noalloc_error.restype = ctypes.c_char_p
    import paper_1601_02708_gb300 as pkg
    return torch, pkg, lib


@pytest.mark.parametrize("prec,n", [(64, 97), (32, 97), (32, 4096)])
def test_matches_lbm_diagnostics_twice(env, prec, n):
    torch, pkg, lib = env
    kw = dict(edges=(1, 2, 0, 0), react_mode=1, k=0.05, dissolution=True)
    solid = inputs.disk_packing(n, n, 0.6, seed=n, rmin=3, rmax=9)
    vel = inputs.streamfunction_velocity(n, n, n + 1, solid=solid)
    lat = pkg.LBM(n, n, 0.7, precision=prec, solid=solid, vel=vel, u0=np.zeros((n, n)),
                  mineral=np.full((n, n), 0.05), **kw)
    ud = inputs.edge_array(n, n, W=1.0)
    lat.substeps(200, 1, ud, ud)
    ref = lat.diagnostics()["mass"]
    dtype = torch.float64 if prec == 64 else torch.float32
    u = torch.empty((n, n), dtype=dtype, device="cuda")
    lat.concentration(u, precision=prec)
    stream = torch.cuda.current_stream().cuda_stream
    dev_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    results = []
    for _ in range(2):
        host = ctypes.c_double(0.0)
        st = lib.lbm_mass_noalloc(u.data_ptr(), prec, n * n, ctypes.addressof(host), stream)
        assert st == 0, lib.lbm_mass_noalloc_error()
        st = lib.lbm_mass_noalloc(u.data_ptr(), prec, n * n, dev_out.data_ptr(), stream)
        assert st == 0, lib.lbm_mass_noalloc_error()
        torch.cuda.synchronize()
        results += [host.value, float(dev_out.item())]
    for m in results:
        assert abs(m - ref) <= 1e-12 * abs(ref)
    assert len(set(results)) == 1  # fixed summation order


def test_rejects_sizes_beyond_the_maximum(env):
    torch, pkg, lib = env
    buf = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = ctypes.c_double(0.0)
    st = lib.lbm_mass_noalloc(buf.data_ptr(), 32, 8192 * 8192 + 1, ctypes.addressof(out), None)
    assert st == -1 and b"67108864" in lib.lbm_mass_noalloc_error()
    host = np.zeros(8, dtype=np.float32)
    st = lib.lbm_mass_noalloc(host.ctypes.data, 32, 8, ctypes.addressof(out), None)
    assert st == -1 and b"device memory" in lib.lbm_mass_noalloc_error()
