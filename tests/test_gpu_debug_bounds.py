"""The debug-bounds build (every computed index of the step, dissolution and
adjoint kernels checked; a failed check is reported by the next read-out as
an error) runs the lattice, the batch and the adjoint on small ragged cases
in a fresh process: no check may fail, and the results must equal those of
the normal build."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cases():
    from paper_1601_02708_gb300 import inputs
    out = []
    for (nx, ny, seed) in ((97, 61, 1), (300, 37, 2), (33, 9, 3)):
        c = inputs.porous_case(nx, ny, seed=seed, k=0.02)
        solid = inputs.disk_packing(nx, ny, 0.7, seed, rmin=2, rmax=6)
        vel = inputs.streamfunction_velocity(nx, ny, seed + 7, solid=solid)
        c.update(solid=solid, vel=vel, mineral=np.full((ny, nx), 0.05))
        out.append(c)
    return out


def _run(pkg, inputs_mod):
    """Lattices (FP32 pipeline and plain kernel, FP64), a batch in the
    pipelined and a plain shape, and an adjoint; returns named arrays."""
    import torch
    keys = ("edges", "solid", "vel", "u0", "react_mode", "k", "dissolution", "mineral")
    res = {}
    for i, c in enumerate(_cases()):
        for prec, kern in ((32, "tma"), (32, "generic"), (64, "auto")):
            lat = pkg.LBM(c["nx"], c["ny"], c["tau"], precision=prec, **{k: c[k] for k in keys})
            lat.set_kernel(kern)
            lat.substeps(37, 1, c["u_dir"], c["u_dir"], c["q_neu"])
            lat.substeps(40, 5, c["u_dir"], c["u_dir"] * 0.5, c["q_neu"])
            res[f"lat{i}_{prec}_{kern}"] = lat.concentration()
            res[f"solid{i}_{prec}_{kern}"] = lat.solid()
    s = torch.cuda.Stream()
    for shape in (6, 0):
        cases = inputs_mod.batch_cases(n_inst=5, seed=5, smin=40, smax=200)
        mem = [pkg.LBM(c["nx"], c["ny"], c["tau"], precision=32, stream=s.cuda_stream,
                       **{k: c[k] for k in keys}) for c in cases]
        b = pkg.LBMBatch(mem)
        b.set_shape(shape)
        ud = [c["u_dir"] for c in cases]
        b.substeps(31, 1, ud, ud)
        for j, m in enumerate(mem):
            res[f"batch{shape}_{j}"] = m.concentration()
    ac = inputs_mod.adjoint_case(nx=150, ny=37)
    for prec in (32, 64):
        lat = pkg.LBM(ac["nx"], ac["ny"], ac["tau"], precision=prec,
                      **{k: ac[k] for k in ("edges", "solid", "vel", "u0", "react_mode", "k_field")})
        r = lat.adjoint(120, 1, ac["u_dir"], ac["u_dir"], ac["q_neu"], stride=11)
        res[f"adj_k_{prec}"] = r["k"]
        res[f"adj_ua_{prec}"] = r["ua"]
    return res


def _child(out):
    sys.path.insert(0, ROOT)
    import paper_1601_02708_gb300 as pkg
    from paper_1601_02708_gb300 import inputs
    np.savez(out, **_run(pkg, inputs))


def test_debug_bounds_build_runs_clean_and_matches(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02708_gb300 import build
    build.build()
    build.build(debug_bounds=True)
    out = str(tmp_path / "debug.npz")
    env = dict(os.environ, LBM_ADE_DEBUG_BOUNDS="1")
    proc = subprocess.run([sys.executable, __file__, "--child", out], env=env, cwd=ROOT,
                          capture_output=True, text=True, timeout=900)
    assert proc.returncode == 0, proc.stdout[-2000:] + proc.stderr[-4000:]
    import paper_1601_02708_gb300 as pkg
    from paper_1601_02708_gb300 import _lib, inputs
    assert _lib.lib_path() == build.LIB  # this process runs the normal build
    ref = _run(pkg, inputs)
    dbg = np.load(out)
    assert set(dbg.files) == set(ref)
    for key, val in ref.items():
        if key.startswith("solid"):
            assert np.array_equal(dbg[key], val), key
        else:
            scale = max(np.abs(val).max(), 1e-300)
            assert np.abs(dbg[key] - val).max() <= 1e-6 * scale, key


if __name__ == "__main__" and len(sys.argv) == 3 and sys.argv[1] == "--child":
    _child(sys.argv[2])
