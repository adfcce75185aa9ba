"""The one-dimensional hybrid of Sec. 7.1 on the GPU (the library's D1Q2
lattice, lbm1d_*, and its continuum solver with one row of elements, coupled
by Algorithm 1 in hybrid1d.Hybrid1D) against the oracle's, node by node, on
rows of the section's tables; the quadratic closed form the coupled loop
must reproduce; the printed errors as upper bounds; and the D1Q2 lattice's
own boundary conditions and refusals."""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "e5_1d_hybrid_tables.txt")


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_02708_gb300 import build
    build.build()
    from paper_1601_02708_gb300 import hybrid1d
    return hybrid1d


def _rows():
    rows = []
    for ln in open(GOLDEN):
        if ln.strip() and not ln.startswith("#"):
            t, hc, hf, eta, L, it, ec, ef = ln.split()
            snap = lambda v: 1e-2 * 2.0 ** -round(math.log2(1e-2 / float(v)))
            rows.append((int(t), snap(hc), snap(hf), int(eta), float(L), int(it), float(ec),
                         float(ef)))
    return rows


@pytest.mark.parametrize("row", [r for r in _rows() if r[1] >= 5e-3 and r[2] >= 1.25e-3])
def test_matches_oracle_and_printed_bounds(pkg, row):
    from oracle import hybrid1d as o
    _, hc, hf, eta, L, it, ec, ef = row
    run = pkg.Hybrid1D(hc, hf, eta, L, it)
    n = run.run(0.4)
    ref = o.run(hc, hf, eta, L, it)
    assert n == ref["n_coarse"]
    scale = np.abs(ref["u_f"]).max()
    assert np.abs(run.coarse() - ref["u_c"]).max() <= 1e-10 * scale
    assert np.abs(run.fine() - ref["u_f"]).max() <= 1e-10 * scale
    E_c, E_f = run.errors()
    assert E_c <= ec and E_f <= ef
    run.close()


def test_lattice_matches_oracle_with_neumann_data(pkg):
    from oracle import hybrid1d as o
    n = 300
    rng = np.random.default_rng(3)
    u0 = rng.uniform(0.2, 1.0, n)
    for left, right in ((1, 2), (2, 1), (1, 1), (2, 2)):
        lat = pkg.LBM1D(n, 0.83, 0.21, u0, left=left, right=right)
        ref = o.D1Q2(n, 0.83, 0.21, u0, left=left, right=right)
        a, b, q = (0.7, 0.2), (0.9, 0.4), (0.01, -0.02)
        lat.substeps(37, 11, a, b, q)
        ref.substeps(37, 11, a, b, q)
        assert np.abs(lat.u() - ref.u).max() <= 1e-13
        blob = lat.save()
        lat.substeps(5, 5, a, b, q)
        u1 = lat.u()
        lat.restore(blob)
        lat.substeps(5, 5, a, b, q)
        assert np.array_equal(lat.u(), u1)
        lat.close()


def test_quadratic_closed_form_on_the_gpu(pkg):
    """u = 1 + b t + (b / 2D) x^2 (v = 0, tau = 1) through the GPU's coupled
    loop: the lattice's far end takes the closed form as Dirichlet data."""
    from paper_1601_02708_gb300 import hybrid1d as hy
    D, b = 1e-2, 0.3
    exact = lambda x, t: 1.0 + b * t + b / (2 * D) * np.asarray(x) ** 2
    run = hy.Hybrid1D(1e-2, 5e-3, 4, 0.1, 3, D=D, v=0.0, init=lambda x: exact(x, 0.0),
                      right=hy.DIRICHLET, right_value=lambda t: exact(1.0, t))
    for _ in range(30):
        run.coarse_step()
    assert np.abs(run.coarse() - exact(run.x_c, run.t)).max() <= 1e-10
    assert np.abs(run.fine() - exact(run.x_f, run.t)).max() <= 1e-10
    run.close()


def test_refusals(pkg):
    from paper_1601_02708_gb300 import LBMError
    with pytest.raises(LBMError):
        pkg.LBM1D(1, 1.0, 0.0)
    with pytest.raises(LBMError):
        pkg.LBM1D(10, 0.5, 0.0)
    with pytest.raises(LBMError):
        pkg.LBM1D(10, 1.0, 1.0)
    with pytest.raises(LBMError):
        pkg.LBM1D(10, 1.0, 0.0, left=0)
