"""Host orchestration of the split lattice (paper_1601_02708_gb300.partition)
on the CPU: run_steps with LocalExchange and with DistExchange over two and
three gloo ranks, driving stand-in slabs -- a NumPy D2Q9 pull-streaming BGK
lattice with ghost rows, whose bounce-back flags evolve between steps like
the library's solid mask -- that speak the library's exchange protocol
(phase 0: the three populations streaming across a cut; phase 1: the
boundary row's flags).  The split runs must equal the unsplit stand-in bit
for bit, which checks which message goes to which side and rank, the ring
of a periodic lattice (two ranks face each other twice) and the order of
the phases."""
import os
import socket

import numpy as np
import pytest

from paper_1601_02708_gb300 import partition as pt

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])
PLANES = {pt.SIDE_S: [4, 7, 8], pt.SIDE_N: [2, 5, 6]}  # leaving across S / N


def _initial(nx, ny, seed):
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.05, 0.15, (9, ny, nx))
    flag = (rng.uniform(0, 1, (ny, nx)) < 0.05).astype(np.int64)
    return f, flag


class ToySlab:
    """Rows y0 .. y1 - 1 of a D2Q9 lattice (periodic in x) with ghost rows:
    pull streaming with bounce-back from flagged nodes, BGK relaxation to a
    fixed-velocity equilibrium; `dissolve` flags nodes whose density passed a
    threshold.  Sides of the lattice (not shared) are flagged walls."""

    def __init__(self, f, flag, y0, y1, periodic):
        import torch
        self.torch = torch
        ny = f.shape[1]
        self.y0, self.y1, self.rows = y0, y1, y1 - y0
        self.nx = f.shape[2]
        self.whole_periodic = periodic and y0 == 0 and y1 == ny
        self.shared = [] if self.whole_periodic else \
            [s for s, c in ((pt.SIDE_S, y0 > 0 or periodic), (pt.SIDE_N, y1 < ny or periodic)) if c]
        self.f = np.zeros((9, self.rows + 2, self.nx))
        self.f[:, 1:-1] = f[:, y0:y1]
        self.flag = np.ones((self.rows + 2, self.nx), np.int64)  # walls unless shared
        self.flag[1:-1] = flag[y0:y1]
        if self.whole_periodic:
            self._wrap()
        else:  # the neighbours' boundary flags of the initial state
            if pt.SIDE_S in self.shared:
                self.flag[0] = flag[(y0 - 1) % ny]
            if pt.SIDE_N in self.shared:
                self.flag[-1] = flag[y1 % ny]
        self.u = None
        self._in = {}

    def _wrap(self):
        self.f[:, 0] = self.f[:, -2]
        self.f[:, -1] = self.f[:, 1]
        self.flag[0] = self.flag[-2]
        self.flag[-1] = self.flag[1]

    def stream(self, j, eta, final):
        if self.whole_periodic:
            self._wrap()
        R, nx = self.rows, self.nx
        new = np.empty((9, R, nx))
        for i in range(9):
            src_rows = slice(1 - CY[i], 1 - CY[i] + R)
            pulled = np.roll(self.f[i, src_rows], CX[i], axis=1)
            bounce = np.roll(self.flag[src_rows], CX[i], axis=1) != 0
            new[i] = np.where(bounce, self.f[OPP[i], 1:-1], pulled)
        u = new[0]
        for i in range(1, 9):
            u = u + new[i]
        vx, vy = 0.03, -0.02
        for i in range(9):
            ev = CX[i] * vx + CY[i] * vy
            feq = W[i] * u * (1 + 3 * ev + 4.5 * ev * ev - 1.5 * (vx * vx + vy * vy))
            new[i] = new[i] - (new[i] - feq) / 0.8
        self.f[:, 1:-1] = new
        self.u = u

    def dissolve(self):
        if self.u is not None:  # the pass before the first step changes nothing here
            self.flag[1:-1] |= (self.u > 1.06).astype(np.int64)

    def _row(self, side):
        return 1 if side == pt.SIDE_S else self.rows

    def pack(self, side, phase):
        r = self._row(side)
        data = self.f[PLANES[side], r].copy() if phase == 0 else self.flag[r].astype(np.float64)
        return self.torch.from_numpy(data.reshape(-1).copy())

    def inbox(self, side, phase):
        key = (side, phase)
        if key not in self._in:
            n = 3 * self.nx if phase == 0 else self.nx
            self._in[key] = self.torch.zeros(n, dtype=self.torch.float64)
        return self._in[key]

    def unpack(self, side, phase, buf):
        g = 0 if side == pt.SIDE_S else self.rows + 1
        data = buf.numpy()
        if phase == 0:
            src = pt.SIDE_N if side == pt.SIDE_S else pt.SIDE_S  # the neighbour's opposite side
            self.f[PLANES[src], g] = data.reshape(3, self.nx)
        else:
            self.flag[g] = data.astype(np.int64)


def _whole(nx, ny, seed, periodic, n):
    f, flag = _initial(nx, ny, seed)
    s = ToySlab(f, flag, 0, ny, periodic)
    if not periodic:
        s.shared = []
    pt.run_steps([s], pt.LocalExchange([s], periodic), n, 1, first=True)
    return s.f[:, 1:-1], s.flag[1:-1]


@pytest.mark.parametrize("parts", [2, 3, 5])
@pytest.mark.parametrize("periodic", [True, False])
def test_local_exchange_matches_unsplit(parts, periodic):
    nx, ny, n = 23, 31, 40
    f0, flag0 = _initial(nx, ny, 7)
    slabs = [ToySlab(f0, flag0, y0, y1, periodic) for y0, y1 in pt.slab_bounds(ny, parts)]
    pt.run_steps(slabs, pt.LocalExchange(slabs, periodic), n, 1, first=True)
    fw, flw = _whole(nx, ny, 7, periodic, n)
    assert np.array_equal(np.concatenate([s.f[:, 1:-1] for s in slabs], axis=1), fw)
    assert np.array_equal(np.concatenate([s.flag[1:-1] for s in slabs], axis=0), flw)
    assert flw.sum() > flag0.sum()  # flags changed during the run


def test_slab_bounds_and_edge_slices():
    assert pt.slab_bounds(10, 3) == [(0, 4), (4, 7), (7, 10)]
    with pytest.raises(ValueError):
        pt.slab_bounds(5, 3)
    nx, ny = 4, 6
    e = np.arange(2 * (nx + ny), dtype=float)
    s = pt.slice_edges(e, nx, ny, 2, 5)
    assert np.array_equal(s, np.concatenate([e[2:5], e[8:11], e[12:16], e[16:20]]))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, periodic, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx, ny = 23, 31
        f0, flag0 = _initial(nx, ny, 7)
        y0, y1 = pt.slab_bounds(ny, world)[rank]
        s = ToySlab(f0, flag0, y0, y1, periodic)
        pt.run_steps([s], pt.DistExchange(s, rank, world, periodic), 40, 1, first=True)
        out.put((rank, s.f[:, 1:-1].copy(), s.flag[1:-1].copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, True), (2, False), (3, True)])
def test_dist_exchange_over_gloo_matches_unsplit(world, periodic):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, periodic, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in procs], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    fw, flw = _whole(23, 31, 7, periodic, 40)
    assert np.array_equal(np.concatenate([r[1] for r in res], axis=1), fw)
    assert np.array_equal(np.concatenate([r[2] for r in res], axis=0), flw)
