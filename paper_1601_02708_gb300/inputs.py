"""Seeded synthetic inputs for the pore-scale workloads.

This module holds no arithmetic of the method: it only draws geometries,
velocity fields and boundary-data arrays.  The CUDA path and the CPU oracle
both take their inputs from here, so each side sees the same numbers.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out below so that the
streams do not depend on the numpy version installed.

Workload recipes (lattice units, D2Q9):
  * porous medium: random overlapping disks, radius uniform in [8, 24] nodes,
    centres uniform over the lattice, added until the solid fraction reaches
    1 - porosity; the first and last columns stay fluid so that the inlet and
    outlet boundary nodes exist;
  * advection velocity: v = (d psi/dy, -d psi/dx) of a stream function made of
    16 random Fourier modes with integer wave vectors in [-8, 8]^2 \\ {0},
    amplitudes N(0,1)/|k| and phases U[0, 2 pi), scaled so that max |v| = umax,
    then zeroed in solids.
"""
from __future__ import annotations

import math

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """Sequential splitmix64 stream."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal(self) -> float:
        """Standard normal by the Box-Muller transform."""
        u1 = 1.0 - self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def uniform_array(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1): element i is the (i+1)-th output of
    SplitMix64(seed), computed vectorised with wrapping uint64 arithmetic."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(int(seed) & _MASK) + i * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def disk_packing(nx: int, ny: int, porosity: float, seed: int,
                 rmin: float = 8.0, rmax: float = 24.0) -> np.ndarray:
    """uint8 [ny, nx] solid mask (1 = solid) of random overlapping disks."""
    rng = SplitMix64(seed)
    solid = np.zeros((ny, nx), dtype=np.uint8)
    target = int(math.ceil((1.0 - porosity) * nx * ny))
    count = 0
    guard = 0
    while count < target and nx > 2:
        cx = rng.uniform() * nx
        cy = rng.uniform() * ny
        r = rmin + (rmax - rmin) * rng.uniform()
        x0, x1 = max(1, int(math.floor(cx - r))), min(nx - 2, int(math.ceil(cx + r)))
        y0, y1 = max(0, int(math.floor(cy - r))), min(ny - 1, int(math.ceil(cy + r)))
        guard += 1
        if guard > 100 * nx * ny:
            break
        if x0 > x1 or y0 > y1:
            continue
        xs = np.arange(x0, x1 + 1, dtype=np.float64)
        ys = np.arange(y0, y1 + 1, dtype=np.float64)
        inside = ((xs[None, :] - cx) ** 2 + (ys[:, None] - cy) ** 2) <= r * r
        box = solid[y0:y1 + 1, x0:x1 + 1]
        count += int(np.count_nonzero(inside & (box == 0)))
        box[inside] = 1
    return solid


def streamfunction_velocity(nx: int, ny: int, seed: int, n_modes: int = 16,
                            umax: float = 0.05, kmax: int = 8,
                            solid: np.ndarray | None = None) -> np.ndarray:
    """float64 [2, ny, nx] divergence-free velocity from a random stream
    function, scaled to max |v| = umax and zeroed at solid nodes."""
    rng = SplitMix64(seed)
    modes = []
    while len(modes) < n_modes:
        kx = int(rng.uniform() * (2 * kmax + 1)) - kmax
        ky = int(rng.uniform() * (2 * kmax + 1)) - kmax
        if kx == 0 and ky == 0:
            continue
        amp = rng.normal() / math.hypot(kx, ky)
        phase = 2.0 * math.pi * rng.uniform()
        modes.append((kx, ky, amp, phase))
    # cos(a(x) + b(y)) = cos a cos b - sin a sin b: every mode is a sum of
    # two outer products, so both components are one [ny, 2M] x [2M, nx]
    # matrix product.
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    cols_x, rows_vx, rows_vy = [], [], []
    for kx, ky, amp, phase in modes:
        a = 2.0 * math.pi * kx * x / nx
        b = 2.0 * math.pi * ky * y / ny + phase
        cols_x += [np.cos(a), -np.sin(a)]
        gy, gx = 2.0 * math.pi * ky / ny, 2.0 * math.pi * kx / nx
        rows_vx += [amp * gy * np.cos(b), amp * gy * np.sin(b)]
        rows_vy += [-amp * gx * np.cos(b), -amp * gx * np.sin(b)]
    X = np.stack(cols_x)                  # [2M, nx]
    vx = np.stack(rows_vx, axis=1) @ X    # [ny, nx]
    vy = np.stack(rows_vy, axis=1) @ X
    speed = np.sqrt(vx * vx + vy * vy).max()
    if speed > 0:
        vx *= umax / speed
        vy *= umax / speed
    vel = np.stack([vx, vy])
    if solid is not None:
        vel[:, solid != 0] = 0.0
    return vel


def edge_array(nx: int, ny: int, W=0.0, E=0.0, S=0.0, N=0.0) -> np.ndarray:
    """Per-edge-node data in the layout [W: ny][E: ny][S: nx][N: nx]; each
    side takes a scalar or an array of that side's length."""
    out = np.zeros(2 * (nx + ny))
    out[0:ny] = W
    out[ny:2 * ny] = E
    out[2 * ny:2 * ny + nx] = S
    out[2 * ny + nx:] = N
    return out


def porous_case(nx: int, ny: int, seed: int, porosity: float = 0.6,
                tau: float = 0.7, k: float = 1e-3, umax: float = 0.05,
                c_in: float = 1.0) -> dict:
    """Reactive porous lattice: disks at the given porosity, stream-function
    velocity, surface reaction rate k with dissolution, Dirichlet c_in on the
    west edge, zero-flux Neumann on the east edge, periodic in y, c0 = 0."""
    solid = disk_packing(nx, ny, porosity, seed)
    vel = streamfunction_velocity(nx, ny, seed + 1_000_003, umax=umax, solid=solid)
    return dict(
        nx=nx, ny=ny, tau=tau, edges=(1, 2, 0, 0), solid=solid, vel=vel,
        u0=np.zeros((ny, nx)), react_mode=1, k=k, dissolution=True,
        mineral=np.ones((ny, nx)), u_dir=edge_array(nx, ny, W=c_in),
        q_neu=edge_array(nx, ny))


def adjoint_case(nx: int = 512, ny: int = 512, seed: int = 4, porosity: float = 0.6,
                 tau: float = 0.7, k: float = 1e-3, k_noise: float = 0.2,
                 umax: float = 0.05, mean_u: float = 0.15, c_in: float = 1.0) -> dict:
    """Reactive porous lattice for the gradient workload: the disks and the
    stream-function stirring of porous_case plus a uniform mean flow mean_u
    along x (zeroed in solids, so the inlet signal crosses the lattice within
    a few thousand steps), a per-node rate k (1 + k_noise U[-1, 1]) at every
    fluid node (bulk mode, fixed mask), Dirichlet c_in west, zero-flux east,
    periodic y, c0 = 0."""
    solid = disk_packing(nx, ny, porosity, seed)
    vel = streamfunction_velocity(nx, ny, seed + 1_000_003, umax=umax)
    vel[0] += mean_u
    vel[:, solid != 0] = 0.0
    kf = k * (1.0 + k_noise * (2.0 * uniform_array(seed + 2_000_003, nx * ny) - 1.0))
    return dict(
        nx=nx, ny=ny, tau=tau, edges=(1, 2, 0, 0), solid=solid, vel=vel,
        u0=np.zeros((ny, nx)), react_mode=2, k_field=kf.reshape(ny, nx),
        u_dir=edge_array(nx, ny, W=c_in), q_neu=edge_array(nx, ny))


def batch_cases(n_inst: int = 256, seed: int = 3, smin: int = 64, smax: int = 1024,
                k: float = 1e-3, rmin: float = 8.0, rmax: float = 24.0) -> list:
    """Independent reactive porous instances: square side log-uniform in
    [smin, smax], porosity U[0.4, 0.8], tau U[0.6, 1.2], the disk and
    stream-function generators of porous_case (instance i seeded 3000 + i),
    surface rate k with dissolution, Dirichlet 1 west, zero-flux east,
    periodic y."""
    rng = SplitMix64(seed)
    cases = []
    for i in range(n_inst):
        side = int(round(math.exp(math.log(smin) + (math.log(smax) - math.log(smin)) * rng.uniform())))
        porosity = 0.4 + 0.4 * rng.uniform()
        tau = 0.6 + 0.6 * rng.uniform()
        solid = disk_packing(side, side, porosity, 3000 + i, rmin=rmin, rmax=rmax)
        vel = streamfunction_velocity(side, side, 3000 + i + 1_000_003, solid=solid)
        cases.append(dict(
            nx=side, ny=side, tau=tau, edges=(1, 2, 0, 0), solid=solid, vel=vel,
            u0=np.zeros((side, side)), react_mode=1, k=k, dissolution=True,
            mineral=np.ones((side, side)), u_dir=edge_array(side, side, W=1.0),
            q_neu=edge_array(side, side), porosity=porosity))
    return cases


# ---- layouts of the two-subdomain hybrid runs --------------------------------
# A layout holds the inputs of one hybrid run: the lattice's arguments, the
# continuum mesh and its Dirichlet node list (fixed nodes first, then the
# nodes of Gamma_f->c that take the lattice's trace), the lattice coordinates
# of those trace points, the physical coordinates of the lattice's Gamma_c->f
# edge nodes and their (contiguous) slot range in the lattice edge layout,
# and the step counts.  Time unit: one lattice step; lattice spacing h.

def hybrid_plain_layout(n_coarse: int = 100) -> dict:
    """Plain hybrid (no solids, no reaction): continuum [0, 0.6] x [0, 0.25]
    on 40 x 10 Q1 elements, lattice 256 x 64 on x in [0.5, 1.0] (h = 0.5/255,
    periodic in y with period 64 h), overlap [0.5, 0.6]; uniform velocity
    0.05 (lattice units) along x, tau 0.8 (D = 0.1 h^2), Gaussian pulse
    c0 = exp(-(x - 0.3)^2 / 0.002), c = 0 at the continuum inlet, zero flux
    at the lattice outlet and the continuum's y sides; 10 substeps per
    coarse step, 3 Schwarz iterations."""
    nfx, nfy = 256, 64
    h = 0.5 / (nfx - 1)
    tau = 0.8
    D = (tau - 0.5) / 3.0 * h * h
    nex, ney = 40, 10
    hx, hy = 0.6 / nex, 0.25 / ney
    nxn = nex + 1
    xs = 0.5 + np.arange(nfx) * h
    u0 = np.tile(np.exp(-(xs - 0.3) ** 2 / 0.002), (nfy, 1))
    vel = np.zeros((2, nfy, nfx))
    vel[0] = 0.05
    node_x = (np.arange((nex + 1) * (ney + 1)) % nxn) * hx
    inlet = [j * nxn for j in range(ney + 1)]
    gamma = [j * nxn + nex for j in range(ney + 1)]
    gamma_xy = np.array([[(0.6 - 0.5) / h, ((j * hy) / h) % nfy] for j in range(ney + 1)])
    pts = np.array([[0.5, j * h] for j in range(nfy)])
    return dict(
        lbm=dict(nx=nfx, ny=nfy, tau=tau, edges=(1, 2, 0, 0), vel=vel, u0=u0),
        fem=dict(nex=nex, ney=ney, x0=0.0, y0=0.0, hx=hx, hy=hy, D=D, v=(0.05 * h, 0.0),
                 theta=0.5, dt=10.0, supg=True, elem_active=None,
                 dirichlet=inlet + gamma, d0=np.exp(-(node_x - 0.3) ** 2 / 0.002)),
        fixed_values=np.zeros(len(inlet)), gamma_lattice_xy=gamma_xy,
        lbm_points=pts, lbm_slots=(0, nfy), q_neu=None,
        eta=10, max_iter=3, n_coarse=n_coarse, h=h)


def hybrid_block_layout(nex: int = 400, ney: int = 100, hole=(170, 230, 20, 80),
                        n_f: int = 2048, seed: int = 5, porosity: float = 0.55,
                        k: float = 5e-4, tau: float = 0.7, eta: int = 50,
                        max_iter: int = 5, n_coarse: int = 200, rmin: float = 8.0,
                        rmax: float = 24.0) -> dict:
    """Continuum [0, 4] x [0, 1] on nex x ney Q1 elements with an element-
    aligned hole (element ranges i0..i1, j0..j1); the pore block covers the
    hole plus two continuum elements on every side and holds an n_f x n_f
    lattice (wet nodes on the block's edges) of the disk / stream-function
    generator with surface reaction k and dissolution.  The continuum has
    v = 0 and the lattice's diffusivity D = (tau - 1/2)/3 h^2; c = 1 at the
    continuum inlet x = 0 and c0 = 1 everywhere; the lattice's four sides
    take the continuum's values (Gamma_c->f), the hole's edge takes the
    lattice's trace (Gamma_f->c)."""
    hc = 4.0 / nex
    assert abs(1.0 / ney - hc) < 1e-12
    i0, i1, j0, j1 = hole
    bx0, bx1 = (i0 - 2) * hc, (i1 + 2) * hc
    by0, by1 = (j0 - 2) * hc, (j1 + 2) * hc
    h = (bx1 - bx0) / (n_f - 1)
    D = (tau - 0.5) / 3.0 * h * h
    act = np.ones((ney, nex), np.uint8)
    act[j0:j1, i0:i1] = 0
    nxn = nex + 1
    inlet = [j * nxn for j in range(ney + 1)]
    ring = [j * nxn + i for j in range(j0, j1 + 1) for i in range(i0, i1 + 1)
            if i in (i0, i1) or j in (j0, j1)]
    gamma_xy = np.array([[((r % nxn) * hc - bx0) / h, ((r // nxn) * hc - by0) / h]
                         for r in ring])
    side = bx0 + np.arange(n_f) * h
    sidey = by0 + np.arange(n_f) * h
    pts = np.concatenate([
        np.stack([np.full(n_f, bx0), sidey], 1),    # W
        np.stack([np.full(n_f, bx1), sidey], 1),    # E
        np.stack([side, np.full(n_f, by0)], 1),     # S
        np.stack([side, np.full(n_f, by1)], 1)])    # N
    solid = disk_packing(n_f, n_f, porosity, seed, rmin=rmin, rmax=rmax)
    vel = streamfunction_velocity(n_f, n_f, seed + 1_000_003, solid=solid)
    u0 = np.where(solid != 0, 0.0, 1.0)
    return dict(
        lbm=dict(nx=n_f, ny=n_f, tau=tau, edges=(1, 1, 1, 1), solid=solid, vel=vel, u0=u0,
                 react_mode=1, k=k, dissolution=True, mineral=np.ones((n_f, n_f))),
        fem=dict(nex=nex, ney=ney, x0=0.0, y0=0.0, hx=hc, hy=hc, D=D, v=(0.0, 0.0),
                 theta=0.5, dt=float(eta), supg=False, elem_active=act,
                 dirichlet=inlet + ring, d0=np.ones((ney + 1) * nxn)),
        fixed_values=np.ones(len(inlet)), gamma_lattice_xy=gamma_xy,
        lbm_points=pts, lbm_slots=(0, 4 * n_f), q_neu=None,
        eta=eta, max_iter=max_iter, n_coarse=n_coarse, h=h)


def hybrid_multiblock_layout(nex: int = 200, ney: int = 50,
                             holes=((30, 60, 10, 40), (100, 120, 20, 40), (150, 190, 5, 25)),
                             n_f=(512, 256, 384), seed: int = 7, porosity: float = 0.55,
                             k: float = 5e-4, tau: float = 0.7, eta: int = 20,
                             max_iter: int = 3, n_coarse: int = 50, rmin: float = 8.0,
                             rmax: float = 24.0) -> dict:
    """Several pore blocks in one continuum (the many-subdomain coupling of
    Algorithm 2 with one continuum subdomain): [0, 4] x [0, 1] on nex x ney
    Q1 elements with one element-aligned hole per block; block b covers its
    hole plus two elements per side and holds an n_f[b] x n_f[b] lattice of
    the disk / stream-function generator (seed + b) with surface reaction and
    dissolution.  One diffusivity D = (tau - 1/2)/3 h_min^2 (h_min the finest
    block spacing, time unit one lattice step) holds everywhere: block b
    relaxes with tau_b = 1/2 + 3 D / h_b^2.  c = 1 at the inlet x = 0 and
    c0 = 1 everywhere.  Blocks must not overlap."""
    hc = 4.0 / nex
    assert abs(1.0 / ney - hc) < 1e-12 and len(holes) == len(n_f)
    act = np.ones((ney, nex), np.uint8)
    nxn = nex + 1
    inlet = [j * nxn for j in range(ney + 1)]
    lbms, gammas, points, slots, rings = [], [], [], [], []
    h_min = min(((i1 - i0 + 4) * hc) / (nf - 1) for (i0, i1, _, _), nf in zip(holes, n_f))
    D = (tau - 0.5) / 3.0 * h_min * h_min
    for b, ((i0, i1, j0, j1), nf) in enumerate(zip(holes, n_f)):
        act[j0:j1, i0:i1] = 0
        bx0, bx1 = (i0 - 2) * hc, (i1 + 2) * hc
        by0, by1 = (j0 - 2) * hc, (j1 + 2) * hc
        nfx = nf
        h = (bx1 - bx0) / (nfx - 1)
        nfy = int(round((by1 - by0) / h)) + 1
        tau_b = 0.5 + 3.0 * D / (h * h)
        ring = [j * nxn + i for j in range(j0, j1 + 1) for i in range(i0, i1 + 1)
                if i in (i0, i1) or j in (j0, j1)]
        rings += ring
        gammas.append(np.array([[((r % nxn) * hc - bx0) / h, ((r // nxn) * hc - by0) / h]
                                for r in ring]))
        xs = bx0 + np.arange(nfx) * h
        ys = by0 + np.arange(nfy) * h
        points.append(np.concatenate([
            np.stack([np.full(nfy, bx0), ys], 1), np.stack([np.full(nfy, bx0 + (nfx - 1) * h), ys], 1),
            np.stack([xs, np.full(nfx, by0)], 1), np.stack([xs, np.full(nfx, by0 + (nfy - 1) * h)], 1)]))
        slots.append((0, 2 * (nfx + nfy)))
        solid = disk_packing(nfx, nfy, porosity, seed + b, rmin=rmin, rmax=rmax)
        vel = streamfunction_velocity(nfx, nfy, seed + b + 1_000_003, solid=solid)
        lbms.append(dict(nx=nfx, ny=nfy, tau=tau_b, edges=(1, 1, 1, 1), solid=solid, vel=vel,
                         u0=np.where(solid != 0, 0.0, 1.0), react_mode=1, k=k, dissolution=True,
                         mineral=np.ones((nfy, nfx))))
    return dict(
        lbms=lbms,
        fem=dict(nex=nex, ney=ney, x0=0.0, y0=0.0, hx=hc, hy=hc, D=D, v=(0.0, 0.0),
                 theta=0.5, dt=float(eta), supg=False, elem_active=act,
                 dirichlet=inlet + rings, d0=np.ones((ney + 1) * nxn)),
        fixed_values=np.ones(len(inlet)), gamma_lattice_xy=gammas, lbm_points=points,
        lbm_slots=slots, q_neu=None, eta=eta, max_iter=max_iter, n_coarse=n_coarse)
