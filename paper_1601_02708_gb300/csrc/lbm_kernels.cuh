// lbm_kernels.cuh -- the fused D2Q9 ADE-LBM step and its companions.
//
// State between steps: post-collision populations f* in SoA planes
// [9][rows][pitch] (padded layout with ghost cells, see lbm_lattice.cuh),
// two buffers swapped every step.  One step pulls f_i(x) = f*_i(x - e_i)
// (Eq. "LBE"), replaces pulls from solid nodes by halfway bounce-back, sets
// the populations pulled from outside the lattice by the maximum-entropy
// conditions (Sec. 4.1.1), takes u = sum f (Eq. "LBM_Macro"), and collides
// with the BGK operator (Eq. "Collision", "LBM_feq") plus the first-order
// sink.  The sequence of states equals the paper's collide -> stream -> BC
// order shifted by half a step: the stored f* is what the next stream moves.
//
// The node update (step_node) is written once and reads its inputs through a
// source object: GlobalSrc reads the padded arrays directly (FP64 mode and
// the generic kernel), the TMA kernel of lbm_tma.cuh reads a shared-memory
// tile.
#pragma once
#include <cstdint>

#include "lbm_lattice.cuh"

namespace lbm {

constexpr int kBX = 32;  // generic kernel: threads along x per block
constexpr int kBY = 8;   // generic kernel: rows per block

template <typename Real>
struct StepArgs {
  const Real* __restrict__ fin;  // f* of the previous step
  Real* __restrict__ fout;       // f* of this step
  const uint32_t* __restrict__ link;  // [rows][pitch] link words
  const Real* __restrict__ vel;  // [2][rows][pitch]
  const Real* __restrict__ kf;   // [rows][pitch] or null
  Real* __restrict__ u_out;      // [rows][pitch], written on the final substep
  Real* __restrict__ ureact;     // [rows][pitch], k u / W_s at reactive nodes
  const double* __restrict__ ua;  // edge data, start of the coarse step
  const double* __restrict__ ub;  // edge data, end of the coarse step
  const double* __restrict__ q;   // Neumann data
  const float* __restrict__ ua32;  // FP32 copies of the edge data (FP32 lattice)
  const float* __restrict__ ub32;
  const float* __restrict__ q32;
  long long* __restrict__ infeasible;  // per edge slot
  double* __restrict__ jnode;          // per east-edge row: sum_t u
  double* __restrict__ partial;        // per block: sum u (final substep)
  int* __restrict__ status;            // device error word (0 = fine)
  unsigned char* __restrict__ bc_root;  // per edge slot: 1 where the Neumann root
                                        // set the unknowns this step (or null)
  long long* __restrict__ wall_infeasible;  // count of wall solves without a root
  int wall_maxent;  // pore walls of the maximum-entropy kind (else bounce-back)
  long long plane;  // pitch * rows
  int nx, ny, pitch;
  int per_x, per_y;
  int edge[4];
  int react_mode;
  int dissolution;
  Real omega;  // 1 / tau
  Real k_scalar;
  double frac;  // j / eta of this substep
};

// Warp + block sum of a double into one value per block (thread 0 holds it).
__device__ __forceinline__ double block_sum(double v, double* smem) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  __syncthreads();
  if (lane == 0) smem[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (tid == 0) {
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    for (int k = 0; k < nw; ++k) s += smem[k];
  }
  return s;
}

// BGK collision with equilibrium
//   f^eq_i = w_i u (1 + e.v / c_s^2 + (e.v)^2 / (2 c_s^4) - v.v / (2 c_s^2))
// and the explicit sink -w_i k u.  The weights sum to one, so sum_i f^eq_i = u
// and the sink removes exactly k u; rounded to FP32 they sum to 1 + 7.5e-9,
// which would create mass at every collision.  The rest population therefore
// takes the remainder (f^eq_0 = u - sum_{i>0} f^eq_i, and likewise for the
// sink): the same quantities in exact arithmetic, without the drift.
template <typename Real>
__device__ __forceinline__ void equilibrium(Real (&feq)[9], Real u, Real vx, Real vy) {
  const Real vv = vx * vx + vy * vy;
  const Real base = (Real)1 - (Real)1.5 * vv;
  Real rest = u;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const Real ev = (Real)cx_of(i) * vx + (Real)cy_of(i) * vy;
    feq[i] = (Real)w_of(i) * u * (base + (Real)3 * ev + (Real)4.5 * ev * ev);
    rest -= feq[i];
  }
  feq[0] = rest;
}

// Collision written for the fewest operations: with P_i = 1 + 3 e.v +
// 4.5 (e.v)^2 - 1.5 v.v, f*_i = (1 - omega) f_i + w_i u (omega P_i - k) for the
// moving populations, evaluated per opposite pair (i, opp i), whose P differ
// only in the sign of 3 e.v; the rest population takes the remainder
// f*_0 = (1 - k) u - sum_{i>0} f*_i, which is the same value in exact
// arithmetic (sum_i f*_i = (1 - k) u) and keeps the stored populations
// summing to the post-reaction mass in FP32.
template <typename Real>
__device__ __forceinline__ void collide(Real (&f)[9], Real u, Real vx, Real vy,
                                        Real omega, Real kr) {
  const Real base = (Real)1 - (Real)1.5 * (vx * vx + vy * vy);
  const Real om1 = (Real)1 - omega;
  Real rest = u - kr * u;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = p < 2 ? p + 1 : p + 3;  // 1, 2, 5, 6; opposites 3, 4, 7, 8
    const int o = opp_of(i);
    const Real wu = (Real)w_of(i) * u;
    const Real ev = (Real)cx_of(i) * vx + (Real)cy_of(i) * vy;
    const Real sym = wu * (omega * ((Real)4.5 * ev * ev + base) - kr);
    const Real anti = wu * omega * (Real)3 * ev;
    f[i] = om1 * f[i] + (sym + anti);
    f[o] = om1 * f[o] + (sym - anti);
    rest -= f[i] + f[o];
  }
  f[0] = rest;
}

// a / b for the reaction split: exact in FP64; the fast reciprocal-based
// quotient in FP32 (the value only feeds the FP64 mineral sum).
__device__ __forceinline__ double share(double a, double b) { return a / b; }
__device__ __forceinline__ float share(float a, float b) { return __fdividef(a, b); }

// Store a node value and, at nodes on a periodic side, its ghost images.
template <typename Real>
__device__ __forceinline__ void store_node(Real* __restrict__ base, long long n, Real v,
                                           bool ghosts, int x, int y, int nx, int ny,
                                           int pitch, int per_x, int per_y,
                                           long long limit = 1ll << 62, int* flag = nullptr) {
  base[dbg_idx(n, limit, flag, kSiteStore)] = v;
  if (ghosts)
    for_each_ghost(x, y, nx, ny, per_x, per_y, [&](int gx, int gy) {
      base[dbg_idx((long long)gy * pitch + gx, limit, flag, kSiteStore)] = v;
    });
}

// Inputs of one node read straight from the padded global arrays.
template <typename Real>
struct GlobalSrc {
  const StepArgs<Real>& a;
  long long n;
  __device__ __forceinline__ long long up(int i) const {  // index of x - e_i
    return n - (long long)cx_of(i) - (long long)cy_of(i) * a.pitch;
  }
  __device__ __forceinline__ long long nd() const { return dbg_idx(n, a.plane, a.status, kSiteNode); }
  __device__ __forceinline__ long long pop(long long i) const {
    return dbg_idx(i, 9 * a.plane, a.status, kSitePull);
  }
  __device__ __forceinline__ uint32_t word() const { return a.link[nd()]; }
  __device__ __forceinline__ Real pull(int i) const { return a.fin[pop(i * a.plane + up(i))]; }
  __device__ __forceinline__ Real own(int i) const { return a.fin[pop(i * a.plane + n)]; }
  // pull of direction i, or halfway bounce-back of the node's own opposite
  // population: one load from the chosen address
  __device__ __forceinline__ Real pull_or_bounce(int i, bool bounce) const {
    return a.fin[pop(bounce ? (long long)opp_of(i) * a.plane + n : i * a.plane + up(i))];
  }
  __device__ __forceinline__ Real vx() const { return a.vel[nd()]; }
  __device__ __forceinline__ Real vy() const { return a.vel[a.plane + nd()]; }
  __device__ __forceinline__ Real kf() const { return a.kf[nd()]; }
};

// One node's step.  (x, y) interior coordinates, n its padded index.  Writes
// f* (and ghost images), ureact, jnode, u_out; returns u (0 at solid nodes)
// for the mass reduction.
// kEdge false: the caller guarantees the node is at least one node away
// from every side, so no pull leaves the lattice, no ghost image exists and
// the node is not on the outlet; the boundary code is then compiled out.
// kWalls: the kernel may meet maximum-entropy pore walls (a.wall_maxent);
// kernels built without it carry no wall code.
template <typename Real, bool kFinal, bool kEdge, bool kWalls = false, class Src>
__device__ __forceinline__ double step_node(const StepArgs<Real>& a, const Src& src,
                                            int x, int y, long long n, double frac) {
  const uint32_t w = src.word();
  const bool ghosts =
      kEdge && ((x == 0) | (x == a.nx - 1) | (y == 0) | (y == a.ny - 1)) &&
      (a.per_x | a.per_y);
  // Solid nodes hold no populations, but a solid node whose 32-byte sector
  // (8 FP32 nodes, aligned since kXO = 8) holds fluid nodes writes zeros, so
  // every sector the warp touches is written whole.  A node that turns
  // fluid before this step collides (pending) gets zero populations anyway.
  const bool solid = (w & kOwnSolid) && !(w & kOwnPending);
  const unsigned active = __activemask();
  const unsigned fluid_lanes = __ballot_sync(active, !solid);
  const unsigned lane = threadIdx.x & 31u;
  const bool fill = ((fluid_lanes >> (lane & 24u)) & 0xFFu) != 0u;
  if (w & kOwnSolid) {
    if ((w & kOwnPending) || (sizeof(Real) == 4 && fill)) {
#pragma unroll
      for (int i = 0; i < 9; ++i)
        store_node(a.fout + i * a.plane, n, (Real)0, ghosts, x, y, a.nx, a.ny, a.pitch,
                   a.per_x, a.per_y, a.plane, a.status);
      if (a.dissolution && (w & kOwnPending))
        store_node(a.ureact, n, (Real)0, ghosts, x, y, a.nx, a.ny, a.pitch, a.per_x,
                   a.per_y, a.plane, a.status);
    }
    if (kFinal) a.u_out[dbg_idx(n, a.plane, a.status, kSiteNode)] = (Real)0;
    return 0.0;
  }
  Real f[9];
  f[0] = src.own(0);
#pragma unroll
  for (int i = 1; i < 9; ++i) f[i] = src.pull_or_bounce(i, w & up_bit(kUpSolidShift, i));
  // pore walls of the maximum-entropy kind, at nodes off the open lattice
  // sides (those keep bounce-back at their solid links)
  if (kWalls && a.wall_maxent && (w & 0xFFu) && !(w & (0xFFu << kUpOutShift)))
    if (maxent_wall(f, (w & 0xFFu) << 1))
      atomicAdd(reinterpret_cast<unsigned long long*>(a.wall_infeasible), 1ull);
  if (kEdge) {
    const unsigned unknown = ((w >> kUpOutShift) & 0xFFu) << 1;  // bit i: direction i
    if (unknown) {
      // Boundary node: Dirichlet wins at corners, else Neumann.
      int dside, nside, sx, sy;
      edge_kind(a.edge, x, y, a.nx, a.ny, &dside, &nside, &sx, &sy);
      bool bad;
      int slot;
      if (dside >= 0) {
        slot = edge_slot(dside, x, y, a.nx, a.ny);
        if constexpr (sizeof(Real) == 4) {
          const float fr = (float)frac;
          bad = maxent_dirichlet_f32(f, unknown, (1.f - fr) * a.ua32[slot] + fr * a.ub32[slot]);
        } else {
          const double up = (1.0 - frac) * a.ua[slot] + frac * a.ub[slot];
          bad = maxent_dirichlet(f, unknown, up);
        }
      } else {
        slot = edge_slot(nside, x, y, a.nx, a.ny);
        int how = -1;
        if constexpr (sizeof(Real) == 4) {
          if (sx == 0 || sy == 0) how = maxent_neumann_side_f32(f, unknown, sx, sy, a.q32[slot]);
        }
        if (how < 0) {  // FP64 lattice, or the corner of two Neumann sides
          Real fbb[9];
#pragma unroll
          for (int i = 0; i < 9; ++i)
            fbb[i] = (unknown & (1u << opp_of(i))) ? src.own(i) : (Real)0;
          how = maxent_neumann(f, unknown, sx, sy, a.q[slot], fbb);
        }
        bad = how == kNeuInfeasible;
        if (a.bc_root) a.bc_root[slot] = how == kNeuRoot;
      }
      if (bad) atomicAdd(reinterpret_cast<unsigned long long*>(a.infeasible + slot), 1ull);
    }
  }
  Real u = f[0];
#pragma unroll
  for (int i = 1; i < 9; ++i) u += f[i];
  // links to solid neighbours after this step's flips: axis links weigh 1/9,
  // diagonal links 1/36
  const uint32_t post = (w >> kUpPostShift) & 0xFFu;
  const bool near_solid = post != 0u;
  Real kr = (Real)0;
  if (a.react_mode == kReactBulk || (a.react_mode == kReactSurface && near_solid))
    kr = a.kf ? src.kf() : a.k_scalar;
  collide(f, u, src.vx(), src.vy(), a.omega, kr);
#pragma unroll
  for (int i = 0; i < 9; ++i)
    store_node(a.fout + i * a.plane, n, f[i], ghosts, x, y, a.nx, a.ny, a.pitch,
               a.per_x, a.per_y, a.plane, a.status);
  // mass this node takes from each solid neighbour per unit link weight
  if (a.dissolution && near_solid) {
    const Real wsolid = (Real)__popc(post & 0x0Fu) * (Real)w_of(1) +
                        (Real)__popc(post & 0xF0u) * (Real)w_of(5);
    store_node(a.ureact, n, share(kr * u, wsolid), ghosts, x, y, a.nx, a.ny, a.pitch,
               a.per_x, a.per_y, a.plane, a.status);
  }
  // one node per row adds to its row's sum: a reduction without a read-back
  if (kEdge && x == a.nx - 1) atomicAdd(a.jnode + y, (double)u);
  if (kFinal) a.u_out[dbg_idx(n, a.plane, a.status, kSiteNode)] = u;
  return (double)u;
}

// True when the warp's 32 consecutive nodes (xs .. xs + 31, row y) all lie
// one node or more inside every side of the lattice: the boundary code can
// be skipped for the whole warp (the test is warp-uniform).
__device__ __forceinline__ bool group_is_interior(int xs, int y, int nx, int ny) {
  return xs >= 1 && xs + 32 <= nx - 1 && y >= 1 && y <= ny - 2;
}

// Generic step: one thread per node, inputs from global memory.  Used in
// FP64 mode; the FP32 path runs the TMA kernel instead.
template <typename Real, bool kFinal, bool kWalls = false>
__global__ void __launch_bounds__(kBX * kBY, sizeof(Real) == 4 ? 4 : 4)
    lbm_step(const StepArgs<Real> a) {
  __shared__ double red[kBX * kBY / 32];
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  double my_u = 0.0;
  if (x < a.nx && y < a.ny) {
    const long long n = (long long)(y + kYO) * a.pitch + (x + kXO);
    GlobalSrc<Real> src{a, n};
    if (group_is_interior(blockIdx.x * kBX, y, a.nx, a.ny))
      my_u = step_node<Real, kFinal, false, kWalls>(a, src, x, y, n, a.frac);
    else
      my_u = step_node<Real, kFinal, true, kWalls>(a, src, x, y, n, a.frac);
  }
  if (kFinal) {
    const double s = block_sum(my_u, red);
    if (threadIdx.x == 0 && threadIdx.y == 0)
      a.partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// Initialisation, Sec. 6.2 (i): f = f^eq(u0), then the collision of the
// first step, so that the stored state is post-collision like every other.
// u0 is a plain [ny][nx] array.
template <typename Real>
__global__ void __launch_bounds__(kBX * kBY)
    lbm_init_kernel(const StepArgs<Real> a, const double* __restrict__ u0) {
  __shared__ double red[kBX * kBY / 32];
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  double my_u = 0.0;
  if (x < a.nx && y < a.ny) {
    const long long n = (long long)(y + kYO) * a.pitch + (x + kXO);
    const bool ghosts = ((x == 0) | (x == a.nx - 1) | (y == 0) | (y == a.ny - 1)) &&
                        (a.per_x | a.per_y);
    const uint32_t w = a.link[n];
    if (w & kOwnSolid) {
      a.u_out[n] = (Real)0;
    } else {
      const Real vx = a.vel[n], vy = a.vel[a.plane + n];
      const Real u = u0 ? (Real)u0[(long long)y * a.nx + x] : (Real)0;
      Real f[9];
      equilibrium(f, u, vx, vy);
      const uint32_t post = (w >> kUpPostShift) & 0xFFu;
      const bool near_solid = post != 0u;
      const Real wsolid = (Real)__popc(post & 0x0Fu) * (Real)w_of(1) +
                          (Real)__popc(post & 0xF0u) * (Real)w_of(5);
      Real kr = (Real)0;
      if (a.react_mode == kReactBulk || (a.react_mode == kReactSurface && near_solid))
        kr = a.kf ? a.kf[n] : a.k_scalar;
      collide(f, u, vx, vy, a.omega, kr);
#pragma unroll
      for (int i = 0; i < 9; ++i)
        store_node(a.fout + i * a.plane, n, f[i], ghosts, x, y, a.nx, a.ny, a.pitch,
                   a.per_x, a.per_y, a.plane, a.status);
      if (a.dissolution && near_solid)
        store_node(a.ureact, n, kr * u / wsolid, ghosts, x, y, a.nx, a.ny, a.pitch,
                   a.per_x, a.per_y, a.plane, a.status);
      a.u_out[n] = u;
      my_u = (double)u;
    }
  }
  const double s = block_sum(my_u, red);
  if (threadIdx.x == 0 && threadIdx.y == 0)
    a.partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

struct DissolveArgs {
  uint32_t* link;
  double* mineral;       // dense [rows][pitch] mineral (nodes not on the list)
  int* slist;            // surface list: padded node index per entry
  double* smin;          // surface list: mineral per entry
  int* scount;           // surface list length
  int* flip_list;        // padded indices of nodes found exhausted this pass
  int* flip_count;
  unsigned* done;
  long long* flips_total;
  int* status;    // the context's status word (index checks of the debug build)
  int nx, ny, pitch, per_x, per_y;
  int check_all;  // also flip untouched solid nodes whose mineral is <= 0
};

__device__ __forceinline__ void node_xy(const DissolveArgs& d, int n, int& x, int& y) {
  y = n / d.pitch - kYO;
  x = n - (y + kYO) * d.pitch - kXO;
}

// Padded index of the in-lattice neighbour z = (x, y) + e_i, or -1.
__device__ __forceinline__ int neighbour(const DissolveArgs& d, int x, int y, int i) {
  int zx = x + cx_of(i), zy = y + cy_of(i);
  if (zx < 0 || zx >= d.nx) {
    if (!d.per_x) return -1;
    zx = zx < 0 ? zx + d.nx : zx - d.nx;
  }
  if (zy < 0 || zy >= d.ny) {
    if (!d.per_y) return -1;
    zy = zy < 0 ? zy + d.ny : zy - d.ny;
  }
  return (zy + kYO) * d.pitch + (zx + kXO);
}

// Atomically clear bit `shift + i - 1` in the link word of every in-lattice
// neighbour z = y + e_i of node (x, y), i.e. the bit that describes y as z's
// upstream node in direction i.
__device__ __forceinline__ void clear_in_neighbours(const DissolveArgs& d, int x, int y,
                                                    int shift) {
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int z = neighbour(d, x, y, i);
    if (z >= 0) atomicAnd(d.link + z, ~up_bit(shift, i));
  }
}

// Mineral lost by solid node n this step (word w): sum over its fluid
// (after this step's flips) in-lattice neighbours s = y - e_j of w_j r(s),
// r(s) = k(s) u(s) / W_s(s) stored by the step.  Summed in the working
// precision in a fixed order; FP64 throughput is scarce and the result only
// enters the FP64 mineral.
template <typename Real>
__device__ __forceinline__ Real mineral_take(const Real* __restrict__ rlink, long long n,
                                             const DissolveArgs& d, uint32_t fluid) {
  const long long plane = (long long)d.pitch * padded_rows(d.ny);
  Real take = (Real)0;
#pragma unroll
  for (int j = 1; j < 9; ++j)
    if (fluid & (1u << (j - 1)))
      take += (Real)w_of(j) *
              rlink[dbg_idx(n - cx_of(j) - (long long)cy_of(j) * d.pitch, plane, d.status,
                            kSiteShare)];
  return take;
}

// Mark every node of the flip list pending (solid for the next streaming,
// fluid for its collision), tell its neighbours through their post-flip bits,
// and put solid neighbours it exposes on the surface list.  Run by one block
// after every node has been examined.
__device__ inline void apply_flips(const DissolveArgs& d, int tid, int nthreads) {
  __threadfence();
  const int cnt = *((volatile int*)d.flip_count);
  for (int k = tid; k < cnt; k += nthreads) {
    const int n = ((volatile int*)d.flip_list)[k];
    int x, y;
    node_xy(d, n, x, y);
    atomicOr(d.link + n, kOwnPending);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const int z = neighbour(d, x, y, i);
      if (z < 0) continue;
      const uint32_t old = atomicAnd(d.link + z, ~up_bit(kUpPostShift, i));
      if ((old & kOwnSolid) && !(old & kListed) &&
          !(atomicOr(d.link + z, kListed) & kListed)) {
        const long long slot =
            dbg_idx(atomicAdd(d.scount, 1), (long long)d.nx * d.ny, d.status, kSiteList);
        d.slist[slot] = z;
        d.smin[slot] = d.mineral[z];
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    *d.flips_total += cnt;
    *d.flip_count = 0;
    *d.done = 0u;
  }
}

// Dissolution after a step, for the solid nodes on the surface list: each
// gathers the mineral it loses (mineral_take); nodes that turned fluid
// before this step's collision (pending) become plain fluid and stop being
// solid upstream for their neighbours; nodes whose mineral is used up are
// collected and, by the last block to finish, marked pending (apply_flips).
// Link-word edits are atomic bit operations on bits no concurrent reader of
// the same word depends on, so the result is independent of timing.
constexpr int kDThreads = 256;

template <typename Real>
__global__ void __launch_bounds__(kDThreads)
    lbm_dissolve_list(const DissolveArgs d, const Real* __restrict__ rlink) {
  const int tid = threadIdx.x;
  bool flipped = false;
  const int count = *d.scount;
  for (int e = blockIdx.x * kDThreads + tid; e < count; e += gridDim.x * kDThreads) {
    const int n = d.slist[e];
    const uint32_t w = d.link[n];
    if (!(w & kOwnSolid)) continue;  // dissolved earlier
    if (w & kOwnPending) {
      int x, y;
      node_xy(d, n, x, y);
      atomicAnd(d.link + n, ~(kOwnSolid | kOwnPending | kListed));
      clear_in_neighbours(d, x, y, kUpSolidShift);
      continue;
    }
    const uint32_t fluid = ~((w >> kUpPostShift) | (w >> kUpOutShift)) & 0xFFu;
    if (!fluid) continue;
    const double m = d.smin[e] - (double)mineral_take(rlink, n, d, fluid);
    d.smin[e] = m;
    if (m <= 0.0) {
      d.flip_list[dbg_idx(atomicAdd(d.flip_count, 1), (long long)d.nx * d.ny, d.status, kSiteList)] = n;
      flipped = true;
    }
  }
  __shared__ bool last;
  if (flipped) __threadfence();
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    last = (atomicAdd(d.done, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) apply_flips(d, tid, kDThreads);
}

// Dissolution pass over every node (used once, after initialisation): the
// same update as lbm_dissolve_list for surface nodes, and with check_all set
// it also flips solid nodes given no mineral.  The mineral is the dense array.
template <typename Real>
__global__ void __launch_bounds__(kDThreads)
    lbm_dissolve_dense(const DissolveArgs d, const Real* __restrict__ rlink) {
  const int tid = threadIdx.x;
  bool flipped = false;
  const long long total = (long long)d.nx * d.ny;
  for (long long id = blockIdx.x * (long long)kDThreads + tid; id < total;
       id += (long long)gridDim.x * kDThreads) {
    const int y = (int)(id / d.nx), x = (int)(id - (long long)y * d.nx);
    const int n = (y + kYO) * d.pitch + (x + kXO);
    const uint32_t w = d.link[n];
    if (!(w & kOwnSolid)) continue;
    if (w & kOwnPending) {
      atomicAnd(d.link + n, ~(kOwnSolid | kOwnPending | kListed));
      clear_in_neighbours(d, x, y, kUpSolidShift);
      continue;
    }
    const uint32_t fluid = ~((w >> kUpPostShift) | (w >> kUpOutShift)) & 0xFFu;
    if (!fluid && !d.check_all) continue;
    const double m = d.mineral[n] - (double)mineral_take(rlink, n, d, fluid);
    if (fluid) d.mineral[n] = m;
    if (m <= 0.0) {
      d.flip_list[dbg_idx(atomicAdd(d.flip_count, 1), (long long)d.nx * d.ny, d.status, kSiteList)] = n;
      flipped = true;
    }
  }
  __shared__ bool last;
  if (flipped) __threadfence();
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    last = (atomicAdd(d.done, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) apply_flips(d, tid, kDThreads);
}

// Build the surface list: every solid node with a fluid in-lattice neighbour
// (or pending) that is not listed yet; its mineral moves to the list.
static __global__ void __launch_bounds__(kDThreads) lbm_list_build(const DissolveArgs d) {
  const long long total = (long long)d.nx * d.ny;
  for (long long id = blockIdx.x * (long long)kDThreads + threadIdx.x; id < total;
       id += (long long)gridDim.x * kDThreads) {
    const int y = (int)(id / d.nx), x = (int)(id - (long long)y * d.nx);
    const int n = (y + kYO) * d.pitch + (x + kXO);
    const uint32_t w = d.link[n];
    if (!(w & kOwnSolid) || (w & kListed)) continue;
    const uint32_t fluid = ~((w >> kUpPostShift) | (w >> kUpOutShift)) & 0xFFu;
    if (!fluid && !(w & kOwnPending)) continue;
    d.link[n] = w | kListed;
    const int slot = atomicAdd(d.scount, 1);
    d.slist[slot] = n;
    d.smin[slot] = d.mineral[n];
  }
}

// Write the list's minerals back into the dense array (before read-out).
static __global__ void lbm_list_scatter(const DissolveArgs d) {
  const int count = *d.scount;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
    d.mineral[d.slist[e]] = d.smin[e];
}

}  // namespace lbm
