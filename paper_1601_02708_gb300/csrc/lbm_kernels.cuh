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

// Rows per block of the plain step kernel (lbm_step).  FP32: 2, so 24
// blocks of 64 threads share an SM: measured 221 against 225 us a launch at
// 4096^2 with 32 x 8 blocks (32 x 16 blocks: 237 us), with the same warps
// active and the same DRAM bytes but DRAM busier (61 against 59% of peak in
// a 2048^2 capture).  FP64: 8, since its interior blocks pack their
// updating nodes into the first lanes, which larger blocks do better (1.40
// against 1.46 ms at 32 x 4).
template <typename Real>
__host__ __device__ constexpr int step_rows() {
  return sizeof(Real) == 4 ? 2 : 8;
}

template <typename Real>
struct StepArgs {
  const Real* __restrict__ fin;  // f* of the previous step
  Real* __restrict__ fout;       // f* of this step
  const uint32_t* __restrict__ link;  // [rows][pitch] link words
  const Real* __restrict__ vel;  // [2][rows][pitch]
  const Real* __restrict__ kf;   // [rows][pitch] or null
  Real* __restrict__ u_out;      // [rows][pitch], written on the final substep
  Real* __restrict__ u_hist;     // [rows][pitch], written every step if not null
                                 // (the adjoint's recomputation)
  void* __restrict__ ureact;     // [rows][pitch] reaction shares at near-solid nodes
                                 // (dissolution): FP64 lattice r = k u / W_s (double);
                                 // FP32 lattice {u, 36 W_s} (ShareF32), r formed in FP64
  const double* __restrict__ ua;  // edge data, start of the coarse step
  const double* __restrict__ ub;  // edge data, end of the coarse step
  const double* __restrict__ q;   // Neumann data
  long long* __restrict__ infeasible;  // per edge slot
  double* __restrict__ jnode;          // per east-edge row: sum_t u
  double* __restrict__ jflux;          // per east-edge row: first moment sum_i f_i e_ix
                                       // at x = nx - 1 of the last step (or null)
  double* __restrict__ partial;        // per block: sum u (final substep)
  int* __restrict__ status;            // device error word (0 = fine)
  unsigned char* __restrict__ bc_root;  // per edge slot: 1 where the Neumann root
                                        // set the unknowns this step (or null)
  long long* __restrict__ wall_infeasible;  // count of wall solves without a root
  long long* __restrict__ newton_fail;      // count of wall solves short of the tolerance
  const int* __restrict__ open_nodes;  // padded indices of the nodes on non-periodic
                                       // sides (boundary warp of the tile pipeline)
  int n_open;
  int open_mask;    // bit s: side s (W, E, S, N) is a Dirichlet or Neumann side
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

// Reaction share of a near-solid node of the FP32 lattice: its concentration
// as stored by the lattice and 36 W_s = 4 (axis links to solid) + (diagonal
// links to solid), an integer in 1 .. 20.  The dissolution pass forms
// k u / W_s from it in FP64.
struct alignas(8) ShareF32 {
  float u;
  uint32_t w36;
};

// Whether interior node (x, y) lies on a Dirichlet or Neumann side (bit s of
// open_mask for side W, E, S, N): its populations pulled from outside the
// lattice are set by a boundary solve.  Periodic sides and the sides a slab
// shares with its neighbours (exchange sides) are not open.
__device__ __forceinline__ bool on_open_side(int x, int y, int nx, int ny, int open_mask) {
  return ((open_mask & 1) && x == 0) || ((open_mask & 2) && x == nx - 1) ||
         ((open_mask & 4) && y == 0) || ((open_mask & 8) && y == ny - 1);
}

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
  // the factors that do not depend on the direction, formed once
  const Real sym0 = omega * base - kr;
  const Real c45 = (Real)4.5 * omega;
  const Real c3 = (Real)3 * omega;
  const Real ev[4] = {vx, vy, vx + vy, vy - vx};  // e.v of directions 1, 2, 5, 6
  Real rest = u - kr * u;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = p < 2 ? p + 1 : p + 3;  // 1, 2, 5, 6; opposites 3, 4, 7, 8
    const int o = opp_of(i);
    const Real wu = (Real)w_of(i) * u;
    const Real sym = wu * (c45 * (ev[p] * ev[p]) + sym0);
    const Real anti = (wu * c3) * ev[p];
    f[i] = om1 * f[i] + (sym + anti);
    f[o] = om1 * f[o] + (sym - anti);
    rest -= f[i] + f[o];
  }
  f[0] = rest;
}

// Store a node value and, at nodes on a periodic side, its ghost images.
template <typename T>
__device__ __forceinline__ void store_node(T* __restrict__ base, long long n, T v,
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

// Reaction share of a near-solid node, stored for the dissolution pass:
// r = k u / W_s on the FP64 lattice; the concentration and 36 W_s on the FP32
// lattice (the pass forms r in FP64).  `post` holds the node's links to solid
// neighbours after this step's flips; post = 0 stores a zero share.
template <typename Real>
__device__ __forceinline__ void store_share(const StepArgs<Real>& a, long long n, Real kr,
                                            Real u, uint32_t post, bool ghosts, int x, int y) {
  const int na = __popc(post & 0x0Fu), nd = __popc(post & 0xF0u);
  if constexpr (sizeof(Real) == 8) {
    const double wsolid = (double)na * w_of(1) + (double)nd * w_of(5);
    store_node((double*)a.ureact, n, post ? (double)kr * (double)u / wsolid : 0.0, ghosts, x, y,
               a.nx, a.ny, a.pitch, a.per_x, a.per_y, a.plane, a.status);
  } else {
    ShareF32 v;
    v.u = (float)u;
    v.w36 = (uint32_t)(4 * na + nd);
    store_node((ShareF32*)a.ureact, n, v, ghosts, x, y, a.nx, a.ny, a.pitch, a.per_x, a.per_y,
               a.plane, a.status);
  }
}

// One node's step.  (x, y) interior coordinates, n its padded index.  Writes
// f* (and ghost images), ureact, jnode, jflux, u_out; returns u (0 at solid
// nodes) for the mass reduction.
// kEdge false: the caller guarantees the node is at least one node away
// from every side, so no pull leaves the lattice, no ghost image exists and
// the node is not on the outlet; the boundary code is then compiled out.
// kSolve: the node may lie on a non-periodic side, whose populations pulled
// from outside are set by the maximum-entropy conditions (in FP64 on either
// lattice); callers that route those nodes elsewhere compile the solves out.
// kWalls: 0, the kernel carries no wall code; 1, maximum-entropy pore walls
// (when a.wall_maxent) solved in the lattice's precision; 2, solved in FP64.
// kLight: the node's inputs are cheap to read (a shared-memory tile), so a
// solid lane runs the fluid lanes' arithmetic on its (finite) inputs and
// discards it: the warp takes one path and issues one set of stores, where
// mixed solid and fluid lanes would otherwise split it in two.  Results are
// the same either way.
// kClear (with !kEdge): the caller has checked that the node is fluid with
// no solid neighbour before or after this step's flips (its link word is
// zero in kClearMask), so the bounce-back, wall, share and solid-lane code is
// compiled out.  Results are the same as without it.
template <typename Real, bool kFinal, bool kEdge, bool kSolve, int kWalls, bool kLight = false,
          bool kClear = false, class Src>
__device__ __forceinline__ double step_node(const StepArgs<Real>& a, const Src& src,
                                            int x, int y, long long n, double frac) {
  static_assert(!(kClear && kEdge), "the clear path is for interior nodes");
  const uint32_t w = kClear ? 0u : src.word();
  const bool ghosts =
      kEdge && ((x == 0) | (x == a.nx - 1) | (y == 0) | (y == a.ny - 1)) &&
      (a.per_x | a.per_y);
  // Solid nodes hold no populations, but a solid node whose 32-byte sector
  // (8 FP32 nodes, aligned since kXO = 8) holds fluid nodes writes zeros, so
  // every sector the warp touches is written whole.  A node that turns
  // fluid before this step collides (pending) gets zero populations anyway.
  const bool own_solid = (w & kOwnSolid) != 0u;
  const bool pending = (w & kOwnPending) != 0u;
  const bool solid = own_solid && !pending;
  const unsigned fluid_lanes = kClear ? 0xFFFFFFFFu : __ballot_sync(__activemask(), !solid);
  const unsigned lane = threadIdx.x & 31u;
  const bool fill = ((fluid_lanes >> (lane & 24u)) & 0xFFu) != 0u;
  if (!kLight && own_solid) {
    if (pending || (sizeof(Real) == 4 && fill)) {
#pragma unroll
      for (int i = 0; i < 9; ++i)
        store_node(a.fout + i * a.plane, n, (Real)0, ghosts, x, y, a.nx, a.ny, a.pitch,
                   a.per_x, a.per_y, a.plane, a.status);
      if (a.dissolution && pending) store_share(a, n, (Real)0, (Real)0, 0u, ghosts, x, y);
    }
    if (kFinal) a.u_out[dbg_idx(n, a.plane, a.status, kSiteNode)] = (Real)0;
    if (a.u_hist) a.u_hist[dbg_idx(n, a.plane, a.status, kSiteNode)] = (Real)0;
    return 0.0;
  }
  Real f[9];
  f[0] = src.own(0);
#pragma unroll
  for (int i = 1; i < 9; ++i) f[i] = src.pull_or_bounce(i, w & up_bit(kUpSolidShift, i));
  // pore walls of the maximum-entropy kind, at nodes off the open lattice
  // sides (those keep bounce-back at their solid links)
  if (kWalls != 0 && a.wall_maxent && !own_solid && (w & 0xFFu) &&
      !(w & (0xFFu << kUpOutShift))) {
    const int r = kWalls == 2 ? maxent_wall<double>(f, (w & 0xFFu) << 1)
                              : maxent_wall<Real>(f, (w & 0xFFu) << 1);
    if (r == kWallNoRoot)
      atomicAdd(reinterpret_cast<unsigned long long*>(a.wall_infeasible), 1ull);
    else if (r == kWallNoConv)
      atomicAdd(reinterpret_cast<unsigned long long*>(a.newton_fail), 1ull);
  }
  if (kEdge && kSolve && !own_solid) {
    const unsigned unknown = ((w >> kUpOutShift) & 0xFFu) << 1;  // bit i: direction i
    if (unknown) {
      // Boundary node: Dirichlet wins at corners, else Neumann.  The solves
      // run in FP64 from the FP64 edge data on either lattice; only their
      // results are rounded to the lattice's precision.
      int dside, nside, sx, sy;
      edge_kind(a.edge, x, y, a.nx, a.ny, &dside, &nside, &sx, &sy);
      bool bad;
      int slot;
      if (dside >= 0) {
        slot = edge_slot(dside, x, y, a.nx, a.ny);
        const double up = (1.0 - frac) * a.ua[slot] + frac * a.ub[slot];
        bad = maxent_dirichlet(f, unknown, up);
      } else {
        slot = edge_slot(nside, x, y, a.nx, a.ny);
        Real fbb[9];
#pragma unroll
        for (int i = 0; i < 9; ++i)
          fbb[i] = (unknown & (1u << opp_of(i))) ? src.own(i) : (Real)0;
        const int how = maxent_neumann(f, unknown, sx, sy, a.q[slot], fbb);
        bad = how == kNeuInfeasible;
        if (a.bc_root) a.bc_root[slot] = how == kNeuRoot;
      }
      if (bad) atomicAdd(reinterpret_cast<unsigned long long*>(a.infeasible + slot), 1ull);
    }
  }
  Real u = f[0];
#pragma unroll
  for (int i = 1; i < 9; ++i) u += f[i];
  // the first moment through the east column (outlet flux of lbm_diagnostics)
  if (kEdge && x == a.nx - 1 && a.jflux && !own_solid)
    a.jflux[y] = ((double)f[1] + (double)f[5] + (double)f[8]) -
                 ((double)f[3] + (double)f[6] + (double)f[7]);
  // links to solid neighbours after this step's flips: axis links weigh 1/9,
  // diagonal links 1/36
  const uint32_t post = (w >> kUpPostShift) & 0xFFu;
  const bool near_solid = post != 0u;
  Real kr = (Real)0;
  if (a.react_mode == kReactBulk || (a.react_mode == kReactSurface && near_solid))
    kr = a.kf ? src.kf() : a.k_scalar;
  collide(f, u, src.vx(), src.vy(), a.omega, kr);
  if (kLight && own_solid) {  // a solid lane: zeros (pending), or nothing to keep
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = (Real)0;
    u = (Real)0;
  }
  if (!kLight || !own_solid || pending || (sizeof(Real) == 4 && fill)) {
#pragma unroll
    for (int i = 0; i < 9; ++i)
      store_node(a.fout + i * a.plane, n, f[i], ghosts, x, y, a.nx, a.ny, a.pitch,
                 a.per_x, a.per_y, a.plane, a.status);
  }
  // what this node takes from its solid neighbours (dissolution pass); a
  // pending node's share is zero
  if (a.dissolution) {
    if (kLight && pending) store_share(a, n, (Real)0, (Real)0, 0u, ghosts, x, y);
    else if (!own_solid && near_solid) store_share(a, n, kr, u, post, ghosts, x, y);
  }
  // one node per row adds to its row's sum: a reduction without a read-back
  if (kEdge && x == a.nx - 1 && !own_solid) atomicAdd(a.jnode + y, (double)u);
  if (kFinal) a.u_out[dbg_idx(n, a.plane, a.status, kSiteNode)] = u;
  if (a.u_hist) a.u_hist[dbg_idx(n, a.plane, a.status, kSiteNode)] = u;
  return (double)u;
}

// True when the warp's 32 consecutive nodes (xs .. xs + 31, row y) all lie
// one node or more inside every side of the lattice: the boundary code can
// be skipped for the whole warp (the test is warp-uniform).
__device__ __forceinline__ bool group_is_interior(int xs, int y, int nx, int ny) {
  return xs >= 1 && xs + 32 <= nx - 1 && y >= 1 && y <= ny - 2;
}

// Inputs of an interior node fetched from global memory in one round: the
// link word, both candidates of every streamed population (the one pulled
// from x - e_i and the node's own opposite one, for bounce-back) and the
// velocity and rate, none of the loads waiting for the link word, which
// then picks between the candidates.
template <typename Real>
struct PreSrc {
  uint32_t w;
  Real f[9];
  Real vx_, vy_, kf_;
  __device__ __forceinline__ uint32_t word() const { return w; }
  __device__ __forceinline__ Real own(int i) const { return f[i]; }  // i = 0 only
  __device__ __forceinline__ Real pull_or_bounce(int i, bool) const { return f[i]; }
  __device__ __forceinline__ Real vx() const { return vx_; }
  __device__ __forceinline__ Real vy() const { return vy_; }
  __device__ __forceinline__ Real kf() const { return kf_; }
  __device__ __forceinline__ ShareF32* keep_ptr() const { return nullptr; }
};
template <typename Real>
__device__ __forceinline__ PreSrc<Real> preload(const StepArgs<Real>& a, long long n) {
  const long long lim = 9 * a.plane;
  PreSrc<Real> p;
  Real own[9], pul[9];
  p.w = a.link[dbg_idx(n, a.plane, a.status, kSiteNode)];
#pragma unroll
  for (int i = 0; i < 9; ++i) own[i] = a.fin[dbg_idx(i * a.plane + n, lim, a.status, kSitePull)];
#pragma unroll
  for (int i = 1; i < 9; ++i)
    pul[i] = a.fin[dbg_idx(i * a.plane + n - cx_of(i) - (long long)cy_of(i) * a.pitch, lim,
                           a.status, kSitePull)];
  p.vx_ = a.vel[dbg_idx(n, a.plane, a.status, kSiteNode)];
  p.vy_ = a.vel[dbg_idx(a.plane + n, 2 * a.plane, a.status, kSiteNode)];
  p.kf_ = a.kf ? a.kf[dbg_idx(n, a.plane, a.status, kSiteNode)] : (Real)0;
  p.f[0] = own[0];
#pragma unroll
  for (int i = 1; i < 9; ++i) p.f[i] = (p.w & up_bit(kUpSolidShift, i)) ? own[opp_of(i)] : pul[i];
  return p;
}

// Generic step: one thread per node, inputs from global memory.  The FP64
// lattice's step, and the FP32 one on large lattices (lbm_set_kernel).
template <typename Real, bool kFinal, int kWalls = 0>
// FP32: 24 blocks of 64 per SM (40 registers, as many threads as six blocks
// of 256) keep more loads in flight than fewer threads; FP64 keeps four
// blocks of 256 (64 registers) for its arithmetic.
__global__ void __launch_bounds__(kBX * step_rows<Real>(), sizeof(Real) == 4 ? 24 : 4)
    lbm_step(const StepArgs<Real> a) {
  constexpr int kBY = step_rows<Real>();
  __shared__ double red[kBX * kBY / 32];
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  double my_u = 0.0;
  const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY;
  if (sizeof(Real) == 8 && x0 >= 1 && x0 + kBX <= a.nx - 1 && y0 >= 1 && y0 + kBY <= a.ny - 1) {
    // FP64 lattice, a block one node inside every side: the FP64 pipe (1/64
    // of the FP32 rate on this part) bounds the update, so the block's nodes
    // that update (fluid, or turning fluid) are packed into the first lanes
    // and solid lanes do not occupy it
    __shared__ unsigned short list[kBX * kBY];
    __shared__ int wcount[kBX * kBY / 32];
    const int tid = threadIdx.y * kBX + threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long n = (long long)(y + kYO) * a.pitch + (x + kXO);
    const uint32_t w = a.link[dbg_idx(n, a.plane, a.status, kSiteNode)];
    const bool active = !(w & kOwnSolid) || (w & kOwnPending);
    if (!active) {
      if (kFinal) a.u_out[dbg_idx(n, a.plane, a.status, kSiteNode)] = (Real)0;
      if (a.u_hist) a.u_hist[dbg_idx(n, a.plane, a.status, kSiteNode)] = (Real)0;
    }
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, active);
    if (lane == 0) wcount[wid] = __popc(bal);
    __syncthreads();
    int off = 0, total = 0;
#pragma unroll
    for (int k = 0; k < kBX * kBY / 32; ++k) {
      off += k < wid ? wcount[k] : 0;
      total += wcount[k];
    }
    if (active) list[off + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)tid;
    __syncthreads();
    if (tid < total) {
      const int t = list[tid];
      const int xx = x0 + (t % kBX), yy = y0 + (t / kBX);
      const long long nn = (long long)(yy + kYO) * a.pitch + (xx + kXO);
      const PreSrc<Real> src = preload(a, nn);
      my_u = step_node<Real, kFinal, false, false, kWalls>(a, src, xx, yy, nn, a.frac);
    }
  } else if (x < a.nx && y < a.ny) {
    const long long n = (long long)(y + kYO) * a.pitch + (x + kXO);
    if (group_is_interior(blockIdx.x * kBX, y, a.nx, a.ny)) {
      // the warp's class by its link words: all clear of solids, all solid
      // (u only), or general (solid lanes compute on their finite inputs and
      // discard the result, so the warp takes one path)
      // (FP32 only: the FP64 lattice's interior blocks are packed above, and
      // its other nodes keep the one path that the batch's FP64 kernels share)
      const PreSrc<Real> src = preload(a, n);
      if (sizeof(Real) == 8)
        my_u = step_node<Real, kFinal, false, false, kWalls>(a, src, x, y, n, a.frac);
      else if (__all_sync(0xFFFFFFFFu, (src.w & kClearMask) == 0u))
        my_u = step_node<Real, kFinal, false, false, kWalls, true, true>(a, src, x, y, n, a.frac);
      else if (__all_sync(0xFFFFFFFFu, (src.w & (kOwnSolid | kOwnPending)) == kOwnSolid)) {
        if (kFinal) a.u_out[dbg_idx(n, a.plane, a.status, kSiteNode)] = (Real)0;
        if (a.u_hist) a.u_hist[dbg_idx(n, a.plane, a.status, kSiteNode)] = (Real)0;
      } else
        my_u = step_node<Real, kFinal, false, false, kWalls, true>(a, src, x, y, n, a.frac);
    } else {
      GlobalSrc<Real> src{a, n};
      my_u = step_node<Real, kFinal, true, true, kWalls>(a, src, x, y, n, a.frac);
    }
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
      Real kr = (Real)0;
      if (a.react_mode == kReactBulk || (a.react_mode == kReactSurface && near_solid))
        kr = a.kf ? a.kf[n] : a.k_scalar;
      collide(f, u, vx, vy, a.omega, kr);
#pragma unroll
      for (int i = 0; i < 9; ++i)
        store_node(a.fout + i * a.plane, n, f[i], ghosts, x, y, a.nx, a.ny, a.pitch,
                   a.per_x, a.per_y, a.plane, a.status);
      if (a.dissolution && near_solid) store_share(a, n, kr, u, post, ghosts, x, y);
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
  int* pass;             // passes run so far (the first, after initialisation, is 0)
  int* flip_step;        // [rows][pitch]: pass that turned the node fluid, -1 if none
  long long* flips_total;
  int* status;    // the context's status word (index checks of the debug build)
  const float* kf32;  // FP32 lattice with a rate field: k per node (else null)
  double k_scalar;    // FP32 lattice without a rate field: k
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

// A pending node (found exhausted by the previous pass, fluid since this
// step's collision) becomes plain fluid: it stops being solid upstream for
// its neighbours, and the pass that turned it fluid is recorded.
__device__ __forceinline__ void finish_flip(const DissolveArgs& d, int n, int pass) {
  int x, y;
  node_xy(d, n, x, y);
  atomicAnd(d.link + n, ~(kOwnSolid | kOwnPending | kListed));
  clear_in_neighbours(d, x, y, kUpSolidShift);
  if (d.flip_step) d.flip_step[n] = pass;
}

// Mineral lost by solid node n this step (word w): sum over its fluid (after
// this step's flips) in-lattice neighbours s = y - e_j of w_j r(s),
// r(s) = k(s) u(s) / W_s(s), in FP64 and a fixed order.
// FP64 lattice: r(s) was stored by the step.
__device__ __forceinline__ double mineral_take(const double* __restrict__ r, long long n,
                                               const DissolveArgs& d, uint32_t fluid,
                                               const double*) {
  const long long plane = (long long)d.pitch * padded_rows(d.ny);
  double take = 0.0;
#pragma unroll
  for (int j = 1; j < 9; ++j)
    if (fluid & (1u << (j - 1)))
      take += w_of(j) * r[dbg_idx(n - cx_of(j) - (long long)cy_of(j) * d.pitch, plane,
                                  d.status, kSiteShare)];
  return take;
}
// FP32 lattice: the step stored u(s) and c = 36 W_s(s); with T[t][c] = 36 w_t / c
// (t = 0 axis, 1 diagonal direction) w_j r(s) = k(s) u(s) T[t_j][c].  GB300
// runs FP64 at 1/64 of the FP32 rate, so the terms and their sum are formed
// in double-float arithmetic on the FP32 pipe -- T as an unevaluated float
// pair, each product by Dekker's splitting with a fused multiply-add, the
// sum by Knuth's two-sum -- carrying about 48 significant bits (relative
// error near 1e-14), and only the final sum is converted and scaled by k in
// FP64.  With a rate field each term is scaled in FP64.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ void two_sum_add(float& s, float& e, float a) {
  const float t = s + a;
  const float bp = t - s;
  e += (s - (t - bp)) + (a - bp);
  s = t;
}
__device__ __forceinline__ double mineral_take(const ShareF32* __restrict__ sh, long long n,
                                               const DissolveArgs& d, uint32_t fluid,
                                               const double* tab) {
  const long long plane = (long long)d.pitch * padded_rows(d.ny);
  const F2* tf = reinterpret_cast<const F2*>(tab + 42);  // the float pairs of T
  if (d.kf32) {
    double take = 0.0;
#pragma unroll
    for (int j = 1; j < 9; ++j)
      if (fluid & (1u << (j - 1))) {
        const long long s = dbg_idx(n - cx_of(j) - (long long)cy_of(j) * d.pitch, plane,
                                    d.status, kSiteShare);
        const ShareF32 v = sh[s];
        take += (double)v.u * tab[(j >= 5 ? 21 : 0) + (int)dbg_idx(v.w36, 21, d.status, kSiteShare)] *
                (double)d.kf32[s];
      }
    return take;
  }
  float S = 0.f, E = 0.f;
#pragma unroll
  for (int j = 1; j < 9; ++j)
    if (fluid & (1u << (j - 1))) {
      const long long s = dbg_idx(n - cx_of(j) - (long long)cy_of(j) * d.pitch, plane,
                                  d.status, kSiteShare);
      const ShareF32 v = sh[s];
      const F2 t = tf[(j >= 5 ? 21 : 0) + (int)dbg_idx(v.w36, 21, d.status, kSiteShare)];
      const float p = v.u * t.hi;
      const float err = fmaf(v.u, t.hi, -p) + v.u * t.lo;  // u T - p, to ~2^-48 of u T
      two_sum_add(S, E, p);
      E += err;
    }
  return ((double)S + (double)E) * d.k_scalar;
}

// The tables of mineral_take for the FP32 lattice: tab[t][c] = 36 w_t / c
// in FP64 (36 w_t = 4 axis, 1 diagonal; tab[t][0] = 0), then the same 42
// values as float pairs hi + lo (hi the float nearest, lo the float nearest
// the remainder).  Computed by the compiler (IEEE division and conversions,
// as on the device) into device memory, so no block spends time building
// them; share_table() returns them as 84 doubles of storage.
struct ShareTab {
  double d[42];
  F2 f[42];
};
constexpr ShareTab make_share_tab() {
  ShareTab t{};
  for (int i = 0; i < 42; ++i) {
    const int c = i % 21;
    const double v = c == 0 ? 0.0 : (i < 21 ? 4.0 : 1.0) / (double)c;
    t.d[i] = v;
    const float hi = (float)v;
    t.f[i] = F2{hi, (float)(v - (double)hi)};
  }
  return t;
}
__device__ const ShareTab kShareTab = make_share_tab();
static_assert(sizeof(ShareTab) == 84 * sizeof(double), "tables of 84 doubles");
__device__ __forceinline__ const double* share_table() {
  return reinterpret_cast<const double*>(&kShareTab);
}

// Mark every node of the flip list pending (solid for the next streaming,
// fluid for its collision), tell its neighbours through their post-flip bits,
// and put solid neighbours it exposes on the surface list.  Run by one block
// after every node has been examined; it closes the pass.
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
    *d.pass += 1;
  }
}

// Dissolution after a step, for the solid nodes on the surface list: each
// gathers the mineral it loses (mineral_take); nodes that turned fluid
// before this step's collision (pending) become plain fluid and stop being
// solid upstream for their neighbours; nodes whose mineral is used up are
// collected and, by the last block to finish, marked pending (apply_flips).
// Link-word edits are atomic bit operations on bits no concurrent reader of
// the same word depends on, so the result is independent of timing.
// Share is double (FP64 lattice) or ShareF32 (FP32 lattice).
constexpr int kDThreads = 256;

template <typename Share>
__global__ void __launch_bounds__(kDThreads)
    lbm_dissolve_list(const DissolveArgs d, const Share* __restrict__ rlink) {
  const double* const tab = share_table();
  const int tid = threadIdx.x;
  const int pass = *(volatile int*)d.pass;
  bool flipped = false;
  const int count = *d.scount;
  for (int e = blockIdx.x * kDThreads + tid; e < count; e += gridDim.x * kDThreads) {
    const int n = d.slist[e];
    const uint32_t w = d.link[n];
    if (!(w & kOwnSolid)) continue;  // dissolved earlier
    if (w & kOwnPending) {
      finish_flip(d, n, pass);
      continue;
    }
    const uint32_t fluid = ~((w >> kUpPostShift) | (w >> kUpOutShift)) & 0xFFu;
    if (!fluid) continue;
    const double m = d.smin[e] - mineral_take(rlink, n, d, fluid, tab);
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
template <typename Share>
__global__ void __launch_bounds__(kDThreads)
    lbm_dissolve_dense(const DissolveArgs d, const Share* __restrict__ rlink) {
  const double* const tab = share_table();
  const int tid = threadIdx.x;
  const int pass = *(volatile int*)d.pass;
  bool flipped = false;
  const long long total = (long long)d.nx * d.ny;
  for (long long id = blockIdx.x * (long long)kDThreads + tid; id < total;
       id += (long long)gridDim.x * kDThreads) {
    const int y = (int)(id / d.nx), x = (int)(id - (long long)y * d.nx);
    const int n = (y + kYO) * d.pitch + (x + kXO);
    const uint32_t w = d.link[n];
    if (!(w & kOwnSolid)) continue;
    if (w & kOwnPending) {
      finish_flip(d, n, pass);
      continue;
    }
    const uint32_t fluid = ~((w >> kUpPostShift) | (w >> kUpOutShift)) & 0xFFu;
    if (!fluid && !d.check_all) continue;
    const double m = d.mineral[n] - mineral_take(rlink, n, d, fluid, tab);
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
