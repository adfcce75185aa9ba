// lbm_kernels.cuh -- the fused D2Q9 ADE-LBM step and its companions.
//
// State between steps: post-collision populations f* in SoA planes
// [9][ny][pitch] (pitch = nx rounded up to 32 elements), two buffers
// swapped every step.  One step (kernel lbm_step) pulls f_i(x) = f*_i(x - e_i)
// (Eq. "LBE"), replaces pulls from solid nodes by halfway bounce-back, sets
// the populations pulled from outside the lattice by the maximum-entropy
// conditions (Sec. 4.1.1), takes u = sum f (Eq. "LBM_Macro"), and collides
// with the BGK operator (Eq. "Collision", "LBM_feq") plus the first-order
// sink.  The sequence of states equals the paper's collide -> stream -> BC
// order shifted by half a step: the stored f* is what the next stream moves.
#pragma once
#include <cstdint>

#include "lbm_lattice.cuh"

namespace lbm {

constexpr int kBX = 32;  // threads along x per block (one warp per row)
constexpr int kBY = 8;   // rows per block

template <typename Real>
struct StepArgs {
  const Real* __restrict__ fin;  // f* of the previous step
  Real* __restrict__ fout;       // f* of this step
  const uint8_t* __restrict__ mask;
  const Real* __restrict__ vel;  // [2][ny][pitch]
  const Real* __restrict__ kf;   // [ny][pitch] or null
  Real* __restrict__ u_out;      // [ny][pitch], written on the final substep
  Real* __restrict__ ureact;     // [ny][pitch], k u / W_s at reactive nodes (dissolution)
  const double* __restrict__ ua;  // edge data, start of the coarse step
  const double* __restrict__ ub;  // edge data, end of the coarse step
  const double* __restrict__ q;   // Neumann data
  long long* __restrict__ infeasible;  // per edge slot
  double* __restrict__ jnode;          // per east-edge row: sum_t u
  double* __restrict__ partial;        // per block: sum u (final substep)
  long long plane;  // pitch * ny
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

template <typename Real>
__device__ __forceinline__ void collide_store(const Real (&f)[9], Real u, Real vx,
                                              Real vy, Real omega, Real kr,
                                              Real* __restrict__ out, long long plane,
                                              long long n) {
  Real feq[9];
  equilibrium(feq, u, vx, vy);
  const Real sink = kr * u;
  Real sink0 = sink;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const Real si = (Real)w_of(i) * sink;
    sink0 -= si;
    out[i * plane + n] = f[i] + omega * (feq[i] - f[i]) - si;
  }
  out[n] = f[0] + omega * (feq[0] - f[0]) - sink0;
}

template <typename Real, bool kFinal>
__global__ void __launch_bounds__(kBX * kBY)
    lbm_step(const StepArgs<Real> a) {
  __shared__ double red[kBX * kBY / 32];
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  double my_u = 0.0;
  if (x < a.nx && y < a.ny) {
    const long long n = (long long)y * a.pitch + x;
    const uint8_t mk = a.mask[n];
    if (mk & kSolid) {
      if (mk & kPending) {  // became fluid with zero populations
#pragma unroll
        for (int i = 0; i < 9; ++i) a.fout[i * a.plane + n] = (Real)0;
        if (a.dissolution) a.ureact[n] = (Real)0;
      }
      if (kFinal) a.u_out[n] = (Real)0;
    } else {
      Real f[9];
      unsigned unknown = 0;
      bool near_solid = false;
      Real wsolid = (Real)0;  // sum of w_i over links to solid neighbours
      f[0] = a.fin[n];
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        // upstream neighbour x - e_i, wrapped through periodic sides
        int sx = x - cx_of(i), sy = y - cy_of(i);
        bool out = false;
        if (sx < 0) { if (a.per_x) sx += a.nx; else out = true; }
        else if (sx >= a.nx) { if (a.per_x) sx -= a.nx; else out = true; }
        if (sy < 0) { if (a.per_y) sy += a.ny; else out = true; }
        else if (sy >= a.ny) { if (a.per_y) sy -= a.ny; else out = true; }
        if (out) {
          unknown |= 1u << i;
          f[i] = (Real)0;
        } else {
          const long long s = (long long)sy * a.pitch + sx;
          const uint8_t ms = a.mask[s];
          if (solid_post(ms)) {
            near_solid = true;
            wsolid += (Real)w_of(opp_of(i));  // the link x -> x - e_i
          }
          f[i] = (ms & kSolid) ? a.fin[opp_of(i) * a.plane + n]
                               : a.fin[i * a.plane + s];
        }
      }
      if (unknown) {
        // Boundary node: Dirichlet wins at corners, else Neumann.
        const bool on[4] = {x == 0 && a.edge[0] != kPeriodic,
                            x == a.nx - 1 && a.edge[1] != kPeriodic,
                            y == 0 && a.edge[2] != kPeriodic,
                            y == a.ny - 1 && a.edge[3] != kPeriodic};
        int dside = -1, nside = -1, sx = 0, sy = 0;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          if (!on[s]) continue;
          if (a.edge[s] == kDirichlet && dside < 0) dside = s;
          if (a.edge[s] == kNeumann) {
            if (nside < 0) nside = s;
            sx += (s == 0) ? -1 : (s == 1) ? 1 : 0;
            sy += (s == 2) ? -1 : (s == 3) ? 1 : 0;
          }
        }
        bool bad;
        int slot;
        if (dside >= 0) {
          slot = edge_slot(dside, x, y, a.nx, a.ny);
          const double up = (1.0 - a.frac) * a.ua[slot] + a.frac * a.ub[slot];
          bad = maxent_dirichlet(f, unknown, up);
        } else {
          slot = edge_slot(nside, x, y, a.nx, a.ny);
          Real fbb[9];
#pragma unroll
          for (int i = 0; i < 9; ++i)
            fbb[i] = (unknown & (1u << opp_of(i))) ? a.fin[i * a.plane + n] : (Real)0;
          bad = maxent_neumann(f, unknown, sx, sy, a.q[slot], fbb);
        }
        if (bad) a.infeasible[slot] += 1;
        // neighbours across the boundary are not solid; the reactive test
        // already saw every in-lattice neighbour
      }
      Real u = f[0];
#pragma unroll
      for (int i = 1; i < 9; ++i) u += f[i];
      Real kr = (Real)0;
      if (a.react_mode == kReactBulk ||
          (a.react_mode == kReactSurface && near_solid))
        kr = a.kf ? a.kf[n] : a.k_scalar;
      const Real vx = a.vel[n], vy = a.vel[a.plane + n];
      collide_store(f, u, vx, vy, a.omega, kr, a.fout, a.plane, n);
      // mass this node takes from each solid neighbour per unit link weight
      if (a.dissolution && near_solid) a.ureact[n] = kr * u / wsolid;
      if (x == a.nx - 1) a.jnode[y] += (double)u;
      if (kFinal) a.u_out[n] = u;
      my_u = (double)u;
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
template <typename Real>
__global__ void __launch_bounds__(kBX * kBY)
    lbm_init_kernel(const StepArgs<Real> a, const double* __restrict__ u0) {
  __shared__ double red[kBX * kBY / 32];
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  double my_u = 0.0;
  if (x < a.nx && y < a.ny) {
    const long long n = (long long)y * a.pitch + x;
    const uint8_t mk = a.mask[n];
    if (mk & kSolid) {
#pragma unroll
      for (int i = 0; i < 9; ++i) a.fout[i * a.plane + n] = (Real)0;
      a.u_out[n] = (Real)0;
    } else {
      const Real vx = a.vel[n], vy = a.vel[a.plane + n];
      const Real u = u0 ? (Real)u0[(long long)y * a.nx + x] : (Real)0;
      Real f[9];
      equilibrium(f, u, vx, vy);
      bool near_solid = false;
      Real wsolid = (Real)0;
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        int sx = x + cx_of(i), sy = y + cy_of(i);
        bool out = false;
        if (sx < 0) { if (a.per_x) sx += a.nx; else out = true; }
        else if (sx >= a.nx) { if (a.per_x) sx -= a.nx; else out = true; }
        if (sy < 0) { if (a.per_y) sy += a.ny; else out = true; }
        else if (sy >= a.ny) { if (a.per_y) sy -= a.ny; else out = true; }
        if (!out && solid_post(a.mask[(long long)sy * a.pitch + sx])) {
          near_solid = true;
          wsolid += (Real)w_of(i);
        }
      }
      Real kr = (Real)0;
      if (a.react_mode == kReactBulk ||
          (a.react_mode == kReactSurface && near_solid))
        kr = a.kf ? a.kf[n] : a.k_scalar;
      collide_store(f, u, vx, vy, a.omega, kr, a.fout, a.plane, n);
      if (a.dissolution && near_solid) a.ureact[n] = kr * u / wsolid;
      a.u_out[n] = u;
      my_u = (double)u;
    }
  }
  const double s = block_sum(my_u, red);
  if (threadIdx.x == 0 && threadIdx.y == 0)
    a.partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

struct DissolveArgs {
  uint8_t* mask;
  double* mineral;
  int* flip_list;
  int* flip_count;
  unsigned* done;
  long long* flips_total;
  int nx, ny, pitch, per_x, per_y;
  int check_all;  // also flip untouched solid nodes whose mineral is <= 0
};

// Dissolution after a step: every solid node y gathers the mineral it loses,
//   m(y) -= sum_j w_j r(s),  s = y - e_j a fluid neighbour,
// where the step stored r(s) = k(s) u(s) / W_s(s) at every fluid node with a
// solid neighbour (W_s = sum of the weights of s's links to solid nodes), so
// the node's sink k u is shared among its solid links in proportion to w_j.
// The order of the sum is fixed: the result is deterministic.  Nodes that
// turned fluid before this step's collision (kPending) are cleared to fluid;
// nodes whose mineral is used up are collected and, by the last block to
// finish, marked kSolid | kPending: solid for the next step's streaming,
// fluid (with zero populations) for its collision.
template <typename Real>
__global__ void __launch_bounds__(kBX * kBY)
    lbm_dissolve(const DissolveArgs d, const Real* __restrict__ rlink) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  bool flipped = false;
  if (x < d.nx && y < d.ny) {
    const long long n = (long long)y * d.pitch + x;
    const uint8_t mk = d.mask[n];
    if (mk & kPending) {
      d.mask[n] = 0;  // solid_post() reads the same before and after
    } else if (mk & kSolid) {
      double take = 0.0;
      bool touched = false;
#pragma unroll
      for (int j = 1; j < 9; ++j) {
        int sx = x - cx_of(j), sy = y - cy_of(j);
        if (sx < 0) { if (!d.per_x) continue; sx += d.nx; }
        else if (sx >= d.nx) { if (!d.per_x) continue; sx -= d.nx; }
        if (sy < 0) { if (!d.per_y) continue; sy += d.ny; }
        else if (sy >= d.ny) { if (!d.per_y) continue; sy -= d.ny; }
        const long long s = (long long)sy * d.pitch + sx;
        if (solid_post(d.mask[s])) continue;
        take += w_of(j) * (double)rlink[s];
        touched = true;
      }
      if (touched || d.check_all) {
        const double m = d.mineral[n] - take;
        if (touched) d.mineral[n] = m;
        if (m <= 0.0) {
          d.flip_list[atomicAdd(d.flip_count, 1)] = (int)n;
          flipped = true;
        }
      }
    }
  }
  // The last block to finish applies the collected flips.  Only threads that
  // appended to the list need their write ordered before the block's ticket.
  __shared__ bool last;
  if (flipped) __threadfence();
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(d.done, 1u);
    last = (ticket == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int cnt = *((volatile int*)d.flip_count);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int k = tid; k < cnt; k += blockDim.x * blockDim.y)
    d.mask[((volatile int*)d.flip_list)[k]] = kSolid | kPending;
  __syncthreads();
  if (tid == 0) {
    *d.flips_total += cnt;
    *d.flip_count = 0;
    *d.done = 0u;
  }
}

}  // namespace lbm
