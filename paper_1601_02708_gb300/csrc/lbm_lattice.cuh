// lbm_lattice.cuh -- D2Q9 lattice constants and the node-level pieces of the
// step: equilibrium, maximum-entropy boundary solves.  Device code only.
#pragma once
#include <cstdint>

namespace lbm {

// D2Q9: 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE (Sec. 4.1, the
// standard DnQm lattice with c_s^2 = 1/3).  constexpr functions so that the
// fully unrolled loops fold every lookup into an immediate.
__host__ __device__ constexpr int cx_of(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int cy_of(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ constexpr int opp_of(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
__host__ __device__ constexpr double w_of(int i) {
  return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// Link word of a node (one uint32 per node).  Byte k of the low three bytes
// has bit i-1 set for direction i = 1..8 when the upstream neighbour x - e_i
//   byte 0: is solid while this step streams (pull -> halfway bounce-back),
//   byte 1: is solid after this step's dissolution flips (reaction, W_s),
//   byte 2: lies outside the lattice across a non-periodic side (unknown);
// bit 24 marks the node itself solid while streaming, bit 25 marks a solid
// node that turns fluid before this step collides (dissolution), bit 26 a
// solid node on the dissolution surface list.  The words
// change only when a node dissolves, so a step decodes its neighbourhood with
// bit tests on one word.
constexpr uint32_t kOwnSolid = 1u << 24;
constexpr uint32_t kOwnPending = 1u << 25;
constexpr uint32_t kListed = 1u << 26;  // solid node on the dissolution surface list
constexpr int kUpSolidShift = 0;
constexpr int kUpPostShift = 8;
constexpr int kUpOutShift = 16;
__host__ __device__ constexpr uint32_t up_bit(int shift, int i) { return 1u << (shift + i - 1); }
// A fluid node without a solid neighbour before or after this step's flips
// has a link word that is zero in these bits.
constexpr uint32_t kClearMask =
    kOwnSolid | kOwnPending | (0xFFu << kUpSolidShift) | (0xFFu << kUpPostShift);

// Index checks of the debug-bounds build (compiled with LBM_DEBUG_BOUNDS, in
// place of a memory checker): an index outside [0, limit) records its check
// site in *flag (the first one wins, the host reports it) and is replaced by
// 0, so the access stays inside the array.  The normal build compiles the
// check away.
#ifdef LBM_DEBUG_BOUNDS
__device__ __forceinline__ long long dbg_idx(long long i, long long limit, int* flag, int site) {
  if (i >= 0 && i < limit) return i;
  if (flag) atomicCAS(flag, 0, site);
  return 0;
}
#else
__device__ __forceinline__ long long dbg_idx(long long i, long long, int*, int) { return i; }
#endif
// Sites (values of the status word >= kSiteBase name the failed check).
enum {
  kSiteBase = 100,
  kSitePull = 101,     // global population read of the step
  kSiteNode = 102,     // per-node global field of the step (word, velocity, rate, u)
  kSiteStore = 103,    // global store of a node value or ghost image
  kSiteSmemPop = 111,  // shared-memory population read (tile pipeline)
  kSiteSmemNode = 112, // shared-memory per-node field (tile pipeline)
  kSiteShare = 121,    // reaction share read by the dissolution
  kSiteList = 122,     // surface-list or flip-list entry
  kSiteAdjGather = 131,  // adjoint state read by the reverse step
  kSiteAdjNode = 132,    // per-node field of the reverse step
};

// Padded layout of every node field: interior node (x, y) lives at column
// x + kXO and row y + kYO of a [rows][pitch] array, pitch a multiple of 32
// with pitch >= nx + 16, rows >= ny + 2.  Column kXO - 1, column nx + kXO,
// row 0 and row ny + 1 are ghost cells: across a periodic side the population
// and reaction fields hold there the image of the wrapped node (written
// through by the node itself).  Eight columns on the left put interior
// x = 0 on a 32-byte sector boundary (8 consecutive FP32 nodes per sector)
// and keep every tile's halo box 16-byte aligned for TMA; the minimum sizes
// (160 columns, 10 rows) let one halo box fit the array.
constexpr int kXO = 8;
constexpr int kYO = 1;

__host__ __device__ constexpr int padded_pitch(int nx) {
  return (nx + 16 + 31) / 32 * 32 < 160 ? 160 : (nx + 16 + 31) / 32 * 32;
}
__host__ __device__ constexpr int padded_rows(int ny) { return ny + 2 < 10 ? 10 : ny + 2; }

// Calls fn(gx, gy) for every ghost image of interior node (x, y) (padded
// coordinates), i.e. its copies across periodic sides within one cell of the
// lattice.
template <class Fn>
__device__ __forceinline__ void for_each_ghost(int x, int y, int nx, int ny, int per_x,
                                               int per_y, Fn&& fn) {
  const int xs[2] = {x, per_x ? (x == 0 ? nx : (x == nx - 1 ? -1 : x)) : x};
  const int ys[2] = {y, per_y ? (y == 0 ? ny : (y == ny - 1 ? -1 : y)) : y};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (a == 0 && b == 0) continue;
      const int gx = xs[a], gy = ys[b];
      if ((a == 1 && gx == x) || (b == 1 && gy == y)) continue;
      fn(gx + kXO, gy + kYO);
    }
}

// Side kinds (lbm_edge_kind); kExchange: a side a slab shares with its
// neighbour in a split lattice (its ghost row is filled by the halo exchange).
enum { kPeriodic = 0, kDirichlet = 1, kNeumann = 2, kExchange = 3 };
enum { kReactNone = 0, kReactSurface = 1, kReactBulk = 2 };


// Index of edge node (x, y) of side s in the edge layout [W|E|S|N].
__device__ __forceinline__ int edge_slot(int s, int x, int y, int nx, int ny) {
  return s == 0 ? y : s == 1 ? ny + y : s == 2 ? 2 * ny + x : 2 * ny + nx + x;
}

// Maximum-entropy Dirichlet, Sec. 4.1.1 (a): the unknowns minimising
// H = sum f log(f/w) under sum f = up are proportional to w.  Computed in
// FP64.  Returns true if the data admit no non-negative solution.
template <typename Real>
__device__ bool maxent_dirichlet(Real (&f)[9], unsigned unknown, double up) {
  double wu = 0.0, known = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    if (unknown & (1u << i)) wu += w_of(i);
    else known += (double)f[i];
  }
  const double rest = up - known;
  const double scale = rest / wu;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    if (unknown & (1u << i)) f[i] = (Real)(w_of(i) * scale);
  return rest < 0.0;
}

// Maximum-entropy Neumann, Sec. 4.1.1 (b), for an outward normal (sx, sy)
// with sx, sy in {-1, 0, 1} (a side, or the corner of two Neumann sides).
// Unknowns with e.n = 0 (corner tangents) take halfway bounce-back of the
// node's own post-collision population fbb[opp(i)].  On a side every M^-
// unknown has e.n = -1 and the root gives f proportional to w; at a corner
// (n = (sx, sy)/sqrt 2) the unknowns have e.n = -1/sqrt 2 or -sqrt 2 and the
// root condition is a quadratic in t = exp(gamma / sqrt 2), solved in closed
// form.  Returns kNeuRoot when the root set the unknowns, else the unknowns
// are 0 (the gamma -> -inf limit) and the return is kNeuInfeasible if the
// data admit no root (R > 0) or kNeuZero if R = 0.
enum { kNeuRoot = 0, kNeuInfeasible = 1, kNeuZero = 2 };
template <typename Real>
__device__ int maxent_neumann(Real (&f)[9], unsigned unknown, int sx, int sy,
                              double q, const Real (&fbb)[9]) {
  const bool corner = (sx != 0) && (sy != 0);
  const double inv_len = corner ? 0.70710678118654752440 : 1.0;
  double R = q;
  double w1 = 0.0, w2 = 0.0;  // weights of M^- with |e.n| = 1/sqrt2 (or 1), sqrt2
  unsigned m1 = 0, m2 = 0;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int d = cx_of(i) * sx + cy_of(i) * sy;
    if (unknown & (1u << i)) {
      if (d == 0) {
        f[i] = fbb[opp_of(i)];
      } else if (d == -1) {
        m1 |= 1u << i;
        w1 += w_of(i);
      } else {  // d == -2 (corner diagonal)
        m2 |= 1u << i;
        w2 += w_of(i);
      }
    } else {
      R -= (double)d * inv_len * (double)f[i];
    }
  }
  const double S = -R;
  if (!(S > 0.0)) {
#pragma unroll
    for (int i = 1; i < 9; ++i)
      if ((m1 | m2) & (1u << i)) f[i] = (Real)0;
    return S < 0.0 ? kNeuInfeasible : kNeuZero;
  }
  if (!corner) {
    const double scale = S / w1;
#pragma unroll
    for (int i = 1; i < 9; ++i)
      if (m1 & (1u << i)) f[i] = (Real)(w_of(i) * scale);
    return kNeuRoot;
  }
  // (w1 / (sqrt2 e)) t + (sqrt2 w2 / e) t^2 = S
  const double inv_e = 0.36787944117144233;  // exp(-1)
  const double A = w1 * 0.70710678118654752440 * inv_e;
  const double B = w2 * 1.41421356237309504880 * inv_e;
  const double t = 2.0 * S / (A + sqrt(A * A + 4.0 * B * S));
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    if (m1 & (1u << i)) f[i] = (Real)(w_of(i) * t * inv_e);
    if (m2 & (1u << i)) f[i] = (Real)(w_of(i) * t * t * inv_e);
  }
  return kNeuRoot;
}

// Boundary kind of an edge node (x, y) whose unknown set is not empty:
// Dirichlet wins at corners (*dside >= 0, the first Dirichlet side), else
// Neumann (*nside, the first Neumann side, with the outward normal (sx, sy)
// summed over the node's Neumann sides).
__device__ __forceinline__ void edge_kind(const int (&edge)[4], int x, int y, int nx, int ny,
                                          int* dside, int* nside, int* sx, int* sy) {
  auto bc = [&](int s) { return edge[s] == kDirichlet || edge[s] == kNeumann; };
  const bool on[4] = {x == 0 && bc(0), x == nx - 1 && bc(1), y == 0 && bc(2),
                      y == ny - 1 && bc(3)};
  *dside = -1;
  *nside = -1;
  *sx = 0;
  *sy = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (!on[s]) continue;
    if (edge[s] == kDirichlet && *dside < 0) *dside = s;
    if (edge[s] == kNeumann) {
      if (*nside < 0) *nside = s;
      *sx += (s == 0) ? -1 : (s == 1) ? 1 : 0;
      *sy += (s == 2) ? -1 : (s == 3) ? 1 : 0;
    }
  }
}

// Pore wall of the maximum-entropy kind: Sec. 4.1.1 (b) with zero flux, the
// option beside halfway bounce-back.  `solid` has bit i set where the source
// x - e_i of pull i is solid; on entry f holds the halfway bounce-back value
// in those directions.  The outward normal is the lattice-weighted direction
// to the solid neighbours, n = -sum_{i in solid} w_i e_i, normalised (where it
// cancels, as in a one-node channel, bounce-back stays throughout; which
// unknowns are tangent to it is decided on 36 n, an integer vector).  Unknowns
// with e_i.n >= 0 keep bounce-back; the others become
// w_i exp(-1 - gamma e_i.n) with gamma making sum_i f_i e_i.n zero.  With
// a_i = e_i.n < 0 the flux of those unknowns is -L(gamma),
// L(gamma) = sum |a_i| w_i exp(-1 + gamma |a_i|), so the root solves
// log L(gamma) = log(-R), R = -sum_{others} a_j f_j; log L is convex and
// increasing with slope between the smallest and largest |a_i|, so Newton's
// method converges from any start (in one step when every |a_i| is equal, as
// on a flat wall).
// S is the precision of the solve (the Lagrange multiplier, the normal, the
// fluxes and the exponentials); the lattice's populations f are read and
// written in their own precision Real.  Returns kWallSet, kWallNoRoot if
// R > 0 (no root: those unknowns are set to zero, the gamma -> -infinity
// limit) or kWallNoConv if Newton's method stopped short of its tolerance
// (the last iterate is used).
enum { kWallSet = 0, kWallNoRoot = 1, kWallNoConv = 2 };
template <typename S, typename Real>
__device__ int maxent_wall(Real (&f)[9], unsigned solid) {
  // the normal scaled by 36 (the weights are 4/36 and 1/36): integers, so
  // which unknowns are tangent to it, and whether it cancels, is exact
  int mx = 0, my = 0;
#pragma unroll
  for (int i = 1; i < 9; ++i)
    if (solid & (1u << i)) {
      const int w36 = (cx_of(i) != 0 && cy_of(i) != 0) ? 1 : 4;
      mx -= w36 * cx_of(i);
      my -= w36 * cy_of(i);
    }
  if (mx == 0 && my == 0) return kWallSet;
  const S inv = (S)1 / sqrt((S)(mx * mx + my * my));
  const S nx = (S)mx * inv, ny = (S)my * inv;
  S a[9], R = (S)0, s1 = (S)0, s2 = (S)0;
  unsigned neg = 0u;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    a[i] = (S)cx_of(i) * nx + (S)cy_of(i) * ny;
    if (((solid >> i) & 1u) && cx_of(i) * mx + cy_of(i) * my < 0) {
      neg |= 1u << i;
      s1 -= (S)w_of(i) * a[i];
      s2 += (S)w_of(i) * a[i] * a[i];
    } else {
      R -= a[i] * (S)f[i];
    }
  }
  if (!neg) return kWallSet;
  if (!(R < (S)0)) {
#pragma unroll
    for (int i = 0; i < 9; ++i)
      if (neg & (1u << i)) f[i] = (Real)0;
    return R > (S)0 ? kWallNoRoot : kWallSet;
  }
  if (sizeof(S) == 4 && -R < (S)1e-30) {
    // far below FP32's normal range the exponentials would underflow: the
    // flux-conserving split w_i (-R) / sum w |a| meets the constraint exactly
    // and differs from the maximum-entropy values by less than 1e-30
#pragma unroll
    for (int i = 0; i < 9; ++i)
      if (neg & (1u << i)) f[i] = (Real)((S)w_of(i) * (-R / s1));
    return kWallSet;
  }
  // tolerance on the relative Newton step: a few units of the solve's
  // rounding (FP64 2.2e-16, FP32 1.2e-7)
  constexpr int kIters = sizeof(S) == 8 ? 60 : 24;
  const S tol = sizeof(S) == 8 ? (S)1e-15 : (S)5e-7;
  // An FP64 solve for FP32 populations stops at the first step below 2e-6
  // in g.  phi(g) = log L(g) is convex, with phi' a weighted mean of the
  // unknowns' |a_i| and phi'' their weighted variance (<= 1/2); |a_i| lies
  // in [1 / sqrt(72), sqrt(2)] (an integer c_i . m over |m| <= sqrt(72)).
  // By convexity the error before a Newton step is at most 12 times the
  // step (at most the step itself from below the root), and after it at
  // most |phi''| / (2 phi') < 2.2 times the square of the error before: a
  // step under 2e-6 leaves g within 1.3e-9 and f within 1.8e-9 relative of
  // the root, 30 times below the FP32 rounding the populations then take.
  constexpr bool kLoose = sizeof(S) == 8 && sizeof(Real) == 4;
  const S logR = log(-R);
  // start: the root if every |a_i| were their weighted mean s2 / s1 (in
  // FP32 where FP32 iterations take it from there)
  S g = (S)0;
  bool started = false;
  if constexpr (sizeof(S) == 8) {
    // FP32 iterations (64 times the FP64 rate on this part) bring g to FP32
    // rounding of the root; the FP64 iterations below then need two or three
    // steps to the FP64 tolerance instead of a full solve.  Outside FP32's
    // range, or without FP32 convergence, the FP64 solve starts as above.
    if (-R > 1e-30 && -R < 1e30) {
      float af[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) af[i] = (float)a[i];
      const float logRf = logf((float)-R);
      float gf = (logRf - logf((float)s1) + 1.f) * ((float)s1 / (float)s2);
      bool okf = false;
      for (int it = 0; it < 24; ++it) {
        float L = 0.f, dL = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i)
          if (neg & (1u << i)) {
            const float e = (float)w_of(i) * expf(gf * -af[i] - 1.f);
            L -= af[i] * e;
            dL += af[i] * af[i] * e;
          }
        if (!(dL > 0.f) || !(L > 0.f)) break;
        const float step = (logf(L) - logRf) * (L / dL);
        gf -= step;
        if (fabsf(step) <= 5e-7f * (1.f + fabsf(gf))) {
          okf = true;
          break;
        }
      }
      // (for FP32 populations any finite FP32 iterate is a start: Newton's
      // method converges from any start, and the loop below stops on its
      // own step)
      if ((okf || kLoose) && isfinite(gf)) {
        g = (S)gf;
        started = true;
      }
    }
  }
  if (!started) g = (logR - log(s1) + (S)1) * (s1 / s2);
  bool conv = false;
  S last = (S)0;
  for (int it = 0; it < kIters; ++it) {
    S L = (S)0, dL = (S)0;
#pragma unroll
    for (int i = 0; i < 9; ++i)
      if (neg & (1u << i)) {
        const S e = (S)w_of(i) * exp(g * -a[i] - (S)1);
        L -= a[i] * e;
        dL += a[i] * a[i] * e;
      }
    if (!(dL > (S)0)) break;
    const S step = (log(L) - logR) * (L / dL);
    g -= step;
    last = step;
    if (kLoose ? fabs(step) <= (S)2e-6 : fabs(step) <= tol * ((S)1 + fabs(g))) {
      conv = true;
      break;
    }
  }
  // an iteration that ended oscillating at its rounding level has converged
  if (!conv && fabs(last) <= (S)16 * tol * ((S)1 + fabs(g))) conv = true;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    if (neg & (1u << i)) f[i] = (Real)((S)w_of(i) * exp(g * -a[i] - (S)1));
  return conv ? kWallSet : kWallNoConv;
}

}  // namespace lbm
