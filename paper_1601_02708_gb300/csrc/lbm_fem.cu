// lbm_fem.cu -- the continuum solver of the hybrid method: Q1 finite
// elements for the advection-diffusion equation on a structured rectangular
// mesh, stepped on the GPU (lbm_fem_*, declared in include/lbm_ade.h).
//
// Sec. 3: Galerkin weak form (Sec. 3.1.1) and SUPG (Sec. 3.1.2, Eq. "SUPG",
// "SUPG_tau"); Sec. 6.1.1: semi-discrete M d' + K d = 0 advanced by the
// generalized trapezoidal rule (Eq. "FEM_discrete"),
//     (M + theta dt K) d^{n+1} = (M - (1 - theta) dt K) d^n,
// Dirichlet nodes taking their prescribed values at t^{n+1}; every other
// boundary (the mesh edge and the edge of switched-off elements) is
// zero-flux.
//
// The element matrices of a bilinear element with uniform D and v are
// tensor products of the 1-D linear-element matrices
//     m(h) = h/6 [[2,1],[1,2]], k(h) = 1/h [[1,-1],[-1,1]],
//     c = 1/2 [[-1,1],[-1,1]]  (int phi_a phi_b'),
// assembled once on the host into 9-diagonal (one per neighbour offset)
// arrays of A = M + theta dt K and B = M - (1 - theta) dt K.  The rows of
// Dirichlet and inactive nodes are the identity in A and zero in B.  Each step
// solves A x = B d^n (+ prescribed values) by Jacobi-preconditioned
// BiCGSTAB in FP64 inside one cooperative launch (grid-wide barriers between
// the phases of an iteration, dot products folded in a fixed order, so the
// result is deterministic); the host reads the outcome once per step.  A
// solve starts from the last converged solution (the previous Schwarz
// iterate inside Algorithm 1), else from d^n.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "lbm_ade.h"
#include "lbm_ctx.h"

namespace {

#define FCK(call)                                                                \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess)                                                       \
      return ctx_fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA, \
                      "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                      __FILE__, __LINE__);                                       \
  } while (0)

constexpr int kThreads = 256;

// Outcome of one solve, written by the solver for the host.
struct Scal {
  double bnorm2, rnorm2;  // squared norms of the free rows' rhs and final residual
  int done;               // converged
  int breakdown;          // BiCGSTAB broke down before converging
};

struct Vec {
  double *x, *r, *rhat, *p, *phat, *v, *s, *shat, *t;
};

// Row (i, j) of A x for the 9-diagonal matrix: A[k][row] multiplies the
// neighbour at offset di = k % 3 - 1, dj = k / 3 - 1.
__device__ __forceinline__ double spmv_row(const double* __restrict__ A, const double* x,
                                           int i, int j, int nxn, int nyn, long long n) {
  const long long row = (long long)j * nxn + i;
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int di = k % 3 - 1, dj = k / 3 - 1;
    const int ii = i + di, jj = j + dj;
    if (ii < 0 || ii >= nxn || jj < 0 || jj >= nyn) continue;
    // x may have been written by other blocks of this launch (behind a grid
    // barrier): read it through L2, not the non-coherent L1
    acc += A[k * n + row] * __ldcg(x + (long long)jj * nxn + ii);
  }
  return acc;
}

// Row (i, j) of A y where y_m = g(m) * invd[m] is formed on the fly from
// vectors complete behind the last grid barrier (read through L2).
template <class G>
__device__ __forceinline__ double spmv_row_of(const double* __restrict__ A,
                                              const double* __restrict__ invd, G g, int i, int j,
                                              int nxn, int nyn, long long n) {
  const long long row = (long long)j * nxn + i;
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int di = k % 3 - 1, dj = k / 3 - 1;
    const int ii = i + di, jj = j + dj;
    if (ii < 0 || ii >= nxn || jj < 0 || jj >= nyn) continue;
    const long long m = (long long)jj * nxn + ii;
    acc += A[k * n + row] * (g(m) * invd[m]);
  }
  return acc;
}
// The search direction's update r + beta (p - omega v), one expression for
// the owner's stored value and for the neighbours' on-the-fly values.
__device__ __forceinline__ double next_dir(double r, double p, double v, double beta,
                                           double omega) {
  return r + beta * (p - omega * v);
}

// ---- the linear solve as one cooperative launch -----------------------------
// Every block runs the same BiCGSTAB iteration over a grid-stride share of the
// nodes; the three points per iteration where a dot product must be summed
// (the vectors the sparse products read are complete there too) are
// grid-wide barriers.  Partial dots are written per block and folded by every block in
// the same fixed order, so all blocks take the same decisions.  Each barrier
// wait is bounded: on expiry the status word is set and the blocks return.

constexpr long long kBarrierSpin = 1ll << 24;

struct Solve {
  const double* A;       // [9][n]
  const double* invd;    // [n] 1 / diagonal of A (the Jacobi preconditioner)
  const double* B;       // [9][n]
  double* d;             // state: d^n in, d^{n+1} out
  const int* fixed_id;   // -1 free, -2 inactive, >= 0 index into fixed_val
  const double* fixed_val;
  double* b;
  Vec w;
  double* part;          // [4][gridDim.x] partial dots
  unsigned* bar;         // [2] barrier count and generation
  int* status;           // 0, or 1 after an expired barrier wait
  Scal* sc;              // results: iterations, norms, breakdown
  int* iters;
  int nxn, nyn;
  long long n;
  double tol;
  int max_iter;
  int warm;  // start from w.x (the last converged solution) instead of d^n
};

// Grid-wide barrier (all blocks are resident: cooperative launch).  Returns
// false if the wait expired.
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
      ok = 1;
    } else {
      long long i = 0;
      while (*gen == g && ++i < kBarrierSpin) {
      }
      ok = *gen != g;
      if (!ok) atomicExch(status, 1);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Block partials of two dot products into part0/part1 [blockIdx.x].
__device__ __forceinline__ void block_dot2(double v0, double v1, double* part0, double* part1) {
  __shared__ double s0[kThreads / 32], s1[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_down_sync(0xffffffffu, v0, o);
    v1 += __shfl_down_sync(0xffffffffu, v1, o);
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (lane == 0) {
    s0[wp] = v0;
    s1[wp] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) {
      a += s0[k];
      c += s1[k];
    }
    part0[blockIdx.x] = a;
    if (part1) part1[blockIdx.x] = c;
  }
}

// Sums of the gridDim.x partials of two dot products, the same in every
// block: thread t adds partials t and t + kThreads, each warp folds its
// threads with a fixed shuffle tree, and every thread adds the warp sums in
// warp order.  Each thread issues its loads together, so a fold costs one
// trip to L2 rather than one per partial.  gridDim.x <= kFoldCap (the host
// clamps the grid).
constexpr int kFoldCap = 2 * kThreads;
__device__ __forceinline__ void grid_fold2(const double* pa, const double* pb, double& ra,
                                           double& rb) {
  __shared__ double wa[kThreads / 32], wb[kThreads / 32];
  const int t = threadIdx.x, nb = (int)gridDim.x;
  // written by other blocks before the last grid barrier: read through L2
  const double a0 = t < nb ? __ldcg(pa + t) : 0.0;
  const double a1 = t + kThreads < nb ? __ldcg(pa + t + kThreads) : 0.0;
  const double b0 = pb && t < nb ? __ldcg(pb + t) : 0.0;
  const double b1 = pb && t + kThreads < nb ? __ldcg(pb + t + kThreads) : 0.0;
  double a = a0 + a1, b = b0 + b1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((t & 31) == 0) {
    wa[t >> 5] = a;
    wb[t >> 5] = b;
  }
  __syncthreads();
  a = 0.0;
  b = 0.0;
#pragma unroll
  for (int k = 0; k < kThreads / 32; ++k) {
    a += wa[k];
    b += wb[k];
  }
  ra = a;
  rb = b;
  __syncthreads();  // the warp sums may be overwritten by the next fold
}
__device__ __forceinline__ double grid_fold(const double* part) {
  double a, b;
  grid_fold2(part, nullptr, a, b);
  return a;
}

__global__ void __launch_bounds__(kThreads) k_bicgstab(const Solve S) {
  const long long n = S.n;
  const int nxn = S.nxn, nyn = S.nyn;
  const long long stride = (long long)gridDim.x * kThreads;
  const long long p0 = blockIdx.x * (long long)kThreads + threadIdx.x;
  double* P0 = S.part;
  double* P1 = S.part + gridDim.x;
  double* P2 = S.part + 2 * gridDim.x;
  double* P3 = S.part + 3 * gridDim.x;
  const Vec w = S.w;
  const double* A = S.A;

  // right-hand side (prescribed rows: their values), initial guess
  double bb = 0.0;
  for (long long p = p0; p < n; p += stride) {
    const int i = (int)(p % nxn), j = (int)(p / nxn);
    const int f = S.fixed_id[p];
    double bv, xv;
    if (f >= 0) {
      bv = S.fixed_val[f];
      xv = bv;
    } else if (f == -2) {  // inactive
      bv = 0.0;
      xv = 0.0;
    } else {
      bv = spmv_row(S.B, S.d, i, j, nxn, nyn, n);
      xv = S.warm ? w.x[p] : S.d[p];
    }
    S.b[p] = bv;
    w.x[p] = xv;
    // the residual is measured against the free rows' right-hand side (the
    // prescribed rows are met exactly from the start and stay so)
    if (f == -1) bb += bv * bv;
  }
  block_dot2(bb, 0.0, P0, nullptr);
  if (!grid_sync(S.bar, S.status)) return;

  // r = b - A x, rhat = r, p = r
  double rr = 0.0;
  for (long long p = p0; p < n; p += stride) {
    const int i = (int)(p % nxn), j = (int)(p / nxn);
    const double r = S.b[p] - spmv_row(A, w.x, i, j, nxn, nyn, n);
    w.r[p] = r;
    w.rhat[p] = r;
    w.p[p] = r;
    w.v[p] = 0.0;  // the first direction update r + 0 (p - 0 v) reads it
    rr += r * r;
  }
  block_dot2(rr, 0.0, P1, nullptr);
  if (!grid_sync(S.bar, S.status)) return;
  double bnorm2, rnorm2;
  grid_fold2(P0, P1, bnorm2, rnorm2);
  double rho = rnorm2, alpha = 0.0, omega = 0.0, beta = 0.0;
  const double tol2 = S.tol * S.tol * bnorm2;
  bool done = rnorm2 <= tol2, breakdown = false;
  int it = 0;
  // Three grid barriers an iteration: each sparse product forms its input
  // vector on the fly from vectors that are complete behind the last barrier
  // (the new search direction p = r + beta (p - omega v) with the
  // preconditioner, then s = r - alpha v with it), so neither needs a
  // barrier of its own.  p and v alternate between two buffers, because the
  // products read the previous ones while the owners write the new ones.
  double* pc = w.p;     // search direction of the last iteration
  double* pn = w.phat;  // this iteration's
  double* vc = w.v;     // A (p invd) of the last iteration
  double* vn = w.shat;  // this iteration's
  while (!done && it < S.max_iter) {
    double d0 = 0.0;
    for (long long p = p0; p < n; p += stride) {
      const int i = (int)(p % nxn), j = (int)(p / nxn);
      pn[p] = next_dir(w.r[p], pc[p], vc[p], beta, omega);
      const double v = spmv_row_of(
          A, S.invd,
          [&](long long m) {
            return next_dir(__ldcg(w.r + m), __ldcg(pc + m), __ldcg(vc + m), beta, omega);
          },
          i, j, nxn, nyn, n);
      vn[p] = v;
      d0 += w.rhat[p] * v;
    }
    block_dot2(d0, 0.0, P0, nullptr);
    if (!grid_sync(S.bar, S.status)) return;
    const double rv = grid_fold(P0);
    if (rv == 0.0 || !isfinite(rv)) {
      breakdown = true;
      break;
    }
    alpha = rho / rv;
    double ts = 0.0, tt = 0.0;
    for (long long p = p0; p < n; p += stride) {
      const int i = (int)(p % nxn), j = (int)(p / nxn);
      const double sv = w.r[p] - alpha * vn[p];
      w.s[p] = sv;
      const double t = spmv_row_of(
          A, S.invd, [&](long long m) { return __ldcg(w.r + m) - alpha * __ldcg(vn + m); }, i, j,
          nxn, nyn, n);
      w.t[p] = t;
      ts += t * sv;
      tt += t * t;
    }
    block_dot2(ts, tt, P0, P1);
    if (!grid_sync(S.bar, S.status)) return;
    double tsum, tsv;
    grid_fold2(P1, P0, tsum, tsv);
    omega = tsum > 0.0 ? tsv / tsum : 0.0;
    double rh = 0.0;
    rr = 0.0;
    for (long long p = p0; p < n; p += stride) {
      const double sv = w.s[p];
      w.x[p] += alpha * (pn[p] * S.invd[p]) + omega * (sv * S.invd[p]);
      const double r = sv - omega * w.t[p];
      w.r[p] = r;
      rh += w.rhat[p] * r;
      rr += r * r;
    }
    block_dot2(rh, rr, P2, P3);
    if (!grid_sync(S.bar, S.status)) return;
    double rho_new;
    grid_fold2(P2, P3, rho_new, rnorm2);
    ++it;
    if (rnorm2 <= tol2) {
      done = true;
      break;
    }
    if (rho_new == 0.0 || omega == 0.0 || !isfinite(rho_new)) {
      breakdown = true;
      break;
    }
    beta = (rho_new / rho) * (alpha / omega);
    rho = rho_new;
    double* tp = pc;
    pc = pn;
    pn = tp;
    double* tv = vc;
    vc = vn;
    vn = tv;
  }
  // every block copies its own share of x: no barrier needed
  for (long long p = p0; p < n; p += stride) S.d[p] = w.x[p];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S.sc->bnorm2 = bnorm2;
    S.sc->rnorm2 = rnorm2;
    S.sc->done = done ? 1 : 0;
    S.sc->breakdown = breakdown ? 1 : 0;
    *S.iters = it;
  }
}

// ---- the linear solve of a small system in one block -----------------------
// The same preconditioned BiCGSTAB with its vectors in shared memory, for
// systems of at most kSmallNodes nodes, run by one block.  One SM then does
// all the FP64 work, at 1/64 of the FP32 rate on this part (an FP64 warp
// instruction holds the SM's FP64 pipe for about 16 cycles), so the work
// that is the same for every thread is done once: each warp folds its
// threads' partial sums, thread 0 adds the warp sums in warp order and forms
// the iteration's scalars (alpha, omega, beta), and the others read them
// from shared memory.  The preconditioned vectors p invd and s invd are
// formed once an iteration behind a barrier, where the cooperative solve
// re-forms them at every neighbour to save grid barriers.
constexpr int kSmallThreads = 256;
constexpr long long kSmallNodes = 2048;
constexpr int kSmallVecs = 9;  // x, r, rhat, p, v, s, t, p invd, s invd

// Warp sums of two values into red[0][warp], red[1][warp].
__device__ __forceinline__ void small_warp_sums(double a, double b, double (*red)[kSmallThreads / 32]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
}

__global__ void __launch_bounds__(kSmallThreads) k_bicgstab_small(const Solve S) {
  extern __shared__ double sm[];
  __shared__ double red[2][kSmallThreads / 32];
  // broadcast of thread 0's scalars: alpha, omega, beta; and its verdict
  __shared__ double bc[3];
  __shared__ int stop;  // 0 go on, 1 converged, 2 broke down
  constexpr int kW = kSmallThreads / 32;
  const int n = (int)S.n, nxn = S.nxn, nyn = S.nyn;
  double* x = sm;
  double* r = sm + n;
  double* rh = sm + 2 * n;
  double* p = sm + 3 * n;
  double* v = sm + 4 * n;
  double* s = sm + 5 * n;
  double* t = sm + 6 * n;
  double* y = sm + 7 * n;  // p invd (and d^n in the prologue)
  double* z = sm + 8 * n;  // s invd (and b in the prologue)
  const int q0 = threadIdx.x;
  const bool lead = threadIdx.x == 0;
  // row q of M u for a vector u in shared memory
  auto row = [&](const double* __restrict__ M, const double* u, int q) {
    const int i = q % nxn, j = q / nxn;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int ii = i + k % 3 - 1, jj = j + k / 3 - 1;
      if (ii < 0 || ii >= nxn || jj < 0 || jj >= nyn) continue;
      acc += __ldg(M + (long long)k * n + q) * u[jj * nxn + ii];
    }
    return acc;
  };
  for (int q = q0; q < n; q += kSmallThreads) y[q] = S.d[q];
  __syncthreads();
  // right-hand side (prescribed rows: their values), initial guess
  double bb = 0.0;
  for (int q = q0; q < n; q += kSmallThreads) {
    const int f = S.fixed_id[q];
    double bv, xv;
    if (f >= 0) {
      bv = S.fixed_val[f];
      xv = bv;
    } else if (f == -2) {
      bv = 0.0;
      xv = 0.0;
    } else {
      bv = row(S.B, y, q);
      xv = S.warm ? S.w.x[q] : y[q];
    }
    z[q] = bv;
    x[q] = xv;
    if (f == -1) bb += bv * bv;
  }
  __syncthreads();
  // r = b - A x, rhat = r, p = r, v = 0
  double rr = 0.0;
  for (int q = q0; q < n; q += kSmallThreads) {
    const double rq = z[q] - row(S.A, x, q);
    r[q] = rq;
    rh[q] = rq;
    p[q] = rq;
    v[q] = 0.0;
    rr += rq * rq;
  }
  small_warp_sums(bb, rr, red);
  __syncthreads();
  // thread 0's state: norms, rho and the iteration count
  double bnorm2 = 0.0, rnorm2 = 0.0, tol2 = 0.0, rho = 0.0;
  int it = 0;
  if (lead) {
    for (int k = 0; k < kW; ++k) {
      bnorm2 += red[0][k];
      rnorm2 += red[1][k];
    }
    tol2 = S.tol * S.tol * bnorm2;
    rho = rnorm2;
    bc[0] = bc[1] = bc[2] = 0.0;
    stop = rnorm2 <= tol2 ? 1 : 0;
  }
  __syncthreads();
  while (!stop) {
    const double beta = bc[2], omega_old = bc[1];
    for (int q = q0; q < n; q += kSmallThreads) {
      const double pq = r[q] + beta * (p[q] - omega_old * v[q]);
      p[q] = pq;
      y[q] = pq * S.invd[q];
    }
    __syncthreads();
    double d0 = 0.0;
    for (int q = q0; q < n; q += kSmallThreads) {
      const double vq = row(S.A, y, q);
      v[q] = vq;
      d0 += rh[q] * vq;
    }
    small_warp_sums(d0, 0.0, red);
    __syncthreads();
    if (lead) {
      double sum = 0.0;
      for (int k = 0; k < kW; ++k) sum += red[0][k];
      if (sum == 0.0 || !isfinite(sum))
        stop = 2;
      else
        bc[0] = rho / sum;
    }
    __syncthreads();
    if (stop) break;
    const double alpha = bc[0];
    for (int q = q0; q < n; q += kSmallThreads) {
      const double sq = r[q] - alpha * v[q];
      s[q] = sq;
      z[q] = sq * S.invd[q];
    }
    __syncthreads();
    double ts = 0.0, tt = 0.0;
    for (int q = q0; q < n; q += kSmallThreads) {
      const double tq = row(S.A, z, q);
      t[q] = tq;
      ts += tq * s[q];
      tt += tq * tq;
    }
    small_warp_sums(ts, tt, red);
    __syncthreads();
    if (lead) {
      double a = 0.0, b = 0.0;
      for (int k = 0; k < kW; ++k) {
        a += red[0][k];
        b += red[1][k];
      }
      bc[1] = b > 0.0 ? a / b : 0.0;
    }
    __syncthreads();
    const double omega = bc[1];
    double rhn = 0.0;
    rr = 0.0;
    for (int q = q0; q < n; q += kSmallThreads) {
      x[q] += alpha * y[q] + omega * z[q];
      const double rq = s[q] - omega * t[q];
      r[q] = rq;
      rhn += rh[q] * rq;
      rr += rq * rq;
    }
    small_warp_sums(rhn, rr, red);
    __syncthreads();
    if (lead) {
      double rho_new = 0.0;
      rnorm2 = 0.0;
      for (int k = 0; k < kW; ++k) {
        rho_new += red[0][k];
        rnorm2 += red[1][k];
      }
      ++it;
      if (rnorm2 <= tol2)
        stop = 1;
      else if (rho_new == 0.0 || omega == 0.0 || !isfinite(rho_new))
        stop = 2;
      else if (it >= S.max_iter)
        stop = 3;
      else
        bc[2] = (rho_new / rho) * (alpha / omega);
      rho = rho_new;
    }
    __syncthreads();
  }
  // the solution, and the warm start of the next solve
  for (int q = q0; q < n; q += kSmallThreads) {
    S.d[q] = x[q];
    S.w.x[q] = x[q];
  }
  if (lead) {
    S.sc->bnorm2 = bnorm2;
    S.sc->rnorm2 = rnorm2;
    S.sc->done = stop == 1 ? 1 : 0;
    S.sc->breakdown = stop == 2 ? 1 : 0;
    *S.iters = it;
  }
}

// FE interpolation (bilinear on the containing element) of d at points
__global__ void k_interp(const double* __restrict__ d, int nex, int ney, double x0, double y0,
                         double hx, double hy, const double* __restrict__ xy, int npts,
                         double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npts) return;
  const double px = (xy[2 * k] - x0) / hx, py = (xy[2 * k + 1] - y0) / hy;
  int i = (int)floor(px), j = (int)floor(py);
  i = i < 0 ? 0 : (i > nex - 1 ? nex - 1 : i);
  j = j < 0 ? 0 : (j > ney - 1 ? ney - 1 : j);
  const double gx = px - i, gy = py - j;
  const int nxn = nex + 1;
  const double* r0 = d + (long long)j * nxn + i;
  const double* r1 = r0 + nxn;
  out[k] = r0[0] * (1 - gx) * (1 - gy) + r0[1] * gx * (1 - gy) + r1[1] * gx * gy +
           r1[0] * (1 - gx) * gy;
}

}  // namespace

struct lbm_fem {
  lbm_fem_params p;
  int nxn = 0, nyn = 0;
  long long n = 0;
  int n_dir = 0;
  cudaStream_t stream = nullptr;
  double* A = nullptr;  // [9][n]
  double* B = nullptr;  // [9][n]
  double* d = nullptr;  // state
  double* b = nullptr;  // right-hand side
  double* invd = nullptr;  // 1 / diagonal of A
  Vec w{};
  double* vecs = nullptr;   // storage of w
  int* fixed_id = nullptr;  // per node: index into the prescribed values, -1 free, -2 inactive
  double* fixed_val = nullptr;
  double* part = nullptr;   // [4][grid] partial dots
  Scal* sc = nullptr;
  int* iters = nullptr;
  unsigned* bar = nullptr;  // grid barrier [2]
  int* status = nullptr;
  int grid = 0;             // blocks of the cooperative solve (all resident)
  double* scratch = nullptr;  // staging of host points / results of lbm_fem_interpolate
  void* pinned = nullptr;     // page-locked read-back of a solve's outcome
  bool small = false;         // solved by k_bicgstab_small (n <= kSmallNodes)
  size_t scratch_n = 0;
  int last_iters = 0;
  double last_resid = 0.0;
  // w.x holds the last converged solution: the next solve starts from it.
  // Within a Schwarz step (Algorithm 1) every iteration after the first
  // solves the same system with nearby Dirichlet data, so the previous
  // iterate is a far better start than d^n; in plain time stepping it is
  // d^n itself.  The answer is the same to the solve's tolerance.
  bool warm = false;
};

namespace {

void fem_free(lbm_fem* f) {
  void* ptrs[] = {f->A, f->B, f->d, f->b, f->vecs, f->fixed_id, f->fixed_val, f->part,
                  f->sc, f->iters, f->scratch, f->bar, f->status, f->invd};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (f->pinned) cudaFreeHost(f->pinned);
  delete f;
}

// Element matrices (Galerkin + SUPG) of one hx x hy element in the local
// node order (0,0), (1,0), (1,1), (0,1).
void element(const lbm_fem_params& p, double tau, double Me[4][4], double Ke[4][4]) {
  const double mx[2][2] = {{p.hx / 3, p.hx / 6}, {p.hx / 6, p.hx / 3}};
  const double my[2][2] = {{p.hy / 3, p.hy / 6}, {p.hy / 6, p.hy / 3}};
  const double kx[2][2] = {{1 / p.hx, -1 / p.hx}, {-1 / p.hx, 1 / p.hx}};
  const double ky[2][2] = {{1 / p.hy, -1 / p.hy}, {-1 / p.hy, 1 / p.hy}};
  const double c[2][2] = {{-0.5, 0.5}, {-0.5, 0.5}};  // int phi_a phi_b'
  const int loc[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const int ia = loc[a][0], ja = loc[a][1], ib = loc[b][0], jb = loc[b][1];
      const double mass = mx[ia][ib] * my[ja][jb];
      const double adv = p.vx * c[ia][ib] * my[ja][jb] + p.vy * mx[ia][ib] * c[ja][jb];
      const double dif = p.D * (kx[ia][ib] * my[ja][jb] + mx[ia][ib] * ky[ja][jb]);
      // SUPG: the test function gains tau v.grad N_a
      const double adv_t = p.vx * c[ib][ia] * my[ja][jb] + p.vy * mx[ia][ib] * c[jb][ja];
      const double vv = p.vx * p.vx * kx[ia][ib] * my[ja][jb] +
                        p.vy * p.vy * mx[ia][ib] * ky[ja][jb] +
                        p.vx * p.vy * (c[ib][ia] * c[ja][jb] + c[ia][ib] * c[jb][ja]);
      Me[a][b] = mass + tau * adv_t;
      Ke[a][b] = adv + dif + tau * vv;
    }
}

// tau_e = h / (2|v|) (coth Pe - 1/Pe), Pe = |v| h / (2D), h the element
// length along the flow, min(hx / |v^_x|, hy / |v^_y|).
double supg_tau(const lbm_fem_params& p) {
  const double speed = std::hypot(p.vx, p.vy);
  if (!p.supg || speed == 0.0) return 0.0;
  const double ux = std::fabs(p.vx) / speed, uy = std::fabs(p.vy) / speed;
  double h = INFINITY;
  if (ux > 0) h = std::fmin(h, p.hx / ux);
  if (uy > 0) h = std::fmin(h, p.hy / uy);
  if (!(p.D > 0.0)) return h / (2.0 * speed);
  const double pe = speed * h / (2.0 * p.D);
  const double xi = pe > 30.0 ? 1.0 - 1.0 / pe : (std::cosh(pe) / std::sinh(pe) - 1.0 / pe);
  return h / (2.0 * speed) * xi;
}

lbm_status fem_setup(lbm_fem* f, const uint8_t* elem_active, const int* dir_nodes,
                     const double* d0) {
  const lbm_fem_params& p = f->p;
  const int nxn = f->nxn;
  const long long n = f->n;
  std::vector<double> A(9 * n, 0.0), B(9 * n, 0.0);
  std::vector<char> touched(n, 0);
  double Me[4][4], Ke[4][4];
  element(p, supg_tau(p), Me, Ke);
  const int loc[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
  const double ca = p.theta * p.dt, cb = -(1.0 - p.theta) * p.dt;
  for (int j = 0; j < p.ney; ++j)
    for (int i = 0; i < p.nex; ++i) {
      if (elem_active && !elem_active[(long long)j * p.nex + i]) continue;
      for (int a = 0; a < 4; ++a) {
        const int ra = (j + loc[a][1]) * nxn + (i + loc[a][0]);
        touched[ra] = 1;
        for (int b = 0; b < 4; ++b) {
          const int di = loc[b][0] - loc[a][0], dj = loc[b][1] - loc[a][1];
          const int k = (dj + 1) * 3 + (di + 1);
          A[k * n + ra] += Me[a][b] + ca * Ke[a][b];
          B[k * n + ra] += Me[a][b] + cb * Ke[a][b];
        }
      }
    }
  std::vector<int> fid(n, -1);
  for (long long q = 0; q < n; ++q)
    if (!touched[q]) fid[q] = -2;
  for (int k = 0; k < f->n_dir; ++k) {
    const int q = dir_nodes[k];
    if (q < 0 || q >= n) return ctx_fail(LBM_ERR_ARG, "lbm_fem_init: Dirichlet node %d out of range", q);
    if (fid[q] >= 0) return ctx_fail(LBM_ERR_ARG, "lbm_fem_init: Dirichlet node %d repeated", q);
    fid[q] = k;
  }
  for (long long q = 0; q < n; ++q)
    if (fid[q] != -1) {  // identity row in A, zero row in B
      for (int k = 0; k < 9; ++k) {
        A[k * n + q] = k == 4 ? 1.0 : 0.0;
        B[k * n + q] = 0.0;
      }
    }
  std::vector<double> invd(n);
  for (long long q = 0; q < n; ++q) invd[q] = 1.0 / A[4 * n + q];
  FCK(cudaMemcpyAsync(f->A, A.data(), 9 * n * sizeof(double), cudaMemcpyHostToDevice, f->stream));
  FCK(cudaMemcpyAsync(f->invd, invd.data(), n * sizeof(double), cudaMemcpyHostToDevice,
                      f->stream));
  FCK(cudaMemcpyAsync(f->B, B.data(), 9 * n * sizeof(double), cudaMemcpyHostToDevice, f->stream));
  FCK(cudaMemcpyAsync(f->fixed_id, fid.data(), n * sizeof(int), cudaMemcpyHostToDevice, f->stream));
  std::vector<double> d(n, 0.0);
  if (d0) {
    const bool dev = ctx_on_device(d0);
    if (dev) FCK(cudaMemcpy(d.data(), d0, n * sizeof(double), cudaMemcpyDeviceToHost));
    else std::memcpy(d.data(), d0, n * sizeof(double));
  }
  for (long long q = 0; q < n; ++q)
    if (fid[q] == -2) d[q] = 0.0;
  FCK(cudaMemcpyAsync(f->d, d.data(), n * sizeof(double), cudaMemcpyHostToDevice, f->stream));
  FCK(cudaStreamSynchronize(f->stream));
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_fem_init(lbm_fem** out, const lbm_fem_params* p, const uint8_t* elem_active,
                        int n_dir, const int* dir_nodes, const double* d0, void* stream) {
  if (!out || !p) return ctx_fail(LBM_ERR_ARG, "lbm_fem_init: null argument");
  *out = nullptr;
  if (p->nex < 1 || p->ney < 1 || !(p->hx > 0) || !(p->hy > 0) || !(p->dt > 0) ||
      !(p->theta >= 0.0 && p->theta <= 1.0) || !(p->D >= 0.0) || n_dir < 0 ||
      (n_dir > 0 && !dir_nodes))
    return ctx_fail(LBM_ERR_ARG, "lbm_fem_init: bad parameters");
  if ((long long)(p->nex + 1) * (p->ney + 1) > (1ll << 30))
    return ctx_fail(LBM_ERR_ARG, "lbm_fem_init: mesh too large");
  lbm_fem* f = new lbm_fem();
  f->p = *p;
  if (!(f->p.tol > 0)) f->p.tol = 1e-12;
  if (f->p.max_iter <= 0) f->p.max_iter = 1000;
  f->nxn = p->nex + 1;
  f->nyn = p->ney + 1;
  f->n = (long long)f->nxn * f->nyn;
  f->n_dir = n_dir;
  f->stream = (cudaStream_t)stream;
  const long long n = f->n;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
  };
  al((void**)&f->A, 9 * n * sizeof(double));
  al((void**)&f->B, 9 * n * sizeof(double));
  al((void**)&f->d, n * sizeof(double));
  al((void**)&f->b, n * sizeof(double));
  al((void**)&f->invd, n * sizeof(double));
  al((void**)&f->vecs, 9 * n * sizeof(double));
  al((void**)&f->fixed_id, n * sizeof(int));
  al((void**)&f->fixed_val, (n_dir > 0 ? n_dir : 1) * sizeof(double));
  {
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bicgstab, kThreads, 0);
    if (e == cudaSuccess && (!coop || per_sm < 1)) {
      fem_free(f);
      return ctx_fail(LBM_ERR_CUDA, "lbm_fem_init: the device has no cooperative launch");
    }
    const long long need = (n + kThreads - 1) / kThreads;
    long long cap = (long long)sms * (per_sm < 2 ? per_sm : 2);
    if (cap > kFoldCap) cap = kFoldCap;  // partials one fold can take
    f->grid = (int)(need < cap ? need : cap);
    f->small = n <= kSmallNodes;
    if (f->small && e == cudaSuccess)
      e = cudaFuncSetAttribute(k_bicgstab_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kSmallVecs * kSmallNodes * sizeof(double)));
  }
  al((void**)&f->part, 4 * (size_t)(f->grid > 0 ? f->grid : 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&f->pinned, 256);
  al((void**)&f->sc, sizeof(Scal));
  al((void**)&f->iters, sizeof(int));
  al((void**)&f->bar, 2 * sizeof(unsigned));
  al((void**)&f->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(f->bar, 0, 2 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(f->status, 0, sizeof(int));
  if (e != cudaSuccess) {
    fem_free(f);
    return ctx_fail(LBM_ERR_NOMEM, "lbm_fem_init: %s", cudaGetErrorString(e));
  }
  double* v = f->vecs;
  f->w = Vec{v, v + n, v + 2 * n, v + 3 * n, v + 4 * n, v + 5 * n, v + 6 * n, v + 7 * n, v + 8 * n};
  const lbm_status st = fem_setup(f, elem_active, dir_nodes, d0);
  if (st != LBM_OK) {
    fem_free(f);
    return st;
  }
  *out = f;
  return LBM_OK;
}

lbm_status lbm_fem_step(lbm_fem* f, const double* dir_values) {
  if (!f) return ctx_fail(LBM_ERR_ARG, "lbm_fem_step: null solver");
  if (f->n_dir > 0 && !dir_values) return ctx_fail(LBM_ERR_ARG, "lbm_fem_step: null values");
  cudaStream_t s = f->stream;
  if (f->n_dir > 0)
    FCK(cudaMemcpyAsync(f->fixed_val, dir_values, f->n_dir * sizeof(double), cudaMemcpyDefault, s));
  Solve S;
  S.A = f->A;
  S.invd = f->invd;
  S.B = f->B;
  S.d = f->d;
  S.fixed_id = f->fixed_id;
  S.fixed_val = f->fixed_val;
  S.b = f->b;
  S.w = f->w;
  S.part = f->part;
  S.bar = f->bar;
  S.status = f->status;
  S.sc = f->sc;
  S.iters = f->iters;
  S.nxn = f->nxn;
  S.nyn = f->nyn;
  S.n = f->n;
  S.tol = f->p.tol;
  S.max_iter = f->p.max_iter;
  S.warm = f->warm ? 1 : 0;
  void* args[] = {&S};
  if (f->small)
    k_bicgstab_small<<<1, kSmallThreads, kSmallVecs * f->n * sizeof(double), s>>>(S);
  else
    FCK(cudaLaunchCooperativeKernel((const void*)k_bicgstab, dim3(f->grid), dim3(kThreads), args,
                                    0, s));
  FCK(cudaGetLastError());
  struct Outcome {
    Scal sc;
    int iters, status;
  };
  static_assert(sizeof(Outcome) <= 256, "the outcome fits its pinned read-back");
  Outcome& h = *(Outcome*)f->pinned;
  FCK(cudaMemcpyAsync(&h.sc, f->sc, sizeof(Scal), cudaMemcpyDeviceToHost, s));
  FCK(cudaMemcpyAsync(&h.iters, f->iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  FCK(cudaMemcpyAsync(&h.status, f->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  FCK(cudaStreamSynchronize(s));
  f->last_iters = h.iters;
  f->last_resid = h.sc.bnorm2 > 0 ? std::sqrt(h.sc.rnorm2 / h.sc.bnorm2) : std::sqrt(h.sc.rnorm2);
  f->warm = !h.status && h.sc.done;
  if (h.status) {
    cudaMemsetAsync(f->status, 0, sizeof(int), s);
    cudaMemsetAsync(f->bar, 0, 2 * sizeof(unsigned), s);
    return ctx_fail(LBM_ERR_TIMEOUT, "lbm_fem_step: a grid barrier wait of the solve expired");
  }
  if (h.sc.breakdown && !h.sc.done)
    return ctx_fail(LBM_ERR_STATE, "lbm_fem_step: BiCGSTAB broke down (relative residual %.3e)",
                    f->last_resid);
  if (!h.sc.done)
    return ctx_fail(LBM_ERR_STATE, "lbm_fem_step: no convergence in %d iterations (residual %.3e)",
                    f->p.max_iter, f->last_resid);
  return LBM_OK;
}

lbm_status lbm_fem_interpolate(lbm_fem* f, int npts, const double* xy, double* out) {
  if (!f || npts < 0 || (npts > 0 && (!xy || !out)))
    return ctx_fail(LBM_ERR_ARG, "lbm_fem_interpolate: bad arguments");
  if (npts == 0) return LBM_OK;
  cudaStream_t s = f->stream;
  const bool xy_dev = ctx_on_device(xy), out_dev = ctx_on_device(out);
  const double* dxy = xy;
  double* dout = out;
  double* tmp = nullptr;
  if (!xy_dev || !out_dev) {
    if (f->scratch_n < 3 * (size_t)npts) {
      FCK(cudaStreamSynchronize(s));
      if (f->scratch) cudaFree(f->scratch);
      f->scratch = nullptr;
      f->scratch_n = 0;
      FCK(cudaMalloc((void**)&f->scratch, 3 * (size_t)npts * sizeof(double)));
      f->scratch_n = 3 * (size_t)npts;
    }
    tmp = f->scratch;
    if (!xy_dev) {
      FCK(cudaMemcpyAsync(tmp, xy, 2 * (size_t)npts * sizeof(double), cudaMemcpyHostToDevice, s));
      dxy = tmp;
    }
    if (!out_dev) dout = tmp + 2 * (size_t)npts;
  }
  const lbm_fem_params& p = f->p;
  k_interp<<<(npts + 127) / 128, 128, 0, s>>>(f->d, p.nex, p.ney, p.x0, p.y0, p.hx, p.hy, dxy,
                                               npts, dout);
  FCK(cudaGetLastError());
  if (!out_dev) FCK(cudaMemcpyAsync(out, dout, (size_t)npts * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (tmp) FCK(cudaStreamSynchronize(s));
  return LBM_OK;
}

lbm_status lbm_fem_get(lbm_fem* f, double* d) {
  if (!f || !d) return ctx_fail(LBM_ERR_ARG, "lbm_fem_get: null argument");
  FCK(cudaMemcpyAsync(d, f->d, f->n * sizeof(double), cudaMemcpyDefault, f->stream));
  if (!ctx_on_device(d)) FCK(cudaStreamSynchronize(f->stream));
  return LBM_OK;
}

lbm_status lbm_fem_set(lbm_fem* f, const double* d) {
  if (!f || !d) return ctx_fail(LBM_ERR_ARG, "lbm_fem_set: null argument");
  FCK(cudaMemcpyAsync(f->d, d, f->n * sizeof(double), cudaMemcpyDefault, f->stream));
  if (!ctx_on_device(d)) FCK(cudaStreamSynchronize(f->stream));
  return LBM_OK;
}

lbm_status lbm_fem_solver_info(lbm_fem* f, int* iters, double* rel_resid) {
  if (!f) return ctx_fail(LBM_ERR_ARG, "lbm_fem_solver_info: null solver");
  if (iters) *iters = f->last_iters;
  if (rel_resid) *rel_resid = f->last_resid;
  return LBM_OK;
}

void lbm_fem_destroy(lbm_fem* f) {
  if (!f) return;
  cudaStreamSynchronize(f->stream);
  fem_free(f);
}

}  // extern "C"
