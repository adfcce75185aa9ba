// lbm_adjoint.cu -- reverse mode of the fused step for a fixed solid mask
// (lbm_adjoint, declared in include/lbm_ade.h).
//
// With the mask fixed, one step maps the stored post-collision populations
// F^{n-1} to F^n through pull streaming with bounce-back, the boundary
// conditions of Sec. 4.1.1 and the collision with the sink; the map is affine
// in the populations and the edge data (a Neumann node switches between the
// root and the zero limit, a branch that is recorded).  The objective is the
// outlet breakthrough J = sum_n sum_{east-edge fluid nodes} u^n.
//
// The adjoint state kept between kernels is pbar, the sensitivity of J to
// the populations a node pulled in (after the boundary conditions have moved
// the sensitivity of the unknowns onto the known populations and the data).
// One adjoint step n, per fluid node y:
//   lambda_j(y) = pbar^{n+1}_j(y + e_j)        downstream fluid (pulled it)
//               = pbar^{n+1}_rev(j)(y)         downstream solid (bounced back)
//               = 0                            downstream outside
//   gbar_j = (1 - omega) lambda_j + omega sum_i w_i P_i lambda_i
//            - k sum_i w_i lambda_i + [y on the east edge]
//   dJ/dk(y) -= u^n(y) sum_i w_i lambda_i       (reactive nodes)
//   boundary nodes, t = sum_U w_i gbar_i / W_U over the unknowns U:
//     Dirichlet: pbar_known = gbar_known - t, dJ/du^p += t (split over the
//       start and end data by 1 - j/eta and j/eta, Eq. "MTS")
//     Neumann with the root: pbar_k = gbar_k + (e_k.n) t, dJ/dq -= t
//   pbar^n = gbar elsewhere, 0 on the unknowns.
// A final pass gathers lambda^0 and adds the first collision's -u^0 sum
// w_i lambda_i, so the state held fixed is the pre-collision one at the start
// of the call.
//
// sqrt(N) checkpointing: the forward run keeps F every L steps; the reverse
// sweep restores each segment's checkpoint, recomputes its L steps storing
// u^n and the Neumann branches, then runs its L adjoint steps backwards.
// With one segment (L >= N) the forward run stores u^n and the branches of
// every step itself and nothing is recomputed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "lbm_ade.h"
#include "lbm_ctx.h"
#include "lbm_kernels.cuh"

namespace {

#define ACK(call)                                                                \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess)                                                       \
      return ctx_fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA, \
                      "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                      __FILE__, __LINE__);                                       \
  } while (0)

#define ATRY(...)                   \
  do {                              \
    lbm_status s_ = (__VA_ARGS__);  \
    if (s_ != LBM_OK) return s_;    \
  } while (0)

template <typename Real>
struct AdjArgs {
  const Real* __restrict__ mu_in;   // pbar of step n + 1, [9][rows][pitch]
  Real* __restrict__ mu_out;        // pbar of step n
  const uint32_t* __restrict__ link;
  const Real* __restrict__ vel;     // [2][rows][pitch]
  const Real* __restrict__ kf;      // [rows][pitch] or null
  const Real* __restrict__ u_n;     // u^n, the input of step n's collision
  const unsigned char* __restrict__ root;  // Neumann root taken at step n, per edge slot
  double* __restrict__ gk;          // [rows][pitch] dJ/dk (FP64 lattice)
  float* __restrict__ gk32;         // [rows][pitch] dJ/dk of the current segment (FP32
                                    // lattice), folded into gk after every segment
  double* __restrict__ g_ua;        // [nedge] dJ/d(start data)
  double* __restrict__ g_ub;        // [nedge] dJ/d(end data)
  double* __restrict__ g_q;         // [nedge] dJ/dq
  int* status;  // the context's status word (index checks of the debug build)
  long long plane;
  int nx, ny, pitch, per_x, per_y;
  int edge[4];
  int react_mode;
  Real omega, k_scalar;
  double frac;  // j / eta of step n
};

template <typename Real, bool kInit, bool kEdge>
__device__ __forceinline__ void adjoint_node(const AdjArgs<Real>& a, int x, int y, long long n) {
  using namespace lbm;
  const long long nn = dbg_idx(n, a.plane, a.status, kSiteAdjNode);
  const long long lim = 9 * a.plane;
  const uint32_t w = a.link[nn];
  if (w & kOwnSolid) return;
  Real lam[9];
  lam[0] = a.mu_in[nn];
#pragma unroll
  for (int j = 1; j < 9; ++j) {
    const int jb = opp_of(j);
    if (kEdge && (w & up_bit(kUpOutShift, jb))) {
      lam[j] = (Real)0;
    } else if (w & up_bit(kUpSolidShift, jb)) {
      lam[j] = a.mu_in[dbg_idx(jb * a.plane + n, lim, a.status, kSiteAdjGather)];
    } else {
      lam[j] = a.mu_in[dbg_idx(j * a.plane + n + cx_of(j) + (long long)cy_of(j) * a.pitch, lim,
                               a.status, kSiteAdjGather)];
    }
  }
  const uint32_t post = (w >> kUpPostShift) & 0xFFu;
  const bool reactive =
      a.react_mode == kReactBulk || (a.react_mode == kReactSurface && post != 0u);
  Real wl = (Real)w_of(0) * lam[0];
#pragma unroll
  for (int i = 1; i < 9; ++i) wl += (Real)w_of(i) * lam[i];
  if (reactive) {
    if constexpr (sizeof(Real) == 4) a.gk32[nn] -= a.u_n[nn] * wl;
    else a.gk[nn] -= (double)a.u_n[nn] * (double)wl;
  }
  if (kInit) return;
  const Real kr = reactive ? (a.kf ? a.kf[nn] : a.k_scalar) : (Real)0;
  const Real vx = a.vel[nn], vy = a.vel[a.plane + nn];
  const Real base = (Real)1 - (Real)1.5 * (vx * vx + vy * vy);
  // sum_i w_i P_i lambda_i, by opposite pairs (P differs in the sign of 3 e.v)
  Real wp = (Real)w_of(0) * base * lam[0];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = p < 2 ? p + 1 : p + 3;
    const int o = opp_of(i);
    const Real ev = (Real)cx_of(i) * vx + (Real)cy_of(i) * vy;
    const Real sym = base + (Real)4.5 * ev * ev;
    const Real anti = (Real)3 * ev;
    wp += (Real)w_of(i) * ((sym + anti) * lam[i] + (sym - anti) * lam[o]);
  }
  Real s = a.omega * wp - kr * wl;
  if (kEdge && x == a.nx - 1) s += (Real)1;  // u^n counts in J
  const Real om1 = (Real)1 - a.omega;
  Real nu[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) nu[j] = om1 * lam[j] + s;
  bool ghosts = false;
  if (kEdge) {
    ghosts = ((x == 0) | (x == a.nx - 1) | (y == 0) | (y == a.ny - 1)) && (a.per_x | a.per_y);
    const unsigned unknown = ((w >> kUpOutShift) & 0xFFu) << 1;
    if (unknown) {
      int dside, nside, sx, sy;
      edge_kind(a.edge, x, y, a.nx, a.ny, &dside, &nside, &sx, &sy);
      // t = sum_U w_i nu_i / W_U over the unknowns, in FP64 on either lattice
      // (the transpose of the forward solves, which run in FP64)
      double t = 0.0, wu = 0.0;
#pragma unroll
      for (int i = 0; i < 9; ++i)
        if (unknown & (1u << i)) {
          t += w_of(i) * (double)nu[i];
          wu += w_of(i);
        }
      t /= wu;
      if (dside >= 0) {
        const int slot = edge_slot(dside, x, y, a.nx, a.ny);
#pragma unroll
        for (int i = 0; i < 9; ++i)
          if (!(unknown & (1u << i))) nu[i] = (Real)((double)nu[i] - t);
        atomicAdd(a.g_ua + slot, (1.0 - a.frac) * t);
        atomicAdd(a.g_ub + slot, a.frac * t);
      } else {
        const int slot = edge_slot(nside, x, y, a.nx, a.ny);
        if (a.root[slot]) {
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            const int d = cx_of(i) * sx + cy_of(i) * sy;
            if (!(unknown & (1u << i)) && d != 0) nu[i] = (Real)((double)nu[i] + d * t);
          }
          atomicAdd(a.g_q + slot, -t);
        }
      }
#pragma unroll
      for (int i = 0; i < 9; ++i)
        if (unknown & (1u << i)) nu[i] = (Real)0;
    }
  }
#pragma unroll
  for (int i = 0; i < 9; ++i)
    store_node(a.mu_out + i * a.plane, n, nu[i], ghosts, x, y, a.nx, a.ny, a.pitch, a.per_x,
               a.per_y, a.plane, a.status);
}

// One adjoint step (kInit: the gather of lambda^0 and the first collision's
// rate term only).  One thread per node in blocks of one warp (32 x
// kAdjRows): the reverse step is bound by the latency of its gathers, and
// one-warp blocks leave no slot waiting for a block's slowest warp.  One
// 5000-step call at 512^2 took 113, 101, 89 and 84 ms with 8, 4, 2 and 1
// rows per block.
constexpr int kAdjRows = 1;
template <typename Real, bool kInit>
__global__ void __launch_bounds__(lbm::kBX * kAdjRows) lbm_adjoint_step(const AdjArgs<Real> a) {
  const int x = blockIdx.x * lbm::kBX + threadIdx.x;
  const int y = blockIdx.y * kAdjRows + threadIdx.y;
  if (x >= a.nx || y >= a.ny) return;
  const long long n = (long long)(y + lbm::kYO) * a.pitch + (x + lbm::kXO);
  if (lbm::group_is_interior(blockIdx.x * lbm::kBX, y, a.nx, a.ny))
    adjoint_node<Real, kInit, false>(a, x, y, n);
  else
    adjoint_node<Real, kInit, true>(a, x, y, n);
}

// gk += gk32 (FP64), gk32 = 0: the end of a segment of the FP32 lattice.
__global__ void k_fold_gk(double* __restrict__ gk, float* __restrict__ gk32, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float g = gk32[i];
    if (g != 0.f) {
      gk[i] += (double)g;
      gk32[i] = 0.f;
    }
  }
}

}  // namespace

// Buffers of the reverse sweep, kept in the context between calls.
struct AdjWork {
  size_t plane_b = 0;  // bytes of one plane in the working precision
  int cap_k = 0, cap_l = 0;
  char* ck = nullptr;        // checkpoints, cap_k x 9 planes
  char* fin = nullptr;       // final state, 9 planes
  char* mu[2] = {nullptr, nullptr};  // adjoint state, 9 planes each
  char* uh = nullptr;        // u history of one segment, cap_l planes
  char* u0 = nullptr;        // u at the start of the call
  unsigned char* roots = nullptr;  // Neumann branches of one segment, cap_l x nedge
  double* gk = nullptr;      // [rows][pitch]
  float* gk32 = nullptr;     // [rows][pitch], FP32 lattice: one segment's share
  double* ge = nullptr;      // [3][nedge]: start, end, Neumann gradients
  double* jn0 = nullptr;     // east-edge sums before the call, [ny]
  double* part = nullptr;    // recompute scratch: mass partials
  double* jn = nullptr;      //   east-edge sums
  long long* inf = nullptr;  //   infeasible counters
};

void ctx_adjoint_free(lbm_ctx* c) {
  AdjWork* w = c->adj;
  if (!w) return;
  void* ptrs[] = {w->ck, w->fin, w->mu[0], w->mu[1], w->uh, w->u0, w->roots,
                  w->gk, w->ge,  w->jn0,   w->part,  w->jn, w->inf, w->gk32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete w;
  c->adj = nullptr;
}

namespace {

lbm_status ensure_work(lbm_ctx* c, int K, int L) {
  AdjWork* w = c->adj;
  if (w && w->cap_k >= K && w->cap_l >= L) return LBM_OK;
  ctx_drop_recorded(c, 1);  // recorded reverse sweeps write the old buffers
  ctx_adjoint_free(c);
  w = new AdjWork();
  c->adj = w;
  w->plane_b = (size_t)c->plane * c->esize;
  w->cap_k = K;
  w->cap_l = L;
  const size_t fb = 9 * w->plane_b;
  const size_t ne = (size_t)c->nedge;
  ACK(cudaMalloc((void**)&w->ck, (size_t)K * fb));
  ACK(cudaMalloc((void**)&w->fin, fb));
  ACK(cudaMalloc((void**)&w->mu[0], fb));
  ACK(cudaMalloc((void**)&w->mu[1], fb));
  ACK(cudaMalloc((void**)&w->uh, (size_t)L * w->plane_b));
  ACK(cudaMalloc((void**)&w->u0, w->plane_b));
  ACK(cudaMalloc((void**)&w->roots, (size_t)L * ne + 1));
  ACK(cudaMalloc((void**)&w->gk, (size_t)c->plane * sizeof(double)));
  ACK(cudaMalloc((void**)&w->gk32, (size_t)c->plane * sizeof(float)));
  ACK(cudaMalloc((void**)&w->ge, 3 * ne * sizeof(double)));
  ACK(cudaMalloc((void**)&w->jn0, (size_t)c->p.ny * sizeof(double)));
  // partials of a 32 x 8 launch or of a step launch, whichever is more
  const size_t parts = std::max((size_t)c->grid.x * c->grid.y, (size_t)c->sgrid.x * c->sgrid.y);
  ACK(cudaMalloc((void**)&w->part, parts * sizeof(double)));
  ACK(cudaMalloc((void**)&w->jn, (size_t)c->p.ny * sizeof(double)));
  ACK(cudaMalloc((void**)&w->inf, ne * sizeof(long long)));
  return LBM_OK;
}

template <typename Real>
AdjArgs<Real> adj_args(lbm_ctx* c, AdjWork* w, int mc, const Real* u_n,
                       const unsigned char* root, double frac) {
  AdjArgs<Real> a;
  a.mu_in = (const Real*)w->mu[mc];
  a.mu_out = (Real*)w->mu[mc ^ 1];
  a.link = c->link;
  a.vel = (const Real*)c->vel;
  a.kf = (const Real*)c->kf;
  a.u_n = u_n;
  a.root = root;
  a.gk = w->gk;
  a.gk32 = w->gk32;
  a.g_ua = w->ge;
  a.g_ub = w->ge + c->nedge;
  a.g_q = w->ge + 2 * c->nedge;
  a.status = c->status;
  a.plane = c->plane;
  a.nx = c->p.nx;
  a.ny = c->p.ny;
  a.pitch = c->pitch;
  a.per_x = c->p.edge[0] == LBM_EDGE_PERIODIC;
  a.per_y = c->p.edge[2] == LBM_EDGE_PERIODIC;
  for (int s = 0; s < 4; ++s) a.edge[s] = c->p.edge[s];
  a.react_mode = c->p.react_mode;
  a.omega = (Real)(1.0 / c->p.tau);
  a.k_scalar = (Real)c->p.k_scalar;
  a.frac = frac;
  return a;
}

template <typename Real>
lbm_status adjoint_impl(lbm_ctx* c, int n, int eta, int L) {
  const int K = (n + L - 1) / L;
  AdjWork* w = c->adj;  // sized by ensure_work(c, K, L) before the call
  const size_t pb = w->plane_b, fb = 9 * pb;
  const size_t ne = (size_t)c->nedge;
  cudaStream_t st = c->stream;
  const dim3 block(lbm::kBX, kAdjRows);
  const dim3 grid((c->p.nx + lbm::kBX - 1) / lbm::kBX, (c->p.ny + kAdjRows - 1) / kAdjRows);

  // forward, keeping a checkpoint every L steps; with one segment (K = 1)
  // the forward run records u and the Neumann branches of every step itself
  // and nothing is recomputed
  const bool whole = K == 1;
  ACK(cudaMemcpyAsync(w->u0, c->u, pb, cudaMemcpyDeviceToDevice, st));
  ACK(cudaMemcpyAsync(w->jn0, c->jnode, (size_t)c->p.ny * sizeof(double),
                      cudaMemcpyDeviceToDevice, st));
  if (whole) ACK(cudaMemsetAsync(w->roots, 0, (size_t)L * ne, st));
  for (int j = 1; j <= n; ++j) {
    if (!whole && (j - 1) % L == 0)
      ACK(cudaMemcpyAsync(w->ck + (size_t)((j - 1) / L) * fb, c->f[c->cur], fb,
                          cudaMemcpyDeviceToDevice, st));
    lbm::StepArgs<Real> a = step_args<Real>(c, (double)j / eta);
    if (whole) {
      a.u_hist = (Real*)(w->uh + (size_t)(j - 1) * pb);
      a.bc_root = w->roots + (size_t)(j - 1) * ne;
    }
    ATRY(ctx_launch_step<Real>(c, a, j == n));
    c->cur ^= 1;
    c->steps += 1;
  }
  const int cur_final = c->cur;
  const int nparts_final = c->nparts;
  ACK(cudaMemcpyAsync(w->fin, c->f[cur_final], fb, cudaMemcpyDeviceToDevice, st));

  // reverse sweep
  ACK(cudaMemsetAsync(w->mu[0], 0, fb, st));
  ACK(cudaMemsetAsync(w->mu[1], 0, fb, st));
  ACK(cudaMemsetAsync(w->gk, 0, (size_t)c->plane * sizeof(double), st));
  ACK(cudaMemsetAsync(w->gk32, 0, (size_t)c->plane * sizeof(float), st));
  ACK(cudaMemsetAsync(w->ge, 0, 3 * ne * sizeof(double), st));
  if (!whole) ACK(cudaMemsetAsync(w->roots, 0, (size_t)L * ne, st));
  int mc = 0;
  const long long fb_blocks = (c->plane + 255) / 256;
  const int fold_grid = (int)(fb_blocks < 4LL * c->num_sms ? fb_blocks : 4LL * c->num_sms);
  for (int s = K - 1; s >= 0; --s) {
    const int n0 = s * L, n1 = n0 + L < n ? n0 + L : n;
    if (!whole) {
      ACK(cudaMemcpyAsync(c->f[0], w->ck + (size_t)s * fb, fb, cudaMemcpyDeviceToDevice, st));
      c->cur = 0;
    }
    for (int j = n0 + 1; !whole && j <= n1; ++j) {
      // recompute: u of every step into the history (no mass sums: not a
      // final substep), the Neumann branches into their record
      lbm::StepArgs<Real> a = step_args<Real>(c, (double)j / eta);
      a.u_hist = (Real*)(w->uh + (size_t)(j - n0 - 1) * pb);
      a.bc_root = w->roots + (size_t)(j - n0 - 1) * ne;
      a.partial = w->part;
      a.jnode = w->jn;
      a.jflux = nullptr;  // the context keeps the forward run's last flux
      a.infeasible = w->inf;
      ATRY(ctx_launch_step<Real>(c, a, false));
      c->cur ^= 1;
    }
    // the FP32 lattice's dJ/dk is folded into the FP64 total after every
    // segment, and every ceil(sqrt(n)) steps of a whole-history sweep
    const int fold_every = whole ? (int)std::ceil(std::sqrt((double)n)) : 0;
    for (int j = n1; j > n0; --j) {
      const auto a = adj_args<Real>(c, w, mc, (const Real*)(w->uh + (size_t)(j - n0 - 1) * pb),
                                    w->roots + (size_t)(j - n0 - 1) * ne, (double)j / eta);
      lbm_adjoint_step<Real, false><<<grid, block, 0, st>>>(a);
      ACK(cudaGetLastError());
      mc ^= 1;
      if (sizeof(Real) == 4 && fold_every > 0 && j > n0 + 1 && (n1 - j + 1) % fold_every == 0) {
        k_fold_gk<<<fold_grid, 256, 0, st>>>(w->gk, w->gk32, c->plane);
        ACK(cudaGetLastError());
      }
    }
    if (sizeof(Real) == 4) {
      k_fold_gk<<<fold_grid, 256, 0, st>>>(w->gk, w->gk32, c->plane);
      ACK(cudaGetLastError());
    }
  }
  const auto a0 = adj_args<Real>(c, w, mc, (const Real*)w->u0, w->roots, 0.0);
  lbm_adjoint_step<Real, true><<<grid, block, 0, st>>>(a0);
  ACK(cudaGetLastError());
  if (sizeof(Real) == 4) {
    k_fold_gk<<<fold_grid, 256, 0, st>>>(w->gk, w->gk32, c->plane);
    ACK(cudaGetLastError());
  }

  // the context ends where the forward run left it
  ACK(cudaMemcpyAsync(c->f[cur_final], w->fin, fb, cudaMemcpyDeviceToDevice, st));
  c->cur = cur_final;
  c->nparts = nparts_final;
  return LBM_OK;
}

struct AdjCall {
  int n, eta, L;
};
template <typename Real>
lbm_status enqueue_adjoint(lbm_ctx* c, void* arg) {
  const AdjCall* a = (const AdjCall*)arg;
  return adjoint_impl<Real>(c, a->n, a->eta, a->L);
}

// A context the adjoint can differentiate: fixed mask, and no corner where
// two Neumann sides meet (that root is not affine in the data).
lbm_status check_adjoint(const lbm_ctx* c) {
  if (c->p.dissolution)
    return ctx_fail(LBM_ERR_STATE,
                    "lbm_adjoint: needs a fixed mask (the context dissolves; a flip is not "
                    "differentiable)");
  if (c->wall_mode != LBM_WALL_BOUNCE)
    return ctx_fail(LBM_ERR_STATE,
                    "lbm_adjoint: covers bounce-back pore walls only (the maximum-entropy "
                    "wall solve is not affine in f)");
  const int* e = c->p.edge;
  if (e[0] != LBM_EDGE_PERIODIC && e[2] != LBM_EDGE_PERIODIC)
    for (int xs = 0; xs < 2; ++xs)
      for (int ys = 2; ys < 4; ++ys)
        if (e[xs] == LBM_EDGE_NEUMANN && e[ys] == LBM_EDGE_NEUMANN)
          return ctx_fail(LBM_ERR_ARG,
                          "lbm_adjoint: two Neumann sides meet at a corner (the corner root "
                          "is not affine in the data)");
  return LBM_OK;
}

lbm_status copy_out(lbm_ctx* c, double* dst, const double* src, size_t count) {
  if (!dst) return LBM_OK;
  ACK(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, c->stream));
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_adjoint(lbm_ctx* c, int n, int eta, int stride, const double* u_dir_t0,
                       const double* u_dir_t1, const double* q_neu, double* J, double* grad_k,
                       double* grad_ua, double* grad_ub, double* grad_q, double* grad_side) {
  ATRY(ctx_check(c));
  if (n < 1 || eta < 1) return ctx_fail(LBM_ERR_ARG, "lbm_adjoint: need n >= 1 and eta >= 1");
  ATRY(check_adjoint(c));
  int L = stride;
  if (stride <= 0) {
    // the whole history when it takes at most a quarter of the free device
    // memory (no recompute), else sqrt(n) checkpoints
    size_t free_b = 0, total_b = 0;
    ACK(cudaMemGetInfo(&free_b, &total_b));
    const size_t whole_b = (size_t)n * ((size_t)c->plane * c->esize + (size_t)c->nedge) +
                           (size_t)c->plane * c->esize * 9;
    const size_t held = c->adj ? (size_t)c->adj->cap_l * c->adj->plane_b : 0;
    L = whole_b <= (free_b + held) / 4 ? n : (int)std::ceil(std::sqrt((double)n));
  }
  if (L > n) L = n;
  ATRY(ctx_stage_edges(c, u_dir_t0, u_dir_t1, q_neu));
  ATRY(ensure_work(c, (n + L - 1) / L, L));
  // the whole device sequence (forward with checkpoints, recompute, reverse
  // sweep) is one launch sequence, recorded on a repeated call and replayed
  AdjCall call{n, eta, L};
  const lbm_ctx::GraphKey key{1, n, eta, L, c->cur, walls_variant(c), c->use_tma ? 1 : 0};
  if (c->timing) ATRY(c->esize == 8 ? adjoint_impl<double>(c, n, eta, L)
                                    : adjoint_impl<float>(c, n, eta, L));
  else ATRY(ctx_run_recorded(c, key, c->esize == 8 ? enqueue_adjoint<double>
                                                    : enqueue_adjoint<float>, &call));
  AdjWork* w = c->adj;
  if (grad_k) ATRY(ctx_field_out_f64(c, w->gk, grad_k));
  const size_t ne = (size_t)c->nedge;
  ATRY(copy_out(c, grad_ua, w->ge, ne));
  ATRY(copy_out(c, grad_ub, w->ge + ne, ne));
  ATRY(copy_out(c, grad_q, w->ge + 2 * ne, ne));
  if (grad_side) {
    // dJ/d(a value held on a whole Dirichlet side): its slots' start and end
    // gradients summed in slot order
    std::vector<double> ge(2 * ne);
    ACK(cudaMemcpyAsync(ge.data(), w->ge, 2 * ne * sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream));
    ACK(cudaStreamSynchronize(c->stream));
    const int nx = c->p.nx, ny = c->p.ny;
    const int first[4] = {0, ny, 2 * ny, 2 * ny + nx}, len[4] = {ny, ny, nx, nx};
    double side[4];
    for (int sd = 0; sd < 4; ++sd) {
      double acc = 0.0;
      if (c->p.edge[sd] == LBM_EDGE_DIRICHLET)
        for (int k = first[sd]; k < first[sd] + len[sd]; ++k) acc += ge[k] + ge[ne + k];
      side[sd] = acc;
    }
    ACK(cudaMemcpyAsync(grad_side, side, sizeof(side), cudaMemcpyDefault, c->stream));
    ACK(cudaStreamSynchronize(c->stream));
  }
  if (J) {
    std::vector<double> after(c->p.ny), before(c->p.ny);
    ACK(cudaMemcpyAsync(after.data(), c->jnode, c->p.ny * sizeof(double),
                        cudaMemcpyDeviceToHost, c->stream));
    ACK(cudaMemcpyAsync(before.data(), w->jn0, c->p.ny * sizeof(double),
                        cudaMemcpyDeviceToHost, c->stream));
    ACK(cudaStreamSynchronize(c->stream));
    double s = 0.0;
    for (int y = 0; y < c->p.ny; ++y) s += after[y] - before[y];
    *J = s;
  }
  return ctx_status(c);
}

}  // extern "C"
