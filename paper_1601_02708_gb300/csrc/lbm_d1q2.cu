// lbm_d1q2.cu -- the D1Q2 lattice of the one-dimensional hybrid (Sec. 7.1),
// declared in include/lbm_ade.h (lbm1d_*).
//
// D1Q2: velocities +-c (c = h / dt), weights 1/2, c_s^2 = c^2; in lattice
// units D dt / h^2 = tau - 1/2 and the equilibrium of Eq. "LBM_feq" is
// f_+- = (u/2)(1 +- vl), vl = v dt / h.  One step streams the stored
// post-collision populations (f_+ moves right, f_- left), sets the one
// unknown population at each end by the maximum-entropy conditions of
// Sec. 4.1.1 (a Dirichlet end: the unknown takes the missing mass; a Neumann
// end: the unknown's e.n = -1, so it equals the known one minus the flux
// datum -- zero flux is bounce-back), takes u = f_+ + f_- (Eq. "LBM_Macro")
// and collides (Eq. "Collision").  The lattice of the 1-D runs has a few
// thousand nodes: one thread block holds it and runs all n substeps of a
// call in one launch, synchronising between steps, in FP64 throughout.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <new>

#include "lbm_ade.h"
#include "lbm_ctx.h"

struct lbm1d {
  int n = 0;
  double tau = 1.0, vl = 0.0;
  int kind[2] = {LBM_EDGE_DIRICHLET, LBM_EDGE_NEUMANN};  // left, right
  double* f[2] = {nullptr, nullptr};  // [2][n] post-collision populations (+, -)
  double* u = nullptr;                // [n] concentration at the current time
  double* data = nullptr;             // [6]: a_left, a_right, b_left, b_right, q_left, q_right
  int cur = 0;
  long long steps = 0;
  cudaStream_t stream = nullptr;
};

namespace {

constexpr int kThreads = 1024;

struct Args1d {
  const double* fin;
  double* fout_a;  // the two buffers: fin is one of them
  double* fout_b;
  double* u;
  const double* data;
  int n, steps, eta, j0;
  int kind_l, kind_r;
  double omega, vl;
};

// One collision of node values (u, f_+, f_-), stored post-collision.
__device__ __forceinline__ void collide1(double u, double& fp, double& fm, double omega,
                                         double vl) {
  const double ep = 0.5 * u * (1.0 + vl), em = 0.5 * u * (1.0 - vl);
  fp = fp - omega * (fp - ep);
  fm = fm - omega * (fm - em);
}

// n substeps j0 + 1 .. j0 + steps of eta in one block: each step pulls from
// the buffer the previous step wrote (the two buffers alternate).
__global__ void __launch_bounds__(kThreads) k_d1q2_steps(Args1d a) {
  const double* src = a.fin;
  double* dst = (src == a.fout_a) ? a.fout_b : a.fout_a;
  for (int s = 1; s <= a.steps; ++s) {
    const double frac = (double)(a.j0 + s) / (double)a.eta;
    for (int x = threadIdx.x; x < a.n; x += blockDim.x) {
      // pull: f_+ from x - 1, f_- from x + 1 (src planes: [0, n) plus, [n, 2n) minus)
      double fp = x > 0 ? src[x - 1] : 0.0;
      double fm = x < a.n - 1 ? src[a.n + x + 1] : 0.0;
      if (x == 0) {  // unknown f_+
        const double up = (1.0 - frac) * a.data[0] + frac * a.data[2];
        fp = a.kind_l == LBM_EDGE_DIRICHLET ? up - fm : fm - a.data[4];
      }
      if (x == a.n - 1) {  // unknown f_-
        const double up = (1.0 - frac) * a.data[1] + frac * a.data[3];
        fm = a.kind_r == LBM_EDGE_DIRICHLET ? up - fp : fp - a.data[5];
      }
      const double u = fp + fm;
      a.u[x] = u;
      collide1(u, fp, fm, a.omega, a.vl);
      dst[x] = fp;
      dst[a.n + x] = fm;
    }
    __syncthreads();
    const double* t = src;
    src = dst;
    dst = const_cast<double*>(t);
  }
}

__global__ void k_d1q2_init(double* f, double* u, const double* u0, int n, double omega,
                            double vl) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    const double u0x = u0 ? u0[x] : 0.0;
    double fp = 0.5 * u0x * (1.0 + vl), fm = 0.5 * u0x * (1.0 - vl);  // f = f^eq(u0)
    u[x] = u0x;
    collide1(u0x, fp, fm, omega, vl);  // stored post-collision, like the 2-D lattice
    f[x] = fp;
    f[n + x] = fm;
  }
}

#define DCK(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return ctx_fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA,   \
                      "%s failed: %s", #call, cudaGetErrorString(e_));                   \
  } while (0)

void free1d(lbm1d* c) {
  if (!c) return;
  for (void* p : {(void*)c->f[0], (void*)c->f[1], (void*)c->u, (void*)c->data})
    if (p) cudaFree(p);
  delete c;
}

}  // namespace

extern "C" {

lbm_status lbm1d_init(lbm1d** out, int n, double tau, double vl, int left, int right,
                      const double* u0, void* stream) {
  if (!out) return ctx_fail(LBM_ERR_ARG, "lbm1d_init: null out");
  *out = nullptr;
  if (n < 2 || !(tau > 0.5) || !(vl > -1.0 && vl < 1.0))
    return ctx_fail(LBM_ERR_ARG, "lbm1d_init: need n >= 2, tau > 1/2, |vl| < 1");
  for (int k : {left, right})
    if (k != LBM_EDGE_DIRICHLET && k != LBM_EDGE_NEUMANN)
      return ctx_fail(LBM_ERR_ARG, "lbm1d_init: ends must be Dirichlet or Neumann");
  lbm1d* c = new (std::nothrow) lbm1d();
  if (!c) return ctx_fail(LBM_ERR_NOMEM, "lbm1d_init: host allocation failed");
  c->n = n;
  c->tau = tau;
  c->vl = vl;
  c->kind[0] = left;
  c->kind[1] = right;
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaMalloc((void**)&c->f[0], 2 * (size_t)n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->f[1], 2 * (size_t)n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->u, (size_t)n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->data, 6 * sizeof(double));
  double* du0 = nullptr;
  if (e == cudaSuccess && u0) {
    e = cudaMalloc((void**)&du0, (size_t)n * sizeof(double));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(du0, u0, (size_t)n * sizeof(double), cudaMemcpyDefault, c->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->data, 0, 6 * sizeof(double), c->stream);
  if (e == cudaSuccess) {
    k_d1q2_init<<<(n + 255) / 256, 256, 0, c->stream>>>(c->f[0], c->u, du0, n, 1.0 / tau, vl);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (du0) cudaFree(du0);
  if (e != cudaSuccess) {
    free1d(c);
    return ctx_fail(LBM_ERR_CUDA, "lbm1d_init: %s", cudaGetErrorString(e));
  }
  *out = c;
  return LBM_OK;
}

lbm_status lbm1d_substeps(lbm1d* c, int n, int eta, const double* ends_t0,
                          const double* ends_t1, const double* q) {
  if (!c) return ctx_fail(LBM_ERR_ARG, "lbm1d_substeps: null lattice");
  if (n < 0 || eta < 1) return ctx_fail(LBM_ERR_ARG, "lbm1d_substeps: need n >= 0, eta >= 1");
  if (n == 0) return LBM_OK;
  double h[6] = {0, 0, 0, 0, 0, 0};
  if (ends_t0) DCK(cudaMemcpy(h, ends_t0, 2 * sizeof(double), cudaMemcpyDefault));
  const double* b = ends_t1 ? ends_t1 : ends_t0;
  if (b) DCK(cudaMemcpy(h + 2, b, 2 * sizeof(double), cudaMemcpyDefault));
  if (q) DCK(cudaMemcpy(h + 4, q, 2 * sizeof(double), cudaMemcpyDefault));
  DCK(cudaMemcpyAsync(c->data, h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
  Args1d a;
  a.fin = c->f[c->cur];
  a.fout_a = c->f[0];
  a.fout_b = c->f[1];
  a.u = c->u;
  a.data = c->data;
  a.n = c->n;
  a.steps = n;
  a.eta = eta;
  a.j0 = 0;
  a.kind_l = c->kind[0];
  a.kind_r = c->kind[1];
  a.omega = 1.0 / c->tau;
  a.vl = c->vl;
  k_d1q2_steps<<<1, kThreads, 0, c->stream>>>(a);
  DCK(cudaGetLastError());
  DCK(cudaStreamSynchronize(c->stream));  // the staged end data live on this frame
  c->cur ^= (n & 1);
  c->steps += n;
  return LBM_OK;
}

lbm_status lbm1d_get(lbm1d* c, double* u) {
  if (!c || !u) return ctx_fail(LBM_ERR_ARG, "lbm1d_get: null argument");
  DCK(cudaMemcpyAsync(u, c->u, (size_t)c->n * sizeof(double), cudaMemcpyDefault, c->stream));
  DCK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm1d_state_bytes(lbm1d* c, size_t* bytes) {
  if (!c || !bytes) return ctx_fail(LBM_ERR_ARG, "lbm1d_state_bytes: null argument");
  *bytes = 3 * (size_t)c->n * sizeof(double);
  return LBM_OK;
}

lbm_status lbm1d_save(lbm1d* c, void* buf, size_t bytes) {
  size_t need = 0;
  const lbm_status st = lbm1d_state_bytes(c, &need);
  if (st != LBM_OK) return st;
  if (!buf || bytes < need) return ctx_fail(LBM_ERR_ARG, "lbm1d_save: buffer too small");
  const size_t fb = 2 * (size_t)c->n * sizeof(double);
  DCK(cudaMemcpyAsync(buf, c->f[c->cur], fb, cudaMemcpyDefault, c->stream));
  DCK(cudaMemcpyAsync((char*)buf + fb, c->u, (size_t)c->n * sizeof(double), cudaMemcpyDefault,
                      c->stream));
  DCK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm1d_restore(lbm1d* c, const void* buf, size_t bytes) {
  size_t need = 0;
  const lbm_status st = lbm1d_state_bytes(c, &need);
  if (st != LBM_OK) return st;
  if (!buf || bytes < need) return ctx_fail(LBM_ERR_ARG, "lbm1d_restore: buffer too small");
  const size_t fb = 2 * (size_t)c->n * sizeof(double);
  DCK(cudaMemcpyAsync(c->f[c->cur], buf, fb, cudaMemcpyDefault, c->stream));
  DCK(cudaMemcpyAsync(c->u, (const char*)buf + fb, (size_t)c->n * sizeof(double),
                      cudaMemcpyDefault, c->stream));
  DCK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

void lbm1d_destroy(lbm1d* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free1d(c);
}

}  // extern "C"
