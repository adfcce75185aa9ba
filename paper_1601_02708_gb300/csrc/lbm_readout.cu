// lbm_readout.cu -- read-outs the step does not need: the smallest stored
// population over the fluid nodes, the check of the condition that keeps
// the populations non-negative (Sec. 4.1, Eq. "NN_Cond", and the
// non-negativity of the maximum-entropy boundary data).  A minimum is the
// same in any order, so the fold is exact.
#include <cuda_runtime.h>

#include <cmath>

#include "lbm_ade.h"
#include "lbm_ctx.h"

namespace {

constexpr int kThreads = 256;

template <typename Real>
__global__ void __launch_bounds__(kThreads)
    k_min_pop(const Real* __restrict__ f, const uint32_t* __restrict__ link, int nx, int ny,
              int pitch, long long plane, double* __restrict__ part) {
  double m = INFINITY;
  const long long total = (long long)nx * ny;
  for (long long id = blockIdx.x * (long long)kThreads + threadIdx.x; id < total;
       id += (long long)gridDim.x * kThreads) {
    const int y = (int)(id / nx), x = (int)(id - (long long)y * nx);
    const long long n = (long long)(y + lbm::kYO) * pitch + (x + lbm::kXO);
    if (link[n] & lbm::kOwnSolid) continue;  // solid (or turning fluid): no populations
#pragma unroll
    for (int i = 0; i < 9; ++i) m = fmin(m, (double)f[i * plane + n]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ double w[kThreads / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = w[0];
    for (int k = 1; k < kThreads / 32; ++k) b = fmin(b, w[k]);
    part[blockIdx.x] = b;
  }
}

__global__ void k_min_fold(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double m = INFINITY;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmin(m, part[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ double w[kThreads / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = w[0];
    for (int k = 1; k < kThreads / 32; ++k) b = fmin(b, w[k]);
    *out = b;
  }
}

}  // namespace

extern "C" lbm_status lbm_min_population(lbm_ctx* c, double* out) {
  const lbm_status chk = ctx_check(c);
  if (chk != LBM_OK) return chk;
  if (!out) return ctx_fail(LBM_ERR_ARG, "lbm_min_population: null out");
  const long long total = (long long)c->p.nx * c->p.ny;
  long long nb = (total + kThreads - 1) / kThreads;
  const long long cap = 8LL * (c->num_sms > 0 ? c->num_sms : 1);
  if (nb > cap) nb = cap;
  if (nb < 1) nb = 1;
  double* buf = nullptr;
  cudaError_t e = cudaMalloc((void**)&buf, (size_t)(nb + 1) * sizeof(double));
  if (e != cudaSuccess)
    return ctx_fail(LBM_ERR_NOMEM, "lbm_min_population: cudaMalloc: %s", cudaGetErrorString(e));
  if (c->esize == 8)
    k_min_pop<double><<<(int)nb, kThreads, 0, c->stream>>>(
        (const double*)c->f[c->cur], c->link, c->p.nx, c->p.ny, c->pitch, c->plane, buf);
  else
    k_min_pop<float><<<(int)nb, kThreads, 0, c->stream>>>(
        (const float*)c->f[c->cur], c->link, c->p.nx, c->p.ny, c->pitch, c->plane, buf);
  k_min_fold<<<1, kThreads, 0, c->stream>>>(buf, (int)nb, buf + nb);
  double h = 0.0;
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h, buf + nb, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(buf);
  if (e != cudaSuccess)
    return ctx_fail(LBM_ERR_CUDA, "lbm_min_population: %s", cudaGetErrorString(e));
  const lbm_status st = ctx_status(c);
  if (st != LBM_OK) return st;
  *out = h;
  return LBM_OK;
}
