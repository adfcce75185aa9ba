// lbm_species.cu -- the algebraic step of an instantaneous bimolecular
// reaction n_A A + n_B B -> n_C C (Sec. 7.2).  The invariants
//     alpha = u_A + (n_A / n_C) u_C,   beta = u_B + (n_B / n_C) u_C
// are not changed by the reaction, so the lattice transports them like any
// concentration; the species follow from them node by node:
//     u_A = max(alpha - (n_A / n_B) beta, 0),
//     u_B = (n_B / n_A) max((n_A / n_B) beta - alpha, 0),
//     u_C = (n_C / n_A) (alpha - u_A).
// Products and differences are rounded one by one (no fused multiply-add),
// so the results are those of the formulas evaluated as written.
#include <cuda_runtime.h>

#include <cmath>

#include "lbm_ade.h"
#include "lbm_ctx.h"

namespace {

__global__ void k_species(const double* __restrict__ al, const double* __restrict__ be,
                          long long n, double rAB, double rBA, double rCA, double* __restrict__ ua,
                          double* __restrict__ ub, double* __restrict__ uc) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double a = al[i];
    const double d = __dsub_rn(a, __dmul_rn(rAB, be[i]));  // alpha - (n_A / n_B) beta
    const double A = d > 0.0 ? d : 0.0;
    ua[i] = A;
    ub[i] = __dmul_rn(rBA, d < 0.0 ? -d : 0.0);
    uc[i] = __dmul_rn(rCA, __dsub_rn(a, A));
  }
}

__global__ void k_invariants(const double* __restrict__ ua, const double* __restrict__ ub,
                             const double* __restrict__ uc, long long n, double rAC, double rBC,
                             double* __restrict__ al, double* __restrict__ be) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double c = uc[i];
    al[i] = __dadd_rn(ua[i], __dmul_rn(rAC, c));
    be[i] = __dadd_rn(ub[i], __dmul_rn(rBC, c));
  }
}

// Calcite at equilibrium (Sec. 7.4, Eq. "Hybrid_Ksp" K_sp = u2 u3 / u1) from
// the invariants psi1 = u1 + u2 and psi2 = u3 - u2 (Eq. "Carbonate_uncoupled";
// the printed u1 - u2 is not conserved by the reaction, u1 + u2 is and gives
// the printed root): u2 is the non-negative root of
// u2^2 + (psi2 + K_sp) u2 - K_sp psi1 = 0.  Written as printed,
// (-(psi2 + K_sp) + sqrt(...)) / 2 cancels catastrophically when
// psi2 + K_sp > 0 and K_sp psi1 is small (K_sp = 3.36e-9: u2 ~ 1e-8 from two
// O(0.1) terms); the same root as 2 K_sp psi1 / ((psi2 + K_sp) + sqrt(...))
// does not, so that form is used there.  u1 = psi1 - u2, u3 = psi2 + u2.
__global__ void k_calcite(const double* __restrict__ p1, const double* __restrict__ p2,
                          long long n, double ksp, double* __restrict__ u1,
                          double* __restrict__ u2, double* __restrict__ u3) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double a = p1[i], b = p2[i];
    const double s = b + ksp;
    const double r = sqrt(s * s + 4.0 * ksp * a);
    const double c = s > 0.0 ? 2.0 * ksp * a / (s + r) : 0.5 * (r - s);
    u1[i] = a - c;
    u2[i] = c;
    u3[i] = b + c;
  }
}

__global__ void k_calcite_inv(const double* __restrict__ u1, const double* __restrict__ u2,
                              const double* __restrict__ u3, long long n,
                              double* __restrict__ p1, double* __restrict__ p2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    p1[i] = u1[i] + u2[i];
    p2[i] = u3[i] - u2[i];
  }
}

bool ratios_ok(double nA, double nB, double nC) {
  return std::isfinite(nA) && std::isfinite(nB) && std::isfinite(nC) && nA > 0 && nB > 0 &&
         nC > 0;
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return (int)b;
}

// Runs `launch(device pointers...)` on `k` input and `m` output arrays of n
// doubles: device arrays are used in place, host arrays are staged through
// one device buffer (and the outputs copied back before returning).
template <class F>
lbm_status with_device_arrays(long long n, cudaStream_t s, const double* const* in, int k,
                              double* const* out, int m, const char* who, F launch) {
  bool all_dev = true;
  for (int i = 0; i < k; ++i) all_dev = all_dev && ctx_on_device(in[i]);
  for (int i = 0; i < m; ++i) all_dev = all_dev && ctx_on_device(out[i]);
  const double* din[3];
  double* dout[3];
  double* buf = nullptr;
  if (all_dev) {
    for (int i = 0; i < k; ++i) din[i] = in[i];
    for (int i = 0; i < m; ++i) dout[i] = out[i];
  } else {
    cudaError_t e = cudaMalloc((void**)&buf, (size_t)(k + m) * n * sizeof(double));
    if (e != cudaSuccess)
      return ctx_fail(LBM_ERR_NOMEM, "%s: cudaMalloc: %s", who, cudaGetErrorString(e));
    for (int i = 0; i < k; ++i) {
      din[i] = buf + (size_t)i * n;
      e = cudaMemcpyAsync(const_cast<double*>(din[i]), in[i], n * sizeof(double),
                          cudaMemcpyDefault, s);
      if (e != cudaSuccess) {
        cudaFree(buf);
        return ctx_fail(LBM_ERR_CUDA, "%s: copy in: %s", who, cudaGetErrorString(e));
      }
    }
    for (int i = 0; i < m; ++i) dout[i] = buf + (size_t)(k + i) * n;
  }
  launch(din, dout);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !all_dev)
    for (int i = 0; i < m && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(out[i], dout[i], n * sizeof(double), cudaMemcpyDefault, s);
  if (e == cudaSuccess && !all_dev) e = cudaStreamSynchronize(s);
  if (buf) cudaFree(buf);
  if (e != cudaSuccess) return ctx_fail(LBM_ERR_CUDA, "%s: %s", who, cudaGetErrorString(e));
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_species_from_invariants(long long n, double nA, double nB, double nC,
                                       const double* alpha, const double* beta, double* uA,
                                       double* uB, double* uC, void* stream) {
  const char* who = "lbm_species_from_invariants";
  if (n < 0 || !ratios_ok(nA, nB, nC) || (n > 0 && (!alpha || !beta || !uA || !uB || !uC)))
    return ctx_fail(LBM_ERR_ARG, "%s: bad arguments", who);
  if (n == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const double rAB = nA / nB, rBA = nB / nA, rCA = nC / nA;
  const double* in[2] = {alpha, beta};
  double* out[3] = {uA, uB, uC};
  return with_device_arrays(n, s, in, 2, out, 3, who, [&](const double* const* d, double* const* o) {
    k_species<<<grid_for(n), 256, 0, s>>>(d[0], d[1], n, rAB, rBA, rCA, o[0], o[1], o[2]);
  });
}

lbm_status lbm_invariants_from_species(long long n, double nA, double nB, double nC,
                                       const double* uA, const double* uB, const double* uC,
                                       double* alpha, double* beta, void* stream) {
  const char* who = "lbm_invariants_from_species";
  if (n < 0 || !ratios_ok(nA, nB, nC) || (n > 0 && (!alpha || !beta || !uA || !uB || !uC)))
    return ctx_fail(LBM_ERR_ARG, "%s: bad arguments", who);
  if (n == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const double rAC = nA / nC, rBC = nB / nC;
  const double* in[3] = {uA, uB, uC};
  double* out[2] = {alpha, beta};
  return with_device_arrays(n, s, in, 3, out, 2, who, [&](const double* const* d, double* const* o) {
    k_invariants<<<grid_for(n), 256, 0, s>>>(d[0], d[1], d[2], n, rAC, rBC, o[0], o[1]);
  });
}

lbm_status lbm_calcite_species(long long n, double ksp, const double* psi1, const double* psi2,
                               double* u1, double* u2, double* u3, void* stream) {
  const char* who = "lbm_calcite_species";
  if (n < 0 || !(std::isfinite(ksp) && ksp > 0.0) ||
      (n > 0 && (!psi1 || !psi2 || !u1 || !u2 || !u3)))
    return ctx_fail(LBM_ERR_ARG, "%s: bad arguments", who);
  if (n == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const double* in[2] = {psi1, psi2};
  double* out[3] = {u1, u2, u3};
  return with_device_arrays(n, s, in, 2, out, 3, who, [&](const double* const* d, double* const* o) {
    k_calcite<<<grid_for(n), 256, 0, s>>>(d[0], d[1], n, ksp, o[0], o[1], o[2]);
  });
}

lbm_status lbm_calcite_invariants(long long n, const double* u1, const double* u2,
                                  const double* u3, double* psi1, double* psi2, void* stream) {
  const char* who = "lbm_calcite_invariants";
  if (n < 0 || (n > 0 && (!u1 || !u2 || !u3 || !psi1 || !psi2)))
    return ctx_fail(LBM_ERR_ARG, "%s: bad arguments", who);
  if (n == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const double* in[3] = {u1, u2, u3};
  double* out[2] = {psi1, psi2};
  return with_device_arrays(n, s, in, 3, out, 2, who, [&](const double* const* d, double* const* o) {
    k_calcite_inv<<<grid_for(n), 256, 0, s>>>(d[0], d[1], d[2], n, o[0], o[1]);
  });
}

}  // extern "C"
