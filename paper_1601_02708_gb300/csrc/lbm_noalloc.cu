// lbm_noalloc.cu -- lbm_mass_noalloc: the FP64 mass reduction without any
// device allocation (declared in include/lbm_ade.h).
//
// The library's own mass sum (lbm_diagnostics) folds per-block partials that
// live in memory the library allocated for the context.  Some callers cannot
// allocate at the time they need the sum: code that works inside a device
// memory budget fixed at start-up (every byte is spoken for, so a new
// allocation can fail at any later point), or a host framework that owns
// every device allocation itself and forbids libraries to call cudaMalloc.
// This entry point takes the concentration field from the caller and keeps
// its partials in a fixed file-scope device array.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "lbm_ade.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 32;
constexpr long long kChunk = (long long)kThreads * kPerThread;  // nodes per block
constexpr int kMaxBlocks = 8192;  // => at most 8192 * 8192 = 67,108,864 nodes
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: one partial sum per block plus
// one slot for a result that goes back to host memory.  Every call overwrites
// the partials it folds, so nothing needs clearing between calls; calls that
// overlap on the GPU (different streams, no ordering) race on this array.
static __device__ __align__(256) double g_mass_scratch[kMaxBlocks + 1];

thread_local char g_msg[256] = "";

lbm_status fail(lbm_status s, const char* msg) {
  snprintf(g_msg, sizeof(g_msg), "%s", msg);
  return s;
}

// Each block sums its chunk of kChunk values (in a fixed order: per thread
// strided, then a fixed tree) into one FP64 partial.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    mass_partials(const T* __restrict__ u, long long n, double* __restrict__ part) {
  __shared__ double s[kThreads];
  const long long base = (long long)blockIdx.x * kChunk;
  double acc = 0.0;
  for (int k = 0; k < kPerThread; ++k) {
    const long long i = base + (long long)k * kThreads + threadIdx.x;
    if (i < n) acc += (double)u[i];
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// One block folds the partials in a fixed order.
__global__ void __launch_bounds__(kThreads)
    mass_fold(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  __shared__ double s[kThreads];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads) acc += part[b];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// Device address of the scratch array, looked up once per device with that
// device current (host code only sees a stand-in for the symbol).
std::mutex g_lock;
double* g_scratch_ptr[kMaxDevices] = {};

lbm_status scratch_for(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(LBM_ERR_ARG, "lbm_mass_noalloc: device id out of range");
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_mass_scratch);
    if (e != cudaSuccess) {
      snprintf(g_msg, sizeof(g_msg), "lbm_mass_noalloc: cudaGetSymbolAddress failed: %s",
               cudaGetErrorString(e));
      return LBM_ERR_CUDA;
    }
    g_scratch_ptr[dev] = (double*)p;
  }
  *out = g_scratch_ptr[dev];
  return LBM_OK;
}

bool is_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

lbm_status lbm_mass_noalloc(const void* u, int precision, long long n, double* mass_out,
                            void* stream) {
  g_msg[0] = 0;
  if (!u || !mass_out) return fail(LBM_ERR_ARG, "lbm_mass_noalloc: null pointer");
  if (precision != 32 && precision != 64)
    return fail(LBM_ERR_ARG, "lbm_mass_noalloc: precision must be 32 or 64");
  if (n < 1 || n > (long long)kMaxBlocks * kChunk)
    return fail(LBM_ERR_ARG,
                "lbm_mass_noalloc: n must be in [1, 67108864] (8192 x 8192 nodes)");
  if (!is_device(u))
    return fail(LBM_ERR_ARG, "lbm_mass_noalloc: the field must be in device memory");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "lbm_mass_noalloc: cudaGetDevice failed");
  double* scratch = nullptr;
  const lbm_status st = scratch_for(dev, &scratch);
  if (st != LBM_OK) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  const bool out_dev = is_device(mass_out);
  if (!out_dev) {
    // a host result needs a copy back and a wait for the stream; a stream in
    // capture mode allows no wait, so the call refuses instead of failing in
    // the middle
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "lbm_mass_noalloc: cudaStreamIsCapturing failed");
    if (cap != cudaStreamCaptureStatusNone)
      return fail(LBM_ERR_ARG,
                  "lbm_mass_noalloc: mass_out must be device memory while the stream is "
                  "being captured");
  }
  const int nblocks = (int)((n + kChunk - 1) / kChunk);
  if (precision == 64)
    mass_partials<double><<<nblocks, kThreads, 0, s>>>((const double*)u, n, scratch);
  else
    mass_partials<float><<<nblocks, kThreads, 0, s>>>((const float*)u, n, scratch);
  double* dst = out_dev ? mass_out : scratch + kMaxBlocks;
  mass_fold<<<1, kThreads, 0, s>>>(scratch, nblocks, dst);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "lbm_mass_noalloc: kernel launch failed");
  if (!out_dev) {
    e = cudaMemcpyAsync(mass_out, dst, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "lbm_mass_noalloc: copy of the result failed");
  }
  return LBM_OK;
}

const char* lbm_mass_noalloc_error(void) { return g_msg; }

}  // extern "C"
