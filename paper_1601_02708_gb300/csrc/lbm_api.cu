// lbm_api.cu -- C ABI of liblbmade.so (declared in include/lbm_ade.h).
//
// Owns the device state of one lattice and launches the kernels of
// lbm_kernels.cuh / lbm_tma.cuh on the context's stream.  Host-side work is
// argument checking, residency detection of caller pointers, layout
// conversion and launch bookkeeping.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "lbm_ade.h"
#include "lbm_kernels.cuh"
#include "lbm_tma.cuh"
#include "lbm_ctx.h"

namespace {

thread_local char g_err[512] = "";

lbm_status fail(lbm_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

#define CK(call)                                                              \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM             \
                                                  : LBM_ERR_CUDA,             \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                  __FILE__, __LINE__);                                        \
  } while (0)

#define TRY(...)                       \
  do {                                 \
    lbm_status s_ = (__VA_ARGS__);     \
    if (s_ != LBM_OK) return s_;       \
  } while (0)

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaMemcpyKind kind_from(const void* p) {
  return on_device(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}

using lbm::kXO;
using lbm::kYO;

// ---- layout conversion kernels (interior [ny][nx] <-> padded) -------------
template <typename T>
__global__ void k_pitch_in(const double* __restrict__ src, T* __restrict__ dst, int nx,
                           int ny, int pitch, int planes, double fill) {
  const long long total = (long long)nx * ny * planes;
  const long long plane = (long long)pitch * lbm::padded_rows(ny);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / ((long long)nx * ny), r = i % ((long long)nx * ny);
    const long long y = r / nx, x = r % nx;
    dst[p * plane + (y + kYO) * pitch + (x + kXO)] = (T)(src ? src[i] : fill);
  }
}

// Link word of every interior node (see lbm_lattice.cuh) from the caller's
// solid array of the whole lattice ([nyg][nx]); the context holds rows
// y0 .. y0 + nyl - 1 of it (all of it unless the lattice is split into
// slabs).  Periodic sides wrap, other sides are outside.  With ghost_s /
// ghost_n set (the slab's S / N side is shared with a neighbouring slab) the
// row beyond it is the neighbour's boundary row: its nodes' own solid bits are
// written into the ghost row, and the links that cross into it are set from
// the whole lattice's mask like any other.
__global__ void k_link_in(const uint8_t* __restrict__ src, uint32_t* __restrict__ link, int nx,
                          int nyl, int y0, int nyg, int pitch, int per_x, int per_yg,
                          int ghost_s, int ghost_n) {
  const int rows = nyl + ghost_s + ghost_n;
  const long long total = (long long)nx * rows;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(id % nx), yl = (int)(id / nx) - ghost_s;
    int yg = y0 + yl;
    if (yg < 0 || yg >= nyg) yg = ((yg % nyg) + nyg) % nyg;  // ghost row across the wrap
    const bool me_solid = src && src[(long long)yg * nx + x];
    uint32_t w = me_solid ? lbm::kOwnSolid : 0u;
    if (yl >= 0 && yl < nyl) {
      for (int i = 1; i < 9; ++i) {
        int sx = x - lbm::cx_of(i), sy = yg - lbm::cy_of(i);
        bool out = false;
        if (sx < 0 || sx >= nx) {
          if (per_x) sx = (sx + nx) % nx; else out = true;
        }
        if (sy < 0 || sy >= nyg) {
          if (per_yg) sy = (sy + nyg) % nyg; else out = true;
        }
        if (out) w |= lbm::up_bit(lbm::kUpOutShift, i);
        else if (src && src[(long long)sy * nx + sx])
          w |= lbm::up_bit(lbm::kUpSolidShift, i) | lbm::up_bit(lbm::kUpPostShift, i);
      }
    }
    link[(long long)(yl + kYO) * pitch + (x + kXO)] = w;
  }
}

template <typename T, typename O>
__global__ void k_pitch_out(const T* __restrict__ src, O* __restrict__ dst, int nx, int ny,
                            int pitch, int planes) {
  const long long total = (long long)nx * ny * planes;
  const long long plane = (long long)pitch * lbm::padded_rows(ny);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / ((long long)nx * ny), r = i % ((long long)nx * ny);
    const long long y = r / nx, x = r % nx;
    dst[i] = (O)src[p * plane + (y + kYO) * pitch + (x + kXO)];
  }
}

__global__ void k_solid_out(const uint32_t* __restrict__ link, uint8_t* __restrict__ dst,
                            int nx, int ny, int pitch) {
  const long long total = (long long)nx * ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long y = i / nx, x = i % nx;
    dst[i] = (link[(y + kYO) * pitch + (x + kXO)] & lbm::kOwnSolid) ? 1 : 0;
  }
}

// Solid-node count (integer sums in any order give the same result).
__global__ void k_count_solid(const uint32_t* __restrict__ link, int nx, int ny, int pitch,
                              unsigned long long* out) {
  unsigned long long c = 0;
  const long long total = (long long)nx * ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long y = i / nx, x = i % nx;
    c += (link[(y + kYO) * pitch + (x + kXO)] & lbm::kOwnSolid) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Fixed-order FP64 reductions for lbm_diagnostics (one block).
__global__ void k_diag(const double* __restrict__ partial, int nparts,
                       const double* __restrict__ jnode, const double* __restrict__ jflux,
                       int ny, const long long* __restrict__ infeas, int nedge, DiagDev* out) {
  __shared__ double sd[256];
  __shared__ long long sl[256];
  const int t = threadIdx.x;
  double m = 0.0, j = 0.0, q = 0.0;
  long long c = 0;
  for (int i = t; i < nparts; i += blockDim.x) m += partial[i];
  for (int i = t; i < ny; i += blockDim.x) j += jnode[i];
  for (int i = t; i < ny; i += blockDim.x) q += jflux[i];
  for (int i = t; i < nedge; i += blockDim.x) c += infeas[i];
  double* outs[3] = {&out->mass, &out->J, &out->flux};
  double vals[3] = {m, j, q};
  for (int k = 0; k < 3; ++k) {
    sd[t] = vals[k];
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      for (int i = 0; i < (int)blockDim.x; ++i) s += sd[i];
      *outs[k] = s;
    }
    __syncthreads();
  }
  sl[t] = c;
  __syncthreads();
  if (t == 0) {
    long long s = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) s += sl[i];
    out->infeasible = s;
  }
}

// LBM -> FEM transfer (Sec. 6.2 (ii)): bilinear patch of the four nodes
// around each point.
template <typename Real>
__global__ void k_trace(const Real* __restrict__ u, int nx, int ny, int pitch, int per_x,
                        int per_y, const double* __restrict__ xy, int npts,
                        double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npts) return;
  const double px = xy[2 * k], py = xy[2 * k + 1];
  const bool bad = !isfinite(px) || !isfinite(py) ||
                   (!per_x && !(px >= 0.0 && px <= nx - 1)) ||
                   (!per_y && !(py >= 0.0 && py <= ny - 1));
  if (bad) {
    out[k] = nan("");
    return;
  }
  int x1 = (int)floor(px), y1 = (int)floor(py);
  if (!per_x && x1 >= nx - 1) x1 = nx - 2;
  if (!per_y && y1 >= ny - 1) y1 = ny - 2;
  const double gx = px - x1, gy = py - y1;
  int ax = x1, ay = y1, bx = x1 + 1, by = y1 + 1;
  if (per_x) { ax = ((ax % nx) + nx) % nx; bx = ((bx % nx) + nx) % nx; }
  if (per_y) { ay = ((ay % ny) + ny) % ny; by = ((by % ny) + ny) % ny; }
  auto U = [&](int xx, int yy) {
    return (double)u[(long long)(yy + kYO) * pitch + (xx + kXO)];
  };
  out[k] = U(ax, ay) * (1 - gx) * (1 - gy) + U(bx, ay) * gx * (1 - gy) +
           U(bx, by) * gx * gy + U(ax, by) * (1 - gx) * gy;
}

int grid1d(long long n) {
  long long b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (int)b;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

namespace {

lbm_status fold_times(lbm_ctx* c, int which) {
  if (c->ev_used[which] == 0) return LBM_OK;
  CK(cudaEventSynchronize(c->ev[which][c->ev_used[which] - 1][1]));
  for (int i = 0; i < c->ev_used[which]; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev[which][i][0], c->ev[which][i][1]));
    c->ms_sum[which] += ms;
  }
  c->launches[which] += c->ev_used[which];
  c->ev_used[which] = 0;
  return LBM_OK;
}

// Record the opening event of a timed launch (which: 0 step, 1 dissolve).
lbm_status time_begin(lbm_ctx* c, int which) {
  if (!c->timing) return LBM_OK;
  if (c->ev_used[which] == lbm_ctx::kPool) TRY(fold_times(c, which));
  cudaEvent_t* e = c->ev[which][c->ev_used[which]];
  if (!e[0]) {
    CK(cudaEventCreate(&e[0]));
    CK(cudaEventCreate(&e[1]));
  }
  CK(cudaEventRecord(e[0], c->stream));
  return LBM_OK;
}
lbm_status time_end(lbm_ctx* c, int which) {
  if (!c->timing) return LBM_OK;
  CK(cudaEventRecord(c->ev[which][c->ev_used[which]][1], c->stream));
  c->ev_used[which] += 1;
  return LBM_OK;
}

// The reaction shares the step stores for the dissolution pass: double on
// the FP64 lattice, ShareF32 on the FP32 lattice.
template <typename Real>
using ShareOf = typename std::conditional<sizeof(Real) == 8, double, lbm::ShareF32>::type;

template <typename Real>
lbm_status launch_dissolve(lbm_ctx* c) {
  TRY(time_begin(c, 1));
  lbm::lbm_dissolve_list<ShareOf<Real>><<<c->dgrid, lbm::kDThreads, 0, c->stream>>>(
      dissolve_args(c), (const ShareOf<Real>*)c->ureact);
  CK(cudaGetLastError());
  return time_end(c, 1);
}

// First dissolution pass after initialisation: over every node (it also
// flips solid nodes given no mineral), then the surface list is built.
template <typename Real>
lbm_status first_dissolve(lbm_ctx* c) {
  lbm::DissolveArgs d = dissolve_args(c);
  d.check_all = 1;
  lbm::lbm_dissolve_dense<ShareOf<Real>><<<c->dgrid, lbm::kDThreads, 0, c->stream>>>(
      d, (const ShareOf<Real>*)c->ureact);
  CK(cudaGetLastError());
  lbm::lbm_list_build<<<c->dgrid, lbm::kDThreads, 0, c->stream>>>(dissolve_args(c));
  CK(cudaGetLastError());
  return LBM_OK;
}

// Dense mineral array up to date (the listed nodes keep theirs on the list).
lbm_status sync_mineral(lbm_ctx* c) {
  if (!c->p.dissolution) return LBM_OK;
  lbm::lbm_list_scatter<<<c->dgrid, lbm::kDThreads, 0, c->stream>>>(dissolve_args(c));
  CK(cudaGetLastError());
  return LBM_OK;
}

// The step kernels are built without wall code and with the two precisions
// of the maximum-entropy wall solve (walls_variant); a context runs the one
// its wall mode needs.
template <typename Real, int kWalls>
lbm_status launch_step_kernels(lbm_ctx* c, const lbm::StepArgs<Real>& a, bool final_step) {
  if (sizeof(Real) == 4 && c->use_tma) {
    const lbm::TmaMaps& m = c->maps[c->cur];
    const auto& af = reinterpret_cast<const lbm::StepArgs<float>&>(a);
    if (final_step)
      lbm::lbm_step_tma<true, kWalls><<<c->tma_grid, lbm::kTmaBlock, lbm::kTmaSmem, c->stream>>>(
          af, m, c->ntx, c->nty);
    else
      lbm::lbm_step_tma<false, kWalls><<<c->tma_grid, lbm::kTmaBlock, lbm::kTmaSmem, c->stream>>>(
          af, m, c->ntx, c->nty);
    if (final_step) c->nparts = c->tma_grid;
  } else {
    if (final_step)
      lbm::lbm_step<Real, true, kWalls><<<c->sgrid, c->sblock, 0, c->stream>>>(a);
    else
      lbm::lbm_step<Real, false, kWalls><<<c->sgrid, c->sblock, 0, c->stream>>>(a);
    if (final_step) c->nparts = (int)(c->sgrid.x * c->sgrid.y);
  }
  CK(cudaGetLastError());
  return LBM_OK;
}

template <typename Real>
lbm_status launch_step_impl(lbm_ctx* c, const lbm::StepArgs<Real>& a, bool final_step) {
  switch (walls_variant(c)) {
    case 0: return launch_step_kernels<Real, 0>(c, a, final_step);
    case 1: return launch_step_kernels<Real, 1>(c, a, final_step);
    default:
      if constexpr (sizeof(Real) == 4) return launch_step_kernels<Real, 2>(c, a, final_step);
      return launch_step_kernels<Real, 1>(c, a, final_step);
  }
}

template <typename Real>
lbm_status run_steps(lbm_ctx* c, int n, int eta) {
  for (int j = 1; j <= n; ++j) {
    TRY(time_begin(c, 0));
    TRY(launch_step_impl<Real>(c, step_args<Real>(c, (double)j / (double)eta), j == n));
    TRY(time_end(c, 0));
    c->cur ^= 1;
    if (c->p.dissolution) TRY(launch_dissolve<Real>(c));
    c->steps += 1;
  }
  return LBM_OK;
}

// Longest call whose launches are recorded into a graph (two kernel nodes a
// step); longer calls launch directly.
constexpr int kGraphMaxSteps = 8192;

struct StepsCall {
  int n, eta;
};
template <typename Real>
lbm_status enqueue_steps_call(lbm_ctx* c, void* arg) {
  const StepsCall* s = (const StepsCall*)arg;
  return run_steps<Real>(c, s->n, s->eta);
}

template <typename Real>
lbm_status run_init(lbm_ctx* c, const double* u0dev) {
  auto a = step_args<Real>(c, 0.0);
  a.fout = (Real*)c->f[0];
  lbm::lbm_init_kernel<Real><<<c->grid, c->block, 0, c->stream>>>(a, u0dev);
  CK(cudaGetLastError());
  c->nparts = (int)(c->grid.x * c->grid.y);
  c->cur = 0;
  if (!c->p.dissolution) return LBM_OK;
  // a slab's first pass gathers shares across its cuts: it waits for the halo
  if (c->p.edge[2] == LBM_EDGE_EXCHANGE || c->p.edge[3] == LBM_EDGE_EXCHANGE) {
    c->first_pass_due = true;
    return LBM_OK;
  }
  return first_dissolve<Real>(c);
}

// Copy a caller array of `count` doubles (host or device) to a device buffer.
lbm_status stage_doubles(lbm_ctx* c, const double* src, size_t count, double** out,
                         bool* owned) {
  *owned = false;
  *out = nullptr;
  if (!src) return LBM_OK;
  if (on_device(src)) {
    *out = const_cast<double*>(src);
    return LBM_OK;
  }
  CK(cudaMalloc((void**)out, count * sizeof(double)));
  *owned = true;
  CK(cudaMemcpyAsync(*out, src, count * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  return LBM_OK;
}

void free_ctx(lbm_ctx* c) {
  if (!c) return;
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
  c->graphs.clear();
  if (c->rec_stream) cudaStreamDestroy(c->rec_stream);
  for (int w = 0; w < 2; ++w)
    for (int i = 0; i < lbm_ctx::kPool; ++i)
      for (int k = 0; k < 2; ++k)
        if (c->ev[w][i][k]) cudaEventDestroy(c->ev[w][i][k]);
  void* ptrs[] = {c->f[0],   c->f[1],     c->link,      c->vel,        c->kf,
                  c->u,      c->ureact,   c->mineral,   c->edge,       c->infeasible,
                  c->jnode,  c->partial,  c->flip_list, c->flip_count, c->counters,
                  c->status, c->diag,     c->scratch,   c->slist,      c->smin,
                  c->jflux,  c->open_nodes, c->flip_step};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->pinned) cudaFreeHost(c->pinned);
  ctx_adjoint_free(c);
  delete c;
}

lbm_status ensure_scratch(lbm_ctx* c, size_t bytes) {
  if (c->scratch_bytes >= bytes) return LBM_OK;
  if (c->scratch) cudaFree(c->scratch);
  c->scratch = nullptr;
  c->scratch_bytes = 0;
  CK(cudaMalloc(&c->scratch, bytes));
  c->scratch_bytes = bytes;
  return LBM_OK;
}

lbm_status make_map(const char* what, CUtensorMap* m, CUtensorMapDataType dt, int rank,
                    void* base, const cuuint64_t* dims, const cuuint64_t* strides,
                    const cuuint32_t* box) {
  auto enc = encode_fn();
  if (!enc) return fail(LBM_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  const cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, dt, (cuuint32_t)rank, base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(LBM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the %s map (%d)", what, (int)r);
  return LBM_OK;
}

// The FP32 step kernel a context runs unless told otherwise: the tile
// pipeline below 8 M nodes or with maximum-entropy pore walls, the
// one-thread-per-node kernel (all inputs of a node in one round, six blocks
// per SM) for larger lattices with bounce-back walls.  Measured per step
// launch: 2048^2, 62 against 68 us; 4096^2, 238 against 226 us; 4096^2
// with maximum-entropy walls (FP32 solve), 214 against 279 us.
constexpr long long kPlainFromNodes = 8ll << 20;
bool tma_by_default(const lbm_ctx* c) {
  return (long long)c->p.nx * c->p.ny < kPlainFromNodes || c->wall_mode != LBM_WALL_BOUNCE;
}

// Tensor maps of the FP32 TMA step (see lbm_tma.cuh for the boxes).
lbm_status setup_tma(lbm_ctx* c) {
  const cuuint64_t P = (cuuint64_t)c->pitch, H = (cuuint64_t)lbm::padded_rows(c->p.ny);
  const cuuint64_t dpop[3] = {P, H, 9}, spop[2] = {P * 4, P * H * 4};
  const cuuint32_t bpop[3] = {lbm::kBoxW, lbm::kBoxH, 9};
  const cuuint64_t dvel[3] = {P, H, 2}, svel[2] = {P * 4, P * H * 4};
  const cuuint32_t bvel[3] = {lbm::kTW, lbm::kTH, 2};
  const cuuint64_t d2[2] = {P, H}, sf[1] = {P * 4};
  const cuuint32_t bk[2] = {lbm::kTW, lbm::kTH};
  for (int b = 0; b < 2; ++b) {
    lbm::TmaMaps& m = c->maps[b];
    TRY(make_map("population", &m.pop, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->f[b], dpop,
                 spop, bpop));
    TRY(make_map("velocity", &m.vel, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->vel, dvel, svel,
                 bvel));
    TRY(make_map("link", &m.link, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, c->link, d2, sf, bk));
    if (c->kf)
      TRY(make_map("rate", &m.kf, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->kf, d2, sf, bk));
    else m.kf = m.link;  // never read without a rate field
  }
  CK(cudaFuncSetAttribute(lbm::lbm_step_tma<true, 0>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, lbm::kTmaSmem));
  CK(cudaFuncSetAttribute(lbm::lbm_step_tma<false, 0>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, lbm::kTmaSmem));
  CK(cudaFuncSetAttribute(lbm::lbm_step_tma<true, 1>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, lbm::kTmaSmem));
  CK(cudaFuncSetAttribute(lbm::lbm_step_tma<false, 1>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, lbm::kTmaSmem));
  CK(cudaFuncSetAttribute(lbm::lbm_step_tma<true, 2>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, lbm::kTmaSmem));
  CK(cudaFuncSetAttribute(lbm::lbm_step_tma<false, 2>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, lbm::kTmaSmem));
  c->ntx = (c->p.nx + lbm::kTW - 1) / lbm::kTW;
  c->nty = (c->p.ny + lbm::kTH - 1) / lbm::kTH;
  const int ntiles = c->ntx * c->nty;
  c->tma_grid = ntiles < c->num_sms ? ntiles : c->num_sms;
  c->tma_ready = true;
  c->use_tma = tma_by_default(c);
  return LBM_OK;
}

lbm_status init_impl(lbm_ctx* c, const uint8_t* solid, const double* vel,
                     const double* k_field, const double* mineral, const double* u0) {
  const lbm_params& p = c->p;
  const size_t nxy = (size_t)p.nx * p.ny;
  c->pitch = lbm::padded_pitch(p.nx);
  c->plane = (long long)c->pitch * lbm::padded_rows(p.ny);
  c->esize = p.precision == 64 ? 8 : 4;
  c->nedge = 2 * (p.nx + p.ny);
  c->block = dim3(lbm::kBX, lbm::kBY);
  c->grid = dim3((p.nx + lbm::kBX - 1) / lbm::kBX, (p.ny + lbm::kBY - 1) / lbm::kBY);
  {
    const int rows = p.precision == 64 ? lbm::step_rows<double>() : lbm::step_rows<float>();
    c->sblock = dim3(lbm::kBX, rows);
    c->sgrid = dim3((p.nx + lbm::kBX - 1) / lbm::kBX, (p.ny + rows - 1) / rows);
  }
  const size_t plane_b = (size_t)c->plane * c->esize;
  const int per_x = p.edge[0] == LBM_EDGE_PERIODIC;
  CK(cudaGetDevice(&c->device));
  CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  {
    const long long blocks = ((long long)p.nx * p.ny + lbm::kDThreads - 1) / lbm::kDThreads;
    const long long cap = 8LL * c->num_sms;  // 8 resident blocks of 256 per SM
    c->dgrid = (int)(blocks < cap ? blocks : cap);
  }
  CK(cudaMalloc(&c->f[0], 9 * plane_b));
  CK(cudaMalloc(&c->f[1], 9 * plane_b));
  CK(cudaMemsetAsync(c->f[0], 0, 9 * plane_b, c->stream));
  CK(cudaMemsetAsync(c->f[1], 0, 9 * plane_b, c->stream));
  CK(cudaMalloc((void**)&c->link, (size_t)c->plane * sizeof(uint32_t)));
  CK(cudaMemsetAsync(c->link, 0, (size_t)c->plane * sizeof(uint32_t), c->stream));
  CK(cudaMalloc(&c->vel, 2 * plane_b));
  CK(cudaMemsetAsync(c->vel, 0, 2 * plane_b, c->stream));
  CK(cudaMalloc(&c->u, plane_b));
  CK(cudaMemsetAsync(c->u, 0, plane_b, c->stream));
  if (k_field) {
    CK(cudaMalloc(&c->kf, plane_b));
    CK(cudaMemsetAsync(c->kf, 0, plane_b, c->stream));
  }
  if (p.dissolution) {
    // reaction shares: 8 bytes a node on either lattice (double, or ShareF32)
    CK(cudaMalloc(&c->ureact, (size_t)c->plane * 8));
    CK(cudaMemsetAsync(c->ureact, 0, (size_t)c->plane * 8, c->stream));
    CK(cudaMalloc((void**)&c->mineral, (size_t)c->plane * sizeof(double)));
    CK(cudaMemsetAsync(c->mineral, 0, (size_t)c->plane * sizeof(double), c->stream));
    CK(cudaMalloc((void**)&c->flip_step, (size_t)c->plane * sizeof(int)));
    CK(cudaMemsetAsync(c->flip_step, 0xFF, (size_t)c->plane * sizeof(int), c->stream));
    CK(cudaMalloc((void**)&c->flip_list, nxy * sizeof(int)));
    CK(cudaMalloc((void**)&c->slist, nxy * sizeof(int)));
    CK(cudaMalloc((void**)&c->smin, nxy * sizeof(double)));
  }
  {
    // the nodes on Dirichlet / Neumann sides, each once (W, E, S, N order);
    // periodic sides and the sides a slab shares with a neighbour are not open
    std::vector<int> open;
    auto add = [&](int x, int y) { open.push_back((y + kYO) * c->pitch + (x + kXO)); };
    auto is_open = [&](int s) {
      return p.edge[s] == LBM_EDGE_DIRICHLET || p.edge[s] == LBM_EDGE_NEUMANN;
    };
    if (is_open(0))
      for (int y = 0; y < p.ny; ++y) add(0, y);
    if (is_open(1))
      for (int y = 0; y < p.ny; ++y) add(p.nx - 1, y);
    const int xa = is_open(0) ? 1 : 0, xb = is_open(1) ? p.nx - 1 : p.nx;
    for (int s : {2, 3})
      if (is_open(s))
        for (int x = xa; x < xb; ++x) add(x, s == 2 ? 0 : p.ny - 1);
    c->n_open = (int)open.size();
    if (!open.empty()) {
      CK(cudaMalloc((void**)&c->open_nodes, open.size() * sizeof(int)));
      CK(cudaMemcpy(c->open_nodes, open.data(), open.size() * sizeof(int),
                    cudaMemcpyHostToDevice));
    }
  }
  CK(cudaMalloc((void**)&c->flip_count, 4 * sizeof(int)));
  CK(cudaMemsetAsync(c->flip_count, 0, 4 * sizeof(int), c->stream));
  CK(cudaMalloc((void**)&c->counters, 4 * sizeof(long long)));
  CK(cudaMemsetAsync(c->counters, 0, 4 * sizeof(long long), c->stream));
  CK(cudaMalloc((void**)&c->status, sizeof(int)));
  CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
  CK(cudaMallocHost(&c->pinned, 256));
  CK(cudaMalloc((void**)&c->edge, 3 * (size_t)c->nedge * sizeof(double)));
  CK(cudaMemsetAsync(c->edge, 0, 3 * (size_t)c->nedge * sizeof(double), c->stream));
  CK(cudaMalloc((void**)&c->infeasible, (size_t)c->nedge * sizeof(long long)));
  CK(cudaMemsetAsync(c->infeasible, 0, (size_t)c->nedge * sizeof(long long), c->stream));
  CK(cudaMalloc((void**)&c->jnode, (size_t)p.ny * sizeof(double)));
  CK(cudaMemsetAsync(c->jnode, 0, (size_t)p.ny * sizeof(double), c->stream));
  CK(cudaMalloc((void**)&c->jflux, (size_t)p.ny * sizeof(double)));
  CK(cudaMemsetAsync(c->jflux, 0, (size_t)p.ny * sizeof(double), c->stream));
  {
    // one partial per block of the generic kernel, and enough for a batch's
    // pipelined tiles plus its boundary-warp chunks of 32 nodes
    const long long generic = (long long)c->sgrid.x * c->sgrid.y;
    const long long tiles = (long long)((p.nx + lbm::kTW - 1) / lbm::kTW) *
                            ((p.ny + lbm::kTH - 1) / lbm::kTH) + (c->n_open + 31) / 32;
    c->partial_cap = (int)((generic > tiles ? generic : tiles) + 1);
  }
  CK(cudaMalloc((void**)&c->partial, (size_t)c->partial_cap * sizeof(double)));
  CK(cudaMemsetAsync(c->partial, 0, (size_t)c->partial_cap * sizeof(double), c->stream));
  CK(cudaMalloc((void**)&c->diag, sizeof(DiagDev)));

  // inputs: host arrays are staged through temporary device buffers
  double *dvel = nullptr, *dk = nullptr, *dmin = nullptr, *du0 = nullptr;
  bool ovel = false, ok = false, omin = false, ou0 = false;
  uint8_t* dsolid = nullptr;
  bool osolid = false;
  lbm_status st = LBM_OK;
  auto cleanup = [&]() {
    cudaStreamSynchronize(c->stream);
    if (ovel) cudaFree(dvel);
    if (ok) cudaFree(dk);
    if (omin) cudaFree(dmin);
    if (ou0) cudaFree(du0);
    if (osolid) cudaFree(dsolid);
  };
  if ((st = stage_doubles(c, vel, 2 * nxy, &dvel, &ovel)) != LBM_OK ||
      (st = stage_doubles(c, k_field, nxy, &dk, &ok)) != LBM_OK ||
      (st = stage_doubles(c, mineral, nxy, &dmin, &omin)) != LBM_OK ||
      (st = stage_doubles(c, u0, nxy, &du0, &ou0)) != LBM_OK) {
    cleanup();
    return st;
  }
  if (solid) {  // the whole lattice's mask (a slab reads its neighbours' rows too)
    const size_t mask_bytes = (size_t)p.nx * c->ny_global;
    if (on_device(solid)) {
      dsolid = const_cast<uint8_t*>(solid);
    } else {
      cudaError_t e = cudaMalloc((void**)&dsolid, mask_bytes);
      if (e != cudaSuccess) {
        cleanup();
        return fail(LBM_ERR_NOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
      }
      osolid = true;
      cudaMemcpyAsync(dsolid, solid, mask_bytes, cudaMemcpyHostToDevice, c->stream);
    }
  }
  const int g = grid1d((long long)nxy * 2);
  {
    const int gs = p.edge[2] == LBM_EDGE_EXCHANGE, gn = p.edge[3] == LBM_EDGE_EXCHANGE;
    k_link_in<<<grid1d((long long)p.nx * (p.ny + 2)), 256, 0, c->stream>>>(
        dsolid, c->link, p.nx, p.ny, c->y0, c->ny_global, c->pitch, per_x, c->per_y_global,
        gs, gn);
  }
  if (c->esize == 8) {
    k_pitch_in<double><<<g, 256, 0, c->stream>>>(dvel, (double*)c->vel, p.nx, p.ny, c->pitch, 2, 0.0);
    if (dk) k_pitch_in<double><<<g, 256, 0, c->stream>>>(dk, (double*)c->kf, p.nx, p.ny, c->pitch, 1, 0.0);
  } else {
    k_pitch_in<float><<<g, 256, 0, c->stream>>>(dvel, (float*)c->vel, p.nx, p.ny, c->pitch, 2, 0.0);
    if (dk) k_pitch_in<float><<<g, 256, 0, c->stream>>>(dk, (float*)c->kf, p.nx, p.ny, c->pitch, 1, 0.0);
  }
  if (p.dissolution)
    k_pitch_in<double><<<g, 256, 0, c->stream>>>(dmin, c->mineral, p.nx, p.ny, c->pitch, 1, 1.0);
  k_count_solid<<<grid1d((long long)nxy), 256, 0, c->stream>>>(
      c->link, p.nx, p.ny, c->pitch, (unsigned long long*)(c->counters + 1));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cleanup();
    return fail(LBM_ERR_CUDA, "input conversion: %s", cudaGetErrorString(e));
  }
  st = c->esize == 8 ? run_init<double>(c, du0) : run_init<float>(c, du0);
  cleanup();
  if (st != LBM_OK) return st;
  CK(cudaGetLastError());
  if (c->esize == 4) TRY(setup_tma(c));
  return LBM_OK;
}

lbm_status check_ctx(const lbm_ctx* c) {
  if (!c) return fail(LBM_ERR_ARG, "null context");
  return LBM_OK;
}

// Reads the device status word (waits for the stream).
lbm_status check_status(lbm_ctx* c) {
  int* hs = (int*)c->pinned;
  CK(cudaMemcpyAsync(hs, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const int st = *hs;
  if (st >= lbm::kSiteBase)
    return fail(LBM_ERR_STATE, "index check %d failed (debug-bounds build)", st);
  if (st) return fail(LBM_ERR_TIMEOUT, "a kernel's bounded wait expired (status %d)", st);
  return LBM_OK;
}

// The status of a call that waited for the stream, after errors: a wall
// Newton solve that stopped short of its tolerance since the last report is
// LBM_ERR_NEWTON; boundary solves whose data had no non-negative solution
// since the last report are LBM_WARN_BC_INFEASIBLE.
lbm_status report(lbm_ctx* c, long long infeasible, long long newton_fail) {
  const long long new_inf = infeasible - c->warned_infeasible;
  const long long new_newton = newton_fail - c->warned_newton;
  c->warned_infeasible = infeasible;
  c->warned_newton = newton_fail;
  if (new_newton > 0)
    return fail(LBM_ERR_NEWTON, "%lld maximum-entropy wall solves stopped short of the Newton "
                "tolerance (the last iterate was used)", new_newton);
  if (new_inf > 0)
    return fail(LBM_WARN_BC_INFEASIBLE, "%lld boundary solves had data with no non-negative "
                "solution", new_inf);
  return LBM_OK;
}

// state blob layout (all sections 256-byte aligned)
struct Section {
  void* ptr;
  size_t bytes;
};
int state_sections(lbm_ctx* c, Section* s) {
  int k = 0;
  const size_t plane_b = (size_t)c->plane * c->esize;
  s[k++] = {c->f[c->cur], 9 * plane_b};
  s[k++] = {c->link, (size_t)c->plane * sizeof(uint32_t)};
  s[k++] = {c->u, plane_b};
  s[k++] = {c->infeasible, (size_t)c->nedge * sizeof(long long)};
  s[k++] = {c->jnode, (size_t)c->p.ny * sizeof(double)};
  s[k++] = {c->partial, (size_t)c->partial_cap * sizeof(double)};
  s[k++] = {c->jflux, (size_t)c->p.ny * sizeof(double)};
  s[k++] = {c->counters, 4 * sizeof(long long)};
  if (c->p.dissolution) {
    const size_t nxy = (size_t)c->p.nx * c->p.ny;
    s[k++] = {c->mineral, (size_t)c->plane * sizeof(double)};
    s[k++] = {c->flip_count, 4 * sizeof(int)};
    s[k++] = {c->slist, nxy * sizeof(int)};
    s[k++] = {c->smin, nxy * sizeof(double)};
    s[k++] = {c->flip_step, (size_t)c->plane * sizeof(int)};
  }
  return k;
}
size_t align256(size_t b) { return (b + 255) / 256 * 256; }
struct BlobHeader {
  unsigned long long magic;
  long long steps;
  int nx, ny, precision, dissolution, nparts, pad;
};
const unsigned long long kMagic = 0x4C424D4144453035ull;  // "LBMADE05"
static_assert(sizeof(BlobHeader) <= 64, "the header fits its pinned read-back slot");

// Write a blob header into device memory byte by byte (any alignment).
__global__ void k_put_blob_header(unsigned char* dst, const BlobHeader h) {
  const unsigned char* src = reinterpret_cast<const unsigned char*>(&h);
  for (int i = threadIdx.x; i < (int)sizeof(BlobHeader); i += blockDim.x) dst[i] = src[i];
}

// Copy a padded device field out to a caller array (host or device) of
// `planes` [ny][nx] planes, converting to O.
template <typename T, typename O>
lbm_status field_out(lbm_ctx* c, const T* src, O* dst, int planes) {
  const size_t bytes = (size_t)planes * c->p.nx * c->p.ny * sizeof(O);
  const bool dev = on_device(dst);
  O* d = dst;
  if (!dev) {
    TRY(ensure_scratch(c, bytes));
    d = (O*)c->scratch;
  }
  k_pitch_out<T, O><<<grid1d((long long)planes * c->p.nx * c->p.ny), 256, 0, c->stream>>>(
      src, d, c->p.nx, c->p.ny, c->pitch, planes);
  CK(cudaGetLastError());
  if (!dev) {
    CK(cudaMemcpyAsync(dst, d, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}

}  // namespace

// ---- services for the other translation units (lbm_ctx.h) ----------------

lbm_status ctx_fail(lbm_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

lbm_status ctx_check(const lbm_ctx* c) { return check_ctx(c); }
lbm_status ctx_status(lbm_ctx* c) { return check_status(c); }
bool ctx_on_device(const void* p) { return on_device(p); }

lbm_status ctx_stage_edges(lbm_ctx* c, const double* ua, const double* ub, const double* q) {
  const size_t eb = (size_t)c->nedge * sizeof(double);
  double* e = c->edge;
  if (ua) CK(cudaMemcpyAsync(e, ua, eb, kind_from(ua), c->stream));
  else CK(cudaMemsetAsync(e, 0, eb, c->stream));
  const double* b = ub ? ub : ua;
  if (b) CK(cudaMemcpyAsync(e + c->nedge, b, eb, kind_from(b), c->stream));
  else CK(cudaMemsetAsync(e + c->nedge, 0, eb, c->stream));
  if (q) CK(cudaMemcpyAsync(e + 2 * c->nedge, q, eb, kind_from(q), c->stream));
  else CK(cudaMemsetAsync(e + 2 * c->nedge, 0, eb, c->stream));
  // host-sourced edge data must not be reused before the copies complete
  if ((ua && !on_device(ua)) || (b && !on_device(b)) || (q && !on_device(q)))
    CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status ctx_run_recorded(lbm_ctx* c, const lbm_ctx::GraphKey& key,
                            lbm_status (*enqueue)(lbm_ctx*, void*), void* arg) {
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    if (c->seen.insert(key).second) return enqueue(c, arg);  // first sighting: run directly
    if (!c->rec_stream) CK(cudaStreamCreateWithFlags(&c->rec_stream, cudaStreamNonBlocking));
    // record: the launches go to the recording stream, the host bookkeeping
    // they do is kept and applied again on every replay
    const int cur0 = c->cur;
    const long long steps0 = c->steps;
    cudaStream_t user = c->stream;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->rec_stream, cudaStreamCaptureModeThreadLocal));
    c->stream = c->rec_stream;
    const lbm_status st = enqueue(c, arg);
    c->stream = user;
    const cudaError_t ce = cudaStreamEndCapture(c->rec_stream, &g);
    if (st != LBM_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      c->cur = cur0;
      c->steps = steps0;
      cudaGetLastError();
      return st != LBM_OK ? st : fail(LBM_ERR_CUDA, "graph recording: %s", cudaGetErrorString(ce));
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    c->cur = cur0;
    c->steps = steps0;
    if (ie != cudaSuccess) return fail(LBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ie));
    it = c->graphs.emplace(key, lbm_ctx::Recorded{ex, c->nparts}).first;
  }
  CK(cudaGraphLaunch(it->second.exec, c->stream));
  // the bookkeeping of the recorded sequence: n steps (key element 1)
  const int n = std::get<1>(key);
  c->cur ^= (n & 1);
  c->steps += n;
  c->nparts = it->second.nparts;
  return LBM_OK;
}

void ctx_drop_recorded(lbm_ctx* c, int kind) {
  for (auto it = c->graphs.begin(); it != c->graphs.end();) {
    if (std::get<0>(it->first) == kind) {
      cudaGraphExecDestroy(it->second.exec);
      it = c->graphs.erase(it);
    } else {
      ++it;
    }
  }
  for (auto it = c->seen.begin(); it != c->seen.end();)
    it = std::get<0>(*it) == kind ? c->seen.erase(it) : std::next(it);
}

lbm_status ctx_make_map(const char* what, CUtensorMap* m, CUtensorMapDataType dt, int rank,
                        void* base, const cuuint64_t* dims, const cuuint64_t* strides,
                        const cuuint32_t* box) {
  return make_map(what, m, dt, rank, base, dims, strides, box);
}

template <typename Real>
lbm_status ctx_launch_step(lbm_ctx* c, const lbm::StepArgs<Real>& a, bool final_step) {
  return launch_step_impl<Real>(c, a, final_step);
}
template lbm_status ctx_launch_step<float>(lbm_ctx*, const lbm::StepArgs<float>&, bool);
template lbm_status ctx_launch_step<double>(lbm_ctx*, const lbm::StepArgs<double>&, bool);

lbm_status ctx_field_out_f64(lbm_ctx* c, const double* padded, double* out) {
  return field_out<double, double>(c, padded, out, 1);
}

extern "C" {

int lbm_abi_version(void) { return LBM_ADE_ABI_VERSION; }

const char* lbm_last_error(void) { return g_err; }

}  // extern "C"

namespace {

lbm_status check_params(const lbm_params* p) {
  if (p->nx < 2 || p->ny < 2) return fail(LBM_ERR_ARG, "lbm_init: nx, ny must be >= 2");
  // launches over the lattice give each row (the adjoint step) or pair of
  // rows a block index in y, at most 65535
  if (p->ny > 65535) return fail(LBM_ERR_ARG, "lbm_init: ny must be <= 65535");
  if ((long long)lbm::padded_pitch(p->nx) * lbm::padded_rows(p->ny) > INT_MAX)
    return fail(LBM_ERR_ARG, "lbm_init: lattice too large (padded plane > INT_MAX)");
  if (p->precision != 32 && p->precision != 64)
    return fail(LBM_ERR_ARG, "lbm_init: precision must be 32 or 64");
  if (!(p->tau > 0.5) || !std::isfinite(p->tau))
    return fail(LBM_ERR_ARG, "lbm_init: tau must be finite and > 1/2");
  for (int s = 0; s < 4; ++s)
    if (p->edge[s] < 0 || p->edge[s] > 2) return fail(LBM_ERR_ARG, "lbm_init: bad edge kind");
  if ((p->edge[0] == LBM_EDGE_PERIODIC) != (p->edge[1] == LBM_EDGE_PERIODIC) ||
      (p->edge[2] == LBM_EDGE_PERIODIC) != (p->edge[3] == LBM_EDGE_PERIODIC))
    return fail(LBM_ERR_ARG, "lbm_init: opposite sides must both be periodic or both not");
  if (p->react_mode < 0 || p->react_mode > 2) return fail(LBM_ERR_ARG, "lbm_init: bad react_mode");
  if (!std::isfinite(p->k_scalar)) return fail(LBM_ERR_ARG, "lbm_init: k_scalar not finite");
  if (p->dissolution && p->react_mode != LBM_REACT_SURFACE)
    return fail(LBM_ERR_ARG, "lbm_init: dissolution needs react_mode = LBM_REACT_SURFACE");
  return LBM_OK;
}

// Rows y0 .. y1 - 1 of `planes` [ny][nx] planes of a caller array (host or
// device) into a new device buffer; *out stays null for a null array.
lbm_status gather_rows(const double* src, int planes, int nx, int ny, int y0, int y1,
                       double** out, cudaStream_t st) {
  *out = nullptr;
  if (!src) return LBM_OK;
  const size_t rows = (size_t)(y1 - y0) * nx;
  CK(cudaMalloc((void**)out, planes * rows * sizeof(double)));
  for (int k = 0; k < planes; ++k)
    CK(cudaMemcpyAsync(*out + k * rows, src + (size_t)k * ny * nx + (size_t)y0 * nx,
                       rows * sizeof(double), cudaMemcpyDefault, st));
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_init(lbm_ctx** out, const lbm_params* p, const uint8_t* solid,
                    const double* vel, const double* k_field, const double* mineral,
                    const double* u0, void* stream) {
  g_err[0] = 0;
  if (!out || !p) return fail(LBM_ERR_ARG, "lbm_init: null out or params");
  *out = nullptr;
  TRY(check_params(p));
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return fail(LBM_ERR_NOMEM, "lbm_init: host allocation failed");
  c->p = *p;
  c->ny_global = p->ny;
  c->per_y_global = p->edge[2] == LBM_EDGE_PERIODIC;
  c->stream = (cudaStream_t)stream;
  lbm_status st = init_impl(c, solid, vel, k_field, mineral, u0);
  if (st != LBM_OK) {
    free_ctx(c);
    return st;
  }
  *out = c;
  return LBM_OK;
}

lbm_status lbm_init_slab(lbm_ctx** out, const lbm_params* p, int y0, int y1,
                         const uint8_t* solid, const double* vel, const double* k_field,
                         const double* mineral, const double* u0, void* stream) {
  g_err[0] = 0;
  if (!out || !p) return fail(LBM_ERR_ARG, "lbm_init_slab: null out or params");
  *out = nullptr;
  TRY(check_params(p));
  if (y0 < 0 || y1 > p->ny || y1 - y0 < 2)
    return fail(LBM_ERR_ARG, "lbm_init_slab: need 0 <= y0, y1 <= ny, at least 2 rows");
  const bool per_yg = p->edge[2] == LBM_EDGE_PERIODIC;
  lbm_params q = *p;
  q.ny = y1 - y0;
  if (!(per_yg && y0 == 0 && y1 == p->ny)) {  // one slab of a periodic lattice stays periodic
    q.edge[2] = (y0 == 0 && !per_yg) ? p->edge[2] : LBM_EDGE_EXCHANGE;
    q.edge[3] = (y1 == p->ny && !per_yg) ? p->edge[3] : LBM_EDGE_EXCHANGE;
  }
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return fail(LBM_ERR_NOMEM, "lbm_init_slab: host allocation failed");
  c->p = q;
  c->y0 = y0;
  c->ny_global = p->ny;
  c->per_y_global = per_yg;
  c->stream = (cudaStream_t)stream;
  double *dv = nullptr, *dk = nullptr, *dm = nullptr, *du = nullptr;
  lbm_status st = gather_rows(vel, 2, p->nx, p->ny, y0, y1, &dv, c->stream);
  if (st == LBM_OK) st = gather_rows(k_field, 1, p->nx, p->ny, y0, y1, &dk, c->stream);
  if (st == LBM_OK) st = gather_rows(mineral, 1, p->nx, p->ny, y0, y1, &dm, c->stream);
  if (st == LBM_OK) st = gather_rows(u0, 1, p->nx, p->ny, y0, y1, &du, c->stream);
  if (st == LBM_OK) st = init_impl(c, solid, dv, dk, dm, du);
  cudaStreamSynchronize(c->stream);
  for (double* t : {dv, dk, dm, du})
    if (t) cudaFree(t);
  if (st != LBM_OK) {
    free_ctx(c);
    return st;
  }
  *out = c;
  return LBM_OK;
}

lbm_status lbm_stage_edges(lbm_ctx* c, const double* u_dir_t0, const double* u_dir_t1,
                           const double* q_neu) {
  TRY(check_ctx(c));
  return ctx_stage_edges(c, u_dir_t0, u_dir_t1, q_neu);
}

lbm_status lbm_step_stream(lbm_ctx* c, int j, int eta, int final_step) {
  TRY(check_ctx(c));
  if (j < 1 || eta < 1) return fail(LBM_ERR_ARG, "lbm_step_stream: need j >= 1, eta >= 1");
  if (c->first_pass_due)
    return fail(LBM_ERR_STATE,
                "lbm_step_stream: the slab's first dissolution pass is due (exchange the "
                "halo, then call lbm_step_dissolve)");
  const double frac = (double)j / (double)eta;
  TRY(time_begin(c, 0));
  if (c->esize == 8) TRY(launch_step_impl<double>(c, step_args<double>(c, frac), final_step != 0));
  else TRY(launch_step_impl<float>(c, step_args<float>(c, frac), final_step != 0));
  TRY(time_end(c, 0));
  c->cur ^= 1;
  c->steps += 1;
  return LBM_OK;
}

lbm_status lbm_step_dissolve(lbm_ctx* c) {
  TRY(check_ctx(c));
  if (!c->p.dissolution) return LBM_OK;
  if (c->first_pass_due) {
    TRY(c->esize == 8 ? first_dissolve<double>(c) : first_dissolve<float>(c));
    c->first_pass_due = false;
    return LBM_OK;
  }
  return c->esize == 8 ? launch_dissolve<double>(c) : launch_dissolve<float>(c);
}

lbm_status lbm_substeps(lbm_ctx* c, int n, int eta, const double* u_dir_t0,
                        const double* u_dir_t1, const double* q_neu) {
  TRY(check_ctx(c));
  if (n < 0 || eta < 1) return fail(LBM_ERR_ARG, "lbm_substeps: need n >= 0, eta >= 1");
  if (c->p.edge[2] == LBM_EDGE_EXCHANGE || c->p.edge[3] == LBM_EDGE_EXCHANGE)
    return fail(LBM_ERR_STATE,
                "lbm_substeps: a slab steps through lbm_step_stream / lbm_step_dissolve with "
                "its halo exchange between them");
  if (n == 0) return LBM_OK;
  TRY(ctx_stage_edges(c, u_dir_t0, u_dir_t1, q_neu));
  if (c->timing || n > kGraphMaxSteps)  // timing records events around every launch
    return c->esize == 8 ? run_steps<double>(c, n, eta) : run_steps<float>(c, n, eta);
  StepsCall call{n, eta};
  const lbm_ctx::GraphKey key{0, n, eta, 0, c->cur, walls_variant(c), c->use_tma ? 1 : 0};
  return ctx_run_recorded(c, key,
                          c->esize == 8 ? enqueue_steps_call<double> : enqueue_steps_call<float>,
                          &call);
}

lbm_status lbm_set_rate_field(lbm_ctx* c, const double* k_field) {
  TRY(check_ctx(c));
  if (!k_field) return fail(LBM_ERR_ARG, "lbm_set_rate_field: null field");
  if (!c->kf)
    return fail(LBM_ERR_STATE,
                "lbm_set_rate_field: the context was created without a rate field");
  const size_t nxy = (size_t)c->p.nx * c->p.ny;
  double* dk = nullptr;
  bool owned = false;
  TRY(stage_doubles(c, k_field, nxy, &dk, &owned));
  const int g = grid1d((long long)nxy);
  if (c->esize == 8)
    k_pitch_in<double><<<g, 256, 0, c->stream>>>(dk, (double*)c->kf, c->p.nx, c->p.ny, c->pitch, 1, 0.0);
  else
    k_pitch_in<float><<<g, 256, 0, c->stream>>>(dk, (float*)c->kf, c->p.nx, c->p.ny, c->pitch, 1, 0.0);
  const cudaError_t e = cudaGetLastError();
  if (owned) {
    cudaStreamSynchronize(c->stream);
    cudaFree(dk);
  }
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "lbm_set_rate_field: %s", cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_interface_trace(lbm_ctx* c, int npts, const double* xy, double* u_out) {
  TRY(check_ctx(c));
  if (npts < 0 || (npts > 0 && (!xy || !u_out)))
    return fail(LBM_ERR_ARG, "lbm_interface_trace: bad arguments");
  if (npts == 0) return LBM_OK;
  const bool xy_dev = on_device(xy), out_dev = on_device(u_out);
  const double* dxy = xy;
  double* dout = u_out;
  const size_t in_b = 2 * (size_t)npts * sizeof(double), out_b = (size_t)npts * sizeof(double);
  if (!xy_dev || !out_dev) TRY(ensure_scratch(c, align256(in_b) + out_b));
  if (!xy_dev) {
    CK(cudaMemcpyAsync(c->scratch, xy, in_b, cudaMemcpyHostToDevice, c->stream));
    dxy = (const double*)c->scratch;
  }
  if (!out_dev) dout = (double*)((char*)c->scratch + align256(in_b));
  const int per_x = c->p.edge[0] == LBM_EDGE_PERIODIC, per_y = c->p.edge[2] == LBM_EDGE_PERIODIC;
  const int g = (npts + 255) / 256;
  if (c->esize == 8)
    k_trace<double><<<g, 256, 0, c->stream>>>((const double*)c->u, c->p.nx, c->p.ny, c->pitch,
                                              per_x, per_y, dxy, npts, dout);
  else
    k_trace<float><<<g, 256, 0, c->stream>>>((const float*)c->u, c->p.nx, c->p.ny, c->pitch,
                                             per_x, per_y, dxy, npts, dout);
  CK(cudaGetLastError());
  if (!out_dev) {
    CK(cudaMemcpyAsync(u_out, dout, out_b, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  } else if (!xy_dev) {
    CK(cudaStreamSynchronize(c->stream));
  } else {
    return LBM_OK;  // device in and out: asynchronous on the stream
  }
  return check_status(c);
}

lbm_status lbm_get_concentration(lbm_ctx* c, void* out, int out_precision) {
  TRY(check_ctx(c));
  if (!out || (out_precision != 32 && out_precision != 64))
    return fail(LBM_ERR_ARG, "lbm_get_concentration: bad arguments");
  if (c->esize == 8)
    TRY(out_precision == 64
            ? field_out<double, double>(c, (const double*)c->u, (double*)out, 1)
            : field_out<double, float>(c, (const double*)c->u, (float*)out, 1));
  else
    TRY(out_precision == 64 ? field_out<float, double>(c, (const float*)c->u, (double*)out, 1)
                            : field_out<float, float>(c, (const float*)c->u, (float*)out, 1));
  return check_status(c);
}

lbm_status lbm_get_populations(lbm_ctx* c, double* out) {
  TRY(check_ctx(c));
  if (!out) return fail(LBM_ERR_ARG, "lbm_get_populations: null out");
  if (c->esize == 8) TRY(field_out<double, double>(c, (const double*)c->f[c->cur], out, 9));
  else TRY(field_out<float, double>(c, (const float*)c->f[c->cur], out, 9));
  return check_status(c);
}

lbm_status lbm_get_solid(lbm_ctx* c, uint8_t* out) {
  TRY(check_ctx(c));
  if (!out) return fail(LBM_ERR_ARG, "lbm_get_solid: null out");
  const size_t bytes = (size_t)c->p.nx * c->p.ny;
  const bool dev = on_device(out);
  uint8_t* d = out;
  if (!dev) {
    TRY(ensure_scratch(c, bytes));
    d = (uint8_t*)c->scratch;
  }
  k_solid_out<<<grid1d((long long)bytes), 256, 0, c->stream>>>(c->link, d, c->p.nx, c->p.ny,
                                                               c->pitch);
  CK(cudaGetLastError());
  if (!dev) {
    CK(cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return check_status(c);
}

lbm_status lbm_get_mineral(lbm_ctx* c, double* out) {
  TRY(check_ctx(c));
  if (!out) return fail(LBM_ERR_ARG, "lbm_get_mineral: null out");
  if (!c->p.dissolution) return fail(LBM_ERR_STATE, "lbm_get_mineral: dissolution is off");
  TRY(sync_mineral(c));
  TRY(field_out<double, double>(c, c->mineral, out, 1));
  return check_status(c);
}

lbm_status lbm_diagnostics(lbm_ctx* c, lbm_diag* out) {
  TRY(check_ctx(c));
  if (!out) return fail(LBM_ERR_ARG, "lbm_diagnostics: null out");
  k_diag<<<1, 256, 0, c->stream>>>(c->partial, c->nparts, c->jnode, c->jflux, c->p.ny,
                                   c->infeasible, c->nedge, c->diag);
  CK(cudaGetLastError());
  DiagDev h;
  long long ctr[4];
  CK(cudaMemcpyAsync(&h, c->diag, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(ctr, c->counters, sizeof(ctr), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  TRY(check_status(c));
  double min_f = 0.0;
  TRY(lbm_min_population(c, &min_f));
  out->mass = h.mass;
  out->outlet_J = h.J;
  out->outlet_flux = h.flux;
  out->min_f = min_f;
  out->steps = c->steps;
  out->bc_infeasible = h.infeasible + ctr[2];
  out->newton_fail = ctr[3];
  out->flips = ctr[0];
  out->n_solid = ctr[1] - ctr[0];
  return report(c, out->bc_infeasible, out->newton_fail);
}

lbm_status lbm_set_wall_mode(lbm_ctx* c, int mode) {
  TRY(check_ctx(c));
  if (mode != LBM_WALL_BOUNCE && mode != LBM_WALL_MAXENT && mode != LBM_WALL_MAXENT_LATTICE)
    return fail(LBM_ERR_ARG,
                "lbm_set_wall_mode: mode must be LBM_WALL_BOUNCE, LBM_WALL_MAXENT or "
                "LBM_WALL_MAXENT_LATTICE");
  c->wall_mode = mode;
  if (c->kernel_auto) c->use_tma = c->tma_ready && tma_by_default(c);
  return LBM_OK;
}

lbm_status lbm_get_flip_steps(lbm_ctx* c, int32_t* out) {
  TRY(check_ctx(c));
  if (!out) return fail(LBM_ERR_ARG, "lbm_get_flip_steps: null out");
  if (!c->p.dissolution) return fail(LBM_ERR_STATE, "lbm_get_flip_steps: dissolution is off");
  TRY(field_out<int, int32_t>(c, c->flip_step, out, 1));
  return check_status(c);
}

lbm_status lbm_state_bytes(lbm_ctx* c, size_t* bytes) {
  TRY(check_ctx(c));
  if (!bytes) return fail(LBM_ERR_ARG, "lbm_state_bytes: null out");
  Section s[16];
  const int k = state_sections(c, s);
  size_t total = align256(sizeof(BlobHeader));
  for (int i = 0; i < k; ++i) total += align256(s[i].bytes);
  *bytes = total;
  return LBM_OK;
}

lbm_status lbm_save(lbm_ctx* c, void* buf, size_t bytes) {
  size_t need = 0;
  TRY(lbm_state_bytes(c, &need));
  if (!buf || bytes < need) return fail(LBM_ERR_ARG, "lbm_save: buffer smaller than lbm_state_bytes");
  const bool dev = on_device(buf);
  const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  TRY(sync_mineral(c));
  BlobHeader h{kMagic, c->steps, c->p.nx, c->p.ny, c->p.precision, c->p.dissolution, c->nparts, 0};
  if (dev) {
    // the header travels as a kernel argument: nothing on this stack frame
    // is read after the call returns, so a save into device memory need
    // not wait
    k_put_blob_header<<<1, 32, 0, c->stream>>>((unsigned char*)buf, h);
    CK(cudaGetLastError());
  } else {
    memcpy(buf, &h, sizeof(h));
  }
  Section s[16];
  const int n = state_sections(c, s);
  size_t off = align256(sizeof(BlobHeader));
  for (int i = 0; i < n; ++i) {
    CK(cudaMemcpyAsync((char*)buf + off, s[i].ptr, s[i].bytes, k, c->stream));
    off += align256(s[i].bytes);
  }
  if (dev) return LBM_OK;
  return check_status(c);  // waits: the host blob is complete on return
}

lbm_status lbm_restore(lbm_ctx* c, const void* buf, size_t bytes) {
  size_t need = 0;
  TRY(lbm_state_bytes(c, &need));
  if (!buf || bytes < need) return fail(LBM_ERR_ARG, "lbm_restore: buffer smaller than lbm_state_bytes");
  const bool dev = on_device(buf);
  BlobHeader h;
  if (dev) {
    BlobHeader* hh = (BlobHeader*)((char*)c->pinned + 64);
    CK(cudaMemcpyAsync(hh, buf, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    h = *hh;
  } else {
    CK(cudaStreamSynchronize(c->stream));  // the sections below overwrite the state
    memcpy(&h, buf, sizeof(h));
  }
  if (h.magic != kMagic || h.nx != c->p.nx || h.ny != c->p.ny ||
      h.precision != c->p.precision || h.dissolution != c->p.dissolution)
    return fail(LBM_ERR_STATE, "lbm_restore: blob does not belong to this lattice");
  const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  Section s[16];
  const int n = state_sections(c, s);
  size_t off = align256(sizeof(BlobHeader));
  for (int i = 0; i < n; ++i) {
    CK(cudaMemcpyAsync(s[i].ptr, (const char*)buf + off, s[i].bytes, k, c->stream));
    off += align256(s[i].bytes);
  }
  c->steps = h.steps;
  c->nparts = h.nparts;
  if (!dev) CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_kernel_timing(lbm_ctx* c, int enable) {
  TRY(check_ctx(c));
  for (int w = 0; w < 2; ++w) {
    TRY(fold_times(c, w));
    c->ms_sum[w] = 0.0;
    c->launches[w] = 0;
  }
  c->timing = enable != 0;
  return LBM_OK;
}

lbm_status lbm_kernel_times_read(lbm_ctx* c, double* step_ms, long long* step_launches,
                                 double* dissolve_ms, long long* dissolve_launches) {
  TRY(check_ctx(c));
  for (int w = 0; w < 2; ++w) TRY(fold_times(c, w));
  if (step_ms) *step_ms = c->ms_sum[0];
  if (step_launches) *step_launches = c->launches[0];
  if (dissolve_ms) *dissolve_ms = c->ms_sum[1];
  if (dissolve_launches) *dissolve_launches = c->launches[1];
  return LBM_OK;
}

lbm_status lbm_set_kernel(lbm_ctx* c, int variant) {
  TRY(check_ctx(c));
  switch (variant) {
    case LBM_KERNEL_AUTO:
      c->kernel_auto = true;
      c->use_tma = c->tma_ready && tma_by_default(c);
      return LBM_OK;
    case LBM_KERNEL_GENERIC:
      c->kernel_auto = false;
      c->use_tma = false;
      return LBM_OK;
    case LBM_KERNEL_TMA:
      if (!c->tma_ready) return fail(LBM_ERR_ARG, "lbm_set_kernel: the tile pipeline is FP32 only");
      c->kernel_auto = false;
      c->use_tma = true;
      return LBM_OK;
    default:
      return fail(LBM_ERR_ARG, "lbm_set_kernel: unknown variant %d", variant);
  }
}

lbm_status lbm_get_kernel(lbm_ctx* c, int* variant) {
  TRY(check_ctx(c));
  if (!variant) return fail(LBM_ERR_ARG, "lbm_get_kernel: null output");
  *variant = (c->esize == 4 && c->use_tma) ? LBM_KERNEL_TMA : LBM_KERNEL_GENERIC;
  return LBM_OK;
}

lbm_status lbm_set_stream(lbm_ctx* c, void* stream) {
  TRY(check_ctx(c));
  CK(cudaStreamSynchronize(c->stream));
  c->stream = (cudaStream_t)stream;
  return LBM_OK;
}

lbm_status lbm_synchronize(lbm_ctx* c) {
  TRY(check_ctx(c));
  TRY(check_status(c));
  long long ctr[4], inf = 0;
  CK(cudaMemcpyAsync(ctr, c->counters, sizeof(ctr), cudaMemcpyDeviceToHost, c->stream));
  std::vector<long long> per(c->nedge);
  CK(cudaMemcpyAsync(per.data(), c->infeasible, per.size() * sizeof(long long),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (long long v : per) inf += v;
  return report(c, inf + ctr[2], ctr[3]);
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

}  // extern "C"
