// lbm_pair.cu -- two lattices of one geometry stepped by one kernel
// (lbm_pair_*, declared in include/lbm_ade.h).
//
// The reaction invariants of Sec. 7.2 (alpha, beta) and Sec. 7.4 (psi1,
// psi2) are two concentrations carried by the same flow through the same
// pores: the same velocity and the same solid links.  The pair kernel is the
// tile pipeline of lbm_tma.cuh over both fields at once: for each 96 x 4 tile
// the producer brings both fields' population boxes (with their one-node
// halo) but the velocity and link-word boxes once; 12 consumer warps update
// each field's 384 nodes; the boundary warp steps both fields' nodes on the
// Dirichlet/Neumann sides (FP64 solves).  Four rows instead of eight keep
// four pipeline stages of both fields in shared memory.  Each field computes
// exactly what stepping its lattice alone computes.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <new>

#include "lbm_ade.h"
#include "lbm_ctx.h"
#include "lbm_tma.cuh"

namespace {

using namespace lbm;

constexpr int kPH = 4;                      // tile rows
constexpr int kPBoxH = kPH + 2;             // population box rows
constexpr int kPWarpsPerField = kTmaThreads / 32 / 2;  // 12: 4 rows x 3 thirds
static_assert(kPWarpsPerField == kPH * kWarpsPerRow, "pair tile mapping");
constexpr int kPPopBytes = 9 * kPBoxH * kBoxW * 4;
constexpr int kPVelBytes = 2 * kPH * kTW * 4;
constexpr int kPNodeBytes = kPH * kTW * 4;
constexpr int kPOffB = round128(kPPopBytes);                 // field B's populations
constexpr int kPOffVel = kPOffB + round128(kPPopBytes);
constexpr int kPOffWord = kPOffVel + round128(kPVelBytes);
constexpr int kPOffKA = kPOffWord + round128(kPNodeBytes);   // rate fields (optional)
constexpr int kPOffKB = kPOffKA + round128(kPNodeBytes);
constexpr int kPStage = kPOffKB + round128(kPNodeBytes);
constexpr int kPSmem = kStages * kPStage;
static_assert(kPSmem <= 227 * 1024, "pair stages exceed shared memory");

struct PairMaps {
  CUtensorMap pop[2];  // field A, field B: box {kBoxW, kPBoxH, 9} of the current buffer
  CUtensorMap vel;     // box {kTW, kPH, 2}
  CUtensorMap link;    // box {kTW, kPH}
  CUtensorMap kf[2];   // box {kTW, kPH} (valid where the field has a rate field)
};

template <bool kFinal>
__global__ void __launch_bounds__(kTmaBlock, 1)
    lbm_step_tma_pair(const StepArgs<float> a0, const StepArgs<float> a1,
                      const __grid_constant__ PairMaps maps, int ntx, int nty) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  __shared__ int2 origin[kStages];
  __shared__ double red[2][kTmaBlock / 32];
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int ntiles = ntx * nty;
  const uint32_t bytes = 2 * kPPopBytes + kPVelBytes + kPNodeBytes +
                         (a0.kf ? kPNodeBytes : 0) + (a1.kf ? kPNodeBytes : 0);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kTmaThreads / 32);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  double u0 = 0.0, u1 = 0.0;  // block's mass of each field
  if (warp == 0) {
    if (lane == 0) {
      int k = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = k % kStages;
        if (k >= kStages && !mbar_wait(&empty[s], (uint32_t)(((k / kStages) - 1) & 1))) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (*(volatile int*)&abort_flag) break;
        unsigned char* st = smem + s * kPStage;
        const int x0 = (t % ntx) * kTW, y0 = (t / ntx) * kPH;
        origin[s] = make_int2(x0, y0);
        mbar_expect_tx(&full[s], bytes);
        tma_load_3d(st, &maps.pop[0], x0 + kXO - 4, y0, 0, &full[s]);
        tma_load_3d(st + kPOffB, &maps.pop[1], x0 + kXO - 4, y0, 0, &full[s]);
        tma_load_3d(st + kPOffVel, &maps.vel, x0 + kXO, y0 + kYO, 0, &full[s]);
        tma_load_2d(st + kPOffWord, &maps.link, x0 + kXO, y0 + kYO, &full[s]);
        if (a0.kf) tma_load_2d(st + kPOffKA, &maps.kf[0], x0 + kXO, y0 + kYO, &full[s]);
        if (a1.kf) tma_load_2d(st + kPOffKB, &maps.kf[1], x0 + kXO, y0 + kYO, &full[s]);
      }
      if (*(volatile int*)&abort_flag) {
        for (int kk = (k >= kStages ? k - kStages : 0); kk < k; ++kk)
          (void)mbar_wait(&full[kk % kStages], (uint32_t)((kk / kStages) & 1));
      }
    }
  } else if (warp == kBoundaryWarp) {
    // both fields' nodes on the Dirichlet / Neumann sides
    const int nopen = a0.n_open;
    for (int e0 = blockIdx.x * 32; e0 < 2 * nopen; e0 += gridDim.x * 32) {
      const int e = e0 + lane;
      if (e < 2 * nopen) {
        const int f = e >= nopen;
        const StepArgs<float>& a = f ? a1 : a0;
        const int n = a.open_nodes[dbg_idx(e - f * nopen, nopen, a.status, kSiteNode)];
        const int y = n / a.pitch - kYO, x = n - (y + kYO) * a.pitch - kXO;
        GlobalSrc<float> src{a, n};
        const double v = step_node<float, kFinal, true, true, 0>(a, src, x, y, n, a.frac);
        if (f) u1 += v;
        else u0 += v;
      }
    }
  } else {
    const int cw = warp - 1;
    const int f = cw / kPWarpsPerField;            // the field this warp updates
    const int w = cw % kPWarpsPerField;
    const int r = w / kWarpsPerRow;                // tile row
    const int cbase = (w % kWarpsPerRow) * 32 + lane;
    const StepArgs<float>& a = f ? a1 : a0;
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
      const int s = k % kStages;
      if (!mbar_wait(&full[s], (uint32_t)((k / kStages) & 1))) {
        atomicExch(&abort_flag, 1);
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      const unsigned char* st = smem + s * kPStage;
      SmemSrcT<kPH> src{(const float*)(st + (f ? kPOffB : 0)), (const float*)(st + kPOffVel),
                        (const float*)(st + (f ? kPOffKB : kPOffKA)),
                        (const uint32_t*)(st + kPOffWord), r, cbase + 4, a.status};
      const int2 o = origin[s];
      const int x = o.x + cbase, y = o.y + r;
      const long long n = (long long)(y + kYO) * a.pitch + (x + kXO);
      double v = 0.0;
      if (group_is_interior(x - lane, y, a.nx, a.ny))
        v = step_interior_group<kFinal, 0>(a, src, x, y, n, a.frac);
      else if (x < a.nx && y < a.ny && !on_open_side(x, y, a.nx, a.ny, a.open_mask))
        v = step_node<float, kFinal, true, false, 0, true>(a, src, x, y, n, a.frac);
      if (f) u1 += v;
      else u0 += v;
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
  __syncthreads();
  if (abort_flag) {
    if (tid == 0) {
      atomicExch(a0.status, 1);
      atomicExch(a1.status, 1);
    }
    return;
  }
  if (kFinal) {
    const double s0 = block_sum(u0, red[0]);
    const double s1 = block_sum(u1, red[1]);
    if (tid == 0) {
      a0.partial[blockIdx.x] = s0;
      a1.partial[blockIdx.x] = s1;
    }
  }
}

// Equal solid links and equal velocity of the two fields, node by node.
__global__ void k_same_geometry(const uint32_t* __restrict__ la, const uint32_t* __restrict__ lb,
                                const float* __restrict__ va, const float* __restrict__ vb,
                                long long plane, int* __restrict__ differ) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane;
       i += (long long)gridDim.x * blockDim.x)
    if (la[i] != lb[i] || va[i] != vb[i] || va[plane + i] != vb[plane + i]) *differ = 1;
}

}  // namespace

struct lbm_pair {
  lbm_ctx* c[2] = {nullptr, nullptr};
  PairMaps maps[2];  // by buffer parity of the pair's current state
  int ntx = 0, nty = 0, grid = 0;
};

extern "C" {

lbm_status lbm_pair_create(lbm_pair** out, lbm_ctx* a, lbm_ctx* b) {
  if (!out || !a || !b || a == b) return ctx_fail(LBM_ERR_ARG, "lbm_pair_create: bad arguments");
  *out = nullptr;
  const lbm_params &p = a->p, &q = b->p;
  bool same = p.nx == q.nx && p.ny == q.ny && a->esize == 4 && b->esize == 4 &&
              a->stream == b->stream && a->device == b->device && a->cur == b->cur &&
              !p.dissolution && !q.dissolution && a->wall_mode == LBM_WALL_BOUNCE &&
              b->wall_mode == LBM_WALL_BOUNCE && a->tma_ready && b->tma_ready && a->y0 == 0 && b->y0 == 0 &&
              a->p.ny == a->ny_global && b->p.ny == b->ny_global;
  for (int s = 0; s < 4; ++s) same = same && p.edge[s] == q.edge[s];
  if (!same)
    return ctx_fail(LBM_ERR_ARG,
                    "lbm_pair_create: the lattices must be FP32 and share size, sides, stream, "
                    "step parity and bounce-back walls, without dissolution");
  int* d = nullptr;
  int differ = 0;
  cudaError_t e = cudaMalloc((void**)&d, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(int), a->stream);
  if (e == cudaSuccess) {
    k_same_geometry<<<256, 256, 0, a->stream>>>(a->link, b->link, (const float*)a->vel,
                                                (const float*)b->vel, a->plane, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&differ, d, sizeof(int), cudaMemcpyDeviceToHost, a->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(a->stream);
  if (d) cudaFree(d);
  if (e != cudaSuccess) return ctx_fail(LBM_ERR_CUDA, "lbm_pair_create: %s", cudaGetErrorString(e));
  if (differ)
    return ctx_fail(LBM_ERR_ARG, "lbm_pair_create: the lattices' solid masks or velocities differ");
  lbm_pair* pr = new (std::nothrow) lbm_pair();
  if (!pr) return ctx_fail(LBM_ERR_NOMEM, "lbm_pair_create: host allocation failed");
  pr->c[0] = a;
  pr->c[1] = b;
  const cuuint64_t P = (cuuint64_t)a->pitch, H = (cuuint64_t)padded_rows(p.ny);
  const cuuint64_t dpop[3] = {P, H, 9}, spop[2] = {P * 4, P * H * 4};
  const cuuint32_t bpop[3] = {kBoxW, kPBoxH, 9};
  const cuuint64_t dvel[3] = {P, H, 2};
  const cuuint32_t bvel[3] = {kTW, kPH, 2};
  const cuuint64_t d2[2] = {P, H}, s2[1] = {P * 4};
  const cuuint32_t b2[2] = {kTW, kPH};
  lbm_status st = LBM_OK;
  for (int par = 0; par < 2 && st == LBM_OK; ++par) {
    PairMaps& m = pr->maps[par];
    for (int f = 0; f < 2 && st == LBM_OK; ++f) {
      lbm_ctx* c = pr->c[f];
      st = ctx_make_map("pair population", &m.pop[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                        c->f[par], dpop, spop, bpop);
      if (st == LBM_OK)
        st = c->kf ? ctx_make_map("pair rate", &m.kf[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                                  c->kf, d2, s2, b2)
                   : ctx_make_map("pair rate", &m.kf[f], CU_TENSOR_MAP_DATA_TYPE_UINT32, 2,
                                  a->link, d2, s2, b2);
    }
    if (st == LBM_OK)
      st = ctx_make_map("pair velocity", &m.vel, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a->vel, dvel,
                        spop, bvel);
    if (st == LBM_OK)
      st = ctx_make_map("pair link", &m.link, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, a->link, d2, s2,
                        b2);
  }
  if (st == LBM_OK &&
      (cudaFuncSetAttribute(lbm_step_tma_pair<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            kPSmem) != cudaSuccess ||
       cudaFuncSetAttribute(lbm_step_tma_pair<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            kPSmem) != cudaSuccess))
    st = ctx_fail(LBM_ERR_CUDA, "lbm_pair_create: cudaFuncSetAttribute failed");
  if (st != LBM_OK) {
    delete pr;
    return st;
  }
  pr->ntx = (p.nx + kTW - 1) / kTW;
  pr->nty = (p.ny + kPH - 1) / kPH;
  const int nt = pr->ntx * pr->nty;
  pr->grid = nt < a->num_sms ? nt : a->num_sms;
  *out = pr;
  return LBM_OK;
}

lbm_status lbm_pair_substeps(lbm_pair* pr, int n, int eta, const double* a_dir_t0,
                             const double* a_dir_t1, const double* a_q, const double* b_dir_t0,
                             const double* b_dir_t1, const double* b_q) {
  if (!pr) return ctx_fail(LBM_ERR_ARG, "lbm_pair_substeps: null pair");
  if (n < 0 || eta < 1) return ctx_fail(LBM_ERR_ARG, "lbm_pair_substeps: need n >= 0, eta >= 1");
  lbm_ctx *a = pr->c[0], *b = pr->c[1];
  if (a->cur != b->cur)
    return ctx_fail(LBM_ERR_STATE,
                    "lbm_pair_substeps: a lattice of the pair was stepped on its own");
  if (n == 0) return LBM_OK;
  lbm_status st = ctx_stage_edges(a, a_dir_t0, a_dir_t1, a_q);
  if (st == LBM_OK) st = ctx_stage_edges(b, b_dir_t0, b_dir_t1, b_q);
  if (st != LBM_OK) return st;
  for (int j = 1; j <= n; ++j) {
    const double frac = (double)j / (double)eta;
    StepArgs<float> s0 = step_args<float>(a, frac), s1 = step_args<float>(b, frac);
    s1.link = a->link;  // one geometry: field B reads field A's links and velocity
    s1.vel = (const float*)a->vel;
    const PairMaps& m = pr->maps[a->cur];
    if (j == n)
      lbm_step_tma_pair<true><<<pr->grid, kTmaBlock, kPSmem, a->stream>>>(s0, s1, m, pr->ntx, pr->nty);
    else
      lbm_step_tma_pair<false><<<pr->grid, kTmaBlock, kPSmem, a->stream>>>(s0, s1, m, pr->ntx, pr->nty);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx_fail(LBM_ERR_CUDA, "lbm_pair_substeps: %s", cudaGetErrorString(e));
    for (lbm_ctx* c : pr->c) {
      c->cur ^= 1;
      c->steps += 1;
      if (j == n) c->nparts = pr->grid;
    }
  }
  return LBM_OK;
}

void lbm_pair_destroy(lbm_pair* pr) { delete pr; }

}  // extern "C"
