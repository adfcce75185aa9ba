// lbm_tma.cuh -- the FP32 fused step as a persistent, TMA-fed tile pipeline.
//
// One CTA per SM walks the lattice in 96 x 8 node tiles (tile t, t + grid,
// ...).  For each tile one cp.async.bulk.tensor 3-D box brings all nine
// population planes with a one-node halo (104 x 10 x 9 floats), and two more
// bring the velocity (96 x 8 x 2) and the link words (96 x 8), optionally
// the rate field; an mbarrier per stage counts the bytes in.  Four stages
// keep three tiles in flight while the CTA's 24 consumer warps update the
// fourth from shared memory with step_node(), which is shared with the
// generic kernel, and store f* with coalesced row writes.  (The update is
// bound by the consumers' instruction latency, so the tile is sized for as
// many consumer warps as the register file holds.)  The nodes on
// non-periodic sides, whose boundary solves run in FP64 (slow on this part),
// are left to one boundary warp per CTA that reads them from global memory
// beside the pipeline, so no consumer warp waits on the FP64 pipe.  Every
// wait on an mbarrier has an iteration limit: on expiry the CTA records a
// status, drains its copies in flight (again with a limit) and returns.
#pragma once
#include <cuda.h>

#include "lbm_kernels.cuh"

namespace lbm {

constexpr int kTW = 96;            // tile width (nodes)
constexpr int kTH = 8;             // tile height (rows)
constexpr int kBoxW = kTW + 8;     // halo box width: 4 columns each side (16 B aligned)
constexpr int kBoxH = kTH + 2;     // halo box height: one row each side
constexpr int kStages = 4;
constexpr int kTmaThreads = 768;   // consumer threads: 24 warps
constexpr int kTmaBlock = kTmaThreads + 64;  // plus one producer and one boundary warp
constexpr int kBoundaryWarp = kTmaThreads / 32 + 1;
constexpr int kWarpsPerRow = (kTmaThreads / 32) / kTH;    // consumer warps sharing a tile row
constexpr int kNodesPerLane = kTW / (32 * kWarpsPerRow);  // nodes of a row per lane
static_assert((kTmaThreads / 32) % kTH == 0 && kNodesPerLane * 32 * kWarpsPerRow == kTW,
              "tile mapping");
// Bounded waits: a wait on an mbarrier gives up after kWaitLimitNs of
// wall-clock time (the kernel then records a status and returns); each poll
// lets the hardware suspend the warp for up to kSuspendNs until the phase
// completes, so a waiting warp issues a handful of instructions, not a spin.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s
constexpr unsigned kSuspendNs = 100000u;                     // 100 us per poll

constexpr int round128(int b) { return (b + 127) / 128 * 128; }
constexpr int kPopBytes = 9 * kBoxH * kBoxW * 4;
constexpr int kVelBytes = 2 * kTH * kTW * 4;
constexpr int kKBytes = kTH * kTW * 4;
constexpr int kWordBytes = kTH * kTW * 4;
constexpr int kOffVel = round128(kPopBytes);
constexpr int kOffK = kOffVel + round128(kVelBytes);
constexpr int kOffWord = kOffK + round128(kKBytes);
constexpr int kStageBytes = kOffWord + round128(kWordBytes);
constexpr int kTmaSmem = kStages * kStageBytes;
static_assert(kTmaSmem <= 227 * 1024, "stages exceed shared memory");

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait; false if the phase did not complete within kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > kWaitLimitNs) return false;
  return true;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0,
                                            int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0,
                                            int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to this CTA's shared memory; completion counts on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Inputs of one node read from the shared-memory tile of its stage: tiles of
// kTW x TH nodes, the population box one node wider on every side.
template <int TH>
struct SmemSrcT {
  static constexpr int kBH = TH + 2;  // box rows
  const float* pop;      // [9][kBH][kBoxW]
  const float* vel;      // [2][TH][kTW]
  const float* kfield;   // [TH][kTW]
  const uint32_t* words; // [TH][kTW] link words
  int r, c;              // node's row in the tile, column in the halo box (xl + 4)
  int* flag;             // status word (index checks of the debug build)
  __device__ __forceinline__ int at(int i) const {  // box offset of x - e_i
    return (r + 1 - cy_of(i)) * kBoxW + (c - cx_of(i));
  }
  __device__ __forceinline__ long long pb(long long i) const {
    return dbg_idx(i, 9 * kBH * kBoxW, flag, kSiteSmemPop);
  }
  __device__ __forceinline__ long long nb(long long i, int planes = 1) const {
    return dbg_idx(i, planes * TH * kTW, flag, kSiteSmemNode);
  }
  __device__ __forceinline__ uint32_t word() const { return words[nb(r * kTW + (c - 4))]; }
  __device__ __forceinline__ float pull(int i) const { return pop[pb(i * kBH * kBoxW + at(i))]; }
  __device__ __forceinline__ float own(int i) const {
    return pop[pb(i * kBH * kBoxW + (r + 1) * kBoxW + c)];
  }
  __device__ __forceinline__ float pull_or_bounce(int i, bool bounce) const {
    return pop[pb(bounce ? opp_of(i) * kBH * kBoxW + (r + 1) * kBoxW + c
                         : i * kBH * kBoxW + at(i))];
  }
  __device__ __forceinline__ float vx() const { return vel[nb(r * kTW + (c - 4), 2)]; }
  __device__ __forceinline__ float vy() const { return vel[nb((TH + r) * kTW + (c - 4), 2)]; }
  __device__ __forceinline__ float kf() const { return kfield[nb(r * kTW + (c - 4))]; }
};
using SmemSrc = SmemSrcT<kTH>;

// Step of a warp's 32 interior nodes from a shared-memory tile, by the
// warp's class (a warp-uniform choice on the link words): every lane clear
// of solids takes the clear path; every lane solid (and not turning fluid)
// has nothing to update but its u; other warps take the general path.
template <bool kFinal, int kWalls, class Src>
__device__ __forceinline__ double step_interior_group(const StepArgs<float>& a, const Src& src,
                                                      int x, int y, long long n, double frac) {
  const uint32_t w = src.word();
  if (__all_sync(0xFFFFFFFFu, (w & kClearMask) == 0u))
    return step_node<float, kFinal, false, false, kWalls, true, true>(a, src, x, y, n, frac);
  if (__all_sync(0xFFFFFFFFu, (w & (kOwnSolid | kOwnPending)) == kOwnSolid)) {
    if (kFinal) a.u_out[dbg_idx(n, a.plane, a.status, kSiteNode)] = 0.0f;
    if (a.u_hist) a.u_hist[dbg_idx(n, a.plane, a.status, kSiteNode)] = 0.0f;
    return 0.0;
  }
  return step_node<float, kFinal, false, false, kWalls, true>(a, src, x, y, n, frac);
}

struct TmaMaps {
  CUtensorMap pop;   // fin: [9][rows][pitch] float, box {kBoxW, kBoxH, 9}
  CUtensorMap vel;   // [2][rows][pitch] float, box {kTW, kTH, 2}
  CUtensorMap link;  // [rows][pitch] uint32 link words, box {kTW, kTH}
  CUtensorMap kf;    // [rows][pitch] float, box {kTW, kTH} (valid if a.kf)
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Warp-specialised pipeline: warp 0 is the producer (one lane issues the TMA
// boxes of tile k into stage k % kStages once all consumer warps have
// released that stage), warps 1..24 are consumers (each updates a third of
// one tile row and releases the stage with one arrival), warp 25 steps the
// CTA's share of the nodes on non-periodic sides from global memory.  No
// CTA-wide barrier sits inside the tile loop.
template <bool kFinal, int kWalls = 0>
__global__ void __launch_bounds__(kTmaBlock, 1)
    lbm_step_tma(const StepArgs<float> a, const __grid_constant__ TmaMaps maps, int ntx,
                 int nty) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  __shared__ int2 origin[kStages];  // tile origin of each stage, set by the producer
  __shared__ double red[kTmaBlock / 32];
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int ntiles = ntx * nty;
  const uint32_t bytes = kPopBytes + kVelBytes + kWordBytes + (a.kf ? kKBytes : 0);

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kTmaThreads / 32);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  double my_u = 0.0;
  if (warp == 0) {
    // ---- producer ------------------------------------------------------
    if (lane == 0) {
      int k = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = k % kStages;
        if (k >= kStages &&
            !mbar_wait(&empty[s], (uint32_t)(((k / kStages) - 1) & 1))) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (*(volatile int*)&abort_flag) break;
        unsigned char* st = smem + s * kStageBytes;
        const int x0 = (t % ntx) * kTW, y0 = (t / ntx) * kTH;
        origin[s] = make_int2(x0, y0);  // published by the arrival below
        mbar_expect_tx(&full[s], bytes);
        tma_load_3d(st, &maps.pop, x0 + kXO - 4, y0, 0, &full[s]);
        tma_load_3d(st + kOffVel, &maps.vel, x0 + kXO, y0 + kYO, 0, &full[s]);
        tma_load_2d(st + kOffWord, &maps.link, x0 + kXO, y0 + kYO, &full[s]);
        if (a.kf) tma_load_2d(st + kOffK, &maps.kf, x0 + kXO, y0 + kYO, &full[s]);
      }
      if (*(volatile int*)&abort_flag) {
        // drain: every issued box must land before shared memory goes away
        for (int kk = (k >= kStages ? k - kStages : 0); kk < k; ++kk)
          (void)mbar_wait(&full[kk % kStages], (uint32_t)((kk / kStages) & 1));
      }
    }
  } else if (warp == kBoundaryWarp) {
    // ---- boundary nodes: FP64 maximum-entropy solves beside the pipeline --
    // (every lane runs the same trip count; lanes past the list idle)
    for (int e0 = blockIdx.x * 32; e0 < a.n_open; e0 += gridDim.x * 32) {
      const int e = e0 + lane;
      if (e < a.n_open) {
        const int n = a.open_nodes[dbg_idx(e, a.n_open, a.status, kSiteNode)];
        const int y = n / a.pitch - kYO, x = n - (y + kYO) * a.pitch - kXO;
        GlobalSrc<float> src{a, n};
        my_u += step_node<float, kFinal, true, true, kWalls>(a, src, x, y, n, a.frac);
      }
    }
  } else {
    // ---- consumers ------------------------------------------------------
    const int cw = warp - 1;                  // 0 .. kTmaThreads / 32 - 1
    const int r = cw / kWarpsPerRow;          // tile row of this warp
    const int cbase = (cw % kWarpsPerRow) * (32 * kNodesPerLane) + lane;  // first column
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
      const int s = k % kStages;
      if (!mbar_wait(&full[s], (uint32_t)((k / kStages) & 1))) {
        atomicExch(&abort_flag, 1);
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      const unsigned char* st = smem + s * kStageBytes;
      SmemSrc src{(const float*)st, (const float*)(st + kOffVel), (const float*)(st + kOffK),
                  (const uint32_t*)(st + kOffWord), r, 0, a.status};
      const int2 o = origin[s];
      const int x0 = o.x, y = o.y + r;
#pragma unroll 1
      for (int j = 0; j < kNodesPerLane; ++j) {
        const int xl = cbase + 32 * j;
        const int x = x0 + xl;
        src.c = xl + 4;
        const long long n = (long long)(y + kYO) * a.pitch + (x + kXO);
        if (group_is_interior(x - lane, y, a.nx, a.ny))
          my_u += step_interior_group<kFinal, kWalls>(a, src, x, y, n, a.frac);
        else if (x < a.nx && y < a.ny && !on_open_side(x, y, a.nx, a.ny, a.open_mask))
          my_u += step_node<float, kFinal, true, false, kWalls, true>(a, src, x, y, n, a.frac);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
  __syncthreads();
  if (abort_flag) {
    if (tid == 0) atomicExch(a.status, 1);
    return;
  }
  if (kFinal) {
    const double s = block_sum(my_u, red);
    if (tid == 0) a.partial[blockIdx.x] = s;
  }
}

}  // namespace lbm
