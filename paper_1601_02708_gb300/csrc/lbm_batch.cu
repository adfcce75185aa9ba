// lbm_batch.cu -- many lattices of different sizes advanced together
// (declared in include/lbm_ade.h).
//
// A batch is built from contexts made by lbm_init; they keep their own
// state, read-out and save/restore.  The batch adds device tables: the step
// arguments of every member for both buffer parities, a tile list over all
// members (member, tile origin, rate-field flag, tile index in the member) and
// a block map over the members' dissolution surface lists.  One persistent
// step kernel walks the tile list and one dissolution kernel walks every
// list, so a time step of the whole batch is two launches whatever the
// number of members (the multi-subdomain loop of Sec. 6.3, Algorithm 2, runs
// many pore-scale subdomains).  Each (n, eta, parity) sequence of launches is
// recorded once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <map>
#include <type_traits>
#include <tuple>
#include <vector>

#include "lbm_ade.h"
#include "lbm_batch_plain.cuh"
#include "lbm_ctx.h"
#include "lbm_kernels.cuh"

namespace {

thread_local char g_err[512] = "";

lbm_status fail(lbm_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

#define BCK(call)                                                                 \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA, \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                \
  } while (0)

using lbm::ArgSlot;
constexpr int kRateBit = lbm::kBatchRateBit;
constexpr int kTileMask = lbm::kBatchTileMask;
constexpr int kPlainShapes = lbm::kBatchPlainShapes;
constexpr int kTmaShape = kPlainShapes;  // the TMA-fed pipeline (FP32), 96 x 8 tiles
constexpr int kNumShapes = kPlainShapes + 1;

// ---- TMA-fed variant (FP32) ---------------------------------------------

// Tensor maps of one member: the population map of either buffer and the
// velocity, link-word and rate maps (boxes as in lbm_tma.cuh).  Kept in
// global memory, written once from the host.
struct MemberMaps {
  CUtensorMap pop[2];
  CUtensorMap vel, link, kf;
};

constexpr int kArgBytes = (int)sizeof(ArgSlot<float>);
constexpr int kOffArgs = lbm::kStageBytes;  // stage: boxes of lbm_tma.cuh, then
constexpr int kOffTd = kOffArgs + kArgBytes;  // the member's arguments, the tile
constexpr int kBStage = lbm::round128(kOffTd + 16);
constexpr int kBTmaSmem = lbm::kStages * kBStage;
static_assert(kArgBytes % 16 == 0, "bulk copies move whole 16-byte units");
static_assert(kBTmaSmem + 1024 <= 227 * 1024, "stages exceed shared memory");

// A tensor map written to global memory by the host is made visible to the
// tensor-map proxy of this thread before its first use.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(
                   reinterpret_cast<uint64_t>(m))
               : "memory");
}

// The pipeline of lbm_step_tma over a tile list of many members: the
// producer lane reads each tile's descriptor, fetches the member's arguments
// (one bulk copy) with the tile's boxes into the stage, and the consumers
// take member, origin and arguments from the stage.  On the final substep
// each tile's mass partial is summed in a fixed order by consumer warp 0
// once the other warps have posted theirs (an mbarrier per stage).  The
// boundary warp steps the nodes on every member's non-periodic sides from
// global memory (FP64 solves), in chunks of 32 nodes of one member:
// otask[32 c + lane] = (member, padded node index or -1, partial slot, 0).
template <bool kFinal, int kWalls = 0>
__global__ void __launch_bounds__(lbm::kTmaBlock, 1)
    lbm_step_tma_batch(const ArgSlot<float>* __restrict__ args,
                       const MemberMaps* __restrict__ maps, int par,
                       const int4* __restrict__ tiles, int ntiles,
                       const int4* __restrict__ otask, int nchunks, double frac) {
  using namespace lbm;
  constexpr int kCW = kTmaThreads / 32;  // consumer warps
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  __shared__ __align__(8) uint64_t summed[kStages];
  __shared__ double red[kStages][kCW];
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const uint32_t base_bytes = kPopBytes + kVelBytes + kWordBytes + kArgBytes;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kCW);
      mbar_init(&summed[s], kCW);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == 0) {
    // ---- producer ------------------------------------------------------
    if (lane == 0) {
      int k = 0, member = -1;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = k % kStages;
        if (k >= kStages && !mbar_wait(&empty[s], (uint32_t)(((k / kStages) - 1) & 1))) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (*(volatile int*)&abort_flag) break;
        const int4 td = tiles[t];
        const bool rate = (td.w & kRateBit) != 0;
        const MemberMaps* mm = maps + td.x;
        if (td.x != member) {
          tensormap_acquire(&mm->pop[par]);
          tensormap_acquire(&mm->vel);
          tensormap_acquire(&mm->link);
          if (rate) tensormap_acquire(&mm->kf);
          member = td.x;
        }
        unsigned char* st = smem + s * kBStage;
        *reinterpret_cast<int4*>(st + kOffTd) = td;  // published by the arrive below
        mbar_expect_tx(&full[s], base_bytes + (rate ? kKBytes : 0));
        bulk_load(st + kOffArgs, args + td.x, kArgBytes, &full[s]);
        tma_load_3d(st, &mm->pop[par], td.y + kXO - 4, td.z, 0, &full[s]);
        tma_load_3d(st + kOffVel, &mm->vel, td.y + kXO, td.z + kYO, 0, &full[s]);
        tma_load_2d(st + kOffWord, &mm->link, td.y + kXO, td.z + kYO, &full[s]);
        if (rate) tma_load_2d(st + kOffK, &mm->kf, td.y + kXO, td.z + kYO, &full[s]);
      }
      if (*(volatile int*)&abort_flag) {
        for (int kk = (k >= kStages ? k - kStages : 0); kk < k; ++kk)
          (void)mbar_wait(&full[kk % kStages], (uint32_t)((kk / kStages) & 1));
      }
    }
  } else if (warp == kBoundaryWarp) {
    // ---- boundary nodes of every member: FP64 solves beside the pipeline --
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
      const int4 task = otask[32 * ch + lane];
      const StepArgs<float>& a = args[task.x].a;  // one member per chunk
      double u = 0.0;
      if (task.y >= 0) {
        const int n = task.y;
        const int y = n / a.pitch - kYO, x = n - (y + kYO) * a.pitch - kXO;
        GlobalSrc<float> src{a, n};
        u = step_node<float, kFinal, true, true, kWalls>(a, src, x, y, n, frac);
      }
      if (kFinal) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
        if (lane == 0) a.partial[task.z] = u;
      }
    }
  } else {
    // ---- consumers ------------------------------------------------------
    const int cw = warp - 1;
    const int r = cw / kWarpsPerRow;
    const int cbase = (cw % kWarpsPerRow) * (32 * kNodesPerLane) + lane;
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
      const int s = k % kStages;
      const uint32_t ph = (uint32_t)((k / kStages) & 1);
      if (!mbar_wait(&full[s], ph)) {
        atomicExch(&abort_flag, 1);
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      const unsigned char* st = smem + s * kBStage;
      const int4 td = *reinterpret_cast<const int4*>(st + kOffTd);
      const StepArgs<float>& a = *reinterpret_cast<const StepArgs<float>*>(st + kOffArgs);
      SmemSrc src{(const float*)st, (const float*)(st + kOffVel), (const float*)(st + kOffK),
                  (const uint32_t*)(st + kOffWord), r, 0, a.status};
      const int x0 = td.y, y = td.z + r;
      double tile_u = 0.0;
#pragma unroll 1
      for (int j = 0; j < kNodesPerLane; ++j) {
        const int xl = cbase + 32 * j;
        const int x = x0 + xl;
        src.c = xl + 4;
        const long long n = (long long)(y + kYO) * a.pitch + (x + kXO);
        if (group_is_interior(x - lane, y, a.nx, a.ny))
          tile_u += step_interior_group<kFinal, kWalls>(a, src, x, y, n, frac);
        else if (x < a.nx && y < a.ny && !on_open_side(x, y, a.nx, a.ny, a.open_mask))
          tile_u += step_node<float, kFinal, true, false, kWalls, true>(a, src, x, y, n, frac);
      }
      if (kFinal) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tile_u += __shfl_down_sync(0xffffffffu, tile_u, o);
        if (lane == 0) {
          red[s][cw] = tile_u;
          mbar_arrive(&summed[s]);
        }
        if (cw == 0) {
          if (!mbar_wait(&summed[s], ph)) {
            atomicExch(&abort_flag, 1);
            break;
          }
          if (lane == 0) {
            double sum = 0.0;
            for (int i = 0; i < kCW; ++i) sum += red[s][i];
            a.partial[td.w & kTileMask] = sum;
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
  __syncthreads();
  if (abort_flag && tid == 0) {
    // every member this CTA served may hold unfinished tiles
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) atomicExch(args[tiles[t].x].a.status, 1);
  }
}

// Dissolution of every member's surface list: block b serves member
// bmap[b].x as its bmap[b].y-th of nblk[member] blocks; the last block of a
// member to finish applies that member's flips (and closes its pass).
template <typename Share>
__global__ void __launch_bounds__(lbm::kDThreads)
    lbm_dissolve_batch(const lbm::DissolveArgs* __restrict__ dargs,
                       const void* const* __restrict__ rlinks, const int2* __restrict__ bmap,
                       const int* __restrict__ nblk) {
  __shared__ lbm::DissolveArgs d;
  __shared__ bool last;
  const double* const tab = lbm::share_table();
  const int tid = threadIdx.x;
  const int2 bm = bmap[blockIdx.x];
  if (tid == 0) d = dargs[bm.x];
  __syncthreads();
  const Share* rlink = (const Share*)rlinks[bm.x];
  const int nb = nblk[bm.x];
  const int pass = *(volatile int*)d.pass;
  bool flipped = false;
  const int count = *d.scount;
  for (int e = bm.y * lbm::kDThreads + tid; e < count; e += nb * lbm::kDThreads) {
    const int n = d.slist[e];
    const uint32_t w = d.link[n];
    if (!(w & lbm::kOwnSolid)) continue;
    if (w & lbm::kOwnPending) {
      lbm::finish_flip(d, n, pass);
      continue;
    }
    const uint32_t fluid = ~((w >> lbm::kUpPostShift) | (w >> lbm::kUpOutShift)) & 0xFFu;
    if (!fluid) continue;
    const double m = d.smin[e] - lbm::mineral_take(rlink, n, d, fluid, tab);
    d.smin[e] = m;
    if (m <= 0.0) {
      d.flip_list[lbm::dbg_idx(atomicAdd(d.flip_count, 1), (long long)d.nx * d.ny, d.status, lbm::kSiteList)] = n;
      flipped = true;
    }
  }
  if (flipped) __threadfence();
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    last = (atomicAdd(d.done, 1u) == (unsigned)nb - 1);
  }
  __syncthreads();
  if (last) lbm::apply_flips(d, tid, lbm::kDThreads);
}

}  // namespace

struct lbm_batch {
  std::vector<lbm_ctx*> m;
  int esize = 4;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int shape = 0;
  // per shape: tile list and each member's tile count
  int4* tiles[kNumShapes] = {};
  int ntiles[kNumShapes] = {};
  std::vector<int> member_tiles[kNumShapes];
  // boundary-warp tasks of the pipelined shape: chunks of 32 nodes of one
  // member on its non-periodic sides, and each member's chunk count
  int4* otask = nullptr;
  int nchunks = 0;
  std::vector<int> member_chunks;
  void* args[2] = {nullptr, nullptr};  // ArgSlot<Real>[n] for fin = f[0] / f[1]
  MemberMaps* maps = nullptr;          // [n], FP32 batches whose members all have maps
  lbm::DissolveArgs* dargs = nullptr;
  void** rlinks = nullptr;
  int2* bmap = nullptr;
  int* nblk = nullptr;
  int dblocks = 0;
  int walls = 0;  // wall variant of the members when the batch was made (walls_variant)
  std::map<std::tuple<int, int, int, int>, cudaGraphExec_t> graphs;  // (n, eta, parity, shape)
};

namespace {

void free_batch(lbm_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (int s = 0; s < kNumShapes; ++s)
    if (b->tiles[s]) cudaFree(b->tiles[s]);
  void* ptrs[] = {b->args[0], b->args[1], b->maps, b->dargs, b->rlinks,
                  b->bmap,    b->nblk,    b->otask};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete b;
}

template <typename Real>
lbm_status upload_args(lbm_batch* b) {
  const int n = (int)b->m.size();
  for (int par = 0; par < 2; ++par) {
    std::vector<ArgSlot<Real>> h(n);
    for (int i = 0; i < n; ++i) {
      lbm_ctx* c = b->m[i];
      const int keep = c->cur;
      c->cur = par;
      h[i].a = step_args<Real>(c, 0.0);
      c->cur = keep;
    }
    BCK(cudaMalloc(&b->args[par], n * sizeof(ArgSlot<Real>)));
    BCK(cudaMemcpy(b->args[par], h.data(), n * sizeof(ArgSlot<Real>), cudaMemcpyHostToDevice));
  }
  return LBM_OK;
}

template <bool kFinal, int kWalls>
lbm_status set_tma_smem() {
  BCK(cudaFuncSetAttribute(lbm_step_tma_batch<kFinal, kWalls>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, kBTmaSmem));
  return LBM_OK;
}

// Tensor maps of every member for the pipelined kernel (FP32 members that
// all carry maps), and its boundary-warp tasks; otherwise that shape stays
// unavailable.
lbm_status upload_maps(lbm_batch* b) {
  if (b->esize != 4) return LBM_OK;
  for (lbm_ctx* c : b->m)
    if (!c->tma_ready) return LBM_OK;
  const int n = (int)b->m.size();
  std::vector<MemberMaps> h(n);
  for (int i = 0; i < n; ++i) {
    const lbm_ctx* c = b->m[i];
    h[i].pop[0] = c->maps[0].pop;
    h[i].pop[1] = c->maps[1].pop;
    h[i].vel = c->maps[0].vel;
    h[i].link = c->maps[0].link;
    h[i].kf = c->maps[0].kf;
  }
  BCK(cudaMalloc((void**)&b->maps, n * sizeof(MemberMaps)));
  BCK(cudaMemcpy(b->maps, h.data(), n * sizeof(MemberMaps), cudaMemcpyHostToDevice));
  lbm_status st = LBM_OK;
  if (st == LBM_OK) st = set_tma_smem<true, 0>();
  if (st == LBM_OK) st = set_tma_smem<false, 0>();
  if (st == LBM_OK) st = set_tma_smem<true, 1>();
  if (st == LBM_OK) st = set_tma_smem<false, 1>();
  if (st == LBM_OK) st = set_tma_smem<true, 2>();
  if (st == LBM_OK) st = set_tma_smem<false, 2>();
  if (st != LBM_OK) return st;
  // boundary tasks: each member's open nodes (device list of its context)
  // in chunks of 32, padded with -1; chunk c of member i owns partial slot
  // member_tiles[kTmaShape][i] + c (the tile list is built before this)
  std::vector<int4> tasks;
  b->member_chunks.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    lbm_ctx* c = b->m[i];
    if (c->n_open == 0) continue;
    std::vector<int> nodes(c->n_open);
    BCK(cudaMemcpy(nodes.data(), c->open_nodes, nodes.size() * sizeof(int),
                   cudaMemcpyDeviceToHost));
    const int chunks = (c->n_open + 31) / 32;
    for (int ch = 0; ch < chunks; ++ch) {
      const int slot = b->member_tiles[kTmaShape][i] + ch;
      if (slot >= c->partial_cap)
        return fail(LBM_ERR_STATE, "lbm_batch_create: member %d has too few partial slots", i);
      for (int l = 0; l < 32; ++l) {
        const int e = 32 * ch + l;
        tasks.push_back(make_int4(i, e < c->n_open ? nodes[e] : -1, slot, 0));
      }
    }
    b->member_chunks[i] = chunks;
  }
  b->nchunks = (int)(tasks.size() / 32);
  if (!tasks.empty()) {
    BCK(cudaMalloc((void**)&b->otask, tasks.size() * sizeof(int4)));
    BCK(cudaMemcpy(b->otask, tasks.data(), tasks.size() * sizeof(int4), cudaMemcpyHostToDevice));
  }
  return LBM_OK;
}

template <typename Real, bool kFinal, int kWalls>
void launch_step_shape(lbm_batch* b, int shape, int par, double frac) {
  if (shape == kTmaShape) {  // FP32 only (set_shape checks)
    if constexpr (sizeof(Real) == 4) {
      const int grid = b->ntiles[shape] < b->num_sms ? b->ntiles[shape] : b->num_sms;
      lbm_step_tma_batch<kFinal, kWalls><<<grid, lbm::kTmaBlock, kBTmaSmem, b->stream>>>(
          (const ArgSlot<float>*)b->args[par], b->maps, par, b->tiles[shape], b->ntiles[shape],
          b->otask, b->nchunks, frac);
    }
    return;
  }
  const int grid = b->ntiles[shape] < 8 * b->num_sms ? b->ntiles[shape] : 8 * b->num_sms;
  lbm::launch_batch_plain<Real, kFinal, kWalls>(shape, grid, b->stream,
                                                (const ArgSlot<Real>*)b->args[par],
                                                b->tiles[shape], b->ntiles[shape], frac);
}

template <typename Real, int kWalls>
void launch_step_walls(lbm_batch* b, bool final_step, int shape, int par, double frac) {
  if (final_step) launch_step_shape<Real, true, kWalls>(b, shape, par, frac);
  else launch_step_shape<Real, false, kWalls>(b, shape, par, frac);
}

// Enqueue n steps starting at buffer parity par (no capture logic here).
template <typename Real>
void enqueue_steps(lbm_batch* b, int n, int eta, int par, int shape) {
  using Share = typename std::conditional<sizeof(Real) == 8, double, lbm::ShareF32>::type;
  for (int j = 1; j <= n; ++j) {
    const double frac = (double)j / (double)eta;
    if (b->walls == 0) {
      launch_step_walls<Real, 0>(b, j == n, shape, par, frac);
    } else if constexpr (sizeof(Real) == 8) {
      launch_step_walls<Real, 1>(b, j == n, shape, par, frac);
    } else {
      if (b->walls == 1) launch_step_walls<Real, 1>(b, j == n, shape, par, frac);
      else launch_step_walls<Real, 2>(b, j == n, shape, par, frac);
    }
    par ^= 1;
    if (b->dblocks > 0)
      lbm_dissolve_batch<Share><<<b->dblocks, lbm::kDThreads, 0, b->stream>>>(
          b->dargs, (const void* const*)b->rlinks, b->bmap, b->nblk);
  }
}

lbm_status run_batch(lbm_batch* b, int n, int eta) {
  const int par = b->m[0]->cur;
  // the recorded graphs fix every member's buffer parity: a member stepped on
  // its own by an odd number of steps would read the wrong buffer
  for (size_t i = 1; i < b->m.size(); ++i)
    if (b->m[i]->cur != par)
      return fail(LBM_ERR_STATE,
                  "lbm_batch: member %d was stepped outside the batch (its buffer parity "
                  "differs from member 0's)", (int)i);
  const auto key = std::make_tuple(n, eta, par, b->shape);
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    if (b->esize == 8) enqueue_steps<double>(b, n, eta, par, b->shape);
    else enqueue_steps<float>(b, n, eta, par, b->shape);
    const cudaError_t le = cudaGetLastError();
    const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return fail(LBM_ERR_CUDA, "batch graph capture failed: %s",
                  cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return fail(LBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ie));
    it = b->graphs.emplace(key, ex).first;
  }
  BCK(cudaGraphLaunch(it->second, b->stream));
  for (size_t i = 0; i < b->m.size(); ++i) {
    lbm_ctx* c = b->m[i];
    c->cur ^= (n & 1);
    c->steps += n;
    c->nparts = b->member_tiles[b->shape][i] + (b->shape == kTmaShape ? b->member_chunks[i] : 0);
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_batch_last_error(void) { return g_err; }

lbm_status lbm_batch_create(lbm_batch** out, int n, lbm_ctx* const* members) {
  g_err[0] = 0;
  if (!out || n < 1 || !members) return fail(LBM_ERR_ARG, "lbm_batch_create: bad arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!members[i]) return fail(LBM_ERR_ARG, "lbm_batch_create: null member %d", i);
    if (members[i]->esize != members[0]->esize || members[i]->stream != members[0]->stream ||
        members[i]->cur != members[0]->cur || members[i]->device != members[0]->device)
      return fail(LBM_ERR_ARG,
                  "lbm_batch_create: members must share precision, stream, device and "
                  "step parity (member %d differs)", i);
    for (int j = 0; j < i; ++j)
      if (members[j] == members[i]) return fail(LBM_ERR_ARG, "lbm_batch_create: member %d repeated", i);
  }
  if (members[0]->stream == nullptr)
    return fail(LBM_ERR_ARG,
                "lbm_batch_create: members must run on a created stream (the batch records "
                "CUDA graphs, which the legacy default stream cannot)");
  lbm_batch* b = new lbm_batch();
  b->m.assign(members, members + n);
  b->esize = (int)members[0]->esize;
  b->stream = members[0]->stream;
  b->num_sms = members[0]->num_sms;
  for (int i = 0; i < n; ++i) {
    const int v = walls_variant(members[i]);
    if (v != 0 && b->walls != 0 && v != b->walls) {
      free_batch(b);
      return fail(LBM_ERR_ARG,
                  "lbm_batch_create: members solve maximum-entropy walls in different "
                  "precisions (member %d)", i);
    }
    if (v != 0) b->walls = v;
  }
  lbm_status st = b->esize == 8 ? upload_args<double>(b) : upload_args<float>(b);
  if (st != LBM_OK) {
    free_batch(b);
    return st;
  }
  bool tma_ok = b->esize == 4;
  for (int i = 0; i < n; ++i) tma_ok = tma_ok && members[i]->tma_ready;
  // tile lists, one per shape
  for (int s = 0; s < kNumShapes; ++s) {
    if (s == kTmaShape && !tma_ok) continue;
    const int tw = s == kTmaShape ? lbm::kTW : 32;
    const int th = s == kTmaShape ? lbm::kTH
                                  : lbm::kBatchShapes[s].by * lbm::kBatchShapes[s].r;
    std::vector<int4> h;
    b->member_tiles[s].assign(n, 0);
    for (int i = 0; i < n; ++i) {
      const lbm_ctx* c = members[i];
      int k = 0;
      for (int y0 = 0; y0 < c->p.ny; y0 += th)
        for (int x0 = 0; x0 < c->p.nx; x0 += tw, ++k) {
          h.push_back(make_int4(i, x0, y0, k | (c->kf ? kRateBit : 0)));
        }
      b->member_tiles[s][i] = k;
    }
    b->ntiles[s] = (int)h.size();
    cudaError_t e = cudaMalloc((void**)&b->tiles[s], h.size() * sizeof(int4));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->tiles[s], h.data(), h.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      free_batch(b);
      return fail(LBM_ERR_CUDA, "lbm_batch_create: %s", cudaGetErrorString(e));
    }
  }
  if (tma_ok && (st = upload_maps(b)) != LBM_OK) {
    free_batch(b);
    return st;
  }
  // dissolution tables for members that dissolve: blocks in proportion to
  // their current surface-list length
  std::vector<lbm::DissolveArgs> dh(n);
  std::vector<void*> rh(n, nullptr);
  std::vector<int2> bm;
  std::vector<int> nb(n, 0);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    lbm_ctx* c = members[i];
    dh[i] = dissolve_args(c);
    rh[i] = c->ureact;
    if (!c->p.dissolution) continue;
    int len = 0;
    e = cudaMemcpy(&len, c->flip_count + 2, sizeof(int), cudaMemcpyDeviceToHost);
    nb[i] = len / 2048 + 1;
    for (int k = 0; k < nb[i]; ++k) bm.push_back(make_int2(i, k));
  }
  b->dblocks = (int)bm.size();
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->dargs, n * sizeof(lbm::DissolveArgs));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->rlinks, n * sizeof(void*));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->nblk, n * sizeof(int));
  if (e == cudaSuccess && !bm.empty()) e = cudaMalloc((void**)&b->bmap, bm.size() * sizeof(int2));
  if (e == cudaSuccess) e = cudaMemcpy(b->dargs, dh.data(), n * sizeof(lbm::DissolveArgs), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->rlinks, rh.data(), n * sizeof(void*), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->nblk, nb.data(), n * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !bm.empty())
    e = cudaMemcpy(b->bmap, bm.data(), bm.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_batch(b);
    return fail(LBM_ERR_CUDA, "lbm_batch_create: %s", cudaGetErrorString(e));
  }
  b->shape = b->maps ? kTmaShape : 0;
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_substeps(lbm_batch* b, int n, int eta, const double* const* u_dir_t0,
                              const double* const* u_dir_t1, const double* const* q_neu) {
  if (!b) return fail(LBM_ERR_ARG, "null batch");
  if (n < 0 || eta < 1) return fail(LBM_ERR_ARG, "lbm_batch_substeps: need n >= 0, eta >= 1");
  if (n == 0) return LBM_OK;
  for (size_t i = 0; i < b->m.size(); ++i) {
    lbm_ctx* c = b->m[i];
    const size_t eb = (size_t)c->nedge * sizeof(double);
    const double* src[3] = {u_dir_t0 ? u_dir_t0[i] : nullptr,
                            u_dir_t1 ? u_dir_t1[i] : (u_dir_t0 ? u_dir_t0[i] : nullptr),
                            q_neu ? q_neu[i] : nullptr};
    for (int k = 0; k < 3; ++k) {
      if (src[k]) BCK(cudaMemcpyAsync(c->edge + k * c->nedge, src[k], eb, cudaMemcpyDefault, b->stream));
      else BCK(cudaMemsetAsync(c->edge + k * c->nedge, 0, eb, b->stream));
    }
  }
  BCK(cudaStreamSynchronize(b->stream));  // host edge data may be reused after return
  return run_batch(b, n, eta);
}

lbm_status lbm_batch_set_shape(lbm_batch* b, int shape) {
  if (!b) return fail(LBM_ERR_ARG, "null batch");
  if (shape < 0 || shape >= kNumShapes) return fail(LBM_ERR_ARG, "lbm_batch_set_shape: shape %d", shape);
  if (shape == kTmaShape && !b->maps)
    return fail(LBM_ERR_ARG,
                "lbm_batch_set_shape: the pipelined shape needs FP32 members with the tile "
                "pipeline set up");
  b->shape = shape;
  return LBM_OK;
}

lbm_status lbm_batch_get_shape(const lbm_batch* b, int* shape) {
  if (!b || !shape) return fail(LBM_ERR_ARG, "lbm_batch_get_shape: null argument");
  *shape = b->shape;
  return LBM_OK;
}

lbm_status lbm_batch_shape_info(int shape, int* tile_w, int* tile_h, int* threads,
                                int* pipelined) {
  if (shape < 0 || shape >= kNumShapes) return fail(LBM_ERR_ARG, "lbm_batch_shape_info: shape %d", shape);
  const bool tma = shape == kTmaShape;
  if (tile_w) *tile_w = tma ? lbm::kTW : 32;
  if (tile_h) *tile_h = tma ? lbm::kTH : lbm::kBatchShapes[shape].by * lbm::kBatchShapes[shape].r;
  if (threads) *threads = tma ? lbm::kTmaBlock : 32 * lbm::kBatchShapes[shape].by;
  if (pipelined) *pipelined = tma ? 1 : 0;
  return LBM_OK;
}

lbm_status lbm_batch_time_steps(lbm_batch* b, int n, float* ms) {
  if (!b || !ms || n < 1) return fail(LBM_ERR_ARG, "lbm_batch_time_steps: bad arguments");
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  BCK(cudaEventRecord(e0, b->stream));
  lbm_status st = run_batch(b, n, 1);
  BCK(cudaEventRecord(e1, b->stream));
  BCK(cudaEventSynchronize(e1));
  BCK(cudaEventElapsedTime(ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

}  // extern "C"
