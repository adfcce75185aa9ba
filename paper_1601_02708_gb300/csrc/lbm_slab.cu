// lbm_slab.cu -- the halo exchange of a lattice split into row slabs
// (lbm_halo_bytes / lbm_halo_pack / lbm_halo_unpack, declared in
// include/lbm_ade.h).
//
// The lattice Boltzmann step reaches one node away (Eq. "LBE": a node pulls
// from its eight neighbours), so a slab needs one row of each neighbouring
// slab: the overlapping decomposition of Sec. 5 with an overlap of one
// lattice row.  A slab keeps that row in the ghost row beyond its shared
// side.  Per time step two messages cross each shared side:
//   phase 0, after the fused step: the three populations that stream across
//     the cut (S side: directions 4, 7, 8 leave downwards; N side: 2, 5, 6)
//     and, with dissolution, the reaction shares of the boundary row, which
//     the neighbour's dissolution pass gathers;
//   phase 1, after the dissolution pass: the link words of the boundary row,
//     whose own bits (solid, turning fluid) decide the links that cross the
//     cut: the receiver sets them from the ghost row (a link "solid while
//     streaming" while the neighbour is solid, "solid after the flips" while
//     it is solid and not turning fluid) and puts a solid boundary node that a
//     neighbour's flip exposed on its surface list, as the unsplit lattice's
//     flip pass does.
// Every row is moved whole (pitch entries: with periodic x its ghost columns
// come along), so a split lattice computes bit for bit what the unsplit one
// does.
#include <cuda_runtime.h>

#include "lbm_ade.h"
#include "lbm_ctx.h"
#include "lbm_kernels.cuh"

namespace {

using lbm::kXO;
using lbm::kYO;

#define SCK(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return ctx_fail(LBM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
  } while (0)

// Population planes a side's message carries: those leaving the slab across
// it (the neighbour's boundary row pulls them from our boundary row).
__host__ __device__ inline int plane_of(int side, int k) {
  return side == LBM_SIDE_S ? (k == 0 ? 4 : k == 1 ? 7 : 8) : (k == 0 ? 2 : k == 1 ? 5 : 6);
}

template <typename Real>
__global__ void k_pack0(const Real* __restrict__ f, const void* __restrict__ share,
                        int share_bytes, long long plane, long long row_off, int pitch,
                        int side, unsigned char* __restrict__ buf) {
  Real* out = (Real*)buf;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pitch; i += gridDim.x * blockDim.x) {
    for (int k = 0; k < 3; ++k) out[k * pitch + i] = f[plane_of(side, k) * plane + row_off + i];
    if (share_bytes) {
      const unsigned long long* sh = (const unsigned long long*)share;
      ((unsigned long long*)(buf + 3 * (size_t)pitch * sizeof(Real)))[i] = sh[row_off + i];
    }
  }
}

// Unpack a neighbour's phase-0 message into the ghost row beyond `side`: the
// neighbour across S sent its N message (planes 2, 5, 6) and vice versa.
template <typename Real>
__global__ void k_unpack0(Real* __restrict__ f, void* __restrict__ share, int share_bytes,
                          long long plane, long long row_off, int pitch, int side,
                          const unsigned char* __restrict__ buf) {
  const Real* in = (const Real*)buf;
  const int from = side == LBM_SIDE_S ? LBM_SIDE_N : LBM_SIDE_S;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pitch; i += gridDim.x * blockDim.x) {
    for (int k = 0; k < 3; ++k) f[plane_of(from, k) * plane + row_off + i] = in[k * pitch + i];
    if (share_bytes) {
      unsigned long long* sh = (unsigned long long*)share;
      sh[row_off + i] = ((const unsigned long long*)(buf + 3 * (size_t)pitch * sizeof(Real)))[i];
    }
  }
}

__global__ void k_pack1(const uint32_t* __restrict__ link, long long row_off, int pitch,
                        uint32_t* __restrict__ buf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pitch; i += gridDim.x * blockDim.x)
    buf[i] = link[row_off + i] & (lbm::kOwnSolid | lbm::kOwnPending);
}

// Phase 1: the neighbour's boundary-row words into the ghost row, then the
// links of our boundary row that cross into it, and the surface list.
__global__ void k_unpack1(uint32_t* __restrict__ link, long long ghost_off, long long row_off,
                          int nx, int pitch, int per_x, int side,
                          const uint32_t* __restrict__ buf, lbm::DissolveArgs d, int dissolution) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pitch; i += gridDim.x * blockDim.x)
    link[ghost_off + i] = buf[i];
  __syncthreads();  // one block: the ghost row is complete before it is read
  const int cy = side == LBM_SIDE_S ? 1 : -1;  // directions whose source is in the ghost row
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    const long long z = row_off + x + kXO;
    uint32_t w = link[z];
    bool exposed = false;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      if (lbm::cy_of(i) != cy) continue;
      int sx = x - lbm::cx_of(i);
      if (sx < 0 || sx >= nx) {
        if (!per_x) continue;  // outside the lattice: the link stays "outside"
        sx = sx < 0 ? sx + nx : sx - nx;
      }
      const uint32_t g = buf[sx + kXO];
      const bool solid = (g & lbm::kOwnSolid) != 0;
      const bool post = solid && !(g & lbm::kOwnPending);
      const uint32_t b0 = lbm::up_bit(lbm::kUpSolidShift, i), b1 = lbm::up_bit(lbm::kUpPostShift, i);
      w = (w & ~(b0 | b1)) | (solid ? b0 : 0u) | (post ? b1 : 0u);
      exposed |= !post;
    }
    if (dissolution && (w & lbm::kOwnSolid) && !(w & lbm::kListed) && exposed) {
      w |= lbm::kListed;
      const int slot = atomicAdd(d.scount, 1);
      d.slist[slot] = (int)z;
      d.smin[slot] = d.mineral[z];
    }
    link[z] = w;
  }
}

lbm_status check_side(const lbm_ctx* c, int side, int phase, const void* buf, const char* who) {
  if (side != LBM_SIDE_S && side != LBM_SIDE_N)
    return ctx_fail(LBM_ERR_ARG, "%s: side must be LBM_SIDE_S or LBM_SIDE_N", who);
  if (c->p.edge[side] != LBM_EDGE_EXCHANGE)
    return ctx_fail(LBM_ERR_ARG, "%s: side %d is not shared with a neighbouring slab", who, side);
  if (phase != 0 && phase != 1) return ctx_fail(LBM_ERR_ARG, "%s: phase must be 0 or 1", who);
  if (!buf || !ctx_on_device(buf))
    return ctx_fail(LBM_ERR_ARG, "%s: the message buffer must be device memory", who);
  return LBM_OK;
}

// Padded offsets of the boundary row next to `side` and of the ghost row beyond it.
long long boundary_row(const lbm_ctx* c, int side) {
  return (long long)(side == LBM_SIDE_S ? kYO : kYO + c->p.ny - 1) * c->pitch;
}
long long ghost_row(const lbm_ctx* c, int side) {
  return (long long)(side == LBM_SIDE_S ? 0 : kYO + c->p.ny) * c->pitch;
}

}  // namespace

extern "C" {

lbm_status lbm_halo_bytes(lbm_ctx* c, int phase, size_t* bytes) {
  const lbm_status chk = ctx_check(c);
  if (chk != LBM_OK) return chk;
  if (!bytes || (phase != 0 && phase != 1)) return ctx_fail(LBM_ERR_ARG, "lbm_halo_bytes: bad arguments");
  const size_t P = (size_t)c->pitch;
  *bytes = phase == 0 ? 3 * P * c->esize + (c->p.dissolution ? P * 8 : 0) : P * 4;
  return LBM_OK;
}

lbm_status lbm_halo_pack(lbm_ctx* c, int side, int phase, void* buf) {
  lbm_status st = ctx_check(c);
  if (st == LBM_OK) st = check_side(c, side, phase, buf, "lbm_halo_pack");
  if (st != LBM_OK) return st;
  const int grid = (c->pitch + 255) / 256;
  const long long row = boundary_row(c, side);
  if (phase == 0) {
    const int sb = c->p.dissolution ? 8 : 0;
    if (c->esize == 8)
      k_pack0<double><<<grid, 256, 0, c->stream>>>((const double*)c->f[c->cur], c->ureact, sb,
                                                   c->plane, row, c->pitch, side,
                                                   (unsigned char*)buf);
    else
      k_pack0<float><<<grid, 256, 0, c->stream>>>((const float*)c->f[c->cur], c->ureact, sb,
                                                  c->plane, row, c->pitch, side,
                                                  (unsigned char*)buf);
  } else {
    k_pack1<<<grid, 256, 0, c->stream>>>(c->link, row, c->pitch, (uint32_t*)buf);
  }
  SCK(cudaGetLastError());
  return LBM_OK;
}

lbm_status lbm_halo_unpack(lbm_ctx* c, int side, int phase, const void* buf) {
  lbm_status st = ctx_check(c);
  if (st == LBM_OK) st = check_side(c, side, phase, buf, "lbm_halo_unpack");
  if (st != LBM_OK) return st;
  if (phase == 0) {
    const int grid = (c->pitch + 255) / 256;
    const int sb = c->p.dissolution ? 8 : 0;
    if (c->esize == 8)
      k_unpack0<double><<<grid, 256, 0, c->stream>>>((double*)c->f[c->cur], c->ureact, sb,
                                                     c->plane, ghost_row(c, side), c->pitch,
                                                     side, (const unsigned char*)buf);
    else
      k_unpack0<float><<<grid, 256, 0, c->stream>>>((float*)c->f[c->cur], c->ureact, sb,
                                                    c->plane, ghost_row(c, side), c->pitch,
                                                    side, (const unsigned char*)buf);
  } else {
    k_unpack1<<<1, 1024, 0, c->stream>>>(c->link, ghost_row(c, side), boundary_row(c, side),
                                         c->p.nx, c->pitch, c->p.edge[0] == LBM_EDGE_PERIODIC,
                                         side, (const uint32_t*)buf, dissolve_args(c),
                                         c->p.dissolution);
  }
  SCK(cudaGetLastError());
  return LBM_OK;
}

}  // extern "C"
