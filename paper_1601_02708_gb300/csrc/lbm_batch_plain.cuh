// lbm_batch_plain.cuh -- the plain (one thread per node) step kernel of a
// batch of lattices, shared by lbm_batch.cu and the translation units that
// instantiate it (lbm_batch_plain_f32.cu, lbm_batch_plain_f64.cu; split so
// that the many shape variants compile in parallel).
#pragma once
#include <cuda_runtime.h>

#include "lbm_kernels.cuh"

namespace lbm {

constexpr int kBatchRateBit = 1 << 29;  // tile descriptor .w: the member has a rate field
constexpr int kBatchTileMask = kBatchRateBit - 1;

// Step arguments of one member, padded to whole 16-byte units so that the
// pipelined kernel can fetch them with one bulk copy.
template <typename Real>
struct alignas(16) ArgSlot {
  StepArgs<Real> a;
};

// Tile shapes of the plain kernel: 32 columns x kBY rows of threads, each
// thread kR rows apart.
struct BatchShape {
  int by, r;
};
constexpr BatchShape kBatchShapes[] = {{8, 1}, {16, 1}, {8, 2}, {4, 2}, {8, 4}, {4, 4}};
constexpr int kBatchPlainShapes = 6;

// One tile list over every member: tile (member, x0, y0, index | rate bit).
// Each block walks tiles t, t + grid, ...; the nodes of a tile step in place
// (boundary solves inline, in FP64).
template <typename Real, bool kFinal, int kBY, int kR, int kWalls>
__global__ void __launch_bounds__(32 * kBY)
    lbm_step_batch(const ArgSlot<Real>* __restrict__ args, const int4* __restrict__ tiles,
                   int ntiles, double frac) {
  static_assert(sizeof(StepArgs<Real>) % sizeof(int) == 0 &&
                    sizeof(StepArgs<Real>) / sizeof(int) <= 32 * kBY,
                "one thread per word of the arguments");
  __shared__ StepArgs<Real> sa;
  __shared__ double red[kBY];
  const int tid = threadIdx.y * 32 + threadIdx.x;
  int member = -1;  // whose arguments sit in sa (consecutive tiles of a block
                    // mostly belong to the same member: reload only on change)
  int4 next = blockIdx.x < ntiles ? tiles[blockIdx.x] : make_int4(0, 0, 0, 0);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int4 td = next;
    if (t + (int)gridDim.x < ntiles) next = tiles[t + gridDim.x];  // prefetch
    if (td.x != member) {
      __syncthreads();  // the previous tile is done with sa
      if (tid < (int)(sizeof(sa) / sizeof(int)))
        reinterpret_cast<int*>(&sa)[tid] = reinterpret_cast<const int*>(&args[td.x].a)[tid];
      __syncthreads();
      member = td.x;
    }
    const StepArgs<Real>& a = sa;
    double my_u = 0.0;
#pragma unroll
    for (int rr = 0; rr < kR; ++rr) {
      const int x = td.y + threadIdx.x, y = td.z + threadIdx.y + rr * kBY;
      if (x < a.nx && y < a.ny) {
        const long long n = (long long)(y + kYO) * a.pitch + (x + kXO);
        GlobalSrc<Real> src{a, n};
        if (group_is_interior(td.y, y, a.nx, a.ny))
          my_u += step_node<Real, kFinal, false, false, kWalls>(a, src, x, y, n, frac);
        else
          my_u += step_node<Real, kFinal, true, true, kWalls>(a, src, x, y, n, frac);
      }
    }
    if (kFinal) {
      const double s = block_sum(my_u, red);
      if (tid == 0) a.partial[td.w & kBatchTileMask] = s;
    }
  }
}

// Launch of the plain kernel in shape `shape` (0 .. kBatchPlainShapes - 1);
// instantiated for every (Real, kFinal, kWalls) the batch uses.
template <typename Real, bool kFinal, int kWalls>
void launch_batch_plain(int shape, int grid, cudaStream_t stream, const ArgSlot<Real>* args,
                        const int4* tiles, int ntiles, double frac);

}  // namespace lbm
