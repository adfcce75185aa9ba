// lbm_batch_plain_impl.cuh -- definition of launch_batch_plain, included by
// the translation units that instantiate it.
#pragma once
#include "lbm_batch_plain.cuh"

namespace lbm {

template <typename Real, bool kFinal, int kWalls>
void launch_batch_plain(int shape, int grid, cudaStream_t stream, const ArgSlot<Real>* a,
                        const int4* tl, int nt, double frac) {
  const BatchShape sh = kBatchShapes[shape];
  const dim3 block(32, sh.by);
  if (sh.by == 8 && sh.r == 1)
    lbm_step_batch<Real, kFinal, 8, 1, kWalls><<<grid, block, 0, stream>>>(a, tl, nt, frac);
  else if (sh.by == 16 && sh.r == 1)
    lbm_step_batch<Real, kFinal, 16, 1, kWalls><<<grid, block, 0, stream>>>(a, tl, nt, frac);
  else if (sh.by == 8 && sh.r == 2)
    lbm_step_batch<Real, kFinal, 8, 2, kWalls><<<grid, block, 0, stream>>>(a, tl, nt, frac);
  else if (sh.by == 4 && sh.r == 2)
    lbm_step_batch<Real, kFinal, 4, 2, kWalls><<<grid, block, 0, stream>>>(a, tl, nt, frac);
  else if (sh.by == 8 && sh.r == 4)
    lbm_step_batch<Real, kFinal, 8, 4, kWalls><<<grid, block, 0, stream>>>(a, tl, nt, frac);
  else
    lbm_step_batch<Real, kFinal, 4, 4, kWalls><<<grid, block, 0, stream>>>(a, tl, nt, frac);
}

}  // namespace lbm
