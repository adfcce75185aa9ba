// lbm_batch_plain_f32_w2.cu -- plain batch step kernels, float lattices,
// wall variant 2 (see lbm_batch_plain.cuh).
#include "lbm_batch_plain_impl.cuh"

namespace lbm {
template void launch_batch_plain<float, true, 2>(int, int, cudaStream_t,
                                                   const ArgSlot<float>*, const int4*, int,
                                                   double);
template void launch_batch_plain<float, false, 2>(int, int, cudaStream_t,
                                                    const ArgSlot<float>*, const int4*, int,
                                                    double);
}  // namespace lbm
