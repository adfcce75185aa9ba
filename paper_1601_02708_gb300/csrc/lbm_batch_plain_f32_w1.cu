// lbm_batch_plain_f32_w1.cu -- plain batch step kernels, float lattices,
// wall variant 1 (see lbm_batch_plain.cuh).
#include "lbm_batch_plain_impl.cuh"

namespace lbm {
template void launch_batch_plain<float, true, 1>(int, int, cudaStream_t,
                                                   const ArgSlot<float>*, const int4*, int,
                                                   double);
template void launch_batch_plain<float, false, 1>(int, int, cudaStream_t,
                                                    const ArgSlot<float>*, const int4*, int,
                                                    double);
}  // namespace lbm
