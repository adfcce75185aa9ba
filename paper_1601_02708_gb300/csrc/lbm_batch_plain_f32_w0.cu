// lbm_batch_plain_f32_w0.cu -- plain batch step kernels, float lattices,
// wall variant 0 (see lbm_batch_plain.cuh).
#include "lbm_batch_plain_impl.cuh"

namespace lbm {
template void launch_batch_plain<float, true, 0>(int, int, cudaStream_t,
                                                   const ArgSlot<float>*, const int4*, int,
                                                   double);
template void launch_batch_plain<float, false, 0>(int, int, cudaStream_t,
                                                    const ArgSlot<float>*, const int4*, int,
                                                    double);
}  // namespace lbm
