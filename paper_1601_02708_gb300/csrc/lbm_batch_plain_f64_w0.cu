// lbm_batch_plain_f64_w0.cu -- plain batch step kernels, double lattices,
// wall variant 0 (see lbm_batch_plain.cuh).
#include "lbm_batch_plain_impl.cuh"

namespace lbm {
template void launch_batch_plain<double, true, 0>(int, int, cudaStream_t,
                                                   const ArgSlot<double>*, const int4*, int,
                                                   double);
template void launch_batch_plain<double, false, 0>(int, int, cudaStream_t,
                                                    const ArgSlot<double>*, const int4*, int,
                                                    double);
}  // namespace lbm
