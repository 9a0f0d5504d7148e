// onchip_linear.cu -- on-chip kernels instantiated for REACH_LINEAR.
#include "onchip_kernels.cuh"

namespace reach {

template int onchip_single_k<REACH_LINEAR>(const OnItem &, int, cudaStream_t);
// a linear system has n <= 256, so it always fits one block: no cluster kernel
template <>
int onchip_cluster_k<REACH_LINEAR>(const OnItem &, cudaStream_t) {
    return REACH_EINVAL;
}
template int onchip_batch_k<REACH_LINEAR>(int, int, const void *, const void *, const void *, const void *, int,
                                     int *, uint64_t *, int, size_t, cudaStream_t);

template int queue_launch_k<REACH_LINEAR>(const QueueArgs &, int, size_t, cudaStream_t);
}  // namespace reach
