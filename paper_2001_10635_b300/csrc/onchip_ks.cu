// onchip_ks.cu -- on-chip kernels instantiated for REACH_KS.
#include "onchip_kernels.cuh"

namespace reach {

template int onchip_single_k<REACH_KS>(const OnItem &, int, cudaStream_t);
template int onchip_cluster_k<REACH_KS>(const OnItem &, cudaStream_t);
template int onchip_batch_k<REACH_KS>(int, int, const void *, const void *, const void *, const void *, int,
                                     int *, uint64_t *, int, size_t, cudaStream_t);

template int queue_launch_k<REACH_KS>(const QueueArgs &, int, size_t, cudaStream_t);
}  // namespace reach
