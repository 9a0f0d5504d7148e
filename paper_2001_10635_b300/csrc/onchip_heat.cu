// onchip_heat.cu -- on-chip kernels instantiated for REACH_HEAT3D.
#include "onchip_kernels.cuh"

namespace reach {

template int onchip_single_k<REACH_HEAT3D>(const OnItem &, int, cudaStream_t);
template int onchip_cluster_k<REACH_HEAT3D>(const OnItem &, cudaStream_t);
template int onchip_batch_k<REACH_HEAT3D>(int, int, const void *, const void *, const void *, const void *, int,
                                     int *, uint64_t *, int, size_t, cudaStream_t);

template int queue_launch_k<REACH_HEAT3D>(const QueueArgs &, int, size_t, cudaStream_t);
}  // namespace reach
