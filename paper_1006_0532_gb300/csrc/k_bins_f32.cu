// Per-element statistics and conditional means, FP32 form (kernels in bins_impl.cuh).
#include "bins_impl.cuh"

namespace pdfx {

template <>
void launch_stats_tiles<float>(const StatsArgs<float>& a, int num_sms, cudaStream_t s,
                               const SideStreams* side) {
  launch_stats_tiles_impl<float>(a, num_sms, s, side);
}

}  // namespace pdfx
