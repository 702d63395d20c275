// Per-element statistics and conditional means, FP32 form (kernels in bins_impl.cuh).
#include "bins_impl.cuh"

namespace pdfx {

template <>
void launch_stats_tiles<float>(const StatsArgs<float>& a, int num_sms, cudaStream_t s_small, cudaStream_t s_mid,
                               cudaStream_t s_large) {
  launch_stats_tiles_impl<float>(a, num_sms, s_small, s_mid, s_large);
}

}  // namespace pdfx
