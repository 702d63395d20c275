// Per-element statistics and conditional means, FP32 form (kernels in bins_impl.cuh).
#include "bins_impl.cuh"

namespace pdfx {

template <>
void launch_stats_warp<float>(const StatsArgs<float>& a, cudaStream_t s) {
  launch_stats_warp_impl<float>(a, s);
}

}  // namespace pdfx
