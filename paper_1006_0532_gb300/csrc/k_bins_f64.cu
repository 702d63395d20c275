// Per-element statistics and conditional means, FP64 form (kernels in bins_impl.cuh).
#include "bins_impl.cuh"

namespace pdfx {

template <>
void launch_stats_warp<double>(const StatsArgs<double>& a, cudaStream_t s) {
  launch_stats_warp_impl<double>(a, s);
}

}  // namespace pdfx
