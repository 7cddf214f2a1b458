// Tensor-core (tcgen05) forms of the travel-time MLP: not built yet.
#include "kernels.h"
#include "spider.h"

namespace spider {

bool mlp_tc_supported(int, int) { return false; }

cudaError_t mlp_tc_prepare(const float* const*, int, int, void** image, float** scales, cudaStream_t) {
  *image = nullptr;
  *scales = nullptr;
  return cudaErrorNotSupported;
}

cudaError_t launch_mlp_tc(const NetView&, const PairSource&, TTOut, int, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace spider
