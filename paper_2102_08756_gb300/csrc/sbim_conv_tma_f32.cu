// Instantiations of the TMA-staged history convolution for FP32 history
// (Section 2.3, the per-mode truncated time convolution).  Shapes: pipeline
// stages x lags per stage x resident CTAs per SM, 24 KB per stage (48 KB for
// shape 3).
#include "sbim_conv_tma.cuh"

namespace sbim {

template <int KAHAN>
static cudaError_t shapes_f32(const StepArgs& a, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep, int tile, bool halves) {
  using S = dev::StoreF32;
  switch (shape) {
    case 1: return tma::launch_tiles<S, KAHAN, 4, 2, 2>(tile, halves, a, st, batch, prep);
    case 2: return tma::launch_tiles<S, KAHAN, 3, 2, 3>(tile, halves, a, st, batch, prep);
    case 3: return tma::launch_tiles<S, KAHAN, 2, 4, 2>(tile, halves, a, st, batch, prep);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_conv_tma_f32(const StepArgs& a, int kahan, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep, int tile, bool halves) {
  return kahan ? shapes_f32<1>(a, shape, st, batch, prep, tile, halves)
               : shapes_f32<0>(a, shape, st, batch, prep, tile, halves);
}

}  // namespace sbim
