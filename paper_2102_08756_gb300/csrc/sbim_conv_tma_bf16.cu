// Instantiations of the TMA-staged history convolution for BF16 hi-only history
// (Section 2.3, the per-mode truncated time convolution).  Shapes: pipeline
// stages x lags per stage x resident CTAs per SM, 12 KB per stage (24 KB for
// shape 3).
#include "sbim_conv_tma.cuh"

namespace sbim {

template <int KAHAN>
static cudaError_t shapes_bf16(const StepArgs& a, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep, int tile, bool halves) {
  using S = dev::StoreBF16<false>;
  switch (shape) {
    case 1: return tma::launch_tiles<S, KAHAN, 8, 2, 2>(tile, halves, a, st, batch, prep);
    case 2: return tma::launch_tiles<S, KAHAN, 6, 2, 3>(tile, halves, a, st, batch, prep);
    case 3: return tma::launch_tiles<S, KAHAN, 4, 4, 2>(tile, halves, a, st, batch, prep);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_conv_tma_bf16(const StepArgs& a, int kahan, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep, int tile, bool halves) {
  return kahan ? shapes_bf16<1>(a, shape, st, batch, prep, tile, halves)
               : shapes_bf16<0>(a, shape, st, batch, prep, tile, halves);
}

}  // namespace sbim
