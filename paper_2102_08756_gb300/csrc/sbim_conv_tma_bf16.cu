// Instantiations of the TMA-staged history convolution for BF16 hi-only history
// (Section 2.3, the per-mode truncated time convolution).  Shapes: pipeline
// stages x lags per stage x resident CTAs per SM, 12 KB per stage (24 KB for
// shape 3).
#include "sbim_conv_tma.cuh"

namespace sbim {

template <int KAHAN>
static cudaError_t shapes_bf16(const StepArgs& a, int shape, cudaStream_t st) {
  using S = dev::StoreBF16<false>;
  switch (shape) {
    case 1: return tma::launch_shape<S, KAHAN, 8, 2, 2>(a, st);
    case 2: return tma::launch_shape<S, KAHAN, 6, 2, 3>(a, st);
    case 3: return tma::launch_shape<S, KAHAN, 4, 4, 2>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_conv_tma_bf16(const StepArgs& a, int kahan, int shape, cudaStream_t st) {
  return kahan ? shapes_bf16<1>(a, shape, st) : shapes_bf16<0>(a, shape, st);
}

}  // namespace sbim
