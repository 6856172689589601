// Instantiations of the TMA-staged history convolution for FP64 history
// (Section 2.3, the per-mode truncated time convolution).  Shapes: pipeline
// stages x lags per stage x resident CTAs per SM, 28 KB per stage at 128 orbits
// per CTA (history 24 KB, precomputed weights 4 KB).
#include "sbim_conv_tma.cuh"

namespace sbim {

cudaError_t launch_conv_tma_f64(const StepArgs& a, int /*kahan*/, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep, int tile, bool halves) {
  using S = dev::StoreF64;
  switch (shape) {
    case 1: return tma::launch_tiles<S, 0, 3, 1, 2>(tile, halves, a, st, batch, prep);
    case 2: return tma::launch_tiles<S, 0, 4, 1, 2>(tile, halves, a, st, batch, prep);
    case 3: return tma::launch_tiles<S, 0, 2, 2, 2>(tile, halves, a, st, batch, prep);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sbim
