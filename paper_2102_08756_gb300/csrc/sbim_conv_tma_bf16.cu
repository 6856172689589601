// Instantiations of the TMA-staged history convolution for BF16 hi-only history
// (Section 2.3, the per-mode truncated time convolution).  Shapes: pipeline
// stages x lags per stage x resident CTAs per SM, 6 KB of history per lag.
//
// The uncompensated kernel is latency-bound on the kernel-table loads at the
// occupancy of 2-lag stages (one thread per record, 12 B per mode and lag, so
// half the FP32 kernel's bytes per instruction): with 1-lag stages the
// prefetched table nodes of the next lag take 16 registers instead of 32, and
// the kernel fits 96 registers per thread, 5 CTAs per SM.  On GB300 at 1024^2 x 4096 the convolution took 4.08 ms with
// 6 x 1 x 5 against 4.46 ms with 6 x 2 x 3 and 4.36 ms with 6 x 1 x 4; 6 x 1 x 6
// spills.  The compensated kernel keeps 2-lag stages (its 80 running sums and
// compensations leave no room for 5 CTAs per SM).
#include "sbim_conv_tma.cuh"

namespace sbim {

template <int KAHAN>
static cudaError_t shapes_bf16(const StepArgs& a, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep, int tile, bool halves) {
  using S = dev::StoreBF16<false>;
  if constexpr (KAHAN) {
    switch (shape) {
      case 1: return tma::launch_tiles<S, KAHAN, 8, 2, 2>(tile, halves, a, st, batch, prep);
      case 2: return tma::launch_tiles<S, KAHAN, 6, 2, 3>(tile, halves, a, st, batch, prep);
      case 3: return tma::launch_tiles<S, KAHAN, 4, 4, 2>(tile, halves, a, st, batch, prep);
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (shape) {
      case 1: return tma::launch_tiles<S, KAHAN, 6, 1, 4>(tile, halves, a, st, batch, prep);
      case 2: return tma::launch_tiles<S, KAHAN, 6, 1, 5>(tile, halves, a, st, batch, prep);
      case 3: return tma::launch_tiles<S, KAHAN, 6, 2, 3>(tile, halves, a, st, batch, prep);
      default: return cudaErrorInvalidValue;
    }
  }
}

cudaError_t launch_conv_tma_bf16(const StepArgs& a, int kahan, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep, int tile, bool halves) {
  return kahan ? shapes_bf16<1>(a, shape, st, batch, prep, tile, halves)
               : shapes_bf16<0>(a, shape, st, batch, prep, tile, halves);
}

}  // namespace sbim
