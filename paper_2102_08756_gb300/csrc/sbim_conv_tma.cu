// Dispatch of the TMA-staged history convolution by history precision and
// pipeline shape (the instantiations live in one translation unit per
// precision so that they compile in parallel).
#include "../../include/sbim.h"
#include "sbim_internal.cuh"

namespace sbim {

cudaError_t launch_conv_tma_f32(const StepArgs& a, int kahan, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep);
cudaError_t launch_conv_tma_bf16x2(const StepArgs& a, int kahan, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep);
cudaError_t launch_conv_tma_bf16(const StepArgs& a, int kahan, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep);
cudaError_t launch_conv_tma_f64(const StepArgs& a, int kahan, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep);

static cudaError_t dispatch(const StepArgs& a, int precision, int kahan, int shape,
                            cudaStream_t st, const BatchLaunch* batch, bool prep) {
  switch (precision) {
    case SBIM_FP64: return launch_conv_tma_f64(a, 0, shape, st, batch, prep);
    case SBIM_FP32: return launch_conv_tma_f32(a, kahan, shape, st, batch, prep);
    case SBIM_BF16X2: return launch_conv_tma_bf16x2(a, kahan, shape, st, batch, prep);
    case SBIM_BF16: return launch_conv_tma_bf16(a, kahan, shape, st, batch, prep);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_conv_tma(const StepArgs& a, int precision, int kahan, int shape,
                            cudaStream_t st, const BatchLaunch* batch) {
  return dispatch(a, precision, kahan, shape, st, batch, false);
}

cudaError_t prepare_conv_tma(int precision, int kahan, int shape) {
  const StepArgs none{};
  return dispatch(none, precision, kahan, shape, nullptr, nullptr, true);
}

int conv_tma_ctas_per_sm(int precision, int shape) {
  if (precision == SBIM_FP64) return 2;
  return shape == 2 ? 3 : 2;
}

}  // namespace sbim
