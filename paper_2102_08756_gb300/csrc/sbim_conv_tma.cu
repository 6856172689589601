// Dispatch of the TMA-staged history convolution by history precision and
// pipeline shape (the instantiations live in one translation unit per
// precision so that they compile in parallel).
#include "../../include/sbim.h"
#include "sbim_conv_tma.cuh"
#include "sbim_internal.cuh"

namespace sbim {

namespace {
// The failure path of the bounded waits, exercised on purpose: the CTA waits on
// an mbarrier that expects one arrival and gets none (no copy is ever issued to
// it), with the same bounded wait the convolution uses.  The wait gives up after
// its wall-time limit and the CTA records the failure in the error word.
__global__ void wait_selftest_kernel(int* err) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    tma::mbar_init(tma::smem_addr(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool landed = tma::mbar_wait(tma::smem_addr(&bar), 0u, err);
  if (!__syncthreads_and(landed) && threadIdx.x == 0) atomicExch(err, 1);
}
}  // namespace

cudaError_t launch_wait_selftest(int* err, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(err);
  return cudaGetLastError();
}

cudaError_t launch_conv_tma_f32(const StepArgs& a, int kahan, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep, int tile, bool halves);
cudaError_t launch_conv_tma_bf16x2(const StepArgs& a, int kahan, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep, int tile, bool halves);
cudaError_t launch_conv_tma_bf16(const StepArgs& a, int kahan, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep, int tile, bool halves);
cudaError_t launch_conv_tma_f64(const StepArgs& a, int kahan, int shape, cudaStream_t st,
                                 const BatchLaunch* batch, bool prep, int tile, bool halves);

static cudaError_t dispatch(const StepArgs& a, int precision, int kahan, int shape,
                            cudaStream_t st, const BatchLaunch* batch, bool prep, int tile,
                            bool halves) {
  switch (precision) {
    case SBIM_FP64: return launch_conv_tma_f64(a, 0, shape, st, batch, prep, tile, halves);
    case SBIM_FP32: return launch_conv_tma_f32(a, kahan, shape, st, batch, prep, tile, halves);
    case SBIM_BF16X2:
      return launch_conv_tma_bf16x2(a, kahan, shape, st, batch, prep, tile, halves);
    case SBIM_BF16: return launch_conv_tma_bf16(a, kahan, shape, st, batch, prep, tile, halves);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_conv_tma(const StepArgs& a, int precision, int kahan, int shape,
                            cudaStream_t st, const BatchLaunch* batch, int tile, bool halves) {
  return dispatch(a, precision, kahan, shape, st, batch, false, tile, halves);
}

cudaError_t prepare_conv_tma(int precision, int kahan, int shape, int tile, bool halves) {
  const StepArgs none{};
  return dispatch(none, precision, kahan, shape, nullptr, nullptr, true, tile, halves);
}

int conv_tma_ctas_per_sm(int precision, int kahan, int shape, int tile) {
  int minb = shape == 2 ? 3 : 2;   // FP32, BF16 hi/lo, compensated BF16 hi-only
  if (precision == SBIM_FP64) minb = 2;
  if (precision == SBIM_BF16 && !kahan) minb = shape == 1 ? 4 : (shape == 2 ? 5 : 3);
  return tma::minb_for_tile(minb, tile);
}

}  // namespace sbim
