// Internal declarations shared by the translation units of libsbim.
//
// Spectral layout used by every kernel (Section 2.3, spectral evaluation of s_i):
//   * Half spectra from the R2C transform: [3][n3][n1/2+1] complex, bin b =
//     r3 * (n1/2+1) + j1.
//   * "Orbits" (records): the library groups the Fourier bins by |k| into
//     records of four "members" in two halves of two; the members of a half
//     share |k|, hence the kernel arguments T = m |k| c_s dt and the convolution
//     weights.  Per-record |k| data (dT, ustep, muq, lmax) is stored per half,
//     [record][2].  Whole-record plans (StepArgs::halves = 0, square grids) give
//     both halves one |k|; half-record plans pair halves of two classes where
//     classes of two bins would otherwise leave half of a record empty
//     (rectangular planes).  A member is one bin seen
//     along one in-plane direction e = k/|k|; a bin on a Nyquist line appears as
//     two (or, at the corner, four) members whose directions differ in the sign
//     of the aliased component, each weighted 1/2 (1/4), which keeps only the
//     part of the operator even in that component.  Orbits are sorted by |k|.
//   * History ring buffer: [n_cut][3][n_orb_pad][4] complex (slot, component
//     xi / 2 / perp, orbit, member); slot = step mod n_cut.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sbim.h"

namespace sbim {

constexpr int kMembers = 4;      // members per orbit
constexpr int kFields = 10;      // real accumulators per member: 5 complex sums
constexpr int kOrbitTile = 128;  // orbits per CTA of the assembly and of the default convolution
                                 // (the TMA convolution also runs 64 or 256: "modes per CTA")

// Everything the per-step kernels read; device pointers unless noted.
struct StepArgs {
  // plan (read-only)
  const int* bin;                  // [n_orb_pad*4] bin index, -1 = padding
  const void* dir;                 // [n_orb_pad*4] (e1, e3) of the member (float2 / double2)
  const float* wout;               // [n_orb_pad*4] output weight of the member
  const void* dT;                  // [n_orb_pad] |k| c_s dt (float or double)
  const unsigned long long* ustep; // [n_orb_pad] dT / h in 32.32 fixed point
  const void* muq;                 // [n_orb_pad] mu |k| (float or double)
  const void* table;               // [table_n] (H11, H22, H33, H12) at T = (j-1) h
  const int* lmax;                 // [n_orb_pad] lags kept per orbit (truncation window), or NULL
  const int* tile_lmax;            // [n_orb_pad/128] max of lmax over each tile, or NULL
  const void* wts;                 // FP64 path: [n_cut][n_orb_pad] precomputed weights
                                   // (11, 22, 33, 12) as 4 doubles, or NULL
  // state
  void* hist;                      // ring buffer (layout per precision)
  long long* step;                 // device step counter n
  int* err;                        // device error word (bounded waits that gave up)
  void* part;                      // [nchunks][40][n_orb_pad] partial sums
  const void* uhat;                // [3][nbins] forward spectra
  void* fhat;                      // [3][nbins] output spectra (scaled 1/(n1 n3))
  // sizes (host values)
  int n_orb_pad;
  int halves;                      // 1: a record's two halves may hold different |k|
  int nbins;
  int n_cut;
  int lc;                          // lags per chunk
  int nchunks;
  int side;
  double eta;
  double inv_n;                    // 1 / (n1 n3)
  long long slot_stride;           // elements of one history plane (BF16X2 lo offset)
};

// Persistent launch over the (update, tile, chunk) items of a batch.
struct BatchLaunch {
  const StepArgs* args;     // [nb] device copies of the members' StepArgs
  const int* item_prefix;   // [nb + 1] first item of each member (tiles x chunks each)
  const int* tile_prefix;   // [nb + 1] first tile of each member (assembly grid)
  int nb;
  int* counter;             // work counter, zero before each launch
  int ctas;                 // persistent CTAs
  int items;                // > 0: one CTA per item (this many), no persistent CTAs
};

cudaError_t launch_conv(const StepArgs& a, int precision, int kahan, cudaStream_t s);
cudaError_t launch_assemble_batch(const BatchLaunch& b, int total_tiles, int precision, int kahan,
                                  cudaStream_t s);
// History convolution with TMA bulk-copy staging of the history slots in shared
// memory (same inputs and outputs as launch_conv).  ctas_per_sm reports the
// residency the launch is sized for.
// shape 1..3 selects the pipeline (stages, lags per stage, CTAs per SM); tile the
// orbits per CTA (64, 128 or 256; n_orb_pad must be a multiple of it).
// halves: the records may hold two |k| (one per half; see StepArgs::halves).
cudaError_t launch_conv_tma(const StepArgs& a, int precision, int kahan, int shape,
                            cudaStream_t s, const BatchLaunch* batch = nullptr,
                            int tile = kOrbitTile, bool halves = false);
int conv_tma_ctas_per_sm(int precision, int kahan, int shape, int tile = kOrbitTile);
// Set the shared-memory attributes of a shape's kernels (done before any launch,
// so that launches can be captured in a CUDA graph).
cudaError_t prepare_conv_tma(int precision, int kahan, int shape, int tile = kOrbitTile,
                             bool halves = false);
// One CTA whose bounded mbarrier wait can never complete (sbim_selftest_wait_timeout).
cudaError_t launch_wait_selftest(int* err, cudaStream_t st);
cudaError_t launch_assemble(const StepArgs& a, int precision, int kahan, cudaStream_t s);
cudaError_t launch_rewind(long long* step, cudaStream_t st);
// FP64 path: out[m][o] = the four convolution weights of orbit o at lag m,
// m < n_cut (the cubic interpolation of the FP64 table the kernels would do).
cudaError_t launch_weights64(const StepArgs& a, void* out, cudaStream_t st);
// *flag = 1 if any of the n values of a or b (b may be NULL) is not finite, else 0.
cudaError_t launch_nonfinite_check(int precision, const void* a, const void* b, long long n,
                                   int* flag, cudaStream_t st);
cudaError_t launch_repeat_lag0(const StepArgs& a, int precision, cudaStream_t st);
cudaError_t launch_epilogue(int precision, const void* s_field, const void* v, void* tau,
                            long long plane, const double coef[3], const double tau_inf[3],
                            long long* step, cudaStream_t st);

cudaError_t launch_adjoint_epilogue(int precision, const void* tau_bar, void* v_bar,
                                    long long plane, const double coef[3], long long* step,
                                    cudaStream_t st);

// FP64 quadrature of the half-space kernels on T_j = j h, j = -1 .. n-2.
// out64 [n][4] doubles; out32 (optional) [n][4] floats.
cudaError_t launch_table_build(double* out64, float* out32, long long n, double h,
                               double eta, const double* gl_x, const double* gl_w,
                               cudaStream_t s);

// Set the calling thread's message returned by sbim_last_error().
void set_last_error(const char* msg);

// Stages of one handle's update, for drivers that batch the convolution of
// several handles (each returns an sbim_status).
StepArgs handle_step_args(sbim_handle h);
int handle_fft_forward(sbim_handle h, const void* u, cudaStream_t st);
int handle_fft_inverse(sbim_handle h, cudaStream_t st);
int handle_epilogue(sbim_handle h, const void* v, void* tau, cudaStream_t st);
void handle_advance(sbim_handle h);
int handle_shape(sbim_handle h, int* precision, int* kahan, int* variant, void** stream);

// Batch over existing handles (not owned); enqueue one step / advance the counters.
int batch_from_handles(sbim_batch* out, const sbim_handle* hs, int n);
int batch_set_conv_config(sbim_batch b, int shape, int lags_per_item);
int batch_set_conv_tile(sbim_batch b, int tile);
// Fork / join of the batch's side streams around per-member stages: after
// batch_fork, work on batch_side(b, i) follows everything enqueued on the
// batch's stream; batch_join makes the batch's stream wait for all of it.
int batch_fork(sbim_batch b);
cudaStream_t batch_side(sbim_batch b, int i);
int batch_join(sbim_batch b);
int batch_enqueue(sbim_batch b, const void* const* u, const void* const* v, void* const* tau);
void batch_advance(sbim_batch b);

}  // namespace sbim
