/*
 * sbim.h -- C ABI of the GB300 spectral-boundary-integral (SBIM) traction update.
 *
 * The operation (Albertini, Elbanna & Kammer, Section 2.3, Eq. (SBI)) maps the
 * displacement history and current velocity of the boundary plane of one elastic
 * half-space to the traction on that plane:
 *
 *     tau_i = tau_i^inf - eta_ij (mu / c_s) du_j/dt + s_i ,
 *
 * with eta_ij = diag(1, c_p/c_s, 1), mu = rho c_s^2, and s_i the non-local term
 * evaluated spectrally (Section 2.3, "spectral approach"): a 2D Fourier transform
 * of the three displacement components over the periodic boundary plane, a
 * truncated time convolution of every Fourier mode's history with the half-space
 * kernels H11, H22, H33, H12(|k| c_s t), and an inverse transform.  One call of
 * sbim_step is step 3 of the hybrid time step of Section 2.4 for one half-space
 * (S+ or S-).
 *
 * Conventions shared by every entry point
 *   - Every function returns an sbim_status; 0 is success.  On failure the
 *     calling thread's message is available from sbim_last_error().  Output
 *     arguments are written only on success.
 *   - Fields are row-major [3][n3][n1] arrays (component, x3, x1 with x1
 *     fastest), in SI units (m, m/s, Pa).  The component index is the Cartesian
 *     direction 1, 2, 3 of the paper, x2 being the normal of the boundary.
 *   - Element type: double for SBIM_FP64 handles, float for every other precision.
 *   - A handle owns all its device memory (history ring buffer, kernel tables,
 *     FFT plans, work buffers), is bound to one CUDA stream, and must not be used
 *     from two threads at once.
 */
#ifndef SBIM_H
#define SBIM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbim_ctx* sbim_handle;

typedef enum {
    SBIM_OK = 0,
    SBIM_ERR_ARG = -1,       /* invalid argument (value, pointer, alignment, size) */
    SBIM_ERR_OOM = -2,       /* device or host allocation failed / would not fit */
    SBIM_ERR_CUDA = -3,      /* a CUDA runtime call or kernel launch failed */
    SBIM_ERR_FFT = -4,       /* a cuFFT call failed */
    SBIM_ERR_TIMEOUT = -5,   /* reserved: a bounded device wait gave up */
    SBIM_ERR_NONFINITE = -6, /* non-finite input detected (opt-in, sbim_set_check_finite) */
    SBIM_ERR_STATE = -7      /* call not valid in the handle's current state */
} sbim_status;

typedef enum {
    SBIM_FP64 = 0,   /* history and arithmetic in double; I/O double */
    SBIM_FP32 = 1,   /* history float, accumulation float (optionally compensated) */
    SBIM_BF16X2 = 2, /* history as bf16 hi + bf16 lo per real, float accumulation */
    SBIM_BF16 = 3    /* history as bf16 hi only, float accumulation */
} sbim_precision;

/*
 * sbim_create -- build a handle for one half-space.
 *
 * Section 2.3 (problem statement of Eq. (SBI)) and Section 2.4 (the boundary S+
 * or S- of the finite-element strip).
 *   n1, n3     grid points along x1 and x3 (even, >= 2); periodic boundary plane
 *   L1, L3     periodic lengths (m), grid spacing L1/n1, L3/n3
 *   cs, cp     shear and dilatational wave speeds (m/s), cp > cs > 0
 *   rho        density (kg/m^3) > 0
 *   dt         time step (s) > 0, the spacing of consecutive sbim_step calls
 *   n_cut      history cutoff in steps (>= 1): the convolution uses the last
 *              min(n+1, n_cut) displacement fields, the current one included
 *   side       +1: half-space x2 > boundary (material above the plane, S+);
 *              -1: half-space x2 < boundary (S-)
 *   precision  an sbim_precision value
 *   kahan      non-zero: compensated (Kahan) float accumulation over the lags
 *              (ignored for SBIM_FP64)
 *   stream     cudaStream_t every call of this handle is ordered on; NULL = the
 *              legacy default stream
 * The kernel tables are built on the device in double precision.  Returns
 * SBIM_ERR_OOM if the history ring buffer (n_cut x 3 x modes, complex) does not
 * fit in free device memory.  An SBIM_FP64 handle also keeps its convolution
 * weights, computed once (n_cut x n_slots x 8 bytes; 17.3 GB at 1024^2 x 4096),
 * when they fit with 512 MB to spare; otherwise it interpolates them from the
 * table every step, with the same result to rounding.  *out is written on
 * success only.
 */
int sbim_create(sbim_handle* out, int n1, int n3, double L1, double L3,
                double cs, double cp, double rho, double dt, int n_cut,
                int side, int precision, int kahan, void* stream);

/*
 * sbim_step -- one traction evaluation, Eq. (SBI), at the next time step n.
 *
 *   u    device pointer, displacement of the boundary at step n      [3][n3][n1]
 *   v    device pointer, velocity at step n (Section 2.4: the FE predicted
 *        velocity), used only by the radiation-damping term          [3][n3][n1]
 *   tau  device pointer, output traction sigma_2i on the boundary    [3][n3][n1]
 * u is appended to the handle's history (step 0 is the first call after
 * sbim_create or sbim_reset; earlier displacements are zero).  The call is
 * asynchronous and ordered on the handle's stream; the caller keeps u, v, tau
 * alive until the stream has passed them.  u, v and tau must not overlap.
 */
int sbim_step(sbim_handle h, const void* u, const void* v, void* tau);

/*
 * sbim_step_host -- as sbim_step, with u, v, tau in HOST memory (pageable or
 * pinned).  Copies the inputs to device work buffers, runs the step, copies
 * tau back and waits for the stream; the device error word comes back with tau
 * and is checked as by sbim_check_device (SBIM_ERR_TIMEOUT if a bounded wait
 * gave up).  Section 2.4 step 2 (displacement and
 * predicted velocity handed from FE to SBI) for a caller whose FE solver runs on the
 * host.  The convolution over lags >= 1 (which needs only the stored history)
 * runs while the inputs are copied and transformed on a side stream; the lag-0
 * term is added to it afterwards, so tau equals sbim_step's up to the rounding
 * of that one addition.  With stage profiling on, the steps run in sbim_step's
 * order instead.
 */
int sbim_step_host(sbim_handle h, const void* u, const void* v, void* tau);

/*
 * sbim_step_adjoint -- transpose of one sbim_step, for reverse-time (adjoint)
 * sweeps that differentiate a function of the tractions (Section 2.3, Eq. (SBI);
 * the transpose of the convolution is the time-reversed correlation with the same
 * kernels).  For a sequence of N forward steps from rest, tau_n(u_0..u_n, v_n),
 * and a cotangent tau_bar_n = dJ/dtau_n, calling this N times with
 * tau_bar_{N-1}, ..., tau_bar_0 on a fresh (or just reset) handle with the same
 * parameters returns, call by call, u_bar_m = dJ/du_m and v_bar_m = dJ/dv_m for
 * m = N-1, ..., 0, with sum_n <tau_n, tau_bar_n> = sum_m <u_m, u_bar_m> + <v_m, v_bar_m>
 * (far-field term excluded).  The handle's history then holds tau_bar spectra:
 * do not interleave forward and adjoint calls without sbim_reset.
 *   tau_bar  device pointer, input  [3][n3][n1]
 *   u_bar    device pointer, output [3][n3][n1]
 *   v_bar    device pointer, output [3][n3][n1] (= -side (mu/c_s) eta tau_bar)
 * The three buffers must be distinct.  Stream-ordered like sbim_step.
 */
int sbim_step_adjoint(sbim_handle h, const void* tau_bar, void* u_bar, void* v_bar);

/*
 * sbim_set_far_field -- tau_i^inf of Eq. (SBI) (Pa), a uniform far-field
 * traction added to every output; default (0, 0, 0).
 */
int sbim_set_far_field(sbim_handle h, const double tau_inf[3]);

/* sbim_reset -- forget the history; the next sbim_step is step 0 again, from the
 * equilibrium start of Section 2.1 (earlier displacements zero in Eq. (SBI)). */
int sbim_reset(sbim_handle h);

/*
 * sbim_step_repeat -- evaluate the level of the last sbim_step again with a new
 * displacement u and velocity v; the result equals sbim_rewind followed by
 * sbim_step(u, v, tau) up to rounding.  Every lag >= 1 of the truncated
 * convolution of Eq. (SBI) is unchanged, so only the lag-0 term, the assembly and
 * the two plane FFTs are recomputed: a predictor-corrector time stepper pays for
 * one history pass per step instead of two.  Needs a preceding sbim_step (or
 * sbim_step_repeat) on this handle with no sbim_step_adjoint, sbim_rewind,
 * sbim_reset, sbim_load, sbim_set_conv_config, sbim_set_window or batched step in
 * between (SBIM_ERR_STATE otherwise).  Arguments as sbim_step; stream-ordered.
 */
int sbim_step_repeat(sbim_handle h, const void* u, const void* v, void* tau);

/*
 * sbim_rewind -- take back the last sbim_step (or sbim_step_adjoint): the step
 * counter goes back by one and the next call evaluates the same time level again,
 * overwriting that level's history entry.  This is what a predictor-corrector
 * time stepper needs (evaluate at a predicted displacement, rewind, evaluate at the
 * corrected one), as the SBIM-only fault solver of Section 3's comparison does.
 * Stream-ordered; SBIM_ERR_STATE at step 0.
 */
int sbim_rewind(sbim_handle h);

/* sbim_get_step -- number of sbim_step calls since creation or the last reset (the time
 * level n of Eq. (SBI)). */
int sbim_get_step(sbim_handle h, long long* n);

/*
 * sbim_save / sbim_load -- checkpoint and restore the handle's state: the step
 * counter n, the far-field traction and the whole history ring (the spectra of
 * every displacement the truncated convolution of Eq. (SBI) can still reach;
 * Section 2.3).  A run restored from a checkpoint continues bit-for-bit as the
 * original run did from the step it was taken at.
 *
 *   sbim_save(h, buf, &bytes)
 *     buf == NULL: writes the size a checkpoint needs to *bytes and returns OK.
 *     Otherwise buf is host memory of capacity *bytes; if it is too small the
 *     call writes the needed size to *bytes and fails with SBIM_ERR_ARG.  On
 *     success *bytes is the size written.  Synchronises the handle's stream.
 *   sbim_load(h, buf, bytes)
 *     buf holds a checkpoint written by sbim_save of a handle with the same
 *     n1, n3, L1, L3, c_s, c_p, rho, dt, n_cut, side and precision; anything else
 *     (wrong magic, version, parameters or size) fails with SBIM_ERR_ARG and leaves
 *     the handle unchanged.  Synchronises the handle's stream; buf may be freed on
 *     return.  The caller owns buf in both calls.
 * A checkpoint holds the raw history layout of this library build and is not a
 * portable file format.
 */
int sbim_save(sbim_handle h, void* buf, size_t* bytes);
int sbim_load(sbim_handle h, const void* buf, size_t bytes);

/*
 * sbim_get_info -- sizes of the handle's spectral work, for throughput
 * accounting.  Any pointer may be NULL.
 *   n_modes     half-spectrum Fourier bins, n3 (n1/2 + 1)
 *   n_slots     storage slots per history step: records of 4 member slots
 *               (Nyquist bins count twice, the corner four times; padding
 *               included).  A record is two halves of 2 slots, each half's
 *               members sharing |k|; whole-record layouts give a record one
 *               class of equal |k|, half-record layouts (used when whole records
 *               would pad the history by more than 3 %, as on rectangular
 *               planes) pair the halves of two classes
 *   hist_bytes  bytes of the history ring buffer
 *   table_nodes entries of the interpolated kernel table
 * Library utility: the paper has no counterpart.
 */
int sbim_get_info(sbim_handle h, long long* n_modes, long long* n_slots,
                  long long* hist_bytes, long long* table_nodes);

/*
 * sbim_plan -- the spectral layout sbim_create builds for a grid, computed on
 * the host without touching the device, so that device memory can be budgeted
 * before any handle exists.  Outputs as sbim_get_info's (any pointer may be
 * NULL): n_modes, n_slots (|k|-sorted records x 4 member slots, padding
 * included; see sbim_get_info) and hist_bytes (the ring buffer of n_cut steps
 * at `precision`).
 * Bins are grouped by exact |k| when L1 / L3 is a ratio of integers up to 4096.
 * SBIM_ERR_ARG for the grid, n_cut and precision rules of sbim_create.
 * Library utility: the paper has no counterpart.
 */
int sbim_plan(int n1, int n3, double L1, double L3, int n_cut, int precision,
              long long* n_modes, long long* n_slots, long long* hist_bytes);

/*
 * sbim_set_check_finite -- opt-in check of every step's input for NaN and
 * infinity.  Eq. (SBI) (Section 2.3) convolves each mode's whole displacement
 * history, so one non-finite value in u would spoil every traction of the next
 * n_cut steps; with the check on, sbim_step, sbim_step_host and sbim_step_repeat
 * (u and v) and sbim_step_adjoint (tau_bar) first run one reduction kernel over
 * their input fields on the handle's stream and read its flag on the host.  If a
 * value is not finite the call returns SBIM_ERR_NONFINITE before anything else is
 * enqueued: no output is written, the history and the step counter are unchanged,
 * and the next call with finite input continues exactly as if the refused call
 * had not been made.  The read synchronises the handle's stream once per step
 * (the check is off by default: steps are then stream-ordered with no host
 * sync).  sbim_step_host takes its plain (non-overlapped) order while the check
 * is on.  Batched steps (sbim_batch_*) do not check.  Library utility: the paper
 * has no counterpart.
 */
int sbim_set_check_finite(sbim_handle h, int enable);

/*
 * sbim_set_profiling / sbim_stage_times -- per-stage device time.  While
 * profiling is on, every sbim_step records CUDA events on the handle's stream
 * around its stages; sbim_stage_times waits for them and returns the summed
 * milliseconds of (0) forward FFT, (1) history convolution, (2) reduction and
 * assembly, (3) inverse FFT, (4) traction epilogue, and the number of steps
 * summed (the stages of the spectral evaluation of Eq. (SBI), Section 2.3).
 * Enabling clears the sums.
 */
int sbim_set_profiling(sbim_handle h, int enable);
int sbim_stage_times(sbim_handle h, double ms[5], long long* steps);

/*
 * sbim_set_conv_config -- launch configuration of the history convolution
 * (Section 2.3, the per-mode time convolution), the knob a tuner turns.
 *   variant       1, 2, 3: history slots staged in shared memory by TMA bulk
 *                 copies, blocked compensated sums; the three pipeline shapes are
 *                 4 stages x 2 lags x 2 CTAs/SM, 3 x 2 x 3, 2 x 4 x 2 (FP32 / BF16
 *                 hi-lo), 8 x 2 x 2, 6 x 2 x 3, 4 x 4 x 2 (compensated BF16
 *                 hi-only), 6 x 1 x 4, 6 x 1 x 5, 6 x 2 x 3 (uncompensated BF16
 *                 hi-only), 3 x 1, 4 x 1, 2 x 2 at 2 CTAs/SM (FP64); 0: per-thread register
 *                 prefetch, per-term compensated sums.  Default: 2 for float,
 *                 bf16 hi/lo and bf16 hi-only history, 1 for double (the
 *                 fastest shapes measured on GB300 at 1024^2 x 4096).
 *   lags_per_cta  lags one CTA convolves (0 = automatic: ~16 waves of resident CTAs)
 * Both variants compute the same sums to within float rounding.  May reallocate
 * the lag-chunk partial buffer (synchronising the stream); on failure the
 * previous configuration is kept.
 */
int sbim_set_conv_config(sbim_handle h, int variant, int lags_per_cta);

/*
 * sbim_set_conv_tile -- orbit records per CTA of the TMA-staged convolution
 * (variants 1-3; Section 2.3's per-mode convolution, one thread per record of 4
 * Fourier-bin members): 64, 128 (the default) or 256, i.e. 256, 512 or 1024
 * member slots ("modes") per CTA.  A shape's shared memory and threads per SM
 * stay the same (twice the resident CTAs at 64, half at 256).  SBIM_ERR_ARG
 * unless the handle's record count (n_slots / 4) is a multiple of it.  The
 * results equal the 128-record launch's to within float rounding.  May
 * reallocate the partial sums; on failure the previous setting is kept.
 * Library utility: the paper has no counterpart.
 */
int sbim_set_conv_tile(sbim_handle h, int orbits_per_cta);

/*
 * sbim_set_window -- mode-dependent truncation of the convolution (Section 1 cites
 * the truncation of Lapusta et al. without giving a rule): a window fixed in the
 * dimensionless time T = |k| c_s t, so mode k keeps its lags m with
 * m |k| c_s dt <= window (at most n_cut; k = 0 keeps n_cut).  Long-wavelength modes
 * keep long histories, short ones short: the bytes read per step drop with the
 * window.  window = 0 restores the uniform cutoff.  The ring buffer keeps n_cut
 * slots either way.  Takes effect for the following steps.
 */
int sbim_set_window(sbim_handle h, double window);

/*
 * sbim_check_device -- wait for the handle's stream and report whether any
 * bounded device-side wait of the convolution gave up since the last check
 * (SBIM_ERR_TIMEOUT; the tractions computed since then are invalid).  Clears the
 * flag.  sbim_step_host performs this check after every step.  Library utility: the
 * paper has no counterpart.
 */
int sbim_check_device(sbim_handle h);

/*
 * sbim_selftest_wait_timeout -- exercises the failure path of the bounded
 * device waits without any fault: one CTA waits, with the convolution's
 * bounded mbarrier wait, on a barrier that nothing ever completes; after the
 * wait's wall-time limit (1 s) it gives up and sets the handle's device error
 * word.  Returns SBIM_OK when sbim_check_device then reports SBIM_ERR_TIMEOUT
 * and the word is clear again (the handle stays usable), SBIM_ERR_STATE if the
 * failure went unreported.  Synchronises the handle's stream; takes ~1 s.  Library
 * utility: the paper has no counterpart.
 */
int sbim_selftest_wait_timeout(sbim_handle h);

/*
 * sbim_spectral_response_noalloc -- the non-local traction spectrum of one
 * half-space for a caller-supplied displacement-spectrum history, without
 * allocating any device memory.  The paper has no counterpart: this entry point
 * exists for callers that may not allocate device memory -- a solver handed its
 * device buffers by a host framework that owns a fixed memory arena, or a
 * plugin whose device footprint must stay constant while the host time-steps --
 * and therefore cannot use sbim_create, which allocates the history ring
 * buffer, the kernel tables and the FFT plans.
 *
 *   n1, n3, L1, L3, cs, cp, rho, dt, side   as for sbim_create
 *   n_lags     number of history steps to convolve (>= 1); lag 0 is the current step
 *   uhat_hist  device pointer, complex float (re, im) [n_lags][3][n3][n1/2+1]: the
 *              unnormalised forward R2C spectra of the three Cartesian displacement
 *              components at steps n, n-1, ..., n-n_lags+1 (lag-major)
 *   fhat       device pointer, complex float [3][n3][n1/2+1], output: the
 *              unnormalised forward spectrum of s_i at step n (s_i is its inverse
 *              R2C transform scaled by 1/(n1 n3))
 *   stream     cudaStream_t the kernels run on (NULL = legacy default stream)
 * Float32 history, compensated accumulation; same kernels, quadrature and Nyquist
 * treatment as sbim_step.  Working memory is one static device array of 64 MiB
 * that every GPU which loads the library keeps until the process exits; it holds
 * the kernel table and the lag-chunk partial sums.  Limits (SBIM_ERR_ARG
 * otherwise): n3 (n1/2+1) <= 655,296 bins, and |k|max c_s dt (n_lags - 1) <= 8191.9.
 * uhat_hist and fhat must be 8-byte aligned memory of the current device (or
 * managed memory); host pointers and misaligned pointers return SBIM_ERR_ARG
 * before any launch.
 * The first call on a device (and any call with a new cp/cs or a longer history
 * range) resolves the array's device address and builds the kernel table, waiting
 * for the stream; make that first call before any stream capture.  All calls
 * share the array and keep the last call's contents: calls whose kernels overlap
 * on the GPU (other streams or host threads) race and must be serialised by the
 * caller.  Calls no cudaMalloc, cudaFree or allocating library routine.
 */
int sbim_spectral_response_noalloc(int n1, int n3, double L1, double L3, double cs,
                                   double cp, double rho, double dt, int side, int n_lags,
                                   const void* uhat_hist, void* fhat, void* stream);

/* ------------------------------------------------------------------------- */
/* Batches of independent updates (Section 2.3) with ragged grids           */
/* ------------------------------------------------------------------------- */
typedef struct sbim_batch_ctx* sbim_batch;

/*
 * sbim_batch_create -- nb independent half-spaces (Eq. (SBI) each), member i with
 * its own grid n1[i] x n3[i], lengths, material, dt, cutoff n_cut[i] and side[i]
 * (arrays of nb HOST values), one precision (SBIM_FP32 / BF16 variants), one
 * compensation flag and one stream.  The members are handles the batch owns
 * (reachable through sbim_batch_member).  A batch step runs the FFTs and the
 * epilogue per member and the history convolution of ALL members in one launch
 * over their (member, orbit tile, lag chunk) work items; each item writes its
 * own partial sums, so results do not depend on the schedule.  The batch sets
 * its members' convolution launch (sbim_set_conv_config) to its own pipeline
 * shape and 1024 lags per item (the default of sbim_batch_set_conv_config).
 */
int sbim_batch_create(sbim_batch* out, int nb, const int* n1, const int* n3, const double* L1,
                      const double* L3, const double* cs, const double* cp, const double* rho,
                      const double* dt, const int* n_cut, const int* side, int precision,
                      int kahan, void* stream);

/* sbim_batch_step -- one update of every member (Eq. (SBI) each): u, v, tau are HOST
 * arrays of nb DEVICE pointers ([3][n3[i]][n1[i]] each), as for sbim_step.
 * Stream-ordered. */
int sbim_batch_step(sbim_batch b, const void* const* u, const void* const* v, void* const* tau);

/*
 * sbim_batch_capture / sbim_batch_replay -- capture one batch step with these
 * (fixed) buffers into a CUDA graph on the batch's stream (which must not be the
 * legacy default stream), then replay it: each replay is one step of every
 * member, reading whatever the buffers hold at that point of the stream.  The
 * capture itself enqueues no work.  Re-capturing replaces the graph.  Library
 * utility: the paper has no counterpart.
 */
int sbim_batch_capture(sbim_batch b, const void* const* u, const void* const* v, void* const* tau);
int sbim_batch_replay(sbim_batch b);

/*
 * sbim_batch_set_conv_config -- launch of the batch's convolution: TMA pipeline
 * shape 1..3 (as in sbim_set_conv_config) on persistent CTAs that take work
 * items from a counter, or 4..6 (shapes 1..3) with one CTA per work item; and
 * lags per work item (0: 1024).  Default: one CTA per 1024-lag item with shape
 * 2 for float history, persistent shape 1 for bf16.  The results are the same
 * for every launch with the same lags per item (each item writes its own
 * partial sums).  Drops a captured graph: capture again before replaying.
 * Library utility (the launch of the Section 2.3 convolution): the paper has no
 * counterpart.
 */
int sbim_batch_set_conv_config(sbim_batch b, int shape, int lags_per_item);

/* sbim_batch_set_conv_tile -- orbit records per CTA of the batch's convolution
 * (64, 128 or 256; as sbim_set_conv_tile), keeping the shape and the lags per
 * item; SBIM_ERR_ARG unless every member's record count is a multiple of it.
 * Drops a captured graph.  Library utility: the paper has no counterpart. */
int sbim_batch_set_conv_tile(sbim_batch b, int orbits_per_cta);

/* sbim_batch_member -- the handle of member i (owned by the batch).  Library utility:
 * the paper has no counterpart. */
int sbim_batch_member(sbim_batch b, int i, sbim_handle* h);

int sbim_batch_destroy(sbim_batch b);

/* ------------------------------------------------------------------------- */
/* Pure-SBIM planar fault (Sections 2.1, 2.3 and 3): the boundary-only       */
/* solver the hybrid scheme is verified against on TPV3.                     */
/* ------------------------------------------------------------------------- */
typedef struct sbim_fault_ctx* sbim_fault;

/*
 * sbim_fault_create -- a planar fault x2 = 0 between two identical elastic
 * half-spaces, each represented only by its boundary through Eq. (SBI) (an
 * upper, side +1, and a lower, side -1, sbim_handle of the given parameters).
 * The paper describes no steps for this solver; each time step is the
 * predictor-corrector of Lapusta et al. (2000): a solve at u* = u_n + dt v_n
 * gives v*, and a solve at u_{n+1} = u_n + dt (v_n + v*)/2 gives v_{n+1}; the
 * corrector's SBIM evaluation re-evaluates the predictor's level
 * (sbim_step_repeat), so each step makes one pass over each history.  One solve
 * at face displacements u+-:
 *   (a) S+- = the non-local tractions of Eq. (SBI) for u+- (velocity 0);
 *   (b) one traction on both faces, tau = S+ - z v+ = S- + z v- with
 *       z = (mu/c_s)(1, c_p/c_s, 1), equal normal velocities (no opening or
 *       interpenetration, Section 2.1), and stick/slip of the shear traction
 *       vector against sigma^n mu(|delta|), sigma^n = sigma0 - tau_2 (Eq. (slipweak)):
 *       V = v+ - v- = 2 (tau_stick - tau)/z_s with tau_stick = (S+ + S-)/2.
 *   precision  any sbim_precision; fields are double for SBIM_FP64, else float
 *   symmetric  1: the symmetry-plane reduction of Section 3 (the lower face is the
 *              mirror image of the upper one, u-_1,3 = -u+_1,3 and u-_2 = u+_2, so
 *              S-_1,3 = S+_1,3, S-_2 = -S+_2, and only the upper half-space is
 *              evaluated: half the memory and time); 0: two half-spaces
 * Fields u, v are [2][3][n3][n1] (face 0 upper, face 1 lower), perturbations
 * from the prestressed equilibrium, starting at rest.  Without
 * sbim_fault_set_fault the fault is welded (V = 0).
 */
int sbim_fault_create(sbim_fault* out, int n1, int n3, double L1, double L3, double cs,
                      double cp, double rho, double dt, int n_cut, int precision, int symmetric,
                      void* stream);

/* sbim_fault_set_fault -- the linear slip-weakening law of Section 2.1 (Eq. (slipweak)),
 * as sbim_hybrid_set_fault: HOST maps [n3][n1] of mu_s and the x1 shear prestress tau0
 * (Pa); mu_k, Dc (m), sigma0 (compression positive, Pa). */
int sbim_fault_set_fault(sbim_fault h, const double* mu_s, const double* tau0, double mu_k,
                         double Dc, double sigma0);

/* sbim_fault_set_state / get_state -- device [2][3][n3][n1] displacement and
 * velocity of the two faces (NULL: zero on set, skip on get), the solver's whole
 * state besides the half-spaces' histories.  The symmetric solver replaces the lower
 * face by the mirror image of the upper one (Section 3's symmetry plane). */
int sbim_fault_set_state(sbim_fault h, const void* u, const void* v);
int sbim_fault_get_state(sbim_fault h, void* u, void* v);

/* sbim_fault_step -- one time step of the solver described at sbim_fault_create
 * (Sections 2.1 and 2.3), stream-ordered, no host sync. */
int sbim_fault_step(sbim_fault h);

/* sbim_fault_fields -- device outputs [3][n3][n1] (any may be NULL): slip u+ - u-,
 * slip rate v+ - v- and fault traction perturbation of the last step (Pa), the fault
 * quantities of Section 2.1. */
int sbim_fault_fields(sbim_fault h, void* slip, void* slip_rate, void* traction);

/* sbim_fault_info -- steps taken and the SBIM handles (lower is NULL when symmetric).
 * Library utility: the paper has no counterpart. */
int sbim_fault_info(sbim_fault h, long long* steps, sbim_handle* upper, sbim_handle* lower);

int sbim_fault_destroy(sbim_fault h);

/* ------------------------------------------------------------------------- */
/* Hybrid FEM-SBIM time step (Section 2.4) with an explicit FEM slab        */
/* (Section 2.2) and a slip-weakening fault (Section 2.1).                   */
/* ------------------------------------------------------------------------- */
typedef struct sbim_hybrid_ctx* sbim_hybrid;

/*
 * sbim_hybrid_create -- a slab of n1 x n2 x n3 8-node hexahedra (cubes of side h,
 * periodic in x1 and x3) between two SBIM half-spaces (Section 2.4, Neumann
 * coupling) or free surfaces.
 *   n1, n3      elements (= nodes) along x1, x3: even, the SBIM grids of S+ and S-
 *   n2          element layers across the slab (even with a fault)
 *   h           element size (m); the SBIM planes are n1 h x n3 h
 *   cs, cp, rho material (homogeneous); dt time step; n_cut SBIM history cutoff
 *   precision   SBIM_FP32 (float fields, float SBIM history with Kahan sums) or
 *               SBIM_FP64
 *   boundaries  1: SBIM half-spaces above (side +1) and below (side -1); 0: free
 *   fault       1: the node plane at element layer n2/2 is split into two copies
 *               (node layers n2/2 and n2/2 + 1); without sbim_hybrid_set_fault
 *               the copies are welded by the stick traction
 * Fields are [L][3][n3][n1] with L = n2 + 2 node layers (n2 + 1 without a fault),
 * layer 0 at the bottom boundary (S-) and L-1 at the top (S+), in the perturbation
 * formulation (departures from the prestressed equilibrium), starting at rest.
 */
int sbim_hybrid_create(sbim_hybrid* out, int n1, int n2, int n3, double h, double cs,
                       double cp, double rho, double dt, int n_cut, int precision,
                       int boundaries, int fault, void* stream);

/*
 * sbim_hybrid_set_fault -- linear slip-weakening law (Eq. (slipweak)) on the split
 * plane: mu_s and tau0 are HOST arrays [n3][n1] (static friction coefficient and
 * x1 shear prestress in Pa); mu_k, Dc (m), sigma0 (normal prestress, compression
 * positive, Pa).  Fault strength sigma^n mu(delta), delta = |tangential slip|,
 * sigma^n = sigma0 - tau_2; stick/slip on the shear traction vector (Eq. (stickslip)).
 */
int sbim_hybrid_set_fault(sbim_hybrid h, const double* mu_s, const double* tau0, double mu_k,
                          double Dc, double sigma0);

/* sbim_hybrid_set_state / get_state -- device pointers [L][3][n3][n1] of the handle's
 * element type for u, v, a (NULL: zero on set, skip on get), the FE state of the time
 * stepping of Section 2.2.  Stream-ordered. */
int sbim_hybrid_set_state(sbim_hybrid h, const void* u, const void* v, const void* a);
int sbim_hybrid_get_state(sbim_hybrid h, void* u, void* v, void* a);

/*
 * sbim_hybrid_step -- one hybrid time step (the seven steps of Section 2.4).
 * force: optional device pointer [L][3][n3][n1], an external nodal force (N)
 * added to f at t_{n+1}; NULL for none.  Stream-ordered, no host sync.
 */
int sbim_hybrid_step(sbim_hybrid h, const void* force);

/* sbim_hybrid_fault_fields -- device outputs [3][n3][n1] (any may be NULL): slip
 * vector u+ - u-, slip rate v+ - v-, and the fault traction perturbation of the
 * last step (Pa): the fault quantities of Section 2.1. */
int sbim_hybrid_fault_fields(sbim_hybrid h, void* slip, void* slip_rate, void* traction);

/*
 * Gradients through the coupled run (reverse sweep).  A forward run that keeps
 * FE states every K steps (sbim_hybrid_get_state) and the boundary tractions of
 * every step (sbim_hybrid_boundary_tractions) can recompute any step without the
 * SBIM half-spaces (sbim_hybrid_step_given), and the transpose of each step is
 * taken in reverse order by sbim_hybrid_adjoint_step.
 *
 * sbim_hybrid_boundary_tractions -- device copies [3][n3][n1] of the top and bottom
 * SBIM tractions of the last step.
 * sbim_hybrid_step_given -- one step with the given boundary tractions in place of
 * the SBIM evaluation (the half-spaces are not advanced).
 * sbim_hybrid_adjoint_step -- transpose of one step of the functional
 * sum_n <tau_n, tau_bar_n> of the fault tractions tau_n (Eqs. (fepred)-(fecorr),
 * (freeslip)-(stickslip), (slipweak), and the SBIM transposes).  h: a handle with
 * the same parameters and fault law whose two SBIM half-spaces (sbim_hybrid_info)
 * were reset before the sweep; they take the sbim_step_adjoint calls.  The call
 * reads no FE state of h, so the same handle may recompute states with
 * sbim_hybrid_step_given between calls.  Call for steps N-1, ..., 0 in that order.
 *   u, v, a           device, the state before step n  [L][3][n3][n1]
 *   tau_top, tau_bot  device, that step's boundary tractions [3][n3][n1]
 *   tau_bar           device, cotangent of the step's fault traction [3][n3][n1] (or NULL)
 *   lu, lv, la        device, in: cotangent of the state after step n; out: before it
 *   dc_bar            device [n3][n1], accumulates d/dDc (per fault node)
 */
int sbim_hybrid_boundary_tractions(sbim_hybrid h, void* tau_top, void* tau_bot);
int sbim_hybrid_step_given(sbim_hybrid h, const void* tau_top, const void* tau_bot);
int sbim_hybrid_adjoint_step(sbim_hybrid h, const void* u, const void* v, const void* a,
                             const void* tau_top, const void* tau_bot, const void* tau_bar,
                             void* lu, void* lv, void* la, void* dc_bar);

/* sbim_hybrid_info -- node layers, steps taken, and the two SBIM handles (NULL
 * with free surfaces), e.g. for profiling or sbim_set_conv_config.  Library utility:
 * the paper has no counterpart. */
int sbim_hybrid_info(sbim_hybrid h, int* layers, long long* steps, sbim_handle* top,
                     sbim_handle* bottom);

int sbim_hybrid_destroy(sbim_hybrid h);

/*
 * Ensembles of independent hybrid scenarios (ragged grids, slab thicknesses,
 * fault laws, cutoffs): sbim_hybrid_batch_create groups existing hybrid handles
 * (SBIM boundaries, SBIM_FP32, one shared stream; not owned by the batch).  A
 * batch step runs every member's FE stages and ONE batched SBIM step over all
 * 2 nb half-spaces (sbim_batch: one batched convolution launch); the members' FE
 * stages run concurrently on side streams.  capture / replay put one batch step in a
 * CUDA graph on the shared (non-default) stream.  Destroy the batch before its
 * members.  Each member steps as in Section 2.4; the batching is a library utility
 * with no counterpart in the paper.
 */
typedef struct sbim_hybrid_batch_ctx* sbim_hybrid_batch;
int sbim_hybrid_batch_create(sbim_hybrid_batch* out, int nb, const sbim_hybrid* members);
int sbim_hybrid_batch_step(sbim_hybrid_batch b);
int sbim_hybrid_batch_capture(sbim_hybrid_batch b);
int sbim_hybrid_batch_replay(sbim_hybrid_batch b);
/* sbim_hybrid_batch_set_conv_config -- as sbim_batch_set_conv_config for the
 * batch's 2 nb half-spaces; drops a captured graph.  Library utility: the paper has
 * no counterpart. */
int sbim_hybrid_batch_set_conv_config(sbim_hybrid_batch b, int shape, int lags_per_item);
/* sbim_hybrid_batch_set_conv_tile -- as sbim_batch_set_conv_tile for the batch's
 * 2 nb half-spaces; drops a captured graph.  Library utility: the paper has no
 * counterpart. */
int sbim_hybrid_batch_set_conv_tile(sbim_hybrid_batch b, int orbits_per_cta);
int sbim_hybrid_batch_destroy(sbim_hybrid_batch b);

/* sbim_destroy -- free everything the handle owns; NULL is accepted.  Library utility:
 * the paper has no counterpart. */
int sbim_destroy(sbim_handle h);

/* sbim_last_error -- message of the calling thread's last failure ("" if none).  Library
 * utility: the paper has no counterpart. */
const char* sbim_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SBIM_H */
