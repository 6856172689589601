// Batches of independent SBIM updates (Section 2.3) with ragged grids and
// history lengths, advanced together: per member the two FFTs and the epilogue,
// and ONE persistent launch of the history convolution over the (member, orbit
// tile, lag chunk) items of all members, plus one batched assembly.  A step can
// be captured once in a CUDA graph and replayed (the step counters live on the
// device, so the replayed graph advances every member's history).
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/sbim.h"
#include "sbim_internal.cuh"

struct sbim_batch_ctx {
  int nb = 0, prec = SBIM_FP32, kahan = 1, shape = 2;
  int tile = sbim::kOrbitTile;   // orbits per CTA of the batched convolution
  int lags = 0;                  // lags per work item last configured
  bool halves = false;           // some member's records hold two |k|
  bool per_item = false;    // one CTA per work item instead of persistent CTAs
  bool owns = true;
  cudaStream_t stream = nullptr;
  std::vector<sbim_handle> h;
  sbim::StepArgs* d_args = nullptr;
  int* d_item_prefix = nullptr;
  int* d_tile_prefix = nullptr;
  int* d_counter = nullptr;
  int total_items = 0, total_tiles = 0, ctas = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // side streams for the members' small stages (FFTs, epilogues): they run
  // concurrently instead of as one serial chain of small launches
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork_ev = nullptr;
};

namespace {

int bfail(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  sbim::set_last_error(buf);
  return code;
}

#define BCU(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return bfail(e_ == cudaErrorMemoryAllocation ? SBIM_ERR_OOM : SBIM_ERR_CUDA,  \
                   "%s: %s", #call, cudaGetErrorString(e_));                       \
  } while (0)

void brelease(sbim_batch_ctx* b) {
  if (!b) return;
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  for (cudaStream_t x : b->side) cudaStreamDestroy(x);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->owns)
    for (sbim_handle x : b->h) sbim_destroy(x);
  void* p[] = {b->d_args, b->d_item_prefix, b->d_tile_prefix, b->d_counter};
  for (void* x : p)
    if (x) cudaFree(x);
  delete b;
}

// Default launch: one CTA per work item of up to 1024 lags of one orbit tile,
// with the single-update kernel's pipeline shape for float history (shape 2:
// 3 stages x 2 lags, 3 CTAs/SM) and persistent CTAs with shape 1 for bf16.  On
// GB300, for a 32-scenario coupled ensemble, the batch autotuner timed 23.67 ms
// per step for this launch against 23.86 ms for the best persistent one (shape 1,
// 1024-lag items) and 24.03-26.74 ms for the other persistent shapes.
// sbim_batch_set_conv_config changes both.
constexpr int kBatchLags = 1024;
constexpr int kBatchShapeF32 = 2;
constexpr int kBatchShapeBF16 = 1;
constexpr int kSideStreams = 8;

int fork(sbim_batch_ctx* b) {
  BCU(cudaEventRecord(b->fork_ev, b->stream));
  for (cudaStream_t x : b->side) BCU(cudaStreamWaitEvent(x, b->fork_ev, 0));
  return SBIM_OK;
}

int join(sbim_batch_ctx* b) {
  for (size_t i = 0; i < b->side.size(); ++i) {
    BCU(cudaEventRecord(b->joins[i], b->side[i]));
    BCU(cudaStreamWaitEvent(b->stream, b->joins[i], 0));
  }
  return SBIM_OK;
}

cudaStream_t side_of(sbim_batch_ctx* b, int i) { return b->side[i % b->side.size()]; }

void drop_graph(sbim_batch_ctx* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// (Re)configure the members' lag chunking and the kernel shape, and upload the
// per-member arguments and item / tile prefix sums.
int configure(sbim_batch_ctx* b, int shape, int lags) {
  for (int i = 0; i < b->nb; ++i) {
    const int rc = sbim_set_conv_config(b->h[i], shape, lags);
    if (rc != SBIM_OK) return rc;
  }
  b->halves = false;
  for (int i = 0; i < b->nb; ++i) b->halves = b->halves || sbim::handle_step_args(b->h[i]).halves;
  BCU(sbim::prepare_conv_tma(b->prec, b->kahan, shape, b->tile, b->halves));
  b->shape = shape;
  b->lags = lags;
  std::vector<sbim::StepArgs> args(b->nb);
  std::vector<int> items(b->nb + 1, 0), tiles(b->nb + 1, 0);
  for (int i = 0; i < b->nb; ++i) {
    args[i] = sbim::handle_step_args(b->h[i]);
    tiles[i + 1] = tiles[i] + args[i].n_orb_pad / sbim::kOrbitTile;   // assembly tiles
    items[i + 1] = items[i] + args[i].n_orb_pad / b->tile * args[i].nchunks;
  }
  b->total_items = items[b->nb];
  b->total_tiles = tiles[b->nb];
  if (!b->d_args) BCU(cudaMalloc(&b->d_args, b->nb * sizeof(sbim::StepArgs)));
  if (!b->d_item_prefix) BCU(cudaMalloc(&b->d_item_prefix, (b->nb + 1) * sizeof(int)));
  if (!b->d_tile_prefix) BCU(cudaMalloc(&b->d_tile_prefix, (b->nb + 1) * sizeof(int)));
  if (!b->d_counter) BCU(cudaMalloc(&b->d_counter, sizeof(int)));
  BCU(cudaMemcpyAsync(b->d_args, args.data(), b->nb * sizeof(sbim::StepArgs),
                      cudaMemcpyHostToDevice, b->stream));
  BCU(cudaMemcpyAsync(b->d_item_prefix, items.data(), (b->nb + 1) * sizeof(int),
                      cudaMemcpyHostToDevice, b->stream));
  BCU(cudaMemcpyAsync(b->d_tile_prefix, tiles.data(), (b->nb + 1) * sizeof(int),
                      cudaMemcpyHostToDevice, b->stream));
  BCU(cudaStreamSynchronize(b->stream));
  int dev = 0, sms = 148;
  BCU(cudaGetDevice(&dev));
  BCU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  b->ctas = sms * sbim::conv_tma_ctas_per_sm(b->prec, b->kahan, b->shape, b->tile);
  return SBIM_OK;
}

int setup(sbim_batch_ctx* b) {
  int prec0 = 0, kahan0 = 0;
  void* st0 = nullptr;
  for (int i = 0; i < b->nb; ++i) {
    int prec, kahan, var;
    void* st;
    sbim::handle_shape(b->h[i], &prec, &kahan, &var, &st);
    (void)var;
    if (i == 0) {
      prec0 = prec; kahan0 = kahan; st0 = st;
    } else if (prec != prec0 || kahan != kahan0 || st != st0) {
      return bfail(SBIM_ERR_ARG, "batch members must share precision, compensation and stream");
    }
    if (prec == SBIM_FP64) return bfail(SBIM_ERR_ARG, "batches use float or bf16 history");
  }
  b->prec = prec0; b->kahan = kahan0; b->stream = (cudaStream_t)st0;
  b->per_item = prec0 == SBIM_FP32;
  const int k = b->nb < kSideStreams ? b->nb : kSideStreams;
  BCU(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming));
  for (int i = 0; i < k; ++i) {
    cudaStream_t x = nullptr;
    cudaEvent_t e = nullptr;
    BCU(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    b->side.push_back(x);
    BCU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->joins.push_back(e);
  }
  return configure(b, prec0 == SBIM_FP32 ? kBatchShapeF32 : kBatchShapeBF16, kBatchLags);
}

// Enqueue one step of every member (pointer arrays are host arrays of device pointers).
int enqueue(sbim_batch_ctx* b, const void* const* u, const void* const* v, void* const* tau) {
  int rc = fork(b);
  for (int i = 0; i < b->nb && rc == SBIM_OK; ++i)
    rc = sbim::handle_fft_forward(b->h[i], u[i], side_of(b, i));
  if (rc == SBIM_OK) rc = join(b);
  if (rc != SBIM_OK) return rc;
  BCU(cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream));
  sbim::BatchLaunch bl;
  bl.args = b->d_args;
  bl.item_prefix = b->d_item_prefix;
  bl.tile_prefix = b->d_tile_prefix;
  bl.nb = b->nb;
  bl.counter = b->d_counter;
  bl.ctas = b->ctas;
  bl.items = b->per_item ? b->total_items : 0;
  const sbim::StepArgs a0 = sbim::handle_step_args(b->h[0]);
  BCU(sbim::launch_conv_tma(a0, b->prec, b->kahan, b->shape, b->stream, &bl, b->tile, b->halves));
  BCU(sbim::launch_assemble_batch(bl, b->total_tiles, b->prec, b->kahan, b->stream));
  rc = fork(b);
  for (int i = 0; i < b->nb && rc == SBIM_OK; ++i) {
    rc = sbim::handle_fft_inverse(b->h[i], side_of(b, i));
    if (rc == SBIM_OK) rc = sbim::handle_epilogue(b->h[i], v[i], tau[i], side_of(b, i));
  }
  if (rc == SBIM_OK) rc = join(b);
  return rc;
}

}  // namespace

namespace sbim {
// A batch over existing handles (not owned), for drivers such as the hybrid batch.
int batch_from_handles(sbim_batch* out, const sbim_handle* hs, int n) {
  if (!out || !hs || n < 1) return bfail(SBIM_ERR_ARG, "bad batch arguments");
  sbim_batch_ctx* b = new sbim_batch_ctx;
  b->nb = n;
  b->owns = false;
  b->h.assign(hs, hs + n);
  const int rc = setup(b);
  if (rc != SBIM_OK) {
    brelease(b);
    return rc;
  }
  *out = b;
  return SBIM_OK;
}
int batch_enqueue(sbim_batch b, const void* const* u, const void* const* v, void* const* tau) {
  return enqueue(b, u, v, tau);
}
int batch_fork(sbim_batch b) { return fork(b); }
cudaStream_t batch_side(sbim_batch b, int i) { return side_of(b, i); }
int batch_join(sbim_batch b) { return join(b); }
int batch_set_conv_config(sbim_batch b, int shape, int lags_per_item) {
  return sbim_batch_set_conv_config(b, shape, lags_per_item);
}
int batch_set_conv_tile(sbim_batch b, int tile) { return sbim_batch_set_conv_tile(b, tile); }
void batch_advance(sbim_batch b) {
  for (sbim_handle x : b->h) handle_advance(x);
}
}  // namespace sbim

extern "C" {

int sbim_batch_create(sbim_batch* out, int nb, const int* n1, const int* n3, const double* L1,
                      const double* L3, const double* cs, const double* cp, const double* rho,
                      const double* dt, const int* n_cut, const int* side, int precision,
                      int kahan, void* stream) {
  if (!out || nb < 1 || !n1 || !n3 || !L1 || !L3 || !cs || !cp || !rho || !dt || !n_cut || !side)
    return bfail(SBIM_ERR_ARG, "NULL or empty batch description");
  if (precision == SBIM_FP64) return bfail(SBIM_ERR_ARG, "batches use float or bf16 history");
  sbim_batch_ctx* b = new sbim_batch_ctx;
  b->nb = nb;
  for (int i = 0; i < nb; ++i) {
    sbim_handle x = nullptr;
    const int rc = sbim_create(&x, n1[i], n3[i], L1[i], L3[i], cs[i], cp[i], rho[i], dt[i],
                               n_cut[i], side[i], precision, kahan, stream);
    if (rc != SBIM_OK) {
      brelease(b);
      return rc;
    }
    b->h.push_back(x);
  }
  const int rc = setup(b);
  if (rc != SBIM_OK) {
    brelease(b);
    return rc;
  }
  *out = b;
  return SBIM_OK;
}

int sbim_batch_step(sbim_batch b, const void* const* u, const void* const* v, void* const* tau) {
  if (!b || !u || !v || !tau) return bfail(SBIM_ERR_ARG, "NULL argument");
  for (int i = 0; i < b->nb; ++i)
    if (!u[i] || !v[i] || !tau[i]) return bfail(SBIM_ERR_ARG, "NULL field pointer (member %d)", i);
  const int rc = enqueue(b, u, v, tau);
  if (rc != SBIM_OK) return rc;
  sbim::batch_advance(b);
  return SBIM_OK;
}

int sbim_batch_capture(sbim_batch b, const void* const* u, const void* const* v, void* const* tau) {
  if (!b || !u || !v || !tau) return bfail(SBIM_ERR_ARG, "NULL argument");
  if (!b->stream) return bfail(SBIM_ERR_ARG, "graph capture needs a non-default stream");
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  BCU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  const int rc = enqueue(b, u, v, tau);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (rc != SBIM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return bfail(SBIM_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  b->graph = g;
  BCU(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return SBIM_OK;
}

int sbim_batch_replay(sbim_batch b) {
  if (!b) return bfail(SBIM_ERR_ARG, "NULL batch");
  if (!b->exec) return bfail(SBIM_ERR_STATE, "no captured step: call sbim_batch_capture first");
  BCU(cudaGraphLaunch(b->exec, b->stream));
  sbim::batch_advance(b);
  return SBIM_OK;
}

int sbim_batch_set_conv_config(sbim_batch b, int shape, int lags_per_item) {
  if (!b) return bfail(SBIM_ERR_ARG, "NULL batch");
  if (shape < 1 || shape > 6) return bfail(SBIM_ERR_ARG, "shape must be 1..6");
  if (lags_per_item < 0) return bfail(SBIM_ERR_ARG, "lags_per_item must be >= 0");
  drop_graph(b);
  b->per_item = shape > 3;
  return configure(b, shape > 3 ? shape - 3 : shape, lags_per_item ? lags_per_item : kBatchLags);
}

int sbim_batch_set_conv_tile(sbim_batch b, int orbits_per_cta) {
  if (!b) return bfail(SBIM_ERR_ARG, "NULL batch");
  if (orbits_per_cta != 64 && orbits_per_cta != 128 && orbits_per_cta != 256)
    return bfail(SBIM_ERR_ARG, "orbits per CTA must be 64, 128 or 256");
  for (int i = 0; i < b->nb; ++i) {
    const int n = sbim::handle_step_args(b->h[i]).n_orb_pad;
    if (n % orbits_per_cta != 0)
      return bfail(SBIM_ERR_ARG, "member %d has %d orbit records, not a multiple of %d", i, n,
                   orbits_per_cta);
  }
  drop_graph(b);
  const int old = b->tile;
  b->tile = orbits_per_cta;
  const int rc = configure(b, b->shape, b->lags);
  if (rc != SBIM_OK) b->tile = old;
  return rc;
}

int sbim_batch_member(sbim_batch b, int i, sbim_handle* h) {
  if (!b || !h || i < 0 || i >= b->nb) return bfail(SBIM_ERR_ARG, "bad member index");
  *h = b->h[i];
  return SBIM_OK;
}

int sbim_batch_destroy(sbim_batch b) {
  if (!b) return SBIM_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  brelease(b);
  return SBIM_OK;
}

}  // extern "C"
