// Per-step kernels of the spectral boundary integral update (Section 2.3, Eq. (SBI)).
//
//  conv_kernel     For every record (four Fourier-bin member slots in two halves,
//                  the members of a half sharing |k|) and one
//                  chunk of lags: rotate the current spectra into the
//                  (xi, 2, perp) frame of each member and write them into the
//                  history ring slot (chunk 0 only), then accumulate the five
//                  truncated convolutions
//                     C11 = sum_m w11(m) D_xi[n-m],   C33 = sum_m w33(m) D_perp[n-m],
//                     C22 = sum_m w22(m) D_2[n-m],    C12a = sum_m w12(m) D_2[n-m],
//                     C12b = sum_m w12(m) D_xi[n-m]
//                  with trapezoid weights w(m) = dT H(m dT) (half at m = 0),
//                  dT = |k| c_s dt.  The weights are interpolated from a table of
//                  H(T) (cubic Lagrange), once per half and lag (once per record
//                  when its halves share |k|), so they cost no HBM bytes.
//  assemble_kernel Sum the chunk partials in chunk order, add the instantaneous
//                  in-plane coupling (2 - eta), apply -side mu |k| to the diagonal
//                  terms, rotate back to (1, 2, 3) and write the output spectrum
//                  scaled by member weight / (n1 n3).
//  epilogue_kernel tau_c = tau_inf_c - side (mu / c_s) eta_c v_c + s_c and the
//                  step counter.
#include "../../include/sbim.h"
#include "sbim_device.cuh"

namespace sbim {

namespace {

using namespace dev;

// Resident CTAs per SM the register budget is sized for: FP64 accumulators
// need twice the registers (and the FP64 path is bound by FP64 issue anyway).
template <class S> struct MinBlocks { static constexpr int value = 3; };
template <> struct MinBlocks<StoreF64> { static constexpr int value = 1; };

// (The half-record variants, with a second weight set, are sized for 2 CTAs/SM.)
template <class S, int KAHAN, bool HALVES>
__global__ void __launch_bounds__(kOrbitTile, HALVES && MinBlocks<S>::value > 2 ? 2 : MinBlocks<S>::value)
conv_kernel(const StepArgs a) {
  using R = typename S::real;
  using C = typename S::cplx;
  using T4 = typename S::tab4;
  const int o = blockIdx.x * kOrbitTile + threadIdx.x;
  const int chunk = blockIdx.y;
  const long long n = *a.step;
  const int n_valid = (n + 1 < (long long)a.n_cut) ? (int)(n + 1) : a.n_cut;
  const int m0 = chunk * a.lc;
  const int m_end = a.tile_lmax ? min(n_valid, a.tile_lmax[blockIdx.x]) : n_valid;
  if (m0 >= m_end) return;
  const int m1 = min(m0 + a.lc, m_end);
  // the two halves' truncation, lag spacing in T and table step
  const int lo0 = a.lmax ? a.lmax[2 * o] : 0x7fffffff, lo1 = a.lmax ? a.lmax[2 * o + 1] : 0x7fffffff;
  const int sn = (int)(n % a.n_cut);
  const R dT0 = reinterpret_cast<const R*>(a.dT)[2 * o], dT1 = reinterpret_cast<const R*>(a.dT)[2 * o + 1];
  const unsigned long long us0 = a.ustep[2 * o], us1 = a.ustep[2 * o + 1];
  const bool same = !HALVES || us0 == us1;   // whole-record plans: always one |k|
  const T4* tab = reinterpret_cast<const T4*>(a.table);
  const long long orb = a.n_orb_pad;
  const long long plane = a.slot_stride;

  R acc[4][kFields], cmp[4][kFields];
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int k = 0; k < kFields; ++k) { acc[g][k] = (R)0; cmp[g][k] = (R)0; }

  int m = m0;
  if (m0 == 0) {
    C D[3][4];
    rotate_current(a, o, D);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      S::store(a.hist, ((long long)sn * 3 + c) * orb + o, plane, D[c]);
      S::round(D[c]);
    }
    R w0[4], w1[4];
    lag_weights(tab, 0ull, dT0 * (R)0.5, w0);
    if (same) {
#pragma unroll
      for (int q = 0; q < 4; ++q) w1[q] = w0[q];
    } else {
      lag_weights(tab, 0ull, dT1 * (R)0.5, w1);
    }
    accumulate<KAHAN>(acc, cmp, w0, w1, D);
    m = 1;
  }
  if (m < m1) {
    int slot = sn - m;
    if (slot < 0) slot += a.n_cut;
    unsigned long long u0 = (unsigned long long)m * us0, u1 = (unsigned long long)m * us1;
    C Dn[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c) S::load(a.hist, ((long long)slot * 3 + c) * orb + o, plane, Dn[c]);
    for (; m < m1; ++m) {
      C D[3][4];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int g = 0; g < 4; ++g) D[c][g] = Dn[c][g];
      if (m + 1 < m1) {
        slot = (slot == 0) ? a.n_cut - 1 : slot - 1;
#pragma unroll
        for (int c = 0; c < 3; ++c) S::load(a.hist, ((long long)slot * 3 + c) * orb + o, plane, Dn[c]);
      }
      R w0[4], w1[4];
      lag_weights(tab, u0, m < lo0 ? dT0 : (R)0, w0);
      if (same) {
#pragma unroll
        for (int q = 0; q < 4; ++q) w1[q] = w0[q];
      } else {
        lag_weights(tab, u1, m < lo1 ? dT1 : (R)0, w1);
      }
      u0 += us0;
      u1 += us1;
      accumulate<KAHAN>(acc, cmp, w0, w1, D);
    }
  }
  R* part = reinterpret_cast<R*>(a.part);
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int k = 0; k < kFields; ++k)
      part[((long long)chunk * (4 * kFields) + g * kFields + k) * orb + o] =
          KAHAN ? acc[g][k] - cmp[g][k] : acc[g][k];
}

template <class S, int KAHAN>
__device__ __forceinline__ void assemble_orbit(const StepArgs& a, int o) {
  using R = typename S::real;
  using C = typename S::cplx;
  const long long n = *a.step;
  const int n_valid = (n + 1 < (long long)a.n_cut) ? (int)(n + 1) : a.n_cut;
  const int m_end = a.tile_lmax ? min(n_valid, a.tile_lmax[o / kOrbitTile]) : n_valid;
  const int nch = (m_end + a.lc - 1) / a.lc;
  const long long orb = a.n_orb_pad;
  const R muq0 = reinterpret_cast<const R*>(a.muq)[2 * o];
  const R muq1 = reinterpret_cast<const R*>(a.muq)[2 * o + 1];
  const R sd = (R)a.side;
  const R inst = (R)(2.0 - a.eta);
  const R* part = reinterpret_cast<const R*>(a.part);
  C* fh = reinterpret_cast<C*>(a.fhat);

  C D[3][4];
  rotate_current(a, o, D);

  // Chunk reduction of the 4 x kFields sums: the chunk loop is outermost so that
  // each iteration issues 40 independent loads (each sum's own order over the
  // chunks, and its compensation, are those of a per-sum loop).
  R sum[4][kFields], cmp[4][kFields];
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int k = 0; k < kFields; ++k) { sum[g][k] = (R)0; cmp[g][k] = (R)0; }
  auto load_chunk = [&](int ch, R (&x)[4][kFields]) {
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
      for (int k = 0; k < kFields; ++k)
        x[g][k] = part[((long long)ch * (4 * kFields) + g * kFields + k) * orb + o];
  };
  if constexpr (KAHAN) {
    for (int ch = 0; ch < nch; ++ch) {
      R x[4][kFields];
      load_chunk(ch, x);
#pragma unroll
      for (int g = 0; g < 4; ++g)
#pragma unroll
        for (int k = 0; k < kFields; ++k) {
          const R y = x[g][k] - cmp[g][k];
          const R t = sum[g][k] + y;
          cmp[g][k] = (t - sum[g][k]) - y;
          sum[g][k] = t;
        }
    }
  } else if constexpr (sizeof(R) == 8) {
    // FP64 sums (their step is bound by the FP64 pipe): one chunk at a time
    for (int ch = 0; ch < nch; ++ch) {
      R x[4][kFields];
      load_chunk(ch, x);
#pragma unroll
      for (int g = 0; g < 4; ++g)
#pragma unroll
        for (int k = 0; k < kFields; ++k) sum[g][k] += x[g][k];
    }
  } else if (nch > 0) {
    // Plain float sums: the next chunk's 40 loads are issued before this chunk's
    // adds (left to the compiler, the uncompensated loop kept few loads in flight
    // and ran at a third of the compensated one's rate on GB300).
    R x[4][kFields], xn[4][kFields];
    load_chunk(0, x);
    for (int ch = 0; ch < nch; ++ch) {
      const bool more = ch + 1 < nch;
      if (more) load_chunk(ch + 1, xn);
#pragma unroll
      for (int g = 0; g < 4; ++g)
#pragma unroll
        for (int k = 0; k < kFields; ++k) sum[g][k] += x[g][k];
      if (more)
#pragma unroll
        for (int g = 0; g < 4; ++g)
#pragma unroll
          for (int k = 0; k < kFields; ++k) x[g][k] = xn[g][k];
    }
  }

  int pend = -1;
  C P1, P2, P3;
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const int b = a.bin[o * 4 + g];
    if (b < 0) continue;
    const R muq = g < 2 ? muq0 : muq1;
    const R* v = sum[g];
    const C dxi = D[0][g], d2 = D[1][g];
    // F_xi = -side mu q C11 + i mu q [(2 - eta) D_2 + C12a]
    const R bxr = inst * d2.x + v[6], bxi = inst * d2.y + v[7];
    C fxi, fp, f2;
    fxi.x = muq * (-sd * v[0] - bxi);
    fxi.y = muq * (-sd * v[1] + bxr);
    // F_perp = -side mu q C33
    fp.x = -sd * muq * v[2];
    fp.y = -sd * muq * v[3];
    // F_2 = -i mu q [(2 - eta) D_xi + C12b] - side mu q C22
    const R b2r = inst * dxi.x + v[8], b2i = inst * dxi.y + v[9];
    f2.x = muq * (b2i - sd * v[4]);
    f2.y = muq * (-b2r - sd * v[5]);
    const C e = reinterpret_cast<const C*>(a.dir)[o * 4 + g];
    const R e1 = e.x, e3 = e.y;
    const R wsc = (R)a.wout[o * 4 + g] * (R)a.inv_n;
    C f1, f3;
    f1.x = wsc * (e1 * fxi.x - e3 * fp.x); f1.y = wsc * (e1 * fxi.y - e3 * fp.y);
    f3.x = wsc * (e3 * fxi.x + e1 * fp.x); f3.y = wsc * (e3 * fxi.y + e1 * fp.y);
    f2.x *= wsc; f2.y *= wsc;
    if (b == pend) {
      P1.x += f1.x; P1.y += f1.y; P2.x += f2.x; P2.y += f2.y; P3.x += f3.x; P3.y += f3.y;
    } else {
      if (pend >= 0) {
        fh[pend] = P1; fh[a.nbins + pend] = P2; fh[2 * (long long)a.nbins + pend] = P3;
      }
      pend = b; P1 = f1; P2 = f2; P3 = f3;
    }
  }
  if (pend >= 0) {
    fh[pend] = P1; fh[a.nbins + pend] = P2; fh[2 * (long long)a.nbins + pend] = P3;
  }
}

template <class S, int KAHAN>
__global__ void __launch_bounds__(kOrbitTile) assemble_kernel(const StepArgs a) {
  const int o = blockIdx.x * kOrbitTile + threadIdx.x;
  if (o >= a.n_orb_pad) return;
  assemble_orbit<S, KAHAN>(a, o);
}

// One CTA per orbit tile of every member of a batch.
template <class S, int KAHAN>
__global__ void __launch_bounds__(kOrbitTile)
assemble_batch_kernel(const StepArgs* __restrict__ args, const int* __restrict__ tile_prefix, int nb) {
  const int t = blockIdx.x;
  int s = 0;
  while (s + 1 < nb && tile_prefix[s + 1] <= t) ++s;
  const StepArgs a = args[s];
  assemble_orbit<S, KAHAN>(a, (t - tile_prefix[s]) * kOrbitTile + threadIdx.x);
}

template <class R>
__global__ void epilogue_kernel(const R* __restrict__ s, const R* __restrict__ v,
                                R* __restrict__ tau, long long plane, R c0, R c1, R c2,
                                R t0, R t1, R t2, long long* step) {
  const long long total = 3 * plane;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / plane);
    const R coef = c == 0 ? c0 : (c == 1 ? c1 : c2);
    const R ti = c == 0 ? t0 : (c == 1 ? t1 : t2);
    tau[i] = ti - coef * v[i] + s[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *step += 1;
}

// Adjoint epilogue: v_bar_c = -side (mu / c_s) eta_c tau_bar_c, and the step counter.
template <class R>
__global__ void adjoint_epilogue_kernel(const R* __restrict__ tau_bar, R* __restrict__ v_bar,
                                        long long plane, R c0, R c1, R c2, long long* step) {
  const long long total = 3 * plane;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / plane);
    const R coef = c == 0 ? c0 : (c == 1 ? c1 : c2);
    v_bar[i] = -coef * tau_bar[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *step += 1;
}

// FP64 weights precomputed once per handle: they depend only on (orbit, lag),
// so the FP64 convolution, bound by the FP64 pipe, streams them beside the
// history instead of re-interpolating them every step.
__global__ void __launch_bounds__(256) weights64_kernel(const StepArgs a, Double4* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)a.n_cut * a.n_orb_pad;
  if (i >= total) return;
  const int o = (int)(i % a.n_orb_pad);
  const long long m = i / a.n_orb_pad;
  double w[4];   // half 0 of the record (the kernel interpolates a differing half 1)
  lag_weights(reinterpret_cast<const Double4*>(a.table), (unsigned long long)m * a.ustep[2 * o],
              reinterpret_cast<const double*>(a.dT)[2 * o], w);
  Double4 r;
  r.x = w[0]; r.y = w[1]; r.z = w[2]; r.w = w[3];
  out[i] = r;
}

// Opt-in input check (sbim_set_check_finite): sets *flag if any of the n values
// of a or b (b may be NULL) is NaN or infinite.  One block-wide vote per pass and
// at most one store per block.
template <class R>
__global__ void __launch_bounds__(256) nonfinite_kernel(const R* __restrict__ a,
                                                        const R* __restrict__ b, long long n,
                                                        int* __restrict__ flag) {
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    bad |= !isfinite(a[i]);
    if (b) bad |= !isfinite(b[i]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) *flag = 1;
}

// Re-evaluation of the current level with a new displacement (sbim_step_repeat).
// Every lag >= 1 of the truncated convolution is unchanged, so chunk 0's partial
// sums take w(0) (D_new - D_old) and the ring slot takes D_new; the assembly then
// runs as usual.  Lag 0 is in chunk 0 of every orbit (its lag limit is >= 1).
template <class S>
__global__ void __launch_bounds__(kOrbitTile) repeat_lag0_kernel(const StepArgs a) {
  using R = typename S::real;
  using C = typename S::cplx;
  using T4 = typename S::tab4;
  const int o = blockIdx.x * kOrbitTile + threadIdx.x;
  if (o >= a.n_orb_pad) return;
  const long long n = *a.step;
  const int sn = (int)(n % a.n_cut);
  const long long orb = a.n_orb_pad;
  C Dn[3][4], Do[3][4];
  rotate_current(a, o, Dn);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long long rec = ((long long)sn * 3 + c) * orb + o;
    S::load(a.hist, rec, a.slot_stride, Do[c]);
    S::store(a.hist, rec, a.slot_stride, Dn[c]);
    S::round(Dn[c]);
  }
  R w0[4], w1[4];
  lag_weights(reinterpret_cast<const T4*>(a.table), 0ull,
              reinterpret_cast<const R*>(a.dT)[2 * o] * (R)0.5, w0);
  lag_weights(reinterpret_cast<const T4*>(a.table), 0ull,
              reinterpret_cast<const R*>(a.dT)[2 * o + 1] * (R)0.5, w1);
  R* part = reinterpret_cast<R*>(a.part);
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const R* w = g < 2 ? w0 : w1;
    C x, d2, dp;
    x.x = Dn[0][g].x - Do[0][g].x;  x.y = Dn[0][g].y - Do[0][g].y;
    d2.x = Dn[1][g].x - Do[1][g].x; d2.y = Dn[1][g].y - Do[1][g].y;
    dp.x = Dn[2][g].x - Do[2][g].x; dp.y = Dn[2][g].y - Do[2][g].y;
    // the field order of accumulate(): C11 (xi), C33 (perp), C22 (2), C12a (2), C12b (xi)
    const R add[kFields] = {w[0] * x.x,  w[0] * x.y,  w[2] * dp.x, w[2] * dp.y, w[1] * d2.x,
                            w[1] * d2.y, w[3] * d2.x, w[3] * d2.y, w[3] * x.x,  w[3] * x.y};
#pragma unroll
    for (int k = 0; k < kFields; ++k) part[((long long)g * kFields + k) * orb + o] += add[k];
  }
}

// Step counter one back (sbim_rewind): the next step rewrites the same ring slot.
__global__ void rewind_kernel(long long* step) {
  if (threadIdx.x == 0 && *step > 0) *step -= 1;
}

template <class S, int KAHAN>
cudaError_t conv_dispatch(const StepArgs& a, cudaStream_t st) {
  const dim3 grid(a.n_orb_pad / kOrbitTile, a.nchunks);
  if (a.halves)
    conv_kernel<S, KAHAN, true><<<grid, kOrbitTile, 0, st>>>(a);
  else
    conv_kernel<S, KAHAN, false><<<grid, kOrbitTile, 0, st>>>(a);
  return cudaGetLastError();
}

template <class S, int KAHAN>
cudaError_t assemble_dispatch(const StepArgs& a, cudaStream_t st) {
  const int grid = a.n_orb_pad / kOrbitTile;
  assemble_kernel<S, KAHAN><<<grid, kOrbitTile, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_conv(const StepArgs& a, int precision, int kahan, cudaStream_t st) {
  switch (precision) {
    case SBIM_FP64: return conv_dispatch<StoreF64, 0>(a, st);
    case SBIM_FP32:
      return kahan ? conv_dispatch<StoreF32, 1>(a, st) : conv_dispatch<StoreF32, 0>(a, st);
    case SBIM_BF16X2:
      return kahan ? conv_dispatch<StoreBF16<true>, 1>(a, st)
                   : conv_dispatch<StoreBF16<true>, 0>(a, st);
    case SBIM_BF16:
      return kahan ? conv_dispatch<StoreBF16<false>, 1>(a, st)
                   : conv_dispatch<StoreBF16<false>, 0>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_assemble(const StepArgs& a, int precision, int kahan, cudaStream_t st) {
  switch (precision) {
    case SBIM_FP64: return assemble_dispatch<StoreF64, 0>(a, st);
    case SBIM_FP32:
      return kahan ? assemble_dispatch<StoreF32, 1>(a, st) : assemble_dispatch<StoreF32, 0>(a, st);
    case SBIM_BF16X2:
      return kahan ? assemble_dispatch<StoreBF16<true>, 1>(a, st)
                   : assemble_dispatch<StoreBF16<true>, 0>(a, st);
    case SBIM_BF16:
      return kahan ? assemble_dispatch<StoreBF16<false>, 1>(a, st)
                   : assemble_dispatch<StoreBF16<false>, 0>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <class S, int KAHAN>
cudaError_t assemble_batch_dispatch(const BatchLaunch& b, int tiles, cudaStream_t st) {
  assemble_batch_kernel<S, KAHAN><<<tiles, kOrbitTile, 0, st>>>(b.args, b.tile_prefix, b.nb);
  return cudaGetLastError();
}

cudaError_t launch_assemble_batch(const BatchLaunch& b, int tiles, int precision, int kahan,
                                  cudaStream_t st) {
  switch (precision) {
    case SBIM_FP64: return assemble_batch_dispatch<StoreF64, 0>(b, tiles, st);
    case SBIM_FP32:
      return kahan ? assemble_batch_dispatch<StoreF32, 1>(b, tiles, st)
                   : assemble_batch_dispatch<StoreF32, 0>(b, tiles, st);
    case SBIM_BF16X2:
      return kahan ? assemble_batch_dispatch<StoreBF16<true>, 1>(b, tiles, st)
                   : assemble_batch_dispatch<StoreBF16<true>, 0>(b, tiles, st);
    case SBIM_BF16:
      return kahan ? assemble_batch_dispatch<StoreBF16<false>, 1>(b, tiles, st)
                   : assemble_batch_dispatch<StoreBF16<false>, 0>(b, tiles, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_epilogue(int precision, const void* s_field, const void* v, void* tau,
                            long long plane, const double coef[3], const double tau_inf[3],
                            long long* step, cudaStream_t st) {
  const int threads = 256;
  long long blocks = (3 * plane + threads - 1) / threads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (precision == SBIM_FP64) {
    epilogue_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(
        (const double*)s_field, (const double*)v, (double*)tau, plane, coef[0], coef[1],
        coef[2], tau_inf[0], tau_inf[1], tau_inf[2], step);
  } else {
    epilogue_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(
        (const float*)s_field, (const float*)v, (float*)tau, plane, (float)coef[0],
        (float)coef[1], (float)coef[2], (float)tau_inf[0], (float)tau_inf[1],
        (float)tau_inf[2], step);
  }
  return cudaGetLastError();
}

cudaError_t launch_repeat_lag0(const StepArgs& a, int precision, cudaStream_t st) {
  const unsigned grid = (unsigned)(a.n_orb_pad / kOrbitTile);
  switch (precision) {
    case SBIM_FP64: repeat_lag0_kernel<StoreF64><<<grid, kOrbitTile, 0, st>>>(a); break;
    case SBIM_FP32: repeat_lag0_kernel<StoreF32><<<grid, kOrbitTile, 0, st>>>(a); break;
    case SBIM_BF16X2: repeat_lag0_kernel<StoreBF16<true>><<<grid, kOrbitTile, 0, st>>>(a); break;
    case SBIM_BF16: repeat_lag0_kernel<StoreBF16<false>><<<grid, kOrbitTile, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_weights64(const StepArgs& a, void* out, cudaStream_t st) {
  const long long total = (long long)a.n_cut * a.n_orb_pad;
  const long long blocks = (total + 255) / 256;
  weights64_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, reinterpret_cast<Double4*>(out));
  return cudaGetLastError();
}

cudaError_t launch_nonfinite_check(int precision, const void* a, const void* b, long long n,
                                   int* flag, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int threads = 256;
  long long blocks = (n + threads - 1) / threads;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  if (precision == SBIM_FP64)
    nonfinite_kernel<double><<<(unsigned)blocks, threads, 0, st>>>((const double*)a,
                                                                   (const double*)b, n, flag);
  else
    nonfinite_kernel<float><<<(unsigned)blocks, threads, 0, st>>>((const float*)a,
                                                                  (const float*)b, n, flag);
  return cudaGetLastError();
}

cudaError_t launch_rewind(long long* step, cudaStream_t st) {
  rewind_kernel<<<1, 32, 0, st>>>(step);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_epilogue(int precision, const void* tau_bar, void* v_bar,
                                    long long plane, const double coef[3], long long* step,
                                    cudaStream_t st) {
  const int threads = 256;
  long long blocks = (3 * plane + threads - 1) / threads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (precision == SBIM_FP64) {
    adjoint_epilogue_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(
        (const double*)tau_bar, (double*)v_bar, plane, coef[0], coef[1], coef[2], step);
  } else {
    adjoint_epilogue_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(
        (const float*)tau_bar, (float*)v_bar, plane, (float)coef[0], (float)coef[1],
        (float)coef[2], step);
  }
  return cudaGetLastError();
}

}  // namespace sbim
