// History convolution with the history slots staged in shared memory by TMA
// bulk copies (Section 2.3, spectral evaluation of s_i: the per-mode truncated
// time convolution, step A4).
//
// One CTA = one tile of TILE orbits (one thread per orbit; TILE = 64, 128 or
// 256, the handle's "modes per CTA") and one chunk of lags.  For every lag the
// tile's history lives in 3 contiguous segments of global memory (one per
// component, TILE records each), so an elected thread stages a
// pipeline stage of KS lags with 3 KS cp.async.bulk copies completing on an
// mbarrier, NS stages deep; the bytes in flight cost no registers.  Threads read
// their own 16-byte chunks from the staged segments with a per-quarter-warp
// rotation of the chunk order that avoids shared-memory bank conflicts.
//
// The convolution weights of stage i+1 are prepared while stage i is computed:
// the four kernel-table nodes of each of its lags are loaded before stage i's
// arithmetic and interpolated after it, so the table's L1/L2 latency overlaps
// the FMA chains.
//
// Compensated accumulation is blocked: the KS terms of one stage are chained by
// FMAs starting from the negated compensation, then a single Kahan update folds
// the block into the running sum (error ~ (KS + 2) eps sum|terms| instead of
// ~2 eps for per-term Kahan, at well under half the instructions).
//
// Every mbarrier wait is bounded; a wait that gives up sets the device error
// word, waits (bounded) for the copies this CTA still has in flight, and
// returns without writing its partial sums.
#pragma once

#include <type_traits>

#include "../../include/sbim.h"
#include "sbim_device.cuh"

namespace sbim {
namespace tma {

using namespace dev;

constexpr unsigned long long kWaitNs = 1000000000ull;   // give up a wait after 1 s

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ const int kNoError = 0;   // drain waits after a failure ignore the flag

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of `parity` to complete.  Bounded: gives up after kWaitNs
// of wall time, or at once when the device error word is already set (another
// CTA gave up), so a failure costs every CTA at most one second.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, const int* err) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 63u) == 63u &&
        (global_ns() - t0 > kWaitNs || *(volatile const int*)err != 0))
      return false;
  }
}

__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes,
                                         unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Whether the next stage's table nodes are loaded during a stage's arithmetic
// (hides their L2 latency, at KS x 16 floats of registers per thread).  The
// compensated BF16 kernels, whose unpacked records and Kahan terms already
// fill the register file, interpolate each stage's weights in place instead.
// Half-record kernels prefetch the nodes of both halves where the register
// budget allows it (<= 2 resident CTAs per 128 records, <= 2 lags per stage,
// float history) and interpolate in place otherwise.
template <class S, int KAHAN, bool HALVES, int NS, int KS, int MINB, int TILE> struct PrefetchNodes {
  static constexpr bool value =
      !HALVES || (KS <= 2 && MINB * TILE <= 2 * 128 && sizeof(typename S::real) == 4);
};
template <bool LO, bool HALVES, int NS, int KS, int MINB, int TILE>
struct PrefetchNodes<dev::StoreBF16<LO>, 1, HALVES, NS, KS, MINB, TILE> {
  static constexpr bool value = false;
};

template <class S, int TILE>
__host__ __device__ constexpr int seg_bytes() { return TILE * S::kRecBytes; }
// FP64 history: a stage also holds each lag's precomputed weights (4 doubles per
// orbit) when the handle keeps them (StepArgs::wts); the float paths interpolate.
template <class S, int TILE>
__host__ __device__ constexpr int wseg_bytes() {
  return std::is_same<S, dev::StoreF64>::value ? TILE * 32 : 0;
}
template <class S, int KS, int TILE>
__host__ __device__ constexpr int stage_bytes() {
  return KS * (3 * S::kPlanes * seg_bytes<S, TILE>() + wseg_bytes<S, TILE>());
}
template <class S, int NS, int KS, int TILE>
__host__ __device__ constexpr int smem_bytes() { return NS * stage_bytes<S, KS, TILE>(); }

// Resident CTAs per SM of a pipeline shape (sized for 128-orbit tiles) at
// another tile: the same shared memory and threads per SM.
__host__ __device__ constexpr int minb_for_tile(int minb, int tile) {
  return tile == 64 ? 2 * minb : (tile == 256 ? (minb / 2 > 0 ? minb / 2 : 1) : minb);
}

// The four table nodes of one lag, and their cubic Lagrange combination (the
// two halves of dev::lag_weights, split so the loads can be issued early).
template <class T4>
__device__ __forceinline__ void fetch_nodes(const T4* __restrict__ tab, unsigned long long u,
                                            T4 nd[4]) {
  const unsigned i = (unsigned)(u >> 32);
  nd[0] = ld_tab(tab + i);
  nd[1] = ld_tab(tab + i + 1);
  nd[2] = ld_tab(tab + i + 2);
  nd[3] = ld_tab(tab + i + 3);
}

template <class R, class T4>
__device__ __forceinline__ void interp_nodes(const T4 nd[4], unsigned long long u, R scale,
                                             R w[4]) {
  const R t = (R)(unsigned)(u & 0xffffffffull) * (R)2.3283064365386962890625e-10;
  const R tm1 = t - (R)1, tm2 = t - (R)2, tp1 = t + (R)1;
  const R sixth = scale * (R)(1.0 / 6.0), halfs = scale * (R)0.5;
  const R l0 = -t * tm1 * tm2 * sixth;
  const R l1 = tp1 * tm1 * tm2 * halfs;
  const R l2 = -tp1 * t * tm2 * halfs;
  const R l3 = tp1 * t * tm1 * sixth;
  w[0] = l0 * nd[0].x + l1 * nd[1].x + l2 * nd[2].x + l3 * nd[3].x;
  w[1] = l0 * nd[0].y + l1 * nd[1].y + l2 * nd[2].y + l3 * nd[3].y;
  w[2] = l0 * nd[0].z + l1 * nd[1].z + l2 * nd[2].z + l3 * nd[3].z;
  w[3] = l0 * nd[0].w + l1 * nd[1].w + l2 * nd[2].w + l3 * nd[3].w;
}

// One work item: orbit tile `tile` and lag chunk `chunk` of the update `a`.
// The NS mbarriers of `full` are initialised once per CTA; their phases carry
// over from item to item through the running stage count `gstage` (stage s of
// this item is global stage gstage + s: buffer (gstage + s) % NS, parity
// ((gstage + s) / NS) & 1).  Returns false if a bounded wait gave up.
template <class S, int KAHAN, int NS, int KS, int MINB, int TILE, bool HALVES>
__device__ __forceinline__ bool conv_tma_item(const StepArgs& a, int tile, int chunk,
                                              unsigned char* smem, unsigned long long* full,
                                              unsigned& gstage) {
  using R = typename S::real;
  using C = typename S::cplx;
  using T4 = typename S::tab4;
  constexpr int SEG = seg_bytes<S, TILE>();
  constexpr int WSEG = wseg_bytes<S, TILE>();
  constexpr int HIST = KS * 3 * S::kPlanes * SEG;   // history part of a stage
  constexpr int STAGE = stage_bytes<S, KS, TILE>();
  constexpr int MPC = S::kChunkMembers, NCH = S::kChunks;

  const int tid = threadIdx.x;
  const int tile0 = tile * TILE;
  const int o = tile0 + tid;
  const long long n = *a.step;
  const int n_valid = (n + 1 < (long long)a.n_cut) ? (int)(n + 1) : a.n_cut;
  const int m0 = chunk * a.lc;
  // the truncation window's lag limit is kept per 128-orbit tile
  int m_end = n_valid;
  if (a.tile_lmax) {
    int lim = 0;
#pragma unroll
    for (int t = 0; t < (TILE + kOrbitTile - 1) / kOrbitTile; ++t)
      lim = max(lim, a.tile_lmax[tile0 / kOrbitTile + t]);
    m_end = min(n_valid, lim);
  }
  if (m0 >= m_end) return true;   // uniform over the CTA
  const int m1 = min(m0 + a.lc, m_end);
  // the record's two halves: truncation, lag spacing in T and table step of each
  // (equal when the record holds one |k|, the usual case on square grids)
  const int lo = a.lmax ? a.lmax[2 * o] : 0x7fffffff;
  const int lo1 = a.lmax ? a.lmax[2 * o + 1] : 0x7fffffff;
  const int sn = (int)(n % a.n_cut);
  const R dT = reinterpret_cast<const R*>(a.dT)[2 * o];
  const R dT1 = reinterpret_cast<const R*>(a.dT)[2 * o + 1];
  const unsigned long long us = a.ustep[2 * o], us1 = a.ustep[2 * o + 1];
  const bool same = !HALVES || us == us1;   // whole-record plans: always one |k|
  const T4* tab = reinterpret_cast<const T4*>(a.table);
  const long long orb = a.n_orb_pad;

  // chunk rotation against bank conflicts: the 8 threads of a quarter warp read
  // 8 different 16-byte bank groups.  Accumulator slot j holds member
  // ((j / MPC + rot) % NCH) * MPC + j % MPC.
  const int rot = (NCH == 2) ? ((tid >> 2) & 1) : (NCH == 4 ? ((tid >> 1) & 3) : 0);

  R acc[4][kFields], cmp[4][kFields];
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int k = 0; k < kFields; ++k) { acc[g][k] = (R)0; cmp[g][k] = (R)0; }

  int mf = m0;
  if (m0 == 0) {  // lag 0: rotate the current spectra, write the ring slot, use them directly
    C D[3][4];
    rotate_current(a, o, D);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      S::store(a.hist, ((long long)sn * 3 + c) * orb + o, a.slot_stride, D[c]);
      S::round(D[c]);
    }
    R w0[4], w1[4];
    lag_weights(tab, 0ull, dT * (R)0.5, w0);
    if constexpr (HALVES) {
      if (same) {
#pragma unroll
        for (int q = 0; q < 4; ++q) w1[q] = w0[q];
      } else {
        lag_weights(tab, 0ull, dT1 * (R)0.5, w1);
      }
    }
    C Dp[3][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < NCH; ++r)
        if (rot == r) {
#pragma unroll
          for (int c = 0; c < 3; ++c) Dp[c][j] = D[c][((j / MPC + r) % NCH) * MPC + j % MPC];
        }
    // slot j holds member ((j / MPC + rot) % NCH) MPC + j % MPC, of half member / 2
    if constexpr (!HALVES) {
      accumulate<KAHAN>(acc, cmp, w0, w0, Dp);
    } else
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool h1 = ((j / MPC + rot) % NCH) * MPC + j % MPC >= 2;
      R wj[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) wj[q] = h1 ? w1[q] : w0[q];
      const C dxi = Dp[0][j], d2 = Dp[1][j], dp = Dp[2][j];
      kadd<KAHAN>(acc[j][0], cmp[j][0], wj[0], dxi.x);
      kadd<KAHAN>(acc[j][1], cmp[j][1], wj[0], dxi.y);
      kadd<KAHAN>(acc[j][2], cmp[j][2], wj[2], dp.x);
      kadd<KAHAN>(acc[j][3], cmp[j][3], wj[2], dp.y);
      kadd<KAHAN>(acc[j][4], cmp[j][4], wj[1], d2.x);
      kadd<KAHAN>(acc[j][5], cmp[j][5], wj[1], d2.y);
      kadd<KAHAN>(acc[j][6], cmp[j][6], wj[3], d2.x);
      kadd<KAHAN>(acc[j][7], cmp[j][7], wj[3], d2.y);
      kadd<KAHAN>(acc[j][8], cmp[j][8], wj[3], dxi.x);
      kadd<KAHAN>(acc[j][9], cmp[j][9], wj[3], dxi.y);
    }
    mf = 1;
  }

  const int nst = (m1 - mf + KS - 1) / KS;
  if (nst > 0) {
    const unsigned char* hist = reinterpret_cast<const unsigned char*>(a.hist);
    const long long plane_bytes = a.slot_stride * S::kRecBytes;
    const unsigned char* wts = reinterpret_cast<const unsigned char*>(a.wts);
    const bool pre = WSEG > 0 && wts != nullptr;   // uniform over the CTA
    auto issue = [&](int s) {
      const int b = (int)((gstage + s) % NS);
      const int mb = mf + s * KS;
      const int kk = min(KS, m1 - mb);
      const unsigned bar = smem_addr(&full[b]);
      mbar_expect_tx(bar, (unsigned)(kk * (3 * S::kPlanes * SEG + (pre ? WSEG : 0))));
      for (int k = 0; k < kk; ++k) {
        int slot = sn - (mb + k);
        if (slot < 0) slot += a.n_cut;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int pl = 0; pl < S::kPlanes; ++pl) {
            const unsigned char* src =
                hist + pl * plane_bytes + (((long long)slot * 3 + c) * orb + tile0) * S::kRecBytes;
            const unsigned dst = smem_addr(smem + b * STAGE + ((k * 3 + c) * S::kPlanes + pl) * SEG);
            bulk_g2s(dst, src, SEG, bar);
          }
        if (pre)
          bulk_g2s(smem_addr(smem + b * STAGE + HIST + k * WSEG),
                   wts + ((long long)(mb + k) * orb + tile0) * 32, WSEG, bar);
      }
    };
    if (tid == 0)
      for (int s = 0; s < min(NS - 1, nst); ++s) issue(s);

    constexpr bool PF = PrefetchNodes<S, KAHAN, HALVES, NS, KS, MINB, TILE>::value;
    constexpr bool HP = PF && HALVES;   // half 1's nodes prefetched as well
    // weights of stage 0 (prefetching shapes)
    R wn[KS][4];
    R wn1[HP ? KS : 1][4];
    if constexpr (PF) if (!pre) {
      T4 nd[KS][4];
#pragma unroll
      for (int k = 0; k < KS; ++k)
        if (mf + k < m1) fetch_nodes(tab, (unsigned long long)(mf + k) * us, nd[k]);
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        if (mf + k < m1 && mf + k < lo) {
          interp_nodes(nd[k], (unsigned long long)(mf + k) * us, dT, wn[k]);
        } else {
          wn[k][0] = wn[k][1] = wn[k][2] = wn[k][3] = (R)0;
        }
      }
      if constexpr (HP) if (!same) {
#pragma unroll
        for (int k = 0; k < KS; ++k)
          if (mf + k < m1) fetch_nodes(tab, (unsigned long long)(mf + k) * us1, nd[k]);
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          if (mf + k < m1 && mf + k < lo1) {
            interp_nodes(nd[k], (unsigned long long)(mf + k) * us1, dT1, wn1[k]);
          } else {
            wn1[k][0] = wn1[k][1] = wn1[k][2] = wn1[k][3] = (R)0;
          }
        }
      }
    }

    bool ok = true;
    int done = 0;   // stages consumed
    for (int i = 0; i < nst; ++i) {
      // The CTA-wide vote makes the give-up decision uniform and certifies that
      // every thread has finished stage i-1, whose buffer is refilled next.
      const unsigned gi = gstage + i;
      const bool landed = mbar_wait(smem_addr(&full[gi % NS]), (gi / NS) & 1u, a.err);
      if (!__syncthreads_and(landed)) {
        ok = false;
        break;
      }
      if (tid == 0 && i + NS - 1 < nst) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(i + NS - 1);
      }
      done = i + 1;
      const int mb = mf + i * KS;
      const int kk = min(KS, m1 - mb);
      R w[KS][4];
      // table nodes of the next stage, in flight during this stage's arithmetic
      const int mn = mb + KS;
      T4 nd[PF ? KS : 1][4];
      T4 nd1[HP ? KS : 1][4];
      if constexpr (WSEG > 0) if (pre) {
        // precomputed weights from the stage; the two 16-byte halves are read in
        // an order that keeps a quarter warp on distinct bank groups
        const unsigned char* wst = smem + (gi % NS) * STAGE + HIST;
        const int h0 = (tid >> 2) & 1;
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          if (mb + k < m1 && mb + k < lo) {
            const double2 p0 = *reinterpret_cast<const double2*>(wst + k * WSEG + tid * 32 + h0 * 16);
            const double2 p1 = *reinterpret_cast<const double2*>(wst + k * WSEG + tid * 32 + (1 - h0) * 16);
            const double2 lo2 = h0 ? p1 : p0, hi2 = h0 ? p0 : p1;
            w[k][0] = lo2.x; w[k][1] = lo2.y; w[k][2] = hi2.x; w[k][3] = hi2.y;
          } else {
            w[k][0] = w[k][1] = w[k][2] = w[k][3] = (R)0;
          }
        }
      }
      if (pre) {
      } else if constexpr (PF) {
#pragma unroll
        for (int k = 0; k < KS; ++k)
#pragma unroll
          for (int q = 0; q < 4; ++q) w[k][q] = wn[k][q];
#pragma unroll
        for (int k = 0; k < KS; ++k)
          if (mn + k < m1) fetch_nodes(tab, (unsigned long long)(mn + k) * us, nd[k]);
      } else {
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          if (mb + k < m1 && mb + k < lo) {
            lag_weights(tab, (unsigned long long)(mb + k) * us, dT, w[k]);
          } else {
            w[k][0] = w[k][1] = w[k][2] = w[k][3] = (R)0;
          }
        }
      }

      // half 1's weights: half 0's when the record holds one |k|, else
      // interpolated here (half 0's are prefetched, precomputed or in place)
      R w1[KS][4];
      if constexpr (!HALVES) {
      } else if (same) {
#pragma unroll
        for (int k = 0; k < KS; ++k)
#pragma unroll
          for (int q = 0; q < 4; ++q) w1[k][q] = w[k][q];
      } else if constexpr (HP) {
#pragma unroll
        for (int k = 0; k < KS; ++k)
#pragma unroll
          for (int q = 0; q < 4; ++q) w1[k][q] = wn1[k][q];
#pragma unroll
        for (int k = 0; k < KS; ++k)
          if (mn + k < m1) fetch_nodes(tab, (unsigned long long)(mn + k) * us1, nd1[k]);
      } else {
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          if (mb + k < m1 && mb + k < lo1) {
            lag_weights(tab, (unsigned long long)(mb + k) * us1, dT1, w1[k]);
          } else {
            w1[k][0] = w1[k][1] = w1[k][2] = w1[k][3] = (R)0;
          }
        }
      }

      const unsigned char* stage = smem + (gi % NS) * STAGE;
#pragma unroll
      for (int r = 0; r < NCH; ++r) {
        const int ch = (r + rot) % NCH;
        // a chunk of <= 2 members lies in one half (ch MPC / 2); a 4-member
        // chunk spans both, selected per member below
        R wc[KS][4];
        if constexpr (MPC <= 2 && HALVES) {
          const bool h1 = ch * MPC >= 2;
#pragma unroll
          for (int k = 0; k < KS; ++k)
#pragma unroll
            for (int q = 0; q < 4; ++q) wc[k][q] = h1 ? w1[k][q] : w[k][q];
        }
        C D[KS][3][MPC];
#pragma unroll
        for (int k = 0; k < KS; ++k)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            if (k < kk) {
              S::chunk_smem(stage + (k * 3 + c) * S::kPlanes * SEG, SEG, tid, ch, D[k][c]);
            } else {
#pragma unroll
              for (int j = 0; j < MPC; ++j) D[k][c][j] = cmake<C>(0, 0);
            }
          }
#pragma unroll
        for (int j = 0; j < MPC; ++j) {
          const int g = r * MPC + j;
          // field -> (kernel, component): 11:xi, 33:perp, 22:2, 12:2, 12:xi (re, im)
          constexpr int kern[kFields] = {0, 0, 2, 2, 1, 1, 3, 3, 3, 3};
          constexpr int comp[kFields] = {0, 0, 2, 2, 1, 1, 1, 1, 0, 0};
          if constexpr (sizeof(R) == 4 && !std::is_same<S, dev::StoreF32>::value) {
            // BF16 history: (re, im) of one field share weight and value, one
            // two-lane op each (the issue-bound kernels gain 10-12 %; the FP32
            // kernels, HBM-bound, keep scalar FMAs, which their batched launch
            // measured faster with)
#pragma unroll
            for (int f = 0; f < kFields; f += 2) {
              float2 y = KAHAN ? make_float2(-cmp[g][f], -cmp[g][f + 1])
                               : make_float2(acc[g][f], acc[g][f + 1]);
#pragma unroll
              for (int k = 0; k < KS; ++k) {
                R wk;
                if constexpr (!HALVES) wk = w[k][kern[f]];
                else if constexpr (MPC <= 2) wk = wc[k][kern[f]];
                else wk = j < 2 ? w[k][kern[f]] : w1[k][kern[f]];
                y = fma2(make_float2(wk, wk), D[k][comp[f]][j], y);
              }
              if (KAHAN) {
                const float2 s = make_float2(acc[g][f], acc[g][f + 1]);
                const float2 t = add2(s, y);
                const float2 e = sub2(sub2(t, s), y);
                acc[g][f] = t.x;
                acc[g][f + 1] = t.y;
                cmp[g][f] = e.x;
                cmp[g][f + 1] = e.y;
              } else {
                acc[g][f] = y.x;
                acc[g][f + 1] = y.y;
              }
            }
          } else {
#pragma unroll
            for (int f = 0; f < kFields; ++f) {
              R y = KAHAN ? -cmp[g][f] : acc[g][f];
#pragma unroll
              for (int k = 0; k < KS; ++k) {
                const C d = D[k][comp[f]][j];
                R wk;
                if constexpr (!HALVES) wk = w[k][kern[f]];
                else if constexpr (MPC <= 2) wk = wc[k][kern[f]];
                else wk = j < 2 ? w[k][kern[f]] : w1[k][kern[f]];
                y = fma(wk, (f & 1) ? d.y : d.x, y);
              }
              if (KAHAN) {
                const R t = acc[g][f] + y;
                cmp[g][f] = (t - acc[g][f]) - y;
                acc[g][f] = t;
              } else {
                acc[g][f] = y;
              }
            }
          }
        }
      }
      if constexpr (PF) if (!pre) {
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          if (mn + k < m1 && mn + k < lo) {
            interp_nodes(nd[k], (unsigned long long)(mn + k) * us, dT, wn[k]);
          } else {
            wn[k][0] = wn[k][1] = wn[k][2] = wn[k][3] = (R)0;
          }
        }
        if constexpr (HP) if (!same) {
#pragma unroll
          for (int k = 0; k < KS; ++k) {
            if (mn + k < m1 && mn + k < lo1) {
              interp_nodes(nd1[k], (unsigned long long)(mn + k) * us1, dT1, wn1[k]);
            } else {
              wn1[k][0] = wn1[k][1] = wn1[k][2] = wn1[k][3] = (R)0;
            }
          }
        }
      }
    }
    if (!ok) {
      if (tid == 0) atomicExch(a.err, 1);
      // let the copies still in flight land before the CTA's shared memory is released
      const int issued = min(nst, done + NS - 1);
      for (int s = done; s < issued; ++s) {
        const unsigned gs = gstage + s;
        mbar_wait(smem_addr(&full[gs % NS]), (gs / NS) & 1u, &kNoError);
      }
      return false;
    }
    gstage += nst;
  }

  R* part = reinterpret_cast<R*>(a.part);
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const int member = (((g / MPC) + rot) % NCH) * MPC + g % MPC;
#pragma unroll
    for (int k = 0; k < kFields; ++k)
      part[((long long)chunk * (4 * kFields) + member * kFields + k) * orb + o] =
          KAHAN ? acc[g][k] - cmp[g][k] : acc[g][k];
  }
  return true;
}

template <int NS>
__device__ __forceinline__ void init_barriers(unsigned long long* full) {
  if (threadIdx.x == 0) {
#pragma unroll
    for (int b = 0; b < NS; ++b) mbar_init(smem_addr(&full[b]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// One CTA per (orbit tile, lag chunk) of one update.
template <class S, int KAHAN, int NS, int KS, int MINB, int TILE, bool HALVES>
__global__ void __launch_bounds__(TILE, MINB) conv_tma_kernel(const StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long full[NS];
  init_barriers<NS>(full);
  unsigned gstage = 0;
  conv_tma_item<S, KAHAN, NS, KS, MINB, TILE, HALVES>(a, blockIdx.x, blockIdx.y, smem, full, gstage);
}

// Persistent CTAs over the (update, tile, chunk) items of a batch of updates
// with ragged grids and history lengths: items are taken from *counter in
// order (item_prefix[s] .. item_prefix[s+1]-1 belong to update s, tile-major
// within each lag chunk).  Every item writes its own partial sums, so the
// result does not depend on which CTA ran it.
template <class S, int KAHAN, int NS, int KS, int MINB, int TILE, bool HALVES>
__global__ void __launch_bounds__(TILE, MINB)
conv_tma_batch_kernel(const StepArgs* __restrict__ args, const int* __restrict__ item_prefix,
                      int nb, int* counter) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long full[NS];
  __shared__ int s_item, s_tile, s_chunk;
  __shared__ StepArgs s_args;   // the item's update, read from shared memory (no registers)
  init_barriers<NS>(full);
  unsigned gstage = 0;
  const int total = item_prefix[nb];
  for (;;) {
    __syncthreads();   // the previous item's buffers and arguments are free
    if (threadIdx.x == 0) {
      const int it = atomicAdd(counter, 1);
      s_item = it;
      if (it < total) {
        int s = 0;
        while (s + 1 < nb && item_prefix[s + 1] <= it) ++s;
        s_args = args[s];
        const int tiles = s_args.n_orb_pad / TILE;
        const int local = it - item_prefix[s];
        s_tile = local % tiles;
        s_chunk = local / tiles;
      }
    }
    __syncthreads();
    if (s_item >= total) break;
    if (!conv_tma_item<S, KAHAN, NS, KS, MINB, TILE, HALVES>(s_args, s_tile, s_chunk, smem, full, gstage))
      return;
  }
}

// One CTA per (update, tile, chunk) item of a batch (the hardware block
// scheduler hands the items out; no work counter, and no barrier phases carried
// from item to item, so its register needs are those of the single-update
// kernel).  Same item order as the persistent kernel.
template <class S, int KAHAN, int NS, int KS, int MINB, int TILE, bool HALVES>
__global__ void __launch_bounds__(TILE, MINB)
conv_tma_items_kernel(const StepArgs* __restrict__ args, const int* __restrict__ item_prefix,
                      int nb) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long full[NS];
  __shared__ int s_tile, s_chunk;
  __shared__ StepArgs s_args;
  if (threadIdx.x == 0) {
    const int it = blockIdx.x;
    int s = 0;
    while (s + 1 < nb && item_prefix[s + 1] <= it) ++s;
    s_args = args[s];
    const int tiles = s_args.n_orb_pad / TILE;
    const int local = it - item_prefix[s];
    s_tile = local % tiles;
    s_chunk = local / tiles;
  }
  init_barriers<NS>(full);   // its __syncthreads publishes the item too
  unsigned gstage = 0;
  conv_tma_item<S, KAHAN, NS, KS, MINB, TILE, HALVES>(s_args, s_tile, s_chunk, smem, full, gstage);
}

// Launch one instantiation (sets the dynamic shared-memory attribute once).
// With `batch` set, launches over the batch's items instead: one CTA per item
// when `batch->items` > 0, else the persistent kernel on `batch->ctas` CTAs.
template <class S, int KAHAN, int NS, int KS, int MINB, int TILE, bool HALVES>
cudaError_t prepare_shape() {
  static bool attr_set = false;
  constexpr int bytes = smem_bytes<S, NS, KS, TILE>();
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(conv_tma_kernel<S, KAHAN, NS, KS, MINB, TILE, HALVES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(conv_tma_batch_kernel<S, KAHAN, NS, KS, MINB, TILE, HALVES>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(conv_tma_items_kernel<S, KAHAN, NS, KS, MINB, TILE, HALVES>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  return cudaSuccess;
}

// With `batch` null and `prepare_only` set, only sets the kernels' attributes.
template <class S, int KAHAN, int NS, int KS, int MINB, int TILE, bool HALVES>
cudaError_t launch_shape(const StepArgs& a, cudaStream_t st, const BatchLaunch* batch = nullptr,
                         bool prepare_only = false) {
  constexpr int bytes = smem_bytes<S, NS, KS, TILE>();
  const cudaError_t pe = prepare_shape<S, KAHAN, NS, KS, MINB, TILE, HALVES>();
  if (pe != cudaSuccess || prepare_only) return pe;
  if (batch && batch->items > 0) {
    conv_tma_items_kernel<S, KAHAN, NS, KS, MINB, TILE, HALVES><<<batch->items, TILE, bytes, st>>>(
        batch->args, batch->item_prefix, batch->nb);
  } else if (batch) {
    conv_tma_batch_kernel<S, KAHAN, NS, KS, MINB, TILE, HALVES><<<batch->ctas, TILE, bytes, st>>>(
        batch->args, batch->item_prefix, batch->nb, batch->counter);
  } else {
    if (a.n_orb_pad % TILE != 0) return cudaErrorInvalidValue;
    const dim3 grid(a.n_orb_pad / TILE, a.nchunks);
    conv_tma_kernel<S, KAHAN, NS, KS, MINB, TILE, HALVES><<<grid, TILE, bytes, st>>>(a);
  }
  return cudaGetLastError();
}

template <class S, int KAHAN, int NS, int KS, int MINB, int TILE>
cudaError_t launch_halves(bool halves, const StepArgs& a, cudaStream_t st,
                          const BatchLaunch* batch, bool prepare_only) {
  return halves ? launch_shape<S, KAHAN, NS, KS, MINB, TILE, true>(a, st, batch, prepare_only)
                : launch_shape<S, KAHAN, NS, KS, MINB, TILE, false>(a, st, batch, prepare_only);
}

// A pipeline shape (sized for 128-orbit tiles: MINB resident CTAs per SM) at the
// orbit tile `tile`, for records of one |k| or (halves) of two.
template <class S, int KAHAN, int NS, int KS, int MINB>
cudaError_t launch_tiles(int tile, bool halves, const StepArgs& a, cudaStream_t st,
                         const BatchLaunch* batch, bool prepare_only) {
  switch (tile) {
    case 64:
      return launch_halves<S, KAHAN, NS, KS, minb_for_tile(MINB, 64), 64>(halves, a, st, batch,
                                                                         prepare_only);
    case 128:
      return launch_halves<S, KAHAN, NS, KS, MINB, 128>(halves, a, st, batch, prepare_only);
    case 256:
      return launch_halves<S, KAHAN, NS, KS, minb_for_tile(MINB, 256), 256>(halves, a, st, batch,
                                                                           prepare_only);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace tma
}  // namespace sbim
