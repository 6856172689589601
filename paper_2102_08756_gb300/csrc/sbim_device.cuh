// Device helpers shared by the convolution kernels (Section 2.3: history
// storage, convolution weights, rotation into the (xi, 2, perp) frame).
#pragma once

#include <cuda_bf16.h>

#include "sbim_internal.cuh"

namespace sbim {
namespace dev {

struct alignas(32) Double4 {
  double x, y, z, w;
};

template <class C> struct RealOf;
template <> struct RealOf<float2> { using type = float; };
template <> struct RealOf<double2> { using type = double; };

__device__ __forceinline__ float4 ld_tab(const float4* p) { return __ldg(p); }
__device__ __forceinline__ Double4 ld_tab(const Double4* p) {
  const double2 lo = __ldg(reinterpret_cast<const double2*>(p));
  const double2 hi = __ldg(reinterpret_cast<const double2*>(p) + 1);
  Double4 r;
  r.x = lo.x; r.y = lo.y; r.z = hi.x; r.w = hi.y;
  return r;
}

// ----------------------------------------------------------------------------
// History storage policies.  A record is the 4 members of one (slot,
// component, orbit): 32 B as float2, 64 B as double2, 16 B per bf16 plane.
// ----------------------------------------------------------------------------
struct StoreF32 {
  using real = float;
  using cplx = float2;
  using tab4 = float4;
  static constexpr int kRecBytes = 32, kPlanes = 1, kChunks = 2, kChunkMembers = 2;
  // 16-byte chunk r of thread t's record in a staged shared-memory segment
  __device__ static void chunk_smem(const unsigned char* seg, int, int t, int r, cplx* out) {
    const float4 v = *reinterpret_cast<const float4*>(seg + t * kRecBytes + r * 16);
    out[0] = make_float2(v.x, v.y);
    out[1] = make_float2(v.z, v.w);
  }
  __device__ static void load(const void* h, long long rec, long long, cplx D[4]) {
    const float4* p = reinterpret_cast<const float4*>(h) + rec * 2;
    const float4 a = __ldcs(p), b = __ldcs(p + 1);
    D[0] = make_float2(a.x, a.y); D[1] = make_float2(a.z, a.w);
    D[2] = make_float2(b.x, b.y); D[3] = make_float2(b.z, b.w);
  }
  __device__ static void store(void* h, long long rec, long long, const cplx D[4]) {
    float4* p = reinterpret_cast<float4*>(h) + rec * 2;
    __stcs(p, make_float4(D[0].x, D[0].y, D[1].x, D[1].y));
    __stcs(p + 1, make_float4(D[2].x, D[2].y, D[3].x, D[3].y));
  }
  __device__ static void round(cplx*) {}
};

struct StoreF64 {
  using real = double;
  using cplx = double2;
  using tab4 = Double4;
  static constexpr int kRecBytes = 64, kPlanes = 1, kChunks = 4, kChunkMembers = 1;
  __device__ static void chunk_smem(const unsigned char* seg, int, int t, int r, cplx* out) {
    out[0] = *reinterpret_cast<const double2*>(seg + t * kRecBytes + r * 16);
  }
  __device__ static void load(const void* h, long long rec, long long, cplx D[4]) {
    const double2* p = reinterpret_cast<const double2*>(h) + rec * 4;
#pragma unroll
    for (int g = 0; g < 4; ++g) D[g] = __ldcs(p + g);
  }
  __device__ static void store(void* h, long long rec, long long, const cplx D[4]) {
    double2* p = reinterpret_cast<double2*>(h) + rec * 4;
#pragma unroll
    for (int g = 0; g < 4; ++g) __stcs(p + g, D[g]);
  }
  __device__ static void round(cplx*) {}
};

__device__ __forceinline__ unsigned pack_bf16(float re, float im) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(re, im);
  return *reinterpret_cast<const unsigned*>(&v);
}
__device__ __forceinline__ float2 unpack_bf16(unsigned w) {
  const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&w);
  return __bfloat1622float2(v);
}

// bf16 hi plane, plus a bf16 lo plane holding x - hi (LO = true).
template <bool LO>
struct StoreBF16 {
  using real = float;
  using cplx = float2;
  using tab4 = float4;
  static constexpr int kRecBytes = 16, kPlanes = LO ? 2 : 1, kChunks = 1, kChunkMembers = 4;
  __device__ static void chunk_smem(const unsigned char* seg, int plane_bytes, int t, int,
                                    cplx* out) {
    const uint4 hi = *reinterpret_cast<const uint4*>(seg + t * kRecBytes);
    out[0] = unpack_bf16(hi.x); out[1] = unpack_bf16(hi.y);
    out[2] = unpack_bf16(hi.z); out[3] = unpack_bf16(hi.w);
    if (LO) {
      const uint4 lo = *reinterpret_cast<const uint4*>(seg + plane_bytes + t * kRecBytes);
      const float2 l0 = unpack_bf16(lo.x), l1 = unpack_bf16(lo.y);
      const float2 l2 = unpack_bf16(lo.z), l3 = unpack_bf16(lo.w);
      out[0].x += l0.x; out[0].y += l0.y; out[1].x += l1.x; out[1].y += l1.y;
      out[2].x += l2.x; out[2].y += l2.y; out[3].x += l3.x; out[3].y += l3.y;
    }
  }
  __device__ static void load(const void* h, long long rec, long long plane, cplx D[4]) {
    const uint4* p = reinterpret_cast<const uint4*>(h) + rec;
    const uint4 hi = __ldcs(p);
    D[0] = unpack_bf16(hi.x); D[1] = unpack_bf16(hi.y);
    D[2] = unpack_bf16(hi.z); D[3] = unpack_bf16(hi.w);
    if (LO) {
      const uint4 lo = __ldcs(p + plane);
      const float2 l0 = unpack_bf16(lo.x), l1 = unpack_bf16(lo.y);
      const float2 l2 = unpack_bf16(lo.z), l3 = unpack_bf16(lo.w);
      D[0].x += l0.x; D[0].y += l0.y; D[1].x += l1.x; D[1].y += l1.y;
      D[2].x += l2.x; D[2].y += l2.y; D[3].x += l3.x; D[3].y += l3.y;
    }
  }
  __device__ static void split(const cplx D[4], uint4& hi, uint4& lo) {
    unsigned hw[4], lw[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      hw[g] = pack_bf16(D[g].x, D[g].y);
      const float2 hv = unpack_bf16(hw[g]);
      lw[g] = pack_bf16(D[g].x - hv.x, D[g].y - hv.y);
    }
    hi = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    lo = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
  __device__ static void store(void* h, long long rec, long long plane, const cplx D[4]) {
    uint4 hi, lo;
    split(D, hi, lo);
    uint4* p = reinterpret_cast<uint4*>(h) + rec;
    __stcs(p, hi);
    if (LO) __stcs(p + plane, lo);
  }
  __device__ static void round(cplx D[4]) {
    uint4 hi, lo;
    split(D, hi, lo);
    const unsigned hw[4] = {hi.x, hi.y, hi.z, hi.w};
    const unsigned lw[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      D[g] = unpack_bf16(hw[g]);
      if (LO) {
        const float2 l = unpack_bf16(lw[g]);
        D[g].x += l.x;
        D[g].y += l.y;
      }
    }
  }
};

// ----------------------------------------------------------------------------
// Convolution weights at lag m of one orbit: cubic Lagrange interpolation of the
// tabulated kernels at T = m dT.  u = m dT / h in 32.32 fixed point; table entry
// j holds node j - 1, so nodes i-1 .. i+2 are entries i .. i+3.
// ----------------------------------------------------------------------------
template <class R, class T4>
__device__ __forceinline__ void lag_weights(const T4* __restrict__ tab, unsigned long long u,
                                            R scale, R w[4]) {
  const unsigned i = (unsigned)(u >> 32);
  const R t = (R)(unsigned)(u & 0xffffffffull) * (R)2.3283064365386962890625e-10;
  const R tm1 = t - (R)1, tm2 = t - (R)2, tp1 = t + (R)1;
  const R sixth = scale * (R)(1.0 / 6.0), halfs = scale * (R)0.5;
  const R l0 = -t * tm1 * tm2 * sixth;
  const R l1 = tp1 * tm1 * tm2 * halfs;
  const R l2 = -tp1 * t * tm2 * halfs;
  const R l3 = tp1 * t * tm1 * sixth;
  const T4 a = ld_tab(tab + i), b = ld_tab(tab + i + 1), c = ld_tab(tab + i + 2), d = ld_tab(tab + i + 3);
  w[0] = l0 * a.x + l1 * b.x + l2 * c.x + l3 * d.x;
  w[1] = l0 * a.y + l1 * b.y + l2 * c.y + l3 * d.y;
  w[2] = l0 * a.z + l1 * b.z + l2 * c.z + l3 * d.z;
  w[3] = l0 * a.w + l1 * b.w + l2 * c.w + l3 * d.w;
}

// Two-lane float arithmetic of the sm_100 family: one instruction applies the
// same operation to both halves of a (re, im) pair, each rounded as the scalar
// instruction rounds it.
__device__ __forceinline__ unsigned long long pack2(float2 v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pack2(a)), "l"(pack2(b)), "l"(pack2(c)));
  return unpack2(d);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack2(a)), "l"(pack2(b)));
  return unpack2(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack2(a)), "l"(pack2(b)));
  return unpack2(d);
}

template <int KAHAN, class R>
__device__ __forceinline__ void kadd(R& s, R& c, R w, R x) {
  if (KAHAN) {
    const R y = fma(w, x, -c);
    const R t = s + y;
    c = (t - s) - y;
    s = t;
  } else {
    s = fma(w, x, s);
  }
}

// acc[g][*] += weights (11, 22, 33, 12) applied to member g's (xi, 2, perp)
// values; members 0, 1 (half 0 of the record) take w0, members 2, 3 take w1.
template <int KAHAN, class R, class C>
__device__ __forceinline__ void accumulate(R (&acc)[4][kFields], R (&cmp)[4][kFields],
                                           const R w0[4], const R w1[4], const C (&D)[3][4]) {
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const R* w = g < 2 ? w0 : w1;
    const C dxi = D[0][g], d2 = D[1][g], dp = D[2][g];
    kadd<KAHAN>(acc[g][0], cmp[g][0], w[0], dxi.x);
    kadd<KAHAN>(acc[g][1], cmp[g][1], w[0], dxi.y);
    kadd<KAHAN>(acc[g][2], cmp[g][2], w[2], dp.x);
    kadd<KAHAN>(acc[g][3], cmp[g][3], w[2], dp.y);
    kadd<KAHAN>(acc[g][4], cmp[g][4], w[1], d2.x);
    kadd<KAHAN>(acc[g][5], cmp[g][5], w[1], d2.y);
    kadd<KAHAN>(acc[g][6], cmp[g][6], w[3], d2.x);
    kadd<KAHAN>(acc[g][7], cmp[g][7], w[3], d2.y);
    kadd<KAHAN>(acc[g][8], cmp[g][8], w[3], dxi.x);
    kadd<KAHAN>(acc[g][9], cmp[g][9], w[3], dxi.y);
  }
}

template <class C> __device__ __forceinline__ C cmake(double re, double im);
template <> __device__ __forceinline__ float2 cmake<float2>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <> __device__ __forceinline__ double2 cmake<double2>(double re, double im) {
  return make_double2(re, im);
}

// Current spectra of the orbit's members rotated into (xi, 2, perp).
template <class C>
__device__ __forceinline__ void rotate_current(const StepArgs& a, int o, C (&D)[3][4]) {
  using R = typename RealOf<C>::type;
  const C* uh = reinterpret_cast<const C*>(a.uhat);
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const int b = a.bin[o * 4 + g];
    if (b >= 0) {
      const C e = reinterpret_cast<const C*>(a.dir)[o * 4 + g];
      const R e1 = e.x, e3 = e.y;
      const C u1 = uh[b], u2 = uh[a.nbins + b], u3 = uh[2 * (long long)a.nbins + b];
      D[0][g].x = e1 * u1.x + e3 * u3.x;  D[0][g].y = e1 * u1.y + e3 * u3.y;
      D[1][g] = u2;
      D[2][g].x = -e3 * u1.x + e1 * u3.x; D[2][g].y = -e3 * u1.y + e1 * u3.y;
    } else {
      D[0][g] = cmake<C>(0, 0); D[1][g] = cmake<C>(0, 0); D[2][g] = cmake<C>(0, 0);
    }
  }
}

}  // namespace dev
}  // namespace sbim
