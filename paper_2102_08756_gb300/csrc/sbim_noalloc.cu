// sbim_spectral_response_noalloc: a handle-free evaluation of the non-local
// traction spectrum that allocates no device memory.
//
// Who needs it: a caller that is handed device buffers by a host framework and
// is not allowed to allocate (a solver running inside a fixed memory arena, a
// plugin whose device footprint must not change while its host time-steps)
// cannot use sbim_create, which allocates the history, tables and FFT plans.
// Here the caller owns the displacement-spectrum history and the output; the
// only working memory is g_noalloc_scratch below, a file-scope device array of
// kNoAllocScratchBytes that every GPU which loads this module keeps until the
// process exits.  It holds the interpolation table of the kernels (rebuilt when
// c_p/c_s changes or a longer table is needed) and the partial sums over lag
// chunks (fully overwritten by every call, so nothing must start at zero).
// All calls share the array: calls whose kernels overlap on the GPU (other
// streams, other host threads) race on it and must be serialised by the caller.
// The first call on a device resolves the array's device address and builds
// the table; make that call before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/sbim.h"
#include "sbim_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;     // 64 MiB per GPU
constexpr long long kTabMax = 1ll << 19;                 // table entries (h = 1/64)
constexpr size_t kTab64Off = 0;                          // double table: 16 MiB
constexpr size_t kTab32Off = kTab64Off + kTabMax * 32;   // float table: 8 MiB
constexpr size_t kGlOff = kTab32Off + kTabMax * 16;      // 32 Gauss-Legendre doubles
constexpr size_t kPartOff = kGlOff + 4096;               // chunk partials: the rest
constexpr size_t kPartBytes = kNoAllocScratchBytes - kPartOff;
constexpr int kFieldsNA = 16;                            // 8 complex sums per bin
constexpr int kTile = 128;
constexpr double kTabH = 1.0 / 64.0;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct DeviceState {
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch
  double eta = 0.0;
  long long tab_n = 0;
};
std::mutex g_mu;
DeviceState g_state[kMaxDevices];

int na_fail(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  sbim::set_last_error(buf);
  return code;
}

struct NAArgs {
  const float2* hist;   // [n_lags][3][nbins]
  float2* fhat;         // [3][nbins]
  const float4* table;  // entry j = node j - 1
  float* part;          // [nchunks][16][nbins]
  int n1, n3, nh, nbins, n_lags, lc, nchunks, side;
  double L1, L3, cs_dt, mu, eta;
};

struct BinGeom {
  float e11, e33, e13, c1, c3, muq;
  unsigned long long ustep;
  float dT;
};

__device__ BinGeom bin_geom(const NAArgs& a, int b) {
  const int j1 = b % a.nh, r3 = b / a.nh;
  const int j3 = r3 <= a.n3 / 2 ? r3 : r3 - a.n3;
  const double k1 = 6.283185307179586476925286766559 * j1 / a.L1;
  const double k3 = 6.283185307179586476925286766559 * j3 / a.L3;
  const double q = sqrt(k1 * k1 + k3 * k3);
  BinGeom g;
  const double qs = q > 0 ? q : 1.0;
  const double e1 = k1 / qs, e3 = k3 / qs;
  const bool ny1 = (j1 == a.n1 / 2), ny3 = (r3 == a.n3 / 2);
  g.e11 = (float)(e1 * e1);
  g.e33 = (float)(e3 * e3);
  g.e13 = (ny1 || ny3) ? 0.f : (float)(e1 * e3);   // odd in an aliased component
  g.c1 = ny1 ? 0.f : (float)e1;
  g.c3 = ny3 ? 0.f : (float)e3;
  g.muq = (float)(a.mu * q);
  const double dT = q * a.cs_dt;
  g.dT = (float)dT;
  g.ustep = __double2ull_rn(dT / kTabH * 4294967296.0);
  return g;
}

__device__ __forceinline__ void na_weights(const float4* __restrict__ tab, unsigned long long u,
                                           float scale, float w[4]) {
  const unsigned i = (unsigned)(u >> 32);
  const float t = (float)(unsigned)(u & 0xffffffffull) * 2.3283064365386962890625e-10f;
  const float tm1 = t - 1.f, tm2 = t - 2.f, tp1 = t + 1.f;
  const float sixth = scale * (1.f / 6.f), halfs = scale * 0.5f;
  const float l0 = -t * tm1 * tm2 * sixth, l1 = tp1 * tm1 * tm2 * halfs;
  const float l2 = -tp1 * t * tm2 * halfs, l3 = tp1 * t * tm1 * sixth;
  const float4 p = __ldg(tab + i), q = __ldg(tab + i + 1), r = __ldg(tab + i + 2), s = __ldg(tab + i + 3);
  w[0] = l0 * p.x + l1 * q.x + l2 * r.x + l3 * s.x;
  w[1] = l0 * p.y + l1 * q.y + l2 * r.y + l3 * s.y;
  w[2] = l0 * p.z + l1 * q.z + l2 * r.z + l3 * s.z;
  w[3] = l0 * p.w + l1 * q.w + l2 * r.w + l3 * s.w;
}

__device__ __forceinline__ void kahan(float& s, float& c, float w, float x) {
  const float y = fmaf(w, x, -c);
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Per bin and lag chunk: Z[a][c] = sum_m w_a(m) Uhat_c[n - m] for the Cartesian
// components the operator needs (11:1, 11:3, 33:1, 33:3, 22:2, 12:1, 12:2, 12:3).
__global__ void __launch_bounds__(kTile) noalloc_conv_kernel(const NAArgs a) {
  const int b = blockIdx.x * kTile + threadIdx.x;
  if (b >= a.nbins) return;
  const int chunk = blockIdx.y;
  const int m0 = chunk * a.lc, m1 = min(m0 + a.lc, a.n_lags);
  const BinGeom g = bin_geom(a, b);
  float s[kFieldsNA], c[kFieldsNA];
#pragma unroll
  for (int k = 0; k < kFieldsNA; ++k) { s[k] = 0.f; c[k] = 0.f; }
  unsigned long long u = (unsigned long long)m0 * g.ustep;
  for (int m = m0; m < m1; ++m, u += g.ustep) {
    float w[4];
    na_weights(a.table, u, m == 0 ? 0.5f * g.dT : g.dT, w);
    const float2* h = a.hist + (long long)m * 3 * a.nbins + b;
    const float2 u1 = h[0], u2 = h[a.nbins], u3 = h[2 * (long long)a.nbins];
    kahan(s[0], c[0], w[0], u1.x);  kahan(s[1], c[1], w[0], u1.y);    // H11 * U1
    kahan(s[2], c[2], w[0], u3.x);  kahan(s[3], c[3], w[0], u3.y);    // H11 * U3
    kahan(s[4], c[4], w[2], u1.x);  kahan(s[5], c[5], w[2], u1.y);    // H33 * U1
    kahan(s[6], c[6], w[2], u3.x);  kahan(s[7], c[7], w[2], u3.y);    // H33 * U3
    kahan(s[8], c[8], w[1], u2.x);  kahan(s[9], c[9], w[1], u2.y);    // H22 * U2
    kahan(s[10], c[10], w[3], u1.x); kahan(s[11], c[11], w[3], u1.y); // H12 * U1
    kahan(s[12], c[12], w[3], u2.x); kahan(s[13], c[13], w[3], u2.y); // H12 * U2
    kahan(s[14], c[14], w[3], u3.x); kahan(s[15], c[15], w[3], u3.y); // H12 * U3
  }
#pragma unroll
  for (int k = 0; k < kFieldsNA; ++k)
    a.part[((long long)chunk * kFieldsNA + k) * a.nbins + b] = s[k] - c[k];
}

// Sum the chunk partials in chunk order and assemble the Cartesian operator;
// the output is the unnormalised spectrum of s (the forward DFT of the field).
__global__ void __launch_bounds__(kTile) noalloc_assemble_kernel(const NAArgs a) {
  const int b = blockIdx.x * kTile + threadIdx.x;
  if (b >= a.nbins) return;
  const BinGeom g = bin_geom(a, b);
  float z[kFieldsNA];
#pragma unroll
  for (int k = 0; k < kFieldsNA; ++k) {
    float s = 0.f, c = 0.f;
    for (int ch = 0; ch < a.nchunks; ++ch) {
      const float x = a.part[((long long)ch * kFieldsNA + k) * a.nbins + b];
      const float y = x - c, t = s + y;
      c = (t - s) - y;
      s = t;
    }
    z[k] = s;
  }
  const float2 u1 = a.hist[b], u2 = a.hist[a.nbins + b], u3 = a.hist[2 * (long long)a.nbins + b];
  const float sd = (float)a.side, inst = (float)(2.0 - a.eta), mq = g.muq;
  // -side mu q [e e^T (H11*U_h) + e_perp e_perp^T (H33*U_h)]
  const float d1r = g.e11 * z[0] + g.e13 * z[2] + g.e33 * z[4] - g.e13 * z[6];
  const float d1i = g.e11 * z[1] + g.e13 * z[3] + g.e33 * z[5] - g.e13 * z[7];
  const float d3r = g.e13 * z[0] + g.e33 * z[2] - g.e13 * z[4] + g.e11 * z[6];
  const float d3i = g.e13 * z[1] + g.e33 * z[3] - g.e13 * z[5] + g.e11 * z[7];
  // in-plane coupling terms
  const float p2r = inst * u2.x + z[12], p2i = inst * u2.y + z[13];
  const float p1r = inst * u1.x + z[10], p1i = inst * u1.y + z[11];
  const float p3r = inst * u3.x + z[14], p3i = inst * u3.y + z[15];
  float2 f1, f2, f3;
  f1.x = mq * (-sd * d1r - g.c1 * p2i);
  f1.y = mq * (-sd * d1i + g.c1 * p2r);
  f3.x = mq * (-sd * d3r - g.c3 * p2i);
  f3.y = mq * (-sd * d3i + g.c3 * p2r);
  const float cr = g.c1 * p1r + g.c3 * p3r, ci = g.c1 * p1i + g.c3 * p3i;
  f2.x = mq * (ci - sd * z[8]);
  f2.y = mq * (-cr - sd * z[9]);
  a.fhat[b] = f1;
  a.fhat[a.nbins + b] = f2;
  a.fhat[2 * (long long)a.nbins + b] = f3;
}

void gl16(double* x, double* w) {
  const double pi = 3.141592653589793238462643383279502884;
  for (int i = 0; i < 16; ++i) {
    double z = std::cos(pi * (i + 0.75) / 16.5), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= 16; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = 16.0 * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// The kernels read and write the spectra as float2: a pointer that is not
// 8-byte aligned, or one the device cannot reach, would fault the caller's
// context.  Accept device memory of the current device and managed memory.
int check_spectrum_pointer(const void* p, const char* what, int dev) {
  if ((uintptr_t)p % alignof(float2) != 0)
    return na_fail(SBIM_ERR_ARG, "%s is not %zu-byte aligned", what, alignof(float2));
  cudaPointerAttributes at;
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return na_fail(SBIM_ERR_ARG, "%s: cudaPointerGetAttributes: %s", what, cudaGetErrorString(e));
  }
  if (at.type == cudaMemoryTypeManaged) return SBIM_OK;
  if (at.type != cudaMemoryTypeDevice)
    return na_fail(SBIM_ERR_ARG, "%s is not device memory", what);
  if (at.device != dev)
    return na_fail(SBIM_ERR_ARG, "%s belongs to device %d, the current device is %d", what,
                   at.device, dev);
  return SBIM_OK;
}

}  // namespace

extern "C" int sbim_spectral_response_noalloc(int n1, int n3, double L1, double L3, double cs,
                                              double cp, double rho, double dt, int side,
                                              int n_lags, const void* uhat_hist, void* fhat,
                                              void* stream) {
  sbim::set_last_error("");
  if (n1 < 2 || n3 < 2 || (n1 & 1) || (n3 & 1))
    return na_fail(SBIM_ERR_ARG, "n1 and n3 must be even and >= 2");
  if (!(L1 > 0) || !(L3 > 0) || !(dt > 0) || !(rho > 0) || !(cs > 0) || !(cp > cs))
    return na_fail(SBIM_ERR_ARG, "need L1, L3, dt, rho, cs > 0 and cp > cs");
  if (side != 1 && side != -1) return na_fail(SBIM_ERR_ARG, "side must be +1 or -1");
  if (n_lags < 1) return na_fail(SBIM_ERR_ARG, "n_lags must be >= 1");
  if (!uhat_hist || !fhat) return na_fail(SBIM_ERR_ARG, "NULL spectrum pointer");
  const int nh = n1 / 2 + 1;
  const long long nbins = (long long)n3 * nh;
  const size_t per_chunk = (size_t)kFieldsNA * sizeof(float) * nbins;
  if (per_chunk > kPartBytes)
    return na_fail(SBIM_ERR_ARG,
                   "grid too large for the %zu-byte static scratch: n3 (n1/2+1) = %lld bins, "
                   "at most %zu", kNoAllocScratchBytes, nbins, kPartBytes / (kFieldsNA * sizeof(float)));
  const double eta = cp / cs;
  const double pi = 3.141592653589793238462643383279502884;
  const double kmax = 2.0 * pi * std::sqrt(std::pow(0.5 * n1 / L1, 2) + std::pow(0.5 * n3 / L3, 2));
  const double t_max = kmax * cs * dt * (n_lags - 1);
  const long long tab_need = (long long)std::floor(t_max / kTabH) + 6;
  if (tab_need > kTabMax)
    return na_fail(SBIM_ERR_ARG,
                   "history too long for the static kernel table: |k|max c_s dt (n_lags - 1) = "
                   "%.1f exceeds %.1f", t_max, (kTabMax - 6) * kTabH);

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(SBIM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev >= kMaxDevices) return na_fail(SBIM_ERR_ARG, "device index %d not supported", dev);
  int rc = check_spectrum_pointer(uhat_hist, "uhat_hist", dev);
  if (rc == SBIM_OK) rc = check_spectrum_pointer(fhat, "fhat", dev);
  if (rc != SBIM_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;

  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState& ds = g_state[dev];
  if (!ds.base) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess)
      return na_fail(SBIM_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    ds.base = (unsigned char*)ptr;
  }
  if (ds.eta != eta || ds.tab_n < tab_need) {
    double gl[32];
    gl16(gl, gl + 16);
    e = cudaMemcpyAsync(ds.base + kGlOff, gl, sizeof gl, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = sbim::launch_table_build((double*)(ds.base + kTab64Off), (float*)(ds.base + kTab32Off),
                                   tab_need, kTabH, eta, (const double*)(ds.base + kGlOff),
                                   (const double*)(ds.base + kGlOff) + 16, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // gl[] leaves scope
    if (e != cudaSuccess) {
      ds.eta = 0.0;
      ds.tab_n = 0;
      return na_fail(SBIM_ERR_CUDA, "kernel table build: %s", cudaGetErrorString(e));
    }
    ds.eta = eta;
    ds.tab_n = tab_need;
  }

  NAArgs a;
  a.hist = (const float2*)uhat_hist;
  a.fhat = (float2*)fhat;
  a.table = (const float4*)(ds.base + kTab32Off);
  a.part = (float*)(ds.base + kPartOff);
  a.n1 = n1; a.n3 = n3; a.nh = nh; a.nbins = (int)nbins; a.n_lags = n_lags; a.side = side;
  a.L1 = L1; a.L3 = L3; a.cs_dt = cs * dt; a.mu = rho * cs * cs; a.eta = eta;
  long long chunks = (long long)(kPartBytes / per_chunk);
  if (chunks > 16) chunks = 16;
  if (chunks > n_lags) chunks = n_lags;
  a.lc = (int)((n_lags + chunks - 1) / chunks);
  a.nchunks = (n_lags + a.lc - 1) / a.lc;
  const dim3 grid((unsigned)((nbins + kTile - 1) / kTile), (unsigned)a.nchunks);
  noalloc_conv_kernel<<<grid, kTile, 0, st>>>(a);
  noalloc_assemble_kernel<<<grid.x, kTile, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(SBIM_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
  return SBIM_OK;
}
