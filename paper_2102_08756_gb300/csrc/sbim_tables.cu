// FP64 device quadrature of the half-space convolution kernels (Section 2.3:
// the elastodynamic kernels of the independent formulation, whose formulas the
// paper defers to its references and which are derived from half-space
// elastodynamics).
//
// For T >= 0 the kernels are cosine / sine transforms of compactly supported
// real-axis densities (upper half-space, eta = c_p / c_s):
//   H_aa(T) = (2/pi) int_0^eta R_aa(y) cos(y T) dy,  a = 1, 2, 3
//   H_12(T) = (2/pi) int_1^eta X_12(y) sin(y T) dy
// with, on 0 <= y <= 1 (a = sqrt(1 - y^2/eta^2), b = sqrt(1 - y^2),
// D = 1 + (1 - y^2)/eta^2):
//   R_11 = a (1 + a b) / D,  R_22 = b (1 + a b) / D,  R_33 = b,
// and on 1 < y <= eta (A = sqrt(1 - y^2/eta^2), B = sqrt(y^2 - 1)):
//   R_11 = A y^2 / (1 + A^2 B^2),  R_22 = -A B^2 y^2 / (1 + A^2 B^2),
//   X_12 = A B y^2 / (1 + A^2 B^2).
// The square-root end points are removed by y = sin(theta) on [0, 1] and
// y = 1 + (eta - 1) sin^2(phi) on [1, eta]; each mapped interval is integrated
// by 16-point Gauss-Legendre panels with at most 6 rad of phase y T per panel.
#include "sbim_internal.cuh"

namespace sbim {

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

__global__ void table_kernel(double* __restrict__ out64, float* __restrict__ out32,
                             long long n, double h, double eta,
                             const double* __restrict__ glx, const double* __restrict__ glw) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const long long j = idx - 1;                 // entry idx holds node j = idx - 1
  const double T = fabs((double)j) * h;
  const double half_pi = 0.5 * kPi;
  const double inv_eta2 = 1.0 / (eta * eta);

  double h11 = 0.0, h22 = 0.0, h33 = 0.0, h12 = 0.0;

  // y = sin(theta), theta in [0, pi/2]
  {
    const int panels = (int)ceil(T * half_pi / 6.0) + 4;
    const double hw = 0.5 * half_pi / panels;
    for (int p = 0; p < panels; ++p) {
      const double mid = (2 * p + 1) * hw;
      for (int k = 0; k < 16; ++k) {
        const double th = mid + hw * glx[k];
        const double w = hw * glw[k];
        double y, b;
        sincos(th, &y, &b);
        const double a = sqrt(1.0 - y * y * inv_eta2);
        const double D = 1.0 + (1.0 - y * y) * inv_eta2;
        const double c = cos(y * T) * w * b;   // b = dy/dtheta
        const double g = (1.0 + a * b) / D;
        h11 += a * g * c;
        h22 += b * g * c;
        h33 += b * c;
      }
    }
  }
  // y = 1 + (eta - 1) sin^2(phi), phi in [0, pi/2]
  {
    const double em1 = eta - 1.0;
    const double sq = sqrt(em1);
    const int panels = (int)ceil(T * em1 * half_pi / 6.0) + 4;
    const double hw = 0.5 * half_pi / panels;
    for (int p = 0; p < panels; ++p) {
      const double mid = (2 * p + 1) * hw;
      for (int k = 0; k < 16; ++k) {
        const double ph = mid + hw * glx[k];
        const double w = hw * glw[k];
        double s, c;
        sincos(ph, &s, &c);
        const double y = 1.0 + em1 * s * s;
        const double B = sq * s * sqrt(y + 1.0);
        const double A = sq * c * sqrt(eta + y) / eta;
        const double jac = 2.0 * em1 * s * c;   // dy/dphi
        const double f = A * y * y / (1.0 + A * A * B * B) * jac * w;
        double sn, cs;
        sincos(y * T, &sn, &cs);
        h11 += f * cs;
        h22 -= f * B * B * cs;
        h12 += f * B * sn;
      }
    }
  }
  const double s = 2.0 / kPi;
  h11 *= s; h22 *= s; h33 *= s; h12 *= s;
  if (j < 0) h12 = -h12;                        // H12 is odd in T, the others even
  out64[4 * idx + 0] = h11;
  out64[4 * idx + 1] = h22;
  out64[4 * idx + 2] = h33;
  out64[4 * idx + 3] = h12;
  if (out32) {
    out32[4 * idx + 0] = (float)h11;
    out32[4 * idx + 1] = (float)h22;
    out32[4 * idx + 2] = (float)h33;
    out32[4 * idx + 3] = (float)h12;
  }
}

}  // namespace

cudaError_t launch_table_build(double* out64, float* out32, long long n, double h,
                               double eta, const double* gl_x, const double* gl_w,
                               cudaStream_t s) {
  const int threads = 128;
  const long long blocks = (n + threads - 1) / threads;
  table_kernel<<<(unsigned)blocks, threads, 0, s>>>(out64, out32, n, h, eta, gl_x, gl_w);
  return cudaGetLastError();
}

}  // namespace sbim
