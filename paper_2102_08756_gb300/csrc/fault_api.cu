// Pure-SBIM planar fault solver: a slip-weakening fault (Section 2.1,
// Eq. (slipweak)) between two identical elastic half-spaces, each represented
// only by its boundary through Eq. (SBI).  The TPV3 benchmark of Section 3 has
// no off-fault nonlinearity, so this boundary-only solver is the reference the
// hybrid scheme is checked against.  One sbim_fault_step enqueues on the
// handle's stream the predictor-corrector of Lapusta et al. (2000):
//   (1) u* = u_n + dt v_n                                      (predict_kernel)
//   (2) solve at u* -> v*                                      (solve, below)
//   (3) u_{n+1} = u_n + dt (v_n + v*)/2                        (correct_kernel)
//   (4) solve at u_{n+1} -> v_{n+1}, re-evaluating the predictor's level: the
//       history sums over lags >= 1 are the predictor's (sbim_step_repeat)
// where one solve is: the non-local tractions S+- of the upper (side +1) and
// lower (side -1) half-spaces, radiation term left out (sbim_step x 2), then
// one traction on both faces, tau = S+ - z v+ = S- + z v-, equal normal
// velocities, stick/slip on the shear vector, v+- = vbar +- V/2 (solve_kernel).
// The one-evaluation explicit update u_{n+1} = u_n + dt v_n is unstable at the
// highest modes; the corrector makes the scheme stable and second order.
// With symmetric = 1 (the symmetry-plane reduction used for TPV3 in Section 3)
// the lower face is the mirror image of the upper one and only the upper
// half-space is evaluated: S-_1,3 = S+_1,3, S-_2 = -S+_2.
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/sbim.h"
#include "sbim_internal.cuh"

struct sbim_fault_ctx {
  int n1 = 0, n3 = 0, prec = SBIM_FP32, symmetric = 0;
  double cs = 0, cp = 0, rho = 0, dt = 0;
  cudaStream_t stream = nullptr;
  sbim_handle up = nullptr, lo = nullptr;
  void* u = nullptr;         // [2][3][n3][n1]: face 0 upper (+), face 1 lower (-)
  void* v = nullptr;
  void* u_pred = nullptr;    // [2][3][n3][n1] predictor displacement
  void* v_pred = nullptr;    // [2][3][n3][n1] predictor velocity
  void* s_up = nullptr;      // [3][n3][n1] non-local tractions
  void* s_lo = nullptr;
  void* zero = nullptr;      // [3][n3][n1] zero velocity for the SBIM calls
  void* mu_s = nullptr;      // [n3][n1]
  void* tau0 = nullptr;      // [n3][n1]
  void* traction = nullptr;  // [3][n3][n1] fault traction perturbation of the last step
  void* rate = nullptr;      // [3][n3][n1] slip rate of the last step
  double mu_k = 0, Dc = 1, sigma0 = 0;
  bool have_law = false;
  long long n = 0;
  size_t rs = 4;
  long long plane() const { return (long long)n1 * n3; }
};

namespace {

int ffail(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  sbim::set_last_error(buf);
  return code;
}

#define FCU(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return ffail(e_ == cudaErrorMemoryAllocation ? SBIM_ERR_OOM : SBIM_ERR_CUDA,   \
                   "%s: %s", #call, cudaGetErrorString(e_));                        \
  } while (0)

constexpr int kThreads = 256;

// Mirror image across x2 = 0 of component c of a face field: 1 and 3 flip.
template <class R>
__device__ __forceinline__ R mirror(R x, int c) {
  return c == 1 ? x : -x;
}

// Step (1): u* = u + dt v; the symmetric solver keeps the lower face at the
// mirror image of the upper one.
template <class R, bool SYM>
__global__ void predict_kernel(const R* __restrict__ u, const R* __restrict__ v,
                               R* __restrict__ out, long long plane, R dt) {
  const long long face = 3 * plane;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < face;
       i += (long long)gridDim.x * blockDim.x) {
    const R up = u[i] + dt * v[i];
    out[i] = up;
    out[face + i] = SYM ? mirror(up, (int)(i / plane)) : u[face + i] + dt * v[face + i];
  }
}

// Step (3): u += dt (v + v*)/2, in place.
template <class R, bool SYM>
__global__ void correct_kernel(R* __restrict__ u, const R* __restrict__ v,
                               const R* __restrict__ vp, long long plane, R dt) {
  const long long face = 3 * plane;
  const R h = (R)0.5 * dt;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < face;
       i += (long long)gridDim.x * blockDim.x) {
    const R up = u[i] + h * (v[i] + vp[i]);
    u[i] = up;
    u[face + i] = SYM ? mirror(up, (int)(i / plane)) : u[face + i] + h * (v[face + i] + vp[face + i]);
  }
}

template <class R>
struct Law {
  const R* mu_s;
  const R* tau0;
  R mu_k, Dc, sigma0;
  int weld;
};

// The solve at one fault node: traction continuity through the radiation
// impedances z = (mu/c_s)(1, c_p/c_s, 1), stick/slip on the shear vector.
template <class R, bool SYM>
__global__ void solve_kernel(const R* __restrict__ u, R* __restrict__ v, const R* __restrict__ s_up,
                             const R* __restrict__ s_lo, R* __restrict__ traction,
                             R* __restrict__ rate, Law<R> law, long long plane, R z_s, R z_p) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= plane) return;
  const long long face = 3 * plane;
  R stick[3], vbar[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R a = s_up[c * plane + q];
    const R b = SYM ? (c == 1 ? -a : a) : s_lo[c * plane + q];
    const R z = c == 1 ? z_p : z_s;
    stick[c] = (R)0.5 * (a + b);
    vbar[c] = (a - b) / ((R)2 * z);
  }
  R tau[3] = {stick[0], stick[1], stick[2]};
  if (!law.weld) {
    const R d1 = u[q] - u[face + q];
    const R d3 = u[2 * plane + q] - u[face + 2 * plane + q];
    const R slip = sqrt(d1 * d1 + d3 * d3);
    const R mus = law.mu_s[q];
    const R fric = slip < law.Dc ? mus - (mus - law.mu_k) * slip / law.Dc : law.mu_k;
    const R strength = (law.sigma0 - stick[1]) * fric;
    const R t1 = law.tau0[q] + stick[0], t3 = stick[2];
    const R mag = sqrt(t1 * t1 + t3 * t3);
    if (mag > strength) {
      const R s = strength / mag;
      tau[0] = t1 * s - law.tau0[q];
      tau[2] = t3 * s;
    }
  }
  const R V[3] = {(R)2 * (stick[0] - tau[0]) / z_s, (R)0, (R)2 * (stick[2] - tau[2]) / z_s};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long long o = c * plane + q;
    v[o] = vbar[c] + (R)0.5 * V[c];
    v[face + o] = vbar[c] - (R)0.5 * V[c];
    traction[o] = tau[c];
    rate[o] = V[c];
  }
}

// slip u+ - u- of the current state
template <class R>
__global__ void slip_kernel(const R* __restrict__ u, R* __restrict__ slip, long long plane) {
  const long long face = 3 * plane;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < face;
       i += (long long)gridDim.x * blockDim.x)
    slip[i] = u[i] - u[face + i];
}

// lower face := mirror image of the upper face (symmetric solver, set_state)
template <class R>
__global__ void mirror_kernel(R* __restrict__ x, long long plane) {
  const long long face = 3 * plane;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < face;
       i += (long long)gridDim.x * blockDim.x)
    x[face + i] = mirror(x[i], (int)(i / plane));
}

int grid_for(long long n) {
  const long long b = (n + kThreads - 1) / kThreads;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

void release(sbim_fault_ctx* c) {
  if (!c) return;
  sbim_destroy(c->up);
  sbim_destroy(c->lo);
  for (void* p : {c->u, c->v, c->u_pred, c->v_pred, c->s_up, c->s_lo, c->zero, c->mu_s, c->tau0, c->traction, c->rate})
    if (p) cudaFree(p);
  delete c;
}

// One solve at face displacements u: the SBIM evaluations (the corrector's
// re-evaluates the predictor's level, reusing its history sums), then the
// traction-continuity / stick-slip kernel writing the face velocities to v_out.
template <class R>
int solve(sbim_fault_ctx* h, const R* u, R* v_out, bool again) {
  const long long np = h->plane();
  const size_t face = 3 * (size_t)np;
  auto eval = again ? sbim_step_repeat : sbim_step;
  int rc = eval(h->up, u, h->zero, h->s_up);
  if (rc != SBIM_OK) return rc;
  if (!h->symmetric) {
    rc = eval(h->lo, u + face, h->zero, h->s_lo);
    if (rc != SBIM_OK) return rc;
  }
  const R mu = (R)(h->rho * h->cs * h->cs);
  const R z_s = mu / (R)h->cs, z_p = z_s * (R)(h->cp / h->cs);
  Law<R> law{(const R*)h->mu_s, (const R*)h->tau0, (R)h->mu_k, (R)h->Dc, (R)h->sigma0,
             h->have_law ? 0 : 1};
  const int blocks = (int)((np + kThreads - 1) / kThreads);
  if (h->symmetric)
    solve_kernel<R, true><<<blocks, kThreads, 0, h->stream>>>(u, v_out, (const R*)h->s_up, nullptr,
                                                              (R*)h->traction, (R*)h->rate, law, np,
                                                              z_s, z_p);
  else
    solve_kernel<R, false><<<blocks, kThreads, 0, h->stream>>>(
        u, v_out, (const R*)h->s_up, (const R*)h->s_lo, (R*)h->traction, (R*)h->rate, law, np,
        z_s, z_p);
  FCU(cudaGetLastError());
  return SBIM_OK;
}

template <class R>
int step_impl(sbim_fault_ctx* h) {
  const long long np = h->plane();
  const R dt = (R)h->dt;
  R* u = (R*)h->u;
  R* v = (R*)h->v;
  R* up = (R*)h->u_pred;
  R* vp = (R*)h->v_pred;
  const int g = grid_for(3 * np);
  if (h->symmetric) predict_kernel<R, true><<<g, kThreads, 0, h->stream>>>(u, v, up, np, dt);
  else predict_kernel<R, false><<<g, kThreads, 0, h->stream>>>(u, v, up, np, dt);
  FCU(cudaGetLastError());
  int rc = solve<R>(h, up, vp, false);
  if (rc != SBIM_OK) return rc;
  if (h->symmetric) correct_kernel<R, true><<<g, kThreads, 0, h->stream>>>(u, v, vp, np, dt);
  else correct_kernel<R, false><<<g, kThreads, 0, h->stream>>>(u, v, vp, np, dt);
  FCU(cudaGetLastError());
  rc = solve<R>(h, u, v, true);
  if (rc != SBIM_OK) return rc;
  ++h->n;
  return SBIM_OK;
}

}  // namespace

extern "C" {

int sbim_fault_create(sbim_fault* out, int n1, int n3, double L1, double L3, double cs, double cp,
                      double rho, double dt, int n_cut, int precision, int symmetric, void* stream) {
  if (!out) return ffail(SBIM_ERR_ARG, "out is NULL");
  if (n1 < 2 || n3 < 2 || (n1 & 1) || (n3 & 1)) return ffail(SBIM_ERR_ARG, "n1, n3 must be even and >= 2");
  if (!(L1 > 0) || !(L3 > 0) || !(dt > 0) || !(rho > 0) || !(cs > 0) || !(cp > cs))
    return ffail(SBIM_ERR_ARG, "need L1, L3, dt, rho, cs > 0 and cp > cs");
  if (precision < SBIM_FP64 || precision > SBIM_BF16) return ffail(SBIM_ERR_ARG, "precision must be 0..3");
  sbim_fault_ctx* c = new sbim_fault_ctx;
  c->n1 = n1; c->n3 = n3; c->prec = precision; c->symmetric = symmetric ? 1 : 0;
  c->cs = cs; c->cp = cp; c->rho = rho; c->dt = dt;
  c->stream = (cudaStream_t)stream;
  c->rs = precision == SBIM_FP64 ? 8 : 4;
  int rc = SBIM_OK;
  auto alloc = [&](void** p, size_t bytes) {
    if (rc != SBIM_OK) return;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) rc = ffail(SBIM_ERR_OOM, "cudaMalloc %zu bytes: %s", bytes, cudaGetErrorString(e));
    else if (cudaMemsetAsync(*p, 0, bytes, c->stream) != cudaSuccess) rc = ffail(SBIM_ERR_CUDA, "memset");
  };
  const size_t pb = 3 * c->plane() * c->rs;
  alloc(&c->u, 2 * pb); alloc(&c->v, 2 * pb); alloc(&c->u_pred, 2 * pb); alloc(&c->v_pred, 2 * pb);
  alloc(&c->s_up, pb); alloc(&c->zero, pb); alloc(&c->traction, pb); alloc(&c->rate, pb);
  if (!c->symmetric) alloc(&c->s_lo, pb);
  alloc(&c->mu_s, c->plane() * c->rs); alloc(&c->tau0, c->plane() * c->rs);
  const int kahan = precision == SBIM_BF16 ? 0 : 1;
  if (rc == SBIM_OK)
    rc = sbim_create(&c->up, n1, n3, L1, L3, cs, cp, rho, dt, n_cut, +1, precision, kahan, stream);
  if (rc == SBIM_OK && !c->symmetric)
    rc = sbim_create(&c->lo, n1, n3, L1, L3, cs, cp, rho, dt, n_cut, -1, precision, kahan, stream);
  if (rc == SBIM_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = ffail(SBIM_ERR_CUDA, "sync");
  if (rc != SBIM_OK) {
    release(c);
    return rc;
  }
  *out = c;
  return SBIM_OK;
}

int sbim_fault_set_fault(sbim_fault h, const double* mu_s, const double* tau0, double mu_k,
                         double Dc, double sigma0) {
  if (!h || !mu_s || !tau0) return ffail(SBIM_ERR_ARG, "NULL argument");
  if (!(Dc > 0)) return ffail(SBIM_ERR_ARG, "Dc must be positive");
  const long long np = h->plane();
  std::vector<float> f1, f2;
  const void* s1 = mu_s;
  const void* s2 = tau0;
  if (h->rs == 4) {
    f1.assign(mu_s, mu_s + np);
    f2.assign(tau0, tau0 + np);
    s1 = f1.data();
    s2 = f2.data();
  }
  FCU(cudaMemcpyAsync(h->mu_s, s1, np * h->rs, cudaMemcpyHostToDevice, h->stream));
  FCU(cudaMemcpyAsync(h->tau0, s2, np * h->rs, cudaMemcpyHostToDevice, h->stream));
  FCU(cudaStreamSynchronize(h->stream));
  h->mu_k = mu_k; h->Dc = Dc; h->sigma0 = sigma0; h->have_law = true;
  return SBIM_OK;
}

int sbim_fault_set_state(sbim_fault h, const void* u, const void* v) {
  if (!h) return ffail(SBIM_ERR_ARG, "NULL handle");
  const size_t fb = 6 * h->plane() * h->rs;
  const void* src[2] = {u, v};
  void* dst[2] = {h->u, h->v};
  for (int i = 0; i < 2; ++i) {
    if (src[i]) FCU(cudaMemcpyAsync(dst[i], src[i], fb, cudaMemcpyDeviceToDevice, h->stream));
    else FCU(cudaMemsetAsync(dst[i], 0, fb, h->stream));
    if (h->symmetric) {
      const long long np = h->plane();
      if (h->rs == 8) mirror_kernel<double><<<grid_for(3 * np), kThreads, 0, h->stream>>>((double*)dst[i], np);
      else mirror_kernel<float><<<grid_for(3 * np), kThreads, 0, h->stream>>>((float*)dst[i], np);
      FCU(cudaGetLastError());
    }
  }
  return SBIM_OK;
}

int sbim_fault_get_state(sbim_fault h, void* u, void* v) {
  if (!h) return ffail(SBIM_ERR_ARG, "NULL handle");
  const size_t fb = 6 * h->plane() * h->rs;
  if (u) FCU(cudaMemcpyAsync(u, h->u, fb, cudaMemcpyDeviceToDevice, h->stream));
  if (v) FCU(cudaMemcpyAsync(v, h->v, fb, cudaMemcpyDeviceToDevice, h->stream));
  return SBIM_OK;
}

int sbim_fault_step(sbim_fault h) {
  if (!h) return ffail(SBIM_ERR_ARG, "NULL handle");
  return h->rs == 8 ? step_impl<double>(h) : step_impl<float>(h);
}

int sbim_fault_fields(sbim_fault h, void* slip, void* slip_rate, void* traction) {
  if (!h) return ffail(SBIM_ERR_ARG, "NULL handle");
  const long long np = h->plane();
  const size_t pb = 3 * np * h->rs;
  if (slip) {
    if (h->rs == 8) slip_kernel<double><<<grid_for(3 * np), kThreads, 0, h->stream>>>((const double*)h->u, (double*)slip, np);
    else slip_kernel<float><<<grid_for(3 * np), kThreads, 0, h->stream>>>((const float*)h->u, (float*)slip, np);
    FCU(cudaGetLastError());
  }
  if (slip_rate) FCU(cudaMemcpyAsync(slip_rate, h->rate, pb, cudaMemcpyDeviceToDevice, h->stream));
  if (traction) FCU(cudaMemcpyAsync(traction, h->traction, pb, cudaMemcpyDeviceToDevice, h->stream));
  return SBIM_OK;
}

int sbim_fault_info(sbim_fault h, long long* steps, sbim_handle* upper, sbim_handle* lower) {
  if (!h) return ffail(SBIM_ERR_ARG, "NULL handle");
  if (steps) *steps = h->n;
  if (upper) *upper = h->up;
  if (lower) *lower = h->lo;
  return SBIM_OK;
}

int sbim_fault_destroy(sbim_fault h) {
  if (!h) return SBIM_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  release(h);
  return SBIM_OK;
}

}  // extern "C"
