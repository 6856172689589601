// Host side of the hybrid FEM-SBIM time step (Section 2.4): an explicit FEM
// slab between two SBIM half-spaces, staggered Neumann coupling, optional
// slip-weakening fault on the mid-plane.  One sbim_hybrid_step enqueues on the
// handle's stream:
//   (1) FE predictor (Eq. (fepred), central-difference displacement update)
//   (2)-(3) sbim_step of the top (side +1) and bottom (side -1) half-spaces with
//       u_{t+1} and the predicted velocity of the boundary layers
//   (4) internal force + boundary forces f = +A tau_top / -A tau_bot
//   (5) fault traction (forward Lagrange multiplier, slip weakening)
//   (6)-(7) acceleration increment and velocity correction (Eqs. (tintf), (fecorr))
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/sbim.h"
#include "fem_internal.cuh"
#include "sbim_internal.cuh"

struct sbim_hybrid_ctx {
  int n1 = 0, n2 = 0, n3 = 0, L = 0, prec = SBIM_FP32, boundaries = 1, fault = 1;
  double h = 0, cs = 0, cp = 0, rho = 0, dt = 0;
  cudaStream_t stream = nullptr;
  sbim_handle top = nullptr, bot = nullptr;
  void* u = nullptr;
  void* v = nullptr;
  void* a = nullptr;
  void* an = nullptr;
  void* tau_top = nullptr;
  void* tau_bot = nullptr;
  void* mu_s = nullptr;
  void* tau0 = nullptr;
  void* traction = nullptr;
  sbim::fem::Stencil<float> stencil_f;
  sbim::fem::Stencil<double> stencil_d;
  void* adj[8] = {};        // reverse sweep: un, vp, af, lun, lvp, lan, lao, lF
  void* adjp[4] = {};       // tb_top, tb_bot, ub, vb ([3][n3][n1])
  double mu_k = 0, Dc = 1, sigma0 = 0;
  bool have_law = false;
  long long n = 0;
  size_t rs = 4;
  long long plane() const { return (long long)n1 * n3; }
  long long elems() const { return (long long)L * 3 * plane(); }
};

struct sbim_hybrid_batch_ctx {
  std::vector<sbim_hybrid> m;
  sbim_batch sb = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

int hfail(int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  sbim::set_last_error(buf);
  return code;
}

#define HCU(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return hfail(e_ == cudaErrorMemoryAllocation ? SBIM_ERR_OOM : SBIM_ERR_CUDA,   \
                   "%s: %s", #call, cudaGetErrorString(e_));                        \
  } while (0)

// 24 x 24 stiffness of a cube of side h, local node a = i + 2 j + 4 k along
// (x1, x2, x3), 2 x 2 x 2 Gauss points, dof 3 a + c.
void hex8_stiffness(double h, double lam, double mu, double K[24][24]) {
  std::memset(K, 0, sizeof(double) * 576);
  const double g = 1.0 / std::sqrt(3.0);
  double D[6][6] = {};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) D[i][j] = lam + (i == j ? 2 * mu : 0.0);
  D[3][3] = D[4][4] = D[5][5] = mu;
  for (int gp = 0; gp < 8; ++gp) {
    const double p[3] = {(gp & 1) ? g : -g, (gp & 2) ? g : -g, (gp & 4) ? g : -g};
    double dN[8][3];
    for (int a = 0; a < 8; ++a) {
      const double s[3] = {(a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0, (a & 4) ? 1.0 : -1.0};
      const double f[3] = {1 + s[0] * p[0], 1 + s[1] * p[1], 1 + s[2] * p[2]};
      dN[a][0] = s[0] * f[1] * f[2] / 8.0 * 2.0 / h;
      dN[a][1] = s[1] * f[0] * f[2] / 8.0 * 2.0 / h;
      dN[a][2] = s[2] * f[0] * f[1] / 8.0 * 2.0 / h;
    }
    double B[6][24] = {};
    for (int a = 0; a < 8; ++a) {
      B[0][3 * a] = dN[a][0];
      B[1][3 * a + 1] = dN[a][1];
      B[2][3 * a + 2] = dN[a][2];
      B[3][3 * a] = dN[a][1]; B[3][3 * a + 1] = dN[a][0];
      B[4][3 * a + 1] = dN[a][2]; B[4][3 * a + 2] = dN[a][1];
      B[5][3 * a] = dN[a][2]; B[5][3 * a + 2] = dN[a][0];
    }
    const double w = std::pow(h / 2.0, 3);
    for (int i = 0; i < 24; ++i)
      for (int j = 0; j < 24; ++j) {
        double s = 0.0;
        for (int r = 0; r < 6; ++r)
          for (int t = 0; t < 6; ++t) s += B[r][i] * D[r][t] * B[t][j];
        K[i][j] += s * w;
      }
  }
}

// Stencil blocks: for side 0 (the 4 elements below a node, the node is their
// top node j = 1) and side 1 (the 4 above, j = 0), offset (o1, o2, o3) with
// o1, o3 in {-1, 0, 1} and o2 in {-1, 0} (below) or {0, 1} (above), the sum of
// the 3x3 blocks K[node][neighbour] over the elements that contain both.
void build_stencil(const double K[24][24], double* out) {
  std::memset(out, 0, 324 * sizeof(double));
  for (int side = 0; side < 2; ++side) {
    const int js = side == 0 ? 1 : 0;
    for (int di = 0; di < 2; ++di)
      for (int dk = 0; dk < 2; ++dk) {
        const int a = di + 2 * js + 4 * dk;
        for (int ox = 0; ox < 3; ++ox)
          for (int oy = 0; oy < 2; ++oy)
            for (int oz = 0; oz < 3; ++oz) {
              const int bi = di + ox - 1, bj = js + (side == 0 ? oy - 1 : oy), bk = dk + oz - 1;
              if (bi < 0 || bi > 1 || bj < 0 || bj > 1 || bk < 0 || bk > 1) continue;
              const int b = bi + 2 * bj + 4 * bk;
              double* blk = out + side * 162 + ((ox * 2 + oy) * 3 + oz) * 9;
              for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) blk[3 * c + d] += K[3 * a + c][3 * b + d];
            }
      }
  }
  // the entries that vanish by the mirror symmetry of the elements (they hold
  // only the rounding of terms that cancel) become exact zeros
  for (int side = 0; side < 2; ++side)
    for (int ox = 0; ox < 3; ++ox)
      for (int oy = 0; oy < 2; ++oy)
        for (int oz = 0; oz < 3; ++oz)
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d)
              if (sbim::fem::stencil_entry_vanishes(ox, oz, c, d))
                out[side * 162 + ((ox * 2 + oy) * 3 + oz) * 9 + 3 * c + d] = 0.0;
}

sbim::fem::MeshArgs mesh_args(const sbim_hybrid_ctx* c) {
  sbim::fem::MeshArgs g;
  g.n1 = c->n1; g.n3 = c->n3; g.L = c->L; g.f = c->n2 / 2; g.fault = c->fault;
  g.area = c->h * c->h;
  g.half_mass = 0.5 * c->rho * c->h * c->h * c->h;
  return g;
}

const sbim::fem::Stencil<float>& stencil_of(const sbim_hybrid_ctx* c, float) { return c->stencil_f; }
const sbim::fem::Stencil<double>& stencil_of(const sbim_hybrid_ctx* c, double) { return c->stencil_d; }

// Stage (1): FE predictor.
template <class R>
int stage_predict(sbim_hybrid_ctx* c, cudaStream_t st) {
  HCU(sbim::fem::predict<R>((R*)c->u, (R*)c->v, (const R*)c->a, c->elems(), (R)c->dt, st));
  return SBIM_OK;
}
template <class R>
int stage_predict(sbim_hybrid_ctx* c) {
  return stage_predict<R>(c, c->stream);
}

// Boundary layers handed to the SBIM half-spaces (top: last layer, bottom: first).
void boundary_ptrs(sbim_hybrid_ctx* c, const void** u_top, const void** v_top,
                   const void** u_bot, const void** v_bot) {
  const long long lay = 3 * c->plane() * (long long)c->rs;
  *u_top = (const char*)c->u + (c->L - 1) * lay;
  *v_top = (const char*)c->v + (c->L - 1) * lay;
  *u_bot = c->u;
  *v_bot = c->v;
}

// Stages (4)-(7): forces, fault traction, acceleration increment, correction.
template <class R>
int stage_finish(sbim_hybrid_ctx* c, const void* src, cudaStream_t st) {
  const R dt = (R)c->dt;
  const long long n = c->elems();
  R* u = (R*)c->u;
  R* v = (R*)c->v;
  R* a = (R*)c->a;
  R* an = (R*)c->an;
  const sbim::fem::MeshArgs g = mesh_args(c);
  HCU(sbim::fem::force<R>(u, an, g, stencil_of(c, R()), c->boundaries ? (const R*)c->tau_top : nullptr,
                          c->boundaries ? (const R*)c->tau_bot : nullptr, (const R*)src, st));
  if (c->fault) {
    sbim::fem::FaultArgs<R> fa;
    fa.mu_s = (const R*)c->mu_s;
    fa.tau0 = (const R*)c->tau0;
    fa.mu_k = (R)c->mu_k;
    fa.Dc = (R)c->Dc;
    fa.sigma0 = (R)c->sigma0;
    fa.traction = (R*)c->traction;
    HCU(sbim::fem::fault<R>(u, v, a, an, g, fa, dt, c->have_law ? 0 : 1, st));
  }
  HCU(sbim::fem::correct<R>(v, a, an, n, dt, st));
  return SBIM_OK;
}
template <class R>
int stage_finish(sbim_hybrid_ctx* c, const void* src) {
  return stage_finish<R>(c, src, c->stream);
}

template <class R>
int step_impl(sbim_hybrid_ctx* c, const void* src) {
  int rc = stage_predict<R>(c);
  if (rc != SBIM_OK) return rc;
  if (c->boundaries) {
    const void *ut, *vt, *ub, *vb;
    boundary_ptrs(c, &ut, &vt, &ub, &vb);
    rc = sbim_step(c->top, ut, vt, c->tau_top);
    if (rc == SBIM_OK) rc = sbim_step(c->bot, ub, vb, c->tau_bot);
    if (rc != SBIM_OK) return rc;
  }
  rc = stage_finish<R>(c, src);
  if (rc == SBIM_OK) ++c->n;
  return rc;
}

template <class R>
int step_given_impl(sbim_hybrid_ctx* c, const void* tau_top, const void* tau_bot) {
  int rc = stage_predict<R>(c);
  if (rc != SBIM_OK) return rc;
  if (tau_top && tau_bot) {
    const size_t pb = 3 * c->plane() * c->rs;
    HCU(cudaMemcpyAsync(c->tau_top, tau_top, pb, cudaMemcpyDeviceToDevice, c->stream));
    HCU(cudaMemcpyAsync(c->tau_bot, tau_bot, pb, cudaMemcpyDeviceToDevice, c->stream));
  }
  rc = stage_finish<R>(c, nullptr);
  if (rc == SBIM_OK) ++c->n;
  return rc;
}

template <class R>
int adjoint_impl(sbim_hybrid_ctx* c, const void* u, const void* v, const void* a,
                 const void* tau_top, const void* tau_bot, const void* tau_bar, void* lu, void* lv,
                 void* la, void* dc_bar) {
  cudaStream_t st = c->stream;
  const size_t fb = c->elems() * c->rs, pb = 3 * c->plane() * c->rs;
  for (void*& x : c->adj)
    if (!x) HCU(cudaMalloc(&x, fb));
  for (void*& x : c->adjp)
    if (!x) HCU(cudaMalloc(&x, pb));
  sbim::fem::AdjointArgs<R> j;
  j.u = (const R*)u; j.v = (const R*)v; j.a = (const R*)a;
  j.un = (R*)c->adj[0]; j.vp = (R*)c->adj[1]; j.af = (R*)c->adj[2];
  j.lu = (R*)lu; j.lv = (R*)lv; j.la = (R*)la;
  j.lun = (R*)c->adj[3]; j.lvp = (R*)c->adj[4]; j.lan = (R*)c->adj[5]; j.lao = (R*)c->adj[6];
  j.lF = (R*)c->adj[7];
  j.tb_top = c->boundaries ? (R*)c->adjp[0] : nullptr;
  j.tb_bot = c->boundaries ? (R*)c->adjp[1] : nullptr;
  j.tau_bar = (const R*)tau_bar;
  j.ddc = (R*)dc_bar;
  j.dt = (R)c->dt;
  j.weld = c->have_law ? 0 : 1;
  const sbim::fem::MeshArgs g = mesh_args(c);
  sbim::fem::FaultArgs<R> fa;
  fa.mu_s = (const R*)c->mu_s; fa.tau0 = (const R*)c->tau0;
  fa.mu_k = (R)c->mu_k; fa.Dc = (R)c->Dc; fa.sigma0 = (R)c->sigma0; fa.traction = nullptr;
  HCU(sbim::fem::adjoint_stages<R>(j, g, stencil_of(c, R()), fa, 0, st));
  HCU(sbim::fem::force<R>(j.un, j.af, g, stencil_of(c, R()), c->boundaries ? (const R*)tau_top : nullptr,
                          c->boundaries ? (const R*)tau_bot : nullptr, nullptr, st));
  for (int stage = 1; stage <= 4; ++stage)
    HCU(sbim::fem::adjoint_stages<R>(j, g, stencil_of(c, R()), fa, stage, st));
  if (c->boundaries) {
    const long long lay = 3 * c->plane();
    R* ub = (R*)c->adjp[2];
    R* vb = (R*)c->adjp[3];
    int rc = sbim_step_adjoint(c->top, j.tb_top, ub, vb);
    if (rc != SBIM_OK) return rc;
    HCU(sbim::fem::layer_add<R>(j.lun + (c->L - 1) * lay, ub, lay, st));
    HCU(sbim::fem::layer_add<R>(j.lvp + (c->L - 1) * lay, vb, lay, st));
    rc = sbim_step_adjoint(c->bot, j.tb_bot, ub, vb);
    if (rc != SBIM_OK) return rc;
    HCU(sbim::fem::layer_add<R>(j.lun, ub, lay, st));
    HCU(sbim::fem::layer_add<R>(j.lvp, vb, lay, st));
  }
  HCU(sbim::fem::adjoint_stages<R>(j, g, stencil_of(c, R()), fa, 5, st));
  ++c->n;
  return SBIM_OK;
}

void hrelease(sbim_hybrid_ctx* c) {
  if (!c) return;
  sbim_destroy(c->top);
  sbim_destroy(c->bot);
  void* p[] = {c->u,     c->v,     c->a,        c->an,      c->tau_top,
               c->tau_bot, c->mu_s, c->tau0, c->traction};
  for (void* x : p)
    if (x) cudaFree(x);
  for (void* x : c->adj)
    if (x) cudaFree(x);
  for (void* x : c->adjp)
    if (x) cudaFree(x);
  delete c;
}

}  // namespace

extern "C" {

int sbim_hybrid_create(sbim_hybrid* out, int n1, int n2, int n3, double h, double cs, double cp,
                       double rho, double dt, int n_cut, int precision, int boundaries,
                       int fault, void* stream) {
  if (!out) return hfail(SBIM_ERR_ARG, "out is NULL");
  if (n1 < 2 || n3 < 2 || (n1 & 1) || (n3 & 1)) return hfail(SBIM_ERR_ARG, "n1, n3 must be even and >= 2");
  if (n2 < 1 || (fault && (n2 < 2 || (n2 & 1))))
    return hfail(SBIM_ERR_ARG, "n2 must be >= 1 (even and >= 2 with a fault)");
  if (!(h > 0) || !(dt > 0) || !(rho > 0) || !(cs > 0) || !(cp > cs))
    return hfail(SBIM_ERR_ARG, "need h, dt, rho, cs > 0 and cp > cs");
  if (precision != SBIM_FP32 && precision != SBIM_FP64)
    return hfail(SBIM_ERR_ARG, "the hybrid step supports SBIM_FP32 and SBIM_FP64");
  sbim_hybrid_ctx* c = new sbim_hybrid_ctx;
  c->n1 = n1; c->n2 = n2; c->n3 = n3; c->h = h; c->cs = cs; c->cp = cp; c->rho = rho; c->dt = dt;
  c->prec = precision; c->boundaries = boundaries ? 1 : 0; c->fault = fault ? 1 : 0;
  c->stream = (cudaStream_t)stream;
  c->L = n2 + (c->fault ? 2 : 1);
  c->rs = precision == SBIM_FP64 ? 8 : 4;
  int rc = SBIM_OK;
  auto alloc = [&](void** p, size_t bytes) {
    if (rc != SBIM_OK) return;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) rc = hfail(SBIM_ERR_OOM, "cudaMalloc %zu bytes: %s", bytes, cudaGetErrorString(e));
    else if (cudaMemsetAsync(*p, 0, bytes, c->stream) != cudaSuccess) rc = hfail(SBIM_ERR_CUDA, "memset");
  };
  const size_t fb = c->elems() * c->rs, pb = 3 * c->plane() * c->rs;
  alloc(&c->u, fb); alloc(&c->v, fb); alloc(&c->a, fb); alloc(&c->an, fb);
  alloc(&c->tau_top, pb); alloc(&c->tau_bot, pb); alloc(&c->traction, pb);
  alloc(&c->mu_s, c->plane() * c->rs); alloc(&c->tau0, c->plane() * c->rs);
  if (rc == SBIM_OK && c->boundaries) {
    rc = sbim_create(&c->top, n1, n3, n1 * h, n3 * h, cs, cp, rho, dt, n_cut, +1, precision, 1, stream);
    if (rc == SBIM_OK)
      rc = sbim_create(&c->bot, n1, n3, n1 * h, n3 * h, cs, cp, rho, dt, n_cut, -1, precision, 1, stream);
  }
  if (rc == SBIM_OK) {
    double K[24][24];
    const double mu = rho * cs * cs, lam = rho * cp * cp - 2 * mu;
    hex8_stiffness(h, lam, mu, K);
    build_stencil(K, c->stencil_d.s);
    for (int i = 0; i < 324; ++i) {
      c->stencil_d.s[i] = -c->stencil_d.s[i];           // the kernels accumulate (-K) u
      c->stencil_f.s[i] = (float)c->stencil_d.s[i];
    }
  }
  if (rc == SBIM_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = hfail(SBIM_ERR_CUDA, "sync");
  if (rc != SBIM_OK) {
    hrelease(c);
    return rc;
  }
  *out = c;
  return SBIM_OK;
}

int sbim_hybrid_set_fault(sbim_hybrid h, const double* mu_s, const double* tau0, double mu_k,
                          double Dc, double sigma0) {
  if (!h || !mu_s || !tau0) return hfail(SBIM_ERR_ARG, "NULL argument");
  if (!h->fault) return hfail(SBIM_ERR_STATE, "the handle was created without a fault");
  if (!(Dc > 0)) return hfail(SBIM_ERR_ARG, "Dc must be positive");
  const long long np = h->plane();
  std::vector<float> f1, f2;
  const void* s1 = mu_s;
  const void* s2 = tau0;
  if (h->prec == SBIM_FP32) {
    f1.assign(mu_s, mu_s + np);
    f2.assign(tau0, tau0 + np);
    s1 = f1.data();
    s2 = f2.data();
  }
  HCU(cudaMemcpyAsync(h->mu_s, s1, np * h->rs, cudaMemcpyHostToDevice, h->stream));
  HCU(cudaMemcpyAsync(h->tau0, s2, np * h->rs, cudaMemcpyHostToDevice, h->stream));
  HCU(cudaStreamSynchronize(h->stream));
  h->mu_k = mu_k; h->Dc = Dc; h->sigma0 = sigma0; h->have_law = true;
  return SBIM_OK;
}

int sbim_hybrid_set_state(sbim_hybrid h, const void* u, const void* v, const void* a) {
  if (!h) return hfail(SBIM_ERR_ARG, "NULL handle");
  const size_t fb = h->elems() * h->rs;
  const void* src[3] = {u, v, a};
  void* dst[3] = {h->u, h->v, h->a};
  for (int i = 0; i < 3; ++i) {
    if (src[i]) HCU(cudaMemcpyAsync(dst[i], src[i], fb, cudaMemcpyDeviceToDevice, h->stream));
    else HCU(cudaMemsetAsync(dst[i], 0, fb, h->stream));
  }
  return SBIM_OK;
}

int sbim_hybrid_get_state(sbim_hybrid h, void* u, void* v, void* a) {
  if (!h) return hfail(SBIM_ERR_ARG, "NULL handle");
  const size_t fb = h->elems() * h->rs;
  void* dst[3] = {u, v, a};
  const void* src[3] = {h->u, h->v, h->a};
  for (int i = 0; i < 3; ++i)
    if (dst[i]) HCU(cudaMemcpyAsync(dst[i], src[i], fb, cudaMemcpyDeviceToDevice, h->stream));
  return SBIM_OK;
}

int sbim_hybrid_step(sbim_hybrid h, const void* force) {
  if (!h) return hfail(SBIM_ERR_ARG, "NULL handle");
  return h->prec == SBIM_FP64 ? step_impl<double>(h, force) : step_impl<float>(h, force);
}

int sbim_hybrid_step_given(sbim_hybrid h, const void* tau_top, const void* tau_bot) {
  if (!h) return hfail(SBIM_ERR_ARG, "NULL handle");
  if (h->boundaries && (!tau_top || !tau_bot))
    return hfail(SBIM_ERR_ARG, "a handle with SBIM boundaries needs both boundary tractions");
  return h->prec == SBIM_FP64 ? step_given_impl<double>(h, tau_top, tau_bot)
                              : step_given_impl<float>(h, tau_top, tau_bot);
}

int sbim_hybrid_boundary_tractions(sbim_hybrid h, void* tau_top, void* tau_bot) {
  if (!h || !tau_top || !tau_bot) return hfail(SBIM_ERR_ARG, "NULL argument");
  if (!h->boundaries) return hfail(SBIM_ERR_STATE, "the handle has free surfaces");
  const size_t pb = 3 * h->plane() * h->rs;
  HCU(cudaMemcpyAsync(tau_top, h->tau_top, pb, cudaMemcpyDeviceToDevice, h->stream));
  HCU(cudaMemcpyAsync(tau_bot, h->tau_bot, pb, cudaMemcpyDeviceToDevice, h->stream));
  return SBIM_OK;
}

int sbim_hybrid_adjoint_step(sbim_hybrid h, const void* u, const void* v, const void* a,
                             const void* tau_top, const void* tau_bot, const void* tau_bar,
                             void* lu, void* lv, void* la, void* dc_bar) {
  if (!h || !u || !v || !a || !lu || !lv || !la || !dc_bar)
    return hfail(SBIM_ERR_ARG, "NULL argument");
  if (h->boundaries && (!tau_top || !tau_bot))
    return hfail(SBIM_ERR_ARG, "a handle with SBIM boundaries needs both boundary tractions");
  if (!h->fault) return hfail(SBIM_ERR_STATE, "the handle was created without a fault");
  return h->prec == SBIM_FP64
             ? adjoint_impl<double>(h, u, v, a, tau_top, tau_bot, tau_bar, lu, lv, la, dc_bar)
             : adjoint_impl<float>(h, u, v, a, tau_top, tau_bot, tau_bar, lu, lv, la, dc_bar);
}

int sbim_hybrid_fault_fields(sbim_hybrid h, void* slip, void* slip_rate, void* traction) {
  if (!h) return hfail(SBIM_ERR_ARG, "NULL handle");
  if (!h->fault) return hfail(SBIM_ERR_STATE, "the handle was created without a fault");
  const sbim::fem::MeshArgs g = mesh_args(h);
  cudaError_t e;
  if (h->prec == SBIM_FP64)
    e = sbim::fem::fault_fields<double>((const double*)h->u, (const double*)h->v, g,
                                        (double*)slip, (double*)slip_rate, h->stream);
  else
    e = sbim::fem::fault_fields<float>((const float*)h->u, (const float*)h->v, g, (float*)slip,
                                       (float*)slip_rate, h->stream);
  if (e != cudaSuccess) return hfail(SBIM_ERR_CUDA, "fault fields: %s", cudaGetErrorString(e));
  if (traction)
    HCU(cudaMemcpyAsync(traction, h->traction, 3 * h->plane() * h->rs, cudaMemcpyDeviceToDevice,
                        h->stream));
  return SBIM_OK;
}

int sbim_hybrid_info(sbim_hybrid h, int* layers, long long* steps, sbim_handle* top,
                     sbim_handle* bottom) {
  if (!h) return hfail(SBIM_ERR_ARG, "NULL handle");
  if (layers) *layers = h->L;
  if (steps) *steps = h->n;
  if (top) *top = h->top;
  if (bottom) *bottom = h->bot;
  return SBIM_OK;
}

int sbim_hybrid_batch_create(sbim_hybrid_batch* out, int nb, const sbim_hybrid* members) {
  if (!out || nb < 1 || !members) return hfail(SBIM_ERR_ARG, "bad batch arguments");
  for (int i = 0; i < nb; ++i) {
    if (!members[i]) return hfail(SBIM_ERR_ARG, "NULL member %d", i);
    if (!members[i]->boundaries || members[i]->prec != SBIM_FP32)
      return hfail(SBIM_ERR_ARG, "batch members need SBIM boundaries and SBIM_FP32");
    if (members[i]->stream != members[0]->stream)
      return hfail(SBIM_ERR_ARG, "batch members must share one stream");
  }
  sbim_hybrid_batch_ctx* b = new sbim_hybrid_batch_ctx;
  b->m.assign(members, members + nb);
  std::vector<sbim_handle> hs;
  for (sbim_hybrid x : b->m) {
    hs.push_back(x->top);
    hs.push_back(x->bot);
  }
  const int rc = sbim::batch_from_handles(&b->sb, hs.data(), (int)hs.size());
  if (rc != SBIM_OK) {
    delete b;
    return rc;
  }
  *out = b;
  return SBIM_OK;
}

namespace {
int hbatch_enqueue(sbim_hybrid_batch b) {
  // the members' FE stages run on the batch's side streams (member k on side
  // stream k mod 8), forked from and joined back into the shared stream
  int rc = sbim::batch_fork(b->sb);
  for (size_t k = 0; k < b->m.size() && rc == SBIM_OK; ++k)
    rc = stage_predict<float>(b->m[k], sbim::batch_side(b->sb, (int)k));
  if (rc == SBIM_OK) rc = sbim::batch_join(b->sb);
  if (rc != SBIM_OK) return rc;
  std::vector<const void*> u, v;
  std::vector<void*> tau;
  for (sbim_hybrid x : b->m) {
    const void *ut, *vt, *ub, *vb;
    boundary_ptrs(x, &ut, &vt, &ub, &vb);
    u.push_back(ut); v.push_back(vt); tau.push_back(x->tau_top);
    u.push_back(ub); v.push_back(vb); tau.push_back(x->tau_bot);
  }
  rc = sbim::batch_enqueue(b->sb, u.data(), v.data(), tau.data());
  if (rc == SBIM_OK) rc = sbim::batch_fork(b->sb);
  for (size_t k = 0; k < b->m.size() && rc == SBIM_OK; ++k)
    rc = stage_finish<float>(b->m[k], nullptr, sbim::batch_side(b->sb, (int)k));
  if (rc == SBIM_OK) rc = sbim::batch_join(b->sb);
  return rc;
}
void hbatch_advance(sbim_hybrid_batch b) {
  sbim::batch_advance(b->sb);
  for (sbim_hybrid x : b->m) ++x->n;
}
}  // namespace

int sbim_hybrid_batch_step(sbim_hybrid_batch b) {
  if (!b) return hfail(SBIM_ERR_ARG, "NULL batch");
  const int rc = hbatch_enqueue(b);
  if (rc == SBIM_OK) hbatch_advance(b);
  return rc;
}

int sbim_hybrid_batch_capture(sbim_hybrid_batch b) {
  if (!b) return hfail(SBIM_ERR_ARG, "NULL batch");
  cudaStream_t st = b->m[0]->stream;
  if (!st) return hfail(SBIM_ERR_ARG, "graph capture needs a non-default stream");
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  HCU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const int rc = hbatch_enqueue(b);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc != SBIM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return hfail(SBIM_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  b->graph = g;
  HCU(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return SBIM_OK;
}

int sbim_hybrid_batch_set_conv_config(sbim_hybrid_batch b, int shape, int lags_per_item) {
  if (!b) return hfail(SBIM_ERR_ARG, "NULL batch");
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  return sbim::batch_set_conv_config(b->sb, shape, lags_per_item);
}

int sbim_hybrid_batch_set_conv_tile(sbim_hybrid_batch b, int orbits_per_cta) {
  if (!b) return hfail(SBIM_ERR_ARG, "NULL batch");
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  return sbim::batch_set_conv_tile(b->sb, orbits_per_cta);
}

int sbim_hybrid_batch_replay(sbim_hybrid_batch b) {
  if (!b) return hfail(SBIM_ERR_ARG, "NULL batch");
  if (!b->exec) return hfail(SBIM_ERR_STATE, "no captured step: call sbim_hybrid_batch_capture");
  HCU(cudaGraphLaunch(b->exec, b->m[0]->stream));
  hbatch_advance(b);
  return SBIM_OK;
}

int sbim_hybrid_batch_destroy(sbim_hybrid_batch b) {
  if (!b) return SBIM_OK;
  cudaStream_t st = b->m.empty() ? nullptr : b->m[0]->stream;
  if (st) cudaStreamSynchronize(st);
  else cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  sbim_batch_destroy(b->sb);   // the SBIM handles stay with their hybrids
  delete b;
  return SBIM_OK;
}

int sbim_hybrid_destroy(sbim_hybrid h) {
  if (!h) return SBIM_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  hrelease(h);
  return SBIM_OK;
}

}  // extern "C"
