// Host side of libsbim: the C ABI declared in include/sbim.h.
//
// sbim_create plans the spectral layout (|k|-sorted orbits of Fourier-bin
// members, Section 2.3 spectral evaluation of s_i), builds the kernel tables
// on the device in FP64, allocates the history ring buffer and creates the
// cuFFT plans.  sbim_step enqueues, on the handle's stream:
//   (0) R2C FFT of u                      (cuFFT)
//   (1) rotate + ring write + convolution  conv_kernel
//   (2) chunk reduction + assembly         assemble_kernel
//   (3) C2R FFT of the traction spectra    (cuFFT)
//   (4) traction epilogue                  epilogue_kernel
// with no host synchronisation.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sbim.h"
#include "sbim_internal.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

const char* fft_name(cufftResult r) {
  switch (r) {
    case CUFFT_SUCCESS: return "CUFFT_SUCCESS";
    case CUFFT_INVALID_PLAN: return "CUFFT_INVALID_PLAN";
    case CUFFT_ALLOC_FAILED: return "CUFFT_ALLOC_FAILED";
    case CUFFT_INVALID_VALUE: return "CUFFT_INVALID_VALUE";
    case CUFFT_INTERNAL_ERROR: return "CUFFT_INTERNAL_ERROR";
    case CUFFT_EXEC_FAILED: return "CUFFT_EXEC_FAILED";
    case CUFFT_SETUP_FAILED: return "CUFFT_SETUP_FAILED";
    case CUFFT_INVALID_SIZE: return "CUFFT_INVALID_SIZE";
    default: return "cuFFT error";
  }
}

#define CU(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(e_ == cudaErrorMemoryAllocation ? SBIM_ERR_OOM : SBIM_ERR_CUDA,   \
                  "%s: %s", #call, cudaGetErrorString(e_));                        \
  } while (0)

#define CF(call)                                                                   \
  do {                                                                             \
    cufftResult r_ = (call);                                                       \
    if (r_ != CUFFT_SUCCESS) return fail(SBIM_ERR_FFT, "%s: %s", #call, fft_name(r_)); \
  } while (0)

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr int kProfRing = 512;
constexpr int kProfEvents = 6;

// 16-point Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_16).
void gauss_legendre16(double* x, double* w) {
  const int n = 16;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

struct Member {
  int bin;
  double e1, e3;
  float w;
};

}  // namespace

struct sbim_ctx {
  int n1 = 0, n3 = 0, nh = 0, nbins = 0, n_cut = 0, side = 1, prec = SBIM_FP32, kahan = 0;
  double L1 = 0, L3 = 0, cs = 0, cp = 0, rho = 0, dt = 0, mu = 0, eta = 0;
  cudaStream_t stream = nullptr;
  int n_orb = 0, n_orb_pad = 0, lc = 1, nchunks = 1;
  int variant = 1;            // 0: register-prefetch loads, 1-3: TMA-staged history shapes
  int tile = sbim::kOrbitTile;  // orbits per CTA of the TMA convolution: 64, 128 or 256
  bool halves = false;        // records may hold two |k| (half-record layout)
  int lags_per_cta = 0;       // 0: automatic
  size_t part_bytes = 0;
  double tab_h = 0;
  long long tab_n = 0;
  size_t real_size = 4;

  int* d_bin = nullptr;
  void* d_dir = nullptr;  // float2, or double2 for the FP64 path
  float* d_wout = nullptr;
  void* d_dT = nullptr;
  unsigned long long* d_ustep = nullptr;
  void* d_muq = nullptr;
  double* d_tab64 = nullptr;
  float* d_tab32 = nullptr;
  double* d_gl = nullptr;
  void* d_hist = nullptr;
  size_t hist_bytes = 0;
  long long plane_records = 0;
  void* d_part = nullptr;
  void* d_uhat = nullptr;
  void* d_fhat = nullptr;
  void* d_s = nullptr;
  long long* d_step = nullptr;
  int* d_err = nullptr;
  int* d_nonfinite = nullptr;  // flag of the opt-in input check
  void* d_wts = nullptr;       // FP64 path: precomputed weights [n_cut][n_orb_pad][4] doubles
  size_t wts_bytes = 0;
  bool check_finite = false;
  int* d_lmax = nullptr;
  int* d_tile_lmax = nullptr;
  double window = 0.0;
  std::vector<double> h_dT;   // |k| c_s dt per half record, [o][2] (host copy)
  void* d_io = nullptr;  // u, v, tau staging and zero spectra for sbim_step_host
  int* h_err = nullptr;  // pinned copy of the error word, read with tau by sbim_step_host
  cudaStream_t io_stream = nullptr;          // sbim_step_host: copies in + forward FFT
  cudaEvent_t io_fork = nullptr, io_join = nullptr;
  cufftHandle plan_fwd = 0, plan_inv = 0;
  bool have_fwd = false, have_inv = false;

  long long n = 0;
  bool can_repeat = false;    // the partial sums hold the last forward level
  double tau_inf[3] = {0, 0, 0};

  bool prof = false;
  std::vector<cudaEvent_t> ev;      // kProfRing * kProfEvents
  long long prof_issued = 0, prof_harvested = 0;
  double prof_ms[5] = {0, 0, 0, 0, 0};

  size_t field_elems() const { return (size_t)3 * n1 * n3; }
};

namespace {

// Integer weights (a, b) with L1 / L3 = a / b exactly, a and b coprime and
// small, so that |k|^2 (L1 L3 / 2 pi)^2 = (j1 b)^2 + (j3 a)^2 is an exact integer
// key; {0, 0} when the period ratio is not such a fraction (or the key could
// overflow), and bins are then grouped by their floating-point |k|^2.
void period_ratio(const sbim_ctx& c, long long& a, long long& b) {
  a = b = 0;
  for (long long bb = 1; bb <= 4096; ++bb) {
    const double aa = std::nearbyint(c.L1 * (double)bb / c.L3);
    if (aa < 1.0 || aa > 4096.0 || c.L1 * (double)bb != c.L3 * aa) continue;
    const double big = std::pow((double)(c.n1 / 2) * (double)bb, 2) +
                       std::pow((double)(c.n3 / 2) * aa, 2);
    if (big < 4e18) {
      a = (long long)aa;
      b = bb;
    }
    return;
  }
}

// Bytes of one 4-member history record (all planes) per precision.
long long history_record_bytes(int prec) {
  switch (prec) {
    case SBIM_FP64: return 64;
    case SBIM_FP32: return 32;
    case SBIM_BF16X2: return 2 * 16;   // hi and lo planes
    default: return 16;
  }
}

// Group the half-spectrum bins into |k|-sorted records of 4 member slots made
// of two halves of 2 slots; each half carries one |k| (q_half[2 r + h]).  The
// members of one bin stay in one record.
//   whole records (halves = false): a class of equal |k| fills records of its
//     own (both halves carry its |k|) -- the layout of square grids, whose
//     generic class {(a, b), (a, -b), (b, a), (b, -a)} is exactly one record;
//   half records (halves = true): a class fills halves (a Nyquist bin's two
//     virtual members take a half, the corner's four a whole record, other bins
//     two to a half); its halves pair up into records of one |k|, and an odd one
//     left over shares a record with the next class's leftover -- for
//     rectangular planes, where most classes are pairs {(j1, j3), (j1, -j3)}
//     and whole records would be half empty.
void plan_orbits(const sbim_ctx& c, std::vector<Member>& mem, std::vector<double>& q_half,
                 bool halves) {
  long long ra, rb;
  period_ratio(c, ra, rb);
  const bool exact = ra > 0;
  struct Rec {
    long long ikey;
    double dkey;
    int j1, r3, j3;
  };
  std::vector<Rec> recs;
  recs.reserve(c.nbins);
  for (int r3 = 0; r3 < c.n3; ++r3) {
    const int j3 = r3 <= c.n3 / 2 ? r3 : r3 - c.n3;
    for (int j1 = 0; j1 < c.nh; ++j1) {
      Rec r;
      r.j1 = j1;
      r.r3 = r3;
      r.j3 = j3;
      r.ikey = exact ? (j1 * rb) * (j1 * rb) + (j3 * ra) * (j3 * ra) : 0;
      const double a = j1 / c.L1, b = j3 / c.L3;
      r.dkey = a * a + b * b;
      recs.push_back(r);
    }
  }
  auto less = [exact](const Rec& x, const Rec& y) {
    if (exact) {
      if (x.ikey != y.ikey) return x.ikey < y.ikey;
    } else if (x.dkey != y.dkey) {
      return x.dkey < y.dkey;
    }
    if (x.j1 != y.j1) return x.j1 < y.j1;
    return x.r3 < y.r3;
  };
  std::sort(recs.begin(), recs.end(), less);
  auto same = [exact](const Rec& x, const Rec& y) {
    return exact ? x.ikey == y.ikey : x.dkey == y.dkey;
  };

  const Member pad{-1, 1.0, 0.0, 0.0f};
  struct Half {
    Member m[2];
    double q;
  };
  auto emit = [&](const Half& x, const Half& y) {
    mem.push_back(x.m[0]);
    mem.push_back(x.m[1]);
    mem.push_back(y.m[0]);
    mem.push_back(y.m[1]);
    q_half.push_back(x.q);
    q_half.push_back(y.q);
  };
  std::vector<Member> cur;
  auto flush_whole = [&](double q) {
    if (cur.empty()) return;
    while (cur.size() < 4) cur.push_back(pad);
    mem.insert(mem.end(), cur.begin(), cur.end());
    q_half.push_back(q);
    q_half.push_back(q);
    cur.clear();
  };
  bool have_left = false;
  Half left{{pad, pad}, 0.0};
  size_t i = 0;
  while (i < recs.size()) {
    size_t j = i;
    while (j < recs.size() && same(recs[i], recs[j])) ++j;
    const double k1c = 2.0 * kPi * recs[i].j1 / c.L1, k3c = 2.0 * kPi * recs[i].j3 / c.L3;
    const double q = std::hypot(k1c, k3c);
    std::vector<Half> hs;
    std::vector<Member> singles;
    for (size_t t = i; t < j; ++t) {
      const Rec& r = recs[t];
      const bool ny1 = (r.j1 == c.n1 / 2), ny3 = (r.r3 == c.n3 / 2);
      const double k1 = 2.0 * kPi * r.j1 / c.L1, k3 = 2.0 * kPi * r.j3 / c.L3;
      const int bin = r.r3 * c.nh + r.j1;
      std::vector<Member> grp;
      const int n_s1 = ny1 ? 2 : 1, n_s3 = ny3 ? 2 : 1;
      const float wgt = 1.0f / (float)(n_s1 * n_s3);
      for (int a = 0; a < n_s1; ++a)
        for (int b = 0; b < n_s3; ++b) {
          const double s1 = a ? -1.0 : 1.0, s3 = b ? -1.0 : 1.0;
          Member m;
          m.bin = bin;
          if (q > 0) {
            m.e1 = s1 * k1 / q;
            m.e3 = s3 * k3 / q;
            m.w = wgt;
          } else {  // k = 0 carries no non-local traction
            m.e1 = 1.0;
            m.e3 = 0.0;
            m.w = 0.0f;
          }
          grp.push_back(m);
        }
      if (!halves) {   // whole records: fill this class's records of 4
        if (cur.size() + grp.size() > 4) flush_whole(q);
        cur.insert(cur.end(), grp.begin(), grp.end());
      } else if (grp.size() == 1) {
        singles.push_back(grp[0]);
      } else {
        for (size_t k = 0; k < grp.size(); k += 2) hs.push_back(Half{{grp[k], grp[k + 1]}, q});
      }
    }
    if (!halves) {
      flush_whole(q);
      i = j;
      continue;
    }
    for (size_t k = 0; k < singles.size(); k += 2)
      hs.push_back(Half{{singles[k], k + 1 < singles.size() ? singles[k + 1] : pad}, q});
    size_t h = 0;
    for (; h + 1 < hs.size(); h += 2) emit(hs[h], hs[h + 1]);
    if (h < hs.size()) {
      if (have_left) {
        emit(left, hs[h]);
        have_left = false;
      } else {
        left = hs[h];
        have_left = true;
      }
    }
    i = j;
  }
  if (have_left) emit(left, Half{{pad, pad}, 0.0});
}

// The record layout of a grid: whole records unless half records would store
// more than 12 % less history.  The half-record kernels stream their bytes
// ~13 % slower (a second weight set per record and lag; on GB300 0.935 against
// 1.07 of the copy bandwidth), so they pay only where whole records are mostly
// padding: rectangular planes (the TPV3 plane: 1.20x the bins as whole records,
// 1.006x as half records) and a few tiny grids; squares of 32^2 and more keep
// whole records.  Returns whether the layout has half records.
bool plan_layout(const sbim_ctx& c, std::vector<Member>& mem, std::vector<double>& q_half) {
  plan_orbits(c, mem, q_half, false);
  if ((double)mem.size() <= 1.03 * c.nbins) return false;
  std::vector<Member> mem_h;
  std::vector<double> q_h;
  plan_orbits(c, mem_h, q_h, true);
  if ((double)mem.size() <= 1.12 * (double)mem_h.size()) return false;
  mem.swap(mem_h);
  q_half.swap(q_h);
  return true;
}

// Lag chunking of the convolution grid: (n_orb_pad / 128) x nchunks CTAs,
// about 16 waves of the variant's resident CTAs, unless lags_per_cta is set.
int choose_chunks(sbim_ctx& c) {
  int dev = 0, sms = 148;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (c.lags_per_cta > 0) {
    c.lc = std::min(c.lags_per_cta, c.n_cut);
  } else {
    const long long tiles = c.n_orb_pad / (c.variant >= 1 ? c.tile : sbim::kOrbitTile);
    const int per_sm = c.variant >= 1 ? sbim::conv_tma_ctas_per_sm(c.prec, c.kahan, c.variant, c.tile)
                                      : (c.prec == SBIM_FP64 ? 1 : 3);
    const long long target = (long long)sms * per_sm * 16;
    long long S = (target + tiles - 1) / tiles;
    const long long smax = std::max(1, (c.n_cut + 15) / 16);
    S = std::max(1LL, std::min(S, smax));
    c.lc = (int)((c.n_cut + S - 1) / S);
  }
  c.nchunks = (c.n_cut + c.lc - 1) / c.lc;
  return SBIM_OK;
}

// (Re)allocate the lag-chunk partial sums for the current chunking; on failure
// the previous buffer is kept.
int alloc_partials(sbim_ctx& c) {
  const size_t need = (size_t)c.nchunks * 4 * sbim::kFields * c.n_orb_pad * c.real_size;
  if (need <= c.part_bytes && c.d_part) return SBIM_OK;
  void* fresh = nullptr;
  CU(cudaMalloc(&fresh, need));
  if (c.d_part) {
    CU(cudaStreamSynchronize(c.stream));
    CU(cudaFree(c.d_part));
  }
  c.d_part = fresh;
  c.part_bytes = need;
  return SBIM_OK;
}

void release(sbim_ctx* c) {
  if (!c) return;
  if (c->have_fwd) cufftDestroy(c->plan_fwd);
  if (c->have_inv) cufftDestroy(c->plan_inv);
  void* ptrs[] = {c->d_bin, c->d_dir, c->d_wout, c->d_dT, c->d_ustep, c->d_muq,
                  c->d_tab64, c->d_tab32, c->d_gl, c->d_hist, c->d_part, c->d_uhat,
                  c->d_fhat, c->d_s, c->d_step, c->d_err, c->d_io, c->d_lmax,
                  c->d_tile_lmax, c->d_nonfinite, c->d_wts};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  if (c->io_fork) cudaEventDestroy(c->io_fork);
  if (c->io_join) cudaEventDestroy(c->io_join);
  if (c->io_stream) cudaStreamDestroy(c->io_stream);
  if (c->h_err) cudaFreeHost(c->h_err);
  delete c;
}

int harvest(sbim_ctx* c, long long upto) {
  while (c->prof_harvested < upto) {
    cudaEvent_t* e = &c->ev[(c->prof_harvested % kProfRing) * kProfEvents];
    CU(cudaEventSynchronize(e[kProfEvents - 1]));
    for (int k = 0; k < 5; ++k) {
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, e[k], e[k + 1]));
      c->prof_ms[k] += ms;
    }
    ++c->prof_harvested;
  }
  return SBIM_OK;
}

sbim::StepArgs step_args(const sbim_ctx* c);

int create_impl(sbim_ctx* c) {
  c->mu = c->rho * c->cs * c->cs;
  c->eta = c->cp / c->cs;
  c->nh = c->n1 / 2 + 1;
  c->nbins = c->n3 * c->nh;
  const bool dbl = c->prec == SBIM_FP64;
  c->real_size = dbl ? 8 : 4;

  std::vector<Member> mem;
  std::vector<double> q_half;
  c->halves = plan_layout(*c, mem, q_half);
  c->n_orb = (int)(q_half.size() / 2);
  c->n_orb_pad = (c->n_orb + sbim::kOrbitTile - 1) / sbim::kOrbitTile * sbim::kOrbitTile;
  mem.resize((size_t)c->n_orb_pad * 4, Member{-1, 1.0, 0.0, 0.0f});
  q_half.resize((size_t)c->n_orb_pad * 2, 0.0);

  // kernel-table resolution: cubic interpolation error ~ 0.0234 h^4 max|H''''|
  c->tab_h = dbl ? 1.0 / 512.0 : 1.0 / 64.0;
  double dT_max = 0.0;
  const int n_half = 2 * c->n_orb_pad;   // per half record: [o][2]
  std::vector<double> dT(n_half), muq(n_half);
  std::vector<unsigned long long> ustep(n_half);
  for (int o = 0; o < n_half; ++o) {
    dT[o] = q_half[o] * c->cs * c->dt;
    muq[o] = c->mu * q_half[o];
    dT_max = std::max(dT_max, dT[o]);
    ustep[o] = (unsigned long long)std::llround(dT[o] / c->tab_h * 4294967296.0);
  }
  c->h_dT = dT;
  const double t_max = dT_max * (c->n_cut - 1);
  c->tab_n = (long long)std::floor(t_max / c->tab_h) + 6;  // nodes -1 .. floor + 4
  if ((double)c->n_cut * (dT_max / c->tab_h + 1.0) * 4294967296.0 > 1.8e19 ||
      c->tab_n > (1LL << 31))
    return fail(SBIM_ERR_ARG, "history too long for the kernel table (n_cut x |k|max c_s dt)");

  std::vector<int> h_bin(mem.size());
  std::vector<float2> h_dir(mem.size());
  std::vector<double2> h_dir64(mem.size());
  std::vector<float> h_w(mem.size());
  for (size_t i = 0; i < mem.size(); ++i) {
    h_bin[i] = mem[i].bin;
    h_dir[i] = make_float2((float)mem[i].e1, (float)mem[i].e3);
    h_dir64[i] = make_double2(mem[i].e1, mem[i].e3);
    h_w[i] = mem[i].w;
  }

  if (choose_chunks(*c) != SBIM_OK) return SBIM_ERR_CUDA;
  if (c->variant >= 1)
    CU(sbim::prepare_conv_tma(c->prec, c->kahan, c->variant, c->tile, c->halves));

  // history size
  c->plane_records = (long long)c->n_cut * 3 * c->n_orb_pad;
  c->hist_bytes = (size_t)c->plane_records * history_record_bytes(c->prec);
  const size_t part_bytes = (size_t)c->nchunks * 4 * sbim::kFields * c->n_orb_pad * c->real_size;
  const size_t cplx = 2 * c->real_size;
  size_t free_b = 0, total_b = 0;
  CU(cudaMemGetInfo(&free_b, &total_b));
  const size_t need = c->hist_bytes + part_bytes + 2 * 3 * (size_t)c->nbins * cplx +
                      4 * c->field_elems() * c->real_size + (size_t)c->tab_n * 48;
  if (need + (256ull << 20) > free_b)
    return fail(SBIM_ERR_OOM, "need %.2f GB of device memory, %.2f GB free",
                need / 1e9, free_b / 1e9);
  // The FP64 path keeps its convolution weights (32 B per orbit and lag) when
  // they fit beside everything else; without them it interpolates every step.
  if (dbl) {
    const size_t wb = (size_t)c->n_cut * c->n_orb_pad * 32;
    if (need + wb + (512ull << 20) <= free_b) c->wts_bytes = wb;
  }

  CU(cudaMalloc(&c->d_bin, h_bin.size() * sizeof(int)));
  CU(cudaMalloc(&c->d_dir, h_dir.size() * (dbl ? sizeof(double2) : sizeof(float2))));
  CU(cudaMalloc(&c->d_wout, h_w.size() * sizeof(float)));
  CU(cudaMalloc(&c->d_dT, 2 * c->n_orb_pad * c->real_size));
  CU(cudaMalloc(&c->d_muq, 2 * c->n_orb_pad * c->real_size));
  CU(cudaMalloc(&c->d_ustep, 2 * c->n_orb_pad * sizeof(unsigned long long)));
  CU(cudaMalloc(&c->d_tab64, (size_t)c->tab_n * 4 * sizeof(double)));
  if (!dbl) CU(cudaMalloc(&c->d_tab32, (size_t)c->tab_n * 4 * sizeof(float)));
  CU(cudaMalloc(&c->d_gl, 32 * sizeof(double)));
  CU(cudaMalloc(&c->d_hist, c->hist_bytes));
  c->d_part = nullptr;
  if (alloc_partials(*c) != SBIM_OK) return SBIM_ERR_OOM;
  CU(cudaMalloc(&c->d_uhat, 3 * (size_t)c->nbins * cplx));
  CU(cudaMalloc(&c->d_fhat, 3 * (size_t)c->nbins * cplx));
  CU(cudaMalloc(&c->d_s, c->field_elems() * c->real_size));
  CU(cudaMalloc(&c->d_step, sizeof(long long)));
  CU(cudaMalloc(&c->d_err, sizeof(int)));
  if (c->wts_bytes) CU(cudaMalloc(&c->d_wts, c->wts_bytes));

  cudaStream_t st = c->stream;
  CU(cudaMemcpyAsync(c->d_bin, h_bin.data(), h_bin.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (dbl)
    CU(cudaMemcpyAsync(c->d_dir, h_dir64.data(), h_dir64.size() * sizeof(double2),
                       cudaMemcpyHostToDevice, st));
  else
    CU(cudaMemcpyAsync(c->d_dir, h_dir.data(), h_dir.size() * sizeof(float2),
                       cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(c->d_wout, h_w.data(), h_w.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(c->d_ustep, ustep.data(), ustep.size() * sizeof(unsigned long long),
                     cudaMemcpyHostToDevice, st));
  if (dbl) {
    CU(cudaMemcpyAsync(c->d_dT, dT.data(), dT.size() * 8, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(c->d_muq, muq.data(), muq.size() * 8, cudaMemcpyHostToDevice, st));
  } else {
    std::vector<float> f1(dT.begin(), dT.end()), f2(muq.begin(), muq.end());
    CU(cudaMemcpyAsync(c->d_dT, f1.data(), f1.size() * 4, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(c->d_muq, f2.data(), f2.size() * 4, cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));  // f1, f2 leave scope
  }
  double gl[32];
  gauss_legendre16(gl, gl + 16);
  CU(cudaMemcpyAsync(c->d_gl, gl, sizeof gl, cudaMemcpyHostToDevice, st));
  CU(sbim::launch_table_build(c->d_tab64, c->d_tab32, c->tab_n, c->tab_h, c->eta, c->d_gl,
                              c->d_gl + 16, st));
  if (c->d_wts) CU(sbim::launch_weights64(step_args(c), c->d_wts, st));
  CU(cudaMemsetAsync(c->d_step, 0, sizeof(long long), st));
  CU(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
  CU(cudaStreamSynchronize(st));

  // cuFFT plans: batch of 3 components, [n3][n1] real <-> [n3][n1/2+1] complex
  int dims[2] = {c->n3, c->n1};
  CF(cufftPlanMany(&c->plan_fwd, 2, dims, nullptr, 1, c->n3 * c->n1, nullptr, 1, c->nbins,
                   dbl ? CUFFT_D2Z : CUFFT_R2C, 3));
  c->have_fwd = true;
  CF(cufftPlanMany(&c->plan_inv, 2, dims, nullptr, 1, c->nbins, nullptr, 1, c->n3 * c->n1,
                   dbl ? CUFFT_Z2D : CUFFT_C2R, 3));
  c->have_inv = true;
  CF(cufftSetStream(c->plan_fwd, st));
  CF(cufftSetStream(c->plan_inv, st));
  return SBIM_OK;
}

sbim::StepArgs step_args(const sbim_ctx* c) {
  sbim::StepArgs a;
  a.bin = c->d_bin;
  a.dir = c->d_dir;
  a.wout = c->d_wout;
  a.dT = c->d_dT;
  a.ustep = c->d_ustep;
  a.muq = c->d_muq;
  a.table = c->prec == SBIM_FP64 ? (const void*)c->d_tab64 : (const void*)c->d_tab32;
  a.lmax = c->window > 0 ? c->d_lmax : nullptr;
  a.tile_lmax = c->window > 0 ? c->d_tile_lmax : nullptr;
  a.wts = c->d_wts;
  a.hist = c->d_hist;
  a.step = c->d_step;
  a.err = c->d_err;
  a.part = c->d_part;
  a.uhat = c->d_uhat;
  a.fhat = c->d_fhat;
  a.n_orb_pad = c->n_orb_pad;
  a.halves = c->halves ? 1 : 0;
  a.nbins = c->nbins;
  a.n_cut = c->n_cut;
  a.lc = c->lc;
  a.nchunks = c->nchunks;
  a.side = c->side;
  a.eta = c->eta;
  a.inv_n = 1.0 / ((double)c->n1 * c->n3);
  a.slot_stride = c->plane_records;
  return a;
}

}  // namespace

namespace sbim {
void set_last_error(const char* msg) { g_err = msg; }

StepArgs handle_step_args(sbim_handle h) { return step_args(h); }

// The batch drivers run members' small stages on side streams: the plans are
// pointed at the given stream for the call and back at the handle's after it.
int handle_fft_forward(sbim_handle c, const void* u, cudaStream_t st) {
  if (st != c->stream) CF(cufftSetStream(c->plan_fwd, st));
  cufftResult r;
  if (c->prec == SBIM_FP64)
    r = cufftExecD2Z(c->plan_fwd, (cufftDoubleReal*)u, (cufftDoubleComplex*)c->d_uhat);
  else
    r = cufftExecR2C(c->plan_fwd, (cufftReal*)u, (cufftComplex*)c->d_uhat);
  if (st != c->stream) CF(cufftSetStream(c->plan_fwd, c->stream));
  CF(r);
  return SBIM_OK;
}

int handle_fft_inverse(sbim_handle c, cudaStream_t st) {
  if (st != c->stream) CF(cufftSetStream(c->plan_inv, st));
  cufftResult r;
  if (c->prec == SBIM_FP64)
    r = cufftExecZ2D(c->plan_inv, (cufftDoubleComplex*)c->d_fhat, (cufftDoubleReal*)c->d_s);
  else
    r = cufftExecC2R(c->plan_inv, (cufftComplex*)c->d_fhat, (cufftReal*)c->d_s);
  if (st != c->stream) CF(cufftSetStream(c->plan_inv, c->stream));
  CF(r);
  return SBIM_OK;
}

int handle_epilogue(sbim_handle c, const void* v, void* tau, cudaStream_t st) {
  const double k = c->side * c->mu / c->cs;
  const double coef[3] = {k, k * c->eta, k};
  CU(launch_epilogue(c->prec, c->d_s, v, tau, (long long)c->n1 * c->n3, coef, c->tau_inf,
                     c->d_step, st));
  return SBIM_OK;
}

void handle_advance(sbim_handle c) {
  ++c->n;
  c->can_repeat = false;   // the batch kept its partial sums in its own buffers
}

int handle_shape(sbim_handle c, int* precision, int* kahan, int* variant, void** stream) {
  *precision = c->prec;
  *kahan = c->kahan;
  *variant = c->variant;
  *stream = (void*)c->stream;
  return SBIM_OK;
}
}  // namespace sbim

extern "C" {

int sbim_plan(int n1, int n3, double L1, double L3, int n_cut, int precision,
              long long* n_modes, long long* n_slots, long long* hist_bytes) {
  g_err.clear();
  if (n1 < 2 || n3 < 2 || (n1 & 1) || (n3 & 1))
    return fail(SBIM_ERR_ARG, "n1 and n3 must be even and >= 2 (got %d, %d)", n1, n3);
  if ((long long)n1 * n3 > (1LL << 28)) return fail(SBIM_ERR_ARG, "grid too large");
  if (!(L1 > 0) || !(L3 > 0)) return fail(SBIM_ERR_ARG, "L1 and L3 must be positive");
  if (n_cut < 1) return fail(SBIM_ERR_ARG, "n_cut must be >= 1");
  if (precision < SBIM_FP64 || precision > SBIM_BF16) return fail(SBIM_ERR_ARG, "bad precision");
  sbim_ctx c;
  c.n1 = n1; c.n3 = n3; c.L1 = L1; c.L3 = L3; c.n_cut = n_cut; c.prec = precision;
  c.nh = n1 / 2 + 1;
  c.nbins = n3 * c.nh;
  std::vector<Member> mem;
  std::vector<double> q_half;
  plan_layout(c, mem, q_half);
  const long long pad =
      ((long long)q_half.size() / 2 + sbim::kOrbitTile - 1) / sbim::kOrbitTile * sbim::kOrbitTile;
  if (n_modes) *n_modes = c.nbins;
  if (n_slots) *n_slots = pad * 4;
  if (hist_bytes) *hist_bytes = (long long)n_cut * 3 * pad * history_record_bytes(precision);
  return SBIM_OK;
}

int sbim_create(sbim_handle* out, int n1, int n3, double L1, double L3, double cs, double cp,
                double rho, double dt, int n_cut, int side, int precision, int kahan,
                void* stream) {
  g_err.clear();
  if (!out) return fail(SBIM_ERR_ARG, "out is NULL");
  if (n1 < 2 || n3 < 2 || (n1 & 1) || (n3 & 1))
    return fail(SBIM_ERR_ARG, "n1 and n3 must be even and >= 2 (got %d, %d)", n1, n3);
  if ((long long)n1 * n3 > (1LL << 28)) return fail(SBIM_ERR_ARG, "grid too large");
  if (!(L1 > 0) || !(L3 > 0) || !(dt > 0) || !(rho > 0) || !(cs > 0))
    return fail(SBIM_ERR_ARG, "L1, L3, dt, rho and cs must be positive");
  if (!(cp > cs)) return fail(SBIM_ERR_ARG, "cp must exceed cs");
  if (n_cut < 1) return fail(SBIM_ERR_ARG, "n_cut must be >= 1");
  if (side != 1 && side != -1) return fail(SBIM_ERR_ARG, "side must be +1 or -1");
  if (precision < SBIM_FP64 || precision > SBIM_BF16) return fail(SBIM_ERR_ARG, "bad precision");
  sbim_ctx* c = new sbim_ctx;
  c->n1 = n1; c->n3 = n3; c->L1 = L1; c->L3 = L3; c->cs = cs; c->cp = cp; c->rho = rho;
  c->dt = dt; c->n_cut = n_cut; c->side = side; c->prec = precision;
  c->kahan = precision == SBIM_FP64 ? 0 : (kahan ? 1 : 0);
  c->stream = (cudaStream_t)stream;
  // default convolution launch: the shapes the autotuner measured fastest on
  // GB300 at 1024^2 x 4096 (shape 2 for every float-class history: 3 stages x
  // 2 lags x 3 CTAs/SM, 6 x 2 x 3 for compensated bf16 hi-only and 6 x 1 x 5
  // for uncompensated bf16 hi-only; 3 x 1 x 2 for double)
  c->variant = precision == SBIM_FP64 ? 1 : 2;
  const int rc = create_impl(c);
  if (rc != SBIM_OK) {
    const std::string msg = g_err;
    release(c);
    cudaGetLastError();
    g_err = msg;
    return rc;
  }
  *out = c;
  return SBIM_OK;
}

}  // extern "C"

namespace {

// One update: forward (in = u, aux = v, out = tau) or its transpose in reverse
// time (in = tau_bar, out = u_bar, aux = v_bar).  The per-bin, per-lag modal
// matrix is Hermitian in the (xi, 2, perp) frame ([a, ib; -ib, d] and a real
// perp entry), so the transpose of R2C -> A -> C2R/N is the same map; applied to
// the tau_bar sequence in reverse time it gives the time-reversed correlation.
// The opt-in input check: a reduction over the step's inputs, read back on the
// host before anything of the step is enqueued, so a refused step leaves the
// handle exactly as it was.
int check_inputs(sbim_ctx* c, const void* a, const void* b) {
  CU(sbim::launch_nonfinite_check(c->prec, a, b, (long long)c->field_elems(), c->d_nonfinite,
                                  c->stream));
  int flag = 0;
  CU(cudaMemcpyAsync(&flag, c->d_nonfinite, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (flag)
    return fail(SBIM_ERR_NONFINITE, "non-finite value (NaN or infinity) in the step's input; "
                                    "the step was not taken");
  return SBIM_OK;
}

int run_step(sbim_ctx* c, const void* in, const void* aux, void* out, bool adjoint,
             bool repeat = false) {
  cudaStream_t st = c->stream;
  if (c->check_finite) {
    const int rc = check_inputs(c, in, adjoint ? nullptr : aux);
    if (rc != SBIM_OK) return rc;
  }
  if (repeat) {                     // back to the level being re-evaluated
    CU(sbim::launch_rewind(c->d_step, st));
    --c->n;
  }
  cudaEvent_t* e = nullptr;
  if (c->prof) {
    if (c->prof_issued - c->prof_harvested >= kProfRing) {
      const int rc = harvest(c, c->prof_issued - kProfRing + 1);
      if (rc != SBIM_OK) return rc;
    }
    e = &c->ev[(c->prof_issued % kProfRing) * kProfEvents];
    CU(cudaEventRecord(e[0], st));
  }
  if (c->prec == SBIM_FP64)
    CF(cufftExecD2Z(c->plan_fwd, (cufftDoubleReal*)in, (cufftDoubleComplex*)c->d_uhat));
  else
    CF(cufftExecR2C(c->plan_fwd, (cufftReal*)in, (cufftComplex*)c->d_uhat));
  if (e) CU(cudaEventRecord(e[1], st));
  const sbim::StepArgs a = step_args(c);
  if (repeat)
    CU(sbim::launch_repeat_lag0(a, c->prec, st));
  else if (c->variant >= 1)
    CU(sbim::launch_conv_tma(a, c->prec, c->kahan, c->variant, st, nullptr, c->tile, c->halves));
  else
    CU(sbim::launch_conv(a, c->prec, c->kahan, st));
  if (e) CU(cudaEventRecord(e[2], st));
  CU(sbim::launch_assemble(a, c->prec, c->kahan, st));
  if (e) CU(cudaEventRecord(e[3], st));
  void* s_dst = adjoint ? out : c->d_s;
  if (c->prec == SBIM_FP64)
    CF(cufftExecZ2D(c->plan_inv, (cufftDoubleComplex*)c->d_fhat, (cufftDoubleReal*)s_dst));
  else
    CF(cufftExecC2R(c->plan_inv, (cufftComplex*)c->d_fhat, (cufftReal*)s_dst));
  if (e) CU(cudaEventRecord(e[4], st));
  const double k = c->side * c->mu / c->cs;
  const double coef[3] = {k, k * c->eta, k};
  const long long plane = (long long)c->n1 * c->n3;
  if (adjoint)
    CU(sbim::launch_adjoint_epilogue(c->prec, in, const_cast<void*>(aux), plane, coef,
                                     c->d_step, st));
  else
    CU(sbim::launch_epilogue(c->prec, c->d_s, aux, out, plane, coef, c->tau_inf, c->d_step, st));
  if (e) {
    CU(cudaEventRecord(e[5], st));
    ++c->prof_issued;
  }
  ++c->n;
  c->can_repeat = !adjoint;
  return SBIM_OK;
}

// The device error word as read after the stream drained: clears it and
// reports SBIM_ERR_TIMEOUT when a bounded wait gave up.
int take_error_word(sbim_ctx* c, int flag) {
  if (flag) {
    CU(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    return fail(SBIM_ERR_TIMEOUT, "a bounded device wait gave up; the outputs since the last check "
                                  "are invalid");
  }
  return SBIM_OK;
}

}  // namespace

extern "C" {

int sbim_step(sbim_handle h, const void* u, const void* v, void* tau) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  if (!u || !v || !tau) return fail(SBIM_ERR_ARG, "NULL field pointer");
  return run_step(h, u, v, tau, false);
}

int sbim_step_repeat(sbim_handle h, const void* u, const void* v, void* tau) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  if (!u || !v || !tau) return fail(SBIM_ERR_ARG, "NULL field pointer");
  if (!h->can_repeat || h->n == 0)
    return fail(SBIM_ERR_STATE, "sbim_step_repeat needs a preceding sbim_step on this handle "
                                "(with no other call that changes its state in between)");
  return run_step(h, u, v, tau, false, true);
}

int sbim_step_adjoint(sbim_handle h, const void* tau_bar, void* u_bar, void* v_bar) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  if (!tau_bar || !u_bar || !v_bar) return fail(SBIM_ERR_ARG, "NULL field pointer");
  if (tau_bar == u_bar || tau_bar == v_bar || u_bar == v_bar)
    return fail(SBIM_ERR_ARG, "tau_bar, u_bar and v_bar must be distinct buffers");
  return run_step(h, tau_bar, v_bar, u_bar, true);
}

int sbim_step_host(sbim_handle h, const void* u, const void* v, void* tau) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  if (!u || !v || !tau) return fail(SBIM_ERR_ARG, "NULL field pointer");
  sbim_ctx* c = h;
  const size_t bytes = c->field_elems() * c->real_size;
  const size_t hat_bytes = (size_t)3 * c->nbins * 2 * c->real_size;
  if (!c->h_err) CU(cudaHostAlloc((void**)&c->h_err, sizeof(int), cudaHostAllocDefault));
  if (!c->d_io) {
    CU(cudaMalloc(&c->d_io, 3 * bytes + hat_bytes));
    CU(cudaMemsetAsync((char*)c->d_io + 3 * bytes, 0, hat_bytes, c->stream));
  }
  char* du = (char*)c->d_io;
  char* dv = du + bytes;
  char* dtau = dv + bytes;
  void* zero_hat = dtau + bytes;   // all-zero spectra: never written after the memset
  cudaStream_t st = c->stream;
  if (c->prof || c->check_finite) {   // stage timing and the input check want the plain order
    CU(cudaMemcpyAsync(du, u, bytes, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(dv, v, bytes, cudaMemcpyHostToDevice, st));
    const int rc = sbim_step(h, du, dv, dtau);
    if (rc != SBIM_OK) return rc;
  } else {
    // Every lag >= 1 of Eq. (SBI)'s convolution reads only the stored history,
    // so it runs while u and v cross to the device and are transformed on the
    // side stream.  The convolution first sees zero spectra (its ring slot
    // holds zeros, lag 0 adds nothing); the lag-0 pass then stores the new
    // spectra and adds w(0) D_n to chunk 0's partial sums, as sbim_step_repeat
    // does.  Equal to sbim_step up to the order of that one addition.
    if (!c->io_stream) {
      CU(cudaStreamCreateWithFlags(&c->io_stream, cudaStreamNonBlocking));
      CU(cudaEventCreateWithFlags(&c->io_fork, cudaEventDisableTiming));
      CU(cudaEventCreateWithFlags(&c->io_join, cudaEventDisableTiming));
    }
    CU(cudaEventRecord(c->io_fork, st));
    CU(cudaStreamWaitEvent(c->io_stream, c->io_fork, 0));
    CU(cudaMemcpyAsync(du, u, bytes, cudaMemcpyHostToDevice, c->io_stream));
    CU(cudaMemcpyAsync(dv, v, bytes, cudaMemcpyHostToDevice, c->io_stream));
    int rc = sbim::handle_fft_forward(c, du, c->io_stream);
    if (rc != SBIM_OK) return rc;
    CU(cudaEventRecord(c->io_join, c->io_stream));
    sbim::StepArgs a = step_args(c);
    a.uhat = zero_hat;
    if (c->variant >= 1)
      CU(sbim::launch_conv_tma(a, c->prec, c->kahan, c->variant, st, nullptr, c->tile, c->halves));
    else
      CU(sbim::launch_conv(a, c->prec, c->kahan, st));
    CU(cudaStreamWaitEvent(st, c->io_join, 0));
    a.uhat = c->d_uhat;
    CU(sbim::launch_repeat_lag0(a, c->prec, st));
    CU(sbim::launch_assemble(a, c->prec, c->kahan, st));
    rc = sbim::handle_fft_inverse(c, st);
    if (rc != SBIM_OK) return rc;
    rc = sbim::handle_epilogue(c, dv, dtau, st);
    if (rc != SBIM_OK) return rc;
    ++c->n;
    c->can_repeat = true;
  }
  // tau and the device error word come back under one synchronisation
  CU(cudaMemcpyAsync(tau, dtau, bytes, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return take_error_word(c, *c->h_err);
}

int sbim_set_window(sbim_handle h, double window) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  if (!(window >= 0)) return fail(SBIM_ERR_ARG, "window must be >= 0");
  h->can_repeat = false;
  if (window == 0) {
    h->window = 0;
    return SBIM_OK;
  }
  // lags kept per half record; a tile's bound is the maximum over its halves
  std::vector<int> lm(2 * h->n_orb_pad), tl(h->n_orb_pad / sbim::kOrbitTile, 1);
  for (int x = 0; x < 2 * h->n_orb_pad; ++x) {
    const double d = h->h_dT[x];
    if (x >= 2 * h->n_orb) lm[x] = 1;                   // padding records
    else if (d <= 0) lm[x] = h->n_cut;                  // k = 0 (and padding halves)
    else lm[x] = (int)std::min<double>(h->n_cut, std::floor(window / d) + 1);
    int& t = tl[(x / 2) / sbim::kOrbitTile];
    t = std::max(t, lm[x]);
  }
  if (!h->d_lmax) CU(cudaMalloc(&h->d_lmax, lm.size() * sizeof(int)));
  if (!h->d_tile_lmax) CU(cudaMalloc(&h->d_tile_lmax, tl.size() * sizeof(int)));
  CU(cudaMemcpyAsync(h->d_lmax, lm.data(), lm.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(h->d_tile_lmax, tl.data(), tl.size() * sizeof(int), cudaMemcpyHostToDevice,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->window = window;
  return SBIM_OK;
}

int sbim_set_check_finite(sbim_handle h, int enable) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  if (enable && !h->d_nonfinite) CU(cudaMalloc(&h->d_nonfinite, sizeof(int)));
  h->check_finite = enable != 0;
  return SBIM_OK;
}

int sbim_check_device(sbim_handle h) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  int flag = 0;
  CU(cudaMemcpyAsync(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return take_error_word(h, flag);
}

int sbim_selftest_wait_timeout(sbim_handle h) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  int rc = sbim_check_device(h);                 // start from a clear error word
  if (rc != SBIM_OK) return rc;
  CU(sbim::launch_wait_selftest(h->d_err, h->stream));
  rc = sbim_check_device(h);                     // waits for the stream
  if (rc == SBIM_ERR_TIMEOUT) {
    g_err.clear();
    return sbim_check_device(h);                 // and the word is clear again
  }
  return fail(SBIM_ERR_STATE, "the bounded wait did not report its failure (status %d)", rc);
}

int sbim_set_conv_config(sbim_handle h, int variant, int lags_per_cta) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  if (variant < 0 || variant > 3) return fail(SBIM_ERR_ARG, "variant must be 0..3");
  if (lags_per_cta < 0) return fail(SBIM_ERR_ARG, "lags_per_cta must be >= 0");
  h->can_repeat = false;
  const int old_v = h->variant, old_l = h->lags_per_cta, old_lc = h->lc, old_nc = h->nchunks;
  h->variant = variant;
  h->lags_per_cta = lags_per_cta;
  if (variant >= 1) {
    const cudaError_t e = sbim::prepare_conv_tma(h->prec, h->kahan, variant, h->tile, h->halves);
    if (e != cudaSuccess) {
      h->variant = old_v;
      h->lags_per_cta = old_l;
      return fail(SBIM_ERR_CUDA, "kernel attributes: %s", cudaGetErrorString(e));
    }
  }
  int rc = choose_chunks(*h);
  if (rc == SBIM_OK) rc = alloc_partials(*h);
  if (rc != SBIM_OK) {
    h->variant = old_v; h->lags_per_cta = old_l; h->lc = old_lc; h->nchunks = old_nc;
    return rc;
  }
  return SBIM_OK;
}

int sbim_set_conv_tile(sbim_handle h, int orbits_per_cta) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  if (orbits_per_cta != 64 && orbits_per_cta != 128 && orbits_per_cta != 256)
    return fail(SBIM_ERR_ARG, "orbits per CTA must be 64, 128 or 256");
  if (h->n_orb_pad % orbits_per_cta != 0)
    return fail(SBIM_ERR_ARG, "the handle's %d orbit records are not a multiple of %d",
                h->n_orb_pad, orbits_per_cta);
  h->can_repeat = false;
  const int old_t = h->tile, old_lc = h->lc, old_nc = h->nchunks;
  h->tile = orbits_per_cta;
  if (h->variant >= 1) {
    const cudaError_t e = sbim::prepare_conv_tma(h->prec, h->kahan, h->variant, h->tile, h->halves);
    if (e != cudaSuccess) {
      h->tile = old_t;
      return fail(SBIM_ERR_CUDA, "kernel attributes: %s", cudaGetErrorString(e));
    }
  }
  int rc = choose_chunks(*h);
  if (rc == SBIM_OK) rc = alloc_partials(*h);
  if (rc != SBIM_OK) {
    h->tile = old_t; h->lc = old_lc; h->nchunks = old_nc;
    return rc;
  }
  return SBIM_OK;
}

int sbim_set_far_field(sbim_handle h, const double tau_inf[3]) {
  if (!h || !tau_inf) return fail(SBIM_ERR_ARG, "NULL argument");
  for (int i = 0; i < 3; ++i) h->tau_inf[i] = tau_inf[i];
  return SBIM_OK;
}

int sbim_reset(sbim_handle h) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  CU(cudaMemsetAsync(h->d_step, 0, sizeof(long long), h->stream));
  h->n = 0;
  h->can_repeat = false;
  return SBIM_OK;
}

int sbim_rewind(sbim_handle h) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  if (h->n == 0) return fail(SBIM_ERR_STATE, "no step to rewind");
  CU(sbim::launch_rewind(h->d_step, h->stream));
  --h->n;
  h->can_repeat = false;
  return SBIM_OK;
}

int sbim_get_step(sbim_handle h, long long* n) {
  if (!h || !n) return fail(SBIM_ERR_ARG, "NULL argument");
  *n = h->n;
  return SBIM_OK;
}

namespace {
// Checkpoint header: the parameters a restored handle must match, then the state.
struct SaveHeader {
  char magic[8];
  int version, n1, n3, n_cut, side, prec, n_orb_pad, pad0;
  double L1, L3, cs, cp, rho, dt;
  long long n, hist_bytes;
  double tau_inf[3];
};
constexpr char kSaveMagic[8] = {'S', 'B', 'I', 'M', 'H', 'S', 'T', '1'};
constexpr int kSaveVersion = 1;

SaveHeader make_header(const sbim_ctx& c) {
  SaveHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kSaveMagic, 8);
  hd.version = kSaveVersion;
  hd.n1 = c.n1; hd.n3 = c.n3; hd.n_cut = c.n_cut; hd.side = c.side; hd.prec = c.prec;
  hd.n_orb_pad = c.n_orb_pad;
  hd.L1 = c.L1; hd.L3 = c.L3; hd.cs = c.cs; hd.cp = c.cp; hd.rho = c.rho; hd.dt = c.dt;
  hd.n = c.n;
  hd.hist_bytes = (long long)c.hist_bytes;
  for (int i = 0; i < 3; ++i) hd.tau_inf[i] = c.tau_inf[i];
  return hd;
}
}  // namespace

int sbim_save(sbim_handle h, void* buf, size_t* bytes) {
  if (!h || !bytes) return fail(SBIM_ERR_ARG, "NULL argument");
  const size_t need = sizeof(SaveHeader) + h->hist_bytes;
  if (!buf) {
    *bytes = need;
    return SBIM_OK;
  }
  if (*bytes < need) {
    const size_t have = *bytes;
    *bytes = need;
    return fail(SBIM_ERR_ARG, "checkpoint buffer holds %zu bytes, %zu needed", have, need);
  }
  const SaveHeader hd = make_header(*h);
  std::memcpy(buf, &hd, sizeof(hd));
  CU(cudaMemcpyAsync((char*)buf + sizeof(hd), h->d_hist, h->hist_bytes, cudaMemcpyDeviceToHost,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));
  *bytes = need;
  return SBIM_OK;
}

int sbim_load(sbim_handle h, const void* buf, size_t bytes) {
  if (!h || !buf) return fail(SBIM_ERR_ARG, "NULL argument");
  if (bytes < sizeof(SaveHeader)) return fail(SBIM_ERR_ARG, "checkpoint is truncated");
  SaveHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  const SaveHeader me = make_header(*h);
  if (std::memcmp(hd.magic, kSaveMagic, 8) != 0) return fail(SBIM_ERR_ARG, "not a checkpoint");
  if (hd.version != kSaveVersion) return fail(SBIM_ERR_ARG, "checkpoint version %d", hd.version);
  if (hd.n1 != me.n1 || hd.n3 != me.n3 || hd.n_cut != me.n_cut || hd.side != me.side ||
      hd.prec != me.prec || hd.n_orb_pad != me.n_orb_pad || hd.L1 != me.L1 || hd.L3 != me.L3 ||
      hd.cs != me.cs || hd.cp != me.cp || hd.rho != me.rho || hd.dt != me.dt ||
      hd.hist_bytes != me.hist_bytes)
    return fail(SBIM_ERR_ARG, "checkpoint was taken from a handle with other parameters");
  if (hd.n < 0) return fail(SBIM_ERR_ARG, "checkpoint step counter is negative");
  if (bytes < sizeof(hd) + (size_t)hd.hist_bytes) return fail(SBIM_ERR_ARG, "checkpoint is truncated");
  CU(cudaMemcpyAsync(h->d_hist, (const char*)buf + sizeof(hd), h->hist_bytes,
                     cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(h->d_step, &hd.n, sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->n = hd.n;
  h->can_repeat = false;
  for (int i = 0; i < 3; ++i) h->tau_inf[i] = hd.tau_inf[i];
  return SBIM_OK;
}

int sbim_get_info(sbim_handle h, long long* n_modes, long long* n_slots, long long* hist_bytes,
                  long long* table_nodes) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  if (n_modes) *n_modes = h->nbins;
  if (n_slots) *n_slots = (long long)h->n_orb_pad * 4;
  if (hist_bytes) *hist_bytes = (long long)h->hist_bytes;
  if (table_nodes) *table_nodes = h->tab_n;
  return SBIM_OK;
}

int sbim_set_profiling(sbim_handle h, int enable) {
  if (!h) return fail(SBIM_ERR_ARG, "NULL handle");
  if (enable && h->ev.empty()) {
    h->ev.resize((size_t)kProfRing * kProfEvents);
    for (auto& e : h->ev) CU(cudaEventCreate(&e));
  }
  if (h->prof) {
    const int rc = harvest(h, h->prof_issued);
    if (rc != SBIM_OK) return rc;
  }
  h->prof = enable != 0;
  h->prof_issued = h->prof_harvested = 0;
  for (double& x : h->prof_ms) x = 0.0;
  return SBIM_OK;
}

int sbim_stage_times(sbim_handle h, double ms[5], long long* steps) {
  if (!h || !ms) return fail(SBIM_ERR_ARG, "NULL argument");
  const int rc = harvest(h, h->prof_issued);
  if (rc != SBIM_OK) return rc;
  for (int k = 0; k < 5; ++k) ms[k] = h->prof_ms[k];
  if (steps) *steps = h->prof_harvested;
  return SBIM_OK;
}

int sbim_destroy(sbim_handle h) {
  if (!h) return SBIM_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  release(h);
  return SBIM_OK;
}

const char* sbim_last_error(void) { return g_err.c_str(); }

}  // extern "C"
