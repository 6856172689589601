// Explicit FEM slab with a slip-weakening fault (Section 2.2) -- the volume part
// of the hybrid time step of Section 2.4.
//
// Mesh: n1 x n2 x n3 cubes of side h, periodic in x1 and x3, node layers
// l = 0 .. L-1 from the bottom; with a fault the node plane at element layer
// f = n2/2 is split into layer f (minus copy, elements below) and f+1 (plus
// copy, elements above).  Fields are [L][3][n3][n1] (x1 fastest), so each
// layer is a [3][n3][n1] block that the SBIM entry points take directly.
//
// Homogeneous material on a regular mesh: K u is a 27-point stencil of 3x3
// blocks.  It splits into the contribution of the four elements below a node
// (offsets o2 in {-1, 0}) and of the four above (o2 in {0, +1}); a node layer
// has elements below unless it is the bottom layer or the fault's plus copy,
// and above unless it is the top layer or the fault's minus copy.  The 2 x 18
// blocks are assembled on the host from the hexahedron stiffness.
#include "../../include/sbim.h"
#include "fem_internal.cuh"

namespace sbim {
namespace fem {

namespace {


// v_pred = v + dt a; u <- u + dt v + dt^2/2 a  (Eq. (fepred); central-difference
// displacement update).  v is overwritten by v_pred.
template <class R>
__global__ void predict_kernel(R* __restrict__ u, R* __restrict__ v, const R* __restrict__ a,
                               long long n, R dt) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const R vi = v[i], ai = a[i];
    u[i] += dt * vi + (R)0.5 * dt * dt * ai;
    v[i] = vi + dt * ai;
  }
}

// One node layer of a field around a node, the 3 x 3 in-plane neighbourhood
// (periodic in x1 and x3) of each component d, held as the nine sums and
// differences of mirrored neighbours that the stencil's mirror symmetry lets
// share one coefficient: with x[oz][ox] the neighbour at offset (ox - 1, oz - 1),
//   CC = x[1][1]                          centre
//   XS, XD = x[1][2] +- x[1][0]           x1 neighbours
//   ZS, ZD = x[2][1] +- x[0][1]           x3 neighbours
//   SS, DS, SD, DD = corners, even/odd (S/D) in x1 then in x3:
//     x[2][2] + sx x[2][0] + sz x[0][2] + sx sz x[0][0].
enum { CC, XS, XD, ZS, ZD, SS, DS, SD, DD };
template <class R>
struct Window {
  R k[3][9];
};

// Columns per CTA of the column march: kTX along x1 (one warp) by kTZ along x3,
// one thread per (i1, i3) column.  Each node layer's values over the tile and a
// one-node halo ([3][kHZ][kHX], periodic wrap) are staged in shared memory by
// asynchronous copies, kStages layers deep, so a thread's 27-value window of a
// layer is 27 shared-memory loads at constant offsets.
constexpr int kTX = 32, kTZ = 4, kColThreads = kTX * kTZ;
constexpr int kHX = kTX + 2, kHZ = kTZ + 2;
constexpr int kLayerTile = 3 * kHZ * kHX;
constexpr int kStages = 3;
constexpr int kFillPer = (kLayerTile + kColThreads - 1) / kColThreads;

template <class R>
__device__ __forceinline__ void cp_async_elem(R* dst, const R* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(sizeof(R))
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// A layer's window from its shared-memory tile: 27 loads, 36 adds.
template <class R>
__device__ __forceinline__ void load_window(const R* __restrict__ tile, int tz, int tx, Window<R>& w) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R x[3][3];
#pragma unroll
    for (int oz = 0; oz < 3; ++oz)
#pragma unroll
      for (int ox = 0; ox < 3; ++ox) x[oz][ox] = tile[(d * kHZ + tz + oz) * kHX + tx + ox];
    const R p = x[2][2] + x[2][0], m = x[2][2] - x[2][0];
    const R q = x[0][2] + x[0][0], r = x[0][2] - x[0][0];
    w.k[d][CC] = x[1][1];
    w.k[d][XS] = x[1][2] + x[1][0];
    w.k[d][XD] = x[1][2] - x[1][0];
    w.k[d][ZS] = x[2][1] + x[0][1];
    w.k[d][ZD] = x[2][1] - x[0][1];
    w.k[d][SS] = p + q;
    w.k[d][DS] = m + r;
    w.k[d][SD] = p - q;
    w.k[d][DD] = m - r;
  }
}

// F += (-K) x from the element layer on one side of the node: side 0 (below)
// spans node layers l-1 (lo) and l (hi), side 1 (above) layers l and l+1.  The
// four elements on one side of a node are mirror-symmetric in x1 and x3, so
// block (c, d) of the neighbour at -x1 equals sx times that at +x1, with
// sx = -1 when exactly one of c, d is the x1 component (likewise sz for x3; the
// assembled stencil holds these equalities to rounding, exactly in float).  Each
// block (c, d) therefore takes the +x1 / +x3 neighbours' coefficients times the
// window's sums (even) or differences (odd): 4, 2, 2 or 1 multiply-adds for
// (sx, sz) = (+, +), (-, +), (+, -), (-, -); 88 per node instead of the 236
// nonzero stencil entries.  Fully unrolled; the stencil holds -K and reaches
// the kernel by value, so every coefficient is a constant-bank operand.
template <int SIDE, class R>
__device__ __forceinline__ void apply_side(const Stencil<R>& S, const Window<R>& lo,
                                           const Window<R>& hi, R (&F)[3]) {
#pragma unroll
  for (int oy = 0; oy < 2; ++oy) {
    const Window<R>& w = oy == 0 ? lo : hi;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        // coefficient of the neighbour at (ox, oz) in block (c, d)
        auto co = [&](int ox, int oz) { return S.s[SIDE * 18 * 9 + ((ox * 2 + oy) * 3 + oz) * 9 + 3 * c + d]; };
        const bool odd_x = (c == 0) != (d == 0), odd_z = (c == 2) != (d == 2);
        if (!odd_x && !odd_z) {
          F[c] = fma(co(1, 1), w.k[d][CC], F[c]);
          F[c] = fma(co(2, 1), w.k[d][XS], F[c]);
          F[c] = fma(co(1, 2), w.k[d][ZS], F[c]);
          F[c] = fma(co(2, 2), w.k[d][SS], F[c]);
        } else if (odd_x && !odd_z) {
          F[c] = fma(co(2, 1), w.k[d][XD], F[c]);
          F[c] = fma(co(2, 2), w.k[d][DS], F[c]);
        } else if (!odd_x && odd_z) {
          F[c] = fma(co(1, 2), w.k[d][ZD], F[c]);
          F[c] = fma(co(2, 2), w.k[d][SD], F[c]);
        } else {
          F[c] = fma(co(2, 2), w.k[d][DD], F[c]);
        }
      }
  }
}

// The stencil -K x for every node of the CTA's kTX x kTZ columns, marching up
// the node layers with two register windows: at layer l one holds layer l-1 and
// the other layer l; after the blocks below the node are applied, the first is
// refilled with layer l+1 (from shared memory) for the blocks above, and the two
// swap roles for layer l+1.  The copy of layer l+2's tile starts as layer l
// begins, into the buffer of layer l-1 (last read while layer l-2 was computed,
// before the barrier of layer l-1), and is waited for one layer later.  A
// layer's element blocks below (down) and above (up) exist unless they cross
// the split fault plane or the slab's faces.  Per node of a column inside the
// grid, epi(l, q0, down, up, F) finishes; threads of columns outside it still
// copy and synchronise.
template <class R, class Epi>
__device__ __forceinline__ void stencil_columns(const R* __restrict__ x, const MeshArgs& g,
                                                const Stencil<R>& S, Epi epi) {
  __shared__ __align__(16) R tiles[kStages][kLayerTile];
  const int tx = threadIdx.x % kTX, tz = threadIdx.x / kTX;
  const int x0 = blockIdx.x * kTX, z0 = blockIdx.y * kTZ;
  const int i1 = x0 + tx, i3 = z0 + tz;
  const bool inside = i1 < g.n1 && i3 < g.n3;
  const long long plane = (long long)g.n1 * g.n3;
  const long long layer = 3 * plane;
  // this thread's share of a layer tile: tile index and in-layer source offset
  int ti[kFillPer];
  long long src[kFillPer];
#pragma unroll
  for (int k = 0; k < kFillPer; ++k) {
    const int e = threadIdx.x + k * kColThreads;
    ti[k] = e < kLayerTile ? e : -1;
    const int c = e / (kHZ * kHX), r = (e / kHX) % kHZ, q = e % kHX;
    const int j3 = ((z0 - 1 + r) % g.n3 + g.n3) % g.n3;
    const int j1 = ((x0 - 1 + q) % g.n1 + g.n1) % g.n1;
    src[k] = c * plane + (long long)j3 * g.n1 + j1;
  }
  auto fill = [&](int l) {
    if (l < g.L) {
      R* t = tiles[l % kStages];
      const R* xl = x + (long long)l * layer;
#pragma unroll
      for (int k = 0; k < kFillPer; ++k)
        if (ti[k] >= 0) cp_async_elem(t + ti[k], xl + src[k]);
    }
    cp_async_commit();   // an empty group past the top layer keeps the count uniform
  };
  const long long q0 = inside ? (long long)i3 * g.n1 + i1 : 0;
  fill(0);
  fill(1);
  cp_async_wait<1>();    // layer 0 landed
  __syncthreads();
  Window<R> A, B;
  load_window(tiles[0], tz, tx, B);
  int l = 0;
  auto node = [&](Window<R>& prev, Window<R>& cur) {
    fill(l + 2);
    const bool down = l > 0 && !(g.fault && l == g.f + 1);
    const bool up = l < g.L - 1 && !(g.fault && l == g.f);
    R F[3] = {(R)0, (R)0, (R)0};
    if (down) apply_side<0>(S, prev, cur, F);
    cp_async_wait<1>();    // layer l+1 landed (layer l+2 may still be in flight)
    __syncthreads();
    if (l + 1 < g.L) load_window(tiles[(l + 1) % kStages], tz, tx, prev);   // prev := layer l+1
    if (up) apply_side<1>(S, cur, prev, F);
    if (inside) epi(l, q0, down, up, F);
    ++l;
  };
  while (l < g.L) {
    node(A, B);
    if (l >= g.L) break;
    node(B, A);
  }
  cp_async_wait<0>();
}

// an = (-K u + f_boundary) / m: the acceleration without fault traction.
// f_boundary = +A tau_top on the top layer, -A tau_bot on the bottom layer.
template <class R>
__global__ void __launch_bounds__(kColThreads) force_kernel(const R* __restrict__ u, R* __restrict__ an,
                                                    MeshArgs g, const __grid_constant__ Stencil<R> S,
                                                    const R* __restrict__ tau_top,
                                                    const R* __restrict__ tau_bot,
                                                    const R* __restrict__ src) {
  const long long plane = (long long)g.n1 * g.n3;
  // 1 / lumped mass of a node with elements on both sides or on one (every node
  // of a slab has elements on at least one side), converted and divided once
  const R hm = (R)g.half_mass;
  const R inv_m1 = (R)1 / hm, inv_m2 = (R)1 / (hm + hm);
  stencil_columns(u, g, S, [&](int l, long long q0, bool down, bool up, R(&F)[3]) {
    if (l == g.L - 1 && tau_top)
#pragma unroll
      for (int c = 0; c < 3; ++c) F[c] += g.area * tau_top[c * plane + q0];
    if (l == 0 && tau_bot)
#pragma unroll
      for (int c = 0; c < 3; ++c) F[c] -= g.area * tau_bot[c * plane + q0];
    const R inv_m = (down && up) ? inv_m2 : inv_m1;
    R* al = an + (long long)l * 3 * plane;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R extra = src ? src[((long long)l * 3 + c) * plane + q0] : (R)0;
      al[c * plane + q0] = (F[c] + extra) * inv_m;
    }
  });
}

// Fault traction by the forward Lagrange-multiplier method (Eqs. (freeslip),
// (sticktraction), (stickslip)) with linear slip weakening (Eq. (slipweak)), in
// the perturbation formulation: shear traction tau0 + tau, normal stress
// (compression positive) sigma0 - tau_2; the normal component always sticks.
// Applies -A tau / m+ to the plus copy and +A tau / m- to the minus copy.
template <class R>
__global__ void fault_kernel(const R* __restrict__ u, const R* __restrict__ vpred,
                             const R* __restrict__ a, R* __restrict__ an, MeshArgs g,
                             FaultArgs<R> fa, R dt, int weld) {
  const long long plane = (long long)g.n1 * g.n3;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= plane) return;
  const long long P = (long long)(g.f + 1) * 3 * plane + q;   // plus copy, component 0
  const long long M = (long long)g.f * 3 * plane + q;         // minus copy
  const R m = (R)g.half_mass;                                 // each copy: 4 elements
  R stick[3], slipc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long long o = c * plane;
    const R vp = vpred[P + o] - (R)0.5 * dt * a[P + o] + dt * an[P + o];
    const R vm = vpred[M + o] - (R)0.5 * dt * a[M + o] + dt * an[M + o];
    stick[c] = (vp - vm) / (dt * (R)g.area * ((R)2 / m));
    slipc[c] = u[P + o] - u[M + o];
  }
  R tau[3] = {stick[0], stick[1], stick[2]};
  if (!weld) {
    const R slip = sqrt(slipc[0] * slipc[0] + slipc[2] * slipc[2]);
    const R mus = fa.mu_s[q];
    const R fric = slip < fa.Dc ? mus - (mus - fa.mu_k) * slip / fa.Dc : fa.mu_k;
    const R strength = (fa.sigma0 - stick[1]) * fric;
    const R t1 = fa.tau0[q] + stick[0], t3 = stick[2];
    const R mag = sqrt(t1 * t1 + t3 * t3);
    if (mag > strength) {
      const R s = strength / mag;
      tau[0] = t1 * s - fa.tau0[q];
      tau[2] = t3 * s;
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long long o = c * plane;
    an[P + o] -= (R)g.area * tau[c] / m;
    an[M + o] += (R)g.area * tau[c] / m;
    if (fa.traction) fa.traction[o + q] = tau[c];
  }
}

// v = v_pred + dt/2 (a_{t+1} - a_t)  (Eq. (fecorr)); a = a_{t+1}.
template <class R>
__global__ void correct_kernel(R* __restrict__ v, R* __restrict__ a, const R* __restrict__ an,
                               long long n, R dt) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const R anew = an[i];
    v[i] += (R)0.5 * dt * (anew - a[i]);
    a[i] = anew;
  }
}

// slip vector, slip rate and (given) traction of the fault plane, [3][n3][n1]
template <class R>
__global__ void fault_fields_kernel(const R* __restrict__ u, const R* __restrict__ v, MeshArgs g,
                                   R* __restrict__ slip, R* __restrict__ rate) {
  const long long plane = (long long)g.n1 * g.n3;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= plane) return;
  const long long P = (long long)(g.f + 1) * 3 * plane + q;
  const long long M = (long long)g.f * 3 * plane + q;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (slip) slip[c * plane + q] = u[P + c * plane] - u[M + c * plane];
    if (rate) rate[c * plane + q] = v[P + c * plane] - v[M + c * plane];
  }
}

// ----------------------------------------------------------------------------
// Transpose of one hybrid step (reverse sweep for gradients).  Notation: for a
// forward quantity x, lx is the cotangent d(functional)/dx.
// ----------------------------------------------------------------------------

// u_new = u + dt v + dt^2/2 a, v_pred = v + dt a (into separate buffers)
template <class R>
__global__ void predict_to_kernel(const R* __restrict__ u, const R* __restrict__ v,
                                  const R* __restrict__ a, R* __restrict__ un, R* __restrict__ vp,
                                  long long n, R dt) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    un[i] = u[i] + dt * v[i] + (R)0.5 * dt * dt * a[i];
    vp[i] = v[i] + dt * a[i];
  }
}

// corrector transpose: lvp = lv, lan = dt/2 lv + la, la_out = -dt/2 lv; lun = lu
template <class R>
__global__ void adj_correct_kernel(const R* __restrict__ lu, const R* __restrict__ lv,
                                   const R* __restrict__ la, R* __restrict__ lun,
                                   R* __restrict__ lvp, R* __restrict__ lan, R* __restrict__ lao,
                                   long long n, R dt) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const R x = lv[i];
    lun[i] = lu[i];
    lvp[i] = x;
    lan[i] = (R)0.5 * dt * x + la[i];
    lao[i] = -(R)0.5 * dt * x;
  }
}

// Fault transpose at one split node.  Recomputes the forward fault quantities
// from u_new, v_pred, a, a_free; lan enters as the cotangent of the
// accelerations with fault forces and leaves (on the two fault layers) as that
// of a_free; adds to lun (slip), lvp and lao (free slip-rate predictor), and
// dDc (strength).
template <class R>
__global__ void adj_fault_kernel(const R* __restrict__ un, const R* __restrict__ vp,
                                 const R* __restrict__ a, const R* __restrict__ af,
                                 R* __restrict__ lan, R* __restrict__ lun, R* __restrict__ lvp,
                                 R* __restrict__ lao, const R* __restrict__ tau_bar,
                                 R* __restrict__ ddc, MeshArgs g, FaultArgs<R> fa, R dt, int weld) {
  const long long plane = (long long)g.n1 * g.n3;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= plane) return;
  const long long P = (long long)(g.f + 1) * 3 * plane + q;
  const long long M = (long long)g.f * 3 * plane + q;
  const R m = (R)g.half_mass;
  const R A = (R)g.area;
  const R imp = dt * A * ((R)2 / m);
  R stick[3], du[3], tb[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long long o = c * plane;
    const R vfp = vp[P + o] - (R)0.5 * dt * a[P + o] + dt * af[P + o];
    const R vfm = vp[M + o] - (R)0.5 * dt * a[M + o] + dt * af[M + o];
    stick[c] = (vfp - vfm) / imp;
    du[c] = un[P + o] - un[M + o];
    tb[c] = -A / m * lan[P + o] + A / m * lan[M + o] + (tau_bar ? tau_bar[o + q] : (R)0);
  }
  R ls[3] = {tb[0], tb[1], tb[2]};
  if (!weld) {
    const R slip = sqrt(du[0] * du[0] + du[2] * du[2]);
    const R mus = fa.mu_s[q];
    const bool weak = slip < fa.Dc;
    const R fric = weak ? mus - (mus - fa.mu_k) * slip / fa.Dc : fa.mu_k;
    const R sig = fa.sigma0 - stick[1];
    const R S = sig * fric;
    const R t1 = fa.tau0[q] + stick[0], t3 = stick[2];
    const R mag = sqrt(t1 * t1 + t3 * t3);
    if (mag > S) {
      const R th1 = t1 / mag, th3 = t3 / mag;
      const R proj = th1 * tb[0] + th3 * tb[2];
      ls[0] = S / mag * (tb[0] - th1 * proj);
      ls[2] = S / mag * (tb[2] - th3 * proj);
      ls[1] = tb[1] - fric * proj;
      const R dmu_dslip = weak ? -(mus - fa.mu_k) / fa.Dc : (R)0;
      const R dmu_ddc = weak ? (mus - fa.mu_k) * slip / (fa.Dc * fa.Dc) : (R)0;
      ddc[q] += proj * sig * dmu_ddc;
      const R lslip = proj * sig * dmu_dslip;
      if (slip > (R)0) {
        lun[P] += lslip * du[0] / slip;
        lun[M] -= lslip * du[0] / slip;
        lun[P + 2 * plane] += lslip * du[2] / slip;
        lun[M + 2 * plane] -= lslip * du[2] / slip;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long long o = c * plane;
    const R lvf = ls[c] / imp;
    lvp[P + o] += lvf;
    lvp[M + o] -= lvf;
    lao[P + o] -= (R)0.5 * dt * lvf;
    lao[M + o] += (R)0.5 * dt * lvf;
    lan[P + o] += dt * lvf;    // from here on: the cotangent of a_free
    lan[M + o] -= dt * lvf;
  }
}

// lF = laf / m (per layer), and the SBIM cotangents tb_top = A lF[top],
// tb_bot = -A lF[0]
template <class R>
__global__ void adj_mass_kernel(const R* __restrict__ laf, R* __restrict__ lF, MeshArgs g,
                                R* __restrict__ tb_top, R* __restrict__ tb_bot) {
  const long long plane = (long long)g.n1 * g.n3;
  const long long n = (long long)g.L * 3 * plane;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(i / (3 * plane));
    const bool down = l > 0 && !(g.fault && l == g.f + 1);
    const bool up = l < g.L - 1 && !(g.fault && l == g.f);
    const R m = (down ? (R)g.half_mass : (R)0) + (up ? (R)g.half_mass : (R)0);
    const R x = laf[i] / m;
    lF[i] = x;
    const long long r = i - (long long)l * 3 * plane;
    if (tb_top && l == g.L - 1) tb_top[r] = (R)g.area * x;
    if (tb_bot && l == 0) tb_bot[r] = -(R)g.area * x;
  }
}

// out += -K x (the stiffness is symmetric: this is the transpose of -K u)
template <class R>
__global__ void __launch_bounds__(kColThreads) stiffness_add_kernel(const R* __restrict__ x,
                                                            R* __restrict__ out, MeshArgs g,
                                                            const __grid_constant__ Stencil<R> S) {
  const long long plane = (long long)g.n1 * g.n3;
  stencil_columns(x, g, S, [&](int l, long long q0, bool, bool, R(&F)[3]) {
    R* ol = out + (long long)l * 3 * plane + q0;
#pragma unroll
    for (int c = 0; c < 3; ++c) ol[c * plane] += F[c];
  });
}

// dst[layer][...] += src[...] on one layer (boundary cotangents from the SBIM transposes)
template <class R>
__global__ void layer_add_kernel(R* __restrict__ dst, const R* __restrict__ src, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] += src[i];
}

// predictor transpose: lu = lun, lv = lvp + dt lun, la = lao + dt lvp + dt^2/2 lun
template <class R>
__global__ void adj_predict_kernel(const R* __restrict__ lun, const R* __restrict__ lvp,
                                   const R* __restrict__ lao, R* __restrict__ lu,
                                   R* __restrict__ lv, R* __restrict__ la, long long n, R dt) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const R x = lun[i], y = lvp[i];
    lu[i] = x;
    lv[i] = y + dt * x;
    la[i] = lao[i] + dt * y + (R)0.5 * dt * dt * x;
  }
}

dim3 column_grid(const MeshArgs& g) {
  return dim3((unsigned)((g.n1 + kTX - 1) / kTX), (unsigned)((g.n3 + kTZ - 1) / kTZ));
}

unsigned grid1(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (unsigned)(b > 152 * 32 ? 152 * 32 : b);
}

}  // namespace

template <class R>
cudaError_t predict(R* u, R* v, const R* a, long long n, R dt, cudaStream_t st) {
  predict_kernel<R><<<grid1(n, 256), 256, 0, st>>>(u, v, a, n, dt);
  return cudaGetLastError();
}

template <class R>
cudaError_t force(const R* u, R* an, const MeshArgs& g, const Stencil<R>& S, const R* tau_top,
                  const R* tau_bot, const R* src, cudaStream_t st) {
  force_kernel<R><<<column_grid(g), kColThreads, 0, st>>>(u, an, g, S, tau_top, tau_bot, src);
  return cudaGetLastError();
}

template <class R>
cudaError_t fault(const R* u, const R* vpred, const R* a, R* an, const MeshArgs& g,
                  const FaultArgs<R>& fa, R dt, int weld, cudaStream_t st) {
  const long long plane = (long long)g.n1 * g.n3;
  fault_kernel<R><<<(unsigned)((plane + 255) / 256), 256, 0, st>>>(u, vpred, a, an, g, fa, dt, weld);
  return cudaGetLastError();
}

template <class R>
cudaError_t correct(R* v, R* a, const R* an, long long n, R dt, cudaStream_t st) {
  correct_kernel<R><<<grid1(n, 256), 256, 0, st>>>(v, a, an, n, dt);
  return cudaGetLastError();
}

template <class R>
cudaError_t fault_fields(const R* u, const R* v, const MeshArgs& g, R* slip, R* rate,
                         cudaStream_t st) {
  const long long plane = (long long)g.n1 * g.n3;
  fault_fields_kernel<R><<<(unsigned)((plane + 255) / 256), 256, 0, st>>>(u, v, g, slip, rate);
  return cudaGetLastError();
}

template <class R>
cudaError_t adjoint_stages(const AdjointArgs<R>& j, const MeshArgs& g, const Stencil<R>& S,
                           const FaultArgs<R>& fa, int stage, cudaStream_t st) {
  const long long n = (long long)g.L * 3 * g.n1 * g.n3;
  const long long plane = (long long)g.n1 * g.n3;
  const R dt = j.dt;
  switch (stage) {
    case 0:
      predict_to_kernel<R><<<grid1(n, 256), 256, 0, st>>>(j.u, j.v, j.a, j.un, j.vp, n, dt);
      break;
    case 1:
      adj_correct_kernel<R><<<grid1(n, 256), 256, 0, st>>>(j.lu, j.lv, j.la, j.lun, j.lvp, j.lan,
                                                             j.lao, n, dt);
      break;
    case 2:
      if (g.fault)
        adj_fault_kernel<R><<<(unsigned)((plane + 255) / 256), 256, 0, st>>>(
            j.un, j.vp, j.a, j.af, j.lan, j.lun, j.lvp, j.lao, j.tau_bar, j.ddc, g, fa, dt,
            j.weld);
      break;
    case 3:
      adj_mass_kernel<R><<<grid1(n, 256), 256, 0, st>>>(j.lan, j.lF, g, j.tb_top, j.tb_bot);
      break;
    case 4: {
      stiffness_add_kernel<R><<<column_grid(g), kColThreads, 0, st>>>(j.lF, j.lun, g, S);
      break;
    }
    case 5:
      adj_predict_kernel<R><<<grid1(n, 256), 256, 0, st>>>(j.lun, j.lvp, j.lao, j.lu, j.lv, j.la,
                                                             n, dt);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class R>
cudaError_t layer_add(R* dst, const R* src, long long n, cudaStream_t st) {
  layer_add_kernel<R><<<grid1(n, 256), 256, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}

#define SBIM_FEM_INST(R)                                                                     \
  template cudaError_t predict<R>(R*, R*, const R*, long long, R, cudaStream_t);             \
  template cudaError_t force<R>(const R*, R*, const MeshArgs&, const Stencil<R>&, const R*,  \
                                const R*, const R*,                                          \
                                cudaStream_t);                                               \
  template cudaError_t fault<R>(const R*, const R*, const R*, R*, const MeshArgs&,           \
                                const FaultArgs<R>&, R, int, cudaStream_t);                  \
  template cudaError_t correct<R>(R*, R*, const R*, long long, R, cudaStream_t);             \
  template cudaError_t fault_fields<R>(const R*, const R*, const MeshArgs&, R*, R*, cudaStream_t); \
  template cudaError_t adjoint_stages<R>(const AdjointArgs<R>&, const MeshArgs&,                  \
                                         const Stencil<R>&, const FaultArgs<R>&, int,            \
                                         cudaStream_t);                                          \
  template cudaError_t layer_add<R>(R*, const R*, long long, cudaStream_t);
SBIM_FEM_INST(float)
SBIM_FEM_INST(double)

}  // namespace fem
}  // namespace sbim
