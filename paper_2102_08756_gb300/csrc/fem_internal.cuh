// Internal declarations of the explicit FEM slab (Section 2.2) used by the
// hybrid FEM-SBIM driver (Section 2.4).
#pragma once

#include <cuda_runtime.h>

namespace sbim {
namespace fem {

struct MeshArgs {
  int n1, n3, L;      // nodes along x1, x3; node layers
  int f;              // minus-copy layer of the split fault plane
  int fault;          // 1 if the plane at layer f is split
  double area;        // h^2: nodal area of boundary and fault nodes
  double half_mass;   // rho h^3 / 2: mass from the 4 elements on one side of a node
};

// The assembled hex8 stiffness, negated (-K), as a 27-point stencil of 3x3
// blocks split by the element layer it comes from: [side: below, above]
// [18 = (ox, oy, oz)][3][3].
// Passed to the kernels by value, so its entries are kernel-parameter constants
// that the multiply-adds read directly (no load instruction per entry).
template <class R>
struct Stencil {
  R s[2 * 18 * 9];
};

// The four elements on one side of a node are mirror-symmetric in x1 and in x3,
// so the block of a neighbour with no offset along x1 (ox == 1) couples the x1
// component only with itself, and likewise for x3 (oz == 1): entry (c, d) of such
// a block vanishes when exactly one of c, d is that axis (components 0 = x1,
// 2 = x3).  88 of the 324 entries vanish; the assembly sets them to exactly 0.
// (The column-march kernels use the symmetry itself: they read only the +x1 /
// +x3 neighbours' coefficients, never a vanishing one.)
__host__ __device__ constexpr bool stencil_entry_vanishes(int ox, int oz, int c, int d) {
  return (ox == 1 && ((c == 0) != (d == 0))) || (oz == 1 && ((c == 2) != (d == 2)));
}

template <class R>
struct FaultArgs {
  const R* mu_s;      // [n3][n1] static friction coefficient
  const R* tau0;      // [n3][n1] x1 shear prestress (Pa)
  R mu_k, Dc, sigma0; // dynamic friction, slip-weakening distance (m), normal prestress (Pa)
  R* traction;        // [3][n3][n1] output: fault traction perturbation (Pa), or NULL
};

// Buffers of the transpose of one step (all [L][3][n3][n1] unless noted).
template <class R>
struct AdjointArgs {
  const R *u, *v, *a;         // state before the step
  R *un, *vp, *af;            // recomputed u_new, v_pred, a_free
  R *lu, *lv, *la;            // in: cotangent after the step; out: before
  R *lun, *lvp, *lan, *lao;   // cotangents of u_new, v_pred, a_with_fault (then a_free), a
  R* lF;                      // cotangent of the force
  R *tb_top, *tb_bot;         // [3][n3][n1] cotangents of the SBIM tractions
  const R* tau_bar;           // [3][n3][n1] cotangent of the fault traction output (or NULL)
  R* ddc;                     // [n3][n1] accumulated d/dDc
  R dt;
  int weld;
};

// stage 0: recompute u_new, v_pred; 1: corrector transpose; 2: fault transpose;
// 3: mass and SBIM cotangents; 4: stiffness transpose; 5: predictor transpose.
template <class R>
cudaError_t adjoint_stages(const AdjointArgs<R>& j, const MeshArgs& g, const Stencil<R>& S,
                           const FaultArgs<R>& fa, int stage, cudaStream_t st);
template <class R> cudaError_t layer_add(R* dst, const R* src, long long n, cudaStream_t st);

template <class R> cudaError_t predict(R* u, R* v, const R* a, long long n, R dt, cudaStream_t st);
template <class R>
cudaError_t force(const R* u, R* an, const MeshArgs& g, const Stencil<R>& S, const R* tau_top,
                  const R* tau_bot, const R* src, cudaStream_t st);
template <class R>
cudaError_t fault(const R* u, const R* vpred, const R* a, R* an, const MeshArgs& g,
                  const FaultArgs<R>& fa, R dt, int weld, cudaStream_t st);
template <class R> cudaError_t correct(R* v, R* a, const R* an, long long n, R dt, cudaStream_t st);
template <class R>
cudaError_t fault_fields(const R* u, const R* v, const MeshArgs& g, R* slip, R* rate,
                         cudaStream_t st);

}  // namespace fem
}  // namespace sbim
