// Coarse part of one step with the coupling weights formed in the kernel.
//
// k_coarse reads the per-draw edge weights K_ij(w) = sum_e c_e^2(w) G_e[i][j]
// that k_edge_weights stored once per solve: 37 % of its DRAM bytes.  The
// random field at the element quadrature points is a lower-order cost
// (Sec. 3.2), so this variant forms every weight it needs from the draw's
// xi and the sample-independent psi rows and G entries instead, with the
// same operations in the same order as k_edge_weights (so the same values
// bit for bit), and is otherwise k_coarse: g = a(u_n) - M^-1 F(t_n) on R,
// the closed-form leapfrog update outside R.  Uniform batches of meshes with
// at most four neighbours per node beyond the overflow list (no second
// neighbour table).
#pragma once
#include "kernels.cuh"

namespace lflts {

// c_e^2 of element t for VEC draws (xr: the draws' padded xi).
template <typename Real, int VEC, int KP>
__device__ __forceinline__ void coef_of_element(const Real* __restrict__ psi, int t, const Real (&xr)[VEC][KP],
                                                Real (&c2)[VEC]) {
  Real pe[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) pe[k] = __ldg(psi + (size_t)t * KP + k);
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    Real acc = Real(0);
#pragma unroll
    for (int k = 0; k < KP; ++k) acc = fma(xr[v][k], pe[k], acc);
    c2[v] = coef_exp(acc);
  }
}

// The weight of edge e for VEC draws: k_edge_weights' sum over its elements.
template <typename Real, int VEC, int KP>
__device__ __forceinline__ Pack<Real, VEC> edge_weight_rc(const int2* __restrict__ ee, const Real* __restrict__ eg,
                                                          const Real* __restrict__ psi, int e,
                                                          const Real (&xr)[VEC][KP]) {
  const int2 el = __ldg(ee + e);
  Pack<Real, VEC> w;
#pragma unroll
  for (int v = 0; v < VEC; ++v) w.v[v] = Real(0);
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int t = side ? el.y : el.x;
    if (t < 0) continue;
    const Real G = __ldg(eg + 2 * e + side);
    Real c2[VEC];
    coef_of_element<Real, VEC, KP>(psi, t, xr, c2);
#pragma unroll
    for (int v = 0; v < VEC; ++v) w.v[v] = fma(c2[v], G, w.v[v]);
  }
  return w;
}

template <typename Real, int VEC, int KP>
__global__ void __launch_bounds__(256)
k_coarse_rc(MeshDev<Real> m, int S, int SB, const int2* __restrict__ ee, const Real* __restrict__ eg,
            const Real* __restrict__ psi, const Real* __restrict__ xi, const Real* __restrict__ u,
            Real* __restrict__ u_next, Real* __restrict__ d, Real* __restrict__ g, Real kappa_gamma,
            const Real* __restrict__ fw, Real famp) {
  const Lane l = lane_of(SB);
  const int s0 = l.sv * VEC;
  if (s0 >= S) return;
  Real xr[VEC][KP];
#pragma unroll
  for (int v = 0; v < VEC; ++v)
#pragma unroll
    for (int k = 0; k < KP; ++k) xr[v][k] = xi[(size_t)(s0 + v) * KP + k];
  for (int i = blockIdx.x * l.NB + l.row; i < m.n_free; i += gridDim.x * l.NB) {
    const size_t is = (size_t)i * S + s0;
    const bool outside = i >= m.n_R;
    const Nb4 nb = load_nb4(m, i);
    const int t0 = m.adj_ptr[i] + 4, t1 = m.adj_ptr[i + 1];
    const Pack<Real, VEC> ui = ldp<Real, VEC>(u + is);
    Pack<Real, VEC> uj[4], dn;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (nb.j[q] >= 0) {
        uj[q] = ldp<Real, VEC>(u + (size_t)nb.j[q] * S + s0);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) uj[q].v[k] = Real(0);
      }
    }
    if (outside) dn = ldp<Real, VEC>(d + is);
    const Real mi = m.minv[i];
    Real acc[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) acc[k] = Real(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Pack<Real, VEC> w;
      if (nb.j[q] >= 0) {
        w = edge_weight_rc<Real, VEC, KP>(ee, eg, psi, nb.e[q], xr);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) w.v[k] = Real(0);
      }
#pragma unroll
      for (int k = 0; k < VEC; ++k) acc[k] = fma(w.v[k], uj[q].v[k] - ui.v[k], acc[k]);
    }
    for (int t = t0; t < t1; ++t) {  // neighbours beyond the fourth
      const int2 o = m.adj[t];
      const Pack<Real, VEC> uo = ldp<Real, VEC>(u + (size_t)o.x * S + s0);
      const Pack<Real, VEC> wo = edge_weight_rc<Real, VEC, KP>(ee, eg, psi, o.y, xr);
#pragma unroll
      for (int k = 0; k < VEC; ++k) acc[k] = fma(wo.v[k], uo.v[k] - ui.v[k], acc[k]);
    }
    Pack<Real, VEC> gi;
    const Real fi = fw ? famp * fw[i] : Real(0);
#pragma unroll
    for (int k = 0; k < VEC; ++k) gi.v[k] = mi * acc[k] - fi;
    if (outside) {
      Pack<Real, VEC> un;
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        dn.v[k] = dn.v[k] - kappa_gamma * gi.v[k];
        un.v[k] = ui.v[k] + dn.v[k];
      }
      stp<Real, VEC>(d + is, dn);
      stp<Real, VEC>(u_next + is, un);
    } else {
      stp<Real, VEC>(g + is, gi);
    }
  }
}

}  // namespace lflts
