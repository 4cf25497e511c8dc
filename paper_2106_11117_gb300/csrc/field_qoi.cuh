// L2(D)-valued QoI of a level pair (Sec. 4: the experiments estimate
// E[u(., T)] in V = L2(D)).  For every draw s the difference of the pair's
// final states on the fine mesh,
//   dU_s = u_l(., T) - I u_{l-1}(., T),
// with I the nodal interpolation of the coarse P1 function at the fine
// mesh's nodes (caller-supplied barycentric weights), and the FP64 sums the
// V-valued MLMC estimator needs: sum_s dU_s at every fine node (Eq.
// MLMCestimator) and ||dU_s||^2_{L2(D)} per draw and summed (Eq. Vell_est in
// the V-norm), the norm being the exact integral of the P1 function (the
// consistent mass matrix, |T|/12 (1 + delta_ab) on every element):
//   ||v||^2 = sum_T |T|/12 (v_a^2 + v_b^2 + v_c^2 + (v_a + v_b + v_c)^2).
// States come as FP64 [node][S] arrays in the caller's node order.
#pragma once
#include "kernels.cuh"

namespace lflts {

// dU in place over uf and the per-node compensated sum over the draws; one
// warp per fine node, lanes over draws, lane partials merged in lane order.
// uc == nullptr: level 0, dU = u_0.
__global__ void __launch_bounds__(256)
k_field_diff(int64_t n_f, int S, double* __restrict__ uf, const double* __restrict__ uc,
             const int* __restrict__ vert, const double* __restrict__ w, double* __restrict__ s1) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (i >= n_f) return;  // the whole warp leaves together (i is per warp)
  int v0 = 0, v1 = 0, v2 = 0;
  double w0 = 0.0, w1 = 0.0, w2 = 0.0;
  if (uc) {
    v0 = vert[3 * i];
    v1 = vert[3 * i + 1];
    v2 = vert[3 * i + 2];
    w0 = w[3 * i];
    w1 = w[3 * i + 1];
    w2 = w[3 * i + 2];
  }
  Neumaier acc;
  for (int s = lane; s < S; s += 32) {
    double x = uf[(size_t)i * S + s];
    if (uc) {
      const double ic = __dadd_rn(__dadd_rn(__dmul_rn(w0, uc[(size_t)v0 * S + s]), __dmul_rn(w1, uc[(size_t)v1 * S + s])),
                                  __dmul_rn(w2, uc[(size_t)v2 * S + s]));
      x = __dsub_rn(x, ic);
      uf[(size_t)i * S + s] = x;
    }
    acc.add(x);
  }
  for (int o = 1; o < 32; ++o) {
    Neumaier t;
    t.s = __shfl_sync(0xffffffffu, acc.s, o);
    t.c = __shfl_sync(0xffffffffu, acc.c, o);
    if (lane == 0) acc.merge(t);
  }
  if (lane == 0) s1[i] = acc.value();
}

// Stage 1 of the per-draw norms: partial sums over chunks of elements.
__global__ void k_field_norm_partial(int64_t n_tri, int S, int chunk, const int* __restrict__ tri,
                                     const double* __restrict__ area, const double* __restrict__ dU,
                                     double* __restrict__ ps, double* __restrict__ pc) {
  const int s = blockIdx.y * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int64_t e0 = (int64_t)blockIdx.x * chunk, e1 = min(n_tri, e0 + chunk);
  Neumaier acc;
  for (int64_t e = e0; e < e1; ++e) {
    const double a = dU[(size_t)tri[3 * e] * S + s];
    const double b = dU[(size_t)tri[3 * e + 1] * S + s];
    const double c = dU[(size_t)tri[3 * e + 2] * S + s];
    const double sq = __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
    const double t = __dadd_rn(__dadd_rn(a, b), c);
    acc.add(__dmul_rn(area[e] / 12.0, __dadd_rn(sq, __dmul_rn(t, t))));
  }
  ps[(size_t)blockIdx.x * S + s] = acc.s;
  pc[(size_t)blockIdx.x * S + s] = acc.c;
}

}  // namespace lflts
