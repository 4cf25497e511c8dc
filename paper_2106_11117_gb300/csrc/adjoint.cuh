// Discrete adjoint of the u-form LF-LTS solve: gradient of the QoI with
// respect to the field parameters xi (included by lflts.cu).
//
// One step of Alg. 2 in u-form is u_{n+1} = 2 T u_n - u_{n-1} with
// T u = u + r_p(u), r_p linear in u and depending on xi through K(xi); the
// start is u_1 = T u_0 + dt v0.  With Q = g_Q . u_N the Lagrange multipliers
// mu_n satisfy mu_N = g_Q, mu_n = 2 T^T mu_{n+1} - mu_{n+2}, and
//   dQ/dxi_k = sum_{n=0}^{N-1} kappa_n mu_{n+1} . (dT/dxi_k) u_n,
// kappa_0 = 1, kappa_n = 2.  T is M-self-adjoint (the z-form step operator is
// symmetric), so nu = M^{-1} mu obeys the forward recursion itself:
//   nu_N = M^{-1} g_Q, nu_n = 2 T nu_{n+1} - nu_{n+2}  (nu_{N+1} = 0),
// and the forward step kernels advance nu (kappa = 2 from the start).
//
// dT/dxi_k u_n differentiates the inner recursion (g = M^-1 K u,
// r_1 = -c_0 g, r_{m+1} = (1+b_m) r_m - b_m r_{m-1} - c_m (g + M^-1 K P r_m)).
// Its adjoint, for the weight sigma = kappa_n nu_{n+1} (scaled by M^{-1}):
//   rho_p = sigma,
//   rho_m = (1+b_m) rho_{m+1} - b_{m+1} rho_{m+2} - c_m P a(rho_{m+1})   (rho_{p+1} = 0)
// and, with dK = dK/dxi_k and y_m = u_n + P r_m,
//   kappa_n mu_{n+1} . dT u_n = sum_{edges ij} dK_ij A^{(n)}_ij,
//   A^{(n)}_ij = c_0 (rho_1,i - rho_1,j)(u_i - u_j)
//              + sum_{m=1}^{p-1} c_m (rho_{m+1},i - rho_{m+1},j)(y_m,i - y_m,j)
// using x^T dK y = -sum_edges dK_ij (x_i - x_j)(y_i - y_j).  On an edge with no
// P endpoint rho_m = alpha_m sigma and y_m = u_n, so A^{(n)} = gamma (sigma_i -
// sigma_j)(u_i - u_j) with gamma = dt^2/2 (the leapfrog adjoint).  Finally
//   dQ/dxi_k = sum_edges A_ij sum_{e ni ij} psi_{e,k} c_e^2 G_e[i][j].
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.cuh"

namespace lflts {

// rho_m on R: dst = a1 s1 src1 - b1 s2 src2 - cm [i in P] a(s1 src1)_i.
template <typename Real, int VEC>
__global__ void __launch_bounds__(256)
k_adj_inner(MeshDev<Real> m, int S, int SB, const Real* __restrict__ W, const Real* __restrict__ src1,
            Real s1, const Real* __restrict__ src2, Real s2, Real* __restrict__ dst, Real a1, Real b1, Real cm) {
  const Lane l = lane_of(SB);
  const int s0 = l.sv * VEC;
  if (s0 >= S) return;
  const int nP = m.n_P, nR = m.n_R;
  for (int i = blockIdx.x * l.NB + l.row; i < nR; i += gridDim.x * l.NB) {
    const size_t is = (size_t)i * S + s0;
    const Pack<Real, VEC> xi = ldp<Real, VEC>(src1 + is);
    Pack<Real, VEC> x2;
    if (src2) {
      x2 = ldp<Real, VEC>(src2 + is);
    } else {
#pragma unroll
      for (int k = 0; k < VEC; ++k) x2.v[k] = Real(0);
    }
    Real acc[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) acc[k] = Real(0);
    if (i < nP) {  // P a(x): only P nodes carry the apply
      const int t1 = m.adj_ptr[i + 1];
      for (int t = m.adj_ptr[i]; t < t1; ++t) {
        const int2 nb = m.adj[t];
        const Pack<Real, VEC> w = ldp<Real, VEC>(W + (size_t)nb.y * S + s0);
        Pack<Real, VEC> xj;
        if (nb.x < nR) {
          xj = ldp<Real, VEC>(src1 + (size_t)nb.x * S + s0);
        } else {  // Dirichlet neighbour (value 0); other nodes are in R
#pragma unroll
          for (int k = 0; k < VEC; ++k) xj.v[k] = Real(0);
        }
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc[k] = fma(w.v[k], s1 * (xj.v[k] - xi.v[k]), acc[k]);
      }
    }
    const Real mi = m.minv[i];
    Pack<Real, VEC> out;
#pragma unroll
    for (int k = 0; k < VEC; ++k) out.v[k] = a1 * (s1 * xi.v[k]) - b1 * (s2 * x2.v[k]) - cm * (mi * acc[k]);
    stp<Real, VEC>(dst + is, out);
  }
}

// Inner-recursion coefficients for the edge accumulation (p <= 64).
struct AdjConsts {
  double c[65];   // c[0] = c_0, c[m] = c_m, m = 1..p-1
  double gamma;   // dt^2/2 from the same recursion
  double kappa;   // weight of this step (1 for n = 0, else 2)
  int p;
};

// A[e] += A^{(n)}_e for every edge (FP64 accumulators, one thread per edge
// and sample).  u: u_n (full), nu: nu_{n+1} (full), gs: a(u_n) on R,
// rs: r_2..r_{p-1} on R ([p-2][n_R][S]), rho: rho_1..rho_{p-1} on R
// ([p-1][n_R][S]); rho_p = kappa nu.
template <typename Real>
__global__ void __launch_bounds__(256)
k_adj_edges(int64_t n_edges, int n_P, int n_R, int S, int SB, const int2* __restrict__ ends,
            const Real* __restrict__ u, const Real* __restrict__ nu, const Real* __restrict__ gs,
            const Real* __restrict__ rs, const Real* __restrict__ rho, double* __restrict__ A, AdjConsts k) {
  const int s = blockIdx.y * SB + (threadIdx.x & (SB - 1));
  if (s >= S) return;
  const int NB = blockDim.x / SB;
  const size_t RS = (size_t)n_R * S;
  for (int64_t e = (int64_t)blockIdx.x * NB + threadIdx.x / SB; e < n_edges; e += (int64_t)gridDim.x * NB) {
    const int2 ij = ends[e];
    const int i = ij.x, j = ij.y;  // i < j
    const double du = (double)u[(size_t)i * S + s] - (double)u[(size_t)j * S + s];
    double acc;
    if (i >= n_P) {  // no P endpoint: leapfrog adjoint term
      const double ds = (double)nu[(size_t)i * S + s] - (double)nu[(size_t)j * S + s];
      acc = k.gamma * k.kappa * ds * du;
    } else {
      // both endpoints are in R (or j is a Dirichlet node, whose values are 0)
      const bool jR = j < n_R, jP = j < n_P;
      const size_t oi = (size_t)i * S + s, oj = (size_t)j * S + s;
      auto rho_at = [&](int mm, bool at_j) -> double {  // rho_mm, mm = 1..p
        if (at_j && !jR) return 0.0;
        const size_t o = at_j ? oj : oi;
        if (mm == k.p) return k.kappa * (double)nu[o];
        return (double)rho[(size_t)(mm - 1) * RS + o];
      };
      auto pr_at = [&](int mm, bool at_j) -> double {  // (P r_mm), mm = 1..p-1
        if (at_j && !jP) return 0.0;
        const size_t o = at_j ? oj : oi;
        if (mm == 1) return -k.c[0] * (double)gs[o];
        return (double)rs[(size_t)(mm - 2) * RS + o];
      };
      acc = k.c[0] * (rho_at(1, false) - rho_at(1, true)) * du;
      for (int mm = 1; mm < k.p; ++mm) {
        const double dy = du + pr_at(mm, false) - pr_at(mm, true);
        acc += k.c[mm] * (rho_at(mm + 1, false) - rho_at(mm + 1, true)) * dy;
      }
    }
    A[(size_t)e * S + s] += acc;
  }
}

// FP32 path of the edge accumulation: VEC draws per thread, FP32 arithmetic
// (the state it reads is FP32), added into a per-segment FP32 accumulator
// Aseg that k_adj_fold adds into the FP64 A at the end of every checkpoint
// segment (so FP32 sums run over at most one segment of steps).  Same terms
// as k_adj_edges.  FP64 work on this GPU runs at a small fraction of the
// FP32 rate, which made the FP64 form of this kernel ALU-bound.
struct AdjConsts32 {
  float c[65];
  float gk;  // gamma * kappa
  float kappa;
  int p;
};

template <int VEC>
__global__ void __launch_bounds__(256)
k_adj_edges32(int64_t n_edges, int n_P, int n_R, int S, int SB, const int2* __restrict__ ends,
              const float* __restrict__ u, const float* __restrict__ nu, const float* __restrict__ gs,
              const float* __restrict__ rs, const float* __restrict__ rho, float* __restrict__ Aseg,
              const AdjConsts32 k) {
  const Lane l = lane_of(SB);
  const int s0 = l.sv * VEC;
  if (s0 >= S) return;
  const size_t RS = (size_t)n_R * S;
  for (int64_t e = (int64_t)blockIdx.x * l.NB + l.row; e < n_edges; e += (int64_t)gridDim.x * l.NB) {
    const int2 ij = ends[e];
    const int i = ij.x, j = ij.y;  // i < j
    const size_t oi = (size_t)i * S + s0, oj = (size_t)j * S + s0;
    const Pack<float, VEC> ui = ldp<float, VEC>(u + oi), uj = ldp<float, VEC>(u + oj);
    const size_t oa = (size_t)e * S + s0;
    Pack<float, VEC> a = ldp<float, VEC>(Aseg + oa);
    float du[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) du[q] = ui.v[q] - uj.v[q];
    if (i >= n_P) {  // no P endpoint: leapfrog adjoint term
      const Pack<float, VEC> vi = ldp<float, VEC>(nu + oi), vj = ldp<float, VEC>(nu + oj);
#pragma unroll
      for (int q = 0; q < VEC; ++q) a.v[q] += k.gk * (vi.v[q] - vj.v[q]) * du[q];
    } else {
      // i in P; j in R, or a Dirichlet node (values 0)
      const bool jR = j < n_R, jP = j < n_P;
      auto rho_of = [&](int mm, size_t o) -> Pack<float, VEC> {  // rho_mm at offset o, mm = 1..p
        if (mm == k.p) {
          Pack<float, VEC> r = ldp<float, VEC>(nu + o);
#pragma unroll
          for (int q = 0; q < VEC; ++q) r.v[q] *= k.kappa;
          return r;
        }
        return ldp<float, VEC>(rho + (size_t)(mm - 1) * RS + o);
      };
      auto pr_of = [&](int mm, size_t o) -> Pack<float, VEC> {  // (P r_mm) at offset o, mm = 1..p-1
        if (mm == 1) {
          Pack<float, VEC> r = ldp<float, VEC>(gs + o);
#pragma unroll
          for (int q = 0; q < VEC; ++q) r.v[q] *= -k.c[0];
          return r;
        }
        return ldp<float, VEC>(rs + (size_t)(mm - 2) * RS + o);
      };
      Pack<float, VEC> zero;
#pragma unroll
      for (int q = 0; q < VEC; ++q) zero.v[q] = 0.f;
      Pack<float, VEC> ri = rho_of(1, oi), rj = jR ? rho_of(1, oj) : zero;
      float acc[VEC];
#pragma unroll
      for (int q = 0; q < VEC; ++q) acc[q] = k.c[0] * (ri.v[q] - rj.v[q]) * du[q];
      for (int mm = 1; mm < k.p; ++mm) {
        const Pack<float, VEC> pi = pr_of(mm, oi), pj = jP ? pr_of(mm, oj) : zero;
        ri = rho_of(mm + 1, oi);
        rj = jR ? rho_of(mm + 1, oj) : zero;
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          const float dy = du[q] + pi.v[q] - pj.v[q];
          acc[q] += k.c[mm] * (ri.v[q] - rj.v[q]) * dy;
        }
      }
#pragma unroll
      for (int q = 0; q < VEC; ++q) a.v[q] += acc[q];
    }
    stp<float, VEC>(Aseg + oa, a);
  }
}

// A += Aseg, Aseg = 0 (end of a checkpoint segment of the FP32 adjoint).
__global__ void k_adj_fold(int64_t n, float* __restrict__ Aseg, double* __restrict__ A) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    A[t] += (double)Aseg[t];
    Aseg[t] = 0.f;
  }
}

// nu_N = M^{-1} g_Q on the QoI nodes (the state arrays are zeroed before).
template <typename Real>
__global__ void k_adj_seed(int nnz, int S, const int* __restrict__ idx, const double* __restrict__ gq,
                           const double* __restrict__ minv_full, int n_free, Real* __restrict__ nu,
                           Real* __restrict__ dnu) {
  const int64_t total = (int64_t)nnz * S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / S), s = (int)(t % S);
    const int r = idx[k];
    if (r >= n_free) continue;  // Dirichlet node: not a degree of freedom
    const Real v = (Real)(gq[k] * minv_full[r]);
    nu[(size_t)r * S + s] = v;
    dnu[(size_t)r * S + s] = v;
  }
}

// Partial contraction over a chunk of edges:
// part[c][s][k] = sum_{e in chunk c} A_e(s) sum_{e' ni e} psi_{e',k} c_{e'}^2(s) G_{e'}.
template <int KP>
__global__ void __launch_bounds__(128)
k_grad_contract(int64_t n_edges, int S, int64_t chunk, const int2* __restrict__ ee, const double* __restrict__ eg,
                const double* __restrict__ psi, const double* __restrict__ xi, int K,
                const double* __restrict__ A, double* __restrict__ part) {
  const int s = blockIdx.y * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int c = blockIdx.x;
  double xr[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) xr[k] = k < K ? xi[(size_t)s * K + k] : 0.0;
  double acc[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) acc[k] = 0.0;
  const int64_t e0 = c * chunk, e1 = min(n_edges, e0 + chunk);
  for (int64_t e = e0; e < e1; ++e) {
    const double a = A[(size_t)e * S + s];
    const int2 el = ee[e];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int t = side ? el.y : el.x;
      if (t < 0) continue;
      const double* pe = psi + (size_t)t * KP;
      double ex = 0.0;
#pragma unroll
      for (int k = 0; k < KP; ++k) ex = fma(xr[k], pe[k], ex);
      const double f = a * exp(ex) * eg[2 * e + side];
#pragma unroll
      for (int k = 0; k < KP; ++k) acc[k] = fma(f, pe[k], acc[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < KP; ++k)
    if (k < K) part[((size_t)c * S + s) * K + k] = acc[k];
}

__global__ void k_grad_finish(int n_chunks, int S, int K, const double* __restrict__ part, double* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)S * K) return;
  Neumaier acc;
  for (int c = 0; c < n_chunks; ++c) acc.add(part[(size_t)c * S * K + t]);
  out[t] = acc.value();
}

}  // namespace lflts
