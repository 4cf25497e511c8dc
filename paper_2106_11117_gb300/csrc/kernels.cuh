// LF-LTS kernels for sm_103a (GB300).  u-form of Alg. 2 in increment variables.
//
// The paper's Alg. 2 is written for z = M^{1/2} u with A = M^{-1/2} K M^{-1/2}.
// M and P are diagonal, so they commute, and multiplying every line of Alg. 2
// by M^{-1/2} gives the same algorithm for u with A replaced by
// a(v) = M^{-1} K v.  The kernels use that u-form and increments, so that FP32
// rounding acts on small quantities:
//   d_n = u_n - u_{n-1}                (d_0 = dt v0)
//   r_m = q_{m/p} - q_0,  q_0 = u_n   (r_0 = 0)
//   g   = a(u_n)       [ = w_n + A P q_0 of Alg. 2, since A is linear ]
//   r_1     = -c_0 g,                      c_0 = dt^2 / (omega delta)
//   r_{m+1} = (1 + beta_m) r_m - beta_m r_{m-1} - c_m (g + a(P r_m)),
//                                          c_m = 2 dt^2 beta_{m+1/2} / omega
//   d_{n+1} = d_n + kappa r_p,  u_{n+1} = u_n + d_{n+1}
// with kappa = 2 (z_{n+1} = 2 q_1 - z_{n-1}) and kappa = 1 on the first step
// (start value z_1 = q_1(z_0) + dt M^{1/2} v0).  A node outside R (no P node
// in any incident element) has a(P r_m) = 0, so its r_p = -gamma g with the
// scalar gamma of the same recursion (gamma = dt^2 / 2: Alg. 2 is leapfrog
// away from the refined region, Sec. 3.3).
//
// Layout: sample-major state [node][S]; the thread (node i, sample s) reads
// neighbours at [j][s], so a warp over 32 consecutive samples of one node
// issues one 128-byte transaction per neighbour.  Element coefficients are
// recomputed in registers: c_e^2 = exp2(sum_k xi_k psi2[e][k]) with psi2
// pre-scaled by log2(e).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace lflts {

template <typename Real> struct Vec2T;
template <> struct Vec2T<float> { using type = float2; };
template <> struct Vec2T<double> { using type = double2; };

template <typename Real>
struct MeshDev {
  int n_free, n_R, n_P;
  const int* __restrict__ inc_ptr;                       // [n_free + 1]
  const int4* __restrict__ inc;                          // (e, j1, j2, 0)
  const typename Vec2T<Real>::type* __restrict__ w;      // (G_i,j1, G_i,j2)
  const Real* __restrict__ minv;                         // [n_free]
  const Real* __restrict__ psi2;                         // [n_tri][KP]
};

__device__ __forceinline__ float exp2_r(float x) { return exp2f(x); }
__device__ __forceinline__ double exp2_r(double x) { return exp2(x); }

// c_e^2 for the draw held in registers.
template <typename Real, int KP>
__device__ __forceinline__ Real coef(const Real (&xr)[KP], const Real* __restrict__ pe) {
  Real acc = Real(0);
#pragma unroll
  for (int k = 0; k < KP; ++k) acc = fma(xr[k], __ldg(pe + k), acc);
  return exp2_r(acc);
}

template <typename Real, int KP>
__device__ __forceinline__ void load_xi(Real (&xr)[KP], const Real* __restrict__ xi, int s) {
#pragma unroll
  for (int k = 0; k < KP; ++k) xr[k] = xi[(size_t)s * KP + k];
}

// ---------------------------------------------------------------------------
// Coarse part of one step, all free nodes: g = a(u_n).
//   outside R: d += -kappa*gamma*g, u_next = u_n + d
//   inside  R: store g and r_1 = -c0 g
// Thread layout: blockDim.x = 256 = SB samples x (256/SB) node rows.
// ---------------------------------------------------------------------------
template <typename Real, int KP>
__global__ void __launch_bounds__(256)
k_coarse(MeshDev<Real> m, const Real* __restrict__ xi, int S, int SB,
         const Real* __restrict__ u, Real* __restrict__ u_next, Real* __restrict__ d,
         Real* __restrict__ g, Real* __restrict__ r1, Real kappa_gamma, Real c0) {
  const int ls = threadIdx.x & (SB - 1);
  const int NB = blockDim.x / SB;
  const int ln = threadIdx.x / SB;
  const int s = blockIdx.y * SB + ls;
  if (s >= S) return;
  Real xr[KP];
  load_xi<Real, KP>(xr, xi, s);
  for (int i = blockIdx.x * NB + ln; i < m.n_free; i += gridDim.x * NB) {
    const size_t is = (size_t)i * S + s;
    const Real ui = u[is];
    Real acc = Real(0);
    const int t1 = m.inc_ptr[i + 1];
    for (int t = m.inc_ptr[i]; t < t1; ++t) {
      const int4 ie = m.inc[t];
      const auto w = m.w[t];
      const Real c2 = coef<Real, KP>(xr, m.psi2 + (size_t)ie.x * KP);
      const Real u1 = u[(size_t)ie.y * S + s];
      const Real u2 = u[(size_t)ie.z * S + s];
      acc = fma(c2, w.x * (u1 - ui) + w.y * (u2 - ui), acc);
    }
    const Real gi = m.minv[i] * acc;
    if (i >= m.n_R) {
      const Real dn = d[is] - kappa_gamma * gi;
      d[is] = dn;
      u_next[is] = ui + dn;
    } else {
      g[is] = gi;
      r1[is] = -c0 * gi;
    }
  }
}

// ---------------------------------------------------------------------------
// One inner substep m on R:  r_{m+1} = (1+beta) r_m - beta r_{m-1} - cm (g + a(P r_m)).
// FIRST: r_{m-1} = r_0 = 0.  LAST: fold r_p into d and u_next instead of storing it.
// ---------------------------------------------------------------------------
template <typename Real, int KP, bool FIRST, bool LAST>
__global__ void __launch_bounds__(256)
k_inner(MeshDev<Real> m, const Real* __restrict__ xi, int S, int SB,
        const Real* __restrict__ r_cur, const Real* __restrict__ r_prev, Real* __restrict__ r_next,
        const Real* __restrict__ g, const Real* __restrict__ u, Real* __restrict__ u_next,
        Real* __restrict__ d, Real one_plus_beta, Real beta, Real cm, Real kappa) {
  const int ls = threadIdx.x & (SB - 1);
  const int NB = blockDim.x / SB;
  const int ln = threadIdx.x / SB;
  const int s = blockIdx.y * SB + ls;
  if (s >= S) return;
  Real xr[KP];
  load_xi<Real, KP>(xr, xi, s);
  const int nP = m.n_P;
  for (int i = blockIdx.x * NB + ln; i < m.n_R; i += gridDim.x * NB) {
    const size_t is = (size_t)i * S + s;
    const Real rc = r_cur[is];
    const bool iP = i < nP;
    const Real vi = iP ? rc : Real(0);
    Real acc = Real(0);
    const int t1 = m.inc_ptr[i + 1];
    for (int t = m.inc_ptr[i]; t < t1; ++t) {
      const int4 ie = m.inc[t];
      const bool p1 = ie.y < nP, p2 = ie.z < nP;
      if (!(iP || p1 || p2)) continue;  // element without P vertex: no AP term
      const auto w = m.w[t];
      const Real c2 = coef<Real, KP>(xr, m.psi2 + (size_t)ie.x * KP);
      const Real v1 = p1 ? r_cur[(size_t)ie.y * S + s] : Real(0);
      const Real v2 = p2 ? r_cur[(size_t)ie.z * S + s] : Real(0);
      acc = fma(c2, w.x * (v1 - vi) + w.y * (v2 - vi), acc);
    }
    const Real rp = FIRST ? Real(0) : r_prev[is];
    const Real rn = one_plus_beta * rc - beta * rp - cm * (g[is] + m.minv[i] * acc);
    if (LAST) {
      const Real dn = d[is] + kappa * rn;
      d[is] = dn;
      u_next[is] = u[is] + dn;
    } else {
      r_next[is] = rn;
    }
  }
}

// ---------------------------------------------------------------------------
// Initial state: u = u0 (both buffers), d = dt v0; xi padded to KP in Real.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_init_state(int64_t n_nodes, int S, const Real* __restrict__ u0,
                             const Real* __restrict__ v0, Real dt, Real* __restrict__ ua,
                             Real* __restrict__ ub, Real* __restrict__ d) {
  const int64_t total = n_nodes * (int64_t)S;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / S;
    const Real v = u0[i];
    ua[k] = v;
    ub[k] = v;
    d[k] = v0 ? dt * v0[i] : Real(0);
  }
}

template <typename Real, int KP>
__global__ void k_xi_pad(int S, int K, const double* __restrict__ xi, Real* __restrict__ out) {
  const int64_t total = (int64_t)S * KP;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / KP;
    const int k = (int)(t % KP);
    out[t] = k < K ? (Real)xi[s * K + k] : Real(0);
  }
}

// ---------------------------------------------------------------------------
// Compensated (Neumaier) FP64 accumulation.
// ---------------------------------------------------------------------------
struct Neumaier {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ void merge(const Neumaier& o) {
    add(o.s);
    c += o.c;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

// QoI stage 1: partial sums of g_k u[idx_k][s] over chunks of the weights.
template <typename Real>
__global__ void k_qoi_partial(const Real* __restrict__ u, int S, const int* __restrict__ idx,
                              const double* __restrict__ gw, int nnz, int chunk,
                              double* __restrict__ ps, double* __restrict__ pc) {
  const int s = blockIdx.y * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int c = blockIdx.x;
  const int k0 = c * chunk, k1 = min(nnz, k0 + chunk);
  Neumaier acc;
  for (int k = k0; k < k1; ++k) acc.add(gw[k] * (double)u[(size_t)idx[k] * S + s]);
  ps[(size_t)c * S + s] = acc.s;
  pc[(size_t)c * S + s] = acc.c;
}

// QoI stage 2: combine the chunk partials in chunk order; flag non-finite Q.
__global__ void k_qoi_final(int n_chunks, int S, const double* __restrict__ ps,
                            const double* __restrict__ pc, double* __restrict__ Q, int* bad) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  Neumaier acc;
  for (int c = 0; c < n_chunks; ++c) {
    acc.add(ps[(size_t)c * S + s]);
    acc.c += pc[(size_t)c * S + s];
  }
  const double q = acc.value();
  Q[s] = q;
  if (!isfinite(q)) atomicMin(bad, s);
}

// Gather the state back to the caller's node order in FP64.
template <typename Real>
__global__ void k_gather_state(int64_t n_nodes, int S, const int* __restrict__ new2old,
                               const Real* __restrict__ u, double* __restrict__ out) {
  const int64_t total = n_nodes * (int64_t)S;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / S, s = k % S;
    out[(int64_t)new2old[i] * S + s] = (double)u[k];
  }
}

// dQ = Qf - Qc for one pair job (Qc == nullptr: level 0, dQ = Qf).
__global__ void k_pair_diff(int S, const double* __restrict__ Qf, const double* __restrict__ Qc,
                            double* __restrict__ dQ, double* __restrict__ Qf_out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double f = Qf[s];
  dQ[s] = Qc ? f - Qc[s] : f;
  if (Qf_out) Qf_out[s] = f;
}

// MLMC level sums: one block, fixed-order compensated reduction.
__global__ void __launch_bounds__(256)
k_level_sums(int64_t S, const double* __restrict__ Qf, const double* __restrict__ Qc,
             double* __restrict__ sums) {
  __shared__ double sh_s[4][256], sh_c[4][256];
  Neumaier a[4];
  for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
    const double f = Qf[s];
    const double dq = Qc ? f - Qc[s] : f;
    a[0].add(dq);
    a[1].add(dq * dq);
    a[2].add(f);
    a[3].add(f * f);
  }
  for (int j = 0; j < 4; ++j) {
    sh_s[j][threadIdx.x] = a[j].s;
    sh_c[j][threadIdx.x] = a[j].c;
  }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      for (int j = 0; j < 4; ++j) {
        Neumaier x;
        x.s = sh_s[j][threadIdx.x];
        x.c = sh_c[j][threadIdx.x];
        Neumaier y;
        y.s = sh_s[j][threadIdx.x + w];
        y.c = sh_c[j][threadIdx.x + w];
        x.merge(y);
        sh_s[j][threadIdx.x] = x.s;
        sh_c[j][threadIdx.x] = x.c;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) sums[j] = sh_s[j][0] + sh_c[j][0];
}

}  // namespace lflts
