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
// away from the refined region, Sec. 3.3).  r_1 is never stored: it is
// -c_0 g wherever it is needed.
//
// Stiffness in edge form: (K u)_i = sum_{j ~ i} K_ij(w) (u_j - u_i) with the
// per-sample edge weights K_ij(w) = sum_e c_e^2(w) G_e[i][j] evaluated once per
// solve (the random field at the element quadrature points, Sec. 3.2: its
// cost is a lower-order term) and stored sample-major [edge][S].
//
// Layout: every per-node and per-edge array is sample-major [index][S]; a
// thread owns VEC consecutive samples of one node (float4 / double2 loads), a
// group of SB threads covers SB*VEC consecutive samples of that node, so
// neighbour reads are contiguous 128..512-byte segments.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace lflts {

template <typename Real>
struct MeshDev {
  int n_free, n_R, n_P;
  const int* __restrict__ adj_ptr;   // [n_free + 1]
  const int2* __restrict__ adj;      // (neighbour, edge), sorted by neighbour
  const int4* __restrict__ ell;      // [n_free][2]: first four (neighbour, edge), neighbour -1 = empty
  const Real* __restrict__ minv;     // [n_free]
  const int4* __restrict__ ell_hi;   // [n_free][2]: entries 5..8, or null (meshes of degree about 4)
};

// The first four neighbours of node i (almost every node of the meshes has
// exactly four stiffness neighbours): two 16-byte loads, no dependent chain.
struct Nb4 {
  int j[4], e[4];
};
template <typename Real>
__device__ __forceinline__ Nb4 load_nb4(const MeshDev<Real>& m, int i, bool hi = false) {
  const int4* tab = hi ? m.ell_hi : m.ell;
  const int4 a = __ldg(tab + 2 * i), b = __ldg(tab + 2 * i + 1);
  Nb4 r;
  r.j[0] = a.x; r.e[0] = a.y; r.j[1] = a.z; r.e[1] = a.w;
  r.j[2] = b.x; r.e[2] = b.y; r.j[3] = b.z; r.e[3] = b.w;
  return r;
}

// --- vector access of VEC consecutive samples -------------------------------
template <typename Real, int V>
struct Pack {
  Real v[V];
};

template <typename Real, int V>
__device__ __forceinline__ Pack<Real, V> ldp(const Real* __restrict__ p) {
  Pack<Real, V> r;
  if constexpr (V == 4 && sizeof(Real) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else if constexpr (V == 2 && sizeof(Real) == 8) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    r.v[0] = t.x; r.v[1] = t.y;
  } else if constexpr (V == 2 && sizeof(Real) == 4) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    r.v[0] = t.x; r.v[1] = t.y;
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) r.v[k] = p[k];
  }
  return r;
}

template <typename Real, int V>
__device__ __forceinline__ void stp(Real* __restrict__ p, const Pack<Real, V>& r) {
  if constexpr (V == 4 && sizeof(Real) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  } else if constexpr (V == 2 && sizeof(Real) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
  } else if constexpr (V == 2 && sizeof(Real) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(r.v[0], r.v[1]);
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) p[k] = r.v[k];
  }
}

// Store of the first nvalid of V values (nvalid >= V: one vector store).
template <typename Real, int V>
__device__ __forceinline__ void stp_lim(Real* __restrict__ p, const Pack<Real, V>& r, int nvalid) {
  if (nvalid >= V) {
    stp<Real, V>(p, r);
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k)
      if (k < nvalid) p[k] = r.v[k];
  }
}

// Ragged batches (draws with their own time step dt_s and step count): the
// step constants belong to a reference step dt_ref and every draw's edge
// weights carry (dt_s / dt_ref)^2, since c_0, c_m and gamma are dt^2 times
// constants of p and nu.  The forcing r(t_n) M^-1 F then needs the same
// factor and the draw's own time t_n = n dt_s; it is evaluated here, on the
// few nodes that carry a load.  dts == nullptr: a uniform batch.
struct RaggedF {
  const double* dts;
  double dt_ref, f0, t0, amp;
  int n;
};
__device__ __forceinline__ double ricker_scaled(const RaggedF& rf, int s) {
  const double dt = rf.dts[s];
  const double t = double(rf.n) * dt, x = M_PI * M_PI * rf.f0 * rf.f0 * (t - rf.t0) * (t - rf.t0);
  const double sc = (dt / rf.dt_ref) * (dt / rf.dt_ref);
  return rf.amp * (1.0 - 2.0 * x) * exp(-x) * sc;
}

// The coefficient c_e^2 = exp(xi . psi_e): the FP32 path keeps psi scaled by
// log2(e) and calls exp2f; the FP64 path keeps psi as given and calls exp,
// so that its c^2 carries no rounding of the scaled basis.
__device__ __forceinline__ float coef_exp(float x) { return exp2f(x); }
__device__ __forceinline__ double coef_exp(double x) { return exp(x); }

// Arithmetic of the inner substeps with every rounding written out (no
// contraction left to the compiler), so that the kernels that run the
// substeps (one launch per substep, all substeps of a small R, tiles of a
// large R) produce the same values bit for bit.
template <typename Real>
struct Rn;
template <>
struct Rn<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <>
struct Rn<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// One coupling term of a(P r_m)_i: acc + W_ij (s r_j - v_i), r_j = 0 off P,
// v_i = s r_i on P (0 off P), s the scale of the stored r_m; s r_j is
// rounded on its own, so that a kernel that stores r_m = s r_j already
// scaled (s = 1) gets the same values.
template <typename Real>
__device__ __forceinline__ Real couple(Real acc, Real w, Real s, Real rj, Real vi) {
  return Rn<Real>::fma(w, Rn<Real>::sub(Rn<Real>::mul(s, rj), vi), acc);
}
// r_{m+1} = (1 + beta_m) r_m - beta_m r_{m-1} - c_m (g + m_i^-1 acc), with
// r_m = src and r_{m-1} = srp
template <typename Real>
__device__ __forceinline__ Real inner_next(Real opb, Real src, Real beta, Real srp, Real cm, Real gi, Real mi,
                                           Real acc) {
  const Real c = Rn<Real>::mul(cm, Rn<Real>::fma(mi, acc, gi));
  return Rn<Real>::fma(opb, src, -Rn<Real>::fma(beta, srp, c));
}

// Thread -> (node row, sample vector) for blockDim.x = 256 threads.
struct Lane {
  int sv;   // sample-vector index (samples sv*VEC .. sv*VEC+VEC-1)
  int row;  // node row within the block
  int NB;   // node rows per block
};
__device__ __forceinline__ Lane lane_of(int SB) {
  Lane l;
  l.sv = blockIdx.y * SB + (threadIdx.x & (SB - 1));
  l.NB = blockDim.x / SB;
  l.row = threadIdx.x / SB;
  return l;
}

// ---------------------------------------------------------------------------
// Per-sample edge weights K_ij(w) = sum_e exp(xi . psi[e]) G_e[i][j].
// One thread per (edge, sample).  Once per solve.
// ---------------------------------------------------------------------------
template <typename Real, int KP>
__global__ void __launch_bounds__(256)
k_edge_weights(int64_t n_edges, int S, int SB, const int2* __restrict__ ee,
               const Real* __restrict__ eg, const Real* __restrict__ psi,
               const Real* __restrict__ xi, Real* __restrict__ W, const Real* __restrict__ sig = nullptr) {
  const int ls = threadIdx.x & (SB - 1);
  const int NB = blockDim.x / SB;
  const int s = blockIdx.y * SB + ls;
  if (s >= S) return;
  Real xr[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) xr[k] = xi[(size_t)s * KP + k];
  const Real sg = sig ? sig[s] : Real(1);  // ragged batch: (dt_s / dt_ref)^2
  for (int64_t e = (int64_t)blockIdx.x * NB + threadIdx.x / SB; e < n_edges; e += (int64_t)gridDim.x * NB) {
    const int2 el = ee[e];
    Real w = Real(0);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int t = side ? el.y : el.x;
      if (t < 0) continue;
      const Real* pe = psi + (size_t)t * KP;
      Real acc = Real(0);
#pragma unroll
      for (int k = 0; k < KP; ++k) acc = fma(xr[k], __ldg(pe + k), acc);
      w = fma(coef_exp(acc), eg[2 * e + side], w);
    }
    W[(size_t)e * S + s] = sig ? w * sg : w;
  }
}

// ---------------------------------------------------------------------------
// Coarse part of one step, all free nodes: g = a(u_n) - M^-1 F(t_n).
//   outside R: d += -kappa*gamma*g, u_next = u_n + d
//   inside  R: store g
// ---------------------------------------------------------------------------
// RAG: a ragged batch (draws [S_lim, S) finished: their u and d are not
// written; per-draw forcing amplitude); otherwise S_lim and rf are unused.
// HI: the mesh has the table of entries 5..8 (general triangulations); the
// neighbours are summed in the same order either way.
template <typename Real, int VEC, int MINB = 1, bool RAG = false, bool HI = false>
__global__ void __launch_bounds__(256, MINB)
k_coarse(MeshDev<Real> m, int S, int SB, const Real* __restrict__ W, const Real* __restrict__ u,
         Real* __restrict__ u_next, Real* __restrict__ d, Real* __restrict__ g, Real kappa_gamma,
         const Real* __restrict__ fw, Real famp, int S_lim, RaggedF rf) {
  const Lane l = lane_of(SB);
  const int s0 = l.sv * VEC;
  const int lim = RAG ? S_lim : S;
  if (s0 >= lim) return;
  const int nvalid = lim - s0;
  for (int i = blockIdx.x * l.NB + l.row; i < m.n_free; i += gridDim.x * l.NB) {
    const size_t is = (size_t)i * S + s0;
    const bool outside = i >= m.n_R;
    // issue every independent load of this node before any arithmetic
    const Nb4 nb = load_nb4(m, i);
    Nb4 nb2;
    if constexpr (HI) nb2 = load_nb4(m, i, true);
    const int t0 = m.adj_ptr[i] + (HI ? 8 : 4), t1 = m.adj_ptr[i + 1];
    const Pack<Real, VEC> ui = ldp<Real, VEC>(u + is);
    Pack<Real, VEC> uj[4], w[4], dn;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (nb.j[q] >= 0) {
        uj[q] = ldp<Real, VEC>(u + (size_t)nb.j[q] * S + s0);
        w[q] = ldp<Real, VEC>(W + (size_t)nb.e[q] * S + s0);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) uj[q].v[k] = w[q].v[k] = Real(0);
      }
    }
    if (outside) dn = ldp<Real, VEC>(d + is);
    const Real mi = m.minv[i];
    Real acc[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) acc[k] = Real(0);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < VEC; ++k) acc[k] = fma(w[q].v[k], uj[q].v[k] - ui.v[k], acc[k]);
    if constexpr (HI) {  // neighbours 5..8: indices already loaded
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (nb2.j[q] >= 0) {
          uj[q] = ldp<Real, VEC>(u + (size_t)nb2.j[q] * S + s0);
          w[q] = ldp<Real, VEC>(W + (size_t)nb2.e[q] * S + s0);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (nb2.j[q] >= 0)
#pragma unroll
          for (int k = 0; k < VEC; ++k) acc[k] = fma(w[q].v[k], uj[q].v[k] - ui.v[k], acc[k]);
    }
    for (int t = t0; t < t1; ++t) {  // neighbours beyond the fourth (eighth with HI)
      const int2 o = m.adj[t];
      const Pack<Real, VEC> uo = ldp<Real, VEC>(u + (size_t)o.x * S + s0);
      const Pack<Real, VEC> wo = ldp<Real, VEC>(W + (size_t)o.y * S + s0);
#pragma unroll
      for (int k = 0; k < VEC; ++k) acc[k] = fma(wo.v[k], uo.v[k] - ui.v[k], acc[k]);
    }
    // g = a(u_n) - M^-1 F(t_n): fw = M^-1 F (sample independent), famp = r(t_n)
    Pack<Real, VEC> gi;
    if constexpr (RAG) {
      const Real f = fw ? fw[i] : Real(0);
      const bool own = rf.dts && f != Real(0);  // the draw's own t_n and dt^2 factor
#pragma unroll
      for (int k = 0; k < VEC; ++k)
        gi.v[k] = mi * acc[k] - (own ? (Real)ricker_scaled(rf, s0 + k) * f : famp * f);
    } else {
      const Real fi = fw ? famp * fw[i] : Real(0);
#pragma unroll
      for (int k = 0; k < VEC; ++k) gi.v[k] = mi * acc[k] - fi;
    }
    if (outside) {
      Pack<Real, VEC> un;
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        dn.v[k] = dn.v[k] - kappa_gamma * gi.v[k];
        un.v[k] = ui.v[k] + dn.v[k];
      }
      if constexpr (RAG) {
        stp_lim<Real, VEC>(d + is, dn, nvalid);
        stp_lim<Real, VEC>(u_next + is, un, nvalid);
      } else {
        stp<Real, VEC>(d + is, dn);
        stp<Real, VEC>(u_next + is, un);
      }
    } else {
      stp<Real, VEC>(g + is, gi);
    }
  }
}

// ---------------------------------------------------------------------------
// One inner substep m on R:
//   r_{m+1} = (1+beta) r_m - beta r_{m-1} - cm (g + a(P r_m)),
// r_m = s_cur * cur, r_{m-1} = s_prev * prev (prev == nullptr: r_0 = 0).
// LAST: fold r_p into d and u_next instead of storing it.
// ---------------------------------------------------------------------------
template <typename Real, int VEC, bool LAST, int MINB = 1, bool RAG = false>
__global__ void __launch_bounds__(256, MINB)
k_inner(MeshDev<Real> m, int S, int SB, const Real* __restrict__ W,
        const Real* __restrict__ cur, Real s_cur, const Real* __restrict__ prev, Real s_prev,
        Real* __restrict__ r_next, const Real* __restrict__ g, const Real* __restrict__ u,
        Real* __restrict__ u_next, Real* __restrict__ d, Real one_plus_beta, Real beta, Real cm,
        Real kappa, int S_lim) {
  const Lane l = lane_of(SB);
  const int s0 = l.sv * VEC;
  const int lim = RAG ? S_lim : S;
  if (s0 >= lim) return;
  const int nvalid = lim - s0;
  const int nP = m.n_P;
  for (int i = blockIdx.x * l.NB + l.row; i < m.n_R; i += gridDim.x * l.NB) {
    const size_t is = (size_t)i * S + s0;
    const bool iP = i < nP;
    // issue every independent load of this node before any arithmetic
    const Nb4 nb = load_nb4(m, i);
    const int t0 = m.adj_ptr[i] + 4, t1 = m.adj_ptr[i + 1];
    const Pack<Real, VEC> rc = ldp<Real, VEC>(cur + is);
    const Pack<Real, VEC> gi = ldp<Real, VEC>(g + is);
    Pack<Real, VEC> rj[4], w[4], rp;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = nb.j[q];
      const bool jP = j >= 0 && j < nP;
      // only P neighbours carry r; a P node also couples to its other neighbours
      if (jP || (iP && j >= 0)) {
        w[q] = ldp<Real, VEC>(W + (size_t)nb.e[q] * S + s0);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) w[q].v[k] = Real(0);
      }
      if (jP) {
        rj[q] = ldp<Real, VEC>(cur + (size_t)j * S + s0);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) rj[q].v[k] = Real(0);
      }
    }
    if (prev) {
      rp = ldp<Real, VEC>(prev + is);
    } else {
#pragma unroll
      for (int k = 0; k < VEC; ++k) rp.v[k] = Real(0);
    }
    const Real mi = m.minv[i];
    Real vi[VEC], acc[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      vi[k] = iP ? Rn<Real>::mul(s_cur, rc.v[k]) : Real(0);
      acc[k] = Real(0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)  // a slot that does not couple has w = 0 and adds an exact zero
#pragma unroll
      for (int k = 0; k < VEC; ++k) acc[k] = couple(acc[k], w[q].v[k], s_cur, rj[q].v[k], vi[k]);
    for (int t = t0; t < t1; ++t) {  // neighbours beyond the fourth (rare)
      const int2 o = m.adj[t];
      const bool jP = o.x < nP;
      if (!jP && !iP) break;  // sorted: no P neighbour left
      const Pack<Real, VEC> wo = ldp<Real, VEC>(W + (size_t)o.y * S + s0);
      if (jP) {
        const Pack<Real, VEC> ro = ldp<Real, VEC>(cur + (size_t)o.x * S + s0);
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc[k] = couple(acc[k], wo.v[k], s_cur, ro.v[k], vi[k]);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc[k] = couple(acc[k], wo.v[k], s_cur, Real(0), vi[k]);
      }
    }
    Pack<Real, VEC> rn;
#pragma unroll
    for (int k = 0; k < VEC; ++k)
      rn.v[k] = inner_next(one_plus_beta, Rn<Real>::mul(s_cur, rc.v[k]), beta, Rn<Real>::mul(s_prev, rp.v[k]), cm,
                           gi.v[k], mi, acc[k]);
    if (LAST) {
      const Pack<Real, VEC> ui = ldp<Real, VEC>(u + is);
      Pack<Real, VEC> dn = ldp<Real, VEC>(d + is), un;
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        dn.v[k] = Rn<Real>::fma(kappa, rn.v[k], dn.v[k]);
        un.v[k] = Rn<Real>::add(ui.v[k], dn.v[k]);
      }
      if constexpr (RAG) {
        stp_lim<Real, VEC>(d + is, dn, nvalid);
        stp_lim<Real, VEC>(u_next + is, un, nvalid);
      } else {
        stp<Real, VEC>(d + is, dn);
        stp<Real, VEC>(u_next + is, un);
      }
    } else {
      stp<Real, VEC>(r_next + is, rn);
    }
  }
}

// ---------------------------------------------------------------------------
// All p-1 inner substeps of one outer step in one launch, for a small R.
//
// CTA b owns the draws [b SL, b SL + SL) (SL = SBf VEC) of every R node.
// Everything the substeps touch is staged in shared memory once: g and the
// recursion r_m of those draws (plane 0 = g, r_1 = -c_0 g is never formed;
// planes 1..3 = r_2, r_3, ... in rotation), the coupling slots of R (target
// and edge weight of the slab's draws, in the order k_inner visits them),
// their offsets and 1/m.  __syncthreads separates the substeps: the draws of
// different CTAs never interact, so no grid-wide synchronisation is needed.
// Per node the arithmetic is that of k_inner, term by term and in the same
// order (the left-out slots add exact zeros), so the result is the same bit
// for bit; only the global traffic differs (g, u, d on R and the P-edge
// weights once per step instead of once per substep).
// Shared memory: (4 n_R SL + n_slots SL + n_R) Real + (n_slots + n_R + 1) int.
template <typename Real>
struct InnerCoef {
  Real opb[64], beta[64], cm[64];  // (1 + beta_m), beta_m, c_m for m = 1..p-1
  Real neg_c0;                     // -c_0 (the scale of r_1 = -c_0 g)
  int p;
};

__host__ __device__ inline size_t fused_real_count(int nR, int n_slots, int SL) {
  return (size_t)4 * nR * SL + (size_t)n_slots * SL + (size_t)nR;
}

template <typename Real, int VEC, bool RAG = false>
__global__ void __launch_bounds__(256)
k_inner_fused(MeshDev<Real> m, int S, int SBf, const Real* __restrict__ W, const Real* __restrict__ g,
              const Real* __restrict__ u, Real* __restrict__ u_next, Real* __restrict__ d,
              const InnerCoef<Real> k, Real kappa, int S_lim, const int* __restrict__ rptr,
              const int2* __restrict__ rslot, int n_slots) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int SL = SBf * VEC;
  const int nR = m.n_R, nP = m.n_P;
  const size_t plane = (size_t)nR * SL;
  Real* wsm = sm + 4 * plane;                       // [n_slots][SL]
  Real* sminv = wsm + (size_t)n_slots * SL;         // [nR]
  const size_t ioff = (fused_real_count(nR, n_slots, SL) * sizeof(Real) + 15) / 16 * 16;
  int* sj = reinterpret_cast<int*>(smem_raw + ioff);  // [n_slots]
  int* sptr = sj + n_slots;                            // [nR + 1]
  const int lane = threadIdx.x % SBf, row = threadIdx.x / SBf, NB = blockDim.x / SBf;
  const int s0 = blockIdx.x * SL + lane * VEC;  // first draw of this thread (VEC divides S)
  const int lim = RAG ? S_lim : S;
  const bool active = s0 < lim;
  const int nvalid = lim - s0;
  const int o = lane * VEC;
  if (s0 < S)
    for (int i = row; i < nR; i += NB)
      stp<Real, VEC>(sm + (size_t)i * SL + o, ldp<Real, VEC>(g + (size_t)i * S + s0));
  for (int t = row; t < n_slots; t += NB) {
    const int2 q = rslot[t];
    if (lane == 0) sj[t] = q.x;
    if (s0 < S) stp<Real, VEC>(wsm + (size_t)t * SL + o, ldp<Real, VEC>(W + (size_t)q.y * S + s0));
  }
  for (int t = threadIdx.x; t <= nR; t += blockDim.x) sptr[t] = rptr[t];
  for (int t = threadIdx.x; t < nR; t += blockDim.x) sminv[t] = m.minv[t];
  __syncthreads();
  const Real* cur = sm;
  Real s_cur = k.neg_c0;
  const Real* prev = nullptr;
  Real s_prev = Real(0);
  int nxt = 1;
  for (int mm = 1; mm < k.p; ++mm) {
    const bool last = (mm == k.p - 1);
    Real* r_next = sm + nxt * plane;
    const Real one_plus_beta = k.opb[mm], beta = k.beta[mm], cm = k.cm[mm];
    if (active) {
      for (int i = row; i < nR; i += NB) {
        const size_t io = (size_t)i * SL + o;
        const bool iP = i < nP;
        const Pack<Real, VEC> rc = ldp<Real, VEC>(cur + io);
        const Pack<Real, VEC> gi = ldp<Real, VEC>(sm + io);
        Pack<Real, VEC> rp;
        if (prev) {
          rp = ldp<Real, VEC>(prev + io);
        } else {
#pragma unroll
          for (int kk = 0; kk < VEC; ++kk) rp.v[kk] = Real(0);
        }
        Real vi[VEC], acc[VEC];
#pragma unroll
        for (int kk = 0; kk < VEC; ++kk) {
          vi[kk] = iP ? Rn<Real>::mul(s_cur, rc.v[kk]) : Real(0);
          acc[kk] = Real(0);
        }
        const int t1 = sptr[i + 1];
        for (int t = sptr[i]; t < t1; ++t) {
          const int jl = sj[t];
          const Pack<Real, VEC> w = ldp<Real, VEC>(wsm + (size_t)t * SL + o);
          Pack<Real, VEC> rj;
          if (jl >= 0) {
            rj = ldp<Real, VEC>(cur + (size_t)jl * SL + o);
          } else {
#pragma unroll
            for (int kk = 0; kk < VEC; ++kk) rj.v[kk] = Real(0);
          }
#pragma unroll
          for (int kk = 0; kk < VEC; ++kk) acc[kk] = couple(acc[kk], w.v[kk], s_cur, rj.v[kk], vi[kk]);
        }
        const Real mi = sminv[i];
        Pack<Real, VEC> rn;
#pragma unroll
        for (int kk = 0; kk < VEC; ++kk)
          rn.v[kk] = inner_next(one_plus_beta, Rn<Real>::mul(s_cur, rc.v[kk]), beta, Rn<Real>::mul(s_prev, rp.v[kk]),
                                cm, gi.v[kk], mi, acc[kk]);
        if (last) {
          const size_t is = (size_t)i * S + s0;
          const Pack<Real, VEC> ui = ldp<Real, VEC>(u + is);
          Pack<Real, VEC> dn = ldp<Real, VEC>(d + is), un;
#pragma unroll
          for (int kk = 0; kk < VEC; ++kk) {
            dn.v[kk] = Rn<Real>::fma(kappa, rn.v[kk], dn.v[kk]);
            un.v[kk] = Rn<Real>::add(ui.v[kk], dn.v[kk]);
          }
          if constexpr (RAG) {
            stp_lim<Real, VEC>(d + is, dn, nvalid);
            stp_lim<Real, VEC>(u_next + is, un, nvalid);
          } else {
            stp<Real, VEC>(d + is, dn);
            stp<Real, VEC>(u_next + is, un);
          }
        } else {
          stp<Real, VEC>(r_next + io, rn);
        }
      }
    }
    __syncthreads();
    prev = cur;
    s_prev = s_cur;
    cur = r_next;
    s_cur = Real(1);
    nxt = nxt % 3 + 1;
  }
}

// ---------------------------------------------------------------------------
// Initial state: u = u0 (both buffers), d = dt v0; xi padded to KP in Real.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void k_init_state(int64_t n_nodes, int S, const Real* __restrict__ u0,
                             const Real* __restrict__ v0, Real dt, Real* __restrict__ ua,
                             Real* __restrict__ ub, Real* __restrict__ d, const double* __restrict__ dts = nullptr) {
  const int64_t total = n_nodes * (int64_t)S;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / S;
    const Real v = u0[i];
    ua[k] = v;
    ub[k] = v;
    d[k] = v0 ? (dts ? (Real)dts[k % S] : dt) * v0[i] : Real(0);  // d_0 = dt v0 (dt of the draw)
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
                              double* __restrict__ ps, double* __restrict__ pc, int s_lo, int s_hi) {
  const int s = s_lo + blockIdx.y * blockDim.x + threadIdx.x;  // draws [s_lo, s_hi)
  if (s >= s_hi) return;
  const int c = blockIdx.x;
  const int k0 = c * chunk, k1 = min(nnz, k0 + chunk);
  Neumaier acc;
  // the product is rounded on its own (no fused multiply-add), so that every
  // reduction of the same values gives the same Q bit for bit
  for (int k = k0; k < k1; ++k) acc.add(__dmul_rn(gw[k], (double)u[(size_t)idx[k] * S + s]));
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
                               const Real* __restrict__ u, double* __restrict__ out, int s_lo, int s_hi) {
  const int64_t w = s_hi - s_lo;  // draws [s_lo, s_hi)
  const int64_t total = n_nodes * w;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / w, s = s_lo + k % w;
    out[(int64_t)new2old[i] * S + s] = (double)u[(size_t)i * S + s];
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
