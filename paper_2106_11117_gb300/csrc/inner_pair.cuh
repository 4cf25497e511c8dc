// Two inner substeps of Alg. 2 in one launch (m + 1 and m + 2), with the
// intermediate r_{m+1} exchanged in shared memory.
//
// R is cut into blocks: square cells of R's bounding box (the core), each
// with a halo, the P nodes outside the core that neighbour a core node.  One
// CTA takes a (block, slab of draws) pair.  It first stages the index data of
// its rows (node id, the four table neighbours and edges, the adjacency
// range, 1/m and, for core rows, the block row of each P neighbour) in
// shared memory, so that every later load of a row depends on shared memory
// only.  Phase A computes r_{m+1} on the core and the halo exactly as
// k_inner does (from r_m, r_{m-1}, g and the coupling weights in global
// memory), keeps it in shared memory and writes the core's part to global
// memory (the next pair's r_{m-1}); phase B computes r_{m+2} on the core
// from the shared r_{m+1} of its P neighbours (or, in the pair that ends the
// step, folds r_p into d and u).  Neighbouring blocks compute a halo node
// again (about 4 / sqrt(core) extra work).  Per two substeps the DRAM
// traffic is r_m, r_{m-1}, g and the coupling weights read once (the second
// reads of phase B hit L2) and r_{m+1}, r_{m+2} written once, instead of all
// of that twice and r_{m+1} read back.  The arithmetic per node is
// k_inner's (kernels.cuh), term by term, so the values are the same bit for
// bit.
#pragma once
#include "kernels.cuh"

namespace lflts {

// Device view of a pair plan (host: build_pair_plan in mesh_prep.h).
struct PairDev {
  int n_blocks;
  int rows_max;        // largest core + halo
  int core_max;        // largest core
  const int* rptr;     // [n_blocks + 1] offsets into row
  const int* ncore;    // [n_blocks] core size
  const int* row;      // rows of every block: core nodes, then halo nodes
  const short* lidx;   // [adjacency entry of an R node]: block row of the neighbour, -1 off P
};

// Shared-memory layout of a CTA (host and device): r_{m+1} rows of the
// slab, then the staged index data.  Every section starts on 16 bytes.
struct PairSmem {
  size_t r1, ell, nid, adj, minv, lid, total;
};
__host__ __device__ inline PairSmem pair_smem_layout(int rows_max, int core_max, int SL, int real_bytes) {
  PairSmem L;
  size_t o = 0;
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  L.r1 = o;
  o = al(o + size_t(rows_max) * SL * real_bytes);
  L.ell = o;
  o = al(o + size_t(rows_max) * 32);
  L.nid = o;
  o = al(o + size_t(rows_max) * 4);
  L.adj = o;
  o = al(o + size_t(rows_max) * 8);
  L.minv = o;
  o = al(o + size_t(rows_max) * real_bytes);
  L.lid = o;
  o = al(o + size_t(core_max) * 8);
  L.total = o;
  return L;
}

// r_{m+1} at node i for the draws [s0, s0 + VEC): k_inner's arithmetic, with
// the node's index data given.
template <typename Real, int VEC>
__device__ __forceinline__ Pack<Real, VEC> inner_one(const MeshDev<Real>& m, int S, int s0, int i, const Nb4& nb,
                                                     int t0, int t1, Real mi, const Real* __restrict__ W,
                                                     const Real* __restrict__ cur, Real s_cur,
                                                     const Real* __restrict__ prev, Real s_prev,
                                                     const Real* __restrict__ g, Real opb, Real beta, Real cm) {
  const int nP = m.n_P;
  const size_t is = (size_t)i * S + s0;
  const bool iP = i < nP;
  const Pack<Real, VEC> rc = ldp<Real, VEC>(cur + is);
  const Pack<Real, VEC> gi = ldp<Real, VEC>(g + is);
  Pack<Real, VEC> rj[4], w[4], rp;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = nb.j[q];
    const bool jP = j >= 0 && j < nP;
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
  Real vi[VEC], acc[VEC];
#pragma unroll
  for (int k = 0; k < VEC; ++k) {
    vi[k] = iP ? Rn<Real>::mul(s_cur, rc.v[k]) : Real(0);
    acc[k] = Real(0);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < VEC; ++k) acc[k] = couple(acc[k], w[q].v[k], s_cur, rj[q].v[k], vi[k]);
  for (int t = t0; t < t1; ++t) {  // neighbours beyond the fourth
    const int2 o = m.adj[t];
    const bool jP = o.x < nP;
    if (!jP && !iP) break;
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
    rn.v[k] = inner_next(opb, Rn<Real>::mul(s_cur, rc.v[k]), beta, Rn<Real>::mul(s_prev, rp.v[k]), cm, gi.v[k], mi,
                         acc[k]);
  return rn;
}

__device__ __forceinline__ Nb4 nb4_of(const int4 a, const int4 b) {
  Nb4 r;
  r.j[0] = a.x; r.e[0] = a.y; r.j[1] = a.z; r.e[1] = a.w;
  r.j[2] = b.x; r.e[2] = b.y; r.j[3] = b.z; r.e[3] = b.w;
  return r;
}

// LAST: the second substep is the step's last one (d, u updated).  Block:
// 256 threads, SB lanes of VEC draws per row (SB * VEC = 32 draws a slab).
// Registers capped for five CTAs per SM (48; the kernel is latency-bound,
// and five CTAs ran the pairs 7 % faster than four, six 60 % slower with
// the spills a 40-register cap takes).
template <typename Real, int VEC, bool LAST>
__global__ void __launch_bounds__(256, 5)
k_inner_pair(MeshDev<Real> m, PairDev pd, int S, int SB, const Real* __restrict__ W,
             const Real* __restrict__ cur, Real s_cur, const Real* __restrict__ prev, Real s_prev,
             const Real* __restrict__ g, Real* __restrict__ out1, Real* __restrict__ out2,
             const Real* __restrict__ u, Real* __restrict__ u_next, Real* __restrict__ d,
             Real opb1, Real beta1, Real cm1, Real opb2, Real beta2, Real cm2, Real kappa) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int SL = SB * VEC;
  const PairSmem L = pair_smem_layout(pd.rows_max, pd.core_max, SL, sizeof(Real));
  Real* const r1 = reinterpret_cast<Real*>(smem_raw + L.r1);     // [rows][SL] r_{m+1}
  int4* const s_ell = reinterpret_cast<int4*>(smem_raw + L.ell);  // [rows][2]
  int* const s_nid = reinterpret_cast<int*>(smem_raw + L.nid);
  int2* const s_adj = reinterpret_cast<int2*>(smem_raw + L.adj);  // adjacency range
  Real* const s_minv = reinterpret_cast<Real*>(smem_raw + L.minv);
  short4* const s_lid = reinterpret_cast<short4*>(smem_raw + L.lid);  // core rows: rows of the 4 table slots

  const int b = blockIdx.x;
  const int r0 = pd.rptr[b], nr = pd.rptr[b + 1] - r0, nc = pd.ncore[b];

  // ---- stage the rows' index data ---------------------------------------
  for (int t = threadIdx.x; t < nr; t += blockDim.x) {
    const int i = pd.row[r0 + t];
    const int a0 = m.adj_ptr[i], a1 = m.adj_ptr[i + 1];
    s_ell[2 * t] = m.ell[2 * i];
    s_ell[2 * t + 1] = m.ell[2 * i + 1];
    s_nid[t] = i;
    s_adj[t] = make_int2(a0, a1);
    s_minv[t] = m.minv[i];
    if (t < nc) {
      const int n = a1 - a0;  // slots past the node's list are never read
      s_lid[t] = make_short4(n > 0 ? pd.lidx[a0] : short(-1), n > 1 ? pd.lidx[a0 + 1] : short(-1),
                             n > 2 ? pd.lidx[a0 + 2] : short(-1), n > 3 ? pd.lidx[a0 + 3] : short(-1));
    }
  }
  __syncthreads();

  const int lane = threadIdx.x % SB, rgrp = threadIdx.x / SB, NB = blockDim.x / SB;
  const int s0 = blockIdx.y * SL + lane * VEC;
  const bool active = s0 < S;  // S is a multiple of VEC
  const int o = lane * VEC;

  // ---- phase A: r_{m+1} on the core and the halo ---------------------------
  if (active) {
    for (int t = rgrp; t < nr; t += NB) {
      const int i = s_nid[t];
      const Nb4 nb = nb4_of(s_ell[2 * t], s_ell[2 * t + 1]);
      const int2 ar = s_adj[t];
      const Pack<Real, VEC> rn = inner_one<Real, VEC>(m, S, s0, i, nb, ar.x + 4, ar.y, s_minv[t], W, cur, s_cur,
                                                       prev, s_prev, g, opb1, beta1, cm1);
      stp<Real, VEC>(r1 + (size_t)t * SL + o, rn);
      if (t < nc && out1) stp<Real, VEC>(out1 + (size_t)i * S + s0, rn);  // not needed after the last pair
    }
  }
  __syncthreads();
  if (!active) return;

  // ---- phase B: r_{m+2} (or d, u) on the core -------------------------------
  const int nP = m.n_P;
  for (int t = rgrp; t < nc; t += NB) {
    const int i = s_nid[t];
    const size_t is = (size_t)i * S + s0;
    const bool iP = i < nP;
    const Nb4 nbq = nb4_of(s_ell[2 * t], s_ell[2 * t + 1]);
    const int2 ar = s_adj[t];
    const short4 l4 = s_lid[t];
    const short lq[4] = {l4.x, l4.y, l4.z, l4.w};
    const Pack<Real, VEC> rc = ldp<Real, VEC>(r1 + (size_t)t * SL + o);  // r_{m+1}, scale 1
    const Pack<Real, VEC> gi = ldp<Real, VEC>(g + is);
    const Pack<Real, VEC> rpv = ldp<Real, VEC>(cur + is);                 // r_m = s_cur cur
    Pack<Real, VEC> rj[4], w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = nbq.j[q];
      const bool jP = j >= 0 && j < nP;
      if (jP || (iP && j >= 0)) {
        w[q] = ldp<Real, VEC>(W + (size_t)nbq.e[q] * S + s0);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) w[q].v[k] = Real(0);
      }
      if (jP) {
        rj[q] = ldp<Real, VEC>(r1 + (size_t)lq[q] * SL + o);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) rj[q].v[k] = Real(0);
      }
    }
    const Real mi = s_minv[t];
    Real vi[VEC], acc[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      vi[k] = iP ? Rn<Real>::mul(Real(1), rc.v[k]) : Real(0);
      acc[k] = Real(0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < VEC; ++k) acc[k] = couple(acc[k], w[q].v[k], Real(1), rj[q].v[k], vi[k]);
    for (int tt = ar.x + 4; tt < ar.y; ++tt) {
      const int2 oo = m.adj[tt];
      const bool jP = oo.x < nP;
      if (!jP && !iP) break;
      const Pack<Real, VEC> wo = ldp<Real, VEC>(W + (size_t)oo.y * S + s0);
      if (jP) {
        const Pack<Real, VEC> ro = ldp<Real, VEC>(r1 + (size_t)pd.lidx[tt] * SL + o);
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc[k] = couple(acc[k], wo.v[k], Real(1), ro.v[k], vi[k]);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc[k] = couple(acc[k], wo.v[k], Real(1), Real(0), vi[k]);
      }
    }
    Pack<Real, VEC> rn;
#pragma unroll
    for (int k = 0; k < VEC; ++k)
      rn.v[k] = inner_next(opb2, Rn<Real>::mul(Real(1), rc.v[k]), beta2, Rn<Real>::mul(s_cur, rpv.v[k]), cm2,
                           gi.v[k], mi, acc[k]);
    if (LAST) {
      const Pack<Real, VEC> ui = ldp<Real, VEC>(u + is);
      Pack<Real, VEC> dn = ldp<Real, VEC>(d + is), un;
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        dn.v[k] = Rn<Real>::fma(kappa, rn.v[k], dn.v[k]);
        un.v[k] = Rn<Real>::add(ui.v[k], dn.v[k]);
      }
      stp<Real, VEC>(d + is, dn);
      stp<Real, VEC>(u_next + is, un);
    } else {
      stp<Real, VEC>(out2 + is, rn);
    }
  }
}

}  // namespace lflts
