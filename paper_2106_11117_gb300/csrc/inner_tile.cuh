// All p-1 inner substeps of one outer step (Alg. 2, the loop over m) for a
// large refined region, tile by tile, with the recursion on chip.
//
// The substeps touch only R and couple nodes only through P: r_{m+1} at a
// node needs r_m at its P neighbours.  A tile is a compact core of R nodes
// (a square cell of R's bounding box) plus p-1 layers of P nodes around it
// (layer k: the P neighbours of layer k-1 not yet in the tile).  Substep m
// computes r_{m+1} on the core and layers 1..p-1-m; after the last substep
// the core's values are exact, since everything they depend on was computed
// inside the tile.  The outermost layer only supplies r_1 = -c_0 g.  Halo
// nodes are computed again by every tile that holds them.
//
// One CTA takes a work unit: a tile and a run of slabs of VEC draws.  Thread
// t owns the tile nodes t, t + NT, ..., t + (IT-1) NT (one node and VEC draws
// each) and keeps their g, r_m, r_{m-1}, coupling weights and neighbour rows
// in registers for all substeps; shared memory holds r_m of the tile for the
// neighbours' reads (two planes, one per parity of m, plus a row of zeros
// that the slots of neighbours off P and unused slots, with weight 0, point
// to: no branch per slot), the tile's node and edge ids, and a staging area
// into which the next slab's g, weights and core u, d are copied
// asynchronously (cp.async) while the current slab's substeps run, so the
// global-memory latency of a slab is hidden behind the previous one.  Per
// step and node the global traffic is g once, the coupling weights once, and
// u, d in and out on the core, instead of r_m, r_{m-1}, g, the weights and
// r_{m+1} in every substep.  The arithmetic per node is that of k_inner term
// by term (same slots in the same order, same roundings, kernels.cuh), so
// the values are the same bit for bit.  PC > 0 fixes p at compile time (the
// substep loop unrolls); PC = 0 reads p from the coefficients.
#pragma once
#include "kernels.cuh"

namespace lflts {

// Device view of a tile plan (built on the host, mesh_prep.h).
struct TileDev {
  const int* ptr;        // [n_tiles + 1] first tile node of every tile
  const int* len;        // [n_tiles][p]: core size, then core + layers 1..k for k = 1..p-1
  const int* node;       // mesh node of every tile node
  const int2* sj;        // [tile node]: local rows of the four slots as 16-bit pairs (lo, hi);
                         //   row n_all (zeros) for a neighbour off P or an unused slot
  const int4* se;        // [tile node]: edge ids of the four slots (-1: unused)
  const int* xp;         // [tile node]: bit 0 node in P; (xp >> 1) & 15 slots beyond the
                         //   fourth, from offset xp >> 5 in xs
  const int2* xs;        // those slots: (local row, edge id)
  const float* minv32;   // [tile node] 1 / m_i
  const double* minv64;
  int n_tiles;
  int n_all_max;         // largest tile (shared-memory planes hold n_all_max + 1 rows)
  int comp_max;          // most computed nodes of a tile (<= the kernel's IT * NT)
  int core_max;          // largest core
  int chunk;             // slabs per work unit
  int chunks;            // work units per tile
  const int* xptr;       // [n_tiles + 1] each tile's range of slots beyond the fourth in xs
  int xs_max;            // most such slots of a tile
};

// Shared-memory layout of k_inner_tile (bytes), the same on host and device.
struct TileSmem {
  size_t plane, node, se, sg, sw, sud, sxs, sxw, total;
};
__host__ __device__ inline TileSmem tile_smem_layout(int n_all_max, int comp_max, int core_max, int xs_max, int vec,
                                                     int real_bytes) {
  TileSmem L;
  const size_t row = size_t(vec) * real_bytes;  // 16 bytes
  L.plane = 0;                                                // 2 x (n_all_max + 1) rows
  L.node = L.plane + 2 * (size_t(n_all_max) + 1) * row;       // n_all_max ints
  L.se = (L.node + size_t(n_all_max) * 4 + 15) / 16 * 16;     // comp_max int4
  L.sg = L.se + size_t(comp_max) * 16;                        // n_all_max rows of g
  L.sw = L.sg + size_t(n_all_max) * row;                      // comp_max x 4 rows of weights
  L.sud = L.sw + size_t(comp_max) * 4 * row;                  // 2 buffers x core_max x (u, d)
  L.sxs = L.sud + 2 * size_t(core_max) * 2 * row;             // xs_max int2: slots beyond the fourth
  L.sxw = (L.sxs + size_t(xs_max) * 8 + 15) / 16 * 16;        // 2 buffers x xs_max rows of their weights
  L.total = L.sxw + 2 * size_t(xs_max) * row;
  return L;
}

__device__ __forceinline__ int slot_of(const int2& v, int q) {
  const int wd = (q < 2) ? v.x : v.y;
  return (q & 1) ? int((unsigned)wd >> 16) : int(wd & 0xffff);
}
__device__ __forceinline__ float tile_minv(const TileDev& tp, int k, float) { return tp.minv32[k]; }
__device__ __forceinline__ double tile_minv(const TileDev& tp, int k, double) { return tp.minv64[k]; }

// 16-byte asynchronous copy global -> shared (completes at cp_wait).
__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename Real, int VEC, int IT, int NT, int PC>
__global__ void __launch_bounds__(NT, 1)
k_inner_tile(TileDev tp, int S, const Real* __restrict__ W, const Real* __restrict__ g,
             const Real* __restrict__ u, Real* __restrict__ u_next, Real* __restrict__ d,
             const InnerCoef<Real> k, Real kappa) {
  static_assert(VEC * sizeof(Real) == 16, "one 16-byte row per node and slab");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TileSmem L = tile_smem_layout(tp.n_all_max, tp.comp_max, tp.core_max, tp.xs_max, VEC, sizeof(Real));
  Real* const plane0 = reinterpret_cast<Real*>(smem_raw + L.plane);
  Real* const plane1 = plane0 + (size_t)(tp.n_all_max + 1) * VEC;
  int* const snode = reinterpret_cast<int*>(smem_raw + L.node);
  int4* const sse = reinterpret_cast<int4*>(smem_raw + L.se);
  Real* const sg = reinterpret_cast<Real*>(smem_raw + L.sg);
  Real* const sw = reinterpret_cast<Real*>(smem_raw + L.sw);
  Real* const sud = reinterpret_cast<Real*>(smem_raw + L.sud);
  int2* const sxs = reinterpret_cast<int2*>(smem_raw + L.sxs);
  Real* const sxw = reinterpret_cast<Real*>(smem_raw + L.sxw);
  __shared__ int slen[64];  // core + layers 1..k of the current tile
  const int p = PC > 0 ? PC : k.p;
  const int n_slabs = S / VEC;
  const int64_t n_units = (int64_t)tp.n_tiles * tp.chunks;
  for (int64_t un = blockIdx.x; un < n_units; un += gridDim.x) {
    const int t = (int)(un / tp.chunks);
    const int sl0 = (int)(un % tp.chunks) * tp.chunk;
    const int sl1 = min(n_slabs, sl0 + tp.chunk);
    if (sl0 >= sl1) continue;  // the same for every thread of the CTA
    const int base = tp.ptr[t];
    const int* len = tp.len + (size_t)t * p;
    const int n_comp = len[p - 2];  // nodes of the first substep
    const int n_all = len[p - 1];
    const int n_core = len[0];
    const int x0 = tp.xptr[t], n_x = tp.xptr[t + 1] - x0;

    // ---- per tile: ids to shared memory, slots and 1/m to registers ---------
    for (int a = threadIdx.x; a < n_all; a += NT) snode[a] = tp.node[base + a];
    for (int a = threadIdx.x; a < n_comp; a += NT) sse[a] = tp.se[base + a];
    for (int e = threadIdx.x; e < n_x; e += NT) sxs[e] = tp.xs[x0 + e];
    for (int q = threadIdx.x; q < p; q += NT) slen[q] = len[q];
    int2 sj[IT];
    Real mi[IT];
    int xp[IT];
#pragma unroll
    for (int j = 0; j < IT; ++j) {
      const int a = threadIdx.x + j * NT;
      sj[j] = make_int2(0, 0);
      xp[j] = 0;
      mi[j] = Real(0);
      if (a < n_comp) {
        sj[j] = tp.sj[base + a];
        xp[j] = tp.xp[base + a];
        mi[j] = tile_minv(tp, base + a, Real(0));
      }
    }
    __syncthreads();

    // copies of one slab: g of every tile node, the weights of the computed
    // nodes' slots, u and d of the core (into buffer b)
    auto prefetch = [&](int sl, int b) {
      const int s0 = sl * VEC;
      for (int a = threadIdx.x; a < n_all; a += NT) cp16(sg + (size_t)a * VEC, g + (size_t)snode[a] * S + s0);
      for (int a = threadIdx.x; a < n_comp; a += NT) {
        const int4 se = sse[a];
        const int e4[4] = {se.x, se.y, se.z, se.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (e4[q] >= 0) cp16(sw + ((size_t)a * 4 + q) * VEC, W + (size_t)e4[q] * S + s0);
      }
      Real* ud = sud + (size_t)b * tp.core_max * 2 * VEC;
      for (int a = threadIdx.x; a < n_core; a += NT) {
        const size_t is = (size_t)snode[a] * S + s0;
        cp16(ud + (size_t)a * 2 * VEC, u + is);
        cp16(ud + ((size_t)a * 2 + 1) * VEC, d + is);
      }
      Real* xw = sxw + (size_t)b * tp.xs_max * VEC;
      for (int e = threadIdx.x; e < n_x; e += NT) cp16(xw + (size_t)e * VEC, W + (size_t)sxs[e].y * S + s0);
      cp_commit();
    };
    prefetch(sl0, 0);

    for (int sl = sl0; sl < sl1; ++sl) {
      const int s0 = sl * VEC;
      const int b = (sl - sl0) & 1;
      cp_wait();
      __syncthreads();  // this slab's copies are visible to every thread

      // ---- staging -> registers: g, r_1 = -c_0 g, weights ------------------
      Pack<Real, VEC> rc[IT], rp[IT], gi[IT], w[IT][4];
#pragma unroll
      for (int j = 0; j < IT; ++j) {
        const int a = threadIdx.x + j * NT;
        if (a < n_comp) {
          gi[j] = ldp<Real, VEC>(sg + (size_t)a * VEC);
          const int4 se = sse[a];
          const int e4[4] = {se.x, se.y, se.z, se.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (e4[q] >= 0) {
              w[j][q] = ldp<Real, VEC>(sw + ((size_t)a * 4 + q) * VEC);
            } else {
#pragma unroll
              for (int c = 0; c < VEC; ++c) w[j][q].v[c] = Real(0);
            }
          }
#pragma unroll
          for (int c = 0; c < VEC; ++c) {
            rc[j].v[c] = Rn<Real>::mul(k.neg_c0, gi[j].v[c]);
            rp[j].v[c] = Real(0);
          }
          stp<Real, VEC>(plane0 + (size_t)a * VEC, rc[j]);
        }
      }
      for (int a = n_comp + threadIdx.x; a < n_all; a += NT) {  // outermost layer: r_1 only
        Pack<Real, VEC> r1 = ldp<Real, VEC>(sg + (size_t)a * VEC);
#pragma unroll
        for (int c = 0; c < VEC; ++c) r1.v[c] = Rn<Real>::mul(k.neg_c0, r1.v[c]);
        stp<Real, VEC>(plane0 + (size_t)a * VEC, r1);
      }
      if (threadIdx.x < VEC) {  // the zero row of both planes
        plane0[(size_t)n_all * VEC + threadIdx.x] = Real(0);
        plane1[(size_t)n_all * VEC + threadIdx.x] = Real(0);
      }
      __syncthreads();  // staging of g and the weights is free again
      if (sl + 1 < sl1) prefetch(sl + 1, b ^ 1);
      const Real* ud = sud + (size_t)b * tp.core_max * 2 * VEC;
      const Real* xw = sxw + (size_t)b * tp.xs_max * VEC;

      // ---- substeps m = 1 .. p-1 --------------------------------------------
#pragma unroll(PC > 0 ? PC - 1 : 1)
      for (int mm = 1; mm < p; ++mm) {
        const Real* cur = (mm & 1) ? plane0 : plane1;
        Real* nxt = (mm & 1) ? plane1 : plane0;
        const bool last = (mm == p - 1);
        const int lm = slen[p - 1 - mm];  // core and layers 1..p-1-m
        const Real opb = k.opb[mm], beta = k.beta[mm], cm = k.cm[mm];
#pragma unroll
        for (int j = 0; j < IT; ++j) {
          const int a = threadIdx.x + j * NT;
          if (a < lm) {
            const bool iP = xp[j] & 1;
            Real vi[VEC], acc[VEC];
#pragma unroll
            for (int c = 0; c < VEC; ++c) {
              vi[c] = iP ? rc[j].v[c] : Real(0);
              acc[c] = Real(0);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // unused slots: weight 0 and the zero row
              const Pack<Real, VEC> rj = ldp<Real, VEC>(cur + (size_t)slot_of(sj[j], q) * VEC);
#pragma unroll
              for (int c = 0; c < VEC; ++c) acc[c] = couple(acc[c], w[j][q].v[c], Real(1), rj.v[c], vi[c]);
            }
            const int nx = (xp[j] >> 1) & 15;
            for (int e = (xp[j] >> 5) - x0; nx > 0 && e < (xp[j] >> 5) - x0 + nx; ++e) {
              // slots beyond the fourth (nodes of the fans), staged like the others
              const Pack<Real, VEC> wo = ldp<Real, VEC>(xw + (size_t)e * VEC);
              const Pack<Real, VEC> rj = ldp<Real, VEC>(cur + (size_t)sxs[e].x * VEC);
#pragma unroll
              for (int c = 0; c < VEC; ++c) acc[c] = couple(acc[c], wo.v[c], Real(1), rj.v[c], vi[c]);
            }
            Pack<Real, VEC> rn;
#pragma unroll
            for (int c = 0; c < VEC; ++c)
              rn.v[c] = inner_next(opb, rc[j].v[c], beta, rp[j].v[c], cm, gi[j].v[c], mi[j], acc[c]);
            if (!last) {
              stp<Real, VEC>(nxt + (size_t)a * VEC, rn);
              rp[j] = rc[j];
              rc[j] = rn;
            } else {  // the core: d_{n+1} = d_n + kappa r_p, u_{n+1} = u_n + d_{n+1}
              const Pack<Real, VEC> ui = ldp<Real, VEC>(ud + (size_t)a * 2 * VEC);
              Pack<Real, VEC> dn = ldp<Real, VEC>(ud + ((size_t)a * 2 + 1) * VEC), unx;
#pragma unroll
              for (int c = 0; c < VEC; ++c) {
                dn.v[c] = Rn<Real>::fma(kappa, rn.v[c], dn.v[c]);
                unx.v[c] = Rn<Real>::add(ui.v[c], dn.v[c]);
              }
              const size_t is = (size_t)snode[a] * S + s0;
              stp<Real, VEC>(d + is, dn);
              stp<Real, VEC>(u_next + is, unx);
            }
          }
        }
        __syncthreads();
      }
    }
    cp_wait();  // nothing in flight when the next unit reuses the buffers
    __syncthreads();
  }
}

}  // namespace lflts
