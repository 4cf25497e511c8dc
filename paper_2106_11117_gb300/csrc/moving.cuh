// Coupling weights of a mesh whose vertices move with the draw.
//
// Sec. 4.3 solves every draw of the channel of random width on one reference
// mesh whose vertices are moved by the map of Eq. MeshTransform; the stiffness
// and the lumped mass of Eq. waveeq_transformed then belong to the moved
// mesh.  Here vertex v of draw s sits at x_v + sum_k xi_{s,k} D_k(v) (K
// displacement modes), and for every adjacency entry t of a free node i
// (neighbour j)
//   W[t][s] = K_ij(s) / m_i(s),
// the P1 stiffness entry of the moved elements that contain edge ij,
// sum_e (E_a . E_b) / (4 |T_e|) with E_a, E_b the moved edge vectors opposite
// i and j, over the lumped mass m_i(s) = sum_{e ni i} |T_e(s)| / 3.  The
// step kernels multiply by 1/m = 1 for such a mesh, so they apply
// M(s)^-1 K(s) of the draw.  Everything in FP64, rounded once to Real.
#pragma once
#include <cuda_runtime.h>

namespace lflts {

struct MovingDev {
  int n_free, n_nodes, K;
  const int* adj_ptr;   // [n_free + 1]
  const int2* adj;      // (neighbour, entry id) per adjacency entry
  const int* dedge;     // [entries] undirected edge of the entry
  const int2* ee;       // [edges] the (one or two) elements of the edge, -1 for none
  const int* tri;       // [n_tri][3] vertices (new ids), counter-clockwise
  const double* xy;     // [n_nodes][2] reference coordinates
  const double* disp;   // [K][n_nodes][2] displacement modes
  const int* nptr;      // [n_free + 1] offsets into nelem
  const int* nelem;     // elements of every free node
};

__device__ __forceinline__ double2 moved_vertex(const MovingDev& g, const double* xi, int v) {
  double x = g.xy[2 * v], y = g.xy[2 * v + 1];
  for (int k = 0; k < g.K; ++k) {
    const double* d = g.disp + (static_cast<size_t>(k) * g.n_nodes + v) * 2;
    x = fma(xi[k], d[0], x);
    y = fma(xi[k], d[1], y);
  }
  return make_double2(x, y);
}

// Twice the signed area of element e and its three moved vertices.
__device__ __forceinline__ double moved_element(const MovingDev& g, const double* xi, int e, int v[3],
                                                double2 X[3]) {
  for (int a = 0; a < 3; ++a) {
    v[a] = g.tri[3 * e + a];
    X[a] = moved_vertex(g, xi, v[a]);
  }
  return (X[1].x - X[0].x) * (X[2].y - X[0].y) - (X[2].x - X[0].x) * (X[1].y - X[0].y);
}

// Lanes of SB threads take consecutive draws of one node; sig (optional) is a
// per-draw factor of a ragged batch.  xi: [S][K] FP64 draws.
template <typename Real>
__global__ void k_moving_weights(MovingDev g, int S, int SB, const double* __restrict__ xi_all,
                                 Real* __restrict__ W, const Real* __restrict__ sig) {
  const int ls = threadIdx.x & (SB - 1);
  const int NB = blockDim.x / SB;
  const int s = blockIdx.y * SB + ls;
  if (s >= S) return;
  double xi[16];
  for (int k = 0; k < g.K; ++k) xi[k] = xi_all[static_cast<size_t>(s) * g.K + k];
  const double sg = sig ? double(sig[s]) : 1.0;
  for (int i = blockIdx.x * NB + threadIdx.x / SB; i < g.n_free; i += gridDim.x * NB) {
    int v[3];
    double2 X[3];
    double mass = 0.0;
    for (int q = g.nptr[i]; q < g.nptr[i + 1]; ++q) mass += moved_element(g, xi, g.nelem[q], v, X) / 6.0;
    const double inv_m = 1.0 / mass;
    for (int t = g.adj_ptr[i]; t < g.adj_ptr[i + 1]; ++t) {
      const int j = g.adj[t].x;
      const int2 el = g.ee[g.dedge[t]];
      double Kij = 0.0;
      for (int side = 0; side < 2; ++side) {
        const int e = side ? el.y : el.x;
        if (e < 0) continue;
        const double a2 = moved_element(g, xi, e, v, X);
        int a = 0, b = 0;
        for (int c = 0; c < 3; ++c) {
          if (v[c] == i) a = c;
          if (v[c] == j) b = c;
        }
        // edge vectors opposite a and b, counter-clockwise
        const double2 Ea = make_double2(X[(a + 2) % 3].x - X[(a + 1) % 3].x, X[(a + 2) % 3].y - X[(a + 1) % 3].y);
        const double2 Eb = make_double2(X[(b + 2) % 3].x - X[(b + 1) % 3].x, X[(b + 2) % 3].y - X[(b + 1) % 3].y);
        Kij += (Ea.x * Eb.x + Ea.y * Eb.y) / (2.0 * a2);
      }
      W[static_cast<size_t>(t) * S + s] = static_cast<Real>(Kij * inv_m * sg);
    }
  }
}

}  // namespace lflts
