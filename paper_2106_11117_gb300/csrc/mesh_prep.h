// Host-side preparation of a P1 mesh for the LF-LTS kernels.
//
// Sec. 3.1 (P1 elements, lumped mass) and Sec. 3.3 (mask P; the products
// A P q "only involve those unknowns inside, or immediately next to, the
// refined region").  The kernels work on a node order grouped as
//   [ P nodes | R \ P nodes | free nodes outside R | Dirichlet nodes ]
// where R = vertices of every element that has a vertex in P: the inner
// substeps of Alg. 2 change exactly the nodes of R, all other free nodes
// follow the closed-form leapfrog update.
//
// The stiffness is applied in edge form.  Rows of a P1 element matrix sum to
// zero, so
//   (K u)_i = sum_{j ~ i} K_ij (u_j - u_i),
//   K_ij(w) = sum over the (one or two) elements e containing edge ij of
//             c_e^2(w) G_e[i][j],
//   G_e[a][b] = |T_e| grad(phi_a) . grad(phi_b) = (E_a . E_b) / (4 |T_e|),
// with E_a the edge vector opposite vertex a in counter-clockwise order.
// Edges whose element entries are all exactly zero (the hypotenuses of the
// right triangles of a uniform grid) are dropped.  Each free node lists its
// edges sorted by neighbour index, so the P neighbours come first.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace lflts {

struct HostMesh {
  int64_t n_nodes = 0, n_free = 0, n_R = 0, n_P = 0, n_tri = 0;
  int K = 0;   // field terms
  int KP = 0;  // K padded to 4, 8 or 16
  std::vector<int32_t> new2old, old2new;   // node permutation
  int64_t n_edges = 0;    // coupling edges kept (at least one free endpoint)
  int64_t n_edges_P = 0;  // edges with a P endpoint (the inner substeps read these)
  std::vector<int32_t> adj_ptr;            // [n_free + 1]
  std::vector<int32_t> adj_j, adj_e;       // neighbour (new id) and edge id
  // The first four entries of every adjacency list again in a fixed-width
  // table [n_free][4] (neighbour, edge), padded with neighbour -1; entries
  // beyond the fourth stay in adj_j/adj_e from adj_ptr[i] + 4 on.
  std::vector<int32_t> ell_j, ell_e;
  std::vector<int32_t> edge_i, edge_j;     // endpoints (new ids), edge_i < edge_j
  std::vector<int32_t> edge_e0, edge_e1;   // element ids (new order), e1 = -1 on the boundary
  std::vector<double> edge_G0, edge_G1;    // G_e0[i][j], G_e1[i][j] (0 when e1 = -1)
  std::vector<double> minv;                // [n_free] 1 / m_i (lumped mass)
  std::vector<double> psi2;                // [n_tri][KP] psi * log2(e), zero padded
};

// Returns 0 on success; on failure fills err and returns a negative status.
int prep_mesh(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
              const uint8_t* dirichlet, const uint8_t* P, const double* psi, int K,
              HostMesh& out, std::string& err);

}  // namespace lflts
