// Host-side preparation of a P1 mesh for the LF-LTS kernels.
//
// Sec. 3.1 (P1 elements, lumped mass) and Sec. 3.3 (mask P; the products
// A P q "only involve those unknowns inside, or immediately next to, the
// refined region").  The kernels work on a node order grouped as
//   [ P nodes | R \ P nodes | free nodes outside R | Dirichlet nodes ]
// where R = vertices of every element that has a vertex in P: the inner
// substeps of Alg. 2 change exactly the nodes of R, all other free nodes
// follow the closed-form leapfrog update.  Each free node lists its
// incident elements with the two element-matrix entries that couple it to
// the element's other vertices:
//   (K u)_i = sum_{e ni i} c_e^2 ( G_e[i][j1] (u_j1 - u_i) + G_e[i][j2] (u_j2 - u_i) )
// which uses that the rows of a P1 element matrix sum to zero.
// G_e[a][b] = |T_e| grad(phi_a) . grad(phi_b) = (E_a . E_b) / (4 |T_e|), with
// E_a the edge vector opposite vertex a taken in counter-clockwise order.
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
  std::vector<int32_t> inc_ptr;            // [n_free + 1]
  std::vector<int32_t> inc_e, inc_j1, inc_j2;  // per incidence (new ids; element = new element id)
  std::vector<double> inc_w1, inc_w2;      // G_e[i][j1], G_e[i][j2]
  std::vector<double> minv;                // [n_free] 1 / m_i (lumped mass)
  std::vector<double> psi2;                // [n_tri][KP] psi * log2(e), zero padded
};

// Returns 0 on success; on failure fills err and returns a negative status.
int prep_mesh(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
              const uint8_t* dirichlet, const uint8_t* P, const double* psi, int K,
              HostMesh& out, std::string& err);

}  // namespace lflts
