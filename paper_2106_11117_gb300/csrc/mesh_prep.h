// Host-side preparation of a P1 mesh for the LF-LTS kernels.
//
// Sec. 3.1 (P1 elements, lumped mass) and Sec. 3.3 (mask P; the products
// A P q "only involve those unknowns inside, or immediately next to, the
// refined region").  The kernels work on a node order grouped as
//   [ P nodes | R \ P nodes | free nodes outside R | Dirichlet nodes ]
// each group in Morton (Z-curve) order of the node coordinates, where
// R = vertices of every element that has a vertex in P: the inner
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
  // Entries 5..8 in a second table of the same shape, built only when at
  // least a quarter of the free nodes have more than four neighbours (empty
  // otherwise); entries beyond the eighth then start at adj_ptr[i] + 8.
  std::vector<int32_t> ell_hi_j, ell_hi_e;
  std::vector<int32_t> edge_i, edge_j;     // endpoints (new ids), edge_i < edge_j
  std::vector<int32_t> edge_e0, edge_e1;   // element ids (new order), e1 = -1 on the boundary
  std::vector<double> edge_G0, edge_G1;    // G_e0[i][j], G_e1[i][j] (0 when e1 = -1)
  std::vector<double> minv;                // [n_free] 1 / m_i (lumped mass)
  std::vector<double> psi;                 // [n_tri][KP] psi, zero padded (new element order)
  std::vector<double> xy;                  // [n_nodes][2] coordinates, internal order
  std::vector<int32_t> tri;                // [n_tri][3] vertices in the caller's numbering and order
  std::vector<double> area;                // [n_tri] |T| in the caller's element order
  // rows of the per-draw coupling weights W: n_edges, or for a moving mesh
  // one row per adjacency entry (directed: W[t] = K_ij / m_i of entry t)
  int64_t n_w = 0;
  // A mesh whose vertices move with the draw (make_moving): adj_e, ell_e and
  // ell_hi_e hold adjacency entry ids, dedge[t] the undirected edge of entry
  // t, tri_new the vertices (new ids) of every element in the new element
  // order, nptr/nelem the elements of every free node, disp the K
  // displacement modes [K][n_nodes][2] in the new node order; minv is 1.
  bool moving = false;
  int K_modes = 0;
  std::vector<int32_t> dedge, tri_new, nptr, nelem;
  std::vector<double> disp;
};

// Coupling slots of the inner substeps on R, in the order the per-substep
// kernel visits them (the four table entries, then the rest of the
// adjacency list), without the slots that add nothing: node i < n_R keeps
// neighbour j when j is in P (r_j enters a(P r)_i) or i is in P (w_ij r_i
// enters).  slot_j = j for j in P, else -1; slot_e = edge id.  ptr has
// n_R + 1 offsets.
void build_r_slots(const HostMesh& m, std::vector<int32_t>& ptr, std::vector<int32_t>& slot_j,
                   std::vector<int32_t>& slot_e);

// Tiles of the on-chip inner substeps (k_inner_tile).  The cores are the
// nodes of R binned into square cells of R's bounding box (each cell's nodes
// in Morton order); tile t holds node[ptr[t] .. ptr[t+1]): its core, then
// p-1 layers of P nodes, layer k being the P neighbours of layer k-1 that are
// not in the tile yet.  len[t*p + k] = core + layers 1..k (k = 0..p-1).
// Substep m computes the prefix len[p-1-m]; the first len[p-2] nodes (at
// most `cap`) are the computed ones.  The cell side is the largest (in steps
// of 5 %) for which every tile fits `cap`.  For every tile node a: the first
// four coupling slots of the per-substep kernel's visiting order
// (build_r_slots) as local rows in 16-bit halves of sj[2 a], sj[2 a + 1]
// (the row n_all of the tile, one past its last node, stands for a neighbour
// off P and for an unused slot: the kernel keeps zeros there), their edge
// ids in se[4 a + q] (-1: unused slot), the slots beyond the fourth in xs as
// (local row, edge) pairs from offset xp[a] >> 5, count (xp[a] >> 1) & 15,
// bit 0 of xp[a] set for a node in P, and minv[a] = 1 / m_i.
struct TilePlan {
  int p = 0, cap = 0;
  int64_t n_all_max = 0;               // largest tile
  std::vector<int32_t> ptr, len, node;
  std::vector<int32_t> sj, se, xp, xs;
  std::vector<double> minv;
};

// Blocks of two fused inner substeps (k_inner_pair).  The cores are the
// nodes of R binned into square cells of R's bounding box of side sqrt(bn)
// times the median over R of each node's shortest edge, so that a cell of a
// uniform part of R holds about bn nodes (cells in row order, each core in
// Morton order); a
// block's rows, row[rptr[b] .. rptr[b+1]), are its core (the first ncore[b])
// and then its halo: the P nodes outside the core that neighbour a core node.
// For every adjacency entry t of an R node i (adj_ptr[i] <= t < adj_ptr[i+1])
// lidx[t] is the row of the neighbour among the rows of i's block, or -1 for
// a neighbour off P.
struct PairPlan {
  int64_t n_blocks = 0, rows_max = 0, core_max = 0;
  std::vector<int32_t> rptr, ncore, row;
  std::vector<int16_t> lidx;
};

// false when R is empty, bn < 1 or a block's rows exceed 32767.
bool build_pair_plan(const HostMesh& m, int bn, PairPlan& out);

// Build the plan for tiles of at most `cap` computed nodes; false (and an
// empty plan) when R is empty, p < 2, a tile would exceed 32000 nodes, no
// cell size fits or a node has more than 15 slots beyond the fourth.
bool build_tile_plan(const HostMesh& m, int p, int64_t cap, TilePlan& out);

// Nodal interpolation between two triangulations of one domain: for every
// point xy_f[k] the vertices vert[3k..3k+2] of a triangle of (xy_c, tri_c)
// that contains it and the barycentric coordinates w[3k..3k+2].  Point
// location through a uniform bucket grid over the triangles' bounding
// boxes; among the candidates the triangle whose smallest coordinate is
// largest is taken.  Returns the number of points outside every triangle
// (smallest coordinate below -tol); their best candidate is still written.
int64_t interp_weights(const double* xy_c, const int32_t* tri_c, int64_t n_tri_c, const double* xy_f,
                       int64_t n_f, int32_t* vert, double* w, double tol);

// Returns 0 on success; on failure fills err and returns a negative status.
// keep_all_edges keeps the edges whose stiffness entries are all zero on the
// given coordinates (needed when the coordinates change with the draw).
int prep_mesh(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
              const uint8_t* dirichlet, const uint8_t* P, const double* psi, int K,
              HostMesh& out, std::string& err, bool keep_all_edges = false);

// Turn a mesh prepared with keep_all_edges into one whose vertices move with
// the draw by sum_k xi_k D_k (disp: [K][n_nodes][2] in the caller's node
// order): directed weight rows, element and node-element tables, 1/m = 1.
int make_moving(HostMesh& m, const double* disp, int K, std::string& err);

}  // namespace lflts
