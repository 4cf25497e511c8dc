// Host-side mesh preparation; see mesh_prep.h for the data it produces.
#include "mesh_prep.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace lflts {

int prep_mesh(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
              const uint8_t* dirichlet, const uint8_t* P, const double* psi, int K,
              HostMesh& out, std::string& err) {
  const int kErrArg = -1, kErrMesh = -6;
  if (!xy || !tri || !dirichlet || !psi || n_nodes < 3 || n_tri < 1) {
    err = "mesh_add: null array or empty mesh";
    return kErrArg;
  }
  if (K < 1 || K > 16) {
    err = "mesh_add: K must be in [1, 16]";
    return kErrArg;
  }
  if (n_nodes >= (int64_t(1) << 31) || n_tri >= (int64_t(1) << 31)) {
    err = "mesh_add: more than 2^31 nodes or triangles";
    return kErrArg;
  }
  HostMesh& m = out;
  m.n_nodes = n_nodes;
  m.n_tri = n_tri;
  m.K = K;
  m.KP = K <= 4 ? 4 : (K <= 8 ? 8 : 16);

  // ---- validation and element areas --------------------------------------
  std::vector<double> area2(n_tri);  // twice the signed area
  for (int64_t e = 0; e < n_tri; ++e) {
    const int32_t a = tri[3 * e], b = tri[3 * e + 1], c = tri[3 * e + 2];
    if (a < 0 || b < 0 || c < 0 || a >= n_nodes || b >= n_nodes || c >= n_nodes ||
        a == b || b == c || a == c) {
      err = "mesh_add: triangle " + std::to_string(e) + " has an invalid vertex index";
      return kErrMesh;
    }
    const double x0 = xy[2 * a], y0 = xy[2 * a + 1];
    const double d = (xy[2 * b] - x0) * (xy[2 * c + 1] - y0) - (xy[2 * c] - x0) * (xy[2 * b + 1] - y0);
    if (!(d > 0.0)) {
      err = "mesh_add: triangle " + std::to_string(e) + " is not counter-clockwise with positive area";
      return kErrMesh;
    }
    area2[e] = d;
  }

  // ---- masks: P (free nodes only), R = vertices of elements touching P ----
  std::vector<uint8_t> inP(n_nodes, 0), inR(n_nodes, 0);
  if (P) {
    for (int64_t i = 0; i < n_nodes; ++i) inP[i] = (P[i] != 0 && dirichlet[i] == 0) ? 1 : 0;
  }
  for (int64_t e = 0; e < n_tri; ++e) {
    const int32_t* v = tri + 3 * e;
    if (inP[v[0]] || inP[v[1]] || inP[v[2]]) {
      for (int a = 0; a < 3; ++a)
        if (dirichlet[v[a]] == 0) inR[v[a]] = 1;
    }
  }

  // ---- node order: [P | R\P | free\R | Dirichlet], stable ---------------
  m.new2old.clear();
  m.new2old.reserve(n_nodes);
  for (int grp = 0; grp < 4; ++grp) {
    for (int64_t i = 0; i < n_nodes; ++i) {
      const bool dir = dirichlet[i] != 0;
      int g;
      if (dir) g = 3;
      else if (inP[i]) g = 0;
      else if (inR[i]) g = 1;
      else g = 2;
      if (g == grp) m.new2old.push_back(static_cast<int32_t>(i));
    }
    if (grp == 0) m.n_P = static_cast<int64_t>(m.new2old.size());
    if (grp == 1) m.n_R = static_cast<int64_t>(m.new2old.size());
    if (grp == 2) m.n_free = static_cast<int64_t>(m.new2old.size());
  }
  m.old2new.assign(n_nodes, 0);
  for (int64_t k = 0; k < n_nodes; ++k) m.old2new[m.new2old[k]] = static_cast<int32_t>(k);

  // ---- element order: by smallest new vertex id (locality of psi reads) --
  std::vector<int32_t> eorder(n_tri);
  std::iota(eorder.begin(), eorder.end(), 0);
  std::vector<int32_t> ekey(n_tri);
  for (int64_t e = 0; e < n_tri; ++e) {
    const int32_t* v = tri + 3 * e;
    ekey[e] = std::min({m.old2new[v[0]], m.old2new[v[1]], m.old2new[v[2]]});
  }
  std::stable_sort(eorder.begin(), eorder.end(), [&](int32_t a, int32_t b) { return ekey[a] < ekey[b]; });
  std::vector<int32_t> enew(n_tri);
  for (int64_t k = 0; k < n_tri; ++k) enew[eorder[k]] = static_cast<int32_t>(k);

  // ---- psi scaled by log2(e), padded, in the new element order -----------
  const double log2e = 1.4426950408889634073599246810019;
  m.psi2.assign(static_cast<size_t>(n_tri) * m.KP, 0.0);
  for (int64_t e = 0; e < n_tri; ++e)
    for (int k = 0; k < K; ++k)
      m.psi2[static_cast<size_t>(enew[e]) * m.KP + k] = psi[static_cast<size_t>(e) * K + k] * log2e;

  // ---- lumped mass ---------------------------------------------------------
  std::vector<double> mass(n_nodes, 0.0);
  for (int64_t e = 0; e < n_tri; ++e)
    for (int a = 0; a < 3; ++a) mass[tri[3 * e + a]] += area2[e] / 6.0;  // |T| / 3
  m.minv.assign(m.n_free, 0.0);
  for (int64_t k = 0; k < m.n_free; ++k) m.minv[k] = 1.0 / mass[m.new2old[k]];

  // ---- incidences of free nodes -------------------------------------------
  std::vector<int32_t> count(m.n_free + 1, 0);
  for (int64_t e = 0; e < n_tri; ++e)
    for (int a = 0; a < 3; ++a) {
      const int32_t nn = m.old2new[tri[3 * e + a]];
      if (nn < m.n_free) count[nn + 1]++;
    }
  m.inc_ptr.assign(m.n_free + 1, 0);
  for (int64_t k = 0; k < m.n_free; ++k) m.inc_ptr[k + 1] = m.inc_ptr[k] + count[k + 1];
  const int64_t n_inc = m.inc_ptr[m.n_free];
  m.inc_e.assign(n_inc, 0);
  m.inc_j1.assign(n_inc, 0);
  m.inc_j2.assign(n_inc, 0);
  m.inc_w1.assign(n_inc, 0.0);
  m.inc_w2.assign(n_inc, 0.0);
  std::vector<int32_t> fill(m.inc_ptr.begin(), m.inc_ptr.end() - 1);
  // visit elements in the new element order so each node's list is sorted
  for (int64_t k = 0; k < n_tri; ++k) {
    const int64_t e = eorder[k];
    const int32_t* v = tri + 3 * e;
    double E[3][2];
    for (int a = 0; a < 3; ++a) {  // edge opposite vertex a, counter-clockwise
      const int32_t p1 = v[(a + 1) % 3], p2 = v[(a + 2) % 3];
      E[a][0] = xy[2 * p2] - xy[2 * p1];
      E[a][1] = xy[2 * p2 + 1] - xy[2 * p1 + 1];
    }
    const double inv4A = 1.0 / (2.0 * area2[e]);  // 1 / (4 |T|)
    for (int a = 0; a < 3; ++a) {
      const int32_t nn = m.old2new[v[a]];
      if (nn >= m.n_free) continue;
      const int b = (a + 1) % 3, c = (a + 2) % 3;
      const int32_t t = fill[nn]++;
      m.inc_e[t] = static_cast<int32_t>(k);
      m.inc_j1[t] = m.old2new[v[b]];
      m.inc_j2[t] = m.old2new[v[c]];
      m.inc_w1[t] = (E[a][0] * E[b][0] + E[a][1] * E[b][1]) * inv4A;
      m.inc_w2[t] = (E[a][0] * E[c][0] + E[a][1] * E[c][1]) * inv4A;
    }
  }
  return 0;
}

}  // namespace lflts
