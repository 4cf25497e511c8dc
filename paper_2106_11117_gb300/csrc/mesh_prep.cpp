// Host-side mesh preparation; see mesh_prep.h for the data it produces.
#include "mesh_prep.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace lflts {

namespace {
uint64_t morton_spread16(uint64_t x) {  // interleave the low 16 bits with zeros
  x &= 0xFFFF;
  x = (x | (x << 8)) & 0x00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0Full;
  x = (x | (x << 2)) & 0x33333333ull;
  x = (x | (x << 1)) & 0x55555555ull;
  return x;
}
}  // namespace

int prep_mesh(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
              const uint8_t* dirichlet, const uint8_t* P, const double* psi, int K,
              HostMesh& out, std::string& err, bool keep_all_edges) {
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

  m.tri.assign(tri, tri + 3 * n_tri);
  m.area.resize(n_tri);
  for (int64_t e = 0; e < n_tri; ++e) m.area[e] = 0.5 * area2[e];

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

  // ---- node order: [P | R\P | free\R | Dirichlet], each group in Morton ----
  // (Z-curve) order of the coordinates, so that index ranges are compact in
  // space and neighbours are close in memory
  double bx0 = 1e300, bx1 = -1e300, by0 = 1e300, by1 = -1e300;
  for (int64_t i = 0; i < n_nodes; ++i) {
    bx0 = std::min(bx0, xy[2 * i]);
    bx1 = std::max(bx1, xy[2 * i]);
    by0 = std::min(by0, xy[2 * i + 1]);
    by1 = std::max(by1, xy[2 * i + 1]);
  }
  const double qx = 65535.0 / std::max(bx1 - bx0, 1e-300), qy = 65535.0 / std::max(by1 - by0, 1e-300);
  std::vector<std::pair<uint64_t, int32_t>> key(n_nodes);
  for (int64_t i = 0; i < n_nodes; ++i) {
    const bool dir = dirichlet[i] != 0;
    const uint64_t grp = dir ? 3 : (inP[i] ? 0 : (inR[i] ? 1 : 2));
    const uint64_t zx = morton_spread16(static_cast<uint64_t>((xy[2 * i] - bx0) * qx));
    const uint64_t zy = morton_spread16(static_cast<uint64_t>((xy[2 * i + 1] - by0) * qy));
    key[i] = {(grp << 40) | zx | (zy << 1), static_cast<int32_t>(i)};
  }
  std::stable_sort(key.begin(), key.end(),
                   [](const std::pair<uint64_t, int32_t>& a, const std::pair<uint64_t, int32_t>& b) {
                     return a.first < b.first;
                   });
  m.new2old.resize(n_nodes);
  m.n_P = m.n_R = m.n_free = 0;
  for (int64_t k = 0; k < n_nodes; ++k) {
    m.new2old[k] = key[k].second;
    const uint64_t grp = key[k].first >> 40;
    if (grp < 1) m.n_P = k + 1;
    if (grp < 2) m.n_R = k + 1;
    if (grp < 3) m.n_free = k + 1;
  }
  m.old2new.assign(n_nodes, 0);
  for (int64_t k = 0; k < n_nodes; ++k) m.old2new[m.new2old[k]] = static_cast<int32_t>(k);
  m.xy.assign(2 * static_cast<size_t>(n_nodes), 0.0);
  for (int64_t k = 0; k < n_nodes; ++k) {
    m.xy[2 * k] = xy[2 * m.new2old[k]];
    m.xy[2 * k + 1] = xy[2 * m.new2old[k] + 1];
  }

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
  if (keep_all_edges) {  // element vertices in the new orders (a moving mesh needs them)
    m.tri_new.resize(static_cast<size_t>(n_tri) * 3);
    for (int64_t k = 0; k < n_tri; ++k)
      for (int a = 0; a < 3; ++a) m.tri_new[3 * k + a] = m.old2new[tri[3 * eorder[k] + a]];
  }

  // ---- psi, padded, in the new element order -------------------------------
  m.psi.assign(static_cast<size_t>(n_tri) * m.KP, 0.0);
  for (int64_t e = 0; e < n_tri; ++e)
    for (int k = 0; k < K; ++k)
      m.psi[static_cast<size_t>(enew[e]) * m.KP + k] = psi[static_cast<size_t>(e) * K + k];

  // ---- lumped mass ---------------------------------------------------------
  std::vector<double> mass(n_nodes, 0.0);
  for (int64_t e = 0; e < n_tri; ++e)
    for (int a = 0; a < 3; ++a) mass[tri[3 * e + a]] += area2[e] / 6.0;  // |T| / 3
  m.minv.assign(m.n_free, 0.0);
  for (int64_t k = 0; k < m.n_free; ++k) m.minv[k] = 1.0 / mass[m.new2old[k]];

  // ---- edges: (lo, hi, element, G) records grouped by edge ---------------
  struct Rec {
    int32_t lo, hi, e;
    double G;
  };
  std::vector<Rec> rec;
  rec.reserve(static_cast<size_t>(n_tri) * 3);
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
      const int b = (a + 1) % 3;
      const int32_t i = m.old2new[v[a]], j = m.old2new[v[b]];
      const double G = (E[a][0] * E[b][0] + E[a][1] * E[b][1]) * inv4A;
      rec.push_back({std::min(i, j), std::max(i, j), static_cast<int32_t>(k), G});
    }
  }
  std::sort(rec.begin(), rec.end(), [](const Rec& x, const Rec& y) {
    return x.lo != y.lo ? x.lo < y.lo : (x.hi != y.hi ? x.hi < y.hi : x.e < y.e);
  });
  m.edge_e0.clear();
  m.edge_e1.clear();
  m.edge_G0.clear();
  m.edge_G1.clear();
  std::vector<int32_t> elo, ehi;
  for (size_t a = 0; a < rec.size();) {
    size_t b = a + 1;
    while (b < rec.size() && rec[b].lo == rec[a].lo && rec[b].hi == rec[a].hi) ++b;
    if (b - a > 2) {
      err = "mesh_add: an edge is shared by more than two triangles";
      return kErrMesh;
    }
    const bool any_free = rec[a].lo < m.n_free || rec[a].hi < m.n_free;
    const bool nonzero = rec[a].G != 0.0 || (b - a == 2 && rec[a + 1].G != 0.0);
    if (any_free && (nonzero || keep_all_edges)) {
      elo.push_back(rec[a].lo);
      ehi.push_back(rec[a].hi);
      m.edge_e0.push_back(rec[a].e);
      m.edge_G0.push_back(rec[a].G);
      m.edge_e1.push_back(b - a == 2 ? rec[a + 1].e : -1);
      m.edge_G1.push_back(b - a == 2 ? rec[a + 1].G : 0.0);
    }
    a = b;
  }
  m.n_edges = static_cast<int64_t>(elo.size());
  m.n_w = m.n_edges;
  m.edge_i = elo;
  m.edge_j = ehi;
  m.n_edges_P = 0;
  for (int64_t k = 0; k < m.n_edges; ++k)
    if (elo[k] < m.n_P) m.n_edges_P++;  // lo < hi, so a P endpoint means lo in P

  // ---- adjacency of free nodes, sorted by neighbour -------------------------
  std::vector<int32_t> count(m.n_free + 1, 0);
  for (int64_t k = 0; k < m.n_edges; ++k) {
    if (elo[k] < m.n_free) count[elo[k] + 1]++;
    if (ehi[k] < m.n_free) count[ehi[k] + 1]++;
  }
  m.adj_ptr.assign(m.n_free + 1, 0);
  for (int64_t k = 0; k < m.n_free; ++k) m.adj_ptr[k + 1] = m.adj_ptr[k] + count[k + 1];
  m.adj_j.assign(m.adj_ptr[m.n_free], 0);
  m.adj_e.assign(m.adj_ptr[m.n_free], 0);
  std::vector<int32_t> fill(m.adj_ptr.begin(), m.adj_ptr.end() - 1);
  for (int64_t k = 0; k < m.n_edges; ++k) {
    if (elo[k] < m.n_free) {
      m.adj_j[fill[elo[k]]] = ehi[k];
      m.adj_e[fill[elo[k]]++] = static_cast<int32_t>(k);
    }
    if (ehi[k] < m.n_free) {
      m.adj_j[fill[ehi[k]]] = elo[k];
      m.adj_e[fill[ehi[k]]++] = static_cast<int32_t>(k);
    }
  }
  std::vector<std::pair<int32_t, int32_t>> row;
  m.ell_j.assign(static_cast<size_t>(m.n_free) * 4, -1);
  m.ell_e.assign(static_cast<size_t>(m.n_free) * 4, 0);
  for (int64_t i = 0; i < m.n_free; ++i) {
    const int32_t a = m.adj_ptr[i], b = m.adj_ptr[i + 1];
    row.clear();
    for (int32_t t = a; t < b; ++t) row.emplace_back(m.adj_j[t], m.adj_e[t]);
    std::sort(row.begin(), row.end());
    for (int32_t t = a; t < b; ++t) {
      m.adj_j[t] = row[t - a].first;
      m.adj_e[t] = row[t - a].second;
      if (t - a < 4) {
        m.ell_j[4 * i + (t - a)] = row[t - a].first;
        m.ell_e[4 * i + (t - a)] = row[t - a].second;
      }
    }
  }
  // entries 5..8 in a second table where many nodes have more than four
  // neighbours (general triangulations: about six)
  int64_t wide = 0;
  for (int64_t i = 0; i < m.n_free; ++i) wide += (m.adj_ptr[i + 1] - m.adj_ptr[i]) > 4;
  m.ell_hi_j.clear();
  m.ell_hi_e.clear();
  if (m.n_free > 0 && 4 * wide >= m.n_free) {
    m.ell_hi_j.assign(static_cast<size_t>(m.n_free) * 4, -1);
    m.ell_hi_e.assign(static_cast<size_t>(m.n_free) * 4, 0);
    for (int64_t i = 0; i < m.n_free; ++i)
      for (int32_t t = m.adj_ptr[i] + 4; t < std::min(m.adj_ptr[i] + 8, m.adj_ptr[i + 1]); ++t) {
        m.ell_hi_j[4 * i + (t - m.adj_ptr[i] - 4)] = m.adj_j[t];
        m.ell_hi_e[4 * i + (t - m.adj_ptr[i] - 4)] = m.adj_e[t];
      }
  }
  return 0;
}

int64_t interp_weights(const double* xy_c, const int32_t* tri_c, int64_t n_tri_c, const double* xy_f,
                       int64_t n_f, int32_t* vert, double* w, double tol) {
  if (n_tri_c < 1 || n_f < 1) return n_f;
  double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
  for (int64_t t = 0; t < n_tri_c; ++t)
    for (int a = 0; a < 3; ++a) {
      const double* p = xy_c + 2 * int64_t(tri_c[3 * t + a]);
      x0 = std::min(x0, p[0]);
      x1 = std::max(x1, p[0]);
      y0 = std::min(y0, p[1]);
      y1 = std::max(y1, p[1]);
    }
  const int64_t G = std::max<int64_t>(1, static_cast<int64_t>(std::sqrt(double(n_tri_c))));
  const double sx = double(G) / std::max(x1 - x0, 1e-300), sy = double(G) / std::max(y1 - y0, 1e-300);
  auto cell = [&](double v, double lo, double sc) {
    return std::min<int64_t>(G - 1, std::max<int64_t>(0, static_cast<int64_t>((v - lo) * sc)));
  };
  // buckets: triangles whose bounding box meets the cell (CSR)
  std::vector<int64_t> count(size_t(G * G) + 1, 0);
  auto for_cells = [&](int64_t t, auto&& fn) {
    double a0 = 1e300, a1 = -1e300, b0 = 1e300, b1 = -1e300;
    for (int a = 0; a < 3; ++a) {
      const double* p = xy_c + 2 * int64_t(tri_c[3 * t + a]);
      a0 = std::min(a0, p[0]);
      a1 = std::max(a1, p[0]);
      b0 = std::min(b0, p[1]);
      b1 = std::max(b1, p[1]);
    }
    for (int64_t j = cell(b0, y0, sy); j <= cell(b1, y0, sy); ++j)
      for (int64_t i = cell(a0, x0, sx); i <= cell(a1, x0, sx); ++i) fn(j * G + i);
  };
  for (int64_t t = 0; t < n_tri_c; ++t) for_cells(t, [&](int64_t c) { ++count[size_t(c) + 1]; });
  for (size_t c = 0; c < size_t(G * G); ++c) count[c + 1] += count[c];
  std::vector<int32_t> items(size_t(count.back()));
  std::vector<int64_t> fill(count.begin(), count.end() - 1);
  for (int64_t t = 0; t < n_tri_c; ++t)
    for_cells(t, [&](int64_t c) { items[size_t(fill[size_t(c)]++)] = static_cast<int32_t>(t); });
  int64_t outside = 0;
  for (int64_t k = 0; k < n_f; ++k) {
    const double px = xy_f[2 * k], py = xy_f[2 * k + 1];
    const int64_t c = cell(py, y0, sy) * G + cell(px, x0, sx);
    double best = -1e300, bl[3] = {0, 0, 0};
    int64_t bt = -1;
    for (int64_t q = count[size_t(c)]; q < count[size_t(c) + 1]; ++q) {
      const int64_t t = items[size_t(q)];
      const double* p0 = xy_c + 2 * int64_t(tri_c[3 * t]);
      const double* p1 = xy_c + 2 * int64_t(tri_c[3 * t + 1]);
      const double* p2 = xy_c + 2 * int64_t(tri_c[3 * t + 2]);
      const double e1x = p1[0] - p0[0], e1y = p1[1] - p0[1], e2x = p2[0] - p0[0], e2y = p2[1] - p0[1];
      const double det = e1x * e2y - e1y * e2x;
      if (det == 0.0) continue;
      const double dx = px - p0[0], dy = py - p0[1];
      const double l1 = (dx * e2y - dy * e2x) / det, l2 = (e1x * dy - e1y * dx) / det, l0 = 1.0 - l1 - l2;
      const double worst = std::min(l0, std::min(l1, l2));
      if (worst > best) {
        best = worst;
        bt = t;
        bl[0] = l0;
        bl[1] = l1;
        bl[2] = l2;
      }
    }
    if (bt < 0 || best < -tol) ++outside;
    for (int a = 0; a < 3; ++a) {
      vert[3 * k + a] = bt < 0 ? 0 : tri_c[3 * bt + a];
      w[3 * k + a] = bt < 0 ? 0.0 : bl[a];
    }
  }
  return outside;
}

void build_r_slots(const HostMesh& m, std::vector<int32_t>& ptr, std::vector<int32_t>& slot_j,
                   std::vector<int32_t>& slot_e) {
  const int64_t nR = m.n_R, nP = m.n_P;
  ptr.assign(1, 0);
  slot_j.clear();
  slot_e.clear();
  for (int64_t i = 0; i < nR; ++i) {
    const bool iP = i < nP;
    for (int q = 0; q < 4; ++q) {
      const int32_t j = m.ell_j[4 * i + q];
      if (j < 0) continue;
      const bool jP = j < nP;
      if (jP || iP) {
        slot_j.push_back(jP ? j : -1);
        slot_e.push_back(m.ell_e[4 * i + q]);
      }
    }
    for (int32_t t = m.adj_ptr[i] + 4; t < m.adj_ptr[i + 1]; ++t) {
      const int32_t j = m.adj_j[t];
      const bool jP = j < nP;
      if (!jP && !iP) break;  // sorted: no P neighbour left
      slot_j.push_back(jP ? j : -1);
      slot_e.push_back(m.adj_e[t]);
    }
    ptr.push_back(static_cast<int32_t>(slot_j.size()));
  }
}

namespace {

// R's nodes in Morton order of their coordinates.
std::vector<int32_t> morton_order_R(const HostMesh& m) {
  const int64_t nR = m.n_R;
  double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
  for (int64_t i = 0; i < nR; ++i) {
    x0 = std::min(x0, m.xy[2 * i]);
    x1 = std::max(x1, m.xy[2 * i]);
    y0 = std::min(y0, m.xy[2 * i + 1]);
    y1 = std::max(y1, m.xy[2 * i + 1]);
  }
  const double sx = 65535.0 / std::max(x1 - x0, 1e-300), sy = 65535.0 / std::max(y1 - y0, 1e-300);
  std::vector<std::pair<uint64_t, int32_t>> key(nR);
  for (int64_t i = 0; i < nR; ++i) {
    const uint64_t qx = static_cast<uint64_t>((m.xy[2 * i] - x0) * sx);
    const uint64_t qy = static_cast<uint64_t>((m.xy[2 * i + 1] - y0) * sy);
    key[i] = {morton_spread16(qx) | (morton_spread16(qy) << 1), static_cast<int32_t>(i)};
  }
  std::sort(key.begin(), key.end());
  std::vector<int32_t> out(nR);
  for (int64_t a = 0; a < nR; ++a) out[a] = key[a].second;
  return out;
}

// Nodes of one tile: the core order[a0, a1), then `layers` layers of P
// nodes (BFS through P neighbours); lens receives core + layers 1..k for
// k = 0..layers.  stamp/mark: per-node scratch, stamp[i] == mark means in
// the tile.
void tile_nodes(const HostMesh& m, const std::vector<int32_t>& order, int64_t a0, int64_t a1, int layers,
                std::vector<int64_t>& stamp, int64_t mark, std::vector<int32_t>& nodes,
                std::vector<int32_t>& lens) {
  const int64_t nP = m.n_P;
  nodes.clear();
  lens.clear();
  for (int64_t a = a0; a < a1; ++a) {
    stamp[order[a]] = mark;
    nodes.push_back(order[a]);
  }
  lens.push_back(static_cast<int32_t>(nodes.size()));
  size_t f0 = 0;
  for (int k = 1; k <= layers; ++k) {
    const size_t f1 = nodes.size();
    for (size_t f = f0; f < f1; ++f) {
      const int32_t i = nodes[f];
      for (int32_t t = m.adj_ptr[i]; t < m.adj_ptr[i + 1]; ++t) {
        const int32_t j = m.adj_j[t];
        if (j < nP && stamp[j] != mark) {
          stamp[j] = mark;
          nodes.push_back(j);
        }
      }
    }
    f0 = f1;
    lens.push_back(static_cast<int32_t>(nodes.size()));
  }
}

}  // namespace

int make_moving(HostMesh& m, const double* disp, int K, std::string& err) {
  if (!disp || K < 1 || K > 16) {
    err = "mesh_add_moving: null displacement modes or K outside [1, 16]";
    return -1;
  }
  if (m.tri_new.size() != static_cast<size_t>(m.n_tri) * 3) {
    err = "mesh_add_moving: mesh not prepared with every edge kept";
    return -1;
  }
  const int64_t na = m.adj_ptr[m.n_free];
  m.moving = true;
  m.K_modes = K;
  m.dedge.assign(m.adj_e.begin(), m.adj_e.end());
  for (int64_t t = 0; t < na; ++t) m.adj_e[t] = static_cast<int32_t>(t);
  for (int64_t i = 0; i < m.n_free; ++i) {
    const int32_t a = m.adj_ptr[i], n = m.adj_ptr[i + 1] - a;
    for (int q = 0; q < 4 && q < n; ++q) m.ell_e[4 * i + q] = a + q;
    if (!m.ell_hi_e.empty())
      for (int q = 0; q < 4 && q + 4 < n; ++q) m.ell_hi_e[4 * i + q] = a + 4 + q;
  }
  m.n_w = na;
  // elements of every free node
  std::vector<int32_t> cnt(m.n_free + 1, 0);
  for (int64_t k = 0; k < m.n_tri; ++k)
    for (int a = 0; a < 3; ++a)
      if (m.tri_new[3 * k + a] < m.n_free) cnt[m.tri_new[3 * k + a] + 1]++;
  m.nptr.assign(m.n_free + 1, 0);
  for (int64_t i = 0; i < m.n_free; ++i) m.nptr[i + 1] = m.nptr[i] + cnt[i + 1];
  m.nelem.assign(m.nptr[m.n_free], 0);
  std::vector<int32_t> fill(m.nptr.begin(), m.nptr.end() - 1);
  for (int64_t k = 0; k < m.n_tri; ++k)
    for (int a = 0; a < 3; ++a) {
      const int32_t v = m.tri_new[3 * k + a];
      if (v < m.n_free) m.nelem[fill[v]++] = static_cast<int32_t>(k);
    }
  m.disp.assign(static_cast<size_t>(K) * m.n_nodes * 2, 0.0);
  for (int k = 0; k < K; ++k)
    for (int64_t v = 0; v < m.n_nodes; ++v)
      for (int c = 0; c < 2; ++c)
        m.disp[(static_cast<size_t>(k) * m.n_nodes + v) * 2 + c] =
            disp[(static_cast<size_t>(k) * m.n_nodes + m.new2old[v]) * 2 + c];
  m.minv.assign(m.n_free, 1.0);  // the weights carry 1 / m_i of the draw
  return 0;
}

bool build_pair_plan(const HostMesh& m, int bn, PairPlan& out) {
  out = PairPlan();
  const int64_t nR = m.n_R, nP = m.n_P;
  if (nR == 0 || bn < 1) return false;
  const std::vector<int32_t> order = morton_order_R(m);
  double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
  for (int64_t i = 0; i < nR; ++i) {
    x0 = std::min(x0, m.xy[2 * i]);
    x1 = std::max(x1, m.xy[2 * i]);
    y0 = std::min(y0, m.xy[2 * i + 1]);
    y1 = std::max(y1, m.xy[2 * i + 1]);
  }
  const double wx = std::max(x1 - x0, 1e-300), wy = std::max(y1 - y0, 1e-300);
  // node spacing of the densest part of R: the median over R of each node's
  // shortest edge; a cell of side L there holds about (L / h)^2 nodes
  std::vector<double> hmin;
  hmin.reserve(static_cast<size_t>(nR));
  for (int64_t i = 0; i < nR; ++i) {
    double best = 1e300;
    for (int32_t t = m.adj_ptr[i]; t < m.adj_ptr[i + 1]; ++t) {
      const int32_t j = m.adj_j[t];
      best = std::min(best, std::hypot(m.xy[2 * j] - m.xy[2 * i], m.xy[2 * j + 1] - m.xy[2 * i + 1]));
    }
    if (best < 1e300) hmin.push_back(best);
  }
  double h = std::sqrt(wx * wy / double(nR));
  if (!hmin.empty()) {
    std::nth_element(hmin.begin(), hmin.begin() + hmin.size() / 2, hmin.end());
    h = hmin[hmin.size() / 2];
  }
  const double L = std::max(h, std::sqrt(double(bn)) * h);
  const int64_t ncx = std::max<int64_t>(1, static_cast<int64_t>(std::ceil(wx / L))),
                ncy = std::max<int64_t>(1, static_cast<int64_t>(std::ceil(wy / L)));
  if (ncx * ncy > (int64_t(1) << 26)) return false;
  std::vector<std::vector<int32_t>> byc(ncx * ncy);
  for (int64_t a = 0; a < nR; ++a) {
    const int32_t i = order[a];
    const int64_t cx = std::min<int64_t>(ncx - 1, static_cast<int64_t>((m.xy[2 * i] - x0) / L));
    const int64_t cy = std::min<int64_t>(ncy - 1, static_cast<int64_t>((m.xy[2 * i + 1] - y0) / L));
    byc[cy * ncx + cx].push_back(i);
  }
  out.rptr.assign(1, 0);
  out.lidx.assign(static_cast<size_t>(m.adj_ptr[nR]), int16_t(-1));
  std::vector<int32_t> local(nR, -1);  // row of a node in the current block (reset after)
  for (const auto& core : byc) {
    if (core.empty()) continue;
    const size_t r0 = out.row.size();
    for (const int32_t i : core) {
      local[i] = static_cast<int32_t>(out.row.size() - r0);
      out.row.push_back(i);
    }
    for (const int32_t i : core)
      for (int32_t t = m.adj_ptr[i]; t < m.adj_ptr[i + 1]; ++t) {
        const int32_t j = m.adj_j[t];
        if (j >= nP) continue;
        if (local[j] < 0) {
          local[j] = static_cast<int32_t>(out.row.size() - r0);
          out.row.push_back(j);
        }
        if (local[j] > 32767) return false;
        out.lidx[t] = static_cast<int16_t>(local[j]);
      }
    for (size_t k = r0; k < out.row.size(); ++k) local[out.row[k]] = -1;
    const int64_t nr = static_cast<int64_t>(out.row.size() - r0);
    out.rows_max = std::max(out.rows_max, nr);
    out.core_max = std::max<int64_t>(out.core_max, static_cast<int64_t>(core.size()));
    out.ncore.push_back(static_cast<int32_t>(core.size()));
    out.rptr.push_back(static_cast<int32_t>(out.row.size()));
    ++out.n_blocks;
  }
  return true;
}

bool build_tile_plan(const HostMesh& m, int p, int64_t cap, TilePlan& out) {
  out = TilePlan();
  const int64_t nR = m.n_R, nP = m.n_P;
  if (nR == 0 || p < 2 || cap < 16) return false;
  std::vector<int32_t> rptr, rsj, rse;
  build_r_slots(m, rptr, rsj, rse);
  const std::vector<int32_t> order = morton_order_R(m);  // Morton order inside each cell
  double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
  for (int64_t i = 0; i < nR; ++i) {
    x0 = std::min(x0, m.xy[2 * i]);
    x1 = std::max(x1, m.xy[2 * i]);
    y0 = std::min(y0, m.xy[2 * i + 1]);
    y1 = std::max(y1, m.xy[2 * i + 1]);
  }
  const double wx = std::max(x1 - x0, 1e-300), wy = std::max(y1 - y0, 1e-300);
  // nodes per unit length if R filled its box; the core of a cell of side L
  // holds about (L / h)^2 nodes and its tile (L / h + 2 (p - 2))^2
  const double h = std::sqrt(wx * wy / double(nR));
  double L = std::max(h, (std::sqrt(double(cap)) - 2.0 * (p - 2)) * h);
  std::vector<int64_t> stamp(nR, -1);
  std::vector<int32_t> nodes, lens;
  std::vector<std::vector<int32_t>> cells;
  int64_t mark = 0;
  for (int attempt = 0;; ++attempt) {
    // cores: the nodes of R binned into cells of side L (each in Morton order)
    const int64_t ncx = std::max<int64_t>(1, static_cast<int64_t>(std::ceil(wx / L))),
                  ncy = std::max<int64_t>(1, static_cast<int64_t>(std::ceil(wy / L)));
    if (ncx * ncy > (int64_t(1) << 26)) return false;
    std::vector<int32_t> cell_of(nR);
    for (int64_t a = 0; a < nR; ++a) {
      const int32_t i = order[a];
      const int64_t cx = std::min<int64_t>(ncx - 1, static_cast<int64_t>((m.xy[2 * i] - x0) / L));
      const int64_t cy = std::min<int64_t>(ncy - 1, static_cast<int64_t>((m.xy[2 * i + 1] - y0) / L));
      // cells in row order, so that consecutive tiles are neighbours
      cell_of[i] = static_cast<int32_t>(cy * ncx + cx);
    }
    cells.clear();
    std::vector<std::vector<int32_t>> byc(ncx * ncy);
    for (int64_t a = 0; a < nR; ++a) byc[cell_of[order[a]]].push_back(order[a]);
    for (auto& v : byc)
      if (!v.empty()) cells.push_back(std::move(v));
    int64_t worst = 0;
    for (const auto& core : cells) {
      tile_nodes(m, core, 0, static_cast<int64_t>(core.size()), p - 1, stamp, mark++, nodes, lens);
      worst = std::max<int64_t>(worst, lens[p - 2]);
      if (lens[p - 1] > 32000) {
        worst = cap + 1;
        break;
      }
    }
    if (worst <= cap) break;
    if (attempt > 80 || L <= 0.5 * h) return false;
    L *= 0.95;
  }
  out.p = p;
  out.cap = static_cast<int>(cap);
  out.ptr.assign(1, 0);
  std::vector<int32_t> local(nR, -1);
  for (const auto& core : cells) {
    tile_nodes(m, core, 0, static_cast<int64_t>(core.size()), p - 1, stamp, mark, nodes, lens);
    const int32_t n_all = static_cast<int32_t>(nodes.size());
    for (int32_t a = 0; a < n_all; ++a) local[nodes[a]] = a;
    const int32_t n_comp = lens[p - 2];
    for (int32_t a = 0; a < n_all; ++a) {
      const int32_t i = nodes[a];
      out.node.push_back(i);
      // slots: local row of the neighbour's r, or the zero row (n_all) for a
      // coupling to a node off P; unused slots: zero row and edge -1
      int32_t q4[4] = {n_all, n_all, n_all, n_all}, e4[4] = {-1, -1, -1, -1};
      int32_t xoff = static_cast<int32_t>(out.xs.size() / 2), xcnt = 0;
      if (a < n_comp) {
        for (int32_t s = rptr[i]; s < rptr[i + 1]; ++s) {
          int32_t lj = n_all;
          if (rsj[s] >= 0) {
            if (stamp[rsj[s]] != mark) return false;  // cannot happen: the layers close the tile
            lj = local[rsj[s]];
          }
          const int32_t q = s - rptr[i];
          if (q < 4) {
            q4[q] = lj;
            e4[q] = rse[s];
          } else {
            out.xs.push_back(lj);
            out.xs.push_back(rse[s]);
            ++xcnt;
          }
        }
        if (xcnt > 15) return false;
      }
      out.sj.push_back(static_cast<int32_t>(uint32_t(uint16_t(q4[0])) | (uint32_t(uint16_t(q4[1])) << 16)));
      out.sj.push_back(static_cast<int32_t>(uint32_t(uint16_t(q4[2])) | (uint32_t(uint16_t(q4[3])) << 16)));
      for (int q = 0; q < 4; ++q) out.se.push_back(e4[q]);
      out.xp.push_back((xcnt ? ((xoff << 5) | (xcnt << 1)) : 0) | (i < nP ? 1 : 0));
      out.minv.push_back(i < m.n_free ? m.minv[i] : 0.0);
    }
    for (int k = 0; k < p; ++k) out.len.push_back(lens[k]);
    out.n_all_max = std::max<int64_t>(out.n_all_max, static_cast<int64_t>(n_all));
    out.ptr.push_back(static_cast<int32_t>(out.node.size()));
    ++mark;
  }
  return true;
}

}  // namespace lflts
