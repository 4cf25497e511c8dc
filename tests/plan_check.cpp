// Host-side checks of the block plans of the paired inner substeps and of
// the tables of a mesh whose vertices move with the draw (no GPU).  Reads a
// mesh written by tests/test_plans_host.py, prepares it as the library does
// and checks the invariants every kernel relies on; prints "OK" or the first
// violation and exits non-zero.
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <set>
#include <string>
#include <vector>

#include "../paper_2106_11117_gb300/csrc/mesh_prep.h"

using namespace lflts;

static int fail(const std::string& what) {
  std::printf("FAIL %s\n", what.c_str());
  return 1;
}

static bool read_all(FILE* f, void* p, size_t size, size_t n) { return std::fread(p, size, n, f) == n; }

int main(int argc, char** argv) {
  if (argc < 2) return fail("usage: plan_check mesh.bin [uniform]");
  const bool uniform = argc > 2 && std::string(argv[2]) == "uniform";
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return fail("cannot open the mesh file");
  int64_t nn = 0, nt = 0;
  int32_t K = 0;
  if (!read_all(f, &nn, 8, 1) || !read_all(f, &nt, 8, 1) || !read_all(f, &K, 4, 1)) return fail("header");
  std::vector<double> xy(2 * nn), psi(nt * K), disp(2 * nn);
  std::vector<int32_t> tri(3 * nt);
  std::vector<uint8_t> dir(nn), P(nn);
  if (!read_all(f, xy.data(), 8, 2 * nn) || !read_all(f, tri.data(), 4, 3 * nt) || !read_all(f, dir.data(), 1, nn) ||
      !read_all(f, P.data(), 1, nn) || !read_all(f, psi.data(), 8, nt * K) || !read_all(f, disp.data(), 8, 2 * nn))
    return fail("body");
  std::fclose(f);

  // ---- pair plans on the fixed mesh -------------------------------------
  HostMesh m;
  std::string err;
  if (prep_mesh(xy.data(), nn, tri.data(), nt, dir.data(), P.data(), psi.data(), K, m, err)) return fail(err);
  const int64_t nR = m.n_R, nP = m.n_P;
  for (int bn : {16, 64, 144}) {
    PairPlan pl;
    if (!build_pair_plan(m, bn, pl)) return fail("no plan for bn " + std::to_string(bn));
    if ((int64_t)pl.rptr.size() != pl.n_blocks + 1 || (int64_t)pl.ncore.size() != pl.n_blocks)
      return fail("plan sizes");
    std::vector<int> seen(nR, 0);
    for (int64_t b = 0; b < pl.n_blocks; ++b) {
      const int r0 = pl.rptr[b], nr = pl.rptr[b + 1] - r0, nc = pl.ncore[b];
      if (nc < 1 || nc > nr || nr > pl.rows_max || nc > pl.core_max) return fail("block bounds");
      std::set<int> core, rows;
      for (int t = 0; t < nr; ++t) {
        const int i = pl.row[r0 + t];
        if (i < 0 || i >= nR) return fail("row outside R");
        if (!rows.insert(i).second) return fail("node twice in a block");
        if (t < nc) {
          core.insert(i);
          seen[i]++;
        } else if (i >= nP) {
          return fail("halo node outside P");
        }
      }
      // every P neighbour of a core node is a row of the block, lidx names it
      std::set<int> needed;
      for (int t = 0; t < nc; ++t) {
        const int i = pl.row[r0 + t];
        for (int a = m.adj_ptr[i]; a < m.adj_ptr[i + 1]; ++a) {
          const int j = m.adj_j[a];
          if (j < nP) {
            const int l = pl.lidx[a];
            if (l < 0 || l >= nr || pl.row[r0 + l] != j) return fail("lidx does not name the neighbour's row");
            needed.insert(j);
          } else if (pl.lidx[a] != -1) {
            return fail("lidx set for a neighbour off P");
          }
        }
      }
      for (int t = nc; t < nr; ++t)
        if (!needed.count(pl.row[r0 + t]) || core.count(pl.row[r0 + t])) return fail("halo node not needed");
    }
    for (int64_t i = 0; i < nR; ++i)
      if (seen[i] != 1) return fail("R node not in exactly one core");
    // cells of a uniform R hold bn nodes (k x k cores)
    if (uniform && pl.core_max != bn)
      return fail("core_max " + std::to_string(pl.core_max) + " for bn " + std::to_string(bn));
  }

  // ---- tables of the moving mesh ------------------------------------------
  HostMesh mv;
  if (prep_mesh(xy.data(), nn, tri.data(), nt, dir.data(), P.data(), psi.data(), K, mv, err, true))
    return fail(err);
  if (make_moving(mv, disp.data(), 1, err)) return fail(err);
  const int64_t na = mv.adj_ptr[mv.n_free];
  if (mv.n_w != na || (int64_t)mv.dedge.size() != na) return fail("moving: weight rows");
  for (int64_t i = 0; i < mv.n_free; ++i) {
    if (mv.minv[i] != 1.0) return fail("moving: 1/m is not 1");
    const int a = mv.adj_ptr[i], n = mv.adj_ptr[i + 1] - a;
    for (int q = 0; q < 4 && q < n; ++q)
      if (mv.ell_e[4 * i + q] != a + q || mv.ell_j[4 * i + q] != mv.adj_j[a + q]) return fail("moving: table ids");
    for (int t = a; t < a + n; ++t) {
      if (mv.adj_e[t] != t) return fail("moving: adjacency ids");
      const int e = mv.dedge[t];
      const int lo = std::min<int>(i, mv.adj_j[t]), hi = std::max<int>(i, mv.adj_j[t]);
      if (mv.edge_i[e] != lo || mv.edge_j[e] != hi) return fail("moving: entry's edge");
    }
    // the node's elements are exactly the elements having it as a vertex
    for (int q = mv.nptr[i]; q < mv.nptr[i + 1]; ++q) {
      const int k = mv.nelem[q];
      if (mv.tri_new[3 * k] != i && mv.tri_new[3 * k + 1] != i && mv.tri_new[3 * k + 2] != i)
        return fail("moving: element list");
    }
  }
  int64_t incid = 0;
  for (int64_t k = 0; k < mv.n_tri; ++k)
    for (int a = 0; a < 3; ++a) incid += mv.tri_new[3 * k + a] < mv.n_free;
  if (incid != mv.nptr[mv.n_free]) return fail("moving: element incidences");
  // displacement modes follow the node order
  for (int64_t v = 0; v < mv.n_nodes; ++v)
    if (mv.disp[2 * v + 1] != disp[2 * mv.new2old[v] + 1]) return fail("moving: mode order");
  std::printf("OK\n");
  return 0;
}
