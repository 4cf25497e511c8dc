// C ABI of the LF-LTS / MLMC library (declared in include/lflts.h).
//
// Host orchestration of the kernels in kernels.cuh and adjoint.cuh: mesh
// upload, per-solve workspaces, the time loop of Alg. 2 (one coarse launch
// and p-1 inner launches per step, or one fused inner launch for a small R),
// the QoI reduction and the MLMC level sums, merged batched solves for level
// pairs (ragged batches for draws with their own time steps, long solves
// queued in slices across streams), CUDA graphs, the launch-shape autotuner,
// the discrete adjoint and profiling counters.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/lflts.h"
#include "adjoint.cuh"
#include "coarse_rc.cuh"
#include "field_qoi.cuh"
#include "inner_pair.cuh"
#include "inner_tile.cuh"
#include "kernels.cuh"
#include "mesh_prep.h"
#include "moving.cuh"
#include "restride.cuh"

using namespace lflts;

namespace {

// Largest batch: 65535 CTA rows of 32 samples (grid y limit).
constexpr int64_t kMaxS = int64_t(65535) * 32;

struct Buf {
  void* p = nullptr;
  size_t n = 0;
};

struct MeshGPU {
  HostMesh h;
  int* adj_ptr = nullptr;
  int2* adj = nullptr;
  int4* ell = nullptr;
  int4* ell_hi = nullptr;   // entries 5..8 (general triangulations) or null
  int2* ee = nullptr;       // elements of each edge
  int2* ends = nullptr;     // endpoints of each edge (i < j)
  float* eg32 = nullptr;    // [n_edges][2] element entries G
  double* eg64 = nullptr;
  float* minv32 = nullptr;
  double* minv64 = nullptr;
  float* psi32 = nullptr;
  double* psi64 = nullptr;
  int* new2old = nullptr;
  // a mesh whose vertices move with the draw: the tables of k_moving_weights
  int* dedge = nullptr;
  int* tri_new = nullptr;
  double* xy64 = nullptr;
  double* disp = nullptr;
  int* nptr = nullptr;
  int* nelem = nullptr;
  MovingDev moving() const {
    return MovingDev{static_cast<int>(h.n_free), static_cast<int>(h.n_nodes), h.K_modes, adj_ptr, adj, dedge,
                     ee, tri_new, xy64, disp, nptr, nelem};
  }
  int* tri_dev = nullptr;    // caller's triangles and areas (L2(D)-valued QoI, uploaded on first use)
  double* area_dev = nullptr;
  // coupling slots of R for the fused inner kernel (built on first use)
  int* rptr = nullptr;
  int2* rslot = nullptr;
  int64_t n_rslots = -1;
  // autotuned (vec, shape code) per (S, precision, p)
  std::map<std::tuple<int64_t, int, int>, std::pair<int, int>> tuned;
  // whether the coarse launch forms its weights (k_coarse_rc), per (S, precision, p)
  std::map<std::tuple<int64_t, int, int>, bool> tuned_rc;
  // tile plans of the on-chip inner substeps per (p, tile capacity), uploaded
  struct DevTiles {
    TileDev dev{};
    bool ok = false;
  };
  std::map<std::pair<int, int64_t>, DevTiles> tiles;
  // block plans of the paired inner substeps per block size, uploaded
  struct DevPairs {
    PairDev dev{};
    bool ok = false;
  };
  std::map<int, DevPairs> pairs;
};

struct Field {
  int mesh;
  float* v32 = nullptr;
  double* v64 = nullptr;
};

struct Source {
  int mesh;
  float* fw32 = nullptr;   // M^-1 F on the free nodes (internal order)
  double* fw64 = nullptr;
};

struct Qoi {
  int mesh;
  int nnz;
  int* idx = nullptr;  // new node ids
  double* g = nullptr;
};

// Nodal interpolation from a coarse to a fine mesh (caller's numbering).
struct Interp {
  int mesh_f, mesh_c;
  int* vert = nullptr;   // [n_nodes_f][3] coarse vertices
  double* w = nullptr;   // [n_nodes_f][3] barycentric weights
};

// Buffers of lflts_run_field_pair.
struct FieldBufs {
  Buf uf, uc, qf, qc, s1, n2, ps, pc, sums, xraw, dq;
};

// Largest solve (in kernels) captured into one CUDA graph.
constexpr int64_t kGraphMaxKernels = 120000;
// Outer steps queued per turn when lflts_run_pairs interleaves long solves.
constexpr int64_t kSliceSteps = 32;

// Everything a captured solve graph depends on.
struct GraphKey {
  int mesh, qoi, u0, v0, precision, p;
  double nu, dt;
  int64_t n_steps, S;
  const void *xi, *Q, *uN, *ua, *ub, *d, *g, *r0, *r1, *r2, *r3, *W, *xipad, *qps, *qpc;
  int vec, cps, source;
  double f0, t0, famp;
  uint64_t ragged;           // segment list of a ragged batch (0: uniform)
  const void *dts, *sig;
  bool operator==(const GraphKey& o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec;
  int64_t kernels;
};

struct Workspace {
  Buf ua, ub, d, g, r0, r1, r2, r3, W, xipad, xraw, qps, qpc, Q, uN;
  Buf cmp;                             // scratch of a ragged batch's stride narrowing
  Buf dts, sig;                        // per-draw dt and (dt / dt_ref)^2 of a ragged batch
  std::vector<double> h_dts;           // host copies of the two (kept for the async copies)
  std::vector<unsigned char> h_sig;
  std::vector<GraphEntry> graphs;
};

// Buffers of the adjoint (gradient) solve.
struct GradBufs {
  Buf ckpt, segU, rs, rho, gs, A, Aseg, nua, nub, dnu, part, xraw, Q, G;
};

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
  double bytes;
};

struct PairRun;  // a level-pair batch between the calls of a sliced run

}  // namespace

struct lflts_ctx {
  int device = -1;  // -1: host-only context (mesh preparation, no solves)
  int sms = 152;
  std::string err;
  std::vector<std::unique_ptr<MeshGPU>> meshes;
  std::vector<Field> fields;
  std::vector<Qoi> qois;
  std::vector<Source> sources;
  std::vector<std::unique_ptr<Workspace>> ws;
  std::unique_ptr<Workspace> gws;   // forward buffers of lflts_grad_xi
  std::unique_ptr<GradBufs> gb;     // adjoint buffers of lflts_grad_xi
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> sync_events;
  int* d_bad = nullptr;
  double* d_scratch = nullptr;  // small FP64 staging (sums)
  bool profiling = false;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> pool;
  int64_t prof_launches[LFLTS_KERNEL_CLASSES] = {0};
  double prof_ms[LFLTS_KERNEL_CLASSES] = {0};
  double prof_bytes[LFLTS_KERNEL_CLASSES] = {0};
  int64_t launches = 0;
  int64_t tune_launches = 0;
  int64_t graph_launches = 0;
  bool graphs = true;
  int64_t graph_cap = 8;  // instantiated solve graphs kept per workspace (least recently used dropped)
  bool autotune = true;
  int fused_mode = 1;            // fused inner kernel: 0 never, 1 autotuned, 2 always where it fits
  int tile_mode = 1;             // tiled inner kernel: 0 never, 1 autotuned, 2 always where it fits
  int64_t tile_cap = 0;          // > 0: at most this many computed nodes per tile
  int pair_mode = 1;             // paired inner substeps: 0 never, 1 autotuned, 2 always where they fit
  int pair_block = 144;          // about this many nodes of R per block of the paired substeps
  int64_t pair_min_r = 0;        // forced paired substeps only where |R| is at least this
  int coarse_rc = 0;             // coarse launch forming its weights: 0 never (measured slower), 1 timed, 2 always
  std::vector<void*> owned;  // device allocations of meshes, fields, QoIs
  std::unique_ptr<PairRun> run;  // lflts_run_pairs_slice: the run in progress, if any
  std::vector<Interp> interps;   // lflts_field_interp_add
  std::unique_ptr<Workspace> fws[2];  // fine and coarse solves of lflts_run_field_pair
  std::unique_ptr<FieldBufs> fb;
  ~lflts_ctx();
};

namespace {

int fail(lflts_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define LF_CUDA(ctx, call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? LFLTS_ERR_OOM : LFLTS_ERR_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

#define LF_TRY(expr)      \
  do {                    \
    int rc_ = (expr);     \
    if (rc_ != 0) return rc_; \
  } while (0)

int ensure(lflts_ctx* c, Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.n >= bytes) return 0;
  if (b.p) {
    cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
  }
  LF_CUDA(c, cudaMalloc(&b.p, bytes));
  b.n = bytes;
  return 0;
}

template <typename T>
int upload(lflts_ctx* c, T** dst, const T* src, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  LF_CUDA(c, cudaMalloc((void**)dst, bytes));
  c->owned.push_back(*dst);
  if (count) LF_CUDA(c, cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
  return 0;
}

int set_device(lflts_ctx* c) {
  if (c->device < 0) return fail(c, LFLTS_ERR_ARG, "host-only context: no device for this call");
  LF_CUDA(c, cudaSetDevice(c->device));
  return 0;
}

cudaEvent_t get_event(lflts_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void harvest(lflts_ctx* c);

struct Prof {
  lflts_ctx* c;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  Prof(lflts_ctx* c_, cudaStream_t st_) : c(c_), st(st_) {
    if (c->profiling) {
      a = get_event(c);
      cudaEventRecord(a, st);
    }
  }
  void end(int cls, double bytes) {
    c->launches++;
    if (c->profiling) {
      cudaEvent_t b = get_event(c);
      cudaEventRecord(b, st);
      c->pending.push_back({cls, a, b, bytes});
      if (c->pending.size() >= 16384) harvest(c);
    }
  }
};

// Books the profiled launches whose end event has completed and recycles
// their events, without waiting: long profiled runs keep a bounded list.
void harvest(lflts_ctx* c) {
  size_t keep = 0;
  for (size_t k = 0; k < c->pending.size(); ++k) {
    ProfRec& r = c->pending[k];
    if (cudaEventQuery(r.b) == cudaSuccess) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        c->prof_ms[r.cls] += ms;
        c->prof_bytes[r.cls] += r.bytes;
        c->prof_launches[r.cls] += 1;
      }
      c->pool.push_back(r.a);
      c->pool.push_back(r.b);
    } else {
      c->pending[keep++] = r;
    }
  }
  c->pending.resize(keep);
  // a query of an event still in flight answers "not ready": not an error of
  // any launch (each launch's own status was taken right after it)
  if (cudaPeekAtLastError() == cudaErrorNotReady) (void)cudaGetLastError();
}

// Chebyshev constants of the stabilised scheme (Sec. 3.3) and the derived
// increment-form coefficients.  out: delta, omega, c0, gamma, then for
// m = 1..p-1: beta_m, c_m.
void lts_constants(int p, double nu, double dt, std::vector<double>& beta, std::vector<double>& cm,
                   double& delta, double& omega, double& c0, double& gamma) {
  delta = 1.0 + nu / (double(p) * p);
  std::vector<double> T(p + 2), U(p + 2);
  T[0] = 1.0;
  T[1] = delta;
  for (int k = 1; k <= p; ++k) T[k + 1] = 2.0 * delta * T[k] - T[k - 1];
  U[0] = 1.0;
  U[1] = 2.0 * delta;
  for (int k = 1; k <= p; ++k) U[k + 1] = 2.0 * delta * U[k] - U[k - 1];
  const double Tp_prime = p * U[p - 1];
  omega = 2.0 * Tp_prime / T[p];
  c0 = dt * dt / (omega * delta);
  beta.assign(p, 0.0);
  cm.assign(p, 0.0);
  for (int m = 1; m < p; ++m) {
    beta[m] = T[m - 1] / T[m + 1];
    cm[m] = 2.0 * dt * dt * (T[m] / T[m + 1]) / omega;
  }
  // gamma: the same recursion for a node whose AP-term vanishes, with g = 1
  double r_prev = 0.0, r = -c0;
  for (int m = 1; m < p; ++m) {
    const double rn = (1.0 + beta[m]) * r - beta[m] * r_prev - cm[m];
    r_prev = r;
    r = rn;
  }
  gamma = -r;
}

struct Geo {
  dim3 grid;
  int SB;
};

// Launch shape of the node/edge kernels: SB lanes per node (a power of two
// up to 32) each owning one sample vector.  Grid x covers the nodes
// (grid-stride), grid y the sample slabs; about 16 CTAs of 256 threads per SM.
// SB is the largest lane count that leaves at most a quarter of the lanes of
// the sample slabs idle.
Geo geometry(const lflts_ctx* c, int64_t n, int64_t SV, int cta_per_sm = 16) {
  int SB = 1;
  for (int sb = 32; sb > 1; sb /= 2) {
    const int64_t waste = ((SV + sb - 1) / sb) * sb - SV;
    if (waste * 4 <= SV) {
      SB = sb;
      break;
    }
  }
  const int NB = 256 / SB;
  const int64_t gy = (SV + SB - 1) / SB;
  const int64_t target = int64_t(c->sms) * cta_per_sm;
  int64_t gx = std::max<int64_t>(1, std::min<int64_t>((n + NB - 1) / NB, std::max<int64_t>(1, target / gy)));
  Geo g;
  g.grid = dim3(static_cast<unsigned>(gx), static_cast<unsigned>(gy), 1);
  g.SB = SB;
  return g;
}

int blocks_for(int64_t total, int threads, int cap) {
  int64_t b = (total + threads - 1) / threads;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(b, cap)));
}

template <typename Real>
struct Sel;
template <>
struct Sel<float> {
  static MeshDev<float> mesh(const MeshGPU& m, int n_R) {
    return MeshDev<float>{(int)m.h.n_free, n_R, (int)m.h.n_P, m.adj_ptr, m.adj, m.ell, m.minv32, m.ell_hi};
  }
  static const float* field(const Field& f) { return f.v32; }
  static const float* eg(const MeshGPU& m) { return m.eg32; }
  static const float* psi(const MeshGPU& m) { return m.psi32; }
  static const float* fw(const Source& s) { return s.fw32; }
};
template <>
struct Sel<double> {
  static MeshDev<double> mesh(const MeshGPU& m, int n_R) {
    return MeshDev<double>{(int)m.h.n_free, n_R, (int)m.h.n_P, m.adj_ptr, m.adj, m.ell, m.minv64, m.ell_hi};
  }
  static const double* field(const Field& f) { return f.v64; }
  static const double* eg(const MeshGPU& m) { return m.eg64; }
  static const double* psi(const MeshGPU& m) { return m.psi64; }
  static const double* fw(const Source& s) { return s.fw64; }
};

// Geometry of the node/edge kernels: SB lanes of VEC samples per node.
Geo geometry_vec(const lflts_ctx* c, int64_t n, int64_t S, int vec, int cta_per_sm = 16) {
  return geometry(c, n, (S + vec - 1) / vec, cta_per_sm);  // a ragged prefix may end inside a vector
}

// Plan of the fused inner kernel (all substeps of a step in one launch, R in
// shared memory): lanes per node SBf (draw slab SL = SBf vec) and dynamic
// shared memory; smem = 0 when R does not fit.
constexpr size_t kFusedSmemMax = 200 * 1024;
inline void fused_plan(const lflts_ctx* c, int n_R, int64_t n_slots, int64_t S, int vec, size_t rb, int& SBf,
                       size_t& smem) {
  (void)c;
  SBf = 1;
  smem = 0;
  if (n_R < 1 || n_slots < 0) return;
  // lanes per node: fill the 256 threads of a CTA when R is small (the
  // kernels of a step are short; fewer, fuller CTAs load less index data)
  while (SBf < 8 && int64_t(n_R) * SBf * 2 <= 256 && int64_t(SBf) * 2 * vec <= S) SBf *= 2;
  const int SL = SBf * vec;
  const size_t need = (fused_real_count(n_R, static_cast<int>(n_slots), SL) * rb + 15) / 16 * 16 +
                      (size_t(n_slots) + size_t(n_R) + 1) * sizeof(int);
  if (need <= kFusedSmemMax) smem = need;
}

// Launch shapes of the tiled inner kernel: draws per node (VEC), nodes per
// thread (IT) and threads (NT); a tile holds at most IT * NT computed nodes.
// All keep their per-node state in registers without spills (ptxas -v).
struct TileShape {
  int vec, it, nt;
};
template <typename Real>
int tile_shapes() {
  return 1;
}
template <typename Real>
TileShape tile_shape(int) {  // one 16-byte row per node and slab
  if (sizeof(Real) == 8) return {2, 3, 384};
  return TileShape{4, 3, 384};
}
template <typename Real>
int64_t tile_cap(const lflts_ctx* c, int var) {
  const TileShape ts = tile_shape<Real>(var);
  const int64_t cap = int64_t(ts.it) * ts.nt;
  return c->tile_cap > 0 ? std::min<int64_t>(c->tile_cap, cap) : cap;
}
template <typename Real>
size_t tile_smem(const TileDev& td, int var) {
  return tile_smem_layout(td.n_all_max, td.comp_max, td.core_max, td.xs_max, tile_shape<Real>(var).vec, sizeof(Real))
      .total;
}
constexpr size_t kTileSmemMax = 220 * 1024;

// Kernels of a tile shape and p (p = 4 and 8 compiled with the substep
// loop unrolled, other p with a runtime loop).
template <typename Real, int V, int IT, int PC>
void tile_go(bool attr_only, int smem_attr, int grid, size_t smem, cudaStream_t st, const TileDev& td, int S,
             const Real* W, const Real* g, const Real* u, Real* un, Real* d, const InnerCoef<Real>& k, Real kappa,
             cudaError_t& e) {
  if (attr_only)
    e = cudaFuncSetAttribute(k_inner_tile<Real, V, IT, 384, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_attr);
  else
    k_inner_tile<Real, V, IT, 384, PC><<<grid, 384, smem, st>>>(td, S, W, g, u, un, d, k, kappa);
}
template <typename Real, int V, int IT>
void tile_go_p(int p, bool attr_only, int smem_attr, int grid, size_t smem, cudaStream_t st, const TileDev& td,
               int S, const Real* W, const Real* g, const Real* u, Real* un, Real* d, const InnerCoef<Real>& k,
               Real kappa, cudaError_t& e) {
  if (p == 8) tile_go<Real, V, IT, 8>(attr_only, smem_attr, grid, smem, st, td, S, W, g, u, un, d, k, kappa, e);
  else if (p == 4) tile_go<Real, V, IT, 4>(attr_only, smem_attr, grid, smem, st, td, S, W, g, u, un, d, k, kappa, e);
  else tile_go<Real, V, IT, 0>(attr_only, smem_attr, grid, smem, st, td, S, W, g, u, un, d, k, kappa, e);
}
template <typename Real>
cudaError_t tile_call(int var, int p, bool attr_only, int smem_attr, int grid, size_t smem, cudaStream_t st,
                      const TileDev& td, int S, const Real* W, const Real* g, const Real* u, Real* un, Real* d,
                      const InnerCoef<Real>& k, Real kappa) {
  cudaError_t e = cudaSuccess;
  if constexpr (sizeof(Real) == 8) {
    (void)var;
    tile_go_p<Real, 2, 3>(p, attr_only, smem_attr, grid, smem, st, td, S, W, g, u, un, d, k, kappa, e);
  } else {
    (void)var;
    tile_go_p<Real, 4, 3>(p, attr_only, smem_attr, grid, smem, st, td, S, W, g, u, un, d, k, kappa, e);
  }
  return e;
}

// Paired inner substeps: the shared memory of a CTA (rows of r_{m+1} for a
// slab of 32 draws and the staged index data).
template <typename Real>
size_t pair_smem(const PairDev& pd, int vec) {
  const int SL = (32 / vec) * vec;
  return pair_smem_layout(pd.rows_max, pd.core_max, SL, sizeof(Real)).total;
}

// Draws per thread of the paired substeps for a shape kind (5, 6, 7: 4, 2, 1
// draws; FP64 takes 2 or 1), 0 for other kinds.  Their slab is always 32
// draws, so the shared memory does not depend on it.
template <typename Real>
int pair_vec_of_kind(int kind) {
  if (kind == 5) return sizeof(Real) == 4 ? 4 : 0;
  if (kind == 6) return 2;
  if (kind == 7) return 1;
  return 0;
}

template <typename Real, int PV>
void launch_pair(bool last2, dim3 grid, size_t smem, cudaStream_t st, const MeshDev<Real>& md, const PairDev& pd,
                 int S, const Real* W, const Real* cur, Real s_cur, const Real* prev, Real s_prev, const Real* g,
                 Real* o1, Real* o2, const Real* uc, Real* un, Real* d, Real a1, Real b1, Real c1, Real a2, Real b2,
                 Real c2, Real kappa) {
  if (last2)
    k_inner_pair<Real, PV, true><<<grid, 256, smem, st>>>(md, pd, S, 32 / PV, W, cur, s_cur, prev, s_prev, g, o1,
                                                          o2, uc, un, d, a1, b1, c1, a2, b2, c2, kappa);
  else
    k_inner_pair<Real, PV, false><<<grid, 256, smem, st>>>(md, pd, S, 32 / PV, W, cur, s_cur, prev, s_prev, g, o1,
                                                           o2, uc, un, d, a1, b1, c1, a2, b2, c2, kappa);
}

// One step of Alg. 2 for one batch (see kernels.cuh for the u-form): the
// coarse launch over the free nodes, then p-1 inner launches over R (or one
// fused launch for a small R).
template <typename Real, int VEC>
struct Stepper {
  lflts_ctx* c = nullptr;
  MeshDev<Real> md{};
  Geo gc{}, gi{};
  std::vector<double> beta, cm;
  double delta = 0, omega = 0, c0 = 0, gamma = 0;
  int p = 1, n_R = 0;
  int64_t S = 0;
  double Srb = 0, coarse_bytes = 0;
  const Real* W = nullptr;
  Real* g = nullptr;
  Real* rbuf[4] = {nullptr, nullptr, nullptr, nullptr};
  bool minb6 = false;
  int cps = 16;
  bool fused = false;  // all inner substeps in one launch (R in shared memory)
  int fSB = 1;
  size_t fsmem = 0;
  int fgrid = 1;
  // coarse launch forming the coupling weights from xi (k_coarse_rc), with
  // its own draws per thread, or the stored weights (k_coarse)
  bool crc = false;
  Geo gcr{};
  int KPs = 0;                  // padded field terms of the mesh
  const Real* xi_pad = nullptr;  // [S][KP] draws (set by the loop that owns the workspace)
  int pvec = 0;  // inner substeps two by two (k_inner_pair) with pvec draws per thread, or 0
  PairDev pdev{};
  size_t psmem = 0;
  int tvar = -1;       // tiled inner kernel shape (-1: not tiled)
  TileDev tdev{};
  size_t tsmem = 0;
  int tgrid = 1;
  InnerCoef<Real> coef{};
  const Real* fw = nullptr;  // M^-1 F or null
  double f0 = 0, t0 = 0, famp = 0, dt = 0;
  int64_t S_act = 0;         // draws [0, S_act) still stepping (ragged batches)
  const double* dts = nullptr;  // per-draw time steps of a ragged batch (device), or null
  const MeshGPU* mgp = nullptr;

  // r(t) of the Ricker wavelet times the amplitude
  Real source_amp(double t) const {
    if (!fw) return Real(0);
    const double a = M_PI * M_PI * f0 * f0 * (t - t0) * (t - t0);
    return (Real)(famp * (1.0 - 2.0 * a) * std::exp(-a));
  }

  Stepper(lflts_ctx* c_, const lflts_solve_desc& ds, const MeshGPU& mg, int n_R_, int64_t S_, const Real* W_,
          Real* g_, Real* r0, Real* r1, Real* r2, int shape = 16, Real* r3 = nullptr)
      : c(c_), p(ds.p), n_R(n_R_), S(S_), W(W_), g(g_), S_act(S_), mgp(&mg) {
    // shape = CTAs per SM target, +100 for the register-capped kernels,
    // +2000 for the fused inner kernel, +3000 for the tiled one, +5000 for
    // the paired substeps with 4 draws per thread (+6000: 2, +7000: 1; they
    // need the fourth r buffer r3)
    // +10000: the coarse launch forms its coupling weights (k_coarse_rc)
    crc = shape >= 10000;
    shape %= 10000;
    minb6 = (shape % 1000) >= 100;
    const int cta_per_sm = shape % 100;
    cps = cta_per_sm;
    dt = ds.dt;
    if (ds.source_id >= 0) {
      fw = Sel<Real>::fw(c->sources[ds.source_id]);
      f0 = ds.src_f0;
      t0 = ds.src_t0;
      famp = ds.src_amp;
    }
    const HostMesh& h = mg.h;
    rbuf[0] = r0;
    rbuf[1] = r1;
    rbuf[2] = r2;
    rbuf[3] = r3;
    lts_constants(p, ds.nu, ds.dt, beta, cm, delta, omega, c0, gamma);
    md = Sel<Real>::mesh(mg, n_R);
    gc = geometry_vec(c, h.n_free, S, VEC, cta_per_sm);
    KPs = h.KP;
    if (crc && (h.moving || mg.ell_hi || S % 2 != 0)) crc = false;
    if (crc) gcr = geometry_vec(c, h.n_free, S, 2, cta_per_sm);
    gi = geometry_vec(c, std::max(n_R, 1), S, VEC, cta_per_sm);
    Srb = double(S) * sizeof(Real);
    coarse_bytes = 3.0 * Srb * double(h.n_free);
    const int kind = shape / 1000;  // 0 per substep, 2 fused, 3.. tiled (shape kind - 3), 5..7 paired
    const int pv = pair_vec_of_kind<Real>(kind);
    if (pv > 0 && n_R > 0 && p > 2 && r3 && S % pv == 0) {
      auto it = mg.pairs.find(c->pair_block);
      if (it != mg.pairs.end() && it->second.ok) {
        pvec = pv;
        pdev = it->second.dev;
        psmem = pair_smem<Real>(pdev, pv);
      }
    }
    if (kind >= 3 && kind - 3 < tile_shapes<Real>() && n_R > 0 && p > 1 && p <= 64 && S % tile_shape<Real>(kind - 3).vec == 0) {
      auto it = mg.tiles.find(std::make_pair(p, tile_cap<Real>(c, kind - 3)));
      if (it != mg.tiles.end() && it->second.ok) {
        tvar = kind - 3;
        tdev = it->second.dev;
        tsmem = tile_smem<Real>(tdev, tvar);
        // work units of a tile and a run of slabs, at least two per SM
        const int64_t n_slabs = S / tile_shape<Real>(tvar).vec;
        const int64_t chunks = std::max<int64_t>(
            1, std::min<int64_t>(n_slabs, (2 * int64_t(c->sms) + tdev.n_tiles - 1) / tdev.n_tiles));
        tdev.chunk = static_cast<int>((n_slabs + chunks - 1) / chunks);
        tdev.chunks = static_cast<int>((n_slabs + tdev.chunk - 1) / tdev.chunk);
        const int64_t units = int64_t(tdev.n_tiles) * tdev.chunks;
        tgrid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(units, c->sms)));
      }
    }
    if (kind >= 2 && n_R > 0 && p > 1 && p <= 64) {
      if (kind == 2) {
        fused_plan(c, n_R, mg.n_rslots, S, VEC, sizeof(Real), fSB, fsmem);
        fused = fsmem > 0;
        const int64_t SL = int64_t(fSB) * VEC;
        fgrid = static_cast<int>((S + SL - 1) / SL);
      }
      coef.p = p;
      coef.neg_c0 = (Real)(-c0);
      for (int m = 1; m < p; ++m) {
        coef.opb[m] = (Real)(1.0 + beta[m]);
        coef.beta[m] = (Real)beta[m];
        coef.cm[m] = (Real)cm[m];
      }
    }
  }

  // Row stride of the arrays after a narrowing copy (S_act unchanged).
  void set_stride(int64_t S_new) { S = S_new; }

  // Narrow the launches to the draws [0, S_new) (a ragged batch whose other
  // draws have reached their own step count).
  void set_active(int64_t S_new) {
    S_act = S_new;
    const HostMesh& h = mgp->h;
    gc = geometry_vec(c, h.n_free, S_act, VEC, cps);
    gi = geometry_vec(c, std::max(n_R, 1), S_act, VEC, cps);
    Srb = double(S_act) * sizeof(Real);
    coarse_bytes = 3.0 * Srb * double(h.n_free);
    if (fused) {
      const int64_t SL = int64_t(fSB) * VEC;
      fgrid = static_cast<int>((S_act + SL - 1) / SL);
    }
  }

  RaggedF ragged(int64_t n) const {
    RaggedF rf{};
    if (dts && fw) {
      rf.dts = dts;
      rf.dt_ref = dt;
      rf.f0 = f0;
      rf.t0 = t0;
      rf.amp = famp;
      rf.n = static_cast<int>(n);
    }
    return rf;
  }

  // u_next = 2 T u_cur - u_prev in increments: d += kappa r_p, u_next = u_cur + d.
  // minb6: the register-capped instantiation (at least 6 CTAs of 256 per SM).
  int step(const Real* uc, Real* un, Real* d, Real kappa, cudaStream_t st, int64_t n = 0) {
    {
      Prof pr(c, st);
      const Real kg = (Real)(double(kappa) * gamma);
      const Real fa = source_amp(double(n) * dt);
      const RaggedF rf = ragged(n);
#define LF_COARSE(B, RG, HI)                                                                              \
  k_coarse<Real, VEC, B, RG, HI><<<gc.grid, 256, 0, st>>>(md, (int)S, gc.SB, W, uc, un, d, g, kg, fw, fa, (int)S_act, \
                                                          rf)
#define LF_COARSE_H(B, RG)         \
  if (md.ell_hi) LF_COARSE(B, RG, true); \
  else LF_COARSE(B, RG, false)
      if (crc && !dts && xi_pad) {  // weights formed in the kernel (2 draws per thread)
        const MeshGPU& mg = *mgp;
        if (KPs == 4)
          k_coarse_rc<Real, 2, 4><<<gcr.grid, 256, 0, st>>>(md, (int)S, gcr.SB, mg.ee, Sel<Real>::eg(mg),
                                                            Sel<Real>::psi(mg), xi_pad, uc, un, d, g, kg, fw, fa);
        else if (KPs == 8)
          k_coarse_rc<Real, 2, 8><<<gcr.grid, 256, 0, st>>>(md, (int)S, gcr.SB, mg.ee, Sel<Real>::eg(mg),
                                                            Sel<Real>::psi(mg), xi_pad, uc, un, d, g, kg, fw, fa);
        else
          k_coarse_rc<Real, 2, 16><<<gcr.grid, 256, 0, st>>>(md, (int)S, gcr.SB, mg.ee, Sel<Real>::eg(mg),
                                                             Sel<Real>::psi(mg), xi_pad, uc, un, d, g, kg, fw, fa);
      } else if (dts) {  // ragged batch (bounded to 64 registers: four CTAs of 256 per SM)
        if (minb6) LF_COARSE_H(6, true);
        else LF_COARSE_H(4, true);
      } else {
        if (minb6) LF_COARSE_H(6, false);
        else LF_COARSE_H(1, false);
      }
#undef LF_COARSE_H
#undef LF_COARSE
      LF_CUDA(c, cudaGetLastError());
      pr.end(LFLTS_KERNEL_COARSE, coarse_bytes);
    }
    if (n_R > 0 && tvar >= 0 && !dts) {
      Prof pr(c, st);
      tile_call<Real>(tvar, p, false, 0, tgrid, tsmem, st, tdev, (int)S, W, g, uc, un, d, coef, kappa);
      LF_CUDA(c, cudaGetLastError());
      // all substeps on chip: the outer-step bytes of R remain
      pr.end(LFLTS_KERNEL_INNER, 3.0 * n_R * Srb);
      return 0;
    }
    if (n_R > 0 && fused) {
      Prof pr(c, st);
      const int ns = static_cast<int>(mgp->n_rslots);
      if (dts)
        k_inner_fused<Real, VEC, true><<<fgrid, 256, fsmem, st>>>(md, (int)S, fSB, W, g, uc, un, d, coef, kappa,
                                                                  (int)S_act, mgp->rptr, mgp->rslot, ns);
      else
        k_inner_fused<Real, VEC, false><<<fgrid, 256, fsmem, st>>>(md, (int)S, fSB, W, g, uc, un, d, coef, kappa,
                                                                   (int)S_act, mgp->rptr, mgp->rslot, ns);
      LF_CUDA(c, cudaGetLastError());
      // all substeps on chip: the outer-step bytes of R remain
      pr.end(LFLTS_KERNEL_INNER, 3.0 * n_R * Srb);
      return 0;
    }
    if (n_R > 0) {
      // r_1 = -c0 g is read from g; r_2.. rotate through the r buffers (a
      // launch never writes a buffer it reads)
      const Real* cur = g;
      Real s_cur = (Real)(-c0);
      const Real* prev = nullptr;
      Real s_prev = Real(0);
      auto pick = [&](const Real* x) -> Real* {
        for (Real* r : rbuf)
          if (r && r != cur && r != prev && r != x) return r;
        return nullptr;
      };
      for (int m = 1; m < p;) {
        // substeps m and m + 1 in one launch; with an odd number of substeps
        // the first (which reads only g) runs alone, so that a pair ends the
        // step
        if (pvec > 0 && !dts && m + 1 < p && (p - m) % 2 == 0) {
          const bool last2 = (m + 1 == p - 1);
          Real* o1 = last2 ? nullptr : pick(nullptr);
          Real* o2 = last2 ? nullptr : pick(o1);
          Prof pr(c, st);
          const dim3 grid(static_cast<unsigned>(pdev.n_blocks), static_cast<unsigned>((S + 31) / 32));
          const Real a1 = (Real)(1.0 + beta[m]), b1 = (Real)beta[m], c1 = (Real)cm[m];
          const Real a2 = (Real)(1.0 + beta[m + 1]), b2 = (Real)beta[m + 1], c2 = (Real)cm[m + 1];
          if constexpr (sizeof(Real) == 4) {
            if (pvec == 4)
              launch_pair<Real, 4>(last2, grid, psmem, st, md, pdev, (int)S, W, cur, s_cur, prev, s_prev, g, o1, o2,
                                   uc, un, d, a1, b1, c1, a2, b2, c2, kappa);
          }
          if (pvec == 2)
            launch_pair<Real, 2>(last2, grid, psmem, st, md, pdev, (int)S, W, cur, s_cur, prev, s_prev, g, o1, o2, uc,
                                 un, d, a1, b1, c1, a2, b2, c2, kappa);
          else if (pvec == 1)
            launch_pair<Real, 1>(last2, grid, psmem, st, md, pdev, (int)S, W, cur, s_cur, prev, s_prev, g, o1, o2, uc,
                                 un, d, a1, b1, c1, a2, b2, c2, kappa);
          LF_CUDA(c, cudaGetLastError());
          // per R node r_m, r_{m-1}, g read and r_{m+1}, r_{m+2} written (the
          // pair that ends the step: u, d read and d, u written instead of
          // r_{m+1}, r_{m+2})
          pr.end(LFLTS_KERNEL_INNER_PAIR, (last2 ? 7.0 : 5.0) * n_R * Srb);
          if (!last2) {
            prev = o1;
            s_prev = Real(1);
            cur = o2;
            s_cur = Real(1);
          }
          m += 2;
          continue;
        }
        const bool last = (m == p - 1);
        const Real opb = (Real)(1.0 + beta[m]), bt = (Real)beta[m], cmm = (Real)cm[m];
        Real* rn = pick(nullptr);
        Prof pr(c, st);
#define LF_INNER(L, B, RG)                                                                                     \
  k_inner<Real, VEC, L, B, RG><<<gi.grid, 256, 0, st>>>(md, (int)S, gi.SB, W, cur, s_cur, prev, s_prev, rn, \
                                                               g, uc, un, d, opb, bt, cmm, kappa, (int)S_act)
        if (dts) {  // ragged batch: only the last substep writes u and d
          if (last) LF_INNER(true, 1, true);
          else LF_INNER(false, 1, false);
        } else if (last) {
          if (minb6) LF_INNER(true, 6, false);
          else LF_INNER(true, 1, false);
        } else {
          if (minb6) LF_INNER(false, 6, false);
          else LF_INNER(false, 1, false);
        }
#undef LF_INNER
        LF_CUDA(c, cudaGetLastError());
        // per R node r_m, r_{m-1} and g read, r_{m+1} written
        pr.end(LFLTS_KERNEL_INNER, 4.0 * n_R * Srb);
        prev = cur;
        s_prev = s_cur;
        cur = rn;
        s_cur = Real(1);
        ++m;
      }
    }
    return 0;
  }
};

// A few steps of Alg. 2 for one batch with a given launch shape (the
// autotuner's timing runs; solves run through SlicedLoop).
template <typename Real, int VEC>
int time_loop(lflts_ctx* c, const lflts_solve_desc& ds, const MeshGPU& mg, int n_R, int64_t S,
              Workspace& ws, Real*& uc_out, cudaStream_t st, int cta_per_sm = 16, int64_t n_steps = -1,
              const double* dts = nullptr) {
  Stepper<Real, VEC> stp(c, ds, mg, n_R, S, static_cast<const Real*>(ws.W.p), static_cast<Real*>(ws.g.p),
                         static_cast<Real*>(ws.r0.p), static_cast<Real*>(ws.r1.p), static_cast<Real*>(ws.r2.p),
                         cta_per_sm, static_cast<Real*>(ws.r3.p));
  stp.dts = dts;  // a ragged batch: its kernels (all draws active)
  stp.xi_pad = static_cast<const Real*>(ws.xipad.p);
  Real* uc = static_cast<Real*>(ws.ua.p);
  Real* un = static_cast<Real*>(ws.ub.p);
  Real* d = static_cast<Real*>(ws.d.p);
  const int64_t N = n_steps >= 0 ? n_steps : ds.n_steps;
  for (int64_t n = 0; n < N; ++n) {
    LF_TRY(stp.step(uc, un, d, (n == 0) ? Real(1) : Real(2), st, n));
    std::swap(uc, un);
  }
  uc_out = uc;
  return 0;
}

template <typename Real>
int time_loop_vec(lflts_ctx* c, const lflts_solve_desc& ds, const MeshGPU& mg, int n_R, int64_t S, Workspace& ws,
                  Real*& uc, cudaStream_t st, int vec, int cps, int64_t n_steps = -1,
                  const double* dts = nullptr) {
  if (vec == 4) return time_loop<Real, 4>(c, ds, mg, n_R, S, ws, uc, st, cps, n_steps, dts);
  if (vec == 2) return time_loop<Real, 2>(c, ds, mg, n_R, S, ws, uc, st, cps, n_steps, dts);
  return time_loop<Real, 1>(c, ds, mg, n_R, S, ws, uc, st, cps, n_steps, dts);
}

// Whether the fused inner kernel can run this batch; raises its dynamic
// shared-memory limit once it can (outside any graph capture).
template <typename Real>
bool fused_ok(lflts_ctx* c, MeshGPU& mg, int n_R, int64_t S, int vec, int p) {
  if (n_R < 1 || p < 2 || p > 64) return false;
  if (mg.n_rslots < 0) {  // coupling slots of R, built and uploaded once per mesh
    std::vector<int32_t> ptr, sj, se;
    build_r_slots(mg.h, ptr, sj, se);
    if (int64_t(sj.size()) > (int64_t(1) << 24)) return false;
    std::vector<int2> sl(sj.size());
    for (size_t t = 0; t < sj.size(); ++t) sl[t] = make_int2(sj[t], se[t]);
    if (upload(c, &mg.rptr, ptr.data(), ptr.size())) return false;
    if (upload(c, &mg.rslot, sl.data(), sl.size())) return false;
    mg.n_rslots = static_cast<int64_t>(sj.size());
  }
  int SBf = 1;
  size_t smem = 0;
  fused_plan(c, n_R, mg.n_rslots, S, vec, sizeof(Real), SBf, smem);
  if (smem == 0) return false;
  cudaError_t e = cudaSuccess;
  const int mx = int(kFusedSmemMax);
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (vec == 4) {
    e = cudaFuncSetAttribute(k_inner_fused<Real, 4, false>, attr, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inner_fused<Real, 4, true>, attr, mx);
  } else if (vec == 2) {
    e = cudaFuncSetAttribute(k_inner_fused<Real, 2, false>, attr, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inner_fused<Real, 2, true>, attr, mx);
  } else {
    e = cudaFuncSetAttribute(k_inner_fused<Real, 1, false>, attr, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inner_fused<Real, 1, true>, attr, mx);
  }
  return e == cudaSuccess;
}

// Whether the tiled inner kernel of shape `var` can run this batch: builds
// and uploads the mesh's tile plan for (p, capacity) once and raises the
// kernel's dynamic shared-memory limit (outside any graph capture).
template <typename Real>
bool tile_ok(lflts_ctx* c, MeshGPU& mg, int n_R, int64_t S, int p, int var) {
  if (n_R < 1 || p < 2 || p > 64 || var < 0 || var >= tile_shapes<Real>()) return false;
  if (S % tile_shape<Real>(var).vec != 0) return false;
  const auto key = std::make_pair(p, tile_cap<Real>(c, var));
  auto it = mg.tiles.find(key);
  if (it == mg.tiles.end()) {
    MeshGPU::DevTiles dt;
    TilePlan tp;
    if (build_tile_plan(mg.h, p, key.second, tp)) {
      int* d_ptr = nullptr;
      int* d_len = nullptr;
      int* d_node = nullptr;
      int* d_sj = nullptr;
      int* d_se = nullptr;
      int* d_xp = nullptr;
      int* d_xs = nullptr;
      float* d_m32 = nullptr;
      double* d_m64 = nullptr;
      const std::vector<float> m32(tp.minv.begin(), tp.minv.end());
      const bool up = !upload(c, &d_m32, m32.data(), m32.size()) && !upload(c, &d_m64, tp.minv.data(), tp.minv.size()) &&
                      !upload(c, &d_ptr, tp.ptr.data(), tp.ptr.size()) &&
                      !upload(c, &d_len, tp.len.data(), tp.len.size()) &&
                      !upload(c, &d_node, tp.node.data(), tp.node.size()) &&
                      !upload(c, &d_sj, tp.sj.data(), tp.sj.size()) &&
                      !upload(c, &d_se, tp.se.data(), tp.se.size()) &&
                      !upload(c, &d_xp, tp.xp.data(), tp.xp.size()) &&
                      !upload(c, &d_xs, tp.xs.data(), tp.xs.size());
      if (up) {
        dt.dev.ptr = d_ptr;
        dt.dev.len = d_len;
        dt.dev.node = d_node;
        dt.dev.sj = reinterpret_cast<const int2*>(d_sj);
        dt.dev.se = reinterpret_cast<const int4*>(d_se);
        dt.dev.xp = d_xp;
        dt.dev.xs = reinterpret_cast<const int2*>(d_xs);
        dt.dev.minv32 = d_m32;
        dt.dev.minv64 = d_m64;
        dt.dev.n_tiles = static_cast<int>(tp.ptr.size()) - 1;
        dt.dev.n_all_max = static_cast<int>(tp.n_all_max);
        int comp_max = 0, core_max = 0;
        for (int t = 0; t < dt.dev.n_tiles; ++t) {
          comp_max = std::max(comp_max, tp.len[size_t(t) * p + p - 2]);
          core_max = std::max(core_max, tp.len[size_t(t) * p]);
        }
        dt.dev.comp_max = comp_max;
        dt.dev.core_max = core_max;
        // each tile's range of slots beyond the fourth: the plan appends them
        // tile after tile, node after node, so the ranges are consecutive
        std::vector<int32_t> xptr(size_t(dt.dev.n_tiles) + 1, 0);
        int xs_max = 0;
        for (int t = 0; t < dt.dev.n_tiles; ++t) {
          int32_t n = 0;
          for (int32_t a = tp.ptr[t]; a < tp.ptr[t + 1]; ++a) {
            const int32_t k = (tp.xp[a] >> 1) & 15;
            if (k && (tp.xp[a] >> 5) != xptr[t] + n) dt.ok = false;  // not consecutive: no tiled kernel
            n += k;
          }
          xptr[t + 1] = xptr[t] + n;
          xs_max = std::max(xs_max, int(n));
        }
        int* d_xptr = nullptr;
        if (upload(c, &d_xptr, xptr.data(), xptr.size())) dt.ok = false;
        dt.dev.xptr = d_xptr;
        dt.dev.xs_max = xs_max;
        dt.ok = true;
      }
    }
    it = mg.tiles.emplace(key, dt).first;
  }
  if (!it->second.ok) return false;
  const size_t smem = tile_smem<Real>(it->second.dev, var);
  if (smem > kTileSmemMax) return false;
  const InnerCoef<Real> k0{};
  return tile_call<Real>(var, p, true, static_cast<int>(kTileSmemMax), 0, 0, nullptr, it->second.dev, 0, nullptr,
                         nullptr, nullptr, nullptr, nullptr, k0, Real(0)) == cudaSuccess;
}

// Draw segments of a ragged batch: draws [off, off + cnt) take n_steps steps
// of dt.  Segments are sorted by n_steps, descending, so that the draws still
// stepping always form a prefix of the batch.  A uniform batch is one segment.
struct RaggedSeg {
  int64_t off, cnt, n_steps;
  double dt;
};
struct RaggedSpec {
  std::vector<RaggedSeg> segs;
  const double* d_dts = nullptr;  // [S] time step of every draw
  const void* d_sig = nullptr;    // [S] (dt_s / dt_ref)^2 in the batch precision
  uint64_t hash = 0;              // of the segment list (graph key)
};

// The time loop of one batch, queued in slices of outer steps.  lflts_run_pairs
// uses the slices to keep several long solves (too long for one graph) on
// their streams at once: a single host thread that queued one solve's whole
// loop would block on that stream's launch queue while the others ran dry.
// When a segment of a ragged batch reaches its step count its QoI is taken
// and the launches narrow to the draws still stepping.
struct SliceTask {
  virtual ~SliceTask() = default;
  virtual int advance(int64_t steps) = 0;  // queue up to `steps` more outer steps
  virtual bool done() const = 0;
  virtual int64_t position() const = 0;    // outer steps queued so far
  virtual int finish() = 0;                // queue the QoI of the last segments
};

template <typename Real>
struct LoopOut {  // what the loop does with finished draws
  std::function<int(const Real* u, int64_t stride, int64_t s_lo, int64_t s_hi)> qoi_range;
  std::function<int()> qoi_final;
  bool restride = false;  // the loop may narrow the row stride (no state gather)
};

template <typename Real, int VEC>
struct SlicedLoop : SliceTask {
  lflts_ctx* c;
  Stepper<Real, VEC> stp;
  Real* uc;
  Real* un;
  Real* d;
  int64_t n = 0, N;
  cudaStream_t st;
  std::vector<RaggedSeg> segs;
  size_t active;  // segments 0 .. active-1 still step
  LoopOut<Real> out;
  Workspace* wsp;
  int64_t S_cur;   // row stride of the arrays
  int64_t n_w;     // rows of W
  SlicedLoop(lflts_ctx* c_, const lflts_solve_desc& ds, const MeshGPU& mg, int n_R, int64_t S, Workspace& ws,
             cudaStream_t st_, int cps, const RaggedSpec* rg, LoopOut<Real> o)
      : c(c_),
        stp(c_, ds, mg, n_R, S, static_cast<const Real*>(ws.W.p), static_cast<Real*>(ws.g.p),
            static_cast<Real*>(ws.r0.p), static_cast<Real*>(ws.r1.p), static_cast<Real*>(ws.r2.p), cps,
            static_cast<Real*>(ws.r3.p)),
        uc(static_cast<Real*>(ws.ua.p)),
        un(static_cast<Real*>(ws.ub.p)),
        d(static_cast<Real*>(ws.d.p)),
        N(ds.n_steps),
        st(st_),
        out(std::move(o)),
        wsp(&ws),
        S_cur(S),
        n_w(mg.h.n_w) {
    stp.xi_pad = static_cast<const Real*>(ws.xipad.p);
    if (rg) {
      segs = rg->segs;
      stp.dts = rg->d_dts;
    } else {
      segs.push_back({0, S, ds.n_steps, ds.dt});
    }
    active = segs.size();
  }
  // QoI of the segments that have taken all their steps (at step n)
  int freeze() {
    bool narrowed = false;
    while (active > 0 && segs[active - 1].n_steps <= n) {
      const RaggedSeg& sg = segs[active - 1];
      LF_TRY(out.qoi_range(uc, S_cur, sg.off, sg.off + sg.cnt));
      --active;
      narrowed = true;
    }
    if (narrowed && active > 0) {
      const int64_t S_act = segs[active - 1].off + segs[active - 1].cnt;
      stp.set_active(S_act);
      const int64_t S_new = (S_act + 7) / 8 * 8;  // 32-byte rows at least (one DRAM sector in FP32)
      if (out.restride && 2 * S_new <= S_cur) LF_TRY(narrow(S_new));
    }
    return 0;
  }
  // Copy u_n, d and W to rows of stride S_new (through the scratch buffer),
  // and u_n again into u_next: a step writes u_next only on free nodes, so its
  // Dirichlet rows must already hold their values at the new stride.  g and
  // the r buffers are written before they are read again.
  int narrow(int64_t S_new) {
    const int64_t n_nodes = stp.mgp->h.n_nodes;
    Real* tmp = static_cast<Real*>(wsp->cmp.p);
    auto one = [&](Real* a, int64_t rows) -> int {
      const int64_t n = rows * S_new;
      k_restride<Real><<<blocks_for(n, 256, c->sms * 32), 256, 0, st>>>(a, tmp, rows, (int)S_cur, (int)S_new);
      LF_CUDA(c, cudaGetLastError());
      c->launches++;
      LF_CUDA(c, cudaMemcpyAsync(a, tmp, size_t(n) * sizeof(Real), cudaMemcpyDeviceToDevice, st));
      return 0;
    };
    LF_TRY(one(uc, n_nodes));
    LF_CUDA(c, cudaMemcpyAsync(un, uc, size_t(n_nodes * S_new) * sizeof(Real), cudaMemcpyDeviceToDevice, st));
    LF_TRY(one(d, n_nodes));
    LF_TRY(one(static_cast<Real*>(wsp->W.p), std::max<int64_t>(n_w, 1)));
    S_cur = S_new;
    stp.set_stride(S_new);
    return 0;
  }
  int advance(int64_t steps) override {
    for (int64_t k = 0; k < steps && n < N; ++k, ++n) {
      LF_TRY(freeze());
      LF_TRY(stp.step(uc, un, d, (n == 0) ? Real(1) : Real(2), st, n));
      std::swap(uc, un);
    }
    return 0;
  }
  bool done() const override { return n >= N; }
  int64_t position() const override { return n; }
  int finish() override {
    LF_TRY(freeze());
    return out.qoi_final();
  }
};

template <typename Real>
std::unique_ptr<SliceTask> make_sliced(lflts_ctx* c, const lflts_solve_desc& ds, const MeshGPU& mg, int n_R,
                                       int64_t S, Workspace& ws, cudaStream_t st, int vec, int cps,
                                       const RaggedSpec* rg, LoopOut<Real> o) {
  if (vec == 4)
    return std::make_unique<SlicedLoop<Real, 4>>(c, ds, mg, n_R, S, ws, st, cps, rg, std::move(o));
  if (vec == 2)
    return std::make_unique<SlicedLoop<Real, 2>>(c, ds, mg, n_R, S, ws, st, cps, rg, std::move(o));
  return std::make_unique<SlicedLoop<Real, 1>>(c, ds, mg, n_R, S, ws, st, cps, rg, std::move(o));
}

// Launch shape of the step kernels for a batch: draws per thread (vec),
// CTAs per SM and the register cap.  Shape code cps: CTAs per SM, +100 for
// the instantiation limited to 40 registers (6 CTAs of 256 per SM), +2000
// for the fused inner kernel.  With autotuning on, the first solve of a (mesh, S, precision, p)
// times every candidate over a few steps on the real buffers (the state is
// re-initialised afterwards) and keeps the fastest.
// Whether the paired inner substeps can run this batch: builds and uploads
// the mesh's block plan once and raises the kernels' dynamic shared-memory
// limit (outside any graph capture).
template <typename Real>
bool pair_ok(lflts_ctx* c, MeshGPU& mg, int n_R, int64_t S, int p) {
  if (n_R < 1 || p < 3 || p > 128 || S < 1) return false;
  auto it = mg.pairs.find(c->pair_block);
  if (it == mg.pairs.end()) {
    MeshGPU::DevPairs dp;
    PairPlan pl;
    if (build_pair_plan(mg.h, c->pair_block, pl) && pl.n_blocks <= INT32_MAX) {
      int* d_rptr = nullptr;
      int* d_ncore = nullptr;
      int* d_row = nullptr;
      int16_t* d_lidx = nullptr;
      const bool up = !upload(c, &d_rptr, pl.rptr.data(), pl.rptr.size()) &&
                      !upload(c, &d_ncore, pl.ncore.data(), pl.ncore.size()) &&
                      !upload(c, &d_row, pl.row.data(), pl.row.size()) &&
                      !upload(c, &d_lidx, pl.lidx.data(), pl.lidx.size());
      if (up) {
        dp.dev.n_blocks = static_cast<int>(pl.n_blocks);
        dp.dev.rows_max = static_cast<int>(pl.rows_max);
        dp.dev.core_max = static_cast<int>(pl.core_max);
        dp.dev.rptr = d_rptr;
        dp.dev.ncore = d_ncore;
        dp.dev.row = d_row;
        dp.dev.lidx = reinterpret_cast<const short*>(d_lidx);
        dp.ok = true;
      }
    }
    it = mg.pairs.emplace(c->pair_block, dp).first;
  }
  if (!it->second.ok) return false;
  const size_t smem = pair_smem<Real>(it->second.dev, 1);  // the same for every draws-per-thread
  if (smem > kTileSmemMax) return false;
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaSuccess;
  if constexpr (sizeof(Real) == 4) {
    e = cudaFuncSetAttribute(k_inner_pair<Real, 4, false>, attr, int(smem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inner_pair<Real, 4, true>, attr, int(smem));
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inner_pair<Real, 2, false>, attr, int(smem));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inner_pair<Real, 2, true>, attr, int(smem));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inner_pair<Real, 1, false>, attr, int(smem));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inner_pair<Real, 1, true>, attr, int(smem));
  return e == cudaSuccess;
}

template <typename Real>
int launch_shape_base(lflts_ctx* c, const lflts_solve_desc& ds, MeshGPU& mg, int n_R, int64_t S, Workspace& ws,
                      cudaStream_t st, int& vec, int& cps, const double* dts) {
  const int vmax = (sizeof(Real) == 4) ? 4 : 2;
  std::vector<int> vecs;
  for (int v = vmax; v >= 1; v /= 2)
    if (S % v == 0) vecs.push_back(v);
  vec = vecs.front();
  cps = 16;
  if (c->pair_mode >= 2 && !dts && n_R >= c->pair_min_r && pair_ok<Real>(c, mg, n_R, S, ds.p)) {
    // 2: 4 draws per thread in FP32, 2 in FP64; 3: 2; 4: 1
    const int kind = c->pair_mode == 2 ? (sizeof(Real) == 4 ? 5 : 6) : c->pair_mode + 3;
    if (S % pair_vec_of_kind<Real>(kind) == 0) {
      cps = 1000 * kind + 16;
      return 0;
    }
  }
  if (c->tile_mode >= 2 && !dts && tile_ok<Real>(c, mg, n_R, S, ds.p, c->tile_mode - 2)) {
    cps = 3016 + 1000 * (c->tile_mode - 2);
    return 0;
  }
  if (c->fused_mode == 2 && fused_ok<Real>(c, mg, n_R, S, vec, ds.p)) {
    cps = 2016;
    return 0;
  }
  if (!c->autotune) return 0;
  const auto key = std::make_tuple(S, ds.precision, ds.p);
  auto it = mg.tuned.find(key);
  if (it != mg.tuned.end()) {
    vec = it->second.first;
    cps = it->second.second;
    return 0;
  }
  cudaEvent_t e0, e1;
  LF_CUDA(c, cudaEventCreate(&e0));
  LF_CUDA(c, cudaEventCreate(&e1));
  const bool prof = c->profiling;
  c->profiling = false;
  const int64_t launches0 = c->launches;
  float best = 1e30f;
  const int64_t steps = std::min<int64_t>(4, ds.n_steps);
  for (int v : vecs) {
    // one draw per thread is timed only for a small R (the fused kernel then
    // gets four times as many CTAs for a small batch)
    if (vecs.size() > 2 && v == 1 && !(n_R >= 1 && n_R <= 2048 && c->fused_mode >= 1)) continue;
    // The fused inner kernel is a candidate where R fits in shared memory.
    // For a small R (at most 2048 nodes) the fused kernel replaces p-1
    // launches of a few microseconds each; a four-step timing does not tell
    // the two apart reliably there, so only the fused shapes are timed.
    std::vector<int> shapes = {8, 16, 32, 108, 116, 132};
    if (c->fused_mode >= 1 && fused_ok<Real>(c, mg, n_R, S, v, ds.p)) {
      if (n_R <= 2048) shapes.clear();
      for (int k : {8, 16, 32, 108, 116, 132}) shapes.push_back(2000 + k);
    }
    // substeps two by two for a large R, with their own draws per thread (4
    // in FP32, 2 in FP64: fewer were slower on every benchmark level), so
    // timed with the first v only
    if (c->pair_mode == 1 && !dts && n_R > 2048 && v == vecs.front() && pair_ok<Real>(c, mg, n_R, S, ds.p)) {
      const int kind = sizeof(Real) == 4 ? 5 : 6;
      if (S % pair_vec_of_kind<Real>(kind) == 0)
        for (int k : {8, 16, 32, 108, 116, 132}) shapes.push_back(1000 * kind + k);
    }
    // the tiled inner kernel (all substeps on chip) for a large R; its own
    // draws per node do not depend on v, so it is timed with the first v only
    if (c->tile_mode == 1 && !dts && n_R > 2048 && v == vecs.front())
      for (int var = 0; var < tile_shapes<Real>(); ++var)
        if (tile_ok<Real>(c, mg, n_R, S, ds.p, var))
          for (int k : {8, 16, 32, 108, 116, 132}) shapes.push_back(3000 + 1000 * var + k);
    for (int k : shapes) {
      Real* uc = nullptr;
      int rc = time_loop_vec<Real>(c, ds, mg, n_R, S, ws, uc, st, v, k, 1, dts);  // warm
      if (!rc) rc = cudaEventRecord(e0, st) == cudaSuccess ? 0 : LFLTS_ERR_CUDA;
      if (!rc) rc = time_loop_vec<Real>(c, ds, mg, n_R, S, ws, uc, st, v, k, steps, dts);
      if (!rc) rc = cudaEventRecord(e1, st) == cudaSuccess ? 0 : LFLTS_ERR_CUDA;
      if (!rc) rc = cudaEventSynchronize(e1) == cudaSuccess ? 0 : LFLTS_ERR_CUDA;
      float ms = 0.f;
      if (!rc) cudaEventElapsedTime(&ms, e0, e1);
      if (rc) {
        c->profiling = prof;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc;
      }
      if (ms < best) {
        best = ms;
        vec = v;
        cps = k;
      }
    }
  }
  c->tune_launches += c->launches - launches0;
  c->launches = launches0;  // tuning launches are reported separately
  c->profiling = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  mg.tuned[key] = std::make_pair(vec, cps);
  return 0;
}

// Launch shape of a solve: draws per thread and shape code (launch_shape_base),
// then whether the coarse launch forms its coupling weights in the kernel
// (+10000, k_coarse_rc): always with LFLTS_OPT_COARSE_RC = 2, timed against
// the stored weights once per (S, precision, p) with 1.
template <typename Real>
int launch_shape(lflts_ctx* c, const lflts_solve_desc& ds, MeshGPU& mg, int n_R, int64_t S, Workspace& ws,
                 cudaStream_t st, int& vec, int& cps, const double* dts) {
  LF_TRY(launch_shape_base<Real>(c, ds, mg, n_R, S, ws, st, vec, cps, dts));
  const bool eligible = c->coarse_rc > 0 && !dts && !mg.h.moving && !mg.ell_hi && S % 2 == 0 && cps < 10000;
  if (!eligible) return 0;
  if (c->coarse_rc == 2) {
    cps += 10000;
    return 0;
  }
  if (!c->autotune) return 0;
  const auto key = std::make_tuple(S, ds.precision, ds.p);
  auto it = mg.tuned_rc.find(key);
  if (it == mg.tuned_rc.end()) {
    cudaEvent_t e0, e1;
    LF_CUDA(c, cudaEventCreate(&e0));
    LF_CUDA(c, cudaEventCreate(&e1));
    const bool prof = c->profiling;
    c->profiling = false;
    const int64_t launches0 = c->launches;
    const int64_t steps = std::min<int64_t>(4, ds.n_steps);
    float t[2] = {0.f, 0.f};
    int rc = 0;
    for (int a = 0; a < 2 && !rc; ++a) {
      Real* uc = nullptr;
      const int k = cps + 10000 * a;
      rc = time_loop_vec<Real>(c, ds, mg, n_R, S, ws, uc, st, vec, k, 1, dts);  // warm
      if (!rc) rc = cudaEventRecord(e0, st) == cudaSuccess ? 0 : LFLTS_ERR_CUDA;
      if (!rc) rc = time_loop_vec<Real>(c, ds, mg, n_R, S, ws, uc, st, vec, k, steps, dts);
      if (!rc) rc = cudaEventRecord(e1, st) == cudaSuccess ? 0 : LFLTS_ERR_CUDA;
      if (!rc) rc = cudaEventSynchronize(e1) == cudaSuccess ? 0 : LFLTS_ERR_CUDA;
      if (!rc) cudaEventElapsedTime(&t[a], e0, e1);
    }
    c->tune_launches += c->launches - launches0;
    c->launches = launches0;
    c->profiling = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    it = mg.tuned_rc.emplace(key, t[1] < t[0]).first;
  }
  if (it->second) cps += 10000;
  return 0;
}

template <typename Real, int KP>
int run_solve_kp(lflts_ctx* c, const lflts_solve_desc& ds, MeshGPU& mg, const Qoi& q,
                 const Field& u0, const Field* v0, const double* d_xi, int64_t S, double* d_Q,
                 double* d_uN, Workspace& ws, cudaStream_t st, std::unique_ptr<SliceTask>* defer,
                 const RaggedSpec* rg, bool allow_graph) {
  const HostMesh& h = mg.h;
  const size_t rb = sizeof(Real);
  const int64_t n_nodes = h.n_nodes;
  const int p = ds.p;
  const int n_R = (p > 1) ? static_cast<int>(h.n_R) : 0;
  const size_t state_bytes = size_t(n_nodes) * S * rb;
  const size_t r_bytes = size_t(std::max(n_R, 1)) * S * rb;
  const int chunk = 512;
  const int n_chunks = std::max(1, (q.nnz + chunk - 1) / chunk);
  // every buffer is sized before the first launch (no allocation during graph capture)
  LF_TRY(ensure(c, ws.ua, state_bytes));
  LF_TRY(ensure(c, ws.ub, state_bytes));
  LF_TRY(ensure(c, ws.d, state_bytes));
  LF_TRY(ensure(c, ws.g, r_bytes));
  LF_TRY(ensure(c, ws.r0, r_bytes));
  LF_TRY(ensure(c, ws.r1, r_bytes));
  LF_TRY(ensure(c, ws.r2, r_bytes));
  LF_TRY(ensure(c, ws.r3, r_bytes));
  LF_TRY(ensure(c, ws.W, size_t(std::max<int64_t>(h.n_w, 1)) * S * rb));
  LF_TRY(ensure(c, ws.xipad, size_t(S) * KP * rb));
  LF_TRY(ensure(c, ws.qps, size_t(n_chunks) * S * sizeof(double)));
  LF_TRY(ensure(c, ws.qpc, size_t(n_chunks) * S * sizeof(double)));
  if (rg && rg->segs.size() > 1 && !d_uN)  // a narrowing copy keeps at most half the stride
    LF_TRY(ensure(c, ws.cmp, size_t(std::max<int64_t>(n_nodes, std::max<int64_t>(h.n_w, 1))) * ((S + 1) / 2 + 8) * rb));
  Real* ua = static_cast<Real*>(ws.ua.p);
  Real* ub = static_cast<Real*>(ws.ub.p);
  Real* d = static_cast<Real*>(ws.d.p);
  Real* xi = static_cast<Real*>(ws.xipad.p);
  Real* W = static_cast<Real*>(ws.W.p);

  auto a1 = [&]() -> int {  // a1: draws, initial state, per-sample edge weights of K(w)
    Prof pr(c, st);
    k_xi_pad<Real, KP><<<blocks_for(S * KP, 256, 4096), 256, 0, st>>>((int)S, h.K, d_xi, xi);
    LF_CUDA(c, cudaGetLastError());
    k_init_state<Real><<<blocks_for(n_nodes * S, 256, c->sms * 32), 256, 0, st>>>(
        n_nodes, (int)S, Sel<Real>::field(u0), v0 ? Sel<Real>::field(*v0) : nullptr, (Real)ds.dt, ua, ub, d,
        rg ? rg->d_dts : nullptr);
    LF_CUDA(c, cudaGetLastError());
    if (h.moving) {  // stiffness and lumped mass of every draw's moved mesh
      const Geo ge = geometry(c, std::max<int64_t>(h.n_free, 1), S);
      k_moving_weights<Real><<<ge.grid, 256, 0, st>>>(mg.moving(), (int)S, ge.SB, d_xi, W,
                                                       rg ? static_cast<const Real*>(rg->d_sig) : nullptr);
    } else {
      const Geo ge = geometry(c, std::max<int64_t>(h.n_edges, 1), S);
      k_edge_weights<Real, KP><<<ge.grid, 256, 0, st>>>(h.n_edges, (int)S, ge.SB, mg.ee, Sel<Real>::eg(mg),
                                                        Sel<Real>::psi(mg), xi, W,
                                                        rg ? static_cast<const Real*>(rg->d_sig) : nullptr);
    }
    LF_CUDA(c, cudaGetLastError());
    pr.end(LFLTS_KERNEL_INIT, double(S) * rb * 3.0 * n_nodes);  // u (twice) and d written
    c->launches += 2;  // three kernels in this class
    return 0;
  };

  int vec = 1, cps = 16;
  if (c->autotune && !mg.tuned.count(std::make_tuple(S, ds.precision, ds.p))) {
    const int64_t l0 = c->launches;
    const bool prof = c->profiling;
    c->profiling = false;
    const int rc = a1();  // edge weights and a valid state for the timing runs
    c->profiling = prof;
    LF_TRY(rc);
    LF_TRY(launch_shape<Real>(c, ds, mg, n_R, S, ws, st, vec, cps, rg ? rg->d_dts : nullptr));
    c->tune_launches += c->launches - l0;
    c->launches = l0;
  } else {
    LF_TRY(launch_shape<Real>(c, ds, mg, n_R, S, ws, st, vec, cps, rg ? rg->d_dts : nullptr));
  }

  // QoI at each draw's final step (Sec. 2.1; FP64 compensated sums), stage 1
  // per finished draw range, stage 2 once; optional gather of u_N.  Captured
  // by value: a sliced solve runs them later.
  const Qoi* qp = &q;
  Workspace* wsp = &ws;
  const int* new2old = mg.new2old;
  int* d_bad = c->d_bad;
  LoopOut<Real> lo;
  lo.restride = rg && rg->segs.size() > 1 && !d_uN;
  lo.qoi_range = [=](const Real* uc, int64_t stride, int64_t s_lo, int64_t s_hi) -> int {
    const int64_t w = s_hi - s_lo;
    const int tb = static_cast<int>(std::min<int64_t>(w, 128));
    Prof pr(c, st);
    const dim3 qg(n_chunks, static_cast<unsigned>((w + tb - 1) / tb));
    if (stride == S)
      k_qoi_partial<Real><<<qg, tb, 0, st>>>(uc, (int)S, qp->idx, qp->g, qp->nnz, chunk,
                                             static_cast<double*>(wsp->qps.p), static_cast<double*>(wsp->qpc.p),
                                             (int)s_lo, (int)s_hi);
    else  // the state's rows narrowed to `stride` (ragged batch)
      k_qoi_partial_rs<Real><<<qg, tb, 0, st>>>(uc, (int)stride, qp->idx, qp->g, qp->nnz, chunk,
                                                static_cast<double*>(wsp->qps.p), static_cast<double*>(wsp->qpc.p),
                                                (int)S, (int)s_lo, (int)s_hi);
    LF_CUDA(c, cudaGetLastError());
    pr.end(LFLTS_KERNEL_QOI, double(qp->nnz) * w * rb);
    if (d_uN) {
      k_gather_state<Real><<<blocks_for(n_nodes * w, 256, c->sms * 32), 256, 0, st>>>(n_nodes, (int)S, new2old,
                                                                                     uc, d_uN, (int)s_lo,
                                                                                     (int)s_hi);
      LF_CUDA(c, cudaGetLastError());
      c->launches++;
    }
    return 0;
  };
  lo.qoi_final = [=]() -> int {
    k_qoi_final<<<blocks_for(S, 128, 1 << 20), 128, 0, st>>>(n_chunks, (int)S, static_cast<double*>(wsp->qps.p),
                                                            static_cast<double*>(wsp->qpc.p), d_Q, d_bad);
    LF_CUDA(c, cudaGetLastError());
    c->launches++;
    return 0;
  };
  auto body = [&]() -> int {
    LF_TRY(a1());
    auto loop = make_sliced<Real>(c, ds, mg, n_R, S, ws, st, vec, cps, rg, lo);
    LF_TRY(loop->advance(ds.n_steps));
    return loop->finish();
  };

  // CUDA graph of the whole solve (one launch instead of ~p N), replayed while
  // the problem, the batch and the buffers stay the same.  Very long solves
  // (more than kGraphMaxKernels kernels) launch directly: their graphs would
  // take seconds and gigabytes of host memory to build, and their kernels
  // outlast the launch cost anyway.
  const int shape_in = cps % 10000;  // the inner kernel's part of the shape code
  const int64_t inner_per_step = n_R == 0 ? 0 : (shape_in >= 5000 ? p / 2 : (shape_in >= 2000 ? 1 : p - 1));
  const int64_t est_kernels = ds.n_steps * (1 + inner_per_step);
  const bool use_graph =
      allow_graph && c->graphs && !c->profiling && st != nullptr && est_kernels <= kGraphMaxKernels;
  if (!use_graph) {
    if (!defer) return body();
    LF_TRY(a1());
    *defer = make_sliced<Real>(c, ds, mg, n_R, S, ws, st, vec, cps, rg, lo);
    return 0;
  }
  GraphKey key;
  std::memset(&key, 0, sizeof(key));  // padding too: keys compare bytewise
  key.mesh = ds.mesh_id;
  key.qoi = ds.qoi_id;
  key.u0 = ds.u0_field;
  key.v0 = ds.v0_field;
  key.precision = ds.precision;
  key.p = ds.p;
  key.nu = ds.nu;
  key.dt = ds.dt;
  key.n_steps = ds.n_steps;
  key.S = S;
  key.xi = d_xi;
  key.Q = d_Q;
  key.uN = d_uN;
  key.ua = ws.ua.p;
  key.ub = ws.ub.p;
  key.d = ws.d.p;
  key.g = ws.g.p;
  key.r0 = ws.r0.p;
  key.r1 = ws.r1.p;
  key.r2 = ws.r2.p;
  key.r3 = ws.r3.p;
  key.W = ws.W.p;
  key.xipad = ws.xipad.p;
  key.qps = ws.qps.p;
  key.qpc = ws.qpc.p;
  key.vec = vec;
  key.cps = cps;
  key.source = ds.source_id;
  key.f0 = ds.src_f0;
  key.t0 = ds.src_t0;
  key.famp = ds.src_amp;
  key.ragged = rg ? rg->hash : 0;
  key.dts = rg ? rg->d_dts : nullptr;
  key.sig = rg ? rg->d_sig : nullptr;
  for (size_t k = 0; k < ws.graphs.size(); ++k)
    if (ws.graphs[k].key == key) {
      // most recently used last: eviction takes the front
      std::rotate(ws.graphs.begin() + k, ws.graphs.begin() + k + 1, ws.graphs.end());
      const GraphEntry& ge = ws.graphs.back();
      LF_CUDA(c, cudaGraphLaunch(ge.exec, st));
      c->launches += ge.kernels;
      c->graph_launches++;
      return 0;
    }
  // a full cache gives up its least recently used graphs first (after the
  // stream has finished with them; outside any capture)
  if (!ws.graphs.empty() && int64_t(ws.graphs.size()) >= c->graph_cap) {
    LF_CUDA(c, cudaStreamSynchronize(st));
    while (!ws.graphs.empty() && int64_t(ws.graphs.size()) >= c->graph_cap) {
      cudaGraphExecDestroy(ws.graphs.front().exec);
      ws.graphs.erase(ws.graphs.begin());
    }
  }
  const int64_t l0 = c->launches;
  LF_CUDA(c, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const int rc = body();
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ec != cudaSuccess) return fail(c, LFLTS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
  const int64_t kernels = c->launches - l0;
  c->launches = l0;
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return fail(c, LFLTS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
  ws.graphs.push_back({key, exec, kernels});
  LF_CUDA(c, cudaGraphLaunch(exec, st));
  c->launches += kernels;
  c->graph_launches++;
  return 0;
}

template <typename Real>
int run_solve(lflts_ctx* c, const lflts_solve_desc& ds, const double* d_xi, int64_t S, double* d_Q,
              double* d_uN, Workspace& ws, cudaStream_t st, std::unique_ptr<SliceTask>* defer,
              const RaggedSpec* rg, bool allow_graph) {
  MeshGPU& mg = *c->meshes[ds.mesh_id];
  const Qoi& q = c->qois[ds.qoi_id];
  const Field& u0 = c->fields[ds.u0_field];
  const Field* v0 = ds.v0_field >= 0 ? &c->fields[ds.v0_field] : nullptr;
  switch (mg.h.KP) {
    case 4: return run_solve_kp<Real, 4>(c, ds, mg, q, u0, v0, d_xi, S, d_Q, d_uN, ws, st, defer, rg, allow_graph);
    case 8: return run_solve_kp<Real, 8>(c, ds, mg, q, u0, v0, d_xi, S, d_Q, d_uN, ws, st, defer, rg, allow_graph);
    default: return run_solve_kp<Real, 16>(c, ds, mg, q, u0, v0, d_xi, S, d_Q, d_uN, ws, st, defer, rg, allow_graph);
  }
}

int check_desc(lflts_ctx* c, const lflts_solve_desc* ds) {
  if (!ds) return fail(c, LFLTS_ERR_ARG, "solve: null descriptor");
  if (ds->mesh_id < 0 || ds->mesh_id >= (int)c->meshes.size()) return fail(c, LFLTS_ERR_ARG, "solve: bad mesh_id");
  if (ds->qoi_id < 0 || ds->qoi_id >= (int)c->qois.size() || c->qois[ds->qoi_id].mesh != ds->mesh_id)
    return fail(c, LFLTS_ERR_ARG, "solve: qoi_id does not belong to the mesh");
  if (ds->u0_field < 0 || ds->u0_field >= (int)c->fields.size() || c->fields[ds->u0_field].mesh != ds->mesh_id)
    return fail(c, LFLTS_ERR_ARG, "solve: u0_field does not belong to the mesh");
  if (ds->v0_field >= 0 && (ds->v0_field >= (int)c->fields.size() || c->fields[ds->v0_field].mesh != ds->mesh_id))
    return fail(c, LFLTS_ERR_ARG, "solve: v0_field does not belong to the mesh");
  if (ds->precision != 32 && ds->precision != 64) return fail(c, LFLTS_ERR_ARG, "solve: precision must be 32 or 64");
  if (ds->p < 1 || ds->p > 128) return fail(c, LFLTS_ERR_ARG, "solve: p must be in [1, 128]");
  if (!(ds->nu >= 0.0 && ds->nu <= 1.0)) return fail(c, LFLTS_ERR_ARG, "solve: nu must be in [0, 1]");
  if (!(ds->dt > 0.0) || !std::isfinite(ds->dt)) return fail(c, LFLTS_ERR_ARG, "solve: dt must be positive");
  if (ds->n_steps < 1) return fail(c, LFLTS_ERR_ARG, "solve: n_steps must be >= 1");
  if (ds->source_id >= 0 && (ds->source_id >= (int)c->sources.size() || c->sources[ds->source_id].mesh != ds->mesh_id))
    return fail(c, LFLTS_ERR_ARG, "solve: source_id does not belong to the mesh");
  if (ds->source_id >= 0 && !(std::isfinite(ds->src_f0) && std::isfinite(ds->src_t0) && std::isfinite(ds->src_amp)))
    return fail(c, LFLTS_ERR_ARG, "solve: non-finite source parameters");
  if (ds->source_id >= 0 && c->meshes[ds->mesh_id]->h.moving)
    return fail(c, LFLTS_ERR_ARG, "solve: a source on a moving mesh is not supported");
  return 0;
}

// defer non-null: a solve that is not captured into a graph only queues its
// start here and returns its time loop as a SliceTask in *defer.
// allow_graph false: never captured (the time loop of a sliced run).
int solve_device(lflts_ctx* c, const lflts_solve_desc& ds, const double* d_xi, int64_t S, double* d_Q,
                 double* d_uN, Workspace& ws, cudaStream_t st, std::unique_ptr<SliceTask>* defer = nullptr,
                 const RaggedSpec* rg = nullptr, bool allow_graph = true) {
  if (ds.precision == 32) return run_solve<float>(c, ds, d_xi, S, d_Q, d_uN, ws, st, defer, rg, allow_graph);
  return run_solve<double>(c, ds, d_xi, S, d_Q, d_uN, ws, st, defer, rg, allow_graph);
}

Workspace& workspace(lflts_ctx* c, size_t slot) {
  while (c->ws.size() <= slot) c->ws.emplace_back(new Workspace());
  return *c->ws[slot];
}

int reset_bad(lflts_ctx* c, cudaStream_t st) {
  LF_CUDA(c, cudaMemsetAsync(c->d_bad, 0x7f, sizeof(int), st));
  return 0;
}

int check_bad(lflts_ctx* c, cudaStream_t st) {
  int bad = INT_MAX;
  LF_CUDA(c, cudaMemcpyAsync(&bad, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  LF_CUDA(c, cudaStreamSynchronize(st));
  if (bad != 0x7f7f7f7f)
    return fail(c, LFLTS_ERR_UNSTABLE, "non-finite QoI (unstable solve), first sample " + std::to_string(bad));
  return 0;
}

// ---------------------------------------------------------------------------
// Gradient of the QoI with respect to xi: discrete adjoint (adjoint.cuh),
// checkpoints every k outer steps, forward recomputation inside a segment.
// ---------------------------------------------------------------------------
template <typename Real, int VEC, int KP>
int run_grad(lflts_ctx* c, const lflts_solve_desc& ds, const double* d_xi, int64_t S, int k_ck, double* d_Q,
             double* d_G, cudaStream_t st) {
  const MeshGPU& mg = *c->meshes[ds.mesh_id];
  const HostMesh& h = mg.h;
  const Qoi& q = c->qois[ds.qoi_id];
  const Field& u0 = c->fields[ds.u0_field];
  const Field* v0 = ds.v0_field >= 0 ? &c->fields[ds.v0_field] : nullptr;
  if (!c->gws) c->gws.reset(new Workspace());
  if (!c->gb) c->gb.reset(new GradBufs());
  Workspace& ws = *c->gws;
  GradBufs& gb = *c->gb;
  const int p = ds.p;
  const int n_R = p > 1 ? static_cast<int>(h.n_R) : 0;
  const int nP_eff = p > 1 ? static_cast<int>(h.n_P) : 0;
  const int64_t N = ds.n_steps;
  const int64_t n_nodes = h.n_nodes;
  const size_t rb = sizeof(Real);
  const size_t state = size_t(n_nodes) * S * rb, rsz = size_t(std::max(n_R, 1)) * S * rb;
  const int64_t k = std::max<int64_t>(1, std::min<int64_t>(k_ck, N));
  const int64_t n_ck = (N + k - 1) / k;
  LF_TRY(ensure(c, ws.ua, state));
  LF_TRY(ensure(c, ws.ub, state));
  LF_TRY(ensure(c, ws.d, state));
  LF_TRY(ensure(c, ws.g, rsz));
  LF_TRY(ensure(c, ws.r0, rsz));
  LF_TRY(ensure(c, ws.r1, rsz));
  LF_TRY(ensure(c, ws.r2, rsz));
  LF_TRY(ensure(c, ws.W, size_t(std::max<int64_t>(h.n_edges, 1)) * S * rb));
  LF_TRY(ensure(c, ws.xipad, size_t(S) * KP * rb));
  LF_TRY(ensure(c, gb.ckpt, size_t(n_ck) * 2 * state));
  LF_TRY(ensure(c, gb.segU, size_t(k) * state));
  LF_TRY(ensure(c, gb.rs, size_t(std::max(p - 2, 1)) * rsz));
  LF_TRY(ensure(c, gb.rho, size_t(std::max(p - 1, 1)) * rsz));
  LF_TRY(ensure(c, gb.gs, rsz));
  LF_TRY(ensure(c, gb.A, size_t(std::max<int64_t>(h.n_edges, 1)) * S * sizeof(double)));
  constexpr bool kF32 = std::is_same<Real, float>::value;  // FP32 edge terms, per-segment FP32 sums
  if (kF32) LF_TRY(ensure(c, gb.Aseg, size_t(std::max<int64_t>(h.n_edges, 1)) * S * sizeof(float)));
  LF_TRY(ensure(c, gb.nua, state));
  LF_TRY(ensure(c, gb.nub, state));
  LF_TRY(ensure(c, gb.dnu, state));
  Real* ua = static_cast<Real*>(ws.ua.p);
  Real* ub = static_cast<Real*>(ws.ub.p);
  Real* d = static_cast<Real*>(ws.d.p);
  Real* xi = static_cast<Real*>(ws.xipad.p);
  Real* W = static_cast<Real*>(ws.W.p);
  Real* ckpt = static_cast<Real*>(gb.ckpt.p);
  Real* segU = static_cast<Real*>(gb.segU.p);
  Real* rs = static_cast<Real*>(gb.rs.p);
  Real* rho = static_cast<Real*>(gb.rho.p);
  Real* gs = static_cast<Real*>(gb.gs.p);
  double* A = static_cast<double*>(gb.A.p);
  const size_t sn = size_t(n_nodes) * S;  // elements per state array
  const size_t rn = size_t(std::max(n_R, 1)) * S;

  {  // a1 and start values, as in lflts_solve
    Prof pr(c, st);
    k_xi_pad<Real, KP><<<blocks_for(S * KP, 256, 4096), 256, 0, st>>>((int)S, h.K, d_xi, xi);
    LF_CUDA(c, cudaGetLastError());
    k_init_state<Real><<<blocks_for(n_nodes * S, 256, c->sms * 32), 256, 0, st>>>(
        n_nodes, (int)S, Sel<Real>::field(u0), v0 ? Sel<Real>::field(*v0) : nullptr, (Real)ds.dt, ua, ub, d);
    LF_CUDA(c, cudaGetLastError());
    const Geo ge = geometry(c, std::max<int64_t>(h.n_edges, 1), S);
    k_edge_weights<Real, KP><<<ge.grid, 256, 0, st>>>(h.n_edges, (int)S, ge.SB, mg.ee, Sel<Real>::eg(mg),
                                                      Sel<Real>::psi(mg), xi, W);
    LF_CUDA(c, cudaGetLastError());
    pr.end(LFLTS_KERNEL_INIT, double(S) * rb * (3.0 * n_nodes + double(h.n_edges)));
    c->launches += 2;
  }
  Stepper<Real, VEC> stp(c, ds, mg, n_R, S, W, static_cast<Real*>(ws.g.p), static_cast<Real*>(ws.r0.p),
                         static_cast<Real*>(ws.r1.p), static_cast<Real*>(ws.r2.p));

  // ---- forward with checkpoints of (u_n, d_n) every k steps --------------
  Real* uc = ua;
  Real* un = ub;
  for (int64_t n = 0; n < N; ++n) {
    if (n % k == 0) {
      LF_CUDA(c, cudaMemcpyAsync(ckpt + (2 * (n / k)) * sn, uc, state, cudaMemcpyDeviceToDevice, st));
      LF_CUDA(c, cudaMemcpyAsync(ckpt + (2 * (n / k) + 1) * sn, d, state, cudaMemcpyDeviceToDevice, st));
    }
    LF_TRY(stp.step(uc, un, d, (n == 0) ? Real(1) : Real(2), st, n));
    std::swap(uc, un);
  }
  {  // QoI of u_N
    const int chunk = 512;
    const int n_chunks = std::max(1, (q.nnz + chunk - 1) / chunk);
    LF_TRY(ensure(c, ws.qps, size_t(n_chunks) * S * sizeof(double)));
    LF_TRY(ensure(c, ws.qpc, size_t(n_chunks) * S * sizeof(double)));
    const int tb = static_cast<int>(std::min<int64_t>(S, 128));
    Prof pr(c, st);
    k_qoi_partial<Real><<<dim3(n_chunks, static_cast<unsigned>((S + tb - 1) / tb)), tb, 0, st>>>(
        uc, (int)S, q.idx, q.g, q.nnz, chunk, static_cast<double*>(ws.qps.p), static_cast<double*>(ws.qpc.p), 0,
        (int)S);
    LF_CUDA(c, cudaGetLastError());
    k_qoi_final<<<blocks_for(S, 128, 1 << 20), 128, 0, st>>>(n_chunks, (int)S, static_cast<double*>(ws.qps.p),
                                                            static_cast<double*>(ws.qpc.p), d_Q, c->d_bad);
    LF_CUDA(c, cudaGetLastError());
    pr.end(LFLTS_KERNEL_QOI, double(q.nnz) * S * rb);
    c->launches++;
  }

  // ---- adjoint seed nu_N = M^-1 g_Q, d nu = nu_N, A = 0 --------------------
  Real* vc = static_cast<Real*>(gb.nua.p);
  Real* vn = static_cast<Real*>(gb.nub.p);
  Real* dv = static_cast<Real*>(gb.dnu.p);
  LF_CUDA(c, cudaMemsetAsync(vc, 0, state, st));
  LF_CUDA(c, cudaMemsetAsync(vn, 0, state, st));
  LF_CUDA(c, cudaMemsetAsync(dv, 0, state, st));
  LF_CUDA(c, cudaMemsetAsync(A, 0, size_t(std::max<int64_t>(h.n_edges, 1)) * S * sizeof(double), st));
  float* Aseg = static_cast<float*>(gb.Aseg.p);
  if (kF32) LF_CUDA(c, cudaMemsetAsync(Aseg, 0, size_t(std::max<int64_t>(h.n_edges, 1)) * S * sizeof(float), st));
  // the step kernels write free nodes only: Dirichlet rows of the recomputed
  // states must hold 0 (the edge accumulation reads them)
  LF_CUDA(c, cudaMemsetAsync(segU, 0, size_t(k) * state, st));
  {
    Prof pr(c, st);
    k_adj_seed<Real><<<blocks_for(int64_t(q.nnz) * S, 256, c->sms * 16), 256, 0, st>>>(
        q.nnz, (int)S, q.idx, q.g, mg.minv64, (int)h.n_free, vc, dv);
    LF_CUDA(c, cudaGetLastError());
    pr.end(LFLTS_KERNEL_GRAD, double(q.nnz) * S * 2.0 * rb);
  }

  MeshDev<Real> mdR = Sel<Real>::mesh(mg, n_R);
  mdR.n_free = n_R;  // g = a(u) on R only
  const Geo gR = geometry_vec(c, std::max(n_R, 1), S, VEC);
  const Geo gE = geometry(c, std::max<int64_t>(h.n_edges, 1), S);
  AdjConsts kc{};
  kc.p = p;
  kc.gamma = stp.gamma;
  kc.c[0] = stp.c0;
  for (int m = 1; m < p; ++m) kc.c[m] = stp.cm[m];
  // algorithmic bytes per launch (profiling): R rows and edges with an R endpoint
  // (R is the index prefix [0, n_R) and edge_i < edge_j)
  int64_t n_edges_R = 0;
  for (int64_t e = 0; e < h.n_edges; ++e) n_edges_R += h.edge_i[e] < n_R;
  const double Srb = double(S) * rb;
  const double edges_bytes = (kF32 ? 8.0 : 16.0) * double(h.n_edges) * S + 2.0 * double(h.n_free) * Srb +
                             double(2 * p - 2) * double(n_R) * Srb;
  const Geo gE32 = geometry(c, std::max<int64_t>(h.n_edges, 1), S / VEC);
  AdjConsts32 kc32{};
  kc32.p = p;
  for (int m = 0; m < p; ++m) kc32.c[m] = float(kc.c[m]);

  // ---- segments, last to first ------------------------------------------------
  for (int64_t seg = n_ck - 1; seg >= 0; --seg) {
    const int64_t n0 = seg * k, n1 = std::min(N, n0 + k);
    LF_CUDA(c, cudaMemcpyAsync(segU, ckpt + (2 * seg) * sn, state, cudaMemcpyDeviceToDevice, st));
    LF_CUDA(c, cudaMemcpyAsync(d, ckpt + (2 * seg + 1) * sn, state, cudaMemcpyDeviceToDevice, st));
    for (int64_t n = n0; n + 1 < n1; ++n)
      LF_TRY(stp.step(segU + (n - n0) * sn, segU + (n - n0 + 1) * sn, d, (n == 0) ? Real(1) : Real(2), st, n));
    for (int64_t n = n1 - 1; n >= n0; --n) {
      const Real kappa = (n == 0) ? Real(1) : Real(2);
      const Real* u_n = segU + (n - n0) * sn;
      if (n_R > 0) {
        // (i) g = a(u_n) on R; (ii) r_2 .. r_{p-1} of the inner recursion
        {
          Prof pr(c, st);
          k_coarse<Real, VEC><<<gR.grid, 256, 0, st>>>(mdR, (int)S, gR.SB, W, u_n, nullptr, nullptr, gs, Real(0),
                                                        stp.fw, stp.source_amp(double(n) * ds.dt), (int)S,
                                                        RaggedF{});
          LF_CUDA(c, cudaGetLastError());
          pr.end(LFLTS_KERNEL_ADJ_INNER, 2.0 * double(n_R) * Srb + double(n_edges_R) * Srb);
        }
        for (int m = 1; m <= p - 2; ++m) {
          Prof pr(c, st);
          const Real* cur = (m == 1) ? gs : rs + (m - 2) * rn;
          const Real s_cur = (m == 1) ? (Real)(-stp.c0) : Real(1);
          const Real* prv = (m == 1) ? nullptr : ((m == 2) ? gs : rs + (m - 3) * rn);
          const Real s_prv = (m == 2) ? (Real)(-stp.c0) : Real(1);
          k_inner<Real, VEC, false><<<gR.grid, 256, 0, st>>>(
              stp.md, (int)S, gR.SB, W, cur, s_cur, prv, s_prv, rs + (m - 1) * rn, gs, nullptr, nullptr, nullptr,
              (Real)(1.0 + stp.beta[m]), (Real)stp.beta[m], (Real)stp.cm[m], Real(0), (int)S);
          LF_CUDA(c, cudaGetLastError());
          pr.end(LFLTS_KERNEL_ADJ_INNER, double(m == 1 ? 2 : (m == 2 ? 3 : 4)) * double(n_R) * Srb);
        }
        // (iii) inner adjoint rho_{p-1} .. rho_1 (rho_p = kappa nu_{n+1})
        for (int m = p - 1; m >= 1; --m) {
          const Real* s1p = (m + 1 == p) ? vc : rho + m * rn;
          const Real s1 = (m + 1 == p) ? kappa : Real(1);
          const Real* s2p = (m + 2 == p) ? vc : ((m + 2 < p) ? rho + (m + 1) * rn : nullptr);
          const Real s2 = (m + 2 == p) ? kappa : Real(1);
          const Real b1 = (m + 1 <= p - 1) ? (Real)stp.beta[m + 1] : Real(0);
          Prof pr(c, st);
          k_adj_inner<Real, VEC><<<gR.grid, 256, 0, st>>>(stp.md, (int)S, gR.SB, W, s1p, s1, s2p, s2,
                                                           rho + (m - 1) * rn, (Real)(1.0 + stp.beta[m]), b1,
                                                           (Real)stp.cm[m]);
          LF_CUDA(c, cudaGetLastError());
          pr.end(LFLTS_KERNEL_ADJ_INNER, double(s2p ? 3 : 2) * double(n_R) * Srb);
        }
      }
      // (iv) edge accumulators
      kc.kappa = double(kappa);
      {
        Prof pr(c, st);
        if constexpr (kF32) {
          kc32.kappa = float(kappa);
          kc32.gk = float(kc.gamma * double(kappa));
          k_adj_edges32<VEC><<<gE32.grid, 256, 0, st>>>(h.n_edges, nP_eff, n_R, (int)S, gE32.SB, mg.ends, u_n, vc,
                                                        gs, rs, rho, Aseg, kc32);
        } else {
          k_adj_edges<Real><<<gE.grid, 256, 0, st>>>(h.n_edges, nP_eff, n_R, (int)S, gE.SB, mg.ends, u_n, vc, gs,
                                                     rs, rho, A, kc);
        }
        LF_CUDA(c, cudaGetLastError());
        pr.end(LFLTS_KERNEL_ADJ_EDGES, edges_bytes);
      }
      // (v) nu_n = 2 T nu_{n+1} - nu_{n+2}
      if (n > 0) {
        const Real* fw_saved = stp.fw;
        stp.fw = nullptr;  // the adjoint recursion has no forcing
        const int rc = stp.step(vc, vn, dv, Real(2), st);
        stp.fw = fw_saved;
        LF_TRY(rc);
        std::swap(vc, vn);
      }
    }
    if constexpr (kF32) {  // end of the segment: A += Aseg, Aseg = 0
      const int64_t ne = std::max<int64_t>(h.n_edges, 1) * S;
      Prof pr(c, st);
      k_adj_fold<<<blocks_for(ne, 256, c->sms * 16), 256, 0, st>>>(ne, Aseg, A);
      LF_CUDA(c, cudaGetLastError());
      pr.end(LFLTS_KERNEL_ADJ_EDGES, 24.0 * double(ne));
    }
  }

  // ---- dQ/dxi_k = sum_edges A_e dK_e/dxi_k ------------------------------------
  const int64_t chunk = 4096;
  const int64_t n_chunks = std::max<int64_t>(1, (h.n_edges + chunk - 1) / chunk);
  LF_TRY(ensure(c, gb.part, size_t(n_chunks) * S * h.K * sizeof(double)));
  const int tb = static_cast<int>(std::min<int64_t>(S, 128));
  Prof pr(c, st);
  k_grad_contract<KP><<<dim3(static_cast<unsigned>(n_chunks), static_cast<unsigned>((S + tb - 1) / tb)), tb, 0, st>>>(
      h.n_edges, (int)S, chunk, mg.ee, mg.eg64, mg.psi64, d_xi, h.K, A, static_cast<double*>(gb.part.p));
  LF_CUDA(c, cudaGetLastError());
  k_grad_finish<<<blocks_for(S * h.K, 128, 1 << 20), 128, 0, st>>>((int)n_chunks, (int)S, h.K,
                                                                   static_cast<double*>(gb.part.p), d_G);
  LF_CUDA(c, cudaGetLastError());
  c->launches++;
  pr.end(LFLTS_KERNEL_GRAD, 8.0 * double(h.n_edges) * S + 8.0 * double(S) * h.K * (1.0 + n_chunks));
  return 0;
}

template <typename Real, int VEC>
int run_grad_kp(lflts_ctx* c, const lflts_solve_desc& ds, const double* d_xi, int64_t S, int k_ck, double* d_Q,
                double* d_G, cudaStream_t st) {
  switch (c->meshes[ds.mesh_id]->h.KP) {
    case 4: return run_grad<Real, VEC, 4>(c, ds, d_xi, S, k_ck, d_Q, d_G, st);
    case 8: return run_grad<Real, VEC, 8>(c, ds, d_xi, S, k_ck, d_Q, d_G, st);
    default: return run_grad<Real, VEC, 16>(c, ds, d_xi, S, k_ck, d_Q, d_G, st);
  }
}

int grad_device(lflts_ctx* c, const lflts_solve_desc& ds, const double* d_xi, int64_t S, int k_ck, double* d_Q,
                double* d_G, cudaStream_t st) {
  if (ds.precision == 32) {
    if (S % 4 == 0) return run_grad_kp<float, 4>(c, ds, d_xi, S, k_ck, d_Q, d_G, st);
    if (S % 2 == 0) return run_grad_kp<float, 2>(c, ds, d_xi, S, k_ck, d_Q, d_G, st);
    return run_grad_kp<float, 1>(c, ds, d_xi, S, k_ck, d_Q, d_G, st);
  }
  if (S % 2 == 0) return run_grad_kp<double, 2>(c, ds, d_xi, S, k_ck, d_Q, d_G, st);
  return run_grad_kp<double, 1>(c, ds, d_xi, S, k_ck, d_Q, d_G, st);
}

// ---------------------------------------------------------------------------
// MLMC level pairs (lflts_run_pairs, lflts_run_pairs_slice).  Solves that
// differ at most in (dt, n_steps) share a batch (a group): identical ones
// form a segment, and a group with several segments is ragged (each draw
// steps with its own dt for its own count; segments sorted by step count).
// ---------------------------------------------------------------------------
struct PairMember {
  int job;
  bool fine;
  int64_t off;
};
struct PairSeg {
  lflts_solve_desc desc;
  int64_t S = 0;
  std::vector<PairMember> members;
};
struct PairGroup {
  std::vector<PairSeg> segs;
  int64_t S = 0;
};
struct PairRun {
  uint64_t sig = 0;
  int next = 0, n_slices = 1;
  std::vector<PairGroup> groups;
  std::vector<RaggedSpec> specs;
  std::vector<std::unique_ptr<SliceTask>> tasks;  // null: the group's whole solve is queued (a graph)
  std::vector<cudaStream_t> gst;                  // stream of each group
  std::vector<int64_t> N;                         // outer steps of each group's time loop
};

// FNV-1a over the jobs' bytes, the memory kind and the slice count: the
// calls of one sliced run must pass the same jobs.
uint64_t jobs_signature(const lflts_pair_job* jobs, int n_jobs, int mem, int n_slices) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t k = 0; k < n; ++k) h = (h ^ b[k]) * 1099511628211ull;
  };
  if (jobs)
    for (int j = 0; j < n_jobs; ++j) {
      const lflts_pair_job& jb = jobs[j];
      for (const lflts_solve_desc* d : {&jb.fine, &jb.coarse}) {
        mix(&d->mesh_id, sizeof(int) * 6);
        mix(&d->nu, sizeof(double) * 2);
        mix(&d->n_steps, sizeof(int64_t));
        mix(&d->source_id, sizeof(int));
        mix(&d->src_f0, sizeof(double) * 3);
      }
      mix(&jb.has_coarse, sizeof(int));
      mix(&jb.xi, sizeof(void*));
      mix(&jb.S, sizeof(int64_t));
      mix(&jb.dQ, sizeof(void*) * 3);
    }
  mix(&mem, sizeof(int));
  mix(&n_slices, sizeof(int));
  return h;
}

// Validate and group the jobs, copy the draws of every group into its
// workspace and queue the start of each group's solve (coefficients, start
// values); the time loops stay in run.tasks unless a whole solve went into a
// graph (n_slices == 1 only).
int pairs_start(lflts_ctx* c, PairRun& run, const lflts_pair_job* jobs, int n_jobs, int mem, int n_slices,
                cudaStream_t st) {
  run.n_slices = n_slices;
  std::vector<PairGroup>& groups = run.groups;
  auto same_batch = [](const lflts_solve_desc& a, const lflts_solve_desc& b) {
    return a.mesh_id == b.mesh_id && a.qoi_id == b.qoi_id && a.u0_field == b.u0_field &&
           a.v0_field == b.v0_field && a.precision == b.precision && a.p == b.p && a.nu == b.nu &&
           a.source_id == b.source_id && a.src_f0 == b.src_f0 && a.src_t0 == b.src_t0 && a.src_amp == b.src_amp;
  };
  auto add_member = [&](const lflts_solve_desc& ds, int j, bool fine, int64_t S) {
    PairGroup* gp = nullptr;
    for (auto& gr : groups)
      if (same_batch(gr.segs[0].desc, ds)) gp = &gr;
    if (!gp) {
      groups.emplace_back();
      gp = &groups.back();
    }
    PairSeg* sp = nullptr;
    for (auto& sg : gp->segs)
      if (sg.desc.dt == ds.dt && sg.desc.n_steps == ds.n_steps) sp = &sg;
    if (!sp) {
      gp->segs.emplace_back();
      sp = &gp->segs.back();
      sp->desc = ds;
    }
    sp->members.push_back({j, fine, sp->S});
    sp->S += S;
    gp->S += S;
  };
  for (int j = 0; j < n_jobs; ++j) {
    const lflts_pair_job& jb = jobs[j];
    if (!jb.xi || !jb.dQ || jb.S < 1)
      return fail(c, LFLTS_ERR_ARG, "run_pairs: job " + std::to_string(j) + " has null xi/dQ or S < 1");
    LF_TRY(check_desc(c, &jb.fine));
    if (jb.has_coarse) {
      LF_TRY(check_desc(c, &jb.coarse));
      if (c->meshes[jb.coarse.mesh_id]->h.K != c->meshes[jb.fine.mesh_id]->h.K)
        return fail(c, LFLTS_ERR_ARG, "run_pairs: fine and coarse meshes have different K");
    }
    add_member(jb.fine, j, true, jb.S);
    if (jb.has_coarse) add_member(jb.coarse, j, false, jb.S);
  }
  for (auto& gr : groups)
    if (gr.S > kMaxS) return fail(c, LFLTS_ERR_ARG, "run_pairs: merged batch larger than 2097120 samples");
  // segments by step count (descending), members' offsets within the batch
  std::vector<RaggedSpec>& specs = run.specs;
  specs.assign(groups.size(), RaggedSpec());
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    PairGroup& gr = groups[gi];
    std::stable_sort(gr.segs.begin(), gr.segs.end(),
                     [](const PairSeg& a, const PairSeg& b) { return a.desc.n_steps > b.desc.n_steps; });
    int64_t off = 0;
    uint64_t hsh = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
      for (int b = 0; b < 8; ++b) hsh = (hsh ^ ((v >> (8 * b)) & 0xff)) * 1099511628211ull;
    };
    for (PairSeg& sg : gr.segs) {
      for (PairMember& mb : sg.members) mb.off += off;
      specs[gi].segs.push_back({off, sg.S, sg.desc.n_steps, sg.desc.dt});
      uint64_t dbits = 0;
      std::memcpy(&dbits, &sg.desc.dt, sizeof(dbits));
      mix(uint64_t(sg.desc.n_steps));
      mix(uint64_t(sg.S));
      mix(dbits);
      off += sg.S;
    }
    specs[gi].hash = hsh;
  }

  // ---- streams and events ----------------------------------------------------
  const size_t ng = groups.size();
  while (c->streams.size() < ng) {
    cudaStream_t s;
    LF_CUDA(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    c->streams.push_back(s);
  }
  while (c->sync_events.size() < ng + 1) {
    cudaEvent_t e;
    LF_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->sync_events.push_back(e);
  }
  LF_TRY(reset_bad(c, st));
  LF_CUDA(c, cudaEventRecord(c->sync_events[ng], st));

  // ---- per group: gather xi, queue the start of the solve -----------------------
  // With per-launch profiling on, every group runs on the caller's stream, one
  // after the other, so that each kernel's event times are its own.
  run.tasks.resize(ng);
  run.gst.assign(ng, st);
  run.N.assign(ng, 0);
  for (size_t gi = 0; gi < ng; ++gi) {
    PairGroup& gr = groups[gi];
    Workspace& ws = workspace(c, 1 + gi);
    const lflts_solve_desc& gd = gr.segs[0].desc;  // the longest segment: dt_ref and the step count
    run.N[gi] = gd.n_steps;
    const int K = c->meshes[gd.mesh_id]->h.K;
    cudaStream_t gs = c->profiling ? st : c->streams[gi];
    run.gst[gi] = gs;
    LF_CUDA(c, cudaStreamWaitEvent(gs, c->sync_events[ng], 0));
    LF_TRY(ensure(c, ws.xraw, size_t(gr.S) * K * sizeof(double)));
    LF_TRY(ensure(c, ws.Q, size_t(gr.S) * sizeof(double)));
    for (const PairSeg& sg : gr.segs)
      for (const PairMember& mb : sg.members) {
        const lflts_pair_job& jb = jobs[mb.job];
        LF_CUDA(c, cudaMemcpyAsync(static_cast<double*>(ws.xraw.p) + mb.off * K, jb.xi,
                                   size_t(jb.S) * K * sizeof(double),
                                   mem == LFLTS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, gs));
      }
    const RaggedSpec* rg = nullptr;
    if (gr.segs.size() > 1) {  // per-draw dt and weight scale of the ragged batch
      const size_t rb = gd.precision == 32 ? sizeof(float) : sizeof(double);
      ws.h_dts.assign(size_t(gr.S), 0.0);
      ws.h_sig.assign(size_t(gr.S) * rb, 0);
      for (const RaggedSeg& sg : specs[gi].segs)
        for (int64_t k = 0; k < sg.cnt; ++k) {
          const double sc = (sg.dt / gd.dt) * (sg.dt / gd.dt);
          ws.h_dts[size_t(sg.off + k)] = sg.dt;
          if (rb == sizeof(float)) {
            const float f = float(sc);
            std::memcpy(ws.h_sig.data() + size_t(sg.off + k) * rb, &f, rb);
          } else {
            std::memcpy(ws.h_sig.data() + size_t(sg.off + k) * rb, &sc, rb);
          }
        }
      LF_TRY(ensure(c, ws.dts, size_t(gr.S) * sizeof(double)));
      LF_TRY(ensure(c, ws.sig, size_t(gr.S) * rb));
      LF_CUDA(c, cudaMemcpyAsync(ws.dts.p, ws.h_dts.data(), size_t(gr.S) * sizeof(double), cudaMemcpyHostToDevice, gs));
      LF_CUDA(c, cudaMemcpyAsync(ws.sig.p, ws.h_sig.data(), size_t(gr.S) * rb, cudaMemcpyHostToDevice, gs));
      specs[gi].d_dts = static_cast<const double*>(ws.dts.p);
      specs[gi].d_sig = ws.sig.p;
      rg = &specs[gi];
    }
    LF_TRY(solve_device(c, gd, static_cast<double*>(ws.xraw.p), gr.S, static_cast<double*>(ws.Q.p), nullptr, ws,
                        gs, &run.tasks[gi], rg, n_slices == 1));
  }
  return 0;
}

// Queue slice k of every group's time loop: outer steps
// [floor(N k / n), floor(N (k+1) / n)), in turns of kSliceSteps steps group
// after group so that every stream keeps work queued; the last slice also
// queues the QoI.  The caller's stream then waits for every group.
int pairs_advance(lflts_ctx* c, PairRun& run, int slice, cudaStream_t st) {
  const size_t ng = run.groups.size();
  std::vector<int64_t> target(ng, 0);
  for (size_t gi = 0; gi < ng; ++gi) target[gi] = run.N[gi] * (slice + 1) / run.n_slices;
  for (bool more = true; more;) {
    more = false;
    for (size_t gi = 0; gi < ng; ++gi) {
      SliceTask* t = run.tasks[gi].get();
      if (!t) continue;
      const int64_t left = target[gi] - t->position();
      if (left <= 0) continue;
      LF_TRY(t->advance(std::min<int64_t>(left, kSliceSteps)));
      more = more || target[gi] - t->position() > 0;
    }
  }
  const bool last = slice + 1 == run.n_slices;
  for (size_t gi = 0; gi < ng; ++gi) {
    if (last && run.tasks[gi]) LF_TRY(run.tasks[gi]->finish());
    LF_CUDA(c, cudaEventRecord(c->sync_events[gi], run.gst[gi]));
  }
  for (size_t gi = 0; gi < ng; ++gi) LF_CUDA(c, cudaStreamWaitEvent(st, c->sync_events[gi], 0));
  return 0;
}

// After the last slice: per job dQ, Qf and the level sums on the caller's
// stream (and the copies to host memory).
int pairs_finish(lflts_ctx* c, PairRun& run, const lflts_pair_job* jobs, int n_jobs, int mem, cudaStream_t st) {
  const size_t ng = run.groups.size();
  Workspace& ws0 = workspace(c, 0);
  int64_t total = 0;
  for (int j = 0; j < n_jobs; ++j) total += jobs[j].S;
  if (mem == LFLTS_MEM_HOST) LF_TRY(ensure(c, ws0.Q, size_t(total) * 2 * sizeof(double) + 4 * sizeof(double) * n_jobs));
  int64_t hoff = 0;
  for (int j = 0; j < n_jobs; ++j) {
    const lflts_pair_job& jb = jobs[j];
    const double* qf = nullptr;
    const double* qc = nullptr;
    for (size_t gi = 0; gi < ng; ++gi)
      for (const PairSeg& sg : run.groups[gi].segs)
        for (const PairMember& mb : sg.members)
          if (mb.job == j) {
            const double* base = static_cast<double*>(workspace(c, 1 + gi).Q.p) + mb.off;
            if (mb.fine) qf = base;
            else qc = base;
          }
    double* dq_dst = jb.dQ;
    double* qf_dst = jb.Qf;
    double* sums_dst = jb.sums;
    if (mem == LFLTS_MEM_HOST) {
      double* base = static_cast<double*>(ws0.Q.p);
      dq_dst = base + hoff;
      qf_dst = base + total + hoff;
      sums_dst = base + 2 * total + 4 * j;
    }
    {
      Prof pr(c, st);
      k_pair_diff<<<blocks_for(jb.S, 128, 1 << 20), 128, 0, st>>>((int)jb.S, qf, qc, dq_dst, qf_dst);
      LF_CUDA(c, cudaGetLastError());
      k_level_sums<<<1, 256, 0, st>>>(jb.S, qf, qc, sums_dst);
      LF_CUDA(c, cudaGetLastError());
      pr.end(LFLTS_KERNEL_SUMS, double(jb.S) * 8.0 * (qc ? 5.0 : 3.0));
      c->launches++;
    }
    if (mem == LFLTS_MEM_HOST) {
      LF_CUDA(c, cudaMemcpyAsync(jb.dQ, dq_dst, size_t(jb.S) * sizeof(double), cudaMemcpyDeviceToHost, st));
      if (jb.Qf) LF_CUDA(c, cudaMemcpyAsync(jb.Qf, qf_dst, size_t(jb.S) * sizeof(double), cudaMemcpyDeviceToHost, st));
      if (jb.sums) LF_CUDA(c, cudaMemcpyAsync(jb.sums, sums_dst, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    hoff += jb.S;
  }
  if (mem == LFLTS_MEM_HOST) return check_bad(c, st);
  return LFLTS_OK;
}

// disp non-null: a mesh whose vertices move with the draw (K modes, psi unused)
int mesh_add_impl(lflts_ctx* c, const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
                  const uint8_t* dirichlet, const uint8_t* P, const double* psi, int K, const double* disp,
                  int* mesh_id) {
  if (!c || !mesh_id) return LFLTS_ERR_ARG;
  c->err.clear();
  std::unique_ptr<MeshGPU> mg(new MeshGPU());
  std::vector<double> zero_psi;
  if (disp) {
    if (K < 1 || K > 16 || n_tri < 1) return fail(c, LFLTS_ERR_ARG, "mesh_add_moving: K must be in [1, 16]");
    zero_psi.assign(static_cast<size_t>(n_tri) * K, 0.0);
    psi = zero_psi.data();
  }
  int rc = prep_mesh(xy, n_nodes, tri, n_tri, dirichlet, P, psi, K, mg->h, c->err, disp != nullptr);
  if (rc) return rc;
  if (disp) {
    rc = make_moving(mg->h, disp, K, c->err);
    if (rc) return rc;
  }
  if (c->device >= 0) {
    LF_TRY(set_device(c));
    const HostMesh& h = mg->h;
    const size_t na = h.adj_j.size(), ne = static_cast<size_t>(h.n_edges);
    std::vector<int2> adj(na), ee(ne);
    for (size_t t = 0; t < na; ++t) adj[t] = make_int2(h.adj_j[t], h.adj_e[t]);
    std::vector<double> eg64(2 * ne);
    for (size_t k = 0; k < ne; ++k) {
      ee[k] = make_int2(h.edge_e0[k], h.edge_e1[k]);
      eg64[2 * k] = h.edge_G0[k];
      eg64[2 * k + 1] = h.edge_G1[k];
    }
    std::vector<float> eg32(eg64.begin(), eg64.end());
    std::vector<float> minv32(h.minv.begin(), h.minv.end());
    const double log2e = 1.4426950408889634073599246810019;
    std::vector<float> psi32(h.psi.size());  // scaled by log2(e) for exp2f
    for (size_t k = 0; k < psi32.size(); ++k) psi32[k] = float(h.psi[k] * log2e);
    LF_TRY(upload(c, &mg->adj_ptr, h.adj_ptr.data(), h.adj_ptr.size()));
    LF_TRY(upload(c, &mg->adj, adj.data(), na));
    std::vector<int4> ell(static_cast<size_t>(h.n_free) * 2);
    for (int64_t i = 0; i < h.n_free; ++i)
      for (int hh = 0; hh < 2; ++hh)
        ell[2 * i + hh] = make_int4(h.ell_j[4 * i + 2 * hh], h.ell_e[4 * i + 2 * hh], h.ell_j[4 * i + 2 * hh + 1],
                                    h.ell_e[4 * i + 2 * hh + 1]);
    LF_TRY(upload(c, &mg->ell, ell.data(), ell.size()));
    if (!h.ell_hi_j.empty()) {
      for (int64_t i = 0; i < h.n_free; ++i)
        for (int hh = 0; hh < 2; ++hh)
          ell[2 * i + hh] = make_int4(h.ell_hi_j[4 * i + 2 * hh], h.ell_hi_e[4 * i + 2 * hh],
                                      h.ell_hi_j[4 * i + 2 * hh + 1], h.ell_hi_e[4 * i + 2 * hh + 1]);
      LF_TRY(upload(c, &mg->ell_hi, ell.data(), ell.size()));
    }
    LF_TRY(upload(c, &mg->ee, ee.data(), ne));
    std::vector<int2> ends(ne);
    for (size_t k = 0; k < ne; ++k) ends[k] = make_int2(h.edge_i[k], h.edge_j[k]);
    LF_TRY(upload(c, &mg->ends, ends.data(), ne));
    LF_TRY(upload(c, &mg->eg32, eg32.data(), eg32.size()));
    LF_TRY(upload(c, &mg->eg64, eg64.data(), eg64.size()));
    LF_TRY(upload(c, &mg->minv32, minv32.data(), minv32.size()));
    LF_TRY(upload(c, &mg->minv64, h.minv.data(), h.minv.size()));
    LF_TRY(upload(c, &mg->psi32, psi32.data(), psi32.size()));
    LF_TRY(upload(c, &mg->psi64, h.psi.data(), h.psi.size()));
    LF_TRY(upload(c, &mg->new2old, h.new2old.data(), h.new2old.size()));
    if (h.moving) {
      LF_TRY(upload(c, &mg->dedge, h.dedge.data(), h.dedge.size()));
      LF_TRY(upload(c, &mg->tri_new, h.tri_new.data(), h.tri_new.size()));
      LF_TRY(upload(c, &mg->xy64, h.xy.data(), h.xy.size()));
      LF_TRY(upload(c, &mg->disp, h.disp.data(), h.disp.size()));
      LF_TRY(upload(c, &mg->nptr, h.nptr.data(), h.nptr.size()));
      LF_TRY(upload(c, &mg->nelem, h.nelem.data(), h.nelem.size()));
    }
  }
  *mesh_id = static_cast<int>(c->meshes.size());
  c->meshes.push_back(std::move(mg));
  return LFLTS_OK;
}

}  // namespace

lflts_ctx::~lflts_ctx() = default;

// Error reporting for entry points defined in other translation units.
int lflts_internal_set_error(lflts_ctx* ctx, int code, const char* msg) {
  if (ctx) ctx->err = msg ? msg : "";
  return code;
}

int lflts_internal_ctx_device(const lflts_ctx* ctx) { return ctx ? ctx->device : -1; }

// ============================================================================
// ABI
// ============================================================================
extern "C" {

int lflts_version(void) { return 200; }

int lflts_create(lflts_ctx** out, int device) {
  if (!out) return LFLTS_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<lflts_ctx> c(new lflts_ctx());
  c->device = device;
  if (device >= 0) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device >= n) return LFLTS_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return LFLTS_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return LFLTS_ERR_CUDA;
    c->sms = prop.multiProcessorCount;
    if (cudaMalloc(&c->d_bad, sizeof(int)) != cudaSuccess) return LFLTS_ERR_OOM;
    if (cudaMalloc(&c->d_scratch, 64 * sizeof(double)) != cudaSuccess) return LFLTS_ERR_OOM;
  }
  *out = c.release();
  return LFLTS_OK;
}

int lflts_destroy(lflts_ctx* c) {
  if (!c) return LFLTS_OK;
  if (c->device >= 0) {
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto& w : c->ws)
      for (auto& ge : w->graphs) cudaGraphExecDestroy(ge.exec);
    for (auto& w : c->fws)
      if (w)
        for (auto& ge : w->graphs) cudaGraphExecDestroy(ge.exec);
    for (auto& w : c->ws)
      for (Buf* b : {&w->ua, &w->ub, &w->d, &w->g, &w->r0, &w->r1, &w->r2, &w->r3, &w->cmp, &w->W, &w->xipad, &w->xraw, &w->qps,
                     &w->qpc, &w->Q, &w->uN, &w->dts, &w->sig})
        if (b->p) cudaFree(b->p);
    for (Workspace* w : {c->gws.get(), c->fws[0].get(), c->fws[1].get()})
      if (w)
        for (Buf* b : {&w->ua, &w->ub, &w->d, &w->g, &w->r0, &w->r1, &w->r2, &w->r3, &w->cmp, &w->W, &w->xipad, &w->xraw, &w->qps,
                       &w->qpc, &w->Q, &w->uN, &w->dts, &w->sig})
          if (b->p) cudaFree(b->p);
    if (c->fb)
      for (Buf* b : {&c->fb->uf, &c->fb->uc, &c->fb->qf, &c->fb->qc, &c->fb->s1, &c->fb->n2, &c->fb->ps,
                     &c->fb->pc, &c->fb->sums, &c->fb->xraw, &c->fb->dq})
        if (b->p) cudaFree(b->p);
    if (c->gb)
      for (Buf* b : {&c->gb->ckpt, &c->gb->segU, &c->gb->rs, &c->gb->rho, &c->gb->gs, &c->gb->A, &c->gb->Aseg,
                     &c->gb->nua, &c->gb->nub, &c->gb->dnu, &c->gb->part, &c->gb->xraw, &c->gb->Q, &c->gb->G})
        if (b->p) cudaFree(b->p);
    for (void* p : c->owned) cudaFree(p);
    for (auto s : c->streams) cudaStreamDestroy(s);
    for (auto e : c->sync_events) cudaEventDestroy(e);
    for (auto& r : c->pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : c->pool) cudaEventDestroy(e);
    if (c->d_bad) cudaFree(c->d_bad);
    if (c->d_scratch) cudaFree(c->d_scratch);
  }
  delete c;
  return LFLTS_OK;
}

const char* lflts_last_error(const lflts_ctx* c) { return c ? c->err.c_str() : "null context"; }

int lflts_mesh_add(lflts_ctx* c, const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
                   const uint8_t* dirichlet, const uint8_t* P, const double* psi, int K, int* mesh_id) {
  return mesh_add_impl(c, xy, n_nodes, tri, n_tri, dirichlet, P, psi, K, nullptr, mesh_id);
}

int lflts_mesh_add_moving(lflts_ctx* c, const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
                          const uint8_t* dirichlet, const uint8_t* P, const double* disp, int K, int* mesh_id) {
  if (c && !disp) return fail(c, LFLTS_ERR_ARG, "mesh_add_moving: null displacement modes");
  return mesh_add_impl(c, xy, n_nodes, tri, n_tri, dirichlet, P, nullptr, K, disp, mesh_id);
}

int lflts_mesh_info(lflts_ctx* c, int mesh_id, int64_t info[8]) {
  if (!c || !info) return LFLTS_ERR_ARG;
  if (mesh_id < 0 || mesh_id >= (int)c->meshes.size()) return fail(c, LFLTS_ERR_ARG, "mesh_info: bad mesh_id");
  const HostMesh& h = c->meshes[mesh_id]->h;
  info[0] = h.n_nodes;
  info[1] = h.n_free;
  info[2] = h.n_R;
  info[3] = h.n_P;
  info[4] = h.n_tri;
  info[5] = h.K;
  info[6] = h.n_edges;
  info[7] = h.n_edges_P;
  return LFLTS_OK;
}

int lflts_mesh_order(lflts_ctx* c, int mesh_id, int32_t* new2old) {
  if (!c || !new2old) return LFLTS_ERR_ARG;
  if (mesh_id < 0 || mesh_id >= (int)c->meshes.size()) return fail(c, LFLTS_ERR_ARG, "mesh_order: bad mesh_id");
  const HostMesh& h = c->meshes[mesh_id]->h;
  std::memcpy(new2old, h.new2old.data(), h.new2old.size() * sizeof(int32_t));
  return LFLTS_OK;
}

int lflts_interp_weights(const double* xy_c, int64_t n_c, const int32_t* tri_c, int64_t n_tri_c,
                         const double* xy_f, int64_t n_f, int32_t* vert, double* w) {
  if (!xy_c || !tri_c || !xy_f || !vert || !w || n_c < 3 || n_tri_c < 1 || n_f < 1) return LFLTS_ERR_ARG;
  for (int64_t k = 0; k < 3 * n_tri_c; ++k)
    if (tri_c[k] < 0 || tri_c[k] >= n_c) return LFLTS_ERR_ARG;
  const int64_t outside = interp_weights(xy_c, tri_c, n_tri_c, xy_f, n_f, vert, w, 1e-10);
  return outside ? LFLTS_ERR_MESH : LFLTS_OK;
}

int lflts_lts_constants(int p, double nu, double dt, double* out) {
  if (!out || p < 1 || p > 128 || !(nu >= 0.0 && nu <= 1.0) || !(dt > 0.0)) return LFLTS_ERR_ARG;
  std::vector<double> beta, cm;
  double delta, omega, c0, gamma;
  lts_constants(p, nu, dt, beta, cm, delta, omega, c0, gamma);
  out[0] = delta;
  out[1] = omega;
  out[2] = c0;
  out[3] = gamma;
  for (int m = 1; m < p; ++m) {
    out[4 + 2 * (m - 1)] = beta[m];
    out[5 + 2 * (m - 1)] = cm[m];
  }
  return LFLTS_OK;
}

int lflts_field_add(lflts_ctx* c, int mesh_id, const double* values, int* field_id) {
  if (!c || !values || !field_id) return LFLTS_ERR_ARG;
  if (mesh_id < 0 || mesh_id >= (int)c->meshes.size()) return fail(c, LFLTS_ERR_ARG, "field_add: bad mesh_id");
  LF_TRY(set_device(c));
  const HostMesh& h = c->meshes[mesh_id]->h;
  std::vector<double> v64(h.n_nodes, 0.0);
  for (int64_t k = 0; k < h.n_free; ++k) {
    const double v = values[h.new2old[k]];
    if (!std::isfinite(v)) return fail(c, LFLTS_ERR_ARG, "field_add: non-finite value");
    v64[k] = v;
  }
  std::vector<float> v32(v64.begin(), v64.end());
  Field f;
  f.mesh = mesh_id;
  LF_TRY(upload(c, &f.v64, v64.data(), v64.size()));
  LF_TRY(upload(c, &f.v32, v32.data(), v32.size()));
  *field_id = static_cast<int>(c->fields.size());
  c->fields.push_back(f);
  return LFLTS_OK;
}

int lflts_source_add(lflts_ctx* c, int mesh_id, const int32_t* nodes, const double* weights, int64_t n,
                     int* source_id) {
  if (!c || !source_id || n < 1 || !nodes || !weights) return LFLTS_ERR_ARG;
  if (mesh_id < 0 || mesh_id >= (int)c->meshes.size()) return fail(c, LFLTS_ERR_ARG, "source_add: bad mesh_id");
  LF_TRY(set_device(c));
  const HostMesh& h = c->meshes[mesh_id]->h;
  std::vector<double> fw64(std::max<int64_t>(h.n_free, 1), 0.0);
  for (int64_t k = 0; k < n; ++k) {
    if (nodes[k] < 0 || nodes[k] >= h.n_nodes) return fail(c, LFLTS_ERR_ARG, "source_add: node out of range");
    if (!std::isfinite(weights[k])) return fail(c, LFLTS_ERR_ARG, "source_add: non-finite weight");
    const int32_t nn = h.old2new[nodes[k]];
    if (nn < h.n_free) fw64[nn] += weights[k] * h.minv[nn];  // M^-1 F; Dirichlet rows dropped
  }
  std::vector<float> fw32(fw64.begin(), fw64.end());
  Source src;
  src.mesh = mesh_id;
  LF_TRY(upload(c, &src.fw64, fw64.data(), fw64.size()));
  LF_TRY(upload(c, &src.fw32, fw32.data(), fw32.size()));
  *source_id = static_cast<int>(c->sources.size());
  c->sources.push_back(src);
  return LFLTS_OK;
}

int lflts_qoi_add(lflts_ctx* c, int mesh_id, const int32_t* idx, const double* g, int64_t nnz, int* qoi_id) {
  if (!c || !qoi_id || (nnz > 0 && (!idx || !g)) || nnz < 0 || nnz >= INT_MAX) return LFLTS_ERR_ARG;
  if (mesh_id < 0 || mesh_id >= (int)c->meshes.size()) return fail(c, LFLTS_ERR_ARG, "qoi_add: bad mesh_id");
  LF_TRY(set_device(c));
  const HostMesh& h = c->meshes[mesh_id]->h;
  std::vector<int32_t> nid(nnz);
  for (int64_t k = 0; k < nnz; ++k) {
    if (idx[k] < 0 || idx[k] >= h.n_nodes) return fail(c, LFLTS_ERR_ARG, "qoi_add: index out of range");
    if (!std::isfinite(g[k])) return fail(c, LFLTS_ERR_ARG, "qoi_add: non-finite weight");
    nid[k] = h.old2new[idx[k]];
  }
  Qoi q;
  q.mesh = mesh_id;
  q.nnz = static_cast<int>(nnz);
  LF_TRY(upload(c, &q.idx, nid.data(), nid.size()));
  LF_TRY(upload(c, &q.g, g, static_cast<size_t>(nnz)));
  *qoi_id = static_cast<int>(c->qois.size());
  c->qois.push_back(q);
  return LFLTS_OK;
}

int lflts_solve(lflts_ctx* c, const lflts_solve_desc* ds, const double* xi, int64_t S, double* Q, double* uN,
                int mem, void* stream) {
  if (!c) return LFLTS_ERR_ARG;
  c->err.clear();
  LF_TRY(set_device(c));
  LF_TRY(check_desc(c, ds));
  if (S < 1 || S > kMaxS) return fail(c, LFLTS_ERR_ARG, "solve: S must be in [1, 2097120]");
  if (!xi || !Q) return fail(c, LFLTS_ERR_ARG, "solve: null xi or Q");
  if (mem != LFLTS_MEM_HOST && mem != LFLTS_MEM_DEVICE) return fail(c, LFLTS_ERR_ARG, "solve: bad mem kind");
  const HostMesh& h = c->meshes[ds->mesh_id]->h;
  if (double(h.n_nodes) * double(S) >= 9.0e18) return fail(c, LFLTS_ERR_ARG, "solve: state too large");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Workspace& ws = workspace(c, 0);
  LF_TRY(reset_bad(c, st));
  if (mem == LFLTS_MEM_DEVICE) return solve_device(c, *ds, xi, S, Q, uN, ws, st);
  // host buffers: stage xi, run, copy results back, synchronise
  LF_TRY(ensure(c, ws.xraw, size_t(S) * h.K * sizeof(double)));
  LF_TRY(ensure(c, ws.Q, size_t(S) * sizeof(double)));
  if (uN) LF_TRY(ensure(c, ws.uN, size_t(h.n_nodes) * S * sizeof(double)));
  LF_CUDA(c, cudaMemcpyAsync(ws.xraw.p, xi, size_t(S) * h.K * sizeof(double), cudaMemcpyHostToDevice, st));
  LF_TRY(solve_device(c, *ds, static_cast<double*>(ws.xraw.p), S, static_cast<double*>(ws.Q.p),
                      uN ? static_cast<double*>(ws.uN.p) : nullptr, ws, st));
  LF_CUDA(c, cudaMemcpyAsync(Q, ws.Q.p, size_t(S) * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (uN) LF_CUDA(c, cudaMemcpyAsync(uN, ws.uN.p, size_t(h.n_nodes) * S * sizeof(double), cudaMemcpyDeviceToHost, st));
  return check_bad(c, st);
}

int lflts_level_sums(lflts_ctx* c, const double* Qf, const double* Qc, int64_t S, double* sums, int mem,
                     void* stream) {
  if (!c) return LFLTS_ERR_ARG;
  c->err.clear();
  LF_TRY(set_device(c));
  if (!Qf || !sums || S < 1) return fail(c, LFLTS_ERR_ARG, "level_sums: null array or S < 1");
  if (mem != LFLTS_MEM_HOST && mem != LFLTS_MEM_DEVICE) return fail(c, LFLTS_ERR_ARG, "level_sums: bad mem kind");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (mem == LFLTS_MEM_DEVICE) {
    Prof pr(c, st);
    k_level_sums<<<1, 256, 0, st>>>(S, Qf, Qc, sums);
    LF_CUDA(c, cudaGetLastError());
    pr.end(LFLTS_KERNEL_SUMS, double(S) * (Qc ? 16.0 : 8.0));
    return LFLTS_OK;
  }
  Workspace& ws = workspace(c, 0);
  LF_TRY(ensure(c, ws.Q, size_t(S) * 2 * sizeof(double)));
  double* dQf = static_cast<double*>(ws.Q.p);
  double* dQc = Qc ? dQf + S : nullptr;
  LF_CUDA(c, cudaMemcpyAsync(dQf, Qf, size_t(S) * sizeof(double), cudaMemcpyHostToDevice, st));
  if (Qc) LF_CUDA(c, cudaMemcpyAsync(dQc, Qc, size_t(S) * sizeof(double), cudaMemcpyHostToDevice, st));
  {
    Prof pr(c, st);
    k_level_sums<<<1, 256, 0, st>>>(S, dQf, dQc, c->d_scratch);
    LF_CUDA(c, cudaGetLastError());
    pr.end(LFLTS_KERNEL_SUMS, double(S) * (Qc ? 16.0 : 8.0));
  }
  LF_CUDA(c, cudaMemcpyAsync(sums, c->d_scratch, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  LF_CUDA(c, cudaStreamSynchronize(st));
  return LFLTS_OK;
}

int lflts_run_pairs(lflts_ctx* c, const lflts_pair_job* jobs, int n_jobs, int mem, void* stream) {
  return lflts_run_pairs_slice(c, jobs, n_jobs, mem, 0, 1, stream);
}

int lflts_run_pairs_slice(lflts_ctx* c, const lflts_pair_job* jobs, int n_jobs, int mem, int slice, int n_slices,
                          void* stream) {
  if (!c) return LFLTS_ERR_ARG;
  c->err.clear();
  LF_TRY(set_device(c));
  if (!jobs || n_jobs < 1 || (mem != LFLTS_MEM_HOST && mem != LFLTS_MEM_DEVICE)) {
    c->run.reset();
    return fail(c, LFLTS_ERR_ARG, "run_pairs: no jobs or bad mem kind");
  }
  if (n_slices < 1 || slice < 0 || slice >= n_slices) {
    c->run.reset();
    return fail(c, LFLTS_ERR_ARG, "run_pairs_slice: need 0 <= slice < n_slices");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t sig = jobs_signature(jobs, n_jobs, mem, n_slices);
  if (slice == 0) {
    c->run.reset();  // a new run replaces one left unfinished
    std::unique_ptr<PairRun> run(new PairRun());
    LF_TRY(pairs_start(c, *run, jobs, n_jobs, mem, n_slices, st));
    run->sig = sig;
    c->run = std::move(run);
  } else if (!c->run || c->run->sig != sig || c->run->next != slice) {
    c->run.reset();
    return fail(c, LFLTS_ERR_ARG,
                "run_pairs_slice: slice " + std::to_string(slice) +
                    " does not continue the run in progress (same jobs, memory kind and n_slices, slices in order)");
  }
  PairRun& run = *c->run;
  const int rc = pairs_advance(c, run, slice, st);
  if (rc) {
    c->run.reset();
    return rc;
  }
  run.next = slice + 1;
  if (slice + 1 < n_slices) {
    if (mem == LFLTS_MEM_HOST) LF_CUDA(c, cudaStreamSynchronize(st));
    return LFLTS_OK;
  }
  const int rf = pairs_finish(c, run, jobs, n_jobs, mem, st);
  c->run.reset();
  return rf;
}

int lflts_field_interp_add(lflts_ctx* c, int mesh_f, int mesh_c, const int32_t* vert, const double* w,
                           int* interp_id) {
  if (!c || !vert || !w || !interp_id) return LFLTS_ERR_ARG;
  c->err.clear();
  LF_TRY(set_device(c));
  const int nm = static_cast<int>(c->meshes.size());
  if (mesh_f < 0 || mesh_f >= nm || mesh_c < 0 || mesh_c >= nm)
    return fail(c, LFLTS_ERR_ARG, "field_interp_add: bad mesh id");
  const int64_t n_f = c->meshes[mesh_f]->h.n_nodes, n_c = c->meshes[mesh_c]->h.n_nodes;
  for (int64_t k = 0; k < 3 * n_f; ++k) {
    if (vert[k] < 0 || vert[k] >= n_c) return fail(c, LFLTS_ERR_ARG, "field_interp_add: vertex out of range");
    if (!std::isfinite(w[k])) return fail(c, LFLTS_ERR_ARG, "field_interp_add: non-finite weight");
  }
  Interp in;
  in.mesh_f = mesh_f;
  in.mesh_c = mesh_c;
  LF_TRY(upload(c, &in.vert, vert, size_t(3 * n_f)));
  LF_TRY(upload(c, &in.w, w, size_t(3 * n_f)));
  *interp_id = static_cast<int>(c->interps.size());
  c->interps.push_back(in);
  return LFLTS_OK;
}

int lflts_run_field_pair(lflts_ctx* c, const lflts_pair_job* jb, int interp_id, double* sum_dU, double* norm2,
                         double* sum_norm2, int mem, void* stream) {
  if (!c) return LFLTS_ERR_ARG;
  c->err.clear();
  LF_TRY(set_device(c));
  if (!jb || !jb->xi || jb->S < 1 || jb->S > kMaxS || !sum_dU || !sum_norm2)
    return fail(c, LFLTS_ERR_ARG, "run_field_pair: null job, xi, sum_dU or sum_norm2, or S out of range");
  if (mem != LFLTS_MEM_HOST && mem != LFLTS_MEM_DEVICE) return fail(c, LFLTS_ERR_ARG, "run_field_pair: bad mem kind");
  LF_TRY(check_desc(c, &jb->fine));
  if (c->meshes[jb->fine.mesh_id]->h.moving)
    return fail(c, LFLTS_ERR_ARG, "run_field_pair: the L2(D) norm on a moving mesh is not supported");
  const Interp* in = nullptr;
  if (jb->has_coarse) {
    LF_TRY(check_desc(c, &jb->coarse));
    if (interp_id < 0 || interp_id >= (int)c->interps.size() || c->interps[interp_id].mesh_f != jb->fine.mesh_id ||
        c->interps[interp_id].mesh_c != jb->coarse.mesh_id)
      return fail(c, LFLTS_ERR_ARG, "run_field_pair: interp_id does not map the coarse mesh to the fine mesh");
    if (c->meshes[jb->coarse.mesh_id]->h.K != c->meshes[jb->fine.mesh_id]->h.K)
      return fail(c, LFLTS_ERR_ARG, "run_field_pair: fine and coarse meshes have different K");
    in = &c->interps[interp_id];
  }
  const int64_t S = jb->S;
  MeshGPU& mf = *c->meshes[jb->fine.mesh_id];
  const HostMesh& hf = mf.h;
  const int64_t n_f = hf.n_nodes;
  const int64_t n_c = in ? c->meshes[jb->coarse.mesh_id]->h.n_nodes : 0;
  if (!mf.tri_dev) {
    LF_TRY(upload(c, &mf.tri_dev, hf.tri.data(), hf.tri.size()));
    LF_TRY(upload(c, &mf.area_dev, hf.area.data(), hf.area.size()));
  }
  for (auto& w : c->fws)
    if (!w) w.reset(new Workspace());
  if (!c->fb) c->fb.reset(new FieldBufs());
  FieldBufs& fb = *c->fb;
  const int chunk = 512;
  const int64_t n_chunks = std::max<int64_t>(1, (hf.n_tri + chunk - 1) / chunk);
  const int K = hf.K;
  LF_TRY(ensure(c, fb.uf, size_t(n_f) * S * sizeof(double)));
  if (in) LF_TRY(ensure(c, fb.uc, size_t(n_c) * S * sizeof(double)));
  LF_TRY(ensure(c, fb.qf, size_t(S) * sizeof(double)));
  LF_TRY(ensure(c, fb.qc, size_t(S) * sizeof(double)));
  LF_TRY(ensure(c, fb.s1, size_t(n_f) * sizeof(double)));
  LF_TRY(ensure(c, fb.n2, size_t(S) * sizeof(double)));
  LF_TRY(ensure(c, fb.ps, size_t(n_chunks) * S * sizeof(double)));
  LF_TRY(ensure(c, fb.pc, size_t(n_chunks) * S * sizeof(double)));
  LF_TRY(ensure(c, fb.sums, 4 * sizeof(double)));
  LF_TRY(ensure(c, fb.dq, size_t(S) * 2 * sizeof(double) + 4 * sizeof(double)));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LF_TRY(reset_bad(c, st));
  const double* d_xi = jb->xi;
  if (mem == LFLTS_MEM_HOST) {
    LF_TRY(ensure(c, fb.xraw, size_t(S) * K * sizeof(double)));
    LF_CUDA(c, cudaMemcpyAsync(fb.xraw.p, jb->xi, size_t(S) * K * sizeof(double), cudaMemcpyHostToDevice, st));
    d_xi = static_cast<const double*>(fb.xraw.p);
  }
  double* uf = static_cast<double*>(fb.uf.p);
  double* uc = in ? static_cast<double*>(fb.uc.p) : nullptr;
  double* qf = static_cast<double*>(fb.qf.p);
  double* qc = static_cast<double*>(fb.qc.p);
  // the pair's solves with their final states gathered in the caller's node order (FP64)
  LF_TRY(solve_device(c, jb->fine, d_xi, S, qf, uf, *c->fws[0], st));
  if (in) LF_TRY(solve_device(c, jb->coarse, d_xi, S, qc, uc, *c->fws[1], st));
  // dU = u_l - I u_{l-1} in place over uf, per-node sums over the draws
  {
    Prof pr(c, st);
    const unsigned nb = static_cast<unsigned>((n_f + 7) / 8);
    k_field_diff<<<nb, 256, 0, st>>>(n_f, (int)S, uf, uc, in ? in->vert : nullptr, in ? in->w : nullptr,
                                     static_cast<double*>(fb.s1.p));
    LF_CUDA(c, cudaGetLastError());
    const int tb = static_cast<int>(std::min<int64_t>(S, 128));
    k_field_norm_partial<<<dim3(static_cast<unsigned>(n_chunks), static_cast<unsigned>((S + tb - 1) / tb)), tb, 0,
                           st>>>(hf.n_tri, (int)S, chunk, mf.tri_dev, mf.area_dev, uf, static_cast<double*>(fb.ps.p),
                                 static_cast<double*>(fb.pc.p));
    LF_CUDA(c, cudaGetLastError());
    k_qoi_final<<<blocks_for(S, 128, 1 << 20), 128, 0, st>>>((int)n_chunks, (int)S, static_cast<double*>(fb.ps.p),
                                                            static_cast<double*>(fb.pc.p),
                                                            static_cast<double*>(fb.n2.p), c->d_bad);
    LF_CUDA(c, cudaGetLastError());
    k_level_sums<<<1, 256, 0, st>>>(S, static_cast<double*>(fb.n2.p), nullptr, static_cast<double*>(fb.sums.p));
    LF_CUDA(c, cudaGetLastError());
    pr.end(LFLTS_KERNEL_QOI, 8.0 * double(S) * (2.0 * n_f + 3.0 * n_c + 3.0 * hf.n_tri));
    c->launches += 3;
  }
  // the scalar QoI of the same solves (dQ, Qf and level sums), when asked for
  double* dq_buf = static_cast<double*>(fb.dq.p);
  if (jb->dQ || jb->Qf || jb->sums) {
    k_pair_diff<<<blocks_for(S, 128, 1 << 20), 128, 0, st>>>((int)S, qf, in ? qc : nullptr, dq_buf, dq_buf + S);
    LF_CUDA(c, cudaGetLastError());
    k_level_sums<<<1, 256, 0, st>>>(S, qf, in ? qc : nullptr, dq_buf + 2 * S);
    LF_CUDA(c, cudaGetLastError());
    c->launches += 2;
  }
  const cudaMemcpyKind kind = mem == LFLTS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  LF_CUDA(c, cudaMemcpyAsync(sum_dU, fb.s1.p, size_t(n_f) * sizeof(double), kind, st));
  LF_CUDA(c, cudaMemcpyAsync(sum_norm2, fb.sums.p, sizeof(double), kind, st));
  if (norm2) LF_CUDA(c, cudaMemcpyAsync(norm2, fb.n2.p, size_t(S) * sizeof(double), kind, st));
  if (jb->dQ) LF_CUDA(c, cudaMemcpyAsync(jb->dQ, dq_buf, size_t(S) * sizeof(double), kind, st));
  if (jb->Qf) LF_CUDA(c, cudaMemcpyAsync(jb->Qf, dq_buf + S, size_t(S) * sizeof(double), kind, st));
  if (jb->sums) LF_CUDA(c, cudaMemcpyAsync(jb->sums, dq_buf + 2 * S, 4 * sizeof(double), kind, st));
  if (mem == LFLTS_MEM_HOST) return check_bad(c, st);
  return LFLTS_OK;
}

int lflts_grad_xi(lflts_ctx* c, const lflts_solve_desc* ds, const double* xi, int64_t S, int ckpt_every,
                  double* Q, double* dQdxi, int mem, void* stream) {
  if (!c) return LFLTS_ERR_ARG;
  c->err.clear();
  LF_TRY(set_device(c));
  LF_TRY(check_desc(c, ds));
  if (c->meshes[ds->mesh_id]->h.moving)
    return fail(c, LFLTS_ERR_ARG, "grad_xi: the gradient on a moving mesh is not supported");
  if (ds->p > 64) return fail(c, LFLTS_ERR_ARG, "grad_xi: p must be in [1, 64]");
  if (S < 1 || S > kMaxS) return fail(c, LFLTS_ERR_ARG, "grad_xi: S must be in [1, 2097120]");
  if (!xi || !Q || !dQdxi) return fail(c, LFLTS_ERR_ARG, "grad_xi: null xi, Q or dQdxi");
  if (ckpt_every < 1) return fail(c, LFLTS_ERR_ARG, "grad_xi: ckpt_every must be >= 1");
  if (mem != LFLTS_MEM_HOST && mem != LFLTS_MEM_DEVICE) return fail(c, LFLTS_ERR_ARG, "grad_xi: bad mem kind");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const HostMesh& h = c->meshes[ds->mesh_id]->h;
  LF_TRY(reset_bad(c, st));
  if (mem == LFLTS_MEM_DEVICE) return grad_device(c, *ds, xi, S, ckpt_every, Q, dQdxi, st);
  if (!c->gb) c->gb.reset(new GradBufs());
  GradBufs& gb = *c->gb;
  LF_TRY(ensure(c, gb.xraw, size_t(S) * h.K * sizeof(double)));
  LF_TRY(ensure(c, gb.Q, size_t(S) * sizeof(double)));
  LF_TRY(ensure(c, gb.G, size_t(S) * h.K * sizeof(double)));
  LF_CUDA(c, cudaMemcpyAsync(gb.xraw.p, xi, size_t(S) * h.K * sizeof(double), cudaMemcpyHostToDevice, st));
  LF_TRY(grad_device(c, *ds, static_cast<double*>(gb.xraw.p), S, ckpt_every, static_cast<double*>(gb.Q.p),
                     static_cast<double*>(gb.G.p), st));
  LF_CUDA(c, cudaMemcpyAsync(Q, gb.Q.p, size_t(S) * sizeof(double), cudaMemcpyDeviceToHost, st));
  LF_CUDA(c, cudaMemcpyAsync(dQdxi, gb.G.p, size_t(S) * h.K * sizeof(double), cudaMemcpyDeviceToHost, st));
  return check_bad(c, st);
}

int lflts_profile_enable(lflts_ctx* c, int on) {
  if (!c) return LFLTS_ERR_ARG;
  c->profiling = on != 0;
  return LFLTS_OK;
}

static int drain(lflts_ctx* c) {
  if (c->pending.empty()) return 0;
  LF_TRY(set_device(c));
  LF_CUDA(c, cudaDeviceSynchronize());
  for (auto& r : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.cls] += ms;
      c->prof_bytes[r.cls] += r.bytes;
      c->prof_launches[r.cls] += 1;
    }
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->pending.clear();
  return 0;
}

int lflts_profile_reset(lflts_ctx* c) {
  if (!c) return LFLTS_ERR_ARG;
  LF_TRY(drain(c));
  for (int k = 0; k < LFLTS_KERNEL_CLASSES; ++k) {
    c->prof_launches[k] = 0;
    c->prof_ms[k] = 0;
    c->prof_bytes[k] = 0;
  }
  return LFLTS_OK;
}

int lflts_profile_read(lflts_ctx* c, int cls, int64_t* launches, double* ms, double* bytes) {
  if (!c || cls < 0 || cls >= LFLTS_KERNEL_CLASSES) return LFLTS_ERR_ARG;
  LF_TRY(drain(c));
  if (launches) *launches = c->prof_launches[cls];
  if (ms) *ms = c->prof_ms[cls];
  if (bytes) *bytes = c->prof_bytes[cls];
  return LFLTS_OK;
}

int lflts_set_option(lflts_ctx* c, int option, int64_t value) {
  if (!c) return LFLTS_ERR_ARG;
  switch (option) {
    case LFLTS_OPT_GRAPHS: c->graphs = value != 0; return LFLTS_OK;
    case LFLTS_OPT_AUTOTUNE: c->autotune = value != 0; return LFLTS_OK;
    case LFLTS_OPT_FUSED_INNER:
      if (value < 0 || value > 2) return fail(c, LFLTS_ERR_ARG, "set_option: fused inner mode must be 0, 1 or 2");
      c->fused_mode = static_cast<int>(value);
      for (auto& m : c->meshes) m->tuned.clear();  // re-tune with the new candidate set
      return LFLTS_OK;
    case LFLTS_OPT_PAIRED_INNER:
      if (value < 0 || value > 4) return fail(c, LFLTS_ERR_ARG, "set_option: paired inner mode must be 0..4");
      c->pair_mode = static_cast<int>(value);
      for (auto& m : c->meshes) m->tuned.clear();
      return LFLTS_OK;
    case LFLTS_OPT_PAIR_BLOCK:
      if (value < 16 || value > 4096)
        return fail(c, LFLTS_ERR_ARG, "set_option: paired-substep block must be 16..4096 nodes");
      c->pair_block = static_cast<int>(value);
      for (auto& m : c->meshes) m->tuned.clear();
      return LFLTS_OK;
    case LFLTS_OPT_COARSE_RC:
      if (value < 0 || value > 2) return fail(c, LFLTS_ERR_ARG, "set_option: coarse weight mode must be 0, 1 or 2");
      c->coarse_rc = static_cast<int>(value);
      for (auto& m : c->meshes) {
        m->tuned.clear();
        m->tuned_rc.clear();
      }
      return LFLTS_OK;
    case LFLTS_OPT_PAIR_MIN_R:
      if (value < 0) return fail(c, LFLTS_ERR_ARG, "set_option: paired-substep minimum |R| must be >= 0");
      c->pair_min_r = value;
      for (auto& m : c->meshes) m->tuned.clear();
      return LFLTS_OK;
    case LFLTS_OPT_GRAPH_CACHE:
      if (value < 1) return fail(c, LFLTS_ERR_ARG, "set_option: graph cache must hold at least 1 graph");
      c->graph_cap = value;
      return LFLTS_OK;
    case LFLTS_OPT_TILED_INNER:
      if (value < 0 || value > 2) return fail(c, LFLTS_ERR_ARG, "set_option: tiled inner mode must be 0, 1 or 2");
      c->tile_mode = static_cast<int>(value);
      for (auto& m : c->meshes) m->tuned.clear();
      return LFLTS_OK;
    case LFLTS_OPT_TILE_CAP:
      if (value < 0 || (value > 0 && value < 16))
        return fail(c, LFLTS_ERR_ARG, "set_option: tile capacity must be 0 or at least 16");
      c->tile_cap = value;
      for (auto& m : c->meshes) m->tuned.clear();
      return LFLTS_OK;
    default: return fail(c, LFLTS_ERR_ARG, "set_option: unknown option");
  }
}

int lflts_get_stats(lflts_ctx* c, int64_t out[4]) {
  if (!c || !out) return LFLTS_ERR_ARG;
  out[0] = c->launches;
  out[1] = c->graph_launches;
  out[2] = c->tune_launches;
  out[3] = 0;
  for (auto& m : c->meshes) out[3] += static_cast<int64_t>(m->tuned.size());
  return LFLTS_OK;
}

int lflts_graph_cache_size(lflts_ctx* c, int64_t* n) {
  if (!c || !n) return LFLTS_ERR_ARG;
  int64_t k = 0;
  for (auto& w : c->ws) k += static_cast<int64_t>(w->graphs.size());
  for (auto& w : c->fws)
    if (w) k += static_cast<int64_t>(w->graphs.size());
  if (c->gws) k += static_cast<int64_t>(c->gws->graphs.size());
  *n = k;
  return LFLTS_OK;
}

int lflts_launch_count(lflts_ctx* c, int64_t* launches) {
  if (!c || !launches) return LFLTS_ERR_ARG;
  *launches = c->launches;
  return LFLTS_OK;
}

}  // extern "C"
