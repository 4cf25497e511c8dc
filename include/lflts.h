/*
 * lflts.h -- C ABI of the GB300 library for MLMC with stabilised leapfrog
 * local time-stepping (LF-LTS) of the mass-lumped P1 wave equation.
 *
 * Method: Grote, Michel, Nobile, "Uncertainty quantification by MLMC and
 * local time-stepping for wave propagation" (arXiv 2106.11117).
 *   - model problem u_tt - div(c^2(x,w) grad u) = 0, u(0) = u0, u_t(0) = v0,
 *     homogeneous Dirichlet boundary (Sec. 2.1, Eq. Wave_hd);
 *   - P1 elements, lumped mass M, stiffness K(w) (Sec. 3.1);
 *   - stabilised LF-LTS with the diagonal 0/1 mask P, ratio p and
 *     stabilisation nu (Sec. 3.3, Alg. 2), leapfrog when p = 1 or P = 0
 *     (Eq. LF2scheme);
 *   - QoI Q(w) = sum_k g_k u_h(x_k, T, w), a linear functional (Sec. 2.1);
 *   - MLMC level sums for the estimator and variance (Sec. 2.2, Eqs.
 *     MLMCestimator and Vell_est); fine/coarse pairs share one draw.
 *
 * Conventions
 *   - Every call returns an lflts_status (0 = success, < 0 = error).  On error
 *     lflts_last_error(ctx) returns a message owned by the context, valid
 *     until the next call on that context.
 *   - Host arrays passed in are owned by the caller and copied before the
 *     call returns.  Device arrays are owned by the caller.
 *   - mem = LFLTS_MEM_HOST: xi and outputs are host pointers; the call copies
 *     xi to the device, runs on `stream` and synchronises the stream before
 *     returning.  mem = LFLTS_MEM_DEVICE: xi and outputs are device pointers of
 *     the context's device; the call only enqueues work on `stream` and
 *     returns (outputs are ready when the stream reaches that point).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).
 *   - A context belongs to one host thread at a time; it owns all device
 *     memory it allocates (meshes, fields, workspaces) and frees it in
 *     lflts_destroy.
 *   - Random coefficients: the field is c_e^2 = exp(sum_k xi_k psi[e][k]) on
 *     each triangle e (the random field evaluated at one quadrature point per
 *     element).  xi is row-major [S][K] FP64, one row per sample.
 */
#ifndef LFLTS_H
#define LFLTS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lflts_ctx lflts_ctx;

typedef enum {
  LFLTS_OK = 0,
  LFLTS_ERR_ARG = -1,      /* invalid argument (sizes, ids, pointers)          */
  LFLTS_ERR_OOM = -2,      /* device or host allocation failed                 */
  LFLTS_ERR_CUDA = -3,     /* a CUDA runtime call failed (message has details) */
  LFLTS_ERR_UNSTABLE = -4, /* a sample produced a non-finite QoI               */
  LFLTS_ERR_TIMEOUT = -5,  /* a bounded device-side wait gave up               */
  LFLTS_ERR_MESH = -6      /* invalid mesh (index range, orientation, masks)   */
} lflts_status;

enum { LFLTS_MEM_HOST = 0, LFLTS_MEM_DEVICE = 1 };

/* Kernel classes for lflts_profile_read (timing and algorithmic bytes). */
enum {
  LFLTS_KERNEL_INIT = 0,   /* state initialisation from u0, v0              */
  LFLTS_KERNEL_COARSE = 1, /* w-part: full apply M^-1 K u_n + update off R  */
  LFLTS_KERNEL_INNER = 2,  /* one inner LTS substep on R (Alg. 2 loop)      */
  LFLTS_KERNEL_QOI = 3,    /* QoI reduction (both stages)                   */
  LFLTS_KERNEL_SUMS = 4,   /* MLMC level sums                               */
  LFLTS_KERNEL_ADJ_INNER = 5, /* lflts_grad_xi: recomputed a(u_n) and r_2..r_{p-1} on R and the
                                 adjoint inner recursion rho_{p-1}..rho_1                 */
  LFLTS_KERNEL_ADJ_EDGES = 6, /* lflts_grad_xi: per-edge FP64 accumulation of the gradient    */
  LFLTS_KERNEL_GRAD = 7,      /* lflts_grad_xi: adjoint seed and the contraction with dK/dxi */
  LFLTS_KERNEL_INNER_PAIR = 8, /* two inner LTS substeps on R in one launch (Alg. 2 loop)   */
  LFLTS_KERNEL_CLASSES = 9
};

/* Options for lflts_set_option. */
enum {
  LFLTS_OPT_GRAPHS = 1,   /* 1 (default): solves on a non-default stream are captured once into a
                             CUDA graph and replayed while problem, batch and buffers are unchanged */
  LFLTS_OPT_AUTOTUNE = 2, /* 1 (default): the first solve of a (mesh, S, precision, p) times the
                             candidate launch shapes (draws per thread, CTAs per SM, register cap)
                             and keeps the best */
  LFLTS_OPT_FUSED_INNER = 5,  /* all p-1 inner substeps of a step in one launch, with R's recursion,
                                 coupling slots, their edge weights and 1/m for a CTA's draws in
                                 shared memory (only where they fit in 200 KB; same results bit for
                                 bit): 0 never; 1 (default) autotuned, and always where it fits and
                                 |R| <= 2048; 2 always where it fits */
  LFLTS_OPT_TILED_INNER = 6,  /* all p-1 inner substeps of a step in one launch for a large R: tiles of
                                 R (a compact core plus p-1 layers of P nodes, recomputed by the
                                 neighbouring tiles) with each node's state in registers and r_m in
                                 shared memory; same results bit for bit, uniform batches only:
                                 0 never; 1 (default) autotuned where |R| > 2048; 2 always */
  LFLTS_OPT_TILE_CAP = 7,     /* 0 (default): tiles as large as the kernel's registers allow; n >= 16:
                                 at most n computed nodes per tile (more, smaller tiles) */
  LFLTS_OPT_GRAPH_CACHE = 8,  /* instantiated solve graphs kept per workspace (default 8, >= 1); a
                                 new graph beyond it first synchronises the stream and destroys the
                                 least recently used ones (an adaptive MLMC run changes its batch
                                 sizes every iteration) */
  LFLTS_OPT_PAIRED_INNER = 9, /* inner substeps two by two in one launch for a large R: blocks of R
                                 (square cells plus a halo of their P neighbours) with r_{m+1}
                                 exchanged in shared memory; same results bit for bit, uniform
                                 batches only; with an odd number of substeps the first runs alone:
                                 0 never; 1 (default) autotuned where |R| > 2048 (4 draws per thread
                                 in FP32, 2 in FP64); always where the blocks fit in shared memory
                                 with 2: 4 draws per thread in FP32, 2 in FP64; 3: 2; 4: 1 */
  LFLTS_OPT_PAIR_BLOCK = 10,  /* about this many nodes of R per block of the paired substeps,
                                 16..4096 (default 144); blocks whose rows do not fit in the shared
                                 memory of a CTA make the batch run one launch per substep */
  LFLTS_OPT_PAIR_MIN_R = 11,  /* with LFLTS_OPT_PAIRED_INNER >= 2: forced only on meshes with at least
                                 this many nodes of R (default 0: every mesh); fixes the shapes a
                                 profiler run uses without timing them */
  LFLTS_OPT_COARSE_RC = 12    /* the coarse launch forms the coupling weights it needs from xi and
                                 the field basis (Sec. 3.2: the field at the quadrature points is
                                 a lower-order cost) instead of reading the stored per-draw weights;
                                 same values bit for bit; uniform batches of fixed meshes with at
                                 most four table neighbours: 0 (default) never, because on GB300
                                 it measured 3x slower than reading the stored weights (issue-bound:
                                 eight exp2 and 72 FMA per node and draw); 1 timed against the
                                 stored weights; 2 always where it applies */
};

/* Library version (major*10000 + minor*100 + patch). */
int lflts_version(void);

/* Create a context on CUDA device `device` (or -1: a host-only context that
 * can prepare meshes but not solve).  *out receives the handle.
 * Errors: LFLTS_ERR_ARG for out == NULL; LFLTS_ERR_CUDA if the device does not exist or cannot be
 * selected; LFLTS_ERR_OOM if its small fixed device buffers cannot be allocated. */
int lflts_create(lflts_ctx** out, int device);

/* Free every device buffer and stream of the context, then the context.
 * Errors: none (a NULL context is accepted and ignored). */
int lflts_destroy(lflts_ctx* ctx);

/* Last error message of the context (never NULL; "" after success). */
const char* lflts_last_error(const lflts_ctx* ctx);

/*
 * Register a P1 triangle mesh with its LTS mask and random-field basis
 * (Sec. 3.1 discretisation; Sec. 3.3 mask P).
 *   xy        [n_nodes][2] FP64 node coordinates
 *   tri       [n_tri][3] int32 vertex indices, counter-clockwise
 *   dirichlet [n_nodes] 0/1, 1 = homogeneous Dirichlet node (u = 0)
 *   P         [n_nodes] 0/1, the diagonal of P (refined region and the
 *             elements adjacent to it); entries on Dirichlet nodes ignored;
 *             may be NULL (P = 0, plain leapfrog)
 *   psi       [n_tri][K] FP64 field basis at the element quadrature point
 *   K         number of field terms, 1 <= K <= 16
 * The library reorders the nodes internally; every nodal array crossing the
 * ABI uses the caller's node order.  Errors: LFLTS_ERR_MESH for indices out
 * of range or a triangle with non-positive signed area.
 */
int lflts_mesh_add(lflts_ctx* ctx, const double* xy, int64_t n_nodes,
                   const int32_t* tri, int64_t n_tri, const uint8_t* dirichlet,
                   const uint8_t* P, const double* psi, int K, int* mesh_id);

/*
 * Register a mesh whose vertices move with the draw (Sec. 4.3): every draw is
 * solved on this reference triangulation with vertex v moved to
 *   x_v + sum_k xi_k D_k(v)
 * (Eq. MeshTransform applied to the vertices; xi_k the draw's entries of the
 * xi array a solve receives, K of them), with wave speed c = 1 and the
 * stiffness and lumped mass of the moved mesh (Eq. waveeq_transformed): the
 * solve forms, per draw and adjacency entry, K_ij / m_i of the moved
 * elements.  Arguments as lflts_mesh_add, with
 *   disp      [K][n_nodes][2] FP64 displacement modes D_k in the caller's
 *             node order (copied)
 *   K         number of modes, 1 <= K <= 16
 * Every edge of the reference mesh is kept (a zero stiffness entry of the
 * reference, such as the diagonal of a right triangle, is not zero once the
 * vertices move).  Not supported on such a mesh: point sources,
 * lflts_grad_xi and lflts_run_field_pair (LFLTS_ERR_ARG).  A draw that folds
 * an element over (non-positive moved area) gives meaningless values; the
 * caller keeps the modes and draws within the map's range.
 * Errors: as lflts_mesh_add; LFLTS_ERR_ARG for disp == NULL or K outside
 * [1, 16].
 */
int lflts_mesh_add_moving(lflts_ctx* ctx, const double* xy, int64_t n_nodes,
                          const int32_t* tri, int64_t n_tri, const uint8_t* dirichlet,
                          const uint8_t* P, const double* disp, int K, int* mesh_id);

/*
 * Sizes of a registered mesh: info[0] n_nodes, [1] n_free (non-Dirichlet),
 * [2] n_R (nodes the inner substeps update: P and its element neighbours),
 * [3] n_P, [4] n_tri, [5] K, [6] n_edges (edges with a nonzero stiffness
 * entry and a free endpoint), [7] n_edges_P (those with an endpoint in P).
 * Errors: LFLTS_ERR_ARG for a NULL context or info, or an unknown mesh_id.
 */
int lflts_mesh_info(lflts_ctx* ctx, int mesh_id, int64_t info[8]);

/*
 * Internal node order of a mesh: new2old [n_nodes] receives, for each
 * internal position k, the caller's node index.  The order is
 * [P nodes | R \ P | other free nodes | Dirichlet nodes], each group in
 * Morton (Z-curve) order of the node coordinates, ties in the caller's order.
 * Works on host-only contexts (device -1).
 * Errors: LFLTS_ERR_ARG for a NULL context or output, or an unknown mesh_id.
 */
int lflts_mesh_order(lflts_ctx* ctx, int mesh_id, int32_t* new2old);

/*
 * Constants of the stabilised scheme (Sec. 3.3) as the library uses them,
 * computed on the host in FP64 (no device needed):
 *   out[0] delta = 1 + nu/p^2, out[1] omega = 2 T_p'(delta)/T_p(delta),
 *   out[2] c0 = dt^2/(omega delta) (first substep, u-form),
 *   out[3] gamma (the factor of the leapfrog update away from P, dt^2/2 in
 *   exact arithmetic), then for m = 1..p-1:
 *   out[4+2(m-1)] beta_m = T_{m-1}/T_{m+1},
 *   out[5+2(m-1)] c_m = 2 dt^2 beta_{m+1/2} / omega.
 * out must hold 4 + 2(p-1) doubles.
 * Errors: LFLTS_ERR_ARG for out == NULL, p outside [1, 128], nu outside [0, 1] or dt <= 0.
 */
int lflts_lts_constants(int p, double nu, double dt, double* out);

/*
 * Nodal interpolation between two meshes of one domain (host only; no
 * context or device): for every node k of the fine mesh, xy_f[2k..2k+1]
 * (caller's numbering), the vertices vert[3k..3k+2] of a triangle of the
 * coarse mesh (xy_c [n_c][2], tri_c [n_tri_c][3], caller's numbering) that
 * contains it and its barycentric coordinates w[3k..3k+2] (they sum to 1),
 * so that the coarse P1 function u_c takes the value
 * sum_a w[3k+a] u_c[vert[3k+a]] there.  This forms dQ_l = u_l - I u_{l-1}
 * of the L2(D)-valued QoI u(., T) (Sec. 4) on the finer mesh of a pair.
 * Caller-owned buffers: vert [n_f][3] int32, w [n_f][3] FP64.
 * Errors: LFLTS_ERR_ARG for null pointers, sizes below 1 or vertex ids
 * outside [0, n_c); LFLTS_ERR_MESH if some fine node lies outside every
 * coarse triangle (a barycentric coordinate below -1e-10).
 */
int lflts_interp_weights(const double* xy_c, int64_t n_c, const int32_t* tri_c, int64_t n_tri_c,
                         const double* xy_f, int64_t n_f, int32_t* vert, double* w);

/*
 * Register a nodal field (initial displacement u0 or velocity v0, Sec. 2.1)
 * on a mesh: values [n_nodes] FP64 in the caller's node order; values on
 * Dirichlet nodes are replaced by 0.
 * Errors: LFLTS_ERR_ARG for NULL pointers, an unknown mesh_id or a non-finite value;
 * LFLTS_ERR_OOM / LFLTS_ERR_CUDA from the upload.
 */
int lflts_field_add(lflts_ctx* ctx, int mesh_id, const double* values, int* field_id);

/*
 * Register a load vector F (the space part of the forcing f(x,t) =
 * r(t) f(x), F_i = (f, phi_i); a point source at x_s has F_i = phi_i(x_s)) on
 * a mesh: nodes [n] node indices, weights [n] FP64.  It enters Alg. 2 through
 * w_n = A (I - P) z_n - F~(t_n), frozen over the inner substeps of a step.
 * Errors: LFLTS_ERR_ARG for NULL pointers, n < 1, an unknown mesh_id, a node outside the mesh
 * or a non-finite weight; LFLTS_ERR_OOM / LFLTS_ERR_CUDA from the upload.
 */
int lflts_source_add(lflts_ctx* ctx, int mesh_id, const int32_t* nodes, const double* weights,
                     int64_t n, int* source_id);

/*
 * Register a linear QoI Q(u) = sum_k g[k] u[idx[k]] on a mesh (Sec. 2.1,
 * V = R).  idx [nnz] int32 node indices, g [nnz] FP64 weights.
 * Errors: LFLTS_ERR_ARG for NULL pointers (with nnz > 0), nnz < 0, an unknown mesh_id, an
 * index outside the mesh or a non-finite weight; LFLTS_ERR_OOM / LFLTS_ERR_CUDA from the upload.
 */
int lflts_qoi_add(lflts_ctx* ctx, int mesh_id, const int32_t* idx,
                  const double* g, int64_t nnz, int* qoi_id);

/* One level solve: the problem statement of Alg. 2 for a batch of draws. */
typedef struct {
  int mesh_id;      /* mesh from lflts_mesh_add                                */
  int qoi_id;       /* QoI from lflts_qoi_add on the same mesh                 */
  int u0_field;     /* initial displacement, field id on the same mesh        */
  int v0_field;     /* initial velocity field id, or -1 for v0 = 0            */
  int precision;    /* 32: FP32 state, FP64 QoI; 64: FP64 throughout          */
  int p;            /* LTS ratio, 1 <= p <= 128 (p = 1: leapfrog; the fused
                       and tiled inner kernels and lflts_grad_xi take
                       p <= 64).  Rounding in the inner recursion grows
                       about like p^2: with precision 32 the QoI is within
                       1e-5 of its scale up to p of about 100 and 2e-5 at
                       p = 128                                                */
  double nu;        /* stabilisation parameter, 0 <= nu <= 1                  */
  double dt;        /* coarse time step                                       */
  int64_t n_steps;  /* N >= 1 steps; the QoI is taken at t_N = N dt           */
  int source_id;    /* load vector from lflts_source_add, or -1 (f = 0)       */
  double src_f0;    /* Ricker wavelet of the source: F(t) = amp r(t) F,       */
  double src_t0;    /*   r(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2) */
  double src_amp;
} lflts_solve_desc;

/*
 * Solve the semidiscrete wave equation for S draws with stabilised LF-LTS
 * (Alg. 2; start z_1 = q_1(z_0) + dt M^{1/2} v0) and evaluate the QoI at t_N.
 *   xi   [S][K] FP64 draws (host or device per `mem`)
 *   Q    [S] FP64 output, Q[s] = QoI of sample s
 *   uN   optional [n_nodes][S] FP64 output of u_h(t_N) in the caller's node
 *        order (same memory kind as Q), or NULL
 * Errors: LFLTS_ERR_ARG for bad ids/sizes, LFLTS_ERR_UNSTABLE (host mode
 * only) if some Q[s] is not finite; the message names the first such s.
 */
int lflts_solve(lflts_ctx* ctx, const lflts_solve_desc* desc, const double* xi,
                int64_t S, double* Q, double* uN, int mem, void* stream);

/*
 * MLMC level sums (Sec. 2.2): with dQ = Qf - Qc (or Qf when Qc is NULL, the
 * coarsest level), sums = {sum dQ, sum dQ^2, sum Qf, sum Qf^2} over the S
 * samples, FP64 with compensated (Neumaier) summation in a fixed order.
 * Qf, Qc [S] FP64; sums [4] FP64; all of the kind given by `mem`.
 * Errors: LFLTS_ERR_ARG for a NULL context, Qf or sums, S < 1 or a bad mem kind;
 * LFLTS_ERR_CUDA / LFLTS_ERR_OOM from the copies (host mode).
 */
int lflts_level_sums(lflts_ctx* ctx, const double* Qf, const double* Qc,
                     int64_t S, double* sums, int mem, void* stream);

/*
 * One MLMC level pair (Alg. 1 step 2a): Q_l and Q_{l-1} of the same draws
 * (the coarse solve is skipped when has_coarse == 0, level 0), the
 * differences dQ and the level sums.  Solves that share mesh, QoI, fields,
 * precision, p, nu and source across the jobs of one call are merged into a
 * single batched solve; when their (dt, n_steps) differ (draws with their
 * own time step, e.g. from a per-draw CFL bound) the batch is ragged: every
 * draw steps with its own dt for its own count and its QoI is taken at its
 * own final time (results equal those of separate batches to rounding).
 * Independent batches run concurrently on streams of the context, joined
 * back into `stream`.
 *   xi [S][K]; dQ, Qf [S] (Qf may be NULL); sums [4] (may be NULL).
 * Errors: LFLTS_ERR_ARG for a bad job (null xi or dQ, S < 1, a descriptor
 * that lflts_solve would refuse, fine and coarse meshes with different K,
 * a merged batch above 2,097,120 draws); LFLTS_ERR_UNSTABLE (host mode only)
 * for a non-finite QoI.
 */
typedef struct {
  lflts_solve_desc fine;
  lflts_solve_desc coarse;
  int has_coarse;
  const double* xi;
  int64_t S;
  double* dQ;
  double* Qf;
  double* sums;
} lflts_pair_job;

int lflts_run_pairs(lflts_ctx* ctx, const lflts_pair_job* jobs, int n_jobs,
                    int mem, void* stream);

/*
 * lflts_run_pairs in time slices (the same computation, cut along the time
 * axis of Alg. 2): the time loop of every merged batch, N outer steps (the
 * longest segment's count in a ragged batch), is split into n_slices parts,
 * and call `slice` (0 <= slice < n_slices) queues the outer steps
 * [floor(N slice / n_slices), floor(N (slice + 1) / n_slices)) of every batch.
 * Call 0 also copies the draws and forms the coefficients and start values;
 * call n_slices - 1 also forms the QoI, dQ, Qf and the level sums.  Calls
 * 0, 1, ..., n_slices - 1 in order, with the same jobs (same descriptors,
 * pointers and S), the same memory kind and the same n_slices, give exactly
 * the results of one lflts_run_pairs call (bit for bit); between them the
 * state stays on the device in the context.  lflts_run_pairs is
 * lflts_run_pairs_slice(..., 0, 1, ...).  Sliced runs are never captured
 * into CUDA graphs.  Host memory (mem = LFLTS_MEM_HOST): call 0 reads xi,
 * the last call writes dQ, Qf and sums; every call synchronises `stream`
 * before it returns.  A call with slice = 0 starts a new run and drops an
 * unfinished one; so does lflts_run_pairs.  The jobs' buffers must stay
 * valid until the last call has completed.
 * Errors: those of lflts_run_pairs; LFLTS_ERR_ARG for slice outside
 * [0, n_slices) or a call that does not continue the run in progress (other
 * jobs, memory kind or n_slices, or slices out of order).  After an error the
 * run is dropped.
 */
int lflts_run_pairs_slice(lflts_ctx* ctx, const lflts_pair_job* jobs, int n_jobs,
                          int mem, int slice, int n_slices, void* stream);

/*
 * Register the nodal interpolation from mesh_c to mesh_f (both registered,
 * same domain), as lflts_interp_weights returns it: for every node k of
 * mesh_f (caller's numbering) the vertices vert[3k..3k+2] of a mesh_c
 * triangle containing it (mesh_c's caller numbering) and the barycentric
 * weights w[3k..3k+2].  Used by lflts_run_field_pair to form the difference
 * of a level pair's L2(D)-valued QoIs on the finer mesh (Sec. 4).
 * Errors: LFLTS_ERR_ARG for null pointers, a bad mesh id, a vertex outside
 * mesh_c or a non-finite weight; LFLTS_ERR_OOM / LFLTS_ERR_CUDA from the upload.
 */
int lflts_field_interp_add(lflts_ctx* ctx, int mesh_f, int mesh_c, const int32_t* vert,
                           const double* w, int* interp_id);

/*
 * One level pair of the L2(D)-valued QoI u(., T) (Sec. 4: V = L2(D)): the
 * fine and coarse solves of `job` (as lflts_run_pairs; the coarse one only
 * when job->has_coarse), then for every draw s the difference on the fine
 * mesh dU_s = u_l(., T) - I u_{l-1}(., T) (I: the interpolation interp_id,
 * from job->coarse's mesh to job->fine's; ignored for level 0, dU_s = u_0)
 * and in FP64 with compensated sums:
 *   sum_dU    [n_nodes_f]  sum_s dU_s at every fine node (caller's order)
 *   norm2     [S] or NULL  ||dU_s||^2 in L2(D), the exact integral of the P1
 *                          function (consistent mass: |T|/12 (1 + delta_ab))
 *   sum_norm2 [1]          sum_s ||dU_s||^2
 * the sums of the V-valued estimator and its V-norm variance (Eqs.
 * MLMCestimator and Vell_est).  job->dQ, Qf, sums may be NULL; when given
 * they receive the scalar QoI of the same solves as in lflts_run_pairs.
 * Memory kinds, streams and synchronisation as lflts_run_pairs.
 * Errors: LFLTS_ERR_ARG for a bad job, a missing or mismatched interp_id;
 * LFLTS_ERR_UNSTABLE (host mode) for a non-finite QoI or norm.
 */
int lflts_run_field_pair(lflts_ctx* ctx, const lflts_pair_job* job, int interp_id, double* sum_dU,
                         double* norm2, double* sum_norm2, int mem, void* stream);

/*
 * Gradient of the QoI with respect to the field parameters: for every draw
 * s, Q[s] (as lflts_solve) and dQdxi[s][k] = dQ/dxi_k, the exact derivative of
 * the computed (discrete) QoI.  Discrete adjoint of the u-form LF-LTS solve:
 * the adjoint variable obeys the same step operator backwards (the LF-LTS
 * step is self-adjoint in the M inner product, the basis of the energy
 * identity of Alg. 2), the inner substeps are differentiated by their own
 * adjoint recursion near P, and the derivative of c_e^2 = exp(xi . psi_e) is
 * psi_{e,k} c_e^2.  States are stored every `ckpt_every` outer steps and
 * recomputed forward within a segment, because running leapfrog backwards
 * in floating point drifts.  The paper has no adjoint: it is an extension
 * for gradient-based use (sensitivities, inversion) of the same solve.
 *   xi     [S][K] FP64 draws;  Q [S] FP64;  dQdxi [S][K] FP64, row-major
 *   memory: about (2 ceil(N/ckpt_every) + ckpt_every + 6) state arrays of
 *           n_nodes x S values plus 2p arrays on R and n_edges x S FP64
 * Errors as lflts_solve; LFLTS_ERR_ARG for ckpt_every < 1.
 */
int lflts_grad_xi(lflts_ctx* ctx, const lflts_solve_desc* desc, const double* xi, int64_t S,
                  int ckpt_every, double* Q, double* dQdxi, int mem, void* stream);

/*
 * QoI reduction that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot let a library allocate device
 * memory: applications whose device memory is owned by their own pool
 * allocator (a library cudaMalloc would fragment it or exceed its budget),
 * or code that must not allocate once it is running (fixed memory plans,
 * latency-bound loops in which a cudaMalloc would synchronise the device).
 * It computes, like the QoI step of lflts_solve,
 *     Q[s] = sum_k g[k] * u[idx[k]][s],   s = 0 .. S-1,
 * in FP64 with compensated summation in the same order as lflts_solve
 * (for the same u and weights the two give the same Q bit for bit).
 *   ctx        optional (may be NULL); receives the error message.  With a
 *              context of a device, that device is made current for the
 *              call; with NULL (or a host-only context) the current device
 *              is used
 *   u          device [n_rows][S] state, FP32 (precision 32) or FP64 (64)
 *   idx, g     device [nnz] row indices and FP64 weights; an index outside
 *              [0, n_rows) is skipped (contributes nothing) and never read
 *   Q          device [S] FP64 output
 *   stream     cudaStream_t the two kernels are enqueued on
 * Scratch: a fixed 2 MiB array in the library's device image, present on
 * every GPU that loads the library until the process exits.  Its limit:
 * ceil(nnz / 512) * S <= 131072 partial sums; larger calls return
 * LFLTS_ERR_ARG without launching anything.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress, with the
 * device current) and keeps it for later calls.  All
 * calls on a device share the array and every call overwrites what it
 * reads, so nothing needs clearing, but calls whose kernels overlap on the
 * GPU (different streams, no ordering between them) race on it.  The call
 * makes no cudaMalloc/cudaFree and no allocating library call.  Unlike
 * lflts_solve it does not check Q: a non-finite Q[s] is written as it is and
 * the call still returns LFLTS_OK.
 * Errors: LFLTS_ERR_ARG for null pointers, sizes below 1, a precision other
 * than 32/64 or a call beyond the scratch limit; LFLTS_ERR_CUDA if the
 * device cannot be selected, the array's address cannot be resolved or a
 * launch fails.
 */
int lflts_qoi_reduce_noalloc(lflts_ctx* ctx, const void* u, int precision, int64_t n_rows,
                             int64_t S, const int32_t* idx, const double* g, int64_t nnz,
                             double* Q, void* stream);

/*
 * Profiling.  When enabled, every kernel launch is bracketed by CUDA events
 * on its stream; lflts_profile_read synchronises the context's device and
 * returns, per kernel class, the launch count, the summed device time in ms
 * and the summed algorithmic bytes: the state values the method must move per
 * node and draw (4 bytes each in FP32, 8 in FP64), counted as 3 values per
 * free node for a coarse launch (u_n and u_{n-1} read, u_{n+1} written), 4
 * per node of R for one inner substep (r_m, r_{m-1} and g read, r_{m+1}
 * written), 5 per node of R for a launch of two substeps (r_m, r_{m-1}, g
 * read, r_{m+1}, r_{m+2} written; 7 for the pair that ends the step, which
 * reads u and d and writes d and u instead of r_{m+1}, r_{m+2}) and 3 per
 * node of R for a launch that runs all substeps of a step on chip; per-draw edge weights and index data are not counted (the
 * coefficient can be recomputed from xi).  Reset clears the
 * counters.  lflts_launch_count returns all kernel launches of the context
 * since creation, whether profiling is on or not.
 */
int lflts_profile_enable(lflts_ctx* ctx, int on);
int lflts_profile_reset(lflts_ctx* ctx);
int lflts_profile_read(lflts_ctx* ctx, int kernel_class, int64_t* launches,
                       double* ms, double* alg_bytes);
int lflts_launch_count(lflts_ctx* ctx, int64_t* launches);
/* Instantiated solve graphs the context holds (all workspaces), for the
 * bound LFLTS_OPT_GRAPH_CACHE sets.  Errors: LFLTS_ERR_ARG for NULL pointers. */
int lflts_graph_cache_size(lflts_ctx* ctx, int64_t* n);

/* Set an LFLTS_OPT_* option of the context.
 * Errors: LFLTS_ERR_ARG for a NULL context, an unknown option, a fused-inner mode
 * outside {0, 1, 2}, a tiled-inner mode outside {0, 1, 2}, a tile capacity
 * in [1, 15] or negative, a graph cache below 1, a paired-inner mode outside
 * 0..4, a paired-substep block outside [16, 4096], a negative paired-substep
 * minimum |R| or a coarse weight mode outside {0, 1, 2}. */
int lflts_set_option(lflts_ctx* ctx, int option, int64_t value);

/*
 * Counters: out[0] kernel launches executed (kernels inside replayed graphs
 * counted one by one), out[1] graph launches, out[2] kernel launches spent
 * in autotuning (not in out[0]), out[3] autotuned launch shapes cached.
 * Errors: LFLTS_ERR_ARG for a NULL context or out.
 */
int lflts_get_stats(lflts_ctx* ctx, int64_t out[4]);

#ifdef __cplusplus
}
#endif
#endif /* LFLTS_H */
