/*
 * fsi_solid.h -- C ABI of the GB300 solid Newton step.
 *
 * The library solves the structure sub-problem of the partitioned FSI method
 * of Langer & Yang (arXiv:1312.5561): the residual-stabilised equal-order
 * P1/P1 displacement-pressure formulation of a nearly incompressible
 * hyperelastic solid (Sec. 3.2 strong form, Sec. 4.2.3 weak form, Eq. stelas
 * PSPG term), linearised by Newton's method (Sec. 4.4, Eq. linsys / globsys)
 * and solved by a Krylov method preconditioned by an aggregation AMG V-cycle
 * (Sec. 5.4-5.5 describe the paper's own Krylov/AMG solvers).
 *
 * Conventions shared by every call:
 *  - Unknowns are ordered per node as (d_x, d_y, d_z, p): "state" arrays are
 *    FP64 [n_nodes][4], row-major, on the device, owned by the caller.
 *  - Host descriptors (mesh, materials, options) are copied at create time;
 *    the caller keeps ownership of them.
 *  - All device work is enqueued on the CUDA stream passed as `stream`
 *    (a cudaStream_t cast to void*; NULL = the legacy default stream).  Every
 *    call returns after its work has finished on that stream (the status it
 *    returns is final).
 *  - A call never exits, aborts or traps; errors come back as fsi_status and
 *    fsi_solid_last_error() returns a one-line description.
 *  - A handle is not thread-safe: use one handle per host thread.
 */
#ifndef FSI_SOLID_H
#define FSI_SOLID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fsi_solid_s* fsi_solid_t;   /* opaque, owned by the library */

typedef enum {
  FSI_OK = 0,
  FSI_ERR_ARG = -1,            /* invalid argument (NULL, size, index out of range) */
  FSI_ERR_CUDA = -2,           /* a CUDA runtime call failed */
  FSI_ERR_OOM = -3,            /* device allocation failed */
  FSI_ERR_INVERTED = -4,       /* an element reached J <= 0 or a non-finite value */
  FSI_ERR_NOT_CONVERGED = -5   /* Newton or Krylov hit its iteration cap */
} fsi_status;

/* Material models (Sec. 2.3.1 and 2.3.2). */
enum { FSI_MODEL_MOONEY_RIVLIN = 0, FSI_MODEL_ARTERY = 1 };

/* Mesh description (host arrays, copied at create time).
 *  X         [n_nodes][3]  reference coordinates
 *  tets      [n_elems][4]  vertex ids, positively oriented (det > 0)
 *  mat_id    [n_elems]     index into the material table
 *  fibre     [n_elems][2][3] unit fibre directions a01, a02 (Eq. arinv46), or
 *                          NULL when no element uses the artery model
 *  dir_mask  [n_nodes][4]  1 = Dirichlet-constrained component (Eq. elasbnd)
 *  neu_faces [n_faces][3]  boundary triangles carrying the dead pressure load;
 *                          the right-hand normal (x1-x0)x(x2-x0) points out
 *  seg_node  [n_nodes]     segment id (batched independent meshes) or NULL:
 *                          ids in [0, n_segments), non-decreasing in the node
 *                          index, and the four vertices of every element in one
 *                          segment; otherwise create returns FSI_ERR_ARG
 *  n_segments              number of segments (read only with seg_node) */
typedef struct {
  int32_t n_nodes;
  int32_t n_elems;
  const double* X;
  const int32_t* tets;
  const int32_t* mat_id;
  const double* fibre;
  const uint8_t* dir_mask;
  int32_t n_faces;
  const int32_t* neu_faces;
  int32_t n_segments;
  const int32_t* seg_node;
} fsi_mesh_desc;

/* One material (Eq. mmreng for Mooney-Rivlin; Eq. areng for the artery).
 * Mooney-Rivlin uses c10, c01; the artery uses c10, k1, k2.  kappa is the bulk
 * modulus, rho the reference density (used only when inertia_coef > 0). */
typedef struct {
  int32_t model;
  double c10, c01, k1, k2, kappa, rho;
} fsi_material;

enum { FSI_PREC_FP64 = 0, FSI_PREC_FP32_IR = 1 };
enum { FSI_KRYLOV_FGMRES = 0, FSI_KRYLOV_BICGSTAB = 1 };
/* Smoother of the finest AMG level (coarser levels: see coarse_smoother).
 *  FSI_SMOOTHER_JACOBI  damped 4x4 block Jacobi, damping omega.
 *  FSI_SMOOTHER_VANKA   the multiplicative Vanka smoother of Sec. 5.5.2
 *                       (Eq. locsys, vankasmooth): one patch per pressure
 *                       unknown p_i holding p_i and the displacements of the
 *                       nodes that B2 couples to it (node i and its mesh
 *                       neighbours, up to 46 unknowns); the local problem is
 *                       the restriction of K to the patch, solved directly, and
 *                       the update is relaxed by vanka_omega.  Patches are
 *                       visited colour by colour (distance-2 node colouring,
 *                       so patches of one colour share no unknown): Gauss-Seidel
 *                       across colours, simultaneous within a colour. */
enum { FSI_SMOOTHER_JACOBI = 0, FSI_SMOOTHER_VANKA = 1 };
/* Preconditioner of the Krylov method.
 *  FSI_PRECOND_AMG       one AMG V-cycle on the whole u-p tangent K (default).
 *  FSI_PRECOND_BLOCK_LT  the block lower-triangular P_L of Sec. 5.4.2,
 *                        Eq. lpre: x_u = A~^-1 r_u by one AMG V-cycle on the
 *                        displacement block A, then
 *                        x_p = S~^-1 (B2 x_u - r_p) with the Schur-complement
 *                        approximation S~ = (1/theta + 1/kappa) diag(M_p) of
 *                        Eq. lpreschur (M_p the P1 pressure mass matrix, kappa
 *                        per element).  The paper pairs it with BiCGStab. */
enum { FSI_PRECOND_AMG = 0, FSI_PRECOND_BLOCK_LT = 1 };
/* Aggregation of the smoothed-aggregation hierarchy (set-up, host, once).
 *  FSI_AGG_RING  a root node takes its 7 strongest free neighbours (block
 *                Frobenius norm), leftovers join their strongest neighbour's
 *                aggregate (default).
 *  FSI_AGG_GROW  an aggregate grows one node at a time by the strongest
 *                connection from any member, up to 8 nodes, and leftovers
 *                join as with FSI_AGG_RING (so an aggregate may end with a
 *                few more): on walls meshed
 *                with many thin element layers it forms lines across the wall,
 *                where FSI_AGG_RING coarsens along the weak directions and the
 *                Krylov iteration stalls. */
enum { FSI_AGG_RING = 0, FSI_AGG_GROW = 1 };
/* Smoother of the coarser AMG levels (7x7 blocks: rigid-body modes and a
 * constant pressure per aggregate).
 *  FSI_COARSE_JACOBI  damped block Jacobi x += omega D^-1 (b - A x), as on the
 *                     finest level.  On the saddle-point coarse operators of
 *                     walls meshed with many thin layers D^-1 A has complex
 *                     eigenvalues far outside the unit disc and the sweep
 *                     diverges.
 *  FSI_COARSE_MR      minimal-residual block Jacobi: z = D^-1 r, w = A z and
 *                     x += a z, r -= a w with a = (r.w)/(w.w), the step length
 *                     that minimises ||r - a w||_2, so no sweep can raise the
 *                     residual (default).  The step length depends on the
 *                     right-hand side, which makes the V-cycle a nonlinear
 *                     preconditioner: FGMRES accepts it; with BiCGStab the
 *                     library falls back to FSI_COARSE_JACOBI. */
enum { FSI_COARSE_JACOBI = 0, FSI_COARSE_MR = 1 };

/* Solver options.  Defaults come from fsi_solid_default_opts(). */
typedef struct {
  int32_t precision;        /* FSI_PREC_*: FP64 throughout, or FP32 tangent and
                               V-cycle under an FP64 residual / outer Krylov */
  int32_t krylov;           /* FSI_KRYLOV_* */
  int32_t restart;          /* FGMRES restart length m (<= 128) */
  int32_t max_krylov;       /* cap on Krylov iterations per linear solve */
  int32_t max_newton;       /* cap on Newton iterations per solve */
  int32_t smoother;         /* FSI_SMOOTHER_* */
  int32_t nu_pre, nu_post;  /* smoothing sweeps before / after the coarse correction */
  int32_t coarse_max_nodes; /* stop coarsening when every component is this small */
  int32_t max_levels;       /* cap on AMG levels */
  int32_t use_pspg;         /* 1: PSPG term W_s of Eq. stelas on; 0: off */
  int32_t adaptive_tol;     /* 1: inner tolerance eps_1,k = eps_2,k-1^2 (Sec. 4.4) */
  int32_t use_graphs;       /* 1: capture the V-cycle in a CUDA graph */
  int32_t nu_coarse;        /* smoothing sweeps before / after on every coarser level */
  double omega;             /* block-Jacobi damping */
  double newton_rtol;       /* stop when ||R(v_k)|| <= newton_rtol ||R(v_0)|| */
  double krylov_rtol;       /* relative residual reduction of each linear solve */
  double fibre_factor;      /* 2: S = 2 dPsi/dC; 1: the factor printed in Eq. arpkt */
  double inertia_coef;      /* 1/(beta dt^2) of the Newmark-beta scheme; 0 = quasi-static */
  int32_t amg_lag;          /* recompute the coarse AMG levels on every (amg_lag+1)-th
                               Newton step only (0: every step); the finest level is
                               always the current tangent */
  int32_t assembly;         /* 0: element buffers + fixed-order gather (default);
                               1: colour-ordered scatter; both bit-reproducible */
  int32_t precond;          /* FSI_PRECOND_* */
  double schur_theta;       /* theta of Eq. lpreschur (the paper takes theta = O(c10));
                               <= 0: c10 of material 0 */
  double vanka_omega;       /* relaxation of the Vanka update (the paper: 0.78 for
                               Mooney-Rivlin, 0.86 for the artery) */
  int32_t aggregation;      /* FSI_AGG_* */
  int32_t coarse_bf16;      /* FSI_PREC_FP32_IR only: the V-cycle reads the coarse-level
                               (7x7) operators as BF16 copies (smoothing and residual;
                               FP32 accumulation); the Galerkin products, transfers,
                               block inverses and coarsest solve stay FP32 */
  int32_t coarse_smoother;  /* FSI_COARSE_* (sweeps: nu_coarse before and after) */
  int32_t autotune;         /* 1: at create, time the launch shapes of the element kernel
                               (CTA of 64 or 128 threads) and of every smoothed level's
                               block-row kernels (4x4 level: CTA of 64, 128 or 256 threads;
                               7x7 levels: one CTA or one warp per block row) on this mesh
                               and keep the fastest (see fsi_solid_get_tuning); 0: defaults.
                               The choice rests on timings, so two handles can pick
                               different shapes; the CTA- and warp-per-row kernels sum a
                               block row in different orders, so their solutions agree to
                               the Krylov tolerance, not bit for bit (autotune = 0 fixes
                               the shapes; one handle is always bit-reproducible) */
  int32_t segment_krylov;   /* meshes of several segments (fsi_mesh_desc.seg_node), FGMRES:
                               1 = one Arnoldi process per segment (per-segment inner
                               products, Hessenberg matrices and stop, so each segment
                               stops at its own convergence); 0 = one process over the
                               union (the segments' right-hand sides scaled to unit norm) */
  int32_t exact_candidates; /* coarse near-null space of the aggregation hierarchy: 1 = the
                               full R factor of each aggregate's QR, so that the tentative
                               prolongator reproduces the rigid-body modes and constant
                               pressure exactly on the free unknowns (P_t B_c = B) also where
                               a mode depends on the others within an aggregate (end planes
                               with u_z fixed); 0 (default) = such a mode is dropped from the
                               coarse space of that aggregate altogether */
  int32_t power_steps;      /* steps of the power iteration estimating lambda_max(D^-1 A) of
                               each level for the prolongator smoothing weight 4/(3 lambda)
                               (default 20; more steps give a closer, larger estimate where
                               the top eigenvalues cluster, hence a smaller weight) */
} fsi_solver_opts;

/* Load of one solve (device arrays owned by the caller; NULL = absent).
 *  dir_values    [n_nodes][4] prescribed values written into the constrained
 *                components of the state before Newton starts (Sec. 4.2.3:
 *                increments vanish on the Dirichlet boundary)
 *  pressure      scale of the dead pressure on neu_faces (traction -P n)
 *  node_pressure [n_nodes] nodal pressure values P_b (P1-interpolated on faces)
 *  face_pressure [n_faces] piecewise constant pressure per face
 *  hist          [n_nodes][3] Newmark history h_s; r_s = rho h_s (Sec. 4.2.3) */
typedef struct {
  const double* dir_values;
  double pressure;
  const double* node_pressure;
  const double* face_pressure;
  const double* hist;
} fsi_load;

/* Per-call statistics. */
typedef struct {
  int32_t newton_its;        /* Newton iterations performed */
  int32_t krylov_its_total;  /* Krylov iterations summed over Newton iterations */
  int32_t krylov_its_last;   /* Krylov iterations of the last linear solve */
  int32_t status;            /* fsi_status of the call */
  int32_t guess_accepted;    /* 1 if the supplied initial increment was kept */
  int32_t n_levels;          /* AMG levels */
  double res0;               /* ||R(v_0)||_2 */
  double res;                /* ||R(v_k)||_2 at return */
  double inc_norm;           /* ||v_k - v_(k-1)||_2 of the last update */
  double lin_res;            /* relative residual of the last linear solve */
  double inc_mnorm;          /* ||v_k - v_(k-1)||_M of the last update: the L2 norm of the
                                displacement and pressure increment, sqrt(dv^T M dv) with
                                M = diag[M_1, M_2] the P1 mass matrices, the quantity the
                                paper's Newton stop (Sec. 4.4, Eq. newstop) measures */
} fsi_info;

/* Default options: FP64, FGMRES(100), block Jacobi 4+4 sweeps on the finest
 * level and minimal-residual block Jacobi 2+2 on coarser levels, omega 0.7,
 * V-cycle replayed from a CUDA graph, coarse levels refreshed every Newton step,
 * Newton rtol 1e-8, Krylov rtol 1e-8, PSPG on, fibre_factor 2. */
void fsi_solid_default_opts(fsi_solver_opts* opts);

/* Build a handle: copies the mesh, computes the P1 geometry on the device,
 * colours the elements (greedy first fit in element order), builds the 4x4
 * block-CSR pattern, the element-to-block map and the AMG aggregation
 * hierarchy.  Allocates all device memory the solver needs. */
fsi_status fsi_solid_create(const fsi_mesh_desc* mesh, int32_t n_mat, const fsi_material* mats,
                            const fsi_solver_opts* opts, fsi_solid_t* out);

/* Release every resource of the handle.  NULL is accepted. */
fsi_status fsi_solid_destroy(fsi_solid_t h);

/* Residual R(v) of Eq. stabweakelas (R^1 rows 0..2, R^2 + W_s row 3 per node),
 * minus the dead load, with zero rows on constrained components; and, when
 * want_tangent != 0, the consistent Jacobian K = dR/dv (Eq. globsys) assembled
 * into the library-owned BSR matrix with constrained rows/columns replaced by
 * identity rows / zero columns.  state, residual: device FP64 [n_nodes][4].
 * residual may be NULL when only the tangent is wanted. */
fsi_status fsi_solid_residual_tangent(fsi_solid_t h, const double* state, const fsi_load* load,
                                      double* residual, int32_t want_tangent, void* stream);

/* The assembled level-0 matrix: 4x4 blocks, row-major within a block.
 * row_ptr [n_nodes+1], col_idx [n_blocks] (device pointers owned by the
 * library, valid until destroy); dtype 0 = FP64 values, 1 = FP32 values. */
fsi_status fsi_solid_get_bsr(fsi_solid_t h, const int32_t** row_ptr, const int32_t** col_idx,
                             const void** vals, int32_t* dtype, int32_t* n_blocks);

/* y = K x with the assembled matrix (device FP64 [n_nodes][4] vectors). */
fsi_status fsi_solid_spmv(fsi_solid_t h, const double* x, double* y, void* stream);

/* Solve K x = b with the assembled matrix by the configured Krylov method and
 * AMG preconditioner to krylov_rtol (b, x device FP64 [n_nodes][4]; x is
 * used as the initial guess). */
fsi_status fsi_solid_linear_solve(fsi_solid_t h, const double* b, double* x, fsi_info* info,
                                  void* stream);

/* One Newton iteration from `state` (Sec. 4.4 steps 1-2): residual, tangent,
 * linear solve of K dv = -R, update state += dv.  info->res0 is ||R|| before. */
fsi_status fsi_solid_newton_step(fsi_solid_t h, double* state, const fsi_load* load,
                                 fsi_info* info, void* stream);

/* Newton's method to newton_rtol for one load step.  Writes load->dir_values
 * into the constrained components first.  guess (device [n_nodes][4] or NULL)
 * is an initial increment: it is kept only if ||R(v + guess)|| <= ||R(v)||,
 * else Newton starts from v (zero increment). */
fsi_status fsi_solid_solve(fsi_solid_t h, double* state, const fsi_load* load, const double* guess,
                           fsi_info* info, void* stream);

/* Partitioned coupling: the Dirichlet-Neumann iteration of Sec. 5.1 with the
 * Aitken relaxation of Sec. 5.2 around fsi_solid_solve.  The interface Gamma^0
 * is the set of vertices of the mesh's loaded faces (neu_faces).  Cycle k
 * computes the fluid pressure from the relaxed interface displacement
 * d_(k-1), solves the solid under it (Newton from the previous cycle's state,
 * stopping relative to the first cycle's initial residual norm), takes
 * d~_k = the solid displacement on Gamma^0 and r_k = d~_k - d_(k-1), stops when
 * |r_k| / sqrt(n_Gamma) < tol, and relaxes d_k = w_(k-1) d~_k + (1 - w_(k-1)) d_(k-1)
 * (Eq. acceit) with w_k = -w_(k-1) r_k.(r_(k+1) - r_k) / |r_(k+1) - r_k|^2
 * (Eq. dnomega), w_0 = omega0.
 *
 * The fluid Dirichlet-to-Neumann map F of Eq. fixedp (a Navier-Stokes solve on
 * the moving fluid domain) is not part of this library; a surrogate added-mass
 * map of the blood column stands in for it: on interface node i
 *   p_i = p0 - added_mass * w_i . (d_i - d_ref_i),
 * w_i the unit direction of the P1 load of a unit pressure at node i.  The
 * resulting nodal pressures load the loaded faces as fsi_load.node_pressure
 * does.  With added_mass large against the wall stiffness, omega = 1 diverges
 * (the added-mass effect); the Aitken step restores convergence. */
typedef struct {
  double p0;              /* fluid pressure at rest */
  double added_mass;      /* >= 0, pressure per unit wall displacement */
  const double* d_ref;    /* device [n_nodes][4] state whose displacement is the wall
                             at rest (previous time level); NULL = reference configuration */
  double omega0;          /* first relaxation factor, (0, 1] */
  double tol;             /* interface residual tolerance (the paper: 1e-8) */
  int32_t max_cycles;     /* cap on DN cycles */
  int32_t aitken;         /* 1: Aitken (Eq. dnomega); 0: fixed omega0 */
} fsi_dn_opts;

typedef struct {
  int32_t cycles;           /* DN cycles run */
  int32_t converged;        /* 1 when |r| / sqrt(n_Gamma) < tol */
  int32_t newton_its_total;
  int32_t krylov_its_total;
  int32_t n_interface;      /* n_Gamma */
  double res_first;         /* |r_1| / sqrt(n_Gamma) */
  double res_last;
  double omega_last;        /* the last relaxation factor used */
} fsi_dn_info;

void fsi_dn_default_opts(fsi_dn_opts* o);

/* state: device FP64 [n_nodes][4], start and result (the solid state of the
 * last cycle).  load: dir_values and hist are used; its pressure fields are
 * replaced by the fluid's.  Returns FSI_ERR_NOT_CONVERGED (info filled) when
 * max_cycles end above tol, FSI_ERR_ARG without loaded faces or with
 * omega0 outside (0, 1] or added_mass < 0, and any status of fsi_solid_solve. */
fsi_status fsi_solid_dn_solve(fsi_solid_t h, double* state, const fsi_load* load, const fsi_dn_opts* o,
                              fsi_dn_info* info, void* stream);

/* Newmark-beta update after the solve of time step n (Sec. 4.1.2):
 *   a_n = (d_n - d_(n-1)) / (beta dt^2) - v_(n-1) / (beta dt) - (1 - 2 beta)/(2 beta) a_(n-1)
 *   v_n = v_(n-1) + dt ((1 - gamma) a_(n-1) + gamma a_n)
 * and the history of the next step h = d_n/(beta dt^2) + v_n/(beta dt) + (1-2beta)/(2beta) a_n
 * (r_s = rho h, see fsi_load.hist).  state: device [n][4] (d_n in columns 0..2);
 * disp [n][3] holds d_(n-1) on entry and d_n on return; vel, acc, hist [n][3]. */
fsi_status fsi_solid_newmark_advance(fsi_solid_t h, const double* state, double* disp, double* vel, double* acc,
                                     double* hist, double beta, double gamma, double dt, void* stream);

/* Host copy of the element colouring in original element order
 * (colour_out [n_elems]); returns the number of colours in *n_colours. */
fsi_status fsi_solid_get_colouring(fsi_solid_t h, int32_t* colour_out, int32_t* n_colours);

/* Launch shapes chosen by the autotuner (opts.autotune; project-written, the
 * paper has no counterpart): out[0] = CTA size of the element kernels,
 * out[1 + l] = shape of the block-row kernels of level l for every smoothed
 * level (level 0: CTA size; coarser levels: 1 = one CTA per block row, 2 = one
 * warp per block row; 0 = the size-based default).  *n_out receives the number
 * of entries; at most capacity are written (host array). */
fsi_status fsi_solid_get_tuning(fsi_solid_t h, int32_t* out, int32_t capacity, int32_t* n_out);

/* AMG level sizes: nodes_out[l] for l < *n_levels (host, capacity max_levels). */
fsi_status fsi_solid_get_levels(fsi_solid_t h, int32_t* nodes_out, int32_t* blocks_out,
                                int32_t capacity, int32_t* n_levels);

/* Kernel classes of the launch accounting below. */
enum {
  FSI_KC_TANGENT = 0,  /* element residual + tangent + colour-ordered block scatter */
  FSI_KC_RESIDUAL,     /* element residual only */
  FSI_KC_JACOBI0,      /* damped block-Jacobi sweep on the finest level */
  FSI_KC_BSR0,         /* other finest-level block-row kernels (SpMV, residual) */
  FSI_KC_COARSE_BSR,   /* block-row kernels on coarser levels */
  FSI_KC_TRANSFER,     /* restriction / prolongation */
  FSI_KC_GALERKIN,     /* per-Newton-step numeric AMG set-up */
  FSI_KC_BLOCKINV,     /* block-diagonal inverses */
  FSI_KC_COARSE,       /* dense coarsest-level factorisation and solve */
  FSI_KC_VECTOR,       /* Krylov vector kernels and reductions */
  FSI_KC_OTHER,
  FSI_KC_LEVEL1_SPMV,  /* w = A z on AMG level 1 inside the minimal-residual sweeps
                          (the coarse-level product with the most bytes) */
  FSI_KC_COUNT
};

/* Number of kernels this library has launched in this process so far. */
int64_t fsi_solid_launch_count(void);

/* Per-class kernel timing of one handle.  Returns in ms_out[FSI_KC_COUNT] the
 * device time (sum of CUDA-event intervals recorded on the launching stream
 * around each launch) and in launches_out[FSI_KC_COUNT] the launch counts
 * accumulated since the previous call, then resets them; enable = 1 keeps
 * (or starts) recording for the following calls on this handle, enable = 0
 * stops it.  While recording, the V-cycle is launched kernel by kernel
 * instead of from its CUDA graph.  Either output pointer may be NULL. */
fsi_status fsi_solid_kernel_timing(fsi_solid_t h, int32_t enable, double* ms_out, int64_t* launches_out);

/* ------------------------------------------------------------------------
 * Learned Newton initial guess (a per-node MLP; the paper has no counterpart:
 * Newton itself, unchanged, corrects whatever the network proposes and the
 * zero increment remains the fallback, see fsi_solid_solve's guess).
 * Layers l = 0..n_layers-1 map sizes[l] -> sizes[l+1]; hidden layers use
 * tanh, the last is affine.  Parameters are FP32, laid out per layer as
 * W_l [sizes[l+1]][sizes[l]] then b_l [sizes[l+1]].  Training minimises
 * L = 1/(2N) sum_n sum_o w_o (Y_no - T_no)^2 with Adam (b1 0.9, b2 0.999,
 * eps 1e-8).  Device arrays: X [n][sizes[0]], T and Y [n][sizes[L]], FP32. */
typedef struct fsi_mlp_s* fsi_mlp_t;

/* Create a network; weights U(-a, a), a = sqrt(6/(fan_in + fan_out)), from a
 * splitmix64 stream seeded by `seed`; biases zero. */
fsi_status fsi_mlp_create(int32_t n_layers, const int32_t* sizes, uint64_t seed, fsi_mlp_t* out);
fsi_status fsi_mlp_destroy(fsi_mlp_t h);
int64_t fsi_mlp_num_params(fsi_mlp_t h);
/* Copy the parameters to (set = 0) or from (set = 1) the host array `host`. */
fsi_status fsi_mlp_params(fsi_mlp_t h, float* host, int32_t set);
/* Y = net(X); bf16 = 1 runs every layer on the tensor cores in BF16 with FP32
 * accumulation (every sizes[l] < sizes[L] must then be a multiple of 16). */
fsi_status fsi_mlp_forward(fsi_mlp_t h, const float* X, int32_t n, float* Y, int32_t bf16, void* stream);
/* Forward + backward on one batch; loss_out (host, may be NULL) gets L,
 * grad_host (host, may be NULL) the gradient; apply = 1 then takes one Adam
 * step with learning rate lr.  w_out: device [sizes[L]] output weights or NULL. */
fsi_status fsi_mlp_train_step(fsi_mlp_t h, const float* X, const float* T, int32_t n, const float* w_out, float lr,
                              int32_t apply, float* loss_out, float* grad_host, void* stream);

/* Allocation-free dot products: out[i] = V_i . y for V_i = V + i * ldv,
 * i < k (device FP64 arrays; out is device memory of k doubles).  The paper
 * has no counterpart: this call is for callers that cannot allocate device
 * memory -- a coupling driver or host application that owns every device
 * allocation and hands this library only fixed buffers, or code that may not
 * call cudaMalloc / cudaFree after start-up because those calls synchronise
 * the device and stall its other streams.  It needs no handle and allocates
 * nothing: its partial sums live in a fixed file-scope device array of
 * FSI_DOTS_STATIC_MAX_VECTORS x 304 doubles (76 KiB) that every GPU which
 * loads the library keeps until the process exits.  k must lie in
 * [1, FSI_DOTS_STATIC_MAX_VECTORS] (FSI_ERR_ARG otherwise) and ldv >= n when
 * k > 1.  The sums use the solver's own deterministic two-pass reduction (304
 * CTA partials, then a fixed-order sum), so repeated calls give identical
 * results, bit-identical to the norms the solver reports.  Each call looks up
 * the array's address in the current context of the current device.  All
 * calls share the one array: calls that overlap on the GPU (different streams
 * or threads) race and must be serialised by the caller.  Returns after the
 * work on `stream` has finished. */
#define FSI_DOTS_STATIC_MAX_VECTORS 32
fsi_status fsi_dots_static(const double* V, int64_t ldv, int32_t k, const double* y, int64_t n, double* out,
                           void* stream);

/* Description of the last error on this handle (static storage of the handle). */
const char* fsi_solid_last_error(fsi_solid_t h);

#ifdef __cplusplus
}
#endif
#endif /* FSI_SOLID_H */
