/*
 * mabd.h -- C ABI of the GB300 (sm_103a) multi-affine-body step library.
 *
 * One call of mabd_step advances M affine bodies joined by K joints by one
 * implicit-Euler step with one Newton iteration, as M-ABD (arXiv 2603.08079)
 * defines it:
 *   Sec. 3.3-3.4, Eq. polar / abd_final: co-rotated per-body update with a
 *       constant prefactored Hbar_A = M_A/h^2 + Kbar_A per body;
 *   Sec. 4.2-4.3, Eq. ball / hinge, Sec. 5.1 Eq. pcpq: joint constraint
 *       Jacobians in affine coordinates (hinge frame frozen at q_n);
 *   Sec. 5, Eq. kkt / dual: the KKT system projected into the dual space of
 *       the joint rows, S lambda = G H^{-1} f + C(q_n) with S = G H^{-1} G^T
 *       (the bottom rhs -C(q_n) of the Sec. 5 footnote is included unless
 *       residual_rhs = 0), solved by block cyclic reduction for chains
 *       (Sec. 5.2 Eq. chain-btd), level-scheduled body-space elimination for
 *       trees (Sec. 5.3 Alg. 2 / Eq. module3-kkt) and block-Jacobi
 *       preconditioned conjugate gradients otherwise (Sec. 5.5);
 *   Sec. 5.2 Eq. recover-dq-explicit: back-propagation
 *       dq_j = H_j^{-1}(f_j - sum_k G_kj^T lambda_k), then
 *       q_{n+1} = q_n + dq and qdot_{n+1} = dq / h.
 *
 * Conventions
 *   Affine coordinates q = [vec(A); t] (12 doubles) with vec stacking the
 *   three columns of A (Eq. abd_dof): A(r,c) = q[3c+r].  A body's rest frame
 *   has its origin at the centre of mass.  The step works in the principal
 *   frame, where second_moment is diagonal (Hbar_A then splits into small
 *   blocks).  A body given with off-diagonal entries above 1e-12 of the
 *   trace is kept in its principal frame Sigma = V diag(w) V^T (V a rotation
 *   found by Jacobi rotations on the host): the library holds A V, turns the
 *   rest-frame anchors, axes and reference directions of its joints by V^T,
 *   and every state it takes or returns (mabd_body_desc, mabd_set_state,
 *   mabd_get_state) stays in the caller's frame.  The step is the same
 *   physical step: elasticity is isotropic, and the polar factor satisfies
 *   polar(A V) = polar(A) V.
 *   Ownership: every host array passed in belongs to the caller; the library
 *   copies what it needs during the call and keeps no pointer.  All device
 *   memory belongs to the context (through dev_alloc/dev_free when given,
 *   else cudaMalloc/cudaFree) and is released by mabd_destroy.
 *   Ordering: all device work is ordered on cfg.stream (NULL = the legacy
 *   default stream).  mabd_step returns once the work is enqueued unless
 *   stats is non-NULL, in which case it synchronizes the stream; with the
 *   PCG solver it also synchronizes after each cooperative solve, or
 *   between chunks of 16 iterations of the one-launch-per-step driver (the
 *   host reads the iteration count and the convergence flag there).  Without statistics the step's
 *   launches are replayed from CUDA graphs recorded at the first such call
 *   on a private stream that is ordered after cfg.stream by events
 *   (environment MABD_NO_GRAPHS=1 launches kernels directly instead;
 *   MABD_DEBUG_SYNC=1 checks every launch synchronously).
 *   Errors: no C++ exception crosses this ABI; every call returns a status.
 *   MABD_ERR_CUDA is sticky (destroy the context).  Device-side failures
 *   (non-positive det A, non-finite state, polar or PCG non-convergence, a
 *   bounded wait that gave up; in a library built with -DMABD_DEBUG also an
 *   out-of-range index read from device memory, reported as
 *   MABD_ERR_INVALID_ARG) set
 *   a status word that the next synchronizing call (mabd_step with stats,
 *   mabd_get_state, mabd_get_lambda, mabd_synchronize) returns and clears;
 *   the state is then undefined until mabd_set_state.
 *   Call order: mabd_add_* after mabd_prefactor and mabd_step before it
 *   return MABD_ERR_BAD_STATE.  Threads: one context must not be used from
 *   two threads at once.  Ids: bodies and joints are numbered densely in
 *   insertion order; lambda is returned joint by joint in that order, with
 *   3 rows per ball and 5 per hinge.
 */
#ifndef MABD_H
#define MABD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mabd_ctx mabd_ctx;

#define MABD_WORLD (-1) /* body index of the world in a joint */

typedef enum {
  MABD_OK = 0,
  MABD_ERR_INVALID_ARG = 1,
  MABD_ERR_BAD_STATE = 2,      /* call order */
  MABD_ERR_OUT_OF_MEMORY = 3,
  MABD_ERR_CUDA = 4,           /* sticky */
  MABD_ERR_NOT_SPD = 5,        /* a prefactored or dual block is not positive definite */
  MABD_ERR_INVERTED = 6,       /* det A <= 0 for some body */
  MABD_ERR_NONFINITE = 7,
  MABD_ERR_NO_CONVERGENCE = 8, /* polar iteration or PCG hit its cap */
  MABD_ERR_TIMEOUT = 9,        /* a bounded device-side wait gave up (cooperative PCG) */
  MABD_ERR_UNSUPPORTED = 10
} mabd_status;

/* Arithmetic of the step.
   MABD_FP64   every product in FP64.
   MABD_MIXED  chains: the unconstrained solve, the Jacobian products, the
               dual Gram blocks and the back-propagation in FP32; the polar
               rotation and the rhs in double-float (pairs of FP32 numbers,
               ~46 bits); the constraint values, the prefactorization and
               the block cyclic reduction of the dual in FP64; then
               refine_steps residual-correction sweeps (primal residual in
               double-float, dual residual in FP64)
               (iterative refinement of the KKT system through the stored
               FP64 factors).  Graphs (PCG solver): every dual solve by FP32
               PCG, refined the same way.  Trees and the loop solver:
               MABD_ERR_UNSUPPORTED at mabd_prefactor.
   MABD_MIXED_FP32_DUAL  as MABD_MIXED, but the chain's cyclic reduction
               runs in FP32 as well (Gram blocks, factors and levels in
               FP32); on trees the body-space elimination runs in FP32; the
               FP64 correction sweeps still refine the FP64 system, so the
               result keeps the mixed form's accuracy while the dual solve
               leaves the FP64 pipe.  On the PCG path it equals MABD_MIXED;
               the loop solver is FP64 only (AUTO picks PCG for loops). */
enum { MABD_FP64 = 0, MABD_MIXED = 1, MABD_MIXED_FP32_DUAL = 2 };
#define MABD_MAX_REFINE 8
/* MABD_SOLVER_LOOP: a single closed loop of bodies (every body joined to two
   others, every joint between two bodies; Sec. 5.4, Case III, eq. loop):
   one joint is the loop breaker, the others form a chain solved by the
   chain's block cyclic reduction, and the breaker's multipliers come from the
   Schur complement of the chain (a few right-hand-side passes through the
   chain's factors).  FP64 form only. */
enum { MABD_SOLVER_AUTO = 0, MABD_SOLVER_CHAIN = 1, MABD_SOLVER_TREE = 2, MABD_SOLVER_PCG = 3,
       MABD_SOLVER_LOOP = 4 };
/* Step variants of the paper, FP64 form only (another precision returns
   MABD_ERR_UNSUPPORTED from mabd_prefactor).
   MABD_ROTATION_NORMALIZED (Sec. 3.4, Alg. 1, Eq. len_preserving): each
     body's unconstrained solve u = H_A^{-1} f_A takes its four 3-blocks to
     the rest frame as A^T f_k rescaled to |f_k| and back as A dp_k rescaled to
     |dp_k| (a zero block stays zero).  That map is not linear, so the dual
     operator G H_A^{-1} G^T and the constraint forces keep the polar R
     (Eq. polar); the step's constraints are still met to first order.  Any
     solver.
   MABD_JACOBIAN_FULL (Sec. 5.1, Eq. constraint_gradient, pcpr, r_gradient):
     the hinge and prismatic rows gain the derivative of their frame, which
     is attached to body a (R_J = dR R_a^T): a row n . d (world direction n,
     gap d of its point pair) adds omega . (n x d) on body a, omega the
     rotation rate of a's polar factor, (tr(P) I - P) w = axial(R^T dA -
     dA^T R), omega = R w, P = R^T A.  This is the exact derivative that the
     printed R ~ A approximation stands in for.  Tree and PCG solvers (AUTO
     picks the tree solver for a tree or forest, else PCG; CHAIN and LOOP,
     whose blocks come from point compliances, return MABD_ERR_UNSUPPORTED);
     a universal joint, whose frame follows both bodies, returns
     MABD_ERR_UNSUPPORTED.  The
     default frozen frame (Eq. pcpq) keeps the anchor rows affine in q, so a
     step closes them exactly; the full gradient does not. */
enum { MABD_ROTATION_POLAR = 0, MABD_ROTATION_NORMALIZED = 1 };
enum { MABD_JACOBIAN_FROZEN = 0, MABD_JACOBIAN_FULL = 1 };
/* MABD_JOINT_UNIVERSAL (Sec. 4.4, 4 rows): anchor_a / anchor_b are the joint
   centre in each rest frame, axis_a the first axis a1 (fixed in body a),
   axis_b the second axis a2 (fixed in body b, perpendicular to a1 at rest),
   axis_len the distance l of b's second point along a2.  Rows: the ball rows
   in the frame R_U = [a1 x a2, a1, a2]^T (a2 made normal to a1, frozen at
   q_n) and a1 . (x_b(p_b + l a2) - x_b(p_b)), which keeps b's axis normal to
   a1.  body_b must be a free body; scenes with universal joints are solved
   by the PCG solver (AUTO picks it; the chain, tree and loop solvers return
   MABD_ERR_UNSUPPORTED). */
/* MABD_JOINT_PRISMATIC (Sec. 4.5, 5 rows): body b slides along the axis
   of body a and nothing else.  anchor_a / anchor_b are a point of the
   sliding line in each rest frame, axis_a / axis_b the sliding direction in
   each rest frame (axis_b a world direction when body_b is MABD_WORLD),
   ref_a / ref_b a direction normal to the axis, the same at rest in both
   frames, axis_len l the spacing of the further points.  The frame R_P =
   [x; y; z] follows body a (y = the axis, x = ref_a made normal to it,
   z = x cross y; frozen at q_n).  Rows: the x and z components of the gaps
   between the points p_a / p_b, p_a + l axis_a / p_b + l axis_b, and
   (z only) p_a + l ref_a / p_b + l ref_b.  Solved by the PCG solver. */
enum { MABD_JOINT_BALL = 0, MABD_JOINT_HINGE = 1, MABD_JOINT_UNIVERSAL = 2, MABD_JOINT_PRISMATIC = 3 };
enum { MABD_TOPO_NONE = 0, MABD_TOPO_CHAIN = 1, MABD_TOPO_TREE = 2, MABD_TOPO_GRAPH = 3,
       MABD_TOPO_LOOP = 4 };

typedef struct {
  double h;             /* time step [s] > 0 */
  double gravity[3];    /* [m/s^2], applied at each centre of mass (Eq. module1-wrench-map) */
  int32_t precision;    /* MABD_FP64, MABD_MIXED or MABD_MIXED_FP32_DUAL */
  int32_t solver;       /* MABD_SOLVER_*; AUTO picks chain, then tree, then loop (FP64), then PCG */
  int32_t pcg_max_iters;/* cap on PCG iterations (>= 1) */
  double pcg_rtol;      /* PCG stops when |r| <= pcg_rtol |b|.  The mixed forms' FP32
                           PCG with the learned preconditioner on (ball-joint
                           graphs) runs each solve as one cooperative launch in
                           the normalized dual space (MABD_PCG_NORMALIZED=0 in
                           the environment turns that off; the step's first
                           solve starts from the previous step's multipliers,
                           MABD_PCG_WARM=0 starts it from 0); otherwise one launch
                           per step of an iteration, or with MABD_PCG_PERSIST=1
                           one cooperative launch per solve.  In a cooperative
                           solve the phases meet at a grid barrier; a wait that
                           gives up (about a second) ends the step with
                           MABD_ERR_TIMEOUT. */
  int32_t refine_steps; /* MABD_MIXED: FP64 correction sweeps per step, 0..MABD_MAX_REFINE */
  int32_t residual_rhs; /* 1: bottom KKT rhs is -C(q_n) (Sec. 5 footnote); 0: zero as printed */
  void *stream;         /* cudaStream_t for all work (NULL: default stream) */
  void *(*dev_alloc)(size_t bytes, void *user); /* optional device allocator */
  void (*dev_free)(void *ptr, void *user);
  void *alloc_user;
  int32_t rotation_mode; /* MABD_ROTATION_POLAR (default) or MABD_ROTATION_NORMALIZED */
  int32_t jacobian_mode; /* MABD_JACOBIAN_FROZEN (default) or MABD_JACOBIAN_FULL */
} mabd_config;

typedef struct {
  double mass;             /* m > 0 [kg] */
  double second_moment[6]; /* Sigma = int rho xbar xbar^T about the COM: xx,yy,zz,xy,xz,yz */
  double volume;           /* V > 0 [m^3] */
  double young, poisson;   /* E > 0 [Pa], 0 <= nu < 0.5 */
  double q[12], qdot[12];  /* initial state */
  int32_t fixed;           /* 1: the body never moves; joints to it are one-sided */
} mabd_body_desc;

typedef struct {
  int32_t type;            /* MABD_JOINT_BALL (3 rows), MABD_JOINT_HINGE (5), MABD_JOINT_UNIVERSAL (4)
                              or MABD_JOINT_PRISMATIC (5) */
  int64_t body_a, body_b;  /* body_b may be MABD_WORLD; body_a must be a body */
  double anchor_a[3];      /* joint point in body a's rest frame */
  double anchor_b[3];      /* ... in body b's rest frame, or a world point */
  double axis_a[3];        /* hinge axis in body a's rest frame (the frame follows body a) */
  double axis_b[3];        /* hinge axis in body b's rest frame, or a world axis */
  double axis_len;         /* distance of the second on-axis point (> 0) */
  double ref_a[3];         /* prismatic: reference direction normal to the axis in a's rest frame */
  double ref_b[3];         /* prismatic: the same direction in b's rest frame, or a world direction */
} mabd_joint_desc;

typedef struct {
  double lin_residual;     /* max over rows of |G dq + C(q_n)| */
  double joint_residual;   /* max over rows of |C(q_{n+1})| (Table 1 |r|) */
  int32_t pcg_iters;       /* PCG iterations of this step (0 for direct solvers) */
  double pcg_rel_residual; /* final |r|/|b| of PCG (0 for direct solvers) */
  double refine_residual;  /* MABD_MIXED: max over rows of |C(q_n) + G dq| (FP64) entering the
                              last correction sweep (0 for FP64 or without sweeps) */
  double polar_iterations; /* mean Newton iterations per body of the polar decomposition
                              R = polar(A) (Eq. polar) in this step */
} mabd_step_stats;

typedef struct {
  int64_t bodies, joints, dual_rows;
  int32_t topology;        /* MABD_TOPO_* chosen at prefactor */
  int32_t solver;          /* MABD_SOLVER_* in use */
  int64_t device_bytes;    /* device memory held by the context */
  int32_t precision;       /* MABD_FP64, MABD_MIXED or MABD_MIXED_FP32_DUAL */
  int32_t refine_steps;    /* correction sweeps per step (MABD_MIXED) */
  int32_t cr_levels;       /* chain solver: levels of the block cyclic reduction (0 otherwise) */
  int32_t cr_tail_level;   /* chain solver: first level run by the single-CTA tail launch
                              (= cr_levels when every level has its own launches) */
  int32_t seg_levels;      /* chain solver, MABD_MIXED_FP32_DUAL with one correction sweep and
                              MABD_CHAIN_SEG=1 in the environment at mabd_prefactor: tile
                              levels of the segment-tiled step (tiles of seg_tile joints, then
                              of 256 rows); 0 when the level-by-level reduction runs */
  int32_t seg_tile;        /* joints per tile of the first level of that reduction */
  int32_t rotation_mode;   /* MABD_ROTATION_* of the context */
  int32_t jacobian_mode;   /* MABD_JACOBIAN_* of the context */
} mabd_info;

/* Fills *cfg with h = 1e-2, gravity (0,0,-9.8), FP64, AUTO, pcg_max_iters 2000,
   pcg_rtol 1e-13, refine_steps 1, residual_rhs 1, default stream, library allocator. */
void mabd_config_default(mabd_config *cfg);

/* Creates a context.  cfg is copied.  INVALID_ARG on h <= 0 or bad fields;
   CUDA when no device is usable. */
mabd_status mabd_create(const mabd_config *cfg, mabd_ctx **out);

/* Appends n bodies (host array, copied).  *first_id (optional) receives the id
   of the first.  INVALID_ARG on non-positive mass/volume/E, nu outside
   [0,0.5), non-finite state or a second moment that is not positive
   definite; a non-diagonal second moment is handled as the conventions
   above say. */
mabd_status mabd_add_bodies(mabd_ctx *ctx, int64_t n, const mabd_body_desc *d, int64_t *first_id);

/* Appends n joints (host array, copied); body ids are checked at prefactor. */
mabd_status mabd_add_joints(mabd_ctx *ctx, int64_t n, const mabd_joint_desc *d, int64_t *first_id);

/* Freezes the scene and h: validates joints, classifies the topology,
   orders bodies/joints for the chosen solver, uploads the state and builds
   the per-body inverse of Hbar_A = M_A/h^2 + Kbar_A (Eq. abd_final).
   NOT_SPD if some Hbar_A is not positive definite; UNSUPPORTED if the
   requested solver does not fit the topology. */
mabd_status mabd_prefactor(mabd_ctx *ctx);

/* Runs nsteps >= 0 steps.  stats: NULL, or a host array of nsteps entries
   (then the call synchronizes and returns any device-side failure). */
mabd_status mabd_step(mabd_ctx *ctx, int32_t nsteps, mabd_step_stats *stats);

/* Host arrays of 12*M doubles each, body by body in insertion order.
   get synchronizes; set enqueues the copy (arrays are staged on the host). */
mabd_status mabd_get_state(mabd_ctx *ctx, double *q, double *qdot);
mabd_status mabd_set_state(mabd_ctx *ctx, const double *q, const double *qdot);

/* Multipliers of the last step, dual_rows doubles in joint order (synchronizes). */
mabd_status mabd_get_lambda(mabd_ctx *ctx, double *lambda);

/* Waits for the context's stream and returns any pending device-side failure. */
mabd_status mabd_synchronize(mabd_ctx *ctx);

mabd_status mabd_get_info(mabd_ctx *ctx, mabd_info *info);

/* Per-kernel timing with CUDA events recorded on the context's stream.
   enable = 1 starts recording around every launch (adds event overhead),
   0 stops.  mabd_kernel_times synchronizes and writes up to cap entries:
   names[i] (static strings), total milliseconds and launch counts since the
   last reset; returns the number of kernel names through *count. */
mabd_status mabd_profile_enable(mabd_ctx *ctx, int32_t enable);
mabd_status mabd_profile_reset(mabd_ctx *ctx);
mabd_status mabd_kernel_times(mabd_ctx *ctx, int32_t cap, const char **names, double *ms,
                              int64_t *launches, int32_t *count);

/* ---- Step without device allocation (the paper has no counterpart) ----
   For callers that cannot call cudaMalloc -- code running inside another
   framework that owns the device allocator, or under a fixed memory budget:
   one implicit step of a single chain of at most MABD_NOALLOC_MAX_BODIES
   bodies, computed by the same step kernels as mabd_step (Hbar^{-1} is formed
   on the device).  Every intermediate lives in one file-scope device array of
   the library (12.8 MB = 1,600,000 doubles, held on every device that loads
   the library until the process exits); nothing is allocated.  The first call on a device looks up that array's device
   address (cudaGetSymbolAddress), so make it before any stream capture.
   All calls on a device share the array and it keeps the last call's
   contents (the call clears what must start at zero): calls that overlap on
   the GPU (two host threads, or two streams) race and give wrong results.
     cfg: h, gravity, residual_rhs and stream are used (precision FP64;
       rotation_mode and jacobian_mode must be the defaults, else
       UNSUPPORTED).
     bodies: device array of M descriptions (their q, qdot are the input
       state), in path order; fixed must be 0.
     joints: device array of K in [M-1, M+1] descriptions in path order:
       an optional pin of body 0 (body_a = 0, body_b = MABD_WORLD), the M-1
       joints between bodies i and i+1 (either orientation), an optional pin
       of body M-1; ball and hinge joints only (universal and prismatic
       joints are rejected with INVALID_ARG).
     q_out, qdot_out: device arrays of 12*M doubles (body by body);
     lambda_out: device array of the dual rows (3 per ball, 5 per hinge).
   Synchronizes cfg->stream.  INVALID_ARG for M outside [1, MAX], K outside
   [M-1, M+1], descriptions that break the layout above, or values that
   mabd_add_bodies / mabd_add_joints reject (non-finite numbers, mass,
   volume or E <= 0, nu outside [0, 0.5), a non-diagonal second moment);
   device-side failures are returned as by mabd_step.  The cached device
   address of the array belongs to the device's current context: after
   cudaDeviceReset the library must be reloaded before this call is used. */
#define MABD_NOALLOC_MAX_BODIES 4096
mabd_status mabd_chain_step_noalloc(const mabd_config *cfg, int32_t M, const mabd_body_desc *bodies,
                                    int32_t K, const mabd_joint_desc *joints, double *q_out,
                                    double *qdot_out, double *lambda_out);

/* Schedule of a tree context's elimination, tuned at mabd_prefactor by
   timing the candidates on the scene's first state: counts[0] = number of
   levels below the roots, counts[1] = counts[2] = 0 (unused), counts[3] = 0
   for the level-scheduled path (one launch per level and pass), or 128 / 64 / 32
   for the persistent kernel (one block of that many threads per tree, both
   passes in one launch).  MABD_TREE_MODE=levels|forest128|forest64|forest32 in the
   environment forces the path (tests). */
mabd_status mabd_tree_schedule(mabd_ctx *ctx, int32_t *counts);

/* ---- Learned block preconditioner of the mixed-precision PCG path -------
   The paper has no counterpart: this extends its dual solve for closed loops
   and irregular networks (Sec. 5.5).  For ball-joint graphs the dual S is
   normalized by the inverse Cholesky factors C_k of its 3x3 diagonal blocks,
   S~ = C S C^T with off-diagonal blocks E (joints sharing a free body); a
   three-layer message-passing network (hidden width 64, BF16 tensor-core
   products with FP32 accumulation) over that joint graph gives per-joint
   scales s and per-edge weights alpha, and the preconditioner is
   M^{-1} = C^T G^T G C with G = diag(s)(I - A), A_kn = alpha_kn E_kn for
   n < k (symmetric positive definite for any parameters; block Jacobi for
   alpha = 0, s = 1).  Parameters are a float vector of mabd_lpc_num_params()
   entries: W1 [16][64], b1 [64], W2 [128][64], b2, W3 [128][64], b3,
   Wa [64][8], Wb [64][8], wd [64], cd, we [2], ce (row-major). */
int32_t mabd_lpc_num_params(void);

/* Uses the learned preconditioner in every FP32 PCG solve of the context
   (params: host array, copied; NULL turns it off).  Needs a prefactored
   MABD_MIXED context on the PCG path whose joints are all balls, else
   MABD_ERR_UNSUPPORTED; non-finite parameters give MABD_ERR_INVALID_ARG.
   A learned solve that misses the tolerance within pcg_max_iters is redone
   with block Jacobi (counted by mabd_lpc_fallbacks). */
mabd_status mabd_set_preconditioner(mabd_ctx *ctx, const float *params);
mabd_status mabd_lpc_fallbacks(mabd_ctx *ctx, int32_t *count);

/* Trainer on the current device: holds captured normalized dual systems of
   one joint graph and trains the parameters with the library's own forward
   and backward kernels (Adam). */
typedef struct mabd_lpc mabd_lpc;
mabd_status mabd_lpc_create(mabd_lpc **out);
/* Captures the normalized dual of ctx at its current state as one batch
   (*batch: its index).  ctx as for mabd_set_preconditioner; every capture
   must come from contexts with the first capture's joint graph. */
mabd_status mabd_lpc_capture(mabd_lpc *t, mabd_ctx *ctx, int32_t *batch);
/* Copies a captured batch out (host arrays): the joint graph's CSR offsets
   off[K+1] and neighbours nbr[nnz] (per joint sorted by neighbour, then by
   shared body) and the normalized blocks E[nnz][9] (row-major, rows: the
   joint, columns: the neighbour). */
mabd_status mabd_lpc_batch_blocks(mabd_lpc *t, int32_t batch, int32_t *off, int32_t *nbr, float *E);
/* Training objective of one batch, X = G S~ G^T, n = 3K, over nv probe
   vectors V (host, [nv][K][3] in joint order; NULL: drawn on the device from
   SplitMix64(seed + i), uniform with unit variance):
     kind 0 (Frobenius)  L = sum_v |X v - v|^2 / (nv n);
     kind 1 (Kaporin)    L = log(sum_v v.X v / (nv n)) - (2/K) sum_k log s_k,
                         the log of Kaporin's condition number of X up to a
                         constant (tr X estimated by the probes, det exact);
   and, when grad is not NULL, dL/dparams (host, mabd_lpc_num_params floats). */
mabd_status mabd_lpc_loss_grad(mabd_lpc *t, int32_t batch, const float *params, int32_t kind,
                               int32_t nv, const float *V, uint64_t seed, double *loss, float *grad);
/* iters Adam steps on `kind` (learning rate lr, fresh moments) on batches
   drawn from the seed; params (host) in: start, out: result; losses[iters]
   if given. */
mabd_status mabd_lpc_train(mabd_lpc *t, float *params, int32_t kind, int32_t iters, float lr,
                           int32_t nv, uint64_t seed, double *losses);
mabd_status mabd_lpc_destroy(mabd_lpc *t);

/* Text of the last CUDA failure seen by the context (error name, message and
   the host source line), or "" if none; owned by the context. */
const char *mabd_error_detail(mabd_ctx *ctx);

mabd_status mabd_destroy(mabd_ctx *ctx);
const char *mabd_status_string(mabd_status s);

#ifdef __cplusplus
}
#endif
#endif /* MABD_H */
