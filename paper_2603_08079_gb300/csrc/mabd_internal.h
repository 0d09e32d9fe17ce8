// Internal declarations shared by the host orchestration (mabd_api.cpp) and
// the CUDA kernels.  Device arrays are structure-of-arrays, component-major:
// component c of item i lives at ptr[c * N + i], so consecutive threads read
// consecutive addresses.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace mabd {

// device-side failure bits (status word)
enum : int {
  ST_INVERTED = 1,
  ST_NONFINITE = 2,
  ST_POLAR_NOCONV = 4,
  ST_NOT_SPD = 8,
  ST_PCG_NOCONV = 16,
  ST_TIMEOUT = 32,  // a bounded device-side wait gave up
  ST_BOUNDS = 64,   // MABD_DEBUG builds: an index read from memory was out of range
};

// Structured inverse of Hbar_A = M_A/h^2 + Kbar_A for a body whose second
// moment is diagonal (principal rest frame).  Hbar_A decouples into:
//   the diagonal entries of A (q[0], q[4], q[8])       -> 3x3 block X
//   the transpose pairs (q[1],q[3]), (q[2],q[6]), (q[5],q[7]) -> three 2x2 blocks
//   the translation q[9..11]                           -> (m/h^2) I3
// HINV layout (16 doubles): [t, X00, X01, X02, X11, X12, X22,
//                            P13_aa, P13_ab, P13_bb, P26_.., P57_..]
constexpr int HINV_N = 16;

struct DevBodies {
  int32_t M;
  double *q;            // [12][M]
  double *qd;           // [12][M]
  const double *sig;    // [3][M]  diagonal second moment
  const double *mass;   // [M]
  const double *vmu;    // [M]     V * mu
  const double *vlam;   // [M]     V * lambda
  const double *hinv;   // [16][M] structured Hbar^{-1}
  const uint8_t *fixed; // [M]
  double *R;            // [9][M]  rotation of the step (row-major 3x3)
  double *ubar;         // [12][M] unconstrained solve in the rest frame
  // mixed-precision form only (null otherwise)
  const float *hinvf;   // [16][M] structured Hbar^{-1} rounded to FP32
  float *fbh, *fbl;     // [12][M] rest-frame rhs of the step, double-float (high, low parts)
  double *dqb;          // [12][M] rest-frame increment diag4(R^T) dq (FP64 accumulator)
  float *ubf;           // [12][M] FP32 Hbar^{-1} of the current rhs (u, then each correction)
  float *Rf;            // [9][M]  R rounded to FP32 (written with R)
  float *Rlo;           // [9][M]  R - Rf: R as a double-float pair (Rf, Rlo)
  // processing order of the per-body kernels that visit joints: thread t
  // handles body order[t] (null: body t); see CHUNK_ORDER
  const int32_t *order;
};

// joint flags
enum : uint8_t { JF_A_FREE = 1, JF_B_BODY = 2, JF_B_FREE = 4 };

// constraint rows of a joint type: ball 3, hinge 5, universal 4, prismatic 5
#ifdef __CUDACC__
__host__ __device__
#endif
inline int joint_nrows(int type) { return type == 1 || type == 3 ? 5 : (type == 2 ? 4 : 3); }

struct DevJoints {
  int32_t K;
  const int8_t *type;    // [K] 0 ball, 1 hinge, 2 universal, 3 prismatic
  const int32_t *ja;     // [K] internal body index of a
  const int32_t *jb;     // [K] internal body index of b, -1 for the world
  const uint8_t *flags;  // [K] JF_*
  const double *pa1;     // [3][K] anchor on a (rest frame)
  const double *pb1;     // [3][K] anchor on b (rest frame) or world point
  const double *pa2;     // [3][K] second on-axis point on a (hinge)
  const double *pb2;     // [3][K] second on-axis point on b (hinge); universal: l a2,
                         //        b's axis as a point difference
  const double *pa3;     // [3][K] prismatic: off-axis point p + l c on a (null: no prismatic joint)
  const double *pb3;     // [3][K] ... on b
  const double *ua;      // [3][K] unit hinge axis in a's rest frame
  double *RH;            // [9][K] hinge frame R_H, universal frame R_U or prismatic frame R_P
                         //        of the step
  double *c;             // [5][K] C(q_n)
  double *b;             // [5][K] dual rhs G u + C(q_n)
  double *lambda;        // [5][K] multipliers (rows beyond C_k are zero)
  double *qf;            // [15][K] MABD_JACOBIAN_FULL (null otherwise): per hinge / prismatic
                         //        row r the rest-frame vector qh_r (components [3r + i]) of
                         //        the frame's gradient term on body a (see full_frame_map)
  double *dlam;          // [5][K] mixed form: multiplier correction of a refinement sweep
  // mixed form: FP32 copies of the joint points and of the hinge frame
  const float *pa1f, *pb1f, *pa2f, *pb2f;  // [3][K]
  const float *pa3f, *pb3f;                // [3][K] (null: no prismatic joint)
  float *RHf;                              // [9][K]
  // processing order of the per-joint kernels: thread t handles joint
  // order[t] (null: joint t); see CHUNK_ORDER
  const int32_t *order;
  // the scene has universal or prismatic joints: the per-body and per-joint
  // kernels run their instantiation with those branches (the others carry
  // only the ball and hinge code, fewer registers)
  bool xj;
};

// Per-joint and per-body kernels run CTAs of CHUNK_ORDER threads over runs of
// CHUNK_ORDER consecutive entries; the processing order partitions each run
// stably by joint type (for a body: by the types of its joints, in incidence
// order), so that a warp sees a single type.  On this GPU an FP64
// instruction occupies a warp for the same time however many of its lanes
// are active, so a warp that mixes ball and hinge joints pays for both paths.
constexpr int CHUNK_ORDER = 128;

// body -> incident joints (CSR over internal body order)
struct DevIncidence {
  const int32_t *off;    // [M+1]
  const int32_t *joint;  // [nnz]
  const int8_t *side;    // [nnz] 0: body is a, 1: body is b
};

// chain dual blocks (block-tridiagonal, 5x5 padded, joint chain order)
struct DevChain {
  int32_t K;
  double *Dfirst;        // [15][K] contribution of the joint's lower body (path order)
  double *Dsecond;       // [15][K] contribution of its upper body
  double *B;             // [25][K] coupling of joint k and k+1 (through their shared body)
  const uint8_t *jflags; // [K] bit0: has lower-body part, bit1: has upper-body part, bit2: has B
  const int8_t *islot;   // [nnz] per incidence entry: 0 -> Dfirst, 1 -> Dsecond
  int32_t off;           // level-0 row n is joint n - off; rows n < off are identity rows
  // FP32 Gram parts for the FP32 reduction of the mixed form (else null)
  float *Dfirst_f, *Dsecond_f, *B_f;
  // loop solver: coupling of joint 0 (rows) and the loop breaker K - 1
  // (columns) through body 0 (5x5 padded); null otherwise
  double *corner;
};

// one level of block cyclic reduction (T: the reduction's precision)
template <typename T>
struct CRLevelT {
  int32_t N;             // rows at this level
  T *D;                  // [15][N] (level 0: assembled from DevChain)
  T *B;                  // [25][N]
  T *b;                  // [5][N]
  T *fac;                // [70][N/2] L, Ya, Yb, y of the odd rows
  T *lam;                // [5][N]
};
using CRLevel = CRLevelT<double>;

// tree (forest) of free bodies in breadth-first order: levels are contiguous
// ranges and the children of a body are a contiguous range
// S: the elimination's type (double: FP64 form; float: the FP32 elimination
// of the mixed form, refined by FP64 correction sweeps)
template <typename S>
struct DevTreeT {
  const int32_t *parent;      // [M] parent body (internal index) or -1
  const int32_t *pjoint;      // [M] joint to the parent (internal index) or -1
  const int8_t *pside;        // [M] side of the body in that joint (0: a, 1: b)
  const int32_t *cfirst;      // [M] first child
  const int32_t *ccount;      // [M] number of children
  const int32_t *root_id;     // [M] index among roots, -1 otherwise
  const int32_t *root_joint;  // [2][nroots] one-sided joints of a root (-1: none)
  const int8_t *root_side;    // [2][nroots]
  int32_t nroots;
  const int32_t *order;       // [nfree] per level: bodies with children, then leaves
  const int32_t *lv_lo;       // [levels + 1] first body of each level
  S *X;                       // [60][M]  Hhat^{-1} G^T in the rest frame (12 x 5)
  S *LD;                      // [15][M]  Cholesky factor of D = G Hhat^{-1} G^T
  S *y;                       // [12][M]  Hhat^{-1} fhat (rest frame)
  S *e;                       // [5][M]   G y + C(q_n)
  S *U;                       // [60][M]  P^T L_D^{-T} in the parent's rest frame (12 x 5)
  S *v;                       // [12][M]  P^T D^{-1} e in the parent's rest frame
  S *dq;                      // [12][M]  world-frame increment of the step
  S *rX;                      // [120][nroots] roots: Hhat^{-1} G_w^T (12 x 10)
  S *rLD;                     // [55][nroots]
  S *re;                      // [10][nroots]
  // right-hand side and outputs of one solve of the KKT system
  // [H G^T; G 0][dq; lambda] = [f; -crr c] (the body rhs enters as ubar = Hbar^{-1} fbar)
  const double *c;            // [5][K] joint values: C(q_n), or a correction's C + G dq
  double crr;                 // their weight: residual_rhs (0 or 1) for a step, 1 for a correction
  double *lam;                // [5][K] multipliers out (FP64)
  double *lam_acc;            // [5][K] multipliers also added here (null: not)
  double *dqb;                // [12][M] null: the state update (FP64 form); else the rest-frame
  int32_t dqb_add;            //   increment, written (0) or added (1)
};
using DevTree = DevTreeT<double>;

// the forest regrouped tree by tree for the persistent kernel: tree t has
// levels lvl[t] .. lvl[t] + nlvl[t] - 1 (records), record r covers
// order[lo[r], lo[r + 1]) with its bodies with children first (up to mid[r]);
// every tree's record list ends with a sentinel record
struct DevForest {
  int32_t ntrees;
  const int32_t *tlvl;   // [ntrees] first record of tree t
  const int32_t *tnl;    // [ntrees] levels of tree t
  const int32_t *lo;     // [records] start of a level in order (sentinels: end of the tree)
  const int32_t *mid;    // [records] first leaf of the level
  const int32_t *order;  // [free bodies] body ids
};

// dual-space preconditioned conjugate gradients (graphs).  Vectors are
// [5][K] (rows beyond C_k stay zero); scalars live on the device.
struct DevPCG {
  double *r, *z, *p, *Sp;     // [5][K]
  double *zb;                 // [12][M] Hbar^{-1} diag4(R^T) G^T p (rest frame)
  double *Lpre;               // [15][K] Cholesky of the diagonal blocks D_k
  double *part;               // [2][nblocks] per-block partial sums
  double *scal;               // [8]: rz, alpha, beta, rr, bnorm2, rtol2, pSp, spare
  int *iter;                  // [2]: iterations done, converged flag
  int nblocks;
};

// FP32 preconditioned conjugate gradients on the dual (mixed form on graphs):
// one solve of S x = rhs from x = 0, block-Jacobi preconditioned; vectors [5][K]
struct DevPCG32 {
  float *r, *z, *p, *Sp, *x;  // [5][K]
  float *zb;                  // [12][M]
  float *Lpre;                // [15][K] Cholesky of D_k, reciprocal diagonal
  double *part;               // [2][nblocks]
  double *scal;               // [8]: rz, alpha, beta, rr, bnorm2, rtol2, pSp, spare
  int *iter;                  // [2]: iterations done, converged flag
  int nblocks;
  // learned preconditioner (t null: block Jacobi): t = C r, y = G t
  float *t, *y;               // [5][K]
  const float *Cl;            // [K][6] inverse Cholesky factors C_k of the learned form
  // persistent solve: per-block partial sums [3][P32_MAXB] and the grid
  // barrier's words (arrivals, generation, error flag, spare)
  double *ppart;
  unsigned *bar;
};
constexpr int P32_MAXB = 4096;  // blocks of the persistent solve at most

// Learned block preconditioner of the dual PCG (k_lpc.cu), ball joints.
// Joints are the nodes of a graph whose edges join joints sharing a free
// body; S~ = C S C^T is the dual normalized by the inverse Cholesky factors
// C_k of its diagonal blocks, E_kk' its off-diagonal blocks.  A message-passing
// network over that graph gives per-edge weights alpha (edges to lower-index
// neighbours) and per-joint scales s; the preconditioner is
//   M^{-1} = C^T G^T G C,  G = diag(s) (I - A),  A_kk' = alpha_kk' E_kk' (k' < k).
constexpr int LPC_F = 8;    // input features per joint
constexpr int LPC_H = 64;   // hidden width
constexpr int LPC_R = 8;    // rank of the bilinear edge head
// parameter vector (FP32): W1 [2F][H], b1, W2 [2H][H], b2, W3 [2H][H], b3,
// Wa [H][R], Wb [H][R], wd [H], cd, we [2], ce
constexpr int LPC_OFF_W1 = 0;
constexpr int LPC_OFF_B1 = LPC_OFF_W1 + 2 * LPC_F * LPC_H;
constexpr int LPC_OFF_W2 = LPC_OFF_B1 + LPC_H;
constexpr int LPC_OFF_B2 = LPC_OFF_W2 + 2 * LPC_H * LPC_H;
constexpr int LPC_OFF_W3 = LPC_OFF_B2 + LPC_H;
constexpr int LPC_OFF_B3 = LPC_OFF_W3 + 2 * LPC_H * LPC_H;
constexpr int LPC_OFF_WA = LPC_OFF_B3 + LPC_H;
constexpr int LPC_OFF_WB = LPC_OFF_WA + LPC_H * LPC_R;
constexpr int LPC_OFF_WD = LPC_OFF_WB + LPC_H * LPC_R;
constexpr int LPC_OFF_CD = LPC_OFF_WD + LPC_H;
constexpr int LPC_OFF_WE = LPC_OFF_CD + 1;
constexpr int LPC_OFF_CE = LPC_OFF_WE + 2;
constexpr int LPC_NPARAM = LPC_OFF_CE + 1;

struct LpcGraph {
  int32_t K, nnz;
  const int32_t *off;       // [K+1] CSR over joints
  const int32_t *nbr;       // [nnz] adjacent joint
  const int32_t *body;      // [nnz] the shared free body
  const int8_t *sk, *sn;    // [nnz] side (0: a, 1: b) of the joint and of the neighbour on it
  const int32_t *rev;       // [nnz] entry of the neighbour that points back
  const uint8_t *onesided;  // [K] 1 if the joint has a single free body
};

constexpr int LPC_ES = 12;  // floats per stored block E_e: 3x3 row-major, padded for 16-byte loads

struct LpcAct {
  float *E;                     // [nnz][LPC_ES] E_kk' row-major (rows: joint k, columns: neighbour)
  float *C;                     // [K][6] inverse Cholesky factor of D_k, packed lower
  float *x;                     // [K][F]
  float *A1, *A2, *A3;          // [K][2F], [K][2H], [K][2H] layer inputs as multiplied (training)
  float *pre1, *pre2, *pre3;    // [K][H] pre-activations (training)
  float *h1, *h2, *h3;          // [K][H]
  float *a, *b;                 // [K][R]
  float *s;                     // [K]
  float *alpha;                 // [nnz] (entries to higher-index neighbours hold 0)
};

// vectors of the normalized-space PCG (k_pcgn.cu), one float4 per joint;
// r and p double-buffered
struct DevPCGN {
  float4 *r[2], *p[2], *q, *x, *y, *z;
  float *cu;  // [nnz] alpha of the reverse entry times s of the neighbour
};

struct LpcNet {
  const float *P;               // [LPC_NPARAM]
  const uint16_t *W1t, *W2t, *W3t;  // bf16 bits, transposed: [H][2F], [H][2H], [H][2H]
};

// Segment-tiled form of the chain solve (k_seg.cu; the mixed form with the
// FP32 reduction).  The dual rows (joints in path order) are cut into tiles of
// SEG_T rows; one CTA per tile does the tile's per-body and per-joint work and
// eliminates the tile's rows by block cyclic reduction in shared memory down
// to its first row.  Row t of the next level's system is tile t's first row:
//   D_t = Dn[t] + Da[t-1],  coupling to row t + 1: Bn[t],
//   b_t = bn[t] + ba[t-1] (+ fl32(b0[t] + dl[t-1]) above the level-0 tiles),
// (Da, ba: what tile t's eliminations add to tile t + 1's first row; b0, dl:
// the level-0 first row's own rhs and the part that the previous tile's last
// body contributes, kept in FP64 so that the correction's rhs, a difference of
// nearly equal parts, is summed before it is rounded).  Upper systems are
// reduced the same way by tiles of SEG_UP_T rows until one tile holds them.
constexpr int SEG_T = 64;
constexpr int SEG_UP_T = 256;

struct SegRhs {
  float *bn, *ba;      // [5][N]
  double *b0, *dl;     // [5][N] (level-0 tiles only, else null)
  float *lam;          // [5][N] multipliers of the tiles' first rows (solution of the next level)
};

struct SegLevel {
  int32_t N;           // tiles of this level = rows of the next level's system
  float *Dn, *Da;      // [15][N] packed lower 5x5
  float *Bn;           // [25][N] row-major 5x5
  SegRhs r[2];         // pass 0: the approximate solve, pass 1: the correction
};

// per-joint flags of the chain in path order: the joint's lower and upper
// path bodies exist (a body of the joint), body a is the lower one, hinge
enum : uint8_t { SEGJ_LO = 1, SEGJ_UP = 2, SEGJ_A_LO = 4, SEGJ_HINGE = 8 };

struct SegChain {
  int32_t nb;          // chain bodies (path order 0 .. nb - 1)
  int32_t sigma;       // joint k joins path bodies k - 1 + sigma (lower) and k + sigma (upper)
  const uint8_t *cjf;  // [K] SEGJ_* flags
  float *ytile;        // [5][K] forward-eliminated rhs of the eliminated rows of the current pass
  float *lam0;         // [5][K] multipliers of the approximate solve
  float *dq0, *z;      // [12][nb] rest-frame increment of the approximate solve; the correction's Hbar^{-1} r
  float *u;            // [12][nb] u = Hbar^{-1} fbar (FP32)
  float *rf;           // [12][nb] fbar - Hbar u (its residual, from double-float, rounded to FP32)
  float *RHlo;         // [9][K] hinge frames as double-float pairs (J.RHf, RHlo)
  float *fac;          // [tiles][65][SEG_T + 4] each level-0 tile's factors (written by FIRST)
  SegLevel lv0;        // level-0 tile outputs
  int32_t write_cj;    // also write J.c and J.RH in FP64 (residual statistics)
  unsigned long long *refine_max;   // max |C + G dq| of the approximate solve (null: not wanted)
  unsigned long long *polar_iters;  // Newton steps of the polar rotation, summed (null: not wanted)
};

struct StepParams {
  double h, inv_h;
  double g[3];
  int32_t residual_rhs;
  int32_t rot_norm;  // 1: unconstrained solve by Alg. 1 (MABD_ROTATION_NORMALIZED)
};

// kernel launchers (k_body.cu)
// iters (may be null): += Newton iterations of the polar decomposition, summed over bodies
void launch_body_prep(const DevBodies &B, const StepParams &p, int *status, cudaStream_t s,
                      unsigned long long *iters = nullptr);
void launch_joint_prep(const DevBodies &B, const DevJoints &J, const StepParams &p, int *status,
                       cudaStream_t s);
void launch_backprop(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                     const StepParams &p, int *status, cudaStream_t s);
void launch_residuals(const DevBodies &B, const DevJoints &J, const StepParams &p,
                      unsigned long long *maxbits /*2*/, int *status, cudaStream_t s);
// stage: q then qdot, [M][12] each in user order; the affine part of every
// body with has_frame[j] times frames[j] (to_lib: caller -> principal frame)
// or its transpose (principal -> caller)
void launch_stage_frames(double *stage, int M, const double *frames, const uint8_t *has_frame,
                         bool to_lib, cudaStream_t s);

// state transfer (k_body.cu): stage = the caller's q then qdot, [M][12] each
// in user body order; boi[internal] = user body index
void launch_state_check(const double *stage, size_t n, int *flag, cudaStream_t s);
void launch_state_in(const double *stage, const int32_t *boi, const DevBodies &B, cudaStream_t s);
void launch_state_out(const DevBodies &B, const int32_t *boi, double *stage, cudaStream_t s);

// chain (k_chain.cu): per-body Gram blocks, then block cyclic reduction.
// Level 0 reads D = Dfirst + Dsecond (+ identity on the padded rows of ball
// joints), B and the joint rhs b directly; its multipliers go to J.lambda.
void launch_chain_gram(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                       const DevChain &C, cudaStream_t s);
void launch_cr_reduce(const DevChain &C, const DevJoints &J, const CRLevel &cur, int level,
                      double *cL, double *cR, double *Bn, int *status, cudaStream_t s);
void launch_cr_combine(const DevChain &C, const DevJoints &J, const CRLevel &cur, int level,
                       const CRLevel &next, const double *cL, const double *cR,
                       const double *Bn, cudaStream_t s);
// reduce + combine of one level in a single launch (fused form of the two
// above); T = double or float (the reduction's precision)
template <typename T>
void launch_cr_level(const DevChain &C, const DevJoints &J, const CRLevelT<T> &cur, int level,
                     const CRLevelT<T> &next, int *status, cudaStream_t s);
// the single remaining row; out64 (FP64, with acc) when the top row is level 0
template <typename T>
void launch_cr_top(const DevChain &C, const DevJoints &J, const CRLevelT<T> &top, int level,
                   int *status, cudaStream_t s, double *out64 = nullptr, double *acc = nullptr);
// back-substitution of `level`; level 0 writes its rows n >= C.off to
// J.lambda (FP64) and, when acc is not null, also adds them to acc ([5][K])
template <typename T>
void launch_cr_back(const DevChain &C, const DevJoints &J, const CRLevelT<T> &cur, const CRLevelT<T> &next,
                    int level, cudaStream_t s, double *acc = nullptr);
// new right-hand side through the stored factors: forward elimination of
// `level` (level 0 reads J.b) writing next.b and the odd rows' y; the top
// row and the back-substitution then run as for a factorization
template <typename T>
void launch_cr_rhs(const DevChain &C, const DevJoints &J, const CRLevelT<T> &cur, int level,
                   const CRLevelT<T> &next, cudaStream_t s);
// levels with at most this many rows run in the single-CTA tail (FP32 reduction)
constexpr int CR_TAIL_ROWS = 512;
// levels l0 .. nl-1 of a pass (elimination, or right-hand side when rhs_only),
// the top row and their back-substitution in one single-CTA launch; d_lv is a
// device copy of the level array, cL/cR/Bn scratch of (20, 20, 25) x (rows of
// level l0) / 2; level 0 (when l0 = 0) writes to Jout.lambda and acc
template <typename T>
void launch_cr_tail(const DevChain &C, const DevJoints &J, const DevJoints &Jout, const CRLevelT<T> *d_lv,
                    int l0, int nl, bool rhs_only, T *cL, T *cR, T *Bn, int *status, double *acc,
                    cudaStream_t s);

// loop solver (k_loop.cu): column t of the breaker's coupling as a chain
// rhs ([5][K], only joints 0 and K-2 written), the chain's solution at joints
// 0 and K-2 into w[10 t..], and the breaker's Schur complement solve
void launch_loop_column(const DevChain &C, int K, double *rb, int t, cudaStream_t s);
void launch_loop_gather(int K, const double *x, double *w, int t, cudaStream_t s);
void launch_loop_schur(const DevChain &C, const DevJoints &J, const double *w, int *status, cudaStream_t s);

// FP32 PCG (k_pcg32.cu): setup from rhs (FP64 [5][K]), iterations, and the
// final copy of x to out (FP64 [5][K]) with acc += x when acc is given
// (lg, la: the learned preconditioner when P.t is set)
struct LpcGraph;
struct LpcAct;
void launch_p32_setup(const DevBodies &B, const DevJoints &J, const DevPCG32 &P, const double *rhs,
                      double rtol, int *status, cudaStream_t s, const LpcGraph *lg = nullptr,
                      const LpcAct *la = nullptr);
void launch_p32_iteration(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                          const DevPCG32 &P, int max_iters, cudaStream_t s, const LpcGraph *lg = nullptr,
                          const LpcAct *la = nullptr);
void launch_p32_finish(const DevJoints &J, const DevPCG32 &P, double *out, double *acc, cudaStream_t s);
// the whole solve in one cooperative launch of nblocks co-resident blocks
// (p32_persist_blocks: the most that fit, 0 if the query fails)
int p32_persist_blocks(bool xj, bool lpc);
cudaError_t launch_p32_persist(const DevBodies &B, const DevJoints &J, const DevIncidence &I, const DevPCG32 &P,
                               const LpcGraph *lg, const LpcAct *la, const double *rhs, double rtol,
                               int max_iters, double *out, double *acc, int *status, int nblocks, cudaStream_t s);

// FP32 PCG of a ball-joint graph in the normalized dual space, the whole
// solve in one cooperative launch (k_pcgn.cu), from x0 when given; needs the
// current C and E of launch_lpc_blocks (and, lpc, the network's alpha and s)
int pcgn_blocks(bool lpc);
cudaError_t launch_pcgn(const LpcGraph &G, const LpcAct &A, const DevPCGN &V, const DevPCG32 &P, bool lpc,
                        const double *rhs, const double *x0, double rtol, int max_iters, double *out, double *acc,
                        int *status, int nblocks, cudaStream_t s);

// learned preconditioner (k_lpc.cu)
// C_k and the normalized blocks E of the current state (needs R/Rf, hinvf)
void launch_lpc_blocks(const DevBodies &B, const DevJoints &J, const LpcGraph &G, const LpcAct &A,
                       int *status, cudaStream_t s);
// bf16 transposed copies of the layer weights from P
void launch_lpc_weights(const float *P, uint16_t *W1t, uint16_t *W2t, uint16_t *W3t, cudaStream_t s);
// features, three message-passing layers, heads: alpha and s (training: also
// keeps the layer inputs and pre-activations)
void launch_lpc_forward(const LpcGraph &G, const LpcNet &N, const LpcAct &A, bool keep, cudaStream_t s);
// z = M^{-1} r for PCG vectors [5][K] (rows 0-2): t = C r is formed by the
// caller's kernel; y = G t (tmp), z = C^T G^T y, partial sums of r.z per block
void launch_lpc_apply(const LpcGraph &G, const LpcAct &A, const float *t, float *y, const float *r,
                      float *z, double *part, int nblocks, cudaStream_t s, const int *iter);

// training (k_lpc_train.cu): work arrays of one batch
struct LpcTrainWork {
  int nv;
  const float *V;                    // [nv][K][3]
  float *t, *u, *w, *q, *gw, *gu;    // [nv][K][3]
  float *dalpha;                     // [nnz]
  float *ds;                         // [K]
  float *dh, *dh2;                   // [K][H]
  float *dA;                         // [K][2H]
  float *dpre;                       // [K][H]
  float *grad;                       // [NPARAM]
  double *part;                      // [2][nblocks]
  double *loss;                      // [2]
};

void launch_lpc_probe(float *V, size_t n, uint64_t seed, cudaStream_t s);
// kind 0: Frobenius objective, 1: Kaporin objective; W.loss[0..1] receive the
// sums the loss is formed from (see k_lpc_train.cu)
void launch_lpc_loss_grad(const LpcGraph &G, const LpcAct &A, const LpcNet &N, const LpcTrainWork &W,
                          int kind, bool grad, cudaStream_t s);
void launch_lpc_adam(float *P, const float *g, float *m, float *v, float lr, int step, cudaStream_t s);

// mixed-precision form of the chain step (k_mixed.cu)
void launch_mx_body_prep(const DevBodies &B, const StepParams &p, int *status, cudaStream_t s,
                         unsigned long long *iters = nullptr);
void launch_mx_joint_prep(const DevBodies &B, const DevJoints &J, const StepParams &p, int *status,
                          cudaStream_t s);
void launch_mx_chain_gram(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                          const DevChain &C, cudaStream_t s, bool f32_blocks = false);
// where a sweep's increment dqb comes from: the approximate solve's u and
// lambda (first chain sweep), the previous correction z and dlambda (later
// chain sweeps), or dqb itself (the tree elimination writes it)
enum { MX_FROM_U = 0, MX_FROM_CORRECTION = 1, MX_FROM_DQB = 2 };
void launch_mx_res_body(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                        const StepParams &p, int mode, cudaStream_t s);
// add_gz: b = G z + (C + G dq) (the chain's dual rhs); false: b = C + G dq
// (the joint values of the tree's correction solve)
void launch_mx_res_joint(const DevBodies &B, const DevJoints &J, const StepParams &p,
                         unsigned long long *maxbit, cudaStream_t s, bool add_gz = true);
void launch_mx_final(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                     const StepParams &p, int mode, cudaStream_t s);

// segment-tiled chain step (k_seg.cu): the level-0 tile kernels of the three
// passes (approximate solve; back-substitution, residuals and the correction's
// rhs; correction back-substitution and state update) and the tile kernels of
// the upper systems (reduce: tiles of `in`'s rows into `out`; top: all of
// `in`'s rows in one CTA; back: `in`'s rows given `next`'s solution)
enum { SEG_FIRST = 0, SEG_CORR = 1, SEG_FINAL = 2 };
// per body: polar rotation, rest-frame rhs, u and its residual; per joint
// (by its body a): the hinge frame and C(q_n)
void launch_seg_body(const DevBodies &B, const DevJoints &J, const StepParams &p, const SegChain &S, int *status,
                     cudaStream_t s);
void launch_seg_tiles(int mode, const DevBodies &B, const DevJoints &J, const StepParams &p, const SegChain &S,
                      int *status, cudaStream_t s);
// (T: rows per tile of the upper systems, a power of two, 2 .. SEG_UP_T)
void launch_seg_up_reduce(const SegLevel &in, const SegLevel &out, int T, int pass, bool write_db,
                          unsigned long long *rmax, int *status, cudaStream_t s);
void launch_seg_up_top(const SegLevel &in, int T, int pass, unsigned long long *rmax, int *status,
                       cudaStream_t s);
void launch_seg_up_back(const SegLevel &in, const SegLevel &next, int T, int pass, int *status, cudaStream_t s);
// sets the kernels' shared-memory limits (once per process and device)
cudaError_t seg_init();

// tree (k_tree.cu): one launch per level, deepest first, then root first;
// level [lo, hi) of the body order T.order (roots = true: the roots' level,
// bodies lo .. hi - 1); a 16-lane group per body of the upward pass
// whole tree elimination (upward and downward passes) of every tree of the
// forest in one launch, one block of `threads` (128, 64 or 32) per tree
// (S = double or float, the elimination's type, for these three launchers)
template <typename S>
void launch_tree_forest(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, const DevForest &F,
                        const StepParams &p, int *status, cudaStream_t s, int threads);
template <typename S>
void launch_tree_up(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int lo, int hi, bool roots,
                    const StepParams &p, int *status, cudaStream_t s);
template <typename S>
void launch_tree_down(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int lo, int hi,
                      const StepParams &p, int *status, cudaStream_t s);
// narrow levels [la, lb) of the downward pass, root first, in one block
template <typename S>
void launch_tree_down_run(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int la, int lb,
                          const StepParams &p, cudaStream_t s);

// PCG (k_pcg.cu)
void launch_pcg_setup(const DevBodies &B, const DevJoints &J, const DevPCG &P, double rtol,
                      int *status, cudaStream_t s);
void launch_pcg_iteration(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                          const DevPCG &P, int max_iters, cudaStream_t s);

}  // namespace mabd
