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
};

// joint flags
enum : uint8_t { JF_A_FREE = 1, JF_B_BODY = 2, JF_B_FREE = 4 };

struct DevJoints {
  int32_t K;
  const int8_t *type;    // [K] 0 ball, 1 hinge
  const int32_t *ja;     // [K] internal body index of a
  const int32_t *jb;     // [K] internal body index of b, -1 for the world
  const uint8_t *flags;  // [K] JF_*
  const double *pa1;     // [3][K] anchor on a (rest frame)
  const double *pb1;     // [3][K] anchor on b (rest frame) or world point
  const double *pa2;     // [3][K] second on-axis point on a (hinge)
  const double *pb2;     // [3][K] second on-axis point on b (hinge)
  const double *ua;      // [3][K] unit hinge axis in a's rest frame
  double *RH;            // [9][K] hinge frame of the step
  double *c;             // [5][K] C(q_n)
  double *b;             // [5][K] dual rhs G u + C(q_n)
  double *lambda;        // [5][K] multipliers (rows beyond C_k are zero)
};

// body -> incident joints (CSR over internal body order)
struct DevIncidence {
  const int32_t *off;    // [M+1]
  const int32_t *joint;  // [nnz]
  const int8_t *side;    // [nnz] 0: body is a, 1: body is b
};

// chain dual blocks (block-tridiagonal, 5x5 padded, joint chain order)
struct DevChain {
  int32_t K;
  double *Dfirst;        // [15][K] contribution of the body for which the joint is its first
  double *Dsecond;       // [15][K] ... its second joint
  double *B;             // [25][K] coupling of joint k and k+1 (through their shared body)
  const uint8_t *jflags; // [K] bit0: has first-body part, bit1: has second-body part, bit2: has B
};

// one level of block cyclic reduction
struct CRLevel {
  int32_t N;             // rows at this level
  double *D;             // [15][N] (level 0: assembled from DevChain)
  double *B;             // [25][N]
  double *b;             // [5][N]
  double *fac;           // [70][N/2] L, Ya, Yb, y of the odd rows
  double *lam;           // [5][N]
};

struct StepParams {
  double h, inv_h;
  double g[3];
  int32_t residual_rhs;
};

// kernel launchers (k_body.cu)
void launch_body_prep(const DevBodies &B, const StepParams &p, int *status, cudaStream_t s);
void launch_joint_prep(const DevBodies &B, const DevJoints &J, const StepParams &p, int *status,
                       cudaStream_t s);
void launch_backprop(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                     const StepParams &p, int *status, cudaStream_t s);
void launch_residuals(const DevBodies &B, const DevJoints &J, const StepParams &p,
                      unsigned long long *maxbits /*2*/, int *status, cudaStream_t s);

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
void launch_cr_top(const DevChain &C, const DevJoints &J, const CRLevel &top, int level,
                   int *status, cudaStream_t s);
void launch_cr_back(const CRLevel &cur, const CRLevel &next, cudaStream_t s);

}  // namespace mabd
