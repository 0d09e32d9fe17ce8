/*
 * CPU FP64 oracle for one M-ABD time step -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded C written from the paper's equations
 * (M-ABD, arXiv 2603.08079, Sec. 3-5).  Only the test-suite, the package's
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table or helper with the CUDA library.
 *
 * Matrices are dense row-major doubles.  Affine coordinates follow Eq. abd_dof:
 * q = [vec(A); t] with vec stacking the columns of A, so A(r,c) = q[3c+r].
 */
#ifndef MABD_ORACLE_H
#define MABD_ORACLE_H
#include <stdint.h>

#define ORA_OK 0
#define ORA_ERR_ARG 1
#define ORA_ERR_NOT_SPD 5
#define ORA_ERR_INVERTED 6
#define ORA_ERR_NONFINITE 7
#define ORA_ERR_NO_CONV 8
#define ORA_ERR_TOPOLOGY 10

#define ORA_WORLD (-1)

enum { ORA_SOLVER_AUTO = 0, ORA_SOLVER_CHAIN = 1, ORA_SOLVER_TREE = 2,
       ORA_SOLVER_CG = 3, ORA_SOLVER_DENSE = 4 };

typedef struct {
  int64_t M, K;
  double h;
  double g[3];
  int32_t residual_rhs;      /* 1: KKT bottom rhs is -C(q_n) (Sec. 5 footnote) */
  const double *mass;        /* M */
  const double *second_moment; /* 6M: xx yy zz xy xz yz about the COM */
  const double *volume, *young, *poisson; /* M each */
  const int32_t *fixed;      /* M */
  const int32_t *jtype;      /* K: 0 ball, 1 hinge, 2 universal, 3 prismatic */
  const int64_t *body_a, *body_b; /* K; body_b may be ORA_WORLD */
  const double *anchor_a, *anchor_b, *axis_a, *axis_b; /* 3K each */
  const double *axis_len;    /* K */
  const double *ref_a, *ref_b; /* 3K each: prismatic reference directions normal to the axis */
  /* 0: every world <-> rest rotation by the polar R (Eq. polar); 1: the
     unconstrained solve H_A^{-1} f by Alg. 1 (the per-vector length-preserving
     map of Eq. len_preserving), the dual operator and the constraint forces
     by R (a linear H_A^{-1} is needed there) */
  int32_t rotation_mode;
  /* 0: frozen-frame Jacobian (Eq. pcpq); 1: full gradient of Eq.
     constraint_gradient, the joint frame attached to body alpha's polar
     rotation (Eq. r_gradient); hinge and prismatic joints (universal: error) */
  int32_t jacobian_mode;
} ora_scene;

typedef struct {
  double lin_residual;   /* max_k |G dq + c|_inf */
  double joint_residual; /* max_k |C_k(q_{n+1})|_inf */
  int32_t solver_used;
  int32_t cg_iters;
  double cg_rel_residual;
} ora_stats;

/* Sec. 3.2 / 3.3 building blocks */
int ora_mass_matrix(double m, const double S[6], double MA[144]);
int ora_stiffness_matrix(double V, double E, double nu, double KA[144]);
int ora_system_matrix(double m, const double S[6], double V, double E, double nu,
                      double h, double H[144]);
int ora_cholesky12(const double A[144], double L[144]);
int ora_polar(const double A[9], double R[9], int32_t *iters);
void ora_elastic_stress(const double F[9], double mu, double lam, double P[9]);
int ora_body_rhs(const ora_scene *sc, int64_t j, const double *q, const double *qd,
                 double f[12], double R[9]);
void ora_hinge_frame(const double a[3], double RH[9]);
/* constraint value and frozen-frame Jacobian of joint k (Eq. ball, hinge, pcpq) */
int ora_joint_eval(const ora_scene *sc, const double *q, int64_t k, double c[5],
                   double Ga[60], double Gb[60], int32_t *rows);
int64_t ora_dual_rows(const ora_scene *sc);
/* Alg. 1: one body's unconstrained solve u = H_A^{-1} f with every rotation
   of a 3-block replaced by A (resp. A^T) rescaled to keep the block's
   length; L = Cholesky factor of Hbar_A, A the body's affine matrix */
void ora_alg1_solve(const double L[144], const double A[9], const double f[12], double u[12]);
/* C_k(q) with the joint frame attached to body alpha as it is at q_ref:
   R_J(q) = R_J(q_ref) R_alpha(q_ref) R_alpha(q)^T (Eq. r_gradient's reading
   of R_H as a constant rotation times alpha's R^T); ball joints: C(q) */
int ora_joint_eval_attached(const ora_scene *sc, const double *q_ref, const double *q, int64_t k,
                            double c[5]);
int ora_topology(const ora_scene *sc);   /* 1 chain, 2 tree/forest, 3 graph, <0 error */

/* dense assembly for small systems: Hw (M*144, world-frame H_A), f (12M),
   G (rows x 12M, row-major), c (rows) */
int ora_assemble_dense(const ora_scene *sc, const double *q, const double *qd,
                       double *Hw, double *f, double *G, double *c);

/* one implicit step, one Newton iteration (Eq. kkt, dual, recover) */
int ora_step(const ora_scene *sc, int32_t solver, const double *q, const double *qd,
             double *q_out, double *qd_out, double *lambda, ora_stats *st);

#endif
