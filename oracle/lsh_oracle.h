/*
 * lsh_oracle.h -- plain, slow FP64 CPU oracle for the Galerkin-discretised
 * Lippmann-Schwinger (LS) equation of Brisard & Legoll, "Periodic
 * homogenization using the Lippmann-Schwinger formalism" (arXiv:1411.0330).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may include, link or call this code.  Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark use it.  It shares
 * no code, table or constant with the GPU path.
 *
 * What it computes (paper section / equation in brackets):
 *   - the discrete system, Eq. (13): for every voxel beta in I0,
 *       (A_beta - A0)^{-1} tau_beta + DFT^{-1}[ Gamma_k tau_k ]_beta = p,
 *     with tau = 0 off I0 (Eq. (4), second line);
 *   - the approximate discrete Green operators of Sec. 3.2: truncated
 *     (Eqs. (14)-(15) plus the Nyquist rule), filtered (Sec. 3.2.2) and the
 *     finite-difference one (Sec. 3.2.3);
 *   - A*_h p = A0 p + h^d sum_beta tau_beta  (Eq. (tau_Astar), Theorem 13);
 *   - the real-space form Eq. (12) by direct summation, for a dense solve.
 *
 * Layout: every field is component-major, [c][n2][n1][n0], axis 0 fastest.
 * Elasticity uses Mandel components (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12).
 */
#ifndef LSH_ORACLE_H
#define LSH_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_SCALAR = 0, OR_ELASTIC = 1 };
/* OR_CONSISTENT: the consistent discrete Green operator of Eq. (11) (2D scalar
 * problems with a diagonal A0 only; not a GPU operator: a check of the others) */
enum { OR_TRUNCATED = 0, OR_FILTERED = 1, OR_FINITE_DIFF = 2, OR_CONSISTENT = 3 };
enum { OR_SOLVER_AUTO = 0, OR_SOLVER_CG = 1, OR_SOLVER_MINRES = 2 };
enum {
  OR_OK = 0,
  OR_ERR_ARG = 1,
  OR_ERR_SINGULAR = 2,     /* A_beta - A0 neither zero nor invertible */
  OR_ERR_REFERENCE = 3,    /* A0 not symmetric positive definite */
  OR_ERR_BREAKDOWN = 4,
  OR_ERR_NOT_CONVERGED = 5,
  OR_ERR_TOO_LARGE = 6,
  OR_ERR_NOMEM = 7
};

typedef struct {
  int dim;                     /* 2 or 3 */
  int n[3];                    /* cells per axis; n[2] is ignored for dim 2 */
  int physics;                 /* OR_SCALAR (c = dim) or OR_ELASTIC (dim 3, c = 6) */
  int green;                   /* OR_TRUNCATED, OR_FILTERED, OR_FINITE_DIFF, OR_CONSISTENT */
  int nphase;
  const double *phase_moduli;  /* scalar: dim*dim symmetric matrix per phase;
                                  elastic: (bulk K, shear mu) per phase        */
  const double *ref_moduli;    /* A0 in the same format as one phase            */
  const unsigned char *phase;  /* phase id per voxel                            */
  const double *scale;         /* optional: A_beta = scale_beta * A_phase, or NULL */
  const double *frac;          /* optional (two phases, neither equal to A0): volume
                                  fraction f_beta of phase 1 in voxel beta; the local
                                  operator is then the voxel average of (A(x) - A0)^{-1},
                                  Eq. (def_ah): f M_1 + (1 - f) M_0; NULL otherwise   */
} or_problem;

int or_ncomp(const or_problem *p);
long or_nvox(const or_problem *p);

/* Default reference medium: half the softest phase, see the function body. */
int or_default_reference(int dim, int physics, int nphase, const double *phase_moduli,
                         double *ref_out);

/* Per-voxel local operator M_beta = (A_beta - A0)^{-1} (Eq. (7); with `frac`
 * the average over the voxel, Eq. (def_ah)), c*c per voxel, and the I0 indicator. */
int or_local_operator(const or_problem *p, double *M, unsigned char *active);

/* Continuous Green operator at a nonzero frequency xi (Sec. 2.2.1):
 * scalar xi xi^T / (xi^T A0 xi); elastic: its strain-polarisation analogue. */
void or_gamma0(const or_problem *p, const double xi[3], double *G);

/* Discrete Green operator Gamma^h_k, k in {0..n-1}^d, c*c row-major complex
 * (interleaved re/im; the truncated and filtered operators are real, the
 * finite-difference one is Hermitian). */
void or_gamma_hat(const or_problem *p, const int k[3], double *G);

/* Unnormalised forward (sign -1) or backward (sign +1) multi-dimensional DFT
 * of a complex array (interleaved re/im) of shape n (axis 0 fastest).  Uses a
 * radix-2 FFT along power-of-two axes and a direct sum along the others. */
void or_dft(int dim, const int n[3], int sign, double *data);

/* Direct O(N^{2d}) DFT by definition, for pinning or_dft on tiny grids. */
void or_dft_naive(int dim, const int n[3], int sign, const double *in, double *out);

/* y = P (M x + DFT^{-1}[Gamma_k DFT(P x)_k]) with P the projection on I0. */
int or_apply(const or_problem *p, const double *x, double *y);

/* Solve Eq. (13) for the macroscopic field `load` (c values).  tau (c*V) is
 * the output.  Stops when ||r||_2 <= tol ||b||_2.  info[0] = iterations,
 * info[1] = final relative residual (as double bits in a double array). */
int or_solve(const or_problem *p, const double *load, double *tau, double tol, int maxit,
             int solver, double *info);

/* Dense route: assemble Eq. (12) by direct summation and solve by LU. */
int or_dense_solve(const or_problem *p, const double *load, double *tau);

/* A*_h from c solves with unit loads.  Astar is c*c row-major:
 * Astar[i*c+j] = e_i . A*_h e_j.  tau_all (c*c*V) may be NULL.  info gets
 * 2 doubles per load (iterations, relative residual). */
int or_effective(const or_problem *p, double tol, int maxit, int solver, double *Astar,
                 double *tau_all, double *info);

/* Variational estimate e_i.A*e_j = A0_ij + h^d (b_i.tau_j + b_j.tau_i - tau_i.K tau_j). */
int or_effective_variational(const or_problem *p, const double *tau_all, double *Astar);

/* Gradient of sum_ij W_ij e_i.A*_h e_j with respect to a per-voxel scale s_beta
 * (A_beta = s_beta A_phase): g_beta = h^d sum_ij W_ij eps_i,beta . A_phase eps_j,beta,
 * eps_j = M tau_j.  tau_all holds the c solutions; W is c*c. */
int or_scale_gradient(const or_problem *p, const double *tau_all, const double *W, double *grad);

#ifdef __cplusplus
}
#endif
#endif
