/*
 * lsh_oracle.c -- plain, slow FP64 CPU oracle for the Galerkin-discretised
 * Lippmann-Schwinger equation (Brisard & Legoll, arXiv:1411.0330).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline leg of bench.py.  The product path never includes or links it.
 *
 * Every routine follows the plain definition written in the paper: the DFT
 * sums of Sec. 3.1, the Green operators of Sec. 3.2, the linear system of
 * Eq. (13), and A*_h of Theorem 13.  No blocking, no fusion, no symmetry
 * shortcuts beyond what those definitions state.  Reductions use Neumaier
 * compensated summation.  Loops over independent frequencies / voxels may run
 * under OpenMP; every reduction is serial so results are reproducible.
 *
 * Readings of points the paper leaves open:
 *  - DFT^{-1} carries the factor 1/N^d (forced by Eqs. (8) and (10)).
 *  - Truncated operator, even N: every k with some k_i = N_i/2 gets A0^{-1}
 *    (Sec. 3.2.1, last paragraph); for elasticity this is C0^{-1}.
 *  - Filtered operator: k runs over {0..N-1}^d as in the DFT sums, the
 *    Gamma0(0) term is 0, and for unequal N_i the frequency is k_i + n_i N_i.
 *  - Elastic Gamma0 is the strain/polarisation Green operator of an isotropic
 *    reference medium (the paper only prints the scalar one).
 *  - Voxels with A_beta = A0 exactly are outside I0: tau = 0 there (Eq. (4)).
 */
#include "lsh_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------- */
/* small helpers                                                             */
/* ------------------------------------------------------------------------- */

typedef struct { double s, c; } ksum;

static void ksum_add(ksum *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static double ksum_get(const ksum *a) { return a->s + a->c; }

static double dot_comp(const double *a, const double *b, long n) {
  ksum s = {0.0, 0.0};
  for (long i = 0; i < n; ++i) ksum_add(&s, a[i] * b[i]);
  return ksum_get(&s);
}

int or_ncomp(const or_problem *p) { return p->physics == OR_ELASTIC ? 6 : p->dim; }

long or_nvox(const or_problem *p) {
  long v = (long)p->n[0] * p->n[1];
  if (p->dim == 3) v *= p->n[2];
  return v;
}

static void grid_dims(const or_problem *p, int n[3]) {
  n[0] = p->n[0];
  n[1] = p->n[1];
  n[2] = (p->dim == 3) ? p->n[2] : 1;
}

/* Mandel index pairs: 11, 22, 33, 23, 13, 12. */
static const int MANDEL_I[6] = {0, 1, 2, 1, 0, 0};
static const int MANDEL_J[6] = {0, 1, 2, 2, 2, 1};

static double mandel_w(int I) { return I < 3 ? 1.0 : sqrt(2.0); }

/* Isotropic Hooke tensor C_ijkl = lambda d_ij d_kl + mu (d_ik d_jl + d_il d_jk)
 * written as a 6x6 Mandel matrix C_IJ = w_I w_J C_{i(I) j(I) k(J) l(J)}. */
static void iso_mandel(double K, double mu, double *C) {
  double lam = K - 2.0 * mu / 3.0;
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      int i = MANDEL_I[I], j = MANDEL_J[I], k = MANDEL_I[J], l = MANDEL_J[J];
      double dij = (i == j), dkl = (k == l), dik = (i == k), djl = (j == l), dil = (i == l),
             djk = (j == k);
      C[I * 6 + J] = mandel_w(I) * mandel_w(J) * (lam * dij * dkl + mu * (dik * djl + dil * djk));
    }
}

/* Material matrix (c*c) of one phase / the reference, in the component basis. */
static void material_matrix(const or_problem *p, const double *mod, double *A) {
  int c = or_ncomp(p);
  if (p->physics == OR_ELASTIC) iso_mandel(mod[0], mod[1], A);
  else
    for (int i = 0; i < c * c; ++i) A[i] = mod[i];
}

/* Gauss-Jordan inverse with partial pivoting.  Returns 0 on success. */
static int mat_inverse(int n, const double *A, double *Ainv) {
  double a[36 * 2];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j)
      a[i * 2 * n + j] = (j < n) ? A[i * n + j] : (double)(j - n == i);
  double scale = 0.0;
  for (int i = 0; i < n * n; ++i) scale = fmax(scale, fabs(A[i]));
  if (!(scale > 0.0)) return 1;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(a[r * 2 * n + col]) > fabs(a[piv * 2 * n + col])) piv = r;
    if (fabs(a[piv * 2 * n + col]) <= 1e-13 * scale) return 1;
    if (piv != col)
      for (int j = 0; j < 2 * n; ++j) {
        double t = a[col * 2 * n + j];
        a[col * 2 * n + j] = a[piv * 2 * n + j];
        a[piv * 2 * n + j] = t;
      }
    double d = a[col * 2 * n + col];
    for (int j = 0; j < 2 * n; ++j) a[col * 2 * n + j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = a[r * 2 * n + col];
      if (f == 0.0) continue;
      for (int j = 0; j < 2 * n; ++j) a[r * 2 * n + j] -= f * a[col * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = a[i * 2 * n + n + j];
  return 0;
}

/* Cholesky test: 1 if the symmetric matrix is positive definite. */
static int is_spd(int n, const double *A) {
  double L[36];
  memset(L, 0, sizeof(L));
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) return 0;
    L[j * n + j] = sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / L[j * n + j];
    }
  }
  return 1;
}

/* ------------------------------------------------------------------------- */
/* reference medium                                                          */
/* ------------------------------------------------------------------------- */

/* Default reference medium, following the choice of Sec. 5 / Table 3 of the
 * paper (mu0 = mu_m / 2 with mu_m the softest shear modulus, nu0 = 0.3):
 *   elastic: mu0 = min_phase(mu) / 2, nu0 = 0.3, K0 = 2 mu0 (1 + nu0) / (3 (1 - 2 nu0));
 *   scalar:  A0 = a0 I with a0 = min over phases of the smallest diagonal entry / 2.
 * With this choice A_beta - A0 is positive definite for isotropic phases, so
 * the matrix of Eq. (13) is symmetric positive definite (Sec. 5). */
int or_default_reference(int dim, int physics, int nphase, const double *mod, double *ref) {
  if (nphase <= 0) return OR_ERR_ARG;
  if (physics == OR_ELASTIC) {
    double mumin = mod[1];
    for (int ph = 1; ph < nphase; ++ph) mumin = fmin(mumin, mod[2 * ph + 1]);
    double mu0 = 0.5 * mumin, nu0 = 0.3;
    ref[0] = 2.0 * mu0 * (1.0 + nu0) / (3.0 * (1.0 - 2.0 * nu0));
    ref[1] = mu0;
  } else {
    double amin = mod[0];
    for (int ph = 0; ph < nphase; ++ph)
      for (int i = 0; i < dim; ++i) amin = fmin(amin, mod[ph * dim * dim + i * dim + i]);
    for (int i = 0; i < dim * dim; ++i) ref[i] = 0.0;
    for (int i = 0; i < dim; ++i) ref[i * dim + i] = 0.5 * amin;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* local term, Eq. (7) and Eq. (def_ah) (one material per voxel)             */
/* ------------------------------------------------------------------------- */

/* M = (A_beta - A0)^{-1} for one voxel; *active = 0 when A_beta == A0. */
static int local_M(const or_problem *p, long vox, double *M, int *active) {
  int c = or_ncomp(p);
  double A[36], A0[36], D[36];
  if (p->frac) {
    /* Eq. (def_ah): the voxel average of (A(x) - A0)^{-1} over its two phases */
    if (p->nphase != 2 || p->scale) return OR_ERR_ARG;
    double M0[36], M1[36];
    material_matrix(p, p->ref_moduli, A0);
    for (int ph = 0; ph < 2; ++ph) {
      material_matrix(p, p->phase_moduli + (long)ph * (p->physics == OR_ELASTIC ? 2 : c * c), A);
      for (int i = 0; i < c * c; ++i) D[i] = A[i] - A0[i];
      if (mat_inverse(c, D, ph ? M1 : M0)) return OR_ERR_SINGULAR;
    }
    const double f = p->frac[vox];
    if (!(f >= 0.0 && f <= 1.0)) return OR_ERR_ARG;
    for (int i = 0; i < c * c; ++i) M[i] = f * M1[i] + (1.0 - f) * M0[i];
    *active = 1;
    return OR_OK;
  }
  int ph = p->phase[vox];
  if (ph >= p->nphase) return OR_ERR_ARG;
  material_matrix(p, p->phase_moduli + (long)ph * (p->physics == OR_ELASTIC ? 2 : c * c), A);
  material_matrix(p, p->ref_moduli, A0);
  double s = p->scale ? p->scale[vox] : 1.0;
  int nonzero = 0;
  for (int i = 0; i < c * c; ++i) {
    D[i] = s * A[i] - A0[i];
    if (D[i] != 0.0) nonzero = 1;
  }
  if (!nonzero) {
    *active = 0;
    for (int i = 0; i < c * c; ++i) M[i] = 0.0;
    return OR_OK;
  }
  *active = 1;
  if (mat_inverse(c, D, M)) return OR_ERR_SINGULAR;
  return OR_OK;
}

int or_local_operator(const or_problem *p, double *M, unsigned char *active) {
  int c = or_ncomp(p);
  long V = or_nvox(p);
  for (long v = 0; v < V; ++v) {
    int a;
    int st = local_M(p, v, M + v * c * c, &a);
    if (st) return st;
    active[v] = (unsigned char)a;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Green operators, Sec. 2.2.1 and Sec. 3.2                                   */
/* ------------------------------------------------------------------------- */

/* Gamma0(xi) for xi != 0.  Scalar: xi xi^T / (xi^T A0 xi).
 * Elastic (isotropic C0 with Lame constants lambda0, mu0), n = xi / |xi|:
 *   Gamma_ijkl = (d_ik n_j n_l + d_il n_j n_k + d_jk n_i n_l + d_jl n_i n_k) / (4 mu0)
 *                - (lambda0 + mu0) / (mu0 (lambda0 + 2 mu0)) n_i n_j n_k n_l,
 * the operator with grad^s u = -Gamma0 * tau for -div(C0 grad^s u + tau) = 0,
 * written as a Mandel matrix. */
void or_gamma0(const or_problem *p, const double xi[3], double *G) {
  int c = or_ncomp(p);
  if (p->physics == OR_ELASTIC) {
    double K0 = p->ref_moduli[0], mu0 = p->ref_moduli[1];
    double lam0 = K0 - 2.0 * mu0 / 3.0;
    double nn = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
    double n[3] = {xi[0] / nn, xi[1] / nn, xi[2] / nn};
    double b = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0));
    for (int I = 0; I < 6; ++I)
      for (int J = 0; J < 6; ++J) {
        int i = MANDEL_I[I], j = MANDEL_J[I], k = MANDEL_I[J], l = MANDEL_J[J];
        double t = ((i == k) * n[j] * n[l] + (i == l) * n[j] * n[k] + (j == k) * n[i] * n[l] +
                    (j == l) * n[i] * n[k]) /
                       (4.0 * mu0) -
                   b * n[i] * n[j] * n[k] * n[l];
        G[I * 6 + J] = mandel_w(I) * mandel_w(J) * t;
      }
  } else {
    const double *A0 = p->ref_moduli;
    double q = 0.0;
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) q += xi[i] * A0[i * c + j] * xi[j];
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) G[i * c + j] = xi[i] * xi[j] / q;
  }
}

/* Consistent discrete Green operator, Eq. (11), 2D scalar, A0 = diag(a1, a2):
 *   G_k = sum_{n in Z^2} F(2 pi (k/N + n))^2 Gamma0(k/N + n),
 *   F(2 pi (x + n))^2 = prod_i sin^2(pi x_i) / (pi (x_i + n_i))^2,  x = k / N,
 *   Gamma0(xi) = xi xi^T / (a1 xi_1^2 + a2 xi_2^2).
 * Write s_i = sin(pi x_i), y = x2 + n2, u = x1 + n1, b = sqrt(a2 / a1) |y|.  For
 * fixed n2 the sums over n1 are classical lattice sums:
 *   A(x, b) = sum_n 1 / ((x + n)^2 + b^2)       = (pi / b) sinh(2 pi b) / (cosh(2 pi b) - cos(2 pi x)),
 *   U(x, b) = sum_n (x + n) / ((x + n)^2 + b^2) = pi sin(2 pi x) / (cosh(2 pi b) - cos(2 pi x)),
 *   sum_n 1 / (x + n) = pi cot(pi x) (symmetric),  sum_n 1 / (x + n)^2 = pi^2 / s^2,
 * and partial fractions give, with T = sum_n2 s2^2 / (pi y)^2 * s1^2 / pi^2 * A(x1, b),
 *   G11 = T / a1,   G22 = (1 - T) / a2   (sum_n2 s2^2 / (pi y)^2 = 1),
 *   G12 = sum_n2 s2^2 / (pi^2 y) * s1^2 / (pi^2 a1 b^2) * (pi cot(pi x1) - U(x1, b)).
 * Once 2 pi b >= 40, A = pi / b and U = 0 to double precision, so the terms with
 * |n2| > M0 are power sums of 1 / y^3, taken from the Hurwitz zeta function
 * Z3(q) = sum_{j >= 0} (q + j)^-3 (direct sum, then the Euler-Maclaurin tail).
 * Axis frequencies (x1 = 0 or x2 = 0) keep the single n term whose weight does
 * not vanish. */
static double hurwitz3(double q) {
  double s = 0.0;
  for (int j = 0; j < 50; ++j) s += 1.0 / ((q + j) * (q + j) * (q + j));
  const double a = q + 50.0, a2 = a * a;
  /* integral, f(a)/2 and the B2, B4, B6 terms of Euler-Maclaurin for x^-3 */
  return s + 1.0 / (2.0 * a2) + 1.0 / (2.0 * a2 * a) + 1.0 / (4.0 * a2 * a2) - 1.0 / (12.0 * a2 * a2 * a2) +
         1.0 / (12.0 * a2 * a2 * a2 * a2);
}
static double lat_A(double x, double b) {
  double e = exp(-2.0 * OR_PI * b), e2 = e * e;
  return OR_PI / b * (1.0 - e2) / (1.0 + e2 - 2.0 * e * cos(2.0 * OR_PI * x));
}
static double lat_U(double x, double b) {
  double e = exp(-2.0 * OR_PI * b), e2 = e * e;
  return OR_PI * 2.0 * e * sin(2.0 * OR_PI * x) / (1.0 + e2 - 2.0 * e * cos(2.0 * OR_PI * x));
}
static void gamma_consistent_2d(double a1, double a2, const int k[3], const int n[3], double *G) {
  G[0] = G[1] = G[2] = G[3] = 0.0;
  const int k1 = k[0] % n[0], k2 = k[1] % n[1];
  if (k1 == 0 && k2 == 0) return;
  if (k2 == 0) { /* only n2 = 0 survives: xi = (x1 + n1, 0), weights summing to 1 */
    G[0] = 1.0 / a1;
    return;
  }
  if (k1 == 0) {
    G[3] = 1.0 / a2;
    return;
  }
  const double x1 = (double)k1 / n[0], x2 = (double)k2 / n[1];
  const double s1 = sin(OR_PI * x1), s2 = sin(OR_PI * x2), pi2 = OR_PI * OR_PI;
  const double r = sqrt(a2 / a1);
  const long M0 = (long)ceil(40.0 / (2.0 * OR_PI * r)) + 1;
  const double cot1 = cos(OR_PI * x1) / s1;
  ksum T, C;
  T.s = T.c = C.s = C.c = 0.0;
  for (long n2 = -M0; n2 <= M0; ++n2) {
    const double y = x2 + (double)n2, b = r * fabs(y);
    const double w2 = s2 * s2 / (pi2 * y * y);
    ksum_add(&T, w2 * s1 * s1 / pi2 * lat_A(x1, b));
    ksum_add(&C, w2 * s1 * s1 * y / (pi2 * a1 * b * b) * (OR_PI * cot1 - lat_U(x1, b)));
  }
  const double zp = hurwitz3((double)(M0 + 1) + x2), zm = hurwitz3((double)(M0 + 1) - x2);
  ksum_add(&T, s1 * s1 * s2 * s2 / (pi2 * OR_PI * r) * (zp + zm));
  ksum_add(&C, s1 * s1 * s2 * s2 * cot1 / (pi2 * OR_PI * a2) * (zp - zm));
  const double t = ksum_get(&T);
  G[0] = t / a1;
  G[3] = (1.0 - t) / a2;
  G[1] = G[2] = ksum_get(&C);
}

void or_gamma_hat(const or_problem *p, const int k[3], double *G) {
  int c = or_ncomp(p), n[3];
  grid_dims(p, n);
  int d = p->dim;
  double g[36];
  for (int i = 0; i < 2 * c * c; ++i) G[i] = 0.0;

  if (p->green == OR_TRUNCATED) {
    /* Eqs. (14)-(15): k is represented in {-M+1..M} (N = 2M) or {-M..M}
     * (N = 2M+1); Gamma0 at that representative.  k = 0 gives 0.  For even N
     * and some k_i = M, Moulinec and Suquet use A0^{-1} (Sec. 3.2.1). */
    double xi[3] = {0, 0, 0};
    int zero = 1, nyq = 0;
    for (int i = 0; i < d; ++i) {
      int ki = k[i] <= n[i] / 2 ? k[i] : k[i] - n[i];
      if (n[i] % 2 == 0 && k[i] == n[i] / 2) nyq = 1;
      xi[i] = ki;
      if (ki != 0) zero = 0;
    }
    if (zero) return;
    if (nyq) {
      double A0[36], inv[36];
      material_matrix(p, p->ref_moduli, A0);
      mat_inverse(c, A0, inv);
      for (int i = 0; i < c * c; ++i) G[2 * i] = inv[i];
      return;
    }
    or_gamma0(p, xi, g);
    for (int i = 0; i < c * c; ++i) G[2 * i] = g[i];
  } else if (p->green == OR_FILTERED) {
    /* Sec. 3.2.2: sum over n in {-1,0}^d of G(2 pi (k/N + n))^2 Gamma0(k/N + n)
     * with G(K) = prod_i cos(K_i / 4); the squared weight is cos^2(pi k_i/(2N_i))
     * for n_i = 0 and sin^2(pi k_i/(2N_i)) for n_i = -1. */
    int nterm = 1 << d;
    for (int t = 0; t < nterm; ++t) {
      double w = 1.0, xi[3] = {0, 0, 0};
      int zero = 1;
      for (int i = 0; i < d; ++i) {
        int ni = (t >> i) & 1 ? -1 : 0;
        double a = OR_PI * (double)k[i] / (2.0 * n[i]);
        double wi = ni == 0 ? cos(a) * cos(a) : sin(a) * sin(a);
        w *= wi;
        xi[i] = (double)k[i] + (double)ni * n[i];
        if (xi[i] != 0.0) zero = 0;
      }
      if (w == 0.0 || zero) continue;
      or_gamma0(p, xi, g);
      for (int i = 0; i < c * c; ++i) G[2 * i] += w * g[i];
    }
  } else if (p->green == OR_CONSISTENT) {
    double g2[4];
    gamma_consistent_2d(p->ref_moduli[0], p->ref_moduli[3], k, n, g2);
    for (int i = 0; i < 4; ++i) G[2 * i] = g2[i];
  } else {
    /* Sec. 3.2.3 (scalar problems): V_k V_k^H / (V_k^H A0 V_k) with
     * V_k,i = exp(2 i pi k_i / N_i) - 1. */
    double vr[3], vi[3];
    int zero = 1;
    for (int i = 0; i < d; ++i) {
      double a = 2.0 * OR_PI * (double)k[i] / n[i];
      vr[i] = cos(a) - 1.0;
      vi[i] = sin(a);
      if (k[i] != 0) zero = 0;
    }
    if (zero) return;
    const double *A0 = p->ref_moduli;
    double den = 0.0; /* V^H A0 V, real for symmetric A0 */
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) den += A0[i * d + j] * (vr[i] * vr[j] + vi[i] * vi[j]);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        /* V_i conj(V_j) */
        G[2 * (i * c + j)] = (vr[i] * vr[j] + vi[i] * vi[j]) / den;
        G[2 * (i * c + j) + 1] = (vi[i] * vr[j] - vr[i] * vi[j]) / den;
      }
  }
}

/* ------------------------------------------------------------------------- */
/* DFT, Sec. 3.1: hat(x)_k = sum_beta x_beta exp(-2 i pi beta.k / N)          */
/* ------------------------------------------------------------------------- */

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* exp(sign 2 i pi num / den) with the angle reduced to [0, den) first. */
static void unit_root(int sign, long num, long den, double *re, double *im) {
  long r = num % den;
  if (r < 0) r += den;
  double a = 2.0 * OR_PI * (double)r / (double)den;
  *re = cos(a);
  *im = sign * sin(a);
}

/* Iterative radix-2 FFT on a contiguous complex line (textbook: bit-reversal
 * permutation followed by log2(n) butterfly sweeps). */
static void fft_radix2(double *a, int n, int sign) {
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double tr = a[2 * i], ti = a[2 * i + 1];
      a[2 * i] = a[2 * j];
      a[2 * i + 1] = a[2 * j + 1];
      a[2 * j] = tr;
      a[2 * j + 1] = ti;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    for (int i = 0; i < n; i += len)
      for (int j = 0; j < len / 2; ++j) {
        double wr, wi;
        unit_root(sign, j, len, &wr, &wi);
        double *u = a + 2 * (i + j), *v = a + 2 * (i + j + len / 2);
        double tr = v[0] * wr - v[1] * wi, ti = v[0] * wi + v[1] * wr;
        v[0] = u[0] - tr;
        v[1] = u[1] - ti;
        u[0] += tr;
        u[1] += ti;
      }
  }
}

/* Direct 1D DFT of a contiguous complex line (any n). */
static void dft_direct(double *a, int n, int sign, double *tmp) {
  for (int k = 0; k < n; ++k) {
    ksum sr = {0, 0}, si = {0, 0};
    for (int j = 0; j < n; ++j) {
      double wr, wi;
      unit_root(sign, (long)j * k, n, &wr, &wi);
      ksum_add(&sr, a[2 * j] * wr - a[2 * j + 1] * wi);
      ksum_add(&si, a[2 * j] * wi + a[2 * j + 1] * wr);
    }
    tmp[2 * k] = ksum_get(&sr);
    tmp[2 * k + 1] = ksum_get(&si);
  }
  memcpy(a, tmp, sizeof(double) * 2 * n);
}

void or_dft(int dim, const int nin[3], int sign, double *data) {
  int n[3] = {nin[0], nin[1], dim == 3 ? nin[2] : 1};
  long stride[3] = {1, n[0], (long)n[0] * n[1]};
  for (int ax = 0; ax < 3; ++ax) {
    int len = n[ax];
    if (len == 1) continue;
    long nlines = (long)n[0] * n[1] * n[2] / len;
#pragma omp parallel
    {
      double *line = (double *)malloc(sizeof(double) * 2 * len);
      double *tmp = (double *)malloc(sizeof(double) * 2 * len);
#pragma omp for schedule(static)
      for (long l = 0; l < nlines; ++l) {
        /* base index of line l along axis ax */
        long rest = l, base = 0;
        for (int b = 0; b < 3; ++b) {
          if (b == ax) continue;
          long idx = rest % n[b];
          rest /= n[b];
          base += idx * stride[b];
        }
        for (int j = 0; j < len; ++j) {
          line[2 * j] = data[2 * (base + j * stride[ax])];
          line[2 * j + 1] = data[2 * (base + j * stride[ax]) + 1];
        }
        if (is_pow2(len)) fft_radix2(line, len, sign);
        else dft_direct(line, len, sign, tmp);
        for (int j = 0; j < len; ++j) {
          data[2 * (base + j * stride[ax])] = line[2 * j];
          data[2 * (base + j * stride[ax]) + 1] = line[2 * j + 1];
        }
      }
      free(line);
      free(tmp);
    }
  }
}

void or_dft_naive(int dim, const int nin[3], int sign, const double *in, double *out) {
  int n[3] = {nin[0], nin[1], dim == 3 ? nin[2] : 1};
  long V = (long)n[0] * n[1] * n[2];
  for (long kk = 0; kk < V; ++kk) {
    int k[3] = {(int)(kk % n[0]), (int)((kk / n[0]) % n[1]), (int)(kk / ((long)n[0] * n[1]))};
    ksum sr = {0, 0}, si = {0, 0};
    for (long bb = 0; bb < V; ++bb) {
      int b[3] = {(int)(bb % n[0]), (int)((bb / n[0]) % n[1]), (int)(bb / ((long)n[0] * n[1]))};
      /* phase = sum_i b_i k_i / n_i, reduced exactly with a common denominator */
      long den = (long)n[0] * n[1] * n[2];
      long num = ((long)b[0] * k[0] % n[0]) * (den / n[0]) + ((long)b[1] * k[1] % n[1]) * (den / n[1]) +
                 ((long)b[2] * k[2] % n[2]) * (den / n[2]);
      double wr, wi;
      unit_root(sign, num, den, &wr, &wi);
      ksum_add(&sr, in[2 * bb] * wr - in[2 * bb + 1] * wi);
      ksum_add(&si, in[2 * bb] * wi + in[2 * bb + 1] * wr);
    }
    out[2 * kk] = ksum_get(&sr);
    out[2 * kk + 1] = ksum_get(&si);
  }
}

/* ------------------------------------------------------------------------- */
/* the operator of Eq. (13)                                                  */
/* ------------------------------------------------------------------------- */

static int check_problem(const or_problem *p) {
  if (p->dim != 2 && p->dim != 3) return OR_ERR_ARG;
  if (p->physics == OR_ELASTIC && p->dim != 3) return OR_ERR_ARG;
  if (p->physics == OR_ELASTIC && p->green == OR_FINITE_DIFF) return OR_ERR_ARG;
  if (p->green == OR_CONSISTENT &&
      (p->physics != OR_SCALAR || p->dim != 2 || p->ref_moduli[1] != 0.0 || p->ref_moduli[2] != 0.0))
    return OR_ERR_ARG;
  for (int i = 0; i < p->dim; ++i)
    if (p->n[i] < 1) return OR_ERR_ARG;
  if (!p->ref_moduli || !p->phase_moduli || !p->phase || p->nphase < 1) return OR_ERR_ARG;
  double A0[36];
  material_matrix(p, p->ref_moduli, A0);
  if (!is_spd(or_ncomp(p), A0)) return OR_ERR_REFERENCE;
  return OR_OK;
}

/* Per-phase cache of M (only when there is no per-voxel scale or fraction). */
typedef struct {
  double *M;            /* nphase * c * c */
  unsigned char *act;   /* nphase */
  int ok;
} mcache;

static int mcache_init(const or_problem *p, mcache *mc) {
  int c = or_ncomp(p);
  mc->M = NULL;
  mc->act = NULL;
  mc->ok = 0;
  if (p->scale || p->frac) return OR_OK;
  mc->M = (double *)calloc((size_t)p->nphase * c * c, sizeof(double));
  mc->act = (unsigned char *)calloc((size_t)p->nphase, 1);
  if (!mc->M || !mc->act) return OR_ERR_NOMEM;
  double A[36], A0[36], D[36];
  material_matrix(p, p->ref_moduli, A0);
  for (int ph = 0; ph < p->nphase; ++ph) {
    material_matrix(p, p->phase_moduli + (long)ph * (p->physics == OR_ELASTIC ? 2 : c * c), A);
    int nonzero = 0;
    for (int i = 0; i < c * c; ++i) {
      D[i] = A[i] - A0[i];
      if (D[i] != 0.0) nonzero = 1;
    }
    mc->act[ph] = (unsigned char)nonzero;
    if (nonzero && mat_inverse(c, D, mc->M + (long)ph * c * c)) {
      /* only an error if a voxel actually uses this phase; checked lazily */
      mc->act[ph] = 2;
    }
  }
  mc->ok = 1;
  return OR_OK;
}

static void mcache_free(mcache *mc) {
  free(mc->M);
  free(mc->act);
}

static int voxel_M(const or_problem *p, const mcache *mc, long v, double *M, int *active) {
  if (mc->ok) {
    int c = or_ncomp(p), ph = p->phase[v];
    if (ph >= p->nphase) return OR_ERR_ARG;
    if (mc->act[ph] == 2) return OR_ERR_SINGULAR;
    *active = mc->act[ph];
    memcpy(M, mc->M + (long)ph * c * c, sizeof(double) * c * c);
    return OR_OK;
  }
  return local_M(p, v, M, active);
}

int or_apply(const or_problem *p, const double *x, double *y) {
  int st = check_problem(p);
  if (st) return st;
  int c = or_ncomp(p), n[3];
  grid_dims(p, n);
  long V = or_nvox(p);
  mcache mc;
  if ((st = mcache_init(p, &mc))) return st;
  unsigned char *act = (unsigned char *)malloc(V);
  double *X = (double *)malloc(sizeof(double) * 2 * c * V);
  if (!act || !X) {
    free(act);
    free(X);
    mcache_free(&mc);
    return OR_ERR_NOMEM;
  }
  /* I0 indicator */
  for (long v = 0; v < V; ++v) {
    double M[36];
    int a;
    if ((st = voxel_M(p, &mc, v, M, &a))) break;
    act[v] = (unsigned char)a;
  }
  if (st) goto done;
  /* forward DFT of each component of P x */
  for (int i = 0; i < c; ++i) {
    double *Xi = X + 2 * (long)i * V;
    for (long v = 0; v < V; ++v) {
      Xi[2 * v] = act[v] ? x[(long)i * V + v] : 0.0;
      Xi[2 * v + 1] = 0.0;
    }
    or_dft(p->dim, n, -1, Xi);
  }
  /* per-frequency product with Gamma^h_k */
#pragma omp parallel for schedule(static)
  for (long kk = 0; kk < V; ++kk) {
    int k[3] = {(int)(kk % n[0]), (int)((kk / n[0]) % n[1]), (int)(kk / ((long)n[0] * n[1]))};
    double G[72], in[12], outv[12];
    or_gamma_hat(p, k, G);
    for (int i = 0; i < c; ++i) {
      in[2 * i] = X[2 * ((long)i * V + kk)];
      in[2 * i + 1] = X[2 * ((long)i * V + kk) + 1];
    }
    for (int i = 0; i < c; ++i) {
      double sr = 0.0, si = 0.0;
      for (int j = 0; j < c; ++j) {
        double gr = G[2 * (i * c + j)], gi = G[2 * (i * c + j) + 1];
        sr += gr * in[2 * j] - gi * in[2 * j + 1];
        si += gr * in[2 * j + 1] + gi * in[2 * j];
      }
      outv[2 * i] = sr;
      outv[2 * i + 1] = si;
    }
    for (int i = 0; i < c; ++i) {
      X[2 * ((long)i * V + kk)] = outv[2 * i];
      X[2 * ((long)i * V + kk) + 1] = outv[2 * i + 1];
    }
  }
  /* inverse DFT with 1/N^d, then local term and projection on I0 */
  for (int i = 0; i < c; ++i) or_dft(p->dim, n, +1, X + 2 * (long)i * V);
  for (long v = 0; v < V; ++v) {
    if (!act[v]) {
      for (int i = 0; i < c; ++i) y[(long)i * V + v] = 0.0;
      continue;
    }
    double M[36];
    int a;
    voxel_M(p, &mc, v, M, &a);
    for (int i = 0; i < c; ++i) {
      double s = X[2 * ((long)i * V + v)] / (double)V;
      for (int j = 0; j < c; ++j) s += M[i * c + j] * x[(long)j * V + v];
      y[(long)i * V + v] = s;
    }
  }
done:
  free(act);
  free(X);
  mcache_free(&mc);
  return st;
}

/* ------------------------------------------------------------------------- */
/* solvers                                                                   */
/* ------------------------------------------------------------------------- */

/* Sign structure of M over I0: +1 all positive definite, -1 all negative
 * definite, 0 otherwise (indefinite operator, e.g. A0 between the phases). */
static int local_sign(const or_problem *p) {
  int c = or_ncomp(p);
  long V = or_nvox(p);
  int pos = 0, neg = 0, other = 0;
  double M[36], Mn[36];
  for (long v = 0; v < V; ++v) {
    int a;
    if (local_M(p, v, M, &a) || !a) continue;
    for (int i = 0; i < c * c; ++i) Mn[i] = -M[i];
    if (is_spd(c, M)) pos = 1;
    else if (is_spd(c, Mn)) neg = 1;
    else other = 1;
  }
  if (other || (pos && neg)) return 0;
  return neg ? -1 : 1;
}

static void rhs(const or_problem *p, const double *load, double *b) {
  int c = or_ncomp(p);
  long V = or_nvox(p);
  mcache mc;
  mcache_init(p, &mc);
  for (long v = 0; v < V; ++v) {
    double M[36];
    int a = 0;
    voxel_M(p, &mc, v, M, &a);
    for (int i = 0; i < c; ++i) b[(long)i * V + v] = a ? load[i] : 0.0;
  }
  mcache_free(&mc);
}

/* Conjugate gradient (Hestenes-Stiefel), x0 = 0. */
static int solve_cg(const or_problem *p, const double *b, double *x, double tol, int maxit,
                    double *info) {
  long N = or_ncomp(p) * or_nvox(p);
  double *r = (double *)malloc(sizeof(double) * N), *d = (double *)malloc(sizeof(double) * N),
         *q = (double *)malloc(sizeof(double) * N);
  if (!r || !d || !q) {
    free(r); free(d); free(q);
    return OR_ERR_NOMEM;
  }
  int st = OR_OK, it = 0;
  memset(x, 0, sizeof(double) * N);
  memcpy(r, b, sizeof(double) * N);
  memcpy(d, b, sizeof(double) * N);
  double bb = dot_comp(b, b, N), rr = bb;
  if (bb == 0.0) {
    info[0] = 0; info[1] = 0.0;
    free(r); free(d); free(q);
    return OR_OK;
  }
  st = OR_ERR_NOT_CONVERGED;
  while (it < maxit) {
    if ((st = or_apply(p, d, q))) break;
    double dq = dot_comp(d, q, N);
    if (!(fabs(dq) > 0.0) || !isfinite(dq)) { st = OR_ERR_BREAKDOWN; break; }
    double alpha = rr / dq;
    for (long i = 0; i < N; ++i) { x[i] += alpha * d[i]; r[i] -= alpha * q[i]; }
    double rrn = dot_comp(r, r, N);
    ++it;
    if (sqrt(rrn / bb) <= tol) { rr = rrn; st = OR_OK; break; }
    double beta = rrn / rr;
    rr = rrn;
    for (long i = 0; i < N; ++i) d[i] = r[i] + beta * d[i];
    st = OR_ERR_NOT_CONVERGED;
  }
  info[0] = it;
  info[1] = sqrt(rr / bb);
  free(r); free(d); free(q);
  return st;
}

/* MINRES (Paige & Saunders): Lanczos tridiagonalisation of the symmetric
 * operator, QR of the tridiagonal by Givens rotations, and the update of x
 * along the directions W = V R^{-1}.  x0 = 0; |eta| is the residual norm. */
static int solve_minres(const or_problem *p, const double *b, double *x, double tol, int maxit,
                        double *info) {
  long N = or_ncomp(p) * or_nvox(p);
  double *vprev = calloc(N, sizeof(double)), *v = malloc(sizeof(double) * N),
         *z = malloc(sizeof(double) * N), *w = calloc(N, sizeof(double)),
         *wprev = calloc(N, sizeof(double)), *wnew = malloc(sizeof(double) * N);
  if (!vprev || !v || !z || !w || !wprev || !wnew) {
    free(vprev); free(v); free(z); free(w); free(wprev); free(wnew);
    return OR_ERR_NOMEM;
  }
  memset(x, 0, sizeof(double) * N);
  double beta1 = sqrt(dot_comp(b, b, N));
  int st = OR_ERR_NOT_CONVERGED, it = 0;
  double eta = beta1;
  if (beta1 == 0.0) {
    info[0] = 0; info[1] = 0.0;
    free(vprev); free(v); free(z); free(w); free(wprev); free(wnew);
    return OR_OK;
  }
  for (long i = 0; i < N; ++i) v[i] = b[i] / beta1;
  double beta_k = 0.0; /* coupling of v_k to v_{k-1} */
  double c_km1 = 1.0, s_km1 = 0.0, c_km2 = 1.0, s_km2 = 0.0;
  while (it < maxit) {
    /* Lanczos step */
    if ((st = or_apply(p, v, z))) break;
    for (long i = 0; i < N; ++i) z[i] -= beta_k * vprev[i];
    double alpha = dot_comp(v, z, N);
    for (long i = 0; i < N; ++i) z[i] -= alpha * v[i];
    double beta_next = sqrt(dot_comp(z, z, N));
    /* previous rotations applied to the new column (beta_k, alpha, beta_next) */
    double eps = s_km2 * beta_k;
    double dbar = c_km2 * beta_k;
    double delta = c_km1 * dbar + s_km1 * alpha;
    double gbar = -s_km1 * dbar + c_km1 * alpha;
    double gamma = sqrt(gbar * gbar + beta_next * beta_next);
    if (!(gamma > 0.0)) { st = OR_ERR_BREAKDOWN; break; }
    double ck = gbar / gamma, sk = beta_next / gamma;
    /* new search direction and solution update */
    for (long i = 0; i < N; ++i) wnew[i] = (v[i] - delta * w[i] - eps * wprev[i]) / gamma;
    double tk = ck * eta;
    for (long i = 0; i < N; ++i) x[i] += tk * wnew[i];
    eta = -sk * eta;
    ++it;
    /* shift */
    double *t = wprev; wprev = w; w = wnew; wnew = t;
    c_km2 = c_km1; s_km2 = s_km1; c_km1 = ck; s_km1 = sk;
    if (fabs(eta) / beta1 <= tol) { st = OR_OK; break; }
    if (!(beta_next > 0.0)) { st = OR_OK; break; } /* invariant subspace: exact */
    for (long i = 0; i < N; ++i) { vprev[i] = v[i]; v[i] = z[i] / beta_next; }
    beta_k = beta_next;
    st = OR_ERR_NOT_CONVERGED;
  }
  info[0] = it;
  info[1] = fabs(eta) / beta1;
  free(vprev); free(v); free(z); free(w); free(wprev); free(wnew);
  return st;
}

int or_solve(const or_problem *p, const double *load, double *tau, double tol, int maxit,
             int solver, double *info) {
  int st = check_problem(p);
  if (st) return st;
  long N = or_ncomp(p) * or_nvox(p);
  double *b = (double *)malloc(sizeof(double) * N);
  if (!b) return OR_ERR_NOMEM;
  rhs(p, load, b);
  if (solver == OR_SOLVER_AUTO) solver = local_sign(p) != 0 ? OR_SOLVER_CG : OR_SOLVER_MINRES;
  if (solver == OR_SOLVER_CG) st = solve_cg(p, b, tau, tol, maxit, info);
  else st = solve_minres(p, b, tau, tol, maxit, info);
  free(b);
  return st;
}

/* ------------------------------------------------------------------------- */
/* dense route, Eq. (12)                                                     */
/* ------------------------------------------------------------------------- */

int or_dense_solve(const or_problem *p, const double *load, double *tau) {
  int st = check_problem(p);
  if (st) return st;
  int c = or_ncomp(p), n[3];
  grid_dims(p, n);
  long V = or_nvox(p);
  /* unknowns: components of tau on I0 */
  long *map = (long *)malloc(sizeof(long) * V);
  long na = 0;
  for (long v = 0; v < V; ++v) {
    double M[36];
    int a;
    if ((st = local_M(p, v, M, &a))) { free(map); return st; }
    map[v] = a ? na++ : -1;
  }
  long nu = na * c;
  if (nu > 4096) { free(map); return OR_ERR_TOO_LARGE; }
  memset(tau, 0, sizeof(double) * c * V);
  if (nu == 0) { free(map); return OR_OK; }
  /* Gamma_delta = N^{-d} sum_k Gamma^h_k exp(+2 i pi delta.k / N): direct sums */
  double *Gk = (double *)malloc(sizeof(double) * V * 2 * c * c);
  double *Gr = (double *)malloc(sizeof(double) * V * c * c);
  double *K = (double *)malloc(sizeof(double) * nu * nu);
  double *rhsv = (double *)malloc(sizeof(double) * nu);
  long *piv = (long *)malloc(sizeof(long) * nu);
  if (!Gk || !Gr || !K || !rhsv || !piv) {
    free(map); free(Gk); free(Gr); free(K); free(rhsv); free(piv);
    return OR_ERR_NOMEM;
  }
  for (long kk = 0; kk < V; ++kk) {
    int k[3] = {(int)(kk % n[0]), (int)((kk / n[0]) % n[1]), (int)(kk / ((long)n[0] * n[1]))};
    or_gamma_hat(p, k, Gk + kk * 2 * c * c);
  }
  long den = (long)n[0] * n[1] * n[2];
#pragma omp parallel for schedule(static)
  for (long dd = 0; dd < V; ++dd) {
    int dl[3] = {(int)(dd % n[0]), (int)((dd / n[0]) % n[1]), (int)(dd / ((long)n[0] * n[1]))};
    for (int e = 0; e < c * c; ++e) {
      ksum sr = {0, 0};
      for (long kk = 0; kk < V; ++kk) {
        int k[3] = {(int)(kk % n[0]), (int)((kk / n[0]) % n[1]), (int)(kk / ((long)n[0] * n[1]))};
        long num = ((long)dl[0] * k[0] % n[0]) * (den / n[0]) + ((long)dl[1] * k[1] % n[1]) * (den / n[1]) +
                   ((long)dl[2] * k[2] % n[2]) * (den / n[2]);
        double wr, wi;
        unit_root(+1, num, den, &wr, &wi);
        ksum_add(&sr, Gk[kk * 2 * c * c + 2 * e] * wr - Gk[kk * 2 * c * c + 2 * e + 1] * wi);
      }
      Gr[dd * c * c + e] = ksum_get(&sr) / (double)V;
    }
  }
  /* K_{(beta,i),(gamma,j)} = delta_{beta gamma} M_beta,ij + Gamma_{beta-gamma},ij */
  for (long bv = 0; bv < V; ++bv) {
    if (map[bv] < 0) continue;
    int b3[3] = {(int)(bv % n[0]), (int)((bv / n[0]) % n[1]), (int)(bv / ((long)n[0] * n[1]))};
    double M[36];
    int a;
    local_M(p, bv, M, &a);
    for (long gv = 0; gv < V; ++gv) {
      if (map[gv] < 0) continue;
      int g3[3] = {(int)(gv % n[0]), (int)((gv / n[0]) % n[1]), (int)(gv / ((long)n[0] * n[1]))};
      int dl[3];
      for (int i = 0; i < 3; ++i) dl[i] = ((b3[i] - g3[i]) % n[i] + n[i]) % n[i];
      long dd = dl[0] + (long)n[0] * (dl[1] + (long)n[1] * dl[2]);
      for (int i = 0; i < c; ++i)
        for (int j = 0; j < c; ++j) {
          double val = Gr[dd * c * c + i * c + j];
          if (bv == gv) val += M[i * c + j];
          K[(map[bv] * c + i) * nu + map[gv] * c + j] = val;
        }
    }
    for (int i = 0; i < c; ++i) rhsv[map[bv] * c + i] = load[i];
  }
  /* LU with partial pivoting, then forward / back substitution */
  for (long col = 0; col < nu; ++col) {
    long pr = col;
    for (long r = col + 1; r < nu; ++r)
      if (fabs(K[r * nu + col]) > fabs(K[pr * nu + col])) pr = r;
    piv[col] = pr;
    if (K[pr * nu + col] == 0.0) { st = OR_ERR_SINGULAR; break; }
    if (pr != col)
      for (long j = 0; j < nu; ++j) {
        double t = K[col * nu + j]; K[col * nu + j] = K[pr * nu + j]; K[pr * nu + j] = t;
      }
    double dgl = K[col * nu + col];
#pragma omp parallel for schedule(static)
    for (long r = col + 1; r < nu; ++r) {
      double f = K[r * nu + col] / dgl;
      K[r * nu + col] = f;
      for (long j = col + 1; j < nu; ++j) K[r * nu + j] -= f * K[col * nu + j];
    }
  }
  if (!st) {
    for (long col = 0; col < nu; ++col)
      if (piv[col] != col) { double t = rhsv[col]; rhsv[col] = rhsv[piv[col]]; rhsv[piv[col]] = t; }
    for (long r = 0; r < nu; ++r)
      for (long j = 0; j < r; ++j) rhsv[r] -= K[r * nu + j] * rhsv[j];
    for (long r = nu - 1; r >= 0; --r) {
      for (long j = r + 1; j < nu; ++j) rhsv[r] -= K[r * nu + j] * rhsv[j];
      rhsv[r] /= K[r * nu + r];
    }
    for (long v = 0; v < V; ++v)
      if (map[v] >= 0)
        for (int i = 0; i < c; ++i) tau[(long)i * V + v] = rhsv[map[v] * c + i];
  }
  free(map); free(Gk); free(Gr); free(K); free(rhsv); free(piv);
  return st;
}

/* ------------------------------------------------------------------------- */
/* effective tensor, Eq. (tau_Astar) and Theorem 13                          */
/* ------------------------------------------------------------------------- */

int or_effective(const or_problem *p, double tol, int maxit, int solver, double *Astar,
                 double *tau_all, double *info) {
  int st = check_problem(p);
  if (st) return st;
  int c = or_ncomp(p);
  long V = or_nvox(p);
  double A0[36];
  material_matrix(p, p->ref_moduli, A0);
  double *tau = (double *)malloc(sizeof(double) * c * V);
  if (!tau) return OR_ERR_NOMEM;
  for (int j = 0; j < c; ++j) {
    double load[6] = {0, 0, 0, 0, 0, 0}, inf[2] = {0, 0};
    load[j] = 1.0;
    st = or_solve(p, load, tau, tol, maxit, solver, inf);
    if (info) { info[2 * j] = inf[0]; info[2 * j + 1] = inf[1]; }
    if (st) break;
    /* A*_h e_j = A0 e_j + h^d sum_beta tau_beta  (h^d = 1/V) */
    for (int i = 0; i < c; ++i) {
      ksum s = {0, 0};
      for (long v = 0; v < V; ++v) ksum_add(&s, tau[(long)i * V + v]);
      Astar[i * c + j] = A0[i * c + j] + ksum_get(&s) / (double)V;
    }
    if (tau_all) memcpy(tau_all + (long)j * c * V, tau, sizeof(double) * c * V);
  }
  free(tau);
  return st;
}

int or_effective_variational(const or_problem *p, const double *tau_all, double *Astar) {
  int st = check_problem(p);
  if (st) return st;
  int c = or_ncomp(p);
  long V = or_nvox(p), N = c * V;
  double A0[36];
  material_matrix(p, p->ref_moduli, A0);
  double *Kt = (double *)malloc(sizeof(double) * N * c), *b = (double *)malloc(sizeof(double) * N * c);
  if (!Kt || !b) { free(Kt); free(b); return OR_ERR_NOMEM; }
  for (int j = 0; j < c; ++j) {
    double load[6] = {0, 0, 0, 0, 0, 0};
    load[j] = 1.0;
    rhs(p, load, b + (long)j * N);
    if ((st = or_apply(p, tau_all + (long)j * N, Kt + (long)j * N))) break;
  }
  if (!st)
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) {
        double v = dot_comp(b + (long)i * N, tau_all + (long)j * N, N) +
                   dot_comp(b + (long)j * N, tau_all + (long)i * N, N) -
                   dot_comp(tau_all + (long)i * N, Kt + (long)j * N, N);
        Astar[i * c + j] = A0[i * c + j] + v / (double)V;
      }
  free(Kt); free(b);
  return st;
}

int or_scale_gradient(const or_problem *p, const double *tau_all, const double *W, double *grad) {
  int st = check_problem(p);
  if (st) return st;
  if (p->frac) return OR_ERR_ARG;  /* the scale derivative needs one material per voxel */
  int c = or_ncomp(p);
  long V = or_nvox(p), N = c * V;
  for (long v = 0; v < V; ++v) {
    double M[36], A[36], eps[6][6];
    int a;
    if ((st = local_M(p, v, M, &a))) return st;
    if (!a) { grad[v] = 0.0; continue; }
    material_matrix(p, p->phase_moduli + (long)p->phase[v] * (p->physics == OR_ELASTIC ? 2 : c * c), A);
    for (int j = 0; j < c; ++j)
      for (int i = 0; i < c; ++i) {
        double s = 0.0;
        for (int l = 0; l < c; ++l) s += M[i * c + l] * tau_all[(long)j * N + (long)l * V + v];
        eps[j][i] = s;
      }
    double g = 0.0;
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) {
        if (W[i * c + j] == 0.0) continue;
        double s = 0.0;
        for (int k = 0; k < c; ++k)
          for (int l = 0; l < c; ++l) s += eps[i][k] * A[k * c + l] * eps[j][l];
        g += W[i * c + j] * s;
      }
    grad[v] = g / (double)V;
  }
  return OR_OK;
}
