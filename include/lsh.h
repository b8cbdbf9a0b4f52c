/*
 * lsh.h -- C ABI of liblsh, a GB300 (sm_103a) implementation of the
 * matrix-free Lippmann-Schwinger (LS) solver of Brisard & Legoll, "Periodic
 * homogenization using the Lippmann-Schwinger formalism" (arXiv:1411.0330).
 *
 * The library solves the Galerkin-discretised LS equation, Sec. 3, Eq. (13):
 * for every voxel beta of the set I0 where A_beta != A0,
 *
 *     (A_beta - A0)^{-1} tau_beta + DFT^{-1}[ Gamma^h_k tau^_k ]_beta = p,
 *
 * tau = 0 off I0, with the truncated (Sec. 3.2.1, Eqs. (14)-(15)) or the
 * filtered (Sec. 3.2.2) discrete Green operator Gamma^h, by conjugate
 * gradients (Sec. 5), and returns the effective tensor
 * A*_h p = A0 p + h^d sum_beta tau_beta (Eq. (tau_Astar), Theorem 13).
 *
 * Conventions shared by every entry point
 *  - Grid: dim = 2 or 3, n[i] cells along axis i, V = n0 n1 (n2) voxels.
 *    A field is component-major, [c][n2][n1][n0] with axis 0 fastest.
 *  - Components: scalar problems (conductivity) have c = dim components, one
 *    per axis.  Isotropic elasticity (dim 3) has c = 6 Mandel components
 *    (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12), so that the Euclidean dot of
 *    two 6-vectors is the double contraction of the tensors.
 *  - Memory: "device" pointers are CUDA device memory of the current device,
 *    "host" pointers are ordinary host memory.  The library never allocates
 *    device memory: everything it needs lives in the caller's workspace
 *    (see lsh_workspace_size).  Inputs given at setup are copied into that
 *    workspace, so the caller may free them afterwards.
 *  - Streams: all device work of a handle is issued on the stream given at
 *    setup.  Entry points returning host results synchronise that stream.
 *  - Errors: every entry point returns an lsh_status; none aborts, throws or
 *    traps.  A handle is not thread-safe; distinct handles are independent.
 */
#ifndef LSH_H
#define LSH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LSH_OK = 0,
  LSH_ERR_INVALID_ARG = 1,          /* null pointer, bad enum, inconsistent sizes        */
  LSH_ERR_UNSUPPORTED_SIZE = 2,     /* a grid length with a prime factor > 7, or too big */
  LSH_ERR_REFERENCE_INDEFINITE = 3, /* A0 is not symmetric positive definite            */
  LSH_ERR_SINGULAR_CONTRAST = 4,    /* A_beta - A0 is neither zero nor invertible       */
  LSH_ERR_BREAKDOWN = 5,            /* CG found (p, K p) = 0 or a non-finite scalar     */
  LSH_ERR_NOT_CONVERGED = 6,        /* tolerance not met within the iteration limits    */
  LSH_ERR_WORKSPACE = 7,            /* workspace too small or misaligned (256 B)        */
  LSH_ERR_CUDA = 8,                 /* a CUDA runtime call failed                       */
  LSH_ERR_UNSUPPORTED = 9           /* valid request this build does not implement      */
} lsh_status;

enum { LSH_SCALAR = 0, LSH_ELASTIC_ISO = 1 };
/* Discrete Green operators of Sec. 3.2: truncated (Moulinec-Suquet, with the
 * Nyquist rule), filtered, and the finite-difference one of Sec. 3.2.3
 * (scalar problems only). */
enum { LSH_GREEN_TRUNCATED = 0, LSH_GREEN_FILTERED = 1, LSH_GREEN_FD = 2 };
/* Arithmetic of the solve.  LSH_FP64: every step in double precision.
 * LSH_MIXED: FFTs, Gamma apply and CG vectors in single precision, inner
 * products and CG scalars in double, wrapped in iterative refinement whose
 * residual b - K x is computed to double-precision accuracy: in double-float
 * arithmetic (see LSH_F64_DF) where the grid allows it, else with the FP64
 * operator.  The environment variable LSH_NO_DF=1 at lsh_setup forces the
 * FP64 operator. */
enum { LSH_FP64 = 0, LSH_MIXED = 1 };
/* element type of fields passed to lsh_apply.  LSH_F64_DF: FP64 fields, the
 * operator evaluated in double-float arithmetic (pairs of FP32 values, 48
 * significant bits) on the FP32 pipes -- the arithmetic of the mixed solver's
 * refinement residual; LSH_MIXED handles on 3D grids of lengths 16..256
 * (powers of two), truncated or filtered operator, 3 or 6 components, no
 * scale or fraction field. */
enum { LSH_F64 = 0, LSH_F32 = 1, LSH_F64_DF = 2 };
/* AUTO: CG when every active phase has A_phase - A0 of one sign (K definite),
 * MINRES (Paige-Saunders, FP64) when the signs differ (K indefinite, e.g. the
 * reference k0 = (k_min + k_max)/2); CG: always CG (with a breakdown check);
 * MINRES: always MINRES (handles of at most 2^22 unknowns, or indefinite);
 * BASIC: the fixed-point scheme of Moulinec and Suquet written on the
 * polarisation, tau <- tau + (A - A0)(b - K tau) (FP64; converges when A0 lies
 * between the phases, e.g. the mean of the extreme moduli, at the rate
 * (A_max - A_min) / (A_max + A_min) for that choice); SYMMLQ: the Lanczos
 * method of Paige and Saunders for symmetric indefinite systems that the paper
 * names (Sec. 1), FP64, same buffers and limits as MINRES, stopping on the
 * residual estimate of its CG point, which it returns. */
enum { LSH_SOLVER_AUTO = 0, LSH_SOLVER_CG = 1, LSH_SOLVER_MINRES = 2, LSH_SOLVER_BASIC = 3, LSH_SOLVER_SYMMLQ = 4 };

/* Problem description (Sec. 2.2 and Sec. 3).  All pointers are read during
 * lsh_setup only. */
typedef struct lsh_problem {
  int dim;                     /* 2 or 3                                                  */
  int n[3];                    /* cells per axis; n[2] ignored (treated as 1) for dim 2   */
  int physics;                 /* LSH_SCALAR or LSH_ELASTIC_ISO (requires dim 3)          */
  int green;                   /* LSH_GREEN_TRUNCATED, _FILTERED or _FD (scalar)          */
  int precision;               /* LSH_FP64 or LSH_MIXED                                   */
  int nphase;                  /* 1..256                                                  */
  const double *phase_moduli;  /* host.  Scalar: dim*dim row-major symmetric conductivity
                                  per phase; anisotropic tensors must commute with the
                                  reference and with each other (Eq. (hyp3): one common
                                  eigenbasis), else LSH_ERR_UNSUPPORTED.  Elastic: (bulk
                                  K, shear mu) per phase.                                 */
  const double *ref_moduli;    /* host, same format as one phase: the reference medium A0
                                  (Sec. 2.2.2).  NULL selects half the softest phase:
                                  elastic mu0 = min(mu)/2, nu0 = 0.3; scalar a0 I with a0 =
                                  min diagonal entry / 2 (not allowed with `scale`).      */
  const unsigned char *phase;  /* phase id per voxel, nbatch*V bytes (microstructure-major);
                                  device or host memory                                   */
  int phase_on_host;           /* nonzero: `phase` (and `scale`) are host pointers        */
  const float *scale;          /* optional per-voxel factor s: A_beta = s_beta A_phase;
                                  nbatch*V floats, or NULL                                */
  int nbatch;                  /* microstructures sharing grid, phases and A0 (<= 1: one) */
  int max_systems;             /* systems (microstructure x load) solved simultaneously;
                                  bounds the workspace.  <= 0: nbatch * c                 */
  int scale_kind;              /* what `scale` holds: 0 a factor s of the phase moduli
                                  (A_beta = s_beta A_phase); 1 the volume fraction f of
                                  phase 1 in each voxel of a two-phase medium, whose
                                  local operator is then the voxel average of
                                  (A(x) - A0)^{-1}, Eq. (def_ah): f M_1 + (1 - f) M_0
                                  (the phase map is not used; no gradient)               */
} lsh_problem;

typedef struct lsh_solve_opts {
  double tol;        /* stop when ||b - K tau||_2 <= tol ||b||_2 (Sec. 5 uses 1e-5)    */
  int maxit;         /* iteration limit (FP64 CG iterations, or inner iterations summed) */
  int solver;        /* LSH_SOLVER_AUTO, _CG, _MINRES, _BASIC or _SYMMLQ                   */
  double inner_tol;  /* LSH_MIXED: relative residual reduction of each inner solve
                        (<= 0 selects 0.5 sqrt(tol) within [1e-6, 1e-3], relaxed on
                        later steps to half of what the least converged system of
                        the wave still needs: two refinement steps)                   */
  int max_outer;     /* LSH_MIXED: refinement steps (<= 0 selects 30)                    */
  int check_every;   /* iterations between host convergence checks (<= 0 selects 8)     */
  int warm_start;    /* lsh_solve: tau holds the initial guess on entry                  */
  int no_graphs;     /* 0: each block of check_every CG iterations is captured once in a
                        CUDA graph (per handle, wave and precision) and replayed;
                        1: the kernels are launched one by one.  Results are identical. */
} lsh_solve_opts;

typedef struct lsh_solve_info {
  int iters;      /* CG iterations (summed over inner solves for LSH_MIXED)             */
  int outer;      /* refinement steps (LSH_MIXED), 0 otherwise                           */
  int applies64;  /* applications of the double-precision operator                      */
  int status;     /* lsh_status of this solve                                            */
  double relres;  /* ||b - K tau|| / ||b|| at exit (recursive residual for FP64 CG,
                     true double-precision residual for LSH_MIXED)                      */
} lsh_solve_info;

typedef struct lsh_handle lsh_handle;

/* Choices and timings of lsh_autotune. */
typedef struct lsh_tune_report {
  int xf_variant; /* FP32 forward x pass in use: 0 shared-memory stages, 1 register FFT  */
  int x_variant;  /* FP32 inverse x pass in use: 0 shared-memory stages, 1 register FFT,
                     2 register FFT in a persistent double-buffered kernel, 3 register
                     FFT in blocks of 128 threads                                      */
  int y_variant;  /* FP32 y pass in use: 0 register FFT, 1 TMA tiles, 2 none: the x and
                     y transforms of each z plane run in one kernel (plane passes, with
                     the z pass on a ky-major spectrum; square planes of 16, 32, 48, 64,
                     96 or 128; the only FP32 passes for 48 and 96)                   */
  int z_variant;  /* FP32 z pass (with Gamma) in use: 0 register FFT; TMA tiles of
                     1: 4 columns double-buffered, 2: 8 columns, 3: 8 columns double-
                     buffered, 4: 16 columns with the FFT exchange in the tile, 5: the
                     same with two components per thread; 6 register FFT in blocks
                     of 4 columns; 7 register FFT in a persistent kernel that stages
                     the next tile's columns by asynchronous copies; 8 register FFT
                     in blocks of 16 columns; 9 the default register kernel loading
                     each frequency's Gamma coefficients when it applies them; 10
                     (plane passes only) persistent kernel on tiles of 8 columns
                     brought in and written back by TMA, double-buffered, with the
                     FFT and Gamma exchanges in the tile's buffer; 11 the same on
                     the plan N = R1 x 4 with the 4-point FFT level and Gamma in one
                     register phase (z lengths up to 128)                           */
  float xf_ms[2]; /* measured time of one launch per candidate (-1: not available)   */
  float x_ms[4];
  float y_ms[2];
  float z_ms[10];
  float xy_ms[2]; /* one CG iteration's passes summed: separate x/y passes, plane passes */
  float zp_ms[7]; /* z pass on the ky-major spectrum, variants 0, 6, 8, 9, 7, 10, 11  */
} lsh_tune_report;

/* Bytes of device workspace lsh_setup needs for this problem. */
lsh_status lsh_workspace_size(const lsh_problem *prob, size_t *bytes);

/* Validate the problem (Eq. (hyp2): A_beta - A0 zero or invertible; A0 SPD),
 * copy the microstructure into `workspace` (device, >= lsh_workspace_size
 * bytes, 256-byte aligned, caller-owned, must outlive the handle), build the
 * FFT plans, twiddles and the per-frequency Gamma^h table, and return a
 * handle.  `stream` is a cudaStream_t (NULL = legacy default stream). */
lsh_status lsh_setup(const lsh_problem *prob, void *workspace, size_t bytes, void *stream,
                     lsh_handle **out);

/* Replace the phase map (and scale field, if the problem has one) of an
 * existing handle: same grid, phases and reference medium.  Host or device
 * pointers per `on_host`.  Asynchronous for device inputs. */
lsh_status lsh_set_microstructure(lsh_handle *h, const unsigned char *phase, const float *scale,
                                  int on_host);

/* y = K x with K = P (M + Gamma) P the operator of Eq. (13) (M_beta =
 * (A_beta - A0)^{-1} of Eq. (7), P the projection on I0: values of x off I0
 * are ignored and y is zero there), for every microstructure of the batch.
 * x, y: device, nbatch*c*V elements of `dtype` (LSH_F64; LSH_F32 for
 * LSH_MIXED handles; LSH_F64_DF, FP64 fields evaluated in double-float, for
 * LSH_MIXED handles of the grids listed at LSH_F64_DF -- else
 * LSH_ERR_UNSUPPORTED), layout [nbatch][c][n2][n1][n0].  Asynchronous. */
lsh_status lsh_apply(lsh_handle *h, int dtype, const void *x, void *y);

/* Solve Eq. (13) for one macroscopic load p (host, c doubles; Mandel
 * components for elasticity) on every microstructure of the batch.  tau:
 * device, nbatch*c*V doubles, receives the polarisations (initial guesses on
 * entry when opts->warm_start).  info: host array of nbatch entries or NULL.
 * Synchronous.  Returns LSH_ERR_NOT_CONVERGED (tau holds the last iterate)
 * if the tolerance is not met. */
lsh_status lsh_solve(lsh_handle *h, const double *load, double *tau, const lsh_solve_opts *opts,
                     lsh_solve_info *info);

/* Effective tensor from c solves with the unit loads e_j (Sec. 2.1 and
 * Theorem 13), for every microstructure b of the batch:
 * Astar[(b*c + i)*c + j] = e_i . A*_h e_j (host, nbatch*c*c doubles).  All
 * nbatch*c systems run together (in waves of max_systems).  tau_all:
 * optional device buffer of nbatch*c*c*V doubles receiving the polarisations
 * [b][load j][component][voxel], NULL to skip.  infos: optional host array
 * of nbatch*c lsh_solve_info.  Synchronous. */
lsh_status lsh_effective(lsh_handle *h, const lsh_solve_opts *opts, double *Astar, double *tau_all,
                         lsh_solve_info *infos);

/* Autotuner (no counterpart in the paper): times the candidate kernels of
 * the FP32 x passes (shared-memory stages or register FFT), y pass and z
 * pass (tile shapes, register-only or TMA-staged, one or two tile buffers) on the handle's own buffers at its full system count, and
 * keeps the fastest for the following calls.  The candidates compute the same
 * operator; results change at most at the rounding level of the FP32 passes
 * (some take their sums in another order or on another FFT plan, e.g. z variant
 * 11 on N = R1 x 4).  Overwrites the handle's spectrum buffer
 * (call it between solves, not inside one).  FP64 handles: no-op.  rep may be
 * NULL.  Synchronous. */
lsh_status lsh_autotune(lsh_handle *h, lsh_tune_report *rep);

/* Select the FP32 forward x / inverse x / y / z pass variants by hand (numbering of lsh_tune_report;
 * no counterpart in the paper: for tests and measurements).  y_variant 2
 * selects the plane passes (x variants ignored; z variant 0 or 6 to 11; a handle
 * of a plane grid starts on z variant 11 where that has a plan, else 0).
 * Returns LSH_ERR_UNSUPPORTED if a variant is not available for this problem
 * (FP64 handles accept only zeros). */
lsh_status lsh_set_variants(lsh_handle *h, int xf_variant, int x_variant, int y_variant, int z_variant);

/* lsh_effective for several handles at once (microstructures of different
 * grids or phase sets; Sec. 5 computes one effective tensor per
 * microstructure).  Each handle runs on its own host thread and its own
 * stream, so the handles' kernels overlap on the device; give every handle a
 * distinct stream (handles that share one stream still give the same results,
 * one after the other).  Astar: host, the handles' nbatch*c*c blocks one after
 * the other in the order of hs; infos: optional host array of the handles'
 * nbatch*c entries in the same order.  A handle may appear once only
 * (LSH_ERR_INVALID_ARG otherwise).  Returns the first status other than
 * LSH_OK in handle order.  Synchronous. */
lsh_status lsh_effective_batch(int nh, lsh_handle *const *hs, const lsh_solve_opts *opts, double *Astar,
                               lsh_solve_info *infos);

/* Gradient of sum_ij W_ij e_i.A*_h e_j with respect to the per-voxel scale
 * s_beta (A_beta = s_beta A_phase; s = 1 without a scale field), for every
 * microstructure: g_beta = h^d sum_ij W_ij eps_i,beta . A_phase(beta)
 * eps_j,beta with eps_j = (A_beta - A0)^{-1} tau_j,beta (the derivative of
 * the symmetric system of Eq. (13)).  tau_all: device, nbatch*c*c*V doubles
 * from lsh_effective.  W: host, c*c.  grad: device, nbatch*V doubles.
 * Synchronous. */
lsh_status lsh_effective_grad(lsh_handle *h, const double *tau_all, const double *W, double *grad);

/* Allocation-free variant of lsh_apply (no counterpart in the paper; an
 * interface for callers that cannot allocate device memory where they need
 * K x: plugins inside host programs that own the device memory and offer no
 * allocator, processes whose memory is already claimed by another
 * framework's pool, or code that must not risk the device synchronisation
 * cudaMalloc / cudaFree may cause).  Computes y = K x as lsh_apply does on a
 * handle built from `prob` (one microstructure, FP64), without a handle or
 * workspace: the scratch (spectrum, Gamma^h table, FFT and phase tables) is a
 * 72 MiB array inside the library that every device loading the library
 * keeps until process exit; problems needing more return
 * LSH_ERR_UNSUPPORTED_SIZE (64^3 elasticity fits, 128^3 does not).  Narrower
 * than lsh_apply: scalar phase and reference tensors must be diagonal
 * (anisotropic commuting ones return LSH_ERR_UNSUPPORTED) and `scale` may only
 * hold a factor (scale_kind 0; volume fractions return LSH_ERR_UNSUPPORTED).
 * prob->phase (and prob->scale) must be device memory (phase_on_host = 0,
 * nbatch <= 1); x, y: device, c*V doubles.  It calls no allocator, host or
 * device.  The first call on a device looks up the array's device address
 * with cudaGetSymbolAddress and caches it (not revalidated after
 * cudaDeviceReset: do not call it again on a device that was reset).  A call
 * copies host tables and synchronises `stream` (a cudaStream_t) before
 * returning, so a stream under capture is refused (LSH_ERR_INVALID_ARG).  All
 * calls share the array: calls whose device work overlaps race on it and must
 * be serialised by the caller. */
lsh_status lsh_apply_noalloc(const lsh_problem *prob, const double *x, double *y, void *stream);

/* Diagnostics (no counterpart in the paper): kernel launches issued by the
 * handle, and, when enabled, the device time of each pass of the CG
 * iteration measured with CUDA events recorded on the handle's stream
 * between consecutive launches.  Pass kinds: 0 x-forward (with the CG
 * prologue), 1 y-forward, 2 z-forward + Gamma^h product + z-inverse,
 * 3 y-inverse, 4 x-inverse (with local term and (p, Kp)), 5 CG update. */
typedef struct lsh_profile {
  long long launches;          /* kernels launched since the last reset            */
  long long timed_iters;       /* CG iterations covered by pass_ms                 */
  double pass_ms[6];           /* summed device milliseconds per pass kind        */
  long long pass_launches[6];  /* launches that did work, per pass kind           */
  long long timed_sys_iters;   /* CG iterations of live (not yet converged) systems
                                  inside the timed iterations, summed over systems:
                                  the work pass_ms covers                          */
} lsh_profile;

/* Per-pass event timing of the CG iterations: 0 off, 1 every iteration, k > 1
 * the iterations of every k-th chunk of check_every iterations (the other
 * chunks replay graphs without event nodes, which add gaps between kernels).
 * Host memory only. */
lsh_status lsh_profile_enable(lsh_handle *h, int enable);

/* Copy the counters into `out` (host); reset them when `reset` is nonzero. */
lsh_status lsh_profile_read(lsh_handle *h, lsh_profile *out, int reset);

/* Failure-path check of the bounded device waits (no counterpart in the
 * paper).  Every wait of the library's kernels on a shared-memory barrier
 * gives up after one second, records a fault word and returns; the next
 * synchronous call reports LSH_ERR_CUDA and clears the word, and the handle
 * stays usable.  This call runs that path on purpose: one kernel on the
 * handle's stream waits `seconds` (0 < seconds <= 10) on a barrier that
 * expects two arrivals and receives one, gives up, and the call returns what
 * a real give-up returns, LSH_ERR_CUDA (LSH_OK would mean the wait was not
 * bounded).  No copy is in flight during the wait.  Synchronous. */
lsh_status lsh_check_bounded_wait(lsh_handle *h, double seconds);

/* Release the handle (host memory only; the workspace stays the caller's). */
void lsh_destroy(lsh_handle *h);

/* Static description of a status code. */
const char *lsh_status_string(lsh_status s);

#ifdef __cplusplus
}
#endif
#endif /* LSH_H */
