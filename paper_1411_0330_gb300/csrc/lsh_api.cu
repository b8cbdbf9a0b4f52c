// lsh_api.cu -- host side of the liblsh C ABI (include/lsh.h).
//
// Setup validates the problem, derives the diagonal local operator per phase,
// builds the FFT plans, twiddles and the Gamma^h table, and carves every
// device buffer out of the caller's workspace.  Solves drive the operator
// passes of kernels.cu from the host: each CG iteration is six launches that
// advance all systems of a wave (microstructure x load) together; the CG
// scalars stay on the device and the host reads the per-system states only
// every `check_every` iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <type_traits>
#include <vector>

#include "df.cuh"
#include "internal.h"
#include "lsh.h"

using namespace lsh;

namespace {

constexpr size_t kAlign = 256;
constexpr int kThreads = 256;
constexpr int kMaxSmem = 227 * 1024;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool getenv_flag(const char* name) {
  const char* e = getenv(name);
  return e && e[0] == '1';
}

// ---------------------------------------------------------------- FFT plans
bool make_plan(int n, Plan1D* p) {
  p->n = n;
  p->nst = 0;
  std::vector<int> r;
  int m = n;
  while (m % 8 == 0) { r.push_back(8); m /= 8; }
  if (m % 4 == 0) { r.push_back(4); m /= 4; }
  if (m % 2 == 0) {
    // 8 * 2 -> 4 * 4 keeps every stage at radix >= 4 where possible
    bool swapped = false;
    for (auto& v : r)
      if (v == 8) { v = 4; r.push_back(4); swapped = true; break; }
    if (!swapped) r.push_back(2);
    m /= 2;
  }
  for (int q : {3, 5, 7})
    while (m % q == 0) { r.push_back(q); m /= q; }
  if (m != 1 || (int)r.size() > LSH_MAX_STAGES) return false;
  p->nst = (int)r.size();
  for (int i = 0; i < p->nst; ++i) p->radix[i] = r[i];
  return true;
}

// position of frequency k after the DIF stages of plan p
int dif_position(const Plan1D& p, int k) {
  int pos = 0, kk = k, L = p.n;
  for (int s = 0; s < p.nst; ++s) {
    const int r = p.radix[s], m = L / r;
    pos += (kk % r) * m;
    kk /= r;
    L = m;
  }
  return pos;
}

template <typename T> void twiddles(int n, std::vector<T>& out) {
  out.resize(2 * (size_t)n);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int t = 0; t < n; ++t) {
    const long double a = 2.0L * pi * (long double)t / (long double)n;
    out[2 * t] = (T)cosl(a);
    out[2 * t + 1] = (T)(-sinl(a));
  }
}

// ---------------------------------------------------------------- derived problem data
struct Derived {
  int dim, c, nx, ny, nz, nxh, hs, ts, ncoef, physics, green, precision, nphase;
  int B;       // microstructures
  int Smax;    // systems per wave
  long long V;
  bool has_scale;
  bool frac = false;  // scale holds volume fractions of phase 1 (two phases)
  Plan1D px, py, pz;
  double ref_in[6];      // diagonal of A0 in the internal basis
  double ref_user[6];    // scalar: diagonal of A0; elastic: (K0, mu0)
  std::vector<double> mod_in;  // nphase * c diagonal of A_phase, internal basis
  std::vector<double> m_in;    // nphase * c diagonal of M (0 when inactive)
  std::vector<unsigned char> act;
  int definite;          // +1 / -1: all active phases same sign; 0: indefinite
  // scalar problems whose A0 and phase tensors are not all diagonal but commute
  // (share eigenvectors): fields are carried in the common eigenbasis,
  // u_internal = R^T u (R's columns are the eigenvectors)
  bool rotated = false;
  double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  double A0full[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  // FP32 plane passes available (kernels_plane.cu): mixed precision, 3D, square
  // planes of a plane length, z a register-FFT length
  bool plane = false;
};

// Eigenvectors of a symmetric n x n matrix (n <= 3) by cyclic Jacobi rotations:
// on return A is (numerically) diagonal and V holds the eigenvectors as columns.
void jacobi_eigen(int n, double* A, double* V) {
  for (int i = 0; i < n * n; ++i) V[i] = (i % (n + 1) == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off < 1e-300) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (apq == 0.0) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- J^T A J
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // V <- V J
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

// R^T M R for n x n matrices
void rot_sandwich(int n, const double* R, const double* M, double* out) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l) s += R[k * n + i] * M[k * n + l] * R[l * n + j];
      out[i * n + j] = s;
    }
}

lsh_status derive(const lsh_problem* pr, Derived* d) {
  if (!pr) return LSH_ERR_INVALID_ARG;
  if (pr->dim != 2 && pr->dim != 3) return LSH_ERR_INVALID_ARG;
  if (pr->physics != LSH_SCALAR && pr->physics != LSH_ELASTIC_ISO) return LSH_ERR_INVALID_ARG;
  if (pr->physics == LSH_ELASTIC_ISO && pr->dim != 3) return LSH_ERR_INVALID_ARG;
  if (pr->green != LSH_GREEN_TRUNCATED && pr->green != LSH_GREEN_FILTERED && pr->green != LSH_GREEN_FD)
    return LSH_ERR_INVALID_ARG;
  if (pr->green == LSH_GREEN_FD && pr->physics != LSH_SCALAR) return LSH_ERR_UNSUPPORTED;
  if (pr->precision != LSH_FP64 && pr->precision != LSH_MIXED) return LSH_ERR_INVALID_ARG;
  if (pr->nphase < 1 || pr->nphase > 256 || !pr->phase_moduli || !pr->phase) return LSH_ERR_INVALID_ARG;
  d->dim = pr->dim;
  d->physics = pr->physics;
  d->green = pr->green;
  d->precision = pr->precision;
  d->nphase = pr->nphase;
  d->nx = pr->n[0];
  d->ny = pr->n[1];
  d->nz = pr->dim == 3 ? pr->n[2] : 1;
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return LSH_ERR_INVALID_ARG;
  if ((long long)d->nx * d->ny * d->nz > (1LL << 31)) return LSH_ERR_UNSUPPORTED_SIZE;
  d->V = (long long)d->nx * d->ny * d->nz;
  d->nxh = d->nx / 2 + 1;
  d->hs = (d->nxh + 3) & ~3;  // 32-byte rows: z-pass column segments start on DRAM sectors
  d->ts = (d->nxh + 7) & ~7;  // the same for the FP32 Gamma table rows
  d->c = pr->physics == LSH_ELASTIC_ISO ? 6 : pr->dim;
  d->ncoef = d->c * (d->c + 1) / 2;
  d->B = pr->nbatch > 1 ? pr->nbatch : 1;
  d->Smax = d->B * d->c;
  if (pr->max_systems > 0) d->Smax = std::min(d->Smax, pr->max_systems);
  if ((long long)d->Smax * d->c * d->nz > 65535LL || (long long)d->B * d->V > (1LL << 40)) return LSH_ERR_UNSUPPORTED_SIZE;
  d->has_scale = pr->scale != nullptr;
  if (pr->scale_kind != 0 && pr->scale_kind != 1) return LSH_ERR_INVALID_ARG;
  d->frac = d->has_scale && pr->scale_kind == 1;
  if (d->frac && pr->nphase != 2) return LSH_ERR_INVALID_ARG;
  if (!make_plan(d->nx, &d->px) || !make_plan(d->ny, &d->py) || !make_plan(d->nz, &d->pz))
    return LSH_ERR_UNSUPPORTED_SIZE;
  d->plane = d->precision == LSH_MIXED && d->dim == 3 && d->nx == d->ny && plane_length(d->nx) &&
             (reg_length(d->nz) || d->nz == 48 || d->nz == 96) && !getenv_flag("LSH_NO_PLANE");
  const int c = d->c, dim = d->dim;
  // reference medium
  if (!pr->ref_moduli && d->has_scale && !d->frac) return LSH_ERR_INVALID_ARG;
  if (pr->physics == LSH_ELASTIC_ISO) {
    double K0, mu0;
    if (pr->ref_moduli) {
      K0 = pr->ref_moduli[0];
      mu0 = pr->ref_moduli[1];
    } else {
      double mumin = pr->phase_moduli[1];
      for (int ph = 1; ph < pr->nphase; ++ph) mumin = std::min(mumin, pr->phase_moduli[2 * ph + 1]);
      mu0 = 0.5 * mumin;
      const double nu0 = 0.3;
      K0 = 2.0 * mu0 * (1.0 + nu0) / (3.0 * (1.0 - 2.0 * nu0));
    }
    if (!(K0 > 0.0) || !(mu0 > 0.0)) return LSH_ERR_REFERENCE_INDEFINITE;
    d->ref_user[0] = K0;
    d->ref_user[1] = mu0;
    d->ref_in[0] = 3.0 * K0;
    for (int i = 1; i < 6; ++i) d->ref_in[i] = 2.0 * mu0;
  } else {
    // full d x d reference (given, or a0 I with a0 half the smallest diagonal entry)
    double A0[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool diag = true;
    for (int ph = 0; ph < pr->nphase; ++ph)
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) {
          const double v = pr->phase_moduli[ph * dim * dim + i * dim + j];
          if (i != j && v != 0.0) diag = false;
          if (v != pr->phase_moduli[ph * dim * dim + j * dim + i]) return LSH_ERR_INVALID_ARG;  // symmetric
        }
    if (pr->ref_moduli) {
      for (int i = 0; i < dim * dim; ++i) A0[i] = pr->ref_moduli[i];
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) {
          if (A0[i * dim + j] != A0[j * dim + i]) return LSH_ERR_INVALID_ARG;
          if (i != j && A0[i * dim + j] != 0.0) diag = false;
        }
    } else {
      double amin = pr->phase_moduli[0];
      for (int ph = 0; ph < pr->nphase; ++ph)
        for (int i = 0; i < dim; ++i) amin = std::min(amin, pr->phase_moduli[ph * dim * dim + i * dim + i]);
      for (int i = 0; i < dim; ++i) A0[i * dim + i] = 0.5 * amin;
    }
    for (int i = 0; i < 9; ++i) d->A0full[i] = i < dim * dim ? A0[i] : 0.0;
    if (diag) {
      for (int i = 0; i < dim; ++i) d->ref_in[i] = A0[i * dim + i];
    } else {
      // tensors that commute share eigenvectors: take those of a generic
      // combination, and check that every tensor is diagonal in them
      if (d->has_scale || pr->green == LSH_GREEN_FD) return LSH_ERR_UNSUPPORTED;
      double Sm[9], R[9];
      double scale = 0.0;
      for (int i = 0; i < dim * dim; ++i) {
        Sm[i] = A0[i];
        scale = std::max(scale, std::fabs(A0[i]));
      }
      for (int ph = 0; ph < pr->nphase; ++ph) {
        const double w = 1.0 / std::sqrt(2.0 + ph * 1.6180339887498949);
        for (int i = 0; i < dim * dim; ++i) {
          Sm[i] += w * pr->phase_moduli[ph * dim * dim + i];
          scale = std::max(scale, std::fabs(pr->phase_moduli[ph * dim * dim + i]));
        }
      }
      jacobi_eigen(dim, Sm, R);
      double D[9];
      rot_sandwich(dim, R, A0, D);
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j)
          if (i != j && std::fabs(D[i * dim + j]) > 1e-12 * scale) return LSH_ERR_UNSUPPORTED;
      for (int i = 0; i < dim; ++i) d->ref_in[i] = D[i * dim + i];
      for (int ph = 0; ph < pr->nphase; ++ph) {
        rot_sandwich(dim, R, pr->phase_moduli + ph * dim * dim, D);
        for (int i = 0; i < dim; ++i)
          for (int j = 0; j < dim; ++j)
            if (i != j && std::fabs(D[i * dim + j]) > 1e-12 * scale) return LSH_ERR_UNSUPPORTED;
      }
      d->rotated = true;
      for (int i = 0; i < 9; ++i) d->R[i] = i < dim * dim ? R[i] : 0.0;
    }
    for (int i = 0; i < dim; ++i) {
      if (!(d->ref_in[i] > 0.0)) return LSH_ERR_REFERENCE_INDEFINITE;
      d->ref_user[i] = d->ref_in[i];
    }
  }
  // per-phase diagonal moduli and local operator, Eq. (7) and Eq. (def_ah)
  d->mod_in.assign((size_t)pr->nphase * c, 0.0);
  d->m_in.assign((size_t)pr->nphase * c, 0.0);
  d->act.assign(256, 0);
  bool pos = false, neg = false;
  for (int ph = 0; ph < pr->nphase; ++ph) {
    double* md = &d->mod_in[(size_t)ph * c];
    if (pr->physics == LSH_ELASTIC_ISO) {
      const double K = pr->phase_moduli[2 * ph], mu = pr->phase_moduli[2 * ph + 1];
      md[0] = 3.0 * K;
      for (int i = 1; i < 6; ++i) md[i] = 2.0 * mu;
    } else if (d->rotated) {
      double D[9];
      rot_sandwich(dim, d->R, pr->phase_moduli + ph * dim * dim, D);
      for (int i = 0; i < dim; ++i) md[i] = D[i * dim + i];
    } else {
      for (int i = 0; i < dim; ++i) md[i] = pr->phase_moduli[ph * dim * dim + i * dim + i];
    }
    if (d->has_scale && !d->frac) {
      // with a scale field every voxel is in I0; the sign structure of
      // s A_phase - A0 is the caller's responsibility (A0 softer than all)
      d->act[ph] = 1;
      pos = true;
      continue;
    }
    bool any = false, allnz = true;
    for (int i = 0; i < c; ++i) {
      const double dd = md[i] - d->ref_in[i];
      if (dd != 0.0) any = true;
      else allnz = false;
    }
    if (!any) continue;  // A_phase == A0: outside I0
    if (!allnz) return LSH_ERR_SINGULAR_CONTRAST;
    d->act[ph] = 1;
    for (int i = 0; i < c; ++i) {
      const double dd = md[i] - d->ref_in[i];
      d->m_in[(size_t)ph * c + i] = 1.0 / dd;
      if (dd > 0) pos = true;
      else neg = true;
    }
  }
  d->definite = (pos && neg) ? 0 : (neg ? -1 : 1);
  if (d->frac) {
    // averaged (A - A0)^{-1} needs both phases away from A0; every voxel is in I0
    if (!d->act[0] || !d->act[1]) return LSH_ERR_SINGULAR_CONTRAST;
  }
  return LSH_OK;
}

// ---------------------------------------------------------------- launch configuration
int choose_ry(int rps, int lsx, size_t cs, int S) {
  int target = std::max(2, 2 * (int)(32768 / (lsx * cs)));
  // keep at least ~4 blocks per SM in flight for small problems
  target = std::min(target, std::max(2, (int)((long long)rps * S / 608)));
  if (target >= rps) return rps;
  int best = 1;
  for (int d = target; d >= 1; --d)
    if (rps % d == 0) {
      if (d % 2 == 0) return d;
      if (best == 1) best = d;
    }
  return best;
}

template <typename T> LaunchCfg make_cfg(const Derived& d) {
  LaunchCfg L{};
  L.threads = kThreads;
  const size_t cs = sizeof(C2<T>);
  const int lsx = d.nx | 1, lsy = d.ny | 1, lsz = d.nz | 1;
  const int rps = d.c * d.nz * d.ny;
  L.RY = choose_ry(rps, lsx, cs, d.Smax);
  L.VEC = (d.nx % (16 / (int)sizeof(T)) == 0) ? 16 / (int)sizeof(T) : 1;
  L.smem_x = d.nx * cs + (size_t)((L.RY + 1) / 2) * lsx * cs + d.nx * sizeof(int);
  L.TY = std::min(sizeof(T) == 8 ? 8 : 16, d.nxh);
  L.smem_y = d.ny * cs + (size_t)L.TY * lsy * cs;
  int TZ = std::min(8, d.nxh);
  while (TZ > 1 && (size_t)d.c * TZ * lsz * cs > 100 * 1024) TZ /= 2;
  L.TZ = TZ;
  L.smem_z = d.nz * cs + (size_t)d.c * TZ * lsz * cs;
  L.grid_x = rps / L.RY;  // per system
  L.grid_yx = (d.nxh + L.TY - 1) / L.TY;
  L.grid_yy = d.c * d.nz;  // per system
  L.grid_zx = (d.nxh + TZ - 1) / TZ;
  L.grid_zy = d.ny;
  const long long n = (long long)d.c * d.V;
  const long long want = (n + kThreads * 8 - 1) / (kThreads * 8);
  L.ew_per_sys = (int)std::max(1LL, std::min(want, std::max(1LL, 2432LL / d.Smax)));
  return L;
}

bool cfg_fits(const LaunchCfg& L) {
  return L.smem_x <= (size_t)kMaxSmem && L.smem_y <= (size_t)kMaxSmem && L.smem_z <= (size_t)kMaxSmem &&
         L.grid_zy <= 65535;
}

int rps_of(const Derived& d) { return d.c * d.nz * d.ny; }

// ---------------------------------------------------------------- workspace layout
struct Layout {
  size_t off_state, off_partials, off_phase, off_scale, off_act, off_posx, off_kofy, off_kofz, off_sums, off_W;
  size_t off_tabd, off_tabf, off_loads_d, off_loads_f, off_bb, off_flags, off_fault;
  size_t off_tw_d, off_tw_f;
  size_t off_fd[4], off_Hd, off_gd;
  size_t off_ff[4], off_Hf, off_gf;
  size_t off_wa, off_wb, off_ms;  // MINRES: two direction fields (FP64) and per-system scalars
  size_t off_gdf, off_twdf;       // double-float Gamma table and twiddles (mixed handles)
  size_t off_nq;                  // FP32 Nyquist columns of the plane passes
  size_t off_kofy32, off_kofz32;  // frequency of each y / z position in the FP32 spectrum
  bool df;                        // double-float residual passes available
  bool minres;                    // MINRES buffers present
  size_t total;
  long long nparts;
};

bool reg_len(int n) { return n == 16 || n == 32 || n == 64 || n == 128 || n == 256; }

// The mixed solver's iterative-refinement residual runs in double-float
// arithmetic (kernels_df.cu) on 3D grids whose lengths have register-FFT
// plans, for tabulated operators without finite-difference phases and phase
// maps without per-voxel scale or fraction fields (those keep the FP64 residual).
bool df_eligible(const Derived& d) {
  // powers of two; the radix-3 lengths 48 and 96 on grids with the plane passes,
  // whose FP32 spectrum order (natural along y and z) the double-float table follows
  const bool pow2 = reg_len(d.nx) && reg_len(d.ny) && reg_len(d.nz);
  return d.precision == LSH_MIXED && d.dim == 3 && (pow2 || d.plane) && d.green != LSH_GREEN_FD &&
         (d.c == 3 || d.c == 6) && !d.has_scale;
}

Layout make_layout(const Derived& d) {
  Layout l{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const int S = d.Smax;
  const long long n = (long long)d.c * d.V;  // elements per system
  const long long nf = (long long)d.nz * d.ny * d.ts;    // Gamma table frequencies (rows padded to ts)
  const long long nfh = (long long)d.nz * d.ny * d.hs;  // half spectrum per component
  LaunchCfg Ld = make_cfg<double>(d), Lf = make_cfg<float>(d);
  long long np = std::max<long long>({(long long)S * Ld.grid_x, (long long)S * Lf.grid_x, (long long)S * Ld.ew_per_sys,
                                      (long long)S * Lf.ew_per_sys, (long long)S * d.c * 152,
                                      (long long)d.B * 1216, (long long)S * (rps_of(d) / 2 + 1),
                                      (long long)S * d.c * d.nz});
  l.nparts = np;
  l.off_state = take(sizeof(SolverState) * (size_t)(3 * S + d.B));
  l.off_partials = take(sizeof(double) * (size_t)np);
  l.off_phase = take((size_t)(d.B * d.V));
  l.off_scale = take(d.has_scale ? sizeof(float) * (size_t)(d.B * d.V) : 0);
  l.off_act = take(256);
  l.off_posx = take(sizeof(int) * d.nx);
  l.off_kofy = take(sizeof(int) * d.ny);
  l.off_kofz = take(sizeof(int) * d.nz);
  l.off_kofy32 = take(sizeof(int) * d.ny);
  l.off_kofz32 = take(sizeof(int) * d.nz);
  l.off_sums = take(sizeof(double) * (size_t)S * d.c);
  l.off_W = take(sizeof(double) * 64);
  l.off_tabd = take(sizeof(double) * 2 * 256 * 6);
  l.off_tabf = take(sizeof(float) * 2 * 256 * 6);
  l.off_loads_d = take(sizeof(double) * 6 * (size_t)S);
  l.off_loads_f = take(sizeof(float) * 6 * (size_t)S);
  l.off_bb = take(sizeof(double) * (size_t)S);
  l.off_flags = take((size_t)S);
  l.off_fault = take(sizeof(int));
  l.off_tw_d = take(sizeof(double2) * (size_t)(d.nx + d.ny + d.nz));
  l.off_tw_f = take(sizeof(float2) * (size_t)(d.nx + d.ny + d.nz));
  // FP64 fields: x, r always; p, q for the FP64 CG (one system's worth of p, q
  // suffices for the Mandel rotations of lsh_apply on a mixed handle)
  const bool mixed = d.precision == LSH_MIXED;
  // MINRES (FP64) needs full-size p, q and two more fields: always for an
  // indefinite operator, otherwise only where they are small (tests, small grids)
  l.minres = d.definite == 0 || (long long)S * n <= (1ll << 22);
  for (int i = 0; i < 4; ++i) {
    const long long ns = (i < 2 || !mixed || l.minres) ? S : 1;
    l.off_fd[i] = take(sizeof(double) * (size_t)(ns * n));
  }
  l.off_wa = take(l.minres ? sizeof(double) * (size_t)(S * n) : 0);
  l.off_wb = take(l.minres ? sizeof(double) * (size_t)(S * n) : 0);
  l.off_ms = take((sizeof(MinresScalars) + sizeof(SymmlqScalars)) * (size_t)S);
  l.off_Hd = take(sizeof(double2) * (size_t)(S * d.c * nfh));
  const int ncop = (d.ncoef + 3) & ~3;  // Gamma coefficients per frequency, padded
  l.off_gd = take(sizeof(double) * (size_t)(ncop * nf));
  if (mixed) {
    for (int i = 0; i < 4; ++i) l.off_ff[i] = take(sizeof(float) * (size_t)(S * n));
    l.off_Hf = take(sizeof(float2) * (size_t)(S * d.c * nfh));
    l.off_gf = take(sizeof(float) * (size_t)(ncop * nf));
  }
  l.off_nq = take(d.plane ? sizeof(float2) * (size_t)S * d.c * d.nz * d.ny : 0);
  l.df = df_eligible(d);
  l.off_gdf = take(l.df ? sizeof(DF) * (size_t)(ncop * nf) : 0);
  l.off_twdf = take(l.df ? sizeof(DF2) * (size_t)(d.nx + d.ny + d.nz) : 0);
  l.total = o;
  return l;
}

template <typename T> struct PrecBufs {
  T *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
  C2<T>* H = nullptr;
  T* gtab = nullptr;
  C2<T>*twx = nullptr, *twy = nullptr, *twz = nullptr;
  T *mtab = nullptr, *modtab = nullptr, *loads = nullptr;
  SolverState* st = nullptr;  // Smax CG states
  LaunchCfg L{};
  OpArgs<T> a{};
  CUtensorMap tmy{};          // y-pass tensor map over H (FP32)
  CUtensorMap tmz{};          // z-pass tensor maps over H (FP32), boxes of 4 and 8 columns
  CUtensorMap tmz8{};
  CUtensorMap tmz16{};
  CUtensorMap tmzp{};         // ky-major spectrum and its Nyquist columns (plane passes)
  CUtensorMap tmzq{};
  bool ytma_ok = false, ztma_ok = false, zpipe_ok = false;
};

}  // namespace

// ---------------------------------------------------------------- the handle
struct lsh_handle {
  Derived d;
  int device = 0;
  double *wa = nullptr, *wb = nullptr;  // MINRES direction fields (null: not available)
  MinresScalars* ms = nullptr;
  SymmlqScalars* sq = nullptr;  // after the S MinresScalars
  int* fault = nullptr;  // device word set by a kernel whose bounded wait ran out
  bool no_tma = false;
  Layout lay;
  cudaStream_t stream;
  unsigned char* base;
  SolverState* st;      // [0,S) FP64 CG, [S,2S) FP32 CG, [2S,3S) residual, [3S,3S+B) setup scan
  double* partials;
  unsigned char *phase, *act, *flags;
  float* scale;
  int *posx, *kofy, *kofz;
  int *kofy32, *kofz32;  // FP32 spectrum positions (natural order with the plane passes)
  double *sums, *Wdev, *tabd, *bbdev;
  PrecBufs<double> pd;
  PrecBufs<float> pf;
  bool dfres = false;  // refinement residual in double-float (else native FP64)
  DF* gdf = nullptr;   // double-float Gamma table (the FP64 one converted)
  DF2* twdf = nullptr; // double-float twiddles, x then y then z
  std::vector<long long> n_active;  // voxels in I0 per microstructure
  // diagnostics
  long long launches = 0;
  bool prof = false;
  int prof_every = 1;           // events in every prof_every-th CG chunk
  long long prof_chunk = 0;
  bool prof_now = false;        // the chunk being enqueued records events
  std::vector<cudaEvent_t> ev;  // 7 per timed iteration
  int ev_used = 0;
  double pass_ms[6] = {0, 0, 0, 0, 0, 0};
  long long pass_n[6] = {0, 0, 0, 0, 0, 0};
  long long timed_iters = 0;
  long long timed_sys_iters = 0;  // live system-iterations inside the timed chunks
  // CUDA graphs of check_every CG iterations, one per (precision, wave, chunk,
  // profiling), captured on a private stream and replayed on `stream`
  struct Graph {
    int prec, sys0, S, sys_per_ms, chunk;
    bool prof;
    cudaGraphExec_t exec;
    long long launches;
  };
  std::vector<Graph> graphs;
  cudaStream_t cap = nullptr;
  bool capturing = false;
  void drop_graphs() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
  }
  ~lsh_handle() {
    drop_graphs();
    if (cap) cudaStreamDestroy(cap);
    for (auto e : ev) cudaEventDestroy(e);
  }
};

namespace {

#define LSH_CK(call)                              \
  do {                                            \
    if ((call) != cudaSuccess) {                  \
      cudaGetLastError();                         \
      return LSH_ERR_CUDA;                        \
    }                                             \
  } while (0)

lsh_status last_launch() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LSH_OK : LSH_ERR_CUDA;
}

template <typename T> PrecBufs<T>& bufs(lsh_handle* h);
template <> PrecBufs<double>& bufs<double>(lsh_handle* h) { return h->pd; }
template <> PrecBufs<float>& bufs<float>(lsh_handle* h) { return h->pf; }

template <typename T>
void init_prec(lsh_handle* h, PrecBufs<T>& P, const size_t* off_f, size_t off_H, size_t off_g, size_t off_tw,
               size_t off_tab, size_t off_loads, SolverState* st) {
  const Derived& d = h->d;
  unsigned char* b = h->base;
  P.x = (T*)(b + off_f[0]);
  P.r = (T*)(b + off_f[1]);
  P.p = (T*)(b + off_f[2]);
  P.q = (T*)(b + off_f[3]);
  P.H = (C2<T>*)(b + off_H);
  P.gtab = (T*)(b + off_g);
  P.twx = (C2<T>*)(b + off_tw);
  P.twy = P.twx + d.nx;
  P.twz = P.twy + d.ny;
  P.mtab = (T*)(b + off_tab);
  P.modtab = P.mtab + 256 * 6;
  P.loads = (T*)(b + off_loads);
  P.st = st;
  P.L = make_cfg<T>(d);
  OpArgs<T>& a = P.a;
  a.nx = d.nx;
  a.ny = d.ny;
  a.nz = d.nz;
  a.nxh = d.nxh;
  a.hs = d.hs;
  a.ts = d.ts;
  a.c = d.c;
  a.V = d.V;
  a.S = d.Smax;
  a.sys0 = 0;
  a.sys_per_ms = d.c;
  a.rps = d.c * d.nz * d.ny;
  a.RY = P.L.RY;
  a.bps = a.rps / a.RY;
  a.TY = P.L.TY;
  a.TZ = P.L.TZ;
  a.lsx = d.nx | 1;
  a.lsy = d.ny | 1;
  a.lsz = d.nz | 1;
  a.px = d.px;
  a.py = d.py;
  a.pz = d.pz;
  a.twx = P.twx;
  a.twy = P.twy;
  a.twz = P.twz;
  a.posx = h->posx;
  a.H = P.H;
  a.gtab = P.gtab;
  a.ncoef = d.ncoef;
  a.phase = h->phase;
  a.scale = h->scale;
  a.frac = d.frac ? 1 : 0;
  a.act = h->act;
  a.nphase = d.nphase;
  a.mtab = P.mtab;
  a.modtab = P.modtab;
  for (int i = 0; i < 6; ++i) a.ref[i] = (T)(i < d.c ? d.ref_in[i] : 0.0);
  a.loads = P.loads;
  // FP32 truncated operator: computed on the fly in the z pass (no table read)
  a.onfly = (sizeof(T) == 4 && d.green == LSH_GREEN_TRUNCATED && !d.rotated) ? 1 : 0;
  a.fdphase = d.green == LSH_GREEN_FD ? 1 : 0;
  a.physics = d.physics;
  a.kofy = h->kofy;
  a.kofz = h->kofz;
  const double invV = 1.0 / (double)d.V;
  a.invV = (T)invV;
  a.yreg = reg_length(d.ny) ? 1 : 0;
  a.zreg = (reg_length(d.nz)) ? 1 : 0;
  a.fault = h->fault;
  a.xreg = 0;  // lsh_autotune measures the register x passes against the shared-memory ones
  a.xfreg = 0;
  a.plane = 0;
  a.tlay = 0;
  a.nq = nullptr;
  // measured on the batched workload: the inverse pass gains (0.61 -> 0.66 of the
  // copy bandwidth), the forward pass loses (0.81 -> 0.70); LSH_L2PF overrides
  a.l2pf = 2;
  if (const char* e = getenv("LSH_L2PF")) a.l2pf = atoi(e) & 3;
  if (sizeof(T) == 4 && d.plane) {
    // natural frequency order along y and z in every FP32 pass; the plane
    // passes (ky-major spectrum) are the default
    a.nq = (C2<T>*)(h->base + h->lay.off_nq);
    a.kofy = h->kofy32;
    a.kofz = h->kofz32;
    a.zreg = 1;
    a.plane = 1;
    a.tlay = 1;
  }
  a.ytma = 0;
  a.tmy = &P.tmy;
  if (sizeof(T) == 4 && a.yreg && d.nz > 1 && !h->no_tma)
    P.ytma_ok = encode_y_map(&P.tmy, P.H, d.hs, d.ny, (long long)d.Smax * d.c * d.nz);
  a.ytma = P.ytma_ok ? 1 : 0;
  // the z pass keeps the register kernel unless lsh_autotune measures a TMA variant faster
  a.ztma = 0;
  a.tmz = &P.tmz;
  a.tmz8 = &P.tmz8;
  a.tmz16 = &P.tmz16;
  if (sizeof(T) == 4 && a.zreg && !h->no_tma)
    P.ztma_ok = encode_z_map(&P.tmz, P.H, d.hs, d.ny, d.nz, d.c, d.Smax, 4) &&
                encode_z_map(&P.tmz8, P.H, d.hs, d.ny, d.nz, d.c, d.Smax, 8) &&
                encode_z_map(&P.tmz16, P.H, d.hs, d.ny, d.nz, d.c, d.Smax, 16);
  a.tmzp = nullptr;
  a.tmzq = nullptr;
  if (sizeof(T) == 4 && d.plane && !h->no_tma &&
      (P.zpipe_ok = encode_zpipe_maps(&P.tmzp, &P.tmzq, P.H, a.nq, d.hs, d.ny, d.nz, d.c, d.Smax))) {
    a.tmzp = &P.tmzp;
    a.tmzq = &P.tmzq;
  }
  for (int i = 0; i < 6; ++i) a.g0[i] = (T)0;
  if (d.physics == LSH_ELASTIC_ISO) {
    const double K0 = d.ref_user[0], mu0 = d.ref_user[1], lam0 = K0 - 2.0 * mu0 / 3.0;
    a.g0[0] = (T)(invV / (2.0 * mu0));
    a.g0[1] = (T)(invV * (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0)));
    a.g0[2] = (T)(invV / (3.0 * K0));
    a.g0[3] = (T)(invV / (2.0 * mu0));
  } else {
    for (int i = 0; i < d.c; ++i) a.g0[i] = (T)d.ref_user[i];
  }
}

// internal basis <-> Mandel for elasticity (see k_rotate)
void to_internal(const Derived& d, const double* m, double* out) {
  for (int i = 0; i < d.c; ++i) out[i] = m[i];
  if (d.rotated) {
    for (int k = 0; k < d.c; ++k) {
      double s = 0.0;
      for (int i = 0; i < d.c; ++i) s += d.R[i * d.c + k] * m[i];
      out[k] = s;
    }
  }
  if (d.physics == LSH_ELASTIC_ISO) {
    const double s3 = 1.0 / std::sqrt(3.0), s2 = 1.0 / std::sqrt(2.0), s6 = 1.0 / std::sqrt(6.0);
    out[0] = (m[0] + m[1] + m[2]) * s3;
    out[1] = (m[0] - m[1]) * s2;
    out[2] = (m[0] + m[1] - 2.0 * m[2]) * s6;
  }
}
void to_mandel(const Derived& d, const double* v, double* out) {
  for (int i = 0; i < d.c; ++i) out[i] = v[i];
  if (d.rotated) {
    for (int i = 0; i < d.c; ++i) {
      double s = 0.0;
      for (int k = 0; k < d.c; ++k) s += d.R[i * d.c + k] * v[k];
      out[i] = s;
    }
  }
  if (d.physics == LSH_ELASTIC_ISO) {
    const double s3 = 1.0 / std::sqrt(3.0), s2 = 1.0 / std::sqrt(2.0), s6 = 1.0 / std::sqrt(6.0);
    out[0] = v[0] * s3 + v[1] * s2 + v[2] * s6;
    out[1] = v[0] * s3 - v[1] * s2 + v[2] * s6;
    out[2] = v[0] * s3 - 2.0 * v[2] * s6;
  }
}

// reference stiffness / conductivity in the component basis of the ABI
void ref_matrix(const Derived& d, double* A0) {
  const int c = d.c;
  for (int i = 0; i < c * c; ++i) A0[i] = 0.0;
  if (d.physics == LSH_ELASTIC_ISO) {
    const double K0 = d.ref_user[0], mu0 = d.ref_user[1], lam0 = K0 - 2.0 * mu0 / 3.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A0[i * 6 + j] = lam0 + (i == j ? 2.0 * mu0 : 0.0);
    for (int i = 3; i < 6; ++i) A0[i * 6 + i] = 2.0 * mu0;
  } else {
    for (int i = 0; i < c * c; ++i) A0[i] = d.A0full[i];
  }
}

lsh_status read_states(lsh_handle* h, const SolverState* dev, int n, SolverState* out) {
  LSH_CK(cudaMemcpyAsync(out, dev, sizeof(SolverState) * n, cudaMemcpyDeviceToHost, h->stream));
  LSH_CK(cudaStreamSynchronize(h->stream));
  return LSH_OK;
}

// A wave: S systems starting at global system sys0, sys_per_ms systems per
// microstructure; loads (internal basis) per system.
struct Wave {
  int S, sys0, sys_per_ms;
  const double* loads;  // host [S][6]
};

template <typename T> OpArgs<T> wave_args(lsh_handle* h, const Wave& w) {
  OpArgs<T> a = bufs<T>(h).a;
  a.S = w.S;
  a.sys0 = w.sys0;
  a.sys_per_ms = w.sys_per_ms;
  return a;
}

lsh_status upload_loads(lsh_handle* h, const Wave& w) {
  std::vector<double> ld(6 * (size_t)w.S);
  std::vector<float> lf(6 * (size_t)w.S);
  for (size_t i = 0; i < ld.size(); ++i) {
    ld[i] = w.loads[i];
    lf[i] = (float)w.loads[i];
  }
  LSH_CK(cudaMemcpyAsync(h->pd.loads, ld.data(), sizeof(double) * ld.size(), cudaMemcpyHostToDevice, h->stream));
  if (h->d.precision == LSH_MIXED)
    LSH_CK(cudaMemcpyAsync(h->pf.loads, lf.data(), sizeof(float) * lf.size(), cudaMemcpyHostToDevice, h->stream));
  return LSH_OK;
}

// ---------------------------------------------------------------- operator sequences
// out = K in (internal basis), precision T, for the systems of `a`.
template <typename T> lsh_status apply_internal(lsh_handle* h, const OpArgs<T>& a, const T* in, T* out) {
  PrecBufs<T>& P = bufs<T>(h);
  cudaStream_t s = h->stream;
  launch_xfwd<T>(a, P.L, 0, in, nullptr, nullptr, nullptr, nullptr, s);
  launch_yfft<T>(a, P.L, false, nullptr, s);
  launch_zgamma<T>(a, P.L, nullptr, s);
  launch_yfft<T>(a, P.L, true, nullptr, s);
  launch_xinv<T>(a, P.L, 0, in, out, nullptr, nullptr, s);
  h->launches += a.plane ? 3 : 5;
  return last_launch();
}

// The arguments of the double-float y and z passes: those of the FP64 wave
// with the spectrum read as double-float pairs and the double-float tables.
OpArgs<DF> df_args(lsh_handle* h, const OpArgs<double>& a) {
  static_assert(sizeof(OpArgs<DF>) == sizeof(OpArgs<double>) && alignof(OpArgs<DF>) == alignof(OpArgs<double>),
                "same layout");
  static_assert(offsetof(OpArgs<DF>, invV) == offsetof(OpArgs<double>, invV) &&
                    offsetof(OpArgs<DF>, xfreg) == offsetof(OpArgs<double>, xfreg),
                "same layout");
  OpArgs<DF> b;
  std::memcpy(static_cast<void*>(&b), &a, sizeof(b));  // every member but the typed ones below
  const Derived& d = h->d;
  b.twx = h->twdf;
  b.twy = h->twdf + d.nx;
  b.twz = h->twdf + d.nx + d.ny;
  b.H = reinterpret_cast<DF2*>(a.H);
  b.gtab = h->gdf;
  b.mtab = b.modtab = b.loads = nullptr;
  for (int i = 0; i < 6; ++i) {
    b.ref[i] = DF(a.ref[i]);
    b.g0[i] = DF(a.g0[i]);
  }
  b.invV = DF(a.invV);
  b.onfly = 0;
  b.fdphase = 0;
  return b;
}

// y = K x in double-float arithmetic (FP64 in and out)
lsh_status apply_df(lsh_handle* h, const OpArgs<double>& a, const double* in, double* out) {
  cudaStream_t s = h->stream;
  const OpArgs<DF> b = df_args(h, a);
  launch_df_x(a, b.twx, -1, in, nullptr, nullptr, nullptr, s);
  launch_yfft_reg<DF>(b, false, nullptr, s);
  launch_df_z(b, s);
  launch_yfft_reg<DF>(b, true, nullptr, s);
  launch_df_x(a, b.twx, 0, in, out, nullptr, nullptr, s);
  h->launches += 7;
  return last_launch();
}

// r = b - K x for the wave, (r, r) -> residual states' aux[0].  df (handles
// with the double-float passes): computed in double-float arithmetic and
// stored as (h, l) FP32 pairs in r's 8-byte elements; otherwise native FP64.
lsh_status residual64(lsh_handle* h, const OpArgs<double>& a, const double* x, double* r, bool df = false) {
  PrecBufs<double>& P = h->pd;
  cudaStream_t s = h->stream;
  SolverState* sres = h->st + 2 * h->d.Smax;
  if (df) {
    const OpArgs<DF> b = df_args(h, a);
    launch_df_x(a, b.twx, -1, x, nullptr, nullptr, nullptr, s);
    launch_yfft_reg<DF>(b, false, nullptr, s);
    launch_df_z(b, s);
    launch_yfft_reg<DF>(b, true, nullptr, s);
    launch_df_x(a, b.twx, 2, x, r, sres, h->partials, s);
    h->launches += 7;
    return last_launch();
  }
  launch_xfwd<double>(a, P.L, 0, x, nullptr, nullptr, nullptr, nullptr, s);
  launch_yfft<double>(a, P.L, false, nullptr, s);
  launch_zgamma<double>(a, P.L, nullptr, s);
  launch_yfft<double>(a, P.L, true, nullptr, s);
  launch_xinv<double>(a, P.L, 2, x, r, sres, h->partials, s);
  h->launches += 5;
  return last_launch();
}

template <typename T> void enqueue_cg_iteration(lsh_handle* h, PrecBufs<T>& P, const OpArgs<T>& a) {
  cudaStream_t s = h->stream;
  const bool timed = h->prof_now && h->ev_used + 7 <= (int)h->ev.size();
  cudaEvent_t* e = timed ? &h->ev[h->ev_used] : nullptr;
  // inside a capture the records become graph nodes that record at replay
  const unsigned rf = h->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (timed) cudaEventRecordWithFlags(e[0], s, rf);
  launch_xfwd<T>(a, P.L, 1, nullptr, P.x, P.r, P.p, P.st, s);
  if (timed) cudaEventRecordWithFlags(e[1], s, rf);
  launch_yfft<T>(a, P.L, false, P.st, s);
  if (timed) cudaEventRecordWithFlags(e[2], s, rf);
  launch_zgamma<T>(a, P.L, P.st, s);
  if (timed) cudaEventRecordWithFlags(e[3], s, rf);
  launch_yfft<T>(a, P.L, true, P.st, s);
  if (timed) cudaEventRecordWithFlags(e[4], s, rf);
  launch_xinv<T>(a, P.L, 1, P.p, P.q, P.st, h->partials, s);
  if (timed) cudaEventRecordWithFlags(e[5], s, rf);
  launch_cg_update<T>(P.r, P.q, (long long)a.c * a.V, a.S, P.st, h->partials, P.L.ew_per_sys, s);
  if (timed) {
    cudaEventRecordWithFlags(e[6], s, rf);
    h->ev_used += 7;
  }
  // the FP32 register inverse x pass adds one small reduction kernel; the plane
  // passes replace the x and y passes (xy forward, z, xy inverse, reduction, update)
  if (a.plane) {
    h->launches += 5;
  } else {
    h->launches += 6 + ((sizeof(T) == 4 && (a.xreg == 1 || a.xreg == 3)) ? 1 : 0);
  }
}

// The graph replaying `chunk` CG iterations of this wave, captured on first use.
// Everything the kernels read is fixed per handle and wave (device pointers,
// OpArgs); the CG scalars and the done flags stay on the device.
template <typename T>
lsh_status chunk_graph(lsh_handle* h, PrecBufs<T>& P, const OpArgs<T>& a, int chunk, lsh_handle::Graph** out) {
  const int prec = (int)sizeof(T);
  for (auto& g : h->graphs)
    if (g.prec == prec && g.sys0 == a.sys0 && g.S == a.S && g.sys_per_ms == a.sys_per_ms && g.chunk == chunk &&
        g.prof == h->prof_now) {
      *out = &g;
      return LSH_OK;
    }
  if (!h->cap) LSH_CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  cudaStream_t user = h->stream;
  const long long l0 = h->launches;
  const int ev0 = h->ev_used;
  h->ev_used = 0;
  h->stream = h->cap;
  h->capturing = true;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int j = 0; j < chunk; ++j) enqueue_cg_iteration<T>(h, P, a);
    e = cudaStreamEndCapture(h->cap, &graph);
  }
  h->capturing = false;
  h->stream = user;
  lsh_handle::Graph g{prec, a.sys0, a.S, a.sys_per_ms, chunk, h->prof_now, nullptr, h->launches - l0};
  h->launches = l0;
  h->ev_used = ev0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LSH_ERR_CUDA;
  }
  h->graphs.push_back(g);
  *out = &h->graphs.back();
  return LSH_OK;
}

// After a host synchronisation: add the pass times of the first `real`
// recorded iterations (later ones returned at once because every system of
// the wave was done).
void harvest_profile(lsh_handle* h, int real, bool plane) {
  const int groups = h->ev_used / 7;
  for (int g = 0; g < groups && g < real; ++g) {
    for (int k = 0; k < 6; ++k) {
      if (plane && (k == 1 || k == 3)) continue;  // no separate y passes
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->ev[7 * g + k], h->ev[7 * g + k + 1]) == cudaSuccess) {
        h->pass_ms[k] += ms;
        h->pass_n[k] += 1;
      }
    }
    h->timed_iters += 1;
  }
  cudaGetLastError();
  h->ev_used = 0;
}

// CG on the states already begun for the wave; finalises x.  `out` receives
// the S states.
template <typename T>
lsh_status cg_run(lsh_handle* h, PrecBufs<T>& P, const OpArgs<T>& a, int maxit, int check_every, bool graphs,
                  std::vector<SolverState>& out) {
  const int S = a.S;
  out.resize(S);
  lsh_status stt = read_states(h, P.st, S, out.data());
  if (stt) return stt;
  auto all_done = [&]() {
    for (int s = 0; s < S; ++s)
      if (!out[s].done) return false;
    return true;
  };
  auto max_iter = [&]() {
    int m = 0;
    for (int s = 0; s < S; ++s) m = std::max(m, out[s].iter);
    return m;
  };
  int it = 0;
  while (!all_done() && it < maxit) {
    const int chunk = std::min(check_every, maxit - it);
    const int before = max_iter();
    h->prof_now = h->prof && (h->prof_chunk++ % h->prof_every) == 0;
    if (graphs && chunk == check_every) {
      lsh_handle::Graph* g = nullptr;
      if ((stt = chunk_graph<T>(h, P, a, chunk, &g))) return stt;
      if (h->prof_now) h->ev_used = 0;
      LSH_CK(cudaGraphLaunch(g->exec, h->stream));
      h->launches += g->launches;
      if (h->prof_now) h->ev_used = (int)std::min<size_t>(7 * (size_t)chunk, h->ev.size() / 7 * 7);
    } else {
      for (int j = 0; j < chunk; ++j) enqueue_cg_iteration<T>(h, P, a);
    }
    if ((stt = last_launch())) return stt;
    it += chunk;
    long long live0 = 0;
    for (int k = 0; k < S; ++k) live0 += out[k].iter;
    if ((stt = read_states(h, P.st, S, out.data()))) return stt;
    if (h->prof_now) {
      for (int k = 0; k < S; ++k) h->timed_sys_iters += out[k].iter;
      h->timed_sys_iters -= live0;
      harvest_profile(h, max_iter() - before, a.plane != 0);
    }
    h->prof_now = false;
  }
  launch_cg_finalize<T>(P.x, P.p, (long long)a.c * a.V, S, P.st, P.L.ew_per_sys, h->stream);
  h->launches += 1;
  if ((stt = last_launch())) return stt;
  return read_states(h, P.st, S, out.data());
}

// MINRES on the FP64 operator for the systems of a wave, whose right-hand
// sides are in pd.r and initial guesses in pd.x (x0 + the MINRES updates);
// rhs2: device (r0, r0) per system, bb: device (b, b) per system (tolerance
// base).  Eight launches per iteration: the five operator passes on r2 and the
// three recurrence kernels.
lsh_status minres_run(lsh_handle* h, const OpArgs<double>& a, int maxit, int check_every, const double* rhs2,
                      double tol, std::vector<SolverState>& out, bool symmlq = false) {
  PrecBufs<double>& P = h->pd;
  cudaStream_t s = h->stream;
  const int S = a.S;
  const long long n = (long long)a.c * a.V;
  const int G = P.L.ew_per_sys;
  LSH_CK(cudaMemcpyAsync(P.p, P.r, sizeof(double) * (size_t)(S * n), cudaMemcpyDeviceToDevice, s));
  LSH_CK(cudaMemsetAsync(h->wa, 0, sizeof(double) * (size_t)(S * n), s));
  if (symmlq)  // SYMMLQ: one direction field (wa) and the right-hand side of this run (wb)
    LSH_CK(cudaMemcpyAsync(h->wb, P.r, sizeof(double) * (size_t)(S * n), cudaMemcpyDeviceToDevice, s));
  else
    LSH_CK(cudaMemsetAsync(h->wb, 0, sizeof(double) * (size_t)(S * n), s));
  launch_minres_begin(P.st, h->ms, rhs2, h->bbdev, tol, S, s);
  h->launches += 1;
  if (symmlq) {
    launch_symmlq_begin(h->sq, S, s);
    h->launches += 1;
  }
  lsh_status stt;
  out.resize(S);
  if ((stt = read_states(h, P.st, S, out.data()))) return stt;
  auto all_done = [&]() {
    for (int k = 0; k < S; ++k)
      if (!out[k].done) return false;
    return true;
  };
  int it = 0;
  while (!all_done() && it < maxit) {
    const int chunk = std::min(check_every, maxit - it);
    for (int j = 0; j < chunk; ++j) {
      launch_xfwd<double>(a, P.L, 0, P.p, nullptr, nullptr, nullptr, nullptr, s);
      launch_yfft<double>(a, P.L, false, P.st, s);
      launch_zgamma<double>(a, P.L, P.st, s);
      launch_yfft<double>(a, P.L, true, P.st, s);
      launch_xinv<double>(a, P.L, 3, P.p, P.q, P.st, h->partials, s);
      if (symmlq)
        launch_symmlq_step(P.x, P.r, P.p, P.q, h->wa, h->wb, n, S, P.st, h->ms, h->sq, h->partials, G, s);
      else
        launch_minres_step(P.x, P.r, P.p, P.q, h->wa, h->wb, n, S, P.st, h->ms, h->partials, G, s);
      h->launches += 8;
    }
    if ((stt = last_launch())) return stt;
    it += chunk;
    if ((stt = read_states(h, P.st, S, out.data()))) return stt;
  }
  return LSH_OK;
}

// The basic scheme on the FP64 operator for the systems of a wave (x holds the
// initial guesses): per iteration one residual r = b - K x (five passes) and
// the update x += (A - A0) r; residual norms read every check_every iterations.
lsh_status basic_run(lsh_handle* h, const OpArgs<double>& a, int maxit, int check_every, double tol,
                     const std::vector<double>& bb, std::vector<int>& iters, std::vector<double>& relres,
                     std::vector<int>& done) {
  PrecBufs<double>& P = h->pd;
  cudaStream_t s = h->stream;
  const int S = a.S;
  SolverState* sres = h->st + 2 * h->d.Smax;
  std::vector<unsigned char> flags(S, 0);
  iters.assign(S, 0);
  relres.assign(S, 0.0);
  done.assign(S, 0);
  for (int k = 0; k < S; ++k)
    if (!(bb[k] > 0.0)) {
      flags[k] = 1;
      done[k] = 1;
    }
  LSH_CK(cudaMemcpyAsync(h->flags, flags.data(), S, cudaMemcpyHostToDevice, s));
  lsh_status stt;
  std::vector<SolverState> rs(S);
  int it = 0;
  while (it < maxit) {
    bool all = true;
    for (int k = 0; k < S; ++k) all = all && done[k];
    if (all) break;
    const int chunk = std::min(check_every, maxit - it);
    for (int j = 0; j < chunk; ++j) {
      if ((stt = residual64(h, a, P.x, P.r))) return stt;
      launch_basic_update(a, P.x, P.r, h->flags, P.L.ew_per_sys, s);
      h->launches += 1;
    }
    it += chunk;
    // the residual of the last update (one more application, not counted as an iteration)
    if ((stt = residual64(h, a, P.x, P.r))) return stt;
    if ((stt = read_states(h, sres, S, rs.data()))) return stt;
    for (int k = 0; k < S; ++k) {
      if (done[k]) continue;
      iters[k] = it;
      relres[k] = bb[k] > 0 ? std::sqrt(std::max(rs[k].aux[0], 0.0) / bb[k]) : 0.0;
      if (!std::isfinite(relres[k])) return LSH_ERR_BREAKDOWN;
      if (relres[k] <= tol) {
        done[k] = 1;
        flags[k] = 1;
      }
    }
    LSH_CK(cudaMemcpyAsync(h->flags, flags.data(), S, cudaMemcpyHostToDevice, s));
  }
  return LSH_OK;
}

// A kernel that gave up a bounded wait (TMA copies) set the fault word.
lsh_status check_fault(lsh_handle* h) {
  int f = 0;
  LSH_CK(cudaMemcpyAsync(&f, h->fault, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LSH_CK(cudaStreamSynchronize(h->stream));
  if (f) {
    LSH_CK(cudaMemsetAsync(h->fault, 0, sizeof(int), h->stream));
    return LSH_ERR_CUDA;
  }
  return LSH_OK;
}

// Solve the systems of a wave; the solutions end in pd.x (internal basis).
// warm: pd.x holds initial guesses.  infos: S entries.
lsh_status solve_wave(lsh_handle* h, const Wave& w, bool warm, const lsh_solve_opts* o, lsh_solve_info* infos) {
  const Derived& d = h->d;
  const int S = w.S;
  const long long n = (long long)d.c * d.V;
  const double tol = o && o->tol > 0 ? o->tol : 1e-10;
  const int maxit = o && o->maxit > 0 ? o->maxit : 10000;
  const int check = o && o->check_every > 0 ? o->check_every : 8;
  const bool graphs = !(o && o->no_graphs);
  lsh_status stt;
  if ((stt = upload_loads(h, w))) return stt;
  // (b, b) per system = |load|^2 x (voxels in I0 of its microstructure)
  std::vector<double> bb(S);
  for (int s = 0; s < S; ++s) {
    double lb = 0.0;
    for (int i = 0; i < d.c; ++i) lb += w.loads[6 * s + i] * w.loads[6 * s + i];
    bb[s] = lb * (double)h->n_active[(w.sys0 + s) / w.sys_per_ms];
  }
  LSH_CK(cudaMemcpyAsync(h->bbdev, bb.data(), sizeof(double) * S, cudaMemcpyHostToDevice, h->stream));
  for (int s = 0; s < S; ++s) infos[s] = lsh_solve_info{};
  PrecBufs<double>& Pd = h->pd;
  const OpArgs<double> ad = wave_args<double>(h, w);
  const int G = Pd.L.ew_per_sys;
  std::vector<SolverState> st;
  const int solver = o ? o->solver : LSH_SOLVER_AUTO;
  if (solver < LSH_SOLVER_AUTO || solver > LSH_SOLVER_SYMMLQ) return LSH_ERR_INVALID_ARG;
  const bool use_symmlq = solver == LSH_SOLVER_SYMMLQ;
  const bool use_minres = use_symmlq || solver == LSH_SOLVER_MINRES || (solver == LSH_SOLVER_AUTO && d.definite == 0);
  if (solver == LSH_SOLVER_BASIC) {
    // Moulinec-Suquet fixed point, FP64 whatever the precision
    if (!warm) {
      launch_fill_rhs<double>(ad, Pd.r, Pd.x, G, h->stream);
      h->launches += 1;
    }
    if ((stt = last_launch())) return stt;
    std::vector<int> its, dn;
    std::vector<double> rel;
    if ((stt = basic_run(h, ad, maxit, check, tol, bb, its, rel, dn))) return stt;
    for (int s = 0; s < S; ++s) {
      infos[s].iters = its[s];
      infos[s].applies64 += its[s];
      infos[s].relres = rel[s];
      infos[s].status = dn[s] ? LSH_OK : LSH_ERR_NOT_CONVERGED;
    }
  } else if (use_minres) {
    // indefinite operator (or asked for): MINRES in FP64 whatever the precision
    if (!h->wa) return LSH_ERR_UNSUPPORTED;
    const double* rhs2 = h->bbdev;
    if (!warm) {
      launch_fill_rhs<double>(ad, Pd.r, Pd.x, G, h->stream);
      h->launches += 1;
    } else {
      if ((stt = residual64(h, ad, Pd.x, Pd.r))) return stt;
      std::vector<SolverState> s2(S);
      if ((stt = read_states(h, h->st + 2 * d.Smax, S, s2.data()))) return stt;
      std::vector<double> r2(S);
      for (int s = 0; s < S; ++s) {
        r2[s] = s2[s].aux[0];
        infos[s].applies64 += 1;
      }
      LSH_CK(cudaMemcpyAsync(h->sums, r2.data(), sizeof(double) * S, cudaMemcpyHostToDevice, h->stream));
      rhs2 = h->sums;
    }
    if ((stt = last_launch())) return stt;
    if ((stt = minres_run(h, ad, maxit, check, rhs2, tol, st, use_symmlq))) return stt;
    for (int s = 0; s < S; ++s) {
      infos[s].iters = st[s].iter;
      infos[s].applies64 += st[s].iter;
      infos[s].relres = st[s].bb > 0 ? std::sqrt(std::max(st[s].rr, 0.0) / st[s].bb) : 0.0;
      infos[s].status = st[s].status ? st[s].status : (st[s].done ? LSH_OK : LSH_ERR_NOT_CONVERGED);
    }
  } else if (d.precision == LSH_FP64) {
    if (!warm) {
      launch_fill_rhs<double>(ad, Pd.r, Pd.x, G, h->stream);
      launch_cg_begin<double>(Pd.r, n, S, Pd.st, h->partials, tol, h->bbdev, G, h->stream);
      h->launches += 2;
    } else {
      if ((stt = residual64(h, ad, Pd.x, Pd.r))) return stt;
      for (int s = 0; s < S; ++s) infos[s].applies64 += 1;
      launch_cg_begin<double>(Pd.r, n, S, Pd.st, h->partials, tol, h->bbdev, G, h->stream);
      h->launches += 1;
    }
    if ((stt = last_launch())) return stt;
    if ((stt = cg_run<double>(h, Pd, ad, maxit, check, graphs, st))) return stt;
    for (int s = 0; s < S; ++s) {
      infos[s].iters = st[s].iter;
      infos[s].applies64 += st[s].iter;
      infos[s].relres = st[s].bb > 0 ? std::sqrt(std::max(st[s].rr, 0.0) / st[s].bb) : 0.0;
      infos[s].status = st[s].status ? st[s].status : (st[s].done ? LSH_OK : LSH_ERR_NOT_CONVERGED);
    }
  } else {
    // mixed precision: iterative refinement, FP64 residual, FP32 inner CG
    PrecBufs<float>& Pf = h->pf;
    const OpArgs<float> af = wave_args<float>(h, w);
    // default: two refinement steps reach tol (each inner solve reduces the
    // residual by 0.5 sqrt(tol)), within what FP32 CG resolves
    const double itol = o && o->inner_tol > 0 ? o->inner_tol : std::min(1e-3, std::max(1e-6, 0.5 * std::sqrt(tol)));
    const int max_outer = o && o->max_outer > 0 ? o->max_outer : 30;
    std::vector<double> rr(S);
    SolverState* sres = h->st + 2 * d.Smax;
    bool rdf = false;  // Pd.r holds double-float pairs (else FP64)
    if (!warm) {
      launch_fill_rhs<double>(ad, Pd.r, Pd.x, G, h->stream);
      h->launches += 1;
      rr = bb;
    } else {
      if ((stt = residual64(h, ad, Pd.x, Pd.r, h->dfres))) return stt;
      rdf = h->dfres;
      for (int s = 0; s < S; ++s) infos[s].applies64 += 1;
      std::vector<SolverState> s2(S);
      if ((stt = read_states(h, sres, S, s2.data()))) return stt;
      for (int s = 0; s < S; ++s) rr[s] = s2[s].aux[0];
    }
    if ((stt = last_launch())) return stt;
    std::vector<unsigned char> active(S);
    std::vector<double> prev = rr;
    std::vector<int> total(S, 0), stall(S, 0);
    int outer = 0, total_max = 0;
    for (;;) {
      int nact = 0;
      for (int s = 0; s < S; ++s) {
        const bool conv = rr[s] <= tol * tol * bb[s];
        const bool failed = infos[s].status != LSH_OK;
        active[s] = (!conv && !failed) ? 1 : 0;
        nact += active[s];
      }
      if (nact == 0) break;
      if (outer >= max_outer || total_max >= maxit) {
        for (int s = 0; s < S; ++s)
          if (active[s]) infos[s].status = LSH_ERR_NOT_CONVERGED;
        break;
      }
      LSH_CK(cudaMemcpyAsync(h->flags, active.data(), S, cudaMemcpyHostToDevice, h->stream));
      // default inner tolerance: relaxed on later steps to what still separates
      // the least converged system from the target (half of it, for the FP32
      // solve's recursive residual running ahead of the true one)
      double itol_k = itol;
      if (!(o && o->inner_tol > 0)) {
        double worst = 0.0;
        for (int s = 0; s < S; ++s)
          if (active[s] && bb[s] > 0) worst = std::max(worst, std::sqrt(rr[s] / bb[s]));
        if (worst > 0.0) itol_k = std::min(1e-3, std::max(itol, 0.5 * tol / worst));
      }
      launch_d2f_begin(Pd.r, rdf, Pf.r, Pf.x, n, S, Pf.st, h->partials, itol_k, h->flags, Pf.L.ew_per_sys,
                       h->stream);
      h->launches += 1;
      if ((stt = cg_run<float>(h, Pf, af, maxit - total_max, check, graphs, st))) return stt;
      launch_f2d_axpy(Pd.x, Pf.x, n * S, h->stream);
      h->launches += 1;
      if ((stt = residual64(h, ad, Pd.x, Pd.r, h->dfres))) return stt;
      rdf = h->dfres;
      std::vector<SolverState> s2(S);
      if ((stt = read_states(h, sres, S, s2.data()))) return stt;
      ++outer;
      for (int s = 0; s < S; ++s) {
        if (!active[s]) continue;
        infos[s].applies64 += 1;
        infos[s].outer += 1;
        total[s] += st[s].iter;
        total_max = std::max(total_max, total[s]);
        rr[s] = s2[s].aux[0];
        if (st[s].status == LSH_ERR_BREAKDOWN && rr[s] >= prev[s]) infos[s].status = LSH_ERR_BREAKDOWN;
        // refinement that stops reducing the true residual has reached the
        // attainable accuracy of the inner solver: give up after 3 such steps
        if (!(rr[s] < 0.5 * prev[s])) {
          if (++stall[s] >= 3) infos[s].status = LSH_ERR_NOT_CONVERGED;
        }
        prev[s] = rr[s];
      }
    }
    for (int s = 0; s < S; ++s) {
      infos[s].iters = total[s];
      infos[s].relres = bb[s] > 0 ? std::sqrt(std::max(rr[s], 0.0) / bb[s]) : 0.0;
    }
  }
  return LSH_OK;
}

lsh_status scan_microstructure(lsh_handle* h) {
  const Derived& d = h->d;
  SolverState* sscan = h->st + 3 * d.Smax;
  std::vector<SolverState> zero(d.B);
  LSH_CK(cudaMemcpyAsync(sscan, zero.data(), sizeof(SolverState) * d.B, cudaMemcpyHostToDevice, h->stream));
  const int G = (int)std::max(1LL, std::min((d.V + kThreads - 1) / kThreads, 1216LL));
  launch_scan_phase(h->phase, d.V, d.B, h->act, d.nphase, sscan, h->partials, G, h->stream);
  lsh_status stt = last_launch();
  if (stt) return stt;
  std::vector<SolverState> s(d.B);
  if ((stt = read_states(h, sscan, d.B, s.data()))) return stt;
  if (s[0].pad >= d.nphase) return LSH_ERR_INVALID_ARG;
  h->n_active.resize(d.B);
  for (int b = 0; b < d.B; ++b) h->n_active[b] = (long long)s[b].aux[1];
  return LSH_OK;
}

lsh_status copy_microstructure(lsh_handle* h, const unsigned char* phase, const float* scale, int on_host) {
  const cudaMemcpyKind k = on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const size_t nv = (size_t)(h->d.B * h->d.V);
  LSH_CK(cudaMemcpyAsync(h->phase, phase, nv, k, h->stream));
  if (h->d.has_scale) {
    if (!scale) return LSH_ERR_INVALID_ARG;
    LSH_CK(cudaMemcpyAsync(h->scale, scale, sizeof(float) * nv, k, h->stream));
  }
  return LSH_OK;
}

lsh_status rotate_or_copy(lsh_handle* h, const double* in, double* out, int nsys, int to_internal) {
  const Derived& d = h->d;
  if (d.physics == LSH_ELASTIC_ISO) {
    launch_rotate<double>(in, out, d.V, nsys, to_internal, h->stream);
    h->launches += 1;
    return last_launch();
  }
  if (d.rotated) {
    launch_rotate_scalar<double>(in, out, d.V, nsys, d.c, d.R, to_internal, h->stream);
    h->launches += 1;
    return last_launch();
  }
  if (in != out) LSH_CK(cudaMemcpyAsync(out, in, sizeof(double) * d.c * d.V * nsys, cudaMemcpyDeviceToDevice, h->stream));
  return LSH_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* lsh_status_string(lsh_status s) {
  switch (s) {
    case LSH_OK: return "ok";
    case LSH_ERR_INVALID_ARG: return "invalid argument";
    case LSH_ERR_UNSUPPORTED_SIZE: return "unsupported grid size";
    case LSH_ERR_REFERENCE_INDEFINITE: return "reference medium is not positive definite";
    case LSH_ERR_SINGULAR_CONTRAST: return "A_beta - A0 is singular but not zero";
    case LSH_ERR_BREAKDOWN: return "CG breakdown";
    case LSH_ERR_NOT_CONVERGED: return "not converged";
    case LSH_ERR_WORKSPACE: return "workspace too small or misaligned";
    case LSH_ERR_CUDA: return "CUDA runtime error";
    case LSH_ERR_UNSUPPORTED: return "unsupported by this build";
  }
  return "unknown status";
}

lsh_status lsh_workspace_size(const lsh_problem* prob, size_t* bytes) {
  if (!bytes) return LSH_ERR_INVALID_ARG;
  Derived d;
  lsh_status s = derive(prob, &d);
  if (s) return s;
  if (!cfg_fits(make_cfg<double>(d)) || !cfg_fits(make_cfg<float>(d))) return LSH_ERR_UNSUPPORTED_SIZE;
  *bytes = make_layout(d).total;
  return LSH_OK;
}

lsh_status lsh_setup(const lsh_problem* prob, void* workspace, size_t bytes, void* stream, lsh_handle** out) {
  if (!out || !workspace) return LSH_ERR_INVALID_ARG;
  *out = nullptr;
  lsh_handle* h = new (std::nothrow) lsh_handle();
  if (!h) return LSH_ERR_INVALID_ARG;
  lsh_status s = derive(prob, &h->d);
  if (s) { delete h; return s; }
  Derived& d = h->d;
  if (!cfg_fits(make_cfg<double>(d)) || !cfg_fits(make_cfg<float>(d))) {
    delete h;
    return LSH_ERR_UNSUPPORTED_SIZE;
  }
  h->lay = make_layout(d);
  if (bytes < h->lay.total || ((uintptr_t)workspace % kAlign) != 0) { delete h; return LSH_ERR_WORKSPACE; }
  h->stream = (cudaStream_t)stream;
  cudaGetDevice(&h->device);
  h->base = (unsigned char*)workspace;
  const Layout& l = h->lay;
  h->st = (SolverState*)(h->base + l.off_state);
  h->partials = (double*)(h->base + l.off_partials);
  h->phase = h->base + l.off_phase;
  h->scale = d.has_scale ? (float*)(h->base + l.off_scale) : nullptr;
  h->act = h->base + l.off_act;
  h->posx = (int*)(h->base + l.off_posx);
  h->kofy = (int*)(h->base + l.off_kofy);
  h->kofz = (int*)(h->base + l.off_kofz);
  h->kofy32 = (int*)(h->base + l.off_kofy32);
  h->kofz32 = (int*)(h->base + l.off_kofz32);
  h->sums = (double*)(h->base + l.off_sums);
  h->Wdev = (double*)(h->base + l.off_W);
  h->tabd = (double*)(h->base + l.off_tabd);
  h->bbdev = (double*)(h->base + l.off_bb);
  h->flags = h->base + l.off_flags;
  h->fault = (int*)(h->base + l.off_fault);
  h->ms = (MinresScalars*)(h->base + l.off_ms);
  h->sq = (SymmlqScalars*)(h->ms + d.Smax);
  if (l.minres) {
    h->wa = (double*)(h->base + l.off_wa);
    h->wb = (double*)(h->base + l.off_wb);
  }
  if (cudaMemsetAsync(h->fault, 0, sizeof(int), h->stream) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return LSH_ERR_CUDA;
  }
  {
    const char* e = getenv("LSH_NO_TMA");
    h->no_tma = e && e[0] == '1';
    const char* f = getenv("LSH_NO_DF");
    h->dfres = l.df && !(f && f[0] == '1');
    if (l.df) {
      h->gdf = (DF*)(h->base + l.off_gdf);
      h->twdf = (DF2*)(h->base + l.off_twdf);
    }
  }
  init_prec<double>(h, h->pd, l.off_fd, l.off_Hd, l.off_gd, l.off_tw_d, l.off_tabd, l.off_loads_d, h->st);
  if (d.precision == LSH_MIXED)
    init_prec<float>(h, h->pf, l.off_ff, l.off_Hf, l.off_gf, l.off_tw_f, l.off_tabf, l.off_loads_f, h->st + d.Smax);

  // host tables
  // register-FFT axes keep natural frequency order; the others are digit-reversed
  std::vector<int> posx(d.nx), kofy(d.ny), kofz(d.nz);
  for (int k = 0; k < d.nx; ++k) posx[k] = dif_position(d.px, k);
  for (int k = 0; k < d.ny; ++k) kofy[h->pd.a.yreg ? k : dif_position(d.py, k)] = k;
  for (int k = 0; k < d.nz; ++k) kofz[h->pd.a.zreg ? k : dif_position(d.pz, k)] = k;
  std::vector<int> kofy32(kofy), kofz32(kofz);
  if (d.plane) {
    for (int k = 0; k < d.ny; ++k) kofy32[k] = k;
    for (int k = 0; k < d.nz; ++k) kofz32[k] = k;
  }
  std::vector<double> twd, tmpd;
  twiddles<double>(d.nx, tmpd); twd.insert(twd.end(), tmpd.begin(), tmpd.end());
  twiddles<double>(d.ny, tmpd); twd.insert(twd.end(), tmpd.begin(), tmpd.end());
  twiddles<double>(d.nz, tmpd); twd.insert(twd.end(), tmpd.begin(), tmpd.end());
  std::vector<float> twf(twd.size());
  for (size_t i = 0; i < twd.size(); ++i) twf[i] = (float)twd[i];
  std::vector<double> tabd(2 * 256 * 6, 0.0);
  std::vector<float> tabf(2 * 256 * 6, 0.0f);
  for (int ph = 0; ph < d.nphase; ++ph)
    for (int i = 0; i < d.c; ++i) {
      tabd[ph * d.c + i] = d.m_in[ph * d.c + i];
      tabd[256 * 6 + ph * d.c + i] = d.mod_in[ph * d.c + i];
    }
  for (size_t i = 0; i < tabd.size(); ++i) tabf[i] = (float)tabd[i];

  cudaStream_t st = h->stream;
  std::vector<SolverState> zero(3 * d.Smax + d.B);
#define SETUP_CK(call) do { if ((call) != cudaSuccess) { cudaGetLastError(); delete h; return LSH_ERR_CUDA; } } while (0)
  SETUP_CK(cudaMemcpyAsync(h->st, zero.data(), sizeof(SolverState) * zero.size(), cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->act, d.act.data(), 256, cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->posx, posx.data(), sizeof(int) * d.nx, cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->kofy, kofy.data(), sizeof(int) * d.ny, cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->kofz, kofz.data(), sizeof(int) * d.nz, cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->kofy32, kofy32.data(), sizeof(int) * d.ny, cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->kofz32, kofz32.data(), sizeof(int) * d.nz, cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->base + l.off_tw_d, twd.data(), sizeof(double) * twd.size(), cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->base + l.off_tw_f, twf.data(), sizeof(float) * twf.size(), cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->base + l.off_tabd, tabd.data(), sizeof(double) * tabd.size(), cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->base + l.off_tabf, tabf.data(), sizeof(float) * tabf.size(), cudaMemcpyHostToDevice, st));
  if (copy_microstructure(h, prob->phase, prob->scale, prob->phase_on_host) != LSH_OK) { delete h; return LSH_ERR_CUDA; }
  set_smem_attrs<double>();
  set_smem_attrs<float>();
  tma_prepare();
  xreg_prepare();
  if (d.plane) {
    plane_prepare();
    zpipe_prepare();
    // the z pass of the plane passes without tuning: the fused TMA kernel where it
    // has a plan (the autotuner's choice on every grid of the batched workload),
    // else the register kernel
    OpArgs<float> az = h->pf.a;
    az.S = 0;
    if (d.precision == LSH_MIXED && launch_zgamma_pipe(az, true, nullptr, 0)) h->pf.a.ztma = 11;
  }
  if (l.df) df_prepare();
  launch_gamma_table<double>(h->pd.a, d.dim, d.physics, d.green, d.ref_user, h->kofy, h->kofz, st,
                             d.rotated ? d.A0full : nullptr, d.rotated ? d.R : nullptr);
  if (d.precision == LSH_MIXED)
    launch_gamma_table<float>(h->pf.a, d.dim, d.physics, d.green, d.ref_user, h->kofy32, h->kofz32, st,
                              d.rotated ? d.A0full : nullptr, d.rotated ? d.R : nullptr);
  if (l.df) {
    const long long nf = (long long)d.nz * d.ny * d.ts, ncop = (d.ncoef + 3) & ~3;
    if (d.plane && !(reg_len(d.ny) && reg_len(d.nz))) {
      // the FP64 table follows the digit-reversed y / z positions of the FP64
      // passes: build one in natural order in the double-float table's own
      // memory (8 bytes per value either way) and convert it there
      OpArgs<double> an = h->pd.a;
      an.gtab = reinterpret_cast<double*>(h->gdf);
      an.kofy = h->kofy32;
      an.kofz = h->kofz32;
      launch_gamma_table<double>(an, d.dim, d.physics, d.green, d.ref_user, h->kofy32, h->kofz32, st,
                                 d.rotated ? d.A0full : nullptr, d.rotated ? d.R : nullptr);
      launch_d2df_inplace(h->gdf, ncop * nf, st);
    } else {
      launch_d2df(h->pd.gtab, h->gdf, ncop * nf, st);
    }
    launch_d2df((const double*)(h->base + l.off_tw_d), reinterpret_cast<DF*>(h->twdf), 2ll * (d.nx + d.ny + d.nz), st);
  }
  if (last_launch() != LSH_OK) { delete h; return LSH_ERR_CUDA; }
  s = scan_microstructure(h);  // synchronises the stream (host vectors may go)
  if (s) { delete h; return s; }
#undef SETUP_CK
  *out = h;
  return LSH_OK;
}

lsh_status lsh_set_microstructure(lsh_handle* h, const unsigned char* phase, const float* scale, int on_host) {
  if (!h || !phase) return LSH_ERR_INVALID_ARG;
  h->drop_graphs();  // the scale pointer in the captured arguments may change
  lsh_status s = copy_microstructure(h, phase, scale, on_host);
  if (s) return s;
  return scan_microstructure(h);
}

lsh_status lsh_apply(lsh_handle* h, int dtype, const void* x, void* y) {
  if (!h || !x || !y) return LSH_ERR_INVALID_ARG;
  const Derived& d = h->d;
  const bool el = d.physics == LSH_ELASTIC_ISO;
  const long long n = (long long)d.c * d.V;
  if (dtype != LSH_F64 && dtype != LSH_F32 && dtype != LSH_F64_DF) return LSH_ERR_INVALID_ARG;
  if (dtype == LSH_F32 && d.precision != LSH_MIXED) return LSH_ERR_UNSUPPORTED;
  if (dtype == LSH_F64_DF && !h->lay.df) return LSH_ERR_UNSUPPORTED;
  // one system per microstructure; in waves when the handle holds fewer systems
  // (FP64 on a mixed handle: one system at a time through the p, q scratch)
  const int per_wave = (dtype != LSH_F32 && d.precision == LSH_MIXED) ? 1 : std::min(d.Smax, d.B);
  for (int b0 = 0; b0 < d.B; b0 += per_wave) {
    const int S = std::min(per_wave, d.B - b0);
    std::vector<double> zl(6 * (size_t)S, 0.0);
    Wave w{S, b0, 1, zl.data()};
    // fields enter and leave in the caller's basis; the kernels work in the internal one
    const bool rot = el || d.rotated;
    auto rotate = [&](auto* in, auto* out, int to_internal) {
      typedef std::remove_const_t<std::remove_pointer_t<decltype(in)>> TT;
      if (el) launch_rotate<TT>(in, out, d.V, S, to_internal, h->stream);
      else launch_rotate_scalar<TT>(in, out, d.V, S, d.c, d.R, to_internal, h->stream);
    };
    if (dtype != LSH_F32) {
      PrecBufs<double>& P = h->pd;
      const double* in = (const double*)x + b0 * n;
      double* o = (double*)y + b0 * n;
      if (rot) {
        rotate(in, P.p, 1);
        in = P.p;
      }
      lsh_status s = dtype == LSH_F64_DF ? apply_df(h, wave_args<double>(h, w), in, rot ? P.q : o)
                                         : apply_internal<double>(h, wave_args<double>(h, w), in, rot ? P.q : o);
      if (s) return s;
      if (rot) rotate((const double*)P.q, o, 0);
    } else {
      PrecBufs<float>& P = h->pf;
      const float* in = (const float*)x + b0 * n;
      float* o = (float*)y + b0 * n;
      // the plane passes move fields in 16-byte pieces: unaligned caller buffers
      // go through the handle's own
      const bool stage = !rot && P.a.plane && (((uintptr_t)in | (uintptr_t)o) & 15) != 0;
      if (rot) {
        rotate(in, P.p, 1);
        in = P.p;
      } else if (stage) {
        LSH_CK(cudaMemcpyAsync(P.p, in, sizeof(float) * (size_t)(S * n), cudaMemcpyDeviceToDevice, h->stream));
        in = P.p;
      }
      lsh_status s = apply_internal<float>(h, wave_args<float>(h, w), in, (rot || stage) ? P.q : o);
      if (s) return s;
      if (rot) rotate((const float*)P.q, o, 0);
      else if (stage)
        LSH_CK(cudaMemcpyAsync(o, P.q, sizeof(float) * (size_t)(S * n), cudaMemcpyDeviceToDevice, h->stream));
    }
  }
  return last_launch();
}

lsh_status lsh_solve(lsh_handle* h, const double* load, double* tau, const lsh_solve_opts* opts,
                     lsh_solve_info* info) {
  if (!h || !load || !tau) return LSH_ERR_INVALID_ARG;
  const Derived& d = h->d;
  const long long n = (long long)d.c * d.V;
  double lin[6] = {0, 0, 0, 0, 0, 0};
  to_internal(d, load, lin);
  const bool warm = opts && opts->warm_start;
  lsh_status worst = LSH_OK;
  const int per_wave = std::min(d.Smax, d.B);
  for (int b0 = 0; b0 < d.B; b0 += per_wave) {
    const int S = std::min(per_wave, d.B - b0);
    std::vector<double> loads(6 * (size_t)S);
    for (int s = 0; s < S; ++s)
      for (int i = 0; i < 6; ++i) loads[6 * s + i] = lin[i];
    Wave w{S, b0, 1, loads.data()};
    if (warm) {
      lsh_status r = rotate_or_copy(h, tau + b0 * n, h->pd.x, S, 1);
      if (r) return r;
    }
    std::vector<lsh_solve_info> inf(S);
    lsh_status r = solve_wave(h, w, warm, opts, inf.data());
    if (r) return r;
    if ((r = check_fault(h))) return r;
    if ((r = rotate_or_copy(h, h->pd.x, tau + b0 * n, S, 0))) return r;
    for (int s = 0; s < S; ++s) {
      if (info) info[b0 + s] = inf[s];
      if (inf[s].status != LSH_OK && worst == LSH_OK) worst = (lsh_status)inf[s].status;
    }
  }
  LSH_CK(cudaStreamSynchronize(h->stream));
  return worst;
}

lsh_status lsh_effective(lsh_handle* h, const lsh_solve_opts* opts, double* Astar, double* tau_all,
                         lsh_solve_info* infos) {
  if (!h || !Astar) return LSH_ERR_INVALID_ARG;
  const Derived& d = h->d;
  const int c = d.c;
  const long long n = (long long)c * d.V;
  double A0[36];
  ref_matrix(d, A0);
  const int nblk = 152;
  const int total = d.B * c;
  lsh_status worst = LSH_OK;
  lsh_solve_opts o = opts ? *opts : lsh_solve_opts{};
  o.warm_start = 0;
  for (int s0 = 0; s0 < total; s0 += d.Smax) {
    const int S = std::min(d.Smax, total - s0);
    // system g = b * c + j: microstructure b, unit load e_j (Mandel)
    std::vector<double> loads(6 * (size_t)S, 0.0);
    for (int s = 0; s < S; ++s) {
      double e[6] = {0, 0, 0, 0, 0, 0};
      e[(s0 + s) % c] = 1.0;
      to_internal(d, e, &loads[6 * s]);
    }
    Wave w{S, s0, c, loads.data()};
    std::vector<lsh_solve_info> inf(S);
    lsh_status r = solve_wave(h, w, false, &o, inf.data());
    if (r) return r;
    if ((r = check_fault(h))) return r;
    // A*_h e_j = A0 e_j + h^d sum_beta tau_beta (Eq. (tau_Astar), Theorem 13)
    launch_comp_sums<double>(h->pd.x, c, d.V, S, h->partials, nblk, h->sums, h->stream);
    h->launches += 2;
    if (tau_all && (r = rotate_or_copy(h, h->pd.x, tau_all + (long long)s0 * n, S, 0))) return r;
    std::vector<double> sums((size_t)S * c);
    LSH_CK(cudaMemcpyAsync(sums.data(), h->sums, sizeof(double) * S * c, cudaMemcpyDeviceToHost, h->stream));
    LSH_CK(cudaStreamSynchronize(h->stream));
    for (int s = 0; s < S; ++s) {
      const int g = s0 + s, b = g / c, j = g % c;
      double mean[6], meanM[6];
      for (int i = 0; i < c; ++i) mean[i] = sums[(size_t)s * c + i] / (double)d.V;
      to_mandel(d, mean, meanM);
      for (int i = 0; i < c; ++i) Astar[((size_t)b * c + i) * c + j] = A0[i * c + j] + meanM[i];
      if (infos) infos[g] = inf[s];
      if (inf[s].status != LSH_OK && worst == LSH_OK) worst = (lsh_status)inf[s].status;
    }
  }
  return worst;
}

lsh_status lsh_effective_batch(int nh, lsh_handle* const* hs, const lsh_solve_opts* opts, double* Astar,
                               lsh_solve_info* infos) {
  if (nh < 0 || (nh > 0 && (!hs || !Astar))) return LSH_ERR_INVALID_ARG;
  std::vector<size_t> aoff(nh + 1, 0), ioff(nh + 1, 0);
  for (int k = 0; k < nh; ++k) {
    if (!hs[k]) return LSH_ERR_INVALID_ARG;
    for (int j = 0; j < k; ++j)
      if (hs[j] == hs[k]) return LSH_ERR_INVALID_ARG;
    const size_t nb = (size_t)hs[k]->d.B, c = (size_t)hs[k]->d.c;
    aoff[k + 1] = aoff[k] + nb * c * c;
    ioff[k + 1] = ioff[k] + nb * c;
  }
  std::vector<lsh_status> st(nh, LSH_OK);
  auto run = [&](int k) {
    if (cudaSetDevice(hs[k]->device) != cudaSuccess) {
      cudaGetLastError();
      st[k] = LSH_ERR_CUDA;
      return;
    }
    st[k] = lsh_effective(hs[k], opts, Astar + aoff[k], nullptr, infos ? infos + ioff[k] : nullptr);
  };
  std::vector<std::thread> pool;
  int k0 = 0;
  try {
    for (; k0 < nh; ++k0) pool.emplace_back(run, k0);
  } catch (...) {
    // no more host threads: the remaining handles run on this one
  }
  for (int k = k0; k < nh; ++k) run(k);
  for (auto& t : pool) t.join();
  for (int k = 0; k < nh; ++k)
    if (st[k] != LSH_OK) return st[k];
  return LSH_OK;
}

lsh_status lsh_effective_grad(lsh_handle* h, const double* tau_all, const double* W, double* grad) {
  if (!h || !tau_all || !W || !grad) return LSH_ERR_INVALID_ARG;
  if (h->d.frac) return LSH_ERR_UNSUPPORTED;
  const Derived& d = h->d;
  double wbuf[64] = {0};
  for (int i = 0; i < d.c * d.c; ++i) wbuf[i] = W[i];
  for (int i = 0; i < 6; ++i) wbuf[40 + i] = i < d.c ? d.ref_in[i] : 0.0;
  LSH_CK(cudaMemcpyAsync(h->Wdev, wbuf, sizeof(wbuf), cudaMemcpyHostToDevice, h->stream));
  launch_scale_grad(tau_all, h->Wdev, h->phase, h->scale, h->tabd + 256 * 6, h->Wdev + 40, d.c,
                    d.physics == LSH_ELASTIC_ISO, d.V, d.B, grad, h->stream);
  h->launches += 1;
  lsh_status s = last_launch();
  if (s) return s;
  LSH_CK(cudaStreamSynchronize(h->stream));
  return LSH_OK;
}

lsh_status lsh_autotune(lsh_handle* h, lsh_tune_report* rep) {
  if (!h) return LSH_ERR_INVALID_ARG;
  lsh_tune_report r;
  r.x_variant = h->pf.a.xreg;
  r.xf_variant = h->pf.a.xfreg;
  for (int k = 0; k < 2; ++k) r.xf_ms[k] = -1.f;
  r.y_variant = h->pf.a.plane ? 2 : h->pf.a.ytma;
  r.z_variant = h->pf.a.ztma;
  for (int k = 0; k < 4; ++k) r.x_ms[k] = -1.f;
  for (int k = 0; k < 2; ++k) r.y_ms[k] = -1.f;
  for (int k = 0; k < 10; ++k) r.z_ms[k] = -1.f;
  for (int k = 0; k < 2; ++k) r.xy_ms[k] = -1.f;
  for (int k = 0; k < 7; ++k) r.zp_ms[k] = -1.f;
  const Derived& d = h->d;
  if (d.precision == LSH_MIXED) {
    PrecBufs<float>& P = h->pf;
    cudaStream_t s = h->stream;
    LSH_CK(cudaMemsetAsync(P.H, 0, sizeof(float2) * (size_t)d.Smax * d.c * d.nz * d.ny * d.hs, s));
    OpArgs<float> a = P.a;
    cudaEvent_t e0, e1;
    LSH_CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaGetLastError();
      return LSH_ERR_CUDA;
    }
    // average of 5 launches after 2 untimed ones; -1 if the variant does not run here
    auto timeit = [&](auto launch) -> float {
      for (int k = 0; k < 2; ++k)
        if (!launch()) return -1.f;
      cudaEventRecord(e0, s);
      for (int k = 0; k < 5; ++k) launch();
      cudaEventRecord(e1, s);
      float ms = -1.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        cudaGetLastError();
        return -1.f;
      }
      return ms / 5.f;
    };
    // the x passes are timed as in a CG iteration, on states of a running solve
    std::vector<SolverState> fake(d.Smax);
    for (auto& f : fake) {
      f = SolverState{};
      f.iter = 1;
      f.rr = 1.0;
    }
    LSH_CK(cudaMemcpyAsync(P.st, fake.data(), sizeof(SolverState) * d.Smax, cudaMemcpyHostToDevice, s));
    // the separate x and y passes need natural y order for the FP32 table on
    // plane grids (powers of two); radix-3 planes have the plane passes only
    const bool sep_ok = !d.plane || reg_length(d.ny);
    a.plane = 0;
    a.tlay = 0;
    if (sep_ok && xfwd_reg_fits(a)) {
      for (int v = 0; v < 2; ++v) {
        a.xfreg = v;
        r.xf_ms[v] = timeit([&]() {
          cudaMemcpyAsync(P.st, fake.data(), sizeof(SolverState) * d.Smax, cudaMemcpyHostToDevice, s);
          if (v == 1) return launch_xfwd_reg(a, 1, nullptr, P.x, P.r, P.p, P.st, s);
          launch_xfwd<float>(a, P.L, 1, nullptr, P.x, P.r, P.p, P.st, s);
          return true;
        });
      }
      r.xf_variant = (r.xf_ms[1] > 0.f && r.xf_ms[1] < r.xf_ms[0]) ? 1 : 0;
      a.xfreg = r.xf_variant;
    }
    if (sep_ok) {
      // inverse x pass with the local term and the (p, Kp) reduction
      int bx = 0;
      for (int v = 0; v < 4; ++v) {
        a.xreg = v;
        r.x_ms[v] = timeit([&]() {
          // fresh states each time: a breakdown flagged on the arbitrary data would stop the next launch
          cudaMemcpyAsync(P.st, fake.data(), sizeof(SolverState) * d.Smax, cudaMemcpyHostToDevice, s);
          if (v >= 1) return launch_xinv_reg(a, 1, P.p, P.q, P.st, h->partials, s, v == 2, v == 3);
          launch_xinv<float>(a, P.L, 1, P.p, P.q, P.st, h->partials, s);
          return true;
        });
        if (r.x_ms[v] > 0.f && r.x_ms[v] < r.x_ms[bx]) bx = v;
      }
      r.x_variant = bx;
      a.xreg = r.x_variant;
    }
    if (sep_ok && a.yreg && P.ytma_ok) {
      for (int v = 0; v < 2; ++v) {
        a.ytma = v;
        r.y_ms[v] = timeit([&]() {
          launch_yfft<float>(a, P.L, false, nullptr, s);
          return true;
        });
      }
      r.y_variant = (r.y_ms[1] > 0.f && (r.y_ms[0] < 0.f || r.y_ms[1] < r.y_ms[0])) ? 1 : 0;
      a.ytma = r.y_variant;
    }
    if (sep_ok && a.zreg) {
      int best = 0;
      for (int v = 0; v < 10; ++v) {
        if (v >= 1 && v <= 5 && !P.ztma_ok) continue;  // TMA tiles need the tensor map
        a.ztma = v;
        r.z_ms[v] = timeit([&]() {
          if (v == 0 || v == 6 || v == 8 || v == 9) {
            launch_zgamma<float>(a, P.L, nullptr, s);
            return true;
          }
          if (v == 7) return launch_zgamma_regp(a, nullptr, s);
          return launch_zgamma_tma(a, v, nullptr, s);
        });
        if (r.z_ms[v] > 0.f && (r.z_ms[best] < 0.f || r.z_ms[v] < r.z_ms[best])) best = v;
      }
      r.z_variant = best;
      a.ztma = best;
    }
    if (d.plane) {
      // the plane passes with the register z kernels on the ky-major spectrum,
      // against the best separate passes, summed over one CG iteration
      OpArgs<float> b = a;
      b.plane = 1;
      b.tlay = 1;
      const int zc[7] = {0, 6, 8, 9, 7, 10, 11};
      int bz = 0;
      for (int k = 0; k < 7; ++k) {
        b.ztma = zc[k];
        r.zp_ms[k] = timeit([&]() {
          if (zc[k] == 7) return launch_zgamma_regp(b, nullptr, s);
          if (zc[k] >= 10) return launch_zgamma_pipe(b, zc[k] == 11, nullptr, s);
          launch_zgamma<float>(b, P.L, nullptr, s);
          return true;
        });
        if (r.zp_ms[k] > 0.f && (r.zp_ms[bz] < 0.f || r.zp_ms[k] < r.zp_ms[bz])) bz = k;
      }
      b.ztma = zc[bz];
      const float f = timeit([&]() {
        cudaMemcpyAsync(P.st, fake.data(), sizeof(SolverState) * d.Smax, cudaMemcpyHostToDevice, s);
        return launch_xyfwd(b, 1, nullptr, P.x, P.r, P.p, P.st, s);
      });
      const float i = timeit([&]() {
        cudaMemcpyAsync(P.st, fake.data(), sizeof(SolverState) * d.Smax, cudaMemcpyHostToDevice, s);
        return launch_xyinv(b, 1, P.p, P.q, P.st, h->partials, s);
      });
      r.xy_ms[1] = (f > 0.f && i > 0.f && r.zp_ms[bz] > 0.f) ? f + r.zp_ms[bz] + i : -1.f;
      if (sep_ok) {
        const float xf = r.xf_ms[a.xfreg] > 0.f ? r.xf_ms[a.xfreg] : r.xf_ms[0];
        const float yy = r.y_ms[a.ytma] > 0.f ? r.y_ms[a.ytma] : -1.f;
        const float zz = r.z_ms[a.ztma], xi = r.x_ms[a.xreg];
        if (xf > 0.f && yy > 0.f && zz > 0.f && xi > 0.f) r.xy_ms[0] = xf + 2.f * yy + zz + xi;
      }
      if (!sep_ok || (r.xy_ms[1] > 0.f && (r.xy_ms[0] < 0.f || r.xy_ms[1] < r.xy_ms[0]))) {
        a = b;
        r.y_variant = 2;
        r.z_variant = b.ztma;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    lsh_status st = last_launch();
    if (st) return st;
    if (h->fault && (st = check_fault(h))) return st;
    P.a.xreg = a.xreg;
    P.a.xfreg = a.xfreg;
    P.a.ytma = a.ytma;
    P.a.ztma = a.ztma;
    P.a.plane = a.plane;
    P.a.tlay = a.tlay;
    h->drop_graphs();  // captured with the previous choices
  }
  if (rep) *rep = r;
  return LSH_OK;
}

lsh_status lsh_set_variants(lsh_handle* h, int xf_variant, int x_variant, int y_variant, int z_variant) {
  if (!h) return LSH_ERR_INVALID_ARG;
  if (xf_variant < 0 || xf_variant > 1 || x_variant < 0 || x_variant > 3 || y_variant < 0 || y_variant > 2 ||
      z_variant < 0 || z_variant > 11)
    return LSH_ERR_INVALID_ARG;
  PrecBufs<float>& P = h->pf;
  if (h->d.precision != LSH_MIXED)
    return (xf_variant || x_variant || y_variant || z_variant) ? LSH_ERR_UNSUPPORTED : LSH_OK;
  if (y_variant == 2) {
    // plane passes: the register z kernels on the ky-major spectrum
    if (!h->d.plane || !(z_variant == 0 || z_variant >= 6)) return LSH_ERR_UNSUPPORTED;
    OpArgs<float> a = P.a;
    a.S = 0;
    a.plane = 1;
    a.tlay = 1;
    if (z_variant == 7 && !launch_zgamma_regp(a, nullptr, 0)) return LSH_ERR_UNSUPPORTED;
    if (z_variant >= 10 && !launch_zgamma_pipe(a, z_variant == 11, nullptr, 0)) return LSH_ERR_UNSUPPORTED;
    P.a.plane = 1;
    P.a.tlay = 1;
    P.a.ztma = z_variant;
    h->drop_graphs();
    return LSH_OK;
  }
  if (h->d.plane && !reg_length(h->d.ny)) return LSH_ERR_UNSUPPORTED;  // radix-3 planes: plane passes only
  if (x_variant >= 1 && !xinv_reg_fits(P.a)) return LSH_ERR_UNSUPPORTED;
  if (xf_variant == 1 && !xfwd_reg_fits(P.a)) return LSH_ERR_UNSUPPORTED;
  if (y_variant == 1 && !P.ytma_ok) return LSH_ERR_UNSUPPORTED;
  if (z_variant >= 6 && !P.a.zreg) return LSH_ERR_UNSUPPORTED;
  if (z_variant >= 10) return LSH_ERR_UNSUPPORTED;  // ky-major spectrum only
  if (z_variant == 7) {
    OpArgs<float> a = P.a;
    a.S = 0;
    if (!launch_zgamma_regp(a, nullptr, 0)) return LSH_ERR_UNSUPPORTED;
  }
  if (z_variant >= 1 && z_variant <= 5 && !P.ztma_ok) return LSH_ERR_UNSUPPORTED;
  if (z_variant >= 1 && z_variant <= 5) {
    // the variant must have a kernel for this length and component count
    OpArgs<float> a = P.a;
    a.S = 0;
    if (!tma_z_variant_fits(a, z_variant)) return LSH_ERR_UNSUPPORTED;
  }
  P.a.xreg = x_variant;
  P.a.xfreg = xf_variant;
  P.a.ytma = y_variant;
  P.a.ztma = z_variant;
  P.a.plane = 0;
  P.a.tlay = 0;
  h->drop_graphs();
  return LSH_OK;
}

lsh_status lsh_check_bounded_wait(lsh_handle* h, double seconds) {
  if (!h || !(seconds > 0.0) || seconds > 10.0) return LSH_ERR_INVALID_ARG;
  launch_wait_probe(h->fault, (unsigned long long)(seconds * 1e9), h->stream);
  h->launches += 1;
  if (last_launch() != LSH_OK) return LSH_ERR_CUDA;
  return check_fault(h);
}

lsh_status lsh_profile_enable(lsh_handle* h, int enable) {
  if (!h) return LSH_ERR_INVALID_ARG;
  if (enable && h->ev.empty()) {
    h->ev.resize(7 * 64);
    for (auto& e : h->ev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return LSH_ERR_CUDA;
      }
  }
  h->prof = enable != 0;
  h->prof_every = enable > 1 ? enable : 1;
  h->prof_chunk = 0;
  h->ev_used = 0;
  return LSH_OK;
}

lsh_status lsh_profile_read(lsh_handle* h, lsh_profile* out, int reset) {
  if (!h || !out) return LSH_ERR_INVALID_ARG;
  out->launches = h->launches;
  out->timed_iters = h->timed_iters;
  out->timed_sys_iters = h->timed_sys_iters;
  for (int k = 0; k < 6; ++k) {
    out->pass_ms[k] = h->pass_ms[k];
    out->pass_launches[k] = h->pass_n[k];
  }
  if (reset) {
    h->launches = 0;
    h->timed_iters = 0;
    h->timed_sys_iters = 0;
    for (int k = 0; k < 6; ++k) {
      h->pass_ms[k] = 0.0;
      h->pass_n[k] = 0;
    }
  }
  return LSH_OK;
}

void lsh_destroy(lsh_handle* h) { delete h; }

}  // extern "C"
