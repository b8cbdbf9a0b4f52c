// lsh_api.cu -- host side of the liblsh C ABI (include/lsh.h).
//
// Setup validates the problem, derives the diagonal local operator per phase,
// builds the FFT plans, twiddles and the Gamma^h table, and carves every
// device buffer out of the caller's workspace.  Solves drive the operator
// passes of kernels.cu from the host: each CG iteration is six launches whose
// scalars (alpha, beta, (r,r)) stay on the device; the host reads the device
// state only every `check_every` iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "lsh.h"

using namespace lsh;

namespace {

constexpr size_t kAlign = 256;
constexpr int kThreads = 256;
constexpr int kMaxSmem = 227 * 1024;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

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
  int dim, c, nx, ny, nz, nxh, ncoef, physics, green, precision, nphase;
  long long V;
  bool has_scale;
  Plan1D px, py, pz;
  double ref_in[6];      // diagonal of A0 in the internal basis
  double ref_user[6];    // scalar: diagonal of A0; elastic: (K0, mu0)
  std::vector<double> mod_in;  // nphase * c diagonal of A_phase, internal basis
  std::vector<double> m_in;    // nphase * c diagonal of M (0 when inactive)
  std::vector<unsigned char> act;
  int definite;          // +1 / -1: all active phases same sign; 0: indefinite
};

lsh_status derive(const lsh_problem* pr, Derived* d) {
  if (!pr) return LSH_ERR_INVALID_ARG;
  if (pr->dim != 2 && pr->dim != 3) return LSH_ERR_INVALID_ARG;
  if (pr->physics != LSH_SCALAR && pr->physics != LSH_ELASTIC_ISO) return LSH_ERR_INVALID_ARG;
  if (pr->physics == LSH_ELASTIC_ISO && pr->dim != 3) return LSH_ERR_INVALID_ARG;
  if (pr->green != LSH_GREEN_TRUNCATED && pr->green != LSH_GREEN_FILTERED) return LSH_ERR_INVALID_ARG;
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
  d->c = pr->physics == LSH_ELASTIC_ISO ? 6 : pr->dim;
  d->ncoef = d->c * (d->c + 1) / 2;
  d->has_scale = pr->scale != nullptr;
  if (!make_plan(d->nx, &d->px) || !make_plan(d->ny, &d->py) || !make_plan(d->nz, &d->pz))
    return LSH_ERR_UNSUPPORTED_SIZE;
  const int c = d->c, dim = d->dim;
  // reference medium
  if (!pr->ref_moduli && d->has_scale) return LSH_ERR_INVALID_ARG;
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
    for (int ph = 0; ph < pr->nphase; ++ph)
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j)
          if (i != j && pr->phase_moduli[ph * dim * dim + i * dim + j] != 0.0) return LSH_ERR_UNSUPPORTED;
    if (pr->ref_moduli) {
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j)
          if (i != j && pr->ref_moduli[i * dim + j] != 0.0) return LSH_ERR_UNSUPPORTED;
      for (int i = 0; i < dim; ++i) d->ref_in[i] = pr->ref_moduli[i * dim + i];
    } else {
      double amin = pr->phase_moduli[0];
      for (int ph = 0; ph < pr->nphase; ++ph)
        for (int i = 0; i < dim; ++i) amin = std::min(amin, pr->phase_moduli[ph * dim * dim + i * dim + i]);
      for (int i = 0; i < dim; ++i) d->ref_in[i] = 0.5 * amin;
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
    } else {
      for (int i = 0; i < dim; ++i) md[i] = pr->phase_moduli[ph * dim * dim + i * dim + i];
    }
    if (d->has_scale) {
      // the scale field makes every voxel of an active phase active; the sign
      // structure is the caller's responsibility (A0 softer than s A_phase)
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
  return LSH_OK;
}

// ---------------------------------------------------------------- workspace layout
template <typename T> struct PrecBufs {
  T *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
  C2<T>* H = nullptr;
  T* gtab = nullptr;
  C2<T>*twx = nullptr, *twy = nullptr, *twz = nullptr;
  T *mtab = nullptr, *modtab = nullptr;
  SolverState* st = nullptr;
  LaunchCfg L{};
  OpArgs<T> a{};
};

struct Layout {
  size_t off_state, off_partials, off_phase, off_scale, off_act, off_posx, off_kofy, off_kofz, off_sums, off_W;
  size_t off_tabd, off_tabf;  // per-phase tables (mtab, modtab) for each precision
  size_t off_tw_d, off_tw_f;
  size_t off_fd[4], off_Hd, off_gd;
  size_t off_ff[4], off_Hf, off_gf;
  size_t total;
  int nparts;
};

template <typename T> LaunchCfg make_cfg(const Derived& d) {
  LaunchCfg L{};
  L.threads = kThreads;
  const size_t cs = sizeof(C2<T>);
  const int lsx = d.nx | 1, lsy = d.ny | 1, lsz = d.nz | 1;
  const int nrows = d.c * d.nz * d.ny;
  int npair = std::max(1, (int)(32768 / (lsx * cs)));
  int RY = 2 * npair;
  RY = std::min(RY, nrows + (nrows & 1));
  L.smem_x = d.nx * cs + (size_t)(RY / 2) * lsx * cs + d.nx * sizeof(int);
  int TY = sizeof(T) == 8 ? 8 : 16;
  TY = std::min(TY, d.nxh);
  L.smem_y = d.ny * cs + (size_t)TY * lsy * cs;
  int TZ = sizeof(T) == 8 ? 8 : 16;
  TZ = std::min(TZ, d.nxh);
  while (TZ > 1 && (size_t)d.c * TZ * lsz * cs > 100 * 1024) TZ /= 2;
  L.smem_z = d.nz * cs + (size_t)d.c * TZ * lsz * cs;
  L.grid_x = (nrows + RY - 1) / RY;
  L.grid_yx = (d.nxh + TY - 1) / TY;
  L.grid_yy = d.c * d.nz;
  L.grid_zx = (d.nxh + TZ - 1) / TZ;
  L.grid_zy = d.ny;
  const long long n = (long long)d.c * d.V;
  L.grid_ew = (int)std::max(1LL, std::min((n + kThreads - 1) / kThreads, 152LL * 8));
  L.RY = RY;
  L.TY = TY;
  L.TZ = TZ;
  return L;
}

template <typename T> bool cfg_fits(const LaunchCfg& L) {
  return L.smem_x <= (size_t)kMaxSmem && L.smem_y <= (size_t)kMaxSmem && L.smem_z <= (size_t)kMaxSmem &&
         L.grid_yy <= 65535 && L.grid_zy <= 65535;
}

Layout make_layout(const Derived& d) {
  Layout l{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const long long n = (long long)d.c * d.V;
  const long long nf = (long long)d.nz * d.ny * d.nxh;
  LaunchCfg Ld = make_cfg<double>(d), Lf = make_cfg<float>(d);
  int np = std::max({Ld.grid_x, Ld.grid_ew, Lf.grid_x, Lf.grid_ew, 152 * 8 * 6});
  l.nparts = np;
  l.off_state = take(sizeof(SolverState) * 4);
  l.off_partials = take(sizeof(double) * 2 * (size_t)np);
  l.off_phase = take((size_t)d.V);
  l.off_scale = take(d.has_scale ? sizeof(float) * (size_t)d.V : 0);
  l.off_act = take(256);
  l.off_posx = take(sizeof(int) * d.nx);
  l.off_kofy = take(sizeof(int) * d.ny);
  l.off_kofz = take(sizeof(int) * d.nz);
  l.off_sums = take(sizeof(double) * 64);
  l.off_W = take(sizeof(double) * 64);
  l.off_tabd = take(sizeof(double) * 2 * 256 * 6);
  l.off_tabf = take(sizeof(float) * 2 * 256 * 6);
  l.off_tw_d = take(sizeof(double2) * (size_t)(d.nx + d.ny + d.nz));
  l.off_tw_f = take(sizeof(float2) * (size_t)(d.nx + d.ny + d.nz));
  for (int i = 0; i < 4; ++i) l.off_fd[i] = take(sizeof(double) * (size_t)n);
  l.off_Hd = take(sizeof(double2) * (size_t)(d.c * nf));
  l.off_gd = take(sizeof(double) * (size_t)(d.ncoef * nf));
  if (d.precision == LSH_MIXED) {
    for (int i = 0; i < 4; ++i) l.off_ff[i] = take(sizeof(float) * (size_t)n);
    l.off_Hf = take(sizeof(float2) * (size_t)(d.c * nf));
    l.off_gf = take(sizeof(float) * (size_t)(d.ncoef * nf));
  }
  l.total = o;
  return l;
}

}  // namespace

// ---------------------------------------------------------------- the handle
struct lsh_handle {
  Derived d;
  Layout lay;
  cudaStream_t stream;
  unsigned char* base;
  SolverState* st;  // [0] FP64 CG, [1] FP32 CG, [2] residual / scratch, [3] setup scan
  double* partials;
  unsigned char *phase, *act;
  float* scale;
  int *posx, *kofy, *kofz;
  double* sums;
  double* Wdev;
  double* tabd;  // mtab (256*6) then modtab (256*6)
  PrecBufs<double> pd;
  PrecBufs<float> pf;
  long long n_active;
  // diagnostics
  long long launches = 0;
  bool prof = false;
  std::vector<cudaEvent_t> ev;  // 7 per timed iteration
  int ev_used = 0;
  double pass_ms[6] = {0, 0, 0, 0, 0, 0};
  long long pass_n[6] = {0, 0, 0, 0, 0, 0};
  long long timed_iters = 0;
  ~lsh_handle() {
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
               size_t off_tab, SolverState* st) {
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
  P.st = st;
  P.L = make_cfg<T>(d);
  OpArgs<T>& a = P.a;
  a.nx = d.nx;
  a.ny = d.ny;
  a.nz = d.nz;
  a.nxh = d.nxh;
  a.c = d.c;
  a.V = d.V;
  a.nrows = d.c * d.nz * d.ny;
  a.lsx = d.nx | 1;
  a.lsy = d.ny | 1;
  a.lsz = d.nz | 1;
  a.RY = P.L.RY;
  a.TY = P.L.TY;
  a.TZ = P.L.TZ;
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
  a.act = h->act;
  a.mtab = P.mtab;
  a.modtab = P.modtab;
  for (int i = 0; i < 6; ++i) {
    a.ref[i] = (T)(i < d.c ? d.ref_in[i] : 0.0);
    a.load[i] = (T)0;
  }
}

// internal basis <-> Mandel for elasticity (see k_rotate)
void to_internal(const Derived& d, const double* m, double* out) {
  for (int i = 0; i < d.c; ++i) out[i] = m[i];
  if (d.physics == LSH_ELASTIC_ISO) {
    const double s3 = 1.0 / std::sqrt(3.0), s2 = 1.0 / std::sqrt(2.0), s6 = 1.0 / std::sqrt(6.0);
    out[0] = (m[0] + m[1] + m[2]) * s3;
    out[1] = (m[0] - m[1]) * s2;
    out[2] = (m[0] + m[1] - 2.0 * m[2]) * s6;
  }
}
void to_mandel(const Derived& d, const double* v, double* out) {
  for (int i = 0; i < d.c; ++i) out[i] = v[i];
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
    for (int i = 0; i < c; ++i) A0[i * c + i] = d.ref_user[i];
  }
}

lsh_status read_state(lsh_handle* h, int idx, SolverState* out) {
  LSH_CK(cudaMemcpyAsync(out, h->st + idx, sizeof(SolverState), cudaMemcpyDeviceToHost, h->stream));
  LSH_CK(cudaStreamSynchronize(h->stream));
  return LSH_OK;
}

// ---------------------------------------------------------------- operator sequences
// out = K in (both in the internal basis), precision T.
template <typename T> lsh_status apply_internal(lsh_handle* h, const T* in, T* out) {
  PrecBufs<T>& P = bufs<T>(h);
  cudaStream_t s = h->stream;
  launch_xfwd<T>(P.a, P.L, 0, in, nullptr, nullptr, nullptr, nullptr, s);
  launch_yfft<T>(P.a, P.L, false, nullptr, s);
  launch_zgamma<T>(P.a, P.L, nullptr, s);
  launch_yfft<T>(P.a, P.L, true, nullptr, s);
  launch_xinv<T>(P.a, P.L, 0, in, out, nullptr, nullptr, s);
  h->launches += 5;
  return last_launch();
}

// r = b - K x in FP64, (r, r) -> st[2].aux[0]
lsh_status residual64(lsh_handle* h, const double* load_in, const double* x, double* r) {
  PrecBufs<double>& P = h->pd;
  cudaStream_t s = h->stream;
  OpArgs<double> a = P.a;
  for (int i = 0; i < 6; ++i) a.load[i] = i < h->d.c ? load_in[i] : 0.0;
  launch_xfwd<double>(a, P.L, 0, x, nullptr, nullptr, nullptr, nullptr, s);
  launch_yfft<double>(a, P.L, false, nullptr, s);
  launch_zgamma<double>(a, P.L, nullptr, s);
  launch_yfft<double>(a, P.L, true, nullptr, s);
  launch_xinv<double>(a, P.L, 2, x, r, h->st + 2, h->partials, s);
  h->launches += 5;
  return last_launch();
}

template <typename T> void enqueue_cg_iteration(lsh_handle* h, PrecBufs<T>& P) {
  cudaStream_t s = h->stream;
  const bool timed = h->prof && h->ev_used + 7 <= (int)h->ev.size();
  cudaEvent_t* e = timed ? &h->ev[h->ev_used] : nullptr;
  if (timed) cudaEventRecord(e[0], s);
  launch_xfwd<T>(P.a, P.L, 1, nullptr, P.x, P.r, P.p, P.st, s);
  if (timed) cudaEventRecord(e[1], s);
  launch_yfft<T>(P.a, P.L, false, P.st, s);
  if (timed) cudaEventRecord(e[2], s);
  launch_zgamma<T>(P.a, P.L, P.st, s);
  if (timed) cudaEventRecord(e[3], s);
  launch_yfft<T>(P.a, P.L, true, P.st, s);
  if (timed) cudaEventRecord(e[4], s);
  launch_xinv<T>(P.a, P.L, 1, P.p, P.q, P.st, h->partials, s);
  if (timed) cudaEventRecord(e[5], s);
  launch_cg_update<T>(P.r, P.q, (long long)h->d.c * h->d.V, P.st, h->partials, P.L.grid_ew, s);
  if (timed) {
    cudaEventRecord(e[6], s);
    h->ev_used += 7;
  }
  h->launches += 6;
}

// After a host synchronisation: add the pass times of the first `real`
// recorded iterations (later ones returned at once because the solve was done).
void harvest_profile(lsh_handle* h, int real) {
  const int groups = h->ev_used / 7;
  for (int g = 0; g < groups && g < real; ++g) {
    for (int k = 0; k < 6; ++k) {
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

// CG on the state already begun in P.st; finalises x.  Returns the state.
template <typename T>
lsh_status cg_run(lsh_handle* h, PrecBufs<T>& P, int maxit, int check_every, SolverState* out) {
  int idx = (P.st == h->st) ? 0 : 1;
  lsh_status stt = read_state(h, idx, out);
  if (stt) return stt;
  int it = 0;
  while (!out->done && it < maxit) {
    const int chunk = std::min(check_every, maxit - it);
    const int before = out->iter;
    for (int j = 0; j < chunk; ++j) enqueue_cg_iteration<T>(h, P);
    if ((stt = last_launch())) return stt;
    it += chunk;
    if ((stt = read_state(h, idx, out))) return stt;
    if (h->prof) harvest_profile(h, out->iter - before);
  }
  launch_cg_finalize<T>(P.x, P.p, (long long)h->d.c * h->d.V, P.st, P.L.grid_ew, h->stream);
  h->launches += 1;
  if ((stt = last_launch())) return stt;
  return read_state(h, idx, out);
}

lsh_status solve_internal(lsh_handle* h, const double* load_in, bool warm, const lsh_solve_opts* o,
                          lsh_solve_info* info) {
  const Derived& d = h->d;
  const long long n = (long long)d.c * d.V;
  double tol = o && o->tol > 0 ? o->tol : 1e-10;
  int maxit = o && o->maxit > 0 ? o->maxit : 10000;
  int check = o && o->check_every > 0 ? o->check_every : 8;
  double lb = 0.0;
  for (int i = 0; i < d.c; ++i) lb += load_in[i] * load_in[i];
  const double bb = (double)h->n_active * lb;
  lsh_solve_info inf{};
  PrecBufs<double>& Pd = h->pd;
  lsh_status stt;
  if (d.precision == LSH_FP64) {
    if (!warm) {
      OpArgs<double> a = Pd.a;
      for (int i = 0; i < 6; ++i) a.load[i] = i < d.c ? load_in[i] : 0.0;
      launch_fill_rhs<double>(a, Pd.r, Pd.x, Pd.L.grid_ew, h->stream);
      launch_cg_begin<double>(Pd.r, n, Pd.st, h->partials, tol, -1.0, Pd.L.grid_ew, h->stream);
      h->launches += 2;
    } else {
      if ((stt = residual64(h, load_in, Pd.x, Pd.r))) return stt;
      inf.applies64 += 1;
      launch_cg_begin<double>(Pd.r, n, Pd.st, h->partials, tol, bb, Pd.L.grid_ew, h->stream);
      h->launches += 1;
    }
    if ((stt = last_launch())) return stt;
    SolverState s;
    if ((stt = cg_run<double>(h, Pd, maxit, check, &s))) return stt;
    inf.iters = s.iter;
    inf.applies64 += s.iter;
    inf.relres = s.bb > 0 ? std::sqrt(std::max(s.rr, 0.0) / s.bb) : 0.0;
    inf.status = s.status ? s.status : (s.done ? LSH_OK : LSH_ERR_NOT_CONVERGED);
  } else {
    // mixed precision: iterative refinement, FP64 residual, FP32 inner CG
    PrecBufs<float>& Pf = h->pf;
    const double itol = o && o->inner_tol > 0 ? o->inner_tol : 1e-4;
    const int max_outer = o && o->max_outer > 0 ? o->max_outer : 30;
    double rr;
    if (!warm) {
      OpArgs<double> a = Pd.a;
      for (int i = 0; i < 6; ++i) a.load[i] = i < d.c ? load_in[i] : 0.0;
      launch_fill_rhs<double>(a, Pd.r, Pd.x, Pd.L.grid_ew, h->stream);
      h->launches += 1;
      rr = bb;
    } else {
      if ((stt = residual64(h, load_in, Pd.x, Pd.r))) return stt;
      inf.applies64 += 1;
      SolverState s2;
      if ((stt = read_state(h, 2, &s2))) return stt;
      rr = s2.aux[0];
    }
    if ((stt = last_launch())) return stt;
    int total = 0, outer = 0, status = LSH_OK;
    double prev = rr;
    while (rr > tol * tol * bb) {
      if (outer >= max_outer || total >= maxit) { status = LSH_ERR_NOT_CONVERGED; break; }
      launch_d2f_begin(Pd.r, Pf.r, Pf.x, n, Pf.st, h->partials, itol, Pf.L.grid_ew, h->stream);
      h->launches += 1;
      SolverState s;
      if ((stt = cg_run<float>(h, Pf, maxit - total, check, &s))) return stt;
      total += s.iter;
      launch_f2d_axpy(Pd.x, Pf.x, n, Pd.L.grid_ew, h->stream);
      h->launches += 1;
      if ((stt = residual64(h, load_in, Pd.x, Pd.r))) return stt;
      inf.applies64 += 1;
      SolverState s2;
      if ((stt = read_state(h, 2, &s2))) return stt;
      rr = s2.aux[0];
      ++outer;
      if (s.status == LSH_ERR_BREAKDOWN && rr >= prev) { status = LSH_ERR_BREAKDOWN; break; }
      if (!(rr < prev) && s.iter == 0) { status = LSH_ERR_NOT_CONVERGED; break; }
      prev = rr;
    }
    inf.iters = total;
    inf.outer = outer;
    inf.relres = bb > 0 ? std::sqrt(std::max(rr, 0.0) / bb) : 0.0;
    inf.status = status;
  }
  if (info) *info = inf;
  return (lsh_status)inf.status;
}

lsh_status scan_microstructure(lsh_handle* h) {
  SolverState zero{};
  LSH_CK(cudaMemcpyAsync(h->st + 3, &zero, sizeof(zero), cudaMemcpyHostToDevice, h->stream));
  launch_scan_phase(h->phase, h->d.V, h->act, h->d.nphase, h->st + 3, h->partials,
                    (int)std::min<long long>((h->d.V + kThreads - 1) / kThreads, 152 * 8), h->stream);
  lsh_status stt = last_launch();
  if (stt) return stt;
  SolverState s;
  if ((stt = read_state(h, 3, &s))) return stt;
  if (s.pad >= h->d.nphase) return LSH_ERR_INVALID_ARG;
  h->n_active = (long long)s.aux[1];
  return LSH_OK;
}

lsh_status copy_microstructure(lsh_handle* h, const unsigned char* phase, const float* scale, int on_host) {
  const cudaMemcpyKind k = on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  LSH_CK(cudaMemcpyAsync(h->phase, phase, (size_t)h->d.V, k, h->stream));
  if (h->d.has_scale) {
    if (!scale) return LSH_ERR_INVALID_ARG;
    LSH_CK(cudaMemcpyAsync(h->scale, scale, sizeof(float) * (size_t)h->d.V, k, h->stream));
  }
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
  if (!cfg_fits<double>(make_cfg<double>(d)) || !cfg_fits<float>(make_cfg<float>(d)))
    return LSH_ERR_UNSUPPORTED_SIZE;
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
  if (!cfg_fits<double>(make_cfg<double>(d)) || !cfg_fits<float>(make_cfg<float>(d))) {
    delete h;
    return LSH_ERR_UNSUPPORTED_SIZE;
  }
  h->lay = make_layout(d);
  if (bytes < h->lay.total || ((uintptr_t)workspace % kAlign) != 0) { delete h; return LSH_ERR_WORKSPACE; }
  h->stream = (cudaStream_t)stream;
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
  h->sums = (double*)(h->base + l.off_sums);
  h->Wdev = (double*)(h->base + l.off_W);
  h->tabd = (double*)(h->base + l.off_tabd);
  init_prec<double>(h, h->pd, l.off_fd, l.off_Hd, l.off_gd, l.off_tw_d, l.off_tabd, h->st + 0);
  if (d.precision == LSH_MIXED) init_prec<float>(h, h->pf, l.off_ff, l.off_Hf, l.off_gf, l.off_tw_f, l.off_tabf, h->st + 1);

  // host tables
  std::vector<int> posx(d.nx), kofy(d.ny), kofz(d.nz);
  for (int k = 0; k < d.nx; ++k) posx[k] = dif_position(d.px, k);
  for (int k = 0; k < d.ny; ++k) kofy[dif_position(d.py, k)] = k;
  for (int k = 0; k < d.nz; ++k) kofz[dif_position(d.pz, k)] = k;
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
  SolverState zero[4] = {};
#define SETUP_CK(call) do { if ((call) != cudaSuccess) { cudaGetLastError(); delete h; return LSH_ERR_CUDA; } } while (0)
  SETUP_CK(cudaMemcpyAsync(h->st, zero, sizeof(zero), cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->act, d.act.data(), 256, cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->posx, posx.data(), sizeof(int) * d.nx, cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->kofy, kofy.data(), sizeof(int) * d.ny, cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->kofz, kofz.data(), sizeof(int) * d.nz, cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->base + l.off_tw_d, twd.data(), sizeof(double) * twd.size(), cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->base + l.off_tw_f, twf.data(), sizeof(float) * twf.size(), cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->base + l.off_tabd, tabd.data(), sizeof(double) * tabd.size(), cudaMemcpyHostToDevice, st));
  SETUP_CK(cudaMemcpyAsync(h->base + l.off_tabf, tabf.data(), sizeof(float) * tabf.size(), cudaMemcpyHostToDevice, st));
  if (copy_microstructure(h, prob->phase, prob->scale, prob->phase_on_host) != LSH_OK) { delete h; return LSH_ERR_CUDA; }
  set_smem_attrs<double>(h->pd.L);
  set_smem_attrs<float>(h->pf.L.threads ? h->pf.L : h->pd.L);
  launch_gamma_table<double>(h->pd.a, d.dim, d.physics, d.green, d.ref_user, h->kofy, h->kofz, st);
  if (d.precision == LSH_MIXED)
    launch_gamma_table<float>(h->pf.a, d.dim, d.physics, d.green, d.ref_user, h->kofy, h->kofz, st);
  if (last_launch() != LSH_OK) { delete h; return LSH_ERR_CUDA; }
  s = scan_microstructure(h);  // synchronises the stream (host vectors may go)
  if (s) { delete h; return s; }
#undef SETUP_CK
  *out = h;
  return LSH_OK;
}

lsh_status lsh_set_microstructure(lsh_handle* h, const unsigned char* phase, const float* scale, int on_host) {
  if (!h || !phase) return LSH_ERR_INVALID_ARG;
  lsh_status s = copy_microstructure(h, phase, scale, on_host);
  if (s) return s;
  return scan_microstructure(h);
}

lsh_status lsh_apply(lsh_handle* h, int dtype, const void* x, void* y) {
  if (!h || !x || !y) return LSH_ERR_INVALID_ARG;
  const Derived& d = h->d;
  const bool el = d.physics == LSH_ELASTIC_ISO;
  const int grid = h->pd.L.grid_ew;
  if (dtype == LSH_F64) {
    PrecBufs<double>& P = h->pd;
    const double* in = (const double*)x;
    if (el) {
      launch_rotate<double>(in, P.p, d.V, 1, grid, h->stream);
      in = P.p;
    }
    lsh_status s = apply_internal<double>(h, in, el ? P.q : (double*)y);
    if (s) return s;
    if (el) launch_rotate<double>(P.q, (double*)y, d.V, 0, grid, h->stream);
  } else if (dtype == LSH_F32) {
    if (d.precision != LSH_MIXED) return LSH_ERR_UNSUPPORTED;
    PrecBufs<float>& P = h->pf;
    const float* in = (const float*)x;
    if (el) {
      launch_rotate<float>(in, P.p, d.V, 1, grid, h->stream);
      in = P.p;
    }
    lsh_status s = apply_internal<float>(h, in, el ? P.q : (float*)y);
    if (s) return s;
    if (el) launch_rotate<float>(P.q, (float*)y, d.V, 0, grid, h->stream);
  } else {
    return LSH_ERR_INVALID_ARG;
  }
  return last_launch();
}

lsh_status lsh_solve(lsh_handle* h, const double* load, double* tau, const lsh_solve_opts* opts,
                     lsh_solve_info* info) {
  if (!h || !load || !tau) return LSH_ERR_INVALID_ARG;
  const Derived& d = h->d;
  double lin[6];
  to_internal(d, load, lin);
  const bool warm = opts && opts->warm_start;
  const int grid = h->pd.L.grid_ew;
  if (warm) {
    if (d.physics == LSH_ELASTIC_ISO) launch_rotate<double>(tau, h->pd.x, d.V, 1, grid, h->stream);
    else if (cudaMemcpyAsync(h->pd.x, tau, sizeof(double) * d.c * d.V, cudaMemcpyDeviceToDevice, h->stream))
      return LSH_ERR_CUDA;
  }
  lsh_status s = solve_internal(h, lin, warm, opts, info);
  if (s != LSH_OK && s != LSH_ERR_NOT_CONVERGED && s != LSH_ERR_BREAKDOWN) return s;
  if (d.physics == LSH_ELASTIC_ISO) launch_rotate<double>(h->pd.x, tau, d.V, 0, grid, h->stream);
  else if (cudaMemcpyAsync(tau, h->pd.x, sizeof(double) * d.c * d.V, cudaMemcpyDeviceToDevice, h->stream))
    return LSH_ERR_CUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LSH_ERR_CUDA;
  return s;
}

lsh_status lsh_effective(lsh_handle* h, const lsh_solve_opts* opts, double* Astar, double* tau_all,
                         lsh_solve_info* infos) {
  if (!h || !Astar) return LSH_ERR_INVALID_ARG;
  const Derived& d = h->d;
  const int c = d.c;
  double A0[36];
  ref_matrix(d, A0);
  const int nblk = 152;
  lsh_status worst = LSH_OK;
  for (int j = 0; j < c; ++j) {
    double e[6] = {0, 0, 0, 0, 0, 0}, lin[6];
    e[j] = 1.0;
    to_internal(d, e, lin);
    lsh_solve_info inf{};
    lsh_solve_opts o = opts ? *opts : lsh_solve_opts{};
    o.warm_start = 0;
    lsh_status s = solve_internal(h, lin, false, &o, &inf);
    if (infos) infos[j] = inf;
    if (s != LSH_OK && s != LSH_ERR_NOT_CONVERGED && s != LSH_ERR_BREAKDOWN) return s;
    if (s != LSH_OK && worst == LSH_OK) worst = s;
    // A*_h e_j = A0 e_j + h^d sum_beta tau_beta (Eq. (tau_Astar), Theorem 13)
    launch_comp_sums<double>(h->pd.x, c, d.V, h->partials, nblk, h->sums, h->stream);
    h->launches += 2;
    if (tau_all) {
      double* dst = tau_all + (long long)j * c * d.V;
      if (d.physics == LSH_ELASTIC_ISO) launch_rotate<double>(h->pd.x, dst, d.V, 0, h->pd.L.grid_ew, h->stream);
      else if (cudaMemcpyAsync(dst, h->pd.x, sizeof(double) * c * d.V, cudaMemcpyDeviceToDevice, h->stream))
        return LSH_ERR_CUDA;
    }
    double sums[6], mean[6], meanM[6];
    LSH_CK(cudaMemcpyAsync(sums, h->sums, sizeof(double) * c, cudaMemcpyDeviceToHost, h->stream));
    LSH_CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < c; ++i) mean[i] = sums[i] / (double)d.V;
    to_mandel(d, mean, meanM);
    for (int i = 0; i < c; ++i) Astar[i * c + j] = A0[i * c + j] + meanM[i];
  }
  return worst;
}

lsh_status lsh_effective_grad(lsh_handle* h, const double* tau_all, const double* W, double* grad) {
  if (!h || !tau_all || !W || !grad) return LSH_ERR_INVALID_ARG;
  const Derived& d = h->d;
  LSH_CK(cudaMemcpyAsync(h->Wdev, W, sizeof(double) * d.c * d.c, cudaMemcpyHostToDevice, h->stream));
  double refd[6];
  for (int i = 0; i < 6; ++i) refd[i] = i < d.c ? d.ref_in[i] : 0.0;
  LSH_CK(cudaMemcpyAsync(h->Wdev + 40, refd, sizeof(refd), cudaMemcpyHostToDevice, h->stream));
  launch_scale_grad(tau_all, h->Wdev, h->phase, h->scale, h->tabd + 256 * 6, h->Wdev + 40, d.c,
                    d.physics == LSH_ELASTIC_ISO, d.V, grad,
                    (int)std::min<long long>((d.V + 127) / 128, 152 * 16), h->stream);
  lsh_status s = last_launch();
  if (s) return s;
  // the host arrays above are stack memory: finish the copies before returning
  LSH_CK(cudaStreamSynchronize(h->stream));
  return LSH_OK;
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
  h->ev_used = 0;
  return LSH_OK;
}

lsh_status lsh_profile_read(lsh_handle* h, lsh_profile* out, int reset) {
  if (!h || !out) return LSH_ERR_INVALID_ARG;
  out->launches = h->launches;
  out->timed_iters = h->timed_iters;
  for (int k = 0; k < 6; ++k) {
    out->pass_ms[k] = h->pass_ms[k];
    out->pass_launches[k] = h->pass_n[k];
  }
  if (reset) {
    h->launches = 0;
    h->timed_iters = 0;
    for (int k = 0; k < 6; ++k) {
      h->pass_ms[k] = 0.0;
      h->pass_n[k] = 0;
    }
  }
  return LSH_OK;
}

void lsh_destroy(lsh_handle* h) { delete h; }

}  // extern "C"
