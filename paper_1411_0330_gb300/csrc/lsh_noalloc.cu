// lsh_noalloc.cu -- lsh_apply_noalloc: the operator application of lsh_apply
// with all of its scratch in a fixed array that is part of the library image.
//
// Who needs this: code that may not call cudaMalloc (or any allocator) at the
// point where it wants K x.  Typical cases are plugins loaded into a host
// program that owns the device memory and hands out no allocator, processes
// whose device memory is already fully claimed by another framework's pool,
// and code paths that must not risk the implicit device synchronisation that
// cudaMalloc / cudaFree can cause.  Such callers pass only their input and
// output fields; the spectrum, the Green-operator table, the twiddles and the
// per-phase tables live in `g_lsh_noalloc_scratch` below.
//
// The array is a file-scope __device__ variable: every device that loads the
// library holds its 72 MiB until the process exits (enough for 64^3 elasticity:
// two rotated fields, the spectrum and the padded Gamma table take 69.6 MB).
// Host code cannot use the symbol as a device address (it is a host-side
// stand-in), so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current and caches it.  The cache
// is not revalidated: after cudaDeviceReset the module may load elsewhere, so
// a process that resets a device must not call this entry point on it again.
// A call copies host tables and synchronises its stream, neither of which a
// capturing stream allows: calls on a stream under capture are refused.  The
// host side here allocates nothing either: plans and per-phase tables live in
// fixed-size structures, the FFT tables are computed on the device.
//
// All calls share the one array and keep the last call's contents.  Nothing
// in it needs to start at zero (every buffer is fully written before it is
// read), but calls whose device work overlaps (different streams, or several
// host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "internal.h"
#include "lsh.h"

using namespace lsh;

#define LSH_NOALLOC_SCRATCH_BYTES (72ull << 20)

static __device__ __align__(256) unsigned char g_lsh_noalloc_scratch[LSH_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
lsh_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return LSH_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_lsh_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return LSH_ERR_CUDA;
    }
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return LSH_OK;
}

bool plan_axis(int n, Plan1D* p) {
  int r[LSH_MAX_STAGES * 4];
  int k = 0, m = n;
  while (m % 8 == 0 && k < 32) { r[k++] = 8; m /= 8; }
  if (m % 4 == 0) { r[k++] = 4; m /= 4; }
  if (m % 2 == 0) {
    bool swapped = false;
    for (int i = 0; i < k; ++i)
      if (r[i] == 8) { r[i] = 4; r[k++] = 4; swapped = true; break; }
    if (!swapped) r[k++] = 2;
    m /= 2;
  }
  const int qs[3] = {3, 5, 7};
  for (int qi = 0; qi < 3; ++qi)
    while (m % qs[qi] == 0 && k < 32) { r[k++] = qs[qi]; m /= qs[qi]; }
  if (m != 1 || k > LSH_MAX_STAGES) return false;
  p->n = n;
  p->nst = k;
  for (int i = 0; i < k; ++i) p->radix[i] = r[i];
  return true;
}

// Twiddles exp(-2 i pi t / n), DIF positions of x frequencies, frequencies of
// y / z positions: one thread per table entry.
__global__ void k_noalloc_tables(Plan1D px, Plan1D py, Plan1D pz, double2* tw, int* posx, int* kofy, int* kofz) {
  const int nx = px.n, ny = py.n, nz = pz.n;
  const int total = nx + ny + nz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const Plan1D& p = i < nx ? px : (i < nx + ny ? py : pz);
    const int k = i < nx ? i : (i < nx + ny ? i - nx : i - nx - ny);
    double s, c;
    sincospi(2.0 * (double)k / (double)p.n, &s, &c);
    tw[i] = make_double2(c, -s);
    int pos = 0, kk = k, L = p.n;
    for (int st = 0; st < p.nst; ++st) {
      const int r = p.radix[st], m = L / r;
      pos += (kk % r) * m;
      kk /= r;
      L = m;
    }
    if (i < nx) posx[k] = pos;
    else if (i < nx + ny) kofy[pos] = k;
    else kofz[pos] = k;
  }
}

size_t up(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" lsh_status lsh_apply_noalloc(const lsh_problem* pr, const double* x, double* y, void* stream) {
  if (!pr || !x || !y || !pr->phase || !pr->phase_moduli) return LSH_ERR_INVALID_ARG;
  if (pr->phase_on_host || pr->nbatch > 1) return LSH_ERR_INVALID_ARG;
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) {
      cudaGetLastError();
      return LSH_ERR_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return LSH_ERR_INVALID_ARG;  // host copies and a synchronisation follow
  }
  if (pr->dim != 2 && pr->dim != 3) return LSH_ERR_INVALID_ARG;
  if (pr->physics != LSH_SCALAR && pr->physics != LSH_ELASTIC_ISO) return LSH_ERR_INVALID_ARG;
  if (pr->physics == LSH_ELASTIC_ISO && pr->dim != 3) return LSH_ERR_INVALID_ARG;
  if (pr->green != LSH_GREEN_TRUNCATED && pr->green != LSH_GREEN_FILTERED && pr->green != LSH_GREEN_FD)
    return LSH_ERR_INVALID_ARG;
  if (pr->green == LSH_GREEN_FD && pr->physics != LSH_SCALAR) return LSH_ERR_UNSUPPORTED;
  if (pr->scale && pr->scale_kind != 0) return LSH_ERR_UNSUPPORTED;
  if (pr->nphase < 1 || pr->nphase > 256) return LSH_ERR_INVALID_ARG;
  if (pr->scale && !pr->ref_moduli) return LSH_ERR_INVALID_ARG;
  const int dim = pr->dim, nx = pr->n[0], ny = pr->n[1], nz = dim == 3 ? pr->n[2] : 1;
  if (nx < 1 || ny < 1 || nz < 1) return LSH_ERR_INVALID_ARG;
  const bool el = pr->physics == LSH_ELASTIC_ISO;
  const int c = el ? 6 : dim, ncoef = c * (c + 1) / 2, nxh = nx / 2 + 1;
  const long long V = (long long)nx * ny * nz;
  Plan1D px, py, pz;
  if (!plan_axis(nx, &px) || !plan_axis(ny, &py) || !plan_axis(nz, &pz)) return LSH_ERR_UNSUPPORTED_SIZE;

  // reference medium and per-phase diagonal tables in the internal basis
  double ref_user[6] = {0, 0, 0, 0, 0, 0}, ref_in[6] = {0, 0, 0, 0, 0, 0};
  if (el) {
    double K0, mu0;
    if (pr->ref_moduli) {
      K0 = pr->ref_moduli[0];
      mu0 = pr->ref_moduli[1];
    } else {
      double mumin = pr->phase_moduli[1];
      for (int ph = 1; ph < pr->nphase; ++ph) mumin = std::min(mumin, pr->phase_moduli[2 * ph + 1]);
      mu0 = 0.5 * mumin;
      K0 = 2.0 * mu0 * 1.3 / (3.0 * 0.4);  // nu0 = 0.3
    }
    if (!(K0 > 0.0) || !(mu0 > 0.0)) return LSH_ERR_REFERENCE_INDEFINITE;
    ref_user[0] = K0;
    ref_user[1] = mu0;
    ref_in[0] = 3.0 * K0;
    for (int i = 1; i < 6; ++i) ref_in[i] = 2.0 * mu0;
  } else {
    for (int ph = 0; ph < pr->nphase; ++ph)
      for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j)
          if (i != j && pr->phase_moduli[ph * dim * dim + i * dim + j] != 0.0) return LSH_ERR_UNSUPPORTED;
    double amin = pr->phase_moduli[0];
    for (int ph = 0; ph < pr->nphase; ++ph)
      for (int i = 0; i < dim; ++i) amin = std::min(amin, pr->phase_moduli[ph * dim * dim + i * dim + i]);
    for (int i = 0; i < dim; ++i) {
      if (pr->ref_moduli)
        for (int j = 0; j < dim; ++j)
          if (i != j && pr->ref_moduli[i * dim + j] != 0.0) return LSH_ERR_UNSUPPORTED;
      ref_in[i] = pr->ref_moduli ? pr->ref_moduli[i * dim + i] : 0.5 * amin;
      if (!(ref_in[i] > 0.0)) return LSH_ERR_REFERENCE_INDEFINITE;
      ref_user[i] = ref_in[i];
    }
  }
  struct Tables {
    unsigned char act[256];
    double mtab[256 * 6];
    double modtab[256 * 6];
  };
  static thread_local Tables tab;  // host, fixed size
  for (int i = 0; i < 256; ++i) tab.act[i] = 0;
  for (int i = 0; i < 256 * 6; ++i) tab.mtab[i] = tab.modtab[i] = 0.0;
  for (int ph = 0; ph < pr->nphase; ++ph) {
    double* md = &tab.modtab[ph * c];
    if (el) {
      md[0] = 3.0 * pr->phase_moduli[2 * ph];
      for (int i = 1; i < 6; ++i) md[i] = 2.0 * pr->phase_moduli[2 * ph + 1];
    } else {
      for (int i = 0; i < dim; ++i) md[i] = pr->phase_moduli[ph * dim * dim + i * dim + i];
    }
    if (pr->scale) {
      tab.act[ph] = 1;
      continue;
    }
    bool any = false, allnz = true;
    for (int i = 0; i < c; ++i) {
      if (md[i] - ref_in[i] != 0.0) any = true;
      else allnz = false;
    }
    if (!any) continue;
    if (!allnz) return LSH_ERR_SINGULAR_CONTRAST;
    tab.act[ph] = 1;
    for (int i = 0; i < c; ++i) tab.mtab[ph * c + i] = 1.0 / (md[i] - ref_in[i]);
  }

  // tile shapes (same rules as the workspace path, one system)
  const size_t cs = sizeof(double2);
  const int lsx = nx | 1, lsy = ny | 1, lsz = nz | 1, rps = c * nz * ny;
  int RY = std::max(2, 2 * (int)(32768 / (lsx * cs)));
  RY = std::min(RY, std::max(2, rps / 608));
  if (RY >= rps) {
    RY = rps;
  } else {
    int best = 1, pick = 0;
    for (int dv = RY; dv >= 1 && !pick; --dv)
      if (rps % dv == 0) {
        if (dv % 2 == 0) pick = dv;
        else if (best == 1) best = dv;
      }
    RY = pick ? pick : best;
  }
  LaunchCfg L{};
  L.threads = 256;
  L.RY = RY;
  L.VEC = (nx % 2 == 0) ? 2 : 1;
  L.smem_x = nx * cs + (size_t)((RY + 1) / 2) * lsx * cs + nx * sizeof(int);
  L.TY = std::min(8, nxh);
  L.smem_y = ny * cs + (size_t)L.TY * lsy * cs;
  int TZ = std::min(8, nxh);
  while (TZ > 1 && (size_t)c * TZ * lsz * cs > 100 * 1024) TZ /= 2;
  L.TZ = TZ;
  L.smem_z = nz * cs + (size_t)c * TZ * lsz * cs;
  L.grid_x = rps / RY;
  L.grid_yx = (nxh + L.TY - 1) / L.TY;
  L.grid_yy = c * nz;
  L.grid_zx = (nxh + TZ - 1) / TZ;
  L.grid_zy = ny;
  const size_t kMax = 227 * 1024;
  if (L.smem_x > kMax || L.smem_y > kMax || L.smem_z > kMax || ny > 65535 || (long long)c * nz > 65535)
    return LSH_ERR_UNSUPPORTED_SIZE;

  // scratch layout
  const long long nf = (long long)nz * ny * nxh;
  size_t o = 0;
  const size_t o_act = o; o = up(o + 256);
  const size_t o_mtab = o; o = up(o + sizeof(double) * 256 * 6);
  const size_t o_modtab = o; o = up(o + sizeof(double) * 256 * 6);
  const size_t o_posx = o; o = up(o + sizeof(int) * nx);
  const size_t o_kofy = o; o = up(o + sizeof(int) * ny);
  const size_t o_kofz = o; o = up(o + sizeof(int) * nz);
  const size_t o_tw = o; o = up(o + sizeof(double2) * (size_t)(nx + ny + nz));
  const size_t o_p = o; o = up(o + (el ? sizeof(double) * (size_t)(c * V) : 0));
  const size_t o_q = o; o = up(o + (el ? sizeof(double) * (size_t)(c * V) : 0));
  const size_t o_H = o; o = up(o + sizeof(double2) * (size_t)(c * nf));
  const long long ntf = (long long)nz * ny * ((nxh + 7) & ~7);  // Gamma table rows padded to 8
  const size_t o_g = o; o = up(o + sizeof(double) * (size_t)(((ncoef + 3) & ~3) * ntf));
  if (o > LSH_NOALLOC_SCRATCH_BYTES) return LSH_ERR_UNSUPPORTED_SIZE;

  void* base_v = nullptr;
  lsh_status st = scratch_address(&base_v);
  if (st) return st;
  unsigned char* base = (unsigned char*)base_v;
  cudaStream_t s = (cudaStream_t)stream;

  OpArgs<double> a{};
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.nxh = nxh;
  a.hs = nxh;
  a.ts = (nxh + 7) & ~7;
  a.fdphase = pr->green == LSH_GREEN_FD ? 1 : 0;
  a.kofy = (const int*)(base + o_kofy);  // frequency of each y / z position (phase rotations)
  a.kofz = (const int*)(base + o_kofz);
  a.c = c;
  a.V = V;
  a.S = 1;
  a.sys0 = 0;
  a.sys_per_ms = 1;
  a.rps = rps;
  a.RY = RY;
  a.bps = rps / RY;
  a.TY = L.TY;
  a.TZ = L.TZ;
  a.lsx = lsx;
  a.lsy = lsy;
  a.lsz = lsz;
  a.px = px;
  a.py = py;
  a.pz = pz;
  a.twx = (const double2*)(base + o_tw);
  a.twy = a.twx + nx;
  a.twz = a.twy + ny;
  a.posx = (const int*)(base + o_posx);
  a.H = (double2*)(base + o_H);
  a.gtab = (const double*)(base + o_g);
  a.ncoef = ncoef;
  a.phase = pr->phase;
  a.scale = pr->scale;
  a.act = base + o_act;
  a.nphase = pr->nphase;
  a.mtab = (const double*)(base + o_mtab);
  a.modtab = (const double*)(base + o_modtab);
  for (int i = 0; i < 6; ++i) a.ref[i] = i < c ? ref_in[i] : 0.0;
  a.loads = nullptr;

  if (cudaMemcpyAsync(base + o_act, tab.act, 256, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + o_mtab, tab.mtab, sizeof(tab.mtab), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + o_modtab, tab.modtab, sizeof(tab.modtab), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return LSH_ERR_CUDA;
  }
  set_smem_attrs<double>();
  const int ntab = nx + ny + nz;
  k_noalloc_tables<<<(ntab + 255) / 256, 256, 0, s>>>(px, py, pz, (double2*)(base + o_tw), (int*)(base + o_posx),
                                                       (int*)(base + o_kofy), (int*)(base + o_kofz));
  launch_gamma_table<double>(a, dim, pr->physics, pr->green, ref_user, (const int*)(base + o_kofy),
                             (const int*)(base + o_kofz), s);
  const double* in = x;
  double* out = y;
  if (el) {
    launch_rotate<double>(x, (double*)(base + o_p), V, 1, 1, s);
    in = (const double*)(base + o_p);
    out = (double*)(base + o_q);
  }
  launch_xfwd<double>(a, L, 0, in, nullptr, nullptr, nullptr, nullptr, s);
  launch_yfft<double>(a, L, false, nullptr, s);
  launch_zgamma<double>(a, L, nullptr, s);
  launch_yfft<double>(a, L, true, nullptr, s);
  launch_xinv<double>(a, L, 0, in, out, nullptr, nullptr, s);
  if (el) launch_rotate<double>(out, y, V, 1, 0, s);
  // the host tables above are copied from pageable memory, which the runtime
  // stages before returning; synchronising keeps the call's contract simple
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return LSH_ERR_CUDA;
  return LSH_OK;
}
