// kernels.cu -- the operator passes and CG kernels of liblsh (sm_103a).
//
// One application of the Lippmann-Schwinger operator of Eq. (13),
//   K x = P (M x + DFT^{-1}[Gamma^h_k DFT(x)_k]),
// is five passes over a half spectrum H[c][nz][ny][nx/2+1]:
//   xfwd   rows along x: two real rows packed as one complex line, DIF, split
//          into the two Hermitian half rows (fused CG prologue p = r + beta p,
//          x += alpha p_old);
//   yfft   columns along y, DIF (forward) or DIT (inverse), in place;
//   zgamma lines along z for all c components at once: DIF, the per-frequency
//          product with the tabulated Gamma^h_k (Sec. 3.2), DIT;
//   xinv   rows along x: rebuild the packed line, DIT, fused local term
//          M_beta x_beta (Eq. (7)), projection on I0 and the CG inner product.
// Fields use an internal component basis in which M_beta is diagonal (for
// isotropic elasticity: hydrostatic, two deviatoric normal and three shear
// Mandel components), so every component plane is independent outside zgamma.
#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

#include <algorithm>

namespace lsh {

static constexpr int kThreads = 256;

// Local coefficient m = (A_beta - A0)^{-1} of component `comp` at voxel `vox`.
template <typename T>
__device__ __forceinline__ T local_coef(const OpArgs<T>& a, long long vox, int comp, int* active) {
  const int ph = a.phase[vox];
  *active = a.act[ph];
  if (a.scale == nullptr) return a.mtab[ph * a.c + comp];
  const T s = (T)a.scale[vox];
  return (T)1 / (s * a.modtab[ph * a.c + comp] - a.ref[comp]);
}

// ------------------------------------------------------------------ x forward
// MODE 0: input field `in`, masked by I0.  MODE 1: CG prologue.
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_xfwd(OpArgs<T> a, const T* __restrict__ in, T* x, const T* r, T* p,
                                                   const SolverState* st) {
  if (MODE == 1 && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* Z = tw + a.nx;
  int* pos = reinterpret_cast<int*>(Z + (a.RY >> 1) * a.lsx);
  const int nx = a.nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    tw[i] = a.twx[i];
    pos[i] = a.posx[i];
  }
  const int row0 = blockIdx.x * a.RY;
  const int nr = min(a.RY, a.nrows - row0);
  const int npair = (nr + 1) >> 1;
  const int rows_per_comp = a.nz * a.ny;
  T alpha = 0, beta = 0;
  int k = 0;
  if (MODE == 1) {
    k = st->iter;
    alpha = (T)st->alpha;
    beta = (T)st->beta;
  }
  const long long gbase = (long long)row0 * nx;
  for (int idx = threadIdx.x; idx < nr * nx; idx += blockDim.x) {
    const int row = idx / nx, xx = idx - row * nx;
    const long long g = gbase + idx;
    T v;
    if (MODE == 0) {
      const int comp = (row0 + row) / rows_per_comp;
      const long long vox = g - (long long)comp * a.V;
      v = a.act[a.phase[vox]] ? in[g] : (T)0;
    } else {
      if (k == 0) {
        v = r[g];
        p[g] = v;
      } else {
        const T po = p[g];
        x[g] += alpha * po;
        v = r[g] + beta * po;
        p[g] = v;
      }
    }
    C2<T>* zc = Z + (row >> 1) * a.lsx + xx;
    if (row & 1) zc->y = v;
    else zc->x = v;
  }
  if (nr & 1)
    for (int xx = threadIdx.x; xx < nx; xx += blockDim.x) Z[(nr >> 1) * a.lsx + xx].y = (T)0;
  __syncthreads();
  fft_lines<T, false>(Z, npair, a.lsx, a.px, tw);
  // split Z = X_a + i X_b into the two Hermitian half rows
  const T h = (T)0.5;
  for (int idx = threadIdx.x; idx < npair * a.nxh; idx += blockDim.x) {
    const int lp = idx / a.nxh, kx = idx - lp * a.nxh;
    const C2<T> z1 = Z[lp * a.lsx + pos[kx]];
    const C2<T> z2 = Z[lp * a.lsx + pos[kx == 0 ? 0 : nx - kx]];
    const long long hrow = row0 + 2 * lp;
    a.H[hrow * a.nxh + kx] = mkc<T>(h * (z1.x + z2.x), h * (z1.y - z2.y));
    if (2 * lp + 1 < nr) a.H[(hrow + 1) * a.nxh + kx] = mkc<T>(h * (z1.y + z2.y), h * (z2.x - z1.x));
  }
}

// ------------------------------------------------------------------ y pass
template <typename T, bool INV>
__global__ void __launch_bounds__(kThreads) k_yfft(OpArgs<T> a, const SolverState* st) {
  if (st != nullptr && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf = tw + a.ny;
  for (int i = threadIdx.x; i < a.ny; i += blockDim.x) tw[i] = a.twy[i];
  const long long plane = blockIdx.y;
  const int kx0 = blockIdx.x * a.TY;
  const int nt = min(a.TY, a.nxh - kx0);
  C2<T>* Hp = a.H + plane * a.ny * a.nxh + kx0;
  for (int idx = threadIdx.x; idx < a.ny * a.TY; idx += blockDim.x) {
    const int y = idx / a.TY, t = idx - y * a.TY;
    if (t < nt) buf[t * a.lsy + y] = Hp[(long long)y * a.nxh + t];
  }
  __syncthreads();
  fft_lines<T, INV>(buf, nt, a.lsy, a.py, tw);
  for (int idx = threadIdx.x; idx < a.ny * a.TY; idx += blockDim.x) {
    const int y = idx / a.TY, t = idx - y * a.TY;
    if (t < nt) Hp[(long long)y * a.nxh + t] = buf[t * a.lsy + y];
  }
}

// ------------------------------------------------------------------ z pass + Gamma
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads) k_zgamma(OpArgs<T> a, const SolverState* st) {
  if (st != nullptr && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf = tw + a.nz;
  for (int i = threadIdx.x; i < a.nz; i += blockDim.x) tw[i] = a.twz[i];
  const int yp = blockIdx.y;
  const int kx0 = blockIdx.x * a.TZ;
  const int nt = min(a.TZ, a.nxh - kx0);
  const int c = NC, nz = a.nz, TZ = a.TZ;
  const long long zstride = (long long)a.ny * a.nxh;  // distance between z planes
  const long long cstride = zstride * nz;
  C2<T>* Hp = a.H + (long long)yp * a.nxh + kx0;
  for (int idx = threadIdx.x; idx < c * nz * TZ; idx += blockDim.x) {
    const int t = idx % TZ, rest = idx / TZ;
    const int z = rest % nz, comp = rest / nz;
    C2<T> v = mkc<T>(0, 0);
    if (t < nt) v = Hp[comp * cstride + z * zstride + t];
    buf[(comp * TZ + t) * a.lsz + z] = v;
  }
  __syncthreads();
  if (nz > 1) fft_lines<T, false>(buf, c * TZ, a.lsz, a.pz, tw);
  // per-frequency product with the symmetric c x c table (packed upper triangle)
  const T* G = a.gtab + (long long)yp * a.nxh + kx0;
  const long long gstride = cstride;  // table has the same [nz][ny][nxh] layout per coefficient
  for (int idx = threadIdx.x; idx < nz * TZ; idx += blockDim.x) {
    const int t = idx % TZ, zp = idx / TZ;
    if (t >= nt) continue;
    C2<T> v[NC], y[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      v[i] = buf[(i * TZ + t) * a.lsz + zp];
      y[i] = mkc<T>(0, 0);
    }
    int coef = 0;
#pragma unroll
    for (int i = 0; i < NC; ++i)
#pragma unroll
      for (int j = i; j < NC; ++j, ++coef) {
        const T g = G[coef * gstride + zp * zstride + t];
        y[i].x += g * v[j].x;
        y[i].y += g * v[j].y;
        if (j != i) {
          y[j].x += g * v[i].x;
          y[j].y += g * v[i].y;
        }
      }
#pragma unroll
    for (int i = 0; i < NC; ++i) buf[(i * TZ + t) * a.lsz + zp] = y[i];
  }
  __syncthreads();
  if (nz > 1) fft_lines<T, true>(buf, c * TZ, a.lsz, a.pz, tw);
  for (int idx = threadIdx.x; idx < c * nz * TZ; idx += blockDim.x) {
    const int t = idx % TZ, rest = idx / TZ;
    const int z = rest % nz, comp = rest / nz;
    if (t < nt) Hp[comp * cstride + z * zstride + t] = buf[(comp * TZ + t) * a.lsz + z];
  }
}

// ------------------------------------------------------------------ x inverse + local term
// MODE 0: out = P (M xin + g).  MODE 1 (CG): q = P (M p + g), (p, q) -> alpha.
// MODE 2 (residual): out = P (load - M xin - g), (r, r) -> st->aux[0].
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_xinv(OpArgs<T> a, const T* __restrict__ xin, T* __restrict__ out,
                                                   SolverState* st, double* partials) {
  if (MODE == 1 && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* Z = tw + a.nx;
  int* pos = reinterpret_cast<int*>(Z + (a.RY >> 1) * a.lsx);
  const int nx = a.nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    tw[i] = a.twx[i];
    pos[i] = a.posx[i];
  }
  __syncthreads();
  const int row0 = blockIdx.x * a.RY;
  const int nr = min(a.RY, a.nrows - row0);
  const int npair = (nr + 1) >> 1;
  // Z = X_a + i X_b over the full line, X(nx - k) = conj X(k) beyond the half
  for (int idx = threadIdx.x; idx < npair * a.nxh; idx += blockDim.x) {
    const int lp = idx / a.nxh, kx = idx - lp * a.nxh;
    const long long hrow = row0 + 2 * lp;
    const C2<T> xa = a.H[hrow * a.nxh + kx];
    const C2<T> xb = (2 * lp + 1 < nr) ? a.H[(hrow + 1) * a.nxh + kx] : mkc<T>(0, 0);
    Z[lp * a.lsx + pos[kx]] = mkc<T>(xa.x - xb.y, xa.y + xb.x);
    if (kx >= 1 && kx <= nx - a.nxh) Z[lp * a.lsx + pos[nx - kx]] = mkc<T>(xa.x + xb.y, xb.x - xa.y);
  }
  __syncthreads();
  fft_lines<T, true>(Z, npair, a.lsx, a.px, tw);
  const int rows_per_comp = a.nz * a.ny;
  const long long gbase = (long long)row0 * nx;
  double acc = 0.0;
  for (int idx = threadIdx.x; idx < nr * nx; idx += blockDim.x) {
    const int row = idx / nx, xx = idx - row * nx;
    const long long g = gbase + idx;
    const C2<T> zc = Z[(row >> 1) * a.lsx + xx];
    const T gv = (row & 1) ? zc.y : zc.x;
    const int comp = (row0 + row) / rows_per_comp;
    const long long vox = g - (long long)comp * a.V;
    int active;
    const T m = local_coef(a, vox, comp, &active);
    const T xv = xin[g];
    if (MODE == 0) {
      out[g] = active ? m * xv + gv : (T)0;
    } else if (MODE == 1) {
      const T qv = active ? m * xv + gv : (T)0;
      out[g] = qv;
      acc += (double)xv * (double)qv;
    } else {
      const T rv = active ? a.load[comp] - (m * xv + gv) : (T)0;
      out[g] = rv;
      acc += (double)rv * (double)rv;
    }
  }
  if (MODE != 0) {
    acc = block_sum(acc);
    if (publish_partial(partials, acc, &st->counter[0])) {
      const double tot = gather_partials(partials, &st->counter[0]);
      if (threadIdx.x == 0) {
        if (MODE == 1) {
          st->pq = tot;
          if (!(fabs(tot) > 0.0) || !isfinite(tot) || !isfinite(st->rr)) {
            st->status = 5;  // LSH_ERR_BREAKDOWN
            st->alpha = 0.0;
            st->done = 1;
          } else {
            st->alpha = st->rr / tot;
          }
        } else {
          st->aux[0] = tot;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ CG vector kernels
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_update(T* __restrict__ r, const T* __restrict__ q, long long n,
                                                        SolverState* st, double* partials) {
  if (st->done) return;
  const T al = (T)st->alpha;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T rv = r[i] - al * q[i];
    r[i] = rv;
    acc += (double)rv * (double)rv;
  }
  acc = block_sum(acc);
  if (publish_partial(partials, acc, &st->counter[1])) {
    const double rrn = gather_partials(partials, &st->counter[1]);
    if (threadIdx.x == 0) {
      st->beta = rrn / st->rr;
      st->rr = rrn;
      st->iter += 1;
      if (!isfinite(rrn)) {
        st->status = 5;
        st->done = 1;
      } else if (rrn <= st->tol2) {
        st->done = 1;
      }
    }
  }
}

template <typename T>
__global__ void k_cg_finalize(T* __restrict__ x, const T* __restrict__ p, long long n, const SolverState* st) {
  const double al = st->alpha;
  if (al == 0.0) return;
  const T a = (T)al;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += a * p[i];
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_begin(const T* __restrict__ r, long long n, SolverState* st,
                                                       double* partials, double tol, double bb_given) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += (double)r[i] * (double)r[i];
  acc = block_sum(acc);
  if (publish_partial(partials, acc, &st->counter[2])) {
    const double rr = gather_partials(partials, &st->counter[2]);
    if (threadIdx.x == 0) {
      const double bb = bb_given >= 0.0 ? bb_given : rr;
      st->rr = rr;
      st->bb = bb;
      st->tol2 = tol * tol * bb;
      st->alpha = 0.0;
      st->beta = 0.0;
      st->pq = 0.0;
      st->iter = 0;
      st->status = 0;
      st->done = (rr <= st->tol2) ? 1 : 0;
    }
  }
}

template <typename T>
__global__ void k_fill_rhs(OpArgs<T> a, T* __restrict__ r, T* __restrict__ x) {
  const long long n = (long long)a.c * a.V;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int comp = (int)(i / a.V);
    const long long vox = i - comp * a.V;
    r[i] = a.act[a.phase[vox]] ? a.load[comp] : (T)0;
    x[i] = (T)0;
  }
}

// Internal basis <-> Mandel for the three normal components (shear unchanged):
// h = (e11+e22+e33)/sqrt3, d1 = (e11-e22)/sqrt2, d2 = (e11+e22-2 e33)/sqrt6.
template <typename T>
__global__ void k_rotate(const T* in, T* out, long long V, int to_internal) {
  const double s3 = 0.57735026918962576450914878050195745565;   // 1/sqrt3
  const double s2 = 0.70710678118654752440084436210484903928;   // 1/sqrt2
  const double s6 = 0.40824829046386301636621401245098189866;   // 1/sqrt6
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const double a0 = in[v], a1 = in[V + v], a2 = in[2 * V + v];
    double b0, b1, b2;
    if (to_internal) {
      b0 = (a0 + a1 + a2) * s3;
      b1 = (a0 - a1) * s2;
      b2 = (a0 + a1 - 2.0 * a2) * s6;
    } else {
      b0 = a0 * s3 + a1 * s2 + a2 * s6;
      b1 = a0 * s3 - a1 * s2 + a2 * s6;
      b2 = a0 * s3 - 2.0 * a2 * s6;
    }
    out[v] = (T)b0;
    out[V + v] = (T)b1;
    out[2 * V + v] = (T)b2;
    if (in != out)
      for (int k = 3; k < 6; ++k) out[k * V + v] = in[k * V + v];
  }
}

// Per-component sums, deterministic: partials[comp][blk], then ordered sums.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_comp_partials(const T* __restrict__ x, long long V, double* partials) {
  const int comp = blockIdx.y;
  const T* xc = x + comp * V;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x)
    acc += (double)xc[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[comp * gridDim.x + blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) k_comp_final(const double* partials, int nblk, double* out) {
  const int comp = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += partials[comp * nblk + i];
  s = block_sum(s);
  if (threadIdx.x == 0) out[comp] = s;
}

// ------------------------------------------------------------------ Gamma^h table
// Continuous Green operator of the reference medium (Sec. 2.2.1) at a nonzero
// frequency xi, in the component basis of the problem (Mandel for elasticity).
struct GammaCtx {
  int dim, physics, green, c;
  int n[3];
  double ref[6];  // scalar: diagonal of A0; elastic: (K0, mu0)
};

__device__ void gamma0_acc(const GammaCtx& g, const double xi[3], double w, double* G) {
  if (g.physics == 0) {
    double q = 0.0;
    for (int i = 0; i < g.dim; ++i) q += g.ref[i] * xi[i] * xi[i];
    for (int i = 0; i < g.c; ++i)
      for (int j = 0; j < g.c; ++j) G[i * g.c + j] += w * xi[i] * xi[j] / q;
    return;
  }
  const double K0 = g.ref[0], mu0 = g.ref[1];
  const double lam0 = K0 - 2.0 * mu0 / 3.0;
  const double cb = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0));
  const double nn = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
  const double n[3] = {xi[0] / nn, xi[1] / nn, xi[2] / nn};
  const double r2 = 1.41421356237309504880168872420969807857;
  const int mi[6] = {0, 1, 2, 1, 0, 0}, mj[6] = {0, 1, 2, 2, 2, 1};
  for (int J = 0; J < 6; ++J) {
    // tensor T of the Mandel unit vector e_J
    double T[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const double val = J < 3 ? 1.0 : 1.0 / r2;
    T[mi[J]][mj[J]] = val;
    T[mj[J]][mi[J]] = val;
    double Tn[3];
    for (int i = 0; i < 3; ++i) Tn[i] = T[i][0] * n[0] + T[i][1] * n[1] + T[i][2] * n[2];
    const double nTn = n[0] * Tn[0] + n[1] * Tn[1] + n[2] * Tn[2];
    // S = (Tn (x) n + n (x) Tn) / (2 mu0) - cb (n.Tn) n (x) n
    for (int I = 0; I < 6; ++I) {
      const int i = mi[I], j = mj[I];
      const double S = (Tn[i] * n[j] + n[i] * Tn[j]) / (2.0 * mu0) - cb * nTn * n[i] * n[j];
      G[I * 6 + J] += w * (I < 3 ? S : r2 * S);
    }
  }
}

template <typename T>
__global__ void k_gamma_table(OpArgs<T> a, GammaCtx g, const int* __restrict__ kofy, const int* __restrict__ kofz) {
  const long long nf = (long long)a.nz * a.ny * a.nxh;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(f % a.nxh);
    const int yp = (int)((f / a.nxh) % a.ny);
    const int zp = (int)(f / ((long long)a.nxh * a.ny));
    const int k[3] = {kx, kofy[yp], kofz[zp]};
    const int c = g.c;
    double G[36];
    for (int i = 0; i < c * c; ++i) G[i] = 0.0;
    bool nyq = false;
    if (g.green == 0) {
      // truncated, Eqs. (14)-(15) with the Nyquist rule of Sec. 3.2.1
      double xi[3] = {0, 0, 0};
      bool zero = true;
      for (int i = 0; i < g.dim; ++i) {
        const int ki = k[i] <= g.n[i] / 2 ? k[i] : k[i] - g.n[i];
        if ((g.n[i] & 1) == 0 && k[i] == g.n[i] / 2) nyq = true;
        xi[i] = ki;
        if (ki != 0) zero = false;
      }
      if (zero) nyq = false;
      else if (!nyq) gamma0_acc(g, xi, 1.0, G);
    } else {
      // filtered, Sec. 3.2.2: weights cos^2 / sin^2 (pi k_i / (2 N_i))
      const int nterm = 1 << g.dim;
      for (int t = 0; t < nterm; ++t) {
        double w = 1.0, xi[3] = {0, 0, 0};
        bool zero = true;
        for (int i = 0; i < g.dim; ++i) {
          const bool shift = (t >> i) & 1;
          double sn, cs;
          sincospi((double)k[i] / (2.0 * g.n[i]), &sn, &cs);
          w *= shift ? sn * sn : cs * cs;
          xi[i] = (double)k[i] - (shift ? (double)g.n[i] : 0.0);
          if (xi[i] != 0.0) zero = false;
        }
        if (w == 0.0 || zero) continue;
        gamma0_acc(g, xi, w, G);
      }
    }
    // to the internal basis: scalar -> unchanged; elastic -> R G R^T with
    // R = [u0; u1; u2] on the normal block (see k_rotate)
    double Gi[36];
    if (nyq) {
      // A0^{-1} (C0^{-1} for elasticity), diagonal in the internal basis
      for (int i = 0; i < c * c; ++i) Gi[i] = 0.0;
      for (int i = 0; i < c; ++i)
        Gi[i * c + i] = g.physics == 0 ? 1.0 / g.ref[i] : (i == 0 ? 1.0 / (3.0 * g.ref[0]) : 1.0 / (2.0 * g.ref[1]));
    } else if (g.physics == 0) {
      for (int i = 0; i < c * c; ++i) Gi[i] = G[i];
    } else {
      const double s3 = 0.57735026918962576450914878050195745565, s2 = 0.70710678118654752440084436210484903928,
                   s6 = 0.40824829046386301636621401245098189866;
      const double R[6][6] = {{s3, s3, s3, 0, 0, 0},     {s2, -s2, 0, 0, 0, 0}, {s6, s6, -2 * s6, 0, 0, 0},
                              {0, 0, 0, 1, 0, 0},        {0, 0, 0, 0, 1, 0},    {0, 0, 0, 0, 0, 1}};
      double RG[36];
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
          double s = 0.0;
          for (int l = 0; l < 6; ++l) s += R[i][l] * G[l * 6 + j];
          RG[i * 6 + j] = s;
        }
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
          double s = 0.0;
          for (int l = 0; l < 6; ++l) s += RG[i * 6 + l] * R[j][l];
          Gi[i * 6 + j] = s;
        }
    }
    const double invV = 1.0 / (double)a.V;
    const long long cstride = nf;
    int coef = 0;
    T* out = const_cast<T*>(a.gtab);
    for (int i = 0; i < c; ++i)
      for (int j = i; j < c; ++j, ++coef) out[coef * cstride + f] = (T)(0.5 * (Gi[i * c + j] + Gi[j * c + i]) * invV);
  }
}

// ------------------------------------------------------------------ mixed precision helpers
__global__ void __launch_bounds__(kThreads) k_d2f_begin(const double* __restrict__ r64, float* __restrict__ r32,
                                                        float* __restrict__ x32, long long n, SolverState* st,
                                                        double* partials, double tol) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = (float)r64[i];
    r32[i] = v;
    x32[i] = 0.0f;
    acc += (double)v * (double)v;
  }
  acc = block_sum(acc);
  if (publish_partial(partials, acc, &st->counter[2])) {
    const double rr = gather_partials(partials, &st->counter[2]);
    if (threadIdx.x == 0) {
      st->rr = rr;
      st->bb = rr;
      st->tol2 = tol * tol * rr;
      st->alpha = st->beta = st->pq = 0.0;
      st->iter = 0;
      st->status = 0;
      st->done = (rr <= st->tol2) ? 1 : 0;
    }
  }
}

__global__ void k_f2d_axpy(double* __restrict__ x64, const float* __restrict__ x32, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x64[i] += (double)x32[i];
}

// Phase scan at setup: number of voxels in I0 (aux[1]) and largest phase id (aux[2]).
__global__ void __launch_bounds__(kThreads) k_scan_phase(const unsigned char* __restrict__ phase, long long V,
                                                         const unsigned char* __restrict__ act, int nphase,
                                                         SolverState* st, double* partials) {
  double cnt = 0.0;
  int mx = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    const int ph = phase[i];
    mx = max(mx, ph);
    if (ph < nphase && act[ph]) cnt += 1.0;
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(&st->pad, mx);
  cnt = block_sum(cnt);
  if (publish_partial(partials, cnt, &st->counter[3])) {
    const double tot = gather_partials(partials, &st->counter[3]);
    if (threadIdx.x == 0) st->aux[1] = tot;
  }
}

// Scale gradient: g = (1/V) sum_ij W_ij eps_i . A_phase eps_j, eps_j = M tau_j
// (internal basis, where M and A_phase are diagonal).  tau_all is Mandel.
__global__ void k_scale_grad(const double* __restrict__ tau_all, const double* __restrict__ W,
                             const unsigned char* __restrict__ phase, const float* __restrict__ scale,
                             const double* __restrict__ modtab, const double* __restrict__ ref, int c, int elastic,
                             long long V, double* __restrict__ grad) {
  const double s3 = 0.57735026918962576450914878050195745565, s2 = 0.70710678118654752440084436210484903928,
               s6 = 0.40824829046386301636621401245098189866;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const int ph = phase[v];
    const double s = scale ? (double)scale[v] : 1.0;
    double A[6], m[6];
    for (int k = 0; k < c; ++k) {
      A[k] = modtab[ph * c + k];
      m[k] = 1.0 / (s * A[k] - ref[k]);
    }
    double eps[6][6];
    for (int j = 0; j < c; ++j) {
      const double* tj = tau_all + (long long)j * c * V;
      double t[6];
      for (int k = 0; k < c; ++k) t[k] = tj[k * V + v];
      if (elastic) {
        const double a0 = t[0], a1 = t[1], a2 = t[2];
        t[0] = (a0 + a1 + a2) * s3;
        t[1] = (a0 - a1) * s2;
        t[2] = (a0 + a1 - 2.0 * a2) * s6;
      }
      for (int k = 0; k < c; ++k) eps[j][k] = m[k] * t[k];
    }
    double gsum = 0.0;
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) {
        const double w = W[i * c + j];
        if (w == 0.0) continue;
        double e = 0.0;
        for (int k = 0; k < c; ++k) e += eps[i][k] * A[k] * eps[j][k];
        gsum += w * e;
      }
    grad[v] = gsum / (double)V;
  }
}

// ------------------------------------------------------------------ launchers
// The attribute is a per-function upper bound shared by every handle: always
// allow the full 227 KB so that one handle never shrinks another's limit.
template <typename T> void set_smem_attrs(const LaunchCfg&) {
  const int mx = 227 * 1024;
  cudaFuncSetAttribute(k_xfwd<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xfwd<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_yfft<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_yfft<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_zgamma<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_zgamma<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_zgamma<T, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

template <typename T>
void launch_xfwd(const OpArgs<T>& a, const LaunchCfg& L, int mode, const T* in, T* x, const T* r, T* p,
                 const SolverState* st, cudaStream_t s) {
  if (mode == 0) k_xfwd<T, 0><<<L.grid_x, L.threads, L.smem_x, s>>>(a, in, x, r, p, st);
  else k_xfwd<T, 1><<<L.grid_x, L.threads, L.smem_x, s>>>(a, in, x, r, p, st);
}

template <typename T>
void launch_yfft(const OpArgs<T>& a, const LaunchCfg& L, bool inv, const SolverState* st, cudaStream_t s) {
  dim3 g(L.grid_yx, L.grid_yy);
  if (inv) k_yfft<T, true><<<g, L.threads, L.smem_y, s>>>(a, st);
  else k_yfft<T, false><<<g, L.threads, L.smem_y, s>>>(a, st);
}

template <typename T>
void launch_zgamma(const OpArgs<T>& a, const LaunchCfg& L, const SolverState* st, cudaStream_t s) {
  dim3 g(L.grid_zx, L.grid_zy);
  if (a.c == 6) k_zgamma<T, 6><<<g, L.threads, L.smem_z, s>>>(a, st);
  else if (a.c == 3) k_zgamma<T, 3><<<g, L.threads, L.smem_z, s>>>(a, st);
  else k_zgamma<T, 2><<<g, L.threads, L.smem_z, s>>>(a, st);
}

template <typename T>
void launch_xinv(const OpArgs<T>& a, const LaunchCfg& L, int mode, const T* xin, T* out, SolverState* st,
                 double* partials, cudaStream_t s) {
  if (mode == 0) k_xinv<T, 0><<<L.grid_x, L.threads, L.smem_x, s>>>(a, xin, out, st, partials);
  else if (mode == 1) k_xinv<T, 1><<<L.grid_x, L.threads, L.smem_x, s>>>(a, xin, out, st, partials);
  else k_xinv<T, 2><<<L.grid_x, L.threads, L.smem_x, s>>>(a, xin, out, st, partials);
}

template <typename T>
void launch_cg_update(T* r, const T* q, long long n, SolverState* st, double* partials, int grid, cudaStream_t s) {
  k_cg_update<T><<<grid, kThreads, 0, s>>>(r, q, n, st, partials);
}
template <typename T>
void launch_cg_finalize(T* x, const T* p, long long n, const SolverState* st, int grid, cudaStream_t s) {
  k_cg_finalize<T><<<grid, kThreads, 0, s>>>(x, p, n, st);
}
template <typename T>
void launch_cg_begin(const T* r, long long n, SolverState* st, double* partials, double tol, double bb_given,
                     int grid, cudaStream_t s) {
  k_cg_begin<T><<<grid, kThreads, 0, s>>>(r, n, st, partials, tol, bb_given);
}
template <typename T> void launch_fill_rhs(const OpArgs<T>& a, T* r, T* x, int grid, cudaStream_t s) {
  k_fill_rhs<T><<<grid, kThreads, 0, s>>>(a, r, x);
}
template <typename T> void launch_rotate(const T* in, T* out, long long V, int to_internal, int grid, cudaStream_t s) {
  k_rotate<T><<<grid, kThreads, 0, s>>>(in, out, V, to_internal);
}
template <typename T>
void launch_comp_sums(const T* x, int c, long long V, double* partials, int nblk, double* out, cudaStream_t s) {
  k_comp_partials<T><<<dim3(nblk, c), kThreads, 0, s>>>(x, V, partials);
  k_comp_final<<<c, kThreads, 0, s>>>(partials, nblk, out);
}
template <typename T>
void launch_gamma_table(const OpArgs<T>& a, int dim, int physics, int green, const double* ref_mandel,
                        const int* kofy, const int* kofz, cudaStream_t s) {
  GammaCtx g;
  g.dim = dim;
  g.physics = physics;
  g.green = green;
  g.c = a.c;
  g.n[0] = a.nx;
  g.n[1] = a.ny;
  g.n[2] = a.nz;
  for (int i = 0; i < 6; ++i) g.ref[i] = ref_mandel[i];
  const long long nf = (long long)a.nz * a.ny * a.nxh;
  const int grid = (int)std::min<long long>((nf + 127) / 128, 152LL * 16);
  k_gamma_table<T><<<grid, 128, 0, s>>>(a, g, kofy, kofz);
}
void launch_d2f_begin(const double* r64, float* r32, float* x32, long long n, SolverState* st, double* partials,
                      double tol, int grid, cudaStream_t s) {
  k_d2f_begin<<<grid, kThreads, 0, s>>>(r64, r32, x32, n, st, partials, tol);
}
void launch_f2d_axpy(double* x64, const float* x32, long long n, int grid, cudaStream_t s) {
  k_f2d_axpy<<<grid, kThreads, 0, s>>>(x64, x32, n);
}
void launch_scan_phase(const unsigned char* phase, long long V, const unsigned char* act, int nphase,
                       SolverState* st, double* partials, int grid, cudaStream_t s) {
  k_scan_phase<<<grid, kThreads, 0, s>>>(phase, V, act, nphase, st, partials);
}
void launch_scale_grad(const double* tau_all, const double* W, const unsigned char* phase, const float* scale,
                       const double* modtab, const double* ref, int c, int elastic, long long V, double* grad,
                       int grid, cudaStream_t s) {
  k_scale_grad<<<grid, 128, 0, s>>>(tau_all, W, phase, scale, modtab, ref, c, elastic, V, grad);
}

#define LSH_INSTANTIATE(T)                                                                                        \
  template void set_smem_attrs<T>(const LaunchCfg&);                                                              \
  template void launch_xfwd<T>(const OpArgs<T>&, const LaunchCfg&, int, const T*, T*, const T*, T*,               \
                               const SolverState*, cudaStream_t);                                                 \
  template void launch_yfft<T>(const OpArgs<T>&, const LaunchCfg&, bool, const SolverState*, cudaStream_t);       \
  template void launch_zgamma<T>(const OpArgs<T>&, const LaunchCfg&, const SolverState*, cudaStream_t);           \
  template void launch_xinv<T>(const OpArgs<T>&, const LaunchCfg&, int, const T*, T*, SolverState*, double*,      \
                               cudaStream_t);                                                                     \
  template void launch_cg_update<T>(T*, const T*, long long, SolverState*, double*, int, cudaStream_t);           \
  template void launch_cg_finalize<T>(T*, const T*, long long, const SolverState*, int, cudaStream_t);            \
  template void launch_cg_begin<T>(const T*, long long, SolverState*, double*, double, double, int, cudaStream_t); \
  template void launch_fill_rhs<T>(const OpArgs<T>&, T*, T*, int, cudaStream_t);                                  \
  template void launch_rotate<T>(const T*, T*, long long, int, int, cudaStream_t);                                \
  template void launch_comp_sums<T>(const T*, int, long long, double*, int, double*, cudaStream_t);               \
  template void launch_gamma_table<T>(const OpArgs<T>&, int, int, int, const double*, const int*, const int*,     \
                                      cudaStream_t);

LSH_INSTANTIATE(double)
LSH_INSTANTIATE(float)

}  // namespace lsh
