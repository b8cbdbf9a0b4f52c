// kernels.cu -- the operator passes and CG kernels of liblsh (sm_103a).
//
// One application of the Lippmann-Schwinger operator of Eq. (13),
//   K x = P (M x + DFT^{-1}[Gamma^h_k DFT(x)_k]),
// is five passes over a half spectrum H[S][c][nz][ny][nx/2+1]:
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
// Every pass handles S independent systems at once (batched loads and
// microstructures); each system has its own CG state and reductions.
#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"
#include "gamma_onfly.cuh"

namespace lsh {

static constexpr int kThreads = 256;
// resident blocks per SM the register allocation must allow: FP64 passes
// are FP64-pipe bound and need 2 blocks to hide latency, FP32 passes are
// memory bound and need 3
template <typename T> struct MinBlocks { static constexpr int value = sizeof(T) == 8 ? 2 : 3; };

template <typename T, int VEC> struct VecOf;
template <> struct VecOf<float, 4> { typedef float4 type; };
template <> struct VecOf<double, 2> { typedef double2 type; };

template <typename T, int VEC> __device__ __forceinline__ void vload(const T* __restrict__ p, T* v) {
  if constexpr (VEC == 1) {
    v[0] = p[0];
  } else {
    typedef typename VecOf<T, VEC>::type V;
    const V w = *reinterpret_cast<const V*>(p);
    const T* q = reinterpret_cast<const T*>(&w);
#pragma unroll
    for (int u = 0; u < VEC; ++u) v[u] = q[u];
  }
}
template <typename T, int VEC> __device__ __forceinline__ void vstore(T* __restrict__ p, const T* v) {
  if constexpr (VEC == 1) {
    p[0] = v[0];
  } else {
    typedef typename VecOf<T, VEC>::type V;
    V w;
    T* q = reinterpret_cast<T*>(&w);
#pragma unroll
    for (int u = 0; u < VEC; ++u) q[u] = v[u];
    *reinterpret_cast<V*>(p) = w;
  }
}

// Local coefficient m = (A_beta - A0)^{-1} of component `comp` at voxel index
// `pv` of the stacked phase map; *active = voxel in I0.
template <typename T>
__device__ __forceinline__ T local_coef(const OpArgs<T>& a, long long pv, int comp, int* active) {
  const int ph = a.phase[pv];
  *active = a.act[ph];
  if (a.scale == nullptr) return a.mtab[ph * a.c + comp];
  const T s = (T)a.scale[pv];
  return (T)1 / (s * a.modtab[ph * a.c + comp] - a.ref[comp]);
}

// ------------------------------------------------------------------ x forward
// MODE 0: input field `in` (masked by I0).  MODE 1: CG prologue.
// Each thread handles VEC consecutive x of a row pair and writes complete
// complex values of the packed line Z = row_even + i row_odd.
template <typename T, int MODE, int VEC>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_xfwd(OpArgs<T> a, const T* __restrict__ in, T* __restrict__ x,
                                                   const T* __restrict__ r, T* __restrict__ p,
                                                   const SolverState* __restrict__ st) {
  const int s = blockIdx.x / a.bps;
  if (MODE == 1 && st[s].done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* Z = tw + a.nx;
  int* pos = reinterpret_cast<int*>(Z + ((a.RY + 1) >> 1) * a.lsx);
  const int nx = a.nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    tw[i] = a.twx[i];
    pos[i] = a.posx[i];
  }
  const int rloc = (blockIdx.x - s * a.bps) * a.RY;  // first row inside the system
  const int nr = a.RY;
  const int npair = (nr + 1) >> 1;
  const long long row0 = (long long)s * a.rps + rloc;  // global row
  T alpha = 0, beta = 0;
  int k = 0;
  if (MODE == 1) {
    k = st[s].iter;
    alpha = (T)st[s].alpha;
    beta = (T)st[s].beta;
  }
  const int nxv = nx / VEC;
  const int rows_per_comp = a.nz * a.ny;
  const long long pbase = (long long)((a.sys0 + s) / a.sys_per_ms) * a.V;
  for (int idx = threadIdx.x; idx < npair * nxv; idx += blockDim.x) {
    const int lp = fdiv(idx, nxv);
    const int xx = (idx - lp * nxv) * VEC;
    T v0[VEC], v1[VEC];
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      T* v = h2 ? v1 : v0;
      const int row = 2 * lp + h2;
      if (row >= nr) {
#pragma unroll
        for (int u = 0; u < VEC; ++u) v[u] = (T)0;
        continue;
      }
      const long long g = (row0 + row) * nx + xx;
      if (MODE == 0) {
        vload<T, VEC>(in + g, v);
        const int rs = rloc + row;
        const int comp = rs / rows_per_comp;
        const long long vox = (long long)(rs - comp * rows_per_comp) * nx + xx;
#pragma unroll
        for (int u = 0; u < VEC; ++u)
          if (!a.act[a.phase[pbase + vox + u]]) v[u] = (T)0;
      } else if (k == 0) {
        vload<T, VEC>(r + g, v);
        vstore<T, VEC>(p + g, v);
      } else {
        T pv[VEC], xv[VEC];
        vload<T, VEC>(p + g, pv);
        vload<T, VEC>(x + g, xv);
        vload<T, VEC>(r + g, v);
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          xv[u] += alpha * pv[u];
          v[u] += beta * pv[u];
        }
        vstore<T, VEC>(x + g, xv);
        vstore<T, VEC>(p + g, v);
      }
    }
#pragma unroll
    for (int u = 0; u < VEC; ++u) Z[lp * a.lsx + xx + u] = mkc<T>(v0[u], v1[u]);
  }
  __syncthreads();
  fft_lines<T, false>(Z, npair, a.lsx, a.px, tw);
  // split Z = X_a + i X_b into the two Hermitian half rows
  const T h = (T)0.5;
  for (int idx = threadIdx.x; idx < npair * a.nxh; idx += blockDim.x) {
    const int lp = fdiv(idx, a.nxh), kx = idx - lp * a.nxh;
    const C2<T> z1 = Z[lp * a.lsx + pos[kx]];
    const C2<T> z2 = Z[lp * a.lsx + pos[kx == 0 ? 0 : nx - kx]];
    const long long hrow = row0 + 2 * lp;
    a.H[hrow * a.hs + kx] = mkc<T>(h * (z1.x + z2.x), h * (z1.y - z2.y));
    if (2 * lp + 1 < nr) a.H[(hrow + 1) * a.hs + kx] = mkc<T>(h * (z1.y + z2.y), h * (z2.x - z1.x));
  }
}

// ------------------------------------------------------------------ y pass
// blockIdx.y = plane (s, comp, z); TY consecutive kx columns per block.
template <typename T, bool INV>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_yfft(OpArgs<T> a, const SolverState* __restrict__ st) {
  const long long plane = blockIdx.y;
  const int s = (int)(plane / (a.c * a.nz));
  if (st != nullptr && st[s].done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf = tw + a.ny;
  for (int i = threadIdx.x; i < a.ny; i += blockDim.x) tw[i] = a.twy[i];
  const int kx0 = blockIdx.x * a.TY;
  const int nt = min(a.TY, a.nxh - kx0);
  const int TY = a.TY;
  C2<T>* __restrict__ Hp = a.H + plane * a.ny * a.hs + kx0;
  const int tot = a.ny * TY;
  for (int base = threadIdx.x; base < tot; base += 4 * blockDim.x) {
    C2<T> v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * blockDim.x;
      const int y = fdiv(idx, TY), t = idx - y * TY;
      if (idx < tot && t < nt) v[u] = Hp[(long long)y * a.hs + t];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * blockDim.x;
      const int y = fdiv(idx, TY), t = idx - y * TY;
      if (idx < tot && t < nt) buf[t * a.lsy + y] = v[u];
    }
  }
  __syncthreads();
  fft_lines<T, INV>(buf, nt, a.lsy, a.py, tw);
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int y = fdiv(idx, TY), t = idx - y * TY;
    if (t < nt) Hp[(long long)y * a.hs + t] = buf[t * a.lsy + y];
  }
}

// ------------------------------------------------------------------ z pass + Gamma
// blockIdx.x = system, blockIdx.y = kx tile, blockIdx.z = y position: the
// blocks of all systems for one tile run together and share its Gamma
// coefficients through L2.
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_zgamma(OpArgs<T> a, const SolverState* __restrict__ st) {
  const int s = blockIdx.x;
  if (st != nullptr && st[s].done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf = tw + a.nz;
  for (int i = threadIdx.x; i < a.nz; i += blockDim.x) tw[i] = a.twz[i];
  const int yp = blockIdx.z;
  const int kx0 = blockIdx.y * a.TZ;
  const int nt = min(a.TZ, a.nxh - kx0);
  const int nz = a.nz, TZ = a.TZ;
  const long long zstride = (long long)a.ny * a.hs;  // distance between z planes of H
  const long long cstride = zstride * nz;
  C2<T>* __restrict__ Hp = a.H + (long long)s * NC * cstride + (long long)yp * a.hs + kx0;
  const int tot = NC * nz * TZ;
  for (int base = threadIdx.x; base < tot; base += 4 * blockDim.x) {
    C2<T> v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * blockDim.x;
      const int rest = fdiv(idx, TZ), t = idx - rest * TZ;
      const int comp = fdiv(rest, nz), z = rest - comp * nz;
      v[u] = mkc<T>(0, 0);
      if (idx < tot && t < nt) v[u] = Hp[comp * cstride + z * zstride + t];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * blockDim.x;
      const int rest = fdiv(idx, TZ), t = idx - rest * TZ;
      const int comp = fdiv(rest, nz), z = rest - comp * nz;
      if (idx < tot) buf[(comp * TZ + t) * a.lsz + z] = v[u];
    }
  }
  __syncthreads();
  if (nz > 1) fft_lines<T, false>(buf, NC * TZ, a.lsz, a.pz, tw);
  // per-frequency product with Gamma^h_k
  const int ky = (a.onfly || a.fdphase) ? a.kofy[yp] : 0;
  for (int idx = threadIdx.x; idx < nz * TZ; idx += blockDim.x) {
    const int zp = fdiv(idx, TZ), t = idx - zp * TZ;
    if (t >= nt) continue;
    C2<T> v[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) v[i] = buf[(i * TZ + t) * a.lsz + zp];
    if (a.onfly) {
      gamma_trunc_onfly<T, NC>(a, kx0 + t, ky, a.kofz[zp], v);
    } else {
      if (a.fdphase) fd_rotate<T, NC>(a, kx0 + t, ky, a.kofz[zp], v, (T)-1);
      gamma_table_apply<T, NC>(a.gtab, ((long long)zp * a.ny + yp) * a.ts + kx0 + t, v);
      if (a.fdphase) fd_rotate<T, NC>(a, kx0 + t, ky, a.kofz[zp], v, (T)1);
    }
#pragma unroll
    for (int i = 0; i < NC; ++i) buf[(i * TZ + t) * a.lsz + zp] = v[i];
  }
  __syncthreads();
  if (nz > 1) fft_lines<T, true>(buf, NC * TZ, a.lsz, a.pz, tw);
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int rest = fdiv(idx, TZ), t = idx - rest * TZ;
    const int comp = fdiv(rest, nz), z = rest - comp * nz;
    if (t < nt) Hp[comp * cstride + z * zstride + t] = buf[(comp * TZ + t) * a.lsz + z];
  }
}

// ------------------------------------------------------------------ x inverse + local term
// MODE 0: out = P (M xin + g).  MODE 1 (CG): q = P (M p + g), (p, q) -> alpha.
// MODE 2 (residual): out = P (load - M xin - g), (r, r) -> st[s].aux[0].
template <typename T, int MODE, int VEC>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_xinv(OpArgs<T> a, const T* __restrict__ xin,
                                                                        T* __restrict__ out,
                                                                        SolverState* __restrict__ st,
                                                                        double* __restrict__ partials) {
  const int s = blockIdx.x / a.bps;
  if ((MODE == 1 || MODE == 3) && st[s].done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T mloc[256 * 6];  // local coefficients (no scale field) or A_phase diagonal
  __shared__ unsigned char aloc[256];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* Z = tw + a.nx;
  int* pos = reinterpret_cast<int*>(Z + ((a.RY + 1) >> 1) * a.lsx);
  const int nx = a.nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    tw[i] = a.twx[i];
    pos[i] = a.posx[i];
  }
  const int ntab = a.nphase * a.c;
  for (int i = threadIdx.x; i < ntab; i += blockDim.x) mloc[i] = (a.scale && !a.frac) ? a.modtab[i] : a.mtab[i];
  for (int i = threadIdx.x; i < a.nphase; i += blockDim.x) aloc[i] = a.act[i];
  __syncthreads();
  const int blk = blockIdx.x - s * a.bps;
  const int rloc = blk * a.RY;
  const int nr = a.RY;
  const int npair = (nr + 1) >> 1;
  const long long row0 = (long long)s * a.rps + rloc;
  const C2<T>* __restrict__ Hb = a.H + row0 * a.hs;
  // Z = X_a + i X_b over the full line, X(nx - k) = conj X(k) beyond the half
  const int nz_items = npair * a.nxh;
  for (int base = threadIdx.x; base < nz_items; base += 4 * blockDim.x) {
    C2<T> xa[4], xb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * blockDim.x;
      xa[u] = xb[u] = mkc<T>(0, 0);
      if (idx < nz_items) {
        const int lp = fdiv(idx, a.nxh), kx = idx - lp * a.nxh;
        xa[u] = Hb[(2 * lp) * a.hs + kx];
        if (2 * lp + 1 < nr) xb[u] = Hb[(2 * lp + 1) * a.hs + kx];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < nz_items) {
        const int lp = fdiv(idx, a.nxh), kx = idx - lp * a.nxh;
        Z[lp * a.lsx + pos[kx]] = mkc<T>(xa[u].x - xb[u].y, xa[u].y + xb[u].x);
        if (kx >= 1 && kx <= nx - a.nxh) Z[lp * a.lsx + pos[nx - kx]] = mkc<T>(xa[u].x + xb[u].y, xb[u].x - xa[u].y);
      }
    }
  }
  __syncthreads();
  fft_lines<T, true>(Z, npair, a.lsx, a.px, tw);
  const int rows_per_comp = a.nz * a.ny;
  const long long pbase = (long long)((a.sys0 + s) / a.sys_per_ms) * a.V;
  const int nxv = nx / VEC;
  Acc<T> acc;
  for (int idx = threadIdx.x; idx < npair * nxv; idx += blockDim.x) {
    const int lp = fdiv(idx, nxv);
    const int xx = (idx - lp * nxv) * VEC;
    // issue every global load of the row pair first
    T xv[2][VEC];
    unsigned char ph[2][VEC];
    int comp[2];
    long long voxs[2];
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int row = 2 * lp + h2;
      const int rs = rloc + min(row, nr - 1);
      comp[h2] = rs / rows_per_comp;
      const long long vox = (long long)(rs - comp[h2] * rows_per_comp) * nx + xx;
      voxs[h2] = pbase + vox;
      if (row < nr) {
        vload<T, VEC>(xin + (row0 + row) * nx + xx, xv[h2]);
        if constexpr (VEC == 4) {
          const uchar4 q = *reinterpret_cast<const uchar4*>(a.phase + pbase + vox);
          ph[h2][0] = q.x; ph[h2][1] = q.y; ph[h2][2] = q.z; ph[h2][3] = q.w;
        } else if constexpr (VEC == 2) {
          const uchar2 q = *reinterpret_cast<const uchar2*>(a.phase + pbase + vox);
          ph[h2][0] = q.x; ph[h2][1] = q.y;
        } else {
          ph[h2][0] = a.phase[pbase + vox];
        }
      }
    }
    C2<T> zc[VEC];
#pragma unroll
    for (int u = 0; u < VEC; ++u) zc[u] = Z[lp * a.lsx + xx + u];
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int row = 2 * lp + h2;
      if (row >= nr) continue;
      const long long g = (row0 + row) * nx + xx;
      T ov[VEC];
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        const int p = ph[h2][u];
        const bool active = aloc[p] != 0;
        T m = mloc[p * a.c + comp[h2]];
        if (a.scale) {
          const T f = (T)a.scale[voxs[h2] + u];
          m = a.frac ? f * mloc[a.c + comp[h2]] + ((T)1 - f) * mloc[comp[h2]]  // Eq. (def_ah)
                     : (T)1 / (f * m - a.ref[comp[h2]]);
        }
        const T gv = h2 ? zc[u].y : zc[u].x;
        const T xq = xv[h2][u];
        if (MODE == 0) {
          ov[u] = active ? m * xq + gv : (T)0;
        } else if (MODE == 1 || MODE == 3) {
          ov[u] = active ? m * xq + gv : (T)0;
          acc.add(xq * ov[u]);
        } else {
          ov[u] = active ? a.loads[s * 6 + comp[h2]] - (m * xq + gv) : (T)0;
          acc.add(ov[u] * ov[u]);
        }
      }
      vstore<T, VEC>(out + g, ov);
    }
  }
  if (MODE != 0) {
    const double tot = block_reduce(acc);
    double* part = partials + (long long)s * a.bps;
    SolverState* sst = st + s;
    if (publish_partial_sys(part, blk, a.bps, tot, &sst->counter[0])) {
      const double sum = gather_partials_sys(part, a.bps, &sst->counter[0]);
      if (threadIdx.x == 0) {
        if (MODE == 1) {
          sst->pq = sum;
          if (!(fabs(sum) > 0.0) || !isfinite(sum) || !isfinite(sst->rr)) {
            sst->status = 5;  // LSH_ERR_BREAKDOWN
            sst->alpha = 0.0;
            sst->done = 1;
          } else {
            sst->alpha = sst->rr / sum;
          }
        } else if (MODE == 3) {
          sst->pq = sum;  // (v, K v) for MINRES: any sign, no breakdown test
        } else {
          sst->aux[0] = sum;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ (p, Kp) from per-block partials
// One block per system sums the partials of its nb blocks in block order and
// sets alpha = (r, r) / (p, Kp) (or flags a breakdown), as the ticket reduction
// of the inverse x pass does.
__global__ void __launch_bounds__(kThreads) k_dot_finalize(SolverState* __restrict__ st,
                                                           const double* __restrict__ partials, int nb) {
  const int s = blockIdx.x;
  SolverState* sst = st + s;
  if (sst->done) return;
  const double* part = partials + (long long)s * nb;
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v += part[i];
  const double sum = block_sum(v);
  if (threadIdx.x == 0) {
    sst->pq = sum;
    if (!(fabs(sum) > 0.0) || !isfinite(sum) || !isfinite(sst->rr)) {
      sst->status = 5;  // LSH_ERR_BREAKDOWN
      sst->alpha = 0.0;
      sst->done = 1;
    } else {
      sst->alpha = sst->rr / sum;
    }
  }
}

// ------------------------------------------------------------------ MINRES vector kernels
// One MINRES iteration after q = K r2 (r2 = beta v, so K v = q / beta) and
// pq = (r2, q) from the inverse x pass:
//   A: y = K v - (beta / oldb) r1, alfa = (v, y)
//   B: y -= (alfa / beta) r2, r1 <- r2, r2 <- y, beta <- |y|, Givens rotation
//   C: w_k = (v - oldeps w_{k-2} - delta w_{k-1}) / gamma, x += phi w_k
// (x0 = 0, r1 = r2 = b; Paige-Saunders recurrences).  Grid (G, S).
__global__ void __launch_bounds__(kThreads) k_mr_a(double* __restrict__ q, const double* __restrict__ r1,
                                                   const double* __restrict__ r2, long long n,
                                                   SolverState* __restrict__ st, MinresScalars* __restrict__ ms,
                                                   double* __restrict__ partials) {
  const int s = blockIdx.y;
  SolverState* sst = st + s;
  if (sst->done) return;
  const double beta = ms[s].beta;
  const double coef = sst->iter > 0 ? beta / ms[s].oldb : 0.0;
  const double ib = 1.0 / beta;
  double* qs = q + s * n;
  const double* r1s = r1 + s * n;
  const double* r2s = r2 + s * n;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    qs[i] = qs[i] * ib - coef * r1s[i];
    acc += r2s[i] * r1s[i];
  }
  const double tot = block_sum(acc);
  double* part = partials + (long long)s * gridDim.x;
  if (publish_partial_sys(part, blockIdx.x, gridDim.x, tot, &sst->counter[1])) {
    const double t2 = gather_partials_sys(part, gridDim.x, &sst->counter[1]);
    if (threadIdx.x == 0) ms[s].alfa = sst->pq * ib * ib - coef * t2 * ib;
  }
}

__global__ void __launch_bounds__(kThreads) k_mr_b(double* __restrict__ q, double* __restrict__ r1,
                                                   double* __restrict__ r2, long long n,
                                                   SolverState* __restrict__ st, MinresScalars* __restrict__ ms,
                                                   double* __restrict__ partials) {
  const int s = blockIdx.y;
  SolverState* sst = st + s;
  if (sst->done) return;
  const double c2 = ms[s].alfa / ms[s].beta;
  double* qs = q + s * n;
  double* r1s = r1 + s * n;
  double* r2s = r2 + s * n;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double y = qs[i] - c2 * r2s[i];
    r1s[i] = r2s[i];
    r2s[i] = y;
    acc += y * y;
  }
  const double tot = block_sum(acc);
  double* part = partials + (long long)s * gridDim.x;
  if (publish_partial_sys(part, blockIdx.x, gridDim.x, tot, &sst->counter[2])) {
    const double yy = gather_partials_sys(part, gridDim.x, &sst->counter[2]);
    if (threadIdx.x == 0) {
      MinresScalars& m = ms[s];
      const double bnew = sqrt(fmax(yy, 0.0));
      m.oldb = m.beta;
      m.beta = bnew;
      m.oldeps = m.epsln;
      m.delta = m.cs * m.dbar + m.sn * m.alfa;
      const double gbar = m.sn * m.dbar - m.cs * m.alfa;
      m.epsln = m.sn * bnew;
      m.dbar = -m.cs * bnew;
      const double gamma = fmax(hypot(gbar, bnew), 1e-300);
      m.cs = gbar / gamma;
      m.sn = bnew / gamma;
      m.phi = m.cs * m.phibar;
      m.phibar = m.sn * m.phibar;
      m.denom = 1.0 / gamma;
      sst->iter += 1;
      sst->rr = m.phibar * m.phibar;  // residual norm estimate, squared
      if (!isfinite(yy) || !isfinite(m.phibar)) {
        sst->status = 5;
        sst->done = 1;
      } else if (m.phibar * m.phibar <= sst->tol2 || bnew == 0.0) {
        m.pending = 1;  // x gets this iteration's update in C, then the system stops
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_mr_c(double* __restrict__ x, double* __restrict__ wa,
                                                   double* __restrict__ wb, const double* __restrict__ r1, long long n,
                                                   SolverState* __restrict__ st, MinresScalars* __restrict__ ms,
                                                   double* __restrict__ partials) {
  const int s = blockIdx.y;
  SolverState* sst = st + s;
  if (sst->done) return;
  const MinresScalars m = ms[s];
  const double iv = 1.0 / m.oldb;  // v = r1 / oldb (r1 holds the previous r2)
  double* xs = x + s * n;
  double* was = wa + s * n;  // w_{k-1}
  double* wbs = wb + s * n;  // w_{k-2}
  const double* r1s = r1 + s * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double a = was[i];
    const double wn = (r1s[i] * iv - m.oldeps * wbs[i] - m.delta * a) * m.denom;
    wbs[i] = a;
    was[i] = wn;
    xs[i] += m.phi * wn;
  }
  double* part = partials + (long long)s * gridDim.x;
  if (publish_partial_sys(part, blockIdx.x, gridDim.x, 0.0, &sst->counter[3])) {
    gather_partials_sys(part, gridDim.x, &sst->counter[3]);
    if (threadIdx.x == 0 && ms[s].pending) sst->done = 1;
  }
}

// ------------------------------------------------------------------ SYMMLQ vector kernels
// The Lanczos step is MINRES's (k_mr_a, then the first half of k_sq_b); the
// tridiagonal T_k is factorised T_k = L_k Q_k by rotations from the right,
// each iteration adds s w + t v to the LQ iterate and turns w, and at
// convergence the CG point x_LQ + zbar w + cb b (cb: the accumulated step
// along the first Lanczos vector b / beta1) is taken.  The estimate of the CG
// point's residual norm is |snprod beta1 beta / gbar|.
__global__ void __launch_bounds__(kThreads) k_sq_b(double* __restrict__ q, double* __restrict__ r1,
                                                   double* __restrict__ r2, long long n,
                                                   SolverState* __restrict__ st, MinresScalars* __restrict__ ms,
                                                   SymmlqScalars* __restrict__ sq, double* __restrict__ partials) {
  const int s = blockIdx.y;
  SolverState* sst = st + s;
  if (sst->done) return;
  const double c2 = ms[s].alfa / ms[s].beta;
  double* qs = q + s * n;
  double* r1s = r1 + s * n;
  double* r2s = r2 + s * n;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double y = qs[i] - c2 * r2s[i];
    r1s[i] = r2s[i];
    r2s[i] = y;
    acc += y * y;
  }
  const double tot = block_sum(acc);
  double* part = partials + (long long)s * gridDim.x;
  if (publish_partial_sys(part, blockIdx.x, gridDim.x, tot, &sst->counter[2])) {
    const double yy = gather_partials_sys(part, gridDim.x, &sst->counter[2]);
    if (threadIdx.x == 0) {
      MinresScalars& m = ms[s];
      SymmlqScalars& l = sq[s];
      const double bnew = sqrt(fmax(yy, 0.0));
      m.oldb = m.beta;
      m.beta = bnew;
      if (sst->iter == 0) {
        l.gbar = m.alfa;
        l.dbar = bnew;
        l.rhs1 = m.beta1;
        l.rhs2 = 0.0;
        l.bstep = 0.0;
        l.snprod = 1.0;
        l.s = l.t = 0.0;  // no update of x or w on the first step
        l.cs = 0.0;
        l.sn = 1.0;
      } else {
        const double gamma = fmax(hypot(l.gbar, m.oldb), 1e-300);
        const double cs = l.gbar / gamma, sn = m.oldb / gamma;
        const double delta = cs * l.dbar + sn * m.alfa;
        l.gbar = sn * l.dbar - cs * m.alfa;
        const double epsln = sn * bnew;
        l.dbar = -cs * bnew;
        const double z = l.rhs1 / gamma;
        l.s = z * cs;
        l.t = z * sn;
        l.cs = cs;
        l.sn = sn;
        l.bstep += l.snprod * cs * z;
        l.snprod *= sn;
        l.rhs1 = l.rhs2 - delta * z;
        l.rhs2 = -epsln * z;
      }
      sst->iter += 1;
      const double cg = l.gbar != 0.0 ? fabs(l.snprod * m.beta1 * bnew / l.gbar) : (bnew == 0.0 ? 0.0 : INFINITY);
      sst->rr = cg * cg;  // CG-point residual norm estimate, squared
      if (!isfinite(yy) || !isfinite(l.rhs1)) {
        sst->status = 5;
        sst->done = 1;
      } else if (cg * cg <= sst->tol2 || bnew == 0.0) {
        l.zbar = l.gbar != 0.0 ? l.rhs1 / l.gbar : 0.0;
        l.cb = (l.bstep + l.snprod * l.zbar) / m.beta1;
        l.pending = 1;
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_sq_c(double* __restrict__ x, double* __restrict__ w,
                                                   const double* __restrict__ b, const double* __restrict__ r1,
                                                   long long n, SolverState* __restrict__ st,
                                                   const MinresScalars* __restrict__ ms,
                                                   const SymmlqScalars* __restrict__ sq, double* __restrict__ partials) {
  const int s = blockIdx.y;
  SolverState* sst = st + s;
  if (sst->done) return;
  const SymmlqScalars l = sq[s];
  const double iv = 1.0 / ms[s].oldb;  // v = r1 / oldb (r1 holds the previous r2)
  double* xs = x + s * n;
  double* ws = w + s * n;
  const double* bs = b + s * n;
  const double* r1s = r1 + s * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = r1s[i] * iv, wo = ws[i];
    const double wn = l.sn * wo - l.cs * v;
    double xv = xs[i] + l.s * wo + l.t * v;
    if (l.pending) xv += l.zbar * wn + l.cb * bs[i];
    xs[i] = xv;
    ws[i] = wn;
  }
  double* part = partials + (long long)s * gridDim.x;
  if (publish_partial_sys(part, blockIdx.x, gridDim.x, 0.0, &sst->counter[3])) {
    gather_partials_sys(part, gridDim.x, &sst->counter[3]);
    if (threadIdx.x == 0 && l.pending) sst->done = 1;
  }
}

__global__ void k_sq_begin(SymmlqScalars* __restrict__ sq, int S) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) sq[s] = SymmlqScalars{};
}

// Basic fixed-point scheme (Moulinec-Suquet): with r = b - K tau, the update
// tau += (A - A0) r equals tau_new = (A - A0)(b - Gamma tau), the classic
// iteration written on the polarisation.  Grid (G, S); systems whose flag is
// set (converged) are left alone.
__global__ void __launch_bounds__(kThreads) k_basic_update(OpArgs<double> a, double* __restrict__ x,
                                                           const double* __restrict__ r,
                                                           const unsigned char* __restrict__ flags) {
  const int s = blockIdx.y;
  if (flags[s]) return;
  const long long n = (long long)a.c * a.V;
  const long long pbase = (long long)((a.sys0 + s) / a.sys_per_ms) * a.V;
  double* xs = x + s * n;
  const double* rs = r + s * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int comp = (int)(i / a.V);
    const long long vox = i - (long long)comp * a.V;
    const int p = a.phase[pbase + vox];
    if (!a.act[p]) continue;
    double d;
    if (a.scale && a.frac) {
      const double f = (double)a.scale[pbase + vox];
      d = 1.0 / (f * a.mtab[a.c + comp] + (1.0 - f) * a.mtab[comp]);  // inverse of the averaged M
    } else {
      double mod = a.modtab[p * a.c + comp];
      if (a.scale) mod *= (double)a.scale[pbase + vox];
      d = mod - a.ref[comp];
    }
    xs[i] += d * rs[i];
  }
}

// Start: beta1 = |r0| (the right-hand side of this MINRES run: b, or b - K x0
// for a warm start), zero recurrence scalars; the tolerance is relative to |b|.
__global__ void k_mr_begin(SolverState* __restrict__ st, MinresScalars* __restrict__ ms,
                           const double* __restrict__ rhs2, const double* __restrict__ bb, double tol, int S) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  SolverState& t = st[s];
  t = SolverState{};
  MinresScalars& m = ms[s];
  m = MinresScalars{};
  const double b1 = sqrt(fmax(rhs2[s], 0.0));
  m.beta1 = b1;
  m.beta = b1;
  m.phibar = b1;
  m.cs = -1.0;
  t.bb = bb[s];
  t.tol2 = tol * tol * bb[s];
  t.rr = rhs2[s];
  if (!(b1 > 0.0) || rhs2[s] <= t.tol2) t.done = 1;
}

// ------------------------------------------------------------------ CG vector kernels
// Grid (G, S): blockIdx.y is the system, n the elements per system.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_update(T* __restrict__ r, const T* __restrict__ q, long long n,
                                                        SolverState* __restrict__ st, double* __restrict__ partials) {
  const int s = blockIdx.y;
  SolverState* sst = st + s;
  if (sst->done) return;
  const T al = (T)sst->alpha;
  T* rs = r + s * n;
  const T* qs = q + s * n;
  Acc<T> acc;
  constexpr int VEC = 16 / sizeof(T);
  // 16-byte accesses only when every system's range starts on a 16-byte boundary
  const long long nv = (n % VEC == 0) ? n / VEC : 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
    T rv[VEC], qv[VEC];
    vload<T, VEC>(rs + i * VEC, rv);
    vload<T, VEC>(qs + i * VEC, qv);
#pragma unroll
    for (int u = 0; u < VEC; ++u) {
      rv[u] -= al * qv[u];
      acc.add(rv[u] * rv[u]);
    }
    vstore<T, VEC>(rs + i * VEC, rv);
  }
  for (long long i = nv * VEC + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T rv = rs[i] - al * qs[i];
    rs[i] = rv;
    acc.add(rv * rv);
  }
  const double tot = block_reduce(acc);
  double* part = partials + (long long)s * gridDim.x;
  if (publish_partial_sys(part, blockIdx.x, gridDim.x, tot, &sst->counter[1])) {
    const double rrn = gather_partials_sys(part, gridDim.x, &sst->counter[1]);
    if (threadIdx.x == 0) {
      sst->beta = rrn / sst->rr;
      sst->rr = rrn;
      sst->iter += 1;
      if (!isfinite(rrn)) {
        sst->status = 5;
        sst->done = 1;
      } else if (rrn <= sst->tol2) {
        sst->done = 1;
      }
    }
  }
}

template <typename T>
__global__ void k_cg_finalize(T* __restrict__ x, const T* __restrict__ p, long long n,
                              const SolverState* __restrict__ st) {
  const int s = blockIdx.y;
  const double al = st[s].alpha;
  if (al == 0.0) return;
  const T a = (T)al;
  T* xs = x + s * n;
  const T* ps = p + s * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    xs[i] += a * ps[i];
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_cg_begin(const T* __restrict__ r, long long n,
                                                       SolverState* __restrict__ st, double* __restrict__ partials,
                                                       double tol, const double* __restrict__ bb_given) {
  const int s = blockIdx.y;
  const T* rs = r + s * n;
  Acc<T> acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc.add(rs[i] * rs[i]);
  const double tot = block_reduce(acc);
  double* part = partials + (long long)s * gridDim.x;
  SolverState* sst = st + s;
  if (publish_partial_sys(part, blockIdx.x, gridDim.x, tot, &sst->counter[2])) {
    const double rr = gather_partials_sys(part, gridDim.x, &sst->counter[2]);
    if (threadIdx.x == 0) {
      const double bb = bb_given != nullptr ? bb_given[s] : rr;
      sst->rr = rr;
      sst->bb = bb;
      sst->tol2 = tol * tol * bb;
      sst->alpha = 0.0;
      sst->beta = 0.0;
      sst->pq = 0.0;
      sst->iter = 0;
      sst->status = 0;
      sst->done = (rr <= sst->tol2) ? 1 : 0;
    }
  }
}

// r = b (load on I0, 0 elsewhere), x = 0.  Grid (G, S).
template <typename T>
__global__ void k_fill_rhs(OpArgs<T> a, T* __restrict__ r, T* __restrict__ x) {
  const int s = blockIdx.y;
  const long long n = (long long)a.c * a.V;
  const long long pbase = (long long)((a.sys0 + s) / a.sys_per_ms) * a.V;
  T* rs = r + s * n;
  T* xs = x + s * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int comp = (int)(i / a.V);
    const long long vox = i - comp * a.V;
    rs[i] = a.act[a.phase[pbase + vox]] ? a.loads[s * 6 + comp] : (T)0;
    xs[i] = (T)0;
  }
}

// Internal basis <-> Mandel for the three normal components (shear unchanged):
// h = (e11+e22+e33)/sqrt3, d1 = (e11-e22)/sqrt2, d2 = (e11+e22-2 e33)/sqrt6.
template <typename T>
__global__ void k_rotate(const T* in, T* out, long long V, long long nvox, int to_internal) {
  const double s3 = 0.57735026918962576450914878050195745565;   // 1/sqrt3
  const double s2 = 0.70710678118654752440084436210484903928;   // 1/sqrt2
  const double s6 = 0.40824829046386301636621401245098189866;   // 1/sqrt6
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nvox; q += (long long)gridDim.x * blockDim.x) {
    const long long sys = q / V, v = q - sys * V;
    const T* i0 = in + sys * 6 * V;
    T* o0 = out + sys * 6 * V;
    const double a0 = i0[v], a1 = i0[V + v], a2 = i0[2 * V + v];
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
    o0[v] = (T)b0;
    o0[V + v] = (T)b1;
    o0[2 * V + v] = (T)b2;
    if (in != out)
      for (int k = 3; k < 6; ++k) o0[k * V + v] = i0[k * V + v];
  }
}

// Scalar fields between the caller's axes and the common eigenbasis of the
// reference and phase tensors: u_int = R^T u (to_internal) or u = R u_int.
struct Rot3 {
  double r[9];
};
template <typename T>
__global__ void k_rotate_scalar(const T* in, T* out, long long V, long long nvox, int d, Rot3 R, int to_internal) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nvox; q += (long long)gridDim.x * blockDim.x) {
    const long long sys = q / V, v = q - sys * V;
    const T* i0 = in + sys * d * V;
    T* o0 = out + sys * d * V;
    double a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    for (int i = 0; i < d; ++i) a[i] = i0[i * V + v];
    for (int i = 0; i < d; ++i)
      for (int k = 0; k < d; ++k) b[i] += (to_internal ? R.r[k * d + i] : R.r[i * d + k]) * a[k];
    for (int i = 0; i < d; ++i) o0[i * V + v] = (T)b[i];
  }
}

// Per-system, per-component sums, deterministic: partials[(s c + comp) nblk + blk].
template <typename T>
__global__ void __launch_bounds__(kThreads) k_comp_partials(const T* __restrict__ x, long long V, int c,
                                                            double* __restrict__ partials) {
  const int comp = blockIdx.y, s = blockIdx.z;
  const T* xc = x + ((long long)s * c + comp) * V;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x)
    acc += (double)xc[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[((long long)s * c + comp) * gridDim.x + blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) k_comp_final(const double* __restrict__ partials, int nblk,
                                                         double* __restrict__ out) {
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += partials[(long long)j * nblk + i];
  s = block_sum(s);
  if (threadIdx.x == 0) out[j] = s;
}

// ------------------------------------------------------------------ Gamma^h table
// Continuous Green operator of the reference medium (Sec. 2.2.1) at a nonzero
// frequency xi, in the component basis of the problem (Mandel for elasticity).
struct GammaCtx {
  int dim, physics, green, c;
  int n[3];
  double ref[6];  // scalar: diagonal of A0 in the internal basis; elastic: (K0, mu0)
  // scalar problems in a rotated basis: the full A0 and the rotation R (columns =
  // internal basis vectors); the table then holds R^T Gamma R
  int rotated;
  double A0[9];
  double R[9];
};

__device__ void gamma0_acc(const GammaCtx& g, const double xi[3], double w, double* G) {
  if (g.physics == 0) {
    double q = 0.0;
    if (g.rotated) {
      for (int i = 0; i < g.dim; ++i)
        for (int j = 0; j < g.dim; ++j) q += g.A0[i * g.dim + j] * xi[i] * xi[j];
    } else {
      for (int i = 0; i < g.dim; ++i) q += g.ref[i] * xi[i] * xi[i];
    }
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
  const int ncop = ((g.c * (g.c + 1) / 2) + 3) & ~3;  // coefficients per frequency, padded
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
    } else if (g.green == 2) {
      // finite differences, Sec. 3.2.3 (scalar): V V^H / (V^H A0 V) with
      // V_i = exp(2 i pi k_i / N_i) - 1 = i exp(i pi k_i / N_i) u_i,
      // u_i = 2 sin(pi k_i / N_i).  For diagonal A0 this is D (u u^T / u^T A0 u) D^H
      // with D = diag(i exp(i pi k_i / N_i)): the table holds the real middle factor,
      // the z pass applies the phases.
      double u[3] = {0, 0, 0};
      double q = 0.0;
      for (int i = 0; i < g.dim; ++i) {
        u[i] = 2.0 * sinpi((double)k[i] / g.n[i]);
        q += g.ref[i] * u[i] * u[i];
      }
      if (q > 0.0)
        for (int i = 0; i < c; ++i)
          for (int j = 0; j < c; ++j) G[i * c + j] = u[i] * u[j] / q;
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
    } else if (g.physics == 0 && g.rotated) {
      // R^T G R: the operator in the common eigenbasis of A0 and the phases
      for (int i = 0; i < c; ++i)
        for (int j = 0; j < c; ++j) {
          double s = 0.0;
          for (int p = 0; p < c; ++p)
            for (int q = 0; q < c; ++q) s += g.R[p * c + i] * G[p * c + q] * g.R[q * c + j];
          Gi[i * c + j] = s;
        }
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
    int coef = 0;
    T* out = const_cast<T*>(a.gtab);
    const long long fi = ((long long)zp * a.ny + yp) * a.ts + kx;
    for (int i = 0; i < c; ++i)
      for (int j = i; j < c; ++j, ++coef)
        out[gamma_elem<T>(fi, coef, ncop)] = (T)(0.5 * (Gi[i * c + j] + Gi[j * c + i]) * invV);
    for (; coef < ncop; ++coef) out[gamma_elem<T>(fi, coef, ncop)] = (T)0;
  }
}

// ------------------------------------------------------------------ mixed precision helpers
// r32 = (float) r64, x32 = 0, inner CG state begun with tolerance tol relative
// to the new right-hand side; systems with active[s] == 0 start done.
// DFIN: r64's elements hold double-float pairs (h, l); the FP32 residual is h
template <bool DFIN>
__global__ void __launch_bounds__(kThreads) k_d2f_begin(const double* __restrict__ r64, float* __restrict__ r32,
                                                        float* __restrict__ x32, long long n,
                                                        SolverState* __restrict__ st, double* __restrict__ partials,
                                                        double tol, const unsigned char* __restrict__ active) {
  const int s = blockIdx.y;
  const double* r64s = r64 + s * n;
  float* r32s = r32 + s * n;
  float* x32s = x32 + s * n;
  Acc<float> acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = DFIN ? reinterpret_cast<const float2*>(r64s)[i].x : (float)r64s[i];
    r32s[i] = v;
    x32s[i] = 0.0f;
    acc.add(v * v);
  }
  const double tot = block_reduce(acc);
  double* part = partials + (long long)s * gridDim.x;
  SolverState* sst = st + s;
  if (publish_partial_sys(part, blockIdx.x, gridDim.x, tot, &sst->counter[2])) {
    const double rr = gather_partials_sys(part, gridDim.x, &sst->counter[2]);
    if (threadIdx.x == 0) {
      sst->rr = rr;
      sst->bb = rr;
      sst->tol2 = tol * tol * rr;
      sst->alpha = sst->beta = sst->pq = 0.0;
      sst->iter = 0;
      sst->status = 0;
      sst->done = (!active[s] || rr <= sst->tol2) ? 1 : 0;
    }
  }
}

__global__ void k_f2d_axpy(double* __restrict__ x64, const float* __restrict__ x32, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x64[i] += (double)x32[i];
}

// Phase scan at setup, grid (G, B): voxels in I0 per microstructure (st[b].aux[1])
// and the largest phase id (st[0].pad via atomicMax).
__global__ void __launch_bounds__(kThreads) k_scan_phase(const unsigned char* __restrict__ phase, long long V,
                                                         const unsigned char* __restrict__ act, int nphase,
                                                         SolverState* __restrict__ st, double* __restrict__ partials) {
  const int b = blockIdx.y;
  const unsigned char* ph = phase + (long long)b * V;
  double cnt = 0.0;
  int mx = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    const int p = ph[i];
    mx = max(mx, p);
    if (p < nphase && act[p]) cnt += 1.0;
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(&st[0].pad, mx);
  cnt = block_sum(cnt);
  double* part = partials + (long long)b * gridDim.x;
  if (publish_partial_sys(part, blockIdx.x, gridDim.x, cnt, &st[b].counter[3])) {
    const double tot = gather_partials_sys(part, gridDim.x, &st[b].counter[3]);
    if (threadIdx.x == 0) st[b].aux[1] = tot;
  }
}

// Scale gradient, grid (G, B): g = (1/V) sum_ij W_ij eps_i . A_phase eps_j with
// eps_j = M tau_j (internal basis, where M and A_phase are diagonal); tau_all is
// [B][c loads][c][V] in Mandel components.
__global__ void k_scale_grad(const double* __restrict__ tau_all, const double* __restrict__ W,
                             const unsigned char* __restrict__ phase, const float* __restrict__ scale,
                             const double* __restrict__ modtab, const double* __restrict__ ref, int c, int elastic,
                             long long V, double* __restrict__ grad) {
  const double s3 = 0.57735026918962576450914878050195745565, s2 = 0.70710678118654752440084436210484903928,
               s6 = 0.40824829046386301636621401245098189866;
  const int b = blockIdx.y;
  const double* tau_b = tau_all + (long long)b * c * c * V;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const long long pv = (long long)b * V + v;
    const int ph = phase[pv];
    const double s = scale ? (double)scale[pv] : 1.0;
    double A[6], m[6];
    for (int k = 0; k < c; ++k) {
      A[k] = modtab[ph * c + k];
      m[k] = 1.0 / (s * A[k] - ref[k]);
    }
    double eps[6][6];
    for (int j = 0; j < c; ++j) {
      const double* tj = tau_b + (long long)j * c * V;
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
    grad[pv] = gsum / (double)V;
  }
}

// ------------------------------------------------------------------ launchers
// The attribute is a per-function upper bound shared by every handle: always
// allow the full 227 KB so that one handle never shrinks another's limit.
template <typename T> void set_smem_attrs() {
  const int mx = 227 * 1024;
  constexpr int VV = 16 / sizeof(T);
  cudaFuncSetAttribute(k_xinv<T, 3, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv<T, 3, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xfwd<T, 0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xfwd<T, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xfwd<T, 0, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xfwd<T, 1, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv<T, 0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv<T, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv<T, 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv<T, 0, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv<T, 1, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv<T, 2, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_yfft<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_yfft<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_zgamma<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_zgamma<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_zgamma<T, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  set_smem_attrs_reg<T>();
}

template <typename T>
void launch_xfwd(const OpArgs<T>& a, const LaunchCfg& L, int mode, const T* in, T* x, const T* r, T* p,
                 const SolverState* st, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (a.plane && launch_xyfwd(a, mode, in, x, r, p, st, s)) return;
    if (a.xfreg && launch_xfwd_reg(a, mode, in, x, r, p, st, s)) return;
  }
  const int grid = a.S * a.bps;
  constexpr int VV = 16 / sizeof(T);
  if (L.VEC == VV) {
    if (mode == 0) k_xfwd<T, 0, VV><<<grid, L.threads, L.smem_x, s>>>(a, in, x, r, p, st);
    else k_xfwd<T, 1, VV><<<grid, L.threads, L.smem_x, s>>>(a, in, x, r, p, st);
  } else {
    if (mode == 0) k_xfwd<T, 0, 1><<<grid, L.threads, L.smem_x, s>>>(a, in, x, r, p, st);
    else k_xfwd<T, 1, 1><<<grid, L.threads, L.smem_x, s>>>(a, in, x, r, p, st);
  }
}

template <typename T>
void launch_yfft(const OpArgs<T>& a, const LaunchCfg& L, bool inv, const SolverState* st, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (a.plane) return;  // the plane passes transform y
    if (a.ytma) {
      launch_yfft_tma(a, inv, st, s);
      return;
    }
  }
  if (a.yreg) {
    launch_yfft_reg<T>(a, inv, st, s);
    return;
  }
  dim3 g(L.grid_yx, a.S * a.c * a.nz);
  if (inv) k_yfft<T, true><<<g, L.threads, L.smem_y, s>>>(a, st);
  else k_yfft<T, false><<<g, L.threads, L.smem_y, s>>>(a, st);
}

template <typename T>
void launch_zgamma(const OpArgs<T>& a, const LaunchCfg& L, const SolverState* st, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    // the TMA variants read the x-major layout only
    if (!a.tlay && a.ztma >= 1 && a.ztma <= 5 && launch_zgamma_tma(a, a.ztma, st, s)) return;
    if (a.ztma == 7 && launch_zgamma_regp(a, st, s)) return;
    if ((a.ztma == 10 || a.ztma == 11) && launch_zgamma_pipe(a, a.ztma == 11, st, s)) return;
  }
  if (a.zreg) {
    int tz = 0;
    if (sizeof(T) == 4) tz = a.ztma == 6 ? 4 : a.ztma == 8 ? 16 : a.ztma == 9 ? -1 : 0;
    launch_zgamma_reg<T>(a, st, s, tz);
    return;
  }
  dim3 g(a.S, L.grid_zx, L.grid_zy);
  if (a.c == 6) k_zgamma<T, 6><<<g, L.threads, L.smem_z, s>>>(a, st);
  else if (a.c == 3) k_zgamma<T, 3><<<g, L.threads, L.smem_z, s>>>(a, st);
  else k_zgamma<T, 2><<<g, L.threads, L.smem_z, s>>>(a, st);
}

template <typename T>
void launch_xinv(const OpArgs<T>& a, const LaunchCfg& L, int mode, const T* xin, T* out, SolverState* st,
                 double* partials, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (a.plane && mode <= 1 && launch_xyinv(a, mode, xin, out, st, partials, s)) return;
    if (a.xreg && mode <= 2 && launch_xinv_reg(a, mode, xin, out, st, partials, s, a.xreg == 2, a.xreg == 3)) return;
  }
  const int grid = a.S * a.bps;
  constexpr int VV = 16 / sizeof(T);
  if (L.VEC == VV) {
    if (mode == 0) k_xinv<T, 0, VV><<<grid, L.threads, L.smem_x, s>>>(a, xin, out, st, partials);
    else if (mode == 1) k_xinv<T, 1, VV><<<grid, L.threads, L.smem_x, s>>>(a, xin, out, st, partials);
    else if (mode == 3) k_xinv<T, 3, VV><<<grid, L.threads, L.smem_x, s>>>(a, xin, out, st, partials);
    else k_xinv<T, 2, VV><<<grid, L.threads, L.smem_x, s>>>(a, xin, out, st, partials);
  } else {
    if (mode == 0) k_xinv<T, 0, 1><<<grid, L.threads, L.smem_x, s>>>(a, xin, out, st, partials);
    else if (mode == 1) k_xinv<T, 1, 1><<<grid, L.threads, L.smem_x, s>>>(a, xin, out, st, partials);
    else if (mode == 3) k_xinv<T, 3, 1><<<grid, L.threads, L.smem_x, s>>>(a, xin, out, st, partials);
    else k_xinv<T, 2, 1><<<grid, L.threads, L.smem_x, s>>>(a, xin, out, st, partials);
  }
}

void launch_dot_finalize(SolverState* st, const double* partials, int nb, int S, cudaStream_t s) {
  k_dot_finalize<<<S, kThreads, 0, s>>>(st, partials, nb);
}

void launch_basic_update(const OpArgs<double>& a, double* x, const double* r, const unsigned char* flags, int G,
                         cudaStream_t s) {
  k_basic_update<<<dim3(G, a.S), kThreads, 0, s>>>(a, x, r, flags);
}

void launch_minres_begin(SolverState* st, MinresScalars* ms, const double* rhs2, const double* bb, double tol, int S,
                         cudaStream_t s) {
  k_mr_begin<<<(S + 127) / 128, 128, 0, s>>>(st, ms, rhs2, bb, tol, S);
}
void launch_symmlq_begin(SymmlqScalars* sq, int S, cudaStream_t s) { k_sq_begin<<<(S + 127) / 128, 128, 0, s>>>(sq, S); }

void launch_symmlq_step(double* x, double* r1, double* r2, double* q, double* w, const double* b, long long n, int S,
                        SolverState* st, MinresScalars* ms, SymmlqScalars* sq, double* partials, int G,
                        cudaStream_t s) {
  k_mr_a<<<dim3(G, S), kThreads, 0, s>>>(q, r1, r2, n, st, ms, partials);
  k_sq_b<<<dim3(G, S), kThreads, 0, s>>>(q, r1, r2, n, st, ms, sq, partials);
  k_sq_c<<<dim3(G, S), kThreads, 0, s>>>(x, w, b, r1, n, st, ms, sq, partials);
}

void launch_minres_step(double* x, double* r1, double* r2, double* q, double* wa, double* wb, long long n, int S,
                        SolverState* st, MinresScalars* ms, double* partials, int G, cudaStream_t s) {
  k_mr_a<<<dim3(G, S), kThreads, 0, s>>>(q, r1, r2, n, st, ms, partials);
  k_mr_b<<<dim3(G, S), kThreads, 0, s>>>(q, r1, r2, n, st, ms, partials);
  k_mr_c<<<dim3(G, S), kThreads, 0, s>>>(x, wa, wb, r1, n, st, ms, partials);
}

template <typename T>
void launch_rotate_scalar(const T* in, T* out, long long V, int nsys, int d, const double* R, int to_internal,
                          cudaStream_t s) {
  Rot3 r;
  for (int i = 0; i < 9; ++i) r.r[i] = R[i];
  const long long nvox = V * nsys;
  const int grid = (int)std::max(1LL, std::min((nvox + 255) / 256, 152LL * 8));
  k_rotate_scalar<T><<<grid, 256, 0, s>>>(in, out, V, nvox, d, r, to_internal);
}

template <typename T>
void launch_cg_update(T* r, const T* q, long long n, int S, SolverState* st, double* partials, int G, cudaStream_t s) {
  k_cg_update<T><<<dim3(G, S), kThreads, 0, s>>>(r, q, n, st, partials);
}
template <typename T>
void launch_cg_finalize(T* x, const T* p, long long n, int S, const SolverState* st, int G, cudaStream_t s) {
  k_cg_finalize<T><<<dim3(G, S), kThreads, 0, s>>>(x, p, n, st);
}
template <typename T>
void launch_cg_begin(const T* r, long long n, int S, SolverState* st, double* partials, double tol,
                     const double* bb_given, int G, cudaStream_t s) {
  k_cg_begin<T><<<dim3(G, S), kThreads, 0, s>>>(r, n, st, partials, tol, bb_given);
}
template <typename T> void launch_fill_rhs(const OpArgs<T>& a, T* r, T* x, int G, cudaStream_t s) {
  k_fill_rhs<T><<<dim3(G, a.S), kThreads, 0, s>>>(a, r, x);
}
template <typename T> void launch_rotate(const T* in, T* out, long long V, int nsys, int to_internal, cudaStream_t s) {
  const long long nvox = V * nsys;
  const int grid = (int)std::max(1LL, std::min((nvox + kThreads - 1) / kThreads, 152LL * 16));
  k_rotate<T><<<grid, kThreads, 0, s>>>(in, out, V, nvox, to_internal);
}
template <typename T>
void launch_comp_sums(const T* x, int c, long long V, int S, double* partials, int nblk, double* out, cudaStream_t s) {
  k_comp_partials<T><<<dim3(nblk, c, S), kThreads, 0, s>>>(x, V, c, partials);
  k_comp_final<<<c * S, kThreads, 0, s>>>(partials, nblk, out);
}
template <typename T>
void launch_gamma_table(const OpArgs<T>& a, int dim, int physics, int green, const double* ref_mandel,
                        const int* kofy, const int* kofz, cudaStream_t s, const double* a0full, const double* rot) {
  GammaCtx g;
  g.rotated = (a0full && rot) ? 1 : 0;
  for (int i = 0; i < 9; ++i) {
    g.A0[i] = g.rotated ? a0full[i] : 0.0;
    g.R[i] = g.rotated ? rot[i] : 0.0;
  }
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
void launch_d2f_begin(const double* r64, bool df_pairs, float* r32, float* x32, long long n, int S, SolverState* st,
                      double* partials, double tol, const unsigned char* active, int G, cudaStream_t s) {
  if (df_pairs) k_d2f_begin<true><<<dim3(G, S), kThreads, 0, s>>>(r64, r32, x32, n, st, partials, tol, active);
  else k_d2f_begin<false><<<dim3(G, S), kThreads, 0, s>>>(r64, r32, x32, n, st, partials, tol, active);
}
void launch_f2d_axpy(double* x64, const float* x32, long long n, cudaStream_t s) {
  const int grid = (int)std::max(1LL, std::min((n + kThreads - 1) / kThreads, 152LL * 16));
  k_f2d_axpy<<<grid, kThreads, 0, s>>>(x64, x32, n);
}
void launch_scan_phase(const unsigned char* phase, long long V, int B, const unsigned char* act, int nphase,
                       SolverState* st, double* partials, int G, cudaStream_t s) {
  k_scan_phase<<<dim3(G, B), kThreads, 0, s>>>(phase, V, act, nphase, st, partials);
}
void launch_scale_grad(const double* tau_all, const double* W, const unsigned char* phase, const float* scale,
                       const double* modtab, const double* ref, int c, int elastic, long long V, int B,
                       double* grad, cudaStream_t s) {
  const int G = (int)std::max(1LL, std::min((V + 127) / 128, 152LL * 8));
  k_scale_grad<<<dim3(G, B), 128, 0, s>>>(tau_all, W, phase, scale, modtab, ref, c, elastic, V, grad);
}

#define LSH_INSTANTIATE(T)                                                                                         \
  template void set_smem_attrs<T>();                                                                               \
  template void launch_xfwd<T>(const OpArgs<T>&, const LaunchCfg&, int, const T*, T*, const T*, T*,                \
                               const SolverState*, cudaStream_t);                                                  \
  template void launch_yfft<T>(const OpArgs<T>&, const LaunchCfg&, bool, const SolverState*, cudaStream_t);        \
  template void launch_zgamma<T>(const OpArgs<T>&, const LaunchCfg&, const SolverState*, cudaStream_t);            \
  template void launch_xinv<T>(const OpArgs<T>&, const LaunchCfg&, int, const T*, T*, SolverState*, double*,       \
                               cudaStream_t);                                                                      \
  template void launch_cg_update<T>(T*, const T*, long long, int, SolverState*, double*, int, cudaStream_t);       \
  template void launch_cg_finalize<T>(T*, const T*, long long, int, const SolverState*, int, cudaStream_t);        \
  template void launch_cg_begin<T>(const T*, long long, int, SolverState*, double*, double, const double*, int,    \
                                   cudaStream_t);                                                                  \
  template void launch_fill_rhs<T>(const OpArgs<T>&, T*, T*, int, cudaStream_t);                                   \
  template void launch_rotate<T>(const T*, T*, long long, int, int, cudaStream_t);                                 \
  template void launch_comp_sums<T>(const T*, int, long long, int, double*, int, double*, cudaStream_t);           \
  template void launch_gamma_table<T>(const OpArgs<T>&, int, int, int, const double*, const int*, const int*,      \
                                      cudaStream_t, const double*, const double*);                                 \
  template void launch_rotate_scalar<T>(const T*, T*, long long, int, int, const double*, int, cudaStream_t);

LSH_INSTANTIATE(double)
LSH_INSTANTIATE(float)

}  // namespace lsh
