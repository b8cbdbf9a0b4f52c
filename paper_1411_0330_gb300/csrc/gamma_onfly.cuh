// gamma_onfly.cuh -- the discrete Green operator applied at one frequency
// inside the z pass: from the tabulated symmetric coefficients, or for the
// truncated operator evaluated on the fly; shared by the z-pass kernels.
#pragma once

#include "common.cuh"
#include "df.cuh"
#include "internal.h"

namespace lsh {

// Truncated Green operator at one frequency, computed in place on the c
// components of the internal basis (Eqs. (14)-(15) and the Nyquist rule of
// Sec. 3.2.1), scaled by 1/V.  Used for FP32, where it is cheaper than
// reading the tabulated coefficients.
template <typename T, int NC>
__device__ __forceinline__ void gamma_trunc_onfly(const OpArgs<T>& a, int kx, int ky, int kz, C2<T>* v) {
  const int kk[3] = {kx, ky, kz};
  const int nn[3] = {a.nx, a.ny, a.nz};
  T xi[3];
  bool zero = true, nyq = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int ki = kk[i] <= nn[i] / 2 ? kk[i] : kk[i] - nn[i];
    if ((nn[i] & 1) == 0 && kk[i] == nn[i] / 2 && nn[i] > 1) nyq = true;
    xi[i] = (T)ki;
    if (ki != 0) zero = false;
  }
  if (zero) {
#pragma unroll
    for (int i = 0; i < NC; ++i) v[i] = mkc<T>(0, 0);
    return;
  }
  if (NC != 6) {
    // scalar: xi (xi . v) / (xi^T A0 xi), or A0^{-1} v at the Nyquist frequencies
    if (nyq) {
#pragma unroll
      for (int i = 0; i < NC; ++i) v[i] = cscale<T>(v[i], a.invV / a.g0[i]);
      return;
    }
    T q = 0;
    C2<T> d = mkc<T>(0, 0);
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      q += a.g0[i] * xi[i] * xi[i];
      d.x += xi[i] * v[i].x;
      d.y += xi[i] * v[i].y;
    }
    const T f = a.invV / q;
#pragma unroll
    for (int i = 0; i < NC; ++i) v[i] = mkc<T>(f * xi[i] * d.x, f * xi[i] * d.y);
    return;
  }
  if (nyq) {
    // C0^{-1}: diagonal in the internal basis
    v[0] = cscale<T>(v[0], a.g0[2]);
#pragma unroll
    for (int i = 1; i < 6; ++i) v[i] = cscale<T>(v[i], a.g0[3]);
    return;
  }
  const T s3 = (T)0.57735026918962576450914878050195745565, s2 = (T)0.70710678118654752440084436210484903928,
          s6 = (T)0.40824829046386301636621401245098189866;
  const T rn = (T)1 / sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
  const T n0 = xi[0] * rn, n1 = xi[1] * rn, n2 = xi[2] * rn;
  // internal -> tensor components (t11, t22, t33, t23, t13, t12)
  C2<T> t11, t22, t33, t23, t13, t12;
  t11 = mkc<T>(v[0].x * s3 + v[1].x * s2 + v[2].x * s6, v[0].y * s3 + v[1].y * s2 + v[2].y * s6);
  t22 = mkc<T>(v[0].x * s3 - v[1].x * s2 + v[2].x * s6, v[0].y * s3 - v[1].y * s2 + v[2].y * s6);
  t33 = mkc<T>(v[0].x * s3 - (T)2 * v[2].x * s6, v[0].y * s3 - (T)2 * v[2].y * s6);
  t23 = cscale<T>(v[3], s2);
  t13 = cscale<T>(v[4], s2);
  t12 = cscale<T>(v[5], s2);
  // Tn and n.Tn
  const C2<T> u0 = mkc<T>(t11.x * n0 + t12.x * n1 + t13.x * n2, t11.y * n0 + t12.y * n1 + t13.y * n2);
  const C2<T> u1 = mkc<T>(t12.x * n0 + t22.x * n1 + t23.x * n2, t12.y * n0 + t22.y * n1 + t23.y * n2);
  const C2<T> u2 = mkc<T>(t13.x * n0 + t23.x * n1 + t33.x * n2, t13.y * n0 + t23.y * n1 + t33.y * n2);
  const C2<T> w = mkc<T>(n0 * u0.x + n1 * u1.x + n2 * u2.x, n0 * u0.y + n1 * u1.y + n2 * u2.y);
  const T a1 = a.g0[0], a2 = a.g0[1];
  // S_ij = a1 (u_i n_j + n_i u_j) - a2 w n_i n_j
#define LSH_SIJ(ui, nj, ni, uj, nij) \
  mkc<T>(a1 * (ui.x * nj + ni * uj.x) - a2 * w.x * nij, a1 * (ui.y * nj + ni * uj.y) - a2 * w.y * nij)
  const C2<T> S11 = LSH_SIJ(u0, n0, n0, u0, n0 * n0);
  const C2<T> S22 = LSH_SIJ(u1, n1, n1, u1, n1 * n1);
  const C2<T> S33 = LSH_SIJ(u2, n2, n2, u2, n2 * n2);
  const C2<T> S23 = LSH_SIJ(u1, n2, n1, u2, n1 * n2);
  const C2<T> S13 = LSH_SIJ(u0, n2, n0, u2, n0 * n2);
  const C2<T> S12 = LSH_SIJ(u0, n1, n0, u1, n0 * n1);
#undef LSH_SIJ
  // tensor -> internal basis (Mandel shear components carry sqrt 2)
  const T r2 = (T)1.41421356237309504880168872420969807857;
  v[0] = mkc<T>((S11.x + S22.x + S33.x) * s3, (S11.y + S22.y + S33.y) * s3);
  v[1] = mkc<T>((S11.x - S22.x) * s2, (S11.y - S22.y) * s2);
  v[2] = mkc<T>((S11.x + S22.x - (T)2 * S33.x) * s6, (S11.y + S22.y - (T)2 * S33.y) * s6);
  v[3] = cscale<T>(S23, r2);
  v[4] = cscale<T>(S13, r2);
  v[5] = cscale<T>(S12, r2);
}

// Finite-difference operator: rotate component i (axis i) by sign * pi k_i / N_i
// (k unsigned, as in the table), before (sign -1) and after (+1) the real table.
template <typename T, int NC>
__device__ __forceinline__ void fd_rotate(const OpArgs<T>& a, int kx, int ky, int kz, C2<T>* v, T sign) {
  if constexpr (NC == 6) return;  // scalar operator only: nothing in the elastic kernels
  const int kk[3] = {kx, ky, kz};
  const int nn[3] = {a.nx, a.ny, a.nz};
#pragma unroll
  for (int i = 0; i < NC && i < 3; ++i) {
    T s, c;
    sincospi((T)kk[i] / (T)nn[i], &s, &c);
    s *= sign;
    v[i] = mkc<T>(c * v[i].x - s * v[i].y, s * v[i].x + c * v[i].y);
  }
}

// The Gamma^h table holds, per frequency f = (z position * ny + y position) *
// ts + kx (ts a multiple of 8), the c(c+1)/2 coefficients of the symmetric
// c x c matrix (packed upper triangle) padded to NCOP, a multiple of 4.  It is
// cut in blocks of 8 consecutive frequencies (f & ~7): inside a block, 16-byte
// vector q of frequency f & 7 sits at vector q * 8 + (f & 7).  Eight threads on
// consecutive kx then read one whole 128-byte line per vector load.
template <int NC> struct GammaPack {
  static constexpr int NCO = NC * (NC + 1) / 2;
  static constexpr int NCOP = (NCO + 3) & ~3;
};

// element index of coefficient `coef` of frequency f (ncop the padded count)
template <typename T> __host__ __device__ __forceinline__ long long gamma_elem(long long f, int coef, int ncop) {
  constexpr int VEC = 16 / (int)sizeof(T);
  return (f & ~7ll) * ncop + (long long)(coef / VEC) * (8 * VEC) + (f & 7) * VEC + coef % VEC;
}

template <typename T, int NC>
__device__ __forceinline__ void gamma_coef_load(const T* __restrict__ G, long long f, T* gc) {
  constexpr int NCO = GammaPack<NC>::NCO, NCOP = GammaPack<NC>::NCOP;
  if constexpr (is_df<T>::value) {
    // two double-float coefficients per 16-byte vector
    const float4* p = reinterpret_cast<const float4*>(G + (f & ~7ll) * NCOP) + (f & 7);
#pragma unroll
    for (int j = 0; j < NCOP / 2; ++j) {
      const float4 v = p[8 * j];
      if (2 * j + 0 < NCO) gc[2 * j + 0] = DF(v.x, v.y);
      if (2 * j + 1 < NCO) gc[2 * j + 1] = DF(v.z, v.w);
    }
  } else if constexpr (sizeof(T) == 4) {
    const float4* p = reinterpret_cast<const float4*>(G + (f & ~7ll) * NCOP) + (f & 7);
#pragma unroll
    for (int j = 0; j < NCOP / 4; ++j) {
      const float4 v = p[8 * j];
      if (4 * j + 0 < NCO) gc[4 * j + 0] = v.x;
      if (4 * j + 1 < NCO) gc[4 * j + 1] = v.y;
      if (4 * j + 2 < NCO) gc[4 * j + 2] = v.z;
      if (4 * j + 3 < NCO) gc[4 * j + 3] = v.w;
    }
  } else {
    const double2* p = reinterpret_cast<const double2*>(G + (f & ~7ll) * NCOP) + (f & 7);
#pragma unroll
    for (int j = 0; j < NCOP / 2; ++j) {
      const double2 v = p[8 * j];
      if (2 * j + 0 < NCO) gc[2 * j + 0] = v.x;
      if (2 * j + 1 < NCO) gc[2 * j + 1] = v.y;
    }
  }
}

// c x c symmetric product with coefficients already in registers, in place.
template <typename T, int NC> __device__ __forceinline__ void gamma_coef_apply(const T* gc, C2<T>* v) {
  C2<T> y[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) y[i] = mkc<T>(0, 0);
  int coef = 0;
#pragma unroll
  for (int i = 0; i < NC; ++i)
#pragma unroll
    for (int j = i; j < NC; ++j, ++coef) {
      const T g = gc[coef];
      y[i].x += g * v[j].x;
      y[i].y += g * v[j].y;
      if (j != i) {
        y[j].x += g * v[i].x;
        y[j].y += g * v[i].y;
      }
    }
#pragma unroll
  for (int i = 0; i < NC; ++i) v[i] = y[i];
}

// Gamma^h of frequency f applied to the c components of that frequency, in place.
template <typename T, int NC>
__device__ __forceinline__ void gamma_table_apply(const T* __restrict__ G, long long f, C2<T>* v) {
  T gc[GammaPack<NC>::NCO];
  gamma_coef_load<T, NC>(G, f, gc);
  gamma_coef_apply<T, NC>(gc, v);
}

}  // namespace lsh
