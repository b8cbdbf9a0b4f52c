// kernels_reg.cu -- y and z passes built on the two-level register FFT
// (regfft.cuh) for the lengths 16, 32, 64, 128 and 256.  Frequencies along y
// and z are then stored in natural order.
//
// A block owns a set of lines.  Regular blocks take TY (TZ) consecutive kx
// columns of one plane, so their global accesses are coalesced along kx;
// the columns left over when nx/2+1 is not a multiple of the tile (the
// Nyquist column for even nx) are gathered TY at a time from several planes
// by extra blocks.
#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"
#include "regfft.cuh"
#include "gamma_onfly.cuh"

namespace lsh {

// ------------------------------------------------------------------ y pass
template <typename T, bool INV, int N>
__global__ void __launch_bounds__(16 * RegPlan<N>::P) k_yfft_reg(OpArgs<T> a, const SolverState* __restrict__ st,
                                                                 int nrt, int nreg) {
  typedef RegLine<T, N> RL;
  constexpr int TY = 16, P = RL::P, R1 = RL::R1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* ex = tw + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.twy[i];
  const int i = threadIdx.x % TY, t = threadIdx.x / TY;
  const long long nplanes = (long long)a.S * a.c * a.nz;
  const int nleft = a.nxh - nreg;
  long long plane;
  int kx;
  bool valid = true;
  if ((long long)blockIdx.x < nplanes * nrt) {
    plane = blockIdx.x / nrt;
    kx = (int)(blockIdx.x - plane * nrt) * TY + i;
    if (st != nullptr && st[plane / (a.c * a.nz)].done) return;  // uniform: one plane per block
  } else {
    const long long l = (blockIdx.x - nplanes * nrt) * (long long)TY + i;
    valid = l < nplanes * nleft;
    plane = valid ? l / nleft : 0;
    kx = valid ? nreg + (int)(l - plane * nleft) : 0;
    if (valid && st != nullptr && st[plane / (a.c * a.nz)].done) valid = false;
  }
  C2<T>* __restrict__ Hl = a.H + plane * a.ny * a.hs + kx;
  const int rs = a.hs;  // row stride
  C2<T> v[R1];
  __syncthreads();
  if (!INV) {
#pragma unroll
    for (int j = 0; j < R1; ++j) v[j] = valid ? Hl[(t + P * j) * rs] : mkc<T>(0, 0);
    RL::fwd_a(v, t, tw, ex + i * RL::LS);
    __syncthreads();
    RL::fwd_b(v, t, tw, ex + i * RL::LS);
    if (valid) {
#pragma unroll
      for (int m = 0; m < R1; ++m) Hl[RL::freq(t, m) * rs] = v[m];
    }
  } else {
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = valid ? Hl[RL::freq(t, m) * rs] : mkc<T>(0, 0);
    RL::inv_a(v, t, tw, ex + i * RL::LS);
    __syncthreads();
    RL::inv_b(v, t, tw, ex + i * RL::LS);
    if (valid) {
#pragma unroll
      for (int j = 0; j < R1; ++j) Hl[(t + P * j) * rs] = v[j];
    }
  }
}

// ------------------------------------------------------------------ z pass + Gamma
template <typename T, int NC, int N, int TZV = 0> struct ZCfg {
  // TZV = 0: 8 columns per block (4 in FP64 or for length 256); else TZV columns
  static constexpr int TZ = TZV > 0 ? TZV : ((sizeof(T) == 8 || N >= 256) ? 4 : 8);
  static constexpr int W = 128 / (int)sizeof(C2<T>);  // complex values per shared wavefront
  static constexpr int KS0 = NC * TZ;
  static constexpr int KS = KS0 + ((TZ - KS0 % W) % W + W) % W;  // KS = TZ (mod W)
  static constexpr int THREADS = TZ * NC * RegPlan<N>::P;
  static constexpr int EXN = NC * TZ * RegLine<T, N>::LS;
  static constexpr int GBN = N * KS;
  static constexpr int BUF = EXN > GBN ? EXN : GBN;
};

template <typename T, int NC, int N, int TZV>
__global__ void __launch_bounds__(ZCfg<T, NC, N, TZV>::THREADS, ZCfg<T, NC, N, TZV>::THREADS <= 192 ? 4 : 2)
    k_zgamma_reg(OpArgs<T> a, const SolverState* __restrict__ st, int nrt, int nreg) {
  typedef RegLine<T, N> RL;
  typedef ZCfg<T, NC, N, TZV> ZC;
  constexpr int TZ = ZC::TZ, P = RL::P, R1 = RL::R1, KS = ZC::KS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf = tw + N;
  __shared__ int line_yp[TZ], line_kx[TZ];
  const int s = blockIdx.x;
  if (st != nullptr && st[s].done) return;
  for (int u = threadIdx.x; u < N; u += blockDim.x) tw[u] = a.twz[u];
  const int tile = blockIdx.y;
  const int nleft = a.nxh - nreg;
  if (threadIdx.x < TZ) {
    const int i = threadIdx.x;
    int yp = -1, kx = 0;
    if (tile < a.ny * nrt) {
      yp = tile / nrt;
      kx = (tile - yp * nrt) * TZ + i;
    } else {
      const int l = (tile - a.ny * nrt) * TZ + i;
      if (l < a.ny * nleft) {
        yp = l / nleft;
        kx = nreg + (l - yp * nleft);
      }
    }
    line_yp[i] = yp;
    line_kx[i] = kx;
  }
  __syncthreads();
  const int i = threadIdx.x % TZ, comp = (threadIdx.x / TZ) % NC, t = threadIdx.x / (TZ * NC);
  const int yp = line_yp[i], kx = line_kx[i];
  const bool valid = yp >= 0;
  const long long zstride = (long long)a.ny * a.hs;  // z planes of H
  const long long cstride = zstride * N;
  const long long gzs = (long long)a.ny * a.ts, gcs = gzs * N;  // the same in the Gamma table
  C2<T>* __restrict__ Hl = a.H + ((long long)s * NC + comp) * cstride + (valid ? (long long)yp * a.hs + kx : 0);
  C2<T>* exl = buf + (comp * TZ + i) * RL::LS;
  C2<T> v[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) v[j] = valid ? Hl[(t + P * j) * zstride] : mkc<T>(0, 0);
  RL::fwd_a(v, t, tw, exl);
  __syncthreads();
  RL::fwd_b(v, t, tw, exl);
  __syncthreads();
  // all components of each frequency meet in buf[kz][comp][i]
#pragma unroll
  for (int m = 0; m < R1; ++m) buf[RL::freq(t, m) * KS + comp * TZ + i] = v[m];
  __syncthreads();
  if (a.onfly) {
    for (int item = threadIdx.x; item < N * TZ; item += blockDim.x) {
      const int kz = item / TZ, li = item - kz * TZ;
      const int lyp = line_yp[li];
      if (lyp < 0) continue;
      C2<T> g[NC];
#pragma unroll
      for (int c2 = 0; c2 < NC; ++c2) g[c2] = buf[kz * KS + c2 * TZ + li];
      gamma_trunc_onfly<T, NC>(a, line_kx[li], a.kofy[lyp], kz, g);
#pragma unroll
      for (int c2 = 0; c2 < NC; ++c2) buf[kz * KS + c2 * TZ + li] = g[c2];
    }
  } else {
    // tabulated Gamma^h_k: the coefficients of a thread's next frequency are
    // loaded while the current one is applied
    constexpr int NCO = NC * (NC + 1) / 2;
    auto off = [&](int item) {
      const int kz = item / TZ, li = item - kz * TZ;
      return kz * gzs + (long long)line_yp[li] * a.ts + line_kx[li];
    };
    auto ok = [&](int item) { return item < N * TZ && line_yp[item % TZ] >= 0; };
    T gc[NCO], gn[NCO];
    int item = threadIdx.x;
    bool have = ok(item);
    if (have) gamma_coef_load<T, NC>(a.gtab, gcs, off(item), gc);
#pragma unroll 1
    for (; item < N * TZ; item += blockDim.x) {
      const int nxt = item + blockDim.x;
      const bool hn = ok(nxt);
      if (hn) gamma_coef_load<T, NC>(a.gtab, gcs, off(nxt), gn);
      if (have) {
        const int kz = item / TZ, li = item - kz * TZ;
        C2<T> g[NC];
#pragma unroll
        for (int c2 = 0; c2 < NC; ++c2) g[c2] = buf[kz * KS + c2 * TZ + li];
        if (a.fdphase) fd_rotate<T, NC>(a, line_kx[li], a.kofy[line_yp[li]], kz, g, (T)-1);
        gamma_coef_apply<T, NC>(gc, g);
        if (a.fdphase) fd_rotate<T, NC>(a, line_kx[li], a.kofy[line_yp[li]], kz, g, (T)1);
#pragma unroll
        for (int c2 = 0; c2 < NC; ++c2) buf[kz * KS + c2 * TZ + li] = g[c2];
      }
#pragma unroll
      for (int c = 0; c < NCO; ++c) gc[c] = gn[c];
      have = hn;
    }
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < R1; ++m) v[m] = buf[RL::freq(t, m) * KS + comp * TZ + i];
  __syncthreads();
  RL::inv_a(v, t, tw, exl);
  __syncthreads();
  RL::inv_b(v, t, tw, exl);
  if (valid) {
#pragma unroll
    for (int j = 0; j < R1; ++j) Hl[(t + P * j) * zstride] = v[j];
  }
}

// ------------------------------------------------------------------ launchers
bool reg_length(int n) { return n == 16 || n == 32 || n == 64 || n == 128 || n == 256; }

template <typename T, bool INV, int N> void launch_y_n(const OpArgs<T>& a, const SolverState* st, cudaStream_t s) {
  constexpr int TY = 16;
  const int nrt = a.nxh / TY, nreg = nrt * TY;
  const long long nplanes = (long long)a.S * a.c * a.nz;
  const long long nleft_lines = nplanes * (a.nxh - nreg);
  const long long grid = nplanes * nrt + (nleft_lines + TY - 1) / TY;
  const size_t smem = sizeof(C2<T>) * (N + TY * RegLine<T, N>::LS);
  k_yfft_reg<T, INV, N><<<(unsigned)grid, TY * RegPlan<N>::P, smem, s>>>(a, st, nrt, nreg);
}

template <typename T, bool INV> void launch_y_reg(const OpArgs<T>& a, const SolverState* st, cudaStream_t s) {
  switch (a.ny) {
    case 16: launch_y_n<T, INV, 16>(a, st, s); break;
    case 32: launch_y_n<T, INV, 32>(a, st, s); break;
    case 64: launch_y_n<T, INV, 64>(a, st, s); break;
    case 128: launch_y_n<T, INV, 128>(a, st, s); break;
    default: launch_y_n<T, INV, 256>(a, st, s); break;
  }
}

template <typename T> void launch_yfft_reg(const OpArgs<T>& a, bool inv, const SolverState* st, cudaStream_t s) {
  if (inv) launch_y_reg<T, true>(a, st, s);
  else launch_y_reg<T, false>(a, st, s);
}

template <typename T, int NC, int N, int TZV> void launch_z_n(const OpArgs<T>& a, const SolverState* st, cudaStream_t s) {
  typedef ZCfg<T, NC, N, TZV> ZC;
  const int nrt = a.nxh / ZC::TZ, nreg = nrt * ZC::TZ;
  const int ntiles = a.ny * nrt + (a.ny * (a.nxh - nreg) + ZC::TZ - 1) / ZC::TZ;
  const size_t smem = sizeof(C2<T>) * (N + ZC::BUF);
  k_zgamma_reg<T, NC, N, TZV><<<dim3(a.S, ntiles), ZC::THREADS, smem, s>>>(a, st, nrt, nreg);
}

template <typename T, int NC, int TZV> void launch_z_nc(const OpArgs<T>& a, const SolverState* st, cudaStream_t s) {
  switch (a.nz) {
    case 16: launch_z_n<T, NC, 16, TZV>(a, st, s); break;
    case 32: launch_z_n<T, NC, 32, TZV>(a, st, s); break;
    case 64: launch_z_n<T, NC, 64, TZV>(a, st, s); break;
    case 128: launch_z_n<T, NC, 128, TZV>(a, st, s); break;
    default: launch_z_n<T, NC, 256, TZV>(a, st, s); break;
  }
}

template <typename T, int TZV> void launch_z_tz(const OpArgs<T>& a, const SolverState* st, cudaStream_t s) {
  if (a.c == 6) launch_z_nc<T, 6, TZV>(a, st, s);
  else if (a.c == 3) launch_z_nc<T, 3, TZV>(a, st, s);
  else launch_z_nc<T, 2, TZV>(a, st, s);
}

// tz = 4: blocks of 4 columns (FP32 autotuner candidate); otherwise the default width
template <typename T> void launch_zgamma_reg(const OpArgs<T>& a, const SolverState* st, cudaStream_t s, int tz) {
  if (sizeof(T) == 4 && tz == 4) launch_z_tz<T, 4>(a, st, s);
  else launch_z_tz<T, 0>(a, st, s);
}

// dynamic shared memory of one instantiation (static shared memory comes on top
// of it, so the attribute is set to exactly what the launch asks for)
template <typename T, int NC, int N> void attr_z_n() {
  const int bytes = (int)(sizeof(C2<T>) * (N + ZCfg<T, NC, N, 0>::BUF));
  cudaFuncSetAttribute(k_zgamma_reg<T, NC, N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (sizeof(T) == 4) {
    const int b4 = (int)(sizeof(C2<T>) * (N + ZCfg<T, NC, N, 4>::BUF));
    cudaFuncSetAttribute(k_zgamma_reg<T, NC, N, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b4);
  }
}
template <typename T, bool INV, int N> void attr_y_n() {
  const int bytes = (int)(sizeof(C2<T>) * (N + 16 * RegLine<T, N>::LS));
  cudaFuncSetAttribute(k_yfft_reg<T, INV, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
template <typename T, int NC> void attr_z_nc() {
  attr_z_n<T, NC, 16>();
  attr_z_n<T, NC, 32>();
  attr_z_n<T, NC, 64>();
  attr_z_n<T, NC, 128>();
  attr_z_n<T, NC, 256>();
}
template <typename T, bool INV> void attr_y() {
  attr_y_n<T, INV, 16>();
  attr_y_n<T, INV, 32>();
  attr_y_n<T, INV, 64>();
  attr_y_n<T, INV, 128>();
  attr_y_n<T, INV, 256>();
}
template <typename T> void set_smem_attrs_reg() {
  attr_y<T, false>();
  attr_y<T, true>();
  attr_z_nc<T, 2>();
  attr_z_nc<T, 3>();
  attr_z_nc<T, 6>();
}
template void set_smem_attrs_reg<double>();
template void set_smem_attrs_reg<float>();

template void launch_yfft_reg<double>(const OpArgs<double>&, bool, const SolverState*, cudaStream_t);
template void launch_yfft_reg<float>(const OpArgs<float>&, bool, const SolverState*, cudaStream_t);
template void launch_zgamma_reg<double>(const OpArgs<double>&, const SolverState*, cudaStream_t, int);
template void launch_zgamma_reg<float>(const OpArgs<float>&, const SolverState*, cudaStream_t, int);

}  // namespace lsh
