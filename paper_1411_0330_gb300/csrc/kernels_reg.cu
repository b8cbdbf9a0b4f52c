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
#include "tma.cuh"

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
  // TZV <= 0: 8 columns per block (4 in FP64 or for length 256); else TZV columns.
  // TZV < 0: the Gamma coefficients are loaded when used, not one frequency ahead.
  static constexpr int TZ = TZV > 0 ? TZV : ((sizeof(T) == 8 || N >= 256) ? 4 : 8);
  static constexpr int W = 128 / (int)sizeof(C2<T>);  // complex values per shared wavefront
  static constexpr int KS0 = NC * TZ;
  static constexpr int KS = KS0 + ((TZ - KS0 % W) % W + W) % W;  // KS = TZ (mod W)
  static constexpr int THREADS = TZ * NC * RegPlan<N>::P;
  static constexpr int EXN = NC * TZ * RegLine<T, N>::LS;
  static constexpr int GBN = N * KS;
  static constexpr int BUF = EXN > GBN ? EXN : GBN;
};

// Gamma^h_k on the NC components of the N x TZ frequencies of a block's tile,
// in place in buf[kz KS + comp TZ + li]; line_yp/line_kx give each line's y
// position (-1: no line) and kx.  PIPE: a thread loads the table coefficients
// of its next frequency while it applies the current ones.
template <typename T, int NC, int N, int TZ, int KS, bool PIPE = true>
__device__ __forceinline__ void z_gamma_block(const OpArgs<T>& a, C2<T>* buf, const int* line_yp,
                                              const int* line_kx) {
  // double-float (T = DF): tabulated coefficients only, no finite-difference phases
  constexpr bool FLY = !is_df<T>::value;
  if (FLY && a.onfly) {
    if constexpr (FLY) {
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
    }
  } else if constexpr (!PIPE) {
    for (int item = threadIdx.x; item < N * TZ; item += blockDim.x) {
      const int kz = item / TZ, li = item - kz * TZ;
      const int lyp = line_yp[li];
      if (lyp < 0) continue;
      C2<T> g[NC];
#pragma unroll
      for (int c2 = 0; c2 < NC; ++c2) g[c2] = buf[kz * KS + c2 * TZ + li];
      if constexpr (FLY)
        if (a.fdphase) fd_rotate<T, NC>(a, line_kx[li], a.kofy[lyp], kz, g, (T)-1);
      gamma_table_apply<T, NC>(a.gtab, ((long long)kz * a.ny + lyp) * a.ts + line_kx[li], g);
      if constexpr (FLY)
        if (a.fdphase) fd_rotate<T, NC>(a, line_kx[li], a.kofy[lyp], kz, g, (T)1);
#pragma unroll
      for (int c2 = 0; c2 < NC; ++c2) buf[kz * KS + c2 * TZ + li] = g[c2];
    }
  } else {
    // tabulated Gamma^h_k: the coefficients of a thread's next frequency are
    // loaded while the current one is applied
    constexpr int NCO = NC * (NC + 1) / 2;
    auto off = [&](int item) {  // frequency index in the table
      const int kz = item / TZ, li = item - kz * TZ;
      return ((long long)kz * a.ny + line_yp[li]) * a.ts + line_kx[li];
    };
    auto ok = [&](int item) { return item < N * TZ && line_yp[item % TZ] >= 0; };
    T gc[NCO], gn[NCO];
    int item = threadIdx.x;
    bool have = ok(item);
    if (have) gamma_coef_load<T, NC>(a.gtab, off(item), gc);
#pragma unroll 1
    for (; item < N * TZ; item += blockDim.x) {
      const int nxt = item + blockDim.x;
      const bool hn = ok(nxt);
      if (hn) gamma_coef_load<T, NC>(a.gtab, off(nxt), gn);
      if (have) {
        const int kz = item / TZ, li = item - kz * TZ;
        C2<T> g[NC];
#pragma unroll
        for (int c2 = 0; c2 < NC; ++c2) g[c2] = buf[kz * KS + c2 * TZ + li];
        if constexpr (FLY)
          if (a.fdphase) fd_rotate<T, NC>(a, line_kx[li], a.kofy[line_yp[li]], kz, g, (T)-1);
        gamma_coef_apply<T, NC>(gc, g);
        if constexpr (FLY)
          if (a.fdphase) fd_rotate<T, NC>(a, line_kx[li], a.kofy[line_yp[li]], kz, g, (T)1);
#pragma unroll
        for (int c2 = 0; c2 < NC; ++c2) buf[kz * KS + c2 * TZ + li] = g[c2];
      }
#pragma unroll
      for (int c = 0; c < NCO; ++c) gc[c] = gn[c];
      have = hn;
    }
  }
}

template <typename T, int NC, int N, int TZV>
__global__ void __launch_bounds__(ZCfg<T, NC, N, TZV>::THREADS,
                                  ZCfg<T, NC, N, TZV>::THREADS > 384
                                      ? 1
                                      : ((ZCfg<T, NC, N, TZV>::THREADS <= 192 && !is_df<T>::value) ? 4 : 2))
    k_zgamma_reg(OpArgs<T> a, const SolverState* __restrict__ st, int nrt, int nreg) {
  typedef RegLine<T, N> RL;
  typedef ZCfg<T, NC, N, TZV> ZC;
  constexpr int TZ = ZC::TZ, P = RL::P, R1 = RL::R1, KS = ZC::KS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* tw = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf = tw + N;
  __shared__ int line_yp[TZ], line_kx[TZ];
  const int nleft = a.nxh - nreg;
  int s, tile;
  if (a.tlay) {
    // ky-major spectrum (plane passes): the kx tiles of one (system, ky) slab
    // are consecutive blocks, so their columns share the slab's contiguous range
    const long long nregb = (long long)a.ny * a.S * nrt;
    const long long lin = blockIdx.x;
    if (lin < nregb) {
      const int yp = (int)(lin / ((long long)a.S * nrt));
      const int rem = (int)(lin - (long long)yp * a.S * nrt);
      s = rem / nrt;
      tile = yp * nrt + (rem - s * nrt);
    } else {
      const int ntl = (a.ny * nleft + TZ - 1) / TZ;
      const int l2 = (int)(lin - nregb);
      s = l2 / ntl;
      tile = a.ny * nrt + (l2 - s * ntl);
    }
  } else {
    s = blockIdx.x;
    tile = blockIdx.y;
  }
  if (st != nullptr && st[s].done) return;
  for (int u = threadIdx.x; u < N; u += blockDim.x) tw[u] = a.twz[u];
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
  if constexpr (sizeof(T) == 4 && TZV >= 0) {
    // the tile's Gamma rows (contiguous per z frequency) go to L2 while the
    // forward transform runs; the first system's block asks for all systems
    if (!a.onfly && s == 0 && tile < a.ny * nrt) {
      constexpr int NCOP = GammaPack<NC>::NCOP;
      for (int kz = threadIdx.x; kz < N; kz += blockDim.x)
        bulk_prefetch_l2(a.gtab + (((long long)kz * a.ny + line_yp[0]) * a.ts + line_kx[0]) * NCOP,
                         (uint32_t)(sizeof(T) * TZ * NCOP));
    }
  }
  const int i = threadIdx.x % TZ, comp = (threadIdx.x / TZ) % NC, t = threadIdx.x / (TZ * NC);
  const int yp = line_yp[i], kx = line_kx[i];
  const bool valid = yp >= 0;
  long long zstride = (long long)a.ny * a.hs;  // z planes of H
  const long long cstride = zstride * N;
  C2<T>* __restrict__ Hl = a.H + ((long long)s * NC + comp) * cstride + (valid ? (long long)yp * a.hs + kx : 0);
  if (a.tlay) {
    if (valid && 2 * kx == a.nx) {
      // the Nyquist column: NQ[s][comp][z][ky]
      Hl = a.nq + ((long long)s * NC + comp) * N * a.ny + yp;
      zstride = a.ny;
    } else {
      Hl = a.H + ((long long)s * NC + comp) * cstride + (valid ? (long long)yp * N * a.hs + kx : 0);
      zstride = a.hs;
    }
  }
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
  z_gamma_block<T, NC, N, TZ, KS, (TZV >= 0)>(a, buf, line_yp, line_kx);
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

// ------------------------------------------------------------------ z pass + Gamma, persistent
// FP32 variant of k_zgamma_reg whose blocks stay resident and walk the tiles
// (system s, TZ lines) with the grid's stride.  The columns of the next tile
// are copied into a staging area of shared memory by per-thread asynchronous
// copies issued right after the current tile has left it, so the strided reads
// along z run under the FFTs and the Gamma^h product of the current tile.
template <int NC, int N> struct ZPCfg {
  typedef ZCfg<float, NC, N, 0> ZC;
  static constexpr int TZ = ZC::TZ, THREADS = ZC::THREADS;
  static constexpr int STAGE = N * NC * TZ;  // complex values of one tile
  static constexpr size_t SMEM = sizeof(float2) * (STAGE + N + ZC::BUF);
  static constexpr bool FITS = SMEM <= 226 * 1024;
};

template <int NC, int N>
__global__ void __launch_bounds__(ZPCfg<NC, N>::THREADS, ZPCfg<NC, N>::THREADS <= 192 ? 4 : 2)
    k_zgamma_regp(OpArgs<float> a, const SolverState* __restrict__ st, int nrt, int nreg, int ntiles) {
  typedef RegLine<float, N> RL;
  typedef ZCfg<float, NC, N, 0> ZC;
  constexpr int TZ = ZC::TZ, P = RL::P, R1 = RL::R1, KS = ZC::KS, THREADS = ZC::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* stage = reinterpret_cast<float2*>(smem_raw);  // [z][comp][li]
  float2* tw = stage + ZPCfg<NC, N>::STAGE;
  float2* buf = tw + N;
  __shared__ int line_yp[TZ], line_kx[TZ];
  for (int u = threadIdx.x; u < N; u += THREADS) tw[u] = a.twz[u];
  const int S = a.S, nleft = a.nxh - nreg, nregt = a.ny * nrt;
  const int total = S * ntiles;  // below 2^31 (checked by the launcher)
  // element strides of H: x-major [S][c][z][y][hs] or ky-major [S][c][y][z][hs]
  const long long ys = a.tlay ? (long long)N * a.hs : a.hs;
  const long long zs = a.tlay ? a.hs : (long long)a.ny * a.hs;
  const long long cstride = (long long)a.ny * a.hs * N;
  // line li of tile `tile`: y position (-1: past the last column) and kx
  auto line = [&](int tile, int li, int& yp, int& kx) {
    if (tile < nregt) {
      yp = tile / nrt;
      kx = (tile - yp * nrt) * TZ + li;
    } else {
      const int l = (tile - nregt) * TZ + li;
      yp = -1;
      kx = 0;
      if (l < a.ny * nleft) {
        yp = l / nleft;
        kx = nreg + (l - yp * nleft);
      }
    }
  };
  // the system and tile of work item tl: systems fastest (x-major spectrum: the
  // systems share the tile's Gamma rows), or kx tiles fastest within a (system,
  // ky) slab (ky-major spectrum: the slab is one contiguous range)
  auto item = [&](int tl, int& s, int& tile) {
    if (!a.tlay) {
      s = tl % S;
      tile = tl / S;
    } else if (tl < nregt * S) {
      const int yp = tl / (S * nrt), rem = tl - yp * S * nrt;
      s = rem / nrt;
      tile = yp * nrt + (rem - s * nrt);
    } else {
      const int ntl = ntiles - nregt, l2 = tl - nregt * S;
      s = l2 / ntl;
      tile = nregt + (l2 - s * ntl);
    }
  };
  // complex element (s, comp, z) of line (yp, kx): the Nyquist column of a
  // ky-major spectrum lives in NQ[S][c][z][ky]
  auto elem = [&](int s, int comp, int z, int yp, int kx) -> float2* {
    if (a.tlay && 2 * kx == a.nx) return a.nq + (((long long)s * NC + comp) * N + z) * a.ny + yp;
    return a.H + ((long long)s * NC + comp) * cstride + (long long)z * zs + (long long)yp * ys + kx;
  };
  auto next_live = [&](int tl) {
    int s, tile;
    while (tl < total && st != nullptr) {
      item(tl, s, tile);
      if (!st[s].done) break;
      tl += gridDim.x;
    }
    return tl;
  };
  // stage the columns of tile tl; its Gamma^h rows go to L2 meanwhile
  auto prefetch = [&](int tl) {
    int s, tile;
    item(tl, s, tile);
    if (tile < nregt) {
      // TZ consecutive columns: rows of TZ / 2 aligned 16-byte pieces
      constexpr int CH = TZ / 2, NCOP = GammaPack<NC>::NCOP;
      const int yp = tile / nrt, kx0 = (tile - yp * nrt) * TZ;
      for (int q = threadIdx.x; q < N * NC * CH; q += THREADS) {
        const int row = q / CH, piece = q - row * CH;  // row = z NC + comp
        const int z = row / NC, comp = row - z * NC;
        cp_async16(stage + row * TZ + 2 * piece, elem(s, comp, z, yp, kx0) + 2 * piece);
      }
      if (!a.onfly)
        for (int kz = threadIdx.x; kz < N; kz += THREADS)
          bulk_prefetch_l2(a.gtab + (((long long)kz * a.ny + yp) * a.ts + kx0) * NCOP,
                           (uint32_t)(sizeof(float) * TZ * NCOP));
    } else {
      for (int q = threadIdx.x; q < N * NC * TZ; q += THREADS) {
        const int row = q / TZ, li = q - row * TZ;
        const int z = row / NC, comp = row - z * NC;
        int yp, kx;
        line(tile, li, yp, kx);
        if (yp >= 0) cp_async8(stage + q, elem(s, comp, z, yp, kx));
      }
    }
    cp_async_commit();
  };
  const int i = threadIdx.x % TZ, comp = (threadIdx.x / TZ) % NC, t = threadIdx.x / (TZ * NC);
  float2* exl = buf + (comp * TZ + i) * RL::LS;
  int cur = next_live(blockIdx.x);
  if (cur < total) prefetch(cur);
  while (cur < total) {
    const int nxt = next_live(cur + gridDim.x);
    int s, tile;
    item(cur, s, tile);
    cp_async_wait_all();
    __syncthreads();  // the tile is staged; the previous tile is done with buf and the line table
    if (threadIdx.x < TZ) {
      int yp, kx;
      line(tile, threadIdx.x, yp, kx);
      line_yp[threadIdx.x] = yp;
      line_kx[threadIdx.x] = kx;
    }
    int yp, kx;
    line(tile, i, yp, kx);
    const bool valid = yp >= 0;
    float2 v[R1];
#pragma unroll
    for (int j = 0; j < R1; ++j) v[j] = valid ? stage[((t + P * j) * NC + comp) * TZ + i] : mkc<float>(0, 0);
    RL::fwd_a(v, t, tw, exl);
    __syncthreads();  // every thread has read the staging area
    if (nxt < total) prefetch(nxt);
    RL::fwd_b(v, t, tw, exl);
    __syncthreads();
#pragma unroll
    for (int m = 0; m < R1; ++m) buf[RL::freq(t, m) * KS + comp * TZ + i] = v[m];
    __syncthreads();
    z_gamma_block<float, NC, N, TZ, KS, false>(a, buf, line_yp, line_kx);
    __syncthreads();
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = buf[RL::freq(t, m) * KS + comp * TZ + i];
    __syncthreads();
    RL::inv_a(v, t, tw, exl);
    __syncthreads();
    RL::inv_b(v, t, tw, exl);
    if (valid) {
      float2* Hl = elem(s, comp, 0, yp, kx);
      const long long step = (a.tlay && 2 * kx == a.nx) ? (long long)a.ny : zs;
#pragma unroll
      for (int j = 0; j < R1; ++j) Hl[(long long)(t + P * j) * step] = v[j];
    }
    cur = nxt;
  }
  cp_async_wait_all();
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
  if constexpr (is_df<T>::value) {
    // radix-3 lengths of the double-float refinement residual
    if (a.ny == 48) {
      launch_y_n<T, INV, 48>(a, st, s);
      return;
    }
    if (a.ny == 96) {
      launch_y_n<T, INV, 96>(a, st, s);
      return;
    }
  }
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
  if constexpr (ZC::THREADS > 1024 || sizeof(C2<T>) * (N + ZC::BUF) > 227 * 1024) {
    launch_z_n<T, NC, N, 0>(a, st, s);  // too wide for one block: the default width
    return;
  }
  const int nrt = a.nxh / ZC::TZ, nreg = nrt * ZC::TZ;
  const int ntiles = a.ny * nrt + (a.ny * (a.nxh - nreg) + ZC::TZ - 1) / ZC::TZ;
  const size_t smem = sizeof(C2<T>) * (N + ZC::BUF);
  if (a.tlay)
    k_zgamma_reg<T, NC, N, TZV><<<(unsigned)((long long)a.S * ntiles), ZC::THREADS, smem, s>>>(a, st, nrt, nreg);
  else
    k_zgamma_reg<T, NC, N, TZV><<<dim3(a.S, ntiles), ZC::THREADS, smem, s>>>(a, st, nrt, nreg);
}

template <typename T, int NC, int TZV> void launch_z_nc(const OpArgs<T>& a, const SolverState* st, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    // radix-3 lengths of the FP32 passes
    if (a.nz == 48) {
      launch_z_n<T, NC, 48, TZV>(a, st, s);
      return;
    }
    if (a.nz == 96) {
      launch_z_n<T, NC, 96, TZV>(a, st, s);
      return;
    }
  }
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

// FP32 autotuner candidates: tz = 4 or 16 columns per block, tz < 0 the default
// width without loading the Gamma coefficients ahead; otherwise the default width
template <typename T> void launch_zgamma_reg(const OpArgs<T>& a, const SolverState* st, cudaStream_t s, int tz) {
  if constexpr (sizeof(T) == 4) {
    if (tz == 4) {
      launch_z_tz<T, 4>(a, st, s);
      return;
    }
    if (tz == 16) {
      launch_z_tz<T, 16>(a, st, s);
      return;
    }
    if (tz < 0) {
      launch_z_tz<T, -1>(a, st, s);
      return;
    }
  }
  launch_z_tz<T, 0>(a, st, s);
}

int multiprocessors() {
  static int n = []() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      v = 1;
    }
    return v;
  }();
  return n;
}

template <int NC, int N> int zp_blocks_per_sm() {
  typedef ZPCfg<NC, N> ZP;
  static int n = []() {
    int v = 0;
    if constexpr (ZP::FITS) {
      cudaFuncSetAttribute(k_zgamma_regp<NC, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZP::SMEM);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_zgamma_regp<NC, N>, ZP::THREADS, ZP::SMEM) !=
          cudaSuccess) {
        cudaGetLastError();
        v = 0;
      }
    }
    return v;
  }();
  return n;
}

template <int NC, int N> bool launch_zp_n(const OpArgs<float>& a, const SolverState* st, cudaStream_t s) {
  typedef ZPCfg<NC, N> ZP;
  if constexpr (!ZP::FITS) {
    return false;
  } else {
    const int bpsm = zp_blocks_per_sm<NC, N>();
    if (bpsm < 1 || a.S < 1) return bpsm >= 1;
    const int nrt = a.nxh / ZP::TZ, nreg = nrt * ZP::TZ;
    const int ntiles = a.ny * nrt + (a.ny * (a.nxh - nreg) + ZP::TZ - 1) / ZP::TZ;
    const long long total = (long long)a.S * ntiles;
    const long long cstride = (long long)a.ny * a.hs * N;
    if (total + (long long)multiprocessors() * bpsm >= (1ll << 31) || cstride >= (1ll << 31)) return false;
    const int grid = (int)std::max<long long>(1, std::min<long long>(total, (long long)multiprocessors() * bpsm));
    k_zgamma_regp<NC, N><<<grid, ZP::THREADS, ZP::SMEM, s>>>(a, st, nrt, nreg, ntiles);
    return true;
  }
}

template <int NC> bool launch_zp_nc(const OpArgs<float>& a, const SolverState* st, cudaStream_t s) {
  switch (a.nz) {
    case 48: return launch_zp_n<NC, 48>(a, st, s);
    case 96: return launch_zp_n<NC, 96>(a, st, s);
    case 16: return launch_zp_n<NC, 16>(a, st, s);
    case 32: return launch_zp_n<NC, 32>(a, st, s);
    case 64: return launch_zp_n<NC, 64>(a, st, s);
    case 128: return launch_zp_n<NC, 128>(a, st, s);
    case 256: return launch_zp_n<NC, 256>(a, st, s);
    default: return false;
  }
}

// Persistent FP32 z pass with staged prefetch; false (nothing launched) when
// the length has no register plan or the kernel does not fit.  With a.S = 0
// it only answers whether it would launch.
bool launch_zgamma_regp(const OpArgs<float>& a, const SolverState* st, cudaStream_t s) {
  if (a.c == 6) return launch_zp_nc<6>(a, st, s);
  if (a.c == 3) return launch_zp_nc<3>(a, st, s);
  if (a.c == 2) return launch_zp_nc<2>(a, st, s);
  return false;
}

template <int NC> void zp_prepare() {
  zp_blocks_per_sm<NC, 48>();
  zp_blocks_per_sm<NC, 96>();
  zp_blocks_per_sm<NC, 16>();
  zp_blocks_per_sm<NC, 32>();
  zp_blocks_per_sm<NC, 64>();
  zp_blocks_per_sm<NC, 128>();
  zp_blocks_per_sm<NC, 256>();
}

// dynamic shared memory of one instantiation (static shared memory comes on top
// of it, so the attribute is set to exactly what the launch asks for)
template <typename T, int NC, int N> void attr_z_n() {
  const int bytes = (int)(sizeof(C2<T>) * (N + ZCfg<T, NC, N, 0>::BUF));
  cudaFuncSetAttribute(k_zgamma_reg<T, NC, N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if constexpr (sizeof(T) == 4) {
    const int b4 = (int)(sizeof(C2<T>) * (N + ZCfg<T, NC, N, 4>::BUF));
    cudaFuncSetAttribute(k_zgamma_reg<T, NC, N, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b4);
    const int bn = (int)(sizeof(C2<T>) * (N + ZCfg<T, NC, N, -1>::BUF));
    cudaFuncSetAttribute(k_zgamma_reg<T, NC, N, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bn);
    typedef ZCfg<T, NC, N, 16> Z16;
    if constexpr (Z16::THREADS <= 1024 && sizeof(C2<T>) * (N + Z16::BUF) <= 227 * 1024) {
      const int b16 = (int)(sizeof(C2<T>) * (N + Z16::BUF));
      cudaFuncSetAttribute(k_zgamma_reg<T, NC, N, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b16);
    }
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
  if constexpr (sizeof(T) == 4) {
    attr_z_n<T, NC, 48>();
    attr_z_n<T, NC, 96>();
  }
}
template <typename T, bool INV> void attr_y() {
  attr_y_n<T, INV, 16>();
  attr_y_n<T, INV, 32>();
  attr_y_n<T, INV, 64>();
  attr_y_n<T, INV, 128>();
  attr_y_n<T, INV, 256>();
  if constexpr (is_df<T>::value) {
    attr_y_n<T, INV, 48>();
    attr_y_n<T, INV, 96>();
  }
}
template <typename T> void set_smem_attrs_reg() {
  attr_y<T, false>();
  attr_y<T, true>();
  if constexpr (!is_df<T>::value) {  // the double-float z pass has kernels of its own
    attr_z_nc<T, 2>();
    attr_z_nc<T, 3>();
    attr_z_nc<T, 6>();
  }
  if constexpr (sizeof(T) == 4) {
    zp_prepare<2>();
    zp_prepare<3>();
    zp_prepare<6>();
  }
}
template void set_smem_attrs_reg<double>();
template void set_smem_attrs_reg<float>();
template void set_smem_attrs_reg<DF>();

template void launch_yfft_reg<double>(const OpArgs<double>&, bool, const SolverState*, cudaStream_t);
template void launch_yfft_reg<float>(const OpArgs<float>&, bool, const SolverState*, cudaStream_t);
template void launch_zgamma_reg<double>(const OpArgs<double>&, const SolverState*, cudaStream_t, int);
template void launch_zgamma_reg<float>(const OpArgs<float>&, const SolverState*, cudaStream_t, int);
template void launch_yfft_reg<DF>(const OpArgs<DF>&, bool, const SolverState*, cudaStream_t);

}  // namespace lsh
