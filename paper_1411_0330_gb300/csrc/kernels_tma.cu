// kernels_tma.cu -- the y pass and the z pass with the Green operator as
// persistent, double-buffered TMA kernels (FP32 spectrum, lengths 16..256).
//
// The half spectrum H[S][c][nz][ny][hs] is seen by the Tensor Memory
// Accelerator as a 3-D array {2 hs floats, ny rows, S c nz planes}.  A tile is
// TY consecutive kx columns of one plane (all ny rows): one TMA load brings it
// into shared memory, the threads transform its columns with the two-level
// register FFT (regfft.cuh), and one TMA store writes it back.  Each block
// owns every gridDim.x-th tile and prefetches its next tile into the second
// buffer while it transforms the current one, so the copy engine keeps HBM
// busy while the SM computes.  Columns past nxh (padding, or the part of the
// last tile beyond the array) are transformed as well and are never read.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"
#include "gamma_onfly.cuh"
#include "regfft.cuh"
#include "tma.cuh"

namespace lsh {

template <int N> struct YTma {
  static constexpr int TY = 16;  // columns per tile: 128-byte FP32 complex rows
  static constexpr int P = RegPlan<N>::P;
  static constexpr int THREADS = TY * P;
  static constexpr int TILE = N * TY;                          // complex elements
  static constexpr int LS = RegLine<float, N>::LS;
  static constexpr size_t TILE_BYTES = sizeof(float2) * TILE;  // multiple of 128
  // shared memory: two tiles (128-byte aligned), exchange area, twiddles
  static constexpr size_t SMEM = 2 * TILE_BYTES + sizeof(float2) * (TY * LS + N) + 128;
};

template <bool INV, int N>
__global__ void __launch_bounds__(YTma<N>::THREADS) k_yfft_tma(const __grid_constant__ CUtensorMap tm, OpArgs<float> a,
                                                               const SolverState* __restrict__ st, int ntx,
                                                               long long ntiles) {
  typedef RegLine<float, N> RL;
  typedef YTma<N> YC;
  constexpr int TY = YC::TY, P = YC::P, R1 = RL::R1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  float2* tile[2] = {reinterpret_cast<float2*>(base), reinterpret_cast<float2*>(base + YC::TILE_BYTES)};
  float2* ex = reinterpret_cast<float2*>(base + 2 * YC::TILE_BYTES);
  float2* tw = ex + TY * YC::LS;
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int fault;
  for (int u = threadIdx.x; u < N; u += blockDim.x) tw[u] = a.twy[u];
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
    fault = 0;
  }
  __syncthreads();
  const int i = threadIdx.x % TY, t = threadIdx.x / TY;
  const long long pps = (long long)a.c * a.nz;  // planes per system
  auto live = [&](long long tl) {
    if (tl >= ntiles) return false;
    if (st == nullptr) return true;
    return st[(tl / ntx) / pps].done == 0;
  };
  auto issue = [&](long long tl, int b) {  // one thread
    const long long plane = tl / ntx;
    const int kx0 = (int)(tl - plane * ntx) * TY;
    mbar_expect_tx(&bar[b], (uint32_t)YC::TILE_BYTES);
    tma_load_3d(tile[b], &tm, 2 * kx0, 0, (int)plane, &bar[b]);
  };
  uint32_t par[2] = {0, 0};
  long long cur = blockIdx.x;
  bool cur_live = live(cur);
  if (cur_live && threadIdx.x == 0) issue(cur, 0);
  int b = 0;
  while (cur < ntiles) {
    const long long nxt = cur + gridDim.x;
    const bool nxt_live = live(nxt);
    if (nxt_live && threadIdx.x == 0) {
      bulk_wait_read_all();  // the store from this buffer has read it
      issue(nxt, b ^ 1);
    }
    if (cur_live) {
      const bool ok = mbar_wait(&bar[b], par[b]);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) fault = 1;
        break;  // par keeps the pending phase of this buffer for the final wait
      }
      par[b] ^= 1;
      float2* T = tile[b];
      float2 v[R1];
      if (!INV) {
#pragma unroll
        for (int j = 0; j < R1; ++j) v[j] = T[(t + P * j) * TY + i];
        RL::fwd_a(v, t, tw, ex + i * YC::LS);
        __syncthreads();
        RL::fwd_b(v, t, tw, ex + i * YC::LS);
#pragma unroll
        for (int m = 0; m < R1; ++m) T[RL::freq(t, m) * TY + i] = v[m];
      } else {
#pragma unroll
        for (int m = 0; m < R1; ++m) v[m] = T[RL::freq(t, m) * TY + i];
        RL::inv_a(v, t, tw, ex + i * YC::LS);
        __syncthreads();
        RL::inv_b(v, t, tw, ex + i * YC::LS);
#pragma unroll
        for (int j = 0; j < R1; ++j) T[(t + P * j) * TY + i] = v[j];
      }
      fence_proxy_async();
      __syncthreads();
      if (threadIdx.x == 0) {
        const long long plane = cur / ntx;
        const int kx0 = (int)(cur - plane * ntx) * TY;
        tma_store_3d(&tm, 2 * kx0, 0, (int)plane, T);
        bulk_commit();
      }
    }
    cur = nxt;
    cur_live = nxt_live;
    b ^= 1;
  }
  if (threadIdx.x == 0) {
    bulk_wait_all();
    // a load still in flight after a fault: give it the same bounded time
    if (fault) {
      mbar_wait(&bar[0], par[0]);
      mbar_wait(&bar[1], par[1]);
      atomicOr(a.fault, 1);
    }
  }
}


// ------------------------------------------------------------------ z pass + Gamma
// H seen as {2 hs floats, ny, nz, S c}; a tile is TZ kx columns at one y
// position, all nz planes, all NC components of one system: one 4-D box.
// Tiles run system-fastest, so the blocks working on the same (y, kx) tile of
// the systems of a launch read the same Gamma coefficients together (L2).
template <int NC, int N, int TZ_, int NB_> struct ZTma {
  static constexpr int TZ = TZ_;  // columns per tile (4: 32-byte, 8: 64-byte FP32 complex rows)
  static constexpr int NB = NB_;  // tile buffers: 2 = prefetch the next tile while computing
  static constexpr int P = RegPlan<N>::P;
  static constexpr int THREADS = TZ * P * NC;
  static constexpr int TILE = NC * N * TZ;
  static constexpr int LS = RegLine<float, N>::LS;
  static constexpr size_t TILE_BYTES = sizeof(float2) * TILE;  // multiple of 128
  static constexpr size_t SMEM = NB * TILE_BYTES + sizeof(float2) * (NC * TZ * LS + N) + 128;
  static constexpr bool FITS = SMEM <= 226 * 1024 && THREADS <= 1024;
  static constexpr int MINB = SMEM <= 110 * 1024 ? 2 : 1;
};

template <int NC, int N, int TZ, int NB>
__global__ void __launch_bounds__(ZTma<NC, N, TZ, NB>::THREADS, ZTma<NC, N, TZ, NB>::MINB)
    k_zgamma_tma(const __grid_constant__ CUtensorMap tm, OpArgs<float> a, const SolverState* __restrict__ st, int ntx,
                 long long ntiles) {
  typedef RegLine<float, N> RL;
  typedef ZTma<NC, N, TZ, NB> ZC;
  constexpr int P = ZC::P, R1 = RL::R1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  float2* tile[2] = {reinterpret_cast<float2*>(base),
                     reinterpret_cast<float2*>(base + (NB - 1) * ZC::TILE_BYTES)};
  float2* ex = reinterpret_cast<float2*>(base + NB * ZC::TILE_BYTES);
  float2* tw = ex + NC * TZ * ZC::LS;
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int fault;
  for (int u = threadIdx.x; u < N; u += blockDim.x) tw[u] = a.twz[u];
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
    fault = 0;
  }
  __syncthreads();
  // a warp runs along z for one component: conflict-free tile rows
  const int i = threadIdx.x % TZ, t = (threadIdx.x / TZ) % P, comp = threadIdx.x / (TZ * P);
  float2* exl = ex + (comp * TZ + i) * ZC::LS;
  const int S = a.S;
  auto live = [&](long long tl) {
    if (tl >= ntiles) return false;
    if (st == nullptr) return true;
    return st[tl % S].done == 0;
  };
  auto coords = [&](long long tl, int& s, int& yp, int& kx0) {
    s = (int)(tl % S);
    const long long sp = tl / S;
    yp = (int)(sp / ntx);
    kx0 = (int)(sp - (long long)yp * ntx) * TZ;
  };
  // one thread; with one buffer both tiles alternate barriers on the same area
  auto issue = [&](long long tl, int b) {
    int s, yp, kx0;
    coords(tl, s, yp, kx0);
    mbar_expect_tx(&bar[b], (uint32_t)ZC::TILE_BYTES);
    tma_load_4d(tile[b], &tm, 2 * kx0, yp, 0, s * NC, &bar[b]);
  };
  uint32_t par[2] = {0, 0};
  long long cur = blockIdx.x;
  bool cur_live = live(cur);
  if (cur_live && threadIdx.x == 0) issue(cur, 0);
  int b = 0;
  while (cur < ntiles) {
    const long long nxt = cur + gridDim.x;
    const bool nxt_live = live(nxt);
    if (NB == 2 && nxt_live && threadIdx.x == 0) {
      bulk_wait_read_all();
      issue(nxt, b ^ 1);
    }
    if (cur_live) {
      const bool ok = mbar_wait(&bar[b], par[b]);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) fault = 1;
        break;  // par keeps the pending phase of this buffer for the final wait
      }
      par[b] ^= 1;
      int s, yp, kx0;
      coords(cur, s, yp, kx0);
      float2* T = tile[b];
      float2* Tl = T + comp * N * TZ + i;  // this thread's line, stride TZ along z
      float2 v[R1];
#pragma unroll
      for (int j = 0; j < R1; ++j) v[j] = Tl[(t + P * j) * TZ];
      RL::fwd_a(v, t, tw, exl);
      __syncthreads();
      RL::fwd_b(v, t, tw, exl);
#pragma unroll
      for (int m = 0; m < R1; ++m) Tl[RL::freq(t, m) * TZ] = v[m];
      __syncthreads();
      // Gamma^h_k on the NC components of each frequency of the tile
      const int ky = a.kofy[yp];
      for (int item = threadIdx.x; item < N * TZ; item += ZC::THREADS) {
        const int kz = item / TZ, li = item - kz * TZ;
        const int kx = kx0 + li;
        if (kx >= a.nxh) continue;
        float2 g[NC];
#pragma unroll
        for (int c2 = 0; c2 < NC; ++c2) g[c2] = T[(c2 * N + kz) * TZ + li];
        if (a.onfly) {
          gamma_trunc_onfly<float, NC>(a, kx, ky, kz, g);
        } else {
          if (a.fdphase) fd_rotate<float, NC>(a, kx, ky, kz, g, -1.f);
          gamma_table_apply<float, NC>(a.gtab, ((long long)kz * a.ny + yp) * a.ts + kx, g);
          if (a.fdphase) fd_rotate<float, NC>(a, kx, ky, kz, g, 1.f);
        }
#pragma unroll
        for (int c2 = 0; c2 < NC; ++c2) T[(c2 * N + kz) * TZ + li] = g[c2];
      }
      __syncthreads();
#pragma unroll
      for (int m = 0; m < R1; ++m) v[m] = Tl[RL::freq(t, m) * TZ];
      RL::inv_a(v, t, tw, exl);
      __syncthreads();
      RL::inv_b(v, t, tw, exl);
#pragma unroll
      for (int j = 0; j < R1; ++j) Tl[(t + P * j) * TZ] = v[j];
      fence_proxy_async();
      __syncthreads();
      if (threadIdx.x == 0) {
        tma_store_4d(&tm, 2 * kx0, yp, 0, s * NC, T);
        bulk_commit();
      }
    }
    if (NB == 1 && nxt_live && threadIdx.x == 0) {
      bulk_wait_read_all();  // the store has read the only buffer
      issue(nxt, b ^ 1);
    }
    cur = nxt;
    cur_live = nxt_live;
    b ^= 1;
  }
  if (threadIdx.x == 0) {
    bulk_wait_all();
    if (fault) {
      mbar_wait(&bar[0], par[0]);
      mbar_wait(&bar[1], par[1]);
      atomicOr(a.fault, 1);
    }
  }
}

// Tiles of 16 columns (128-byte rows, the DRAM-friendly width along z): the
// FFT exchange runs in place in the tile, whose rows of 16 complex values make
// every warp access two whole 128-byte rows (no bank conflicts) and leave room
// for two buffers.  CPT components per thread (1 or 2) trades threads for
// registers.
template <int NC, int N, int CPT> struct ZTma16 {
  static constexpr int TZ = 16;
  static constexpr int P = RegPlan<N>::P;
  static constexpr int NCG = NC / CPT;  // component groups running together
  static constexpr int THREADS = TZ * P * NCG;
  static constexpr int TILE = NC * N * TZ;
  static constexpr size_t TILE_BYTES = sizeof(float2) * TILE;
  static constexpr int NB = 2 * TILE_BYTES + sizeof(float2) * N + 128 <= 200 * 1024 ? 2 : 1;
  static constexpr size_t SMEM = NB * TILE_BYTES + sizeof(float2) * N + 128;
  static constexpr bool FITS = SMEM <= 226 * 1024 && THREADS <= 1024 && NC % CPT == 0;
};

template <int NC, int N, int CPT>
__global__ void __launch_bounds__(ZTma16<NC, N, CPT>::THREADS, 1)
    k_zgamma_tma16(const __grid_constant__ CUtensorMap tm, OpArgs<float> a, const SolverState* __restrict__ st,
                   int ntx, long long ntiles) {
  typedef RegLine<float, N> RL;
  typedef ZTma16<NC, N, CPT> ZC;
  constexpr int TZ = 16, P = ZC::P, R1 = RL::R1, NB = ZC::NB, NCG = ZC::NCG;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  float2* tile[2] = {reinterpret_cast<float2*>(base),
                     reinterpret_cast<float2*>(base + (NB - 1) * ZC::TILE_BYTES)};
  float2* tw = reinterpret_cast<float2*>(base + NB * ZC::TILE_BYTES);
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int fault;
  for (int u = threadIdx.x; u < N; u += blockDim.x) tw[u] = a.twz[u];
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
    fault = 0;
  }
  __syncthreads();
  const int i = threadIdx.x % TZ, t = (threadIdx.x / TZ) % P, cg = threadIdx.x / (TZ * P);
  const int S = a.S;
  auto live = [&](long long tl) {
    if (tl >= ntiles) return false;
    if (st == nullptr) return true;
    return st[tl % S].done == 0;
  };
  auto coords = [&](long long tl, int& s, int& yp, int& kx0) {
    s = (int)(tl % S);
    const long long sp = tl / S;
    yp = (int)(sp / ntx);
    kx0 = (int)(sp - (long long)yp * ntx) * TZ;
  };
  auto issue = [&](long long tl, int b) {
    int s, yp, kx0;
    coords(tl, s, yp, kx0);
    mbar_expect_tx(&bar[b], (uint32_t)ZC::TILE_BYTES);
    tma_load_4d(tile[b], &tm, 2 * kx0, yp, 0, s * NC, &bar[b]);
  };
  uint32_t par[2] = {0, 0};
  long long cur = blockIdx.x;
  bool cur_live = live(cur);
  if (cur_live && threadIdx.x == 0) issue(cur, 0);
  int b = 0;
  while (cur < ntiles) {
    const long long nxt = cur + gridDim.x;
    const bool nxt_live = live(nxt);
    if (NB == 2 && nxt_live && threadIdx.x == 0) {
      bulk_wait_read_all();
      issue(nxt, b ^ 1);
    }
    if (cur_live) {
      const bool ok = mbar_wait(&bar[b], par[b]);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) fault = 1;
        break;  // par keeps the pending phase of this buffer for the final wait
      }
      par[b] ^= 1;
      int s, yp, kx0;
      coords(cur, s, yp, kx0);
      float2* T = tile[b];
      float2 v[R1];
#pragma unroll 1
      for (int k = 0; k < CPT; ++k) {
        float2* Tl = T + (cg + k * NCG) * N * TZ + i;
#pragma unroll
        for (int j = 0; j < R1; ++j) v[j] = Tl[(t + P * j) * TZ];
        __syncthreads();
        RL::template fwd_a_s<TZ>(v, t, tw, Tl);
        __syncthreads();
        RL::template fwd_b_s<TZ>(v, t, tw, Tl);
        __syncthreads();
#pragma unroll
        for (int m = 0; m < R1; ++m) Tl[RL::freq(t, m) * TZ] = v[m];
      }
      __syncthreads();
      const int ky = a.kofy[yp];
      for (int item = threadIdx.x; item < N * TZ; item += ZC::THREADS) {
        const int kz = item / TZ, li = item - kz * TZ;
        const int kx = kx0 + li;
        if (kx >= a.nxh) continue;
        float2 g[NC];
#pragma unroll
        for (int c2 = 0; c2 < NC; ++c2) g[c2] = T[(c2 * N + kz) * TZ + li];
        if (a.onfly) {
          gamma_trunc_onfly<float, NC>(a, kx, ky, kz, g);
        } else {
          if (a.fdphase) fd_rotate<float, NC>(a, kx, ky, kz, g, -1.f);
          gamma_table_apply<float, NC>(a.gtab, ((long long)kz * a.ny + yp) * a.ts + kx, g);
          if (a.fdphase) fd_rotate<float, NC>(a, kx, ky, kz, g, 1.f);
        }
#pragma unroll
        for (int c2 = 0; c2 < NC; ++c2) T[(c2 * N + kz) * TZ + li] = g[c2];
      }
      __syncthreads();
#pragma unroll 1
      for (int k = 0; k < CPT; ++k) {
        float2* Tl = T + (cg + k * NCG) * N * TZ + i;
#pragma unroll
        for (int m = 0; m < R1; ++m) v[m] = Tl[RL::freq(t, m) * TZ];
        __syncthreads();
        RL::template inv_a_s<TZ>(v, t, tw, Tl);
        __syncthreads();
        RL::template inv_b_s<TZ>(v, t, tw, Tl);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < R1; ++j) Tl[(t + P * j) * TZ] = v[j];
      }
      fence_proxy_async();
      __syncthreads();
      if (threadIdx.x == 0) {
        tma_store_4d(&tm, 2 * kx0, yp, 0, s * NC, T);
        bulk_commit();
      }
    }
    if (NB == 1 && nxt_live && threadIdx.x == 0) {
      bulk_wait_read_all();
      issue(nxt, b ^ 1);
    }
    cur = nxt;
    cur_live = nxt_live;
    b ^= 1;
  }
  if (threadIdx.x == 0) {
    bulk_wait_all();
    if (fault) {
      mbar_wait(&bar[0], par[0]);
      mbar_wait(&bar[1], par[1]);
      atomicOr(a.fault, 1);
    }
  }
}

// ------------------------------------------------------------------ host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

int sm_count() {
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

template <bool INV, int N> int y_blocks_per_sm() {
  static int n = []() {
    cudaFuncSetAttribute(k_yfft_tma<INV, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)YTma<N>::SMEM);
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_yfft_tma<INV, N>, YTma<N>::THREADS, YTma<N>::SMEM) !=
            cudaSuccess ||
        v < 1) {
      cudaGetLastError();
      v = 1;
    }
    return v;
  }();
  return n;
}

template <bool INV, int N> void launch_y_tma_n(const OpArgs<float>& a, const SolverState* st, cudaStream_t s) {
  const int ntx = (a.nxh + YTma<N>::TY - 1) / YTma<N>::TY;
  const long long ntiles = (long long)a.S * a.c * a.nz * ntx;
  const long long cap = (long long)sm_count() * y_blocks_per_sm<INV, N>();
  const int grid = (int)std::max<long long>(1, std::min<long long>(ntiles, cap));
  k_yfft_tma<INV, N><<<grid, YTma<N>::THREADS, YTma<N>::SMEM, s>>>(*a.tmy, a, st, ntx, ntiles);
}

template <int NC, int N, int TZ, int NB> int z_blocks_per_sm() {
  typedef ZTma<NC, N, TZ, NB> ZC;
  static int n = []() {
    int v = 0;
    if constexpr (ZC::FITS) {
      cudaFuncSetAttribute(k_zgamma_tma<NC, N, TZ, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZC::SMEM);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_zgamma_tma<NC, N, TZ, NB>, ZC::THREADS, ZC::SMEM) !=
          cudaSuccess) {
        cudaGetLastError();
        v = 0;
      }
    }
    return v;
  }();
  return n;
}

template <int NC, int N, int CPT> int z16_blocks_per_sm() {
  typedef ZTma16<NC, N, CPT> ZC;
  static int n = []() {
    int v = 0;
    if constexpr (ZC::FITS) {
      cudaFuncSetAttribute(k_zgamma_tma16<NC, N, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZC::SMEM);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_zgamma_tma16<NC, N, CPT>, ZC::THREADS, ZC::SMEM) !=
          cudaSuccess) {
        cudaGetLastError();
        v = 0;
      }
    }
    return v;
  }();
  return n;
}

template <int NC, int N, int CPT>
bool launch_z16(const OpArgs<float>& a, const SolverState* st, cudaStream_t s) {
  typedef ZTma16<NC, N, CPT> ZC;
  if constexpr (!ZC::FITS) {
    return false;
  } else {
    const int bpsm = z16_blocks_per_sm<NC, N, CPT>();
    if (bpsm < 1) return false;
    const int ntx = (a.nxh + 15) / 16;
    const long long ntiles = (long long)a.S * a.ny * ntx;
    const long long cap = (long long)sm_count() * bpsm;
    const int grid = (int)std::max<long long>(1, std::min<long long>(ntiles, cap));
    k_zgamma_tma16<NC, N, CPT><<<grid, ZC::THREADS, ZC::SMEM, s>>>(*a.tmz16, a, st, ntx, ntiles);
    return true;
  }
}

// Launch variant `var` (1: 4 columns double-buffered, 2: 8 columns single
// buffer, 3: 8 columns double-buffered, 4: 16 columns in-place exchange, 5:
// the same with two components per thread); false if it does not fit this
// length.
template <int NC, int N, int TZ, int NB>
bool launch_z_tma_v(const OpArgs<float>& a, const CUtensorMap* tm, const SolverState* st, cudaStream_t s) {
  typedef ZTma<NC, N, TZ, NB> ZC;
  if constexpr (!ZC::FITS) {
    return false;
  } else {
    const int bpsm = z_blocks_per_sm<NC, N, TZ, NB>();
    if (bpsm < 1) return false;
    const int ntx = (a.nxh + TZ - 1) / TZ;
    const long long ntiles = (long long)a.S * a.ny * ntx;
    const long long cap = (long long)sm_count() * bpsm;
    const int grid = (int)std::max<long long>(1, std::min<long long>(ntiles, cap));
    k_zgamma_tma<NC, N, TZ, NB><<<grid, ZC::THREADS, ZC::SMEM, s>>>(*tm, a, st, ntx, ntiles);
    return true;
  }
}

template <int NC, int N> bool launch_z_tma_n(const OpArgs<float>& a, int var, const SolverState* st, cudaStream_t s) {
  switch (var) {
    case 1: return launch_z_tma_v<NC, N, 4, 2>(a, a.tmz, st, s);
    case 2: return launch_z_tma_v<NC, N, 8, 1>(a, a.tmz8, st, s);
    case 3: return launch_z_tma_v<NC, N, 8, 2>(a, a.tmz8, st, s);
    case 4: return launch_z16<NC, N, 1>(a, st, s);
    case 5: return (NC % 2 == 0) ? launch_z16<NC, N, (NC % 2 == 0 ? 2 : 1)>(a, st, s) : false;
    default: return false;
  }
}

template <int NC> bool launch_z_tma_nc(const OpArgs<float>& a, int var, const SolverState* st, cudaStream_t s) {
  switch (a.nz) {
    case 16: return launch_z_tma_n<NC, 16>(a, var, st, s);
    case 32: return launch_z_tma_n<NC, 32>(a, var, st, s);
    case 64: return launch_z_tma_n<NC, 64>(a, var, st, s);
    case 128: return launch_z_tma_n<NC, 128>(a, var, st, s);
    default: return launch_z_tma_n<NC, 256>(a, var, st, s);
  }
}

template <int NC, int N> void z_prepare_n() {
  z_blocks_per_sm<NC, N, 4, 2>();
  z_blocks_per_sm<NC, N, 8, 1>();
  z_blocks_per_sm<NC, N, 8, 2>();
  z16_blocks_per_sm<NC, N, 1>();
  z16_blocks_per_sm<NC, N, (NC % 2 == 0 ? 2 : 1)>();
}

template <int NC> void z_prepare() {
  z_prepare_n<NC, 16>();
  z_prepare_n<NC, 32>();
  z_prepare_n<NC, 64>();
  z_prepare_n<NC, 128>();
  z_prepare_n<NC, 256>();
}

template <bool INV> void launch_y_tma_inv(const OpArgs<float>& a, const SolverState* st, cudaStream_t s) {
  switch (a.ny) {
    case 16: launch_y_tma_n<INV, 16>(a, st, s); break;
    case 32: launch_y_tma_n<INV, 32>(a, st, s); break;
    case 64: launch_y_tma_n<INV, 64>(a, st, s); break;
    case 128: launch_y_tma_n<INV, 128>(a, st, s); break;
    default: launch_y_tma_n<INV, 256>(a, st, s); break;
  }
}

}  // namespace

template <int NC, int N> bool z_fits_n(int var) {
  switch (var) {
    case 1: return ZTma<NC, N, 4, 2>::FITS && z_blocks_per_sm<NC, N, 4, 2>() > 0;
    case 2: return ZTma<NC, N, 8, 1>::FITS && z_blocks_per_sm<NC, N, 8, 1>() > 0;
    case 3: return ZTma<NC, N, 8, 2>::FITS && z_blocks_per_sm<NC, N, 8, 2>() > 0;
    case 4: return ZTma16<NC, N, 1>::FITS && z16_blocks_per_sm<NC, N, 1>() > 0;
    case 5: return NC % 2 == 0 && ZTma16<NC, N, (NC % 2 == 0 ? 2 : 1)>::FITS &&
                   z16_blocks_per_sm<NC, N, (NC % 2 == 0 ? 2 : 1)>() > 0;
    default: return false;
  }
}

template <int NC> bool z_fits_nc(int nz, int var) {
  switch (nz) {
    case 16: return z_fits_n<NC, 16>(var);
    case 32: return z_fits_n<NC, 32>(var);
    case 64: return z_fits_n<NC, 64>(var);
    case 128: return z_fits_n<NC, 128>(var);
    case 256: return z_fits_n<NC, 256>(var);
    default: return false;
  }
}

bool tma_z_variant_fits(const OpArgs<float>& a, int var) {
  if (a.c == 6) return z_fits_nc<6>(a.nz, var);
  if (a.c == 3) return z_fits_nc<3>(a.nz, var);
  return z_fits_nc<2>(a.nz, var);
}

bool launch_zgamma_tma(const OpArgs<float>& a, int var, const SolverState* st, cudaStream_t s) {
  if (a.c == 6) return launch_z_tma_nc<6>(a, var, st, s);
  if (a.c == 3) return launch_z_tma_nc<3>(a, var, st, s);
  return launch_z_tma_nc<2>(a, var, st, s);
}

void launch_yfft_tma(const OpArgs<float>& a, bool inv, const SolverState* st, cudaStream_t s) {
  if (inv) launch_y_tma_inv<true>(a, st, s);
  else launch_y_tma_inv<false>(a, st, s);
}

// Instantiate the launch attributes and occupancy of every TMA kernel once,
// outside any stream capture.
void tma_prepare() {
  (void)sm_count();
  (void)encode_fn();
  y_blocks_per_sm<false, 16>(); y_blocks_per_sm<true, 16>();
  y_blocks_per_sm<false, 32>(); y_blocks_per_sm<true, 32>();
  y_blocks_per_sm<false, 64>(); y_blocks_per_sm<true, 64>();
  y_blocks_per_sm<false, 128>(); y_blocks_per_sm<true, 128>();
  y_blocks_per_sm<false, 256>(); y_blocks_per_sm<true, 256>();
  z_prepare<2>();
  z_prepare<3>();
  z_prepare<6>();
}

// The tensor map of an FP32 half spectrum for the y pass: {2 hs, ny, planes}
// floats, box {2 TY, ny, 1}.  False when the driver entry point is missing or
// the geometry is not encodable (the caller then keeps the non-TMA pass).
bool encode_y_map(CUtensorMap* out, void* H, int hs, int ny, long long planes) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn || !reg_length(ny) || planes < 1 || planes > (1ll << 31) - 1) return false;
  if (((uintptr_t)H & 15) != 0 || (hs & 1) != 0) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * hs, (cuuint64_t)ny, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)hs * sizeof(float2), (cuuint64_t)hs * ny * sizeof(float2)};
  const cuuint32_t box[3] = {2 * 16, (cuuint32_t)ny, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, H, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace lsh

namespace lsh {

// The tensor map of an FP32 half spectrum for the z pass: {2 hs, ny, nz, S c}
// floats, box {2 tz, 1, nz, c}.
bool encode_z_map(CUtensorMap* out, void* H, int hs, int ny, int nz, int c, long long nsys, int tz) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn || !reg_length(nz) || nsys < 1 || nsys * c > (1ll << 31) - 1) return false;
  if (((uintptr_t)H & 15) != 0 || (hs & 1) != 0) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)2 * hs, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)(nsys * c)};
  const cuuint64_t strides[3] = {(cuuint64_t)hs * sizeof(float2), (cuuint64_t)hs * ny * sizeof(float2),
                                 (cuuint64_t)hs * ny * nz * sizeof(float2)};
  const cuuint32_t box[4] = {(cuuint32_t)(2 * tz), 1, (cuuint32_t)nz, (cuuint32_t)c};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, H, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Failure-path probe of the bounded waits: a barrier initialised for two
// arrivals receives one, so its phase never completes; the wait gives up after
// limit_ns and records the fault word exactly as a TMA kernel whose copies
// did not land would.  No copy is in flight.
__global__ void k_wait_probe(int* fault, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_arrive(&bar);
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, limit_ns);
  if (!ok && threadIdx.x == 0) atomicOr(fault, 1);
}

void launch_wait_probe(int* fault, unsigned long long limit_ns, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(fault, limit_ns);
}

}  // namespace lsh
