// kernels_zpipe.cu -- FP32 z pass with the Green-operator product (Eq. (13):
// z transform, Gamma^h_k, inverse z transform) on the ky-major spectrum of the
// plane passes, fed and drained by the Tensor Memory Accelerator.
//
// A tile is 8 consecutive kx columns of one (system, ky) slab, every component
// and every z (one 4-D TMA box of NC N rows of 64 bytes), or 8 consecutive ky
// of the Nyquist column kx = nx/2 (one 3-D box of the same shape).  Blocks are
// persistent and double-buffered: the next tile's box is requested before the
// current tile is transformed, and every exchange of the two-level register FFT
// (regfft.cuh) and of the Gamma^h product runs in place in the tile's buffer, so
// that two buffers per block leave room for a second block on the SM.  The
// result leaves through one TMA store from the same buffer.
//
// Two variants.  The unfused one (variant 10) runs the register plans of
// regfft.cuh; the c components of each frequency then meet for the Gamma^h
// product in a layout of their own.  The fused one (variant 11) runs the plan
// N = R1 x 4 and lets one thread per (k1, column) take the 4-point transforms
// of all components, the product and the inverse 4-point transforms in
// registers: two fewer exchanges and four fewer barriers per tile.
//
// Buffer layouts (a row is the 8 columns of one component at one position, 64
// bytes; rows alternate between the two 64-byte halves of a 128-byte bank row):
//   dense (the TMA box)          row c N + z
//   unfused: transform exchange  row c NX + e + e / R1   (NX = N + N / R1)
//            Gamma^h product     row c N + kz ^ ((kz / Q) & 1) for even Q = R1 / P,
//                                row c N + kz for odd Q
//   fused: transform exchange    row c N + (e ^ ((e >> 2) & 1))
// A warp holds the 8 columns of 4 consecutive line positions t of one
// component (in the fused product phase: of 4 consecutive k1); in each layout
// the four rows a warp touches split two and two between the halves (no bank
// conflicts), and every offset is a compile-time constant from one of a few
// per-thread bases.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "gamma_onfly.cuh"
#include "internal.h"
#include "regfft.cuh"
#include "tma.cuh"

namespace lsh {

// FUSED: every length runs the plan N = R1 x 4 (P = 4); one thread per (k1,
// column) takes the 4-point DFTs of all NC components, the Gamma^h product at
// its 4 frequencies k1 + R1 k2 and the inverse 4-point DFTs in registers (the
// (k1, column) pairs go round the block when there are more of them than
// threads).  Its exchange needs no padding: element e sits in row
// e ^ ((e >> 2) & 1), which splits the four rows of every warp access two and
// two between the bank halves both when 4 threads t write k1 P + t and when 4
// consecutive k1 read k1 P + u.
template <int N, bool FUSED> struct ZPlan {
  static constexpr int P = FUSED ? 4 : RegPlan<N>::P, R1 = FUSED ? N / 4 : RegPlan<N>::R1;
};
template <int NC, int N, bool FUSED = false> struct ZPipe {
  static constexpr int TZ = 8;                   // columns per tile
  static constexpr int P = ZPlan<N, FUSED>::P, R1 = ZPlan<N, FUSED>::R1, Q = R1 / P;
  static constexpr int THREADS = TZ * P * NC;
  static constexpr int NX = FUSED ? N : N + N / R1;  // exchange rows per component
  static constexpr bool FUSABLE = R1 <= 32;      // register DFTs of up to 32 points
  static constexpr int BUF = NC * NX * TZ;       // complex values per buffer
  static constexpr uint32_t BOX_BYTES = (uint32_t)(sizeof(float2) * NC * N * TZ);
  static constexpr size_t SMEM = 2 * sizeof(float2) * BUF + sizeof(float2) * N + 128;
  static constexpr bool FITS = THREADS <= 1024 && SMEM <= 227 * 1024 && (NX % 2) == 0 && (!FUSED || FUSABLE);
  static constexpr int MINB = (2 * SMEM <= 226 * 1024 && 2 * THREADS <= 1024) ? 2 : 1;
};

// Row of frequency kz in the Gamma^h layout (a permutation of 0..N-1).
template <int Q> __device__ __forceinline__ int zp_grow(int kz) {
  if constexpr ((Q & 1) == 0) return kz ^ ((kz / Q) & 1);
  else return kz;
}

// The middle of the FUSED kernel: thread (k1, column li) reads element k1 P + u
// (u < P) of every component's line from the exchange (row 4 k1 + (u ^ (k1 & 1))),
// transforms over u, applies Gamma^h_k at kz = k1 + R1 k2 to the NC components
// of each k2, transforms back and writes the same rows.  The coefficients of
// the next k2 load while the current ones are applied.
template <int NC, int N>
__device__ __forceinline__ void zp_fused_item(const OpArgs<float>& a, float2* B, int item, bool nyq, int yp,
                                              int kx0) {
  typedef ZPipe<NC, N, true> ZC;
  constexpr int TZ = ZC::TZ, P = ZC::P, R1 = ZC::R1, NX = ZC::NX;
  const int li = item & (TZ - 1), k1 = item / TZ, kb = k1 & 1;
  // rows of even u one up for odd k1, rows of odd u one down
  float2* const ev = B + (4 * k1 + kb) * TZ + li;
  float2* const od = B + (4 * k1 - kb) * TZ + li;
  const int kx = nyq ? kx0 : kx0 + li, ypos = nyq ? yp + li : yp;
  float2 d[NC][P];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
#pragma unroll
    for (int u = 0; u < P; ++u) d[c][u] = ((u & 1) ? od : ev)[(c * NX + u) * TZ];
    Dft<float, P, false>::run(d[c], nullptr, N);
  }
  if (a.onfly) {
    const int ky = a.kofy[ypos];
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) {
      float2 g[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) g[c] = d[c][k2];
      gamma_trunc_onfly<float, NC>(a, kx, ky, k1 + R1 * k2, g);
#pragma unroll
      for (int c = 0; c < NC; ++c) d[c][k2] = g[c];
    }
  } else {
    constexpr int NCO = GammaPack<NC>::NCO;
    const long long f0 = ((long long)k1 * a.ny + ypos) * a.ts + kx;  // frequency (kx, ky, k1)
    const long long fs = (long long)R1 * a.ny * a.ts;                // kz step R1
    float gc[2][NCO];
    gamma_coef_load<float, NC>(a.gtab, f0, gc[0]);
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) {
      if (k2 + 1 < P) gamma_coef_load<float, NC>(a.gtab, f0 + (k2 + 1) * fs, gc[(k2 + 1) & 1]);
      float2 g[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) g[c] = d[c][k2];
      if (a.fdphase) fd_rotate<float, NC>(a, kx, a.kofy[ypos], k1 + R1 * k2, g, -1.f);
      gamma_coef_apply<float, NC>(gc[k2 & 1], g);
      if (a.fdphase) fd_rotate<float, NC>(a, kx, a.kofy[ypos], k1 + R1 * k2, g, 1.f);
#pragma unroll
      for (int c = 0; c < NC; ++c) d[c][k2] = g[c];
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    Dft<float, P, true>::run(d[c], nullptr, N);
#pragma unroll
    for (int u = 0; u < P; ++u) ((u & 1) ? od : ev)[(c * NX + u) * TZ] = d[c][u];
  }
}

template <int NC, int N, bool FUSED>
__global__ void __launch_bounds__(ZPipe<NC, N, FUSED>::THREADS, ZPipe<NC, N, FUSED>::MINB)
    k_zgamma_pipe(const __grid_constant__ CUtensorMap tmH, const __grid_constant__ CUtensorMap tmQ, OpArgs<float> a,
                  const SolverState* __restrict__ st, int nkt, int nregular, int total) {
  typedef ZPipe<NC, N, FUSED> ZC;
  constexpr int TZ = ZC::TZ, P = ZC::P, R1 = ZC::R1, Q = ZC::Q, NX = ZC::NX, THREADS = ZC::THREADS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // 128-byte aligned start, kept as an offset into the shared array (shared-window accesses)
  float2* const buf0 = reinterpret_cast<float2*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));
  float2* const tw = buf0 + 2 * ZC::BUF;  // buffer b at buf0 + b BUF
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int fault;
  // the tile each buffer holds, published by warp 0: live, system, y position, first kx
  __shared__ int tile_live[2], tile_s[2], tile_yp[2], tile_kx0[2];
  for (int u = threadIdx.x; u < N; u += THREADS) tw[u] = a.twz[u];
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
    fault = 0;
  }
  __syncthreads();

  // Warp 0 walks the block's tiles (grid stride, skipping converged systems),
  // requests each box one tile ahead and brings the tile's Gamma rows into L2.
  // Regular tiles are ordered (ky, system, kx tile) -- the kx tiles of a slab run
  // together, and so do the systems sharing the tile's Gamma rows -- then come
  // the Nyquist tiles (system, ky tile).
  int tl_next = blockIdx.x;  // warp 0: the next tile index to consider
  auto advance = [&](int b) {
    const int S = a.S, nqt = a.ny / TZ;
    int s = 0, yp = 0, kx0 = 0, tl = tl_next;
    for (; tl < total; tl += gridDim.x) {
      if (tl < nregular) {
        const int ys = tl / nkt;
        kx0 = (tl - ys * nkt) * TZ;
        yp = ys / S;
        s = ys - yp * S;
      } else {
        const int l = tl - nregular;
        s = l / nqt;
        yp = (l - s * nqt) * TZ;
        kx0 = a.nx / 2;
      }
      if (st == nullptr || !st[s].done) break;
    }
    tl_next = tl + gridDim.x;
    const bool live = tl < total;
    if (threadIdx.x == 0) {
      tile_live[b] = live;
      tile_s[b] = s;
      tile_yp[b] = yp;
      tile_kx0[b] = kx0;
      if (live) {
        bulk_wait_read_all();  // the store of the buffer's previous tile has read it
        mbar_expect_tx(&bar[b], ZC::BOX_BYTES);
        if (tl < nregular) tma_load_4d(buf0 + b * ZC::BUF, &tmH, 2 * kx0, 0, yp, s * NC, &bar[b]);
        else tma_load_3d(buf0 + b * ZC::BUF, &tmQ, 2 * yp, 0, s * NC, &bar[b]);
      }
    }
    if (live && tl < nregular && s == 0 && !a.onfly) {
      constexpr int NCOP = GammaPack<NC>::NCOP;
      for (int kz = threadIdx.x; kz < N; kz += 32)
        bulk_prefetch_l2(a.gtab + (((long long)kz * a.ny + yp) * a.ts + kx0) * NCOP,
                         (uint32_t)(sizeof(float) * TZ * NCOP));
    }
  };

  const int i = threadIdx.x & (TZ - 1), t = (threadIdx.x / TZ) % P, comp = threadIdx.x / (TZ * P);
  // per-thread bases (complex offsets within a buffer)
  const int od = (comp * N + t) * TZ + i;             // dense: x[t + P j] at od + j P TZ
  // exchange, element k1 P + t: row k1 P + k1 / Q + t, or (FUSED) 4 k1 + (t ^ (k1 & 1))
  const int oa = (comp * NX + t) * TZ + i;
  const int oa1 = (comp * NX + (FUSED ? (t ^ 1) : t)) * TZ + i;  // odd k1 (FUSED)
  auto xa = [&](int k1) { return FUSED ? ((k1 & 1) ? oa1 : oa) + 4 * k1 * TZ : oa + (k1 * P + k1 / Q) * TZ; };
  const int ob = (comp * NX + t * (R1 + 1)) * TZ + i; // exchange, element (t Q + q) P + u
  // Gamma layout, frequency kz(m) = t Q + m / P + R1 (m % P): for even Q its row
  // is kz ^ (t & 1), i.e. one row up or down by the parity of m / P
  const int og0 = (comp * N + t * Q + (((Q & 1) == 0) ? (t & 1) : 0)) * TZ + i;
  const int og1 = (comp * N + t * Q - (((Q & 1) == 0) ? (t & 1) : 0)) * TZ + i;

  if (threadIdx.x < 32) advance(0);
  __syncthreads();
  uint32_t par = 0;  // bit b: parity of the next phase of buffer b's barrier
  int b = 0;
  while (tile_live[b]) {
    const int s = tile_s[b], yp = tile_yp[b], kx0 = tile_kx0[b];
    const bool nyq = 2 * kx0 == a.nx;
    if (threadIdx.x < 32) advance(b ^ 1);
    const bool ok = mbar_wait(&bar[b], (par >> b) & 1u);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) fault = 1;
      break;  // par still holds the pending phases of both buffers
    }
    par ^= 1u << b;
    float2* const B = buf0 + b * ZC::BUF;
    float2 v[R1];
    // forward transform along z (tw[0] = 1: thread t = 0 multiplies by one)
#pragma unroll
    for (int j = 0; j < R1; ++j) v[j] = B[od + j * P * TZ];
    __syncthreads();
    Dft<float, R1, false>::run(v, tw, N);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul<float>(v[k1], tw[t * k1]);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) B[xa(k1)] = v[k1];
    __syncthreads();
    if constexpr (FUSED) {
      for (int item = threadIdx.x; item < R1 * TZ; item += THREADS) zp_fused_item<NC, N>(a, B, item, nyq, yp, kx0);
    } else {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      float2 c[P];
#pragma unroll
      for (int u = 0; u < P; ++u) c[u] = B[ob + (q * P + u) * TZ];
      Dft<float, P, false>::run(c, tw, N);
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) v[q * P + k2] = c[k2];
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < R1; ++m) B[(((m / P) & 1) ? og1 : og0) + ((m / P) + R1 * (m % P)) * TZ] = v[m];
    __syncthreads();
    // Gamma^h_k on the NC components of each of the tile's N x 8 frequencies
    {
      // frequency `item` = kz TZ + li of the tile: its y position and kx
      auto ypos = [&](int li) { return nyq ? yp + li : yp; };
      auto kxof = [&](int li) { return nyq ? kx0 : kx0 + li; };
      auto gptr = [&](int item) { return B + zp_grow<Q>(item / TZ) * TZ + (item & (TZ - 1)); };
      if (a.onfly) {
        for (int item = threadIdx.x; item < N * TZ; item += THREADS) {
          const int kz = item / TZ, li = item & (TZ - 1);
          float2* gp = gptr(item);
          float2 g[NC];
#pragma unroll
          for (int c2 = 0; c2 < NC; ++c2) g[c2] = gp[c2 * N * TZ];
          gamma_trunc_onfly<float, NC>(a, kxof(li), a.kofy[ypos(li)], kz, g);
#pragma unroll
          for (int c2 = 0; c2 < NC; ++c2) gp[c2 * N * TZ] = g[c2];
        }
      } else {
        // tabulated coefficients, loaded one frequency ahead into two register
        // sets used in turn (no copies between them)
        constexpr int NCO = GammaPack<NC>::NCO;
        auto off = [&](int item) {
          const int li = item & (TZ - 1);
          return ((long long)(item / TZ) * a.ny + ypos(li)) * a.ts + kxof(li);
        };
        auto apply = [&](int item, const float* gc) {
          const int kz = item / TZ, li = item & (TZ - 1);
          float2* gp = gptr(item);
          float2 g[NC];
#pragma unroll
          for (int c2 = 0; c2 < NC; ++c2) g[c2] = gp[c2 * N * TZ];
          if (a.fdphase) fd_rotate<float, NC>(a, kxof(li), a.kofy[ypos(li)], kz, g, -1.f);
          gamma_coef_apply<float, NC>(gc, g);
          if (a.fdphase) fd_rotate<float, NC>(a, kxof(li), a.kofy[ypos(li)], kz, g, 1.f);
#pragma unroll
          for (int c2 = 0; c2 < NC; ++c2) gp[c2 * N * TZ] = g[c2];
        };
        float ga[NCO], gb[NCO];
        int item = threadIdx.x;
        if (item < N * TZ) gamma_coef_load<float, NC>(a.gtab, off(item), ga);
#pragma unroll 1
        for (; item < N * TZ; item += 2 * THREADS) {
          const int i1 = item + THREADS, i2 = item + 2 * THREADS;
          if (i1 < N * TZ) gamma_coef_load<float, NC>(a.gtab, off(i1), gb);
          apply(item, ga);
          if (i1 >= N * TZ) break;
          if (i2 < N * TZ) gamma_coef_load<float, NC>(a.gtab, off(i2), ga);
          apply(i1, gb);
        }
      }
    }
    __syncthreads();
    // inverse transform along z
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = B[(((m / P) & 1) ? og1 : og0) + ((m / P) + R1 * (m % P)) * TZ];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      float2 c[P];
#pragma unroll
      for (int u = 0; u < P; ++u) c[u] = v[q * P + u];
      Dft<float, P, true>::run(c, tw, N);
#pragma unroll
      for (int u = 0; u < P; ++u) B[ob + (q * P + u) * TZ] = c[u];
    }
    }  // !FUSED
    __syncthreads();
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = B[xa(k1)];
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmulc<float>(v[k1], tw[t * k1]);
    Dft<float, R1, true>::run(v, tw, N);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < R1; ++j) B[od + j * P * TZ] = v[j];
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!nyq) tma_store_4d(&tmH, 2 * kx0, 0, yp, s * NC, B);
      else tma_store_3d(&tmQ, 2 * yp, 0, s * NC, B);
      bulk_commit();
    }
    b ^= 1;
  }
  if (threadIdx.x == 0) {
    bulk_wait_all();
    if (fault) {
      // a box still in flight lands before the block's shared memory is released
      if (tile_live[b ^ 1]) mbar_wait(&bar[b ^ 1], (par >> (b ^ 1)) & 1u);
      mbar_wait(&bar[b], (par >> b) & 1u);
      atomicOr(a.fault, 1);
    }
  }
}

// ------------------------------------------------------------------ host side
namespace {

template <int NC, int N, bool FUSED> int zpipe_blocks_per_sm() {
  typedef ZPipe<NC, N, FUSED> ZC;
  static int n = []() {
    int v = 0;
    if constexpr (ZC::FITS) {
      cudaFuncSetAttribute(k_zgamma_pipe<NC, N, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZC::SMEM);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_zgamma_pipe<NC, N, FUSED>, ZC::THREADS, ZC::SMEM) !=
          cudaSuccess) {
        cudaGetLastError();
        v = 0;
      }
    }
    return v;
  }();
  return n;
}

template <int NC, int N, bool FUSED>
bool launch_zpipe_n(const OpArgs<float>& a, const SolverState* st, cudaStream_t s) {
  typedef ZPipe<NC, N, FUSED> ZC;
  if constexpr (!ZC::FITS) {
    return false;
  } else {
    const int bpsm = zpipe_blocks_per_sm<NC, N, FUSED>();
    if (bpsm < 1) return false;
    if (a.S < 1) return true;
    const int nkt = (a.nx / 2) / ZC::TZ;
    const long long nregular = (long long)a.ny * a.S * nkt;
    const long long total = nregular + (long long)a.S * (a.ny / ZC::TZ);
    const long long grid = std::max<long long>(1, std::min<long long>(total, (long long)multiprocessors() * bpsm));
    if (total + grid >= (1ll << 31)) return false;
    k_zgamma_pipe<NC, N, FUSED><<<(unsigned)grid, ZC::THREADS, ZC::SMEM, s>>>(*a.tmzp, *a.tmzq, a, st, nkt,
                                                                              (int)nregular, (int)total);
    return true;
  }
}

template <int NC, bool FUSED> bool launch_zpipe_nc(const OpArgs<float>& a, const SolverState* st, cudaStream_t s) {
  switch (a.nz) {
    case 16: return launch_zpipe_n<NC, 16, FUSED>(a, st, s);
    case 32: return launch_zpipe_n<NC, 32, FUSED>(a, st, s);
    case 48: return launch_zpipe_n<NC, 48, FUSED>(a, st, s);
    case 64: return launch_zpipe_n<NC, 64, FUSED>(a, st, s);
    case 96: return launch_zpipe_n<NC, 96, FUSED>(a, st, s);
    case 128: return launch_zpipe_n<NC, 128, FUSED>(a, st, s);
    case 256: return launch_zpipe_n<NC, 256, FUSED>(a, st, s);
    default: return false;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 zp_encode_fn() {
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

}  // namespace

// Pipelined TMA z pass on the ky-major spectrum (fused: the P = 4 variant that
// takes the level-b DFTs and Gamma^h in one register phase); false (nothing launched) when
// the spectrum is not ky-major, the maps are missing, the geometry has no
// tiling or the kernel does not fit.  With a.S = 0 it only answers whether it
// would launch.
bool launch_zgamma_pipe(const OpArgs<float>& a, bool fused, const SolverState* st, cudaStream_t s) {
  if (!a.tlay || a.nq == nullptr || a.tmzp == nullptr || a.tmzq == nullptr) return false;
  if ((a.nx & 15) != 0 || (a.ny & 7) != 0) return false;  // whole 8-column tiles of kx < nx/2 and of ky
  if (a.c == 6) return fused ? launch_zpipe_nc<6, true>(a, st, s) : launch_zpipe_nc<6, false>(a, st, s);
  if (a.c == 3) return fused ? launch_zpipe_nc<3, true>(a, st, s) : launch_zpipe_nc<3, false>(a, st, s);
  return false;
}

// Tensor maps of the ky-major FP32 spectrum H[S c][ky][z][hs] ({2 hs, nz, ny, S c}
// floats, box {16, nz, 1, c}) and of its Nyquist columns NQ[S c][z][ky]
// ({2 ny, nz, S c} floats, box {16, nz, c}).  False when the driver entry point
// is missing or the geometry is not encodable.
bool encode_zpipe_maps(CUtensorMap* th, CUtensorMap* tq, void* H, void* NQ, int hs, int ny, int nz, int c,
                       long long nsys) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = zp_encode_fn();
  if (!fn || nz < 1 || nz > 256 || c < 1 || c > 6 || nsys < 1 || nsys * c > (1ll << 31) - 1) return false;
  if (((uintptr_t)H & 15) != 0 || ((uintptr_t)NQ & 15) != 0 || (hs & 1) != 0 || (ny & 7) != 0) return false;
  const cuuint64_t dh[4] = {(cuuint64_t)2 * hs, (cuuint64_t)nz, (cuuint64_t)ny, (cuuint64_t)(nsys * c)};
  const cuuint64_t sh[3] = {(cuuint64_t)hs * sizeof(float2), (cuuint64_t)hs * nz * sizeof(float2),
                            (cuuint64_t)hs * nz * ny * sizeof(float2)};
  const cuuint32_t bh[4] = {16, (cuuint32_t)nz, 1, (cuuint32_t)c};
  const cuuint32_t e4[4] = {1, 1, 1, 1};
  if (fn(th, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, H, dh, sh, bh, e4, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS)
    return false;
  const cuuint64_t dq[3] = {(cuuint64_t)2 * ny, (cuuint64_t)nz, (cuuint64_t)(nsys * c)};
  const cuuint64_t sq[2] = {(cuuint64_t)ny * sizeof(float2), (cuuint64_t)ny * nz * sizeof(float2)};
  const cuuint32_t bq[3] = {16, (cuuint32_t)nz, (cuuint32_t)c};
  const cuuint32_t e3[3] = {1, 1, 1};
  return fn(tq, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, NQ, dq, sq, bq, e3, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <int NC, bool FUSED> void zpipe_prepare_nc() {
  zpipe_blocks_per_sm<NC, 16, FUSED>();
  zpipe_blocks_per_sm<NC, 32, FUSED>();
  zpipe_blocks_per_sm<NC, 48, FUSED>();
  zpipe_blocks_per_sm<NC, 64, FUSED>();
  zpipe_blocks_per_sm<NC, 96, FUSED>();
  zpipe_blocks_per_sm<NC, 128, FUSED>();
  zpipe_blocks_per_sm<NC, 256, FUSED>();
}

void zpipe_prepare() {
  zpipe_prepare_nc<3, false>();
  zpipe_prepare_nc<6, false>();
  zpipe_prepare_nc<3, true>();
  zpipe_prepare_nc<6, true>();
}

}  // namespace lsh
