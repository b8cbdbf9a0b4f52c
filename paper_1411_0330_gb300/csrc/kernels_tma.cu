// kernels_tma.cu -- the y pass as a persistent, double-buffered TMA kernel
// (FP32 spectrum, lengths 16..256).
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
      par[b] ^= 1;
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) fault = 1;
        break;
      }
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
