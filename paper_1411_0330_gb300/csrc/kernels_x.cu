// kernels_x.cu -- the inverse x pass with the local term (FP32, lengths
// 16..256) on the two-level register FFT.
//
// A block owns RY consecutive rows of one system (RY/2 packed lines, P threads
// per line).  Its rows of the half spectrum are one contiguous range of H,
// copied to shared memory with 16-byte loads; each thread gathers the R1
// frequencies of its line it needs (X(N - k) = conj X(k) beyond the half),
// runs the register inverse FFT, and the real rows go back through shared
// memory to a coalesced epilogue: local term, projection on I0, the CG inner
// product and its deterministic per-system reduction -- the same epilogue as
// the shared-memory DIT kernel of kernels.cu.
#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"
#include "regfft.cuh"
#include "tma.cuh"

namespace lsh {

template <int N> struct XReg {
  static constexpr int P = RegPlan<N>::P;
  static constexpr int THREADS = 256;
  static constexpr int LINES = THREADS / P;  // packed lines (row pairs) per block
  static constexpr int RY = 2 * LINES;       // rows per block
  static constexpr int OSTR = N + 4;         // shared row stride of the real output (floats)
  static constexpr int LS = RegLine<float, N>::LS;
};

template <int N> size_t xreg_smem(int hs) {
  typedef XReg<N> XC;
  const size_t rows = std::max(sizeof(float2) * (size_t)XC::RY * hs, sizeof(float) * (size_t)XC::RY * XC::OSTR);
  const size_t rows16 = (rows + 15) & ~(size_t)15;
  return rows16 + sizeof(float2) * ((size_t)XC::LINES * XC::LS + N);
}

// MODE 0: out = P (M xin + g).  MODE 1 (CG): q = P (M p + g), (p, q) -> alpha.
// MODE 2 (residual): out = P (load - M xin - g), (r, r) -> st[s].aux[0].
template <int MODE, int N>
__global__ void __launch_bounds__(256, 2) k_xinv_reg(OpArgs<float> a, const float* __restrict__ xin,
                                                     float* __restrict__ out, SolverState* __restrict__ st,
                                                     double* __restrict__ partials, int bps, size_t rows_bytes) {
  typedef RegLine<float, N> RL;
  typedef XReg<N> XC;
  constexpr int P = XC::P, R1 = RL::R1, Q = RL::Q, RY = XC::RY, OSTR = XC::OSTR;
  const int s = blockIdx.x / bps;
  if (MODE == 1 && st[s].done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float mloc[256 * 6];
  __shared__ unsigned char aloc[256];
  __shared__ __align__(8) uint64_t bar;
  float2* HS = reinterpret_cast<float2*>(smem_raw);  // [RY][hs] spectrum rows, later [RY][OSTR] real rows
  float* OS = reinterpret_cast<float*>(smem_raw);
  float2* ex = reinterpret_cast<float2*>(smem_raw + rows_bytes);
  float2* tw = ex + XC::LINES * XC::LS;
  for (int u = threadIdx.x; u < N; u += blockDim.x) tw[u] = a.twx[u];
  const int ntab = a.nphase * a.c;
  for (int u = threadIdx.x; u < ntab; u += blockDim.x) mloc[u] = a.scale ? a.modtab[u] : a.mtab[u];
  for (int u = threadIdx.x; u < a.nphase; u += blockDim.x) aloc[u] = a.act[u];
  const int blk = blockIdx.x - s * bps;
  const int rloc = blk * RY;                            // first row inside the system
  const long long row0 = (long long)s * a.rps + rloc;  // global row
  const int hs = a.hs;
  // the block's spectrum rows are one contiguous range: a single bulk copy
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
    const uint32_t bytes = (uint32_t)(sizeof(float2) * (size_t)RY * hs);
    mbar_expect_tx(&bar, bytes);
    bulk_load_1d(HS, a.H + row0 * hs, bytes, &bar);
  }
  const int rows_per_comp = a.nz * a.ny;
  const long long pbase = (long long)((a.sys0 + s) / a.sys_per_ms) * a.V;
  constexpr int NV = N / 4;
  constexpr int IT = RY * NV / XC::THREADS;  // float4 groups per thread
  static_assert(RY * NV % XC::THREADS == 0, "epilogue tiling");
  // the epilogue's global loads go out while the copy and the FFT run
  float4 xq4s[IT];
  uchar4 ph4s[IT];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int idx = threadIdx.x + it * XC::THREADS;
    const int row = idx / NV;
    const int xx = (idx - row * NV) * 4;
    const int rs = rloc + row;
    const int comp = rs / rows_per_comp;
    const long long vox = (long long)(rs - comp * rows_per_comp) * N + xx;
    xq4s[it] = *reinterpret_cast<const float4*>(xin + (row0 + row) * N + xx);
    ph4s[it] = *reinterpret_cast<const uchar4*>(a.phase + pbase + vox);
  }
  __syncthreads();
  if (__syncthreads_or(!mbar_wait(&bar, 0))) {
    if (threadIdx.x == 0) {
      mbar_wait(&bar, 0);
      atomicOr(a.fault, 1);
    }
    return;
  }
  const int t = threadIdx.x % P, l = threadIdx.x / P;
  float2 v[R1];
  {
    const float2* xa_row = HS + (2 * l) * hs;
    const float2* xb_row = xa_row + hs;
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int f = t * Q + q + R1 * u;
        const bool lo = f <= N / 2;
        const int k = lo ? f : N - f;
        const float sg = lo ? 1.f : -1.f;
        const float2 xa = xa_row[k], xb = xb_row[k];
        // Z(f) = X_a(f) + i X_b(f), X(N - k) = conj X(k)
        v[q * P + u] = make_float2(xa.x - sg * xb.y, sg * xa.y + xb.x);
      }
  }
  float2* exl = ex + l * XC::LS;
  RL::inv_a(v, t, tw, exl);
  __syncthreads();
  RL::inv_b(v, t, tw, exl);
  // real rows 2l (Re) and 2l + 1 (Im); HS is no longer read
#pragma unroll
  for (int j = 0; j < R1; ++j) {
    OS[(2 * l) * OSTR + t + P * j] = v[j].x;
    OS[(2 * l + 1) * OSTR + t + P * j] = v[j].y;
  }
  __syncthreads();
  Acc<float> acc;
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int idx = threadIdx.x + it * XC::THREADS;
    const int row = idx / NV;
    const int xx = (idx - row * NV) * 4;
    const int rs = rloc + row;
    const int comp = rs / rows_per_comp;
    const long long vox = (long long)(rs - comp * rows_per_comp) * N + xx;
    const long long g = (row0 + row) * N + xx;
    const float4 xq4 = xq4s[it];
    const uchar4 ph4 = ph4s[it];
    const float4 g4 = *reinterpret_cast<const float4*>(OS + row * OSTR + xx);
    const float xq[4] = {xq4.x, xq4.y, xq4.z, xq4.w};
    const unsigned char ph[4] = {ph4.x, ph4.y, ph4.z, ph4.w};
    const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
    float ov[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int p = ph[u];
      const bool active = aloc[p] != 0;
      float m = mloc[p * a.c + comp];
      if (a.scale) m = 1.f / (a.scale[pbase + vox + u] * m - a.ref[comp]);
      if (MODE == 0) {
        ov[u] = active ? m * xq[u] + gv[u] : 0.f;
      } else if (MODE == 1) {
        ov[u] = active ? m * xq[u] + gv[u] : 0.f;
        acc.add(xq[u] * ov[u]);
      } else {
        ov[u] = active ? a.loads[s * 6 + comp] - (m * xq[u] + gv[u]) : 0.f;
        acc.add(ov[u] * ov[u]);
      }
    }
    *reinterpret_cast<float4*>(out + g) = make_float4(ov[0], ov[1], ov[2], ov[3]);
  }
  if (MODE != 0) {
    const double tot = block_reduce(acc);
    double* part = partials + (long long)s * bps;
    SolverState* sst = st + s;
    if (publish_partial_sys(part, blk, bps, tot, &sst->counter[0])) {
      const double sum = gather_partials_sys(part, bps, &sst->counter[0]);
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
        } else {
          sst->aux[0] = sum;
        }
      }
    }
  }
}

namespace {

template <int N> bool launch_xinv_reg_n(const OpArgs<float>& a, int mode, const float* xin, float* out,
                                        SolverState* st, double* partials, cudaStream_t s) {
  typedef XReg<N> XC;
  if (a.rps % XC::RY != 0 || (a.hs & 1)) return false;
  const int bps = a.rps / XC::RY;
  const size_t rows = std::max(sizeof(float2) * (size_t)XC::RY * a.hs, sizeof(float) * (size_t)XC::RY * XC::OSTR);
  const size_t rows16 = (rows + 15) & ~(size_t)15;
  const size_t smem = xreg_smem<N>(a.hs);
  if (smem > 200 * 1024) return false;
  const int grid = a.S * bps;
  if (mode == 0) k_xinv_reg<0, N><<<grid, XC::THREADS, smem, s>>>(a, xin, out, st, partials, bps, rows16);
  else if (mode == 1) k_xinv_reg<1, N><<<grid, XC::THREADS, smem, s>>>(a, xin, out, st, partials, bps, rows16);
  else k_xinv_reg<2, N><<<grid, XC::THREADS, smem, s>>>(a, xin, out, st, partials, bps, rows16);
  return true;
}

template <int N> void xreg_attrs() {
  const int mx = 200 * 1024;
  cudaFuncSetAttribute(k_xinv_reg<0, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_reg<1, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_reg<2, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

}  // namespace

bool xinv_reg_fits(const OpArgs<float>& a) {
  switch (a.nx) {
    case 16: return a.rps % XReg<16>::RY == 0 && xreg_smem<16>(a.hs) <= 200 * 1024;
    case 32: return a.rps % XReg<32>::RY == 0 && xreg_smem<32>(a.hs) <= 200 * 1024;
    case 64: return a.rps % XReg<64>::RY == 0 && xreg_smem<64>(a.hs) <= 200 * 1024;
    case 128: return a.rps % XReg<128>::RY == 0 && xreg_smem<128>(a.hs) <= 200 * 1024;
    case 256: return a.rps % XReg<256>::RY == 0 && xreg_smem<256>(a.hs) <= 200 * 1024;
    default: return false;
  }
}

// False when this grid has no register inverse x pass (the caller keeps the
// shared-memory kernel).
bool launch_xinv_reg(const OpArgs<float>& a, int mode, const float* xin, float* out, SolverState* st,
                     double* partials, cudaStream_t s) {
  switch (a.nx) {
    case 16: return launch_xinv_reg_n<16>(a, mode, xin, out, st, partials, s);
    case 32: return launch_xinv_reg_n<32>(a, mode, xin, out, st, partials, s);
    case 64: return launch_xinv_reg_n<64>(a, mode, xin, out, st, partials, s);
    case 128: return launch_xinv_reg_n<128>(a, mode, xin, out, st, partials, s);
    case 256: return launch_xinv_reg_n<256>(a, mode, xin, out, st, partials, s);
    default: return false;
  }
}

void xreg_prepare() {
  xreg_attrs<16>();
  xreg_attrs<32>();
  xreg_attrs<64>();
  xreg_attrs<128>();
  xreg_attrs<256>();
}

}  // namespace lsh
