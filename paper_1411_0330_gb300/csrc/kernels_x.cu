// kernels_x.cu -- the x passes (FP32, lengths 16..256) on the two-level
// register FFT, with bulk copies between HBM and shared memory.
//
// Forward: a block owns RY consecutive rows of one system.  The CG prologue
// (x += alpha p_old, p = r + beta p_old) or the projection on I0 (apply) runs
// on rows brought in by bulk copies; two real rows form one complex line, the
// register FFT transforms it, the two Hermitian half rows are split out and
// one bulk store writes the block's contiguous range of the half spectrum.
//
// Inverse:
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

template <int N, int TH = 256> struct XReg {
  static constexpr int P = RegPlan<N>::P;
  static constexpr int THREADS = TH;
  static constexpr int LINES = THREADS / P;  // packed lines (row pairs) per block
  static constexpr int RY = 2 * LINES;       // rows per block
  static constexpr int OSTR = N + 4;         // shared row stride of the real output (floats)
  static constexpr int LS = RegLine<float, N>::LS;
};

template <int N, int TH = 256> size_t xreg_smem(int hs) {
  typedef XReg<N, TH> XC;
  const size_t rows = std::max(sizeof(float2) * (size_t)XC::RY * hs, sizeof(float) * (size_t)XC::RY * XC::OSTR);
  const size_t rows16 = (rows + 15) & ~(size_t)15;
  return rows16 + sizeof(float2) * ((size_t)XC::LINES * XC::LS + N);
}

// The work on one block of RY rows whose spectrum rows are being copied into
// HS (bulk copy completing on `bar`, phase `parity`): gather, register inverse
// FFT, epilogue, reduction.  False (uniform) if the copy did not land in time.
// MODE 0: out = P (M xin + g).  MODE 1 (CG): q = P (M p + g), (p, q) -> alpha.
// MODE 2 (residual): out = P (load - M xin - g), (r, r) -> st[s].aux[0].
template <int MODE, int N, int TH = 256>
__device__ __forceinline__ bool xinv_rows(const OpArgs<float>& a, const float* __restrict__ xin,
                                          float* __restrict__ out, SolverState* __restrict__ st,
                                          double* __restrict__ partials, int bps, long long rb, float2* HS,
                                          float2* ex, const float2* tw, const float* mloc,
                                          const unsigned char* aloc, uint64_t* bar, uint32_t parity) {
  typedef RegLine<float, N> RL;
  typedef XReg<N, TH> XC;
  constexpr int P = XC::P, R1 = RL::R1, Q = RL::Q, RY = XC::RY, OSTR = XC::OSTR;
  float* OS = reinterpret_cast<float*>(HS);  // the real rows replace the spectrum rows
  const int s = (int)(rb / bps);
  const int blk = (int)(rb - (long long)s * bps);
  const int rloc = blk * RY;                            // first row inside the system
  const long long row0 = (long long)s * a.rps + rloc;  // global row
  const int hs = a.hs;
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
  if (__syncthreads_or(!mbar_wait(bar, parity))) return false;
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
      if (a.scale) {
        const float f = a.scale[pbase + vox + u];
        m = a.frac ? f * mloc[a.c + comp] + (1.f - f) * mloc[comp]  // Eq. (def_ah)
                   : 1.f / (f * m - a.ref[comp]);
      }
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
  return true;
}

// One block per RY rows (standalone body; the persistent kernel below runs the
// same arithmetic through xinv_rows).
// MODE 0: out = P (M xin + g).  MODE 1 (CG): q = P (M p + g), (p, q) -> alpha.
// MODE 2 (residual): out = P (load - M xin - g), (r, r) -> st[s].aux[0].
template <int MODE, int N, int TH = 256>
__global__ void __launch_bounds__(TH, TH == 256 ? 2 : 4) k_xinv_reg(OpArgs<float> a, const float* __restrict__ xin,
                                                                   float* __restrict__ out,
                                                                   SolverState* __restrict__ st,
                                                                   double* __restrict__ partials, int bps,
                                                                   size_t rows_bytes) {
  typedef RegLine<float, N> RL;
  typedef XReg<N, TH> XC;
  constexpr int P = XC::P, R1 = RL::R1, Q = RL::Q, RY = XC::RY, OSTR = XC::OSTR;
  const int s = blockIdx.x / bps;
  if ((MODE == 1 || MODE == 4) && st[s].done) return;
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
  for (int u = threadIdx.x; u < ntab; u += blockDim.x) mloc[u] = (a.scale && !a.frac) ? a.modtab[u] : a.mtab[u];
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
      if (a.scale) {
        const float f = a.scale[pbase + vox + u];
        m = a.frac ? f * mloc[a.c + comp] + (1.f - f) * mloc[comp]  // Eq. (def_ah)
                   : 1.f / (f * m - a.ref[comp]);
      }
      if (MODE == 0) {
        ov[u] = active ? m * xq[u] + gv[u] : 0.f;
      } else if (MODE == 1 || MODE == 4) {
        ov[u] = active ? m * xq[u] + gv[u] : 0.f;
        acc.add(xq[u] * ov[u]);
      } else {
        ov[u] = active ? a.loads[s * 6 + comp] - (m * xq[u] + gv[u]) : 0.f;
        acc.add(ov[u] * ov[u]);
      }
    }
    *reinterpret_cast<float4*>(out + g) = make_float4(ov[0], ov[1], ov[2], ov[3]);
  }
  if (MODE == 4) {
    // (p, Kp) partial of this block only; k_dot_finalize sums them (no fence, no ticket)
    const double tot = block_reduce(acc);
    if (threadIdx.x == 0) partials[(long long)s * bps + blk] = tot;
  } else if (MODE != 0) {
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

// Persistent: a block walks every gridDim.x-th row block and prefetches the
// next one's spectrum rows into its second buffer while it works on the
// current one.
template <int MODE, int N>
__global__ void __launch_bounds__(256, 2) k_xinv_regp(OpArgs<float> a, const float* __restrict__ xin,
                                                      float* __restrict__ out, SolverState* __restrict__ st,
                                                      double* __restrict__ partials, int bps, size_t rows_bytes,
                                                      long long nrb) {
  typedef XReg<N> XC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  float2* HSb[2] = {reinterpret_cast<float2*>(smem_raw), reinterpret_cast<float2*>(smem_raw + rows_bytes)};
  float2* ex = reinterpret_cast<float2*>(smem_raw + 2 * rows_bytes);
  float2* tw = ex + XC::LINES * XC::LS;
  float* mloc = reinterpret_cast<float*>(tw + N);
  const int ntab = a.nphase * a.c;
  unsigned char* aloc = reinterpret_cast<unsigned char*>(mloc + ntab);
  for (int u = threadIdx.x; u < N; u += blockDim.x) tw[u] = a.twx[u];
  for (int u = threadIdx.x; u < ntab; u += blockDim.x) mloc[u] = (a.scale && !a.frac) ? a.modtab[u] : a.mtab[u];
  for (int u = threadIdx.x; u < a.nphase; u += blockDim.x) aloc[u] = a.act[u];
  const uint32_t bytes = (uint32_t)(sizeof(float2) * (size_t)XC::RY * a.hs);
  auto live = [&](long long rb) { return rb < nrb && (MODE != 1 || st[rb / bps].done == 0); };
  auto issue = [&](long long rb, int b) {  // one thread
    const int s = (int)(rb / bps);
    const long long row0 = (long long)s * a.rps + (rb - (long long)s * bps) * XC::RY;
    mbar_expect_tx(&bar[b], bytes);
    bulk_load_1d(HSb[b], a.H + row0 * a.hs, bytes, &bar[b]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  uint32_t par[2] = {0, 0};
  long long rb = blockIdx.x;
  bool cur = live(rb);
  if (cur && threadIdx.x == 0) issue(rb, 0);
  int b = 0;
  bool fault = false;
  while (rb < nrb) {
    const long long nxt = rb + gridDim.x;
    const bool nl = live(nxt);
    if (nl && threadIdx.x == 0) issue(nxt, b ^ 1);  // that buffer was released at the end of the last round
    if (cur) {
      if (!xinv_rows<MODE, N>(a, xin, out, st, partials, bps, rb, HSb[b], ex, tw, mloc, aloc, &bar[b], par[b])) {
        fault = true;
        break;
      }
      par[b] ^= 1;
      fence_proxy_async();  // our reads of this buffer come before the next copy into it
      __syncthreads();
    }
    rb = nxt;
    cur = nl;
    b ^= 1;
  }
  if (fault && threadIdx.x == 0) {
    mbar_wait(&bar[0], par[0]);
    mbar_wait(&bar[1], par[1]);
    atomicOr(a.fault, 1);
  }
}

template <int N> size_t xfwd_region(int hs) {
  typedef XReg<N> XC;
  const size_t a = std::max(sizeof(float) * (size_t)XC::RY * N, sizeof(float2) * (size_t)XC::RY * hs);
  return (a + 15) & ~(size_t)15;
}
template <int N> size_t xfwd_smem(int hs) {
  typedef XReg<N> XC;
  const size_t ex = std::max(sizeof(float2) * (size_t)XC::LINES * XC::LS, sizeof(float) * (size_t)XC::RY * XC::OSTR);
  return 2 * xfwd_region<N>(hs) + ((ex + 15) & ~(size_t)15) + sizeof(float2) * N;
}

// MODE 0: spectrum of P in (apply).  MODE 1 (CG): x += alpha p_old, p = r + beta
// p_old (p = r at the first iteration), spectrum of p.
template <int MODE, int N>
__global__ void __launch_bounds__(256, 2) k_xfwd_reg(OpArgs<float> a, const float* __restrict__ in,
                                                     float* __restrict__ x, const float* __restrict__ r,
                                                     float* __restrict__ p, const SolverState* __restrict__ st,
                                                     int bps, size_t region) {
  typedef RegLine<float, N> RL;
  typedef XReg<N> XC;
  constexpr int P = XC::P, R1 = RL::R1, RY = XC::RY, OSTR = XC::OSTR, LINES = XC::LINES;
  const int s = blockIdx.x / bps;
  if (MODE == 1 && st[s].done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned char aloc[256];
  __shared__ __align__(8) uint64_t bar;
  unsigned char* R0 = smem_raw;           // p (or in) rows; later the packed spectra Zs
  unsigned char* R1b = smem_raw + region;  // r rows (or phase bytes); later the half-spectrum rows
  float* PN = reinterpret_cast<float*>(smem_raw + 2 * region);  // padded FFT input rows; later the exchange
  float2* ex = reinterpret_cast<float2*>(PN);
  constexpr size_t exa = sizeof(float2) * (size_t)LINES * XC::LS, exr = sizeof(float) * (size_t)RY * OSTR;
  constexpr size_t exb = exa > exr ? exa : exr;
  float2* tw = reinterpret_cast<float2*>(smem_raw + 2 * region + ((exb + 15) & ~(size_t)15));
  for (int u = threadIdx.x; u < N; u += blockDim.x) tw[u] = a.twx[u];
  if (MODE == 0)
    for (int u = threadIdx.x; u < a.nphase; u += blockDim.x) aloc[u] = a.act[u];
  const int blk = blockIdx.x - s * bps;
  const int rloc = blk * RY;
  const long long row0 = (long long)s * a.rps + rloc;
  const int hs = a.hs;
  const int rows_per_comp = a.nz * a.ny;
  const int comp = rloc / rows_per_comp;  // the block's rows lie in one component plane
  const long long pbase = (long long)((a.sys0 + s) / a.sys_per_ms) * a.V;
  const long long vox0 = (long long)(rloc - comp * rows_per_comp) * N;
  int k = 0;
  float alpha = 0.f, beta = 0.f;
  if (MODE == 1) {
    k = st[s].iter;
    alpha = (float)st[s].alpha;
    beta = (float)st[s].beta;
  }
  const uint32_t rows_bytes = (uint32_t)(sizeof(float) * RY * N);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
    if (MODE == 0) {
      mbar_expect_tx(&bar, rows_bytes + (uint32_t)(RY * N));
      bulk_load_1d(R0, in + row0 * N, rows_bytes, &bar);
      bulk_load_1d(R1b, a.phase + pbase + vox0, (uint32_t)(RY * N), &bar);
    } else if (k == 0) {
      mbar_expect_tx(&bar, rows_bytes);
      bulk_load_1d(R1b, r + row0 * N, rows_bytes, &bar);
    } else {
      mbar_expect_tx(&bar, 2 * rows_bytes);
      bulk_load_1d(R0, p + row0 * N, rows_bytes, &bar);
      bulk_load_1d(R1b, r + row0 * N, rows_bytes, &bar);
    }
  }
  constexpr int NV = N / 4;
  constexpr int IT = RY * NV / XC::THREADS;
  static_assert(RY * NV % XC::THREADS == 0, "prologue tiling");
  float4 x4s[IT];
  if (MODE == 1 && k > 0) {
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int idx = threadIdx.x + it * XC::THREADS;
      const int row = idx / NV, xx = (idx - row * NV) * 4;
      x4s[it] = *reinterpret_cast<const float4*>(x + (row0 + row) * N + xx);
    }
  }
  __syncthreads();
  if (__syncthreads_or(!mbar_wait(&bar, 0))) {
    if (threadIdx.x == 0) {
      mbar_wait(&bar, 0);
      atomicOr(a.fault, 1);
    }
    return;
  }
  // prologue: the FFT input rows into PN (padded rows)
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int idx = threadIdx.x + it * XC::THREADS;
    const int row = idx / NV, xx = (idx - row * NV) * 4;
    float4 v;
    if (MODE == 0) {
      v = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(R0) + row * N + xx);
      const uchar4 ph = *reinterpret_cast<const uchar4*>(R1b + row * N + xx);
      if (!aloc[ph.x]) v.x = 0.f;
      if (!aloc[ph.y]) v.y = 0.f;
      if (!aloc[ph.z]) v.z = 0.f;
      if (!aloc[ph.w]) v.w = 0.f;
    } else {
      const float4 r4 = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(R1b) + row * N + xx);
      const long long g = (row0 + row) * N + xx;
      if (k == 0) {
        v = r4;
      } else {
        const float4 p4 = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(R0) + row * N + xx);
        float4 x4 = x4s[it];
        x4.x += alpha * p4.x;
        x4.y += alpha * p4.y;
        x4.z += alpha * p4.z;
        x4.w += alpha * p4.w;
        *reinterpret_cast<float4*>(x + g) = x4;
        v = make_float4(r4.x + beta * p4.x, r4.y + beta * p4.y, r4.z + beta * p4.z, r4.w + beta * p4.w);
      }
      *reinterpret_cast<float4*>(p + g) = v;
    }
    *reinterpret_cast<float4*>(PN + row * OSTR + xx) = v;
  }
  __syncthreads();
  const int t = threadIdx.x % P, l = threadIdx.x / P;
  float2 v[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j)
    v[j] = make_float2(PN[(2 * l) * OSTR + t + P * j], PN[(2 * l + 1) * OSTR + t + P * j]);
  __syncthreads();  // PN becomes the exchange area
  float2* exl = ex + l * XC::LS;
  RL::fwd_a(v, t, tw, exl);
  __syncthreads();
  RL::fwd_b(v, t, tw, exl);
  // packed spectra of the lines, natural order, padded rows
  constexpr int ZS = N + 4;
  float2* Zs = reinterpret_cast<float2*>(R0);
#pragma unroll
  for (int m = 0; m < R1; ++m) Zs[l * ZS + RL::freq(t, m)] = v[m];
  __syncthreads();
  // split Z = X_a + i X_b into the two Hermitian half rows (zero padding columns)
  float2* HSo = reinterpret_cast<float2*>(R1b);
  const int nxh = a.nxh;
  for (int item = threadIdx.x; item < LINES * hs; item += XC::THREADS) {
    const int ln = item / hs, kx = item - ln * hs;
    float2 xa = make_float2(0.f, 0.f), xb = xa;
    if (kx < nxh) {
      const float2 z1 = Zs[ln * ZS + kx];
      const float2 z2 = Zs[ln * ZS + (kx == 0 ? 0 : N - kx)];
      xa = make_float2(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y));
      xb = make_float2(0.5f * (z1.y + z2.y), 0.5f * (z2.x - z1.x));
    }
    HSo[(2 * ln) * hs + kx] = xa;
    HSo[(2 * ln + 1) * hs + kx] = xb;
  }
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    bulk_store_1d(a.H + row0 * hs, HSo, (uint32_t)(sizeof(float2) * (size_t)RY * hs));
    bulk_commit();
    bulk_wait_all();
  }
}

namespace {

template <int N> bool launch_xfwd_reg_n(const OpArgs<float>& a, int mode, const float* in, float* xx, const float* r,
                                        float* p, const SolverState* st, cudaStream_t s) {
  typedef XReg<N> XC;
  if (a.rps % XC::RY != 0 || (a.nz * a.ny) % XC::RY != 0 || (a.hs & 1)) return false;
  if (mode == 0 && ((uintptr_t)in & 15) != 0) return false;  // bulk copies need 16-byte addresses
  const int bps = a.rps / XC::RY;
  const size_t smem = xfwd_smem<N>(a.hs);
  if (smem > 200 * 1024) return false;
  const int grid = a.S * bps;
  const size_t region = xfwd_region<N>(a.hs);
  if (mode == 0) k_xfwd_reg<0, N><<<grid, XC::THREADS, smem, s>>>(a, in, xx, r, p, st, bps, region);
  else k_xfwd_reg<1, N><<<grid, XC::THREADS, smem, s>>>(a, in, xx, r, p, st, bps, region);
  return true;
}

template <int N, int TH = 256> bool launch_xinv_reg_n(const OpArgs<float>& a, int mode, const float* xin, float* out,
                                                      SolverState* st, double* partials, cudaStream_t s) {
  typedef XReg<N, TH> XC;
  if (a.rps % XC::RY != 0 || (a.hs & 1)) return false;
  const int bps = a.rps / XC::RY;
  const size_t rows = std::max(sizeof(float2) * (size_t)XC::RY * a.hs, sizeof(float) * (size_t)XC::RY * XC::OSTR);
  const size_t rows16 = (rows + 15) & ~(size_t)15;
  const size_t smem = xreg_smem<N, TH>(a.hs);
  if (smem > 200 * 1024) return false;
  const int grid = a.S * bps;
  if (mode == 0) k_xinv_reg<0, N, TH><<<grid, XC::THREADS, smem, s>>>(a, xin, out, st, partials, bps, rows16);
  else if (mode == 1) {
    // CG: partials per block, then one small kernel per system turns them into alpha
    k_xinv_reg<4, N, TH><<<grid, XC::THREADS, smem, s>>>(a, xin, out, st, partials, bps, rows16);
    launch_dot_finalize(st, partials, bps, a.S, s);
  } else k_xinv_reg<2, N, TH><<<grid, XC::THREADS, smem, s>>>(a, xin, out, st, partials, bps, rows16);
  return true;
}

template <int N> size_t xregp_smem(const OpArgs<float>& a, size_t* rows16) {
  typedef XReg<N> XC;
  const size_t rows = std::max(sizeof(float2) * (size_t)XC::RY * a.hs, sizeof(float) * (size_t)XC::RY * XC::OSTR);
  *rows16 = (rows + 15) & ~(size_t)15;
  return 2 * *rows16 + sizeof(float2) * ((size_t)XC::LINES * XC::LS + N) + sizeof(float) * a.nphase * a.c + a.nphase;
}

template <int N> int xregp_blocks_per_sm(size_t smem) {
  int v = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_xinv_regp<1, N>, 256, smem) != cudaSuccess) {
    cudaGetLastError();
    v = 0;
  }
  return v;
}

template <int N> bool launch_xinv_regp_n(const OpArgs<float>& a, int mode, const float* xin, float* out,
                                         SolverState* st, double* partials, cudaStream_t s) {
  typedef XReg<N> XC;
  if (a.rps % XC::RY != 0 || (a.hs & 1)) return false;
  const int bps = a.rps / XC::RY;
  size_t rows16 = 0;
  const size_t smem = xregp_smem<N>(a, &rows16);
  if (smem > 200 * 1024) return false;
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  const int bpsm = std::max(1, xregp_blocks_per_sm<N>(smem));
  const long long nrb = (long long)a.S * bps;
  const int grid = (int)std::min<long long>(nrb, (long long)nsm * bpsm);
  if (mode == 0) k_xinv_regp<0, N><<<grid, XC::THREADS, smem, s>>>(a, xin, out, st, partials, bps, rows16, nrb);
  else if (mode == 1) k_xinv_regp<1, N><<<grid, XC::THREADS, smem, s>>>(a, xin, out, st, partials, bps, rows16, nrb);
  else k_xinv_regp<2, N><<<grid, XC::THREADS, smem, s>>>(a, xin, out, st, partials, bps, rows16, nrb);
  return true;
}

template <int N> void xreg_attrs() {
  const int mx = 200 * 1024;
  cudaFuncSetAttribute(k_xinv_reg<4, N, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_reg<4, N, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_reg<0, N, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_reg<1, N, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_reg<2, N, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_regp<0, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_regp<1, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_regp<2, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xfwd_reg<0, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xfwd_reg<1, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_reg<0, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_reg<1, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xinv_reg<2, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

}  // namespace

bool launch_xfwd_reg(const OpArgs<float>& a, int mode, const float* in, float* x, const float* r, float* p,
                     const SolverState* st, cudaStream_t s) {
  switch (a.nx) {
    case 16: return launch_xfwd_reg_n<16>(a, mode, in, x, r, p, st, s);
    case 32: return launch_xfwd_reg_n<32>(a, mode, in, x, r, p, st, s);
    case 64: return launch_xfwd_reg_n<64>(a, mode, in, x, r, p, st, s);
    case 128: return launch_xfwd_reg_n<128>(a, mode, in, x, r, p, st, s);
    case 256: return launch_xfwd_reg_n<256>(a, mode, in, x, r, p, st, s);
    default: return false;
  }
}

bool xfwd_reg_fits(const OpArgs<float>& a) {
  switch (a.nx) {
    case 16: return a.rps % XReg<16>::RY == 0 && (a.nz * a.ny) % XReg<16>::RY == 0 && xfwd_smem<16>(a.hs) <= 200 * 1024;
    case 32: return a.rps % XReg<32>::RY == 0 && (a.nz * a.ny) % XReg<32>::RY == 0 && xfwd_smem<32>(a.hs) <= 200 * 1024;
    case 64: return a.rps % XReg<64>::RY == 0 && (a.nz * a.ny) % XReg<64>::RY == 0 && xfwd_smem<64>(a.hs) <= 200 * 1024;
    case 128:
      return a.rps % XReg<128>::RY == 0 && (a.nz * a.ny) % XReg<128>::RY == 0 && xfwd_smem<128>(a.hs) <= 200 * 1024;
    case 256:
      return a.rps % XReg<256>::RY == 0 && (a.nz * a.ny) % XReg<256>::RY == 0 && xfwd_smem<256>(a.hs) <= 200 * 1024;
    default: return false;
  }
}

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
// shared-memory kernel).  persistent: the double-buffered persistent kernel.
bool launch_xinv_reg(const OpArgs<float>& a, int mode, const float* xin, float* out, SolverState* st,
                     double* partials, cudaStream_t s, bool persistent, bool small) {
  if (small) {
    switch (a.nx) {
      case 16: return launch_xinv_reg_n<16, 128>(a, mode, xin, out, st, partials, s);
      case 32: return launch_xinv_reg_n<32, 128>(a, mode, xin, out, st, partials, s);
      case 64: return launch_xinv_reg_n<64, 128>(a, mode, xin, out, st, partials, s);
      case 128: return launch_xinv_reg_n<128, 128>(a, mode, xin, out, st, partials, s);
      case 256: return launch_xinv_reg_n<256, 128>(a, mode, xin, out, st, partials, s);
      default: return false;
    }
  }
  if (persistent) {
    switch (a.nx) {
      case 16: return launch_xinv_regp_n<16>(a, mode, xin, out, st, partials, s);
      case 32: return launch_xinv_regp_n<32>(a, mode, xin, out, st, partials, s);
      case 64: return launch_xinv_regp_n<64>(a, mode, xin, out, st, partials, s);
      case 128: return launch_xinv_regp_n<128>(a, mode, xin, out, st, partials, s);
      case 256: return launch_xinv_regp_n<256>(a, mode, xin, out, st, partials, s);
      default: return false;
    }
  }
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
