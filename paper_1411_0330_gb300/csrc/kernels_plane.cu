// kernels_plane.cu -- the x and y transforms of one z plane in one kernel
// (FP32, square planes nx = ny = N with N in {16, 32, 48, 64, 96, 128}).
//
// The operator of Eq. (13) transforms along x, y and z around the per-
// frequency Gamma^h product.  A z plane of one component (N^2 reals, at most
// 68 KB as a half spectrum) fits in shared memory, so both in-plane axes are
// done by one block and the spectrum makes one HBM round trip less per axis
// than with separate x and y passes.
//
// Forward (k_xyfwd): the CG prologue (x += alpha p_old, p = r + beta p_old) or
// the projection on I0 runs on coalesced 16-byte global accesses and leaves
// the real plane in shared memory.  Rows 2l and 2l+1 form one complex line,
// transformed along x by the two-level register FFT with the exchange inside
// the pair's own storage, and split into two Hermitian half rows
// X(kx) = (Z(kx) + conj Z(N-kx)) / 2, (Z(kx) - conj Z(N-kx)) / 2i.  Then the
// columns are transformed along y; columns 0 and N/2 hold real sequences and
// travel as one complex column X0 + i XN, separated afterwards.  The plane
// leaves as N rows of the half spectrum, one bulk copy per row, in the
// ky-major layout H[S][c][ky][z][hs]: the z pass then reads each (system,
// component, ky) slab [z][kx] as one contiguous range.  The Nyquist column
// kx = N/2 also goes to a compact array NQ[S][c][z][ky], so the z pass reads
// that column as 8 consecutive ky per z instead of one complex per row.
//
// Inverse (k_xyinv): the rows come back by bulk copies (bounded wait), the
// Nyquist column from NQ, the y and x inverse transforms run the same steps
// backwards (unnormalised: the Gamma table carries 1/V), and the epilogue
// adds the local term M_beta x_beta of Eq. (7), projects on I0 (zero where
// A_beta = A0, Eq. (4)) and, in a CG iteration, reduces this block's part of
// (p, K p) in FP64; k_dot_finalize sums the blocks of a system into alpha.
#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"
#include "regfft.cuh"
#include "tma.cuh"

namespace lsh {

template <int N> struct PlaneCfg {
  typedef RegLine<float, N> RL;
  static constexpr int P = RL::P, R1 = RL::R1, Q = RL::Q;
  // row stride of the plane in shared memory (complex values, even: 16-byte
  // rows for the bulk copies), at least N/2 + 1.  A warp of the x phases holds
  // 32 / P row pairs; their bases, 2 RS apart, must fall on distinct banks for
  // the accesses along a line (stride 1 in t): RS = 4 (mod 8) for P = 8 (row
  // pairs 8 complex values apart modulo 16), RS = 2 (mod 8) for P = 4 (4 apart).
  // The global rows keep the handle's stride hs >= RS (32-byte rows for the z
  // pass); a bulk copy moves the first RS values of a row.
  static constexpr int RS = P >= 8 ? (N / 2 + 1 + 3) / 8 * 8 + 4 : (N / 2 + 6) / 8 * 8 + 2;
  static constexpr int LINES = N / 2;  // row pairs along x, packed columns along y
  static constexpr int TH = LINES * P < 256 ? LINES * P : 256;
  static constexpr int LPR = TH / P;   // lines per round
  static constexpr int ROUNDS = LINES / LPR;
  static constexpr int NV = N / 4;     // float4 groups per real row
  static constexpr int IT = N * NV / TH;
  static constexpr size_t SMEM = sizeof(float2) * ((size_t)N * RS + N);
  // resident blocks per SM the register budget must allow (three 70 KB planes at 128^2)
  static constexpr int MINB = N == 128 ? 3 : 4;
  static_assert(LINES % LPR == 0 && (N * NV) % TH == 0, "tiling");
  static_assert(N + N / R1 <= 2 * RS, "padded exchange fits in a row pair");
};

// x transform of the row pairs of the plane: real rows in, half rows out.
template <int N> __device__ __forceinline__ void plane_x_fwd(float2* PL, const float2* tw) {
  typedef PlaneCfg<N> PC;
  typedef typename PC::RL RL;
  constexpr int P = PC::P, R1 = PC::R1, RS = PC::RS;
  constexpr int NK = (RS + P - 1) / P;
  const int t = threadIdx.x % P, lr = threadIdx.x / P;
#pragma unroll 1
  for (int rd = 0; rd < PC::ROUNDS; ++rd) {
    float2* pair = PL + 2 * (lr + rd * PC::LPR) * RS;
    const float* ra = reinterpret_cast<const float*>(pair);
    const float* rb = ra + 2 * RS;
    float2 v[R1];
#pragma unroll
    for (int j = 0; j < R1; ++j) v[j] = make_float2(ra[t + P * j], rb[t + P * j]);
    __syncwarp();
    RL::fwd_a_p(v, t, tw, pair);
    __syncwarp();
    RL::fwd_b_p(v, t, tw, pair);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < R1; ++m) pair[RL::freq(t, m)] = v[m];
    __syncwarp();
    // kx = t + P i lies in [P i, P (i + 1)): inside 0..N/2 for every t while
    // P (i + 1) <= N/2, for t = 0 only at i = N / (2P), outside beyond; kx = 0
    // pairs with itself
    float2 xa[NK], xb[NK];
#pragma unroll
    for (int i = 0; i < NK; ++i) {
      const int kx = t + P * i;
      xa[i] = make_float2(0.f, 0.f);
      xb[i] = xa[i];
      const bool in = P * (i + 1) <= N / 2 || (P * i <= N / 2 && kx <= N / 2);
      if (in) {
        const float2 z1 = pair[kx], z2 = pair[(i == 0 && t == 0) ? 0 : N - kx];
        xa[i] = make_float2(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y));
        xb[i] = make_float2(0.5f * (z1.y + z2.y), 0.5f * (z2.x - z1.x));
      }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < NK; ++i) {
      const int kx = t + P * i;
      if (P * (i + 1) <= RS || kx < RS) {
        pair[kx] = xa[i];
        pair[RS + kx] = xb[i];
      }
    }
  }
}

// y transform of the columns 0 .. N/2 (0 and N/2 packed), forward.
template <int N> __device__ __forceinline__ void plane_y_fwd(float2* PL, const float2* tw) {
  typedef PlaneCfg<N> PC;
  typedef typename PC::RL RL;
  constexpr int P = PC::P, R1 = PC::R1, RS = PC::RS, LPR = PC::LPR;
  const int t = threadIdx.x / LPR, cl = threadIdx.x % LPR;
#pragma unroll 1
  for (int rd = 0; rd < PC::ROUNDS; ++rd) {
    const int col = cl + rd * LPR;
    float2* cp = PL + col;
    float2 v[R1];
    if (col == 0) {  // columns 0 and N/2 (real) as one complex column
#pragma unroll
      for (int j = 0; j < R1; ++j) v[j] = make_float2(PL[(t + P * j) * RS].x, PL[(t + P * j) * RS + N / 2].x);
    } else {
#pragma unroll
      for (int j = 0; j < R1; ++j) v[j] = cp[(t + P * j) * RS];
    }
    __syncthreads();
    RL::template fwd_a_s<RS>(v, t, tw, cp);
    __syncthreads();
    RL::template fwd_b_s<RS>(v, t, tw, cp);
    __syncthreads();
#pragma unroll
    for (int m = 0; m < R1; ++m) cp[RL::freq(t, m) * RS] = v[m];
  }
  __syncthreads();
  // W = X0 + i XN with X0, XN Hermitian in ky: X0 = (W(k) + conj W(-k)) / 2,
  // XN = (W(k) - conj W(-k)) / 2i; the thread of ky also writes N - ky
  for (int ky = threadIdx.x; ky <= N / 2; ky += PC::TH) {
    const int km = ky == 0 ? 0 : N - ky;
    const float2 w1 = PL[ky * RS], w2 = PL[km * RS];
    const float2 x0 = make_float2(0.5f * (w1.x + w2.x), 0.5f * (w1.y - w2.y));
    const float2 xn = make_float2(0.5f * (w1.y + w2.y), 0.5f * (w2.x - w1.x));
    PL[ky * RS] = x0;
    PL[ky * RS + N / 2] = xn;
    if (km != ky) {
      PL[km * RS] = make_float2(x0.x, -x0.y);
      PL[km * RS + N / 2] = make_float2(xn.x, -xn.y);
    }
  }
  __syncthreads();
}

// y inverse transform of the columns (0 and N/2 packed), unnormalised.
template <int N> __device__ __forceinline__ void plane_y_inv(float2* PL, const float2* tw) {
  typedef PlaneCfg<N> PC;
  typedef typename PC::RL RL;
  constexpr int P = PC::P, R1 = PC::R1, RS = PC::RS, LPR = PC::LPR;
  const int t = threadIdx.x / LPR, cl = threadIdx.x % LPR;
#pragma unroll 1
  for (int rd = 0; rd < PC::ROUNDS; ++rd) {
    const int col = cl + rd * LPR;
    float2* cp = PL + col;
    float2 v[R1];
    if (col == 0) {
#pragma unroll
      for (int m = 0; m < R1; ++m) {
        const int f = RL::freq(t, m);
        const float2 x0 = PL[f * RS], xn = PL[f * RS + N / 2];
        v[m] = make_float2(x0.x - xn.y, x0.y + xn.x);  // X0 + i XN
      }
    } else {
#pragma unroll
      for (int m = 0; m < R1; ++m) v[m] = cp[RL::freq(t, m) * RS];
    }
    __syncthreads();
    RL::template inv_a_s<RS>(v, t, tw, cp);
    __syncthreads();
    RL::template inv_b_s<RS>(v, t, tw, cp);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < R1; ++j) {
      const int y = t + P * j;
      if (col == 0) {
        // the inverse of X0 + i XN is x0 + i xN with x0, xN real
        PL[y * RS] = make_float2(v[j].x, 0.f);
        PL[y * RS + N / 2] = make_float2(v[j].y, 0.f);
      } else {
        cp[y * RS] = v[j];
      }
    }
  }
  __syncthreads();
}

// x inverse transform of the row pairs: half rows in, N x real rows out.
template <int N> __device__ __forceinline__ void plane_x_inv(float2* PL, const float2* tw) {
  typedef PlaneCfg<N> PC;
  typedef typename PC::RL RL;
  constexpr int P = PC::P, R1 = PC::R1, Q = PC::Q, RS = PC::RS;
  const int t = threadIdx.x % P, lr = threadIdx.x / P;
#pragma unroll 1
  for (int rd = 0; rd < PC::ROUNDS; ++rd) {
    float2* pair = PL + 2 * (lr + rd * PC::LPR) * RS;
    float2 v[R1];
    // frequency f = t Q + q + R1 u lies in [R1 u, R1 (u + 1)): below N/2 for u < P/2,
    // read at N - f from u = P/2 on (f = N/2 included: X(N/2) of a row is real)
    const float2* up = pair + t * Q;      // X(f) at up[q + R1 u]
    const float2* dn = pair + N - t * Q;  // X(N - f) at dn[-(q + R1 u)]
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int u = 0; u < P; ++u) {
        const int c = q + R1 * u;
        // Z(f) = X_a(f) + i X_b(f), X(N - k) = conj X(k)
        if (u < P / 2) {
          const float2 xa = up[c], xb = up[RS + c];
          v[q * P + u] = make_float2(xa.x - xb.y, xa.y + xb.x);
        } else {
          const float2 xa = dn[-c], xb = dn[RS - c];
          v[q * P + u] = make_float2(xa.x + xb.y, xb.x - xa.y);
        }
      }
    __syncwarp();
    RL::inv_a_p(v, t, tw, pair);
    __syncwarp();
    RL::inv_b_p(v, t, tw, pair);
    __syncwarp();
    float* ra = reinterpret_cast<float*>(pair);
    float* rb = ra + 2 * RS;
#pragma unroll
    for (int j = 0; j < R1; ++j) {
      ra[t + P * j] = v[j].x;
      rb[t + P * j] = v[j].y;
    }
  }
}

// MODE 0: spectrum of P in (apply).  MODE 1 (CG): x += alpha p_old, p = r +
// beta p_old (p = r at the first iteration), spectrum of p.
template <int N, int MODE>
__global__ void __launch_bounds__(PlaneCfg<N>::TH, PlaneCfg<N>::MINB) k_xyfwd(OpArgs<float> a, const float* __restrict__ in,
                                                           float* __restrict__ x, const float* __restrict__ r,
                                                           float* __restrict__ p, const SolverState* __restrict__ st) {
  typedef PlaneCfg<N> PC;
  constexpr int RS = PC::RS, TH = PC::TH, NV = PC::NV;
  const int cnz = a.c * a.nz;
  const int s = blockIdx.x / cnz;
  const int blk = blockIdx.x - s * cnz;  // comp * nz + z
  const int comp = blk / a.nz, z = blk - comp * a.nz;
  if (MODE == 1 && st[s].done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* PL = reinterpret_cast<float2*>(smem_raw);  // [N][RS]
  float2* tw = PL + N * RS;
  float* PR = reinterpret_cast<float*>(PL);  // real row y at PR + 2 RS y
  __shared__ unsigned char aloc[256];
  for (int u = threadIdx.x; u < N; u += TH) tw[u] = a.twx[u];
  if (MODE == 0)
    for (int u = threadIdx.x; u < a.nphase; u += TH) aloc[u] = a.act[u];
  const long long plane = (long long)blockIdx.x * N * N;  // [S][c][nz] planes of N^2
  const long long pbase = (long long)((a.sys0 + s) / a.sys_per_ms) * a.V + (long long)z * N * N;
  int k = 0;
  float alpha = 0.f, beta = 0.f;
  if (MODE == 1) {
    k = st[s].iter;
    alpha = (float)st[s].alpha;
    beta = (float)st[s].beta;
  }
  if (MODE == 0) {
    __syncthreads();  // aloc
#pragma unroll 4
    for (int it = 0; it < PC::IT; ++it) {
      const int idx = threadIdx.x + it * TH;
      const int row = idx / NV, xx = (idx - row * NV) * 4;
      const long long g = plane + (long long)row * N + xx;
      float4 v = *reinterpret_cast<const float4*>(in + g);
      const uchar4 ph = *reinterpret_cast<const uchar4*>(a.phase + pbase + row * N + xx);
      if (!aloc[ph.x]) v.x = 0.f;
      if (!aloc[ph.y]) v.y = 0.f;
      if (!aloc[ph.z]) v.z = 0.f;
      if (!aloc[ph.w]) v.w = 0.f;
      *reinterpret_cast<float4*>(PR + 2 * RS * row + xx) = v;
    }
  } else {
    // The r plane comes into the real rows of the plane buffer by one bulk copy
    // per row; p and x go through registers in batches of B groups of four
    // reals, each batch's loads in flight while the previous batch is combined.
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      mbar_init_fence();
      mbar_expect_tx(&bar, (uint32_t)(sizeof(float) * N * N));
    }
    __syncthreads();
    for (int row = threadIdx.x; row < N; row += TH)
      bulk_load_1d(PR + 2 * RS * row, r + plane + (long long)row * N, (uint32_t)(sizeof(float) * N), &bar);
    constexpr int B = PC::IT % 4 == 0 ? 4 : (PC::IT % 3 == 0 ? 3 : (PC::IT % 2 == 0 ? 2 : 1));
    static_assert(PC::IT % B == 0, "batches");
    float4 pb[B], xb[B];
    auto load_batch = [&](int it0) {
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int idx = threadIdx.x + (it0 + b) * TH;
        const int row = idx / NV, xx = (idx - row * NV) * 4;
        const long long g = plane + (long long)row * N + xx;
        pb[b] = *reinterpret_cast<const float4*>(p + g);
        xb[b] = *reinterpret_cast<const float4*>(x + g);
      }
    };
    if (k > 0) load_batch(0);
    if (__syncthreads_or(!mbar_wait(&bar, 0))) {
      if (threadIdx.x == 0) {
        mbar_wait(&bar, 0);  // no copy may still be writing this block's shared memory
        atomicOr(a.fault, 1);
      }
      return;
    }
#pragma unroll
    for (int it0 = 0; it0 < PC::IT; it0 += B) {
      float4 pc[B], xc[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        pc[b] = pb[b];
        xc[b] = xb[b];
      }
      if (k > 0 && it0 + B < PC::IT) load_batch(it0 + B);
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int idx = threadIdx.x + (it0 + b) * TH;
        const int row = idx / NV, xx = (idx - row * NV) * 4;
        const long long g = plane + (long long)row * N + xx;
        float4* rs = reinterpret_cast<float4*>(PR + 2 * RS * row + xx);
        const float4 r4 = *rs;
        float4 v = r4;
        if (k > 0) {
          const float4 p4 = pc[b];
          float4 x4 = xc[b];
          x4.x += alpha * p4.x;
          x4.y += alpha * p4.y;
          x4.z += alpha * p4.z;
          x4.w += alpha * p4.w;
          *reinterpret_cast<float4*>(x + g) = x4;
          v = make_float4(r4.x + beta * p4.x, r4.y + beta * p4.y, r4.z + beta * p4.z, r4.w + beta * p4.w);
          *rs = v;
        }
        *reinterpret_cast<float4*>(p + g) = v;
      }
    }
  }
  __syncthreads();
  plane_x_fwd<N>(PL, tw);
  __syncthreads();
  plane_y_fwd<N>(PL, tw);
  // N rows of the half spectrum to H[s][comp][ky][z][:]; the Nyquist column to NQ
  fence_proxy_async();
  __syncthreads();
  const long long slab = (long long)(s * a.c + comp) * N;
  for (int ky = threadIdx.x; ky < N; ky += TH) {
    bulk_store_1d(a.H + ((slab + ky) * a.nz + z) * a.hs, PL + ky * RS, (uint32_t)(sizeof(float2) * RS));
    a.nq[(long long)blockIdx.x * N + ky] = PL[ky * RS + N / 2];
  }
  bulk_commit();
  bulk_wait_read_all();
}

// MODE 0: out = P (M xin + g).  MODE 4 (CG): q = P (M p + g) and this block's
// part of (p, q) in partials[s * c nz + block of the system].
template <int N, int MODE>
__global__ void __launch_bounds__(PlaneCfg<N>::TH, PlaneCfg<N>::MINB) k_xyinv(OpArgs<float> a, const float* __restrict__ xin,
                                                           float* __restrict__ out, const SolverState* __restrict__ st,
                                                           double* __restrict__ partials) {
  typedef PlaneCfg<N> PC;
  constexpr int RS = PC::RS, TH = PC::TH, NV = PC::NV;
  const int cnz = a.c * a.nz;
  const int s = blockIdx.x / cnz;
  const int blk = blockIdx.x - s * cnz;
  const int comp = blk / a.nz, z = blk - comp * a.nz;
  if (MODE == 4 && st[s].done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* PL = reinterpret_cast<float2*>(smem_raw);
  float2* tw = PL + N * RS;
  float* PR = reinterpret_cast<float*>(PL);
  // per-phase tables after the plane (sized by the launch: nphase * (4 c + 1) bytes)
  float* mloc = reinterpret_cast<float*>(tw + N);
  unsigned char* aloc = reinterpret_cast<unsigned char*>(mloc + a.nphase * a.c);
  __shared__ __align__(8) uint64_t bar;
  const long long slab = (long long)(s * a.c + comp) * N;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
    mbar_expect_tx(&bar, (uint32_t)(sizeof(float2) * N * RS));
  }
  __syncthreads();
  for (int ky = threadIdx.x; ky < N; ky += TH)
    bulk_load_1d(PL + ky * RS, a.H + ((slab + ky) * a.nz + z) * a.hs, (uint32_t)(sizeof(float2) * RS), &bar);
  for (int u = threadIdx.x; u < N; u += TH) tw[u] = a.twx[u];
  const int ntab = a.nphase * a.c;
  for (int u = threadIdx.x; u < ntab; u += TH) mloc[u] = (a.scale && !a.frac) ? a.modtab[u] : a.mtab[u];
  for (int u = threadIdx.x; u < a.nphase; u += TH) aloc[u] = a.act[u];
  // the epilogue's p plane and phase plane go to L2 while the transforms run
  const long long plane = (long long)blockIdx.x * N * N;
  const long long pbase = (long long)((a.sys0 + s) / a.sys_per_ms) * a.V + (long long)z * N * N;
  if ((a.l2pf & 2) && threadIdx.x < 9) {
    constexpr uint32_t PB = (uint32_t)(sizeof(float) * N * N);
    if (threadIdx.x < 8) bulk_prefetch_l2(reinterpret_cast<const char*>(xin + plane) + threadIdx.x * (PB / 8), PB / 8);
    else if ((pbase & 15) == 0) bulk_prefetch_l2(a.phase + pbase, (uint32_t)(N * N));
  }
  float2 nqv = make_float2(0.f, 0.f);
  if (threadIdx.x < N) nqv = a.nq[(long long)blockIdx.x * N + threadIdx.x];
  if (__syncthreads_or(!mbar_wait(&bar, 0))) {
    if (threadIdx.x == 0) {
      mbar_wait(&bar, 0);  // no copy may still be writing this block's shared memory
      atomicOr(a.fault, 1);
    }
    return;
  }
  for (int ky = threadIdx.x; ky < N; ky += TH)
    PL[ky * RS + N / 2] = ky == (int)threadIdx.x ? nqv : a.nq[(long long)blockIdx.x * N + ky];
  __syncthreads();
  plane_y_inv<N>(PL, tw);
  // the epilogue's p and phase loads go out in batches of B groups of four
  // voxels, each batch in flight while the previous one is worked on; two
  // register sets take the batches in turn (no copies between them)
  constexpr int B = PC::IT % 2 == 0 ? 2 : 1;
  float4 xb0[B], xb1[B];
  uchar4 hb0[B], hb1[B];
  auto load_batch = [&](int it0, float4* xb, uchar4* hb) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int idx = threadIdx.x + (it0 + b) * TH;
      const int row = idx / NV, xx = (idx - row * NV) * 4;
      xb[b] = *reinterpret_cast<const float4*>(xin + plane + (long long)row * N + xx);
      hb[b] = *reinterpret_cast<const uchar4*>(a.phase + pbase + (long long)row * N + xx);
    }
  };
  plane_x_inv<N>(PL, tw);
  load_batch(0, xb0, hb0);
  __syncthreads();
  Acc<float> acc;
  // two phases without a voxel field (the common case): both phases' M and
  // activity in registers, selected per voxel instead of read from the tables;
  // both active (A0 differs from both phases): no projection to apply
  const bool two = a.nphase <= 2 && !a.scale;
  const float m0 = mloc[comp], m1 = a.nphase > 1 ? mloc[a.c + comp] : m0;
  const bool act0 = aloc[0] != 0, act1 = a.nphase > 1 ? aloc[1] != 0 : act0;
  const bool both = two && act0 && act1;
  auto work = [&](int it0, const float4* xc, const uchar4* hc) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int idx = threadIdx.x + (it0 + b) * TH;
      const int row = idx / NV, xx = (idx - row * NV) * 4;
      const long long g = plane + (long long)row * N + xx;
      const long long vox = pbase + (long long)row * N + xx;
      const float4 g4 = *reinterpret_cast<const float4*>(PR + 2 * RS * row + xx);
      const float xq[4] = {xc[b].x, xc[b].y, xc[b].z, xc[b].w};
      const unsigned char ph[4] = {hc[b].x, hc[b].y, hc[b].z, hc[b].w};
      const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
      float ov[4];
      if (both) {
#pragma unroll
        for (int u = 0; u < 4; ++u) ov[u] = fmaf(ph[u] != 0 ? m1 : m0, xq[u], gv[u]);
      } else if (two) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool p1 = ph[u] != 0;
          ov[u] = (p1 ? act1 : act0) ? fmaf(p1 ? m1 : m0, xq[u], gv[u]) : 0.f;
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int pp = ph[u];
          const bool active = aloc[pp] != 0;
          float m = mloc[pp * a.c + comp];
          if (a.scale) {
            const float f = a.scale[vox + u];
            m = a.frac ? f * mloc[a.c + comp] + (1.f - f) * mloc[comp]  // Eq. (def_ah)
                       : 1.f / (f * m - a.ref[comp]);
          }
          ov[u] = active ? m * xq[u] + gv[u] : 0.f;
        }
      }
      // (p, K p): the group's four products summed in FP32, then one compensated add
      if (MODE == 4) acc.add(fmaf(xq[3], ov[3], fmaf(xq[2], ov[2], fmaf(xq[1], ov[1], xq[0] * ov[0]))));
      *reinterpret_cast<float4*>(out + g) = make_float4(ov[0], ov[1], ov[2], ov[3]);
    }
  };
#pragma unroll 1
  for (int it0 = 0; it0 < PC::IT; it0 += 2 * B) {
    if (it0 + B < PC::IT) load_batch(it0 + B, xb1, hb1);
    work(it0, xb0, hb0);
    if (it0 + B >= PC::IT) break;
    if (it0 + 2 * B < PC::IT) load_batch(it0 + 2 * B, xb0, hb0);
    work(it0 + B, xb1, hb1);
  }
  if (MODE == 4) {
    const double tot = block_reduce(acc);
    if (threadIdx.x == 0) partials[(long long)s * cnz + blk] = tot;
  }
}

namespace {

// dynamic shared memory of the inverse kernel: the plane, the twiddles and the phase tables
template <int N> size_t plane_inv_smem(const OpArgs<float>& a) {
  return PlaneCfg<N>::SMEM + (((size_t)a.nphase * (4 * a.c + 1) + 15) & ~(size_t)15);
}

template <int N> void plane_attrs() {
  const int sm = (int)PlaneCfg<N>::SMEM;
  const int smi = (int)(PlaneCfg<N>::SMEM + 256 * 25);  // up to 256 phases of 6 components
  cudaFuncSetAttribute(k_xyfwd<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_xyfwd<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_xyinv<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smi);
  cudaFuncSetAttribute(k_xyinv<N, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smi);
}

template <int N> bool plane_fwd_n(const OpArgs<float>& a, int mode, const float* in, float* x, const float* r,
                                  float* p, const SolverState* st, cudaStream_t s) {
  typedef PlaneCfg<N> PC;
  if (a.hs < PC::RS || (a.hs & 1) != 0) return false;
  const unsigned grid = (unsigned)((long long)a.S * a.c * a.nz);
  if (mode == 0) k_xyfwd<N, 0><<<grid, PC::TH, PC::SMEM, s>>>(a, in, x, r, p, st);
  else k_xyfwd<N, 1><<<grid, PC::TH, PC::SMEM, s>>>(a, in, x, r, p, st);
  return true;
}

template <int N> bool plane_inv_n(const OpArgs<float>& a, int mode, const float* xin, float* out, SolverState* st,
                                  double* partials, cudaStream_t s) {
  typedef PlaneCfg<N> PC;
  if (a.hs < PC::RS || (a.hs & 1) != 0) return false;
  const unsigned grid = (unsigned)((long long)a.S * a.c * a.nz);
  const size_t smem = plane_inv_smem<N>(a);
  if (mode == 0) {
    k_xyinv<N, 0><<<grid, PC::TH, smem, s>>>(a, xin, out, st, partials);
  } else {
    k_xyinv<N, 4><<<grid, PC::TH, smem, s>>>(a, xin, out, st, partials);
    launch_dot_finalize(st, partials, a.c * a.nz, a.S, s);
  }
  return true;
}

}  // namespace

bool plane_length(int n) { return n == 16 || n == 32 || n == 48 || n == 64 || n == 96 || n == 128; }

bool launch_xyfwd(const OpArgs<float>& a, int mode, const float* in, float* x, const float* r, float* p,
                  const SolverState* st, cudaStream_t s) {
  if (a.nx != a.ny || mode < 0 || mode > 1) return false;
  switch (a.nx) {
    case 16: return plane_fwd_n<16>(a, mode, in, x, r, p, st, s);
    case 32: return plane_fwd_n<32>(a, mode, in, x, r, p, st, s);
    case 48: return plane_fwd_n<48>(a, mode, in, x, r, p, st, s);
    case 64: return plane_fwd_n<64>(a, mode, in, x, r, p, st, s);
    case 96: return plane_fwd_n<96>(a, mode, in, x, r, p, st, s);
    case 128: return plane_fwd_n<128>(a, mode, in, x, r, p, st, s);
    default: return false;
  }
}

bool launch_xyinv(const OpArgs<float>& a, int mode, const float* xin, float* out, SolverState* st, double* partials,
                  cudaStream_t s) {
  if (a.nx != a.ny || mode < 0 || mode > 1) return false;
  switch (a.nx) {
    case 16: return plane_inv_n<16>(a, mode, xin, out, st, partials, s);
    case 32: return plane_inv_n<32>(a, mode, xin, out, st, partials, s);
    case 48: return plane_inv_n<48>(a, mode, xin, out, st, partials, s);
    case 64: return plane_inv_n<64>(a, mode, xin, out, st, partials, s);
    case 96: return plane_inv_n<96>(a, mode, xin, out, st, partials, s);
    case 128: return plane_inv_n<128>(a, mode, xin, out, st, partials, s);
    default: return false;
  }
}

void plane_prepare() {
  plane_attrs<16>();
  plane_attrs<32>();
  plane_attrs<48>();
  plane_attrs<64>();
  plane_attrs<96>();
  plane_attrs<128>();
}

}  // namespace lsh
