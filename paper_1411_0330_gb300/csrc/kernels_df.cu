// kernels_df.cu -- the operator of Eq. (13) in double-float arithmetic (df.cuh):
// FP64 fields in HBM, every step of the five passes on the FP32 pipes with 48
// significant bits.  It serves the iterative-refinement residual of the mixed
// solver (r = b - K x, which must resolve about 1e-11 of ||b||) and the
// emulated-FP64 apply; on GB300 it runs several times faster than the same
// passes in native FP64, whose pipe issues 1/64 of the FP32 rate.
//
// The y pass is the register-FFT kernel of kernels_reg.cu instantiated for DF.
// The z pass runs as three launches: the z transform, the Gamma^h product
// (one thread per frequency, its coefficients read once for all systems),
// the inverse z transform: one fused kernel holding the double-float 6 x 6
// product and both transforms needed 168 registers and missed the
// instruction cache (1.64 ms against 0.39 + 0.42 + 0.40 ms for the three at
// 128^3 with 6 systems).
// The x passes below read and write FP64: a block owns RY consecutive rows of
// one system, two real rows form one complex line of N points held by P
// threads (two-level register FFT, regfft.cuh).
//   forward (apply):  projection on I0, FFT, split into the two Hermitian half
//                     rows, store of the half spectrum (double-float pairs);
//   inverse:          gather of each line's frequencies (X(N - k) = conj X(k)
//                     beyond the half), inverse FFT, local term M x,
//                     projection, and for the residual (r, r).
#include <algorithm>

#include "common.cuh"
#include "df.cuh"
#include "fft.cuh"
#include "gamma_onfly.cuh"
#include "internal.h"
#include "regfft.cuh"

namespace lsh {

template <int N> struct XDf {
  static constexpr int P = RegPlan<N>::P;
  static constexpr int THREADS = 128;
  static constexpr int LINES = THREADS / P;  // packed lines (row pairs) per block
  static constexpr int RY = 2 * LINES;       // rows per block
  static constexpr int LS = RegLine<DF, N>::LS;
  static constexpr int ZS = N + 1;           // shared row stride of the packed spectra
  static constexpr int EXN = LINES * (LS > ZS ? LS : ZS);
  static constexpr size_t SMEM = sizeof(DF2) * (size_t)(EXN + N);
};

__global__ void k_d2df(const double* __restrict__ in, DF* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = df_from(in[i]);
}

// The half spectrum of P x (apply), x FP64 [S][c][nz][ny][nx].
template <int N>
__global__ void __launch_bounds__(128) k_df_xfwd(OpArgs<double> a, const DF2* __restrict__ twx,
                                                 const double* __restrict__ in, int bps) {
  typedef RegLine<DF, N> RL;
  typedef XDf<N> XC;
  constexpr int P = XC::P, R1 = RL::R1, RY = XC::RY, LINES = XC::LINES, ZS = XC::ZS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DF2* ex = reinterpret_cast<DF2*>(smem_raw);
  DF2* tw = ex + XC::EXN;
  __shared__ unsigned char aloc[256];
  for (int u = threadIdx.x; u < N; u += XC::THREADS) tw[u] = twx[u];
  for (int u = threadIdx.x; u < a.nphase; u += XC::THREADS) aloc[u] = a.act[u];
  const int s = blockIdx.x / bps, blk = blockIdx.x - s * bps;
  const int rloc = blk * RY;
  const long long row0 = (long long)s * a.rps + rloc;
  const int rows_per_comp = a.nz * a.ny;
  const int comp = rloc / rows_per_comp;  // the block's rows lie in one component plane
  const long long pbase = (long long)((a.sys0 + s) / a.sys_per_ms) * a.V;
  const long long vox0 = (long long)(rloc - comp * rows_per_comp) * N;
  __syncthreads();
  // P x into padded shared rows with row-contiguous 16-byte loads (the FP64
  // pipe converts: it has room in this pass)
  constexpr int GS = N + 4, NP = N / 2;
  static_assert(RY * GS <= XC::EXN * 2, "rows fit in the exchange area");
  DF* G = reinterpret_cast<DF*>(ex);
  for (int e = threadIdx.x; e < RY * NP; e += XC::THREADS) {
    const int rowl = e / NP, x = 2 * (e - rowl * NP);
    const double2 xv = *reinterpret_cast<const double2*>(in + (row0 + rowl) * N + x);
    const uchar2 ph = *reinterpret_cast<const uchar2*>(a.phase + pbase + vox0 + (long long)rowl * N + x);
    G[rowl * GS + x] = aloc[ph.x] ? df_from(xv.x) : DF(0.f, 0.f);
    G[rowl * GS + x + 1] = aloc[ph.y] ? df_from(xv.y) : DF(0.f, 0.f);
  }
  __syncthreads();
  const int t = threadIdx.x % P, l = threadIdx.x / P;
  DF2 v[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) {
    v[j].x = G[(2 * l) * GS + t + P * j];
    v[j].y = G[(2 * l + 1) * GS + t + P * j];
  }
  __syncthreads();  // the rows become the exchange area
  DF2* exl = ex + l * XC::LS;
  RL::fwd_a(v, t, tw, exl);
  __syncthreads();
  RL::fwd_b(v, t, tw, exl);
  __syncthreads();  // the exchange area becomes the packed spectra
  DF2* Zs = ex;
#pragma unroll
  for (int m = 0; m < R1; ++m) Zs[l * ZS + RL::freq(t, m)] = v[m];
  __syncthreads();
  // split Z = X_a + i X_b into the two Hermitian half rows (zero padding columns)
  const int hs = a.hs, nxh = a.nxh;
  DF2* H = reinterpret_cast<DF2*>(a.H);
  for (int item = threadIdx.x; item < LINES * hs; item += XC::THREADS) {
    const int ln = item / hs, kx = item - ln * hs;
    DF2 ya, yb;
    ya.x = ya.y = yb.x = yb.y = DF(0.f, 0.f);
    if (kx < nxh) {
      const DF2 z1 = Zs[ln * ZS + kx];
      const DF2 z2 = Zs[ln * ZS + (kx == 0 ? 0 : N - kx)];
      ya.x = df_scale2(z1.x + z2.x, 0.5f);
      ya.y = df_scale2(z1.y - z2.y, 0.5f);
      yb.x = df_scale2(z1.y + z2.y, 0.5f);
      yb.y = df_scale2(z2.x - z1.x, 0.5f);
    }
    H[(row0 + 2 * ln) * hs + kx] = ya;
    H[(row0 + 2 * ln + 1) * hs + kx] = yb;
  }
}

// MODE 0: out = P (M xin + g) (FP64).  MODE 2 (residual): out = P (load - M xin
// - g) as double-float pairs (h, l) in the 8 bytes of each element, (out, out)
// -> st[s].aux[0].  g = the inverse transform of the spectrum.
template <int MODE, int N>
__global__ void __launch_bounds__(128) k_df_xinv(OpArgs<double> a, const DF2* __restrict__ twx,
                                                 const double* __restrict__ xin, double* __restrict__ out,
                                                 SolverState* __restrict__ st, double* __restrict__ partials,
                                                 int bps) {
  typedef RegLine<DF, N> RL;
  typedef XDf<N> XC;
  constexpr int P = XC::P, R1 = RL::R1, Q = RL::Q, RY = XC::RY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DF2* ex = reinterpret_cast<DF2*>(smem_raw);
  DF2* tw = ex + XC::EXN;
  __shared__ DF mloc[256 * 6];
  __shared__ unsigned char aloc[256];
  for (int u = threadIdx.x; u < N; u += XC::THREADS) tw[u] = twx[u];
  const int ntab = a.nphase * a.c;
  for (int u = threadIdx.x; u < ntab; u += XC::THREADS) mloc[u] = df_from(a.mtab[u]);
  for (int u = threadIdx.x; u < a.nphase; u += XC::THREADS) aloc[u] = a.act[u];
  const int s = blockIdx.x / bps, blk = blockIdx.x - s * bps;
  const int rloc = blk * RY;
  const long long row0 = (long long)s * a.rps + rloc;
  const int rows_per_comp = a.nz * a.ny;
  const int comp = rloc / rows_per_comp;
  const long long pbase = (long long)((a.sys0 + s) / a.sys_per_ms) * a.V;
  const long long vox0 = (long long)(rloc - comp * rows_per_comp) * N;
  const int t = threadIdx.x % P, l = threadIdx.x / P;
  const int hs = a.hs;
  const DF2* Ha = reinterpret_cast<const DF2*>(a.H) + (row0 + 2 * l) * hs;
  const DF2* Hb = Ha + hs;
  DF2 v[R1];
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const int f = t * Q + q + R1 * u;
      const bool lo = f <= N / 2;
      const int k = lo ? f : N - f;
      const DF2 ya = Ha[k], yb = Hb[k];
      // Z(f) = X_a(f) + i X_b(f), X(N - k) = conj X(k)
      DF2 z;
      if (lo) {
        z.x = ya.x - yb.y;
        z.y = ya.y + yb.x;
      } else {
        z.x = ya.x + yb.y;
        z.y = yb.x - ya.y;
      }
      v[q * P + u] = z;
    }
  __syncthreads();  // tw, mloc, aloc in place
  DF2* exl = ex + l * XC::LS;
  RL::inv_a(v, t, tw, exl);
  __syncthreads();
  RL::inv_b(v, t, tw, exl);
  // v[j] = (g of row 2l, g of row 2l + 1) at x = t + P j; through shared memory
  // (rows padded by 4 values: conflict-free) to an epilogue whose global
  // accesses run along the rows
  constexpr int GS = N + 4;
  static_assert(RY * GS <= XC::EXN * 2, "g rows fit in the exchange area");
  DF* G = reinterpret_cast<DF*>(ex);
  __syncthreads();  // every thread has read the exchange area
#pragma unroll
  for (int j = 0; j < R1; ++j) {
    G[(2 * l) * GS + t + P * j] = v[j].x;
    G[(2 * l + 1) * GS + t + P * j] = v[j].y;
  }
  __syncthreads();
  const DF loaddf = MODE == 2 ? df_from(a.loads[s * 6 + comp]) : DF(0.f, 0.f);
  float acc_s = 0.f, acc_c = 0.f;  // compensated (r, r) of this thread
  constexpr int NP = N / 2;         // element pairs per row
  for (int e = threadIdx.x; e < RY * NP; e += XC::THREADS) {
    const int rowl = e / NP, x = 2 * (e - rowl * NP);
    const long long vox = vox0 + (long long)rowl * N + x;
    const long long gi = (row0 + rowl) * N + x;
    const double2 xv = *reinterpret_cast<const double2*>(xin + gi);
    const uchar2 ph = *reinterpret_cast<const uchar2*>(a.phase + pbase + vox);
    DF o[2];
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int p = h2 == 0 ? ph.x : ph.y;
      o[h2] = DF(0.f, 0.f);
      if (aloc[p]) {
        DF m = mloc[p * a.c + comp];
        if (a.scale) {  // per-voxel moduli: M in FP64, then split
          const double fr = (double)a.scale[pbase + vox + h2];
          const double m0 = a.mtab[comp], m1 = a.mtab[a.c + comp], mp = a.modtab[p * a.c + comp];
          m = df_from(a.frac ? fr * m1 + (1.0 - fr) * m0  // Eq. (def_ah)
                             : 1.0 / (fr * mp - a.ref[comp]));
        }
        const DF mx = m * df_split(h2 == 0 ? xv.x : xv.y) + G[rowl * GS + x + h2];
        if (MODE == 0) {
          o[h2] = mx;
        } else {
          o[h2] = loaddf - mx;
          const float y = __fsub_rn(__fmul_rn(o[h2].h, o[h2].h), acc_c);
          const float tt = __fadd_rn(acc_s, y);
          acc_c = __fsub_rn(__fsub_rn(tt, acc_s), y);
          acc_s = tt;
        }
      }
    }
    if (MODE == 0) *reinterpret_cast<double2*>(out + gi) = make_double2(df_to(o[0]), df_to(o[1]));
    else *reinterpret_cast<float4*>(out + gi) = make_float4(o[0].h, o[0].l, o[1].h, o[1].l);
  }
  if (MODE == 2) {
    Acc<float> acc;
    acc.s = acc_s;
    acc.c = acc_c;
    const double tot = block_reduce(acc);
    double* part = partials + (long long)s * bps;
    SolverState* sst = st + s;
    if (publish_partial_sys(part, blk, bps, tot, &sst->counter[0])) {
      const double sum = gather_partials_sys(part, bps, &sst->counter[0]);
      if (threadIdx.x == 0) sst->aux[0] = sum;
    }
  }
}

// z transform (INV: inverse) of the double-float half spectrum: a block owns
// 16 consecutive kx columns at one (system, component, y); the columns left
// over when nx/2+1 is not a multiple of 16 are gathered 16 at a time.
template <bool INV, int N>
__global__ void __launch_bounds__(16 * RegPlan<N>::P) k_df_zfft(OpArgs<DF> a, int nrt, int nreg) {
  typedef RegLine<DF, N> RL;
  constexpr int TZ = 16, P = RL::P, R1 = RL::R1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DF2* tw = reinterpret_cast<DF2*>(smem_raw);
  DF2* ex = tw + N;
  for (int u = threadIdx.x; u < N; u += blockDim.x) tw[u] = a.twz[u];
  const int i = threadIdx.x % TZ, t = threadIdx.x / TZ;
  const long long nplanes = (long long)a.S * a.c * a.ny;  // (system, component, y)
  const int nleft = a.nxh - nreg;
  long long plane;
  int kx;
  bool valid = true;
  if ((long long)blockIdx.x < nplanes * nrt) {
    plane = blockIdx.x / nrt;
    kx = (int)(blockIdx.x - plane * nrt) * TZ + i;
  } else {
    const long long l = (blockIdx.x - nplanes * nrt) * (long long)TZ + i;
    valid = l < nplanes * nleft;
    plane = valid ? l / nleft : 0;
    kx = valid ? nreg + (int)(l - plane * nleft) : 0;
  }
  const long long sc = plane / a.ny, yp = plane - sc * a.ny;
  DF2* __restrict__ Hl = a.H + (sc * a.nz * a.ny + yp) * a.hs + kx;
  const long long rs = (long long)a.ny * a.hs;  // z stride
  DF2 v[R1];
  __syncthreads();
  if (!INV) {
#pragma unroll
    for (int j = 0; j < R1; ++j) v[j] = valid ? Hl[(t + P * j) * rs] : DF2{DF(0.f, 0.f), DF(0.f, 0.f)};
    RL::fwd_a(v, t, tw, ex + i * RL::LS);
    __syncthreads();
    RL::fwd_b(v, t, tw, ex + i * RL::LS);
    if (valid) {
#pragma unroll
      for (int m = 0; m < R1; ++m) Hl[RL::freq(t, m) * rs] = v[m];
    }
  } else {
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = valid ? Hl[RL::freq(t, m) * rs] : DF2{DF(0.f, 0.f), DF(0.f, 0.f)};
    RL::inv_a(v, t, tw, ex + i * RL::LS);
    __syncthreads();
    RL::inv_b(v, t, tw, ex + i * RL::LS);
    if (valid) {
#pragma unroll
      for (int j = 0; j < R1; ++j) Hl[(t + P * j) * rs] = v[j];
    }
  }
}

// Gamma^h_k applied to the NC components of every system at each frequency
// (natural z and y order); a thread reads its frequency's coefficients once.
template <int NC> __global__ void __launch_bounds__(256) k_df_gamma(OpArgs<DF> a) {
  const long long nfr = (long long)a.nz * a.ny * a.nxh;
  const long long cstride = (long long)a.nz * a.ny * a.hs;  // one component plane
  for (long long f = blockIdx.x * 256ll + threadIdx.x; f < nfr; f += (long long)gridDim.x * 256) {
    const long long r = f / a.nxh;  // z position * ny + y position
    const int kx = (int)(f - r * a.nxh);
    DF gc[GammaPack<NC>::NCO];
    gamma_coef_load<DF, NC>(a.gtab, r * a.ts + kx, gc);
    for (int s = 0; s < a.S; ++s) {
      DF2* h = a.H + (long long)s * NC * cstride + r * a.hs + kx;
      DF2 v[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) v[c] = h[c * cstride];
      gamma_coef_apply<DF, NC>(gc, v);
#pragma unroll
      for (int c = 0; c < NC; ++c) h[c * cstride] = v[c];
    }
  }
}

template <int N> size_t df_z_smem() { return sizeof(DF2) * (size_t)(N + 16 * RegLine<DF, N>::LS); }

template <bool INV, int N> void launch_df_zfft_n(const OpArgs<DF>& a, cudaStream_t s) {
  constexpr int TZ = 16;
  const int nrt = a.nxh / TZ, nreg = nrt * TZ;
  const long long nplanes = (long long)a.S * a.c * a.ny;
  const long long grid = nplanes * nrt + (nplanes * (a.nxh - nreg) + TZ - 1) / TZ;
  k_df_zfft<INV, N><<<(unsigned)grid, TZ * RegPlan<N>::P, df_z_smem<N>(), s>>>(a, nrt, nreg);
}

template <bool INV> void launch_df_zfft(const OpArgs<DF>& a, cudaStream_t s) {
  switch (a.nz) {
    case 48: launch_df_zfft_n<INV, 48>(a, s); break;
    case 96: launch_df_zfft_n<INV, 96>(a, s); break;
    case 16: launch_df_zfft_n<INV, 16>(a, s); break;
    case 32: launch_df_zfft_n<INV, 32>(a, s); break;
    case 64: launch_df_zfft_n<INV, 64>(a, s); break;
    case 128: launch_df_zfft_n<INV, 128>(a, s); break;
    default: launch_df_zfft_n<INV, 256>(a, s); break;
  }
}

// the z pass with Gamma^h in double-float: three launches
void launch_df_z(const OpArgs<DF>& a, cudaStream_t s) {
  launch_df_zfft<false>(a, s);
  const long long nfr = (long long)a.nz * a.ny * a.nxh;
  const unsigned g = (unsigned)std::min<long long>((nfr + 255) / 256, 152ll * 8);
  if (a.c == 6) k_df_gamma<6><<<g, 256, 0, s>>>(a);
  else k_df_gamma<3><<<g, 256, 0, s>>>(a);
  launch_df_zfft<true>(a, s);
}

bool df_length(int n) { return n == 16 || n == 32 || n == 48 || n == 64 || n == 96 || n == 128 || n == 256; }

// The double-float passes cover 3D grids whose three lengths have register
// plans and operators without finite-difference phases.
bool df_supported(const OpArgs<double>& a) {
  return df_length(a.nx) && df_length(a.ny) && df_length(a.nz) && !a.fdphase && (a.c == 6 || a.c == 3);
}

void launch_d2df(const double* in, DF* out, long long n, cudaStream_t s) {
  if (n <= 0) return;
  const long long g = std::min<long long>((n + 255) / 256, 4096);
  k_d2df<<<(unsigned)g, 256, 0, s>>>(in, out, n);
}

// FP64 values converted to double-float pairs in place (both 8 bytes per value).
__global__ void k_d2df_inplace(void* buf, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = reinterpret_cast<const double*>(buf)[i];
    reinterpret_cast<DF*>(buf)[i] = df_from(v);
  }
}

void launch_d2df_inplace(void* buf, long long n, cudaStream_t s) {
  if (n <= 0) return;
  const long long g = std::min<long long>((n + 255) / 256, 4096);
  k_d2df_inplace<<<(unsigned)g, 256, 0, s>>>(buf, n);
}

template <int N> void launch_df_x_n(const OpArgs<double>& a, const DF2* twx, int mode, const double* in, double* out,
                                    SolverState* st, double* partials, cudaStream_t s) {
  typedef XDf<N> XC;
  const int bps = a.rps / XC::RY;
  const unsigned grid = (unsigned)(a.S * bps);
  if (mode < 0) k_df_xfwd<N><<<grid, XC::THREADS, XC::SMEM, s>>>(a, twx, in, bps);
  else if (mode == 0) k_df_xinv<0, N><<<grid, XC::THREADS, XC::SMEM, s>>>(a, twx, in, out, st, partials, bps);
  else k_df_xinv<2, N><<<grid, XC::THREADS, XC::SMEM, s>>>(a, twx, in, out, st, partials, bps);
}

// mode -1: forward x pass of P in; 0: inverse x pass, out = P (M in + g);
// 2: inverse x pass, out = P (load - M in - g) as double-float pairs, with
// (out, out) -> st[s].aux[0].
void launch_df_x(const OpArgs<double>& a, const DF2* twx, int mode, const double* in, double* out, SolverState* st,
                 double* partials, cudaStream_t s) {
  switch (a.nx) {
    case 48: launch_df_x_n<48>(a, twx, mode, in, out, st, partials, s); break;
    case 96: launch_df_x_n<96>(a, twx, mode, in, out, st, partials, s); break;
    case 16: launch_df_x_n<16>(a, twx, mode, in, out, st, partials, s); break;
    case 32: launch_df_x_n<32>(a, twx, mode, in, out, st, partials, s); break;
    case 64: launch_df_x_n<64>(a, twx, mode, in, out, st, partials, s); break;
    case 128: launch_df_x_n<128>(a, twx, mode, in, out, st, partials, s); break;
    default: launch_df_x_n<256>(a, twx, mode, in, out, st, partials, s); break;
  }
}

template <int N> void df_attrs_n() {
  const int zb = (int)df_z_smem<N>();
  cudaFuncSetAttribute(k_df_zfft<false, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, zb);
  cudaFuncSetAttribute(k_df_zfft<true, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, zb);
  const int bytes = (int)XDf<N>::SMEM;
  cudaFuncSetAttribute(k_df_xfwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_df_xinv<0, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_df_xinv<2, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// launch attributes, set once outside any stream capture
void df_prepare() {
  df_attrs_n<16>();
  df_attrs_n<32>();
  df_attrs_n<48>();
  df_attrs_n<96>();
  df_attrs_n<64>();
  df_attrs_n<128>();
  df_attrs_n<256>();
  set_smem_attrs_reg<DF>();
}

}  // namespace lsh
