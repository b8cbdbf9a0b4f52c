// regfft.cuh -- two-level register FFT of lines of length N = R1 * P.
//
// A line is held by P threads; thread t owns the R1 values x[t + P j],
// j < R1.  With n = t + P j and k = k1 + R1 k2,
//   X[k] = sum_t w_P^(t k2) [ w_N^(t k1) sum_j x[t + P j] w_R1^(j k1) ],
// so the forward transform is: an R1-point DFT in registers, the twiddle
// w_N^(t k1), one transpose through shared memory, and P-point DFTs in
// registers (each thread takes Q = R1 / P of the k1).  Frequencies come out
// in natural order.  The inverse runs the same steps backwards with
// conjugate twiddles and is unnormalised.  Compared with one shared-memory
// round trip per radix stage this moves every element through shared memory
// once per transform.
#pragma once

#include "fft.cuh"

namespace lsh {

template <int N> struct RegPlan;
template <> struct RegPlan<16> { static constexpr int R1 = 4, P = 4; };
template <> struct RegPlan<32> { static constexpr int R1 = 8, P = 4; };
template <> struct RegPlan<64> { static constexpr int R1 = 8, P = 8; };
template <> struct RegPlan<128> { static constexpr int R1 = 16, P = 8; };
// radix-3 lengths (FP32 passes): R1 = 3 P keeps Q = R1 / P whole
template <> struct RegPlan<48> { static constexpr int R1 = 12, P = 4; };
template <> struct RegPlan<96> { static constexpr int R1 = 24, P = 4; };
template <> struct RegPlan<256> { static constexpr int R1 = 16, P = 16; };

template <typename T, int N> struct RegLine {
  static constexpr int R1 = RegPlan<N>::R1, P = RegPlan<N>::P, Q = R1 / P;
  static constexpr int EXS = P + 1;                    // row stride of the exchange area
  static constexpr int RAW = R1 * EXS;                 // complex elements of one line
  static constexpr int LS = RAW | 1;                   // odd line stride: conflict-free across lines

  // a[j] = x[t + P j] in; a[k1] = w_N^(t k1) DFT_R1(...)[k1] written to ex, natural k1.
  static __device__ __forceinline__ void fwd_a(C2<T>* a, int t, const C2<T>* tw, C2<T>* ex) {
    Dft<T, R1, false>::run(a, tw, N);
    if (t != 0) {
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) a[k1] = cmul<T>(a[k1], tw[t * k1]);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) ex[k1 * EXS + t] = a[k1];
  }
  // after a barrier: a[q P + k2] = X[(t Q + q) + R1 k2]
  static __device__ __forceinline__ void fwd_b(C2<T>* a, int t, const C2<T>* tw, const C2<T>* ex) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k1 = t * Q + q;
      C2<T> b[P];
#pragma unroll
      for (int u = 0; u < P; ++u) b[u] = ex[k1 * EXS + u];
      Dft<T, P, false>::run(b, tw, N);
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) a[q * P + k2] = b[k2];
    }
  }
  // a[q P + k2] = X[(t Q + q) + R1 k2] in; P-point inverse DFTs written to ex
  static __device__ __forceinline__ void inv_a(const C2<T>* a, int t, const C2<T>* tw, C2<T>* ex) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k1 = t * Q + q;
      C2<T> b[P];
#pragma unroll
      for (int u = 0; u < P; ++u) b[u] = a[q * P + u];
      Dft<T, P, true>::run(b, tw, N);
#pragma unroll
      for (int u = 0; u < P; ++u) ex[k1 * EXS + u] = b[u];
    }
  }
  // after a barrier: a[j] = N x[t + P j]
  static __device__ __forceinline__ void inv_b(C2<T>* a, int t, const C2<T>* tw, const C2<T>* ex) {
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) a[k1] = ex[k1 * EXS + t];
    if (t != 0) {
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) a[k1] = cmulc<T>(a[k1], tw[t * k1]);
    }
    Dft<T, R1, true>::run(a, tw, N);
  }
  // The same four steps with the exchange held in a line of N elements at
  // stride ST (element e = k1 P + u at ex[e ST]), e.g. in place in a tile whose
  // columns are ST apart.
  template <int ST> static __device__ __forceinline__ void fwd_a_s(C2<T>* a, int t, const C2<T>* tw, C2<T>* ex) {
    Dft<T, R1, false>::run(a, tw, N);
    if (t != 0) {
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) a[k1] = cmul<T>(a[k1], tw[t * k1]);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) ex[(k1 * P + t) * ST] = a[k1];
  }
  template <int ST> static __device__ __forceinline__ void fwd_b_s(C2<T>* a, int t, const C2<T>* tw, const C2<T>* ex) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k1 = t * Q + q;
      C2<T> b[P];
#pragma unroll
      for (int u = 0; u < P; ++u) b[u] = ex[(k1 * P + u) * ST];
      Dft<T, P, false>::run(b, tw, N);
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) a[q * P + k2] = b[k2];
    }
  }
  template <int ST> static __device__ __forceinline__ void inv_a_s(const C2<T>* a, int t, const C2<T>* tw, C2<T>* ex) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k1 = t * Q + q;
      C2<T> b[P];
#pragma unroll
      for (int u = 0; u < P; ++u) b[u] = a[q * P + u];
      Dft<T, P, true>::run(b, tw, N);
#pragma unroll
      for (int u = 0; u < P; ++u) ex[(k1 * P + u) * ST] = b[u];
    }
  }
  template <int ST> static __device__ __forceinline__ void inv_b_s(C2<T>* a, int t, const C2<T>* tw, const C2<T>* ex) {
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) a[k1] = ex[(k1 * P + t) * ST];
    if (t != 0) {
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) a[k1] = cmulc<T>(a[k1], tw[t * k1]);
    }
    Dft<T, R1, true>::run(a, tw, N);
  }
  // The four steps with the exchange held in a line of N + N / R1 elements,
  // element e at ex[e + e / R1]: the R1 values a thread writes stay adjacent,
  // the ones it reads sit R1 + 1 apart (conflict-free for odd R1 + 1 banks).
  static __device__ __forceinline__ int xp(int e) { return e + e / R1; }
  static __device__ __forceinline__ void fwd_a_p(C2<T>* a, int t, const C2<T>* tw, C2<T>* ex) {
    Dft<T, R1, false>::run(a, tw, N);
    if (t != 0) {
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) a[k1] = cmul<T>(a[k1], tw[t * k1]);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) ex[xp(k1 * P + t)] = a[k1];
  }
  static __device__ __forceinline__ void fwd_b_p(C2<T>* a, int t, const C2<T>* tw, const C2<T>* ex) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      C2<T> b[P];
#pragma unroll
      for (int u = 0; u < P; ++u) b[u] = ex[t * (R1 + 1) + q * P + u];
      Dft<T, P, false>::run(b, tw, N);
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) a[q * P + k2] = b[k2];
    }
  }
  static __device__ __forceinline__ void inv_a_p(const C2<T>* a, int t, const C2<T>* tw, C2<T>* ex) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      C2<T> b[P];
#pragma unroll
      for (int u = 0; u < P; ++u) b[u] = a[q * P + u];
      Dft<T, P, true>::run(b, tw, N);
#pragma unroll
      for (int u = 0; u < P; ++u) ex[t * (R1 + 1) + q * P + u] = b[u];
    }
  }
  static __device__ __forceinline__ void inv_b_p(C2<T>* a, int t, const C2<T>* tw, const C2<T>* ex) {
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) a[k1] = ex[xp(k1 * P + t)];
    if (t != 0) {
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) a[k1] = cmulc<T>(a[k1], tw[t * k1]);
    }
    Dft<T, R1, true>::run(a, tw, N);
  }
  // frequency held in slot m of thread t after fwd_b (and expected by inv_a)
  static __device__ __forceinline__ int freq(int t, int m) { return (t * Q + m / P) + R1 * (m % P); }
};

}  // namespace lsh
