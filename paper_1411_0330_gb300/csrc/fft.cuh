// fft.cuh -- batched in-place mixed-radix FFT of lines held in shared memory.
//
// Forward transforms are decimation-in-frequency (DIF): natural-order input,
// digit-reversed output.  Inverse transforms are decimation-in-time (DIT):
// digit-reversed input, natural-order output, unnormalised.  Because the
// Green-operator product between them is per frequency, the spectrum is never
// permuted: the kernels only need the frequency k stored at each position.
//
// Stage s of a DIF with radix r acts on spans of length L (L = n for the
// first stage, divided by r after each stage), m = L / r.  For j < m:
//   y_p = (sum_q a_q w_r^{pq}) w_L^{pj},  a_q = x[j + q m],  y_p -> x[j + p m],
// with w_N = exp(-2 i pi / N).  The frequency k of an n-point transform ends up
// at position pos(k) = sum_s d_s m_s, where k = d_1 + r_1 (d_2 + r_2 (...)).
// The DIT stage is the exact inverse of the DIF stage up to the factor r.
//
// All threads of the block cooperate; each stage ends with __syncthreads().
// Twiddles come from a per-axis table tw[t] = exp(-2 i pi t / n), t < n.
#pragma once

#include "common.cuh"

namespace lsh {

template <typename T, int R, bool INV> struct Dft;

template <typename T, bool INV> struct Dft<T, 2, INV> {
  static __device__ __forceinline__ void run(C2<T>* a, const C2<T>*, int) {
    C2<T> t = a[1];
    a[1] = csub<T>(a[0], t);
    a[0] = cadd<T>(a[0], t);
  }
};

template <typename T, bool INV> struct Dft<T, 4, INV> {
  static __device__ __forceinline__ void run(C2<T>* a, const C2<T>*, int) {
    C2<T> t0 = cadd<T>(a[0], a[2]), t1 = csub<T>(a[0], a[2]);
    C2<T> t2 = cadd<T>(a[1], a[3]), t3 = csub<T>(a[1], a[3]);
    C2<T> r3 = INV ? cmul_pi<T>(t3) : cmul_mi<T>(t3);  // w_4^{1} t3
    a[0] = cadd<T>(t0, t2);
    a[2] = csub<T>(t0, t2);
    a[1] = cadd<T>(t1, r3);
    a[3] = csub<T>(t1, r3);
  }
};

template <typename T, bool INV> struct Dft<T, 8, INV> {
  static __device__ __forceinline__ void run(C2<T>* a, const C2<T>* tw, int n) {
    const T h = (T)0.70710678118654752440084436210484903928;  // 1/sqrt(2)
    C2<T> e[4] = {a[0], a[2], a[4], a[6]};
    C2<T> o[4] = {a[1], a[3], a[5], a[7]};
    Dft<T, 4, INV>::run(e, tw, n);
    Dft<T, 4, INV>::run(o, tw, n);
    // o_p *= w_8^p
    C2<T> o1 = o[1], o3 = o[3];
    if (!INV) {
      o[1] = mkc<T>((o1.x + o1.y) * h, (o1.y - o1.x) * h);
      o[2] = cmul_mi<T>(o[2]);
      o[3] = mkc<T>((o3.y - o3.x) * h, -(o3.x + o3.y) * h);
    } else {
      o[1] = mkc<T>((o1.x - o1.y) * h, (o1.x + o1.y) * h);
      o[2] = cmul_pi<T>(o[2]);
      o[3] = mkc<T>(-(o3.x + o3.y) * h, (o3.x - o3.y) * h);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      a[p] = cadd<T>(e[p], o[p]);
      a[p + 4] = csub<T>(e[p], o[p]);
    }
  }
};

template <typename T, bool INV> struct Dft<T, 3, INV> {
  static __device__ __forceinline__ void run(C2<T>* a, const C2<T>*, int) {
    const T s3 = (T)0.86602540378443864676372317075293618347;  // sqrt(3)/2
    C2<T> s = cadd<T>(a[1], a[2]), d = csub<T>(a[1], a[2]);
    C2<T> m = mkc<T>(a[0].x - (T)0.5 * s.x, a[0].y - (T)0.5 * s.y);
    C2<T> rd = INV ? cmul_pi<T>(d) : cmul_mi<T>(d);  // +-i d
    a[0] = cadd<T>(a[0], s);
    a[1] = mkc<T>(m.x + s3 * rd.x, m.y + s3 * rd.y);
    a[2] = mkc<T>(m.x - s3 * rd.x, m.y - s3 * rd.y);
  }
};

template <typename T, bool INV> struct Dft<T, 5, INV> {
  static __device__ __forceinline__ void run(C2<T>* a, const C2<T>*, int) {
    const T c1 = (T)0.30901699437494742410229341718281905886;   // cos(2pi/5)
    const T c2 = (T)-0.80901699437494742410229341718281905886;  // cos(4pi/5)
    const T s1 = (T)0.95105651629515357211643933337938214340;   // sin(2pi/5)
    const T s2 = (T)0.58778525229247312916870595463907276860;   // sin(4pi/5)
    C2<T> p14 = cadd<T>(a[1], a[4]), m14 = csub<T>(a[1], a[4]);
    C2<T> p23 = cadd<T>(a[2], a[3]), m23 = csub<T>(a[2], a[3]);
    C2<T> b1 = mkc<T>(a[0].x + c1 * p14.x + c2 * p23.x, a[0].y + c1 * p14.y + c2 * p23.y);
    C2<T> b2 = mkc<T>(a[0].x + c2 * p14.x + c1 * p23.x, a[0].y + c2 * p14.y + c1 * p23.y);
    C2<T> u1 = mkc<T>(s1 * m14.x + s2 * m23.x, s1 * m14.y + s2 * m23.y);
    C2<T> u2 = mkc<T>(s2 * m14.x - s1 * m23.x, s2 * m14.y - s1 * m23.y);
    // forward: y1 = b1 - i u1, y4 = b1 + i u1, y2 = b2 - i u2, y3 = b2 + i u2
    C2<T> iu1 = INV ? cmul_pi<T>(u1) : cmul_mi<T>(u1);
    C2<T> iu2 = INV ? cmul_pi<T>(u2) : cmul_mi<T>(u2);
    a[0] = mkc<T>(a[0].x + p14.x + p23.x, a[0].y + p14.y + p23.y);
    a[1] = cadd<T>(b1, iu1);
    a[4] = csub<T>(b1, iu1);
    a[2] = cadd<T>(b2, iu2);
    a[3] = csub<T>(b2, iu2);
  }
};

// 16 = 4 x 4: x[n2 + 4 n1] -> X[k1 + 4 k2] = sum_n2 w4^(n2 k2) w16^(n2 k1) sum_n1 x[n2 + 4 n1] w4^(n1 k1)
template <typename T, bool INV> struct Dft<T, 16, INV> {
  static __device__ __forceinline__ void run(C2<T>* a, const C2<T>* tw, int n) {
    const T c1 = (T)0.92387953251128675612818318939678828682;  // cos(pi/8)
    const T s1 = (T)0.38268343236508977172845998403039886676;  // sin(pi/8)
    const T h = (T)0.70710678118654752440084436210484903928;   // cos(pi/4)
    C2<T> b[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      C2<T> c[4] = {a[n2], a[n2 + 4], a[n2 + 8], a[n2 + 12]};
      Dft<T, 4, INV>::run(c, tw, n);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) b[n2][k1] = c[k1];
    }
    // twiddles w16^m, m = n2 k1: (cos, -+sin) of 2 pi m / 16
    const T sg = INV ? (T)1 : (T)-1;
    const C2<T> w1 = mkc<T>(c1, sg * s1), w2 = mkc<T>(h, sg * h), w3 = mkc<T>(s1, sg * c1);
    const C2<T> w6 = mkc<T>(-h, sg * h), w9 = mkc<T>(-c1, -sg * s1);
    b[1][1] = cmul<T>(b[1][1], w1);
    b[1][2] = cmul<T>(b[1][2], w2);
    b[1][3] = cmul<T>(b[1][3], w3);
    b[2][1] = cmul<T>(b[2][1], w2);
    b[2][2] = INV ? cmul_pi<T>(b[2][2]) : cmul_mi<T>(b[2][2]);  // w16^4 = -+i
    b[2][3] = cmul<T>(b[2][3], w6);
    b[3][1] = cmul<T>(b[3][1], w3);
    b[3][2] = cmul<T>(b[3][2], w6);
    b[3][3] = cmul<T>(b[3][3], w9);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C2<T> d[4] = {b[0][k1], b[1][k1], b[2][k1], b[3][k1]};
      Dft<T, 4, INV>::run(d, tw, n);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = d[k2];
    }
  }
};

// 32 = 2 x 16: X[k] = E[k] + w32^k O[k], X[k + 16] = E[k] - w32^k O[k] with E, O
// the 16-point DFTs of the even and odd samples (w32 = exp(-+2 i pi / 32)).
template <typename T, bool INV> struct Dft<T, 32, INV> {
  static __device__ __forceinline__ void run(C2<T>* a, const C2<T>* tw, int n) {
    // cos(pi k / 16), k = 0..8 (sin(pi k / 16) = cos(pi (8 - k) / 16))
    const T cs[9] = {(T)1.0,
                     (T)0.98078528040323044912618223613424,
                     (T)0.92387953251128675612818318939679,
                     (T)0.83146961230254523707878837761791,
                     (T)0.70710678118654752440084436210485,
                     (T)0.55557023301960222474283081394853,
                     (T)0.38268343236508977172845998403040,
                     (T)0.19509032201612826784828486847702,
                     (T)0.0};
    C2<T> e[16], o[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      e[j] = a[2 * j];
      o[j] = a[2 * j + 1];
    }
    Dft<T, 16, INV>::run(e, tw, n);
    Dft<T, 16, INV>::run(o, tw, n);
    const T sg = INV ? (T)1 : (T)-1;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      C2<T> w;
      if (k <= 8) w = mkc<T>(cs[k], sg * cs[8 - k]);
      else w = mkc<T>(-cs[16 - k], sg * cs[k - 8]);
      const C2<T> ow = k == 0 ? o[k] : cmul<T>(o[k], w);
      a[k] = cadd<T>(e[k], ow);
      a[k + 16] = csub<T>(e[k], ow);
    }
  }
};

// Direct DFT for the remaining small prime (7), from the twiddle table.
template <typename T, bool INV> struct Dft<T, 7, INV> {
  static __device__ __forceinline__ void run(C2<T>* a, const C2<T>* tw, int n) {
    const int st = n / 7;
    C2<T> y[7];
#pragma unroll
    for (int p = 0; p < 7; ++p) {
      C2<T> s = a[0];
#pragma unroll
      for (int q = 1; q < 7; ++q) {
        C2<T> w = tw[((p * q) % 7) * st];
        s = cadd<T>(s, INV ? cmulc<T>(a[q], w) : cmul<T>(a[q], w));
      }
      y[p] = s;
    }
#pragma unroll
    for (int p = 0; p < 7; ++p) a[p] = y[p];
  }
};

// cos and sin of 2 pi m / 24 (multiples of 15 degrees) from the closed forms
// cos 15 = (sqrt 6 + sqrt 2) / 4, sin 15 = (sqrt 6 - sqrt 2) / 4, cos 30 = sqrt 3 / 2,
// cos 45 = sqrt 2 / 2; once the loops are unrolled m is a constant and these fold.
__host__ __device__ constexpr double cos24(int m) {
  constexpr double c15 = 0.96592582628906828674974319972889736763, s15 = 0.25881904510252076234889883762404832835;
  constexpr double c30 = 0.86602540378443864676372317075293618347, c45 = 0.70710678118654752440084436210484903928;
  switch (((m % 24) + 24) % 24) {
    case 0: return 1.0;
    case 1: return c15;
    case 2: return c30;
    case 3: return c45;
    case 4: return 0.5;
    case 5: return s15;
    case 6: return 0.0;
    case 7: return -s15;
    case 8: return -0.5;
    case 9: return -c45;
    case 10: return -c30;
    case 11: return -c15;
    case 12: return -1.0;
    case 13: return -c15;
    case 14: return -c30;
    case 15: return -c45;
    case 16: return -0.5;
    case 17: return -s15;
    case 18: return 0.0;
    case 19: return s15;
    case 20: return 0.5;
    case 21: return c45;
    case 22: return c30;
    default: return c15;
  }
}
__host__ __device__ constexpr double sin24(int m) { return cos24(m - 6); }

// Composite lengths R = A * B in registers (Cooley-Tukey with B-point outer
// and A-point inner DFTs): x[B n1 + n2] -> X[k1 + A k2] =
//   sum_n2 w_B^(n2 k2) [ w_R^(n2 k1) sum_n1 x[B n1 + n2] w_A^(n1 k1) ];
// the twiddles w_R^m are constants for R dividing 24 (the radix-3 lengths 6,
// 12, 24), else they come from the line's table tw of length n (stride n / R).
template <typename T, int A, int B, bool INV> struct DftAB {
  static __device__ __forceinline__ C2<T> twiddle(const C2<T>& c, int m, const C2<T>* tw, int st) {
    constexpr int R = A * B;
    if constexpr (24 % R == 0) {
      const int m24 = m * (24 / R);
      const C2<T> w = mkc<T>((T)cos24(m24), (T)(INV ? sin24(m24) : -sin24(m24)));
      return cmul<T>(c, w);
    } else {
      return INV ? cmulc<T>(c, tw[m * st]) : cmul<T>(c, tw[m * st]);
    }
  }
  static __device__ __forceinline__ void run(C2<T>* a, const C2<T>* tw, int n) {
    constexpr int R = A * B;
    const int st = n / R;
    C2<T> b[B][A];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
      C2<T> c[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) c[n1] = a[B * n1 + n2];
      Dft<T, A, INV>::run(c, tw, n);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1)
        b[n2][k1] = (n2 == 0 || k1 == 0) ? c[k1] : twiddle(c[k1], n2 * k1, tw, st);
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      C2<T> d[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) d[n2] = b[n2][k1];
      Dft<T, B, INV>::run(d, tw, n);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) a[k1 + A * k2] = d[k2];
    }
  }
};
template <typename T, bool INV> struct Dft<T, 6, INV> : DftAB<T, 2, 3, INV> {};
template <typename T, bool INV> struct Dft<T, 12, INV> : DftAB<T, 4, 3, INV> {};
template <typename T, bool INV> struct Dft<T, 24, INV> : DftAB<T, 8, 3, INV> {};

template <typename T, int R, bool INV>
__device__ __forceinline__ void butterfly(C2<T>* base, int m, int te, const C2<T>* tw, int n) {
  C2<T> a[R];
#pragma unroll
  for (int q = 0; q < R; ++q) a[q] = base[q * m];
  if (!INV) {
    Dft<T, R, false>::run(a, tw, n);
    if (te != 0) {
#pragma unroll
      for (int p = 1; p < R; ++p) a[p] = cmul<T>(a[p], tw[p * te]);
    }
  } else {
    if (te != 0) {
#pragma unroll
      for (int p = 1; p < R; ++p) a[p] = cmulc<T>(a[p], tw[p * te]);
    }
    Dft<T, R, true>::run(a, tw, n);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) base[q * m] = a[q];
}

// One stage over `nlines` lines of length n (line stride ls, element stride 1).
template <typename T, bool INV>
__device__ __forceinline__ void fft_stage(C2<T>* __restrict__ buf, int nlines, int ls, int n, int r, int L,
                                          const C2<T>* __restrict__ tw) {
  const int m = L / r, nb = n / r, total = nb * nlines, tws = n / L;
  const bool jmajor = m >= 16;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    int line, b;
    if (jmajor) {
      line = fdiv(w, nb);
      b = w - line * nb;
    } else {
      b = fdiv(w, nlines);
      line = w - b * nlines;
    }
    const int sp = fdiv(b, m), j = b - sp * m;
    C2<T>* base = buf + line * ls + sp * L + j;
    const int te = j * tws;
    switch (r) {
      case 8: butterfly<T, 8, INV>(base, m, te, tw, n); break;
      case 4: butterfly<T, 4, INV>(base, m, te, tw, n); break;
      case 2: butterfly<T, 2, INV>(base, m, te, tw, n); break;
      case 3: butterfly<T, 3, INV>(base, m, te, tw, n); break;
      case 5: butterfly<T, 5, INV>(base, m, te, tw, n); break;
      default: butterfly<T, 7, INV>(base, m, te, tw, n); break;
    }
  }
}

// ---------------------------------------------------------------- compile-time schedules
// For the common lengths the radix sequence is a template argument: every
// index split becomes a shift or a mask and the stage loop unrolls.
template <typename T, bool INV, int N, int R, int L>
__device__ __forceinline__ void stage_ct(C2<T>* __restrict__ buf, int nlines, int ls, const C2<T>* __restrict__ tw) {
  constexpr int m = L / R, nb = N / R, tws = N / L;
  constexpr bool jmajor = m >= 16;
  const int total = nb * nlines;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    int line, b;
    if (jmajor) {
      line = w / nb;
      b = w - line * nb;
    } else {
      b = fdiv(w, nlines);
      line = w - b * nlines;
    }
    const int sp = b / m, j = b - sp * m;
    butterfly<T, R, INV>(buf + line * ls + sp * L + j, m, j * tws, tw, N);
  }
}

template <typename T, int N, int L, int... Rs> struct DifStages {
  static __device__ __forceinline__ void run(C2<T>*, int, int, const C2<T>*) {}
};
template <typename T, int N, int L, int R, int... Rs> struct DifStages<T, N, L, R, Rs...> {
  static __device__ __forceinline__ void run(C2<T>* buf, int nlines, int ls, const C2<T>* tw) {
    stage_ct<T, false, N, R, L>(buf, nlines, ls, tw);
    __syncthreads();
    DifStages<T, N, L / R, Rs...>::run(buf, nlines, ls, tw);
  }
};
// DIT stages run the DIF radices in reverse; the span of a stage is its radix
// times the product of the radices after it.
template <typename T, int N, int... Rs> struct DitStages {
  static constexpr int P = 1;
  static __device__ __forceinline__ void run(C2<T>*, int, int, const C2<T>*) {}
};
template <typename T, int N, int R, int... Rs> struct DitStages<T, N, R, Rs...> {
  static constexpr int P = R * DitStages<T, N, Rs...>::P;
  static __device__ __forceinline__ void run(C2<T>* buf, int nlines, int ls, const C2<T>* tw) {
    DitStages<T, N, Rs...>::run(buf, nlines, ls, tw);
    stage_ct<T, true, N, R, P>(buf, nlines, ls, tw);
    __syncthreads();
  }
};

template <int... Rs> __device__ __forceinline__ bool plan_is(const Plan1D& pl) {
  constexpr int r[] = {Rs...};
  constexpr int k = sizeof...(Rs);
  if (pl.nst != k) return false;
#pragma unroll
  for (int i = 0; i < k; ++i)
    if (pl.radix[i] != r[i]) return false;
  return true;
}

template <typename T, bool INV, int N, int... Rs>
__device__ __forceinline__ bool try_fixed(C2<T>* buf, int nlines, int ls, const Plan1D& pl, const C2<T>* tw) {
  if (pl.n != N || !plan_is<Rs...>(pl)) return false;
  if (INV) DitStages<T, N, Rs...>::run(buf, nlines, ls, tw);
  else DifStages<T, N, N, Rs...>::run(buf, nlines, ls, tw);
  return true;
}

template <typename T, bool INV>
__device__ void fft_lines_generic(C2<T>* buf, int nlines, int ls, const Plan1D& pl, const C2<T>* tw);

// Forward (DIF) or inverse (DIT) transform of nlines lines; ends synchronised.
// The fixed schedules mirror the host's radix choice (8s first, an 8*2 pair
// becomes 4*4, then 3, 5, 7); any other plan runs the generic stage loop.
template <typename T, bool INV>
__device__ void fft_lines(C2<T>* buf, int nlines, int ls, const Plan1D& pl, const C2<T>* tw) {
  if (try_fixed<T, INV, 128, 4, 8, 4>(buf, nlines, ls, pl, tw)) return;
  if (try_fixed<T, INV, 64, 8, 8>(buf, nlines, ls, pl, tw)) return;
  if (try_fixed<T, INV, 256, 8, 8, 4>(buf, nlines, ls, pl, tw)) return;
  if (try_fixed<T, INV, 32, 8, 4>(buf, nlines, ls, pl, tw)) return;
  if (try_fixed<T, INV, 96, 8, 4, 3>(buf, nlines, ls, pl, tw)) return;
  if (try_fixed<T, INV, 48, 4, 4, 3>(buf, nlines, ls, pl, tw)) return;
  if (try_fixed<T, INV, 16, 4, 4>(buf, nlines, ls, pl, tw)) return;
  fft_lines_generic<T, INV>(buf, nlines, ls, pl, tw);
}

template <typename T, bool INV>
__device__ void fft_lines_generic(C2<T>* buf, int nlines, int ls, const Plan1D& pl, const C2<T>* tw) {
  const int n = pl.n;
  if (!INV) {
    int L = n;
    for (int s = 0; s < pl.nst; ++s) {
      fft_stage<T, false>(buf, nlines, ls, n, pl.radix[s], L, tw);
      L /= pl.radix[s];
      __syncthreads();
    }
  } else {
    int L = 1;
    for (int s = pl.nst - 1; s >= 0; --s) {
      L *= pl.radix[s];
      fft_stage<T, true>(buf, nlines, ls, n, pl.radix[s], L, tw);
      __syncthreads();
    }
  }
}

}  // namespace lsh
