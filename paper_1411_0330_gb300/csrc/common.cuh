// common.cuh -- device-side types and helpers shared by the liblsh kernels.
//
// Precision-generic complex arithmetic (float2 / double2), the device-resident
// CG state, and deterministic block / grid reductions (per-block partials in
// FP64, summed in block-index order by the last block to finish: no spin
// waits, bit-identical results run to run).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lsh {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { typedef float2 type; };
template <> struct cplx_of<double> { typedef double2 type; };
template <typename T> using C2 = typename cplx_of<T>::type;

template <typename T> __device__ __forceinline__ C2<T> mkc(T a, T b) {
  C2<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T> __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return mkc<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return mkc<T>(a.x - b.x, a.y - b.y); }
// a * b
template <typename T> __device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __device__ __forceinline__ C2<T> cmulc(C2<T> a, C2<T> b) {
  return mkc<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// a * (-i)  and  a * (+i)
template <typename T> __device__ __forceinline__ C2<T> cmul_mi(C2<T> a) { return mkc<T>(a.y, -a.x); }
template <typename T> __device__ __forceinline__ C2<T> cmul_pi(C2<T> a) { return mkc<T>(-a.y, a.x); }
template <typename T> __device__ __forceinline__ C2<T> cscale(C2<T> a, T s) { return mkc<T>(a.x * s, a.y * s); }

// Device-resident state of one Krylov solve.  Scalars are always FP64.
struct SolverState {
  double rr;        // (r_k, r_k)
  double bb;        // (b, b) of the system being solved
  double tol2;      // stop when rr <= tol2 (= tol^2 bb)
  double alpha;     // alpha of the last completed iteration (0 after breakdown)
  double beta;      // beta_{k-1}
  double pq;        // (p_k, K p_k)
  double aux[4];    // extra reduction results (component sums, ...)
  int iter;         // completed CG iterations
  int done;         // nonzero: converged or failed, later kernels return at once
  int status;       // lsh_status-compatible code set on device (0, breakdown)
  int pad;
  unsigned int counter[4];  // last-block counters, reset by the last block
};

// Per-thread accumulator for inner products.  FP64 fields: plain double sum.
// FP32 fields: Kahan-compensated float sum (the FP64 pipe of GB300 is 64x
// slower than the FP32 one), handed to the FP64 block / grid reduction.
template <typename T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double get() const { return s; }
};
template <> struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// Block sum of per-thread accumulators; result valid in thread 0.  FP32
// compensated pairs are first merged across the warp in FP32 (TwoSum keeps
// the rounding error of each merge), so only one value per warp touches the
// FP64 pipe.
__device__ __forceinline__ double block_sum(double v);
__device__ __forceinline__ double block_reduce(const Acc<double>& a) { return block_sum(a.get()); }
__device__ __forceinline__ void warp_merge_pair(float& s, float& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_down_sync(0xffffffffu, s, o);
    const float c2 = __shfl_down_sync(0xffffffffu, c, o);
    const float t = s + s2;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (s2 - bp);  // s + s2 = t + e exactly
    s = t;
    c = c + c2 - e;
  }
}
__device__ __forceinline__ double block_reduce(const Acc<float>& a) {
  __shared__ float pair_sh[2][32];
  float s = a.s, c = a.c;  // value = s - c
  warp_merge_pair(s, c);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    pair_sh[0][w] = s;
    pair_sh[1][w] = c;
  }
  __syncthreads();
  double out = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    s = l < nw ? pair_sh[0][l] : 0.0f;
    c = l < nw ? pair_sh[1][l] : 0.0f;
    warp_merge_pair(s, c);
    if (l == 0) out = (double)s - (double)c;
  }
  return out;
}

// a / d with a shift when d is a power of two (d is uniform across the block).
__device__ __forceinline__ int fdiv(int a, int d) { return (d & (d - 1)) == 0 ? (a >> (__ffs(d) - 1)) : a / d; }

// FFT plan of one axis: length n = product of the radices, DIF stage order.
#define LSH_MAX_STAGES 8
struct Plan1D {
  int n;
  int nst;
  int radix[LSH_MAX_STAGES];
};

// ---------------------------------------------------------------- reductions
// Sum of one double per thread; result valid in thread 0.  Deterministic for a
// fixed block size.  Every thread of the block must call it.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red_sh[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red_sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < (unsigned)nw) ? red_sh[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Publish this block's partial and report whether the block is the last one
// of the grid to do so.  The last block then owns partials[0..nblocks).
__device__ __forceinline__ bool publish_partial(double* partials, double v, unsigned int* counter) {
  __shared__ int is_last;
  const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
  const unsigned int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  if (threadIdx.x == 0) {
    partials[b] = v;
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    is_last = (t == nb - 1);
  }
  __syncthreads();
  return is_last != 0;
}

// In the last block: ordered sum of the partials (result in thread 0), and
// counter reset for the next launch.
__device__ __forceinline__ double gather_partials(const double* partials, unsigned int* counter) {
  __threadfence();
  const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
  double s = 0.0;
  for (unsigned int i = threadIdx.x; i < nb; i += blockDim.x) s += __ldcg(partials + i);
  s = block_sum(s);
  if (threadIdx.x == 0) *counter = 0u;
  return s;
}

// Variants for a reduction over `nb` blocks of one system out of many in the
// grid: block `b` (0..nb-1 within its system) publishes to partials[b].
__device__ __forceinline__ bool publish_partial_sys(double* partials, unsigned int b, unsigned int nb, double v,
                                                    unsigned int* counter) {
  __shared__ int is_last_sys;
  if (threadIdx.x == 0) {
    partials[b] = v;
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    is_last_sys = (t == nb - 1);
  }
  __syncthreads();
  return is_last_sys != 0;
}

__device__ __forceinline__ double gather_partials_sys(const double* partials, unsigned int nb, unsigned int* counter) {
  __threadfence();
  double s = 0.0;
  for (unsigned int i = threadIdx.x; i < nb; i += blockDim.x) s += __ldcg(partials + i);
  s = block_sum(s);
  if (threadIdx.x == 0) *counter = 0u;
  return s;
}

// Scalars of one system's MINRES recurrence (Lanczos + Givens, Paige-Saunders),
// kept on the device next to its SolverState.
struct MinresScalars {
  double beta1, beta, oldb, alfa;
  double dbar, epsln, oldeps, phibar;
  double cs, sn, phi, delta, denom;
  int pending;  // converged after this iteration's update of x
  int pad;
};

// Scalars of one system's SYMMLQ recurrence (Lanczos as for MINRES, whose
// MinresScalars keep beta1, beta, oldb and alfa; LQ factorisation of the
// tridiagonal matrix by rotations from the right, Paige-Saunders 1975).
struct SymmlqScalars {
  double gbar, dbar, rhs1, rhs2;
  double bstep, snprod;     // step along the first Lanczos vector, product of the sines
  double s, t, cs, sn;      // this iteration's update x += s w + t v, w <- sn w - cs v
  double zbar, cb;          // at exit: x += zbar w + cb b (the CG point)
  int pending;
  int pad;
};

}  // namespace lsh
