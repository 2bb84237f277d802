// lse_common.cuh -- small complex type, phase helpers and block reductions
// shared by the kernels of the line-spectral-estimation library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lse {

// ---------------------------------------------------------------------------
// complex numbers over float or double, 2*sizeof(T)-aligned so that one
// element moves in a single vector load/store
// ---------------------------------------------------------------------------
template <class T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

template <class T> __host__ __device__ __forceinline__ cx<T> mk(T r, T i) { cx<T> z; z.re = r; z.im = i; return z; }
template <class T> __host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <class T> __host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <class T> __host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class T> __host__ __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk(s * a.re, s * a.im); }
template <class T> __host__ __device__ __forceinline__ cx<T> conj(cx<T> a) { return mk(a.re, -a.im); }
template <class T> __host__ __device__ __forceinline__ cx<T> conj_mul(cx<T> a, cx<T> b) {  // conj(a) * b
  return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
template <class T> __host__ __device__ __forceinline__ T norm2(cx<T> a) { return a.re * a.re + a.im * a.im; }
template <class T> __host__ __device__ __forceinline__ cx<T> mul_j(cx<T> a) { return mk(-a.im, a.re); }  // j*a
template <class T> __host__ __device__ __forceinline__ cx<T> zero() { return mk<T>(0, 0); }

template <class D, class S> __host__ __device__ __forceinline__ cx<D> cvt(cx<S> a) { return mk<D>((D)a.re, (D)a.im); }

using c64 = cx<float>;
using c128 = cx<double>;

// ---------------------------------------------------------------------------
// exp(j 2 pi n theta) for integer n >= 0 with n*theta reduced modulo 1 without
// rounding error: fma gives the exact low part of the product, so the
// fractional phase is exact to ~1 ulp of 1 even for n*theta ~ 1e5.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double frac_product(double n, double theta) {
  double p = n * theta;
  double e = fma(n, theta, -p);  // exact: p + e = n*theta
  double f = p - floor(p);       // exact for p < 2^52
  f += e;
  f -= floor(f);
  return f;
}

__device__ __forceinline__ c128 unit_phase(double n, double theta, double sign) {
  double s, c;
  sincospi(2.0 * frac_product(n, theta), &s, &c);
  return mk(c, sign * s);
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one value per thread; the result is returned to every
// thread.  `red` is shared scratch of at least NT/32 elements.  Contains two
// __syncthreads and may be called back to back.
template <int NT, class T> __device__ T block_sum(T v, T* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T r = 0;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) r += red[i];
  return r;
}

// Block-wide (value, index) minimum with ties broken towards the lower index.
struct MinLoc {
  double v;
  int i;
};
__device__ __forceinline__ MinLoc minloc(MinLoc a, MinLoc b) {
  if (b.v < a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}
__device__ __forceinline__ MinLoc warp_minloc(MinLoc m) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    MinLoc n;
    n.v = __shfl_xor_sync(0xffffffffu, m.v, o);
    n.i = __shfl_xor_sync(0xffffffffu, m.i, o);
    m = minloc(m, n);
  }
  return m;
}
template <int NT> __device__ MinLoc block_minloc(MinLoc m, MinLoc* red) {
  m = warp_minloc(m);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = m;
  __syncthreads();
  MinLoc r = red[0];
#pragma unroll
  for (int i = 1; i < NT / 32; ++i) r = minloc(r, red[i]);
  return r;
}

__host__ __device__ __forceinline__ int ilog2(uint32_t x) {
  int r = 0;
  while ((1u << r) < x) ++r;
  return r;
}
__host__ __device__ __forceinline__ uint32_t next_pow2(uint32_t x) { return 1u << ilog2(x); }

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.28318530717958647692;

}  // namespace lse
