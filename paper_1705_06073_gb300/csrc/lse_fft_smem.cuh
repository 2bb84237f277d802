// lse_fft_smem.cuh -- one block computes one length-M FFT entirely in shared
// memory (M * sizeof(complex) fits on chip): Stockham decimation in
// frequency with radix-16 passes (a 16-point DFT in registers, as 4 x 4) and
// a radix-4 / radix-2 remainder, in place with a barrier between the reads
// and the writes of every pass.  Twiddles come from two small shared tables
// (W^k = hi[k >> b] lo[k & (2^b - 1)]); shared indices are padded by one
// element per 16 so that the radix-16 scatter of a warp hits distinct banks.
// The last pass hands every output to an epilogue functor instead of
// storing it, so results go straight to global memory, coalesced.
#pragma once

#include "lse_common.cuh"

namespace lse {

__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }

template <class T>
struct SmemTwiddles {
  const cx<T>* lo;
  const cx<T>* hi;
  int lb, mask;
  __device__ __forceinline__ cx<T> w(int k) const { return hi[k >> lb] * lo[k & mask]; }  // W_M^k
};

// Fill the two tables for W_M = exp(-j 2 pi / M) from the global table
// tw[k] = exp(-j 2 pi k / 2^log2max).  lo: 2^lb entries, hi: 2^(log2M-lb).
template <int NT, class T>
__device__ SmemTwiddles<T> make_smem_twiddles(cx<T>* lo, cx<T>* hi, int log2M, const cx<T>* tw, int log2max) {
  const int lb = (log2M + 1) >> 1;
  const int nlo = 1 << lb, nhi = 1 << (log2M - lb);
  const int sh = log2max - log2M;
  for (int j = threadIdx.x; j < nlo; j += NT) lo[j] = tw[(size_t)j << sh];
  for (int j = threadIdx.x; j < nhi; j += NT) hi[j] = tw[(size_t)j << (sh + lb)];
  return SmemTwiddles<T>{lo, hi, lb, nlo - 1};
}

// 4-point DFT in place: forward uses W_4 = -j, inverse +j
template <class T>
__device__ __forceinline__ void dft4(cx<T>& a, cx<T>& b, cx<T>& c, cx<T>& d, bool inverse) {
  const cx<T> apc = a + c, amc = a - c, bpd = b + d, jbmd = mul_j(b - d);
  a = apc + bpd;
  c = apc - bpd;
  const cx<T> y1 = inverse ? amc + jbmd : amc - jbmd;
  const cx<T> y3 = inverse ? amc - jbmd : amc + jbmd;
  b = y1;
  d = y3;
}

// 16-point DFT of x[0..15] in place, r = 4 r1 + r2, u = u1 + 4 u2:
//   X[u1 + 4u2] = sum_r2 W_4^{r2 u2} W_16^{r2 u1} sum_r1 x[4r1 + r2] W_4^{r1 u1}.
// The result is left transposed: X[u] is in x[4 (u % 4) + u / 4]
// (dft16_out(u) gives that position), which saves a 16-element copy.
__host__ __device__ constexpr int dft16_out(int u) { return 4 * (u & 3) + (u >> 2); }

template <class T>
__device__ __forceinline__ void dft16(cx<T>* x, bool inverse) {
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173, h = (T)0.70710678118654752440;
  const T sg = inverse ? (T)1 : (T)-1;  // imaginary sign of the twiddles
#pragma unroll
  for (int r2 = 0; r2 < 4; ++r2) dft4(x[r2], x[4 + r2], x[8 + r2], x[12 + r2], inverse);
  // x[4 u1 + r2] now holds A[r2][u1]; twiddle by W_16^{r2 u1}
  // W_16^k = cos(k pi/8) + sg j sin(k pi/8)
  const cx<T> w1 = mk(c1, sg * s1), w2 = mk(h, sg * h), w3 = mk(s1, sg * c1);
  const cx<T> w6 = mk(-h, sg * h), w9 = mk(-c1, -sg * s1);
  x[5] = x[5] * w1;   // u1=1 r2=1
  x[6] = x[6] * w2;   // u1=1 r2=2
  x[7] = x[7] * w3;   // u1=1 r2=3
  x[9] = x[9] * w2;   // u1=2 r2=1
  x[10] = mk((T)0, sg) * x[10];  // W_16^4 = sg j
  x[11] = x[11] * w6;  // u1=2 r2=3
  x[13] = x[13] * w3;  // u1=3 r2=1
  x[14] = x[14] * w6;  // u1=3 r2=2
  x[15] = x[15] * w9;  // u1=3 r2=3
  // 4-point DFTs over r2 for each u1, in place: x[4u1 + u2] = X[u1 + 4u2]
#pragma unroll
  for (int u1 = 0; u1 < 4; ++u1) dft4(x[4 * u1], x[4 * u1 + 1], x[4 * u1 + 2], x[4 * u1 + 3], inverse);
}

// The FFT (M <= MMAX).  The first pass reads its input through gen(i) (no
// separate fill pass; zero padding costs nothing); later passes read sm at
// padded positions spad(i).  R16 selects radix-16 passes (else radix-4
// only).  epi(index, value) receives the outputs of the last pass.
template <int NT, int MMAX, bool R16, class T, class Gen, class Epi>
__device__ void smem_fft_run(Gen gen, cx<T>* sm, int log2M, bool inverse, const SmemTwiddles<T>& tw, Epi epi) {
  const int M = 1 << log2M;
  int n = M, s = 1, log2s = 0;
  // number of passes, to know which one is last
  int npass = 0;
  {
    int m = log2M;
    if (R16) { npass += m / 4; m %= 4; }
    npass += m / 2 + (m & 1);
  }
  int pass = 0;
  if (R16) {
    constexpr int MAXB = (MMAX / 16 + NT - 1) / NT;  // radix-16 butterflies per thread
    while (n >= 16) {
      ++pass;
      const bool last = pass == npass;
      const int n16 = n >> 4;
      const int M16 = M >> 4;
      cx<T> v[MAXB][16];
#pragma unroll
      for (int jb = 0; jb < MAXB; ++jb) {
        const int t = threadIdx.x + jb * NT;
        if (t < M16) {
          const int p = t >> log2s, q = t & (s - 1);
          if (pass == 1) {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[jb][r] = gen(q + s * (p + r * n16));
          } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[jb][r] = sm[spad(q + s * (p + r * n16))];
          }
        }
      }
      if (pass > 1) __syncthreads();
#pragma unroll
      for (int jb = 0; jb < MAXB; ++jb) {
        const int t = threadIdx.x + jb * NT;
        if (t < M16) {
          const int p = t >> log2s, q = t & (s - 1);
          dft16(v[jb], inverse);
          const int o = q + s * 16 * p;
          cx<T> w1 = tw.w(p * s);
          if (inverse) w1 = conj(w1);
          cx<T> w = w1;  // W^u, built by repeated products (about u ulp)
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            cx<T> z = v[jb][dft16_out(u)];
            if (u) {
              z = w * z;
              w = w * w1;
            }
            if (last) epi(o + u * s, z);
            else sm[spad(o + u * s)] = z;
          }
        }
      }
      __syncthreads();
      n >>= 4; s <<= 4; log2s += 4;
    }
  }
  while (n >= 4) {
    ++pass;
    const bool last = pass == npass;
    const int n4 = n >> 2;
    const int M4 = M >> 2;
    constexpr int MAXB = (MMAX / 4 + NT - 1) / NT;  // radix-4 butterflies per thread
    cx<T> v[MAXB][4];
#pragma unroll
    for (int jb = 0; jb < MAXB; ++jb) {
      const int t = threadIdx.x + jb * NT;
      if (t < M4) {
        const int p = t >> log2s, q = t & (s - 1);
        if (pass == 1) {
#pragma unroll
          for (int r = 0; r < 4; ++r) v[jb][r] = gen(q + s * (p + r * n4));
        } else {
#pragma unroll
          for (int r = 0; r < 4; ++r) v[jb][r] = sm[spad(q + s * (p + r * n4))];
        }
      }
    }
    if (pass > 1) __syncthreads();
#pragma unroll
    for (int jb = 0; jb < MAXB; ++jb) {
      const int t = threadIdx.x + jb * NT;
      if (t < M4) {
        const int p = t >> log2s, q = t & (s - 1);
        dft4(v[jb][0], v[jb][1], v[jb][2], v[jb][3], inverse);
        const int o = q + s * 4 * p;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          cx<T> z = v[jb][u];
          if (u) {
            cx<T> w = tw.w(p * u * s);
            if (inverse) w = conj(w);
            z = w * z;
          }
          if (last) epi(o + u * s, z);
          else sm[spad(o + u * s)] = z;
        }
      }
    }
    __syncthreads();
    n >>= 2; s <<= 2; log2s += 2;
  }
  if (n == 2) {
    const bool first = pass == 0;
    for (int q = threadIdx.x; q < (M >> 1); q += NT) {
      const cx<T> a = first ? gen(q) : sm[spad(q)], b = first ? gen(q + s) : sm[spad(q + s)];
      epi(q, a + b);
      epi(q + s, a - b);
    }
    __syncthreads();
  }
}

// shared memory (bytes) the FFT needs for length M: padded data + twiddles
__host__ __device__ inline size_t smem_fft_bytes(int log2M, size_t elem) {
  const size_t M = size_t(1) << log2M;
  const int lb = (log2M + 1) >> 1;
  return elem * (M + (M >> 4) + (size_t(1) << lb) + (size_t(1) << (log2M - lb)));
}

}  // namespace lse
