// lse_nufft.cuh -- the off-grid sums at arbitrary frequencies (the active
// components' q, r, u and the generator sums behind s, t, v, x of Sec. III-B,
// III-C and App. B; the re-scored grid points) by a type-2 non-uniform FFT,
// the route the paper names for them (Sec. III-B footnote): O(N log N + K W)
// per set of sums instead of the O(N K) direct sums.
//
// For a sequence f_n, n = 0..N-1, the sum S(theta) = sum_n f_n e^{-j2pi n theta}
// is written with the centred modes n' = n - n0 (n0 = N/2):
//   S(theta) = e^{-j2pi n0 theta} sum_{n'} f_{n'+n0} e^{-j2pi n' theta}.
// With a kernel psi of width W/M (M >= 2N points, a power of two) and its
// Fourier transform psi^(nu) = int psi(u) e^{j2pi nu u} du,
//   sum_{n'} f e^{-j2pi n' theta} ~ (1/M) sum_m F(m) psi(theta - m/M),
//   F(m) = sum_{n'} (f_{n'+n0} / psi^(n')) e^{-j2pi n' m / M},
// the rectangle rule of the convolution of the deconvolved series with psi;
// its error is set by the aliases psi^(n' + pM)/psi^(n') (|n'| <= N/2,
// |n' + pM| >= M - N/2).  The kernel is Kaiser-Bessel in grid units
// t = u M:  psi(t) = I0(beta sqrt(1 - (2t/W)^2)), |t| <= W/2, whose transform
// has the closed form  W sinh(r)/r, r = sqrt(beta^2 - (pi W nu / M)^2)
// (Kaiser-Bessel window/transform pair, e.g. Jackson et al., IEEE TMI 10,
// 1991), with beta = pi sqrt(W^2 (sigma - 1/2)^2 / sigma^2 - 0.8),
// sigma = M / N (Beatty, Nishimura, Pauly, IEEE TMI 24, 2005).  W = 16 and
// sigma >= 2 keep the approximation error near 1e-14 of sum |f_n|, the level
// of the FFT's own rounding.
//
// Scaling: the deconvolution factors are stored as c_n = I0(beta) r/sinh(r)
// (order one) and the interpolation weights as psi(t) / (W I0(beta)), so that
// S = e^{-j2pi n0 theta} sum_m DFT_M(f c)(m) psi(t_m)/(W I0(beta)) with no
// factor of M (the 1/M of the rectangle rule cancels the M of psi^).
//
// The arithmetic is the Schur recursion's policy (PolDF or Pol64): the FFTs
// are pol_fft's batched transforms.
#pragma once

#include "lse_common.cuh"
#include "lse_df64.cuh"
#include "lse_schur.cuh"

namespace lse {

constexpr int kNufftW = 16;  // kernel width in grid points

__host__ __device__ inline double nufft_beta(int N, int M) {
  const double sg = (double)M / (double)N;
  const double W = (double)kNufftW;
  return kPi * sqrt(W * W * (sg - 0.5) * (sg - 0.5) / (sg * sg) - 0.8);
}

// deconvolution factors c_n (n = 0..N-1, mode n' = n - N/2) in FP64 and as
// double-float pairs; every thread of the block calls it
template <int NT>
__device__ void nufft_factors(int N, int M, double* c64, float2* cdf) {
  const double beta = nufft_beta(N, M);
  const double i0b = cyl_bessel_i0(beta);
  const int n0 = N / 2;
  for (int n = threadIdx.x; n < N; n += NT) {
    const double a = kPi * (double)kNufftW * (double)(n - n0) / (double)M;
    const double r = sqrt(beta * beta - a * a);  // > 0: |a| <= pi W / 4 < beta
    const double c = i0b * r / sinh(r);
    c64[n] = c;
    const f2 d = to_f2(c);
    cdf[n] = make_float2(d.h, d.l);
  }
  __syncthreads();
}

template <class Pol>
struct NufftReal;
template <>
struct NufftReal<PolDF> {
  using R = f2;
  __device__ __forceinline__ static R of(double d) { return to_f2(d); }
  __device__ __forceinline__ static R tab(const double*, const float2* t, int n) { return f2{t[n].x, t[n].y}; }
  __device__ __forceinline__ static R mulr(R a, R b) { return mul(a, b); }
  __device__ __forceinline__ static R exact(float w) { return f2{w, 0.f}; }
  __device__ __forceinline__ static cf2 scale(cf2 v, R r) { return cf2{mul_f(v.re, r), mul_f(v.im, r)}; }
};
template <>
struct NufftReal<Pol64> {
  using R = double;
  __device__ __forceinline__ static R of(double d) { return d; }
  __device__ __forceinline__ static R tab(const double* t, const float2*, int n) { return t[n]; }
  __device__ __forceinline__ static R mulr(R a, R b) { return a * b; }
  __device__ __forceinline__ static R exact(float w) { return (double)w; }
  __device__ __forceinline__ static c128 scale(c128 v, R r) { return r * v; }
};

// The seven off-grid sums per frequency of lse_device.cuh's block_active_sums
// (R_a = sum (n-c)^a rho_n e^{-j2pi n theta}, a = 0..3, and for every
// snapshot X_a = sum (n-c)^a x_n e^{-j2pi n theta}, a = 0..2; c = (N-2)/2)
// for theta[0..K), written to sums_g[7k + j] of every snapshot g
// (sums_g = sums + g * stride; the R sums are repeated in every snapshot's
// slots).  rho and x0 + g xstride (snapshot g): the sequences in the
// policy's storage (float4: double float, or a c128); fac64/facdf:
// nufft_factors; buf: 2 nb M float4 of workspace, nb = 4 + 3G.  Every thread
// of the block calls it.
template <int NT, class Pol>
__device__ void block_sums_nufft(const Pol& Pl, const float4* rho, const float4* x0, size_t xstride, int G,
                                 const double* theta, int K, int N, int log2M, const double* fac64,
                                 const float2* facdf, float4* buf, c128* sums, size_t stride) {
  using T = typename Pol::T;
  using RR = NufftReal<Pol>;
  using R = typename RR::R;
  const int M = 1 << log2M;
  const int n0 = N / 2;
  const int nb = 4 + 3 * G;
  const float cen = 0.5f * (float)(N - 2);  // exact: N < 2^24
  float4* F = buf;
  float4* tmp = buf + (size_t)nb * M;
  // F_j = DFT_M of (weight_j(n) * c_n * v_j(n)) at the centred modes
  pol_fft<NT>(
      Pl, nb,
      [=] __device__(int j, int i) -> T {
        const int np = i < (M >> 1) ? i : i - M;
        const int n = np + n0;
        if (n < 0 || n >= N) return Pol::zero();
        int a;
        const float4* v;
        if (j < 4) {
          a = j;
          v = rho;
        } else {
          const int g = (j - 4) / 3;
          a = (j - 4) - 3 * g;
          v = x0 + (size_t)g * xstride;
        }
        const R w = RR::exact((float)n - cen);
        R f = RR::tab(fac64, facdf, n);
        for (int e = 0; e < a; ++e) f = RR::mulr(f, w);
        return RR::scale(Pol::ld(v + n), f);
      },
      F, tmp, log2M, false);
  // interpolation: one warp per frequency, lane l < W holds kernel tap l
  const double beta = nufft_beta(N, M);
  const double inv_norm = 1.0 / ((double)kNufftW * cyl_bessel_i0(beta));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = warp; k < K; k += NT / 32) {
    const double th = theta[k];
    const double x = th * (double)M;  // exact: M a power of two
    const int m0 = (int)floor(x - 0.5 * kNufftW) + 1;
    const int l = lane & (kNufftW - 1);
    const double t = x - (double)(m0 + l);  // in (-W/2, W/2]
    const double q = 2.0 * t / (double)kNufftW;
    const double psi = cyl_bessel_i0(beta * sqrt(fmax(0.0, 1.0 - q * q))) * inv_norm;
    const R kw = RR::of(psi);
    const int m = (m0 + l) & (M - 1);
    const T ph = Pl.of(unit_phase((double)n0, th, -1.0));
    for (int j = 0; j < nb; ++j) {
      T v = lane < kNufftW ? RR::scale(Pol::ld(F + (size_t)j * M + m), kw) : Pol::zero();
#pragma unroll
      for (int o = kNufftW / 2; o > 0; o >>= 1) v = v + Pol::shfl_xor(v, o);
      if (lane == 0) {
        const c128 s = Pol::to_c128(ph * v);
        if (j < 4) {
          for (int g = 0; g < G; ++g) sums[(size_t)g * stride + 7 * (size_t)k + j] = s;
        } else {
          const int g = (j - 4) / 3;
          sums[(size_t)g * stride + 7 * (size_t)k + 4 + ((j - 4) - 3 * g)] = s;
        }
      }
    }
  }
  __syncthreads();
}

}  // namespace lse
