// lse_semifast.cuh -- device functions of the semifast evaluation of Sec. IV
// (Hansen, Fleury, Rao, "Superfast Line Spectral Estimation") for incomplete
// observations: instance b observes M samples y_m = z(n_m) of an N-sample
// signal (Phi a row selection), and at a state (theta, gamma, beta) of K
// components every quantity of the method follows from Woodbury's identity
// (eq. CfromSigma)
//   C^{-1} = I/beta - A Sigma A^H / beta^2,   Sigma^{-1} = A^H A/beta + Gamma^{-1},
// with A = Phi Psi(theta), through K x K matrices and one Cholesky
// factorisation Sigma^{-1} = L L^H:
//   ln|C| = M ln beta + sum ln gamma_k + 2 sum ln L_kk  (determinant lemma)
//   y^H C^{-1} y = (||y||^2 - ||L^{-1} h0||^2 / beta) / beta
//   q, r, u = (h_a - G_a Sigma h0 / beta) / beta,            a = 0, 1, 2
//   s, t, v = (diag G_a - diag(G_a Sigma G0) / beta) / beta, a = 0, 1, 2
//   x       = (diag G2 - diag(G1 Sigma G1^H) / beta) / beta
// with G_a = A_{D^a}^H A (eq. AhA; [G_a]_{ik} = w_a(theta_i - theta_k),
// w_a(phi) = sum_m (2 pi n_m)^a e^{-j 2 pi n_m phi}) and h_a = A_{D^a}^H y.
// The w_a and h_a are type-2 non-uniform FFT sums (lse_nufft.cuh): the mask
// and the zero-filled y, weighted by (2 pi n)^a, deconvolved and transformed
// once per instance (they do not depend on the state), then interpolated at
// the K^2 differences and the K frequencies.  On the grid theta_l = l/L
// (Sec. IV, evaluating q and s for all theta):
//   b_l[k] = [A^H A(theta_l)]_k = w_0(theta_k - l/L),
//   s(l) = M/beta - ||L^{-1} b_l||^2 / beta^2,
//   q(l) = (Y(l) - sum_k conj(b_l[k]) (Sigma h0)_k / beta) / beta,
// Y the length-L FFT of the zero-filled y: the O(L K^2) contraction of the
// method, one forward substitution per grid point.
//
// One thread block per instance.  The K x K algebra is FP64; the transforms,
// the interpolations and the grid contraction use the precision policy
// (Pol64, or PolDF: double-float on the FP32 pipes).
#pragma once

#include "lse_common.cuh"
#include "lse_device.cuh"
#include "lse_df64.cuh"
#include "lse_nufft.cuh"
#include "lse_schur.cuh"

namespace lse {

constexpr int kSNT = 256;  // threads per block of the semifast kernels

template <class Pol>
struct SemiReal;
template <>
struct SemiReal<PolDF> : NufftReal<PolDF> {
  __device__ __forceinline__ static f2 add(f2 a, f2 b) { return add_s(a, b); }
  __device__ __forceinline__ static f2 norm(cf2 v) { return add_s(mul_f(v.re, v.re), mul_f(v.im, v.im)); }
  __device__ __forceinline__ static double d(f2 a) { return to_d(a); }
  __device__ __forceinline__ static f2 zr() { return f2{0.f, 0.f}; }
};
template <>
struct SemiReal<Pol64> : NufftReal<Pol64> {
  __device__ __forceinline__ static double add(double a, double b) { return a + b; }
  __device__ __forceinline__ static double norm(c128 v) { return norm2(v); }
  __device__ __forceinline__ static double d(double a) { return a; }
  __device__ __forceinline__ static double zr() { return 0.0; }
};

template <class Pol>
__device__ inline Pol semi_pol(const Tables& t);
template <>
__device__ inline PolDF semi_pol<PolDF>(const Tables& t) { return PolDF{t.twdf, t.log2max}; }
template <>
__device__ inline Pol64 semi_pol<Pol64>(const Tables& t) { return Pol64{t.tw64, t.log2max}; }

// Workspace of one block for instances up to (Kmax, Nmax, Lmax).
struct SemiLayout {
  size_t G, Lc, Z, h, ystar, mask, F, fac64, facdf, Yh, B, total;
};

__host__ __device__ inline SemiLayout semi_layout(int Kmax, int Nmax, int Lmax) {
  SemiLayout S;
  const size_t M2 = (size_t)1 << ilog2(2u * (uint32_t)Nmax);
  const size_t K = (size_t)(Kmax > 0 ? Kmax : 1);
  size_t o = 0;
  auto put = [&](size_t bytes) { size_t r = o; o += (bytes + 255) & ~size_t(255); return r; };
  S.G = put(sizeof(c128) * 3 * K * K);
  S.Lc = put(sizeof(c128) * K * K);
  S.Z = put(sizeof(c128) * 3 * K * K);
  S.h = put(sizeof(c128) * 6 * K);  // h0, h1, h2, L^{-1} h0, Sigma h0, scratch
  S.ystar = put(sizeof(float4) * (size_t)Nmax);
  S.mask = put(sizeof(float) * (size_t)Nmax);
  S.F = put(sizeof(float4) * 2 * 6 * M2);
  S.fac64 = put(sizeof(double) * (size_t)Nmax);
  S.facdf = put(sizeof(float2) * (size_t)Nmax);
  S.Yh = put(sizeof(float4) * 2 * (size_t)Lmax);
  S.B = put(sizeof(float4) * K * (size_t)Lmax);
  S.total = o;
  return S;
}

// shared memory of the grid contraction: the factor L (K x K) in the policy's
// storage, Sigma h0 / beta and 1/L_kk; or the interpolation weights of one
// component (r weight sets of 16 taps and their first taps)
__host__ __device__ inline size_t semi_smem_bytes(int Kmax, int r_max) {
  const size_t K = (size_t)(Kmax > 0 ? Kmax : 1);
  const size_t a = sizeof(float4) * K * K + sizeof(float4) * K + sizeof(double) * K;
  const size_t b = sizeof(double) * (size_t)r_max * kNufftW + sizeof(int) * (size_t)r_max;
  return a > b ? a : b;
}

template <class Pol>
struct SemiEval {
  using T = typename Pol::T;
  using RR = SemiReal<Pol>;
  using R = typename RR::R;
  Pol P;
  int M, N, L, M2, log2M2, log2L, n0;
  double nbeta, inv_norm, yy;
  c128 *G, *Lc, *Z, *h;
  float4* ystar;
  float* mask;
  float4* F;
  double* fac64;
  float2* facdf;
  float4 *Yh, *Bm;
  char* smem;     // dynamic shared memory (semi_smem_bytes)
  double* red;    // kSNT / 32 doubles of shared memory
  int* bad;       // one shared int: 1 = Sigma^{-1} not positive definite, 2 = index out of range

  __device__ void carve(char* base, const SemiLayout& S) {
    G = (c128*)(base + S.G);
    Lc = (c128*)(base + S.Lc);
    Z = (c128*)(base + S.Z);
    h = (c128*)(base + S.h);
    ystar = (float4*)(base + S.ystar);
    mask = (float*)(base + S.mask);
    F = (float4*)(base + S.F);
    fac64 = (double*)(base + S.fac64);
    facdf = (float2*)(base + S.facdf);
    Yh = (float4*)(base + S.Yh);
    Bm = (float4*)(base + S.B);
  }

  // Per instance, independent of the state: the zero-filled y and the mask,
  // ||y||^2, the six non-uniform-FFT transforms and, when the grid is wanted,
  // Y = FFT_L(zero-filled y).
  __device__ void prepare(const float* yin, const int* obs, int M_, int N_, int L_, bool want_grid) {
    M = M_;
    N = N_;
    L = L_;
    log2M2 = ilog2(2u * (uint32_t)N);
    M2 = 1 << log2M2;
    log2L = ilog2((uint32_t)L);
    n0 = N / 2;
    if (threadIdx.x == 0) *bad = 0;
    for (int n = threadIdx.x; n < N; n += kSNT) {
      Pol::st(ystar + n, Pol::zero());
      mask[n] = 0.f;
    }
    __syncthreads();
    double part = 0.0;
    for (int m = threadIdx.x; m < M; m += kSNT) {
      const int n = obs[m];
      if (n < 0 || n >= N) {  // an index outside the signal: reported, never used
        *bad = 2;
        continue;
      }
      const c128 v = mk((double)yin[2 * m], (double)yin[2 * m + 1]);
      part += norm2(v);
      Pol::st(ystar + n, Pol::of(v));
      mask[n] = 1.f;
    }
    yy = block_sum<kSNT>(part, red);
    nufft_factors<kSNT>(N, M2, fac64, facdf);
    const int Nl = N, M2l = M2, n0l = n0;
    const float* maskl = mask;
    const float4* ysl = ystar;
    const double* f64l = fac64;
    const float2* fdfl = facdf;
    pol_fft<kSNT>(
        P, 6,
        [=] __device__(int j, int i) -> T {
          const int np = i < (M2l >> 1) ? i : i - M2l;
          const int n = np + n0l;
          if (n < 0 || n >= Nl) return Pol::zero();
          const int e = j < 3 ? j : j - 3;
          R f = RR::tab(f64l, fdfl, n);
          const R w = RR::of(kTwoPi * (double)n);
          for (int q = 0; q < e; ++q) f = RR::mulr(f, w);
          const T v = j < 3 ? (maskl[n] != 0.f ? Pol::one() : Pol::zero()) : Pol::ld(ysl + n);
          return RR::scale(v, f);
        },
        F, F + 6 * (size_t)M2, log2M2, false);
    nbeta = nufft_beta(N, M2);
    inv_norm = 1.0 / ((double)kNufftW * cyl_bessel_i0(nbeta));
    if (want_grid)
      pol_fft<kSNT>(
          P, 1, [=] __device__(int, int i) -> T { return i < Nl ? Pol::ld(ysl + i) : Pol::zero(); }, Yh, Yh + L,
          log2L, false);
  }

  // S_j(phi) = sum_n f_j(n) e^{-j 2 pi n phi} of transform j, by the calling
  // warp (lane < 16: one kernel tap each); every lane returns the sum.
  __device__ c128 interp(int j, double phi) const {
    const int lane = threadIdx.x & 31;
    const double x = phi * (double)M2;
    const int m0 = (int)floor(x - 0.5 * kNufftW) + 1;
    const int l = lane & (kNufftW - 1);
    const double t = x - (double)(m0 + l);
    const double q = 2.0 * t / (double)kNufftW;
    const double psi = cyl_bessel_i0(nbeta * sqrt(fmax(0.0, 1.0 - q * q))) * inv_norm;
    T v = lane < kNufftW ? RR::scale(Pol::ld(F + (size_t)j * M2 + ((m0 + l) & (M2 - 1))), RR::of(psi)) : Pol::zero();
#pragma unroll
    for (int o = kNufftW / 2; o > 0; o >>= 1) v = v + Pol::shfl_xor(v, o);
    return unit_phase((double)n0, phi, -1.0) * Pol::to_c128(v);
  }

  // G_a[i][k] = w_a(theta_i - theta_k) and h_a[k] = S_{3+a}(theta_k) (with
  // vectors = false only G0 and h0, all a trial evaluation needs)
  __device__ void gram(const double* th, int K, bool vectors) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int na = vectors ? 3 : 1;
    for (int p = warp; p < K * K; p += kSNT / 32) {
      const int i = p / K, k = p - i * K;
      double phi = th[i] - th[k];
      phi -= floor(phi);
      for (int a = 0; a < na; ++a) {
        const c128 v = interp(a, phi);
        if (lane == 0) G[(size_t)a * K * K + p] = v;
      }
    }
    for (int k = warp; k < K; k += kSNT / 32)
      for (int a = 0; a < na; ++a) {
        const c128 v = interp(3 + a, th[k]);
        if (lane == 0) h[a * K + k] = v;
      }
    __syncthreads();
  }

  // Sigma^{-1} = G0 / beta + Gamma^{-1} = L L^H (FP64, column by column), then
  // w = L^{-1} h0 and Sigma h0 = L^{-H} w.  Sets *bad = 1 if a pivot is not
  // positive and finite.
  __device__ void factor(const double* ga, int K, double beta) {
    const double ib = 1.0 / beta;
    for (int j = 0; j < K; ++j) {
      if (threadIdx.x == 0) {
        double dj = G[(size_t)j * K + j].re * ib + 1.0 / ga[j];
        for (int p = 0; p < j; ++p) dj -= norm2(Lc[(size_t)j * K + p]);
        if ((!(dj > 0.0) || !isfinite(dj)) && *bad == 0) *bad = 1;
        Lc[(size_t)j * K + j] = mk(sqrt(fmax(dj, 1e-300)), 0.0);
      }
      __syncthreads();
      const double ljj = Lc[(size_t)j * K + j].re;
      for (int i = j + 1 + threadIdx.x; i < K; i += kSNT) {
        c128 v = ib * G[(size_t)i * K + j];
        for (int p = 0; p < j; ++p) v = v - Lc[(size_t)i * K + p] * conj(Lc[(size_t)j * K + p]);
        Lc[(size_t)i * K + j] = (1.0 / ljj) * v;
      }
      __syncthreads();
    }
    c128* w0 = h + 3 * K;
    c128* Sh = h + 4 * K;
    if (threadIdx.x == 0) {
      for (int i = 0; i < K; ++i) {
        c128 v = h[i];
        for (int p = 0; p < i; ++p) v = v - Lc[(size_t)i * K + p] * w0[p];
        w0[i] = (1.0 / Lc[(size_t)i * K + i].re) * v;
      }
      for (int i = K - 1; i >= 0; --i) {
        c128 v = w0[i];
        for (int p = i + 1; p < K; ++p) v = v - conj(Lc[(size_t)p * K + i]) * Sh[p];
        Sh[i] = (1.0 / Lc[(size_t)i * K + i].re) * v;
      }
    }
    __syncthreads();
  }

  // ln|C| and y^H C^{-1} y (after factor); every thread gets them
  __device__ void scalars(const double* ga, int K, double beta, double& logdet, double& yCy) {
    const double ib = 1.0 / beta;
    const c128* w0 = h + 3 * K;
    double pl = 0.0, pw = 0.0;
    for (int k = threadIdx.x; k < K; k += kSNT) {
      pl += log(ga[k]) + 2.0 * log(Lc[(size_t)k * K + k].re);
      pw += norm2(w0[k]);
    }
    pl = block_sum<kSNT>(pl, red);
    pw = block_sum<kSNT>(pw, red);
    logdet = (double)M * log(beta) + pl;
    yCy = ib * (yy - ib * pw);
  }

  // ||C^{-1} y||^2 = (||y||^2 - 2 Re(h0^H Sigma h0)/beta + (Sigma h0)^H G0 (Sigma h0)/beta^2)/beta^2
  // (C^{-1} y = (y - A Sigma h0 / beta)/beta); every thread gets it
  __device__ double residual_norm2(int K, double beta) {
    const double ib = 1.0 / beta;
    const c128* Sh = h + 4 * K;
    double p1 = 0.0, p2 = 0.0;
    for (int k = threadIdx.x; k < K; k += kSNT) {
      p1 += (conj(h[k]) * Sh[k]).re;
      c128 g = mk(0.0, 0.0);
      for (int p = 0; p < K; ++p) g = g + G[(size_t)k * K + p] * Sh[p];
      p2 += (conj(Sh[k]) * g).re;
    }
    p1 = block_sum<kSNT>(p1, red);
    p2 = block_sum<kSNT>(p2, red);
    return ib * ib * (yy - 2.0 * ib * p1 + ib * ib * p2);
  }

  // eqs. (q)-(x) at the K components into vo[7k + j] (q, r, u, s, t, v, x;
  // s and x real): per column k, z0 = L^{-1} G0 e_k, z1 = L^{-1} G1^H e_k,
  // z2 = L^{-1} G2^H e_k (thread k)
  __device__ void vectors(int K, double beta, c128* vo) {
    const double ib = 1.0 / beta;
    const c128* Sh = h + 4 * K;
    for (int k = threadIdx.x; k < K; k += kSNT) {
      c128* z0 = Z + (size_t)k * K;
      c128* z1 = Z + (size_t)K * K + (size_t)k * K;
      c128* z2 = Z + 2 * (size_t)K * K + (size_t)k * K;
      double n00 = 0.0, n11 = 0.0;
      c128 d10 = mk(0.0, 0.0), d20 = mk(0.0, 0.0);
      for (int i = 0; i < K; ++i) {
        c128 a0 = G[(size_t)i * K + k];
        c128 a1 = conj(G[(size_t)K * K + (size_t)k * K + i]);
        c128 a2 = conj(G[2 * (size_t)K * K + (size_t)k * K + i]);
        for (int p = 0; p < i; ++p) {
          const c128 l = Lc[(size_t)i * K + p];
          a0 = a0 - l * z0[p];
          a1 = a1 - l * z1[p];
          a2 = a2 - l * z2[p];
        }
        const double il = 1.0 / Lc[(size_t)i * K + i].re;
        z0[i] = il * a0;
        z1[i] = il * a1;
        z2[i] = il * a2;
        n00 += norm2(z0[i]);
        n11 += norm2(z1[i]);
        d10 = d10 + conj(z1[i]) * z0[i];
        d20 = d20 + conj(z2[i]) * z0[i];
      }
      c128 gs[3] = {mk(0.0, 0.0), mk(0.0, 0.0), mk(0.0, 0.0)};
      for (int p = 0; p < K; ++p)
        for (int a = 0; a < 3; ++a) gs[a] = gs[a] + G[(size_t)a * K * K + (size_t)k * K + p] * Sh[p];
      const c128 g0 = G[(size_t)k * K + k], g1 = G[(size_t)K * K + (size_t)k * K + k],
                 g2 = G[2 * (size_t)K * K + (size_t)k * K + k];
      vo[7 * k + 0] = ib * (h[k] - ib * gs[0]);
      vo[7 * k + 1] = ib * (h[K + k] - ib * gs[1]);
      vo[7 * k + 2] = ib * (h[2 * K + k] - ib * gs[2]);
      vo[7 * k + 3] = mk(ib * (g0.re - ib * n00), 0.0);
      vo[7 * k + 4] = ib * (g1 - ib * d10);
      vo[7 * k + 5] = ib * (g2 - ib * d20);
      vo[7 * k + 6] = mk(ib * (g2.re - ib * n11), 0.0);
    }
    __syncthreads();
  }

  // The grid: out(l, s, q) for every l < L (each l by one thread).
  template <class Out>
  __device__ void grid(const double* th, int K, double beta, Out out) {
    const double ib = 1.0 / beta;
    const int r = L / M2;  // L >= M2, both powers of two
    const c128* Sh = h + 4 * K;
    // B[k][l] = w_0(theta_k - l/L): for l = r a + c the taps are m0_c - a + tap
    // with weights that depend on c only
    for (int k = 0; k < K; ++k) {
      double* wts = (double*)smem;
      int* m0s = (int*)(wts + r * kNufftW);
      __syncthreads();
      for (int e = threadIdx.x; e < r * kNufftW; e += kSNT) {
        const int c = e / kNufftW, tap = e - c * kNufftW;
        const double x = th[k] * (double)M2 - (double)c / (double)r;
        const int m0 = (int)floor(x - 0.5 * kNufftW) + 1;
        const double t = x - (double)(m0 + tap);
        const double q = 2.0 * t / (double)kNufftW;
        wts[e] = cyl_bessel_i0(nbeta * sqrt(fmax(0.0, 1.0 - q * q))) * inv_norm;
        if (tap == 0) m0s[c] = m0;
      }
      __syncthreads();
      const T pk = Pol::of(unit_phase((double)n0, th[k], -1.0));
      for (int l = threadIdx.x; l < L; l += kSNT) {
        const int a = l / r, c = l - a * r;
        const int mb = m0s[c] - a;
        T v = Pol::zero();
#pragma unroll 4
        for (int tap = 0; tap < kNufftW; ++tap)
          v = v + RR::scale(Pol::ld(F + ((mb + tap) & (M2 - 1))), RR::of(wts[c * kNufftW + tap]));
        // e^{+j 2 pi n0 l / L} from the twiddle table
        const T tl = conj(P.w((int)(((int64_t)n0 * l) & (L - 1)), log2L));
        Pol::st(Bm + (size_t)k * L + l, pk * tl * v);
      }
    }
    __syncthreads();
    float4* Ls = (float4*)smem;
    for (int e = threadIdx.x; e < K * K; e += kSNT) Pol::st(Ls + e, Pol::of(Lc[e]));
    T* shb = (T*)(Ls + K * K);  // 16-byte aligned
    R* il = (R*)(shb + K);
    for (int k = threadIdx.x; k < K; k += kSNT) {
      il[k] = RR::of(1.0 / Lc[(size_t)k * K + k].re);
      shb[k] = Pol::of(ib * Sh[k]);
    }
    __syncthreads();
    const double Mb = (double)M * ib, ib2 = ib * ib;
    for (int l = threadIdx.x; l < L; l += kSNT) {
      R nz = RR::zr();
      T qs = Pol::zero();
      for (int i = 0; i < K; ++i) {
        const T b = Pol::ld(Bm + (size_t)i * L + l);
        qs = qs + conj(b) * shb[i];
        T v = b;
        for (int p = 0; p < i; ++p) v = v - Pol::ld(Ls + (size_t)i * K + p) * Pol::ld(Bm + (size_t)p * L + l);
        v = RR::scale(v, il[i]);
        Pol::st(Bm + (size_t)i * L + l, v);
        nz = RR::add(nz, RR::norm(v));
      }
      out(l, Mb - ib2 * RR::d(nz), ib * Pol::to_c128(Pol::ld(Yh + l) - qs));
    }
    __syncthreads();
  }
};

}  // namespace lse
