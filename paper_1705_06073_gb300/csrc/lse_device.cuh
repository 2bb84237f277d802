// lse_device.cuh -- block-level building blocks of the superfast evaluation
// (Sec. III of Hansen, Fleury, Rao, "Superfast Line Spectral Estimation").
//
// Every function here is executed by one whole thread block (NT threads) on
// data of one problem instance; arrays are generic pointers (shared or
// global memory).  Control flow inside is block-uniform and every function
// begins and ends at a __syncthreads(), so callers may chain them freely.
#pragma once

#include "lse_common.cuh"

namespace lse {

// ---------------------------------------------------------------------------
// Twiddle table: tw[k] = exp(-j 2 pi k / Mmax), k < Mmax.  W_M^k (M | Mmax)
// is tw[k * (Mmax / M)].
// ---------------------------------------------------------------------------
template <class T>
struct Twiddles {
  const cx<T>* tw;
  int log2max;
  __device__ __forceinline__ cx<T> w(int k, int log2M) const {  // exp(-j 2 pi k / M), 0 <= k < M
    return tw[(size_t)k << (log2max - log2M)];
  }
};

// ---------------------------------------------------------------------------
// Stockham radix-4 FFT (decimation in frequency, self-sorting).
//
// For length n and m = p + r n/4, k = 4k' + u:
//   X[4k'+u] = sum_p W_{n/4}^{pk'} [ W_n^{pu} sum_r x[p + r n/4] W_4^{ru} ],
// so each level does n/4 four-point DFTs, twiddles by W_n^{pu} and hands four
// interleaved length-n/4 problems to the next level (stride s grows by 4).
// A radix-2 level closes odd powers of two.  The first level reads its input
// through `gen(i)` (so zero padding, weights and pointwise products cost no
// extra pass); the levels alternate between `tmp` and `dst` so that the last
// one writes `dst`.  `gen` must not read `dst` or `tmp`.  inverse = true gives
// the unscaled inverse transform (sum x[m] W^{-mk}).
// ---------------------------------------------------------------------------
template <int NT, class T, class Gen>
__device__ void block_fft(Gen gen, cx<T>* dst, cx<T>* tmp, int log2M, bool inverse, const Twiddles<T>& tw) {
  const int M = 1 << log2M;
  const int npass = (log2M >> 1) + (log2M & 1);
  int pass = 0;
  const cx<T>* in = nullptr;
  int n = M, s = 1, log2s = 0;
  while (n >= 4) {
    ++pass;
    cx<T>* out = ((npass - pass) & 1) ? tmp : dst;
    const int n4 = n >> 2;
    for (int t = threadIdx.x; t < (M >> 2); t += NT) {
      const int p = t >> log2s, q = t & (s - 1);
      cx<T> a, b, c, d;
      if (pass == 1) {
        a = gen(q + s * p); b = gen(q + s * (p + n4)); c = gen(q + s * (p + 2 * n4)); d = gen(q + s * (p + 3 * n4));
      } else {
        a = in[q + s * p]; b = in[q + s * (p + n4)]; c = in[q + s * (p + 2 * n4)]; d = in[q + s * (p + 3 * n4)];
      }
      const cx<T> apc = a + c, amc = a - c, bpd = b + d, jbmd = mul_j(b - d);
      cx<T> y1 = inverse ? amc + jbmd : amc - jbmd;
      cx<T> y3 = inverse ? amc - jbmd : amc + jbmd;
      cx<T> y2 = apc - bpd;
      cx<T> w1 = tw.w(p * s, log2M), w2 = tw.w(2 * p * s, log2M), w3 = tw.w(3 * p * s, log2M);
      if (inverse) { w1 = conj(w1); w2 = conj(w2); w3 = conj(w3); }
      out[q + s * (4 * p + 0)] = apc + bpd;
      out[q + s * (4 * p + 1)] = w1 * y1;
      out[q + s * (4 * p + 2)] = w2 * y2;
      out[q + s * (4 * p + 3)] = w3 * y3;
    }
    __syncthreads();
    in = out;
    n >>= 2; s <<= 2; log2s += 2;
  }
  if (n == 2) {
    ++pass;
    cx<T>* out = dst;  // the last pass always writes dst
    for (int q = threadIdx.x; q < (M >> 1); q += NT) {
      cx<T> a, b;
      if (pass == 1) { a = gen(q); b = gen(q + s); } else { a = in[q]; b = in[q + s]; }
      out[q] = a + b;
      out[q + s] = a - b;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// First column of C (Sec. III intro; C of eq. py):
//   c_m = beta [m = 0] + sum_k gamma_k exp(j 2 pi m theta_k),  m = 0..N-1.
// m is split as m = S h + l (S = 2^ceil(log2 sqrt N)); per component the
// shared tables gamma_k e^{j2pi l theta_k} and e^{j2pi S h theta_k} (exact
// phase reduction) turn every (m, k) term into one complex product.
// smem must hold KC*(S + H) complex doubles.
// ---------------------------------------------------------------------------
constexpr int kFirstColumnChunk = 8;

__host__ __device__ inline void first_column_split(int N, int& S, int& H) {
  int lg = ilog2((uint32_t)N);
  S = 1 << ((lg + 1) >> 1);
  H = (N + S - 1) / S;
}

template <int NT>
__device__ void block_first_column(c128* c, const double* theta, const double* gamma, int K, double beta, int N,
                                   c128* smem) {
  int S, H;
  first_column_split(N, S, H);
  const int KC = kFirstColumnChunk;
  c128* lo = smem;              // [KC][S]
  c128* hi = smem + KC * S;     // [KC][H]
  for (int m = threadIdx.x; m < N; m += NT) c[m] = mk(m == 0 ? beta : 0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += KC) {
    const int kc = min(KC, K - k0);
    __syncthreads();
    for (int i = threadIdx.x; i < kc * S; i += NT) {
      const int k = i / S, l = i - k * S;
      lo[k * S + l] = gamma[k0 + k] * unit_phase((double)l, theta[k0 + k], 1.0);
    }
    for (int i = threadIdx.x; i < kc * H; i += NT) {
      const int k = i / H, h = i - k * H;
      hi[k * H + h] = unit_phase((double)h * S, theta[k0 + k], 1.0);
    }
    __syncthreads();
    for (int m = threadIdx.x; m < N; m += NT) {
      const int h = m / S, l = m - h * S;
      c128 acc = c[m];
      for (int k = 0; k < kc; ++k) acc = acc + lo[k * S + l] * hi[k * H + h];
      c[m] = acc;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Levinson-Durbin recursion for the Hermitian positive definite Toeplitz C
// with first column c (the O(N^2) route to the Gohberg-Semencul generators,
// Sec. III intro).  Order n -> n+1:
//   e_n = sum_{i<n} a_i c_{n-i},  k = -e_n / delta_{n-1},
//   a_i <- a_i + k conj(a_{n-i})  (i = 0..n, a_n = 0 before),
//   delta_n = delta_{n-1} (1 - |k|^2).
// a solves C a = delta_{N-1} e_0, so the last column of C^{-1} normalised to
// end in 1 (eq. gohberg-semencul) is rho_n = conj(a_{N-1-n}); delta_n are the
// pivots of C = L B L^H and ln|C| = sum_n ln delta_n (Sec. III-A).
// The update and the next inner product are fused: the thread owning the pair
// (i, n-i) updates both entries and adds their terms of e_{n+1}, so every
// order costs one pass over a and two barriers.
// `red` needs NT complex doubles of shared memory.
// ---------------------------------------------------------------------------
struct LevShared {
  c128 k;        // current reflection coefficient
  float4 kdf;    // the same as a double-float pair (double-float recursion)
  double delta;  // current pivot
  double mant;   // ln|C| accumulated as mant * 2^expo
  double logdet; // ln|C| (double-float recursion: result for the whole block)
  int expo;
  int status;    // 0 ok, 1 non-positive / non-finite pivot
  int ctrl[2];   // cluster recursion: go / stop word of the last two barriers
};

struct LevResult {
  double delta_last;
  double logdet;
  int status;
};

template <int NT>
__device__ LevResult block_levinson(const c128* c, c128* a, int N, c128* red, LevShared* sh) {
  for (int i = threadIdx.x; i < N; i += NT) a[i] = mk(i == 0 ? 1.0 : 0.0, 0.0);
  if (threadIdx.x == 0) {
    const double d0 = c[0].re;
    sh->status = (d0 > 0.0 && isfinite(d0)) ? 0 : 1;
    sh->delta = d0;
    int ex;
    sh->mant = frexp(d0, &ex);
    sh->expo = ex;
    if (N > 1) sh->k = (-1.0 / d0) * c[1];
  }
  __syncthreads();
  for (int n = 1; n < N; ++n) {
    if (sh->status) break;
    const c128 k = sh->k;
    const bool more = (n + 1) < N;
    c128 part = zero<double>();
    for (int i = threadIdx.x; 2 * i <= n; i += NT) {
      const int j = n - i;
      const c128 ai = a[i], aj = a[j];
      const c128 ain = ai + k * conj(aj);
      a[i] = ain;
      if (j != i) {
        const c128 ajn = aj + k * conj(ai);
        a[j] = ajn;
        if (more) part = part + ajn * c[i + 1];
      }
      if (more) part = part + ain * c[n + 1 - i];
    }
    red[threadIdx.x] = part;
    __syncthreads();
    if (threadIdx.x < 32) {
      c128 e = zero<double>();
#pragma unroll
      for (int r = 0; r < NT / 32; ++r) e = e + red[threadIdx.x + 32 * r];
      e.re = warp_sum(e.re);
      e.im = warp_sum(e.im);
      if (threadIdx.x == 0) {
        const double dn = sh->delta * (1.0 - norm2(k));
        if (!(dn > 0.0) || !isfinite(dn) || !isfinite(e.re) || !isfinite(e.im)) {
          sh->status = 1;
        } else {
          sh->delta = dn;
          double m = sh->mant * dn;
          int ex;
          m = frexp(m, &ex);
          sh->mant = m;
          sh->expo += ex;
          if (more) sh->k = (-1.0 / dn) * e;
        }
      }
    }
    __syncthreads();
  }
  LevResult r;
  r.status = sh->status;
  r.delta_last = sh->delta;
  r.logdet = log(sh->mant) + sh->expo * 0.69314718055994530942;
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// x = C^{-1} y by eq. (gohberg-semencul) (Sec. III-A, III-B):
//   x = delta_{N-1}^{-1} (T1^H (T1 y) - T0 (T0^H y)),
// [T0]_{ik} = rho_{i-k-1}, [T1]_{ik} = rho_{N-1+i-k}.  Each triangular
// Toeplitz product is a linear convolution done with length-M2 FFTs
// (M2 >= 2N); with P = FFT(rho) and W = exp(-j 2 pi / M2) the kernels'
// transforms are W^{-(N-1)w} P (T1), W^{(N-1)w} conj(P) (T1^H),
// W^{-w} conj(P) (T0^H) and W^{w} P (T0).  The two inner products are
// truncated to length N before the outer ones.
// Yf = FFT_M2(y) is computed once per instance.  bufs: 5 arrays of M2.
// ---------------------------------------------------------------------------
template <int NT>
__device__ void block_gs_apply(const c128* rho, const c128* Yf, c128* x, int N, int log2M2, double delta_last,
                               c128* const* bufs, const Twiddles<double>& tw) {
  const int M2 = 1 << log2M2;
  const int msk = M2 - 1;
  const double inv = 1.0 / (double)M2;
  c128 *P = bufs[0], *B1 = bufs[1], *B2 = bufs[2], *B3 = bufs[3], *T = bufs[4];
  block_fft<NT, double>([=] __device__(int i) { return i < N ? rho[i] : zero<double>(); }, P, T, log2M2, false, tw);
  // u = T1 y
  block_fft<NT, double>([=] __device__(int w) { return Yf[w] * conj(tw.w((int)(((int64_t)(N - 1) * w) & msk), log2M2)) * P[w]; },
                        B1, T, log2M2, true, tw);
  block_fft<NT, double>([=] __device__(int i) { return i < N ? inv * B1[i] : zero<double>(); }, B2, T, log2M2, false, tw);
  // z = T0^H y
  block_fft<NT, double>([=] __device__(int w) { return Yf[w] * conj(tw.w(w, log2M2)) * conj(P[w]); }, B1, T, log2M2, true, tw);
  block_fft<NT, double>([=] __device__(int i) { return i < N ? inv * B1[i] : zero<double>(); }, B3, T, log2M2, false, tw);
  // x = (T1^H u - T0 z) / delta
  block_fft<NT, double>(
      [=] __device__(int w) {
        const c128 g1 = tw.w((int)(((int64_t)(N - 1) * w) & msk), log2M2) * conj(P[w]);
        const c128 g0 = tw.w(w, log2M2) * P[w];
        return g1 * B2[w] - g0 * B3[w];
      },
      B1, T, log2M2, true, tw);
  const double sc = inv / delta_last;
  for (int i = threadIdx.x; i < N; i += NT) x[i] = sc * B1[i];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Off-grid sums at the active frequencies (Sec. III-B, III-C).  With the
// centre c = (N-2)/2 and phases e^{-j 2 pi n theta_k}:
//   R_a = sum_n (n-c)^a rho_n e^{-j2pi n theta},  a = 0..3
//   X_a = sum_n (n-c)^a x_n  e^{-j2pi n theta},  a = 0..2   (x = C^{-1} y).
// Every quantity of eqs. (q)-(x) with the centred D_c = 2 pi diag(n - c)
// follows from these (see component_vectors); the derivatives of eq. (obj)
// do not depend on the centre.  One warp per component; phases rotate by
// e^{-j2pi 32 theta} and are re-anchored exactly every 16 steps.
// Output: sums[k*7 + j] = (R0,R1,R2,R3,X0,X1,X2)[j] for component k.
// ---------------------------------------------------------------------------
template <int NT, class T>
__device__ void block_active_sums(const cx<T>* rho, const cx<T>* x, const double* theta, int K, int N,
                                  cx<T>* sums) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double cen = 0.5 * (double)(N - 2);
  for (int k = warp; k < K; k += NT / 32) {
    const double th = theta[k];
    const c128 stp64 = unit_phase(32.0, th, -1.0);
    const cx<T> stp = cvt<T>(stp64);
    cx<T> acc[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) acc[j] = zero<T>();
    cx<T> e = zero<T>();
    int it = 0;
    for (int n = lane; n < N; n += 32, ++it) {
      if ((it & 15) == 0) e = cvt<T>(unit_phase((double)n, th, -1.0));
      const T w = (T)((double)n - cen);
      const cx<T> pr = rho[n] * e;
      const cx<T> px = x[n] * e;
      const T w2 = w * w;
      acc[0] = acc[0] + pr;
      acc[1] = acc[1] + w * pr;
      acc[2] = acc[2] + w2 * pr;
      acc[3] = acc[3] + (w2 * w) * pr;
      acc[4] = acc[4] + px;
      acc[5] = acc[5] + w * px;
      acc[6] = acc[6] + w2 * px;
      e = e * stp;
    }
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      acc[j].re = warp_sum(acc[j].re);
      acc[j].im = warp_sum(acc[j].im);
    }
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < 7; ++j) sums[k * 7 + j] = acc[j];
    }
  }
  __syncthreads();
}

// The vectors of eqs. (q)-(x) at one active component from its sums, in the
// centred frame D_c = 2 pi diag(n - c), c = (N-2)/2.  The quadratic forms
// follow from Appendix B: with i = p - q and p, q the row/column indices the
// weights c_s, c_t, c_v, c_x of the appendix become, after shifting both
// indices by c, polynomials whose coefficients do not depend on N:
//   s  = (1/d)        [R1 R0* + R0 R1*]
//   t  = (2pi/d)  1/2 [R2 R0* + R1 R0* + R0 R1* - R0 R2*]
//   v  = (4pi^2/d)    [(R3 R0* + R0 R3*)/3 + (R2 R0* - R0 R2*)/2 + (R1 R0* + R0 R1*)/6]
//   x  = (4pi^2/d)    [Re(R1 R2*) + Re(R1 R0*)/3 - Re(R3 R0*)/3]
// (products R_a R_b* stand for the bilinear sums over (q, p) of
// (q-c)^a (p-c)^b rho_q rho_p^* e^{j2pi(p-q)theta}), and
//   q = X0, r = 2pi X1, u = 4pi^2 X2.
// d = delta_{N-1}.  q is also the uncentred q of eq. (q) (alpha = gamma q).
struct CompVec {
  c128 q, r, u, t, v;
  double s, x;
};

template <class T>
__device__ __forceinline__ CompVec component_vectors(const cx<T>* sm, double inv_delta) {
  const c128 R0 = cvt<double>(sm[0]), R1 = cvt<double>(sm[1]), R2 = cvt<double>(sm[2]), R3 = cvt<double>(sm[3]);
  const c128 X0 = cvt<double>(sm[4]), X1 = cvt<double>(sm[5]), X2 = cvt<double>(sm[6]);
  const c128 r1r0 = R1 * conj(R0), r2r0 = R2 * conj(R0), r3r0 = R3 * conj(R0), r1r2 = R1 * conj(R2);
  CompVec o;
  o.s = 2.0 * r1r0.re * inv_delta;
  // R0 R1* = conj(r1r0), R0 R2* = conj(r2r0), R0 R3* = conj(r3r0)
  o.t = (kPi * inv_delta) * (r2r0 - conj(r2r0) + r1r0 + conj(r1r0));
  const double f = 4.0 * kPi * kPi * inv_delta;
  o.v = f * ((1.0 / 3.0) * (r3r0 + conj(r3r0)) + 0.5 * (r2r0 - conj(r2r0)) + (1.0 / 6.0) * (r1r0 + conj(r1r0)));
  o.x = f * (r1r2.re + r1r0.re / 3.0 - r3r0.re / 3.0);
  o.q = X0;
  o.r = kTwoPi * X1;
  o.u = (4.0 * kPi * kPi) * X2;
  return o;
}

// First and second partial derivatives of eq. (obj) in theta_k and gamma_k
// (eqs. derivative, derivative2).
struct Derivs {
  double gt, gg, ht, hg;
};
__device__ __forceinline__ Derivs objective_derivatives(const CompVec& c, double g) {
  Derivs d;
  const double aq2 = norm2(c.q), ar2 = norm2(c.r);
  const c128 qcr = conj(c.q) * c.r;
  d.gt = 2.0 * g * (c.t.im - qcr.im);
  d.gg = c.s - aq2;
  const c128 tt = c.t * c.t;
  const c128 trq = c.t * c.r * conj(c.q);
  const c128 uq = c.u * conj(c.q);
  const double inner = (c.x - c.v.re) + g * (tt.re - c.x * c.s) + g * (c.x * aq2 + c.s * ar2 - 2.0 * trq.re) + (uq.re - ar2);
  d.ht = 2.0 * g * inner;
  d.hg = 2.0 * c.s * aq2 - c.s * c.s;
  return d;
}

}  // namespace lse
