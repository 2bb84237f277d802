// lse_df64.cuh -- double-float arithmetic on the FP32 pipes and the
// Levinson-Durbin recursion carried out in it.
//
// GB300 executes FP64 at about 1/70 of its FP32 rate, and the O(N^2)
// Levinson recursion is the dominant cost of the method.  A double-float
// number is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// which carries a 48-bit significand.  Sums and products are formed with the
// error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and TwoProd
// via FMA (e.g. Ogita, Rump, Oishi, "Accurate sum and dot product", SIAM J.
// Sci. Comput. 26, 2005); the explicit _rn intrinsics keep the compiler from
// contracting or reassociating the operations these transformations rely on.
#pragma once

#include "lse_common.cuh"

namespace lse {

struct f2 {
  float h, l;
};

__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return f2{s, e};
}

// p + e = x * y up to the dropped x.l * y.l term (relative 2^-48)
__device__ __forceinline__ void prod_terms(f2 x, f2 y, float& p, float& e) {
  p = __fmul_rn(x.h, y.h);
  e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
}

__device__ __forceinline__ f2 neg(f2 x) { return f2{-x.h, -x.l}; }

// x + y1*z1 + y2*z2, renormalised
__device__ __forceinline__ f2 axpy2(f2 x, f2 y1, f2 z1, f2 y2, f2 z2) {
  float p1, e1, p2, e2;
  prod_terms(y1, z1, p1, e1);
  prod_terms(y2, z2, p2, e2);
  const f2 s = two_sum(x.h, p1);
  const f2 t = two_sum(s.h, p2);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(x.l, e1), __fadd_rn(e2, s.l)), t.l);
  return two_sum(t.h, lo);
}

// running sum S + E += x * y (E collects all rounding errors)
__device__ __forceinline__ void acc_prod(float& S, float& E, f2 x, f2 y) {
  float p, e;
  prod_terms(x, y, p, e);
  const f2 t = two_sum(S, p);
  S = t.h;
  E = __fadd_rn(E, __fadd_rn(t.l, e));
}

// (S1 + E1) + (S2 + E2)
__device__ __forceinline__ void acc_merge(float& S, float& E, float S2, float E2) {
  const f2 t = two_sum(S, S2);
  S = t.h;
  E = __fadd_rn(__fadd_rn(E, E2), t.l);
}

__device__ __forceinline__ f2 to_f2(double d) {
  const float h = (float)d;
  return f2{h, (float)(d - (double)h)};
}
__device__ __forceinline__ double to_d(f2 x) { return (double)x.h + (double)x.l; }

// complex double-float stored as float4 {re.h, re.l, im.h, im.l}
__device__ __forceinline__ float4 pack(f2 re, f2 im) { return make_float4(re.h, re.l, im.h, im.l); }
__device__ __forceinline__ f2 re_of(float4 v) { return f2{v.x, v.y}; }
__device__ __forceinline__ f2 im_of(float4 v) { return f2{v.z, v.w}; }

// double-float product x*y, renormalised
__device__ __forceinline__ f2 mul(f2 x, f2 y) {
  float p, e;
  prod_terms(x, y, p, e);
  return two_sum(p, e);
}
// x - y
__device__ __forceinline__ f2 sub(f2 x, f2 y) {
  const f2 s = two_sum(x.h, -y.h);
  return two_sum(s.h, __fadd_rn(__fsub_rn(x.l, y.l), s.l));
}
// 1 / y (one Newton correction after the FP32 reciprocal)
__device__ __forceinline__ f2 recip(f2 y) {
  const float r = __fdiv_rn(1.f, y.h);
  const f2 e = sub(f2{1.f, 0.f}, mul(y, f2{r, 0.f}));
  return two_sum(r, __fmul_rn(r, e.h));
}

// x / y (one correction step after the FP32 quotient)
__device__ __forceinline__ f2 div(f2 x, f2 y) {
  const float q1 = __fdiv_rn(x.h, y.h);
  const f2 r = sub(x, mul(f2{q1, 0.f}, y));
  const float q2 = __fdiv_rn(r.h, y.h);
  return two_sum(q1, q2);
}

// ---------------------------------------------------------------------------
// The Levinson-Durbin recursion of block_levinson (same orders, same fused
// update + next inner product per pair (i, n-i)), with the vectors, the
// reflection coefficient, the pivot and the running product of pivots all in
// double-float on the FP32 pipes.  The first column is scaled by 1/c_0 so that
// every value stays near unit magnitude; pivots and ln|C| are returned in the
// unscaled units.
//
// One barrier per order: every warp writes its partial inner product into a
// double-buffered slot, and after the barrier every warp reduces all slots and
// forms the next reflection coefficient itself (the same operations on the
// same data, so all warps agree exactly).  The inner product is split over
// four accumulators per thread to shorten dependency chains.
// c: FP64 first column, converted in place to double-float (same 16 bytes per
// element); a: output predictor in FP64.  red: 2*NT/32 float4 of shared memory.
// ---------------------------------------------------------------------------
template <int NT>
__device__ LevResult block_levinson_df(c128* c64, c128* a64, int N, float4* red, LevShared* sh) {
  constexpr int NW = NT / 32;
  float4* c = reinterpret_cast<float4*>(c64);
  float4* a = reinterpret_cast<float4*>(a64);
  const double c0 = c64[0].re;
  __syncthreads();
  const double inv_c0 = 1.0 / c0;
  for (int i = threadIdx.x; i < N; i += NT) {
    const c128 v = c64[i];
    c[i] = pack(to_f2(v.re * inv_c0), to_f2(v.im * inv_c0));
    a[i] = make_float4(i == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // per-thread copies of the scalar state (identical in every thread)
  f2 kr{0.f, 0.f}, ki{0.f, 0.f};
  if (N > 1) {
    const float4 c1 = c[1];
    kr = neg(re_of(c1));
    ki = neg(im_of(c1));
  }
  f2 delta{1.f, 0.f}, mant{1.f, 0.f};
  int expo = 0;
  int bad = !(c0 > 0.0 && isfinite(c0));
  for (int n = 1; n < N && !bad; ++n) {
    const bool more = (n + 1) < N;
    // pivot of this order, delta_n = delta_{n-1} (1 - |k_n|^2), and its
    // reciprocal: they need only k_n, so they are issued before the pair loop
    // and their latency hides behind it
    float p1, q1, p2, q2;
    prod_terms(kr, kr, p1, q1);
    prod_terms(ki, ki, p2, q2);
    const f2 k2a = two_sum(p1, p2);
    const f2 k2 = two_sum(k2a.h, __fadd_rn(__fadd_rn(q1, q2), k2a.l));
    const f2 dn = mul(delta, sub(f2{1.f, 0.f}, k2));
    const f2 inv_dn = recip(dn);
    float S0 = 0.f, E0 = 0.f, S1 = 0.f, E1 = 0.f, S2 = 0.f, E2 = 0.f, S3 = 0.f, E3 = 0.f;
    for (int i = threadIdx.x; 2 * i <= n; i += NT) {
      const int j = n - i;
      const float4 ai = a[i], aj = a[j];
      const f2 air = re_of(ai), aii = im_of(ai), ajr = re_of(aj), aji = im_of(aj);
      // a_i + k conj(a_j)
      const f2 nir = axpy2(air, kr, ajr, ki, aji);
      const f2 nii = axpy2(aii, ki, ajr, neg(kr), aji);
      a[i] = pack(nir, nii);
      if (more) {
        const float4 cc = c[n + 1 - i];
        const f2 cr = re_of(cc), ci = im_of(cc);
        acc_prod(S0, E0, nir, cr);
        acc_prod(S1, E1, neg(nii), ci);
        acc_prod(S2, E2, nir, ci);
        acc_prod(S3, E3, nii, cr);
      }
      if (j != i) {
        const f2 njr = axpy2(ajr, kr, air, ki, aii);
        const f2 nji = axpy2(aji, ki, air, neg(kr), aii);
        a[j] = pack(njr, nji);
        if (more) {
          const float4 cc = c[i + 1];
          const f2 cr = re_of(cc), ci = im_of(cc);
          acc_prod(S0, E0, njr, cr);
          acc_prod(S1, E1, neg(nji), ci);
          acc_prod(S2, E2, njr, ci);
          acc_prod(S3, E3, nji, cr);
        }
      }
    }
    acc_merge(S0, E0, S1, E1);
    acc_merge(S2, E2, S3, E3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float sr = __shfl_xor_sync(0xffffffffu, S0, o), er = __shfl_xor_sync(0xffffffffu, E0, o);
      const float si = __shfl_xor_sync(0xffffffffu, S2, o), ei = __shfl_xor_sync(0xffffffffu, E2, o);
      acc_merge(S0, E0, sr, er);
      acc_merge(S2, E2, si, ei);
    }
    float4* slot = red + (n & 1) * NW;
    if (lane == 0) slot[warp] = make_float4(S0, E0, S2, E2);
    __syncthreads();
    // every warp: total of all partials (butterfly: all lanes end with it)
    const float4 v = lane < NW ? slot[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    float s0 = v.x, e0 = v.y, s1 = v.z, e1 = v.w;
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) {
      const float a0 = __shfl_xor_sync(0xffffffffu, s0, o), b0 = __shfl_xor_sync(0xffffffffu, e0, o);
      const float a1 = __shfl_xor_sync(0xffffffffu, s1, o), b1 = __shfl_xor_sync(0xffffffffu, e1, o);
      acc_merge(s0, e0, a0, b0);
      acc_merge(s1, e1, a1, b1);
    }
    // lanes < NW now hold the total; give every lane lane 0's copy so that all
    // threads of the block continue from bit-identical scalars (the loop exit
    // below must be block-uniform)
    s0 = __shfl_sync(0xffffffffu, s0, 0);
    e0 = __shfl_sync(0xffffffffu, e0, 0);
    s1 = __shfl_sync(0xffffffffu, s1, 0);
    e1 = __shfl_sync(0xffffffffu, e1, 0);
    if (!(dn.h > 0.f) || !isfinite(dn.h) || !isfinite(s0) || !isfinite(s1)) {
      bad = 1;
      break;
    }
    delta = dn;
    // running product of the pivots, kept in [0.5, 1) with a separate exponent
    const f2 m = mul(mant, dn);
    int ex;
    const float mh = frexpf(m.h, &ex);
    mant = f2{mh, ldexpf(m.l, -ex)};
    expo += ex;
    if (more) {
      const f2 er = two_sum(s0, e0), ei = two_sum(s1, e1);
      kr = neg(mul(er, inv_dn));
      ki = neg(mul(ei, inv_dn));
    }
  }
  LevResult r;
  r.status = bad;
  r.delta_last = to_d(delta) * c0;
  r.logdet = log(to_d(mant)) + expo * 0.69314718055994530942 + (double)N * log(c0);
  __syncthreads();
  // back to FP64 in place
  for (int i = threadIdx.x; i < N; i += NT) {
    const float4 v = a[i];
    a64[i] = mk(to_d(re_of(v)), to_d(im_of(v)));
  }
  __syncthreads();
  (void)sh;
  return r;
}

// ---------------------------------------------------------------------------
// Off-grid sums of block_active_sums (R_0..R_3 from rho, X_0..X_2 from x with
// the centred weights (n - c)^a, phases e^{-j2pi n theta_k}) in double-float
// on the FP32 pipes.  rho_df, x_df: the FP64 vectors converted once per
// evaluation (float4 {re.h, re.l, im.h, im.l}).  One warp per component;
// lane l visits n = l + 32 j with the phase advanced by e^{-j2pi 32 theta}
// and restarted every 64 steps from e^{-j2pi l theta} (e^{-j2pi 2048 theta})^i,
// all three phase factors formed once per component in FP64.  Output in FP64,
// same layout as block_active_sums.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cmul_df(f2 ar, f2 ai, f2 br, f2 bi, f2& cr, f2& ci) {
  cr = axpy2(f2{0.f, 0.f}, ar, br, neg(ai), bi);
  ci = axpy2(f2{0.f, 0.f}, ar, bi, ai, br);
}

template <int NT>
__device__ void block_active_sums_df(const float4* rho_df, const float4* x_df, const double* theta, int K, int N,
                                     c128* sums) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float cen = 0.5f * (float)(N - 2);  // exact: N < 2^24
  for (int k = warp; k < K; k += NT / 32) {
    const double th = theta[k];
    const c128 st64 = unit_phase(32.0, th, -1.0);
    const c128 big64 = unit_phase(2048.0, th, -1.0);
    const c128 e064 = unit_phase((double)lane, th, -1.0);
    const f2 sr = to_f2(st64.re), si = to_f2(st64.im);
    const f2 br = to_f2(big64.re), bi = to_f2(big64.im);
    f2 ar = to_f2(e064.re), ai = to_f2(e064.im);  // anchor e^{-j2pi (l + 2048 i) theta}
    f2 er = ar, ei = ai;
    float S[14], E[14];
#pragma unroll
    for (int j = 0; j < 14; ++j) { S[j] = 0.f; E[j] = 0.f; }
    int it = 0;
    for (int n = lane; n < N; n += 32, ++it) {
      if (it && (it & 63) == 0) {  // next anchor
        f2 nr, ni;
        cmul_df(ar, ai, br, bi, nr, ni);
        ar = nr; ai = ni;
        er = ar; ei = ai;
      }
      const float4 rv = rho_df[n], xv = x_df[n];
      f2 pr, pi, qr, qi;
      cmul_df(re_of(rv), im_of(rv), er, ei, pr, pi);  // rho_n e
      cmul_df(re_of(xv), im_of(xv), er, ei, qr, qi);  // x_n e
      const f2 w1{(float)n - cen, 0.f};               // exact (half-integer at worst)
      float w2h, w2l;
      w2h = __fmul_rn(w1.h, w1.h);
      w2l = __fmaf_rn(w1.h, w1.h, -w2h);
      const f2 w2{w2h, w2l};
      const f2 w3 = mul(w2, w1);
      acc_merge(S[0], E[0], pr.h, pr.l);
      acc_merge(S[1], E[1], pi.h, pi.l);
      acc_prod(S[2], E[2], pr, w1);
      acc_prod(S[3], E[3], pi, w1);
      acc_prod(S[4], E[4], pr, w2);
      acc_prod(S[5], E[5], pi, w2);
      acc_prod(S[6], E[6], pr, w3);
      acc_prod(S[7], E[7], pi, w3);
      acc_merge(S[8], E[8], qr.h, qr.l);
      acc_merge(S[9], E[9], qi.h, qi.l);
      acc_prod(S[10], E[10], qr, w1);
      acc_prod(S[11], E[11], qi, w1);
      acc_prod(S[12], E[12], qr, w2);
      acc_prod(S[13], E[13], qi, w2);
      f2 nr, ni;
      cmul_df(er, ei, sr, si, nr, ni);
      er = nr; ei = ni;
    }
#pragma unroll
    for (int j = 0; j < 14; ++j) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, S[j], o), e2 = __shfl_xor_sync(0xffffffffu, E[j], o);
        acc_merge(S[j], E[j], s2, e2);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < 7; ++j)
        sums[k * 7 + j] = mk((double)S[2 * j] + (double)E[2 * j], (double)S[2 * j + 1] + (double)E[2 * j + 1]);
    }
  }
  __syncthreads();
}

}  // namespace lse
