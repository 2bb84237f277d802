// lse_schur.cuh -- the Gohberg-Semencul generator of a Hermitian positive
// definite Toeplitz matrix by a divide-and-conquer ("superfast") Schur
// recursion: O(N log^2 N) work instead of the O(N^2) Levinson-Durbin
// recursion, which the paper names as the faster alternative for large N
// (Sec. III intro; Sec. III-E), organised for one thread block, or for a
// pair of blocks in a thread-block cluster sharing the passes of the FFT
// stages kept in global memory (the "team" arguments below).
//
// Notation (the same as block_levinson).  C has first column c; the order-n
// predictor a^(n) (a_0 = 1) and its reversed conjugate b^(n)_i =
// conj(a^(n)_{n-i}) give the polynomials A_n(z), B_n(z), and one order is
//   [A_n; B_n] = [[1, k_n z], [conj(k_n), z]] [A_{n-1}; B_{n-1}],
//   k_n = -e_n / delta_{n-1},  delta_n = delta_{n-1} (1 - |k_n|^2).
// The Schur generators are the residual sequences U_n = A_n c and
// V_n = B_n c (polynomial times series, only non-negative lags of c are
// involved where they are used): U_n(n+1) = e_{n+1} and V_n(n) = delta_n, so
//   k_{n+1} = -U_n(n+1) / V_n(n),
//   U_{n+1}(i) = U_n(i) + k V_n(i-1),   V_{n+1}(i) = V_n(i-1) + conj(k) U_n(i).
// A run of d orders m+1..m+d is one 2x2 polynomial matrix
//   Theta = [[P, Q], [R, S]],  R_j = conj(Q_{d-j}), S_j = conj(P_{d-j})
// (so only P and Q are kept; deg P <= d-1, deg Q <= d, Q_0 = 0), and it maps
// the generators as it maps the predictors: U_{m+d} = P U_m + Q V_m,
// V_{m+d} = R U_m + S V_m.  The orders of a run need only the windows
// U_m(m+1..m+d) and V_m(m..m+d-1).  A run is split in two halves; the first
// half's Theta, applied to the run's windows by FFT convolution, gives the
// second half's windows, and the run's Theta is the product of the halves'
// (FFT again).  Runs of at most 32 orders are done directly by one warp.
// At the top, A_{N-1} = P + Q, and the generator of eq. (gohberg-semencul)
// is rho_n = conj(a_{N-1-n}).
//
// The arithmetic is a policy: PolDF (double-float pairs on the FP32 pipes)
// or Pol64 (FP64).  Both store a complex number in 16 bytes (a float4
// {re.h, re.l, im.h, im.l}, or the two doubles of a c128).
#pragma once

#include "lse_common.cuh"
#include "lse_device.cuh"
#include "lse_df64.cuh"

namespace lse {

// ---------------------------------------------------------------- policies --
struct PolDF {
  using T = cf2;
  static constexpr int kDirectM = 64;  // runs up to this FFT length merge by direct sums
  const float4* tw;  // exp(-j 2 pi k / 2^log2max), double-float
  int log2max;
  __device__ __forceinline__ static T ld(const float4* p) { return ld_cf2(*p); }
  __device__ __forceinline__ static void st(float4* p, T v) { *p = st_cf2(v); }
  __device__ __forceinline__ T w(int k, int log2M) const { return ld_cf2(tw[(size_t)k << (log2max - log2M)]); }
  __device__ __forceinline__ static T zero() { return cf2_zero(); }
  __device__ __forceinline__ static T one() { return cf2{f2{1.f, 0.f}, f2{0.f, 0.f}}; }
  __device__ __forceinline__ static T scale2(float s, T v) { return lse::scale2(s, v); }  // s a power of two
  __device__ __forceinline__ static T of(c128 v) { return cf2_of(v); }
  __device__ __forceinline__ static c128 to_c128(T v) { return mk(to_d(v.re), to_d(v.im)); }
  __device__ __forceinline__ static double re_d(T v) { return to_d(v.re); }
  // -u / d for a real d (the real part of dv); ok: d > 0 and the result
  // finite (checked on the FP32 heads: no FP64 on this path)
  __device__ __forceinline__ static T neg_div_re(T u, T dv, bool& ok) {
    const float r0 = __frcp_rn(dv.re.h);
    const f2 e = sub(f2{1.f, 0.f}, mul(dv.re, f2{r0, 0.f}));
    const f2 r = fast_two_sum(r0, __fmul_rn(r0, e.h));  // one Newton step: 1/d to ~2^-46
    const T k = cf2{neg(mul_f(u.re, r)), neg(mul_f(u.im, r))};
    ok = dv.re.h > 0.f && isfinite(dv.re.h) && isfinite(k.re.h) && isfinite(k.im.h);
    return k;
  }
  __device__ __forceinline__ static T shfl(T v, int src) {
    return cf2{f2{__shfl_sync(0xffffffffu, v.re.h, src), __shfl_sync(0xffffffffu, v.re.l, src)},
               f2{__shfl_sync(0xffffffffu, v.im.h, src), __shfl_sync(0xffffffffu, v.im.l, src)}};
  }
  __device__ __forceinline__ static T shfl_up1(T v) {
    return cf2{f2{__shfl_up_sync(0xffffffffu, v.re.h, 1), __shfl_up_sync(0xffffffffu, v.re.l, 1)},
               f2{__shfl_up_sync(0xffffffffu, v.im.h, 1), __shfl_up_sync(0xffffffffu, v.im.l, 1)}};
  }
  __device__ __forceinline__ static T shfl_xor(T v, int m) {
    return cf2{f2{__shfl_xor_sync(0xffffffffu, v.re.h, m), __shfl_xor_sync(0xffffffffu, v.re.l, m)},
               f2{__shfl_xor_sync(0xffffffffu, v.im.h, m), __shfl_xor_sync(0xffffffffu, v.im.l, m)}};
  }
};

struct Pol64 {
  using T = c128;
  static constexpr int kDirectM = 0;  // FP64 multiply-adds are slow on GB300: always FFTs
  const c128* tw;
  int log2max;
  __device__ __forceinline__ static T ld(const float4* p) { return *reinterpret_cast<const c128*>(p); }
  __device__ __forceinline__ static void st(float4* p, T v) { *reinterpret_cast<c128*>(p) = v; }
  __device__ __forceinline__ T w(int k, int log2M) const { return tw[(size_t)k << (log2max - log2M)]; }
  __device__ __forceinline__ static T zero() { return mk(0.0, 0.0); }
  __device__ __forceinline__ static T one() { return mk(1.0, 0.0); }
  __device__ __forceinline__ static T scale2(float s, T v) { return (double)s * v; }
  __device__ __forceinline__ static T of(c128 v) { return v; }
  __device__ __forceinline__ static c128 to_c128(T v) { return v; }
  __device__ __forceinline__ static double re_d(T v) { return v.re; }
  __device__ __forceinline__ static T neg_div_re(T u, T dv, bool& ok) {
    const T k = (-1.0 / dv.re) * u;
    ok = dv.re > 0.0 && isfinite(dv.re) && isfinite(k.re) && isfinite(k.im);
    return k;
  }
  __device__ __forceinline__ static T shfl(T v, int src) {
    return mk(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
  }
  __device__ __forceinline__ static T shfl_up1(T v) {
    return mk(__shfl_up_sync(0xffffffffu, v.re, 1), __shfl_up_sync(0xffffffffu, v.im, 1));
  }
  __device__ __forceinline__ static T shfl_xor(T v, int m) {
    return mk(__shfl_xor_sync(0xffffffffu, v.re, m), __shfl_xor_sync(0xffffffffu, v.im, m));
  }
};

// ------------------------------------------------------------- teams -------
// A recursion can be shared by the blocks of a thread-block cluster (a team of
// csize blocks, this one of rank crank): the work of a step is split over the
// team's threads and its steps are separated by cluster barriers (release /
// acquire at cluster scope, so the global-memory stores of one block are seen
// by the other).  csize = 1: one block, block barriers.
__device__ __forceinline__ void team_sync(int csize) {
  if (csize > 1) cluster_barrier();
  else __syncthreads();
}
// a 32-bit store into the same shared-memory object of block `rank`
__device__ __forceinline__ void st_cluster_u32(const void* local, unsigned rank, unsigned v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr(local, rank)), "r"(v) : "memory");
}

// ------------------------------------------------------ batched block FFT --
// one radix-4 butterfly of a decimation-in-frequency Stockham pass (stride s,
// group p, offset q), twiddled and stored into out
template <class Pol>
__device__ __forceinline__ void pol_bfly4(const Pol& P, typename Pol::T a, typename Pol::T b, typename Pol::T c,
                                          typename Pol::T d, float4* out, int p, int q, int s, int log2M,
                                          bool inverse) {
  using T = typename Pol::T;
  const T apc = a + c, amc = a - c, bpd = b + d, jbmd = mul_j(b - d);
  const T y1 = inverse ? amc + jbmd : amc - jbmd;
  const T y3 = inverse ? amc - jbmd : amc + jbmd;
  const T y2 = apc - bpd;
  T w1 = P.w(p * s, log2M), w2 = P.w(2 * p * s, log2M), w3 = P.w(3 * p * s, log2M);
  if (inverse) { w1 = conj(w1); w2 = conj(w2); w3 = conj(w3); }
  Pol::st(out + q + s * (4 * p + 0), apc + bpd);
  Pol::st(out + q + s * (4 * p + 1), w1 * y1);
  Pol::st(out + q + s * (4 * p + 2), w2 * y2);
  Pol::st(out + q + s * (4 * p + 3), w3 * y3);
}

// nb independent length-M FFTs (radix-4 Stockham, decimation in frequency,
// radix-2 closing an odd power of two), every pass spread over the whole
// block: job j reads gen(j, i) in the first pass and ends in dst + j*M; the
// passes alternate between tmp + j*M and dst + j*M.  inverse: the unscaled
// inverse transform.  gen must not read dst or tmp.  A thread issues the
// loads of two butterflies before it computes either, so that in global
// memory (L2) their latencies overlap.  A team of csize blocks (rank crank)
// splits every pass (gen, dst and tmp then in global memory).
template <int NT, class Pol, class Gen>
__device__ __noinline__ void pol_fft(const Pol& P, int nb, Gen gen, float4* dst, float4* tmp, int log2M, bool inverse,
                                     int crank = 0, int csize = 1) {
  using T = typename Pol::T;
  constexpr int UN = 2;
  const int M = 1 << log2M;
  const int g0 = crank * NT + (int)threadIdx.x, S = csize * NT;  // this thread in the team, the team's threads
  const int npass = (log2M >> 1) + (log2M & 1);
  int pass = 0;
  const float4* in = nullptr;
  int n = M, s = 1, log2s = 0;
  while (n >= 4) {
    ++pass;
    float4* out = ((npass - pass) & 1) ? tmp : dst;
    const int n4 = n >> 2;
    const int lq = log2M - 2;
    const int total = nb << lq;
    if (pass == 1) {
      // the first pass reads through gen (which may do its own loads): one
      // butterfly at a time
      for (int t = g0; t < total; t += S) {
        const int j = t >> lq, tt = t & ((1 << lq) - 1);
        const int p = tt >> log2s, q = tt & (s - 1);
        const T a = gen(j, q + s * p), b = gen(j, q + s * (p + n4)), c = gen(j, q + s * (p + 2 * n4)),
                d = gen(j, q + s * (p + 3 * n4));
        pol_bfly4(P, a, b, c, d, out + (size_t)j * M, p, q, s, log2M, inverse);
      }
    } else {
      for (int t0 = g0; t0 < total; t0 += UN * S) {
        T a[UN], b[UN], c[UN], d[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
          const int t = t0 + u * S;
          if (t < total) {
            const int j = t >> lq, tt = t & ((1 << lq) - 1);
            const int p = tt >> log2s, q = tt & (s - 1);
            const float4* ij = in + (size_t)j * M;
            a[u] = Pol::ld(ij + q + s * p); b[u] = Pol::ld(ij + q + s * (p + n4));
            c[u] = Pol::ld(ij + q + s * (p + 2 * n4)); d[u] = Pol::ld(ij + q + s * (p + 3 * n4));
          }
        }
#pragma unroll
        for (int u = 0; u < UN; ++u) {
          const int t = t0 + u * S;
          if (t < total) {
            const int j = t >> lq, tt = t & ((1 << lq) - 1);
            const int p = tt >> log2s, q = tt & (s - 1);
            pol_bfly4(P, a[u], b[u], c[u], d[u], out + (size_t)j * M, p, q, s, log2M, inverse);
          }
        }
      }
    }
    team_sync(csize);
    in = out;
    n >>= 2; s <<= 2; log2s += 2;
  }
  if (n == 2) {
    ++pass;
    const int lh = log2M - 1;
    for (int t = g0; t < (nb << lh); t += S) {
      const int j = t >> lh, q = t & ((1 << lh) - 1);
      T a, b;
      if (pass == 1) {
        a = gen(j, q); b = gen(j, q + s);
      } else {
        const float4* ij = in + (size_t)j * M;
        a = Pol::ld(ij + q); b = Pol::ld(ij + q + s);
      }
      float4* oj = dst + (size_t)j * M;
      Pol::st(oj + q, a + b);
      Pol::st(oj + q + s, a - b);
    }
    team_sync(csize);
  }
}

// ------------------------------------------------------------- workspace --
constexpr int kSchurLeaf = 32;  // orders done directly by one warp (a run of at most 32)

__host__ __device__ inline int schur_top_m(int N) { return N > 2 ? (int)next_pow2((uint32_t)(N - 1)) : 1; }

// buffer of a run whose FFT length is M: 4 M transforms, M for the second
// half's windows, M + 16 for the halves' Theta.  Along the path of pending
// runs M strictly decreases (a half has at most ceil(d/2) orders), so one
// buffer per FFT length suffices: the buffer of length 2^l sits after those of
// every longer length.
__host__ __device__ inline size_t schur_level_elems(int M) { return 6 * (size_t)M + 16; }

// offset of the buffer for FFT length 2^l among the lengths 2^lo..2^hi
__host__ __device__ inline size_t schur_level_offset(int l, int hi) {
  size_t o = 0;
  for (int k = hi; k > l; --k) o += schur_level_elems(1 << k);
  return o;
}

// Runs whose FFT length is at most 2^lsm keep their buffers (and their FFT
// scratch) in shared memory: the small runs are many and latency-bound.  The
// caller picks lsm (8 or 9) from the shared memory it can spare.
constexpr int kSchurMinLog2M = 6;  // the shortest run that is not a leaf has 33 orders

__host__ __device__ inline size_t schur_smem_elems(int lsm) {
  return schur_level_offset(kSchurMinLog2M - 1, lsm) + 4 * ((size_t)1 << lsm) + 32;
}
__host__ __device__ inline size_t schur_smem_bytes(int lsm) { return 16 * schur_smem_elems(lsm); }

// largest lsm in [lo, hi] whose shared part fits in `bytes`, or 0
__host__ __device__ inline int schur_pick_lsm(size_t bytes) {
  for (int l = 9; l >= kSchurMinLog2M; --l)
    if (schur_smem_bytes(l) <= bytes) return l;
  return 0;
}

// FFT length of the refinement step: a power of two >= 2N
__host__ __device__ inline int schur_refine_m(int N) { return (int)next_pow2(2u * (uint32_t)N); }

__host__ __device__ inline size_t schur_workspace_elems(int Nmax) {
  const int M = schur_top_m(Nmax);
  size_t e = 2 * (size_t)Nmax + 2 * ((size_t)Nmax + 16) + 2 * (size_t)Nmax;  // root windows, root Theta, delta, k
  e += 4 * (size_t)M;                                                        // FFT scratch
  e += schur_level_offset(kSchurMinLog2M - 1, ilog2((uint32_t)M));           // every run length's buffer
  e += 8 * (size_t)schur_refine_m(Nmax);                                     // refinement step
  return e + 64;
}

struct SchurWork {
  float4* Uw;     // root windows: c(1..N-1), c(0..N-2) (scaled by 1/c_0)
  float4* Vw;
  float4* Pc;     // root Theta
  float4* Qc;
  float4* delta;  // delta_n / c_0, n = 0..N-2 (real part)
  float4* ks;     // k_{n+1}, n = 0..N-2
  float4* scratch;  // 4 M (global)
  float4* levels;   // buffers of runs with FFT length > 2^lsm (global)
  float4* slevels;  // buffers of runs with FFT length <= 2^lsm (shared)
  float4* sscratch; // 4 2^lsm (shared)
  float4* sk;       // 32 reflection coefficients of the current leaf (shared)
  float4* refine;   // 8 schur_refine_m(N) (global)
  int Mtop, lsm;
  int* bad;         // shared flag: a pivot <= 0 or not finite
};

__device__ inline SchurWork schur_carve(float4* base, int Nmax) {
  SchurWork w;
  w.Mtop = schur_top_m(Nmax);
  float4* p = base;
  w.Uw = p; p += Nmax;
  w.Vw = p; p += Nmax;
  w.Pc = p; p += Nmax + 16;
  w.Qc = p; p += Nmax + 16;
  w.delta = p; p += Nmax;
  w.ks = p; p += Nmax;
  w.scratch = p; p += 4 * (size_t)w.Mtop;
  w.levels = p; p += schur_level_offset(kSchurMinLog2M - 1, ilog2((uint32_t)w.Mtop));
  w.refine = p;
  w.slevels = w.sscratch = w.sk = nullptr;
  w.bad = nullptr;
  return w;
}

// the shared-memory part: smem holds schur_smem_bytes(lsm)
__device__ inline void schur_carve_smem(SchurWork& w, float4* smem, int lsm) {
  w.lsm = lsm;
  w.slevels = smem;
  w.sscratch = smem + schur_level_offset(kSchurMinLog2M - 1, lsm);
  w.sk = w.sscratch + 4 * ((size_t)1 << lsm);
}

// ---------------------------------------------------------------- leaves --
// d <= 32 orders m+1..m+d by warps 0-2 (lane t: window and coefficient index
// t).  Warp 0 holds U[t] = U_m(m+1+t), V[t] = V_m(m+t): per order j its lane
// j forms k and publishes it in W.sk, and then the generators are updated.
// Warp 1 updates P and R (P' = P + k z R, R' = conj(k) P + z R) and warp 2
// updates Q and S (Q' = Q + k z S, S' = conj(k) Q + z S), each on its own; one
// named barrier per order orders the three.  Q_d = k_{m+d} (the leading
// coefficient of S is 1).  Writes Pc[0..d], Qc[0..d], delta[m..m+d-1],
// ks[m..m+d-1].
template <class Pol>
__device__ void schur_leaf(const Pol& Pl, const SchurWork& W, int m, int d, const float4* Uw, const float4* Vw,
                           float4* Pc, float4* Qc) {
  using T = typename Pol::T;
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  if (warp > 2) return;
  if (warp == 0) {
    T U = t < d ? Pol::ld(Uw + t) : Pol::zero();
    T V = t < d ? Pol::ld(Vw + t) : Pol::zero();
    T kt = Pol::zero(), dt = Pol::zero();  // lane t's order: k_{m+t+1} and delta_{m+t}
    bool ok = true;
    for (int j = 0; j < d; ++j) {
      // every lane shuffles (full mask); lane 0 drops what it received
      const T Up = Pol::shfl_up1(U), Vp = Pol::shfl_up1(V);
      if (t == j) {
        bool okj;
        kt = Pol::neg_div_re(U, V, okj);
        dt = V;
        ok = okj;
        Pol::st(W.sk + j, kt);
      }
      asm volatile("bar.sync 2, 96;" ::: "memory");
      const T k = Pol::ld(W.sk + j);
      U = U + k * V;
      V = Vp + conj(k) * Up;
    }
    if (t < d) {
      Pol::st(W.delta + m + t, dt);
      Pol::st(W.ks + m + t, kt);
    }
    const bool bad = __any_sync(0xffffffffu, !ok);
    if (t == 0 && bad) *W.bad = 1;
    if (t == d - 1 || (d == 32 && t == 31)) {
      Pol::st(Qc + d, Pol::ld(W.sk + d - 1));  // Q_d = k_{m+d}
      Pol::st(Pc + d, Pol::zero());             // deg P <= d - 1
    }
  } else {
    // warp 1: X = P, Y = R; warp 2: X = Q, Y = S.  X' = X + k z Y, Y' = conj(k) X + z Y
    T X = (warp == 1 && t == 0) ? Pol::one() : Pol::zero();
    T Y = (warp == 2 && t == 0) ? Pol::one() : Pol::zero();
    for (int j = 0; j < d; ++j) {
      const T Yr = Pol::shfl_up1(Y);
      const T zY = t ? Yr : Pol::zero();
      asm volatile("bar.sync 2, 96;" ::: "memory");
      const T k = Pol::ld(W.sk + j);
      const T Xn = X + k * zY;
      Y = conj(k) * X + zY;
      X = Xn;
    }
    if (t < d) Pol::st((warp == 1 ? Pc : Qc) + t, X);
  }
}

// ------------------------------------------------------- direct sums ------
// out[o] = sum_{j < nterms} term(o, j) for o < nout, G consecutive threads
// per output (each summing every G-th term, then a butterfly over the group);
// store(o, value) receives each sum.  Used for the short runs, where direct
// convolution beats three latency-bound FFT passes.
template <int NT, int G, class Pol, class Term, class Store>
__device__ __forceinline__ void group_sums(int nout, int nterms, Term term, Store store) {
  using T = typename Pol::T;
  static_assert((G & (G - 1)) == 0 && G <= 32 && NT % G == 0, "groups within a warp");
  const int g = threadIdx.x & (G - 1);
  for (int base = 0; base < nout; base += NT / G) {  // uniform across the block
    const int o = base + (int)threadIdx.x / G;
    T acc = Pol::zero();
    if (o < nout)
      for (int j = g; j < nterms; j += G) acc = acc + term(o, j);
#pragma unroll
    for (int off = G >> 1; off > 0; off >>= 1) acc = acc + Pol::shfl_xor(acc, off);
    if (g == 0 && o < nout) store(o, acc);
  }
}

// ----------------------------------------------------------------- runs --
// The orders 1..d (d = N - 1) from the root windows, depth first: a run of d
// orders m+1..m+d has the windows Uw[t] = U_m(m+1+t), Vw[t] = V_m(m+t),
// t < d, and leaves its Theta in Pc, Qc [0..d].  A run longer than
// kSchurLeaf is done in three stages: (0) its first half (its windows are
// the prefixes of the run's); (1) the transforms of the first half's Theta
// and of the run's windows, and from them the second half's windows;
// (2) the second half's Theta transformed and multiplied into the run's.
// The stack of pending runs is the same in every thread (block-uniform
// control flow); the buffers of depth k sit at a fixed offset.
//
// A team of csize blocks (rank crank): every block walks the same stack; the
// FFT stages of runs whose buffers are in global memory are shared (a cluster
// barrier before and after, the passes split), and everything else (leaves,
// direct sums, runs in shared memory) is done by rank 0 alone, the others
// skipping it.  The results are those of one block, bit for bit.
constexpr int kSchurMaxDepth = 16;  // enough for N <= 2^20

struct SchurNode {
  int m, d, stage;
  const float4 *Uw, *Vw;
  float4 *Pc, *Qc;
};

template <int NT, class Pol>
__device__ __noinline__ void schur_solve(const Pol& Pl, const SchurWork& W, int d0, int crank = 0, int csize = 1) {
  using T = typename Pol::T;
  SchurNode st[kSchurMaxDepth];
  int top = 0;
  st[0] = SchurNode{0, d0, 0, W.Uw, W.Vw, W.Pc, W.Qc};
  const bool lead = crank == 0;
  while (top >= 0) {
    const SchurNode nd = st[top];
    const int m = nd.m, d = nd.d;
    if (d <= kSchurLeaf) {
      if (lead) {
        schur_leaf<Pol>(Pl, W, m, d, nd.Uw, nd.Vw, nd.Pc, nd.Qc);
        __syncthreads();
      }
      --top;
      continue;
    }
    const int d1 = d >> 1, d2 = d - d1;
    const int log2M = ilog2((uint32_t)d);
    const int M = 1 << log2M;
    const int msk = M - 1;
    const bool sm = log2M <= W.lsm;
    // the team shares the FFT stages of runs kept in global memory
    const bool team = csize > 1 && !sm && M > Pol::kDirectM;
    const int tr = team ? crank : 0, ts = team ? csize : 1;
    const int gt = tr * NT + (int)threadIdx.x, St = ts * NT;  // this thread in the team, the team's threads
    const bool work = team || lead;
    float4* lev = sm ? W.slevels + schur_level_offset(log2M, W.lsm)
                     : W.levels + schur_level_offset(log2M, ilog2((uint32_t)W.Mtop));
    float4* scr = sm ? W.sscratch : W.scratch;
    float4* F = lev;  // F0 = FFT(P1), F1 = FFT(Q1), F2, F3
    float4* Uh = lev + 4 * (size_t)M;
    float4* Vh = Uh + (M >> 1);
    float4* Pch = lev + 5 * (size_t)M;  // the halves' Theta (first, then second)
    float4* Qch = Pch + (M >> 1) + 8;
    const float inv = 1.0f / (float)M;  // a power of two: exact
    const Pol P2 = Pl;
    if (nd.stage == 0) {
      st[top].stage = 1;
      st[top + 1] = SchurNode{m, d1, 0, nd.Uw, nd.Vw, Pch, Qch};
      ++top;
      continue;
    }
    if (nd.stage == 1 && M <= Pol::kDirectM) {
      if (lead) {
      // the first half's Theta kept for stage 2 (the second half reuses Pch, Qch)
      for (int i = threadIdx.x; i <= d1; i += NT) {
        Pol::st(F + i, Pol::ld(Pch + i));
        Pol::st(F + M + i, Pol::ld(Qch + i));
      }
      const float4 *Uw = nd.Uw, *Vw = nd.Vw;
      // U_h(h+1+s) = sum_j P1_j Uw[d1+s-j] + Q1_j Vw[d1+1+s-j],
      // V_h(h+s)   = sum_j conj(Q1_{d1-j}) Uw[d1+s-1-j] + conj(P1_{d1-j}) Vw[d1+s-j]
      group_sums<NT, 4, Pol>(
          2 * d2, d1 + 1,
          [=] __device__(int o, int j) {
            if (o < d2) {
              const int s2 = o;
              T v = Pol::ld(Pch + j) * Pol::ld(Uw + d1 + s2 - j);
              if (j >= 1) v = v + Pol::ld(Qch + j) * Pol::ld(Vw + d1 + 1 + s2 - j);
              return v;
            }
            const int s2 = o - d2;
            T v = conj(Pol::ld(Pch + d1 - j)) * Pol::ld(Vw + d1 + s2 - j);
            if (j <= d1 - 1) v = v + conj(Pol::ld(Qch + d1 - j)) * Pol::ld(Uw + d1 + s2 - 1 - j);
            return v;
          },
          [=] __device__(int o, T v) { Pol::st(o < d2 ? Uh + o : Vh + (o - d2), v); });
      __syncthreads();
      }
      st[top].stage = 2;
      st[top + 1] = SchurNode{m + d1, d2, 0, Uh, Vh, Pch, Qch};
      ++top;
      continue;
    }
    if (nd.stage == 2 && M <= Pol::kDirectM) {
      if (lead) {
      // P_i = sum_j P2_j P1_{i-j} + Q2_j conj(Q1_{d1-i+j}),
      // Q_i = sum_j P2_j Q1_{i-j} + Q2_j conj(P1_{d1-i+j})  (P1, Q1 saved in F)
      float4 *Pc = nd.Pc, *Qc = nd.Qc;
      const float4 *P1 = F, *Q1 = F + M;
      group_sums<NT, 4, Pol>(
          2 * (d + 1), d2 + 1,
          [=] __device__(int o, int j) {
            const bool isq = o > d;
            const int i = isq ? o - d - 1 : o;
            const int t = i - j;
            if (t < 0 || t > d1) return Pol::zero();
            const T x1 = isq ? Pol::ld(Q1 + t) : Pol::ld(P1 + t);
            const T y1 = conj(isq ? Pol::ld(P1 + d1 - t) : Pol::ld(Q1 + d1 - t));
            return Pol::ld(Pch + j) * x1 + Pol::ld(Qch + j) * y1;
          },
          [=] __device__(int o, T v) {
            if (o > d) Pol::st(Qc + (o - d - 1), v);
            else Pol::st(Pc + o, v);
          });
      __syncthreads();
      }
      --top;
      continue;
    }
    if (nd.stage == 1) {
      if (work) {
      if (team) cluster_barrier();  // the first half (rank 0's, if short) complete
      const float4 *Uw = nd.Uw, *Vw = nd.Vw;
      pol_fft<NT, Pol>(
          Pl, 4,
          [=] __device__(int j, int i) {
            if (j == 0) return i <= d1 ? Pol::ld(Pch + i) : Pol::zero();
            if (j == 1) return i <= d1 ? Pol::ld(Qch + i) : Pol::zero();
            if (j == 2) return i < d ? Pol::ld(Uw + i) : Pol::zero();
            return i < d ? Pol::ld(Vw + i) : Pol::zero();
          },
          F, scr, log2M, false, tr, ts);
      // second half's windows: U_h(h+1+s) = (P1 * Uw)[d1+s] + (Q1 * Vw)[d1+1+s],
      // V_h(h+s) = (R1 * Uw)[d1+s-1] + (S1 * Vw)[d1+s]; FFT(R1) = W^{d1 w}
      // conj(F1), FFT(S1) = W^{d1 w} conj(F0), and a shift by one lag is a
      // factor W^{-w} or W^{w} (W = exp(-j 2 pi / M))
      pol_fft<NT, Pol>(
          Pl, 2,
          [=] __device__(int j, int w) {
            const T f0 = Pol::ld(F + w), f1 = Pol::ld(F + M + w), f2 = Pol::ld(F + 2 * M + w),
                    f3 = Pol::ld(F + 3 * M + w);
            if (j == 0) return f0 * f2 + P2.w((M - w) & msk, log2M) * (f1 * f3);
            return P2.w((int)(((int64_t)(d1 + 1) * w) & msk), log2M) * (conj(f1) * f2) +
                   P2.w((int)(((int64_t)d1 * w) & msk), log2M) * (conj(f0) * f3);
          },
          scr, scr + 2 * (size_t)M, log2M, true, tr, ts);
      for (int s = gt; s < d2; s += St) {
        Pol::st(Uh + s, Pol::scale2(inv, Pol::ld(scr + d1 + s)));
        Pol::st(Vh + s, Pol::scale2(inv, Pol::ld(scr + M + d1 + s)));
      }
      team_sync(ts);
      }
      st[top].stage = 2;
      st[top + 1] = SchurNode{m + d1, d2, 0, Uh, Vh, Pch, Qch};
      ++top;
      continue;
    }
    // stage 2: Theta = Theta2 Theta1, P = P2 P1 + Q2 R1, Q = P2 Q1 + Q2 S1
    if (work) {
    if (team) cluster_barrier();  // the second half complete
    pol_fft<NT, Pol>(
        Pl, 2,
        [=] __device__(int j, int i) {
          if (j == 0) return i <= d2 ? Pol::ld(Pch + i) : Pol::zero();
          return i <= d2 ? Pol::ld(Qch + i) : Pol::zero();
        },
        F + 2 * (size_t)M, scr, log2M, false, tr, ts);
    pol_fft<NT, Pol>(
        Pl, 2,
        [=] __device__(int j, int w) {
          const T f0 = Pol::ld(F + w), f1 = Pol::ld(F + M + w), g0 = Pol::ld(F + 2 * M + w), g1 = Pol::ld(F + 3 * M + w);
          const T tw = P2.w((int)(((int64_t)d1 * w) & msk), log2M);
          if (j == 0) return g0 * f0 + tw * (g1 * conj(f1));
          return g0 * f1 + tw * (g1 * conj(f0));
        },
        scr, scr + 2 * (size_t)M, log2M, true, tr, ts);
    float4 *Pc = nd.Pc, *Qc = nd.Qc;
    for (int i = gt; i <= d; i += St) {
      T p = i < M ? Pol::scale2(inv, Pol::ld(scr + i)) : Pol::zero();
      T q = i < M ? Pol::scale2(inv, Pol::ld(scr + M + i)) : Pol::zero();
      if (M == d) {  // coefficient d of Q aliased onto 0 (Q_0 = 0; deg P <= d - 1)
        if (i == 0) q = Pol::zero();
        if (i == d) q = Pol::scale2(inv, Pol::ld(scr + M));
      }
      Pol::st(Pc + i, p);
      Pol::st(Qc + i, q);
    }
    team_sync(ts);
    }
    --top;
  }
}

// ------------------------------------------------------------ refinement --
// One step of iterative refinement of the generator (the superfast runs'
// rounding error grows with N; one step brings it back to the kappa(C) eps
// of the arithmetic).  With Ct = C / c_0, the approximate generator rho and
// pivot dl (of Ct): z0 = rho / dl approximates Ct^{-1} e_{N-1}; the residual
// r = e_{N-1} - Ct z0 is one Toeplitz product (Ct embedded in a circulant of
// length M2 >= 2N); z1 = z0 + Ct^{-1} r with Ct^{-1} applied by eq.
// (gohberg-semencul) from rho (as block_gs_apply); then rho = z1 / z1_{N-1},
// dl = 1 / z1_{N-1}.  a (FP64) is read and rewritten in place (rho_n =
// conj(a_{N-1-n})); c is the FP64 first column, inv_c0 = 1 / c_0.  Returns
// the refined pivot of Ct.  A team (csize > 1) shares every step; c and a
// are then in global memory.
template <int NT, class Pol>
__device__ double schur_refine(const Pol& Pl, const SchurWork& W, const c128* c, double inv_c0, c128* a, int N,
                               double dl, int crank = 0, int csize = 1) {
  using T = typename Pol::T;
  const int M2 = schur_refine_m(N);
  const int lg = ilog2((uint32_t)M2);
  const int msk = M2 - 1;
  // P | H | R contiguous; UZ 2 M2; X; tmp 2 M2.  No FFT reads its own output.
  float4* P = W.refine;  // transform of rho
  float4* H = P + M2;    // transform of the circulant's column; then of r; then T1 r truncated
  float4* R = H + M2;    // r; then T0^H r truncated
  float4* UZ = R + M2;   // T1 r | T0^H r
  float4* X = UZ + 2 * (size_t)M2;
  float4* tmp = X + M2;  // 2 M2
  const T inv_dl = Pol::of(mk(1.0 / dl, 0.0));
  const float inv = 1.0f / (float)M2;  // a power of two: exact
  const Pol P2 = Pl;
  const int gt = crank * NT + (int)threadIdx.x, St = csize * NT;  // this thread in the team, the team's threads
  // transforms of rho and of the circulant's first column
  // [c_0..c_{N-1}, 0.., conj(c_{N-1})..conj(c_1)] (scaled by 1/c_0)
  pol_fft<NT, Pol>(
      Pl, 2,
      [=] __device__(int j, int i) {
        if (j == 0) return i < N ? Pol::of(conj(a[N - 1 - i])) : Pol::zero();
        if (i < N) return Pol::of(inv_c0 * c[i]);
        if (i > M2 - N) return Pol::of(inv_c0 * conj(c[M2 - i]));
        return Pol::zero();
      },
      P, tmp, lg, false, crank, csize);
  // Ct z0 (z0 = rho / dl), then r = e_{N-1} - Ct z0 and its transform
  pol_fft<NT, Pol>(
      Pl, 1, [=] __device__(int, int w) { return (Pol::ld(H + w) * Pol::ld(P + w)) * inv_dl; }, R, UZ, lg, true, crank,
      csize);
  for (int i = gt; i < M2; i += St) {
    T v = Pol::zero();
    if (i < N) {
      v = Pol::scale2(-inv, Pol::ld(R + i));
      if (i == N - 1) v = Pol::one() + v;
    }
    Pol::st(R + i, v);
  }
  team_sync(csize);
  pol_fft<NT, Pol>(Pl, 1, [=] __device__(int, int i) { return Pol::ld(R + i); }, H, UZ, lg, false, crank, csize);
  // Ct^{-1} r by eq. (gohberg-semencul) as in block_gs_apply: u = T1 r and
  // z = T0^H r, truncated to N and transformed again, then T1^H u - T0 z
  pol_fft<NT, Pol>(
      Pl, 2,
      [=] __device__(int j, int w) {
        const T rf = Pol::ld(H + w), p = Pol::ld(P + w);
        if (j == 0) return rf * conj(P2.w((int)(((int64_t)(N - 1) * w) & msk), lg)) * p;
        return rf * conj(P2.w(w, lg)) * conj(p);
      },
      UZ, tmp, lg, true, crank, csize);
  pol_fft<NT, Pol>(
      Pl, 2,
      [=] __device__(int j, int i) { return i < N ? Pol::scale2(inv, Pol::ld(UZ + (size_t)j * M2 + i)) : Pol::zero(); },
      H, tmp, lg, false, crank, csize);
  pol_fft<NT, Pol>(
      Pl, 1,
      [=] __device__(int, int w) {
        const T p = Pol::ld(P + w);
        const T g1 = P2.w((int)(((int64_t)(N - 1) * w) & msk), lg) * conj(p), g0 = P2.w(w, lg) * p;
        return g1 * Pol::ld(H + w) - g0 * Pol::ld(R + w);
      },
      X, UZ, lg, true, crank, csize);
  // z1 = z0 + X / (M2 dl) = (rho + X / M2) / dl; rho' = z1 / z1_{N-1}, dl' = 1 / Re z1_{N-1}
  const c128 den = mk(1.0, 0.0) + Pol::to_c128(Pol::scale2(inv, Pol::ld(X + N - 1)));
  const double dd = norm2(den);
  const c128 inv_den = mk(den.re / dd, -den.im / dd);
  for (int n = gt; n < N; n += St) {
    const c128 z = conj(a[N - 1 - n]) + Pol::to_c128(Pol::scale2(inv, Pol::ld(X + n)));
    a[N - 1 - n] = conj(z * inv_den);
  }
  team_sync(csize);
  return dl / den.re;
}

// ------------------------------------------------------------- GS apply --
// x = C^{-1} y by eq. (gohberg-semencul) as FFT convolutions of length M2 =
// 2^log2M2 >= 2N: the six transforms of block_gs_apply_df, each by pol_fft
// (the same butterflies in the same order), so that a team of csize blocks
// can share them.  rho, Yf = FFT_M2(y) and x in FP64 (global memory for a
// team); bufs: 5 arrays of M2 16-byte elements (global memory).
template <int NT, class Pol>
__device__ void team_gs_apply(const Pol& Pl, const c128* rho, const c128* Yf, c128* x, int N, int log2M2,
                              double delta_last, c128* const* bufs, int crank = 0, int csize = 1) {
  using T = typename Pol::T;
  const int M2 = 1 << log2M2;
  const int msk = M2 - 1;
  const float inv = 1.0f / (float)M2;  // a power of two: exact
  const Pol P2 = Pl;
  float4* P = reinterpret_cast<float4*>(bufs[0]);
  float4* B1 = reinterpret_cast<float4*>(bufs[1]);
  float4* B2 = reinterpret_cast<float4*>(bufs[2]);
  float4* B3 = reinterpret_cast<float4*>(bufs[3]);
  float4* Tm = reinterpret_cast<float4*>(bufs[4]);
  pol_fft<NT, Pol>(
      Pl, 1, [=] __device__(int, int i) { return i < N ? Pol::of(rho[i]) : Pol::zero(); }, P, Tm, log2M2, false,
      crank, csize);
  // u = T1 y
  pol_fft<NT, Pol>(
      Pl, 1,
      [=] __device__(int, int w) {
        return Pol::of(Yf[w]) * conj(P2.w((int)(((int64_t)(N - 1) * w) & msk), log2M2)) * Pol::ld(P + w);
      },
      B1, Tm, log2M2, true, crank, csize);
  pol_fft<NT, Pol>(
      Pl, 1, [=] __device__(int, int i) { return i < N ? Pol::scale2(inv, Pol::ld(B1 + i)) : Pol::zero(); }, B2, Tm,
      log2M2, false, crank, csize);
  // z = T0^H y
  pol_fft<NT, Pol>(
      Pl, 1, [=] __device__(int, int w) { return Pol::of(Yf[w]) * conj(P2.w(w, log2M2)) * conj(Pol::ld(P + w)); },
      B1, Tm, log2M2, true, crank, csize);
  pol_fft<NT, Pol>(
      Pl, 1, [=] __device__(int, int i) { return i < N ? Pol::scale2(inv, Pol::ld(B1 + i)) : Pol::zero(); }, B3, Tm,
      log2M2, false, crank, csize);
  // x = (T1^H u - T0 z) / delta
  pol_fft<NT, Pol>(
      Pl, 1,
      [=] __device__(int, int w) {
        const T g1 = P2.w((int)(((int64_t)(N - 1) * w) & msk), log2M2) * conj(Pol::ld(P + w));
        const T g0 = P2.w(w, log2M2) * Pol::ld(P + w);
        return g1 * Pol::ld(B2 + w) - g0 * Pol::ld(B3 + w);
      },
      B1, Tm, log2M2, true, crank, csize);
  const double sc = (double)inv / delta_last;
  for (int i = crank * NT + (int)threadIdx.x; i < N; i += csize * NT) {
    const c128 v = Pol::to_c128(Pol::ld(B1 + i));
    x[i] = mk(sc * v.re, sc * v.im);
  }
  team_sync(csize);
}

// ------------------------------------------------------------- the block --
// rho's predictor a (FP64, a_0 = 1) of the Hermitian positive definite
// Toeplitz matrix with first column c (FP64), with delta_{N-1} and ln|C| =
// sum_n ln delta_n, by the runs above and one step of refinement.  Called by every thread of the block
// (NT threads); c and a may be shared or global memory; ws holds
// schur_workspace_elems(N) float4s (global), smem schur_smem_bytes(lsm) of
// shared memory (lsm from schur_pick_lsm); sh_bad one shared int; sh_red NT/32 doubles and NT/32 ints
// of shared memory.
// A team of csize blocks of a cluster (this one of rank crank) shares the
// recursion's global-memory FFT stages and the refinement: every block of the
// team calls this with the same c, a, N, ws and lsm (c and a in global
// memory, sh_bad and sh_rex at the same shared-memory offsets in every
// block); rank 0's result is the one returned, the other ranks' is empty.
template <int NT, class Pol>
__device__ __noinline__ LevResult block_superfast(const Pol& Pl, const c128* c, c128* a, int N, float4* ws, float4* smem,
                                     int lsm, int* sh_bad, double* sh_red, int* sh_rex, int crank = 0,
                                     int csize = 1) {
  using T = typename Pol::T;
  static_assert(NT >= 96, "the leaves use three warps");
  SchurWork W = schur_carve(ws, N);
  schur_carve_smem(W, smem, lsm);
  W.bad = sh_bad;
  const double c0 = c[0].re;
  const bool c0_ok = c0 > 0.0 && isfinite(c0);
  const double inv_c0 = c0_ok ? 1.0 / c0 : 0.0;
  if (threadIdx.x == 0) *sh_bad = !c0_ok;
  for (int t = crank * NT + (int)threadIdx.x; t < N - 1; t += csize * NT) {
    Pol::st(W.Uw + t, Pol::of(inv_c0 * c[t + 1]));
    Pol::st(W.Vw + t, Pol::of(inv_c0 * c[t]));
  }
  team_sync(csize);
  if (N > 1) schur_solve<NT, Pol>(Pl, W, N - 1, crank, csize);
  double dlast = 1.0;
  bool refine = false;
  if (crank == 0) {
    // a = P + Q (the predictor of order N-1)
    for (int i = threadIdx.x; i < N; i += NT)
      a[i] = N > 1 ? Pol::to_c128(Pol::ld(W.Pc + i) + Pol::ld(W.Qc + i)) : mk(1.0, 0.0);
    // ln|C| / c_0^N = sum_n ln(delta_n / c_0): a product kept as mantissa and
    // exponent, in a fixed order; delta_{N-1} = delta_{N-2} (1 - |k_{N-1}|^2)
    if (N > 1) {
      const double dp = Pol::re_d(Pol::ld(W.delta + N - 2));
      const c128 kl = Pol::to_c128(Pol::ld(W.ks + N - 2));
      dlast = dp * (1.0 - norm2(kl));
    }
    __syncthreads();  // a complete, the leaves' flag visible
    refine = N > 1 && !*sh_bad && dlast > 0.0 && isfinite(dlast);
  }
  if (csize > 1) {
    // rank 0 hands the decision and the pivot to the others (their sh_bad and
    // sh_rex[0..1]; rank 0's own stay as they are)
    if (crank == 0 && threadIdx.x == 0)
      for (int r = 1; r < csize; ++r) {
        st_cluster_u32(sh_bad, (unsigned)r, refine ? 1u : 0u);
        st_cluster_u32(sh_rex, (unsigned)r, (unsigned)__double2loint(dlast));
        st_cluster_u32(sh_rex + 1, (unsigned)r, (unsigned)__double2hiint(dlast));
      }
    cluster_barrier();  // a and the decision visible to the team
    if (crank != 0) {
      refine = *sh_bad != 0;
      dlast = __hiloint2double(sh_rex[1], sh_rex[0]);
    }
  }
  if (refine) dlast = schur_refine<NT, Pol>(Pl, W, c, inv_c0, a, N, dlast, crank, csize);
  if (crank != 0) return LevResult{};
  double pm = 1.0;
  int pe = 0;
  for (int n = 1 + threadIdx.x; n < N; n += NT) {
    const double dn = n < N - 1 ? Pol::re_d(Pol::ld(W.delta + n)) : dlast;
    int ex;
    pm = frexp(pm * dn, &ex);
    pe += ex;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double m2 = __shfl_xor_sync(0xffffffffu, pm, o);
    const int e2 = __shfl_xor_sync(0xffffffffu, pe, o);
    int ex;
    pm = frexp(pm * m2, &ex);
    pe += e2 + ex;
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh_red[w] = pm;
    sh_rex[w] = pe;
  }
  __syncthreads();
  double tm = 1.0;
  int te = 0;
  for (int i = 0; i < NT / 32; ++i) {
    int ex;
    tm = frexp(tm * sh_red[i], &ex);
    te += sh_rex[i] + ex;
  }
  LevResult r;
  r.status = (*sh_bad || !(dlast > 0.0) || !isfinite(dlast) || !(tm > 0.0)) ? 1 : 0;
  r.delta_last = dlast * c0;
  r.logdet = log(tm) + te * 0.69314718055994530942 + (double)N * log(c0);
  __syncthreads();
  return r;
}

}  // namespace lse
