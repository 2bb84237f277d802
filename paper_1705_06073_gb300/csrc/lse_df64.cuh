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

// a + b when |a| >= |b| (or a = 0): Dekker's Fast2Sum, exact under that
// condition (used only to renormalise a head and its small correction)
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return f2{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// x + y1*z1 + y2*z2 with the final renormalisation by Fast2Sum
__device__ __forceinline__ f2 axpy2f(f2 x, f2 y1, f2 z1, f2 y2, f2 z2) {
  float p1, e1, p2, e2;
  prod_terms(y1, z1, p1, e1);
  prod_terms(y2, z2, p2, e2);
  const f2 s = two_sum(x.h, p1);
  const f2 t = two_sum(s.h, p2);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(x.l, e1), __fadd_rn(e2, s.l)), t.l);
  return fast_two_sum(t.h, lo);
}

// the four running sums of one thread's share of e = sum_i a_i c_{n+1-i}:
// Re a Re c, -Im a Im c, Re a Im c, Im a Re c (each S + E)
struct LevAcc {
  float S0, E0, S1, E1, S2, E2, S3, E3;
};

__device__ __forceinline__ void lev_acc(LevAcc& A, f2 r, f2 i, float4 c4) {
  const f2 cr = re_of(c4), ci = im_of(c4);
  acc_prod(A.S0, A.E0, r, cr);
  acc_prod(A.S1, A.E1, neg(i), ci);
  acc_prod(A.S2, A.E2, r, ci);
  acc_prod(A.S3, A.E3, i, cr);
}

// barrier over the first NTL threads of the block (named barrier 1)
template <int NTL>
__device__ __forceinline__ void lev_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(NTL) : "memory");
}

// ---- thread-block clusters (two blocks of a cluster share one recursion) ----
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// every thread of every block of the cluster; release/acquire at cluster scope
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of the same shared-memory object in block `rank` of the cluster
__device__ __forceinline__ unsigned cluster_addr(const void* p, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster(unsigned addr, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
__device__ __forceinline__ float4 ld_cluster(unsigned addr) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

// One pair (i, j = n - i) of an order: a_i + k conj(a_j) and a_j + k conj(a_i)
// from the loaded old values, stored where st_i / st_j (MIRROR: also into the
// other block's copy of a at peer_a), and both new values' products with
// their column entries (ci4 for entry i, cj4 for entry j; a zero entry adds
// exactly nothing) accumulated into A.
template <bool MIRROR>
__device__ __forceinline__ void lev_pair(float4* a, unsigned peer_a, float4 ai, float4 aj, f2 kr, f2 ki, int i, int j,
                                         bool st_i, bool st_j, float4 ci4, float4 cj4, LevAcc& A) {
  const f2 air = re_of(ai), aii = im_of(ai), ajr = re_of(aj), aji = im_of(aj);
  const f2 nir = axpy2f(air, kr, ajr, ki, aji);
  const f2 nii = axpy2f(aii, ki, ajr, neg(kr), aji);
  const f2 njr = axpy2f(ajr, kr, air, ki, aii);
  const f2 nji = axpy2f(aji, ki, air, neg(kr), aii);
  if (st_i) {
    const float4 v = pack(nir, nii);
    a[i] = v;
    if constexpr (MIRROR) st_cluster(peer_a + 16u * (unsigned)i, v);
  }
  if (st_j) {
    const float4 v = pack(njr, nji);
    a[j] = v;
    if constexpr (MIRROR) st_cluster(peer_a + 16u * (unsigned)j, v);
  }
  lev_acc(A, nir, nii, ci4);
  lev_acc(A, njr, nji, cj4);
}

// loads of the recursion's vectors: shared memory, or (G) global memory read
// through L2 only, since other SMs of the cluster rewrite a between orders
template <bool G>
__device__ __forceinline__ float4 lev_ld(const float4* p) {
  if constexpr (G) return __ldcg(p);
  else return *p;
}

// Sum of NS double-float partial sums {S_re, E_re, S_im, E_im} in a fixed
// pairwise tree (groups of at most 8, then the group totals), so that every
// thread that calls it gets bit-identical totals.
template <int NS>
__device__ __forceinline__ float4 tree8(const float4* slot) {
  static_assert(NS >= 1 && NS <= 8 && (NS & (NS - 1)) == 0, "tree of 1..8 slots");
  float4 v[NS];
#pragma unroll
  for (int w = 0; w < NS; ++w) v[w] = slot[w];
#pragma unroll
  for (int st = 1; st < NS; st <<= 1) {
#pragma unroll
    for (int w = 0; w < NS; w += 2 * st) {
      acc_merge(v[w].x, v[w].y, v[w + st].x, v[w + st].y);
      acc_merge(v[w].z, v[w].w, v[w + st].z, v[w + st].w);
    }
  }
  return v[0];
}

template <int NS>
__device__ __forceinline__ float4 slot_total(const float4* slot) {
  if constexpr (NS <= 8) {
    return tree8<NS>(slot);
  } else {
    static_assert(NS % 8 == 0 && NS <= 64, "up to 64 slots");
    float4 g[NS / 8];
#pragma unroll
    for (int k = 0; k < NS / 8; ++k) g[k] = tree8<8>(slot + 8 * k);
    return tree8<NS / 8>(g);
  }
}

constexpr int kLevGo = 1, kLevStop = 2;

// ---------------------------------------------------------------------------
// The orders of the double-float Levinson-Durbin recursion (the same orders
// and the same update of every pair (i, n-i) fused with the next inner product
// as block_levinson), run by the first NTL threads of C blocks:
//  - C = 1: one block, c and a in its shared memory;
//  - C = 2, G = false: the two blocks of a cluster, each holding a full copy
//    of c and a in its own shared memory; every stored entry is mirrored
//    into the other copy;
//  - G = true: the C blocks of a cluster share one c and a in global memory
//    (large N), read through L2.
// The pairs are dealt to the C * NTL threads; a thread takes two pairs per
// step without branches (a missing pair reads c[0], stores nothing and
// accumulates zeros).  Every order ends with each warp's partial inner
// product in a double-buffered slot (C > 1: written into every block of the
// cluster) and one barrier over the participating threads (C > 1: a cluster
// barrier, whose release/acquire also orders the stores of a); then every
// thread sums the C * NTL / 32 slots in the same fixed tree and forms the
// next reflection coefficient itself, so all of them hold bit-identical
// scalars and leave the loop together.  The pivot of the order, which needs
// only k_n, is formed in the same straight-line block as the first two pairs
// so that its dependency chain overlaps their arithmetic.
// c, a: double-float (c scaled by 1/c_0, a[0] = 1, rest 0); red: 2 * C *
// NTL / 32 float4 of shared memory.  C > 1: before every cluster barrier
// thread 0 writes sh->ctrl[barrier index & 1] (kLevGo, or kLevStop before
// the last one) for the block's threads that take no pairs (lev_shadow).
// Thread 0 leaves the status, pivot delta_{N-1} and ln|C| (unscaled) in sh.
// ---------------------------------------------------------------------------
template <int NTL, int C, bool G = false>
__device__ void lev_orders(const float4* c, float4* a, int N, double c0, float4* red, LevShared* sh, unsigned rank) {
  constexpr int NW = NTL / 32;
  constexpr int V = C * NTL;  // threads sharing the pairs
  constexpr bool MIRROR = (C == 2) && !G;
  static_assert(C == 1 || C == 2 || G, "shared-memory copies are mirrored between two blocks only");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int vt = threadIdx.x + NTL * (int)rank;
  unsigned peer_a = 0;
  if constexpr (MIRROR) peer_a = cluster_addr(a, rank ^ 1u);
  f2 kr{0.f, 0.f}, ki{0.f, 0.f};
  if (N > 1) {
    const float4 c1 = lev_ld<G>(c + 1);
    kr = neg(re_of(c1));
    ki = neg(im_of(c1));
  }
  f2 delta{1.f, 0.f}, mant{1.f, 0.f};
  int expo = 0;
  int bad = !(c0 > 0.0 && isfinite(c0));
  int bidx = 0;  // cluster barriers passed
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int n = 1; n < N && !bad; ++n) {
    const bool more = (n + 1) < N;
    LevAcc A{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    f2 dn, inv_dn;
    {
      const int i0 = vt, i1 = vt + V;
      const bool v0 = 2 * i0 <= n, v1 = 2 * i1 <= n;
      const int ia = v0 ? i0 : 0, ib = v1 ? i1 : 0;
      const int ja = v0 ? n - ia : 0, jb = v1 ? n - ib : 0;
      const float4* pa = v0 ? a : c;
      const float4* pb = v1 ? a : c;
      const float4 aa_i = lev_ld<G>(pa + ia), aa_j = lev_ld<G>(pa + ja), ab_i = lev_ld<G>(pb + ib),
                   ab_j = lev_ld<G>(pb + jb);
      const bool wa_i = v0 && more, wa_j = wa_i && ja != ia, wb_i = v1 && more, wb_j = wb_i && jb != ib;
      const float4 ca_i = lev_ld<G>(c + (wa_i ? n + 1 - ia : 0)), ca_j = lev_ld<G>(c + (wa_j ? ia + 1 : 0));
      const float4 cb_i = lev_ld<G>(c + (wb_i ? n + 1 - ib : 0)), cb_j = lev_ld<G>(c + (wb_j ? ib + 1 : 0));
      // pivot of this order, delta_n = delta_{n-1} (1 - |k_n|^2), and 1/delta_n
      float p1, q1, p2, q2;
      prod_terms(kr, kr, p1, q1);
      prod_terms(ki, ki, p2, q2);
      const f2 k2a = two_sum(p1, p2);
      const f2 k2 = two_sum(k2a.h, __fadd_rn(__fadd_rn(q1, q2), k2a.l));
      dn = mul(delta, sub(f2{1.f, 0.f}, k2));
      inv_dn = recip(dn);
      lev_pair<MIRROR>(a, peer_a, aa_i, aa_j, kr, ki, ia, ja, v0, v0 && ja != ia, wa_i ? ca_i : z4, wa_j ? ca_j : z4, A);
      lev_pair<MIRROR>(a, peer_a, ab_i, ab_j, kr, ki, ib, jb, v1, v1 && jb != ib, wb_i ? cb_i : z4, wb_j ? cb_j : z4, A);
    }
    for (int ia = vt + 2 * V; 2 * ia <= n; ia += 2 * V) {
      const int i1 = ia + V;
      const bool v1 = 2 * i1 <= n;
      const int ib = v1 ? i1 : 0;
      const int ja = n - ia, jb = v1 ? n - ib : 0;
      const float4* pb = v1 ? a : c;
      const float4 aa_i = lev_ld<G>(a + ia), aa_j = lev_ld<G>(a + ja), ab_i = lev_ld<G>(pb + ib),
                   ab_j = lev_ld<G>(pb + jb);
      const bool wa_j = more && ja != ia, wb_i = v1 && more, wb_j = wb_i && jb != ib;
      const float4 ca_i = lev_ld<G>(c + (more ? n + 1 - ia : 0)), ca_j = lev_ld<G>(c + (wa_j ? ia + 1 : 0));
      const float4 cb_i = lev_ld<G>(c + (wb_i ? n + 1 - ib : 0)), cb_j = lev_ld<G>(c + (wb_j ? ib + 1 : 0));
      lev_pair<MIRROR>(a, peer_a, aa_i, aa_j, kr, ki, ia, ja, true, ja != ia, more ? ca_i : z4, wa_j ? ca_j : z4, A);
      lev_pair<MIRROR>(a, peer_a, ab_i, ab_j, kr, ki, ib, jb, v1, v1 && jb != ib, wb_i ? cb_i : z4, wb_j ? cb_j : z4, A);
    }
    acc_merge(A.S0, A.E0, A.S1, A.E1);
    acc_merge(A.S2, A.E2, A.S3, A.E3);
    float S0 = A.S0, E0 = A.E0, S2 = A.S2, E2 = A.E2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float sr = __shfl_xor_sync(0xffffffffu, S0, o), er = __shfl_xor_sync(0xffffffffu, E0, o);
      const float si = __shfl_xor_sync(0xffffffffu, S2, o), ei = __shfl_xor_sync(0xffffffffu, E2, o);
      acc_merge(S0, E0, sr, er);
      acc_merge(S2, E2, si, ei);
    }
    float4* slot = red + (n & 1) * C * NW;
    if (lane == 0) {
      const float4 v = make_float4(S0, E0, S2, E2);
      const int si = (int)rank * NW + warp;
      slot[si] = v;
      if constexpr (C > 1) {
#pragma unroll
        for (unsigned r = 1; r < (unsigned)C; ++r)
          st_cluster(cluster_addr(slot + si, (rank + r) % (unsigned)C), v);
      }
    }
    if constexpr (C > 1) {
      if (threadIdx.x == 0) sh->ctrl[bidx & 1] = kLevGo;
      cluster_barrier();
      ++bidx;
    } else {
      lev_bar<NTL>();
    }
    // the same fixed tree over the slots in every thread
    const float4 tot = slot_total<C * NW>(slot);
    const float s0 = tot.x, e0 = tot.y, s1 = tot.z, e1 = tot.w;
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
  if constexpr (C > 1) {
    if (threadIdx.x == 0) sh->ctrl[bidx & 1] = kLevStop;
    cluster_barrier();
  }
  if (threadIdx.x == 0) {
    sh->status = bad;
    sh->delta = to_d(delta) * c0;
    sh->logdet = log(to_d(mant)) + expo * 0.69314718055994530942 + (double)N * log(c0);
  }
}

// The threads of a block that take no pairs in a cluster recursion: they pass
// the same cluster barriers as the others (a cluster barrier counts every
// thread of both blocks) and stop after the one announced by kLevStop.
__device__ __forceinline__ void lev_shadow(const LevShared* sh) {
  for (int bidx = 0;; ++bidx) {
    cluster_barrier();
    if (((volatile const int*)sh->ctrl)[bidx & 1] == kLevStop) break;
  }
}

// c (FP64 first column, in shared memory) -> double-float in place, scaled by
// 1/c_0; a <- e_0.  Returns c_0.
template <int NT>
__device__ double lev_prologue(c128* c64, c128* a64, int N) {
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
  return c0;
}

// a (double-float) -> FP64 in place; results of lev_orders from sh
template <int NT>
__device__ LevResult lev_epilogue(c128* a64, int N, const LevShared* sh) {
  const float4* a = reinterpret_cast<const float4*>(a64);
  LevResult r;
  r.status = sh->status;
  r.delta_last = sh->delta;
  r.logdet = sh->logdet;
  for (int i = threadIdx.x; i < N; i += NT) {
    const float4 v = a[i];
    a64[i] = mk(to_d(re_of(v)), to_d(im_of(v)));
  }
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// The double-float Levinson-Durbin recursion in one block: the orders run on
// the first NTL = 128 threads (one warp per SM sub-partition) and the rest of
// the block waits at the closing barrier.  The per-order reduction and scalar
// work is paid per warp, which is why fewer, busier warps win: at N = 4096
// four warps ran the recursion about 13% faster than eight.
// c: FP64 first column, converted in place to double-float (same 16 bytes per
// element); a: output predictor in FP64.  red: 2*NTL/32 float4 of shared
// memory; sh: carries the results to the threads that did not take part.
// ---------------------------------------------------------------------------
template <int NT, int NTL = 128>
__device__ __noinline__ LevResult block_levinson_df(c128* c64, c128* a64, int N, float4* red, LevShared* sh) {
  static_assert(NTL % 32 == 0 && NTL <= NT, "recursion threads");
  const double c0 = lev_prologue<NT>(c64, a64, N);
  if (threadIdx.x < NTL)
    lev_orders<NTL, 1>(reinterpret_cast<const float4*>(c64), reinterpret_cast<float4*>(a64), N, c0, red, sh, 0u);
  __syncthreads();
  return lev_epilogue<NT>(a64, N, sh);
}

// ---------------------------------------------------------------------------
// The same recursion shared by the two blocks of a cluster (each on its own
// SM), called by every thread of both blocks with the same N and c_0.  c: the
// double-float column (scaled by 1/c_0) already in this block's shared memory;
// a: this block's copy of the predictor (the pairs each block updates are
// stored into both copies).  Returns with a complete in both blocks, still in
// double-float; the caller converts what it needs.  One cluster barrier per
// order (about 0.2 us on GB300) against half the pair work per SM.
// Not inlined: the two blocks of a cluster then run one copy of the code.
// Two inlined copies (one in each block's caller) measured 16% slower on the
// whole fit, with instruction-fetch stalls as the top stall reason; the two
// SMs of a cluster evidently share an instruction cache level.
// ---------------------------------------------------------------------------
template <int NT, int NTL = 128>
__device__ __noinline__ LevResult cluster_levinson_df(const c128* c64, c128* a64, int N, double c0, float4* red, LevShared* sh) {
  static_assert(NTL % 32 == 0 && NTL <= NT, "recursion threads");
  const unsigned rank = cluster_ctarank();
  float4* a = reinterpret_cast<float4*>(a64);
  for (int i = threadIdx.x; i < N; i += NT) a[i] = make_float4(i == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);
  cluster_barrier();  // both copies initialised before any mirrored store
  if (threadIdx.x < NTL) lev_orders<NTL, 2>(reinterpret_cast<const float4*>(c64), a, N, c0, red, sh, rank);
  else lev_shadow(sh);
  __syncthreads();
  LevResult r;
  r.status = sh->status;
  r.delta_last = sh->delta;
  r.logdet = sh->logdet;
  return r;
}

// A recursion request from the first block of a cluster to the others
// (op 1: shared-memory recursion of order N with c_0, two blocks; op 2: the
// same on the global vectors c, a; op 0: no more work).
struct alignas(16) LevCmd {
  int op, N;
  double c0;
  c128 *c, *a;
};

// write `v` into the LevCmd at the same shared address in blocks 1..csize-1
__device__ __forceinline__ void lev_send_cmd(const LevCmd* local, int csize, const LevCmd& v) {
  const float4 v0 = make_float4(__int_as_float(v.op), __int_as_float(v.N), __int_as_float(__double2loint(v.c0)),
                                __int_as_float(__double2hiint(v.c0)));
  const unsigned long long pc = (unsigned long long)v.c, pa = (unsigned long long)v.a;
  const float4 v1 = make_float4(__int_as_float((int)(pc & 0xffffffffu)), __int_as_float((int)(pc >> 32)),
                                __int_as_float((int)(pa & 0xffffffffu)), __int_as_float((int)(pa >> 32)));
  for (int r = 1; r < csize; ++r) {
    const unsigned dst = cluster_addr(local, (unsigned)r);
    st_cluster(dst, v0);
    st_cluster(dst + 16u, v1);
  }
}

// ---------------------------------------------------------------------------
// The recursion of a large instance shared by the C blocks of a cluster, with
// c and a in global memory (the instance's workspace; L2-resident), called by
// every thread of every block with the same arguments.  All NT threads of a
// block take pairs.  c: double-float, scaled by 1/c_0 (written before the
// cluster barrier that precedes this call); a is initialised here.  Returns
// with a complete in global memory, still in double-float.  Not inlined, so
// the blocks of a cluster run one copy of the code.
// ---------------------------------------------------------------------------
template <int NT, int C>
__device__ __noinline__ LevResult cluster_levinson_global(const c128* c64, c128* a64, int N, double c0, float4* red,
                                                          LevShared* sh) {
  const unsigned rank = cluster_ctarank();
  float4* a = reinterpret_cast<float4*>(a64);
  for (int i = threadIdx.x + NT * (int)rank; i < N; i += NT * C) a[i] = make_float4(i == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);
  cluster_barrier();  // a initialised (and c visible) in every block
  lev_orders<NT, C, true>(reinterpret_cast<const float4*>(c64), a, N, c0, red, sh, rank);
  __syncthreads();
  LevResult r;
  r.status = sh->status;
  r.delta_last = sh->delta;
  r.logdet = sh->logdet;
  return r;
}

// ---------------------------------------------------------------------------
// Double-float FFT and Gohberg-Semencul apply (the double-float fit path).
// Complex double-float values are float4 {re.h, re.l, im.h, im.l}.  Sums use
// the "sloppy" double-float addition (TwoSum of the heads, the tails added,
// Fast2Sum renormalisation), whose error is relative to the operands'
// magnitudes, the usual FFT error model; products keep the cross terms.
// ---------------------------------------------------------------------------
__device__ __forceinline__ f2 add_s(f2 a, f2 b) {
  const f2 s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ f2 sub_s(f2 a, f2 b) { return add_s(a, neg(b)); }
__device__ __forceinline__ f2 mul_f(f2 a, f2 b) {
  float p, e;
  prod_terms(a, b, p, e);
  return fast_two_sum(p, e);
}

struct cf2 {
  f2 re, im;
};
__device__ __forceinline__ cf2 ld_cf2(float4 v) { return cf2{f2{v.x, v.y}, f2{v.z, v.w}}; }
__device__ __forceinline__ float4 st_cf2(cf2 a) { return make_float4(a.re.h, a.re.l, a.im.h, a.im.l); }
__device__ __forceinline__ cf2 cf2_of(c128 v) { return cf2{to_f2(v.re), to_f2(v.im)}; }
__device__ __forceinline__ cf2 operator+(cf2 a, cf2 b) { return cf2{add_s(a.re, b.re), add_s(a.im, b.im)}; }
__device__ __forceinline__ cf2 operator-(cf2 a, cf2 b) { return cf2{sub_s(a.re, b.re), sub_s(a.im, b.im)}; }
__device__ __forceinline__ cf2 operator*(cf2 a, cf2 b) {
  return cf2{sub_s(mul_f(a.re, b.re), mul_f(a.im, b.im)), add_s(mul_f(a.re, b.im), mul_f(a.im, b.re))};
}
__device__ __forceinline__ cf2 conj(cf2 a) { return cf2{a.re, neg(a.im)}; }
__device__ __forceinline__ cf2 mul_j(cf2 a) { return cf2{neg(a.im), a.re}; }
// multiplication by a power of two (exact)
__device__ __forceinline__ cf2 scale2(float s, cf2 a) {
  return cf2{f2{a.re.h * s, a.re.l * s}, f2{a.im.h * s, a.im.l * s}};
}
__device__ __forceinline__ cf2 cf2_zero() { return cf2{f2{0.f, 0.f}, f2{0.f, 0.f}}; }

// exp(-j 2 pi k / M), 0 <= k < M, from the double-float table of 2^log2max points
struct TwiddlesDF {
  const float4* tw;
  int log2max;
  __device__ __forceinline__ cf2 w(int k, int log2M) const { return ld_cf2(tw[(size_t)k << (log2max - log2M)]); }
};

// block_fft (Stockham radix-4, decimation in frequency; first level reads
// gen(i), levels alternate between tmp and dst) in double-float
template <int NT, class Gen>
__device__ void block_fft_df(Gen gen, float4* dst, float4* tmp, int log2M, bool inverse, const TwiddlesDF& tw) {
  const int M = 1 << log2M;
  const int npass = (log2M >> 1) + (log2M & 1);
  int pass = 0;
  const float4* in = nullptr;
  int n = M, s = 1, log2s = 0;
  while (n >= 4) {
    ++pass;
    float4* out = ((npass - pass) & 1) ? tmp : dst;
    const int n4 = n >> 2;
    for (int t = threadIdx.x; t < (M >> 2); t += NT) {
      const int p = t >> log2s, q = t & (s - 1);
      cf2 a, b, c, d;
      if (pass == 1) {
        a = gen(q + s * p); b = gen(q + s * (p + n4)); c = gen(q + s * (p + 2 * n4)); d = gen(q + s * (p + 3 * n4));
      } else {
        a = ld_cf2(in[q + s * p]); b = ld_cf2(in[q + s * (p + n4)]);
        c = ld_cf2(in[q + s * (p + 2 * n4)]); d = ld_cf2(in[q + s * (p + 3 * n4)]);
      }
      const cf2 apc = a + c, amc = a - c, bpd = b + d, jbmd = mul_j(b - d);
      const cf2 y1 = inverse ? amc + jbmd : amc - jbmd;
      const cf2 y3 = inverse ? amc - jbmd : amc + jbmd;
      const cf2 y2 = apc - bpd;
      cf2 w1 = tw.w(p * s, log2M), w2 = tw.w(2 * p * s, log2M), w3 = tw.w(3 * p * s, log2M);
      if (inverse) { w1 = conj(w1); w2 = conj(w2); w3 = conj(w3); }
      out[q + s * (4 * p + 0)] = st_cf2(apc + bpd);
      out[q + s * (4 * p + 1)] = st_cf2(w1 * y1);
      out[q + s * (4 * p + 2)] = st_cf2(w2 * y2);
      out[q + s * (4 * p + 3)] = st_cf2(w3 * y3);
    }
    __syncthreads();
    in = out;
    n >>= 2; s <<= 2; log2s += 2;
  }
  if (n == 2) {
    ++pass;
    for (int q = threadIdx.x; q < (M >> 1); q += NT) {
      cf2 a, b;
      if (pass == 1) { a = gen(q); b = gen(q + s); } else { a = ld_cf2(in[q]); b = ld_cf2(in[q + s]); }
      dst[q] = st_cf2(a + b);
      dst[q + s] = st_cf2(a - b);
    }
    __syncthreads();
  }
}

// block_gs_apply in double-float: x = C^{-1} y by the Gohberg-Semencul
// formula (eq. gohberg-semencul) as FFT convolutions, the same six
// transforms of length M2; rho, Yf = FFT_M2(y) and x in FP64.
// bufs: 5 arrays of M2 complex (16 bytes each, used as double-float).
template <int NT>
__device__ void block_gs_apply_df(const c128* rho, const c128* Yf, c128* x, int N, int log2M2, double delta_last,
                                  c128* const* bufs, const TwiddlesDF& tw) {
  const int M2 = 1 << log2M2;
  const int msk = M2 - 1;
  const float inv = 1.0f / (float)M2;  // a power of two: exact
  float4* P = reinterpret_cast<float4*>(bufs[0]);
  float4* B1 = reinterpret_cast<float4*>(bufs[1]);
  float4* B2 = reinterpret_cast<float4*>(bufs[2]);
  float4* B3 = reinterpret_cast<float4*>(bufs[3]);
  float4* T = reinterpret_cast<float4*>(bufs[4]);
  block_fft_df<NT>([=] __device__(int i) { return i < N ? cf2_of(rho[i]) : cf2_zero(); }, P, T, log2M2, false, tw);
  // u = T1 y
  block_fft_df<NT>(
      [=] __device__(int w) {
        return cf2_of(Yf[w]) * conj(tw.w((int)(((int64_t)(N - 1) * w) & msk), log2M2)) * ld_cf2(P[w]);
      },
      B1, T, log2M2, true, tw);
  block_fft_df<NT>([=] __device__(int i) { return i < N ? scale2(inv, ld_cf2(B1[i])) : cf2_zero(); }, B2, T, log2M2,
                   false, tw);
  // z = T0^H y
  block_fft_df<NT>([=] __device__(int w) { return cf2_of(Yf[w]) * conj(tw.w(w, log2M2)) * conj(ld_cf2(P[w])); }, B1,
                   T, log2M2, true, tw);
  block_fft_df<NT>([=] __device__(int i) { return i < N ? scale2(inv, ld_cf2(B1[i])) : cf2_zero(); }, B3, T, log2M2,
                   false, tw);
  // x = (T1^H u - T0 z) / delta
  block_fft_df<NT>(
      [=] __device__(int w) {
        const cf2 g1 = tw.w((int)(((int64_t)(N - 1) * w) & msk), log2M2) * conj(ld_cf2(P[w]));
        const cf2 g0 = tw.w(w, log2M2) * ld_cf2(P[w]);
        return g1 * ld_cf2(B2[w]) - g0 * ld_cf2(B3[w]);
      },
      B1, T, log2M2, true, tw);
  const double sc = (double)inv / delta_last;
  for (int i = threadIdx.x; i < N; i += NT) {
    const cf2 v = ld_cf2(B1[i]);
    x[i] = mk(sc * to_d(v.re), sc * to_d(v.im));
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// block_first_column (Sec. III intro; C of eq. py) with the per-element sums
// in double-float: c_m = beta [m = 0] + sum_k gamma_k e^{j2pi m theta_k}, the
// shared tables gamma_k e^{j2pi l theta_k} and e^{j2pi S h theta_k} (m = S h
// + l) formed in FP64 with exactly reduced phases and kept as double-float;
// each (m, k) term is one double-float complex product, added with the
// accurate double-float sum.  Output in FP64.  smem: KC*(S + H) complex
// doubles, as for block_first_column.
// ---------------------------------------------------------------------------
__device__ __forceinline__ f2 add_a(f2 a, f2 b) {  // accurate double-float sum
  f2 s = two_sum(a.h, b.h);
  const f2 t = two_sum(a.l, b.l);
  s = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(s.h, __fadd_rn(s.l, t.l));
}

template <int NT>
__device__ void block_first_column_df(c128* c, const double* theta, const double* gamma, int K, double beta, int N,
                                      c128* smem) {
  int S, H;
  first_column_split(N, S, H);
  const int KC = kFirstColumnChunk;
  float4* lo = reinterpret_cast<float4*>(smem);  // [KC][S]
  float4* hi = lo + KC * S;                      // [KC][H]
  float4* c4 = reinterpret_cast<float4*>(c);     // running sums, double-float in place
  for (int m = threadIdx.x; m < N; m += NT) c4[m] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k0 = 0; k0 < K; k0 += KC) {
    const int kc = min(KC, K - k0);
    __syncthreads();
    for (int i = threadIdx.x; i < kc * S; i += NT) {
      const int k = i / S, l = i - k * S;
      const c128 v = gamma[k0 + k] * unit_phase((double)l, theta[k0 + k], 1.0);
      lo[k * S + l] = pack(to_f2(v.re), to_f2(v.im));
    }
    for (int i = threadIdx.x; i < kc * H; i += NT) {
      const int k = i / H, h = i - k * H;
      const c128 v = unit_phase((double)h * S, theta[k0 + k], 1.0);
      hi[k * H + h] = pack(to_f2(v.re), to_f2(v.im));
    }
    __syncthreads();
    for (int m = threadIdx.x; m < N; m += NT) {
      const int h = m / S, l = m - h * S;
      cf2 acc = ld_cf2(c4[m]);
      for (int k = 0; k < kc; ++k) {
        const cf2 t = ld_cf2(lo[k * S + l]) * ld_cf2(hi[k * H + h]);
        acc = cf2{add_a(acc.re, t.re), add_a(acc.im, t.im)};
      }
      c4[m] = st_cf2(acc);
    }
  }
  __syncthreads();
  for (int m = threadIdx.x; m < N; m += NT) {
    const cf2 v = ld_cf2(c4[m]);
    c[m] = mk((m == 0 ? beta : 0.0) + to_d(v.re), to_d(v.im));
  }
  __syncthreads();
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
