// lse_grid.cu -- grid evaluation of Sec. III-D (Hansen, Fleury, Rao,
// "Superfast Line Spectral Estimation"): for a given state (theta, gamma,
// beta) compute q(theta_l), s(theta_l) and their first and second
// theta-derivatives at theta_l = l/L.
//
// Two kernels:
//  factor_kernel  one block (or, double-float, one thread-block cluster) per
//                 instance: first column of C, Levinson recursion
//                 (Gohberg-Semencul generators rho, delta) and x = C^{-1} y
//                 by FFT convolutions (Sec. III-A, III-B).
//  grid kernels   the length-L spectra (on chip, or in four steps for L too
//                 large for one block) with the outputs written directly.
//                 With c = (N-2)/2 and
//                   Q_a = DFT_L((n-c)^a rho_n),  X_a = DFT_L(n^a x_n)
//                 the grid quantities are (Appendix B weights, centred)
//                   s   = (2/d) Re(Q1 Q0*)
//                   s'  = (4 pi/d) Im(Q2 Q0*)
//                   s'' = (8 pi^2/d) [Re(Q2 Q1*) - Re(Q3 Q0*)]
//                   q = X0,  q' = -j 2 pi X1,  q'' = -4 pi^2 X2
//                 (d = delta_{N-1}; DFT_L(v)(l) = sum_n v_n e^{-j 2 pi n l / L}).
#include <vector>

#include "lse_device.cuh"
#include "lse_df64.cuh"
#include "lse_fft_smem.cuh"
#include "lse_internal.h"
#include "lse_schur.cuh"

namespace lse {

namespace {

constexpr int kFNT = 256;
template <bool DF>
__host__ __device__ constexpr int factor_threads() { return 256; }

struct FactorLayout {
  size_t y, c, a, Yf, buf, sf, total, M2;
};
// sf: whether some instance runs the superfast recursion (its workspace)
__host__ __device__ inline FactorLayout factor_layout(int Nmax, bool sf) {
  FactorLayout L;
  const size_t M2 = (size_t)1 << ilog2(2u * (uint32_t)Nmax);
  size_t o = 0;
  auto put = [&](size_t bytes) { size_t r = o; o += (bytes + 255) & ~size_t(255); return r; };
  L.y = put(sizeof(c128) * Nmax);
  L.c = put(sizeof(c128) * Nmax);
  L.a = put(sizeof(c128) * Nmax);
  L.Yf = put(sizeof(c128) * M2);
  L.buf = put(sizeof(c128) * M2 * 5);
  L.sf = put(sf ? sizeof(float4) * schur_workspace_elems(Nmax) : 0);
  L.total = o;
  L.M2 = M2;
  return L;
}

// blocks per cluster for large-N recursions of the double-float factor kernel
constexpr int kFactorCluster = 8;

// csize > 1: clusters of csize blocks, one instance per cluster.  Levinson
// clusters (double-float only): the first block does everything and the
// others join its Levinson recursion (csize 2: shared-memory copies;
// kFactorCluster: global memory, for an instance too large for shared
// memory), or are released.
// sf_pair (csize 2, every instance of the launch on the superfast recursion):
// the second block follows the same steps, skipping the first block's own
// work, and takes half of every pass of the recursion's global-memory FFT
// stages and refinement, of the Gohberg-Semencul apply and of the two
// omega_s transforms; the results are the one-block ones, bit for bit.
template <bool DF>
__global__ void __launch_bounds__(factor_threads<DF>(), 1)
    factor_kernel(const float* y, const InstDesc* inst, int Nmax, const double* theta, const double* gamma,
                  const double* beta, Tables tab, char* ws, size_t ws_bytes, c128* rho_out, c128* x_out,
                  c128* omega_out, c64* omega32_out, c64* x32_out, double* delta_out, int* status, int csize,
                  int sf_min_n, int sf_pair) {
  constexpr int kFNT = factor_threads<DF>();
  __shared__ c128 red[kFNT];
  __shared__ LevShared lev;
  __shared__ LevCmd cmd;
  __shared__ int sf_bad;
  __shared__ double sf_red[kFNT / 32];
  __shared__ int sf_rex[kFNT / 32];
  extern __shared__ __align__(16) char dsm[];
  int b = blockIdx.x;
  int crank = 0;  // rank in a superfast pair
  if (csize > 1) {
    cluster_barrier();  // every block running before any store between them
    if (sf_pair) {
      crank = (int)cluster_ctarank();
    } else if (cluster_ctarank() != 0) {
      if constexpr (DF) {  // Levinson clusters: double-float only
        cluster_barrier();  // the request (or the release) is in cmd
        if (cmd.op == 1 && csize == 2) {
          // shared-memory recursion: copy the first block's double-float column
          const int n = cmd.N;
          c128* c = reinterpret_cast<c128*>(dsm);
          const unsigned src = cluster_addr(c, 0u);
          float4* c4 = reinterpret_cast<float4*>(c);
          for (int i = threadIdx.x; i < n; i += kFNT) c4[i] = ld_cluster(src + 16u * (unsigned)i);
          __syncthreads();
          cluster_levinson_df<kFNT>(c, c + n, n, cmd.c0, (float4*)red, &lev);
        } else if (cmd.op == 2 && csize == kFactorCluster) {
          cluster_levinson_global<kFNT, kFactorCluster>(cmd.c, cmd.a, cmd.N, cmd.c0, (float4*)red, &lev);
        }
      }
      return;
    }
    b = blockIdx.x / csize;
  }
  const InstDesc d = inst[b];
  const int N = d.N;
  const bool lead = crank == 0;
  char* base = ws + (size_t)b * ws_bytes;
  const FactorLayout FL = factor_layout(Nmax, sf_min_n > 0 && Nmax >= sf_min_n);
  // the superfast Schur recursion (lse_schur.cuh) for this instance?
  bool sf = sf_min_n > 0 && N >= sf_min_n;
  if constexpr (DF) sf = sf && tab.twdf != nullptr;
  c128* yv = (c128*)(base + FL.y);
  c128* Yf = (c128*)(base + FL.Yf);
  c128* bufp = (c128*)(base + FL.buf);
  c128* bufs[5];
  for (int j = 0; j < 5; ++j) bufs[j] = bufp + (size_t)j * FL.M2;
  const Twiddles<double> tw{tab.tw64, tab.log2max};
  const int log2M2 = ilog2(2u * (uint32_t)N);
  const float* yin = y + 2 * d.y_off;
  if (lead)
    for (int n = threadIdx.x; n < N; n += kFNT) yv[n] = mk((double)yin[2 * n], (double)yin[2 * n + 1]);
  __syncthreads();
  int S, H;
  first_column_split(N, S, H);
  const size_t tab_bytes = sizeof(c128) * kFirstColumnChunk * (S + H);
  const int smem_cap = 200 * 1024;
  c128 *cc, *aa, *tables;
  if (!sf && 2 * sizeof(c128) * (size_t)N + tab_bytes <= (size_t)smem_cap) {
    cc = (c128*)dsm; aa = cc + N; tables = aa + N;
  } else {
    cc = (c128*)(base + FL.c); aa = (c128*)(base + FL.a); tables = (c128*)dsm;
  }
  if (lead) {
    if constexpr (DF) block_first_column_df<kFNT>(cc, theta + d.k_off, gamma + d.k_off, d.K, beta[b], N, tables);
    else block_first_column<kFNT>(cc, theta + d.k_off, gamma + d.k_off, d.K, beta[b], N, tables);
  }
  LevResult lr;
  if (sf) {
    // a cluster launch still owes its other blocks their release
    if (DF && csize > 1 && !sf_pair) {
      if (threadIdx.x == 0) lev_send_cmd(&cmd, csize, LevCmd{0, N, 0.0, cc, aa});
      cluster_barrier();
    }
    float4* sfw = (float4*)(base + FL.sf);
    const size_t tb = (tab_bytes + 255) & ~size_t(255);
    float4* sfs = reinterpret_cast<float4*>(dsm + tb);
    const int lsm = schur_pick_lsm(smem_cap - tb);
    if (sf_pair) cluster_barrier();  // the first column (global memory) complete
    if constexpr (DF)
      lr = block_superfast<kFNT>(PolDF{tab.twdf, tab.log2max}, cc, aa, N, sfw, sfs, lsm, &sf_bad, sf_red, sf_rex,
                                 crank, sf_pair ? 2 : 1);
    else
      lr = block_superfast<kFNT>(Pol64{tab.tw64, tab.log2max}, cc, aa, N, sfw, sfs, lsm, &sf_bad, sf_red, sf_rex,
                                 crank, sf_pair ? 2 : 1);
  } else if constexpr (DF) {
    if (csize > 1) {
      // exactly one request per launch: the shared recursion, or a release
      const bool in_smem = cc == (c128*)dsm;
      const int op = (csize == 2 && in_smem) ? 1 : (csize == kFactorCluster && !in_smem) ? 2 : 0;
      double c0 = 0.0;
      if (op) c0 = lev_prologue<kFNT>(cc, aa, N);
      if (threadIdx.x == 0) lev_send_cmd(&cmd, csize, LevCmd{op, N, c0, cc, aa});
      cluster_barrier();
      if (op == 1) {
        cluster_levinson_df<kFNT>(cc, aa, N, c0, (float4*)red, &lev);
        lr = lev_epilogue<kFNT>(aa, N, &lev);
      } else if (op == 2) {
        cluster_levinson_global<kFNT, kFactorCluster>(cc, aa, N, c0, (float4*)red, &lev);
        float4* a4 = reinterpret_cast<float4*>(aa);
        for (int i = threadIdx.x; i < N; i += kFNT) {  // other SMs stored parts of a: read through L2
          const float4 v = __ldcg(a4 + i);
          aa[i] = mk(to_d(re_of(v)), to_d(im_of(v)));
        }
        __syncthreads();
        lr.status = lev.status;
        lr.delta_last = lev.delta;
        lr.logdet = lev.logdet;
      } else {
        lr = block_levinson_df<kFNT>(cc, aa, N, (float4*)red, &lev);
      }
    } else {
      lr = block_levinson_df<kFNT>(cc, aa, N, (float4*)red, &lev);
    }
  } else {
    lr = block_levinson<kFNT>(cc, aa, N, red, &lev);
  }
  c128* rho = rho_out + d.y_off;
  c128* x = x_out + d.y_off;
  if (lead && !lr.status) {
    for (int n = threadIdx.x; n < N; n += kFNT) rho[n] = conj(aa[N - 1 - n]);
    block_fft<kFNT, double>([=] __device__(int i) { return i < N ? yv[i] : zero<double>(); }, Yf, bufs[4], log2M2,
                            false, tw);
  }
  const int tr = sf_pair ? crank : 0, ts = sf_pair ? 2 : 1;  // the pair shares the transforms below
  if (sf_pair) {
    // the second block learns whether they run, and delta_{N-1} (in its
    // sf_rex[2..4], words the recursion's own hand-over does not use)
    if (lead && threadIdx.x == 0) {
      st_cluster_u32(&sf_rex[2], 1u, lr.status ? 0u : 1u);
      st_cluster_u32(&sf_rex[3], 1u, (unsigned)__double2loint(lr.delta_last));
      st_cluster_u32(&sf_rex[4], 1u, (unsigned)__double2hiint(lr.delta_last));
    }
    cluster_barrier();  // rho and Y = FFT(y) complete
    if (!lead) {
      lr.status = sf_rex[2] ? 0 : 1;
      lr.delta_last = __hiloint2double(sf_rex[4], sf_rex[3]);
    }
  }
  if (lr.status) {
    if (lead) {
      if (threadIdx.x == 0) { status[b] = 4; delta_out[b] = 0.0; }
      for (int n = threadIdx.x; n < N; n += kFNT) { rho[n] = zero<double>(); x[n] = zero<double>(); }
    }
    return;
  }
  // double-float transforms (Gohberg-Semencul apply and the omega_s
  // correlation) when the table exists, else FP64
  bool dft = false;
  if constexpr (DF) dft = tab.twdf != nullptr;
  if (dft && sf_pair) team_gs_apply<kFNT>(PolDF{tab.twdf, tab.log2max}, rho, Yf, x, N, log2M2, lr.delta_last, bufs, tr, ts);
  else if (dft) block_gs_apply_df<kFNT>(rho, Yf, x, N, log2M2, lr.delta_last, bufs, TwiddlesDF{tab.twdf, tab.log2max});
  else  // FP64: the same transforms as block_gs_apply on the batched FFT, one block or shared by a pair
    team_gs_apply<kFNT>(Pol64{tab.tw64, tab.log2max}, rho, Yf, x, N, log2M2, lr.delta_last, bufs, tr, ts);
  // Diagonal sums of C^{-1} (Sec. III-C, Appendix B):
  //   omega_s(i) = (1/d) sum_q [(q-c) + (q+i-c)] rho_q conj(rho_{q+i}),  |i| < N,
  // two cross-correlations; with P = FFT(rho) (still in bufs[0] after the
  // Gohberg-Semencul apply) and Pw = FFT((n-c) rho_n):
  //   omega_s(i) = IFFT(2 Re(Pw conj(P)))(-i) / (d M2).
  {
    const double cen = 0.5 * (double)(N - 2);
    const double sc = 1.0 / (lr.delta_last * (double)(1 << log2M2));
    const int msk = (1 << log2M2) - 1;
    c128* om = omega_out + 2 * d.y_off;
    c64* om32 = omega32_out + 2 * d.y_off;
    if (dft) {
      // P = FFT(rho) left in bufs[0] (double-float) by the apply
      const float4* P = reinterpret_cast<const float4*>(bufs[0]);
      float4* Pw = reinterpret_cast<float4*>(bufs[1]);
      float4* G = reinterpret_cast<float4*>(bufs[2]);
      float4* T = reinterpret_cast<float4*>(bufs[4]);
      const PolDF Pd{tab.twdf, tab.log2max};
      const f2 cen2 = f2{(float)cen, 0.f};  // a half-integer below 2^24: exact
      // (pol_fft: the butterflies of block_fft_df, shared by a pair)
      pol_fft<kFNT, PolDF>(
          Pd, 1,
          [=] __device__(int, int i) {
            if (i >= N) return cf2_zero();
            const cf2 r = cf2_of(rho[i]);
            const f2 wi = sub_s(f2{(float)i, 0.f}, cen2);
            return cf2{mul_f(wi, r.re), mul_f(wi, r.im)};
          },
          Pw, T, log2M2, false, tr, ts);
      pol_fft<kFNT, PolDF>(
          Pd, 1,
          [=] __device__(int, int k) {
            const cf2 v = ld_cf2(Pw[k]) * conj(ld_cf2(P[k]));
            return cf2{f2{2.f * v.re.h, 2.f * v.re.l}, f2{0.f, 0.f}};
          },
          G, T, log2M2, true, tr, ts);
      if (!lead) return;
      for (int i = (int)threadIdx.x - (N - 1); i <= N - 1; i += kFNT) {
        const cf2 g = ld_cf2(G[(-i) & msk]);
        const c128 v = mk(sc * to_d(g.re), sc * to_d(g.im));
        om[i + N - 1] = v;
        om32[i + N - 1] = cvt<float>(v);
      }
    } else {
      const c128* P = bufs[0];
      c128* Pw = bufs[1];
      c128* G = bufs[2];
      const Pol64 P6{tab.tw64, tab.log2max};
      // (pol_fft: the butterflies of block_fft, shared by a pair)
      pol_fft<kFNT, Pol64>(
          P6, 1, [=] __device__(int, int i) { return i < N ? ((double)i - cen) * rho[i] : zero<double>(); },
          reinterpret_cast<float4*>(Pw), reinterpret_cast<float4*>(bufs[4]), log2M2, false, tr, ts);
      pol_fft<kFNT, Pol64>(
          P6, 1, [=] __device__(int, int k) { return mk(2.0 * (Pw[k] * conj(P[k])).re, 0.0); },
          reinterpret_cast<float4*>(G), reinterpret_cast<float4*>(bufs[4]), log2M2, true, tr, ts);
      if (!lead) return;
      for (int i = (int)threadIdx.x - (N - 1); i <= N - 1; i += kFNT) {
        const c128 v = sc * G[(-i) & msk];
        om[i + N - 1] = v;
        om32[i + N - 1] = cvt<float>(v);
      }
    }
    c64* x32 = x32_out + d.y_off;
    for (int n = threadIdx.x; n < N; n += kFNT) x32[n] = cvt<float>(x[n]);
    __syncthreads();
  }
  if (threadIdx.x == 0) { status[b] = 0; delta_out[b] = lr.delta_last; }
}

// ------------------------------------------------------------------ grid ---
// Grid outputs as five independent length-L transforms per instance:
//   job 0: Z = sum_i (1 - i/N) omega_s(i) e^{+j2pi i l/L} -> s = Re Z, s' = 2 pi N Im Z
//          (s and s'/(2 pi N) are real transforms of Hermitian sequences and
//          share one complex FFT; the 1/(2 pi N) keeps both parts the same size)
//   job 1: s'' = Re sum_i (-4 pi^2 i^2) omega_s(i) e^{+j2pi i l/L}
//   jobs 2-4: q^(a) = sum_n (-j 2 pi n)^a x_n e^{-j2pi n l/L}, a = 0, 1, 2
// (Sec. III-D: the grid vectors are FFTs; omega_s from the factor kernel.)
// A task is (instance, job, partner, aux): a paired s'' job also transforms a
// second instance of the same N and L in the imaginary part (both inputs
// Hermitian, both outputs real).  GridJob gives a task's input sequence and
// takes its outputs; the on-chip kernel (one block per task, L on chip) and
// the four-step kernels (L too large for one block) share it.
template <class T>
struct GridPtrs {
  T *q, *dq, *d2q, *s, *ds, *d2s;
};

template <class T>
__host__ __device__ constexpr int grid_mmax() { return sizeof(T) == 4 ? 16384 : 8192; }

template <class T>
struct GridJob {
  int N, L, job;
  bool pair;
  int64_t g, g2;
  const cx<T> *om, *om2, *x;
  T invN, fpp, tp, f;
  T *o0, *o1;
  // input sequence at l (the lag i = l mod L for the s jobs)
  __device__ __forceinline__ cx<T> in(int l) const {
    cx<T> v = zero<T>();
    if (job <= 1) {
      const int i = l < N ? l : l - L;
      if (i > -N && i < N) {
        const cx<T> o = om[i];
        const T fi = (T)i;
        if (job == 0) {
          v = ((T)1 - fi * invN) * o;
        } else {
          v = (fpp * fi * fi) * o;
          if (pair) v = v + mul_j((fpp * fi * fi) * om2[i]);
        }
      }
    } else if (l < N) {
      const T w = tp * (T)l;
      v = x[l];
      if (job == 3) v = mk(w * v.im, -w * v.re);  // -j w x
      if (job == 4) v = (-w * w) * v;
    }
    return v;
  }
  __device__ __forceinline__ void out(int l, cx<T> z) const {
    if (job >= 2) {
      ((cx<T>*)o0)[g + l] = z;
    } else {
      if (o0) o0[g + l] = z.re;
      if (o1) o1[(job == 0 ? g : g2) + l] = f * z.im;
    }
  }
  __device__ __forceinline__ bool inverse() const { return job <= 1; }
};

template <class T>
__device__ __forceinline__ GridJob<T> make_grid_job(const InstDesc* inst, int4 task, const cx<T>* omega_all,
                                                   const cx<T>* x_all, const GridPtrs<T>& out) {
  GridJob<T> J;
  const int b = task.x, b2 = task.z;
  const InstDesc d = inst[b];
  J.N = d.N;
  J.L = d.L;
  J.job = task.y;
  J.pair = b2 >= 0;
  J.g = d.g_off;
  J.g2 = b2 >= 0 ? inst[b2].g_off : 0;
  J.om = omega_all + 2 * d.y_off + (d.N - 1);  // om[i], |i| < N
  J.om2 = b2 >= 0 ? omega_all + 2 * inst[b2].y_off + (d.N - 1) : J.om;
  J.x = x_all + d.y_off;
  // scalars in the element type: the FP64 pipe is slow enough that a per-
  // thread FP64 division showed up in the profile
  J.invN = (T)1 / (T)d.N;
  J.fpp = (T)(-4.0 * kPi * kPi);
  J.tp = (T)kTwoPi;
  const int job = J.job;
  J.o0 = job == 0 ? out.s : job == 1 ? out.d2s : job == 2 ? out.q : job == 3 ? out.dq : out.d2q;
  J.o1 = job == 0 ? out.ds : (J.pair ? out.d2s : nullptr);
  J.f = job == 0 ? J.tp * (T)d.N : (T)1;
  return J;
}

// ------------------------------------------------------- grid (on chip) ---
// One block per task, the whole length-L FFT in shared memory
// (lse_fft_smem.cuh): the first pass reads the input through the task's
// generator and the last pass writes the outputs straight to global memory.
template <class T, int NT, bool R16>
__global__ void __launch_bounds__(NT)
    grid_fft_kernel(const InstDesc* inst, const cx<T>* omega_all, const cx<T>* x_all, Tables tab, GridPtrs<T> out,
                    const int4* tasks) {
  extern __shared__ __align__(16) char gsm[];
  const GridJob<T> J = make_grid_job<T>(inst, tasks[blockIdx.x], omega_all, x_all, out);
  const int log2L = ilog2((uint32_t)J.L);
  cx<T>* sm = (cx<T>*)gsm;
  cx<T>* tlo = sm + J.L + (J.L >> 4);
  cx<T>* thi = tlo + (1 << ((log2L + 1) >> 1));
  const cx<T>* gtw = (const cx<T>*)(sizeof(T) == 8 ? (const void*)tab.tw64 : (const void*)tab.tw32);
  const SmemTwiddles<T> tw = make_smem_twiddles<NT, T>(tlo, thi, log2L, gtw, tab.log2max);
  constexpr int MMAX = grid_mmax<T>();
  __syncthreads();  // twiddle tables
  smem_fft_run<NT, MMAX, R16, T>([&] __device__(int l) { return J.in(l); }, sm, log2L, J.inverse(), tw,
                                 [&] __device__(int l, cx<T> z) { J.out(l, z); });
}

// ----------------------------------------------------- grid (four-step) ---
// L too large for one block: L = L1 L2 (L1 = 2^ceil(p/2), L2 = 2^floor(p/2),
// L = 2^p), and with m = L2 n1 + n2, k = k1 + L1 k2 the transform is
//   Y[k1][n2] = W_L^{n2 k1} sum_{n1} x[L2 n1 + n2] W_{L1}^{n1 k1}   (columns)
//   X[k1 + L1 k2] = sum_{n2} Y[k1][n2] W_{L2}^{n2 k2}               (rows)
// (W = e^{-+j 2 pi / .}).  Y (one length-L buffer per task) lives in the
// workspace and stays in L2.  Each block transforms a few columns (or rows)
// at once in shared memory; loads and stores run over consecutive columns
// (rows) so that they coalesce.  Tasks of several sizes share a launch: a
// block past its task's extent returns.
constexpr int kG4Threads = 256;
constexpr int kG4SmemBytes = 64 * 1024;  // two ping-pong buffers

// sequences of length len a block transforms at once (count of them in all):
// up to 8, as shared memory allows, never more than there are
template <class T>
__host__ __device__ inline int g4_group(int len, int count) {
  int g = kG4SmemBytes / (2 * len * (int)sizeof(cx<T>));
  if (g > 8) g = 8;
  return g < count ? g : count;
}

// nb sequences of length 2^lg at a + f 2^lg, radix-4/2 Stockham between a and
// b; returns the buffer holding the result.
template <class T, int NT>
__device__ cx<T>* smem_batch_fft(cx<T>* a, cx<T>* b, int nb, int lg, bool inverse, const cx<T>* tw, int log2max) {
  const int n = 1 << lg;
  int len = n, s = 1, log2s = 0;
  cx<T>* in = a;
  cx<T>* out = b;
  while (len >= 4) {
    const int n4 = len >> 2;
    for (int t = threadIdx.x; t < (nb << (lg - 2)); t += NT) {
      const int f = t >> (lg - 2), tt = t & ((n >> 2) - 1);
      const int p = tt >> log2s, q = tt & (s - 1);
      const cx<T>* i0 = in + (size_t)f * n;
      cx<T>* o0 = out + (size_t)f * n;
      const cx<T> x0 = i0[q + s * p], x1 = i0[q + s * (p + n4)], x2 = i0[q + s * (p + 2 * n4)], x3 = i0[q + s * (p + 3 * n4)];
      const cx<T> apc = x0 + x2, amc = x0 - x2, bpd = x1 + x3, jbmd = mul_j(x1 - x3);
      const cx<T> y1 = inverse ? amc + jbmd : amc - jbmd;
      const cx<T> y3 = inverse ? amc - jbmd : amc + jbmd;
      const cx<T> y2 = apc - bpd;
      const int sh = log2max - lg;
      cx<T> w1 = tw[(size_t)(p * s) << sh], w2 = tw[(size_t)(2 * p * s) << sh], w3 = tw[(size_t)(3 * p * s) << sh];
      if (inverse) { w1 = conj(w1); w2 = conj(w2); w3 = conj(w3); }
      o0[q + s * (4 * p + 0)] = apc + bpd;
      o0[q + s * (4 * p + 1)] = w1 * y1;
      o0[q + s * (4 * p + 2)] = w2 * y2;
      o0[q + s * (4 * p + 3)] = w3 * y3;
    }
    __syncthreads();
    cx<T>* t2 = in; in = out; out = t2;
    len >>= 2; s <<= 2; log2s += 2;
  }
  if (len == 2) {
    for (int t = threadIdx.x; t < (nb << (lg - 1)); t += NT) {
      const int f = t >> (lg - 1), q = t & ((n >> 1) - 1);
      const cx<T>* i0 = in + (size_t)f * n;
      cx<T>* o0 = out + (size_t)f * n;
      const cx<T> x0 = i0[q], x1 = i0[q + s];
      o0[q] = x0 + x1;
      o0[q + s] = x0 - x1;
    }
    __syncthreads();
    cx<T>* t2 = in; in = out; out = t2;
  }
  return in;
}

__host__ __device__ inline void g4_split(int L, int& p1, int& p2) {
  const int p = ilog2((uint32_t)L);
  p1 = (p + 1) >> 1;
  p2 = p - p1;
}

// columns: block (cb, task) transforms columns n2 in [cb G, cb G + G)
template <class T>
__global__ void __launch_bounds__(kG4Threads)
    grid4_cols_kernel(const InstDesc* inst, const cx<T>* omega_all, const cx<T>* x_all, Tables tab, GridPtrs<T> out,
                      const int4* tasks, cx<T>* ws) {
  extern __shared__ __align__(16) char gsm[];
  const int4 task = tasks[blockIdx.y];
  const GridJob<T> J = make_grid_job<T>(inst, task, omega_all, x_all, out);
  int p1, p2;
  g4_split(J.L, p1, p2);
  const int L1 = 1 << p1, L2 = 1 << p2;
  const int G = g4_group<T>(L1, L2);
  const int c0 = blockIdx.x * G;
  if (c0 >= L2) return;
  cx<T>* a = (cx<T>*)gsm;
  cx<T>* b = a + (size_t)G * L1;
  for (int e = threadIdx.x; e < G * L1; e += kG4Threads) {
    const int n1 = e / G, f = e - n1 * G;
    a[(size_t)f * L1 + n1] = J.in(L2 * n1 + c0 + f);
  }
  __syncthreads();
  const cx<T>* tw = (const cx<T>*)(sizeof(T) == 8 ? (const void*)tab.tw64 : (const void*)tab.tw32);
  const bool inv = J.inverse();
  const cx<T>* r = smem_batch_fft<T, kG4Threads>(a, b, G, p1, inv, tw, tab.log2max);
  cx<T>* Y = ws + (int64_t)task.w * 1024;
  const int p = p1 + p2;
  const int sh = tab.log2max - p;
  const int msk = J.L - 1;
  for (int e = threadIdx.x; e < G * L1; e += kG4Threads) {
    const int k1 = e / G, f = e - k1 * G;
    const int n2 = c0 + f;
    cx<T> w = tw[(size_t)((n2 * k1) & msk) << sh];
    if (inv) w = conj(w);
    Y[(size_t)k1 * L2 + n2] = w * r[(size_t)f * L1 + k1];
  }
}

// rows: block (rb, task) transforms rows k1 in [rb G, rb G + G) and writes
// the outputs X[k1 + L1 k2]
template <class T>
__global__ void __launch_bounds__(kG4Threads)
    grid4_rows_kernel(const InstDesc* inst, const cx<T>* omega_all, const cx<T>* x_all, Tables tab, GridPtrs<T> out,
                      const int4* tasks, const cx<T>* ws) {
  extern __shared__ __align__(16) char gsm[];
  const int4 task = tasks[blockIdx.y];
  const GridJob<T> J = make_grid_job<T>(inst, task, omega_all, x_all, out);
  int p1, p2;
  g4_split(J.L, p1, p2);
  const int L1 = 1 << p1, L2 = 1 << p2;
  const int G = g4_group<T>(L2, L1);
  const int r0 = blockIdx.x * G;
  if (r0 >= L1) return;
  cx<T>* a = (cx<T>*)gsm;
  cx<T>* b = a + (size_t)G * L2;
  const cx<T>* Y = ws + (int64_t)task.w * 1024;
  for (int e = threadIdx.x; e < G * L2; e += kG4Threads) a[e] = Y[(size_t)r0 * L2 + e];
  __syncthreads();
  const cx<T>* tw = (const cx<T>*)(sizeof(T) == 8 ? (const void*)tab.tw64 : (const void*)tab.tw32);
  const cx<T>* r = smem_batch_fft<T, kG4Threads>(a, b, G, p2, J.inverse(), tw, tab.log2max);
  for (int e = threadIdx.x; e < G * L2; e += kG4Threads) {
    const int k2 = e / G, f = e - k2 * G;
    J.out(r0 + f + L1 * k2, r[(size_t)f * L2 + k2]);
  }
}

}  // namespace

size_t factor_workspace_bytes(int Nmax, int sf_min_n) {
  return factor_layout(Nmax, sf_min_n > 0 && Nmax >= sf_min_n).total;
}

template <bool DF>
static cudaError_t launch_factor_t(int sf_min_n, int Nmin, const float* y, const InstDesc* inst, int B, int Nmax,
                                   const double* theta,
                                   const double* gamma, const double* beta, const Tables& tab, void* ws,
                                   c128* rho_out, c128* x_out, c128* omega_out, c64* omega32_out, c64* x32_out,
                                   double* delta_out, int* status, bool allow_cluster, cudaStream_t stream) {
  const int smem = 200 * 1024;
  cudaError_t e = cudaFuncSetAttribute(factor_kernel<DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  // clusters (double-float): of two blocks when every recursion runs in
  // shared memory and the launch leaves a spare SM per instance; of
  // kFactorCluster blocks when some recursion is too large for shared memory
  // and the launch leaves the SMs for them
  int csize = 1, sf_pair = 0;
  const bool any_levinson = sf_min_n <= 0 || Nmin < sf_min_n || (DF && !tab.twdf);
  if (allow_cluster && !any_levinson) {  // pairs sharing the superfast recursions (every precision)
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && 2 * B <= sms) {
      csize = 2;
      sf_pair = 1;
    }
  } else if (DF && allow_cluster) {
    int S, H;
    first_column_split(Nmax, S, H);
    const size_t need = 2 * sizeof(c128) * (size_t)Nmax + sizeof(c128) * kFirstColumnChunk * (S + H);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
      if (need <= (size_t)smem) {
        if (2 * B <= sms) csize = 2;
      } else if (kFactorCluster * B <= sms) {
        csize = kFactorCluster;
      }
    }
  }
  const size_t wsb = factor_workspace_bytes(Nmax, sf_min_n);
  if (csize > 1) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(csize * B);
    lc.blockDim = dim3(factor_threads<DF>());
    lc.dynamicSmemBytes = smem;
    lc.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, factor_kernel<DF>, y, inst, Nmax, theta, gamma, beta, tab, (char*)ws, wsb, rho_out,
                              x_out, omega_out, omega32_out, x32_out, delta_out, status, csize, sf_min_n, sf_pair);
  }
  factor_kernel<DF><<<B, factor_threads<DF>(), smem, stream>>>(y, inst, Nmax, theta, gamma, beta, tab, (char*)ws, wsb,
                                                               rho_out, x_out, omega_out, omega32_out, x32_out,
                                                               delta_out, status, 1, sf_min_n, 0);
  return cudaGetLastError();
}

cudaError_t launch_factor(bool df, int sf_min_n, int Nmin, const float* y, const InstDesc* inst, int B, int Nmax,
                          const double* theta, const double* gamma, const double* beta, const Tables& tab, void* ws,
                          c128* rho_out, c128* x_out, c128* omega_out, c64* omega32_out, c64* x32_out,
                          double* delta_out, int* status, bool allow_cluster, cudaStream_t stream) {
  return df ? launch_factor_t<true>(sf_min_n, Nmin, y, inst, B, Nmax, theta, gamma, beta, tab, ws, rho_out, x_out,
                                    omega_out, omega32_out, x32_out, delta_out, status, allow_cluster, stream)
            : launch_factor_t<false>(sf_min_n, Nmin, y, inst, B, Nmax, theta, gamma, beta, tab, ws, rho_out, x_out,
                                     omega_out, omega32_out, x32_out, delta_out, status, allow_cluster, stream);
}

size_t grid_workspace_bytes(size_t ws_elems, bool f32) { return ws_elems * (f32 ? sizeof(c64) : sizeof(c128)); }

// Schedules of the grid FFT for grids that fit on chip: the on-chip kernel
// with (threads per block, radix-16 passes), or (threads 0) the four-step
// kernels.  The autotuner in lse_api.cu times them on the live batch and
// keeps the fastest per (element type, grid size).
static const GridVariant kGridVariants[] = {{256, true}, {512, true}, {1024, true}, {512, false}, {0, false}};
int grid_variant_count() { return (int)(sizeof(kGridVariants) / sizeof(kGridVariants[0])); }
GridVariant grid_variant(int i) { return kGridVariants[i]; }

template <class T, int NT, bool R16>
static cudaError_t launch_grid_fft_v(const InstDesc* inst, const int4* tasks, int ntasks, const cx<T>* omega,
                                     const cx<T>* x, const Tables& tab, int Lmax, const GridPtrs<T>& o,
                                     cudaStream_t stream) {
  const int smem = (int)smem_fft_bytes(ilog2((uint32_t)Lmax), sizeof(cx<T>));
  cudaError_t e = cudaFuncSetAttribute(grid_fft_kernel<T, NT, R16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  grid_fft_kernel<T, NT, R16><<<ntasks, NT, smem, stream>>>(inst, omega, x, tab, o, tasks);
  return cudaGetLastError();
}

template <class T>
static cudaError_t launch_grid_fft(int variant, const InstDesc* inst, const int4* tasks, int ntasks,
                                   const cx<T>* omega, const cx<T>* x, const Tables& tab, int Lmax, void* q, void* dq,
                                   void* d2q, void* s, void* ds, void* d2s, cudaStream_t stream) {
  if (!ntasks) return cudaSuccess;
  const GridPtrs<T> o{(T*)q, (T*)dq, (T*)d2q, (T*)s, (T*)ds, (T*)d2s};
  switch (variant) {
    case 0: return launch_grid_fft_v<T, 256, true>(inst, tasks, ntasks, omega, x, tab, Lmax, o, stream);
    case 1: return launch_grid_fft_v<T, 512, true>(inst, tasks, ntasks, omega, x, tab, Lmax, o, stream);
    case 2: return launch_grid_fft_v<T, 1024, true>(inst, tasks, ntasks, omega, x, tab, Lmax, o, stream);
    default: return launch_grid_fft_v<T, 512, false>(inst, tasks, ntasks, omega, x, tab, Lmax, o, stream);
  }
}

// Tasks of a batch: one per (instance, output family); the s'' jobs of
// consecutive instances of equal N and L share one.  The tasks the on-chip
// kernel can take come first (n_small of them), then those whose L is too
// large for it.  Every task carries the offset of its four-step intermediate
// buffer (in units of 1024 elements) in .w (any task may run in four steps);
// *ws_elems receives the intermediate buffers' total size.
int grid_tasks(const InstDesc* inst, int B, bool f32, bool q, bool dq, bool d2q, bool s, bool ds, bool d2s, int4* out,
               int* n_small, size_t* ws_elems) {
  std::vector<int4> all;
  int pend = -1;  // an instance whose s'' job waits for a partner of the same N and L
  for (int b = 0; b < B; ++b) {
    if (s || ds) all.push_back(make_int4(b, 0, -1, 0));
    if (q) all.push_back(make_int4(b, 2, -1, 0));
    if (dq) all.push_back(make_int4(b, 3, -1, 0));
    if (d2q) all.push_back(make_int4(b, 4, -1, 0));
    if (d2s) {
      if (pend >= 0 && inst[pend].N == inst[b].N && inst[pend].L == inst[b].L) {
        all.push_back(make_int4(pend, 1, b, 0));
        pend = -1;
      } else {
        if (pend >= 0) all.push_back(make_int4(pend, 1, -1, 0));
        pend = b;
      }
    }
  }
  if (pend >= 0) all.push_back(make_int4(pend, 1, -1, 0));
  const int lim = f32 ? grid_mmax<float>() : grid_mmax<double>();
  int n = 0, ns = 0;
  size_t off = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (const int4& t : all) {
      const int L = inst[t.x].L;
      if ((L <= lim) != (pass == 0)) continue;
      out[n++] = make_int4(t.x, t.y, t.z, (int)(off / 1024));
      off += (size_t)(L < 1024 ? 1024 : L);
      ns += pass == 0;
    }
  *n_small = ns;
  *ws_elems = off;
  return n;
}

bool grid_on_chip(bool f32, int L) { return L <= (f32 ? grid_mmax<float>() : grid_mmax<double>()); }

template <class T>
static cudaError_t launch_grid4(const InstDesc* inst, const int4* tasks, int n, int Lmax, const cx<T>* omega,
                                const cx<T>* x, const Tables& tab, void* ws, const GridPtrs<T>& o,
                                cudaStream_t stream) {
  if (!n) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(grid4_cols_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kG4SmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(grid4_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kG4SmemBytes);
  if (e != cudaSuccess) return e;
  int p1, p2;
  g4_split(Lmax, p1, p2);
  // the largest L needs the most blocks per task (smaller L need no more)
  const int gx_cols = (1 << p2) / g4_group<T>(1 << p1, 1 << p2);
  const int gx_rows = (1 << p1) / g4_group<T>(1 << p2, 1 << p1);
  grid4_cols_kernel<T><<<dim3(gx_cols, n), kG4Threads, kG4SmemBytes, stream>>>(inst, omega, x, tab, o, tasks,
                                                                             (cx<T>*)ws);
  grid4_rows_kernel<T><<<dim3(gx_rows, n), kG4Threads, kG4SmemBytes, stream>>>(inst, omega, x, tab, o, tasks,
                                                                             (const cx<T>*)ws);
  return cudaGetLastError();
}

cudaError_t launch_grid(int variant, bool f32, const InstDesc* inst, int Lmax_small, int Lmax_large, const c128* omega,
                        const c128* x, const c64* omega32, const c64* x32, const Tables& tab, void* ws,
                        const int4* tasks, int n_small, int n_large, void* q, void* dq, void* d2q, void* s, void* ds,
                        void* d2s, cudaStream_t stream) {
  cudaError_t e = cudaSuccess;
  if (n_small && kGridVariants[variant].threads == 0) {  // everything in four steps
    n_large += n_small;
    Lmax_large = Lmax_large > Lmax_small ? Lmax_large : Lmax_small;
    n_small = 0;
  }
  if (n_small)
    e = f32 ? launch_grid_fft<float>(variant, inst, tasks, n_small, omega32, x32, tab, Lmax_small, q, dq, d2q, s, ds,
                                     d2s, stream)
            : launch_grid_fft<double>(variant, inst, tasks, n_small, omega, x, tab, Lmax_small, q, dq, d2q, s, ds,
                                      d2s, stream);
  if (e != cudaSuccess || !n_large) return e;
  if (f32)
    return launch_grid4<float>(inst, tasks + n_small, n_large, Lmax_large, omega32, x32, tab, ws,
                               GridPtrs<float>{(float*)q, (float*)dq, (float*)d2q, (float*)s, (float*)ds, (float*)d2s},
                               stream);
  return launch_grid4<double>(inst, tasks + n_small, n_large, Lmax_large, omega, x, tab, ws,
                              GridPtrs<double>{(double*)q, (double*)dq, (double*)d2q, (double*)s, (double*)ds,
                                               (double*)d2s},
                              stream);
}

}  // namespace lse
