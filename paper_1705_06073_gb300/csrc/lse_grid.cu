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
//  grid_kernel    the length-L spectra of index-weighted generators and the
//                 pointwise combine.  With c = (N-2)/2 and
//                   Q_a = DFT_L((n-c)^a rho_n),  X_a = DFT_L(n^a x_n)
//                 the grid quantities are (Appendix B weights, centred)
//                   s   = (2/d) Re(Q1 Q0*)
//                   s'  = (4 pi/d) Im(Q2 Q0*)
//                   s'' = (8 pi^2/d) [Re(Q2 Q1*) - Re(Q3 Q0*)]
//                   q = X0,  q' = -j 2 pi X1,  q'' = -4 pi^2 X2
//                 (d = delta_{N-1}; DFT_L(v)(l) = sum_n v_n e^{-j 2 pi n l / L}).
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

// csize > 1 (double-float only): clusters of csize blocks, one instance per
// cluster; the first block does everything and the others join its Levinson
// recursion (csize 2: shared-memory copies; kFactorCluster: global memory,
// for an instance too large for shared memory), or are released.
template <bool DF>
__global__ void __launch_bounds__(factor_threads<DF>(), 1)
    factor_kernel(const float* y, const InstDesc* inst, int Nmax, const double* theta, const double* gamma,
                  const double* beta, Tables tab, char* ws, size_t ws_bytes, c128* rho_out, c128* x_out,
                  c128* omega_out, c64* omega32_out, c64* x32_out, double* delta_out, int* status, int csize,
                  int sf_min_n) {
  constexpr int kFNT = factor_threads<DF>();
  __shared__ c128 red[kFNT];
  __shared__ LevShared lev;
  __shared__ LevCmd cmd;
  __shared__ int sf_bad;
  __shared__ double sf_red[kFNT / 32];
  __shared__ int sf_rex[kFNT / 32];
  extern __shared__ __align__(16) char dsm[];
  int b = blockIdx.x;
  if constexpr (DF) {
    if (csize > 1) {
      cluster_barrier();  // every block running before any store between them
      if (cluster_ctarank() != 0) {
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
        return;
      }
      b = blockIdx.x / csize;
    }
  }
  const InstDesc d = inst[b];
  const int N = d.N;
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
  if constexpr (DF) block_first_column_df<kFNT>(cc, theta + d.k_off, gamma + d.k_off, d.K, beta[b], N, tables);
  else block_first_column<kFNT>(cc, theta + d.k_off, gamma + d.k_off, d.K, beta[b], N, tables);
  LevResult lr;
  if (sf) {
    // a cluster launch still owes its other blocks their release
    if (DF && csize > 1) {
      if (threadIdx.x == 0) lev_send_cmd(&cmd, csize, LevCmd{0, N, 0.0, cc, aa});
      cluster_barrier();
    }
    float4* sfw = (float4*)(base + FL.sf);
    const size_t tb = (tab_bytes + 255) & ~size_t(255);
    float4* sfs = reinterpret_cast<float4*>(dsm + tb);
    const int lsm = schur_pick_lsm(smem_cap - tb);
    if constexpr (DF)
      lr = block_superfast<kFNT>(PolDF{tab.twdf, tab.log2max}, cc, aa, N, sfw, sfs, lsm, &sf_bad, sf_red, sf_rex);
    else
      lr = block_superfast<kFNT>(Pol64{tab.tw64, tab.log2max}, cc, aa, N, sfw, sfs, lsm, &sf_bad, sf_red, sf_rex);
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
  if (lr.status) {
    if (threadIdx.x == 0) { status[b] = 4; delta_out[b] = 0.0; }
    for (int n = threadIdx.x; n < N; n += kFNT) { rho[n] = zero<double>(); x[n] = zero<double>(); }
    return;
  }
  for (int n = threadIdx.x; n < N; n += kFNT) rho[n] = conj(aa[N - 1 - n]);
  block_fft<kFNT, double>([=] __device__(int i) { return i < N ? yv[i] : zero<double>(); }, Yf, bufs[4], log2M2, false,
                          tw);
  // double-float transforms (Gohberg-Semencul apply and the omega_s
  // correlation) when the table exists, else FP64
  bool dft = false;
  if constexpr (DF) dft = tab.twdf != nullptr;
  if (dft) block_gs_apply_df<kFNT>(rho, Yf, x, N, log2M2, lr.delta_last, bufs, TwiddlesDF{tab.twdf, tab.log2max});
  else block_gs_apply<kFNT>(rho, Yf, x, N, log2M2, lr.delta_last, bufs, tw);
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
      const TwiddlesDF twd{tab.twdf, tab.log2max};
      const f2 cen2 = f2{(float)cen, 0.f};  // a half-integer below 2^24: exact
      block_fft_df<kFNT>(
          [=] __device__(int i) {
            if (i >= N) return cf2_zero();
            const cf2 r = cf2_of(rho[i]);
            const f2 wi = sub_s(f2{(float)i, 0.f}, cen2);
            return cf2{mul_f(wi, r.re), mul_f(wi, r.im)};
          },
          Pw, T, log2M2, false, twd);
      block_fft_df<kFNT>(
          [=] __device__(int k) {
            const cf2 v = ld_cf2(Pw[k]) * conj(ld_cf2(P[k]));
            return cf2{f2{2.f * v.re.h, 2.f * v.re.l}, f2{0.f, 0.f}};
          },
          G, T, log2M2, true, twd);
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
      block_fft<kFNT, double>([=] __device__(int i) { return i < N ? ((double)i - cen) * rho[i] : zero<double>(); },
                              Pw, bufs[4], log2M2, false, tw);
      block_fft<kFNT, double>([=] __device__(int k) { return mk(2.0 * (Pw[k] * conj(P[k])).re, 0.0); }, G, bufs[4],
                              log2M2, true, tw);
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
// One block per (instance, family): family 0 makes s, s', s'' from Q0..Q3,
// family 1 makes q, q', q'' from X0..X2.  Spectra are built with the block
// FFT in the workspace (L2-resident) and combined pointwise.
template <class T>
__global__ void __launch_bounds__(kFNT, 1)
    grid_kernel(const InstDesc* inst, const c128* rho_all, const c128* x_all, const double* delta, Tables tab,
                char* ws, const int64_t* ws_off, T* q, T* dq, T* d2q, T* s, T* ds, T* d2s) {
  const int b = blockIdx.x >> 1, fam = blockIdx.x & 1;
  const InstDesc d = inst[b];
  const int N = d.N, L = d.L, log2L = ilog2((uint32_t)L);
  const Twiddles<T> tw{(const cx<T>*)(sizeof(T) == 8 ? (const void*)tab.tw64 : (const void*)tab.tw32), tab.log2max};
  cx<T>* buf = (cx<T>*)(ws + ws_off[b] + (size_t)fam * 5 * L * sizeof(cx<T>));
  cx<T>* B[5];
  for (int j = 0; j < 5; ++j) B[j] = buf + (size_t)j * L;
  const int64_t g = d.g_off;
  if (fam == 0) {
    const c128* rho = rho_all + d.y_off;
    const double cen = 0.5 * (double)(N - 2);
    const double inv_d = 1.0 / delta[b];
    for (int a = 0; a < 4; ++a) {
      block_fft<kFNT, T>(
          [=] __device__(int i) {
            if (i >= N) return zero<T>();
            const double w = (double)i - cen;
            double p = 1.0;
            for (int e = 0; e < a; ++e) p *= w;
            return cvt<T>(p * rho[i]);
          },
          B[a], B[4], log2L, false, tw);
    }
    for (int l = threadIdx.x; l < L; l += kFNT) {
      const cx<T> Q0 = B[0][l], Q1 = B[1][l], Q2 = B[2][l], Q3 = B[3][l];
      const cx<T> q10 = Q1 * conj(Q0), q20 = Q2 * conj(Q0), q21 = Q2 * conj(Q1), q30 = Q3 * conj(Q0);
      if (s) s[g + l] = (T)(2.0 * inv_d) * q10.re;
      if (ds) ds[g + l] = (T)(4.0 * kPi * inv_d) * q20.im;
      if (d2s) d2s[g + l] = (T)(8.0 * kPi * kPi * inv_d) * (q21.re - q30.re);
    }
  } else {
    const c128* x = x_all + d.y_off;
    for (int a = 0; a < 3; ++a) {
      block_fft<kFNT, T>(
          [=] __device__(int i) {
            if (i >= N) return zero<T>();
            double p = 1.0;
            for (int e = 0; e < a; ++e) p *= (double)i;
            return cvt<T>(p * x[i]);
          },
          B[a], B[4], log2L, false, tw);
    }
    cx<T>* Q = (cx<T>*)q;
    cx<T>* DQ = (cx<T>*)dq;
    cx<T>* D2Q = (cx<T>*)d2q;
    for (int l = threadIdx.x; l < L; l += kFNT) {
      if (Q) Q[g + l] = B[0][l];
      if (DQ) DQ[g + l] = (T)(-kTwoPi) * mul_j(B[1][l]);
      if (D2Q) D2Q[g + l] = (T)(-4.0 * kPi * kPi) * B[2][l];
    }
  }
}


// ------------------------------------------------------- grid (on chip) ---
// Grid outputs as five independent length-L FFTs, each done by one block in
// shared memory (lse_fft_smem.cuh):
//   job 0: Z = sum_i (1 - i/N) omega_s(i) e^{+j2pi i l/L} -> s = Re Z, s' = 2 pi N Im Z
//          (s and s'/(2 pi N) are real transforms of Hermitian sequences and
//          share one complex FFT; the 1/(2 pi N) keeps both parts the same size)
//   job 1: s'' = Re sum_i (-4 pi^2 i^2) omega_s(i) e^{+j2pi i l/L}
//   jobs 2-4: q^(a) = sum_n (-j 2 pi n)^a x_n e^{-j2pi n l/L}, a = 0, 1, 2
// (Sec. III-D: the grid vectors are FFTs; omega_s from the factor kernel.)
template <class T>
struct GridPtrs {
  T *q, *dq, *d2q, *s, *ds, *d2s;
};

template <class T>
__host__ __device__ constexpr int grid_mmax() { return sizeof(T) == 4 ? 16384 : 8192; }

template <class T, int NT, bool R16>
__global__ void __launch_bounds__(NT)
    grid_fft_kernel(const InstDesc* inst, const cx<T>* omega_all, const cx<T>* x_all, Tables tab, GridPtrs<T> out,
                    const int4* tasks) {
  extern __shared__ __align__(16) char gsm[];
  // task: x = instance, y = job, z = partner instance of a paired s'' job (or -1)
  const int4 task = tasks[blockIdx.x];
  const int b = task.x, job = task.y, b2 = task.z;
  const InstDesc d = inst[b];
  const int N = d.N, L = d.L, log2L = ilog2((uint32_t)L);
  const int64_t g = d.g_off;
  cx<T>* sm = (cx<T>*)gsm;
  cx<T>* tlo = sm + L + (L >> 4);
  cx<T>* thi = tlo + (1 << ((log2L + 1) >> 1));
  const cx<T>* gtw = (const cx<T>*)(sizeof(T) == 8 ? (const void*)tab.tw64 : (const void*)tab.tw32);
  const SmemTwiddles<T> tw = make_smem_twiddles<NT, T>(tlo, thi, log2L, gtw, tab.log2max);
  constexpr int MMAX = grid_mmax<T>();
  // one FFT instantiation for every job (the job only changes the input
  // functor, the direction and the epilogue) keeps the kernel's code small
  const cx<T>* om = omega_all + 2 * d.y_off + (N - 1);  // om[i], |i| < N
  // a paired s'' job also transforms a second instance of the same N and L in
  // the imaginary part (both inputs are Hermitian, both outputs real)
  const cx<T>* om2 = b2 >= 0 ? omega_all + 2 * inst[b2].y_off + (N - 1) : om;
  const int64_t g2 = b2 >= 0 ? inst[b2].g_off : 0;
  const cx<T>* x = x_all + d.y_off;
  // scalars in the element type: the FP64 pipe is slow enough that a per-
  // thread FP64 division showed up in the profile
  const T invN = (T)1 / (T)N;
  const T fpp = (T)(-4.0 * kPi * kPi);
  const T tp = (T)kTwoPi;
  auto gen = [=] __device__(int l) {
    cx<T> v = zero<T>();
    if (job <= 1) {
      const int i = l < N ? l : l - L;  // lag stored at l = i mod L
      if (i > -N && i < N) {
        const cx<T> o = om[i];
        const T fi = (T)i;
        if (job == 0) {
          v = ((T)1 - fi * invN) * o;
        } else {
          v = (fpp * fi * fi) * o;
          if (b2 >= 0) v = v + mul_j((fpp * fi * fi) * om2[i]);
        }
      }
    } else if (l < N) {
      const T w = tp * (T)l;
      v = x[l];
      if (job == 3) v = mk(w * v.im, -w * v.re);  // -j w x
      if (job == 4) v = (-w * w) * v;
    }
    return v;
  };
  T* o0 = job == 0 ? out.s : job == 1 ? out.d2s : job == 2 ? out.q : job == 3 ? out.dq : out.d2q;
  T* o1 = job == 0 ? out.ds : (b2 >= 0 ? out.d2s : nullptr);
  const T f = job == 0 ? tp * (T)N : (T)1;
  const int64_t go = job == 0 ? g : g2;
  auto epi = [=] __device__(int l, cx<T> z) {
    if (job >= 2) {
      ((cx<T>*)o0)[g + l] = z;
    } else {
      if (o0) o0[g + l] = z.re;
      if (o1) o1[go + l] = f * z.im;
    }
  };
  __syncthreads();  // twiddle tables
  smem_fft_run<NT, MMAX, R16, T>(gen, sm, log2L, job <= 1, tw, epi);
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
  int csize = 1;
  // clusters serve the Levinson recursion only
  const bool any_levinson = sf_min_n <= 0 || Nmin < sf_min_n || !tab.twdf;
  if (DF && allow_cluster && any_levinson) {
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
                              x_out, omega_out, omega32_out, x32_out, delta_out, status, csize, sf_min_n);
  }
  factor_kernel<DF><<<B, factor_threads<DF>(), smem, stream>>>(y, inst, Nmax, theta, gamma, beta, tab, (char*)ws, wsb,
                                                               rho_out, x_out, omega_out, omega32_out, x32_out,
                                                               delta_out, status, 1, sf_min_n);
  return cudaGetLastError();
}

cudaError_t launch_factor(bool df, int sf_min_n, int Nmin, const float* y, const InstDesc* inst, int B, int Nmax,
                          const double* theta, const double* gamma, const double* beta, const Tables& tab, void* ws,
                          c128* rho_out, c128* x_out, c128* omega_out, c64* omega32_out, c64* x32_out,
                          double* delta_out, int* status, bool allow_cluster, cudaStream_t stream) {
  return df ? launch_factor_t<true>(sf_min_n, Nmin, y, inst, B, Nmax, theta, gamma, beta, tab, ws, rho_out, x_out,
                                    omega_out, omega32_out, x32_out, delta_out, status, allow_cluster, stream)
            : launch_factor_t<false>(sf_min_n, Nmin, y, inst, B, Nmax, theta, gamma, beta, tab, ws, rho_out, x_out,
                                     omega_out, omega32_out, x32_out, delta_out, status, false, stream);
}

size_t grid_workspace_bytes(int B, int64_t total_L, bool f32) {
  (void)B;
  return (size_t)total_L * 2 * 5 * (f32 ? sizeof(c64) : sizeof(c128));
}

// Schedules of the on-chip grid FFT: (threads per block, radix-16 passes).
// The autotuner in lse_api.cu times them on the live batch and keeps the
// fastest per (element type, grid size).
static const GridVariant kGridVariants[] = {{256, true}, {512, true}, {1024, true}, {512, false}};
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

int grid_tasks(const InstDesc* inst, int B, bool q, bool dq, bool d2q, bool s, bool ds, bool d2s, int4* out) {
  int n = 0;
  int pend = -1;  // an instance whose s'' job waits for a partner of the same N and L
  for (int b = 0; b < B; ++b) {
    if (s || ds) out[n++] = make_int4(b, 0, -1, 0);
    if (q) out[n++] = make_int4(b, 2, -1, 0);
    if (dq) out[n++] = make_int4(b, 3, -1, 0);
    if (d2q) out[n++] = make_int4(b, 4, -1, 0);
    if (d2s) {
      if (pend >= 0 && inst[pend].N == inst[b].N && inst[pend].L == inst[b].L) {
        out[n++] = make_int4(pend, 1, b, 0);
        pend = -1;
      } else {
        if (pend >= 0) out[n++] = make_int4(pend, 1, -1, 0);
        pend = b;
      }
    }
  }
  if (pend >= 0) out[n++] = make_int4(pend, 1, -1, 0);
  return n;
}

bool grid_on_chip(bool f32, int Lmax) { return Lmax <= (f32 ? grid_mmax<float>() : grid_mmax<double>()); }

cudaError_t launch_grid(int variant, bool f32, const InstDesc* inst, int B, int Lmax, const c128* rho, const c128* x,
                        const c128* omega, const c64* x32, const c64* omega32, const double* delta, const Tables& tab,
                        void* ws, const int64_t* ws_off, const int4* tasks, int ntasks, void* q, void* dq, void* d2q,
                        void* s, void* ds, void* d2s, cudaStream_t stream) {
  if (grid_on_chip(f32, Lmax))
    return f32 ? launch_grid_fft<float>(variant, inst, tasks, ntasks, omega32, x32, tab, Lmax, q, dq, d2q, s, ds, d2s,
                                        stream)
               : launch_grid_fft<double>(variant, inst, tasks, ntasks, omega, x, tab, Lmax, q, dq, d2q, s, ds, d2s,
                                         stream);
  // instance b's buffers start ws_off[b] bytes into ws
  char* base = (char*)ws;
  if (f32)
    grid_kernel<float><<<2 * B, kFNT, 0, stream>>>(inst, rho, x, delta, tab, base, ws_off, (float*)q, (float*)dq,
                                                   (float*)d2q, (float*)s, (float*)ds, (float*)d2s);
  else
    grid_kernel<double><<<2 * B, kFNT, 0, stream>>>(inst, rho, x, delta, tab, base, ws_off, (double*)q, (double*)dq,
                                                    (double*)d2q, (double*)s, (double*)ds, (double*)d2s);
  return cudaGetLastError();
}

}  // namespace lse
