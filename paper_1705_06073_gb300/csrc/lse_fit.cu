// lse_fit.cu -- persistent fit kernel: one thread block runs the whole
// block-coordinate-descent estimator (Sec. II-D, II-E of Hansen, Fleury,
// Rao, "Superfast Line Spectral Estimation") for one instance at a time,
// pulling instances from a device work counter, with every model evaluation
// done by the superfast route of Sec. III (superfast Schur or Levinson
// recursion for the Gohberg-Semencul generators, FFT convolutions, FFT grid,
// direct or non-uniform-FFT off-grid sums).  A batch that leaves a spare SM
// per instance runs as thread-block clusters: the first block of each
// cluster runs the estimator and the other blocks only take their share of
// the work it hands over (the superfast recursion's global-memory FFT passes,
// its refinement and the Gohberg-Semencul applies, on every precision path;
// on the double-float path also the Levinson recursion).
//
// Readings of the paper (the same ones the CPU oracle follows):
//  - (theta, gamma) update: one per-component diagonal Newton step with the
//    diagonal Hessian of eqs. (derivative2) (non-positive entries replaced by
//    (50N)^2 and gamma^-2, Sec. II-C1), step cut to 0.99 of the distance at
//    which a gamma would reach 0, Armijo backtracking (c = 1e-4, <= 30
//    halvings) on ln|C| + y^H C^{-1} y; theta modulo 1.
//  - step 4 runs <= max_inner iterations and stops after the iteration whose
//    squared Newton decrement is below N 1e-8 (that iteration takes no step
//    but still checks deactivation).
//  - deactivation removes, one at a time, the qualifying component whose
//    removal lowers eq. (obj) most (ties: earliest activated).
//  - gamma-bar is the mean active gamma, or the candidate's own
//    eq. (activate_gamma) value when no component is active.
//  - approximate activation runs in outer iterations 1..approx_iters while it
//    activates something; candidates are cyclic local minima
//    (strict on the left) with Delta L <= Delta L_min / 5 < 0, visited in
//    ascending Delta L; a pass that activates nothing falls through to exact
//    activation, which the later iterations use.
//  - eps_beta = 1e-12 ||y||^2/N, eps_L = 2^-52, K_max = N, termination when
//    the objective changes by less than N 1e-7 over an outer iteration.
//
// The file builds as several translation units, so that the three kernel
// instantiations compile in parallel: LSE_FIT_UNIT = 0, 1, 2 holds the
// launch of fit_kernel<PREC> for that precision, 3 the host code; left
// undefined, one unit holds everything.
#include <cfloat>

#include "../../include/lse.h"
#include "lse_device.cuh"
#include "lse_df64.cuh"
#include "lse_internal.h"
#include "lse_nufft.cuh"
#include "lse_schur.cuh"

namespace lse {

namespace {

// threads per block (all precisions): 8 warps; for the double-float recursion,
// 256 measured slightly faster than 512 at N = 4096 (fewer copies of the
// per-order reduction and reflection-coefficient work that every warp does).
template <int PREC>
__host__ __device__ constexpr int threads_for() { return 256; }
constexpr int kSmemBytes = 200 * 1024;
constexpr double kEpsL = 2.220446049250313e-16;
constexpr int kST_OK = 0, kST_NUMERIC = 4, kST_NOTCONV = 5;
// blocks per cluster for recursions too large for shared memory
constexpr int kBigCluster = 8;
// smallest N that uses the superfast Schur recursion by default
constexpr int kSuperfastMinN = 64;
// fewest frequencies whose off-grid sums go through the non-uniform FFT by default
constexpr int kNufftMinK = 32;

// whether the recursion's c and a (2N complex doubles) and the first-column
// tables fit in the block's dynamic shared memory
__host__ __device__ inline bool lev_in_smem(int N) {
  int S, H;
  first_column_split(N, S, H);
  const size_t tab_bytes = sizeof(c128) * kFirstColumnChunk * (S + H);
  return (2 * sizeof(c128) * (size_t)N + tab_bytes) <= (size_t)kSmemBytes;
}

// the superfast recursion's shared-memory part: after the first-column
// tables of an instance of N samples, with the largest short-run length that fits
__device__ inline void superfast_smem(char* dsm, int N, float4*& smem, int& lsm) {
  int S, H;
  first_column_split(N, S, H);
  const size_t tb = (sizeof(c128) * kFirstColumnChunk * (S + H) + 255) & ~size_t(255);
  smem = reinterpret_cast<float4*>(dsm + tb);
  lsm = schur_pick_lsm(kSmemBytes - tb);
}

template <int kNT>
struct FitShared {
  c128 red[kNT];
  MinLoc ml[kNT / 32];
  double dred[kNT / 32];
  LevShared lev;
  LevCmd cmd;  // cluster mode: request from the first block (lev_send_cmd)
  int sf_bad;  // superfast recursion: a pivot <= 0 or not finite
  // L-BFGS memory: pairs in a ring of kLbfgsJ, and whether a step awaits its gradient
  int lb_count, lb_head, lb_pending;
  double lb_rho[10], lb_a[10];
  int sf_rex[kNT / 32];
  // instance state (written by thread 0, read by all after a barrier)
  int inst, K, status, n_evals, n_grid, cand_count, flag;
  double beta, zeta, eps_beta, tau;
  double logdet, yCy, delta_last, f_cur, yy;
  double lpo, gbar;
  // grid decisions of the mixed paths: best FP32 candidates re-scored in FP64
  int ntop, sel;
  int top[32];
  double top_dl[32], top_s[32], top_Q[32];
};

// Per-block global workspace for an instance of size up to (Nmax, Lmax) with
// G snapshots (Sec. V; G = 1 for a single measurement vector).  Per-snapshot
// arrays hold snapshot g at g * (their per-snapshot stride).
template <class TG>
struct Work {
  int ny, nyf;      // per-snapshot strides: Nmax (y, x, x_df, 7 Nmax for sums), M2max (Yf)
  c128 *y, *c, *a, *rho, *x, *Yf;
  c128* buf[5];     // FFT buffers, M2max each (GS apply)
  cx<TG>* gbuf[4];  // grid FFT buffers, Lmax each
  double *theta, *gamma, *th_t, *ga_t, *dth, *dga;
  c128* sums;       // G x 7 Nmax off-grid sums (FP64 on every path)
  float4 *rho_df, *x_df;  // Nmax and G x Nmax: rho and x as double-float pairs (double-float path)
  double* dl;       // Lmax
  int* cand;        // Lmax
  double *cand_dl, *cand_s;  // Lmax: decision values of the candidates
  double* cand_Q;   // Lmax: sum over snapshots of |q|^2 at the candidates
  double* rs_theta;  // kRescore: frequencies being re-scored
  c128* rs_sums;     // G x 7 kRescore
  float4* sf;        // superfast Schur recursion (schur_workspace_elems(Nmax))
  double* gq2;       // Lmax: sum over snapshots of |q|^2 on the grid (G > 1)
  // L-BFGS (one base pointer; the arrays are derived where used): the pairs
  // S and Y (kLbfgsJ x 2 Nmax each), then 2 Nmax each of the gradient, the
  // diagonal Hessian, the pending step and its gradient
  double* lb;
  float4* nu;        // 2 (4 + 3G) M2max: transforms of the non-uniform FFT sums
  double* nfac64;    // Nmax: its deconvolution factors (FP64)
  float2* nfacdf;    // Nmax: the same as double-float pairs
  __device__ c128* yg(int g) const { return y + (size_t)g * ny; }
  __device__ c128* xg(int g) const { return x + (size_t)g * ny; }
  __device__ c128* Yfg(int g) const { return Yf + (size_t)g * nyf; }
  __device__ float4* xdfg(int g) const { return x_df + (size_t)g * ny; }
  __device__ c128* sumsg(int g) const { return sums + (size_t)g * 7 * ny; }
  __device__ c128* rssumsg(int g) const { return rs_sums + (size_t)g * 7 * kRescoreW; }
  static constexpr int kRescoreW = 1024;
};

constexpr int kRescore = Work<double>::kRescoreW;  // grid points re-scored in FP64 per batch
constexpr int kLbfgsJ = 10;  // L-BFGS pairs kept (Sec. II-C1: J = 10)

struct Layout {
  size_t off[48];
  size_t total;
};

template <class TG>
__host__ __device__ inline Layout make_layout(int Nmax, int Lmax, int G) {
  Layout L;
  const int M2 = 1 << ilog2(2u * (uint32_t)Nmax);
  size_t o = 0;
  int i = 0;
  auto put = [&](size_t bytes) { L.off[i++] = o; o += (bytes + 255) & ~size_t(255); };
  put(sizeof(c128) * (size_t)Nmax * G);                                 // y
  for (int j = 0; j < 3; ++j) put(sizeof(c128) * (size_t)Nmax);       // c a rho
  put(sizeof(c128) * (size_t)Nmax * G);                                 // x
  put(sizeof(c128) * (size_t)Nmax);                                     // (spare)
  put(sizeof(c128) * (size_t)M2 * G);                                   // Yf
  for (int j = 0; j < 5; ++j) put(sizeof(c128) * (size_t)M2);          // buf
  for (int j = 0; j < 4; ++j) put(sizeof(cx<TG>) * (size_t)Lmax);      // gbuf
  for (int j = 0; j < 6; ++j) put(sizeof(double) * (size_t)Nmax);      // theta..dga
  put(sizeof(c128) * 7 * (size_t)Nmax * G);                             // sums
  put(sizeof(float4) * (size_t)Nmax);                                   // rho_df
  put(sizeof(float4) * (size_t)Nmax * G);                               // x_df
  put(sizeof(double) * (size_t)Lmax);                                   // dl
  put(sizeof(int) * (size_t)Lmax);                                      // cand
  put(sizeof(double) * (size_t)Lmax);                                   // cand_dl
  put(sizeof(double) * (size_t)Lmax);                                   // cand_s
  put(sizeof(double) * (size_t)Lmax);                                   // cand_Q
  put(sizeof(double) * (size_t)kRescore);                               // rs_theta
  put(sizeof(c128) * 7 * (size_t)kRescore * G);                         // rs_sums
  put(sizeof(float4) * schur_workspace_elems(Nmax));                     // sf
  put(G > 1 ? sizeof(double) * (size_t)Lmax : 0);                       // gq2
  put(sizeof(double) * (2 * kLbfgsJ + 4) * 2 * (size_t)Nmax);           // lb
  put(sizeof(float4) * 2 * (size_t)(4 + 3 * G) * M2);                   // nu
  put(sizeof(double) * (size_t)Nmax);                                   // nfac64
  put(sizeof(float2) * (size_t)Nmax);                                   // nfacdf
  L.total = o;
  return L;
}

template <class TG>
__device__ Work<TG> carve(char* base, int Nmax, int Lmax, int G) {
  Layout L = make_layout<TG>(Nmax, Lmax, G);
  Work<TG> w;
  w.ny = Nmax;
  w.nyf = 1 << ilog2(2u * (uint32_t)Nmax);
  int i = 0;
  w.y = (c128*)(base + L.off[i++]);
  w.c = (c128*)(base + L.off[i++]);
  w.a = (c128*)(base + L.off[i++]);
  w.rho = (c128*)(base + L.off[i++]);
  w.x = (c128*)(base + L.off[i++]);
  i++;
  w.Yf = (c128*)(base + L.off[i++]);
  for (int j = 0; j < 5; ++j) w.buf[j] = (c128*)(base + L.off[i++]);
  for (int j = 0; j < 4; ++j) w.gbuf[j] = (cx<TG>*)(base + L.off[i++]);
  w.theta = (double*)(base + L.off[i++]);
  w.gamma = (double*)(base + L.off[i++]);
  w.th_t = (double*)(base + L.off[i++]);
  w.ga_t = (double*)(base + L.off[i++]);
  w.dth = (double*)(base + L.off[i++]);
  w.dga = (double*)(base + L.off[i++]);
  w.sums = (c128*)(base + L.off[i++]);
  w.rho_df = (float4*)(base + L.off[i++]);
  w.x_df = (float4*)(base + L.off[i++]);
  w.dl = (double*)(base + L.off[i++]);
  w.cand = (int*)(base + L.off[i++]);
  w.cand_dl = (double*)(base + L.off[i++]);
  w.cand_s = (double*)(base + L.off[i++]);
  w.cand_Q = (double*)(base + L.off[i++]);
  w.rs_theta = (double*)(base + L.off[i++]);
  w.rs_sums = (c128*)(base + L.off[i++]);
  w.sf = (float4*)(base + L.off[i++]);
  w.gq2 = (double*)(base + L.off[i++]);
  w.lb = (double*)(base + L.off[i++]);
  w.nu = (float4*)(base + L.off[i++]);
  w.nfac64 = (double*)(base + L.off[i++]);
  w.nfacdf = (float2*)(base + L.off[i++]);
  return w;
}

struct FitArgs {
  const float* y;
  const InstDesc* inst;
  int B, Nmax, Lmax;
  FitConfig cfg;
  Tables tab;
  FitOut out;
  char* ws;
  size_t ws_bytes;
  int* counter;
  int cluster;  // blocks per cluster: 1, 2 (shared-memory recursion) or kBigCluster (global)
};

__device__ __forceinline__ double prior_term(int K, int N, double zeta) {
  const double a = K ? K * log(zeta) : 0.0;
  const double b = (N - K) ? (N - K) * log1p(-zeta) : 0.0;
  return a + b;
}

__device__ __forceinline__ double log_prior_odds(double zeta) {
  return zeta <= 0.0 ? HUGE_VAL : log1p(-zeta) - log(zeta);
}

__device__ __forceinline__ double mod1(double t) {
  double r = t - floor(t);
  if (r >= 1.0) r -= 1.0;
  return r;
}

// PREC: 0 = FP64 throughout, 1 = FP32 grid (FP64 recursion), 2 = FP32 grid and
// double-float recursion on the FP32 pipes.
template <int PREC>
struct Fitter {
  static constexpr int kNT = threads_for<PREC>();
  using TG = typename std::conditional<PREC != 0, float, double>::type;
  FitShared<kNT>* sh;
  char* dsm;  // dynamic shared memory
  Work<TG> w;
  const FitArgs* A;
  int N, L, log2L, log2M2;
  int G;      // snapshots of the instance (Sec. V); 1 for a single measurement vector
  double Gd;  // G as a double
  bool lev_smem;
  c128 *lev_c, *lev_a, *tables;
  float4* sf_smem;  // superfast recursion: its shared-memory part (after the tables)
  int sf_lsm;
  Twiddles<double> tw64;
  Twiddles<TG> twg;

  // ---------------------------------------------------------------- eval ---
  // One evaluation of the model at (theta, gamma, beta): ln|C|, y^H C^{-1} y,
  // rho, x = C^{-1} y and (optionally) the off-grid sums.  Returns 0 or 1
  // (Levinson breakdown).
  __device__ int evaluate(const double* th, const double* ga, int K, bool want_sums) {
    const double beta = sh->beta;
    if constexpr (PREC == 2) block_first_column_df<kNT>(lev_c, th, ga, K, beta, N, tables);
    else block_first_column<kNT>(lev_c, th, ga, K, beta, N, tables);
    LevResult lr;
    if (superfast()) {
      // on a two-block cluster the recursion is shared with the other block
      // (c, a and w.sf are in global memory)
      const int cs = A->cluster == 2 ? 2 : 1;
      if (cs == 2) {
        if (threadIdx.x == 0) send_cmd(3, N, 0.0, lev_c, lev_a);
        cluster_barrier();
      }
      if constexpr (PREC == 2)
        lr = block_superfast<kNT>(PolDF{A->tab.twdf, A->tab.log2max}, lev_c, lev_a, N, w.sf, sf_smem, sf_lsm,
                                  &sh->sf_bad, sh->dred, sh->sf_rex, 0, cs);
      else
        lr = block_superfast<kNT>(Pol64{A->tab.tw64, A->tab.log2max}, lev_c, lev_a, N, w.sf, sf_smem, sf_lsm,
                                  &sh->sf_bad, sh->dred, sh->sf_rex, 0, cs);
    } else if constexpr (PREC == 2) {
      if (A->cluster == 2 && lev_smem) lr = cluster_levinson();
      else if (A->cluster == kBigCluster && !lev_smem) lr = cluster_levinson_big();
      else lr = block_levinson_df<kNT>(lev_c, lev_a, N, (float4*)sh->red, &sh->lev);
    } else {
      lr = block_levinson<kNT>(lev_c, lev_a, N, sh->red, &sh->lev);
    }
    if (threadIdx.x == 0) sh->n_evals++;
    if (!lr.status)
      for (int n = threadIdx.x; n < N; n += kNT) w.rho[n] = conj(lev_a[N - 1 - n]);
    // a recursion shared with the other block of the cluster: the
    // Gohberg-Semencul applies are shared too (the other block learns
    // whether they run, and delta_{N-1}, in its sf_rex[2..4], words that
    // the recursion's own hand-over does not use)
    const bool paired = A->cluster == 2 && superfast();
    if (paired) {
      if (threadIdx.x == 0) {
        st_cluster_u32(&sh->sf_rex[2], 1u, lr.status ? 0u : 1u);
        st_cluster_u32(&sh->sf_rex[3], 1u, (unsigned)__double2loint(lr.delta_last));
        st_cluster_u32(&sh->sf_rex[4], 1u, (unsigned)__double2hiint(lr.delta_last));
      }
      cluster_barrier();
    }
    if (lr.status) {
      __syncthreads();
      return 1;
    }
    __syncthreads();
    c128* bufs[5] = {w.buf[0], w.buf[1], w.buf[2], w.buf[3], w.buf[4]};
    double part = 0.0;
    for (int g = 0; g < G; ++g) {  // x_g = C^{-1} y_g, one Gohberg-Semencul apply per snapshot
      bool gs_done = false;
      if constexpr (PREC == 2) {  // double-float transforms when the table exists
        if (paired) {
          team_gs_apply<kNT>(PolDF{A->tab.twdf, A->tab.log2max}, w.rho, w.Yfg(g), w.xg(g), N, log2M2, lr.delta_last,
                             bufs, 0, 2);
          gs_done = true;
        } else if (A->tab.twdf) {
          block_gs_apply_df<kNT>(w.rho, w.Yfg(g), w.xg(g), N, log2M2, lr.delta_last, bufs,
                                 TwiddlesDF{A->tab.twdf, A->tab.log2max});
          gs_done = true;
        }
      }
      // FP64: the same transforms as block_gs_apply on the batched FFT, one
      // block or shared by a pair
      if (!gs_done)
        team_gs_apply<kNT>(Pol64{A->tab.tw64, A->tab.log2max}, w.rho, w.Yfg(g), w.xg(g), N, log2M2, lr.delta_last,
                           bufs, 0, paired ? 2 : 1);
      const c128 *yv = w.yg(g), *xv = w.xg(g);
      for (int n = threadIdx.x; n < N; n += kNT) part += (conj(yv[n]) * xv[n]).re;
    }
    const double yCy = block_sum<kNT>(part, sh->dred);
    if (threadIdx.x == 0) {
      sh->logdet = lr.logdet;
      sh->yCy = yCy;
      sh->delta_last = lr.delta_last;
      sh->f_cur = Gd * lr.logdet + yCy;  // eq. (obj); G ln|C| + sum_g y_g^H C^{-1} y_g for G snapshots (Sec. V)
    }
    __syncthreads();
    if constexpr (PREC == 2) {  // double-float copies for the sums
      for (int n = threadIdx.x; n < N; n += kNT) {
        const c128 r = w.rho[n];
        w.rho_df[n] = pack(to_f2(r.re), to_f2(r.im));
      }
      for (int g = 0; g < G; ++g) {
        const c128* xv = w.xg(g);
        float4* xd = w.xdfg(g);
        for (int n = threadIdx.x; n < N; n += kNT) {
          const c128 v = xv[n];
          xd[n] = pack(to_f2(v.re), to_f2(v.im));
        }
      }
      __syncthreads();
    }
    if (want_sums && K > 0) compute_sums(th, K);
    return 0;
  }

  // the superfast Schur recursion (lse_schur.cuh) for this instance?  On the
  // double-float path it needs the double-float twiddle table.
  __device__ bool superfast() const {
    if (A->cfg.sf_min_n <= 0 || N < A->cfg.sf_min_n) return false;
    if constexpr (PREC == 2) return A->tab.twdf != nullptr;
    return true;
  }

  // The recursion shared with the second block of the cluster: convert c,
  // hand the request over, run the orders together, and convert a back.
  __device__ LevResult cluster_levinson() {
    const double c0 = lev_prologue<kNT>(lev_c, lev_a, N);
    if (threadIdx.x == 0) send_cmd(1, N, c0, nullptr, nullptr);
    cluster_barrier();
    cluster_levinson_df<kNT>(lev_c, lev_a, N, c0, (float4*)sh->red, &sh->lev);
    return lev_epilogue<kNT>(lev_a, N, &sh->lev);
  }
  // A large instance: c and a stay in the workspace (global memory) and all
  // kBigCluster blocks of the cluster work on them.
  __device__ LevResult cluster_levinson_big() {
    const double c0 = lev_prologue<kNT>(lev_c, lev_a, N);
    if (threadIdx.x == 0) send_cmd(2, N, c0, lev_c, lev_a);
    cluster_barrier();
    cluster_levinson_global<kNT, kBigCluster>(lev_c, lev_a, N, c0, (float4*)sh->red, &sh->lev);
    // the other blocks' entries of a were stored on other SMs: read through L2
    float4* a4 = reinterpret_cast<float4*>(lev_a);
    for (int i = threadIdx.x; i < N; i += kNT) {
      const float4 v = __ldcg(a4 + i);
      lev_a[i] = mk(to_d(re_of(v)), to_d(im_of(v)));
    }
    __syncthreads();
    LevResult r;
    r.status = sh->lev.status;
    r.delta_last = sh->lev.delta;
    r.logdet = sh->lev.logdet;
    return r;
  }
  // write the request into every other block of the cluster
  __device__ void send_cmd(int op, int n, double c0, c128* c, c128* a) const {
    lev_send_cmd(&sh->cmd, A->cluster, LevCmd{op, n, c0, c, a});
  }

  // The Newton sums keep FP64 accuracy on every path (FP64, or double-float
  // on the FP32 pipes for the double-float path): in FP32 the gradient terms
  // (e.g. s - |q|^2 near convergence) cancel catastrophically, the Newton
  // directions disagree with the FP64 objective and the line search stalls.
  __device__ void compute_sums(const double* th, int K) {
    if (K <= 0) return;
    if (use_nufft(K)) {
      sums_nufft(th, K, w.sums, 7 * (size_t)w.ny);
      return;
    }
    for (int g = 0; g < G; ++g) {
      if constexpr (PREC == 2) block_active_sums_df<kNT>(w.rho_df, w.xdfg(g), th, K, N, w.sumsg(g));
      else block_active_sums<kNT, double>(w.rho, w.xg(g), th, K, N, w.sumsg(g));
    }
  }

  // the off-grid sums by the non-uniform FFT (lse_nufft.cuh) rather than
  // directly: for K frequencies at least cfg.nufft_min_k (0: never) and N >= 64
  __device__ bool use_nufft(int K) const { return A->cfg.nufft_min_k > 0 && K >= A->cfg.nufft_min_k && N >= 64; }

  __device__ void sums_nufft(const double* th, int K, c128* out, size_t stride) {
    if constexpr (PREC == 2) {
      block_sums_nufft<kNT>(PolDF{A->tab.twdf, A->tab.log2max}, w.rho_df, w.x_df, (size_t)w.ny, G, th, K, N,
                            log2M2, w.nfac64, w.nfacdf, w.nu, out, stride);
    } else {
      block_sums_nufft<kNT>(Pol64{A->tab.tw64, A->tab.log2max}, (const float4*)w.rho, (const float4*)w.x,
                            (size_t)w.ny, G, th, K, N, log2M2, w.nfac64, w.nfacdf, w.nu, out, stride);
    }
  }

  // ---------------------------------------------------------------- grid ---
  // q(theta_l), s(theta_l) on the L-point grid (Sec. III-D) from length-L FFTs:
  //   Q0 = FFT(rho), Q1 = FFT((n-c) rho_n), q = FFT(x), s = 2 Re(Q1 conj Q0)/delta
  // and Delta L(theta_l) of eq. (delta_L) with gamma-bar = gbar (K > 0) or the
  // point's own eq. (activate_gamma) value (K = 0).  Fills w.dl.
  __device__ void grid_delta(int K) {
    if (threadIdx.x == 0) sh->n_grid++;
    const double cen = 0.5 * (double)(N - 2);
    const c128* rho = w.rho;
    const c128* x = w.x;
    const int n_ = N;
    block_fft<kNT, TG>([=] __device__(int i) { return i < n_ ? cvt<TG>(rho[i]) : zero<TG>(); }, w.gbuf[0], w.gbuf[3],
                       log2L, false, twg);
    block_fft<kNT, TG>([=] __device__(int i) { return i < n_ ? cvt<TG>(((double)i - cen) * rho[i]) : zero<TG>(); },
                       w.gbuf[1], w.gbuf[3], log2L, false, twg);
    block_fft<kNT, TG>([=] __device__(int i) { return i < n_ ? cvt<TG>(x[i]) : zero<TG>(); }, w.gbuf[2], w.gbuf[3],
                       log2L, false, twg);
    if (G > 1) {  // Q = sum_g |q_g|^2 on the grid (Sec. V): one transform per snapshot
      for (int l = threadIdx.x; l < L; l += kNT) w.gq2[l] = norm2(cvt<double>(w.gbuf[2][l]));
      for (int g = 1; g < G; ++g) {
        __syncthreads();
        const c128* xv = w.xg(g);
        block_fft<kNT, TG>([=] __device__(int i) { return i < n_ ? cvt<TG>(xv[i]) : zero<TG>(); }, w.gbuf[2],
                           w.gbuf[3], log2L, false, twg);
        for (int l = threadIdx.x; l < L; l += kNT) w.gq2[l] += norm2(cvt<double>(w.gbuf[2][l]));
      }
      __syncthreads();
    }
    double gsum = 0.0;
    for (int k = threadIdx.x; k < K; k += kNT) gsum += w.gamma[k];
    gsum = block_sum<kNT>(gsum, sh->dred);
    const double gbar = K ? gsum / K : 0.0;
    const double lpo = log_prior_odds(sh->zeta);
    const double inv_delta = 1.0 / sh->delta_last;
    for (int l = threadIdx.x; l < L; l += kNT) {
      const c128 Q0 = cvt<double>(w.gbuf[0][l]), Q1 = cvt<double>(w.gbuf[1][l]);
      const double s = 2.0 * inv_delta * (Q1 * conj(Q0)).re;
      const double aq2 = G > 1 ? w.gq2[l] : norm2(cvt<double>(w.gbuf[2][l]));
      double gb = gbar;
      if (K == 0) gb = activate_gamma(aq2, s);
      w.dl[l] = Gd * log1p(gb * s) + lpo - gb * aq2 / (1.0 + gb * s);
    }
    if (threadIdx.x == 0) {
      sh->gbar = gbar;
      sh->lpo = lpo;
    }
    __syncthreads();
  }

  // s and Q = sum_g |q_g|^2 at grid point l (after grid_delta)
  __device__ void grid_point(int l, double& s, double& Q) const {
    const c128 Q0 = cvt<double>(w.gbuf[0][l]), Q1 = cvt<double>(w.gbuf[1][l]);
    Q = G > 1 ? w.gq2[l] : norm2(cvt<double>(w.gbuf[2][l]));
    s = 2.0 / sh->delta_last * (Q1 * conj(Q0)).re;
  }

  // gamma-hat of eq. (activate_gamma) from Q = sum_g |q_g|^2 and s: the
  // minimiser of the single-component objective, (Q/G - s)/s^2 for G
  // snapshots (Sec. V, eq. singlecomp-mmv)
  __device__ double activate_gamma(double Q, double s) const {
    const double Qg = Q / Gd;
    return Qg > s ? (Qg - s) / (s * s) : 0.0;
  }

  // eq. (activate_criterion) (tau = 0: eq. activate_derived) in the mean
  // per-snapshot form Q/(G s) > (1 + 1/(gb s)) (ln(1 + gb s) + ln((1-zeta)/zeta)/G) + tau
  __device__ bool activation_test(double Q, double s, double gb, double tau) const {
    const double gs = gb * s;
    const double rhs = (1.0 + 1.0 / gs) * (log1p(gs) + sh->lpo / Gd) + tau;
    return Q / Gd / s > rhs;
  }

  // Delta L of eq. (delta_L) (eq. singlecomp-mmv for G snapshots) from s and
  // Q = sum_g |q_g|^2 at a grid point.
  __device__ double delta_L(double s, double Q, int K) const {
    double gb = sh->gbar;
    if (K == 0) gb = activate_gamma(Q, s);
    return Gd * log1p(gb * s) + sh->lpo - gb * Q / (1.0 + gb * s);
  }

  // FP64 re-evaluation of s, q and Delta L at grid points ls[0..n), n <=
  // kRescore, by the direct off-grid sums of Sec. III-B/C on the FP64
  // generators (mixed paths: the FP32 grid only proposes candidates).
  __device__ void rescore(const int* ls, int n, double* dl_out, double* s_out, double* Q_out, int K) {
    for (int j = threadIdx.x; j < n; j += kNT) w.rs_theta[j] = (double)ls[j] / (double)L;
    __syncthreads();
    if (use_nufft(n)) {
      sums_nufft(w.rs_theta, n, w.rs_sums, 7 * (size_t)kRescore);
    } else {
      for (int g = 0; g < G; ++g) {
        if constexpr (PREC == 2) block_active_sums_df<kNT>(w.rho_df, w.xdfg(g), w.rs_theta, n, N, w.rssumsg(g));
        else block_active_sums<kNT, double>(w.rho, w.xg(g), w.rs_theta, n, N, w.rssumsg(g));
      }
    }
    const double inv_delta = 1.0 / sh->delta_last;
    for (int j = threadIdx.x; j < n; j += kNT) {
      const c128* sm = w.rs_sums + 7 * j;
      const double sv = 2.0 * inv_delta * (sm[1] * conj(sm[0])).re;
      double Qv = norm2(sm[4]);
      for (int g = 1; g < G; ++g) Qv += norm2(w.rssumsg(g)[7 * j + 4]);
      dl_out[j] = delta_L(sv, Qv, K);
      s_out[j] = sv;
      Q_out[j] = Qv;
    }
    __syncthreads();
  }

  // The 8 smallest grid values of Delta L and their cyclic neighbours into
  // sh->top (deduplicated), then re-scored in FP64 into sh->top_dl/s/q.
  __device__ void top_candidates(int K) {
    if (threadIdx.x == 0) sh->ntop = 0;
    __syncthreads();
    for (int r = 0; r < 8; ++r) {
      const int nt = sh->ntop;
      MinLoc m{HUGE_VAL, 0x7fffffff};
      for (int l = threadIdx.x; l < L; l += kNT) {
        bool taken = false;
        for (int j = 0; j < nt; ++j) taken |= (sh->top[j] == l);
        if (!taken) m = minloc(m, MinLoc{w.dl[l], l});
      }
      m = block_minloc<kNT>(m, sh->ml);
      if (m.i == 0x7fffffff) break;
      if (threadIdx.x == 0) {
        for (int dd = -1; dd <= 1; ++dd) {
          const int l2 = (m.i + dd + L) & (L - 1);
          bool have = false;
          for (int j = 0; j < sh->ntop; ++j) have |= (sh->top[j] == l2);
          if (!have && sh->ntop < 32) sh->top[sh->ntop++] = l2;
        }
      }
      __syncthreads();
    }
    rescore(sh->top, sh->ntop, sh->top_dl, sh->top_s, sh->top_Q, K);
  }

  // ---------------------------------------------------- exact activation ---
  __device__ int exact_activation(bool have_grid) {
    int n_act = 0;
    while (sh->K < N && sh->zeta > 0.0 && sh->status == kST_OK) {
      const int K = sh->K;
      if (!have_grid) grid_delta(K);
      have_grid = false;
      MinLoc m{HUGE_VAL, 0x7fffffff};
      if constexpr (PREC == 0) {
        for (int l = threadIdx.x; l < L; l += kNT) m = minloc(m, MinLoc{w.dl[l], l});
        m = block_minloc<kNT>(m, sh->ml);
      } else {
        top_candidates(K);
        for (int j = 0; j < sh->ntop; ++j) m = minloc(m, MinLoc{sh->top_dl[j], sh->top[j]});
      }
      if (threadIdx.x == 0) {
        double s = 0.0, Q = 0.0;
        // no grid point compares below +inf (every Delta L NaN or +inf): nothing to activate
        const bool found = m.i >= 0 && m.i < L;
        if (!found) {
        } else if constexpr (PREC == 0) {
          grid_point(m.i, s, Q);
        } else {
          int jm = 0;
          for (int j = 0; j < sh->ntop; ++j)
            if (sh->top[j] == m.i) jm = j;
          s = sh->top_s[jm];
          Q = sh->top_Q[jm];
        }
        const double ghat = found ? activate_gamma(Q, s) : 0.0;
        const double gb = K ? sh->gbar : ghat;
        const bool ok = found && ghat > 0.0 && m.v < -kEpsL && activation_test(Q, s, gb, sh->tau);
        sh->flag = ok;
        if (ok) {
          w.theta[K] = (double)m.i / (double)L;
          w.gamma[K] = ghat;
          sh->K = K + 1;
        }
      }
      __syncthreads();
      if (!sh->flag) break;
      ++n_act;
      if (evaluate(w.theta, w.gamma, sh->K, true)) {
        if (threadIdx.x == 0) sh->status = kST_NUMERIC;
        __syncthreads();
      }
    }
    return n_act;
  }

  // ---------------------------------------------- approximate activation ---
  // One pass of the scheme of Sec. II-E.  Returns the number activated.
  __device__ int approximate_activation(bool& grid_valid) {
    grid_valid = false;
    if (sh->zeta <= 0.0 || sh->K >= N) return 0;
    const int K0 = sh->K;
    grid_delta(K0);
    grid_valid = true;  // until a component is activated the grid stays that of the current state
    // global minimum of Delta L (equals the minimum over the local minima)
    double dlmin, slack = 0.0;
    if constexpr (PREC == 0) {
      MinLoc m{HUGE_VAL, 0x7fffffff};
      for (int l = threadIdx.x; l < L; l += kNT) m = minloc(m, MinLoc{w.dl[l], l});
      m = block_minloc<kNT>(m, sh->ml);
      dlmin = m.v;
    } else {
      top_candidates(K0);
      dlmin = HUGE_VAL;
      for (int j = 0; j < sh->ntop; ++j) dlmin = fmin(dlmin, sh->top_dl[j]);
    }
    if (!(dlmin < 0.0)) return 0;
    const double thr = dlmin / 5.0;
    if constexpr (PREC != 0) slack = 1e-3 * fabs(thr);  // FP32 grid error, candidates re-scored below
    if (threadIdx.x == 0) sh->cand_count = 0;
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += kNT) {
      const double v = w.dl[l];
      const double vl = w.dl[(l + L - 1) & (L - 1)], vr = w.dl[(l + 1) & (L - 1)];
      if (v < vl && v <= vr && v <= thr + slack) {
        const int slot = atomicAdd(&sh->cand_count, 1);
        w.cand[slot] = l;
      }
    }
    __syncthreads();
    const int nc = sh->cand_count;
    __syncthreads();
    // decision values of every candidate: the FP64 grid (FP64 path) or an FP64
    // re-evaluation (mixed paths)
    if constexpr (PREC == 0) {
      for (int j = threadIdx.x; j < nc; j += kNT) {
        const int l = w.cand[j];
        double sv, Qv;
        grid_point(l, sv, Qv);
        w.cand_dl[j] = w.dl[l];
        w.cand_s[j] = sv;
        w.cand_Q[j] = Qv;
      }
      __syncthreads();
    } else {
      for (int j0 = 0; j0 < nc; j0 += kRescore)
        rescore(w.cand + j0, min(kRescore, nc - j0), w.cand_dl + j0, w.cand_s + j0, w.cand_Q + j0, K0);
    }
    int n_act = 0;
    const double min_sep = 0.05 / (double)N;
    for (int it = 0; it < nc; ++it) {
      MinLoc b{HUGE_VAL, 0x7fffffff};
      for (int j = threadIdx.x; j < nc; j += kNT) {
        const int l = w.cand[j];
        if (l >= 0 && w.cand_dl[j] <= thr) b = minloc(b, MinLoc{w.cand_dl[j], l});
      }
      b = block_minloc<kNT>(b, sh->ml);
      if (b.i == 0x7fffffff) break;
      const int l = b.i;
      // strike it out and remember its slot
      for (int j = threadIdx.x; j < nc; j += kNT)
        if (w.cand[j] == l) {
          w.cand[j] = -1;
          sh->sel = j;
        }
      const double th = (double)l / (double)L;
      int close = 0;
      for (int k = threadIdx.x; k < sh->K; k += kNT) {
        double d = fabs(th - w.theta[k]);
        d = fmin(d, 1.0 - d);
        close |= (d < min_sep);
      }
      close = __syncthreads_or(close);
      if (threadIdx.x == 0 && !close && sh->K < N) {
        const double s = w.cand_s[sh->sel];
        const double Q = w.cand_Q[sh->sel];
        const double ghat = activate_gamma(Q, s);
        const double gb = K0 ? sh->gbar : ghat;
        if (ghat > 0.0 && activation_test(Q, s, gb, 0.0)) {
          w.theta[sh->K] = th;
          w.gamma[sh->K] = ghat;
          sh->K = sh->K + 1;
        }
      }
      __syncthreads();
    }
    n_act = sh->K - K0;
    if (n_act) {
      grid_valid = false;
      if (evaluate(w.theta, w.gamma, sh->K, true)) {
        if (threadIdx.x == 0) sh->status = kST_NUMERIC;
        __syncthreads();
      }
    }
    return n_act;
  }

  // ------------------------------------------------------ Newton update ---
  // Returns the squared Newton decrement.
  __device__ double newton_iteration() {
    const int K = sh->K;
    const double inv_delta = 1.0 / sh->delta_last;
    const double h_theta_fb = (50.0 * N) * (50.0 * N);
    double dec = 0.0, slope = 0.0, amax = HUGE_VAL;
    for (int k = threadIdx.x; k < K; k += kNT) {
      const double g = w.gamma[k];
      Derivs d = objective_derivatives(component_vectors<double>(w.sums + 7 * k, inv_delta), g);
      for (int gi = 1; gi < G; ++gi) {  // Sec. V: the derivatives sum over snapshots
        const Derivs e = objective_derivatives(component_vectors<double>(w.sumsg(gi) + 7 * k, inv_delta), g);
        d.gt += e.gt;
        d.gg += e.gg;
        d.ht += e.ht;
        d.hg += e.hg;
      }
      const double ht = d.ht > 0.0 ? d.ht : h_theta_fb;
      const double hg = d.hg > 0.0 ? d.hg : 1.0 / (g * g);
      const double dt = -d.gt / ht, dg = -d.gg / hg;
      w.dth[k] = dt;
      w.dga[k] = dg;
      dec += d.gt * d.gt / ht + d.gg * d.gg / hg;
      slope += d.gt * dt + d.gg * dg;
      if (dg < 0.0) amax = fmin(amax, g / -dg);
    }
    dec = block_sum<kNT>(dec, sh->dred);
    slope = block_sum<kNT>(slope, sh->dred);
    MinLoc am{amax, 0};
    am = block_minloc<kNT>(am, sh->ml);
    if (dec < (double)(G * N) * 1e-8) return dec;
    double alpha = am.v < HUGE_VAL ? fmin(1.0, 0.99 * am.v) : 1.0;
    const double f0 = sh->f_cur;
    for (int j = 0; j < 31; ++j) {
      for (int k = threadIdx.x; k < K; k += kNT) {
        w.th_t[k] = mod1(w.theta[k] + alpha * w.dth[k]);
        w.ga_t[k] = w.gamma[k] + alpha * w.dga[k];
      }
      __syncthreads();
      const int bad = evaluate(w.th_t, w.ga_t, K, false);
      if (!bad && sh->f_cur <= f0 + 1e-4 * alpha * slope) {
        for (int k = threadIdx.x; k < K; k += kNT) {
          w.theta[k] = w.th_t[k];
          w.gamma[k] = w.ga_t[k];
        }
        __syncthreads();
        compute_sums(w.theta, K);
        return dec;
      }
      alpha *= 0.5;
    }
    // no step accepted: restore the evaluation of the current state
    if (evaluate(w.theta, w.gamma, K, true)) {
      if (threadIdx.x == 0) sh->status = kST_NUMERIC;
      __syncthreads();
    }
    return dec;
  }

  // ------------------------------------------------------------- L-BFGS ---
  __device__ double* lb_S() const { return w.lb; }
  __device__ double* lb_Y() const { return w.lb + (size_t)kLbfgsJ * 2 * A->Nmax; }
  __device__ double* lb_g() const { return w.lb + (size_t)(2 * kLbfgsJ) * 2 * A->Nmax; }
  __device__ double* lb_h() const { return w.lb + (size_t)(2 * kLbfgsJ + 1) * 2 * A->Nmax; }
  __device__ double* lb_ps() const { return w.lb + (size_t)(2 * kLbfgsJ + 2) * 2 * A->Nmax; }
  __device__ double* lb_pg() const { return w.lb + (size_t)(2 * kLbfgsJ + 3) * 2 * A->Nmax; }
  // The L-BFGS update of Sec. II-C1 (readings L1-L4 of the oracle): with the
  // gradient g and the diagonal Hessian h (2K entries, theta then gamma) in
  // lbg / lbh, first turn a pending step into a pair (kept when s.y > 0, at
  // most kLbfgsJ, the oldest overwritten), then d = -H g by the two-loop
  // recursion with H_0 = diag(1/h) into dth / dga; dec = g.H g, slope = g.d.
  __device__ double dot2(const double* a, const double* b, int n) {
    double p = 0.0;
    for (int i = threadIdx.x; i < n; i += kNT) p += a[i] * b[i];
    return block_sum<kNT>(p, sh->dred);
  }
  __device__ void lbfgs_reset() {
    if (threadIdx.x == 0) {
      sh->lb_count = 0;
      sh->lb_head = 0;
      sh->lb_pending = 0;
    }
    __syncthreads();
  }
  // one L-BFGS update of (theta, gamma): the step rule of newton_iteration
  // with the direction of lbfgs_direction; returns g.H g
  __device__ __noinline__ double lbfgs_iteration() {
    const int K = sh->K;
    const double inv_delta = 1.0 / sh->delta_last;
    const double h_theta_fb = (50.0 * N) * (50.0 * N);
    for (int k = threadIdx.x; k < K; k += kNT) {
      const double g = w.gamma[k];
      Derivs d = objective_derivatives(component_vectors<double>(w.sums + 7 * k, inv_delta), g);
      for (int gi = 1; gi < G; ++gi) {
        const Derivs e = objective_derivatives(component_vectors<double>(w.sumsg(gi) + 7 * k, inv_delta), g);
        d.gt += e.gt;
        d.gg += e.gg;
        d.ht += e.ht;
        d.hg += e.hg;
      }
      lb_g()[k] = d.gt;
      lb_g()[K + k] = d.gg;
      lb_h()[k] = d.ht > 0.0 ? d.ht : h_theta_fb;
      lb_h()[K + k] = d.hg > 0.0 ? d.hg : 1.0 / (g * g);
    }
    double dec, slope;
    lbfgs_direction(K, dec, slope);
    double amax = HUGE_VAL;
    for (int k = threadIdx.x; k < K; k += kNT)
      if (w.dga[k] < 0.0) amax = fmin(amax, w.gamma[k] / -w.dga[k]);
    MinLoc am{amax, 0};
    am = block_minloc<kNT>(am, sh->ml);
    if (dec < (double)(G * N) * 1e-8) return dec;
    double alpha = am.v < HUGE_VAL ? fmin(1.0, 0.99 * am.v) : 1.0;
    const double f0 = sh->f_cur;
    for (int j = 0; j < 31; ++j) {
      for (int k = threadIdx.x; k < K; k += kNT) {
        w.th_t[k] = mod1(w.theta[k] + alpha * w.dth[k]);
        w.ga_t[k] = w.gamma[k] + alpha * w.dga[k];
      }
      __syncthreads();
      const int bad = evaluate(w.th_t, w.ga_t, K, false);
      if (!bad && sh->f_cur <= f0 + 1e-4 * alpha * slope) {
        for (int k = threadIdx.x; k < K; k += kNT) {
          w.theta[k] = w.th_t[k];
          w.gamma[k] = w.ga_t[k];
          // the step and its gradient wait for the next gradient (a pair)
          lb_ps()[k] = alpha * w.dth[k];
          lb_ps()[K + k] = alpha * w.dga[k];
          lb_pg()[k] = lb_g()[k];
          lb_pg()[K + k] = lb_g()[K + k];
        }
        if (threadIdx.x == 0) sh->lb_pending = 1;
        __syncthreads();
        compute_sums(w.theta, K);
        return dec;
      }
      alpha *= 0.5;
    }
    if (evaluate(w.theta, w.gamma, K, true)) {
      if (threadIdx.x == 0) sh->status = kST_NUMERIC;
      __syncthreads();
    }
    return dec;
  }

  __device__ __noinline__ void lbfgs_direction(int K, double& dec, double& slope) {
    const int n = 2 * K;
    const size_t st = 2 * (size_t)A->Nmax;
    __syncthreads();
    if (sh->lb_pending) {
      const int slot = sh->lb_head;
      double* s_ = lb_S() + slot * st;
      double* y_ = lb_Y() + slot * st;
      for (int i = threadIdx.x; i < n; i += kNT) {
        s_[i] = lb_ps()[i];
        y_[i] = lb_g()[i] - lb_pg()[i];
      }
      __syncthreads();
      const double sy = dot2(s_, y_, n);
      if (threadIdx.x == 0) {
        sh->lb_pending = 0;
        if (sy > 0.0) {
          sh->lb_rho[slot] = 1.0 / sy;
          sh->lb_head = (slot + 1) % kLbfgsJ;
          sh->lb_count = min(sh->lb_count + 1, kLbfgsJ);
        }
      }
      __syncthreads();
    }
    const int cnt = sh->lb_count, head = sh->lb_head;
    // q = g (in lbps, free now), newest pair first
    double* q = lb_ps();
    for (int i = threadIdx.x; i < n; i += kNT) q[i] = lb_g()[i];
    __syncthreads();
    for (int t = 0; t < cnt; ++t) {
      const int slot = (head - 1 - t + kLbfgsJ) % kLbfgsJ;
      const double* s_ = lb_S() + slot * st;
      const double* y_ = lb_Y() + slot * st;
      const double a = sh->lb_rho[slot] * dot2(s_, q, n);
      if (threadIdx.x == 0) sh->lb_a[slot] = a;
      for (int i = threadIdx.x; i < n; i += kNT) q[i] -= a * y_[i];
      __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += kNT) q[i] /= lb_h()[i];
    __syncthreads();
    for (int t = cnt - 1; t >= 0; --t) {
      const int slot = (head - 1 - t + kLbfgsJ) % kLbfgsJ;
      const double* s_ = lb_S() + slot * st;
      const double* y_ = lb_Y() + slot * st;
      const double b = sh->lb_rho[slot] * dot2(y_, q, n);
      const double a = sh->lb_a[slot];
      for (int i = threadIdx.x; i < n; i += kNT) q[i] += (a - b) * s_[i];
      __syncthreads();
    }
    for (int k = threadIdx.x; k < K; k += kNT) {
      w.dth[k] = -q[k];
      w.dga[k] = -q[K + k];
    }
    dec = dot2(lb_g(), q, n);  // g.H g
    slope = -dec;
  }

  // ---------------------------------------------------------- deactivation ---
  __device__ void deactivation() {
    while (sh->K > 0 && sh->status == kST_OK) {
      const int K = sh->K;
      const double inv_delta = 1.0 / sh->delta_last;
      const double thr = log_prior_odds(sh->zeta);
      MinLoc m{HUGE_VAL, 0x7fffffff};
      for (int k = threadIdx.x; k < K; k += kNT) {
        const double g = w.gamma[k];
        const CompVec cv = component_vectors<double>(w.sums + 7 * k, inv_delta);
        const double den = 1.0 - g * cv.s;
        const double st = cv.s / den;
        double qq = norm2(cv.q);
        for (int gi = 1; gi < G; ++gi) qq += norm2(w.sumsg(gi)[7 * k + 4]);
        const double aq2 = qq / (den * den);
        const double stat = g * aq2 / (1.0 + g * st) - Gd * log1p(g * st);
        if (stat < thr) m = minloc(m, MinLoc{stat, k});
      }
      m = block_minloc<kNT>(m, sh->ml);
      if (m.i == 0x7fffffff) break;
      // stable removal of component m.i
      double th = 0.0, ga = 0.0;
      const int k = threadIdx.x;
      for (int base = 0; base < K; base += kNT) {
        const int kk = base + k;
        if (kk >= m.i && kk + 1 < K) {
          th = w.theta[kk + 1];
          ga = w.gamma[kk + 1];
        }
        __syncthreads();
        if (kk >= m.i && kk + 1 < K) {
          w.theta[kk] = th;
          w.gamma[kk] = ga;
        }
      }
      if (threadIdx.x == 0) sh->K = K - 1;
      __syncthreads();
      if (evaluate(w.theta, w.gamma, sh->K, true)) {
        if (threadIdx.x == 0) sh->status = kST_NUMERIC;
        __syncthreads();
      }
    }
  }

  // ---------------------------------------------------------------- run ---
  __device__ void run(int b) {
    const InstDesc d = A->inst[b];
    N = d.N;
    L = d.L;
    log2L = ilog2((uint32_t)L);
    log2M2 = ilog2(2u * (uint32_t)N);
    G = A->cfg.G;
    Gd = (double)G;
    double part = 0.0;
    for (int g = 0; g < G; ++g) {  // snapshot g of instance b at G y_off + g N (complex elements)
      const float* yin = A->y + 2 * ((int64_t)G * d.y_off + (int64_t)g * N);
      c128* yv = w.yg(g);
      for (int n = threadIdx.x; n < N; n += kNT) {
        const c128 v = mk((double)yin[2 * n], (double)yin[2 * n + 1]);
        yv[n] = v;
        part += norm2(v);
      }
    }
    const double yy = block_sum<kNT>(part, sh->dred);
    // Levinson arrays in shared memory when they fit and the Levinson
    // recursion runs; the superfast recursion uses the shared memory after
    // the first-column tables for its short runs instead
    const bool sf = superfast();
    lev_smem = !sf && lev_in_smem(N);
    if (lev_smem) {
      lev_c = (c128*)dsm;
      lev_a = lev_c + N;
      tables = lev_a + N;
    } else {
      lev_c = w.c;
      lev_a = w.a;
      tables = (c128*)dsm;
    }
    superfast_smem(dsm, N, sf_smem, sf_lsm);
    if (threadIdx.x == 0) {
      sh->yy = yy;
      sh->K = 0;
      sh->status = kST_OK;
      sh->n_evals = 0;
      sh->n_grid = 0;
      sh->beta = 0.01 * yy / (double)(G * N);
      sh->eps_beta = 1e-12 * yy / (double)(G * N);
      sh->zeta = 0.2;
      sh->tau = A->cfg.tau;
    }
    __syncthreads();
    FitOut o = A->out;
    const int ob = d.idx;  // result slot of this instance
    if (yy == 0.0) {  // degenerate: nothing to estimate
      if (threadIdx.x == 0) {
        o.K[ob] = 0; o.beta[ob] = 0.0; o.objective[ob] = 0.0; o.iters[ob] = 0; o.n_evals[ob] = 0; o.n_grid[ob] = 0;
        o.status[ob] = kST_OK;
      }
      __syncthreads();
      return;
    }
    if (A->cfg.nufft_min_k > 0 && N >= 64) nufft_factors<kNT>(N, 1 << log2M2, w.nfac64, w.nfacdf);
    const int n_ = N;
    for (int g = 0; g < G; ++g) {
      const c128* yv = w.yg(g);
      block_fft<kNT, double>([=] __device__(int i) { return i < n_ ? yv[i] : zero<double>(); }, w.Yfg(g), w.buf[4],
                             log2M2, false, tw64);
    }
    int st = evaluate(w.theta, w.gamma, 0, true);
    double L_prev = sh->f_cur - prior_term(0, N, sh->zeta);
    bool approx = A->cfg.approx_iters > 0;
    bool converged = false;
    int it = 0;
    if (st) {
      if (threadIdx.x == 0) sh->status = kST_NUMERIC;
      __syncthreads();
    }
    for (it = 1; it <= A->cfg.max_outer && sh->status == kST_OK; ++it) {
      // step 1: activation
      if (approx && it <= A->cfg.approx_iters) {
        bool grid_valid;
        const int n = approximate_activation(grid_valid);
        if (n == 0) {
          approx = false;
          exact_activation(grid_valid);
        }
      } else {
        exact_activation(false);
      }
      if (sh->status != kST_OK) break;
      // step 2: zeta (eq. zetaUpdate)
      // step 3: beta (eq. betaUpdate with the Woodbury forms of Sec. II-C3)
      {
        const int K = sh->K;
        const double inv_delta = 1.0 / sh->delta_last;
        double sg = 0.0, xx = 0.0;
        for (int k = threadIdx.x; k < K; k += kNT) {
          const c128* sm = w.sums + 7 * k;
          const c128 r1r0 = sm[1] * conj(sm[0]);
          sg += 2.0 * r1r0.re * inv_delta * w.gamma[k];
        }
        for (int g = 0; g < G; ++g) {
          const c128* xv = w.xg(g);
          for (int n = threadIdx.x; n < N; n += kNT) xx += norm2(xv[n]);
        }
        sg = block_sum<kNT>(sg, sh->dred);
        xx = block_sum<kNT>(xx, sh->dred);
        if (threadIdx.x == 0) {
          sh->zeta = fmin(0.5, (double)K / (double)N);
          const double b0 = sh->beta;
          // Sec. V: the residual term is the mean over snapshots
          sh->beta = fmax(sh->eps_beta, (b0 * sg + b0 * b0 * (xx / Gd)) / N);
        }
        __syncthreads();
        if (evaluate(w.theta, w.gamma, K, true)) {
          if (threadIdx.x == 0) sh->status = kST_NUMERIC;
          __syncthreads();
          break;
        }
      }
      // step 4 (the L-BFGS memory starts empty, and is emptied again when a
      // component is removed)
      if (A->cfg.lbfgs) lbfgs_reset();
      for (int inner = 0; inner < A->cfg.max_inner && sh->status == kST_OK; ++inner) {
        if (sh->K == 0) break;
        const double dec = A->cfg.lbfgs ? lbfgs_iteration() : newton_iteration();
        const int K_before = sh->K;
        deactivation();
        if (A->cfg.lbfgs && sh->K != K_before) lbfgs_reset();
        if (dec < (double)(G * N) * 1e-8) break;
      }
      if (sh->status != kST_OK) break;
      const double L_cur = sh->f_cur - prior_term(sh->K, N, sh->zeta);
      if (fabs(L_cur - L_prev) < (double)(G * N) * 1e-7) {
        converged = true;
        break;
      }
      L_prev = L_cur;
    }
    // ------------------------------------------------------------ output --
    const int K = sh->K;
    const int64_t ro = d.y_off;
    // rank sort by frequency (ties by index)
    for (int k = threadIdx.x; k < K; k += kNT) {
      const double t = w.theta[k];
      int r = 0;
      for (int j = 0; j < K; ++j) {
        const double u = w.theta[j];
        r += (u < t) || (u == t && j < k);
      }
      const double g = w.gamma[k];
      o.theta[ro + r] = t;
      o.gamma[ro + r] = g;
      for (int gi = 0; gi < G; ++gi)  // alpha^(g) = gamma q_g at G ro + g N (eq. bmu, Sec. V)
        o.alpha[(int64_t)G * ro + (int64_t)gi * N + r] = g * w.sumsg(gi)[7 * k + 4];
    }
    if (threadIdx.x == 0) {
      o.K[ob] = K;
      o.beta[ob] = sh->beta;
      o.objective[ob] = sh->f_cur - prior_term(K, N, sh->zeta);
      o.iters[ob] = min(it, A->cfg.max_outer);
      o.n_evals[ob] = sh->n_evals;
      o.n_grid[ob] = sh->n_grid;
      o.status[ob] = sh->status != kST_OK ? sh->status : (converged ? kST_OK : kST_NOTCONV);
    }
    __syncthreads();
  }
};

// The other blocks of a cluster: they wait for recursion requests from the
// first block and run their share of each (double-float path only): a
// Levinson recursion in shared memory (op 1) or global memory (op 2), or the
// global-memory FFT stages and the refinement of a superfast one (op 3).
template <int PREC, int kNT = threads_for<PREC>()>
__device__ void cluster_helper(FitShared<kNT>& sh, char* dsm, int csize, const FitArgs& args, int unit) {
  for (;;) {
    cluster_barrier();  // a request (or the end) is in sh.cmd
    const int op = sh.cmd.op, n = sh.cmd.N;
    const double c0 = sh.cmd.c0;
    bool lev = false;  // a Levinson request (double-float path only)
    if constexpr (PREC == 2) {
      if (op == 1 && csize == 2) {
        c128* c = reinterpret_cast<c128*>(dsm);
        c128* a = c + n;
        const unsigned src = cluster_addr(c, 0u);
        float4* c4 = reinterpret_cast<float4*>(c);
        for (int i = threadIdx.x; i < n; i += kNT) c4[i] = ld_cluster(src + 16u * (unsigned)i);
        __syncthreads();
        cluster_levinson_df<kNT>(c, a, n, c0, (float4*)sh.red, &sh.lev);
        lev = true;
      } else if (op == 2 && csize == kBigCluster) {
        cluster_levinson_global<kNT, kBigCluster>(sh.cmd.c, sh.cmd.a, n, c0, (float4*)sh.red, &sh.lev);
        lev = true;
      }
    }
    if (lev) {
      continue;
    } else if (op == 3 && csize == 2) {
      float4* smem;
      int lsm;
      superfast_smem(dsm, n, smem, lsm);
      using TG = typename Fitter<PREC>::TG;
      const Work<TG> w = carve<TG>(args.ws + (size_t)unit * args.ws_bytes, args.Nmax, args.Lmax, args.cfg.G);
      if constexpr (PREC == 2)
        block_superfast<kNT>(PolDF{args.tab.twdf, args.tab.log2max}, sh.cmd.c, sh.cmd.a, n, w.sf, smem, lsm,
                             &sh.sf_bad, sh.dred, sh.sf_rex, 1, 2);
      else
        block_superfast<kNT>(Pol64{args.tab.tw64, args.tab.log2max}, sh.cmd.c, sh.cmd.a, n, w.sf, smem, lsm,
                             &sh.sf_bad, sh.dred, sh.sf_rex, 1, 2);
      // then this block's share of the Gohberg-Semencul applies, if the
      // factorisation succeeded (the first block's words in sf_rex[2..4])
      cluster_barrier();
      if (sh.sf_rex[2]) {
        const double delta_last = __hiloint2double(sh.sf_rex[4], sh.sf_rex[3]);
        c128* bufs[5] = {w.buf[0], w.buf[1], w.buf[2], w.buf[3], w.buf[4]};
        const int log2M2 = ilog2(2u * (uint32_t)n);
        for (int g = 0; g < args.cfg.G; ++g) {
          if constexpr (PREC == 2)
            team_gs_apply<kNT>(PolDF{args.tab.twdf, args.tab.log2max}, w.rho, w.Yfg(g), w.xg(g), n, log2M2,
                               delta_last, bufs, 1, 2);
          else
            team_gs_apply<kNT>(Pol64{args.tab.tw64, args.tab.log2max}, w.rho, w.Yfg(g), w.xg(g), n, log2M2,
                               delta_last, bufs, 1, 2);
        }
      }
    } else {
      break;
    }
  }
}

template <int PREC>
__global__ void __launch_bounds__(threads_for<PREC>(), 1) fit_kernel(FitArgs args) {
  using TG = typename Fitter<PREC>::TG;
  __shared__ FitShared<threads_for<PREC>()> sh;
  extern __shared__ __align__(16) char dsm[];
  int unit = blockIdx.x;  // workspace index
  if (args.cluster) {
    cluster_barrier();  // both blocks running before any shared-memory store between them
    if (cluster_ctarank() != 0) {
      cluster_helper<PREC>(sh, dsm, args.cluster, args, (int)(blockIdx.x / args.cluster));
      return;
    }
    unit = blockIdx.x / args.cluster;
  }
  Fitter<PREC> F;
  F.sh = &sh;
  F.dsm = dsm;
  F.A = &args;
  F.w = carve<TG>(args.ws + (size_t)unit * args.ws_bytes, args.Nmax, args.Lmax, args.cfg.G);
  F.tw64 = Twiddles<double>{args.tab.tw64, args.tab.log2max};
  if constexpr (PREC != 0) F.twg = Twiddles<TG>{(const cx<TG>*)args.tab.tw32, args.tab.log2max};
  else F.twg = Twiddles<TG>{(const cx<TG>*)args.tab.tw64, args.tab.log2max};
  for (;;) {
    if (threadIdx.x == 0) sh.inst = atomicAdd(args.counter, 1);
    __syncthreads();
    const int b = sh.inst;
    __syncthreads();
    if (b >= args.B) break;
    F.run(b);
  }
  if (args.cluster) {  // release the other blocks
    if (threadIdx.x == 0) F.send_cmd(0, 0, 0.0, nullptr, nullptr);
    cluster_barrier();
  }
}

}  // namespace

#ifndef LSE_FIT_UNIT
#define LSE_FIT_UNIT 4
#endif

// launch of fit_kernel<PREC>; args is a FitArgs (a type local to each unit)
cudaError_t fit_launch_prec0(const void* args, int grid, cudaStream_t stream);
cudaError_t fit_launch_prec1(const void* args, int grid, cudaStream_t stream);
cudaError_t fit_launch_prec2(const void* args, int grid, cudaStream_t stream);

#if LSE_FIT_UNIT == 3 || LSE_FIT_UNIT == 4
int superfast_min_n(uint64_t flags) { return (flags & LSE_FLAG_LEVINSON) ? 0 : kSuperfastMinN; }
int nufft_min_k(uint64_t flags) { return (flags & LSE_FLAG_DIRECT_SUMS) ? 0 : kNufftMinK; }

size_t fit_workspace_bytes(int Nmax, int Lmax, int prec, int G) {
  return prec ? make_layout<float>(Nmax, Lmax, G).total : make_layout<double>(Nmax, Lmax, G).total;
}
int fit_smem_bytes() { return kSmemBytes; }
#endif

template <int PREC>
static cudaError_t launch_prec(const FitArgs& a, int grid, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(fit_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  if (a.cluster) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(a.cluster * grid);
    lc.blockDim = dim3(threads_for<PREC>());
    lc.dynamicSmemBytes = kSmemBytes;
    lc.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = a.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, fit_kernel<PREC>, a);
  }
  fit_kernel<PREC><<<grid, threads_for<PREC>(), kSmemBytes, stream>>>(a);
  return cudaGetLastError();
}

#if LSE_FIT_UNIT == 0 || LSE_FIT_UNIT == 4
cudaError_t fit_launch_prec0(const void* args, int grid, cudaStream_t stream) {
  return launch_prec<0>(*static_cast<const FitArgs*>(args), grid, stream);
}
#endif
#if LSE_FIT_UNIT == 1 || LSE_FIT_UNIT == 4
cudaError_t fit_launch_prec1(const void* args, int grid, cudaStream_t stream) {
  return launch_prec<1>(*static_cast<const FitArgs*>(args), grid, stream);
}
#endif
#if LSE_FIT_UNIT == 2 || LSE_FIT_UNIT == 4
cudaError_t fit_launch_prec2(const void* args, int grid, cudaStream_t stream) {
  return launch_prec<2>(*static_cast<const FitArgs*>(args), grid, stream);
}
#endif

#if LSE_FIT_UNIT == 3 || LSE_FIT_UNIT == 4
cudaError_t launch_fit(int prec, const float* y, const InstDesc* inst, int B, int Nmax, int Lmax,
                       const FitConfig& cfg, const Tables& tab, const FitOut& out, void* ws, int* counter, int grid,
                       cudaStream_t stream) {
  FitArgs a;
  a.y = y;
  a.inst = inst;
  a.B = B;
  a.Nmax = Nmax;
  a.Lmax = Lmax;
  a.cfg = cfg;
  a.tab = tab;
  a.out = out;
  a.ws = (char*)ws;
  a.ws_bytes = fit_workspace_bytes(Nmax, Lmax, prec, cfg.G);
  a.counter = counter;
  // Clusters (double-float path): of two blocks, sharing every recursion
  // through shared memory, when the batch leaves a spare SM per instance and
  // every instance's recursion fits in shared memory; of kBigCluster blocks,
  // sharing the recursions of the instances too large for shared memory
  // through global memory, when the batch leaves kBigCluster SMs per instance.
  // Instances that run the superfast recursion share its global-memory FFT
  // stages, its refinement and the Gohberg-Semencul applies with the second
  // block of a two-block cluster (every precision; on the FP64 and mixed
  // paths when every instance of the launch runs the superfast recursion).
  a.cluster = 0;
  const bool any_levinson = cfg.sf_min_n <= 0 || cfg.Nmin < cfg.sf_min_n || (prec == 2 && !tab.twdf);
  if (cfg.cluster && (prec == 2 || !any_levinson)) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
      if (!any_levinson || lev_in_smem(Nmax)) {
        if (2 * grid <= sms) a.cluster = 2;
      } else if (kBigCluster * grid <= sms) {
        a.cluster = kBigCluster;
      }
    }
  }
  switch (prec) {
    case 0: return fit_launch_prec0(&a, grid, stream);
    case 1: return fit_launch_prec1(&a, grid, stream);
    default: return fit_launch_prec2(&a, grid, stream);
  }
}
#endif

}  // namespace lse
