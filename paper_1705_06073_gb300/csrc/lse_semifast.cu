// lse_semifast.cu -- kernels for incomplete observations (Sec. IV of Hansen,
// Fleury, Rao, "Superfast Line Spectral Estimation"), built on the semifast
// evaluation of lse_semifast.cuh:
//  semifast_kernel      one evaluation per instance (ln|C|, y^H C^{-1} y,
//                       eqs. (q)-(x) at the components, grid q and s);
//  semifast_fit_kernel  the estimator of Sec. II on the observed samples,
//                       every model evaluation done the semifast way, one
//                       persistent block per instance.
//
// Readings of the fit (the same as oracle/incomplete.py): those of the
// complete-data fit (lse_fit.cu), with M where the paper counts observations
// (K_max = M, zeta = K/M, beta over M, the M 1e-7 and M 1e-8 thresholds of
// Sec. II-D, eps_beta and the initial beta over M) and N where it measures
// frequency resolution ((50N)^2, 0.05/N).  The grid values are computed at
// FP64-class precision on both paths (FP64, or double-float), so grid
// decisions are taken on them directly.  The semifast kernels hold K <= 96
// components (the K x K factor is staged in shared memory for the grid), so
// activation stops at min(M, 96).
#include <vector>

#include "lse_internal.h"
#include "lse_semifast.cuh"

namespace lse {

namespace {

constexpr double kEpsLS = 2.220446049250313e-16;

// ----------------------------------------------------------- evaluation ---
struct SemiArgs {
  const float* y;
  const int* obs;
  const SemiDesc* inst;
  const double *theta, *gamma, *beta;
  Tables tab;
  char* ws;
  size_t ws_bytes;
  int Kmax, Nmax, Lmax;
  double* scal;  // [2B]: ln|C|, y^H C^{-1} y
  c128* vec;     // [7 sum K]
  void* qg;      // grid q (complex)
  void* sg;      // grid s (real)
  int f64_out;
  int* status;
};

template <class Pol>
__global__ void __launch_bounds__(kSNT, 1) semifast_kernel(SemiArgs a) {
  extern __shared__ __align__(16) char ssm[];
  __shared__ double red[kSNT / 32];
  __shared__ int bad;
  const SemiDesc d = a.inst[blockIdx.x];
  const int K = d.K;
  const double beta = a.beta[d.idx];
  SemiEval<Pol> E;
  E.P = semi_pol<Pol>(a.tab);
  E.carve(a.ws + (size_t)blockIdx.x * a.ws_bytes, semi_layout(a.Kmax, a.Nmax, a.Lmax));
  E.smem = ssm;
  E.red = red;
  E.bad = &bad;
  const bool grid = a.qg || a.sg;
  E.prepare(a.y + 2 * d.m_off, a.obs + d.m_off, d.M, d.N, d.L, grid);
  const double* th = a.theta + d.k_off;
  const double* ga = a.gamma + d.k_off;
  E.gram(th, K, true);
  E.factor(ga, K, beta);
  double logdet, yCy;
  E.scalars(ga, K, beta, logdet, yCy);
  E.vectors(K, beta, a.vec + 7 * d.k_off);
  if (threadIdx.x == 0) {
    a.scal[2 * d.idx] = logdet;
    a.scal[2 * d.idx + 1] = yCy;
    a.status[d.idx] = bad == 2 ? 1 : (bad ? 4 : 0);  // LSE_EINVAL: an observed index out of range
  }
  if (!grid) return;
  const bool f64o = a.f64_out;
  void* qg = a.qg;
  void* sg = a.sg;
  const int64_t g0 = d.g_off;
  E.grid(th, K, beta, [=] __device__(int l, double s, c128 q) {
    if (sg) {
      if (f64o) ((double*)sg)[g0 + l] = s;
      else ((float*)sg)[g0 + l] = (float)s;
    }
    if (qg) {
      if (f64o) ((c128*)qg)[g0 + l] = q;
      else ((c64*)qg)[g0 + l] = mk((float)q.re, (float)q.im);
    }
  });
}

// ------------------------------------------------------------------ fit ---
struct SemiFitLayout {
  SemiLayout S;
  size_t theta, gamma, th_t, ga_t, dth, dga, vec, dl, gs, gq, cand, total;
};

__host__ __device__ inline SemiFitLayout semi_fit_layout(int Kcap, int Nmax, int Lmax) {
  SemiFitLayout F;
  F.S = semi_layout(Kcap, Nmax, Lmax);
  size_t o = F.S.total;
  auto put = [&](size_t bytes) { size_t r = o; o += (bytes + 255) & ~size_t(255); return r; };
  const size_t K = (size_t)Kcap + 1;
  F.theta = put(sizeof(double) * K);
  F.gamma = put(sizeof(double) * K);
  F.th_t = put(sizeof(double) * K);
  F.ga_t = put(sizeof(double) * K);
  F.dth = put(sizeof(double) * K);
  F.dga = put(sizeof(double) * K);
  F.vec = put(sizeof(c128) * 7 * K);
  F.dl = put(sizeof(double) * (size_t)Lmax);
  F.gs = put(sizeof(double) * (size_t)Lmax);
  F.gq = put(sizeof(double) * (size_t)Lmax);
  F.cand = put(sizeof(int) * (size_t)Lmax);
  F.total = o;
  return F;
}

struct SemiFitArgs {
  const float* y;
  const int* obs;
  const SemiDesc* inst;
  int B, Kcap, Nmax, Lmax;
  FitConfig cfg;
  Tables tab;
  FitOut out;
  char* ws;
  size_t ws_bytes;
  int* counter;
};

struct SemiFitShared {
  double red[kSNT / 32];
  MinLoc ml[kSNT / 32];
  int bad, inst, K, status, n_evals, n_grid, flag, cand_count;
  double beta, zeta, eps_beta, tau, f_cur, lpo, gbar;
};

template <class Pol>
struct SemiFitter {
  SemiFitShared* sh;
  const SemiFitArgs* A;
  SemiEval<Pol> E;
  double *theta, *gamma, *th_t, *ga_t, *dth, *dga, *dl, *gs, *gq;
  c128* vec;
  int* cand;
  int M, N, L, Kcap;

  __device__ static double prior(int K, int Kmax, double zeta) {
    const double a = K ? K * log(zeta) : 0.0;
    const double b = (Kmax - K) ? (Kmax - K) * log1p(-zeta) : 0.0;
    return a + b;
  }
  __device__ static double lpo_of(double zeta) { return zeta <= 0.0 ? HUGE_VAL : log1p(-zeta) - log(zeta); }

  // ln|C| + y^H C^{-1} y at (th, ga) into sh->f_cur (and the vectors of eqs.
  // (q)-(x) when asked); returns 1 if Sigma^{-1} is not positive definite
  __device__ int evaluate(const double* th, const double* ga, int K, bool vectors, bool count = true) {
    if (threadIdx.x == 0) {
      if (count) sh->n_evals++;
      if (sh->bad == 1) sh->bad = 0;  // a failed trial state does not carry over
    }
    __syncthreads();
    E.gram(th, K, vectors);
    E.factor(ga, K, sh->beta);
    double logdet, yCy;
    E.scalars(ga, K, sh->beta, logdet, yCy);
    if (vectors) E.vectors(K, sh->beta, vec);
    const int bad = sh->bad;
    if (threadIdx.x == 0) sh->f_cur = logdet + yCy;
    __syncthreads();
    return bad ? 1 : 0;
  }
  __device__ void fail_numeric() {
    if (threadIdx.x == 0) sh->status = 4;
    __syncthreads();
  }

  // grid s, q and Delta L (eq. delta_L) with gamma-bar by reading R4
  __device__ void grid_delta(int K) {
    if (threadIdx.x == 0) sh->n_grid++;
    double gsum = 0.0;
    for (int k = threadIdx.x; k < K; k += kSNT) gsum += gamma[k];
    gsum = block_sum<kSNT>(gsum, sh->red);
    const double gbar = K ? gsum / K : 0.0;
    const double lpo = lpo_of(sh->zeta);
    double *dlp = dl, *gsp = gs, *gqp = gq;
    E.grid(theta, K, sh->beta, [=] __device__(int l, double s, c128 q) {
      const double aq2 = norm2(q);
      const double gb = K ? gbar : (aq2 > s ? (aq2 - s) / (s * s) : 0.0);
      dlp[l] = log1p(gb * s) + lpo - gb * aq2 / (1.0 + gb * s);
      gsp[l] = s;
      gqp[l] = aq2;
    });
    if (threadIdx.x == 0) {
      sh->gbar = gbar;
      sh->lpo = lpo;
    }
    __syncthreads();
  }

  __device__ int exact_activation(bool have_grid) {
    int n_act = 0;
    while (sh->K < Kcap && sh->zeta > 0.0 && sh->status == 0) {
      const int K = sh->K;
      if (!have_grid) grid_delta(K);
      have_grid = false;
      MinLoc m{HUGE_VAL, 0x7fffffff};
      for (int l = threadIdx.x; l < L; l += kSNT) m = minloc(m, MinLoc{dl[l], l});
      m = block_minloc<kSNT>(m, sh->ml);
      if (threadIdx.x == 0) {
        const bool found = m.i >= 0 && m.i < L;
        const double s = found ? gs[m.i] : 1.0, Q = found ? gq[m.i] : 0.0;
        const double ghat = Q > s ? (Q - s) / (s * s) : 0.0;
        const double gb = K ? sh->gbar : ghat;
        const double g_s = gb * s;
        const double rhs = (1.0 + 1.0 / g_s) * (log1p(g_s) + sh->lpo) + sh->tau;
        const bool ok = found && ghat > 0.0 && m.v < -kEpsLS && Q / s > rhs;
        sh->flag = ok;
        if (ok) {
          theta[K] = (double)m.i / (double)L;
          gamma[K] = ghat;
          sh->K = K + 1;
        }
      }
      __syncthreads();
      if (!sh->flag) break;
      ++n_act;
      if (evaluate(theta, gamma, sh->K, true)) fail_numeric();
    }
    return n_act;
  }

  // one pass of Sec. II-E (reading R6)
  __device__ int approximate_activation(bool& grid_valid) {
    grid_valid = false;
    if (sh->zeta <= 0.0 || sh->K >= Kcap) return 0;
    const int K0 = sh->K;
    grid_delta(K0);
    grid_valid = true;
    MinLoc m{HUGE_VAL, 0x7fffffff};
    for (int l = threadIdx.x; l < L; l += kSNT) m = minloc(m, MinLoc{dl[l], l});
    m = block_minloc<kSNT>(m, sh->ml);
    const double dlmin = m.v;
    if (!(dlmin < 0.0)) return 0;
    const double thr = dlmin / 5.0;
    if (threadIdx.x == 0) sh->cand_count = 0;
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += kSNT) {
      const double v = dl[l];
      const double vl = dl[(l + L - 1) & (L - 1)], vr = dl[(l + 1) & (L - 1)];
      if (v < vl && v <= vr && v <= thr) cand[atomicAdd(&sh->cand_count, 1)] = l;
    }
    __syncthreads();
    const int nc = sh->cand_count;
    __syncthreads();
    const double min_sep = 0.05 / (double)N;
    for (int it = 0; it < nc; ++it) {
      MinLoc b{HUGE_VAL, 0x7fffffff};
      for (int j = threadIdx.x; j < nc; j += kSNT) {
        const int l = cand[j];
        if (l >= 0) b = minloc(b, MinLoc{dl[l], l});
      }
      b = block_minloc<kSNT>(b, sh->ml);
      if (b.i == 0x7fffffff) break;
      const int l = b.i;
      for (int j = threadIdx.x; j < nc; j += kSNT)
        if (cand[j] == l) cand[j] = -1;
      const double th = (double)l / (double)L;
      int close = 0;
      for (int k = threadIdx.x; k < sh->K; k += kSNT) {
        double dd = fabs(th - theta[k]);
        dd = fmin(dd, 1.0 - dd);
        close |= (dd < min_sep);
      }
      close = __syncthreads_or(close);
      if (threadIdx.x == 0 && !close && sh->K < Kcap) {
        const double s = gs[l], Q = gq[l];
        const double ghat = Q > s ? (Q - s) / (s * s) : 0.0;
        const double gb = K0 ? sh->gbar : ghat;
        const double g_s = gb * s;
        const double rhs = (1.0 + 1.0 / g_s) * (log1p(g_s) + sh->lpo);
        if (ghat > 0.0 && Q / s > rhs) {
          theta[sh->K] = th;
          gamma[sh->K] = ghat;
          sh->K = sh->K + 1;
        }
      }
      __syncthreads();
    }
    const int n_act = sh->K - K0;
    if (n_act) {
      grid_valid = false;
      if (evaluate(theta, gamma, sh->K, true)) fail_numeric();
    }
    return n_act;
  }

  __device__ CompVec comp(int k) const {
    CompVec c;
    const c128* v = vec + 7 * k;
    c.q = v[0];
    c.r = v[1];
    c.u = v[2];
    c.s = v[3].re;
    c.t = v[4];
    c.v = v[5];
    c.x = v[6].re;
    return c;
  }

  __device__ double newton_iteration() {
    const int K = sh->K;
    const double h_theta_fb = (50.0 * N) * (50.0 * N);
    double dec = 0.0, slope = 0.0, amax = HUGE_VAL;
    for (int k = threadIdx.x; k < K; k += kSNT) {
      const double g = gamma[k];
      const Derivs d = objective_derivatives(comp(k), g);
      const double ht = d.ht > 0.0 ? d.ht : h_theta_fb;
      const double hg = d.hg > 0.0 ? d.hg : 1.0 / (g * g);
      const double dt = -d.gt / ht, dg = -d.gg / hg;
      dth[k] = dt;
      dga[k] = dg;
      dec += d.gt * d.gt / ht + d.gg * d.gg / hg;
      slope += d.gt * dt + d.gg * dg;
      if (dg < 0.0) amax = fmin(amax, g / -dg);
    }
    dec = block_sum<kSNT>(dec, sh->red);
    slope = block_sum<kSNT>(slope, sh->red);
    MinLoc am{amax, 0};
    am = block_minloc<kSNT>(am, sh->ml);
    if (dec < (double)M * 1e-8) return dec;
    double alpha = am.v < HUGE_VAL ? fmin(1.0, 0.99 * am.v) : 1.0;
    const double f0 = sh->f_cur;
    for (int j = 0; j < 31; ++j) {
      for (int k = threadIdx.x; k < K; k += kSNT) {
        double t = theta[k] + alpha * dth[k];
        t -= floor(t);
        if (t >= 1.0) t -= 1.0;
        th_t[k] = t;
        ga_t[k] = gamma[k] + alpha * dga[k];
      }
      __syncthreads();
      const int bad = evaluate(th_t, ga_t, K, false);
      if (!bad && sh->f_cur <= f0 + 1e-4 * alpha * slope) {
        for (int k = threadIdx.x; k < K; k += kSNT) {
          theta[k] = th_t[k];
          gamma[k] = ga_t[k];
        }
        __syncthreads();
        if (evaluate(theta, gamma, K, true, false)) fail_numeric();  // the vectors at the accepted state
        return dec;
      }
      alpha *= 0.5;
    }
    if (evaluate(theta, gamma, K, true)) fail_numeric();  // restore the current state
    return dec;
  }

  __device__ void deactivation() {
    while (sh->K > 0 && sh->status == 0) {
      const int K = sh->K;
      const double thr = lpo_of(sh->zeta);
      MinLoc m{HUGE_VAL, 0x7fffffff};
      for (int k = threadIdx.x; k < K; k += kSNT) {
        const double g = gamma[k];
        const CompVec cv = comp(k);
        const double den = 1.0 - g * cv.s;
        const double st = cv.s / den;
        const double aq2 = norm2(cv.q) / (den * den);
        const double stat = g * aq2 / (1.0 + g * st) - log1p(g * st);
        if (stat < thr) m = minloc(m, MinLoc{stat, k});
      }
      m = block_minloc<kSNT>(m, sh->ml);
      if (m.i == 0x7fffffff) break;
      double t = 0.0, gg = 0.0;
      for (int base = 0; base < K; base += kSNT) {
        const int kk = base + threadIdx.x;
        if (kk >= m.i && kk + 1 < K) {
          t = theta[kk + 1];
          gg = gamma[kk + 1];
        }
        __syncthreads();
        if (kk >= m.i && kk + 1 < K) {
          theta[kk] = t;
          gamma[kk] = gg;
        }
      }
      if (threadIdx.x == 0) sh->K = K - 1;
      __syncthreads();
      if (evaluate(theta, gamma, sh->K, true)) fail_numeric();
    }
  }

  __device__ void run(int b) {
    const SemiDesc d = A->inst[b];
    M = d.M;
    N = d.N;
    L = d.L;
    Kcap = min(M, A->Kcap);
    E.prepare(A->y + 2 * d.m_off, A->obs + d.m_off, M, N, L, true);
    const double yy = E.yy;
    FitOut o = A->out;
    const int ob = d.idx;
    if (threadIdx.x == 0) {
      sh->K = 0;
      sh->status = sh->bad == 2 ? 1 : 0;
      sh->n_evals = 0;
      sh->n_grid = 0;
      sh->beta = 0.01 * yy / M;
      sh->eps_beta = 1e-12 * yy / M;
      sh->zeta = 0.2;
      sh->tau = A->cfg.tau;
    }
    __syncthreads();
    if (yy == 0.0 || sh->status) {  // degenerate (R11), or an index out of range
      if (threadIdx.x == 0) {
        o.K[ob] = 0; o.beta[ob] = 0.0; o.objective[ob] = 0.0; o.iters[ob] = 0; o.n_evals[ob] = 0; o.n_grid[ob] = 0;
        o.status[ob] = sh->status;
      }
      __syncthreads();
      return;
    }
    if (evaluate(theta, gamma, 0, true)) fail_numeric();
    double L_prev = sh->f_cur - prior(0, M, sh->zeta);
    bool approx = A->cfg.approx_iters > 0;
    bool converged = false;
    int it = 0;
    for (it = 1; it <= A->cfg.max_outer && sh->status == 0; ++it) {
      if (approx && it <= A->cfg.approx_iters) {
        bool grid_valid;
        if (approximate_activation(grid_valid) == 0) {
          approx = false;
          exact_activation(grid_valid);
        }
      } else {
        exact_activation(false);
      }
      if (sh->status) break;
      {  // zeta (eq. zetaUpdate) and beta (eq. betaUpdate, over M)
        const int K = sh->K;
        double sg = 0.0;
        for (int k = threadIdx.x; k < K; k += kSNT) sg += vec[7 * k + 3].re * gamma[k];
        sg = block_sum<kSNT>(sg, sh->red);
        const double xx = E.residual_norm2(K, sh->beta);
        if (threadIdx.x == 0) {
          sh->zeta = fmin(0.5, (double)K / (double)M);
          const double b0 = sh->beta;
          sh->beta = fmax(sh->eps_beta, (b0 * sg + b0 * b0 * xx) / M);
        }
        __syncthreads();
        if (evaluate(theta, gamma, K, true)) {
          fail_numeric();
          break;
        }
      }
      for (int inner = 0; inner < A->cfg.max_inner && sh->status == 0; ++inner) {
        if (sh->K == 0) break;
        const double dec = newton_iteration();
        deactivation();
        if (dec < (double)M * 1e-8) break;
      }
      if (sh->status) break;
      const double L_cur = sh->f_cur - prior(sh->K, M, sh->zeta);
      if (fabs(L_cur - L_prev) < (double)M * 1e-7) {
        converged = true;
        break;
      }
      L_prev = L_cur;
    }
    const int K = sh->K;
    const int64_t ro = d.m_off;
    for (int k = threadIdx.x; k < K; k += kSNT) {
      const double t = theta[k];
      int r = 0;
      for (int j = 0; j < K; ++j) {
        const double u = theta[j];
        r += (u < t) || (u == t && j < k);
      }
      o.theta[ro + r] = t;
      o.gamma[ro + r] = gamma[k];
      o.alpha[ro + r] = gamma[k] * vec[7 * k];
    }
    if (threadIdx.x == 0) {
      o.K[ob] = K;
      o.beta[ob] = sh->beta;
      o.objective[ob] = sh->f_cur - prior(K, M, sh->zeta);
      o.iters[ob] = min(it, A->cfg.max_outer);
      o.n_evals[ob] = sh->n_evals;
      o.n_grid[ob] = sh->n_grid;
      o.status[ob] = sh->status ? sh->status : (converged ? 0 : 5);
    }
    __syncthreads();
  }
};

template <class Pol>
__global__ void __launch_bounds__(kSNT, 1) semifast_fit_kernel(SemiFitArgs a) {
  extern __shared__ __align__(16) char ssm[];
  __shared__ SemiFitShared sh;
  const SemiFitLayout FL = semi_fit_layout(a.Kcap, a.Nmax, a.Lmax);
  char* base = a.ws + (size_t)blockIdx.x * a.ws_bytes;
  SemiFitter<Pol> F;
  F.sh = &sh;
  F.A = &a;
  F.E.P = semi_pol<Pol>(a.tab);
  F.E.carve(base, FL.S);
  F.E.smem = ssm;
  F.E.red = sh.red;
  F.E.bad = &sh.bad;
  F.theta = (double*)(base + FL.theta);
  F.gamma = (double*)(base + FL.gamma);
  F.th_t = (double*)(base + FL.th_t);
  F.ga_t = (double*)(base + FL.ga_t);
  F.dth = (double*)(base + FL.dth);
  F.dga = (double*)(base + FL.dga);
  F.vec = (c128*)(base + FL.vec);
  F.dl = (double*)(base + FL.dl);
  F.gs = (double*)(base + FL.gs);
  F.gq = (double*)(base + FL.gq);
  F.cand = (int*)(base + FL.cand);
  for (;;) {
    if (threadIdx.x == 0) sh.inst = atomicAdd(a.counter, 1);
    __syncthreads();
    const int b = sh.inst;
    __syncthreads();
    if (b >= a.B) break;
    F.run(b);
  }
}

}  // namespace

size_t semifast_workspace_bytes(int Kmax, int Nmax, int Lmax) { return semi_layout(Kmax, Nmax, Lmax).total; }
size_t semifast_smem_bytes(int Kmax, int r_max) { return semi_smem_bytes(Kmax, r_max); }
size_t semifast_fit_workspace_bytes(int Kcap, int Nmax, int Lmax) { return semi_fit_layout(Kcap, Nmax, Lmax).total; }

cudaError_t launch_semifast(bool df, const float* y, const int* obs, const SemiDesc* inst, int B, int Kmax, int Nmax,
                            int Lmax, const double* theta, const double* gamma, const double* beta, const Tables& tab,
                            void* ws, double* scal, c128* vec, void* qg, void* sg, bool f64_out, int* status,
                            size_t smem, cudaStream_t stream) {
  SemiArgs a;
  a.y = y;
  a.obs = obs;
  a.inst = inst;
  a.theta = theta;
  a.gamma = gamma;
  a.beta = beta;
  a.tab = tab;
  a.ws = (char*)ws;
  a.ws_bytes = semifast_workspace_bytes(Kmax, Nmax, Lmax);
  a.Kmax = Kmax;
  a.Nmax = Nmax;
  a.Lmax = Lmax;
  a.scal = scal;
  a.vec = vec;
  a.qg = qg;
  a.sg = sg;
  a.f64_out = f64_out ? 1 : 0;
  a.status = status;
  cudaError_t e;
  if (df) {
    e = cudaFuncSetAttribute(semifast_kernel<PolDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    semifast_kernel<PolDF><<<B, kSNT, smem, stream>>>(a);
  } else {
    e = cudaFuncSetAttribute(semifast_kernel<Pol64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    semifast_kernel<Pol64><<<B, kSNT, smem, stream>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_semifast_fit(bool df, const float* y, const int* obs, const SemiDesc* inst, int B, int Kcap,
                                int Nmax, int Lmax, const FitConfig& cfg, const Tables& tab, const FitOut& out,
                                void* ws, int* counter, int grid, size_t smem, cudaStream_t stream) {
  SemiFitArgs a;
  a.y = y;
  a.obs = obs;
  a.inst = inst;
  a.B = B;
  a.Kcap = Kcap;
  a.Nmax = Nmax;
  a.Lmax = Lmax;
  a.cfg = cfg;
  a.tab = tab;
  a.out = out;
  a.ws = (char*)ws;
  a.ws_bytes = semifast_fit_workspace_bytes(Kcap, Nmax, Lmax);
  a.counter = counter;
  cudaError_t e;
  if (df) {
    e = cudaFuncSetAttribute(semifast_fit_kernel<PolDF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    semifast_fit_kernel<PolDF><<<grid, kSNT, smem, stream>>>(a);
  } else {
    e = cudaFuncSetAttribute(semifast_fit_kernel<Pol64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    semifast_fit_kernel<Pol64><<<grid, kSNT, smem, stream>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace lse
