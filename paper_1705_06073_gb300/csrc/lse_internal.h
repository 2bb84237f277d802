// lse_internal.h -- host-side declarations shared by the translation units of
// the library (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/lse.h"
#include "lse_common.cuh"

struct lse_ctx;
// the stream a context enqueues on (lse_api.cu)
cudaStream_t lse_ctx_stream(lse_ctx* c);
// grow a context's device memory (fit workspace, twiddle tables, launch
// descriptors and their pinned staging) for fits of B instances up to
// (Nmax, Lmax), so that such fits allocate nothing; waits for the device
lse_status lse_ctx_reserve_fit(lse_ctx* c, int Nmax, int Lmax, int B);

namespace lse {

// One instance of a batched launch.
struct InstDesc {
  int64_t y_off;   // offset of y (complex elements) in the batch
  int32_t N;
  int32_t L;       // grid size (power of two >= 2N)
  int64_t k_off;   // eval-grid: offset of this instance's components; fit: unused
  int32_t K;       // eval-grid: number of components
  int32_t idx;     // fit: index of the instance's result slots (queue order may differ)
  int64_t g_off;   // eval-grid: offset of this instance's grid outputs
};

struct FitConfig {
  double tau;
  int max_outer, max_inner, approx_iters;
  int cluster;    // thread-block clusters allowed for the Levinson recursion (double-float path)
  int sf_min_n;   // instances with N >= sf_min_n use the superfast Schur recursion (0: none)
  int Nmin;       // smallest N of the launch
  int G = 1;      // snapshots per instance (multiple measurement vectors, Sec. V)
  int nufft_min_k = 0;  // off-grid sums at >= this many frequencies by the non-uniform FFT (0: never)
  int lbfgs = 0;        // step 4a by L-BFGS (Sec. II-C1) instead of diagonal Newton
};

// nufft_min_k for the lse_config flags (LSE_FLAG_DIRECT_SUMS: 0)
int nufft_min_k(uint64_t flags);

// Smallest N for which the superfast Schur recursion replaces the Levinson
// recursion, given the lse_config flags (LSE_FLAG_LEVINSON: never).
int superfast_min_n(uint64_t flags);

// Device outputs of the fit kernel (see lse_batch_out).
struct FitOut {
  double* theta;
  double* gamma;
  c128* alpha;
  int* K;
  double* beta;
  double* objective;
  int* iters;
  int* n_evals;
  int* n_grid;
  int* status;
};

struct Tables {
  const c128* tw64;
  const c64* tw32;
  int log2max;
  // the same table as double-float pairs {re.h, re.l, im.h, im.l}, or null
  // (then the double-float fit path applies the Gohberg-Semencul formula in FP64)
  const float4* twdf;
};

// Per-CTA workspace needed by the fit kernel for instances up to (Nmax, Lmax)
// with G snapshots each.
size_t fit_workspace_bytes(int Nmax, int Lmax, int prec, int G = 1);
int fit_smem_bytes();

// Launch the persistent fit kernel over B instances on `stream` with `grid`
// CTAs; `ws` holds grid * fit_workspace_bytes(Nmax, Lmax, prec) bytes and
// `counter` one zeroed int (work queue).
cudaError_t launch_fit(int prec, const float* y, const InstDesc* inst, int B, int Nmax, int Lmax, const FitConfig& cfg,
                       const Tables& tab, const FitOut& out, void* ws, int* counter, int grid, cudaStream_t stream);

// Eval-grid: per-instance factorisation (first column, Levinson, GS apply).
size_t factor_workspace_bytes(int Nmax, int sf_min_n);
cudaError_t launch_factor(bool df, int sf_min_n, int Nmin, const float* y, const InstDesc* inst, int B, int Nmax,
                          const double* theta,
                          const double* gamma, const double* beta, const Tables& tab, void* ws, c128* rho_out,
                          c128* x_out, c128* omega_out, c64* omega32_out, c64* x32_out, double* delta_out,
                          int* status, bool allow_cluster, cudaStream_t stream);
// Eval-grid: spectra and combine.  outputs in T (float for mixed, double for fp64).
// Schedule of the on-chip grid FFT kernel.
struct GridVariant {
  int threads;
  bool radix16;
};
int grid_variant_count();
GridVariant grid_variant(int i);

// Grid outputs of a batch from the factor kernel's omega_s and x (complex128,
// and their complex64 copies for the FP32 outputs).  tasks: the n_small
// on-chip tasks, then the n_large four-step tasks (grid_tasks); ws: the
// four-step intermediate buffers (grid_workspace_bytes); variant: the on-chip
// schedule; Lmax_small / Lmax_large: the largest L of each group.
cudaError_t launch_grid(int variant, bool f32, const InstDesc* inst, int Lmax_small, int Lmax_large, const c128* omega,
                        const c128* x, const c64* omega32, const c64* x32, const Tables& tab, void* ws,
                        const int4* tasks, int n_small, int n_large, void* q, void* dq, void* d2q, void* s, void* ds,
                        void* d2s, cudaStream_t stream);
// The grid tasks of a batch (host): one per (instance, output family), the
// s'' transforms of consecutive instances of equal N and L paired; the tasks
// with L small enough for the on-chip kernel first (*n_small), then the others
// with their intermediate offsets; *ws_elems the intermediates' total length.
// `out` needs 5 B entries; returns the count.
int grid_tasks(const InstDesc* inst, int B, bool f32, bool q, bool dq, bool d2q, bool s, bool ds, bool d2s, int4* out,
               int* n_small, size_t* ws_elems);
// Semifast evaluation (incomplete observations, Sec. IV): one instance of a
// batched launch.
struct SemiDesc {
  int64_t m_off;  // offset of y and obs (elements)
  int32_t M, N, L, K;
  int64_t k_off;  // offset of the components
  int64_t g_off;  // offset of the grid outputs
  int32_t idx;    // instance index (scalars, status)
};
size_t semifast_workspace_bytes(int Kmax, int Nmax, int Lmax);
size_t semifast_fit_workspace_bytes(int Kcap, int Nmax, int Lmax);
cudaError_t launch_semifast_fit(bool df, const float* y, const int* obs, const SemiDesc* inst, int B, int Kcap,
                                int Nmax, int Lmax, const FitConfig& cfg, const Tables& tab, const FitOut& out,
                                void* ws, int* counter, int grid, size_t smem, cudaStream_t stream);
size_t semifast_smem_bytes(int Kmax, int r_max);
cudaError_t launch_semifast(bool df, const float* y, const int* obs, const SemiDesc* inst, int B, int Kmax, int Nmax,
                            int Lmax, const double* theta, const double* gamma, const double* beta, const Tables& tab,
                            void* ws, double* scal, c128* vec, void* qg, void* sg, bool f64_out, int* status,
                            size_t smem, cudaStream_t stream);

// whether a grid of size L fits the on-chip FFT kernel
bool grid_on_chip(bool f32, int L);
size_t grid_workspace_bytes(size_t ws_elems, bool f32);

}  // namespace lse
