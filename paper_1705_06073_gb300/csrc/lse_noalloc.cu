// lse_noalloc.cu -- a fit entry point that never allocates device memory.
//
// Why it exists: some callers cannot allocate device memory at the moment
// they want a fit.  Examples are processing loops with a fixed per-frame
// deadline (cudaMalloc/cudaFree can block for milliseconds and synchronise
// the whole device), host code that runs inside another framework which owns
// every allocation on the GPU, and code that must not touch the allocator
// once set-up is over.  lse_fit_noalloc_d serves them: the caller passes its
// own device input and output buffers, and every piece of scratch memory the
// fit kernel needs comes from fixed-size arrays compiled into this library.
//
// The arrays below live in device memory of every GPU that loads the library
// until the process exits.  Host code cannot use their names as addresses;
// the set-up step looks the addresses up with cudaGetSymbolAddress (once per
// device, with that device current) and hands them to the kernel.
//
// The paper has no counterpart to this entry point: it is a deployment
// convenience of this library.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/lse.h"
#include "lse_internal.h"

using namespace lse;

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB of fit workspace
constexpr int kMaxN = 4096;
constexpr int kMaxLog2L = 15;                       // L <= 32768
constexpr int kMaxDevices = 64;

// Workspace of the one block that runs the fit.  Shared by every call.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
// Twiddle tables exp(-j 2 pi k / 2^15) in FP64, FP32 and double-float
// {re.h, re.l, im.h, im.l}, filled once per device at set-up.
static __device__ __align__(256) c128 g_tw64[1 << kMaxLog2L];
static __device__ __align__(256) c64 g_tw32[1 << kMaxLog2L];
static __device__ __align__(256) float4 g_twdf[1 << kMaxLog2L];
// Instance descriptor and work counter of the launch.
static __device__ __align__(16) InstDesc g_desc;
static __device__ int g_counter;

struct DeviceSetup {
  bool done = false;
  void* scratch = nullptr;
  c128* tw64 = nullptr;
  c64* tw32 = nullptr;
  float4* twdf = nullptr;
  InstDesc* desc = nullptr;
  int* counter = nullptr;
};

std::mutex g_mu;
DeviceSetup g_setup[kMaxDevices];

__global__ void fill_twiddles(c128* t64, c64* t32, float4* tdf) {
  const int M = 1 << kMaxLog2L;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)k / (double)M, &s, &c);
    t64[k] = mk(c, -s);
    t32[k] = mk((float)c, (float)-s);
    const float ch = (float)c, sh = (float)-s;
    tdf[k] = make_float4(ch, (float)(c - (double)ch), sh, (float)(-s - (double)sh));
  }
}

// The launch's instance descriptor, passed by value (a kernel parameter, so
// no host buffer has to outlive the call), and the zeroed work counter.  The
// device code names the static arrays directly.
__global__ void prepare_launch(InstDesc d) {
  g_desc = d;
  g_counter = 0;
}

// The entry point has no context to keep a message in; the status code is
// the whole report, and `msg` documents each rejection at its call site.
lse_status set_err(lse_status s, const char* msg) {
  (void)msg;
  return s;
}

// Look up the device addresses of the static arrays on the current device and
// fill its twiddle tables.  Runs once per device, on the first call there;
// it waits for the fill on that call's stream, so later calls on any stream
// find the tables complete.  The addresses are those of the device's current
// primary context: after cudaDeviceReset they are stale, and the entry point
// is not meant to be used past a reset.
lse_status setup(int dev, cudaStream_t st, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSetup& d = g_setup[dev];
  if (!d.done) {
    if (cudaGetSymbolAddress((void**)&d.scratch, g_scratch) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.tw64, g_tw64) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.tw32, g_tw32) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.twdf, g_twdf) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.desc, g_desc) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.counter, g_counter) != cudaSuccess)
      return set_err(LSE_ECUDA, "cudaGetSymbolAddress failed for the static scratch arrays");
    fill_twiddles<<<64, 256, 0, st>>>(d.tw64, d.tw32, d.twdf);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
      return set_err(LSE_ECUDA, "twiddle set-up failed");
    d.done = true;
  }
  *out = &d;
  return LSE_OK;
}

}  // namespace

extern "C" {

LSE_API lse_status lse_fit_noalloc_d(const lse_config* cfg, const float* y_d, int32_t N,
                                     const lse_batch_out* out, void* stream) {
  lse_config c;
  if (cfg) c = *cfg; else lse_config_default(&c);
  if (!y_d || !out) return set_err(LSE_EINVAL, "y_d and out must not be NULL");
  if (N < 2 || N > kMaxN) return set_err(LSE_EINVAL, "lse_fit_noalloc_d: N must be in [2, 4096]");
  if (c.grid_size < 0) return set_err(LSE_EINVAL, "lse_fit_noalloc_d: grid_size must be >= 0");
  if (c.flags & ~(uint64_t)(LSE_FLAG_NO_AUTOTUNE | LSE_FLAG_NO_CLUSTER | LSE_FLAG_LEVINSON | LSE_FLAG_DIRECT_SUMS |
                            LSE_FLAG_LBFGS))
    return set_err(LSE_EINVAL, "lse_fit_noalloc_d: unknown flag bits");
  const int L = c.grid_size ? c.grid_size : 1 << (int)std::lround(std::log2(8.0 * N));
  if ((L & (L - 1)) || L < 2 * N || L > (1 << kMaxLog2L))
    return set_err(LSE_EINVAL, "lse_fit_noalloc_d: L must be a power of two with 2N <= L <= 32768");
  if (c.precision != LSE_PREC_FP64 && c.precision != LSE_PREC_MIXED && c.precision != LSE_PREC_MIXED_DF)
    return set_err(LSE_EINVAL, "lse_fit_noalloc_d: unknown precision");
  if (c.max_outer < 1 || c.max_inner < 0 || c.approx_activation_iters < 0 || !(c.tau >= 0.0))
    return set_err(LSE_EINVAL, "lse_fit_noalloc_d: bad iteration limits or tau");
  const int prec = c.precision;
  if (fit_workspace_bytes(N, L, prec) > kScratchBytes)
    return set_err(LSE_EINVAL, "lse_fit_noalloc_d: workspace for this N and L exceeds the 8 MiB static scratch");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_err(LSE_ECUDA, "lse_fit_noalloc_d: no usable current device");
  cudaStream_t st = (cudaStream_t)stream;
  DeviceSetup* d = nullptr;
  lse_status s = setup(dev, st, &d);
  if (s != LSE_OK) return s;
  const InstDesc h{0, N, L, 0, 0, 0, 0};  // result slot 0
  prepare_launch<<<1, 1, 0, st>>>(h);
  if (cudaGetLastError() != cudaSuccess)
    return set_err(LSE_ECUDA, "lse_fit_noalloc_d: staging the launch descriptor failed");
  const FitConfig fc{c.tau, c.max_outer, c.max_inner, c.approx_activation_iters, !(c.flags & LSE_FLAG_NO_CLUSTER),
                     superfast_min_n(c.flags), N, 1, nufft_min_k(c.flags), (c.flags & LSE_FLAG_LBFGS) ? 1 : 0};
  const FitOut fo{out->theta, out->gamma, (c128*)out->alpha, out->K, out->beta, out->objective, out->iters,
                  out->n_evals, out->n_grid, out->status};
  const Tables tab{d->tw64, d->tw32, kMaxLog2L, d->twdf};
  if (launch_fit(prec, y_d, d->desc, 1, N, L, fc, tab, fo, d->scratch, d->counter, 1, st) != cudaSuccess)
    return set_err(LSE_ECUDA, "lse_fit_noalloc_d: fit kernel launch failed");
  return LSE_OK;
}

}  // extern "C"
