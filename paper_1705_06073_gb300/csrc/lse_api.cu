// lse_api.cu -- the C ABI declared in include/lse.h: context, device memory,
// argument checking, launches and host<->device staging.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lse.h"
#include "lse_internal.h"

using namespace lse;

namespace {

struct TimedLaunch {
  cudaEvent_t a, b;
};

// Device buffer that only grows.
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
};

// Launch metadata (instance descriptors, grid offsets, task lists) kept on the
// device: uploaded only when its content changes, from one of two pinned
// host slots whose previous upload is known complete (its event), so a call
// never waits on the device for it.
struct Staged {
  DevBuf dev;
  std::vector<char> last;  // what dev holds
  char* pinned[2] = {nullptr, nullptr};
  size_t pcap[2] = {0, 0};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int next = 0;
};

}  // namespace

struct lse_plan;

struct lse_ctx {
  lse_config cfg;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  // twiddle tables exp(-j 2 pi k / 2^log2max)
  c128* tw64 = nullptr;
  c64* tw32 = nullptr;
  float4* twdf = nullptr;
  int log2max = 0;
  DevBuf ws, counter, stage_in, stage_out, fac, semi;
  Staged fit_meta, grid_meta, semi_meta;
  size_t allocated = 0;
  std::vector<TimedLaunch> timed[3];
  std::string err;
  // autotuned schedule of the on-chip grid FFT per (FP32?, L)
  std::map<std::pair<int, int>, int> grid_variant;
};

struct lse_plan {
  lse_ctx* ctx = nullptr;
  int B = 0, Nmax = 0, Lmax = 0, Nmin = 0, grid = 0, prec = 0;
  DevBuf desc, counter, ws;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const float* g_y = nullptr;  // arguments baked into the captured graph
  lse_batch_out g_out{};
};

namespace {

// snapshots per instance accepted by the multiple-measurement-vector fits
constexpr int32_t kMaxSnapshots = 1024;
// components per instance accepted by the semifast evaluation (its K x K
// factor is staged in shared memory for the grid contraction)
constexpr int32_t kMaxSemifastK = 96;

lse_status fail(lse_ctx* c, lse_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

lse_status cuda_fail(lse_ctx* c, cudaError_t e, const char* where) {
  return fail(c, LSE_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LSE_CUDA(ctx, call)                                  \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

lse_status ensure(lse_ctx* c, DevBuf& b, size_t bytes, bool capturing = false) {
  if (b.n >= bytes) return LSE_OK;
  if (capturing)
    return fail(c, LSE_EINVAL, "the call needs more device memory than the context holds, which cannot be "
                               "allocated during stream capture: make one call with these shapes first");
  const size_t grow = bytes - b.n;
  if (c->cfg.hbm_budget_bytes && c->allocated + grow > c->cfg.hbm_budget_bytes)
    return fail(c, LSE_EBUDGET, "request needs " + std::to_string(c->allocated + grow) +
                                    " bytes of device memory, budget is " +
                                    std::to_string((unsigned long long)c->cfg.hbm_budget_bytes));
  if (b.p) {
    cudaStreamSynchronize(c->stream);
    cudaFree(b.p);
    c->allocated -= b.n;
    b.p = nullptr;
    b.n = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return fail(c, LSE_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  b.n = bytes;
  c->allocated += bytes;
  return LSE_OK;
}

__global__ void twiddle_kernel(c128* t64, c64* t32, float4* tdf, int log2m) {
  const int M = 1 << log2m;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)k / (double)M, &s, &c);
    t64[k] = mk(c, -s);
    t32[k] = mk((float)c, (float)-s);
    const float ch = (float)c, sh = (float)-s;
    tdf[k] = make_float4(ch, (float)(c - (double)ch), sh, (float)(-s - (double)sh));
  }
}

lse_status ensure_tables(lse_ctx* c, int log2m) {
  if (log2m < 2) log2m = 2;
  if (c->tw64 && c->log2max >= log2m) return LSE_OK;
  if (c->tw64) {
    cudaStreamSynchronize(c->stream);
    cudaFree(c->tw64);
    cudaFree(c->tw32);
    cudaFree(c->twdf);
    c->tw64 = nullptr;
    c->tw32 = nullptr;
    c->twdf = nullptr;
  }
  const size_t M = size_t(1) << log2m;
  LSE_CUDA(c, cudaMalloc(&c->tw64, M * sizeof(c128)));
  LSE_CUDA(c, cudaMalloc(&c->tw32, M * sizeof(c64)));
  LSE_CUDA(c, cudaMalloc(&c->twdf, M * sizeof(float4)));
  twiddle_kernel<<<256, 256, 0, c->stream>>>(c->tw64, c->tw32, c->twdf, log2m);
  LSE_CUDA(c, cudaGetLastError());
  c->log2max = log2m;
  return LSE_OK;
}

Tables tables(const lse_ctx* c) { return Tables{c->tw64, c->tw32, c->log2max, c->twdf}; }

int default_L(int N) {
  // 8N rounded to the nearest power of two (Sec. II-C5 footnote)
  double l = std::log2(8.0 * N);
  return 1 << (int)std::lround(l);
}

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

bool is_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// Make s.dev hold `bytes` of `data`, enqueuing the upload on st if it does not
// already.  Stream order protects the device copy (every launch that reads it
// is ordered before the next upload); the pinned slot is reused only after
// the upload that last read it has completed.
lse_status stage(lse_ctx* c, Staged& s, const void* data, size_t bytes, cudaStream_t st, bool capturing) {
  if (s.dev.p && s.last.size() == bytes && std::memcmp(s.last.data(), data, bytes) == 0) return LSE_OK;
  if (capturing)
    return fail(c, LSE_EINVAL, "launch descriptors differ from the previous call's, and uploading them cannot be "
                               "captured: make one call with these shapes before capturing");
  lse_status r = ensure(c, s.dev, bytes);
  if (r) return r;
  const int k = s.next;
  s.next ^= 1;
  if (!s.ev[k]) LSE_CUDA(c, cudaEventCreateWithFlags(&s.ev[k], cudaEventDisableTiming));
  else LSE_CUDA(c, cudaEventSynchronize(s.ev[k]));
  if (s.pcap[k] < bytes) {
    if (s.pinned[k]) cudaFreeHost(s.pinned[k]);
    s.pinned[k] = nullptr;
    s.pcap[k] = 0;
    LSE_CUDA(c, cudaMallocHost((void**)&s.pinned[k], bytes));
    s.pcap[k] = bytes;
  }
  std::memcpy(s.pinned[k], data, bytes);
  LSE_CUDA(c, cudaMemcpyAsync(s.dev.p, s.pinned[k], bytes, cudaMemcpyHostToDevice, st));
  LSE_CUDA(c, cudaEventRecord(s.ev[k], st));
  s.last.assign((const char*)data, (const char*)data + bytes);
  return LSE_OK;
}

void release(Staged& s) {
  if (s.dev.p) cudaFree(s.dev.p);
  for (int k = 0; k < 2; ++k) {
    if (s.pinned[k]) cudaFreeHost(s.pinned[k]);
    if (s.ev[k]) cudaEventDestroy(s.ev[k]);
  }
}

// `from` waits for everything enqueued so far on `to`'s side: used to order a
// caller stream after the context stream and back.
lse_status order_after(lse_ctx* c, cudaStream_t waiter, cudaStream_t done) {
  cudaEvent_t e;
  LSE_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaEventRecord(e, done);
  cudaStreamWaitEvent(waiter, e, 0);
  cudaEventDestroy(e);
  return LSE_OK;
}

void record(lse_ctx* c, int which, cudaStream_t st, bool start) {
  if (is_capturing(st)) return;  // events recorded into a graph carry no time
  if (start && c->timed[which].size() >= 4096) {  // nobody reads them (a server's slot): keep the newest half
    auto& v = c->timed[which];
    for (size_t i = 0; i < v.size() / 2; ++i) {
      cudaEventDestroy(v[i].a);
      cudaEventDestroy(v[i].b);
    }
    v.erase(v.begin(), v.begin() + v.size() / 2);
  }
  if (start) {
    TimedLaunch t;
    cudaEventCreate(&t.a);
    cudaEventCreate(&t.b);
    cudaEventRecord(t.a, st);
    c->timed[which].push_back(t);
  } else {
    cudaEventRecord(c->timed[which].back().b, st);
  }
}

// Autotune cache file: lines "grid <f32|f64> <L> <variant>".
const char* autotune_path() { return std::getenv("LSE_AUTOTUNE_CACHE"); }

void load_autotune(lse_ctx* c) {
  const char* path = autotune_path();
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char kind[16], dt[8];
  int L, v;
  while (std::fscanf(f, "%15s %7s %d %d", kind, dt, &L, &v) == 4)
    if (!std::strcmp(kind, "grid") && v >= 0 && v < grid_variant_count())
      c->grid_variant[{std::strcmp(dt, "f32") == 0 ? 1 : 0, L}] = v;
  std::fclose(f);
}

void save_autotune(const lse_ctx* c) {
  const char* path = autotune_path();
  if (!path) return;
  FILE* f = std::fopen(path, "w");
  if (!f) return;
  for (const auto& kv : c->grid_variant)
    std::fprintf(f, "grid %s %d %d\n", kv.first.first ? "f32" : "f64", kv.first.second, kv.second);
  std::fclose(f);
}

// Descriptors of a batched fit, in the order the instances are handed out:
// largest N first (longest-processing-time order) so that a ragged batch does
// not end waiting on a big instance started last.  idx keeps the result slot.
lse_status plan_fit_descs(lse_ctx* ctx, const int64_t* offsets, int32_t B, std::vector<InstDesc>& d, int& Nmax,
                          int& Lmax, int* Nmin = nullptr) {
  if (B < 1 || !offsets) return fail(ctx, LSE_EINVAL, "null offsets or B < 1");
  if (offsets[0] != 0) return fail(ctx, LSE_EINVAL, "offsets[0] must be 0");
  d.resize(B);
  Nmax = 0;
  Lmax = 0;
  for (int b = 0; b < B; ++b) {
    const int64_t n = offsets[b + 1] - offsets[b];
    if (n < 2 || n > (1 << 17)) return fail(ctx, LSE_EINVAL, "instance " + std::to_string(b) + ": N out of range");
    const int N = (int)n;
    const int L = ctx->cfg.grid_size ? ctx->cfg.grid_size : default_L(N);
    if (L < 2 * N) return fail(ctx, LSE_EINVAL, "grid size L must be >= 2N");
    d[b] = InstDesc{offsets[b], N, L, 0, 0, b, 0};
    Nmax = std::max(Nmax, N);
    Lmax = std::max(Lmax, L);
  }
  std::stable_sort(d.begin(), d.end(), [](const InstDesc& a, const InstDesc& b) { return a.N > b.N; });
  if (Nmin) *Nmin = d.back().N;
  return LSE_OK;
}

}  // namespace

cudaStream_t lse_ctx_stream(lse_ctx* c) { return c ? c->stream : nullptr; }

lse_status lse_ctx_reserve_fit(lse_ctx* ctx, int Nmax, int Lmax, int B) {
  if (!ctx || Nmax < 2 || Lmax < 2 * Nmax || B < 1) return LSE_EINVAL;
  cudaSetDevice(ctx->cfg.device);
  lse_status s;
  if ((s = ensure_tables(ctx, std::max(ilog2((uint32_t)Lmax), ilog2(2u * (uint32_t)Nmax))))) return s;
  const int grid = std::min(B, ctx->sm_count);
  if ((s = ensure(ctx, ctx->ws, fit_workspace_bytes(Nmax, Lmax, ctx->cfg.precision) * grid))) return s;
  const size_t db = (size_t)B * sizeof(InstDesc);
  if ((s = ensure(ctx, ctx->fit_meta.dev, db))) return s;
  Staged& st = ctx->fit_meta;
  for (int k = 0; k < 2; ++k) {
    if (!st.ev[k]) LSE_CUDA(ctx, cudaEventCreateWithFlags(&st.ev[k], cudaEventDisableTiming));
    if (st.pcap[k] < db) {
      LSE_CUDA(ctx, cudaEventSynchronize(st.ev[k]));
      if (st.pinned[k]) cudaFreeHost(st.pinned[k]);
      st.pinned[k] = nullptr;
      st.pcap[k] = 0;
      LSE_CUDA(ctx, cudaMallocHost((void**)&st.pinned[k], db));
      st.pcap[k] = db;
    }
  }
  LSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return LSE_OK;
}

extern "C" {

void lse_config_default(lse_config* cfg) {
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->precision = LSE_PREC_FP64;
  cfg->hbm_budget_bytes = 0;
  cfg->grid_size = 0;
  cfg->tau = 5.0;
  cfg->max_outer = 200;
  cfg->max_inner = 5;
  cfg->approx_activation_iters = 10;
  cfg->flags = 0;
}

const char* lse_strerror(lse_status s) {
  switch (s) {
    case LSE_OK: return "ok";
    case LSE_EINVAL: return "invalid argument";
    case LSE_ENOMEM: return "out of device memory";
    case LSE_EBUDGET: return "request exceeds the device-memory budget";
    case LSE_ENUMERIC: return "Levinson recursion broke down (covariance not numerically positive definite)";
    case LSE_ENOTCONV: return "iteration limit reached before convergence";
    case LSE_ETIMEOUT: return "device-side wait timed out";
    case LSE_ECUDA: return "CUDA runtime error";
    case LSE_ECAPACITY: return "result capacity too small";
  }
  return "unknown status";
}

const char* lse_last_error(const lse_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

lse_status lse_create(const lse_config* cfg, lse_ctx** out) {
  if (!out) return LSE_EINVAL;
  *out = nullptr;
  lse_config c;
  if (cfg) c = *cfg; else lse_config_default(&c);
  if (c.precision != LSE_PREC_FP64 && c.precision != LSE_PREC_MIXED && c.precision != LSE_PREC_MIXED_DF)
    return LSE_EINVAL;
  if (c.max_outer < 1 || c.max_inner < 0 || c.approx_activation_iters < 0 || !(c.tau >= 0.0) ||
      (c.flags & ~(uint64_t)(LSE_FLAG_NO_AUTOTUNE | LSE_FLAG_NO_CLUSTER | LSE_FLAG_LEVINSON | LSE_FLAG_DIRECT_SUMS |
                             LSE_FLAG_LBFGS)))
    return LSE_EINVAL;
  if (c.grid_size < 0 || (c.grid_size > 0 && !is_pow2(c.grid_size))) return LSE_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) return LSE_ECUDA;
  if (cudaSetDevice(c.device) != cudaSuccess) return LSE_ECUDA;
  lse_ctx* ctx = new lse_ctx();
  ctx->cfg = c;
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, c.device);
  if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete ctx;
    return LSE_ECUDA;
  }
  load_autotune(ctx);
  lse_status s = ensure_tables(ctx, 17);
  if (s == LSE_OK) s = ensure(ctx, ctx->counter, 256);
  if (s != LSE_OK) {
    lse_destroy(ctx);
    return s;
  }
  *out = ctx;
  return LSE_OK;
}

void lse_destroy(lse_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->cfg.device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (DevBuf* b : {&ctx->ws, &ctx->counter, &ctx->stage_in, &ctx->stage_out, &ctx->fac, &ctx->semi})
    if (b->p) cudaFree(b->p);
  release(ctx->fit_meta);
  release(ctx->grid_meta);
  release(ctx->semi_meta);
  if (ctx->tw64) cudaFree(ctx->tw64);
  if (ctx->tw32) cudaFree(ctx->tw32);
  if (ctx->twdf) cudaFree(ctx->twdf);
  for (auto& v : ctx->timed)
    for (auto& t : v) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

lse_status lse_kernel_time(lse_ctx* ctx, int32_t which, double* total_ms, int64_t* launches) {
  if (!ctx || which < 0 || which > 2) return LSE_EINVAL;
  double tot = 0.0;
  int64_t n = 0;
  for (auto& t : ctx->timed[which]) {
    LSE_CUDA(ctx, cudaEventSynchronize(t.b));
    float ms = 0.f;
    LSE_CUDA(ctx, cudaEventElapsedTime(&ms, t.a, t.b));
    tot += ms;
    ++n;
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  ctx->timed[which].clear();
  if (total_ms) *total_ms = tot;
  if (launches) *launches = n;
  return LSE_OK;
}

}  // extern "C"

namespace {

// Batched fit of B instances with G snapshots each (G = 1: lse_fit_batch_d;
// G > 1: lse_fit_mmv_batch_d).
lse_status fit_batch_d(lse_ctx* ctx, const float* y_d, const int64_t* offsets, int32_t B, int32_t G,
                       const lse_batch_out* out, void* stream) {
  if (!ctx || !y_d || !offsets || B < 1 || !out) return fail(ctx, LSE_EINVAL, "null argument or B < 1");
  if (G < 1 || G > kMaxSnapshots) return fail(ctx, LSE_EINVAL, "G out of range");
  if (offsets[0] != 0) return fail(ctx, LSE_EINVAL, "offsets[0] must be 0");
  cudaSetDevice(ctx->cfg.device);
  cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
  const bool cap = is_capturing(st);
  std::vector<InstDesc> d;
  int Nmax = 0, Lmax = 0, Nmin = 0;
  lse_status s = plan_fit_descs(ctx, offsets, B, d, Nmax, Lmax, &Nmin);
  if (s) return s;
  const int prec = ctx->cfg.precision;
  const int log2t = std::max(ilog2((uint32_t)Lmax), ilog2(2u * (uint32_t)Nmax));
  if (cap && (!ctx->tw64 || ctx->log2max < log2t))
    return fail(ctx, LSE_EINVAL, "twiddle tables must grow, which cannot be captured: make one call first");
  if ((s = ensure_tables(ctx, log2t))) return s;
  const int grid = std::min(B, ctx->sm_count);
  const size_t per = fit_workspace_bytes(Nmax, Lmax, prec, G);
  if ((s = ensure(ctx, ctx->ws, per * grid, cap))) return s;
  if (!cap && st != ctx->stream && (s = order_after(ctx, st, ctx->stream))) return s;
  if ((s = stage(ctx, ctx->fit_meta, d.data(), d.size() * sizeof(InstDesc), st, cap))) return s;
  LSE_CUDA(ctx, cudaMemsetAsync(ctx->counter.p, 0, sizeof(int), st));
  FitConfig fc{ctx->cfg.tau, ctx->cfg.max_outer, ctx->cfg.max_inner, ctx->cfg.approx_activation_iters,
               !(ctx->cfg.flags & LSE_FLAG_NO_CLUSTER), superfast_min_n(ctx->cfg.flags), Nmin, G,
               nufft_min_k(ctx->cfg.flags),
               (ctx->cfg.flags & LSE_FLAG_LBFGS) ? 1 : 0};
  FitOut fo{out->theta, out->gamma, (c128*)out->alpha, out->K, out->beta, out->objective, out->iters,
            out->n_evals, out->n_grid, out->status};
  record(ctx, 0, st, true);
  cudaError_t e = launch_fit(prec, y_d, (const InstDesc*)ctx->fit_meta.dev.p, B, Nmax, Lmax, fc, tables(ctx), fo,
                             ctx->ws.p, (int*)ctx->counter.p, grid, st);
  record(ctx, 0, st, false);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fit kernel launch");
  // later work of this context on its own stream must follow this launch
  if (!cap && st != ctx->stream && (s = order_after(ctx, ctx->stream, st))) return s;
  return LSE_OK;
}

// Host-array batched fit with G snapshots per instance: stage y in, run
// fit_batch_d, copy the results back and unpack them per instance.
lse_status fit_batch_host(lse_ctx* ctx, const float* y, const int64_t* offsets, int32_t B, int32_t G,
                          lse_result* outs, lse_status* per_instance) {
  if (!ctx || !y || !offsets || B < 1 || !outs) return fail(ctx, LSE_EINVAL, "null argument or B < 1");
  if (G < 1 || G > kMaxSnapshots) return fail(ctx, LSE_EINVAL, "G out of range");
  cudaSetDevice(ctx->cfg.device);
  const int64_t tot = offsets[B];
  if (tot <= 0) return fail(ctx, LSE_EINVAL, "empty batch");
  // device staging: y | theta | gamma | alpha | K | beta | obj | iters | nevals | status
  const size_t yb = (size_t)tot * G * 2 * sizeof(float);
  const size_t ob = (size_t)tot * (2 + 2 * G) * sizeof(double) + (size_t)B * (5 * sizeof(int) + 2 * sizeof(double)) +
                    1024;
  lse_status s;
  if ((s = ensure(ctx, ctx->stage_in, yb))) return s;
  if ((s = ensure(ctx, ctx->stage_out, ob))) return s;
  char* o = (char*)ctx->stage_out.p;
  lse_batch_out bo;
  bo.theta = (double*)o; o += tot * sizeof(double);
  bo.gamma = (double*)o; o += tot * sizeof(double);
  bo.alpha = (double*)o; o += tot * G * 2 * sizeof(double);
  bo.beta = (double*)o; o += B * sizeof(double);
  bo.objective = (double*)o; o += B * sizeof(double);
  bo.K = (int32_t*)o; o += B * sizeof(int);
  bo.iters = (int32_t*)o; o += B * sizeof(int);
  bo.n_evals = (int32_t*)o; o += B * sizeof(int);
  bo.n_grid = (int32_t*)o; o += B * sizeof(int);
  bo.status = (int32_t*)o; o += B * sizeof(int);
  LSE_CUDA(ctx, cudaMemcpyAsync(ctx->stage_in.p, y, yb, cudaMemcpyHostToDevice, ctx->stream));
  if ((s = fit_batch_d(ctx, (const float*)ctx->stage_in.p, offsets, B, G, &bo, ctx->stream))) return s;
  std::vector<char> host(ob);
  LSE_CUDA(ctx, cudaMemcpyAsync(host.data(), ctx->stage_out.p, ob, cudaMemcpyDeviceToHost, ctx->stream));
  LSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const char* h = host.data();
  const double* th = (const double*)h;
  const double* ga = th + tot;
  const double* al = ga + tot;
  const double* be = al + 2 * G * tot;
  const double* ob_ = be + B;
  const int32_t* K = (const int32_t*)(ob_ + B);
  const int32_t* it = K + B;
  const int32_t* ne = it + B;
  const int32_t* ng = ne + B;
  const int32_t* stt = ng + B;
  for (int b = 0; b < B; ++b) {
    lse_result& r = outs[b];
    lse_status sb = (lse_status)stt[b];
    r.K = K[b];
    r.beta = be[b];
    r.objective = ob_[b];
    r.iters = it[b];
    r.n_evals = ne[b];
    r.n_grid = ng[b];
    if (K[b] > r.K_cap) {
      sb = LSE_ECAPACITY;
    } else {
      const int64_t off = offsets[b], Nb = offsets[b + 1] - offsets[b];
      for (int k = 0; k < K[b]; ++k) {
        if (r.theta) r.theta[k] = th[off + k];
        if (r.gamma) r.gamma[k] = ga[off + k];
        if (r.alpha)
          for (int g = 0; g < G; ++g) {
            const int64_t src = 2 * ((int64_t)G * off + g * Nb + k), dst = 2 * ((int64_t)g * r.K_cap + k);
            r.alpha[dst] = al[src];
            r.alpha[dst + 1] = al[src + 1];
          }
      }
    }
    if (per_instance) per_instance[b] = sb;
  }
  return LSE_OK;
}

}  // namespace

extern "C" {

lse_status lse_fit_batch_d(lse_ctx* ctx, const float* y_d, const int64_t* offsets, int32_t B,
                           const lse_batch_out* out, void* stream) {
  return fit_batch_d(ctx, y_d, offsets, B, 1, out, stream);
}

lse_status lse_fit_mmv_batch_d(lse_ctx* ctx, const float* y_d, const int64_t* offsets, int32_t B, int32_t G,
                               const lse_batch_out* out, void* stream) {
  return fit_batch_d(ctx, y_d, offsets, B, G, out, stream);
}

lse_status lse_fit_mmv(lse_ctx* ctx, const float* y, int32_t N, int32_t G, lse_result* out) {
  if (!ctx || !y || !out || N < 2) return fail(ctx, LSE_EINVAL, "null argument or N < 2");
  const int64_t off[2] = {0, N};
  lse_status per = LSE_OK;
  lse_status s = fit_batch_host(ctx, y, off, 1, G, out, &per);
  return s ? s : per;
}

lse_status lse_plan_fit(lse_ctx* ctx, const int64_t* offsets, int32_t B, lse_plan** out) {
  if (!ctx || !out) return fail(ctx, LSE_EINVAL, "null argument");
  *out = nullptr;
  cudaSetDevice(ctx->cfg.device);
  std::vector<InstDesc> d;
  int Nmax = 0, Lmax = 0, Nmin = 0;
  lse_status s = plan_fit_descs(ctx, offsets, B, d, Nmax, Lmax, &Nmin);
  if (s) return s;
  if ((s = ensure_tables(ctx, std::max(ilog2((uint32_t)Lmax), ilog2(2u * (uint32_t)Nmax))))) return s;
  lse_plan* p = new lse_plan();
  p->ctx = ctx;
  p->B = B;
  p->Nmax = Nmax;
  p->Lmax = Lmax;
  p->Nmin = Nmin;
  p->prec = ctx->cfg.precision;
  p->grid = std::min(B, ctx->sm_count);
  if ((s = ensure(ctx, p->desc, d.size() * sizeof(InstDesc))) || (s = ensure(ctx, p->counter, 256)) ||
      (s = ensure(ctx, p->ws, fit_workspace_bytes(Nmax, Lmax, p->prec) * p->grid))) {
    lse_plan_destroy(p);
    return s;
  }
  if (cudaMemcpy(p->desc.p, d.data(), d.size() * sizeof(InstDesc), cudaMemcpyHostToDevice) != cudaSuccess) {
    lse_plan_destroy(p);
    return fail(ctx, LSE_ECUDA, "descriptor upload failed");
  }
  *out = p;
  return LSE_OK;
}

lse_status lse_plan_launch(lse_plan* p, const float* y_d, const lse_batch_out* out, void* stream) {
  if (!p || !y_d || !out) return LSE_EINVAL;
  lse_ctx* ctx = p->ctx;
  cudaStream_t st = (cudaStream_t)stream;
  LSE_CUDA(ctx, cudaMemsetAsync(p->counter.p, 0, sizeof(int), st));
  const FitConfig fc{ctx->cfg.tau, ctx->cfg.max_outer, ctx->cfg.max_inner, ctx->cfg.approx_activation_iters,
                     !(ctx->cfg.flags & LSE_FLAG_NO_CLUSTER), superfast_min_n(ctx->cfg.flags), p->Nmin, 1,
                     nufft_min_k(ctx->cfg.flags),
               (ctx->cfg.flags & LSE_FLAG_LBFGS) ? 1 : 0};
  const FitOut fo{out->theta, out->gamma, (c128*)out->alpha, out->K, out->beta, out->objective, out->iters,
                  out->n_evals, out->n_grid, out->status};
  const cudaError_t e = launch_fit(p->prec, y_d, (const InstDesc*)p->desc.p, p->B, p->Nmax, p->Lmax, fc, tables(ctx),
                                   fo, p->ws.p, (int*)p->counter.p, p->grid, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fit kernel launch");
  return LSE_OK;
}

lse_status lse_plan_graph_launch(lse_plan* p, const float* y_d, const lse_batch_out* out, void* stream) {
  if (!p || !y_d || !out) return LSE_EINVAL;
  lse_ctx* ctx = p->ctx;
  const bool same = p->exec && p->g_y == y_d && !std::memcmp(&p->g_out, out, sizeof(*out));
  if (!same) {
    // capture on the context's own (non-legacy) stream; the graph is launched
    // on the caller's stream
    cudaGraph_t g = nullptr;
    LSE_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const lse_status s = lse_plan_launch(p, y_d, out, ctx->stream);
    const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
    if (s) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamEndCapture");
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = g;
    LSE_CUDA(ctx, cudaGraphInstantiate(&p->exec, g, 0));
    p->g_y = y_d;
    p->g_out = *out;
  }
  LSE_CUDA(ctx, cudaGraphLaunch(p->exec, (cudaStream_t)stream));
  return LSE_OK;
}

void lse_plan_destroy(lse_plan* p) {
  if (!p) return;
  lse_ctx* ctx = p->ctx;
  cudaSetDevice(ctx->cfg.device);
  cudaDeviceSynchronize();
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (DevBuf* b : {&p->desc, &p->counter, &p->ws})
    if (b->p) {
      cudaFree(b->p);
      ctx->allocated -= b->n;
    }
  delete p;
}

lse_status lse_fit_batch(lse_ctx* ctx, const float* y, const int64_t* offsets, int32_t B, lse_result* outs,
                         lse_status* per_instance) {
  return fit_batch_host(ctx, y, offsets, B, 1, outs, per_instance);
}

lse_status lse_fit(lse_ctx* ctx, const float* y, int32_t N, lse_result* out) {
  if (!ctx || !y || !out || N < 2) return fail(ctx, LSE_EINVAL, "null argument or N < 2");
  const int64_t off[2] = {0, N};
  lse_status per = LSE_OK;
  lse_status s = lse_fit_batch(ctx, y, off, 1, out, &per);
  return s ? s : per;
}

lse_status lse_eval_semifast_batch_d(lse_ctx* ctx, const float* y_d, const int32_t* obs_d, const int64_t* m_offsets,
                                     int32_t B, const int32_t* N, const double* theta_d, const double* gamma_d,
                                     const int64_t* k_offsets, const double* beta_d, const int32_t* L, int32_t dtype,
                                     double* scal_d, double* vec_d, void* q, void* s, int32_t* status_d,
                                     void* stream) {
  if (!ctx || !y_d || !obs_d || !m_offsets || !N || !k_offsets || !beta_d || !L || !scal_d || !vec_d ||
      !status_d || B < 1)
    return fail(ctx, LSE_EINVAL, "null argument or B < 1");
  if (m_offsets[0] != 0 || k_offsets[0] != 0) return fail(ctx, LSE_EINVAL, "offsets must start at 0");
  const bool f64 = ctx->cfg.precision == LSE_PREC_FP64;
  if (dtype != (f64 ? LSE_F64 : LSE_F32))
    return fail(ctx, LSE_EINVAL, "dtype must be LSE_F64 for an FP64 context and LSE_F32 for a mixed one");
  cudaSetDevice(ctx->cfg.device);
  cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
  const bool cap = is_capturing(st);
  std::vector<SemiDesc> d(B);
  int Nmax = 0, Lmax = 0, Kmax = 0, rmax = 1;
  int64_t g = 0;
  for (int b = 0; b < B; ++b) {
    const int64_t m = m_offsets[b + 1] - m_offsets[b];
    const int64_t k = k_offsets[b + 1] - k_offsets[b];
    if (N[b] < 2 || N[b] > (1 << 17) || m < 1 || m > N[b])
      return fail(ctx, LSE_EINVAL, "instance " + std::to_string(b) + ": N or M out of range");
    if (k < 0 || k > kMaxSemifastK || k > m)
      return fail(ctx, LSE_EINVAL, "instance " + std::to_string(b) + ": K must be in [0, min(M, " +
                                       std::to_string(kMaxSemifastK) + ")]");
    if (!is_pow2(L[b]) || L[b] < 2 * N[b]) return fail(ctx, LSE_EINVAL, "L must be a power of two >= 2N");
    d[b] = SemiDesc{m_offsets[b], (int)m, N[b], L[b], (int)k, k_offsets[b], g, b};
    g += L[b];
    Nmax = std::max(Nmax, N[b]);
    Lmax = std::max(Lmax, L[b]);
    Kmax = std::max(Kmax, (int)k);
    rmax = std::max(rmax, L[b] / (1 << ilog2(2u * (uint32_t)N[b])));
  }
  const int log2t = std::max(ilog2((uint32_t)Lmax), ilog2(2u * (uint32_t)Nmax));
  if (cap && (!ctx->tw64 || ctx->log2max < log2t))
    return fail(ctx, LSE_EINVAL, "twiddle tables must grow, which cannot be captured: make one call first");
  lse_status sst = ensure_tables(ctx, log2t);
  if (sst) return sst;
  const size_t per = semifast_workspace_bytes(Kmax, Nmax, Lmax);
  if ((sst = ensure(ctx, ctx->semi, per * (size_t)B, cap))) return sst;
  if (!cap && st != ctx->stream && (sst = order_after(ctx, st, ctx->stream))) return sst;
  if ((sst = stage(ctx, ctx->semi_meta, d.data(), d.size() * sizeof(SemiDesc), st, cap))) return sst;
  const size_t smem = semifast_smem_bytes(Kmax, rmax);
  if (smem > 200 * 1024) return fail(ctx, LSE_EINVAL, "K too large for the semifast kernel's shared memory");
  record(ctx, 1, st, true);
  const cudaError_t e = launch_semifast(!f64, y_d, obs_d, (const SemiDesc*)ctx->semi_meta.dev.p, B, Kmax, Nmax, Lmax,
                                        theta_d, gamma_d, beta_d, tables(ctx), ctx->semi.p, scal_d, (c128*)vec_d, q,
                                        s, f64, status_d, smem, st);
  record(ctx, 1, st, false);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "semifast kernel launch");
  if (!cap && st != ctx->stream && (sst = order_after(ctx, ctx->stream, st))) return sst;
  return LSE_OK;
}

lse_status lse_fit_incomplete_batch_d(lse_ctx* ctx, const float* y_d, const int32_t* obs_d, const int64_t* m_offsets,
                                      int32_t B, const int32_t* N, const lse_batch_out* out, void* stream) {
  if (!ctx || !y_d || !obs_d || !m_offsets || !N || !out || B < 1) return fail(ctx, LSE_EINVAL, "null argument or B < 1");
  if (m_offsets[0] != 0) return fail(ctx, LSE_EINVAL, "m_offsets[0] must be 0");
  cudaSetDevice(ctx->cfg.device);
  cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
  const bool cap = is_capturing(st);
  std::vector<SemiDesc> d(B);
  int Nmax = 0, Lmax = 0, rmax = 1;
  for (int b = 0; b < B; ++b) {
    const int64_t m = m_offsets[b + 1] - m_offsets[b];
    if (N[b] < 2 || N[b] > (1 << 17) || m < 1 || m > N[b])
      return fail(ctx, LSE_EINVAL, "instance " + std::to_string(b) + ": N or M out of range");
    const int L = ctx->cfg.grid_size ? ctx->cfg.grid_size : default_L(N[b]);
    if (L < 2 * N[b]) return fail(ctx, LSE_EINVAL, "grid size L must be >= 2N");
    d[b] = SemiDesc{m_offsets[b], (int)m, N[b], L, 0, 0, 0, b};
    Nmax = std::max(Nmax, N[b]);
    Lmax = std::max(Lmax, L);
    rmax = std::max(rmax, L / (1 << ilog2(2u * (uint32_t)N[b])));
  }
  // largest first, as the complete-data batches
  std::stable_sort(d.begin(), d.end(), [](const SemiDesc& a, const SemiDesc& b) { return a.N > b.N; });
  const int log2t = std::max(ilog2((uint32_t)Lmax), ilog2(2u * (uint32_t)Nmax));
  if (cap && (!ctx->tw64 || ctx->log2max < log2t))
    return fail(ctx, LSE_EINVAL, "twiddle tables must grow, which cannot be captured: make one call first");
  lse_status sst = ensure_tables(ctx, log2t);
  if (sst) return sst;
  const int grid = std::min(B, ctx->sm_count);
  const size_t per = semifast_fit_workspace_bytes(kMaxSemifastK, Nmax, Lmax);
  if ((sst = ensure(ctx, ctx->semi, per * (size_t)grid, cap))) return sst;
  if (!cap && st != ctx->stream && (sst = order_after(ctx, st, ctx->stream))) return sst;
  if ((sst = stage(ctx, ctx->semi_meta, d.data(), d.size() * sizeof(SemiDesc), st, cap))) return sst;
  LSE_CUDA(ctx, cudaMemsetAsync(ctx->counter.p, 0, sizeof(int), st));
  const FitConfig fc{ctx->cfg.tau, ctx->cfg.max_outer, ctx->cfg.max_inner, ctx->cfg.approx_activation_iters, 0, 0,
                     0, 1, 0};
  const FitOut fo{out->theta, out->gamma, (c128*)out->alpha, out->K, out->beta, out->objective, out->iters,
                  out->n_evals, out->n_grid, out->status};
  const size_t smem = semifast_smem_bytes(kMaxSemifastK, rmax);
  record(ctx, 0, st, true);
  const cudaError_t e = launch_semifast_fit(ctx->cfg.precision != LSE_PREC_FP64, y_d, obs_d,
                                            (const SemiDesc*)ctx->semi_meta.dev.p, B, kMaxSemifastK, Nmax, Lmax, fc,
                                            tables(ctx), fo, ctx->semi.p, (int*)ctx->counter.p, grid, smem, st);
  record(ctx, 0, st, false);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "semifast fit kernel launch");
  if (!cap && st != ctx->stream && (sst = order_after(ctx, ctx->stream, st))) return sst;
  return LSE_OK;
}

lse_status lse_fit_incomplete(lse_ctx* ctx, const float* y, const int32_t* obs, int32_t M, int32_t N,
                              lse_result* out) {
  if (!ctx || !y || !obs || !out || M < 1 || N < 2 || M > N) return fail(ctx, LSE_EINVAL, "null argument or M, N out of range");
  cudaSetDevice(ctx->cfg.device);
  const size_t yb = (size_t)M * 2 * sizeof(float), ib = (size_t)M * sizeof(int32_t);
  const size_t ob = (size_t)M * 4 * sizeof(double) + 2 * sizeof(double) + 5 * sizeof(int32_t) + 256;
  lse_status s;
  if ((s = ensure(ctx, ctx->stage_in, yb + ib + 256))) return s;
  if ((s = ensure(ctx, ctx->stage_out, ob))) return s;
  char* in = (char*)ctx->stage_in.p;
  char* o = (char*)ctx->stage_out.p;
  lse_batch_out bo;
  bo.theta = (double*)o; o += M * sizeof(double);
  bo.gamma = (double*)o; o += M * sizeof(double);
  bo.alpha = (double*)o; o += M * 2 * sizeof(double);
  bo.beta = (double*)o; o += sizeof(double);
  bo.objective = (double*)o; o += sizeof(double);
  bo.K = (int32_t*)o; o += sizeof(int32_t);
  bo.iters = (int32_t*)o; o += sizeof(int32_t);
  bo.n_evals = (int32_t*)o; o += sizeof(int32_t);
  bo.n_grid = (int32_t*)o; o += sizeof(int32_t);
  bo.status = (int32_t*)o;
  const size_t obs_off = (yb + 255) & ~size_t(255);
  LSE_CUDA(ctx, cudaMemcpyAsync(in, y, yb, cudaMemcpyHostToDevice, ctx->stream));
  LSE_CUDA(ctx, cudaMemcpyAsync(in + obs_off, obs, ib, cudaMemcpyHostToDevice, ctx->stream));
  const int64_t offs[2] = {0, M};
  if ((s = lse_fit_incomplete_batch_d(ctx, (const float*)in, (const int32_t*)(in + obs_off), offs, 1, &N, &bo,
                                      ctx->stream)))
    return s;
  std::vector<char> host(ob);
  LSE_CUDA(ctx, cudaMemcpyAsync(host.data(), ctx->stage_out.p, ob, cudaMemcpyDeviceToHost, ctx->stream));
  LSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const char* h = host.data();
  const double* th = (const double*)h;
  const double* ga = th + M;
  const double* al = ga + M;
  const double* be = al + 2 * (size_t)M;
  const int32_t* ii = (const int32_t*)(be + 2);
  const int32_t K = ii[0];
  out->K = K;
  out->beta = be[0];
  out->objective = be[1];
  out->iters = ii[1];
  out->n_evals = ii[2];
  out->n_grid = ii[3];
  lse_status st = (lse_status)ii[4];
  if (K > out->K_cap) return LSE_ECAPACITY;
  for (int k = 0; k < K; ++k) {
    if (out->theta) out->theta[k] = th[k];
    if (out->gamma) out->gamma[k] = ga[k];
    if (out->alpha) { out->alpha[2 * k] = al[2 * k]; out->alpha[2 * k + 1] = al[2 * k + 1]; }
  }
  return st;
}

lse_status lse_eval_grid_batch_d(lse_ctx* ctx, const float* y_d, const int64_t* y_offsets, int32_t B,
                                 const double* theta_d, const double* gamma_d, const int64_t* k_offsets,
                                 const double* beta_d, const int32_t* L, int32_t dtype, void* q, void* dq, void* d2q,
                                 void* s, void* ds, void* d2s, void* stream) {
  if (!ctx || !y_d || !y_offsets || !k_offsets || !beta_d || !L || B < 1)
    return fail(ctx, LSE_EINVAL, "null argument or B < 1");
  const bool f32 = ctx->cfg.precision != LSE_PREC_FP64;
  if (dtype != (f32 ? LSE_F32 : LSE_F64))
    return fail(ctx, LSE_EINVAL, "dtype must be LSE_F64 for an FP64 context and LSE_F32 for a mixed one");
  cudaSetDevice(ctx->cfg.device);
  cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
  const bool cap = is_capturing(st);
  std::vector<InstDesc> d(B);
  int Nmax = 0, Lmax = 0;
  int64_t g = 0;
  for (int b = 0; b < B; ++b) {
    const int64_t n = y_offsets[b + 1] - y_offsets[b];
    const int64_t k = k_offsets[b + 1] - k_offsets[b];
    if (n < 2 || n > (1 << 17) || k < 0 || k > n)
      return fail(ctx, LSE_EINVAL, "instance " + std::to_string(b) + ": N or K out of range");
    if (!is_pow2(L[b]) || L[b] < 2 * n) return fail(ctx, LSE_EINVAL, "L must be a power of two >= 2N");
    d[b] = InstDesc{y_offsets[b], (int)n, L[b], k_offsets[b], (int)k, b, g};
    g += L[b];
    Nmax = std::max(Nmax, (int)n);
    Lmax = std::max(Lmax, (int)L[b]);
  }
  const int log2t = std::max(ilog2((uint32_t)Lmax), ilog2(2u * (uint32_t)Nmax));
  if (cap && (!ctx->tw64 || ctx->log2max < log2t))
    return fail(ctx, LSE_EINVAL, "twiddle tables must grow, which cannot be captured: make one call first");
  lse_status sst = ensure_tables(ctx, log2t);
  if (sst) return sst;
  const int64_t totN = y_offsets[B];
  const int sfmin = superfast_min_n(ctx->cfg.flags);
  int Nmin = Nmax;
  for (int b = 0; b < B; ++b) Nmin = std::min(Nmin, d[b].N);
  // grid tasks: on-chip ones first, then four-step ones with their offsets
  std::vector<int4> tasks(5 * (size_t)B);
  int n_small = 0;
  size_t g4_elems = 0;
  const int ntasks = grid_tasks(d.data(), B, f32, q, dq, d2q, s, ds, d2s, tasks.data(), &n_small, &g4_elems);
  const int n_large = ntasks - n_small;
  int Lmax_small = 0, Lmax_large = 0;
  for (int b = 0; b < B; ++b) {
    if (grid_on_chip(f32, d[b].L)) Lmax_small = std::max(Lmax_small, d[b].L);
    else Lmax_large = std::max(Lmax_large, d[b].L);
  }
  const size_t fws = factor_workspace_bytes(Nmax, sfmin) * B;
  const size_t gws = grid_workspace_bytes(g4_elems, f32);
  const size_t fac_bytes =
      (size_t)totN * (4 * sizeof(c128) + 3 * sizeof(c64)) + (size_t)B * (sizeof(double) + sizeof(int)) + 1024;
  if ((sst = ensure(ctx, ctx->ws, std::max(fws, gws), cap))) return sst;
  if ((sst = ensure(ctx, ctx->fac, fac_bytes, cap))) return sst;
  // launch metadata, one block: descriptors | grid task list
  const size_t desc_b = ((size_t)B * sizeof(InstDesc) + 15) & ~size_t(15);
  std::vector<char> meta(desc_b + (size_t)std::max(ntasks, 1) * sizeof(int4), 0);
  std::memcpy(meta.data(), d.data(), (size_t)B * sizeof(InstDesc));
  std::memcpy(meta.data() + desc_b, tasks.data(), (size_t)ntasks * sizeof(int4));
  if (!cap && st != ctx->stream && (sst = order_after(ctx, st, ctx->stream))) return sst;
  if ((sst = stage(ctx, ctx->grid_meta, meta.data(), meta.size(), st, cap))) return sst;
  const char* mdev = (const char*)ctx->grid_meta.dev.p;
  const InstDesc* desc_d = (const InstDesc*)mdev;
  const int4* tasks_d = (const int4*)(mdev + desc_b);
  c128* rho = (c128*)ctx->fac.p;
  c128* x = rho + totN;
  c128* omega = x + totN;  // 2N per instance (2N-1 used)
  double* delta = (double*)(omega + 2 * totN);
  int* status = (int*)(delta + B);
  c64* omega32 = (c64*)(((uintptr_t)(status + B) + 255) & ~(uintptr_t)255);
  c64* x32 = omega32 + 2 * totN;
  record(ctx, 1, st, true);
  cudaError_t e = launch_factor(ctx->cfg.precision == LSE_PREC_MIXED_DF, sfmin, Nmin, y_d, desc_d, B, Nmax, theta_d,
                                gamma_d, beta_d, tables(ctx), ctx->ws.p, rho, x, omega, omega32, x32, delta, status,
                                !(ctx->cfg.flags & LSE_FLAG_NO_CLUSTER), st);
  record(ctx, 1, st, false);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "factor kernel launch");
  // schedule of the on-chip grid FFT: cached, or tuned now on this batch
  // (tuning waits for the device once; it is skipped while capturing)
  int variant = 1;
  if (n_small) {
    const auto key = std::make_pair(f32 ? 1 : 0, Lmax_small);
    auto it = ctx->grid_variant.find(key);
    if (it != ctx->grid_variant.end()) {
      variant = it->second;
    } else if (!(ctx->cfg.flags & LSE_FLAG_NO_AUTOTUNE) && !cap) {
      const int nv = grid_variant_count();
      std::vector<cudaEvent_t> ev(nv + 1);
      for (auto& x : ev) LSE_CUDA(ctx, cudaEventCreate(&x));
      cudaEventRecord(ev[0], st);
      for (int v = 0; v < nv; ++v) {
        e = launch_grid(v, f32, desc_d, Lmax_small, 0, omega, x, omega32, x32, tables(ctx), ctx->ws.p, tasks_d,
                        n_small, 0, q, dq, d2q, s, ds, d2s, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "grid kernel launch (autotune)");
        cudaEventRecord(ev[v + 1], st);
      }
      LSE_CUDA(ctx, cudaEventSynchronize(ev[nv]));
      float best = 1e30f;
      for (int v = 0; v < nv; ++v) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[v], ev[v + 1]);
        if (ms < best) { best = ms; variant = v; }
      }
      for (auto& x : ev) cudaEventDestroy(x);
      ctx->grid_variant[key] = variant;
      save_autotune(ctx);
    }
  }
  record(ctx, 2, st, true);
  e = launch_grid(variant, f32, desc_d, Lmax_small, Lmax_large, omega, x, omega32, x32, tables(ctx), ctx->ws.p, tasks_d,
                  n_small, n_large, q, dq, d2q, s, ds, d2s, st);
  record(ctx, 2, st, false);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "grid kernel launch");
  if (!cap && st != ctx->stream && (sst = order_after(ctx, ctx->stream, st))) return sst;
  return LSE_OK;
}

lse_status lse_eval_grid(lse_ctx* ctx, const float* y, int32_t N, const double* theta, const double* gamma,
                         int32_t K, double beta, int32_t L, int32_t dtype, void* q, void* dq, void* d2q, void* s,
                         void* ds, void* d2s) {
  if (!ctx || !y || N < 2 || K < 0 || K > N || (K > 0 && (!theta || !gamma)) || !(beta > 0.0))
    return fail(ctx, LSE_EINVAL, "bad argument");
  const bool f32 = ctx->cfg.precision != LSE_PREC_FP64;
  if (dtype != (f32 ? LSE_F32 : LSE_F64))
    return fail(ctx, LSE_EINVAL, "dtype must be LSE_F64 for an FP64 context and LSE_F32 for a mixed one");
  if (!is_pow2(L) || L < 2 * N) return fail(ctx, LSE_EINVAL, "L must be a power of two >= 2N");
  cudaSetDevice(ctx->cfg.device);
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  const size_t yb = (size_t)N * 2 * sizeof(float);
  const size_t pb = ((size_t)2 * K + 1) * sizeof(double);
  const size_t outb = (size_t)L * 9 * es;
  lse_status st;
  if ((st = ensure(ctx, ctx->stage_in, yb + pb + 512))) return st;
  if ((st = ensure(ctx, ctx->stage_out, outb + 512))) return st;
  char* in = (char*)ctx->stage_in.p;
  float* yd = (float*)in;
  double* thd = (double*)(in + ((yb + 255) & ~size_t(255)));
  double* gad = thd + K;
  double* bed = gad + K;
  LSE_CUDA(ctx, cudaMemcpyAsync(yd, y, yb, cudaMemcpyHostToDevice, ctx->stream));
  if (K) {
    LSE_CUDA(ctx, cudaMemcpyAsync(thd, theta, K * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    LSE_CUDA(ctx, cudaMemcpyAsync(gad, gamma, K * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  }
  LSE_CUDA(ctx, cudaMemcpyAsync(bed, &beta, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  char* o = (char*)ctx->stage_out.p;
  void* dev[6];
  void* host[6] = {q, dq, d2q, s, ds, d2s};
  const size_t sz[6] = {2 * L * es, 2 * L * es, 2 * L * es, L * es, L * es, L * es};
  for (int i = 0; i < 6; ++i) {
    dev[i] = host[i] ? (void*)o : nullptr;
    o += sz[i];
  }
  const int64_t yo[2] = {0, N}, ko[2] = {0, K};
  const int32_t Ls[1] = {L};
  if ((st = lse_eval_grid_batch_d(ctx, yd, yo, 1, thd, gad, ko, bed, Ls, dtype, dev[0], dev[1], dev[2], dev[3],
                                  dev[4], dev[5], ctx->stream)))
    return st;
  for (int i = 0; i < 6; ++i)
    if (host[i]) LSE_CUDA(ctx, cudaMemcpyAsync(host[i], dev[i], sz[i], cudaMemcpyDeviceToHost, ctx->stream));
  int fst = 0;
  const int* status = (const int*)((double*)((c128*)ctx->fac.p + 4 * (size_t)N) + 1);
  LSE_CUDA(ctx, cudaMemcpyAsync(&fst, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  LSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (fst) return fail(ctx, LSE_ENUMERIC, "Levinson recursion broke down");
  return LSE_OK;
}

}  // extern "C"
