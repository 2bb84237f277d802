// lse_serve.cu -- continuous-batching server for line-spectral fits.
//
// Requests (y, N) arrive one at a time.  The server keeps a FIFO of pending
// requests and a set of slots, each a CUDA stream with its own context and
// device buffers.  lse_serve_poll (non-blocking) harvests the slots whose
// work has finished and hands their results back, then admits pending
// requests: an idle slot takes the oldest pending requests (up to max_group)
// whose device memory fits what the budget leaves, copies their inputs in
// and launches one persistent fit kernel over them.  Requests that arrive
// while other groups run start on another slot, so their work overlaps on
// the device.  Every instance is computed with the same arithmetic as a lone
// lse_fit: one thread block per instance, or a two-block cluster on the
// double-float path when the group is small enough (the two differ only in
// the order the recursion's inner products are summed).  So a result does
// not depend on the mix it ran in, bit for bit whenever the group and the
// lone fit run in the same mode (always with LSE_FLAG_NO_CLUSTER), and to
// rounding otherwise.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "../../include/lse.h"
#include "lse_internal.h"

using namespace lse;

namespace {

struct Request {
  int64_t id;
  int32_t N;
  std::vector<float> y;  // complex64, interleaved
};

struct Slot {
  lse_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;  // the context's own stream
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<Request> group;
  std::vector<int64_t> offsets;
  // device buffers
  float* y_d = nullptr;
  char* out_d = nullptr;
  size_t cap_n = 0, cap_b = 0;  // capacity (sum N, B) of the buffers
  size_t dev_bytes = 0;          // bytes this slot holds (buffers + context workspace estimate)
  // pinned host staging
  float* y_h = nullptr;
  char* out_h = nullptr;
};

size_t out_bytes(size_t n, size_t b) { return n * 4 * sizeof(double) + b * (2 * sizeof(double) + 5 * sizeof(int)) + 256; }

int default_L(int N) { return 1 << (int)std::lround(std::log2(8.0 * N)); }

}  // namespace

struct lse_server {
  lse_config cfg;
  int max_group = 0;
  uint64_t budget = 0;
  std::vector<Slot> slots;
  std::deque<Request> pending;
  std::deque<lse_serve_result> done;  // harvested, not yet returned
  std::deque<std::vector<double>> storage;  // theta/gamma/alpha of harvested results
  int sm_count = 0;
  uint64_t in_use = 0;
  int64_t submitted = 0, completed = 0, rejected = 0;
};

namespace {

// device memory a group needs on a slot: fit workspace (one unit per
// instance up to the SM count) plus the input and output buffers
uint64_t group_bytes(const lse_server* s, const std::vector<Request>& g) {
  int Nmax = 0, Lmax = 0;
  size_t sumN = 0;
  for (const Request& r : g) {
    Nmax = std::max(Nmax, r.N);
    Lmax = std::max(Lmax, s->cfg.grid_size ? s->cfg.grid_size : default_L(r.N));
    sumN += r.N;
  }
  const size_t blocks = std::min<size_t>(g.size(), (size_t)s->sm_count);
  return fit_workspace_bytes(Nmax, Lmax, s->cfg.precision) * blocks + sumN * 2 * sizeof(float) +
         out_bytes(sumN, g.size());
}

lse_status grow_slot(Slot& sl, size_t n, size_t b) {
  if (sl.cap_n >= n && sl.cap_b >= b) return LSE_OK;
  cudaStreamSynchronize(sl.stream);
  if (sl.y_d) cudaFree(sl.y_d);
  if (sl.out_d) cudaFree(sl.out_d);
  if (sl.y_h) cudaFreeHost(sl.y_h);
  if (sl.out_h) cudaFreeHost(sl.out_h);
  sl.y_d = nullptr; sl.out_d = nullptr; sl.y_h = nullptr; sl.out_h = nullptr;
  n = std::max(n, 2 * sl.cap_n);
  b = std::max(b, 2 * sl.cap_b);
  if (cudaMalloc(&sl.y_d, n * 2 * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&sl.out_d, out_bytes(n, b)) != cudaSuccess ||
      cudaMallocHost(&sl.y_h, n * 2 * sizeof(float)) != cudaSuccess ||
      cudaMallocHost(&sl.out_h, out_bytes(n, b)) != cudaSuccess) {
    sl.cap_n = sl.cap_b = 0;
    return LSE_ENOMEM;
  }
  sl.cap_n = n;
  sl.cap_b = b;
  return LSE_OK;
}

lse_batch_out carve_out(char* base, size_t tot, size_t B) {
  lse_batch_out o;
  char* p = base;
  o.theta = (double*)p; p += tot * sizeof(double);
  o.gamma = (double*)p; p += tot * sizeof(double);
  o.alpha = (double*)p; p += tot * 2 * sizeof(double);
  o.beta = (double*)p; p += B * sizeof(double);
  o.objective = (double*)p; p += B * sizeof(double);
  o.K = (int32_t*)p; p += B * sizeof(int);
  o.iters = (int32_t*)p; p += B * sizeof(int);
  o.n_evals = (int32_t*)p; p += B * sizeof(int);
  o.n_grid = (int32_t*)p; p += B * sizeof(int);
  o.status = (int32_t*)p;
  return o;
}

lse_status launch_group(lse_server* s, Slot& sl) {
  const size_t B = sl.group.size();
  sl.offsets.assign(B + 1, 0);
  for (size_t i = 0; i < B; ++i) sl.offsets[i + 1] = sl.offsets[i] + sl.group[i].N;
  const size_t tot = (size_t)sl.offsets[B];
  lse_status st = grow_slot(sl, tot, B);
  if (st) return st;
  for (size_t i = 0; i < B; ++i)
    std::memcpy(sl.y_h + 2 * sl.offsets[i], sl.group[i].y.data(), sl.group[i].y.size() * sizeof(float));
  if (cudaMemcpyAsync(sl.y_d, sl.y_h, tot * 2 * sizeof(float), cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
    return LSE_ECUDA;
  const lse_batch_out o = carve_out(sl.out_d, tot, B);
  st = lse_fit_batch_d(sl.ctx, sl.y_d, sl.offsets.data(), (int32_t)B, &o, sl.stream);
  if (st) return st;
  if (cudaMemcpyAsync(sl.out_h, sl.out_d, out_bytes(tot, B), cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
      cudaEventRecord(sl.done, sl.stream) != cudaSuccess)
    return LSE_ECUDA;
  sl.busy = true;
  return LSE_OK;
}

void harvest(lse_server* s, Slot& sl) {
  const size_t B = sl.group.size();
  const size_t tot = (size_t)sl.offsets[B];
  const lse_batch_out o = carve_out(sl.out_h, tot, B);
  for (size_t i = 0; i < B; ++i) {
    lse_serve_result r;
    std::memset(&r, 0, sizeof(r));
    r.request_id = sl.group[i].id;
    r.status = o.status[i];
    r.K = o.K[i];
    r.N = sl.group[i].N;
    r.beta = o.beta[i];
    r.objective = o.objective[i];
    r.iters = o.iters[i];
    r.n_evals = o.n_evals[i];
    const int64_t off = sl.offsets[i];
    std::vector<double> buf(4 * (size_t)r.K);
    for (int k = 0; k < r.K; ++k) {
      buf[k] = o.theta[off + k];
      buf[r.K + k] = o.gamma[off + k];
      buf[2 * r.K + 2 * k] = o.alpha[2 * (off + k)];
      buf[2 * r.K + 2 * k + 1] = o.alpha[2 * (off + k) + 1];
    }
    s->storage.push_back(std::move(buf));
    s->done.push_back(r);
  }
  s->completed += (int64_t)B;
  s->in_use -= sl.dev_bytes;
  sl.dev_bytes = 0;
  sl.group.clear();
  sl.busy = false;
}

void admit(lse_server* s) {
  for (Slot& sl : s->slots) {
    if (s->pending.empty()) return;
    if (sl.busy) continue;
    std::vector<Request> g;
    while (!s->pending.empty() && (int)g.size() < s->max_group) {
      g.push_back(s->pending.front());
      if (s->budget && s->in_use + group_bytes(s, g) > s->budget) {
        g.pop_back();
        break;
      }
      s->pending.pop_front();
    }
    if (g.empty()) return;  // the oldest request waits for memory to free up
    sl.group = std::move(g);
    sl.dev_bytes = group_bytes(s, sl.group);
    s->in_use += sl.dev_bytes;
    if (launch_group(s, sl) != LSE_OK) {
      // report the group as failed rather than losing it
      for (const Request& r : sl.group) {
        lse_serve_result e;
        std::memset(&e, 0, sizeof(e));
        e.request_id = r.id;
        e.status = LSE_ECUDA;
        e.N = r.N;
        s->storage.emplace_back();
        s->done.push_back(e);
      }
      s->in_use -= sl.dev_bytes;
      sl.dev_bytes = 0;
      sl.group.clear();
      sl.busy = false;
    }
  }
}

}  // namespace

extern "C" {

lse_status lse_serve_create(const lse_config* cfg, int32_t streams, int32_t max_group, lse_server** out) {
  if (!out || streams < 1 || streams > 64 || max_group < 1) return LSE_EINVAL;
  *out = nullptr;
  lse_server* s = new lse_server();
  if (cfg) s->cfg = *cfg; else lse_config_default(&s->cfg);
  s->budget = s->cfg.hbm_budget_bytes;
  s->max_group = max_group;
  lse_config c = s->cfg;
  c.hbm_budget_bytes = 0;  // the server enforces the budget across its slots
  s->slots.resize(streams);
  for (Slot& sl : s->slots) {
    lse_status st = lse_create(&c, &sl.ctx);
    if (st) {
      lse_serve_destroy(s);
      return st;
    }
    sl.stream = lse_ctx_stream(sl.ctx);
    if (cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
      lse_serve_destroy(s);
      return LSE_ECUDA;
    }
  }
  cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->cfg.device);
  *out = s;
  return LSE_OK;
}

lse_status lse_serve_submit(lse_server* s, const float* y, int32_t N, int64_t request_id) {
  if (!s || !y || N < 2 || N > (1 << 17)) return LSE_EINVAL;
  Request r;
  r.id = request_id;
  r.N = N;
  if (s->budget && group_bytes(s, std::vector<Request>{Request{request_id, N, {}}}) > s->budget) {
    ++s->rejected;
    return LSE_EBUDGET;
  }
  r.y.assign(y, y + 2 * (size_t)N);
  s->pending.push_back(std::move(r));
  ++s->submitted;
  admit(s);
  return LSE_OK;
}

int32_t lse_serve_poll(lse_server* s, lse_serve_result* results, int32_t cap) {
  if (!s) return -1;
  for (Slot& sl : s->slots)
    if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) harvest(s, sl);
  admit(s);
  int32_t n = 0;
  while (n < cap && !s->done.empty()) {
    lse_serve_result r = s->done.front();
    s->done.pop_front();
    // results[n] arrays belong to the caller; copy what fits
    const std::vector<double>& buf = s->storage.front();
    if (results) {
      lse_serve_result& o = results[n];
      double* th = o.theta;
      double* ga = o.gamma;
      double* al = o.alpha;
      const int kc = o.K_cap;
      o = r;
      o.theta = th;
      o.gamma = ga;
      o.alpha = al;
      o.K_cap = kc;
      if (r.K > kc) {
        o.status = LSE_ECAPACITY;
      } else {
        for (int k = 0; k < r.K; ++k) {
          if (th) th[k] = buf[k];
          if (ga) ga[k] = buf[r.K + k];
          if (al) { al[2 * k] = buf[2 * r.K + 2 * k]; al[2 * k + 1] = buf[2 * r.K + 2 * k + 1]; }
        }
      }
    }
    s->storage.pop_front();
    ++n;
  }
  return n;
}

int32_t lse_serve_in_flight(const lse_server* s) {
  if (!s) return 0;
  int32_t n = (int32_t)s->pending.size() + (int32_t)s->done.size();
  for (const Slot& sl : s->slots)
    if (sl.busy) n += (int32_t)sl.group.size();
  return n;
}

uint64_t lse_serve_device_bytes(const lse_server* s) { return s ? s->in_use : 0; }

lse_status lse_serve_reserve(lse_server* s, int32_t n_max) {
  if (!s || n_max < 2 || n_max > (1 << 17)) return LSE_EINVAL;
  const int L = s->cfg.grid_size ? s->cfg.grid_size : default_L(n_max);
  if (L < 2 * n_max) return LSE_EINVAL;
  for (Slot& sl : s->slots) {
    if (sl.busy) {  // its group must finish before its buffers can change
      cudaEventSynchronize(sl.done);
      harvest(s, sl);
    }
    lse_status st = grow_slot(sl, (size_t)s->max_group * (size_t)n_max, (size_t)s->max_group);
    if (st) return st;
    if ((st = lse_ctx_reserve_fit(sl.ctx, n_max, L, s->max_group))) return st;
  }
  return LSE_OK;
}

void lse_serve_destroy(lse_server* s) {
  if (!s) return;
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.y_d) cudaFree(sl.y_d);
    if (sl.out_d) cudaFree(sl.out_d);
    if (sl.y_h) cudaFreeHost(sl.y_h);
    if (sl.out_h) cudaFreeHost(sl.out_h);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.ctx) lse_destroy(sl.ctx);
  }
  delete s;
}

}  // extern "C"
