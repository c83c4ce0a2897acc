// C ABI of the blocked Floyd-Warshall APSP library (declared in include/apsp.h).
//
// The problem is the paper's Sec. 3 (lengths of all pairs shortest paths of an
// undirected weighted graph given by its adjacency matrix); the solver is the
// three-phase blocked algorithm of Sec. 4.4/4.5 (Alg. 3, Alg. 4) run as CUDA
// kernels on one GPU.  Nothing here computes on the host: every step of a
// solve is a kernel launched on the caller's stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/apsp.h"
#include "fw_launch.h"

namespace {

constexpr int64_t kDefaultMaxEdges = int64_t(1) << 26;

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct Request {
  uint64_t ticket = 0;
  apsp_request req{};
  int64_t bytes = 0;
  bool admitted = false;
  bool finished = false;  // done event observed complete
  bool released = false;
  apsp_status err = APSP_OK;
  void *D = nullptr;
  void *colT = nullptr;
  int *status = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t copy_ev = nullptr;
  cudaEvent_t done_ev = nullptr;
};

// Event pairs around phase launches (apsp_profile).
struct Profiler : apsp::PhaseTimer {
  struct Pair {
    cudaEvent_t a, b;
    int phase;
    double relax;
  };
  std::vector<Pair> pairs;       // recorded, not yet read
  std::vector<cudaEvent_t> pool; // free events
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  cudaEvent_t pending = nullptr;
  void before(int, cudaStream_t s) override {
    pending = get();
    cudaEventRecord(pending, s);
  }
  void after(int phase, cudaStream_t s, double relax) override {
    cudaEvent_t b = get();
    cudaEventRecord(b, s);
    pairs.push_back({pending, b, phase, relax});
    pending = nullptr;
  }
  void read(int64_t *launches, double *ms, double *relax) {
    for (int p = 0; p < 3; ++p) {
      if (launches) launches[p] = 0;
      if (ms) ms[p] = 0;
      if (relax) relax[p] = 0;
    }
    for (Pair &q : pairs) {
      cudaEventSynchronize(q.b);
      float t = 0.f;
      cudaEventElapsedTime(&t, q.a, q.b);
      if (launches) launches[q.phase] += 1;
      if (ms) ms[q.phase] += t;
      if (relax) relax[q.phase] += q.relax;
      pool.push_back(q.a);
      pool.push_back(q.b);
    }
    pairs.clear();
  }
  ~Profiler() {
    for (Pair &q : pairs) {
      cudaEventDestroy(q.a);
      cudaEventDestroy(q.b);
    }
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

}  // namespace

struct apsp_handle {
  apsp_config cfg{};
  std::mutex mu;  // serializes solve-path workspace use and last_error
  void *colT = nullptr;
  size_t colT_bytes = 0;
  void *ws16 = nullptr;
  size_t ws16_bytes = 0;
  int *d_status = nullptr;
  int *h_status = nullptr;  // pinned
  std::string last_error;
  std::atomic<int64_t> launches{0};
  std::unique_ptr<Profiler> prof;  // non-null while apsp_profile(h, 1) is on

  // ---- request loop
  std::mutex smu;
  std::condition_variable scv;
  std::thread worker;
  bool worker_started = false;
  bool stopping = false;
  uint64_t next_ticket = 1;
  std::deque<uint64_t> queue;                         // waiting for admission (FIFO)
  std::map<uint64_t, std::unique_ptr<Request>> reqs;  // every live ticket
  int64_t budget = 0;
  int64_t used = 0;
  int running = 0;
  std::vector<cudaStream_t> free_streams;
};

namespace {

thread_local std::string tls_error;

apsp_status set_err(apsp_handle *h, apsp_status st, const std::string &msg) {
  if (h) {
    std::lock_guard<std::mutex> g(h->mu);
    h->last_error = msg;
  }
  return st;
}

apsp_status cuda_fail(apsp_handle *h, cudaError_t e, const char *where) {
  return set_err(h, APSP_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define APSP_CUDA(h, call)                                   \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return cuda_fail((h), _e, #call); \
  } while (0)

// Grows a device buffer (the old one may still be read by work already queued
// on some stream, so the device is synchronized before it is freed).
cudaError_t ensure(void **p, size_t *cur, size_t need) {
  if (*cur >= need && *p) return cudaSuccess;
  if (*p) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    cudaFree(*p);
    *p = nullptr;
    *cur = 0;
  }
  cudaError_t e = cudaMalloc(p, need);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  *cur = need;
  return cudaSuccess;
}

bool valid_dtype(int d) { return d == APSP_I32 || d == APSP_U16 || d == APSP_F32; }

int64_t panel_ld(int64_t n) { return round_up(n > 0 ? n : 1, 256); }

// Enqueues the q rounds on D (already holding W) using the handle's panel buffer.
apsp_status run_rounds_locked(apsp_handle *h, int dtype, void *D, int64_t n, int64_t ld, cudaStream_t s) {
  const int64_t bk = apsp::round_width(dtype);
  const int64_t ldT = panel_ld(n);
  const size_t need = (size_t)bk * ldT * 4;  // panel buffer of 32-bit words
  cudaError_t e = ensure(&h->colT, &h->colT_bytes, need);
  if (e != cudaSuccess) {
    h->last_error = std::string("panel workspace: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? APSP_E_NOMEM : APSP_E_CUDA;
  }
  int64_t l = 0;
  e = apsp::launch_rounds(dtype, D, ld, n, h->colT, ldT, s, &l, h->prof.get());
  h->launches += l;
  if (e != cudaSuccess) {
    h->last_error = std::string("rounds: ") + cudaGetErrorString(e);
    return APSP_E_CUDA;
  }
  return APSP_OK;
}

apsp_status solve_locked(apsp_handle *h, int dtype, const void *W, int64_t n, int64_t ld, void *D, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(h->d_status, 0, sizeof(int), s);
  if (e != cudaSuccess) {
    h->last_error = std::string("status reset: ") + cudaGetErrorString(e);
    return APSP_E_CUDA;
  }
  if (n == 0) return APSP_OK;
  int64_t l = 0;
  if (dtype != APSP_AUTO) {
    e = apsp::launch_ingest(dtype, W, D, n, ld, h->d_status, s, &l);
    h->launches += l;
    if (e != cudaSuccess) {
      h->last_error = std::string("ingest: ") + cudaGetErrorString(e);
      return APSP_E_CUDA;
    }
    return run_rounds_locked(h, dtype, D, n, ld, s);
  }
  // AUTO: int32 in and out; packed 16-bit when the bound allows (north-star
  // precision selection).  The bound synchronizes the stream.
  e = apsp::launch_ingest(APSP_I32, W, const_cast<void *>(W), n, ld, h->d_status, s, &l);  // checks only (W == D: no copy)
  if (e != cudaSuccess) {
    h->launches += l;
    h->last_error = std::string("ingest: ") + cudaGetErrorString(e);
    return APSP_E_CUDA;
  }
  int64_t bound = 0;
  int ok = 0;
  e = apsp::bound_from_dense(static_cast<const int32_t *>(W), n, ld, std::max<int64_t>(kDefaultMaxEdges, 32 * n), s,
                             &bound, &ok, &l);
  h->launches += l;
  l = 0;
  if (e != cudaSuccess) {
    h->last_error = std::string("16-bit bound: ") + cudaGetErrorString(e);
    return APSP_E_CUDA;
  }
  if (ok) {
    const int64_t ld16 = round_up(n, 8);
    e = ensure(&h->ws16, &h->ws16_bytes, (size_t)n * ld16 * 2);
    if (e == cudaSuccess) {
      uint16_t *P = static_cast<uint16_t *>(h->ws16);
      e = apsp::launch_pack(static_cast<const int32_t *>(W), ld, P, ld16, n, s, &l);
      h->launches += l;
      l = 0;
      if (e != cudaSuccess) {
        h->last_error = std::string("pack: ") + cudaGetErrorString(e);
        return APSP_E_CUDA;
      }
      apsp_status st = run_rounds_locked(h, APSP_U16, P, n, ld16, s);
      if (st != APSP_OK) return st;
      e = apsp::launch_unpack(P, ld16, static_cast<int32_t *>(D), ld, n, s, &l);
      h->launches += l;
      if (e != cudaSuccess) {
        h->last_error = std::string("unpack: ") + cudaGetErrorString(e);
        return APSP_E_CUDA;
      }
      return APSP_OK;
    }
    // no room for the 16-bit copy: solve in int32 instead
    cudaGetLastError();
  }
  if (W != D) {
    e = cudaMemcpy2DAsync(D, (size_t)ld * 4, W, (size_t)ld * 4, (size_t)n * 4, (size_t)n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
      h->last_error = std::string("copy: ") + cudaGetErrorString(e);
      return APSP_E_CUDA;
    }
  }
  return run_rounds_locked(h, APSP_I32, D, n, ld, s);
}

}  // namespace

extern "C" {

void apsp_config_default(apsp_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->dtype = APSP_I32;
  cfg->block_k = 0;
  cfg->max_batch = 64;
  cfg->queue_depth = 4096;
  cfg->memory_budget = 0;
  cfg->spin_limit = 0;
}

apsp_status apsp_create(apsp_handle **out, const apsp_config *cfg) {
  if (!out) return APSP_E_INVALID;
  *out = nullptr;
  apsp_config c;
  apsp_config_default(&c);
  if (cfg) c = *cfg;
  if (c.dtype != APSP_AUTO && !valid_dtype(c.dtype)) return APSP_E_INVALID;
  if (c.block_k != 0 && c.block_k != 64) return APSP_E_INVALID;
  if (c.max_batch <= 0) c.max_batch = 64;
  if (c.queue_depth <= 0) c.queue_depth = 4096;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) return APSP_E_CUDA;
  if (cudaSetDevice(c.device) != cudaSuccess) return APSP_E_CUDA;
  std::unique_ptr<apsp_handle> h(new apsp_handle());
  h->cfg = c;
  if (cudaMalloc(&h->d_status, 64) != cudaSuccess) return APSP_E_CUDA;
  if (cudaMemset(h->d_status, 0, 64) != cudaSuccess) return APSP_E_CUDA;
  if (cudaMallocHost(&h->h_status, 64) != cudaSuccess) {
    cudaFree(h->d_status);
    return APSP_E_CUDA;
  }
  *out = h.release();
  return APSP_OK;
}

static void free_request_device(Request *r) {
  if (r->D) cudaFree(r->D);
  if (r->colT) cudaFree(r->colT);
  if (r->status) cudaFree(r->status);
  if (r->copy_ev) cudaEventDestroy(r->copy_ev);
  if (r->done_ev) cudaEventDestroy(r->done_ev);
  r->D = r->colT = nullptr;
  r->status = nullptr;
  r->copy_ev = r->done_ev = nullptr;
}

apsp_status apsp_destroy(apsp_handle *h) {
  if (!h) return APSP_OK;
  cudaSetDevice(h->cfg.device);
  {
    std::unique_lock<std::mutex> g(h->smu);
    h->stopping = true;
  }
  h->scv.notify_all();
  if (h->worker.joinable()) h->worker.join();
  cudaDeviceSynchronize();
  for (auto &kv : h->reqs) free_request_device(kv.second.get());
  h->reqs.clear();
  for (cudaStream_t s : h->free_streams) cudaStreamDestroy(s);
  if (h->colT) cudaFree(h->colT);
  if (h->ws16) cudaFree(h->ws16);
  if (h->d_status) cudaFree(h->d_status);
  if (h->h_status) cudaFreeHost(h->h_status);
  delete h;
  return APSP_OK;
}

apsp_status apsp_solve_t(apsp_handle *h, int dtype, const void *W, int64_t n, int64_t ld, void *D, void *stream) {
  if (!h) return APSP_E_INVALID;
  if (dtype != APSP_AUTO && !valid_dtype(dtype)) return set_err(h, APSP_E_INVALID, "unknown dtype");
  if (n < 0 || ld < n || (n > 0 && (!W || !D))) return set_err(h, APSP_E_INVALID, "need n >= 0, ld >= n, W and D");
  if (n > (int64_t(1) << 31) - 1) return set_err(h, APSP_E_INVALID, "n too large");
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  std::lock_guard<std::mutex> g(h->mu);
  return solve_locked(h, dtype, W, n, ld, D, static_cast<cudaStream_t>(stream));
}

apsp_status apsp_solve(apsp_handle *h, const void *W, int64_t n, int64_t ld, void *D, void *stream) {
  if (!h) return APSP_E_INVALID;
  return apsp_solve_t(h, h->cfg.dtype, W, n, ld, D, stream);
}

apsp_status apsp_solve_edges(apsp_handle *h, int dtype, const int32_t *src, const int32_t *dst, const void *w,
                             int64_t m, int64_t n, void *D, int64_t ld, void *stream) {
  if (!h) return APSP_E_INVALID;
  if (dtype != APSP_AUTO && !valid_dtype(dtype)) return set_err(h, APSP_E_INVALID, "unknown dtype");
  if (n < 0 || ld < n || m < 0 || (n > 0 && !D) || (m > 0 && (!src || !dst || !w)))
    return set_err(h, APSP_E_INVALID, "bad edge-list arguments");
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(h->mu);
  e = cudaMemsetAsync(h->d_status, 0, sizeof(int), s);
  if (e != cudaSuccess) {
    h->last_error = std::string("status reset: ") + cudaGetErrorString(e);
    return APSP_E_CUDA;
  }
  if (n == 0) return APSP_OK;
  int solve_dtype = dtype;
  int64_t l = 0;
  if (dtype == APSP_U16 || dtype == APSP_AUTO) {
    int64_t bound = 0;
    int ok = 0;
    e = apsp::bound_from_edges(src, dst, w, dtype == APSP_U16 ? 1 : 0, m, n, s, &bound, &ok, &l);
    h->launches += l;
    l = 0;
    if (e != cudaSuccess) {
      h->last_error = std::string("16-bit bound: ") + cudaGetErrorString(e);
      return APSP_E_CUDA;
    }
    if (dtype == APSP_U16 && !ok) {
      h->last_error = "16-bit bound fails: 2*eccentricity = " + std::to_string(bound) + " >= 32767";
      return APSP_E_RANGE;
    }
    solve_dtype = (dtype == APSP_U16) ? APSP_U16 : APSP_I32;
    if (dtype == APSP_AUTO && ok) {
      // dense int32 output, solved through a packed copy
      const int64_t ld16 = round_up(n, 8);
      e = ensure(&h->ws16, &h->ws16_bytes, (size_t)n * ld16 * 2);
      if (e == cudaSuccess) {
        uint16_t *P = static_cast<uint16_t *>(h->ws16);
        e = apsp::launch_densify(APSP_I32, src, dst, w, m, D, n, ld, h->d_status, s, &l);
        if (e == cudaSuccess) e = apsp::launch_pack(static_cast<const int32_t *>(D), ld, P, ld16, n, s, &l);
        h->launches += l;
        l = 0;
        if (e != cudaSuccess) return cuda_fail(h, e, "densify/pack");
        apsp_status st = run_rounds_locked(h, APSP_U16, P, n, ld16, s);
        if (st != APSP_OK) return st;
        e = apsp::launch_unpack(P, ld16, static_cast<int32_t *>(D), ld, n, s, &l);
        h->launches += l;
        if (e != cudaSuccess) return cuda_fail(h, e, "unpack");
        return APSP_OK;
      }
      cudaGetLastError();
    }
  }
  e = apsp::launch_densify(solve_dtype, src, dst, w, m, D, n, ld, h->d_status, s, &l);
  h->launches += l;
  if (e != cudaSuccess) {
    h->last_error = std::string("densify: ") + cudaGetErrorString(e);
    return APSP_E_CUDA;
  }
  return run_rounds_locked(h, solve_dtype, D, n, ld, s);
}

apsp_status apsp_last_status(apsp_handle *h, void *stream) {
  if (!h) return APSP_E_INVALID;
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(h->mu);
  e = cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    h->last_error = std::string("status read: ") + cudaGetErrorString(e);
    return APSP_E_CUDA;
  }
  const int st = *h->h_status;
  if (st & 1) {
    h->last_error = "input check: negative weight, bad vertex id or non-zero diagonal";
    return APSP_E_INVALID;
  }
  if (st & 2) {
    h->last_error = "input check: a finite weight is >= INF";
    return APSP_E_RANGE;
  }
  return APSP_OK;
}

apsp_status apsp_int16_bound(apsp_handle *h, const int32_t *W, int64_t n, int64_t ld, int64_t *bound, int *ok,
                             void *stream) {
  if (!h || !bound || !ok || n < 0 || ld < n || (n > 0 && !W)) return APSP_E_INVALID;
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  int64_t l = 0;
  e = apsp::bound_from_dense(W, n, ld, std::max<int64_t>(kDefaultMaxEdges, 32 * n), static_cast<cudaStream_t>(stream),
                             bound, ok, &l);
  h->launches += l;
  if (e != cudaSuccess) return cuda_fail(h, e, "16-bit bound");
  return APSP_OK;
}

apsp_status apsp_minplus(apsp_handle *h, int dtype, const void *A, int64_t lda, const void *B, int64_t ldb, void *C,
                         int64_t ldc, int64_t m, int64_t k, int64_t n, void *stream) {
  if (!h || !valid_dtype(dtype)) return APSP_E_INVALID;
  if (m < 0 || k < 0 || n < 0 || lda < k || ldb < n || ldc < n) return set_err(h, APSP_E_INVALID, "bad shape");
  if (m > 0 && n > 0 && (!C || (k > 0 && (!A || !B)))) return set_err(h, APSP_E_INVALID, "null matrix");
  if ((m + 127) / 128 > 65535) return set_err(h, APSP_E_INVALID, "m too large");
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  int64_t l = 0;
  e = apsp::launch_minplus(dtype, A, lda, B, ldb, C, ldc, m, k, n, static_cast<cudaStream_t>(stream), &l);
  h->launches += l;
  if (e != cudaSuccess) return cuda_fail(h, e, "minplus");
  return APSP_OK;
}

apsp_status apsp_pack_u16(const int32_t *src, int64_t lds, uint16_t *dst, int64_t ldd, int64_t n, void *stream) {
  if (n < 0 || lds < n || ldd < n || (n > 0 && (!src || !dst))) return APSP_E_INVALID;
  return apsp::launch_pack(src, lds, dst, ldd, n, static_cast<cudaStream_t>(stream), nullptr) == cudaSuccess
             ? APSP_OK
             : APSP_E_CUDA;
}

apsp_status apsp_unpack_u16(const uint16_t *src, int64_t lds, int32_t *dst, int64_t ldd, int64_t n, void *stream) {
  if (n < 0 || lds < n || ldd < n || (n > 0 && (!src || !dst))) return APSP_E_INVALID;
  return apsp::launch_unpack(src, lds, dst, ldd, n, static_cast<cudaStream_t>(stream), nullptr) == cudaSuccess
             ? APSP_OK
             : APSP_E_CUDA;
}

const char *apsp_strerror(apsp_status s) {
  switch (s) {
    case APSP_OK: return "ok";
    case APSP_E_INVALID: return "invalid argument";
    case APSP_E_CUDA: return "CUDA error";
    case APSP_E_NOMEM: return "out of memory (budget)";
    case APSP_E_RANGE: return "value out of range";
    case APSP_E_BUSY: return "request queue full";
    case APSP_E_NOTFOUND: return "unknown ticket";
    case APSP_E_TIMEOUT: return "device wait timed out";
    case APSP_E_CANCELLED: return "cancelled";
    case APSP_E_NOTREADY: return "not ready";
    case APSP_E_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *apsp_last_error(apsp_handle *h) {
  if (!h) return "null handle";
  std::lock_guard<std::mutex> g(h->mu);
  tls_error = h->last_error;
  return tls_error.c_str();
}

int64_t apsp_launch_count(apsp_handle *h) { return h ? h->launches.load() : 0; }

apsp_status apsp_profile(apsp_handle *h, int enable) {
  if (!h) return APSP_E_INVALID;
  cudaSetDevice(h->cfg.device);
  std::lock_guard<std::mutex> g(h->mu);
  if (enable && !h->prof) h->prof.reset(new Profiler());
  if (!enable && h->prof) {
    cudaDeviceSynchronize();
    h->prof.reset();
  }
  return APSP_OK;
}

apsp_status apsp_profile_read(apsp_handle *h, int64_t launches[3], double ms[3], double relaxations[3]) {
  if (!h) return APSP_E_INVALID;
  cudaSetDevice(h->cfg.device);
  std::lock_guard<std::mutex> g(h->mu);
  if (!h->prof) {
    for (int p = 0; p < 3; ++p) {
      if (launches) launches[p] = 0;
      if (ms) ms[p] = 0;
      if (relaxations) relaxations[p] = 0;
    }
    return APSP_OK;
  }
  h->prof->read(launches, ms, relaxations);
  return APSP_OK;
}

}  // extern "C"

// ============================================================== request loop
// Continuous batching over streams: the worker admits queued requests in
// arrival order while their footprint (n^2 * 4 bytes of D plus the panel
// buffer) fits the memory budget and fewer than max_batch are in flight; each
// admitted request gets its own stream, so rounds of co-arriving graphs
// overlap on the device; completions free memory and slots for the next ones.
namespace {

int64_t request_bytes(int64_t n) {
  return n * n * 4 + (int64_t)apsp::round_width(APSP_I32) * panel_ld(n) * 4 + 256;
}

// Admits one request (called by the worker with smu held).
apsp_status admit(apsp_handle *h, Request *r) {
  const int64_t n = r->req.n;
  cudaStream_t s;
  if (!h->free_streams.empty()) {
    s = h->free_streams.back();
    h->free_streams.pop_back();
  } else if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    return APSP_E_CUDA;
  }
  r->stream = s;
  const int64_t ldT = panel_ld(n);
  if (cudaMallocAsync(&r->D, (size_t)std::max<int64_t>(1, n * n) * 4, s) != cudaSuccess ||
      cudaMallocAsync(&r->colT, (size_t)apsp::round_width(APSP_I32) * ldT * 4, s) != cudaSuccess ||
      cudaMallocAsync((void **)&r->status, 64, s) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->copy_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming) != cudaSuccess)
    return APSP_E_CUDA;
  if (n > 0) {
    if (cudaMemcpy2DAsync(r->D, (size_t)n * 4, r->req.W, (size_t)r->req.ld * 4, (size_t)n * 4, (size_t)n,
                          r->req.is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return APSP_E_CUDA;
  }
  cudaEventRecord(r->copy_ev, s);
  cudaMemsetAsync(r->status, 0, sizeof(int), s);
  int64_t l = 0;
  cudaError_t e = apsp::launch_ingest(APSP_I32, r->D, r->D, n, n, r->status, s, &l);
  if (e == cudaSuccess) e = apsp::launch_rounds(APSP_I32, r->D, n, n, r->colT, ldT, s, &l);
  h->launches += l;
  if (e != cudaSuccess) return APSP_E_CUDA;
  cudaEventRecord(r->done_ev, s);
  r->admitted = true;
  return APSP_OK;
}

void worker_loop(apsp_handle *h) {
  cudaSetDevice(h->cfg.device);
  std::unique_lock<std::mutex> g(h->smu);
  while (!h->stopping) {
    // completions
    for (auto &kv : h->reqs) {
      Request *r = kv.second.get();
      if (r->admitted && !r->finished && cudaEventQuery(r->done_ev) == cudaSuccess) {
        r->finished = true;
        int st = 0;
        cudaMemcpy(&st, r->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (st & 1) r->err = APSP_E_INVALID;
        else if (st & 2) r->err = APSP_E_RANGE;
        cudaFreeAsync(r->colT, r->stream);
        cudaFreeAsync(r->status, r->stream);
        r->colT = nullptr;
        r->status = nullptr;
        h->used -= (int64_t)apsp::round_width(APSP_I32) * panel_ld(r->req.n) * 4 + 256;
        h->free_streams.push_back(r->stream);
        --h->running;
        h->scv.notify_all();
      }
    }
    // admissions, in arrival order
    while (!h->queue.empty() && h->running < h->cfg.max_batch) {
      Request *r = h->reqs[h->queue.front()].get();
      if (h->used + r->bytes > h->budget && h->running > 0) break;  // wait for memory to free up
      h->queue.pop_front();
      apsp_status st = admit(h, r);
      h->used += r->bytes;
      if (st != APSP_OK) {
        r->err = st;
        r->finished = true;
        r->admitted = true;
        h->used -= r->bytes;
        continue;
      }
      ++h->running;
    }
    h->scv.wait_for(g, std::chrono::microseconds(h->running > 0 ? 50 : 2000));
  }
}

void start_worker(apsp_handle *h) {
  if (h->worker_started) return;
  if (h->cfg.memory_budget > 0) {
    h->budget = h->cfg.memory_budget;
  } else {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    const int64_t reserve = int64_t(4) << 30;
    h->budget = (int64_t)fr > reserve ? (int64_t)fr - reserve : (int64_t)fr / 2;
  }
  h->worker = std::thread(worker_loop, h);
  h->worker_started = true;
}

}  // namespace

extern "C" {

apsp_status apsp_submit(apsp_handle *h, const apsp_request *r, uint64_t *ticket) {
  if (!h || !r || !ticket) return APSP_E_INVALID;
  if (r->n < 0 || r->ld < r->n || (r->n > 0 && !r->W)) return set_err(h, APSP_E_INVALID, "bad request");
  cudaSetDevice(h->cfg.device);
  std::unique_lock<std::mutex> g(h->smu);
  start_worker(h);
  const int64_t bytes = request_bytes(r->n);
  if (bytes > h->budget) return APSP_E_NOMEM;
  if ((int64_t)h->queue.size() >= h->cfg.queue_depth) return APSP_E_BUSY;
  std::unique_ptr<Request> q(new Request());
  q->ticket = h->next_ticket++;
  q->req = *r;
  q->bytes = bytes;
  *ticket = q->ticket;
  h->queue.push_back(q->ticket);
  h->reqs[q->ticket] = std::move(q);
  g.unlock();
  h->scv.notify_all();
  return APSP_OK;
}

apsp_status apsp_poll(apsp_handle *h, uint64_t ticket, apsp_state *st, const void **D_dev) {
  if (!h || !st) return APSP_E_INVALID;
  std::unique_lock<std::mutex> g(h->smu);
  auto it = h->reqs.find(ticket);
  if (it == h->reqs.end()) return APSP_E_NOTFOUND;
  Request *r = it->second.get();
  if (r->err != APSP_OK) {
    *st = APSP_ERROR;
    return r->err;
  }
  if (!r->admitted) {
    *st = APSP_QUEUED;
    return APSP_OK;
  }
  if (r->finished || cudaEventQuery(r->done_ev) == cudaSuccess) {
    *st = APSP_DONE;
    if (D_dev) *D_dev = r->D;
    return APSP_OK;
  }
  *st = cudaEventQuery(r->copy_ev) == cudaSuccess ? APSP_RUNNING : APSP_QUEUED;
  return APSP_OK;
}

apsp_status apsp_wait(apsp_handle *h, uint64_t ticket, int64_t timeout_ms) {
  if (!h) return APSP_E_INVALID;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    apsp_state st;
    apsp_status s = apsp_poll(h, ticket, &st, nullptr);
    if (s != APSP_OK) return s;
    if (st == APSP_DONE) {
      // make the result visible to the caller's streams
      std::unique_lock<std::mutex> g(h->smu);
      Request *r = h->reqs[ticket].get();
      if (r->done_ev) cudaEventSynchronize(r->done_ev);
      return APSP_OK;
    }
    if (timeout_ms >= 0 && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
      return APSP_E_NOTREADY;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

apsp_status apsp_fetch(apsp_handle *h, uint64_t ticket, void *dst, int64_t ldd, void *stream) {
  if (!h || !dst) return APSP_E_INVALID;
  std::unique_lock<std::mutex> g(h->smu);
  auto it = h->reqs.find(ticket);
  if (it == h->reqs.end()) return APSP_E_NOTFOUND;
  Request *r = it->second.get();
  if (r->err != APSP_OK) return r->err;
  if (!r->admitted) return APSP_E_NOTREADY;
  const int64_t n = r->req.n;
  if (ldd < n) return APSP_E_INVALID;
  if (n == 0) return APSP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamWaitEvent(s, r->done_ev, 0) != cudaSuccess) return APSP_E_CUDA;
  if (cudaMemcpy2DAsync(dst, (size_t)ldd * 4, r->D, (size_t)n * 4, (size_t)n * 4, (size_t)n, cudaMemcpyDefault, s) !=
      cudaSuccess)
    return APSP_E_CUDA;
  return APSP_OK;
}

apsp_status apsp_release(apsp_handle *h, uint64_t ticket) {
  if (!h) return APSP_E_INVALID;
  std::unique_lock<std::mutex> g(h->smu);
  auto it = h->reqs.find(ticket);
  if (it == h->reqs.end()) return APSP_E_NOTFOUND;
  Request *r = it->second.get();
  if (r->admitted && !r->finished && r->err == APSP_OK) {
    // still running: wait for it, then free
    cudaEventSynchronize(r->done_ev);
    return APSP_E_NOTREADY;
  }
  if (!r->admitted) {
    h->queue.erase(std::remove(h->queue.begin(), h->queue.end(), ticket), h->queue.end());
  } else if (r->D) {
    cudaFreeAsync(r->D, r->stream);
    r->D = nullptr;
    h->used -= r->req.n * r->req.n * 4;
  }
  if (r->copy_ev) cudaEventDestroy(r->copy_ev);
  if (r->done_ev) cudaEventDestroy(r->done_ev);
  r->copy_ev = r->done_ev = nullptr;
  h->reqs.erase(it);
  h->scv.notify_all();
  return APSP_OK;
}

apsp_status apsp_cancel(apsp_handle *h, uint64_t ticket) {
  if (!h) return APSP_E_INVALID;
  std::unique_lock<std::mutex> g(h->smu);
  auto it = h->reqs.find(ticket);
  if (it == h->reqs.end()) return APSP_E_NOTFOUND;
  Request *r = it->second.get();
  if (r->admitted) return APSP_E_BUSY;  // already on the device: it finishes
  h->queue.erase(std::remove(h->queue.begin(), h->queue.end(), ticket), h->queue.end());
  r->err = APSP_E_CANCELLED;
  r->admitted = true;
  r->finished = true;
  return APSP_OK;
}

}  // extern "C"
