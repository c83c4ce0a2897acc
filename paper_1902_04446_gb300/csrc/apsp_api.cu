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
#include <fstream>
#include <sstream>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/apsp.h"
#include "batch.h"
#include "fw_launch.h"

namespace {

constexpr int64_t kDefaultMaxEdges = int64_t(1) << 26;

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// A group: requests admitted together and solved by one batched launch on
// one stream.
struct Group {
  cudaStream_t stream = nullptr;
  cudaEvent_t copy_ev = nullptr;  // all inputs copied (callers may reuse W)
  cudaEvent_t done_ev = nullptr;  // batched launch finished
  void *ws = nullptr;             // plan tables + panel buffers (freed at completion)
  int *status = nullptr;          // device words: [i] input checks of request i, [count] kernel errors
  apsp::BatchGraph *graphs_dev = nullptr;
  std::vector<uint64_t> tickets;
  int64_t transient = 0;          // budget bytes returned at completion
  bool finished = false;
  // set by the serving thread once copy_ev is recorded / every launch is
  // enqueued (the device work is enqueued outside the serving lock)
  std::atomic<bool> copy_recorded{false}, enqueued{false};
  ~Group() {
    if (copy_ev) cudaEventDestroy(copy_ev);
    if (done_ev) cudaEventDestroy(done_ev);
  }
};

struct Request {
  uint64_t ticket = 0;
  apsp_request req{};
  int64_t bytes = 0;      // n^2 * 4 (held until release)
  int64_t transient = 0;  // panel share (held until the group finishes)
  bool admitted = false;
  bool finished = false;
  bool alone = false;     // runs in its own group on the per-round kernels
  apsp_status err = APSP_OK;
  void *D = nullptr;
  std::shared_ptr<Group> group;
  int gidx = -1;
};

// Event pairs around phase launches (apsp_profile).
struct Profiler : apsp::PhaseTimer {
  struct Pair {
    cudaEvent_t a, b;
    int phase;
    double relax, relax_alt;
    int *flag;  // pinned copy of a device mode flag (0: relax, else relax_alt), or nullptr
  };
  std::vector<Pair> pairs;       // recorded, not yet read
  std::vector<cudaEvent_t> pool; // free events
  std::vector<int *> flags;      // free pinned flag slots
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
    pairs.push_back({pending, b, phase, relax, relax, nullptr});
    pending = nullptr;
  }
  void after_choice(int phase, cudaStream_t s, double relax_sym, double relax_gen, const int *dflag) override {
    int *f = nullptr;
    if (!flags.empty()) {
      f = flags.back();
      flags.pop_back();
    } else if (cudaHostAlloc(&f, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
      f = nullptr;
      cudaGetLastError();
    }
    if (f && cudaMemcpyAsync(f, dflag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
      flags.push_back(f);
      f = nullptr;
    }
    cudaEvent_t b = get();  // after the flag copy: the pair's end event covers it
    cudaEventRecord(b, s);
    pairs.push_back({pending, b, phase, relax_sym, relax_gen, f});
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
      if (relax) relax[q.phase] += (q.flag && *q.flag != 0) ? q.relax_alt : q.relax;
      if (q.flag) flags.push_back(q.flag);
      pool.push_back(q.a);
      pool.push_back(q.b);
    }
    pairs.clear();
  }
  ~Profiler() {
    for (Pair &q : pairs) {
      cudaEventDestroy(q.a);
      cudaEventDestroy(q.b);
      if (q.flag) cudaFreeHost(q.flag);
    }
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    for (int *f : flags) cudaFreeHost(f);
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
  void *wsb = nullptr;  // batched solve: plan + panel buffers
  size_t wsb_bytes = 0;
  void *rowP = nullptr;  // symmetric mode, packed 16-bit: element panel
  size_t rowP_bytes = 0;
  void *mpT = nullptr;  // min-plus product: A^T (32-bit words)
  size_t mpT_bytes = 0;
  int *d_status = nullptr;
  int *h_status = nullptr;  // pinned
  std::string last_error;
  std::atomic<int64_t> launches{0};
  std::unique_ptr<Profiler> prof;  // non-null while apsp_profile(h, 1) is on
  std::map<std::pair<int, int64_t>, apsp::RoundConfig> tuned;  // (dtype, n bucket) -> round shape

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
  std::vector<std::shared_ptr<Group>> groups;  // in flight
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

int64_t bucket_of(int64_t n) {
  int64_t b = 128;
  while (b < n) b <<= 1;
  return b;
}

// Round shape for (dtype, n): a forced block_k, else the tuned bucket (the
// largest tuned bucket for larger n), else the defaults by n and dtype.
apsp::RoundConfig config_for(apsp_handle *h, int dtype, int64_t n) {
  apsp::RoundConfig c;
  c.p3 = apsp::default_phase3(n, dtype);
  c.bk = apsp::default_round_width(n, dtype);
  const int64_t b = bucket_of(n);
  auto it = h->tuned.find({dtype, b});
  if (it != h->tuned.end()) {
    c = it->second;
  } else {
    for (auto r = h->tuned.rbegin(); r != h->tuned.rend(); ++r)
      if (r->first.first == dtype && r->first.second < b) {
        c = r->second;
        break;
      }
  }
  if (h->cfg.block_k == 32 || h->cfg.block_k == 64 || h->cfg.block_k == 128) c.bk = h->cfg.block_k;
  if (h->cfg.phase3_variant >= 1 && h->cfg.phase3_variant <= 5) c.p3 = h->cfg.phase3_variant - 1;
  return c;
}

// Enqueues the q rounds on D (already holding W) using the handle's panel buffer.
// known_sym: D is symmetric by construction (edge-list input).
apsp_status run_rounds_locked(apsp_handle *h, int dtype, void *D, int64_t n, int64_t ld, cudaStream_t s,
                              bool known_sym = false) {
  const int64_t ldT = panel_ld(n);
  apsp::RoundConfig rc = config_for(h, dtype, n);
  cudaError_t e = ensure(&h->colT, &h->colT_bytes, apsp::panel_buffer_bytes(n, ldT, rc.p3 == 4));
  if (e != cudaSuccess) {
    h->last_error = std::string("panel workspace: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? APSP_E_NOMEM : APSP_E_CUDA;
  }
  if (h->cfg.symmetric == 1 || (h->cfg.symmetric == 0 && known_sym)) {
    rc.sym = true;
  } else if (h->cfg.symmetric == 0 && n > 1 && apsp::single_launch(dtype, D, ld, n, rc)) {
    // device check of W == W^T whose answer the single launch reads itself:
    // no host round trip before the rounds are enqueued
    int *flag = h->d_status + 1;
    e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess) e = apsp::launch_symmetry_check(dtype, D, n, ld, flag, s);
    if (e != cudaSuccess) {
      h->last_error = std::string("symmetry check: ") + cudaGetErrorString(e);
      return APSP_E_CUDA;
    }
    h->launches += 1;
    rc.sym_flag = flag;
  } else if (h->cfg.symmetric == 0 && n > 1) {
    // device check of W == W^T; the answer is read back before the rounds are enqueued
    int *flag = h->d_status + 1;
    e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess) e = apsp::launch_symmetry_check(dtype, D, n, ld, flag, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_status + 1, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      h->last_error = std::string("symmetry check: ") + cudaGetErrorString(e);
      return APSP_E_CUDA;
    }
    h->launches += 1;
    rc.sym = h->h_status[1] == 0;
  }
  if ((rc.sym || rc.sym_flag) && dtype == APSP_U16) {
    e = ensure(&h->rowP, &h->rowP_bytes, apsp::row_panel_bytes(ldT, rc.p3 == 4));
    if (e != cudaSuccess) {
      h->last_error = std::string("panel workspace: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? APSP_E_NOMEM : APSP_E_CUDA;
    }
    rc.rowP = h->rowP;
  }
  int64_t l = 0;
  e = apsp::launch_rounds(dtype, D, ld, n, h->colT, ldT, s, &l, h->prof.get(), rc, h->d_status);
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
  // AUTO: int32 in and out; packed 16-bit when the bound allows (precision
  // selection).  The bound synchronizes the stream.
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
      // the bound accepts only a symmetric W, so the packed copy is symmetric
      apsp_status st = run_rounds_locked(h, APSP_U16, P, n, ld16, s, true);
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
  if (c.block_k != 0 && c.block_k != 32 && c.block_k != 64 && c.block_k != 128) return APSP_E_INVALID;
  if (c.phase3_variant < 0 || c.phase3_variant > 5) return APSP_E_INVALID;
  if (c.symmetric < 0 || c.symmetric > 2) return APSP_E_INVALID;
  if (c.serving_large_n < 0 || c.serving_large_grid < 0) return APSP_E_INVALID;
  if (c.max_batch <= 0) c.max_batch = 64;
  if (c.queue_depth <= 0) c.queue_depth = 4096;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) return APSP_E_CUDA;
  if (cudaSetDevice(c.device) != cudaSuccess) return APSP_E_CUDA;
  std::unique_ptr<apsp_handle> h(new apsp_handle());
  h->cfg = c;
  {
    // stream-ordered allocations (request loop, bound pass) stay in the pool
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, c.device) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      // memory freed on one group's stream is not handed to another group by
      // making that group's stream wait for the first (which would chain
      // independent requests one after another)
      int no = 0;
      cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
  }
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
  r->D = nullptr;
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
  for (auto &g : h->groups) {
    if (g->ws) cudaFree(g->ws);
    if (g->status) cudaFree(g->status);
    g->ws = nullptr;
    g->status = nullptr;
  }
  h->groups.clear();
  for (cudaStream_t s : h->free_streams) cudaStreamDestroy(s);
  if (h->colT) cudaFree(h->colT);
  if (h->ws16) cudaFree(h->ws16);
  if (h->wsb) cudaFree(h->wsb);
  if (h->rowP) cudaFree(h->rowP);
  if (h->mpT) cudaFree(h->mpT);
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
        apsp_status st = run_rounds_locked(h, APSP_U16, P, n, ld16, s, true);
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
  return run_rounds_locked(h, solve_dtype, D, n, ld, s, true);
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
  if (st & 4) {
    h->last_error = "a bounded device wait gave up";
    return APSP_E_TIMEOUT;
  }
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

// The product into C with the library's A^T workspace (the warp-specialized
// kernel) when it can be had, else the one-CTA-per-tile kernel.  h->mu held.
static cudaError_t minplus_locked(apsp_handle *h, int dtype, const void *A, int64_t lda, const void *B, int64_t ldb,
                                  void *C, int64_t ldc, int64_t m, int64_t k, int64_t n, cudaStream_t s) {
  const size_t need = apsp::minplus_scratch_bytes(m, k);
  void *scr = nullptr;
  if (need > 0) {
    if (ensure(&h->mpT, &h->mpT_bytes, need) == cudaSuccess) scr = h->mpT;
    else cudaGetLastError();  // out of memory: the kernel without workspace
  }
  int64_t l = 0;
  cudaError_t e = apsp::launch_minplus(dtype, A, lda, B, ldb, C, ldc, m, k, n, s, &l, scr, scr ? h->mpT_bytes : 0,
                                       h->d_status);
  h->launches += l;
  return e;
}

apsp_status apsp_minplus(apsp_handle *h, int dtype, const void *A, int64_t lda, const void *B, int64_t ldb, void *C,
                         int64_t ldc, int64_t m, int64_t k, int64_t n, void *stream) {
  if (!h || !valid_dtype(dtype)) return APSP_E_INVALID;
  if (m < 0 || k < 0 || n < 0 || lda < k || ldb < n || ldc < n) return set_err(h, APSP_E_INVALID, "bad shape");
  if (m > 0 && n > 0 && (!C || (k > 0 && (!A || !B)))) return set_err(h, APSP_E_INVALID, "null matrix");
  if ((m + 127) / 128 > 65535) return set_err(h, APSP_E_INVALID, "m too large");
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(h->mu);
  if ((e = cudaMemsetAsync(h->d_status, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(h, e, "status reset");
  e = minplus_locked(h, dtype, A, lda, B, ldb, C, ldc, m, k, n, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "minplus");
  return APSP_OK;
}

apsp_status apsp_solve_squaring(apsp_handle *h, int dtype, const void *W, int64_t n, int64_t ld, void *D,
                                void *stream) {
  if (!h) return APSP_E_INVALID;
  if (!valid_dtype(dtype)) return set_err(h, APSP_E_INVALID, "dtype must be APSP_I32, APSP_U16 or APSP_F32");
  if (n < 0 || ld < n || (n > 0 && (!W || !D))) return set_err(h, APSP_E_INVALID, "need n >= 0, ld >= n, W and D");
  if ((n + 127) / 128 > 65535) return set_err(h, APSP_E_INVALID, "n too large");
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(h->mu);
  if ((e = cudaMemsetAsync(h->d_status, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(h, e, "status reset");
  if (n == 0) return APSP_OK;
  int64_t l = 0;
  e = apsp::launch_ingest(dtype, W, D, n, ld, h->d_status, s, &l);
  h->launches += l;
  if (e != cudaSuccess) return cuda_fail(h, e, "ingest");
  // a shortest path has at most n - 1 edges; after i squarings every path of
  // up to 2^i edges is accounted for (Alg. 1).  In place: each value read
  // during a product is already a valid upper bound, so it converges no later
  int rounds = 0;
  while ((int64_t(1) << rounds) < n - 1) ++rounds;
  for (int i = 0; i < rounds; ++i) {
    e = minplus_locked(h, dtype, D, ld, D, ld, D, ld, n, n, n, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "squaring");
  }
  return APSP_OK;
}

apsp_status apsp_tri_layout(int dtype, int64_t n, int64_t *rows, int64_t *ld, int64_t *bytes) {
  if (!valid_dtype(dtype) || n < 0 || (!rows && !ld && !bytes)) return APSP_E_INVALID;
  int64_t r = 0, l = 0;
  apsp::tri_shape(n, dtype, &r, &l);
  if (rows) *rows = r;
  if (ld) *ld = l;
  if (bytes) *bytes = r * l * (dtype == APSP_U16 ? 2 : 4);
  return APSP_OK;
}

apsp_status apsp_tri_from_dense(apsp_handle *h, int dtype, const void *W, int64_t n, int64_t ldw, void *T,
                                void *stream) {
  if (!h) return APSP_E_INVALID;
  if (!valid_dtype(dtype)) return set_err(h, APSP_E_INVALID, "dtype must be APSP_I32, APSP_U16 or APSP_F32");
  if (n < 0 || ldw < n || (n > 0 && (!W || !T))) return set_err(h, APSP_E_INVALID, "need n >= 0, ldw >= n, W and T");
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(h->mu);
  if ((e = cudaMemsetAsync(h->d_status, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(h, e, "status reset");
  int64_t l = 0;
  e = apsp::launch_tri_fill(dtype, W, ldw, T, n, h->d_status, s, &l);
  h->launches += l;
  if (e != cudaSuccess) return cuda_fail(h, e, "tri_from_dense");
  return APSP_OK;
}

apsp_status apsp_tri_from_edges(apsp_handle *h, int dtype, const int32_t *src, const int32_t *dst, const void *w,
                                int64_t m, int64_t n, void *T, void *stream) {
  if (!h) return APSP_E_INVALID;
  if (!valid_dtype(dtype)) return set_err(h, APSP_E_INVALID, "dtype must be APSP_I32, APSP_U16 or APSP_F32");
  if (n < 0 || m < 0 || (n > 0 && !T) || (m > 0 && (!src || !dst || !w)))
    return set_err(h, APSP_E_INVALID, "bad edge-list arguments");
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(h->mu);
  if ((e = cudaMemsetAsync(h->d_status, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(h, e, "status reset");
  if (n == 0) return APSP_OK;
  int64_t l = 0;
  if (dtype == APSP_U16) {
    int64_t bound = 0;
    int ok = 0;
    e = apsp::bound_from_edges(src, dst, w, 1, m, n, s, &bound, &ok, &l);
    h->launches += l;
    l = 0;
    if (e != cudaSuccess) return cuda_fail(h, e, "16-bit bound");
    if (!ok) {
      h->last_error = "16-bit bound fails: 2*eccentricity = " + std::to_string(bound) + " >= 32767";
      return APSP_E_RANGE;
    }
  }
  e = apsp::launch_tri_from_edges(dtype, src, dst, w, m, T, n, h->d_status, s, &l);
  h->launches += l;
  if (e != cudaSuccess) return cuda_fail(h, e, "tri_from_edges");
  return APSP_OK;
}

apsp_status apsp_solve_tri(apsp_handle *h, int dtype, void *T, int64_t n, void *stream) {
  if (!h) return APSP_E_INVALID;
  if (!valid_dtype(dtype)) return set_err(h, APSP_E_INVALID, "dtype must be APSP_I32, APSP_U16 or APSP_F32");
  if (n < 0 || (n > 0 && !T)) return set_err(h, APSP_E_INVALID, "need n >= 0 and T");
  if (n > (int64_t(1) << 31) - 1) return set_err(h, APSP_E_INVALID, "n too large");
  if (reinterpret_cast<uintptr_t>(T) % 16 != 0) return set_err(h, APSP_E_INVALID, "T must be 16-byte aligned");
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(h->mu);
  if (n == 0) return APSP_OK;
  const int64_t ldT = panel_ld(n);
  apsp::RoundConfig rc = config_for(h, dtype, n);
  e = ensure(&h->colT, &h->colT_bytes, apsp::panel_buffer_bytes(n, ldT, false));
  if (e == cudaSuccess && dtype == APSP_U16) {
    e = ensure(&h->rowP, &h->rowP_bytes, apsp::row_panel_bytes(ldT, false));
    rc.rowP = h->rowP;
  }
  if (e != cudaSuccess) {
    h->last_error = std::string("panel workspace: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? APSP_E_NOMEM : APSP_E_CUDA;
  }
  int64_t l = 0;
  e = apsp::launch_rounds_tri(dtype, T, n, h->colT, ldT, s, &l, h->prof.get(), rc, h->d_status);
  h->launches += l;
  if (e != cudaSuccess) return cuda_fail(h, e, "rounds (upper-triangular storage)");
  return APSP_OK;
}

apsp_status apsp_tri_to_dense(int dtype, const void *T, int64_t n, void *D, int64_t ld, void *stream) {
  if (!valid_dtype(dtype) || n < 0 || ld < n || (n > 0 && (!T || !D))) return APSP_E_INVALID;
  return apsp::launch_tri_to_dense(dtype, T, n, D, ld, static_cast<cudaStream_t>(stream), nullptr) == cudaSuccess
             ? APSP_OK
             : APSP_E_CUDA;
}

apsp_status apsp_tri_rows(int dtype, const void *T, int64_t n, const int64_t *rows, int64_t k, void *out, int64_t ldo,
                          void *stream) {
  if (!valid_dtype(dtype) || n < 0 || k < 0 || ldo < n || (n > 0 && k > 0 && (!T || !rows || !out)))
    return APSP_E_INVALID;
  return apsp::launch_tri_rows(dtype, T, n, rows, k, out, ldo, nullptr, static_cast<cudaStream_t>(stream), nullptr) ==
                 cudaSuccess
             ? APSP_OK
             : APSP_E_CUDA;
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

}  // extern "C"

namespace {

// Lays out the batched-solve workspace: plan tables, then one panel buffer
// per graph.  Returns the total bytes; fills colT pointers relative to base.
size_t batch_layout(const std::vector<int64_t> &n, char *base, std::vector<uint32_t *> &colT, size_t plan_bytes) {
  size_t off = (plan_bytes + 255) / 256 * 256;
  colT.resize(n.size());
  for (size_t i = 0; i < n.size(); ++i) {
    colT[i] = reinterpret_cast<uint32_t *>(base + off);
    off += ((size_t)64 * apsp::batch_panel_ld(n[i]) * 4 + 255) / 256 * 256;
  }
  return off;
}

// Enqueues ingest checks and one batched launch (the handle lock is held).
apsp_status batch_locked(apsp_handle *h, const std::vector<const int32_t *> &W, const std::vector<int64_t> &n,
                         const std::vector<int64_t> &ld, const std::vector<int32_t *> &D, cudaStream_t s,
                         int64_t spin_limit, const int *gate) {
  cudaError_t e = cudaMemsetAsync(h->d_status, 0, sizeof(int), s);
  if (e != cudaSuccess) return APSP_E_CUDA;
  std::vector<int32_t *> Dl;
  std::vector<int64_t> nl, ldl;
  for (size_t i = 0; i < n.size(); ++i) {
    if (n[i] == 0) continue;
    int64_t l = 0;
    e = apsp::launch_ingest(APSP_I32, W[i], D[i], n[i], ld[i], h->d_status, s, &l);
    h->launches += l;
    if (e != cudaSuccess) {
      h->last_error = std::string("ingest: ") + cudaGetErrorString(e);
      return APSP_E_CUDA;
    }
    Dl.push_back(D[i]);
    nl.push_back(n[i]);
    ldl.push_back(ld[i]);
  }
  if (Dl.empty()) return APSP_OK;
  // plan sizes do not depend on the panel pointers: build once to size, once for real
  apsp::BatchPlan plan;
  std::vector<uint32_t *> colT(Dl.size(), nullptr);
  plan.build(Dl, nl, ldl, colT);
  const size_t plan_bytes = plan.workspace_bytes();
  const size_t need = batch_layout(nl, nullptr, colT, plan_bytes);
  e = ensure(&h->wsb, &h->wsb_bytes, need);
  if (e != cudaSuccess) {
    h->last_error = std::string("batch workspace: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? APSP_E_NOMEM : APSP_E_CUDA;
  }
  batch_layout(nl, static_cast<char *>(h->wsb), colT, plan_bytes);
  plan.build(Dl, nl, ldl, colT);
  int64_t l = 0;
  e = apsp::launch_batch(plan, h->wsb, s, spin_limit, gate, h->d_status, nullptr, &l);
  h->launches += l;
  if (e != cudaSuccess) {
    h->last_error = std::string("batched launch: ") + cudaGetErrorString(e);
    return APSP_E_CUDA;
  }
  return APSP_OK;
}

}  // namespace

extern "C" {

apsp_status apsp_solve_batch(apsp_handle *h, int64_t count, const int32_t *const *W, const int64_t *n,
                             const int64_t *ld, int32_t *const *D, void *stream) {
  if (!h) return APSP_E_INVALID;
  if (count < 0 || (count > 0 && (!W || !n || !ld || !D))) return set_err(h, APSP_E_INVALID, "bad batch arrays");
  for (int64_t i = 0; i < count; ++i)
    if (n[i] < 0 || ld[i] < n[i] || n[i] > (int64_t(1) << 31) - 1 || (n[i] > 0 && (!W[i] || !D[i])))
      return set_err(h, APSP_E_INVALID, "bad graph " + std::to_string(i) + " in batch");
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  std::lock_guard<std::mutex> g(h->mu);
  std::vector<const int32_t *> Wv(W, W + count);
  std::vector<int64_t> nv(n, n + count), ldv(ld, ld + count);
  std::vector<int32_t *> Dv(D, D + count);
  return batch_locked(h, Wv, nv, ldv, Dv, static_cast<cudaStream_t>(stream), h->cfg.spin_limit, nullptr);
}

apsp_status apsp_check_bounded_wait(apsp_handle *h, int64_t spin_limit) {
  if (!h || spin_limit <= 0) return APSP_E_INVALID;
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  std::lock_guard<std::mutex> g(h->mu);
  // two checks: the batched kernel on a 96-node path (two rounds), and every
  // round of a 320-node path in one persistent launch (five rounds)
  const int64_t n = 96, n1 = 320, ldT = 512;
  const size_t oD1 = (size_t)n * n * 4, oT = oD1 + (size_t)n1 * n1 * 4;
  const size_t oG = oT + ((apsp::panel_buffer_bytes(n1, ldT, true) + 255) & ~size_t(255));
  void *buf = nullptr;
  e = cudaMalloc(&buf, oG + 256);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc");
  char *b = static_cast<char *>(buf);
  int32_t *D = reinterpret_cast<int32_t *>(b), *D1 = reinterpret_cast<int32_t *>(b + oD1);
  int *gate = reinterpret_cast<int *>(b + oG), *err1 = gate + 1;
  cudaStream_t s = nullptr;
  apsp_status st = APSP_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) st = APSP_E_CUDA;
  // valid graphs (paths), and a gate flag that nothing ever sets
  auto path = [](int64_t m) {
    std::vector<int32_t> w((size_t)m * m, APSP_INF_I32);
    for (int64_t i = 0; i < m; ++i) {
      w[(size_t)i * m + i] = 0;
      if (i + 1 < m) w[(size_t)i * m + i + 1] = w[(size_t)(i + 1) * m + i] = 1;
    }
    return w;
  };
  if (st == APSP_OK) {
    const std::vector<int32_t> w = path(n), w1 = path(n1);
    if (cudaMemcpy(D, w.data(), w.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(D1, w1.data(), w1.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(gate, 0, 2 * sizeof(int)) != cudaSuccess)
      st = APSP_E_CUDA;
  }
  auto read_flag = [&](const int *flag) {  // the word a kernel ORs 4 into when a wait gave up
    e = cudaMemcpyAsync(h->h_status, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "sync");
    return (*h->h_status & 4) ? APSP_E_TIMEOUT : APSP_OK;
  };
  if (st == APSP_OK) {
    std::vector<const int32_t *> Wv{D};
    std::vector<int64_t> nv{n}, ldv{n};
    std::vector<int32_t *> Dv{D};
    st = batch_locked(h, Wv, nv, ldv, Dv, s, spin_limit, gate);
    if (st == APSP_OK) st = read_flag(h->d_status);
  }
  if (st == APSP_E_TIMEOUT) {
    apsp::RoundConfig rc;
    rc.bk = 64;
    rc.p3 = 4;
    rc.gate = gate;
    rc.dep_spins = (uint32_t)std::min<int64_t>(spin_limit, 0xFFFFFFFFll);
    if (!apsp::single_launch(APSP_I32, D1, n1, n1, rc)) st = APSP_E_UNSUPPORTED;
    else {
      int64_t l = 0;
      e = apsp::launch_rounds(APSP_I32, D1, n1, n1, b + oT, ldT, s, &l, nullptr, rc, err1);
      st = e != cudaSuccess ? cuda_fail(nullptr, e, "launch_rounds") : read_flag(err1);
    }
  }
  if (s) cudaStreamDestroy(s);
  cudaFree(buf);
  if (st == APSP_E_TIMEOUT) h->last_error = "bounded waits gave up as expected";
  return st;
}

}  // extern "C"

namespace {

struct TuneEntry {
  std::string gpu;
  int dtype = 0;
  int64_t n = 0;
  int bk = 64, tma = 1;
  double ms = 0;
};

std::string json_str_field(const std::string &obj, const char *key) {
  const std::string k = std::string("\"") + key + "\"";
  size_t p = obj.find(k);
  if (p == std::string::npos) return "";
  p = obj.find('"', obj.find(':', p) + 1);
  if (p == std::string::npos) return "";
  const size_t q = obj.find('"', p + 1);
  return q == std::string::npos ? "" : obj.substr(p + 1, q - p - 1);
}

double json_num_field(const std::string &obj, const char *key, double dflt) {
  const std::string k = std::string("\"") + key + "\"";
  size_t p = obj.find(k);
  if (p == std::string::npos) return dflt;
  p = obj.find(':', p);
  if (p == std::string::npos) return dflt;
  return std::strtod(obj.c_str() + p + 1, nullptr);
}

// The cache is a JSON object {"entries": [{...}, ...]}; every entry is one
// flat object, read back field by field.
std::vector<TuneEntry> read_cache(const char *path) {
  std::vector<TuneEntry> out;
  if (!path) return out;
  std::ifstream f(path);
  if (!f) return out;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string txt = ss.str();
  size_t p = txt.find('[');
  while (p != std::string::npos) {
    const size_t a = txt.find('{', p);
    if (a == std::string::npos) break;
    const size_t b = txt.find('}', a);
    if (b == std::string::npos) break;
    const std::string obj = txt.substr(a, b - a + 1);
    TuneEntry e;
    e.gpu = json_str_field(obj, "gpu");
    e.dtype = (int)json_num_field(obj, "dtype", -1);
    e.n = (int64_t)json_num_field(obj, "n", 0);
    e.bk = (int)json_num_field(obj, "bk", 64);
    e.tma = (int)json_num_field(obj, "tma", 1);
    e.ms = json_num_field(obj, "ms", 0);
    if (!e.gpu.empty() && e.dtype >= 0 && e.n > 0 && (e.bk == 32 || e.bk == 64 || e.bk == 128) && e.tma >= 0 && e.tma <= 4)
      out.push_back(e);
    p = b + 1;
  }
  return out;
}

bool write_cache(const char *path, const std::vector<TuneEntry> &es) {
  if (!path) return true;
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp);
    if (!f) return false;
    f << "{\"entries\": [\n";
    for (size_t i = 0; i < es.size(); ++i) {
      const TuneEntry &e = es[i];
      f << "  {\"gpu\": \"" << e.gpu << "\", \"dtype\": " << e.dtype << ", \"n\": " << e.n << ", \"bk\": " << e.bk
        << ", \"tma\": " << e.tma << ", \"ms\": " << e.ms << "}" << (i + 1 < es.size() ? "," : "") << "\n";
    }
    f << "]}\n";
  }
  return std::rename(tmp.c_str(), path) == 0;
}

}  // namespace

extern "C" {

apsp_status apsp_autotune(apsp_handle *h, int dtype, int64_t n_max, const char *cache_path) {
  if (!h || !valid_dtype(dtype) || n_max < 1) return APSP_E_INVALID;
  cudaError_t e = cudaSetDevice(h->cfg.device);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, h->cfg.device)) != cudaSuccess) return cuda_fail(h, e, "properties");
  const std::string gpu = prop.name;
  std::vector<TuneEntry> cache = read_cache(cache_path);
  std::lock_guard<std::mutex> g(h->mu);
  const int64_t top = bucket_of(n_max);
  const size_t es = dtype == APSP_U16 ? 2 : 4;
  bool wrote = false;
  for (int64_t b = 128; b <= top; b <<= 1) {
    bool cached = false;
    for (const TuneEntry &t : cache)
      if (t.gpu == gpu && t.dtype == dtype && t.n == b) {
        apsp::RoundConfig c;
        c.bk = t.bk;
        c.p3 = t.tma;
        h->tuned[{dtype, b}] = c;
        cached = true;
      }
    if (cached) continue;
    void *M = nullptr;
    if ((e = cudaMalloc(&M, (size_t)b * b * es)) != cudaSuccess) return cuda_fail(h, e, "autotune matrix");
    const int64_t ldT = panel_ld(b);
    if ((e = ensure(&h->colT, &h->colT_bytes, apsp::panel_buffer_bytes(b, ldT, true))) != cudaSuccess) {
      cudaFree(M);
      return cuda_fail(h, e, "autotune panel");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    apsp::RoundConfig best_c;
    for (int bk : {32, 64, 128})
      for (int var : {4, 3, 2, 1, 0}) {
        if (bk == 128 && var != 3 && var != 0) continue;  // width 128: per-tile or warp-specialized, per round
        apsp::RoundConfig c;
        c.bk = bk;
        c.p3 = var;
        double t_min = 1e30;
        for (int rep = 0; rep < 4; ++rep) {
          apsp::launch_synth(dtype, M, b, b, nullptr);
          cudaEventRecord(e0, nullptr);
          int64_t l = 0;
          e = apsp::launch_rounds(dtype, M, b, b, h->colT, ldT, nullptr, &l, nullptr, c);
          cudaEventRecord(e1, nullptr);
          if (e != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) break;
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) t_min = std::min(t_min, (double)ms);  // first run warms up
        }
        if (e != cudaSuccess) break;
        if (t_min < best) {
          best = t_min;
          best_c = c;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(M);
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune run");
    h->tuned[{dtype, b}] = best_c;
    TuneEntry t;
    t.gpu = gpu;
    t.dtype = dtype;
    t.n = b;
    t.bk = best_c.bk;
    t.tma = best_c.p3;
    t.ms = best;
    cache.push_back(t);
    wrote = true;
  }
  if (wrote && !write_cache(cache_path, cache)) return set_err(nullptr, APSP_E_INVALID, "cannot write cache");
  return APSP_OK;
}

apsp_status apsp_tuned_config(apsp_handle *h, int dtype, int64_t n, int *block_k, int *tma) {
  if (!h || !block_k || !tma || !valid_dtype(dtype) || n < 0) return APSP_E_INVALID;
  std::lock_guard<std::mutex> g(h->mu);
  const apsp::RoundConfig c = config_for(h, dtype, n);
  *block_k = c.bk;
  *tma = c.p3;
  return APSP_OK;
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
// Continuous batching: the worker admits queued requests in arrival order
// while their footprint (n^2 * 4 bytes of D plus the panel buffer) fits the
// memory budget; requests admitted in one pass form a group that is solved by
// ONE batched persistent launch on its own stream, so the rounds of its
// graphs interleave on the device, and groups admitted later run concurrently
// with the earlier ones.  A group's completion returns its panel memory; a
// request's matrix is returned by apsp_release.
namespace {

constexpr int kMaxGroupsInFlight = 16;
// Default size from which a request gets its own group and the per-round
// kernels (persistent TMA Phase 3) instead of the batched kernel
// (apsp_config.serving_large_n).
constexpr int64_t kLargeN = 1536;
int64_t large_n(const apsp_handle *h) { return h->cfg.serving_large_n > 0 ? h->cfg.serving_large_n : kLargeN; }

int64_t panel_bytes(int64_t n) { return 64 * apsp::batch_panel_ld(n) * 4 + 256; }

// Round shape of a large request: the size's own shape, but with the whole GPU
// (serving_large_grid 0) one launch per round, so that the batched groups on
// other streams keep running between its rounds; with a capped grid (the cap
// leaves SMs to the other groups) the size's default.
apsp::RoundConfig large_round_config(apsp_handle *h, int dtype, int64_t n) {
  apsp::RoundConfig rc = config_for(h, dtype, n);
  rc.grid_cap = h->cfg.serving_large_grid;
  if (rc.p3 == 4 && rc.grid_cap == 0) rc.p3 = 3;
  return rc;
}

// Workspace of a large request's own group beyond panel_bytes: the panel
// buffer (doubled, with counters, when every round runs in one launch), and for
// APSP_AUTO the element panel and the packed 16-bit copy.
int64_t large_extra_bytes(apsp_handle *h, const apsp_request &q) {
  const int64_t ldT = panel_ld(q.n);
  const bool all = large_round_config(h, q.dtype == APSP_AUTO ? APSP_U16 : APSP_I32, q.n).p3 == 4;
  int64_t b = (int64_t)apsp::panel_buffer_bytes(q.n, ldT, all);
  if (q.dtype == APSP_AUTO)
    b += 512 + (int64_t)apsp::row_panel_bytes(ldT, all) + q.n * round_up(q.n, 8) * 2;
  return b;
}

// Marks a finished group's requests DONE or ERROR and frees its transient
// memory (called with smu held, after done_ev completed).
void finish_group(apsp_handle *h, const std::shared_ptr<Group> &g) {
  if (g->finished) return;
  g->finished = true;
  const size_t cnt = g->tickets.size();
  std::vector<int> st(cnt + 1, 0);
  cudaMemcpy(st.data(), g->status, (cnt + 1) * sizeof(int), cudaMemcpyDeviceToHost);
  std::vector<apsp::BatchGraph> G(g->tickets.size());
  if (g->graphs_dev && !G.empty())
    cudaMemcpy(G.data(), g->graphs_dev, G.size() * sizeof(apsp::BatchGraph), cudaMemcpyDeviceToHost);
  for (size_t i = 0; i < g->tickets.size(); ++i) {
    auto it = h->reqs.find(g->tickets[i]);
    if (it == h->reqs.end()) continue;
    Request *r = it->second.get();
    r->finished = true;
    if (st[i] & 1) r->err = APSP_E_INVALID;
    else if (st[i] & 2) r->err = APSP_E_RANGE;
    else if (g->graphs_dev ? (G[i].status & 4) != 0 : (st[cnt] & 4) != 0) r->err = APSP_E_TIMEOUT;
    h->used -= r->transient;
    r->transient = 0;
  }
  cudaFreeAsync(g->ws, g->stream);
  cudaFreeAsync(g->status, g->stream);
  g->ws = nullptr;
  g->status = nullptr;
  h->free_streams.push_back(g->stream);
  h->groups.erase(std::remove(h->groups.begin(), h->groups.end(), g), h->groups.end());
  h->scv.notify_all();
}

void poll_groups(apsp_handle *h) {
  std::vector<std::shared_ptr<Group>> done;
  for (auto &g : h->groups)
    if (g->enqueued && cudaEventQuery(g->done_ev) == cudaSuccess) done.push_back(g);
  for (auto &g : done) finish_group(h, g);
}

// Gives back what a failed admission took -- the requests' matrices and the
// group's workspace (stream-ordered frees, after the work already queued), the
// stream, and the requests' share of the budget -- and marks the requests
// ERROR with `st`.  (smu held.)
void undo_admission(apsp_handle *h, const std::vector<Request *> &rs, const std::shared_ptr<Group> &g,
                    apsp_status st) {
  cudaStream_t s = g->stream;
  for (Request *r : rs) {
    if (r->D) cudaFreeAsync(r->D, s);
    r->D = nullptr;
    h->used -= r->bytes + r->transient;
    r->transient = 0;
    r->group.reset();
    r->err = st;
    r->finished = true;
  }
  if (g->ws) cudaFreeAsync(g->ws, s);
  if (g->status) cudaFreeAsync(g->status, s);
  g->ws = nullptr;
  g->status = nullptr;
  g->finished = true;
  if (s) h->free_streams.push_back(s);
  h->groups.erase(std::remove(h->groups.begin(), h->groups.end(), g), h->groups.end());
}

// The device work of an admitted group: matrices, input copies, checks, the
// rounds (one batched launch, or a large request's own rounds).  Runs in the
// serving thread WITHOUT smu, so that apsp_poll answers (APSP_ADMITTED) while
// hundreds of launches are enqueued; it touches only the group and its
// requests' device fields, which other threads read once g->enqueued is set.
apsp_status admit_group_steps(apsp_handle *h, const std::vector<Request *> &rs, Group *g) {
  if (!g->stream) return APSP_E_CUDA;
  cudaStream_t s = g->stream;
  std::vector<int32_t *> D;
  std::vector<int64_t> n, ld;
  for (Request *r : rs) {
    const int64_t rn = r->req.n;
    if (cudaMallocAsync(&r->D, (size_t)std::max<int64_t>(1, rn * rn) * 4, s) != cudaSuccess) {
      r->D = nullptr;
      return APSP_E_CUDA;
    }
    if (rn > 0 && cudaMemcpy2DAsync(r->D, (size_t)rn * 4, r->req.W, (size_t)r->req.ld * 4, (size_t)rn * 4,
                                    (size_t)rn, r->req.is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                    s) != cudaSuccess)
      return APSP_E_CUDA;
    if (rn > 0) {
      D.push_back(static_cast<int32_t *>(r->D));
      n.push_back(rn);
      ld.push_back(rn);
    }
  }
  if (cudaEventCreateWithFlags(&g->copy_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->done_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(g->copy_ev, s) != cudaSuccess)
    return APSP_E_CUDA;
  g->copy_recorded = true;
  // [i] input checks of request i, [count] kernel errors, [count + 1] a large
  // request's symmetry flag
  const size_t sbytes = (rs.size() + 2) * sizeof(int);
  if (cudaMallocAsync((void **)&g->status, sbytes, s) != cudaSuccess) {
    g->status = nullptr;
    return APSP_E_CUDA;
  }
  if (cudaMemsetAsync(g->status, 0, sbytes, s) != cudaSuccess) return APSP_E_CUDA;
  int64_t l = 0;
  for (size_t i = 0; i < rs.size(); ++i) {
    const int64_t rn = rs[i]->req.n;
    if (rn > 0 && apsp::launch_ingest(APSP_I32, rs[i]->D, rs[i]->D, rn, rn, g->status + i, s, &l) != cudaSuccess)
      return APSP_E_CUDA;
  }
  if (rs.size() == 1 && (rs[0]->req.n >= large_n(h) || rs[0]->alone)) {
    // one large graph: per-round kernels on the group's stream; an undirected
    // (symmetric) matrix takes the symmetric mode, decided by a device check
    const int64_t rn = rs[0]->req.n;
    const int64_t ldT = panel_ld(rn);
    if (rs[0]->req.dtype == APSP_AUTO) {
      // precision selection: the 16-bit bound (synchronizes the group's
      // stream), then the rounds in packed 16-bit when it holds
      int64_t bound = 0;
      int ok = 0;
      if (apsp::bound_from_dense(static_cast<const int32_t *>(rs[0]->D), rn, rn,
                                 std::max<int64_t>(kDefaultMaxEdges, 32 * rn), s, &bound, &ok, &l) != cudaSuccess)
        return APSP_E_CUDA;
      if (ok) {
        apsp::RoundConfig rc = large_round_config(h, APSP_U16, rn);
        rc.sym = true;  // the bound accepts only a symmetric W
        const int64_t ld16 = round_up(rn, 8);
        const bool all = rc.p3 == 4;
        const size_t pb = (apsp::panel_buffer_bytes(rn, ldT, all) + 255) & ~size_t(255);
        const size_t pbytes = (size_t)rn * ld16 * 2;
        const size_t rpb = (apsp::row_panel_bytes(ldT, all) + 255) & ~size_t(255);
        if (cudaMallocAsync(&g->ws, pb + rpb + pbytes, s) != cudaSuccess) {
          g->ws = nullptr;
          return APSP_E_CUDA;
        }
        char *wsb = static_cast<char *>(g->ws);
        rc.rowP = wsb + pb;
        uint16_t *P = reinterpret_cast<uint16_t *>(wsb + pb + rpb);
        int32_t *Dr = static_cast<int32_t *>(rs[0]->D);
        if (apsp::launch_pack(Dr, rn, P, ld16, rn, s, &l) != cudaSuccess ||
            apsp::launch_rounds(APSP_U16, P, ld16, rn, g->ws, ldT, s, &l, nullptr, rc, g->status + 1) !=
                cudaSuccess ||
            apsp::launch_unpack(P, ld16, Dr, rn, rn, s, &l) != cudaSuccess)
          return APSP_E_CUDA;
        h->launches += l;
        if (cudaEventRecord(g->done_ev, s) != cudaSuccess) return APSP_E_CUDA;
        g->graphs_dev = nullptr;
        return APSP_OK;
      }
    }
    apsp::RoundConfig rc = large_round_config(h, APSP_I32, rn);
    if (cudaMallocAsync(&g->ws, apsp::panel_buffer_bytes(rn, ldT, rc.p3 == 4), s) != cudaSuccess) {
      g->ws = nullptr;
      return APSP_E_CUDA;
    }
    if (h->cfg.symmetric == 1) {
      rc.sym = true;
    } else if (h->cfg.symmetric == 0) {
      int *dflag = g->status + 2;  // zeroed with the status words
      if (apsp::launch_symmetry_check(APSP_I32, rs[0]->D, rn, rn, dflag, s) != cudaSuccess) return APSP_E_CUDA;
      if (apsp::single_launch(APSP_I32, rs[0]->D, rn, rn, rc)) {
        rc.sym_flag = dflag;  // every round in one launch: the kernel reads the answer itself
      } else {
        // one launch per round: the answer is read back before the rounds are enqueued
        int flag = 0;
        if (cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
          return APSP_E_CUDA;
        rc.sym = flag == 0;
      }
    }
    if (apsp::launch_rounds(APSP_I32, rs[0]->D, rn, rn, g->ws, ldT, s, &l, nullptr, rc, g->status + 1) !=
        cudaSuccess)
      return APSP_E_CUDA;
    h->launches += l;
    if (cudaEventRecord(g->done_ev, s) != cudaSuccess) return APSP_E_CUDA;
    g->graphs_dev = nullptr;
    return APSP_OK;
  }
  // only graphs with n > 0 take part; group indices follow the tickets
  apsp::BatchPlan plan;
  std::vector<uint32_t *> colT(D.size(), nullptr);
  plan.build(D, n, ld, colT);
  const size_t plan_bytes = plan.workspace_bytes();
  const size_t need = batch_layout(n, nullptr, colT, plan_bytes);
  if (cudaMallocAsync(&g->ws, need, s) != cudaSuccess) {
    g->ws = nullptr;
    return APSP_E_CUDA;
  }
  batch_layout(n, static_cast<char *>(g->ws), colT, plan_bytes);
  plan.build(D, n, ld, colT);
  if (!D.empty() &&
      apsp::launch_batch(plan, g->ws, s, h->cfg.spin_limit, nullptr, g->status + rs.size(), &g->graphs_dev, &l) !=
          cudaSuccess)
    return APSP_E_CUDA;
  h->launches += l;
  if (cudaEventRecord(g->done_ev, s) != cudaSuccess) return APSP_E_CUDA;
  // graphs_dev indexes only n > 0 graphs; map statuses back by skipping n == 0
  if (D.size() != rs.size()) g->graphs_dev = nullptr;
  return APSP_OK;
}

void worker_loop(apsp_handle *h) {
  cudaSetDevice(h->cfg.device);
  std::unique_lock<std::mutex> g(h->smu);
  while (!h->stopping) {
    poll_groups(h);
    // one group per pass from the front of the queue, in arrival order
    if (!h->queue.empty() && (int)h->groups.size() < kMaxGroupsInFlight) {
      std::vector<Request *> rs;
      int64_t add = 0;
      // a request that finds the server idle (nothing in flight, nothing
      // queued behind it) runs alone on the per-round kernels, like a large one:
      // with nothing to share the GPU with, the batched kernel only adds its
      // setup and its lower tile rate
      const bool lone = h->groups.empty() && h->queue.size() == 1;
      while (!h->queue.empty() && (int)rs.size() < h->cfg.max_batch) {
        Request *r = h->reqs[h->queue.front()].get();
        const bool big = r->req.n >= large_n(h);
        bool large = lone || big;
        if (large && !rs.empty()) break;  // a large request starts its own group
        int64_t b = r->bytes + panel_bytes(r->req.n) + (large ? large_extra_bytes(h, r->req) : 0);
        if (large && !big && h->used + add + b > h->budget) {
          large = false;  // no room for the per-round workspace: the batched kernel after all
          b = r->bytes + panel_bytes(r->req.n);
        }
        if (h->used + add + b > h->budget) break;  // wait for memory to free up
        h->queue.pop_front();
        r->alone = large;
        r->transient = b - r->bytes;
        add += b;
        rs.push_back(r);
        if (large) break;
      }
      if (!rs.empty()) {
        h->used += add;
        // admitted: the requests join a group (in flight, not yet enqueued),
        // then the device work is enqueued without the lock
        auto grp = std::make_shared<Group>();
        if (!h->free_streams.empty()) {
          grp->stream = h->free_streams.back();
          h->free_streams.pop_back();
        } else if (cudaStreamCreateWithFlags(&grp->stream, cudaStreamNonBlocking) != cudaSuccess) {
          grp->stream = nullptr;
        }
        for (Request *r : rs) {
          r->group = grp;
          r->gidx = (int)grp->tickets.size();
          grp->tickets.push_back(r->ticket);
          grp->transient += r->transient;
          r->admitted = true;
        }
        h->groups.push_back(grp);
        g.unlock();
        const apsp_status st = admit_group_steps(h, rs, grp.get());
        g.lock();
        if (st == APSP_OK) grp->enqueued = true;
        else undo_admission(h, rs, grp, st);
        continue;  // look for more work right away
      }
    }
    h->scv.wait_for(g, std::chrono::microseconds(h->groups.empty() ? 2000 : 20));
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
  if (r->dtype != APSP_I32 && r->dtype != APSP_AUTO)
    return set_err(h, APSP_E_UNSUPPORTED, "requests are APSP_I32 or APSP_AUTO");
  cudaSetDevice(h->cfg.device);
  std::unique_lock<std::mutex> g(h->smu);
  start_worker(h);
  const int64_t bytes = r->n * r->n * 4;
  if (bytes + panel_bytes(r->n) > h->budget) return APSP_E_NOMEM;
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
  if (r->admitted && !r->finished && r->group && r->group->enqueued &&
      cudaEventQuery(r->group->done_ev) == cudaSuccess)
    finish_group(h, r->group);
  if (r->err != APSP_OK) {
    *st = APSP_ERROR;
    return r->err;
  }
  if (!r->admitted) {
    *st = APSP_QUEUED;
    return APSP_OK;
  }
  if (r->finished) {
    *st = APSP_DONE;
    if (D_dev) *D_dev = r->D;
    return APSP_OK;
  }
  // admitted: the device work being enqueued or the input copy in flight
  // (ADMITTED), or the copy done and the rounds running (RUNNING)
  *st = (r->group && r->group->copy_recorded && cudaEventQuery(r->group->copy_ev) == cudaSuccess) ? APSP_RUNNING
                                                                                                : APSP_ADMITTED;
  return APSP_OK;
}

apsp_status apsp_wait(apsp_handle *h, uint64_t ticket, int64_t timeout_ms) {
  if (!h) return APSP_E_INVALID;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    apsp_state st;
    apsp_status s = apsp_poll(h, ticket, &st, nullptr);
    if (s != APSP_OK) return s;
    if (st == APSP_DONE) return APSP_OK;
    if (timeout_ms >= 0 && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
      return APSP_E_NOTREADY;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

apsp_status apsp_fetch(apsp_handle *h, uint64_t ticket, void *dst, int64_t ldd, void *stream) {
  if (!h || !dst) return APSP_E_INVALID;
  std::unique_lock<std::mutex> g(h->smu);
  auto it = h->reqs.find(ticket);
  if (it == h->reqs.end()) return APSP_E_NOTFOUND;
  Request *r = it->second.get();
  if (r->err != APSP_OK) return r->err;
  if (!r->admitted || !r->group || !r->group->enqueued) return APSP_E_NOTREADY;
  const int64_t n = r->req.n;
  if (ldd < n) return APSP_E_INVALID;
  if (n == 0) return APSP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamWaitEvent(s, r->group->done_ev, 0) != cudaSuccess) return APSP_E_CUDA;
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
  if (r->admitted && !r->finished && r->group) {
    if (!r->group->enqueued || cudaEventQuery(r->group->done_ev) != cudaSuccess)
      return APSP_E_NOTREADY;  // still being enqueued or running
    finish_group(h, r->group);
  }
  if (!r->admitted) {
    h->queue.erase(std::remove(h->queue.begin(), h->queue.end(), ticket), h->queue.end());
  } else if (r->D) {
    cudaFreeAsync(r->D, r->group ? r->group->stream : nullptr);
    r->D = nullptr;
    h->used -= r->bytes;
  }
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
