// Batched persistent blocked Floyd-Warshall: many graphs of uneven n solved in
// one launch.
//
// The rounds of every graph (Phase 1 -> Phase 2 -> Phase 3 per round, the
// paper's Alg. 3/4) are cut into tasks: one Phase-1 task, one task per
// row-panel and column-panel chunk, one task per Phase-3 output tile.  The
// host lists them as segments in the order
//     for round r: for phase p: for every graph with more than r rounds,
// which is a topological order of the dependencies below.  Resident CTAs take
// task ids from a device counter in that order, wait for the task's
// dependency, run it, and count it done:
//     Phase 1 of round r   waits for all Phase-3 tasks of round r-1,
//     Phase 2 of round r   waits for Phase 1 of round r,
//     Phase 3 of round r   waits for all Phase-2 tasks of round r.
// A task only ever waits for tasks with smaller ids, which running CTAs have
// already taken, so the launch always makes progress; rounds of different
// graphs interleave and fill the GPU.  Every wait is bounded: past the spin
// limit the task marks its graph timed out, and the graph's remaining tasks
// are skipped (still counted done) so that nothing waits forever.
//
// Data written earlier in the same launch is read through L2 only
// (ld.global.cg); producers publish with __threadfence + atomicAdd.
#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "batch.h"
#include "fw_tasks.cuh"

namespace apsp {

namespace {

constexpr int BK = 64;
constexpr int NT = 256;
constexpr int P2_ROW_BNW = 256;  // row-panel chunk: 64 x 256 words
constexpr int P2_COL_BM = 256;   // column-panel chunk: 256 x 64 words
constexpr int SMEM_WORDS = BK * BK + BK * P2_ROW_BNW;  // 80 KB: the largest task (Phase 2)
static_assert(SMEM_WORDS >= BK * P2_COL_BM + BK * BK && SMEM_WORDS >= 2 * BK * 128 &&
                  SMEM_WORDS * 4 >= (int)sizeof(P1Smem<OpI32, BK>),
              "shared memory");

__device__ __forceinline__ int ld_volatile(const int *p) { return *reinterpret_cast<const volatile int *>(p); }

// Each task kind is compiled as its own function so that its register
// allocation does not add to the others' under the kernel's 128-register cap.
__device__ __noinline__ void task_p1(const BatchGraph &g, int64_t p0, uint32_t *smem, int tid) {
  auto &s = *reinterpret_cast<P1Smem<OpI32, BK> *>(smem);
  phase1_body<OpI32, BK, NT, true>(g.D, g.ld, g.n, p0, g.colT, g.ldT, s, tid);
}
__device__ __noinline__ void task_p2_row(const BatchGraph &g, int64_t p0, int64_t p1, int idx, uint32_t *smem,
                                         int tid) {
  p2_row_task<OpI32, BK, P2_ROW_BNW, NT, true>(g.D, g.ld, g.n, p0, p1, g.colT, g.ldT, (int64_t)idx * P2_ROW_BNW,
                                              g.vec != 0, smem, tid);
}
__device__ __noinline__ void task_p2_col(const BatchGraph &g, int64_t p0, int64_t p1, int idx, uint32_t *smem,
                                         int tid) {
  p2_col_task<OpI32, BK, P2_COL_BM, NT, true>(g.D, g.ld, g.n, p0, p1, g.colT, g.ldT, (int64_t)idx * P2_COL_BM,
                                             g.vec != 0, smem, tid);
}
__device__ __noinline__ void task_p3(const BatchGraph &g, int64_t p0, int64_t p1, int idx, uint32_t *smem, int tid) {
  const int64_t row0 = (int64_t)(idx / g.tiles_x) * 128;
  const int64_t col0 = (int64_t)(idx % g.tiles_x) * 128;
  p3_task<OpI32, BK, true>(g.D, g.ld, g.n, p0, p1, g.colT, g.ldT, row0, col0, g.vec != 0, smem, tid);
}

__global__ void __launch_bounds__(NT, 2)
    fw_batch_kernel(BatchGraph *G, const BatchSeg *__restrict__ segs, int nsegs, long long total,
                    unsigned long long *head, int *cnt, long long spin_limit, const int *gate, int *err) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ long long s_task;
  __shared__ int s_seg, s_ok;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      const long long task = (long long)atomicAdd(head, 1ull);
      s_task = task;
      if (task < total) {
        int lo = 0, hi = nsegs - 1;  // last segment with first <= task
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (segs[mid].first <= task) lo = mid;
          else hi = mid - 1;
        }
        s_seg = lo;
        const BatchSeg sg = segs[lo];
        const BatchGraph &g = G[sg.graph];
        int ok = ld_volatile(&G[sg.graph].status) == 0;
        const int *dep = nullptr;
        int target = 0;
        if (sg.phase == 0) {
          if (sg.round > 0) {
            dep = cnt + g.cnt_base + (sg.round - 1) * 3 + 2;
            target = g.tiles;
          } else if (gate) {
            dep = gate;
            target = 1;
          }
        } else if (sg.phase == 1) {
          dep = cnt + g.cnt_base + sg.round * 3 + 0;
          target = 1;
        } else {
          dep = cnt + g.cnt_base + sg.round * 3 + 1;
          target = g.nrow + g.ncol;
        }
        if (ok && dep) {
          long long spins = 0;
          while (ld_volatile(dep) < target) {
            if (++spins > spin_limit) {
              atomicOr(&G[sg.graph].status, 4);
              atomicOr(err, 4);
              ok = 0;
              break;
            }
            __nanosleep(64);
          }
          __threadfence();
        }
        s_ok = ok;
      }
    }
    __syncthreads();
    const long long task = s_task;
    if (task >= total) break;
    const BatchSeg sg = segs[s_seg];
    if (s_ok) {
      const BatchGraph g = G[sg.graph];
      const int idx = (int)(task - sg.first);
      const int64_t p0 = (int64_t)sg.round * BK;
      const int64_t p1 = (p0 + BK < g.n) ? p0 + BK : g.n;
      if (sg.phase == 0) task_p1(g, p0, smem, tid);
      else if (sg.phase == 1 && idx < g.nrow) task_p2_row(g, p0, p1, idx, smem, tid);
      else if (sg.phase == 1) task_p2_col(g, p0, p1, idx - g.nrow, smem, tid);
      else task_p3(g, p0, p1, idx, smem, tid);
    }
    __syncthreads();  // every thread's writes of this task are done
    if (tid == 0) {
      __threadfence();
      atomicAdd(cnt + G[sg.graph].cnt_base + sg.round * 3 + sg.phase, 1);
    }
  }
}

int sm_count_now() {
  int dev = 0, c = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
  return c > 0 ? c : 1;
}

}  // namespace

int64_t batch_panel_ld(int64_t n) { return ((n > 0 ? n : 1) + 255) / 256 * 256; }

size_t BatchPlan::workspace_bytes() const {
  const size_t a = graphs.size() * sizeof(BatchGraph);
  const size_t b = segs.size() * sizeof(BatchSeg);
  const size_t c = (size_t)ncounters * sizeof(int);
  return ((a + 255) / 256 + (b + 255) / 256 + (c + 255) / 256 + 1) * 256;
}

void BatchPlan::build(const std::vector<int32_t *> &D, const std::vector<int64_t> &n, const std::vector<int64_t> &ld,
                      const std::vector<uint32_t *> &colT) {
  graphs.clear();
  segs.clear();
  ncounters = 0;
  int maxq = 0;
  for (size_t i = 0; i < D.size(); ++i) {
    BatchGraph g{};
    g.D = D[i];
    g.colT = colT[i];
    g.n = n[i];
    g.ld = ld[i];
    g.vec = (reinterpret_cast<uintptr_t>(D[i]) % 16 == 0 && (ld[i] * 4) % 16 == 0) ? 1 : 0;
    g.ldT = batch_panel_ld(n[i]);
    g.q = (int)((n[i] + BK - 1) / BK);
    g.nrow = (int)((n[i] + P2_ROW_BNW - 1) / P2_ROW_BNW);
    g.ncol = (int)((n[i] + P2_COL_BM - 1) / P2_COL_BM);
    g.tiles_x = (int)((n[i] + 127) / 128);
    g.tiles = g.tiles_x * g.tiles_x;
    g.cnt_base = ncounters;
    g.status = 0;
    ncounters += 3 * std::max(1, g.q);
    maxq = std::max(maxq, g.q);
    graphs.push_back(g);
  }
  long long first = 0;
  for (int r = 0; r < maxq; ++r)
    for (int p = 0; p < 3; ++p)
      for (size_t i = 0; i < graphs.size(); ++i) {
        const BatchGraph &g = graphs[i];
        if (g.q <= r) continue;
        // a single round closes the whole matrix in Phase 1
        const int count = p == 0 ? 1 : (g.q == 1 ? 0 : (p == 1 ? g.nrow + g.ncol : g.tiles));
        if (count == 0) continue;
        segs.push_back(BatchSeg{first, (int)i, r, p, count});
        first += count;
      }
  total = first;
}

cudaError_t launch_batch(const BatchPlan &plan, void *workspace, cudaStream_t s, int64_t spin_limit,
                         const int *gate, int *err, BatchGraph **graphs_dev, int64_t *launches) {
  if (plan.total == 0) return cudaSuccess;
  char *w = static_cast<char *>(workspace);
  BatchGraph *G = reinterpret_cast<BatchGraph *>(w);
  w += (plan.graphs.size() * sizeof(BatchGraph) + 255) / 256 * 256;
  BatchSeg *S = reinterpret_cast<BatchSeg *>(w);
  w += (plan.segs.size() * sizeof(BatchSeg) + 255) / 256 * 256;
  int *cnt = reinterpret_cast<int *>(w);
  w += ((size_t)plan.ncounters * sizeof(int) + 255) / 256 * 256;
  unsigned long long *head = reinterpret_cast<unsigned long long *>(w);
  cudaError_t e;
  e = cudaMemcpyAsync(G, plan.graphs.data(), plan.graphs.size() * sizeof(BatchGraph), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(S, plan.segs.data(), plan.segs.size() * sizeof(BatchSeg), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(cnt, 0, (size_t)plan.ncounters * sizeof(int), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(head, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int smem = SMEM_WORDS * 4;
  e = cudaFuncSetAttribute(fw_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const long long grid = std::min<long long>(2LL * sm_count_now(), plan.total);
  fw_batch_kernel<<<(unsigned)grid, NT, smem, s>>>(G, S, (int)plan.segs.size(), plan.total, head, cnt,
                                                   spin_limit > 0 ? spin_limit : kDefaultSpinLimit, gate, err);
  if (launches) *launches += 1;
  if (graphs_dev) *graphs_dev = G;
  return cudaGetLastError();
}

}  // namespace apsp
