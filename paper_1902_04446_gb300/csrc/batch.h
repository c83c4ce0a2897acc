// Batched persistent blocked Floyd-Warshall (internal; see batch.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace apsp {

// Default bound on every dependency wait of the batched kernel (polls with a
// 64 ns sleep between them: on the order of a second).
constexpr int64_t kDefaultSpinLimit = int64_t(1) << 24;

struct BatchGraph {
  int32_t *D;      // n x n int32 matrix, leading dimension ld (solved in place)
  uint32_t *colT;  // 64 x ldT panel buffer (32-bit words)
  int64_t n, ld, ldT;
  int q;           // rounds
  int nrow, ncol;  // Phase-2 tasks per round (row-panel, column-panel chunks)
  int tiles_x, tiles;  // Phase-3 tasks per round
  int cnt_base;    // first of this graph's 3 * q done-counters
  int vec;         // 16-byte vector access allowed
  int status;      // device-written: 4 = a wait timed out
};

struct BatchSeg {  // tasks [first, first + count) = (graph, round, phase, 0 .. count-1)
  long long first;
  int graph, round, phase, count;
};

struct BatchPlan {
  std::vector<BatchGraph> graphs;
  std::vector<BatchSeg> segs;
  long long total = 0;
  int ncounters = 0;
  void build(const std::vector<int32_t *> &D, const std::vector<int64_t> &n, const std::vector<int64_t> &ld,
             const std::vector<uint32_t *> &colT);
  size_t workspace_bytes() const;
};

// Panel-buffer leading dimension for a graph of n vertices (words per row; 64 rows).
int64_t batch_panel_ld(int64_t n);

// Uploads the plan into `workspace` (plan.workspace_bytes() device bytes) and
// launches the persistent kernel on s.  gate (nullable): round 0 of every
// graph also waits for *gate >= 1.  err |= 4 when a wait timed out; the graph's
// status (at (*graphs_dev)[i].status after the stream syncs) says which.
cudaError_t launch_batch(const BatchPlan &plan, void *workspace, cudaStream_t s, int64_t spin_limit, const int *gate,
                         int *err, BatchGraph **graphs_dev, int64_t *launches);

}  // namespace apsp
