// Precision selection for packed 16-bit distances.
//
// For a connected component c with smallest vertex r_c, every finite distance
// inside c satisfies d(i,j) <= d(i,r_c) + d(r_c,j) <= 2 ecc(r_c) (triangle
// inequality through r_c; the graph is undirected, Sec. 3).  So if
// max_c 2 ecc(r_c) < 0x7FFF every finite distance fits below the 16-bit INF.
//
// Components and single-source distances are found together by one
// Bellman-Ford over the edge list on 64-bit keys key[v] = (label << 32) | dist,
// starting from key[v] = (v << 32) | 0 and relaxing key[v] = min(key[v],
// (label(u) << 32) | (dist(u) + w(u,v))) along every edge in both directions.
// At the fixed point label(v) is the smallest vertex of v's component and
// dist(v) its distance from that vertex.  Distances saturate at 2^32 - 1.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "fw_launch.h"

namespace apsp {

namespace {

__device__ __forceinline__ unsigned long long relax_key(unsigned long long ku, unsigned long long w) {
  const unsigned long long d = (ku & 0xFFFFFFFFull) + w;
  return (ku & 0xFFFFFFFF00000000ull) | (d > 0xFFFFFFFFull ? 0xFFFFFFFFull : d);
}

__global__ void init_keys(unsigned long long *key, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    key[v] = (unsigned long long)v << 32;
}

template <typename WT>
__global__ void bf_sweep(const int32_t *__restrict__ src, const int32_t *__restrict__ dst, const WT *__restrict__ w,
                         int64_t m, int64_t n, uint64_t inf, unsigned long long *key, int *changed) {
  int ch = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = src[e], v = dst[e];
    const WT wt = w[e];
    if (u < 0 || u >= n || v < 0 || v >= n || u == v) continue;
    if ((int64_t)wt < 0 || (uint64_t)wt >= inf) continue;
    const unsigned long long ku = *((volatile unsigned long long *)&key[u]);
    const unsigned long long kv = *((volatile unsigned long long *)&key[v]);
    const unsigned long long cu = relax_key(ku, (unsigned long long)wt);
    if (cu < kv) { atomicMin(&key[v], cu); ch = 1; }
    const unsigned long long cv = relax_key(kv, (unsigned long long)wt);
    if (cv < ku) { atomicMin(&key[u], cv); ch = 1; }
  }
  if (ch) *changed = 1;
}

__global__ void max_dist(const unsigned long long *key, int64_t n, unsigned long long *out) {
  unsigned long long mx = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long d = key[v] & 0xFFFFFFFFull;
    mx = d > mx ? d : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_down_sync(0xFFFFFFFFu, mx, o);
    mx = x > mx ? x : mx;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

// finite off-diagonal entries per row (one warp per row)
__global__ void count_finite(const int32_t *__restrict__ W, int64_t n, int64_t ld, int64_t *cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; i < n; i += warps) {
    int64_t c = 0;
    for (int64_t j = lane; j < n; j += 32) {
      const int32_t x = W[i * ld + j];
      c += (j != i && x < 1073741823) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    if (lane == 0) cnt[i] = c;
  }
}

// exclusive scan of cnt[0..n) into off[0..n], one block
__global__ void scan_counts(const int64_t *cnt, int64_t n, int64_t *off) {
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < n; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t x = i < n ? cnt[i] : 0;
    int64_t s = x;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane == 31) warp_sums[wid] = s;
    __syncthreads();
    if (wid == 0) {
      int64_t ws = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xFFFFFFFFu, ws, o);
        if (lane >= o) ws += y;
      }
      warp_sums[lane] = ws;  // inclusive
    }
    __syncthreads();
    const int64_t before = (wid > 0 ? warp_sums[wid - 1] : 0) + carry;
    if (i < n) off[i] = before + s - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + s;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[n] = carry;
}

// writes the finite off-diagonal entries of row i at off[i].. (one warp per row)
// and flags an entry whose transpose differs
__global__ void fill_edges(const int32_t *__restrict__ W, int64_t n, int64_t ld, const int64_t *__restrict__ off,
                           int32_t *src, int32_t *dst, int32_t *w, int *asym) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; i < n; i += warps) {
    int64_t pos = off[i];
    for (int64_t j0 = 0; j0 < n; j0 += 32) {
      const int64_t j = j0 + lane;
      int32_t x = 0;
      bool keep = false;
      if (j < n) {
        x = W[i * ld + j];
        keep = (j != i && x < 1073741823);
      }
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
      if (keep) {
        const int64_t p = pos + __popc(bal & ((1u << lane) - 1u));
        src[p] = (int32_t)i;
        dst[p] = (int32_t)j;
        w[p] = x;
        if (W[j * ld + i] != x) bad = 1;
      }
      pos += __popc(bal);
    }
  }
  if (bad) *asym = 1;
}

// Stream-ordered scratch (cudaMallocAsync from the device's memory pool, which
// the library keeps from returning memory to the system, so repeated solves
// reuse it without synchronizing the device).
struct DevBuf {
  void *p = nullptr;
  cudaStream_t s = nullptr;
  explicit DevBuf(cudaStream_t st) : s(st) {}
  cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes, s); }
  ~DevBuf() {
    if (p) cudaFreeAsync(p, s);
  }
};

template <typename WT>
cudaError_t run_bf(const int32_t *src, const int32_t *dst, const WT *w, int64_t m, int64_t n, uint64_t inf,
                   cudaStream_t s, int64_t *bound, int *ok, int64_t *launches) {
  *bound = 0;
  *ok = 1;
  if (n <= 0) return cudaSuccess;
  constexpr int kMaxGroup = 64;  // sweeps between two host checks, at most
  DevBuf keyb(s), aux(s);
  cudaError_t e = keyb.alloc((size_t)n * sizeof(unsigned long long));
  if (e != cudaSuccess) return e;
  e = aux.alloc(64 + kMaxGroup * sizeof(int));
  if (e != cudaSuccess) return e;
  unsigned long long *key = static_cast<unsigned long long *>(keyb.p);
  unsigned long long *mx = static_cast<unsigned long long *>(aux.p);
  int *changed = reinterpret_cast<int *>(static_cast<char *>(aux.p) + 64);  // one flag per sweep of a group
  const unsigned gb = (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  init_keys<<<gb, 256, 0, s>>>(key, n);
  *launches += 1;
  const int64_t eb = (m + 255) / 256;
  const unsigned ge = (unsigned)(eb < 1 ? 1 : (eb > 152 * 8 ? 152 * 8 : eb));
  // At most n + 1 sweeps are needed (each sweep fixes one more hop of every
  // shortest-path tree); a sweep that changes nothing means the keys are final.
  // Sweeps run in groups between host checks, each sweep with its own flag;
  // the groups double (4, 8, ..., 64) so that deep graphs need few round trips
  // while shallow ones stop after a few sweeps.
  bool converged = false;
  int h_flags[kMaxGroup];
  for (int64_t done = 0, group = 4; !converged && done <= n + 1; done += group, group = std::min<int64_t>(2 * group, kMaxGroup)) {
    e = cudaMemsetAsync(changed, 0, (size_t)group * sizeof(int), s);
    if (e != cudaSuccess) return e;
    for (int r = 0; r < group; ++r) bf_sweep<WT><<<ge, 256, 0, s>>>(src, dst, w, m, n, inf, key, changed + r);
    *launches += group;
    e = cudaMemcpyAsync(h_flags, changed, (size_t)group * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    for (int r = 0; r < group && !converged; ++r) converged = h_flags[r] == 0;
  }
  e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  max_dist<<<gb, 256, 0, s>>>(key, n, mx);
  *launches += 1;
  unsigned long long h_mx = 0;
  e = cudaMemcpyAsync(&h_mx, mx, sizeof(h_mx), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  *bound = 2 * (int64_t)h_mx;
  *ok = (*bound < 0x7FFF) && converged;
  return cudaGetLastError();
}

}  // namespace

cudaError_t bound_from_edges(const int32_t *src, const int32_t *dst, const void *w, int wtype, int64_t m, int64_t n,
                             cudaStream_t s, int64_t *bound, int *ok, int64_t *launches) {
  if (wtype == 1)
    return run_bf<uint16_t>(src, dst, static_cast<const uint16_t *>(w), m, n, 0x7FFF, s, bound, ok, launches);
  return run_bf<int32_t>(src, dst, static_cast<const int32_t *>(w), m, n, 1073741823, s, bound, ok, launches);
}

cudaError_t bound_from_dense(const int32_t *W, int64_t n, int64_t ld, int64_t max_edges, cudaStream_t s,
                             int64_t *bound, int *ok, int64_t *launches) {
  *bound = 0;
  *ok = 1;
  if (n <= 0) return cudaSuccess;
  DevBuf offb(s);
  cudaError_t e = offb.alloc((size_t)(2 * n + 2) * sizeof(int64_t) + 64);
  if (e != cudaSuccess) return e;
  int64_t *cnt = static_cast<int64_t *>(offb.p);
  int64_t *off = cnt + n;
  int *asym = reinterpret_cast<int *>(off + n + 1);
  const unsigned gw = (unsigned)((n + 7) / 8 < 152 * 16 ? (n + 7) / 8 : 152 * 16);
  count_finite<<<gw, 256, 0, s>>>(W, n, ld, cnt);
  scan_counts<<<1, 1024, 0, s>>>(cnt, n, off);
  *launches += 2;
  int64_t m = 0;
  e = cudaMemcpyAsync(&m, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (m > max_edges) {
    *bound = INT64_MAX / 4;
    *ok = 0;
    return cudaSuccess;
  }
  DevBuf eb(s);
  e = eb.alloc((size_t)(m > 0 ? m : 1) * 3 * sizeof(int32_t));
  if (e != cudaSuccess) return e;
  int32_t *src = static_cast<int32_t *>(eb.p);
  int32_t *dst = src + m;
  int32_t *w = dst + m;
  e = cudaMemsetAsync(asym, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  fill_edges<<<gw, 256, 0, s>>>(W, n, ld, off, src, dst, w, asym);
  *launches += 1;
  int h_asym = 0;
  e = cudaMemcpyAsync(&h_asym, asym, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = run_bf<int32_t>(src, dst, w, m, n, 1073741823, s, bound, ok, launches);
  if (e != cudaSuccess) return e;
  if (h_asym) *ok = 0;
  return cudaSuccess;
}

}  // namespace apsp
