// apsp_solve_i32_noalloc: an int32 solve that allocates no memory.
//
// Who needs it: callers that must not call cudaMalloc (or anything that
// allocates device memory) from the thread or phase they solve in -- for
// example code running under a custom or pre-reserved memory pool that forbids
// outside allocations, a plugin invoked inside another framework's allocator
// hooks, or a real-time loop where an allocation's implicit device
// synchronization is not allowed.  apsp_solve needs a handle, and the handle
// allocates its panel buffer and status word; this entry point needs neither.
//
// Its only scratch memory (the round's panel buffer and one word for the
// bounded-wait flag) is a fixed array in this file, in device global memory,
// sized for n <= APSP_NOALLOC_MAX_N.  Every GPU that loads the library holds
// that array until the process exits.  The flag word of the last call stays
// in the array after the call; apsp_noalloc_status reads it back (a copy
// into the caller's stack, no allocation), so a caller learns when a bounded
// wait of the Phase-3 kernel gave up and left D incomplete.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/apsp.h"
#include "fw_launch.h"

namespace {

// panel buffer: 64 rows (the widest round) x APSP_NOALLOC_MAX_N words, then 64
// words of which the first is the wait flag
constexpr int64_t kPanelWords = 64 * (int64_t)APSP_NOALLOC_MAX_N;
static_assert(APSP_NOALLOC_MAX_N % 256 == 0, "panel rows are padded to 256 words");

static __device__ __align__(256) uint32_t g_noalloc_scratch[kPanelWords + 64];

std::mutex g_mu;
uint32_t *g_scratch_addr[128] = {};  // device address of the array, per device ordinal

// The array's device address for the current device.  The first call on a
// device looks it up with cudaGetSymbolAddress (the host-side name of the
// array is only a stand-in, never a device address).
cudaError_t scratch_for_current_device(uint32_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<uint32_t *>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" apsp_status apsp_solve_i32_noalloc(const int32_t *W, int64_t n, int64_t ld, int32_t *D, void *stream) {
  if (n < 0 || ld < n || (n > 0 && (!W || !D))) return APSP_E_INVALID;
  if (n > APSP_NOALLOC_MAX_N) return APSP_E_RANGE;
  if (n == 0) return APSP_OK;
  uint32_t *scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return APSP_E_CUDA;
  uint32_t *panel = scratch;
  int *wait_flag = reinterpret_cast<int *>(scratch + kPanelWords);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (W != D && cudaMemcpy2DAsync(D, (size_t)ld * 4, W, (size_t)ld * 4, (size_t)n * 4, (size_t)n,
                                  cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return APSP_E_CUDA;
  // the flag must start at zero; the panel buffer is fully rewritten every round
  if (cudaMemsetAsync(wait_flag, 0, sizeof(int), s) != cudaSuccess) return APSP_E_CUDA;
  const int64_t ldT = (n + 255) / 256 * 256;
  apsp::RoundConfig rc;
  rc.bk = 64;  // the static panel holds 64 rows
  if (apsp::launch_rounds(APSP_I32, D, ld, n, panel, ldT, s, nullptr, nullptr, rc, wait_flag) != cudaSuccess)
    return APSP_E_CUDA;
  return APSP_OK;
}

extern "C" apsp_status apsp_noalloc_status(void *stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return APSP_E_CUDA;
  // the flag word sits right after the panel words; a copy from the symbol
  // into a host int (pageable: the copy completes before the call returns)
  int flag = 0;
  if (cudaMemcpyFromSymbol(&flag, g_noalloc_scratch, sizeof(int), kPanelWords * sizeof(uint32_t),
                           cudaMemcpyDeviceToHost) != cudaSuccess)
    return APSP_E_CUDA;
  return (flag & 4) ? APSP_E_TIMEOUT : APSP_OK;
}
