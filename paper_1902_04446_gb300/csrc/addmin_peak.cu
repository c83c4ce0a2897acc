// Measurement support for the ALU roofline of Phase 3: the issue rate of the
// library's own add-min forms on this GPU, and the element-wise add-min itself
// so that its lane semantics can be checked against a host reference.
//
// The relaxation c = min(c, a + b) is the min-plus step of the paper's Table 1
// (MatProd followed by MatMin).  Phase 3 is bound by how many of these the SMs
// issue per clock, so the roofline denominator is that rate:
//   APSP_I32  __viaddmin_s32: one relaxation per 32-bit lane-op
//   APSP_U16  __viaddmin_u16x2: two relaxations per 32-bit lane-op
//   APSP_F32  the Phase-3 tile's form: two k-steps at a time, the sums of two
//             neighbouring columns by one packed pair add (add.rn.f32x2) and
//             each output's two sums taken by one three-input minimum
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/apsp.h"

namespace {

constexpr int kChains = 16;  // independent add-min chains per thread

__device__ __forceinline__ float min3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

template <int DT>
__device__ __forceinline__ uint32_t addmin_op(uint32_t a, uint32_t b, uint32_t c) {
  if constexpr (DT == APSP_I32) return (uint32_t)__viaddmin_s32((int)a, (int)b, (int)c);
  else if constexpr (DT == APSP_U16) return __viaddmin_u16x2(a, b, c);
  else return __float_as_uint(fminf(__uint_as_float(a) + __uint_as_float(b), __uint_as_float(c)));
}

// kChains independent chains per thread: c_j <- addmin(c_j, a_j, c_{j+1}); the
// slowest CTA's clock64 span gives lane-ops per clock per SM.  fp32: kChains
// accumulators as 2 rows x 8 columns of a tile, two k-steps per iteration:
// the row values (taken from the accumulators, so that nothing is
// loop-invariant) duplicated into packed pairs, added to the columns' packed
// pairs, and each accumulator lowered by its two sums with one three-input
// minimum -- 2 kChains relaxations per iteration.
template <int DT>
__global__ void addmin_rate_kernel(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int iters,
                                   unsigned long long *__restrict__ cycles) {
  uint32_t c[kChains], a[kChains];
  const int t = threadIdx.x;
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    c[j] = in[(t + j) & 1023];
    a[j] = in[(3 * t + j) & 1023];
  }
  const unsigned long long t0 = clock64();
  if constexpr (DT == APSP_F32) {
    uint64_t bp[2][4];  // the columns' values, packed in neighbouring pairs, for two k-steps
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int p = 0; p < 4; ++p) bp[k][p] = (uint64_t)a[8 * k + 2 * p] | ((uint64_t)a[8 * k + 2 * p + 1] << 32);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        uint64_t ad[2];
#pragma unroll
        for (int k = 0; k < 2; ++k)
          asm("mov.b64 %0, {%1, %1};" : "=l"(ad[k]) : "r"(c[(8 * r + 8 + k) % kChains]));
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          uint64_t s0, s1;
          asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s0) : "l"(ad[0]), "l"(bp[0][p]));
          asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s1) : "l"(ad[1]), "l"(bp[1][p]));
          float x0, y0, x1, y1;
          asm("mov.b64 {%0, %1}, %2;" : "=f"(x0), "=f"(y0) : "l"(s0));
          asm("mov.b64 {%0, %1}, %2;" : "=f"(x1), "=f"(y1) : "l"(s1));
          const int j = 8 * r + 2 * p;
          c[j] = __float_as_uint(min3f(__uint_as_float(c[j]), x0, x1));
          c[j + 1] = __float_as_uint(min3f(__uint_as_float(c[j + 1]), y0, y1));
        }
      }
    }
  } else {
    for (int it = 0; it < iters; ++it) {
      uint32_t nx[kChains];
#pragma unroll
      for (int j = 0; j < kChains; ++j) nx[j] = addmin_op<DT>(a[j], c[j], c[(j + 1) % kChains]);
#pragma unroll
      for (int j = 0; j < kChains; ++j) c[j] = nx[j];
    }
  }
  const unsigned long long t1 = clock64();
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s ^= c[j];
  out[blockIdx.x * blockDim.x + t] = s;  // keeps the chains live
  if (t == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int DT>
__global__ void addmin_eval_kernel(const uint32_t *a, const uint32_t *b, const uint32_t *c, uint32_t *o, int64_t m) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = addmin_op<DT>(a[i], b[i], c[i]);
}

// Relaxations per kernel-iteration step of one chain: 1 per 32-bit lane-op, 2
// for packed 16-bit and for the fp32 form (two k-steps per accumulator).
template <int DT>
constexpr double relax_per_chain_step() { return DT == APSP_I32 ? 1.0 : 2.0; }

template <int DT>
cudaError_t measure(int sms, uint32_t *din, uint32_t *dout, unsigned long long *dcyc, int grid, int threads,
                    double *lanes, double *ms_out) {
  const int iters = 1 << 14;
  addmin_rate_kernel<DT><<<grid, threads>>>(din, dout, 64, dcyc);  // warm-up
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  if (e == cudaSuccess) {
    addmin_rate_kernel<DT><<<grid, threads>>>(din, dout, iters, dcyc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  std::vector<unsigned long long> cyc(grid);
  if (e == cudaSuccess) e = cudaMemcpy(cyc.data(), dcyc, grid * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const unsigned long long span = *std::max_element(cyc.begin(), cyc.end());
  const double relax = (double)grid * threads * iters * kChains * relax_per_chain_step<DT>();
  *lanes = span ? relax / sms / (double)span : 0.0;
  *ms_out = ms;
  return cudaSuccess;
}

}  // namespace

extern "C" apsp_status apsp_addmin_peak(int device, int dtype, double *relax_per_clk_per_sm, double *relax_per_s) {
  if (!relax_per_clk_per_sm || !relax_per_s) return APSP_E_INVALID;
  if (dtype != APSP_I32 && dtype != APSP_U16 && dtype != APSP_F32) return APSP_E_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) return APSP_E_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
    return APSP_E_CUDA;
  const int threads = 256, grid = 4 * sms;  // one full wave: 4 CTAs of 256 threads per SM
  std::vector<uint32_t> h(1024);
  for (int i = 0; i < 1024; ++i) {
    if (dtype == APSP_F32) {  // ordinary non-negative floats (distances), not bit patterns of tiny ones
      const float v = 1.0f + 0.25f * (float)(i % 977);
      std::memcpy(&h[i], &v, sizeof(v));
    } else {
      h[i] = (uint32_t)(i * 2654435761u) & 0x00FF00FFu;
    }
  }
  uint32_t *din = nullptr, *dout = nullptr;
  unsigned long long *dcyc = nullptr;
  cudaError_t e = cudaMalloc(&din, 1024 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&dout, (size_t)grid * threads * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&dcyc, (size_t)grid * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemcpy(din, h.data(), 1024 * sizeof(uint32_t), cudaMemcpyHostToDevice);
  double lanes = 0.0, ms = 0.0;
  if (e == cudaSuccess) {
    if (dtype == APSP_I32) e = measure<APSP_I32>(sms, din, dout, dcyc, grid, threads, &lanes, &ms);
    else if (dtype == APSP_U16) e = measure<APSP_U16>(sms, din, dout, dcyc, grid, threads, &lanes, &ms);
    else e = measure<APSP_F32>(sms, din, dout, dcyc, grid, threads, &lanes, &ms);
  }
  if (din) cudaFree(din);
  if (dout) cudaFree(dout);
  if (dcyc) cudaFree(dcyc);
  if (e != cudaSuccess) return APSP_E_CUDA;
  const double per_step = dtype == APSP_I32 ? 1.0 : 2.0;
  *relax_per_clk_per_sm = lanes;
  *relax_per_s = ms > 0 ? (double)grid * threads * (double)(1 << 14) * kChains * per_step / (ms * 1e-3) : 0.0;
  return APSP_OK;
}

extern "C" apsp_status apsp_addmin_eval(int dtype, const uint32_t *a, const uint32_t *b, const uint32_t *c,
                                        uint32_t *out, int64_t m, void *stream) {
  if (m < 0 || (m > 0 && (!a || !b || !c || !out))) return APSP_E_INVALID;
  if (m == 0) return APSP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned grid = (unsigned)std::min<int64_t>((m + 255) / 256, 4096);
  if (dtype == APSP_I32) addmin_eval_kernel<APSP_I32><<<grid, 256, 0, s>>>(a, b, c, out, m);
  else if (dtype == APSP_U16) addmin_eval_kernel<APSP_U16><<<grid, 256, 0, s>>>(a, b, c, out, m);
  else if (dtype == APSP_F32) addmin_eval_kernel<APSP_F32><<<grid, 256, 0, s>>>(a, b, c, out, m);
  else return APSP_E_INVALID;
  return cudaGetLastError() == cudaSuccess ? APSP_OK : APSP_E_CUDA;
}
