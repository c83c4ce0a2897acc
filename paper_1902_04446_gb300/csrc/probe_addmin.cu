// Add-min issue-rate probe (a standalone program, not part of libapsp.so).
// Independent add-min chains in registers, one variant per template MODE;
// prints lane-ops per clock per SM (from clock64) and checks the 16-bit lane
// semantics (wrapping add) on edge values.  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/probe_addmin \
//        paper_1902_04446_gb300/csrc/probe_addmin.cu && /tmp/probe_addmin
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define NCH 16
template <int MODE>
__device__ __forceinline__ uint32_t op(uint32_t c, uint32_t a, uint32_t c1, uint32_t one) {
  if (MODE == 0) return (uint32_t)__viaddmin_s32((int)c, (int)a, (int)c1);
  if (MODE == 1) { int s = (int)c + (int)a; return (uint32_t)min(s, (int)c1); }
  if (MODE == 2) return __viaddmin_u16x2(c, a, c1);
  if (MODE == 3) return __viaddmin_s16x2(c, a, c1);
  if (MODE == 4) return __vminu2(__vadd2(c, a), c1);
  if (MODE == 5) { float r = fminf(__uint_as_float(c) + __uint_as_float(a), __uint_as_float(c1)); return __float_as_uint(r); }
  if (MODE == 6) { int s; asm volatile("mad.lo.s32 %0, %1, %2, %3;" : "=r"(s) : "r"((int)c), "r"((int)one), "r"((int)a)); return (uint32_t)min(s, (int)c1); }
  if (MODE == 7) return __viaddmin_u32(c, a, c1);
  return 0;
}

template <int MODE>
__global__ void probe(const uint32_t* in, uint32_t* out, int iters, unsigned long long* cyc) {
  uint32_t c[NCH], a[NCH];
  uint32_t one = in[1024];
  int t = threadIdx.x;
#pragma unroll
  for (int j = 0; j < NCH; ++j) { c[j] = in[(t + j) & 1023]; a[j] = in[(t * 3 + j) & 1023]; }
  unsigned long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    uint32_t n[NCH];
#pragma unroll
    for (int j = 0; j < NCH; ++j) n[j] = op<MODE>(c[j], a[j], c[(j + 1) % NCH], one);
#pragma unroll
    for (int j = 0; j < NCH; ++j) c[j] = n[j];
  }
  unsigned long long t1 = clock64();
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < NCH; ++j) s ^= c[j];
  out[blockIdx.x * blockDim.x + t] = s;
  if (t == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void semantics(const uint32_t* a, const uint32_t* b, const uint32_t* c, uint32_t* o, int m) {
  int i = threadIdx.x;
  if (i < m) {
    o[4 * i + 0] = __viaddmin_u16x2(a[i], b[i], c[i]);
    o[4 * i + 1] = __viaddmin_s16x2(a[i], b[i], c[i]);
    o[4 * i + 2] = (uint32_t)__viaddmin_s32((int)a[i], (int)b[i], (int)c[i]);
    o[4 * i + 3] = __vminu2(__vadd2(a[i], b[i]), c[i]);
  }
}

template <int MODE>
void run(const char* name, const uint32_t* din, uint32_t* dout, unsigned long long* dcyc, int sms, int blocks_per_sm, int threads) {
  int iters = 1 << 14;
  int grid = sms * blocks_per_sm;
  probe<MODE><<<grid, threads>>>(din, dout, 64, dcyc);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  cudaDeviceSynchronize();
  cudaEventRecord(e0);
  probe<MODE><<<grid, threads>>>(din, dout, iters, dcyc);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  unsigned long long h[4096]; cudaMemcpy(h, dcyc, grid * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  unsigned long long mx = 0; for (int i = 0; i < grid; ++i) mx = h[i] > mx ? h[i] : mx;
  double ops = (double)grid * threads * iters * NCH;
  double per_sm_clk = ops / sms / (double)mx;
  printf("%-22s grid=%d thr=%d ms=%.3f Gop/s=%.1f ops/clk/SM(by clock64)=%.2f implied_MHz=%.0f err=%s\n", name, grid, threads, ms,
         ops / ms / 1e6, per_sm_clk, (double)mx / (ms * 1e3), cudaGetErrorString(cudaGetLastError()));
}

int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  printf("%s sms=%d cc=%d.%d\n", p.name, p.multiProcessorCount, p.major, p.minor);
  int sms = p.multiProcessorCount;
  uint32_t h[1025]; for (int i = 0; i < 1024; ++i) h[i] = (i * 2654435761u) & 0x00ff00ffu; h[1024] = 1;
  uint32_t *din, *dout; unsigned long long* dcyc;
  cudaMalloc(&din, sizeof(h)); cudaMemcpy(din, h, sizeof(h), cudaMemcpyHostToDevice);
  cudaMalloc(&dout, sizeof(uint32_t) * sms * 8 * 1024); cudaMalloc(&dcyc, sizeof(unsigned long long) * 4096);
  for (int cfg = 0; cfg < 2; ++cfg) {
    int bps = cfg == 0 ? 4 : 8, thr = cfg == 0 ? 256 : 256;
    run<0>("viaddmin_s32", din, dout, dcyc, sms, bps, thr);
    run<1>("iadd+imin", din, dout, dcyc, sms, bps, thr);
    run<7>("viaddmin_u32", din, dout, dcyc, sms, bps, thr);
    run<6>("imad(one)+imin", din, dout, dcyc, sms, bps, thr);
    run<2>("viaddmin_u16x2", din, dout, dcyc, sms, bps, thr);
    run<3>("viaddmin_s16x2", din, dout, dcyc, sms, bps, thr);
    run<4>("vadd2+vminu2", din, dout, dcyc, sms, bps, thr);
    run<5>("fadd+fmin", din, dout, dcyc, sms, bps, thr);
  }
  // semantics on edge values (lane layout / wrap vs saturate)
  const int m = 6;
  uint32_t a[m] = {0x7FFF7FFFu, 0xFFFF0001u, 0x80000000u, 0x40000000u, 0x3FFF7FFEu, 0x7FFFFFFFu};
  uint32_t b[m] = {0x7FFF7FFFu, 0x00010001u, 0x80000000u, 0x40000000u, 0x00010001u, 0x00000001u};
  uint32_t c[m] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0x7FFFFFFFu, 0x7FFFFFFFu, 0xFFFFFFFFu, 0x7FFFFFFFu};
  uint32_t *da, *db, *dc, *dout2; uint32_t o[4 * m];
  cudaMalloc(&da, sizeof(a)); cudaMalloc(&db, sizeof(b)); cudaMalloc(&dc, sizeof(c)); cudaMalloc(&dout2, sizeof(o));
  cudaMemcpy(da, a, sizeof(a), cudaMemcpyHostToDevice); cudaMemcpy(db, b, sizeof(b), cudaMemcpyHostToDevice); cudaMemcpy(dc, c, sizeof(c), cudaMemcpyHostToDevice);
  semantics<<<1, 32>>>(da, db, dc, dout2, m);
  cudaMemcpy(o, dout2, sizeof(o), cudaMemcpyDeviceToHost);
  for (int i = 0; i < m; ++i) printf("a=%08x b=%08x c=%08x | u16x2=%08x s16x2=%08x s32=%08x vadd2+vminu2=%08x\n", a[i], b[i], c[i], o[4*i], o[4*i+1], o[4*i+2], o[4*i+3]);
  printf("final err=%s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
