// Blocked Floyd-Warshall kernels for sm_103a (the paper's Sec. 4.4/4.5,
// Alg. 3 and 4, Fig. 1 "processing phases").
//
// Round k covers the vertex range [p0, p1) = [k*BK, min(n, (k+1)*BK)).
//   Phase 1  fw_phase1: Floyd-Warshall closure of the diagonal block D_kk in one
//            CTA (Table 1 FloydWarshall).  Also writes D_kk transposed into the
//            panel buffer colT.
//   Phase 2  fw_phase2: row panel D_kJ = min(D_kJ, D_kk (x) D_kJ) and column
//            panel D_Ik = min(D_Ik, D_Ik (x) D_kk) (Table 1 MinPlus, Alg. 4
//            line "rowcol").  Column-panel CTAs also write their block
//            transposed into colT, so that Phase 3 reads both operands as
//            contiguous rows.
//   Phase 3  fw_phase3: D_IJ = min(D_IJ, D_Ik (x) D_kJ) for every block outside
//            row k and column k (Table 1 MatProd + MatMin, Alg. 4 "offcol").
// The product with a closed D_kk equals the in-place sweep over t of the
// original algorithm: the shortest path from i in block k to j that uses
// intermediate vertices of block k ends with one step from its last block-k
// vertex t, and D_kk(i, t) already holds the best way to reach t.
//
// Layout: D is the caller's row-major matrix (n rows of ld elements).  colT is
// a library-owned BK x ldT buffer (ldT a multiple of 256 elements, >= n):
// colT[t][i] = D[i][p0 + t] after Phase 2.  Elements outside the matrix are
// read as INF; INF never improves a finite value, so ragged edges need no
// other handling.
#include <cstdint>
#include <cuda_runtime.h>

#include "fw_device.cuh"
#include "fw_launch.h"

namespace apsp {

constexpr int P1_THREADS = 256;

// ---------------------------------------------------------------- Phase 1
template <class Op, int BK>
__global__ void __launch_bounds__(P1_THREADS) fw_phase1(typename Op::elem *__restrict__ D, int64_t ld, int64_t n,
                                                        int64_t p0, typename Op::elem *__restrict__ colT,
                                                        int64_t ldT) {
  using S = typename Op::scalar;
  constexpr int G = 16;        // 16 x 16 thread grid
  constexpr int PT = BK / G;   // each thread owns PT x PT entries
  static_assert(BK % G == 0, "BK must be a multiple of 16");
  __shared__ S s[BK][BK + 1];
  const int tid = threadIdx.x;
  const int by = tid / G, bx = tid % G;
  const S INF = Op::to_s(Op::inf_elem());
  for (int idx = tid; idx < BK * BK; idx += P1_THREADS) {
    const int i = idx / BK, j = idx % BK;
    const int64_t r = p0 + i, c = p0 + j;
    s[i][j] = (r < n && c < n) ? Op::to_s(D[r * ld + c]) : INF;
  }
  __syncthreads();
  S v[PT][PT];
#pragma unroll
  for (int r = 0; r < PT; ++r)
#pragma unroll
    for (int c = 0; c < PT; ++c) v[r][c] = s[by + G * r][bx + G * c];
  // Step t relaxes every entry through vertex p0 + t.  Row t and column t do
  // not change in step t (D_tt = 0, and INF + x >= x on padded vertices), so
  // one barrier per step orders the steps.
  for (int t = 0; t < BK; ++t) {
    S a[PT], b[PT];
#pragma unroll
    for (int r = 0; r < PT; ++r) a[r] = s[by + G * r][t];
#pragma unroll
    for (int c = 0; c < PT; ++c) b[c] = s[t][bx + G * c];
#pragma unroll
    for (int r = 0; r < PT; ++r)
#pragma unroll
      for (int c = 0; c < PT; ++c) {
        v[r][c] = Op::s_addmin(a[r], b[c], v[r][c]);
        s[by + G * r][bx + G * c] = v[r][c];
      }
    __syncthreads();
  }
  for (int idx = tid; idx < BK * BK; idx += P1_THREADS) {
    const int i = idx / BK, j = idx % BK;
    const int64_t r = p0 + i, c = p0 + j;
    if (r < n && c < n) D[r * ld + c] = Op::from_s(s[i][j]);
  }
  for (int idx = tid; idx < BK * BK; idx += P1_THREADS) {
    const int t = idx / BK, i = idx % BK;
    colT[t * ldT + p0 + i] = Op::from_s(s[i][t]);
  }
}

// ---------------------------------------------------------------- smem loaders
// As[t][i] = dup(colT[t][i0 + i]) for t < BK, i < BM (colT rows are aligned).
template <class Op, int BM, int BK, int NT>
__device__ __forceinline__ void load_As_colT(uint32_t *As, const typename Op::elem *__restrict__ colT, int64_t ldT,
                                             int64_t i0, int tid) {
  constexpr int CH = BK * BM / 4;
  for (int c = tid; c < CH; c += NT) {
    const int t = c / (BM / 4);
    const int i = (c % (BM / 4)) * 4;
    const typename Op::elem *p = colT + t * ldT + i0 + i;
    uint4 v;
    if constexpr (Op::EPW == 1) {
      v = __ldg(reinterpret_cast<const uint4 *>(p));
    } else {
      const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
      v = make_uint4(Op::dup((typename Op::elem)(u.x & 0xFFFFu)), Op::dup((typename Op::elem)(u.x >> 16)),
                     Op::dup((typename Op::elem)(u.y & 0xFFFFu)), Op::dup((typename Op::elem)(u.y >> 16)));
    }
    *reinterpret_cast<uint4 *>(As + t * BM + i) = v;
  }
}

// Bs[t][w] = word w of row (r0 + t), element columns c0 .. c0 + BNW*EPW.
template <class Op, int BNW, int BK, int NT>
__device__ __forceinline__ void load_Bs_rows(uint32_t *Bs, const typename Op::elem *__restrict__ M, int64_t ld,
                                             int64_t nrows, int64_t ncols, int64_t r0, int64_t c0, bool vec,
                                             int tid) {
  constexpr int CH = BK * BNW / 4;
  for (int c = tid; c < CH; c += NT) {
    const int t = c / (BNW / 4);
    const int w = (c % (BNW / 4)) * 4;
    const uint4 v = load_chunk<Op>(M, ld, nrows, ncols, r0 + t, c0 + (int64_t)w * Op::EPW, vec);
    *reinterpret_cast<uint4 *>(Bs + t * BNW + w) = v;
  }
}

// As[t][i] = dup(M[i0 + i][c0 + t]) for t < BK, i < BM: a transposing load of a
// BM x BK block (consecutive threads take consecutive rows, so the scalar
// shared-memory stores hit consecutive banks).
template <class Op, int BM, int BK, int NT>
__device__ __forceinline__ void load_As_transposed(uint32_t *As, const typename Op::elem *__restrict__ M, int64_t ld,
                                                   int64_t nrows, int64_t ncols, int64_t i0, int64_t c0, bool vec,
                                                   int tid) {
  constexpr int E = 4 * Op::EPW;
  constexpr int CH = BM * (BK / E);
  for (int c = tid; c < CH; c += NT) {
    const int i = c % BM;
    const int tq = (c / BM) * E;
    const uint4 v = load_chunk<Op>(M, ld, nrows, ncols, i0 + i, c0 + tq, vec);
#pragma unroll
    for (int e = 0; e < E; ++e)
      As[(tq + e) * BM + i] = Op::dup(bits_elem<Op>(chunk_get<Op>(v, e)));
  }
}

// ---------------------------------------------------------------- Phase 2
// Row-panel CTAs: tile BK x 128 words; column-panel CTAs: tile
// (128 * EPW) x (BK / EPW) words.  Both use 128 threads.
template <class Op, int BK>
struct P2Cfg {
  static constexpr int ROW_BM = BK, ROW_BNW = 128;
  static constexpr int COL_BM = 128 * Op::EPW, COL_BNW = BK / Op::EPW;
  static constexpr int THREADS = 128;
  static_assert(TileMap<ROW_BM, ROW_BNW>::THREADS == THREADS, "row tile");
  static_assert(TileMap<COL_BM, COL_BNW>::THREADS == THREADS, "col tile");
  static constexpr int ROW_SMEM = (BK * ROW_BM + BK * ROW_BNW) * 4;
  static constexpr int COL_SMEM = (BK * COL_BM + BK * COL_BNW) * 4;
  static constexpr int SMEM = ROW_SMEM > COL_SMEM ? ROW_SMEM : COL_SMEM;
};

template <class Op, int BK>
__global__ void __launch_bounds__(128) fw_phase2(typename Op::elem *__restrict__ D, int64_t ld, int64_t n, int64_t p0,
                                                 int64_t p1, typename Op::elem *__restrict__ colT, int64_t ldT,
                                                 int nrow_ctas, int vec) {
  using C = P2Cfg<Op, BK>;
  extern __shared__ __align__(16) uint32_t smem[];
  const int tid = threadIdx.x;
  uint32_t acc[8][8];
  if ((int)blockIdx.x < nrow_ctas) {
    // row panel: D_kJ = min(D_kJ, D_kk (x) D_kJ); A = D_kk (from colT), B = C = D_kJ
    using Map = TileMap<C::ROW_BM, C::ROW_BNW>;
    uint32_t *As = smem;
    uint32_t *Bs = smem + BK * C::ROW_BM;
    const int tx = tid % Map::TX, ty = tid / Map::TX;
    const int64_t col0 = (int64_t)blockIdx.x * C::ROW_BNW * Op::EPW;
    load_As_colT<Op, C::ROW_BM, BK, C::THREADS>(As, colT, ldT, p0, tid);
    load_Bs_rows<Op, C::ROW_BNW, BK, C::THREADS>(Bs, D, ld, n, n, p0, col0, vec, tid);
    load_acc<Op, C::ROW_BM, C::ROW_BNW>(D, ld, n, n, p0, col0, vec, acc, ty, tx);
    __syncthreads();
    tile_minplus<Op, C::ROW_BM, C::ROW_BNW, BK>(As, Bs, acc, ty, tx);
    store_acc<Op, C::ROW_BM, C::ROW_BNW>(D, ld, n, n, p0, col0, 0, 0, p0, p1, vec, acc, ty, tx);
  } else {
    // column panel: D_Ik = min(D_Ik, D_Ik (x) D_kk); A = C = D_Ik, B = D_kk
    using Map = TileMap<C::COL_BM, C::COL_BNW>;
    uint32_t *As = smem;
    uint32_t *Bs = smem + BK * C::COL_BM;
    const int tx = tid % Map::TX, ty = tid / Map::TX;
    const int64_t row0 = (int64_t)(blockIdx.x - nrow_ctas) * C::COL_BM;
    load_As_transposed<Op, C::COL_BM, BK, C::THREADS>(As, D, ld, n, n, row0, p0, vec, tid);
    load_Bs_rows<Op, C::COL_BNW, BK, C::THREADS>(Bs, D, ld, n, n, p0, p0, vec, tid);
    load_acc<Op, C::COL_BM, C::COL_BNW>(D, ld, n, n, row0, p0, vec, acc, ty, tx);
    __syncthreads();
    tile_minplus<Op, C::COL_BM, C::COL_BNW, BK>(As, Bs, acc, ty, tx);
    store_acc<Op, C::COL_BM, C::COL_BNW>(D, ld, n, n, row0, p0, p0, p1, 0, 0, vec, acc, ty, tx);
    // transposed copy: colT[t][row0 + i] = D_Ik[i][t] for rows outside [p0, p1)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int ib = Map::row(ty, 4 * g);   // 4 consecutive rows ib .. ib+3
        const int64_t rb = row0 + ib;
        const bool all_out = (rb + 3 < p0) || (rb >= p1);
#pragma unroll
        for (int cw = 0; cw < 4; ++cw) {
          const int w = Map::wcol(tx, h) + cw;
#pragma unroll
          for (int lane = 0; lane < Op::EPW; ++lane) {
            const int t = w * Op::EPW + lane;
            typename Op::elem e4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const uint32_t word = acc[4 * g + q][4 * h + cw];
              e4[q] = bits_elem<Op>(Op::EPW == 2 ? (lane ? (word >> 16) : (word & 0xFFFFu)) : word);
            }
            typename Op::elem *dst = colT + (int64_t)t * ldT + rb;
            if (all_out) {
              if constexpr (Op::EPW == 1) {
                *reinterpret_cast<uint4 *>(dst) =
                    make_uint4(elem_bits<Op>(e4[0]), elem_bits<Op>(e4[1]), elem_bits<Op>(e4[2]), elem_bits<Op>(e4[3]));
              } else {
                *reinterpret_cast<uint2 *>(dst) =
                    make_uint2(elem_bits<Op>(e4[0]) | (elem_bits<Op>(e4[1]) << 16),
                               elem_bits<Op>(e4[2]) | (elem_bits<Op>(e4[3]) << 16));
              }
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (rb + q < p0 || rb + q >= p1) dst[q] = e4[q];
            }
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------- Phase 3
template <class Op>
struct P3Cfg {
  static constexpr int BM = 128, BNW = 128;
  static constexpr int THREADS = TileMap<BM, BNW>::THREADS;  // 256
};

template <class Op, int BK>
__global__ void __launch_bounds__(256, 2) fw_phase3(typename Op::elem *__restrict__ D, int64_t ld, int64_t n,
                                                    int64_t p0, int64_t p1,
                                                    const typename Op::elem *__restrict__ colT, int64_t ldT,
                                                    int vec) {
  using Cfg = P3Cfg<Op>;
  using Map = TileMap<Cfg::BM, Cfg::BNW>;
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t *As = smem;
  uint32_t *Bs = smem + BK * Cfg::BM;
  const int tid = threadIdx.x;
  const int tx = tid % Map::TX, ty = tid / Map::TX;
  const int64_t row0 = (int64_t)blockIdx.y * Cfg::BM;
  const int64_t col0 = (int64_t)blockIdx.x * Cfg::BNW * Op::EPW;
  uint32_t acc[8][8];
  load_As_colT<Op, Cfg::BM, BK, Cfg::THREADS>(As, colT, ldT, row0, tid);
  load_Bs_rows<Op, Cfg::BNW, BK, Cfg::THREADS>(Bs, D, ld, n, n, p0, col0, vec, tid);
  load_acc<Op, Cfg::BM, Cfg::BNW>(D, ld, n, n, row0, col0, vec, acc, ty, tx);
  __syncthreads();
  tile_minplus<Op, Cfg::BM, Cfg::BNW, BK>(As, Bs, acc, ty, tx);
  store_acc<Op, Cfg::BM, Cfg::BNW>(D, ld, n, n, row0, col0, p0, p1, p0, p1, vec, acc, ty, tx);
}

// ---------------------------------------------------------------- general min-plus
// C = min(C, A (x) B) for A m x k, B k x n, C m x n (Table 1 MatProd + MatMin).
template <class Op, int BK>
__global__ void __launch_bounds__(256, 2) minplus_kernel(const typename Op::elem *__restrict__ A, int64_t lda,
                                                         const typename Op::elem *__restrict__ B, int64_t ldb,
                                                         typename Op::elem *__restrict__ Cm, int64_t ldc, int64_t m,
                                                         int64_t k, int64_t nn, int veca, int vecb, int vecc) {
  using Cfg = P3Cfg<Op>;
  using Map = TileMap<Cfg::BM, Cfg::BNW>;
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t *As = smem;
  uint32_t *Bs = smem + BK * Cfg::BM;
  const int tid = threadIdx.x;
  const int tx = tid % Map::TX, ty = tid / Map::TX;
  const int64_t row0 = (int64_t)blockIdx.y * Cfg::BM;
  const int64_t col0 = (int64_t)blockIdx.x * Cfg::BNW * Op::EPW;
  uint32_t acc[8][8];
  load_acc<Op, Cfg::BM, Cfg::BNW>(Cm, ldc, m, nn, row0, col0, vecc, acc, ty, tx);
  for (int64_t t0 = 0; t0 < k; t0 += BK) {
    load_As_transposed<Op, Cfg::BM, BK, Cfg::THREADS>(As, A, lda, m, k, row0, t0, veca, tid);
    load_Bs_rows<Op, Cfg::BNW, BK, Cfg::THREADS>(Bs, B, ldb, k, nn, t0, col0, vecb, tid);
    __syncthreads();
    tile_minplus<Op, Cfg::BM, Cfg::BNW, BK>(As, Bs, acc, ty, tx);
    __syncthreads();
  }
  store_acc<Op, Cfg::BM, Cfg::BNW>(Cm, ldc, m, nn, row0, col0, 0, 0, 0, 0, vecc, acc, ty, tx);
}

// ---------------------------------------------------------------- ingest / checks
// Copies W to D (when they differ) and checks the input: diagonal 0, weights
// >= 0, finite weights < INF.  status |= 1 (invalid) or 2 (range).
template <class Op>
__global__ void ingest_kernel(const typename Op::elem *__restrict__ W, typename Op::elem *__restrict__ D, int64_t n,
                              int64_t ld, int copy, int *status) {
  int bad = 0;
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
      const typename Op::elem e = W[i * ld + j];
      if constexpr (Op::DTYPE == 2) {
        if (!(e >= 0.0f)) bad |= 1;              // negative or NaN
        if (i == j && e != 0.0f) bad |= 1;
      } else if constexpr (Op::DTYPE == 1) {
        if (e > Op::inf_elem()) bad |= 2;
        if (i == j && e != 0) bad |= 1;
      } else {
        if (e < 0) bad |= 1;
        if (e > Op::inf_elem()) bad |= 2;
        if (i == j && e != 0) bad |= 1;
      }
      if (copy) D[i * ld + j] = e;
    }
  }
  if (bad) atomicOr(status, bad);
}

__global__ void pack_kernel(const int32_t *__restrict__ s, int64_t lds, uint16_t *__restrict__ d, int64_t ldd,
                            int64_t n) {
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y)
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
      const int32_t v = s[i * lds + j];
      d[i * ldd + j] = (uint16_t)(v >= 0x7FFF ? 0x7FFF : v);
    }
}

__global__ void unpack_kernel(const uint16_t *__restrict__ s, int64_t lds, int32_t *__restrict__ d, int64_t ldd,
                              int64_t n) {
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y)
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
      const uint16_t v = s[i * lds + j];
      d[i * ldd + j] = v >= 0x7FFF ? 1073741823 : (int32_t)v;
    }
}

// D = INF off the diagonal, 0 on it (n x n region of D).
template <class Op>
__global__ void fill_inf_kernel(typename Op::elem *__restrict__ D, int64_t n, int64_t ld) {
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y)
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
      D[i * ld + j] = (i == j) ? (typename Op::elem)0 : Op::inf_elem();
}

// Minimum of a 16-bit element by a 16-bit compare-and-swap loop.
__device__ __forceinline__ void atomic_min_u16(uint16_t *p, uint16_t v) {
  unsigned short *a = reinterpret_cast<unsigned short *>(p);
  unsigned short old = *a, assumed;
  do {
    assumed = old;
    if (assumed <= v) return;
    old = atomicCAS(a, assumed, (unsigned short)v);
  } while (old != assumed);
}

// Scatters an undirected edge list into D (min over duplicates; self loops
// ignored).  status |= 1 for a bad vertex id or negative weight, 2 for a
// weight >= INF.
template <class Op>
__global__ void scatter_edges_kernel(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                                     const typename Op::elem *__restrict__ w, int64_t m, typename Op::elem *D,
                                     int64_t n, int64_t ld, int *status) {
  int bad = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = src[e], v = dst[e];
    const typename Op::elem x = w[e];
    if (u < 0 || u >= n || v < 0 || v >= n) { bad |= 1; continue; }
    if constexpr (Op::DTYPE == 2) {
      if (!(x >= 0.0f)) { bad |= 1; continue; }
    } else if constexpr (Op::DTYPE == 0) {
      if (x < 0) { bad |= 1; continue; }
    }
    if (x >= Op::inf_elem()) { if (!(Op::DTYPE == 2 && x == Op::inf_elem())) bad |= 2; continue; }
    if (u == v) continue;
    if constexpr (Op::DTYPE == 1) {
      atomic_min_u16(&D[u * ld + v], x);
      atomic_min_u16(&D[v * ld + u], x);
    } else if constexpr (Op::DTYPE == 2) {
      // non-negative IEEE floats order like their bit patterns
      atomicMin(reinterpret_cast<int *>(&D[u * ld + v]), __float_as_int(x));
      atomicMin(reinterpret_cast<int *>(&D[v * ld + u]), __float_as_int(x));
    } else {
      atomicMin(reinterpret_cast<int *>(&D[u * ld + v]), (int)x);
      atomicMin(reinterpret_cast<int *>(&D[v * ld + u]), (int)x);
    }
  }
  if (bad) atomicOr(status, bad);
}

// ---------------------------------------------------------------- host launchers
static inline unsigned grid_rows(int64_t n) { return (unsigned)(n < 65535 ? (n > 0 ? n : 1) : 65535); }
static inline unsigned grid_cols(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return (unsigned)(g < 1 ? 1 : (g > 64 ? 64 : g));
}

template <class Op, int BK>
static cudaError_t rounds_impl(void *Dv, int64_t ld, int64_t n, void *colTv, int64_t ldT, bool vec, cudaStream_t s,
                               int64_t *launches, PhaseTimer *tm) {
  using E = typename Op::elem;
  E *D = static_cast<E *>(Dv);
  E *colT = static_cast<E *>(colTv);
  using C2 = P2Cfg<Op, BK>;
  using C3 = P3Cfg<Op>;
  constexpr int SMEM3 = (BK * C3::BM + BK * C3::BNW) * 4;
  // the attributes are per device, so they are set on every call (a cheap host call)
  cudaError_t e = cudaFuncSetAttribute(fw_phase2<Op, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2::SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fw_phase3<Op, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM3);
  if (e != cudaSuccess) return e;
  const int64_t q = (n + BK - 1) / BK;
  const int nrow = (int)((n + C2::ROW_BNW * Op::EPW - 1) / (C2::ROW_BNW * Op::EPW));
  const int ncol = (int)((n + C2::COL_BM - 1) / C2::COL_BM);
  const dim3 g3((unsigned)((n + C3::BNW * Op::EPW - 1) / (C3::BNW * Op::EPW)), (unsigned)((n + C3::BM - 1) / C3::BM));
  for (int64_t k = 0; k < q; ++k) {
    const int64_t p0 = k * BK;
    const int64_t p1 = (p0 + BK < n) ? p0 + BK : n;
    const double w = (double)(p1 - p0), rest = (double)(n - (p1 - p0));
    if (tm) tm->before(0, s);
    fw_phase1<Op, BK><<<1, P1_THREADS, 0, s>>>(D, ld, n, p0, colT, ldT);
    if (tm) tm->after(0, s, w * w * w);
    if (q > 1) {
      if (tm) tm->before(1, s);
      fw_phase2<Op, BK><<<nrow + ncol, C2::THREADS, C2::SMEM, s>>>(D, ld, n, p0, p1, colT, ldT, nrow, vec ? 1 : 0);
      if (tm) tm->after(1, s, 2.0 * rest * w * w);
      if (tm) tm->before(2, s);
      fw_phase3<Op, BK><<<g3, C3::THREADS, SMEM3, s>>>(D, ld, n, p0, p1, colT, ldT, vec ? 1 : 0);
      if (tm) tm->after(2, s, rest * rest * w);
    }
    if (launches) *launches += (q > 1) ? 3 : 1;
  }
  return cudaGetLastError();
}

static bool aligned16(const void *p, int64_t ld, size_t esz) {
  return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && ((ld * (int64_t)esz) % 16 == 0);
}

cudaError_t launch_rounds(int dtype, void *D, int64_t ld, int64_t n, void *colT, int64_t ldT, cudaStream_t s,
                          int64_t *launches, PhaseTimer *tm) {
  if (n <= 0) return cudaSuccess;
  switch (dtype) {
    case 0: return rounds_impl<OpI32, 64>(D, ld, n, colT, ldT, aligned16(D, ld, 4), s, launches, tm);
    case 1: return rounds_impl<OpU16, 64>(D, ld, n, colT, ldT, aligned16(D, ld, 2), s, launches, tm);
    case 2: return rounds_impl<OpF32, 64>(D, ld, n, colT, ldT, aligned16(D, ld, 4), s, launches, tm);
    default: return cudaErrorInvalidValue;
  }
}

int64_t round_width(int dtype) {
  (void)dtype;
  return 64;
}

template <class Op>
static cudaError_t ingest_impl(const void *W, void *D, int64_t n, int64_t ld, int *status, cudaStream_t s,
                               int64_t *launches) {
  using E = typename Op::elem;
  dim3 g(grid_cols(n, 256), grid_rows(n));
  ingest_kernel<Op><<<g, 256, 0, s>>>(static_cast<const E *>(W), static_cast<E *>(D), n, ld, W != D ? 1 : 0, status);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_ingest(int dtype, const void *W, void *D, int64_t n, int64_t ld, int *status, cudaStream_t s,
                          int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  switch (dtype) {
    case 0: return ingest_impl<OpI32>(W, D, n, ld, status, s, launches);
    case 1: return ingest_impl<OpU16>(W, D, n, ld, status, s, launches);
    case 2: return ingest_impl<OpF32>(W, D, n, ld, status, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pack(const int32_t *src, int64_t lds, uint16_t *dst, int64_t ldd, int64_t n, cudaStream_t s,
                        int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  dim3 g(grid_cols(n, 256), grid_rows(n));
  pack_kernel<<<g, 256, 0, s>>>(src, lds, dst, ldd, n);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_unpack(const uint16_t *src, int64_t lds, int32_t *dst, int64_t ldd, int64_t n, cudaStream_t s,
                          int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  dim3 g(grid_cols(n, 256), grid_rows(n));
  unpack_kernel<<<g, 256, 0, s>>>(src, lds, dst, ldd, n);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

template <class Op>
static cudaError_t densify_impl(const int32_t *src, const int32_t *dst, const void *w, int64_t m, void *D, int64_t n,
                                int64_t ld, int *status, cudaStream_t s, int64_t *launches) {
  using E = typename Op::elem;
  dim3 g(grid_cols(n, 256), grid_rows(n));
  fill_inf_kernel<Op><<<g, 256, 0, s>>>(static_cast<E *>(D), n, ld);
  if (m > 0) {
    int64_t blocks = (m + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    scatter_edges_kernel<Op><<<(unsigned)blocks, 256, 0, s>>>(src, dst, static_cast<const E *>(w), m,
                                                              static_cast<E *>(D), n, ld, status);
  }
  if (launches) *launches += m > 0 ? 2 : 1;
  return cudaGetLastError();
}

cudaError_t launch_densify(int dtype, const int32_t *src, const int32_t *dst, const void *w, int64_t m, void *D,
                           int64_t n, int64_t ld, int *status, cudaStream_t s, int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  switch (dtype) {
    case 0: return densify_impl<OpI32>(src, dst, w, m, D, n, ld, status, s, launches);
    case 1: return densify_impl<OpU16>(src, dst, w, m, D, n, ld, status, s, launches);
    case 2: return densify_impl<OpF32>(src, dst, w, m, D, n, ld, status, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

template <class Op>
static cudaError_t minplus_impl(const void *A, int64_t lda, const void *B, int64_t ldb, void *Cm, int64_t ldc,
                                int64_t m, int64_t k, int64_t nn, cudaStream_t s, int64_t *launches) {
  using E = typename Op::elem;
  using C3 = P3Cfg<Op>;
  constexpr int BK = 64;
  constexpr int SMEM = (BK * C3::BM + BK * C3::BNW) * 4;
  cudaError_t e = cudaFuncSetAttribute(minplus_kernel<Op, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  if (e != cudaSuccess) return e;
  const int64_t gx = (nn + C3::BNW * Op::EPW - 1) / (C3::BNW * Op::EPW);
  const int64_t gy = (m + C3::BM - 1) / C3::BM;
  if (gy > 65535) return cudaErrorInvalidValue;
  const size_t es = sizeof(E);
  minplus_kernel<Op, BK><<<dim3((unsigned)gx, (unsigned)gy), C3::THREADS, SMEM, s>>>(
      static_cast<const E *>(A), lda, static_cast<const E *>(B), ldb, static_cast<E *>(Cm), ldc, m, k, nn,
      aligned16(A, lda, es) ? 1 : 0, aligned16(B, ldb, es) ? 1 : 0, aligned16(Cm, ldc, es) ? 1 : 0);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_minplus(int dtype, const void *A, int64_t lda, const void *B, int64_t ldb, void *Cm, int64_t ldc,
                           int64_t m, int64_t k, int64_t nn, cudaStream_t s, int64_t *launches) {
  if (m <= 0 || nn <= 0) return cudaSuccess;
  switch (dtype) {
    case 0: return minplus_impl<OpI32>(A, lda, B, ldb, Cm, ldc, m, k, nn, s, launches);
    case 1: return minplus_impl<OpU16>(A, lda, B, ldb, Cm, ldc, m, k, nn, s, launches);
    case 2: return minplus_impl<OpF32>(A, lda, B, ldb, Cm, ldc, m, k, nn, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace apsp
