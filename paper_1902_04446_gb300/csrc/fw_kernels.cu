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
// a library-owned BK x ldT buffer of 32-bit words (ldT a multiple of 256,
// >= n): after Phase 2, colT[t][i] holds D[i][p0 + t] as an A-operand word
// (for packed 16-bit the value sits in both lanes).  Elements outside the
// matrix are read as INF; INF never improves a finite value, so ragged edges
// need no other handling.
#include <cstdint>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <utility>

#include <cudaTypedefs.h>

#include "fw_device.cuh"
#include "fw_launch.h"
#include "fw_tasks.cuh"
#include "tma.cuh"

namespace apsp {

constexpr int P1_THREADS = 256;

// ---------------------------------------------------------------- Phase 1
template <class Op, int BK>
__global__ void __launch_bounds__(P1_THREADS) fw_phase1(typename Op::elem *__restrict__ D, Layout L, int64_t n,
                                                        int64_t p0, uint32_t *__restrict__ colT, int64_t ldT) {
  __shared__ P1Smem<Op, BK> s;
  pdl_trigger();
  pdl_wait();
  phase1_body<Op, BK, P1_THREADS, false>(D, L, n, p0, colT, ldT, s, threadIdx.x);
}

// Phase 1 of a 128-wide round: the pivot-block scheme of phase1_body
// (fw_tasks.cuh) on a 32 x 32 grid of threads, each owning a 4 x 4 block of
// D_kk in registers (1024 threads, at most 64 registers each).  Per pivot
// block p (pivots 4p .. 4p+3) every thread closes the 4 x 4 corner K, then
// for each of its rows r forms a' = a (x) K* from the row's pivot-column
// values a (read from shared memory one row at a time, which keeps the
// registers within the limit) and lowers its row by a' (x) b, b = the
// pivot-row values of its columns.  Reading a later than phase1_body does is
// covered by the same argument: a value written back meanwhile is a' itself,
// and a' (x) K* = a' since K* is closed.  Outputs as phase1_body: D_kk, the
// transposed panel rows in colT and, with rowP, the element panel.
constexpr int P1W_THREADS = 1024;
template <class Op>
__device__ __forceinline__ void phase1_body_w128(typename Op::elem *__restrict__ D, Layout L, int64_t n, int64_t p0,
                                                 uint32_t *__restrict__ colT, int64_t ldT, P1Smem<Op, 128> &sm,
                                                 int tid, typename Op::elem *__restrict__ rowP) {
  using S = typename Op::scalar;
  constexpr int BK = 128, G = 32, PT = 4, NT = P1W_THREADS;
  static_assert(G * PT == BK && G * G == NT, "phase 1 layout");
  auto &s = sm.s;
  const int by = tid / G, bx = tid % G;
  const S INF = Op::to_s(Op::inf_elem());
  for (int idx = tid; idx < BK * BK; idx += NT) {
    const int64_t r = p0 + idx / BK, c = p0 + idx % BK;
    s[idx / BK][idx % BK] = (r < n && c < n) ? Op::to_s(D[L.off(r, c)]) : INF;
  }
  __syncthreads();
  S v[PT][PT];
#pragma unroll
  for (int r = 0; r < PT; ++r)
#pragma unroll
    for (int c = 0; c < PT; ++c) v[r][c] = s[by * PT + r][bx * PT + c];
#pragma unroll 1
  for (int p = 0; p < G; ++p) {
    const int t0 = p * PT;
    S K[PT][PT], b[PT][PT];
#pragma unroll
    for (int i = 0; i < PT; ++i)
#pragma unroll
      for (int j = 0; j < PT; ++j) {
        K[i][j] = s[t0 + i][t0 + j];
        b[i][j] = s[t0 + i][bx * PT + j];
      }
#pragma unroll
    for (int m = 0; m < PT; ++m)
#pragma unroll
      for (int i = 0; i < PT; ++i)
#pragma unroll
        for (int j = 0; j < PT; ++j) K[i][j] = Op::s_addmin(K[i][m], K[m][j], K[i][j]);
#pragma unroll
    for (int r = 0; r < PT; ++r) {
      S a[PT], a2[PT];
#pragma unroll
      for (int i = 0; i < PT; ++i) a[i] = s[by * PT + r][t0 + i];
#pragma unroll
      for (int j = 0; j < PT; ++j) {
        S x = a[j];
#pragma unroll
        for (int i = 0; i < PT; ++i) x = Op::s_addmin(a[i], K[i][j], x);
        a2[j] = x;
      }
#pragma unroll
      for (int c = 0; c < PT; ++c)
#pragma unroll
        for (int j = 0; j < PT; ++j) v[r][c] = Op::s_addmin(a2[j], b[j][c], v[r][c]);
    }
    if (p + 1 < G && (by == p + 1 || bx == p + 1)) {
#pragma unroll
      for (int r = 0; r < PT; ++r)
#pragma unroll
        for (int c = 0; c < PT; ++c) s[by * PT + r][bx * PT + c] = v[r][c];
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < PT; ++r)
#pragma unroll
    for (int c = 0; c < PT; ++c) s[by * PT + r][bx * PT + c] = v[r][c];
  __syncthreads();
  for (int idx = tid; idx < BK * BK; idx += NT) {
    const int i = idx / BK, j = idx % BK;
    const int64_t r = p0 + i, c = p0 + j;
    if (r < n && c < n) D[L.off(r, c)] = Op::from_s(s[i][j]);
  }
  for (int idx = tid; idx < BK * BK; idx += NT) {
    const int t = idx / BK, i = idx % BK;
    colT[t * ldT + p0 + i] = Op::dup(Op::from_s(s[i][t]));
  }
  if (rowP) {
    for (int idx = tid; idx < BK * BK; idx += NT) {
      const int t = idx / BK, j = idx % BK;
      rowP[t * ldT + p0 + j] = Op::from_s(s[t][j]);
    }
  }
}

template <class Op>
__global__ void __launch_bounds__(P1W_THREADS) fw_phase1_w128(typename Op::elem *__restrict__ D, Layout L, int64_t n,
                                                              int64_t p0, uint32_t *__restrict__ colT, int64_t ldT,
                                                              typename Op::elem *rowP) {
  extern __shared__ __align__(16) uint8_t p1w_raw[];
  pdl_trigger();
  pdl_wait();
  phase1_body_w128<Op>(D, L, n, p0, colT, ldT, *reinterpret_cast<P1Smem<Op, 128> *>(p1w_raw), threadIdx.x, rowP);
}

// shared-memory loaders: load_As_colT, load_Bs_rows, load_As_transposed (fw_device.cuh)

// ---------------------------------------------------------------- Phase 2
// Row-panel CTAs: tile BK x 128 words; column-panel CTAs: tile
// (128 * EPW) x (BK / EPW) words.  Both use 128 threads.
// 8 x 4 words per thread (twice the warps of 8 x 8): Phase 2 has little work
// per round and is latency-bound.
// Chunks are 128 elements wide (row panel) and 128 rows tall (column panel)
// for every element type, so a round has as many Phase-2 CTAs for packed
// 16-bit as for int32.
template <class Op, int BK>
struct P2Cfg {
  static constexpr int TN = 4;
  static constexpr int ROW_BM = BK, ROW_BNW = 128 / Op::EPW;
  static constexpr int COL_BM = 128, COL_BNW = BK / Op::EPW;
  static constexpr int THREADS = (BK / 8) * (ROW_BNW / TN);
  static_assert(TileMap<ROW_BM, ROW_BNW, TN>::THREADS == THREADS, "row tile");
  static_assert(TileMap<COL_BM, COL_BNW, TN>::THREADS == THREADS, "col tile");
  static constexpr int ROW_SMEM = (BK * ROW_BM + BK * ROW_BNW) * 4;
  static constexpr int COL_SMEM = (BK * COL_BM + BK * COL_BNW) * 4;
  static constexpr int SMEM = ROW_SMEM > COL_SMEM ? ROW_SMEM : COL_SMEM;
};

// The first nrow_ctas CTAs take row-panel chunks row_chunk0, row_chunk0 + 1,
// ...; the rest take column-panel chunks 0, 1, ....  sym != 0: symmetric
// mode (see p2_row_task / p2_col_task).
template <class Op, int BK>
__global__ void __launch_bounds__(P2Cfg<Op, BK>::THREADS)
    fw_phase2(typename Op::elem *__restrict__ D, Layout L, int64_t n, int64_t p0, int64_t p1,
              uint32_t *__restrict__ colT, int64_t ldT, int nrow_ctas, int vec, int row_chunk0, int sym,
              SymPanel<Op> sp) {
  using C = P2Cfg<Op, BK>;
  extern __shared__ __align__(16) uint32_t smem[];
  const SymPanel<Op> *spp = sym ? &sp : nullptr;
  pdl_trigger();
  pdl_wait();
  if ((int)blockIdx.x < nrow_ctas)
    p2_row_task<Op, BK, C::ROW_BNW, C::THREADS, false, C::TN>(
        D, L, n, p0, p1, colT, ldT, (int64_t)(row_chunk0 + (int)blockIdx.x) * C::ROW_BNW * Op::EPW, vec, smem,
        threadIdx.x, spp);
  else
    p2_col_task<Op, BK, C::COL_BM, C::THREADS, false, C::TN>(D, L, n, p0, p1, colT, ldT,
                                                             (int64_t)(blockIdx.x - nrow_ctas) * C::COL_BM, vec,
                                                             smem, threadIdx.x, spp);
}

// Symmetric mode, after Phase 2: for x < p0 (the column-panel part of the
// symmetric panel, written by the column-panel CTAs as colT words), copy
// row t of colT to the element panel rowP[t][x] (packed 16-bit only) and to
// the row panel's lower-triangle elements D[p0 + t][x] inside the diagonal
// tile band x >= band_start (the only ones that Phase-3 tiles read).
// Coalesced: one block row per panel row t.
template <class Op>
__global__ void panel_finalize(typename Op::elem *__restrict__ D, Layout L, int64_t n, int64_t p0,
                               const uint32_t *__restrict__ colT, int64_t ldT, typename Op::elem *__restrict__ rowP,
                               int64_t band_start) {
  pdl_trigger();
  pdl_wait();
  const int t = blockIdx.y;
  const int64_t row = p0 + t;
  const int64_t x0 = rowP ? 0 : band_start;  // without an element panel only the band is needed
  for (int64_t x = x0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < p0; x += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t w = colT[(int64_t)t * ldT + x];
    const typename Op::elem e = bits_elem<Op>(Op::EPW == 2 ? (w & 0xFFFFu) : w);
    if (rowP) rowP[(int64_t)t * ldT + x] = e;
    if (x >= band_start && row < n) D[L.off(row, x)] = e;
  }
}

// Phase 1 kernel with the optional element panel (symmetric mode).
template <class Op, int BK>
__global__ void __launch_bounds__(P1_THREADS) fw_phase1_sym(typename Op::elem *__restrict__ D, Layout L, int64_t n,
                                                            int64_t p0, uint32_t *__restrict__ colT, int64_t ldT,
                                                            typename Op::elem *rowP) {
  __shared__ P1Smem<Op, BK> s;
  pdl_trigger();
  pdl_wait();
  phase1_body<Op, BK, P1_THREADS, false>(D, L, n, p0, colT, ldT, s, threadIdx.x, rowP);
}

// ---------------------------------------------------------------- symmetry
// D[r][c] = D[c][r] for every r > c (the lower triangle from the upper), by
// 32 x 32 blocks through shared memory; block (R, C) with R >= C.
template <class Op>
__global__ void mirror_kernel(typename Op::elem *__restrict__ D, int64_t n, int64_t ld, const int *sym_flag) {
  __shared__ typename Op::elem tile[32][33];
  if (sym_flag && *sym_flag != 0) return;  // the device found D not symmetric: the general path ran
  const int64_t R = blockIdx.y, Cb = blockIdx.x;
  if (R < Cb) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  // read block (Cb, R) of the upper triangle: rows Cb*32.., columns R*32..
  for (int k = ty; k < 32; k += 8) {
    const int64_t r = Cb * 32 + k, c = R * 32 + tx;
    if (r < n && c < n) tile[k][tx] = D[r * ld + c];
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int64_t r = R * 32 + k, c = Cb * 32 + tx;  // target (r, c) = source (c, r)
    if (r < n && c < n && r > c) D[r * ld + c] = tile[tx][k];
  }
}

// flag |= 1 when some D[r][c] != D[c][r] (compared bitwise), same blocking.
template <class Op>
__global__ void symmetry_check_kernel(const typename Op::elem *__restrict__ D, int64_t n, int64_t ld, int *flag) {
  __shared__ typename Op::elem tile[32][33];
  const int64_t R = blockIdx.y, Cb = blockIdx.x;
  if (R < Cb) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int k = ty; k < 32; k += 8) {
    const int64_t r = Cb * 32 + k, c = R * 32 + tx;
    if (r < n && c < n) tile[k][tx] = D[r * ld + c];
  }
  __syncthreads();
  int bad = 0;
  for (int k = ty; k < 32; k += 8) {
    const int64_t r = R * 32 + k, c = Cb * 32 + tx;
    if (r < n && c < n && elem_bits<Op>(D[r * ld + c]) != elem_bits<Op>(tile[tx][k])) bad = 1;
  }
  if (__syncthreads_or(bad) && tx == 0 && ty == 0) atomicOr(flag, 1);
}

// ---------------------------------------------------------------- Phase 3
template <class Op>
struct P3Cfg {
  static constexpr int BM = 128, BNW = 128;
  static constexpr int THREADS = TileMap<BM, BNW>::THREADS;  // 256
};

template <class Op, int BK>
__global__ void __launch_bounds__(256, 2) fw_phase3(typename Op::elem *__restrict__ D, int64_t ld, int64_t n,
                                                    int64_t p0, int64_t p1, const uint32_t *__restrict__ colT,
                                                    int64_t ldT, int vec, const typename Op::elem *symB) {
  extern __shared__ __align__(16) uint32_t smem[];
  // symmetric mode (symB != nullptr): tiles below the band are skipped and B is the panel
  if (symB && (int)blockIdx.x < (int)blockIdx.y / Op::EPW) return;
  p3_task<Op, BK, false>(D, ld, n, p0, p1, colT, ldT, (int64_t)blockIdx.y * P3Cfg<Op>::BM,
                         (int64_t)blockIdx.x * P3Cfg<Op>::BNW * Op::EPW, vec, smem, threadIdx.x, symB);
}

// ---------------------------------------------------------------- Phase 3, persistent + TMA
// One CTA per SM walks a contiguous range of output tiles (row-major over the
// tile grid).  Shared memory holds two stages of {A tile 64 x 128 words, B tile
// 64 x 128 words} and one C tile (128 x 128 words): while the add-min loop
// runs on tile i, TMA brings tile i+1's operands into the other stage and its
// C block into the C buffer; results go back to D from registers.
//   A = colT[0..64)[row0 .. row0+128)   (column panel, transposed, words)
//   B = D[p0 .. p0+64)[col0 ..)         (row panel)
//   C = D[row0 .. row0+128)[col0 ..)
// TMA fills out-of-range elements with zeros.  That only reaches (a) C and B
// columns >= n, which feed output columns that are never stored, (b) C rows
// >= n, never stored, and (c) B rows >= n of the last, partial round, which
// meet A words colT[t][.] that Phases 1 and 2 set to INF for those t, so the
// sum is INF and never wins.
constexpr int P3T_C_BYTES = 128 * 128 * 4;
constexpr uint32_t P3T_WAIT_LIMIT = 1u << 26;
constexpr uint32_t P3T_SLEEP_NS = 256;  // longest sleep of one wait try in the persistent kernels' producers
// A stage holds KS k-steps of the A and B tiles: the whole round for round
// widths up to 64, half of it for width 128 (whose tiles then take two stages
// each and store their C block once per 128 k-steps).
template <int BK>
struct P3T {
  static constexpr int KS = BK < 64 ? BK : 64;
  static constexpr int NSPLIT = BK / KS;  // stages per tile
  static_assert(NSPLIT == 1 || NSPLIT == 2, "round width 32, 64 or 128");
  static constexpr int STAGE_BYTES = 2 * KS * 128 * 4;  // A + B tiles
  static constexpr int SMEM = 2 * STAGE_BYTES + P3T_C_BYTES + 1024;
};

// TN = 8: 256 threads with 8 x 8 words each; TN = 4: 512 threads with 8 x 4
// words each (twice the warps per SM to hide instruction latency).
// Symmetric mode (sym = 1): only tiles (ty, tx) with tx >= ty / EPW -- the
// tiles that touch the upper triangle -- are processed, in row-major order,
// and B comes from the symmetric panel (mapB over the panel buffer) instead of
// D's row panel.  Number of processed tiles before tile row ty:
// ty * tiles_x - sum_{y < ty} floor(y / EPW).
__device__ __forceinline__ long long sym_prefix(int ty, int tiles_x, int epw) {
  long long f;
  if (epw == 1) {
    f = (long long)ty * (ty - 1) / 2;
  } else {
    const long long a = ty / 2;
    f = (ty % 2 == 0) ? a * (a - 1) : a * a;
  }
  return (long long)ty * tiles_x - f;
}

template <class Op, int BK, int TN>
__global__ void __launch_bounds__(TileMap<128, 128, TN>::THREADS, 1)
    fw_phase3_tma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  const __grid_constant__ CUtensorMap mapC, typename Op::elem *__restrict__ D, int64_t ld, int64_t n,
                  int64_t p0, int64_t p1, int tiles_x, int tiles_total, int *err, int sym, int tiles_y) {
  constexpr int BM = 128, BNW = 128;
  constexpr int P3T_STAGE_BYTES = P3T<BK>::STAGE_BYTES;
  using Map = TileMap<BM, BNW, TN>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar_ab[2];
  __shared__ __align__(8) uint64_t bar_c;
  __shared__ int abort_flag;
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // stage s: A at base + s * STAGE, B right after it; C after both stages
  auto stA = [&](int s) { return reinterpret_cast<uint32_t *>(base + s * P3T_STAGE_BYTES); };
  auto stB = [&](int s) { return reinterpret_cast<uint32_t *>(base + s * P3T_STAGE_BYTES) + BK * BM; };
  uint32_t *Cs = reinterpret_cast<uint32_t *>(base + 2 * P3T_STAGE_BYTES);

  const int tid = threadIdx.x;
  const int tx = tid % Map::TX, ty = tid / Map::TX;
  const int per = tiles_total / (int)gridDim.x, extra = tiles_total % (int)gridDim.x;
  const int t_begin = (int)blockIdx.x * per + min((int)blockIdx.x, extra);
  const int t_end = t_begin + per + ((int)blockIdx.x < extra ? 1 : 0);
  if (t_begin >= t_end) return;

  if (tid == 0) {
    mbar_init(&bar_ab[0], 1);
    mbar_init(&bar_ab[1], 1);
    mbar_init(&bar_c, 1);
    fence_barrier_init();
    prefetch_tensormap(&mapA);
    prefetch_tensormap(&mapB);
    prefetch_tensormap(&mapC);
    abort_flag = 0;
  }
  __syncthreads();

  // tile coordinates advance incrementally (row-major over the tile grid)
  int cur_ty, cur_tx;
  if (!sym) {
    cur_ty = t_begin / tiles_x;
    cur_tx = t_begin % tiles_x;
  } else {
    int lo = 0, hi = tiles_y - 1;  // last tile row whose prefix <= t_begin
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sym_prefix(mid, tiles_x, Op::EPW) <= t_begin) lo = mid;
      else hi = mid - 1;
    }
    cur_ty = lo;
    cur_tx = lo / Op::EPW + (int)(t_begin - sym_prefix(lo, tiles_x, Op::EPW));
  }
  auto issue_ab = [&](int ty_, int tx_, int s) {
    mbar_arrive_expect_tx(&bar_ab[s], P3T_STAGE_BYTES);
    tma_load_2d(stA(s), &mapA, &bar_ab[s], ty_ * BM, 0);
    tma_load_2d(stB(s), &mapB, &bar_ab[s], tx_ * BNW * Op::EPW, sym ? 0 : (int)p0);
  };
  auto issue_c = [&](int ty_, int tx_) {
    mbar_arrive_expect_tx(&bar_c, P3T_C_BYTES);
    tma_load_2d(Cs, &mapC, &bar_c, tx_ * BNW * Op::EPW, ty_ * BM);
  };
  if (tid == 0) {
    issue_ab(cur_ty, cur_tx, 0);
    issue_c(cur_ty, cur_tx);
  }
  // parity of the next completion of bar_c (bit 0) and bar_ab[s] (bit 1 + s);
  // `pend` has the same bits set while a copy on that barrier is in flight
  uint32_t par = 0u, pend = 1u | 2u;
  uint32_t acc[8][TN];
  for (int t = t_begin; t < t_end; ++t) {
    const int s = (t - t_begin) & 1;
    const int nxt_ty = (cur_tx + 1 == tiles_x) ? cur_ty + 1 : cur_ty;
    const int nxt_tx = (cur_tx + 1 == tiles_x) ? (sym ? nxt_ty / Op::EPW : 0) : cur_tx + 1;
    if (!mbar_wait_bounded(&bar_c, par & 1u, P3T_WAIT_LIMIT)) abort_flag = 1;
    par ^= 1u;
    pend &= ~1u;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int h = 0; h < Map::NH; ++h) {
        const uint4 v = *reinterpret_cast<const uint4 *>(Cs + Map::row(ty, r) * BNW + Map::wcol(tx, h));
        acc[r][4 * h + 0] = v.x;
        acc[r][4 * h + 1] = v.y;
        acc[r][4 * h + 2] = v.z;
        acc[r][4 * h + 3] = v.w;
      }
    }
    __syncthreads();  // C buffer read by all; stage s^1 no longer read (tile t-1 done)
    if (abort_flag) break;
    if (t + 1 < t_end) {
      if (tid == 0) {
        issue_c(nxt_ty, nxt_tx);
        issue_ab(nxt_ty, nxt_tx, s ^ 1);
      }
      pend |= 1u | (2u << (s ^ 1));
    }
    const uint32_t bit = 2u << s;
    if (!mbar_wait_bounded(&bar_ab[s], (par & bit) ? 1u : 0u, P3T_WAIT_LIMIT)) abort_flag = 1;
    par ^= bit;
    pend &= ~bit;
    __syncwarp();
    if (abort_flag) break;
    tile_minplus<Op, BM, BNW, BK, TN>(stA(s), stB(s), acc, ty, tx);
    const int64_t r0 = (int64_t)cur_ty * BM, c0 = (int64_t)cur_tx * BNW * Op::EPW;
    const bool interior = r0 + BM <= n && c0 + BNW * Op::EPW <= n && (r0 + BM <= p0 || r0 >= p1) &&
                          (c0 + BNW * Op::EPW <= p0 || c0 >= p1);
    if (interior)
      store_acc_interior<Op, BM, BNW, TN>(D, ld, r0, c0, acc, ty, tx);
    else
      store_acc<Op, BM, BNW, TN>(D, ld, n, n, r0, c0, p0, p1, p0, p1, true, acc, ty, tx);
    cur_tx = nxt_tx;
    cur_ty = nxt_ty;
  }
  if (abort_flag && tid == 0) {
    // a wait gave up: wait (bounded) for this CTA's copies still in flight
    // before the CTA's shared memory is released
    if (pend & 1u) mbar_wait_bounded(&bar_c, par & 1u, P3T_WAIT_LIMIT);
    for (int st = 0; st < 2; ++st)
      if (pend & (2u << st)) mbar_wait_bounded(&bar_ab[st], (par & (2u << st)) ? 1u : 0u, P3T_WAIT_LIMIT);
  }
  if (abort_flag && tid == 0) atomicOr(err, 4);
}

// Phase 3, warp-specialized persistent kernel: 8 consumer warps (8 x 8 words
// each, one 128-row x 128-word tile per CTA at a time) and one producer warp
// that moves all data with TMA.  The consumers never wait on each other:
// full/empty mbarriers hand the two A/B stages back and forth, and the
// accumulators start at INF, so C is needed only at the end of the tile:
//   RED (int32 and fp32): the consumers write acc into the C buffer and the
//     producer applies it with a TMA min-reduction, D = min(D, acc), carried
//     out in L2.  C is never loaded.  fp32 distances are non-negative floats
//     (ingest rejects negatives and NaN and stores -0.0 as +0.0) or +inf,
//     whose bit patterns order like the values under a signed int32 compare,
//     so fp32 tiles reduce through an int32 tensor map over the same bytes.
//     Every tile is reduced, the panel rows and columns included: there the
//     int32 update reproduces the current values exactly (after Phase 2 the
//     row panel R' = min(R, D_kk (x) R) with D_kk closed, so D_kk (x) R' >= R';
//     likewise for the column panel and D_kk itself), so other CTAs may read
//     the row panel while it is rewritten.  In fp32 a rounded sum may come out
//     one unit in the last place lower there: still the rounded length of a
//     real path, so readers see either value and the result stays within
//     the rounding tolerance.
//   !RED (packed 16-bit; no 16-bit-lane min reduction exists for TMA): the
//     producer loads C by TMA during the tile; the consumers merge it (min)
//     at the end; interior tiles go back through
//     the C buffer and a TMA store, edge tiles (panel rows or columns, ragged
//     edge) by masked stores that leave the panels untouched.
// Round width 128 (P3T<128>::NSPLIT = 2): each tile takes two 64-step stages
// in a row -- the producer streams (tile, k-half) items, item j in stage
// j & 1 -- and the consumers run the epilogue once per tile, after both.
// Symmetric mode and the tile order are as in fw_phase3_tma.  Every wait is
// bounded; a CTA that gives up waits (bounded) for its copies in flight and
// ORs 4 into *err.
constexpr int P3W_THREADS = 9 * 32;
// Element types whose Phase-3 tiles leave by the int32 TMA min-reduction.
template <class Op>
constexpr bool kRedOp = Op::DTYPE != 1;

// int32 results leave by a TMA min-reduction over a tensor map that ends at
// n4 = n rounded down to 4 elements (16 bytes): at the tensor's x edge the
// reduction writes whole 16-byte units, so the last n - n4 columns are merged
// here instead, element by element, by the threads that own them (the tile's
// other elements are never touched by this).
__device__ __forceinline__ int64_t red_cols(int64_t n) { return n & ~(int64_t)3; }

template <int BM, int BNW, int TN>
__device__ __forceinline__ void red_tail_store(int32_t *D, int64_t ld, int64_t nrows, int64_t ncols, int64_t r0,
                                               int64_t c0, const uint32_t (&acc)[8][TN], int ty, int tx) {
  using Map = TileMap<BM, BNW, TN>;
  const int64_t n4 = red_cols(ncols);
#pragma unroll
  for (int h = 0; h < Map::NH; ++h) {
    const int64_t cw = c0 + Map::wcol(tx, h);
    if (cw + 4 <= n4 || cw >= ncols) continue;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int64_t row = r0 + Map::row(ty, r);
      if (row >= nrows) continue;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t c = cw + e;
        if (c >= n4 && c < ncols) {
          int32_t *p = D + row * ld + c;
          *p = (int32_t)OpI32::addmin(acc[r][4 * h + e], 0u, (uint32_t)*p);
        }
      }
    }
  }
}

template <class Op, int BK, bool RED>
__global__ void __launch_bounds__(P3W_THREADS, 1)
    fw_phase3_ws(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 const __grid_constant__ CUtensorMap mapC, typename Op::elem *__restrict__ D, Layout L, int64_t n,
                 int64_t p0, int64_t p1, int tiles_x, int tiles_total, int *err, int sym, int tiles_y) {
  constexpr int BM = 128, BNW = 128, TN = 8;
  using Map = TileMap<BM, BNW, TN>;
  constexpr int NCW = Map::THREADS / 32;  // consumer warps
  static_assert(Map::THREADS + 32 == P3W_THREADS, "one producer warp after the consumers");
  constexpr int STAGE = P3T<BK>::STAGE_BYTES;
  constexpr int KS = P3T<BK>::KS, NSPLIT = P3T<BK>::NSPLIT;  // k-steps per stage, stages per tile
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_ab[2], empty_ab[2], full_c, cdone, cfree;
  __shared__ int abort_flag;
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  auto stA = [&](int s) { return reinterpret_cast<uint32_t *>(base + s * STAGE); };
  auto stB = [&](int s) { return reinterpret_cast<uint32_t *>(base + s * STAGE) + KS * BM; };
  uint32_t *Cs = reinterpret_cast<uint32_t *>(base + 2 * STAGE);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int per = tiles_total / (int)gridDim.x, extra = tiles_total % (int)gridDim.x;
  const int t_begin = (int)blockIdx.x * per + min((int)blockIdx.x, extra);
  const int t_end = t_begin + per + ((int)blockIdx.x < extra ? 1 : 0);
  pdl_trigger();
  if (t_begin >= t_end) return;
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full_ab[i], 1);
      mbar_init(&empty_ab[i], NCW);
    }
    mbar_init(&full_c, 1);
    mbar_init(&cdone, NCW);
    mbar_init(&cfree, 1);
    fence_barrier_init();
    prefetch_tensormap(&mapA);
    prefetch_tensormap(&mapB);
    prefetch_tensormap(&mapC);
    abort_flag = 0;
  }
  __syncthreads();
  pdl_wait();  // the round's panels (previous launches) are complete from here on

  // first tile of this CTA and the row-major step over the (symmetric) tile set
  int ty0, tx0;
  if (!sym) {
    ty0 = t_begin / tiles_x;
    tx0 = t_begin % tiles_x;
  } else {
    int lo = 0, hi = tiles_y - 1;  // last tile row whose prefix <= t_begin
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sym_prefix(mid, tiles_x, Op::EPW) <= t_begin) lo = mid;
      else hi = mid - 1;
    }
    ty0 = lo;
    tx0 = lo / Op::EPW + (int)(t_begin - sym_prefix(lo, tiles_x, Op::EPW));
  }
  auto step = [&](int &ty_, int &tx_) {
    if (++tx_ == tiles_x) {
      ++ty_;
      tx_ = sym ? ty_ / Op::EPW : 0;
    }
  };
  auto interior_of = [&](int64_t r0, int64_t c0) {
    return r0 + BM <= n && c0 + BNW * Op::EPW <= n && (r0 + BM <= p0 || r0 >= p1) &&
           (c0 + BNW * Op::EPW <= p0 || c0 >= p1);
  };
  // TMA coordinates of tile (ty, tx) in the storage of D (the rectangle of the
  // upper-triangular layout, or D itself); the reduction map of a dense D ends
  // at red_cols(n), that of the upper-triangular rectangle covers its padding
  auto cxy = [&](int ty_, int tx_, int &x, int &y) {
    int64_t pr, pc;
    L.phys((int64_t)ty_ * BM, (int64_t)tx_ * BNW * Op::EPW, pr, pc);
    x = (int)pc;
    y = (int)pr;
  };
  const int64_t ncr = L.tri() ? INT64_MAX : red_cols(n);

  if (warp == NCW) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int n_ab[2] = {0, 0}, n_c = 0;
      bool ok = true;
      // k-steps [h * KS, (h + 1) * KS) of tile (ty_, tx_) into stage s
      auto issue_ab = [&](int ty_, int tx_, int h, int s) {
        mbar_arrive_expect_tx(&full_ab[s], STAGE);
        tma_load_2d(stA(s), &mapA, &full_ab[s], ty_ * BM, h * KS);
        tma_load_2d(stB(s), &mapB, &full_ab[s], tx_ * BNW * Op::EPW, (sym ? 0 : (int)p0) + h * KS);
        if (s == 0) ++n_ab[0];
        else ++n_ab[1];
      };
      auto issue_c = [&](int ty_, int tx_) {
        int x, y;
        cxy(ty_, tx_, x, y);
        mbar_arrive_expect_tx(&full_c, P3T_C_BYTES);
        tma_load_2d(Cs, &mapC, &full_c, x, y);
        ++n_c;
      };
      // the item stream: (tile, k-part h) in tile order, item j in stage j & 1
      const int n_items = (t_end - t_begin) * NSPLIT;
      int aty = ty0, atx = tx0, ah = 0;  // next item to load
      auto next_item = [&]() {
        if (++ah == NSPLIT) {
          ah = 0;
          step(aty, atx);
        }
      };
      int cty = ty0, ctx = tx0;  // tile whose result is written next
      issue_ab(aty, atx, ah, 0);
      next_item();
      if (n_items > 1) {
        issue_ab(aty, atx, ah, 1);
        next_item();
      }
      if (!RED) issue_c(cty, ctx);
      for (int t = t_begin; t < t_end; ++t) {
        const int i = t - t_begin;
        for (int h = 0; h < NSPLIT; ++h) {
          const int j = i * NSPLIT + h, s = j & 1;
          if (!mbar_wait_sleep_bounded(&empty_ab[s], (uint32_t)(j >> 1) & 1u, P3T_WAIT_LIMIT, P3T_SLEEP_NS)) {
            ok = false;
            break;
          }
          if (j + 2 < n_items) {
            issue_ab(aty, atx, ah, s);
            next_item();
          }
        }
        if (!ok) break;
        if (!mbar_wait_sleep_bounded(&cdone, (uint32_t)i & 1u, P3T_WAIT_LIMIT, P3T_SLEEP_NS)) {
          ok = false;
          break;
        }
        const int r0 = cty * BM, c0 = ctx * BNW * Op::EPW;
        int cx, cy;
        cxy(cty, ctx, cx, cy);
        if (RED) {
          if (c0 < ncr) {  // a dense D's mapC ends at red_cols(n) in this mode
            tma_reduce_min_2d(&mapC, Cs, cx, cy);
            bulk_commit();
            bulk_wait_read_all();
          }
          mbar_arrive(&cfree);
        } else if (interior_of(r0, c0)) {
          tma_store_2d(&mapC, Cs, cx, cy);
          bulk_commit();
          bulk_wait_read_all();
        }
        step(cty, ctx);
        if (!RED && t + 1 < t_end) issue_c(cty, ctx);
      }
      bulk_wait_all();
      if (!ok) {
        abort_flag = 1;
        for (int st = 0; st < 2; ++st)
          if (n_ab[st] > 0) mbar_wait_bounded(&full_ab[st], (uint32_t)(n_ab[st] - 1) & 1u, P3T_WAIT_LIMIT);
        if (n_c > 0) mbar_wait_bounded(&full_c, (uint32_t)(n_c - 1) & 1u, P3T_WAIT_LIMIT);
      }
    }
  } else {
    // ------------------------------------------------------------ consumers
    const int tx = tid % Map::TX, ty = tid / Map::TX;
    int cty = ty0, ctx = tx0;
    uint32_t acc[8][TN];
    for (int t = t_begin; t < t_end; ++t) {
      const int i = t - t_begin;
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = Op::INF_WORD;
      bool bad = false;
#pragma unroll 1
      for (int h = 0; h < NSPLIT; ++h) {  // the tile's k-parts, one stage each (one copy of the k-loop)
        const int j = i * NSPLIT + h, s = j & 1;
        bad = !mbar_wait_bounded(&full_ab[s], (uint32_t)(j >> 1) & 1u, P3T_WAIT_LIMIT);
        if (__any_sync(0xffffffffu, bad)) break;
        tile_minplus<Op, BM, BNW, KS, TN>(stA(s), stB(s), acc, ty, tx);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_ab[s]);
      }
      if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) abort_flag = 1;
        break;
      }
      const int64_t r0 = (int64_t)cty * BM, c0 = (int64_t)ctx * BNW * Op::EPW;
      if (RED) {
        // the previous tile's reduction has finished reading the C buffer
        bad = i > 0 && !mbar_wait_bounded(&cfree, (uint32_t)(i - 1) & 1u, P3T_WAIT_LIMIT);
        if (__any_sync(0xffffffffu, bad)) {
          if (lane == 0) abort_flag = 1;
          break;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int h = 0; h < Map::NH; ++h)
            *reinterpret_cast<uint4 *>(Cs + Map::row(ty, r) * BNW + Map::wcol(tx, h)) =
                make_uint4(acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
        fence_proxy_async_smem();
        if constexpr (Op::DTYPE != 1)
          if (!L.tri() && c0 + BNW > red_cols(n) && c0 < n)
            red_tail_store<BM, BNW, TN>(reinterpret_cast<int32_t *>(D), L.ld, n, n, r0, c0, acc, ty, tx);
      } else {
        bad = !mbar_wait_bounded(&full_c, (uint32_t)i & 1u, P3T_WAIT_LIMIT);
        if (__any_sync(0xffffffffu, bad)) {
          if (lane == 0) abort_flag = 1;
          break;
        }
        const bool interior = interior_of(r0, c0);
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int h = 0; h < Map::NH; ++h) {
            uint4 *cp = reinterpret_cast<uint4 *>(Cs + Map::row(ty, r) * BNW + Map::wcol(tx, h));
            const uint4 v = *cp;
            acc[r][4 * h + 0] = Op::addmin(acc[r][4 * h + 0], 0u, v.x);
            acc[r][4 * h + 1] = Op::addmin(acc[r][4 * h + 1], 0u, v.y);
            acc[r][4 * h + 2] = Op::addmin(acc[r][4 * h + 2], 0u, v.z);
            acc[r][4 * h + 3] = Op::addmin(acc[r][4 * h + 3], 0u, v.w);
            if (interior)
              *cp = make_uint4(acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
          }
        if (interior) fence_proxy_async_smem();
        else store_acc<Op, BM, BNW, TN>(D, L, n, n, r0, c0, p0, p1, p0, p1, true, acc, ty, tx);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&cdone);
      step(cty, ctx);
    }
  }
  __syncthreads();
  if (abort_flag && tid == 0) atomicOr(err, 4);
}

// ---------------------------------------------------------------- lookahead rounds
// Pieces of the next-round tasks that the Phase-3 kernel runs on its consumer
// warps (fw_solve_ws): Phase 1, Phase-2 chunks shaped for 256 threads, and the
// symmetric-mode panel publication.  A task runs on the 256 consumer threads
// with the bounded group barrier below, in the C buffer (int32) or in the two
// stage buffers (the producer takes no new item meanwhile).
// Phase-2 shape for 256 threads (the consumer warps).
template <class Op, int BK>
struct LaP2 {
  static constexpr int TN = 4;
  static constexpr int ROW_BNW = 8192 / BK;             // 64 x 128 words for BK = 64
  static constexpr int COL_BNW = BK / Op::EPW;
  static constexpr int COL_BM = 8192 * Op::EPW / BK;    // 128 rows (256 for packed 16-bit) for BK = 64
  static_assert(TileMap<BK, ROW_BNW, TN>::THREADS == 256, "row chunk");
  static_assert(TileMap<COL_BM, COL_BNW, TN>::THREADS == 256, "column chunk");
  static constexpr int SMEM = (BK * BK + BK * ROW_BNW) > (BK * COL_BM + BK * COL_BNW) ? (BK * BK + BK * ROW_BNW) * 4
                                                                                     : (BK * COL_BM + BK * COL_BNW) * 4;
};
// Lookahead rounds are built for round width 64 (the tasks of width 32 do not
// fit the 256-thread chunk shapes and the two 32 KB stage buffers).
template <int BK>
constexpr bool kLookaheadWidth = BK == 64;

constexpr int LA_TILE = 0, LA_P1 = 1, LA_P2 = 2, LA_FIN = 3, LA_END = -1, LA_SKIP = 5;
constexpr int LA_FIN_ROWS = 8;  // panel rows per publication task (packed 16-bit element panel)

// Consumer-warp barrier of the next-round tasks: an mbarrier that each of the 8
// consumer warps arrives on once per sync, with a bounded wait.  Unlike a
// hardware named barrier it cannot hang when a warp has left after a timeout:
// the others give up, set la_grp_abort, and every later sync returns at once
// (the launch then reports the timeout).
__shared__ __align__(8) uint64_t la_grp_bar;
__shared__ uint32_t la_grp_par[8];  // phase parity of each consumer warp's next sync
__shared__ int la_grp_abort;

// A bounded mbarrier wait that also gives up once *a, or *b when given, is
// nonzero (read after every 32 failed tries, so a launch that is being aborted
// ends without waiting out the full limit).
__device__ __forceinline__ bool mbar_wait_or(uint64_t *bar, uint32_t parity, uint32_t limit, const int *a,
                                             const int *b) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 31) == 31 &&
        (*reinterpret_cast<const volatile int *>(a) || (b && *reinterpret_cast<const volatile int *>(b))))
      return false;
  }
  return false;
}

struct GroupBar {
  __device__ __forceinline__ static void sync() {
    __syncwarp();
    if (*reinterpret_cast<volatile int *>(&la_grp_abort)) return;
    const int w = threadIdx.x >> 5;
    const uint32_t par = la_grp_par[w];
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&la_grp_bar);
    const bool ok = mbar_wait_or(&la_grp_bar, par, P3T_WAIT_LIMIT, &la_grp_abort, nullptr);
    __syncwarp();
    if ((threadIdx.x & 31) == 0) la_grp_par[w] = par ^ 1u;
    if (!ok) la_grp_abort = 1;
    __syncwarp();
  }
};

template <class Op, int BK>
__device__ __noinline__ void la_task_p1(typename Op::elem *D, int64_t ld, int64_t n, int64_t p0, uint32_t *colT,
                                        int64_t ldT, typename Op::elem *rowP, uint32_t *smem, int tid) {
  auto &sm = *reinterpret_cast<P1Smem<Op, BK> *>(smem);
  phase1_body<Op, BK, 256, true, GroupBar>(D, ld, n, p0, colT, ldT, sm, tid, rowP);
}

template <class Op, int BK>
__device__ __noinline__ void la_task_p2(typename Op::elem *D, int64_t ld, int64_t n, int64_t p0, int64_t p1,
                                        uint32_t *colT, int64_t ldT, int idx, int n_row, int row_first, bool vec,
                                        SymPanel<Op> sp, bool sym, uint32_t *smem, int tid) {
  using F = LaP2<Op, BK>;
  const SymPanel<Op> *spp = sym ? &sp : nullptr;
  if (idx < n_row)
    p2_row_task<Op, BK, F::ROW_BNW, 256, true, F::TN, GroupBar>(
        D, ld, n, p0, p1, colT, ldT, (int64_t)(row_first + idx) * F::ROW_BNW * Op::EPW, vec, smem, tid, spp);
  else
    p2_col_task<Op, BK, F::COL_BM, 256, true, F::TN, GroupBar>(D, ld, n, p0, p1, colT, ldT,
                                                                   (int64_t)(idx - n_row) * F::COL_BM, vec, smem,
                                                                   tid, spp);
}

// Symmetric-mode publication (the panel_finalize pass) for panel rows [t0, t1):
// 16-byte panel loads, four per thread in flight (p0 and band_start are
// multiples of 4, and so is every x visited).
template <class Op>
__device__ __noinline__ void la_task_fin(typename Op::elem *D, int64_t ld, int64_t n, int64_t p0,
                                         const uint32_t *colT, int64_t ldT, typename Op::elem *rowP,
                                         int64_t band_start, int t0, int t1, int tid) {
  using E = typename Op::elem;
  constexpr int U = 4, STEP = 4 * 256;
  const int64_t x0 = rowP ? 0 : band_start;
  for (int t = t0; t < t1; ++t) {
    const int64_t row = p0 + t;
    const uint32_t *src = colT + (int64_t)t * ldT;
    for (int64_t xb = x0 + 4 * tid; xb < p0; xb += (int64_t)U * STEP) {
      uint4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t x = xb + (int64_t)u * STEP;
        v[u] = x < p0 ? __ldcg(reinterpret_cast<const uint4 *>(src + x)) : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t x = xb + (int64_t)u * STEP;
        if (x >= p0) continue;
        const uint32_t w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
        E e[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) e[j] = bits_elem<Op>(Op::EPW == 2 ? (w[j] & 0xFFFFu) : w[j]);
        if constexpr (Op::EPW == 2) {
          if (rowP)
            *reinterpret_cast<uint2 *>(rowP + (int64_t)t * ldT + x) =
                make_uint2((uint32_t)e[0] | ((uint32_t)e[1] << 16), (uint32_t)e[2] | ((uint32_t)e[3] << 16));
        }
        if (row < n && x + 4 > band_start) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (x + j >= band_start) D[row * ld + x + j] = e[j];
        }
      }
    }
  }
}

// ---------------------------------------------------------------- all rounds in one launch
// The lookahead scheme carried across the whole solve: one persistent launch
// takes work items from one device counter, so round k+1's tiles start while
// round k's last tiles finish, with no launch boundary between rounds.  Items
// come in blocks: block 0 = round 0's Phase 1 and Phase-2 chunks; block j >= 1
// = round j-1's Phase-3 tiles (first the priority tiles that round j's tasks
// read or write: tile row R' and tile column C' of round j's diagonal block)
// with round j's tasks inserted a few tile waves later (P1 two waves after the
// priority tiles, the Phase-2 chunks four more, the publication three more),
// padded to a common size (padding items are skipped).  Each item waits only for items
// with smaller ids:
//   tile of round k        <- every task of round k done (P1, P2 chunks,
//                             publication); packed 16-bit also the same tile
//                             of round k-1 written (its C is loaded, merged and
//                             stored, which must not overlap)
//   P1 of round j          <- round j-1's priority tiles written, and every
//                             tile of round j-2 written (those read the panel
//                             buffer that round j overwrites, and carry the last
//                             contributions the diagonal block needs)
//   P2 chunks of round j   <- P1 of round j
//   publication, round j   <- every P2 chunk of round j
// int32 and fp32 tiles of rounds k and k+1 may overlap on the same tile: both
// are TMA min-reductions, which commute; and a tile of round k may read a
// row-panel value that round k+1 has already lowered.  Every value is always a
// real path length no larger than the one the sequential order would hold at
// that point, so the int32 result is the same exact matrix.  In fp32 every
// value is the rounded length of a real path and, rounding being monotone, no
// larger than the sequential order's; the result is within the rounding
// tolerance of the exact one, and may differ from another run's in the last
// bit of an entry.
template <class Op>
struct SolvePlan {
  int64_t n, ld, ldT;
  int q, tiles_x, tiles_y, tiles_total, grid, sym, vec;
  int block, base1;  // items per block j >= 1 (padded), items of block 0
  uint32_t *colT[2];
  typename Op::elem *rowP[2];
  unsigned long long *items;  // work items taken (64-bit: blocks x block size can pass 2^31)
  int *cnt;          // 6 per round r: [0] priority tiles for round r, [1] P1(r), [2] P2(r), [3] all tasks of r,
                     // [4] tiles of round r written
  int *tile_round;   // packed 16-bit: rounds written per tile
};

// The plan of each mode ([0] general, [1] symmetric) and, when the host left
// the choice to the device, the symmetry flag (0 = symmetric) to pick it by.
// abort: a zeroed device word that a CTA sets when it gives up, so that the
// others stop at their next wait instead of timing out one by one.  gate
// (nullable): round 0's Phase 1 also waits for *gate >= 1 (a diagnostic of
// the bounded waits).  dep_spins: the limit of each wait on another item.
template <class Op>
struct SolvePlans {
  SolvePlan<Op> p[2];
  const int *sym_flag;
  int *abort;
  const int *gate;
  uint32_t dep_spins;
};

// Round j's tasks and the priority tiles (of round j-1) they depend on.
struct SolveRound {
  int64_t p0, p1, band_start, band_end;
  int R, C, row_x0, col_y1, n_prio, n_p2row, p2_row_first, n_p2col, n_fin;
  int b1, b2, b3, len_t, total;  // positions in block j, tile-stream length, items of block j
};

template <class Op, int BK>
__host__ __device__ inline SolveRound solve_round(int64_t n, int q, int tiles_x, int tiles_y, int tiles_total, int grid,
                                                  int sym, bool has_rowP, int j) {
  using F = LaP2<Op, BK>;
  SolveRound r{};
  r.p0 = (int64_t)j * BK;
  r.p1 = r.p0 + BK < n ? r.p0 + BK : n;
  if (j >= q) {  // the last block: the final round's tiles, no tasks
    r.len_t = tiles_total;
    r.total = tiles_total;
    r.R = -1;
    r.C = -1;
    r.b1 = r.b2 = r.b3 = tiles_total;
    return r;
  }
  const int E = Op::EPW;
  r.R = (int)(r.p0 / 128);
  r.C = (int)(r.p0 / (128 * E));
  r.row_x0 = sym ? r.C : 0;
  r.col_y1 = sym ? (r.C * E + E < tiles_y ? r.C * E + E : tiles_y) : tiles_y;
  r.n_prio = j == 0 ? 0 : (tiles_x - r.row_x0) + (r.col_y1 - (r.R < r.col_y1 ? 1 : 0));
  const int nrow = (int)((n + F::ROW_BNW * E - 1) / (F::ROW_BNW * E));
  const int ncol = (int)((n + F::COL_BM - 1) / F::COL_BM);
  if (sym) {
    r.p2_row_first = (int)(r.p1 / (F::ROW_BNW * E));
    r.n_p2row = nrow - r.p2_row_first > 0 ? nrow - r.p2_row_first : 0;
    r.n_p2col = (int)((r.p0 + F::COL_BM - 1) / F::COL_BM);
  } else {
    r.p2_row_first = 0;
    r.n_p2row = nrow;
    r.n_p2col = ncol;
  }
  r.band_start = (r.p0 / (128 * E)) * (128 * E);
  r.band_end = r.band_start + 128 * E;
  const int w = (int)(r.p1 - r.p0);
  r.n_fin = 0;
  if (sym && r.p0 > 0) r.n_fin = has_rowP ? (w + LA_FIN_ROWS - 1) / LA_FIN_ROWS : (r.p0 > r.band_start ? 1 : 0);
  if (j == 0) {  // block 0: round 0's tasks only
    r.len_t = 0;
    r.b1 = r.b2 = r.b3 = 0;
    r.total = 1 + r.n_p2row + r.n_p2col + r.n_fin;
    return r;
  }
  r.len_t = r.n_prio + tiles_total;
  r.b1 = r.n_prio + 2 * grid < r.len_t ? r.n_prio + 2 * grid : r.len_t;
  r.b2 = r.b1 + 4 * grid < r.len_t ? r.b1 + 4 * grid : r.len_t;
  r.b3 = r.b2 + 3 * grid < r.len_t ? r.b2 + 3 * grid : r.len_t;
  r.total = r.len_t + 1 + r.n_p2row + r.n_p2col + r.n_fin;
  return r;
}

template <class Op, int BK, bool RED>
__global__ void __launch_bounds__(P3W_THREADS, 1)
    fw_solve_ws(const __grid_constant__ CUtensorMap mapA0, const __grid_constant__ CUtensorMap mapA1,
                const __grid_constant__ CUtensorMap mapB0, const __grid_constant__ CUtensorMap mapB1,
                const __grid_constant__ CUtensorMap mapBg, const __grid_constant__ CUtensorMap mapC,
                typename Op::elem *__restrict__ D, int *err, const SolvePlans<Op> PP) {
  // mapB0/mapB1: B of symmetric mode (the element panel of each parity); mapBg: B of the general mode (D)
  const SolvePlan<Op> P = PP.p[PP.sym_flag ? (__ldcg(PP.sym_flag) == 0 ? 1 : 0) : 0];
  constexpr int BM = 128, BNW = 128, TN = 8;
  using Map = TileMap<BM, BNW, TN>;
  constexpr int NCW = Map::THREADS / 32;
  static_assert(Map::THREADS == 256 && Map::THREADS + 32 == P3W_THREADS, "8 consumer warps + producer");
  constexpr int STAGE = P3T<BK>::STAGE_BYTES;
  static_assert(LaP2<Op, BK>::SMEM <= 2 * STAGE && (int)sizeof(P1Smem<Op, BK>) <= 2 * STAGE, "task memory");
  constexpr bool TASK_IN_C = RED && LaP2<Op, BK>::SMEM <= P3T_C_BYTES && (int)sizeof(P1Smem<Op, BK>) <= P3T_C_BYTES;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_ab[2], empty_ab[2], full_c, cdone, cfree;
  __shared__ int slot_kind[2], slot_info[2], slot_round[2];
  __shared__ int abort_flag;
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  auto stA = [&](int s) { return reinterpret_cast<uint32_t *>(base + s * STAGE); };
  auto stB = [&](int s) { return reinterpret_cast<uint32_t *>(base + s * STAGE) + BK * BM; };
  uint32_t *Cs = reinterpret_cast<uint32_t *>(base + 2 * STAGE);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n = P.n, ld = P.ld;
  const bool has_rowP = P.rowP[0] != nullptr;
  auto cnt = [&](int r, int f) { return P.cnt + 6 * r + f; };
  auto vload = [](const int *p) { return *reinterpret_cast<const volatile int *>(p); };
  auto round_info = [&](int j) {
    return solve_round<Op, BK>(n, P.q, P.tiles_x, P.tiles_y, P.tiles_total, P.grid, P.sym, has_rowP, j);
  };
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full_ab[i], 1);
      mbar_init(&empty_ab[i], NCW);
    }
    mbar_init(&full_c, 1);
    mbar_init(&cdone, NCW);
    mbar_init(&cfree, 1);
    mbar_init(&la_grp_bar, NCW);
    for (int w = 0; w < NCW; ++w) la_grp_par[w] = 0;
    la_grp_abort = 0;
    fence_barrier_init();
    prefetch_tensormap(&mapA0);
    prefetch_tensormap(&mapA1);
    prefetch_tensormap(&mapB0);
    prefetch_tensormap(&mapB1);
    prefetch_tensormap(&mapBg);
    prefetch_tensormap(&mapC);
    abort_flag = 0;
  }
  __syncthreads();
  auto span = [&](int k, int64_t &p0, int64_t &p1) {
    p0 = (int64_t)k * BK;
    p1 = p0 + BK < n ? p0 + BK : n;
  };
  auto interior_of = [&](int k, int64_t r0, int64_t c0) {
    int64_t p0, p1;
    span(k, p0, p1);
    return r0 + BM <= n && c0 + BNW * Op::EPW <= n && (r0 + BM <= p0 || r0 >= p1) &&
           (c0 + BNW * Op::EPW <= p0 || c0 >= p1);
  };
  // a bounded wait for a counter, by one thread; false: gave up, or another CTA did
  auto wait_count = [&](const int *c, int target) {
    uint32_t spins = 0;
    while (vload(c) < target) {
      if (++spins > PP.dep_spins || ((spins & 31) == 0 && vload(PP.abort))) return false;
      __nanosleep(64);
    }
    __threadfence();
    return true;
  };
  // this CTA gives up: its other warps stop at their next wait, the other CTAs at theirs
  auto give_up = [&]() {
    la_grp_abort = 1;
    abort_flag = 1;
    *reinterpret_cast<volatile int *>(PP.abort) = 1;
  };

  if (warp == NCW) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      // The per-item bookkeeping stays cheap: this thread shares its SM
      // sub-partition's integer pipe with two consumer warps.  One CTA's items
      // only increase, so the round of the last block met, the block's first
      // item and the last tile row of the stream met are kept and reused.
      SolveRound cr{};
      int cr_j = -1;
      auto round_at = [&](int j) -> const SolveRound & {
        if (j != cr_j) {
          cr = round_info(j);
          cr_j = j;
        }
        return cr;
      };
      long long blk_lo = 0;  // first item of block blk_j, relative to base1
      int blk_j = 0;
      int sy = -1;  // tile row sy holds the stream positions [spre, snext)
      long long spre = 0, snext = 0;
      auto row_prefix = [&](int y) -> long long {
        return P.sym ? sym_prefix(y, P.tiles_x, Op::EPW) : (long long)y * P.tiles_x;
      };
      // tile-stream position -> packed tile, or -1 for a priority tile met again
      auto stream_tile = [&](const SolveRound &r, int j) -> int {
        int y, x;
        if (j < r.n_prio) {
          const int nr = P.tiles_x - r.row_x0;
          if (j < nr) {
            y = r.R;
            x = r.row_x0 + j;
          } else {
            y = j - nr;
            if (y >= r.R) ++y;
            x = r.C;
          }
          return (y << 16) | x;
        }
        const int idx = j - r.n_prio;
        if (sy < 0 || idx < spre || idx >= snext) {
          y = -1;
          if (sy >= 0 && idx >= snext)  // a few rows on
            for (int c = sy + 1; c < sy + 5 && c < P.tiles_y; ++c)
              if (idx < row_prefix(c + 1)) {
                y = c;
                break;
              }
          if (y < 0) {  // the last row whose first position is <= idx
            int lo = 0, hi = P.tiles_y - 1;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (row_prefix(mid) <= idx) lo = mid;
              else hi = mid - 1;
            }
            y = lo;
          }
          sy = y;
          spre = row_prefix(y);
          snext = row_prefix(y + 1);
        }
        y = sy;
        x = (P.sym ? sy / Op::EPW : 0) + (int)(idx - spre);
        const bool prio = r.n_prio > 0 && ((y == r.R && x >= r.row_x0) || (x == r.C && y < r.col_y1));
        return prio ? -1 : ((y << 16) | x);
      };
      // item -> kind, round (tiles: their round; tasks: the round they build), info
      auto decode = [&](long long item, int &kind, int &rnd, int &info) {
        if (item < P.base1) {
          const SolveRound &r0 = round_at(0);
          rnd = 0;
          if (item == 0) { kind = LA_P1; info = 0; }
          else if (item < 1 + r0.n_p2row + r0.n_p2col) { kind = LA_P2; info = (int)item - 1; }
          else { kind = LA_SKIP; info = 0; }
          return;
        }
        const long long rel = item - P.base1;
        if (blk_j > 0 && rel >= blk_lo + P.block && rel < blk_lo + 2 * (long long)P.block) {
          ++blk_j;
          blk_lo += P.block;
        } else if (blk_j == 0 || rel < blk_lo || rel >= blk_lo + P.block) {
          blk_j = 1 + (int)(rel / P.block);
          blk_lo = (long long)(blk_j - 1) * P.block;
        }
        const int j = blk_j, pos = (int)(rel - blk_lo);
        if (j > P.q) { kind = LA_END; rnd = P.q; info = 0; return; }
        const SolveRound &r = round_at(j);
        if (pos >= r.total) { kind = LA_SKIP; rnd = j; info = 0; return; }
        const int n_p2 = r.n_p2row + r.n_p2col;
        if (j < P.q) {
          const int o1 = r.b1, o2 = r.b2 + 1, o3 = r.b3 + 1 + n_p2;
          int t;
          if (pos < o1) t = pos;
          else if (pos == o1) { kind = LA_P1; rnd = j; info = 0; return; }
          else if (pos < o2) t = pos - 1;
          else if (pos < o2 + n_p2) { kind = LA_P2; rnd = j; info = pos - o2; return; }
          else if (pos < o3) t = pos - 1 - n_p2;
          else if (pos < o3 + r.n_fin) { kind = LA_FIN; rnd = j; info = pos - o3; return; }
          else t = pos - 1 - n_p2 - r.n_fin;
          const int pk = stream_tile(r, t);
          kind = pk < 0 ? LA_SKIP : LA_TILE;
          rnd = j - 1;
          info = pk;
        } else {
          kind = LA_TILE;
          rnd = j - 1;
          info = stream_tile(r, pos);
        }
      };
      // The producer never blocks on another item: a claimed tile whose round's
      // panels are not complete yet waits in the queue [issued, claimed) (slots
      // are issued strictly in order, as the stage barriers require), and so does
      // a C load whose tile has not been written by the previous round; both are
      // retried inside every wait below.  Blocking on them could wait for a tile
      // this producer has not published yet.
      int rk[4], rt[4], rr[4];  // kind, packed tile / task index and round of the last four slots
      int claimed = 0, issued = 0, hold = -1, c_next = 0;
      int n_ab[2] = {0, 0}, n_c = 0;
      int ready = -1;  // rounds up to this one have every task done
      bool stop = false, ok = true, cs_free = true;
      long long q0 = -1, q1 = -1;  // items taken and not yet used, in increasing order
      auto next_item = [&]() -> long long {
        if (q0 < 0) return (long long)atomicAdd(P.items, 1ull);
        const long long r = q0;
        q0 = q1;
        q1 = -1;
        return r;
      };
      auto panels_ready = [&](int k) {  // non-blocking
        if (k <= ready) return true;
        const SolveRound r = round_info(k);
        if (vload(cnt(k, 3)) < 1 + r.n_p2row + r.n_p2col + r.n_fin) return false;
        __threadfence();
        fence_proxy_async_global();  // the panels written by other CTAs are read by TMA next
        ready = k;
        return true;
      };
      auto issue_slots = [&]() {  // non-blocking, in slot order
        while (issued < claimed) {
          const int slot = issued, s = slot & 1, kind = rk[slot & 3], info = rt[slot & 3], rnd = rr[slot & 3];
          if (kind == LA_TILE) {
            if (!panels_ready(rnd)) return;
            int64_t p0, p1;
            span(rnd, p0, p1);
            const CUtensorMap *mA = (rnd & 1) ? &mapA1 : &mapA0;
            const CUtensorMap *mB = P.sym ? ((rnd & 1) ? &mapB1 : &mapB0) : &mapBg;
            mbar_arrive_expect_tx(&full_ab[s], STAGE);
            tma_load_2d(stA(s), mA, &full_ab[s], (info >> 16) * BM, 0);
            tma_load_2d(stB(s), mB, &full_ab[s], (info & 0xFFFF) * BNW * Op::EPW, P.sym ? 0 : (int)p0);
          } else {
            mbar_arrive(&full_ab[s]);  // a task or the end: no data
          }
          if (s == 0) ++n_ab[0];
          else ++n_ab[1];
          ++issued;
        }
      };
      auto issue_c = [&]() {  // !RED, non-blocking: the next tile's C once the C buffer is free and the tile's
                              // previous round is written
        if (RED) return;
        while (c_next < claimed && rk[c_next & 3] != LA_TILE) ++c_next;
        if (!cs_free || c_next >= claimed) return;
        const int pk = rt[c_next & 3], k = rr[c_next & 3];
        if (vload(P.tile_round + (pk >> 16) * P.tiles_x + (pk & 0xFFFF)) < k) return;
        __threadfence();
        fence_proxy_async_global();
        mbar_arrive_expect_tx(&full_c, P3T_C_BYTES);
        tma_load_2d(Cs, &mapC, &full_c, (pk & 0xFFFF) * BNW * Op::EPW, (pk >> 16) * BM);
        ++n_c;
        cs_free = false;
        ++c_next;
      };
      auto progress = [&]() {
        issue_slots();
        issue_c();
      };
      auto aborted = [&]() { return *reinterpret_cast<volatile int *>(&abort_flag) || vload(PP.abort); };
      // bounded, making progress meanwhile; with nothing to progress the thread
      // sleeps in the wait instead of spinning (its instructions would take issue
      // and integer-pipe cycles from the consumer warps of its sub-partition)
      auto wait_bar = [&](uint64_t *bar, uint32_t parity) {
        for (uint32_t it = 0; it < P3T_WAIT_LIMIT; ++it) {
          if (issued < claimed || (!RED && cs_free && c_next < claimed)) {
            if (mbar_try_wait(bar, parity)) return true;
            progress();
          } else if (mbar_try_wait_sleep(bar, parity, P3T_SLEEP_NS)) {
            return true;
          }
          if ((it & 31) == 31 && aborted()) return false;
        }
        return false;
      };
      auto claim = [&]() {
        const int slot = claimed;
        int kind, rnd, info;
        do {
          decode(next_item(), kind, rnd, info);
        } while (kind == LA_SKIP);
        rk[slot & 3] = kind;
        rt[slot & 3] = info;
        rr[slot & 3] = rnd;
        if (kind == LA_END) stop = true;
        else if (kind != LA_TILE && !TASK_IN_C) hold = slot;
        ++claimed;
        // the consumers read the slot's kind after its full barrier completes,
        // which happens only once it is issued (in order)
        slot_kind[slot & 1] = kind;
        slot_info[slot & 1] = info;
        slot_round[slot & 1] = rnd;
        progress();
      };
      q0 = (long long)atomicAdd(P.items, 2ull);
      q1 = q0 + 1;
      claim();
      if (!stop && hold < 0) claim();
      for (int i = 0; ok; ++i) {
        const int kind = rk[i & 3], s = i & 1;
        if (kind == LA_END) {
          // the end slot (and anything before it) must reach the consumers
          uint32_t it = 0;
          while (issued < claimed && ++it < P3T_WAIT_LIMIT && ((it & 31) != 0 || !aborted())) progress();
          ok = issued == claimed;
          break;
        }
        if (!wait_bar(&empty_ab[s], (uint32_t)(i >> 1) & 1u)) {
          ok = false;
          break;
        }
        if (!stop && hold < 0 && claimed < i + 3) claim();
        if (!wait_bar(&cdone, (uint32_t)i & 1u)) {
          ok = false;
          break;
        }
        if (kind == LA_TILE) {
          const int pk = rt[i & 3], k = rr[i & 3];
          const int ty_ = pk >> 16, tx_ = pk & 0xFFFF;
          const int r0 = ty_ * BM, c0 = tx_ * BNW * Op::EPW;
          // Cs is free again once the copy out has read it; the next tile's C
          // load (merge path) starts while this tile's copy completes
          if (RED) {
            if (c0 < red_cols(n)) {  // mapC ends at red_cols(n) in this mode
              tma_reduce_min_2d(&mapC, Cs, c0, r0);
              bulk_commit();
              bulk_wait_read_all();
            }
            mbar_arrive(&cfree);
          } else {
            if (interior_of(k, r0, c0)) {
              tma_store_2d(&mapC, Cs, c0, r0);
              bulk_commit();
              bulk_wait_read_all();
            }
            cs_free = true;
            issue_c();
          }
          // the tile of round k is written once its copy has completed: publish it
          bulk_wait_all();
          fence_proxy_async_global();
          __threadfence();
          if (!RED) atomicExch(P.tile_round + ty_ * P.tiles_x + tx_, k + 1);
          atomicAdd(cnt(k, 4), 1);
          if (k + 1 < P.q) {
            const SolveRound &r = round_at(k + 1);
            if ((ty_ == r.R && tx_ >= r.row_x0) || (tx_ == r.C && ty_ < r.col_y1)) atomicAdd(cnt(k + 1, 0), 1);
          }
          progress();
        } else if (!TASK_IN_C) {
          // a task finished: both stage buffers are free again
          hold = -1;
          while (!stop && hold < 0 && claimed < i + 3) claim();
        }
      }
      bulk_wait_all();
      if (!ok) {
        give_up();
        // the copies in flight land before the CTA exits (these waits end: TMA completes)
        for (int st = 0; st < 2; ++st)
          if (n_ab[st] > 0) mbar_wait_bounded(&full_ab[st], (uint32_t)(n_ab[st] - 1) & 1u, P3T_WAIT_LIMIT);
        if (n_c > 0) mbar_wait_bounded(&full_c, (uint32_t)(n_c - 1) & 1u, P3T_WAIT_LIMIT);
      }
    }
  } else {
    // ------------------------------------------------------------ consumers
    const int tx = tid % Map::TX, ty = tid / Map::TX;
    uint32_t acc[8][TN];
    int ct = 0;  // tiles done by this CTA
    for (int i = 0;; ++i) {
      const int s = i & 1;
      const bool bad = !mbar_wait_or(&full_ab[s], (uint32_t)(i >> 1) & 1u, P3T_WAIT_LIMIT, &abort_flag, PP.abort);
      if (__any_sync(0xffffffffu, bad)) {
        give_up();
        break;
      }
      const int kind = slot_kind[s], info = slot_info[s], rnd = slot_round[s];
      if (kind == LA_END) break;
      if (kind == LA_TILE) {
        const int cty = info >> 16, ctx = info & 0xFFFF;
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < TN; ++c) acc[r][c] = Op::INF_WORD;
        tile_minplus<Op, BM, BNW, BK, TN, 4>(stA(s), stB(s), acc, ty, tx);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_ab[s]);
        const int64_t r0 = (int64_t)cty * BM, c0 = (int64_t)ctx * BNW * Op::EPW;
        bool ebad;
        if (RED) {
          ebad = ct > 0 && !mbar_wait_or(&cfree, (uint32_t)(ct - 1) & 1u, P3T_WAIT_LIMIT, &abort_flag, PP.abort);
          if (!__any_sync(0xffffffffu, ebad)) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
              for (int h = 0; h < Map::NH; ++h)
                *reinterpret_cast<uint4 *>(Cs + Map::row(ty, r) * BNW + Map::wcol(tx, h)) =
                    make_uint4(acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
            fence_proxy_async_smem();
            if constexpr (Op::DTYPE != 1)
              if (c0 + BNW > red_cols(n) && c0 < n)
                red_tail_store<BM, BNW, TN>(reinterpret_cast<int32_t *>(D), ld, n, n, r0, c0, acc, ty, tx);
          }
        } else {
          ebad = !mbar_wait_or(&full_c, (uint32_t)ct & 1u, P3T_WAIT_LIMIT, &abort_flag, PP.abort);
          if (!__any_sync(0xffffffffu, ebad)) {
            int64_t p0, p1;
            span(rnd, p0, p1);
            const bool interior = interior_of(rnd, r0, c0);
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
              for (int h = 0; h < Map::NH; ++h) {
                uint4 *cp = reinterpret_cast<uint4 *>(Cs + Map::row(ty, r) * BNW + Map::wcol(tx, h));
                const uint4 v = *cp;
                acc[r][4 * h + 0] = Op::addmin(acc[r][4 * h + 0], 0u, v.x);
                acc[r][4 * h + 1] = Op::addmin(acc[r][4 * h + 1], 0u, v.y);
                acc[r][4 * h + 2] = Op::addmin(acc[r][4 * h + 2], 0u, v.z);
                acc[r][4 * h + 3] = Op::addmin(acc[r][4 * h + 3], 0u, v.w);
                if (interior)
                  *cp = make_uint4(acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
              }
            if (interior) fence_proxy_async_smem();
            else store_acc<Op, BM, BNW, TN>(D, ld, n, n, r0, c0, p0, p1, p0, p1, true, acc, ty, tx);
          }
        }
        ++ct;
        if (__any_sync(0xffffffffu, ebad)) {
          give_up();
          break;
        }
      } else {
        // a task of round rnd
        if (TASK_IN_C) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty_ab[s]);
          const bool cb = ct > 0 && !mbar_wait_or(&cfree, (uint32_t)(ct - 1) & 1u, P3T_WAIT_LIMIT, &abort_flag, PP.abort);
          if (__any_sync(0xffffffffu, cb)) {
            give_up();
            break;
          }
        }
        const SolveRound r = round_info(rnd);
        const int n_p2 = r.n_p2row + r.n_p2col;
        bool dbad = false;
        if (lane == 0) {
          if (kind == LA_P1) {
            if (rnd == 0 && PP.gate) dbad = !wait_count(PP.gate, 1);
            if (rnd >= 1) dbad = !wait_count(cnt(rnd, 0), r.n_prio);
            if (!dbad && rnd >= 2) dbad = !wait_count(cnt(rnd - 2, 4), P.tiles_total);
          } else if (kind == LA_P2) {
            dbad = !wait_count(cnt(rnd, 1), 1);
          } else {
            dbad = !wait_count(cnt(rnd, 2), n_p2);
          }
        }
        if (__any_sync(0xffffffffu, dbad)) {
          give_up();
          break;
        }
        GroupBar::sync();  // every consumer warp is here: the task's memory is no longer read
        if (*reinterpret_cast<volatile int *>(&la_grp_abort)) {
          give_up();
          break;
        }
        uint32_t *tsm = TASK_IN_C ? Cs : reinterpret_cast<uint32_t *>(base);
        uint32_t *colT = P.colT[rnd & 1];
        typename Op::elem *rowP = P.rowP[rnd & 1];
        if (kind == LA_P1) {
          la_task_p1<Op, BK>(D, ld, n, r.p0, colT, P.ldT, rowP, tsm, tid);
        } else if (kind == LA_P2) {
          la_task_p2<Op, BK>(D, ld, n, r.p0, r.p1, colT, P.ldT, info, r.n_p2row, r.p2_row_first, P.vec != 0,
                             SymPanel<Op>{rowP, r.band_end}, P.sym != 0, tsm, tid);
        } else {
          const int rows = rowP ? LA_FIN_ROWS : BK;
          la_task_fin<Op>(D, ld, n, r.p0, colT, P.ldT, rowP, r.band_start, info * rows,
                          min((int)(r.p1 - r.p0), (info + 1) * rows), tid);
        }
        fence_proxy_async_smem();  // the task's shared memory is refilled by TMA next
        GroupBar::sync();          // every consumer's writes of the task are done
        if (*reinterpret_cast<volatile int *>(&la_grp_abort)) {
          give_up();
          break;
        }
        if (tid == 0) {
          __threadfence();
          if (kind == LA_P1) atomicAdd(cnt(rnd, 1), 1);
          else if (kind == LA_P2) atomicAdd(cnt(rnd, 2), 1);
          atomicAdd(cnt(rnd, 3), 1);
        }
        if (!TASK_IN_C) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty_ab[s]);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&cdone);
    }
  }
  __syncthreads();
  if (abort_flag && tid == 0) atomicOr(err, 4);
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

// A^T as the k-major operand of the warp-specialized product: AT[t][i] =
// word(A[i][t]) (the value in both halves for packed 16-bit) for t < k, i < m;
// the padding rows t in [k, k_pad) and columns i >= m hold INF words, so
// TMA's zero fill of B's missing rows (t >= k) never meets a finite A.
template <class Op>
__global__ void transpose_dup_kernel(const typename Op::elem *__restrict__ A, int64_t lda, int64_t m, int64_t k,
                                     uint32_t *__restrict__ AT, int64_t ldat, int64_t k_pad) {
  __shared__ uint32_t tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, t0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {             // read A[i0 + r][t0 + tx]
    const int64_t i = i0 + r, t = t0 + tx;
    tile[r][tx] = (i < m && t < k) ? Op::dup(A[i * lda + t]) : Op::INF_WORD;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {  // write AT[t0 + r][i0 + tx]
    const int64_t t = t0 + r, i = i0 + tx;
    if (t < k_pad && i < ldat) AT[t * ldat + i] = tile[tx][r];
  }
}

// C = min(C, A (x) B) for general shapes, warp-specialized like fw_phase3_ws:
// 8 consumer warps own 8 x 8 words of a 128 x 128-word output tile and walk
// its k in chunks of 64 (one work slot per chunk; the accumulators start at INF
// with the first chunk); a producer warp moves A^T and B chunks by TMA and
// applies the tile after its last chunk: TMA min-reduction for int32 (the map
// ends at ncols rounded down to 4 elements, the tail merged by its owners),
// merge with a TMA-loaded C and TMA store (interior) or masked stores (edge)
// otherwise.  Static contiguous tile ranges per CTA; bounded waits.
template <class Op, bool RED>
__global__ void __launch_bounds__(P3W_THREADS, 1)
    fw_minplus_ws(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  const __grid_constant__ CUtensorMap mapC, typename Op::elem *__restrict__ C, int64_t ldc, int64_t m,
                  int64_t ncols, int nk, int tiles_x, int tiles_total, int *err) {
  constexpr int BK = 64, BM = 128, BNW = 128, TN = 8;
  using Map = TileMap<BM, BNW, TN>;
  constexpr int NCW = Map::THREADS / 32;
  constexpr int STAGE = P3T<BK>::STAGE_BYTES;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_ab[2], empty_ab[2], full_c, cdone, cfree;
  __shared__ int abort_flag;
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  auto stA = [&](int s) { return reinterpret_cast<uint32_t *>(base + s * STAGE); };
  auto stB = [&](int s) { return reinterpret_cast<uint32_t *>(base + s * STAGE) + BK * BM; };
  uint32_t *Cs = reinterpret_cast<uint32_t *>(base + 2 * STAGE);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int per = tiles_total / (int)gridDim.x, extra = tiles_total % (int)gridDim.x;
  const int t_begin = (int)blockIdx.x * per + min((int)blockIdx.x, extra);
  const int t_end = t_begin + per + ((int)blockIdx.x < extra ? 1 : 0);
  if (t_begin >= t_end) return;
  const long long n_slots = (long long)(t_end - t_begin) * nk;
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full_ab[i], 1);
      mbar_init(&empty_ab[i], NCW);
    }
    mbar_init(&full_c, 1);
    mbar_init(&cdone, NCW);
    mbar_init(&cfree, 1);
    fence_barrier_init();
    prefetch_tensormap(&mapA);
    prefetch_tensormap(&mapB);
    prefetch_tensormap(&mapC);
    abort_flag = 0;
  }
  __syncthreads();
  auto interior_of = [&](int64_t r0, int64_t c0) { return r0 + BM <= m && c0 + BNW * Op::EPW <= ncols; };

  if (warp == NCW) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int n_ab[2] = {0, 0}, n_c = 0;
      bool ok = true;
      auto issue_ab = [&](long long j) {
        const int s = (int)(j & 1);
        const int t = t_begin + (int)(j / nk), c = (int)(j % nk);
        mbar_arrive_expect_tx(&full_ab[s], STAGE);
        tma_load_2d(stA(s), &mapA, &full_ab[s], (t / tiles_x) * BM, c * BK);
        tma_load_2d(stB(s), &mapB, &full_ab[s], (t % tiles_x) * BNW * Op::EPW, c * BK);
        if (s == 0) ++n_ab[0];
        else ++n_ab[1];
      };
      auto issue_c = [&](int t) {
        mbar_arrive_expect_tx(&full_c, P3T_C_BYTES);
        tma_load_2d(Cs, &mapC, &full_c, (t % tiles_x) * BNW * Op::EPW, (t / tiles_x) * BM);
        ++n_c;
      };
      issue_ab(0);
      if (n_slots > 1) issue_ab(1);
      if (!RED) issue_c(t_begin);
      for (long long j = 0; j < n_slots; ++j) {
        const int s = (int)(j & 1);
        if (!mbar_wait_sleep_bounded(&empty_ab[s], (uint32_t)(j >> 1) & 1u, P3T_WAIT_LIMIT, P3T_SLEEP_NS)) {
          ok = false;
          break;
        }
        if (j + 2 < n_slots) issue_ab(j + 2);
        if (j % nk != nk - 1) continue;
        const int ti = (int)(j / nk), t = t_begin + ti;  // the tile's last chunk: write it back
        if (!mbar_wait_sleep_bounded(&cdone, (uint32_t)ti & 1u, P3T_WAIT_LIMIT, P3T_SLEEP_NS)) {
          ok = false;
          break;
        }
        const int r0 = (t / tiles_x) * BM, c0 = (t % tiles_x) * BNW * Op::EPW;
        if (RED) {
          if (c0 < red_cols(ncols)) {  // mapC ends at red_cols(ncols) in this mode
            tma_reduce_min_2d(&mapC, Cs, c0, r0);
            bulk_commit();
            bulk_wait_read_all();
          }
          mbar_arrive(&cfree);
        } else {
          if (interior_of(r0, c0)) {
            tma_store_2d(&mapC, Cs, c0, r0);
            bulk_commit();
            bulk_wait_read_all();
          }
          if (t + 1 < t_end) issue_c(t + 1);
        }
      }
      bulk_wait_all();
      if (!ok) {
        abort_flag = 1;
        for (int st = 0; st < 2; ++st)
          if (n_ab[st] > 0) mbar_wait_bounded(&full_ab[st], (uint32_t)(n_ab[st] - 1) & 1u, P3T_WAIT_LIMIT);
        if (n_c > 0) mbar_wait_bounded(&full_c, (uint32_t)(n_c - 1) & 1u, P3T_WAIT_LIMIT);
      }
    }
  } else {
    // ------------------------------------------------------------ consumers
    const int tx = tid % Map::TX, ty = tid / Map::TX;
    uint32_t acc[8][TN];
    for (long long j = 0; j < n_slots; ++j) {
      const int s = (int)(j & 1), c = (int)(j % nk);
      if (c == 0) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int q = 0; q < TN; ++q) acc[r][q] = Op::INF_WORD;
      }
      bool bad = !mbar_wait_bounded(&full_ab[s], (uint32_t)(j >> 1) & 1u, P3T_WAIT_LIMIT);
      if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) abort_flag = 1;
        break;
      }
      tile_minplus<Op, BM, BNW, BK, TN, 1>(stA(s), stB(s), acc, ty, tx);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty_ab[s]);
      if (c != nk - 1) continue;
      const int ti = (int)(j / nk), t = t_begin + ti;
      const int64_t r0 = (int64_t)(t / tiles_x) * BM, c0 = (int64_t)(t % tiles_x) * BNW * Op::EPW;
      if (RED) {
        bad = ti > 0 && !mbar_wait_bounded(&cfree, (uint32_t)(ti - 1) & 1u, P3T_WAIT_LIMIT);
        if (__any_sync(0xffffffffu, bad)) {
          if (lane == 0) abort_flag = 1;
          break;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int h = 0; h < Map::NH; ++h)
            *reinterpret_cast<uint4 *>(Cs + Map::row(ty, r) * BNW + Map::wcol(tx, h)) =
                make_uint4(acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
        fence_proxy_async_smem();
        if constexpr (Op::DTYPE == 0)
          if (c0 + BNW > red_cols(ncols) && c0 < ncols)
            red_tail_store<BM, BNW, TN>(reinterpret_cast<int32_t *>(C), ldc, m, ncols, r0, c0, acc, ty, tx);
      } else {
        bad = !mbar_wait_bounded(&full_c, (uint32_t)ti & 1u, P3T_WAIT_LIMIT);
        if (__any_sync(0xffffffffu, bad)) {
          if (lane == 0) abort_flag = 1;
          break;
        }
        const bool interior = interior_of(r0, c0);
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int h = 0; h < Map::NH; ++h) {
            uint4 *cp = reinterpret_cast<uint4 *>(Cs + Map::row(ty, r) * BNW + Map::wcol(tx, h));
            const uint4 v = *cp;
            acc[r][4 * h + 0] = Op::addmin(acc[r][4 * h + 0], 0u, v.x);
            acc[r][4 * h + 1] = Op::addmin(acc[r][4 * h + 1], 0u, v.y);
            acc[r][4 * h + 2] = Op::addmin(acc[r][4 * h + 2], 0u, v.z);
            acc[r][4 * h + 3] = Op::addmin(acc[r][4 * h + 3], 0u, v.w);
            if (interior) *cp = make_uint4(acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
          }
        if (interior) fence_proxy_async_smem();
        else store_acc<Op, BM, BNW, TN>(C, ldc, m, ncols, r0, c0, 0, 0, 0, 0, true, acc, ty, tx);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&cdone);
    }
  }
  __syncthreads();
  if (abort_flag && tid == 0) atomicOr(err, 4);
}

// ---------------------------------------------------------------- ingest / checks
// Copies W to D (when they differ) and checks the input: diagonal 0, weights
// >= 0, finite weights < INF.  status |= 1 (invalid) or 2 (range).
// fp32: a -0.0 is written as +0.0 (also in place), so that every stored
// distance is a non-negative float whose bit pattern orders like the value
// under a signed int32 compare -- the Phase-3 tiles leave by an int32 TMA
// min-reduction on those bits.
template <class Op>
__global__ void ingest_kernel(const typename Op::elem *__restrict__ W, typename Op::elem *__restrict__ D, int64_t n,
                              int64_t ld, int copy, int *status) {
  int bad = 0;
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
      typename Op::elem e = W[i * ld + j];
      if constexpr (Op::DTYPE == 2) {
        if (!(e >= 0.0f)) bad |= 1;              // negative or NaN
        if (i == j && e != 0.0f) bad |= 1;
        if (__float_as_uint(e) == 0x80000000u) {  // -0.0
          e = 0.0f;
          if (!copy) D[i * ld + j] = e;
        }
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
    typename Op::elem x = w[e];
    if (u < 0 || u >= n || v < 0 || v >= n) { bad |= 1; continue; }
    if constexpr (Op::DTYPE == 2) {
      if (!(x >= 0.0f)) { bad |= 1; continue; }
      if (x == 0.0f) x = 0.0f;  // -0.0 -> +0.0 (the stored bits order like the values)
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

// Synthetic symmetric graph for the autotuner: edge (i, j) with probability
// about 8/n, weight 1..1000, from an integer hash of (min(i,j), max(i,j)).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

template <class Op>
__global__ void synth_kernel(typename Op::elem *__restrict__ D, int64_t n, int64_t ld) {
  const uint32_t thresh = (uint32_t)(4294967295.0 * (8.0 / (double)(n > 8 ? n : 8)));
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y)
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
      const uint32_t a = (uint32_t)(i < j ? i : j), b = (uint32_t)(i < j ? j : i);
      const uint32_t h = mix32(a * 0x9E3779B9U ^ mix32(b));
      typename Op::elem v = Op::inf_elem();
      if (i == j) v = (typename Op::elem)0;
      else if (h < thresh) v = (typename Op::elem)(1 + mix32(h) % (Op::DTYPE == 1 ? 16u : 1000u));
      D[i * ld + j] = v;
    }
}

// ---------------------------------------------------------------- upper-triangular storage
// Every stored element (r, c) of the layout (rows [0, T S), columns
// [S floor(r / S), T S)): from the dense W when r, c < n (W == nullptr: 0 on
// the diagonal, INF elsewhere), INF in the padding.  With W, the input is
// checked as in ingest_kernel (status |= 1 invalid, 2 range); fp32 -0.0 is
// stored as +0.0.
template <class Op>
__global__ void tri_fill_kernel(const typename Op::elem *__restrict__ W, int64_t ldw, typename Op::elem *__restrict__ D,
                                Layout L, int64_t n, int *status) {
  using E = typename Op::elem;
  const int64_t rows = (int64_t)L.T << L.sh;
  int bad = 0;
  for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
    const int64_t c_first = (r >> L.sh) << L.sh;
    const int64_t o = L.off(r, c_first) - c_first;  // D[o + c] is element (r, c) for stored c
    for (int64_t c = c_first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < rows;
         c += (int64_t)gridDim.x * blockDim.x) {
      E e = Op::inf_elem();
      if (r < n && c < n) {
        if (!W) {
          e = r == c ? (E)0 : Op::inf_elem();
        } else {
          e = W[r * ldw + c];
          if constexpr (Op::DTYPE == 2) {
            if (!(e >= 0.0f)) bad |= 1;
            if (r == c && e != 0.0f) bad |= 1;
            if (e == 0.0f) e = 0.0f;
          } else if constexpr (Op::DTYPE == 1) {
            if (e > Op::inf_elem()) bad |= 2;
            if (r == c && e != 0) bad |= 1;
          } else {
            if (e < 0) bad |= 1;
            if (e > Op::inf_elem()) bad |= 2;
            if (r == c && e != 0) bad |= 1;
          }
        }
      }
      D[o + c] = e;
    }
  }
  if (bad && status) atomicOr(status, bad);
}

// Scatters an undirected edge list into the layout: min over duplicates into
// (u, v) and (v, u), whichever of them is stored; checks as scatter_edges_kernel.
template <class Op>
__global__ void tri_scatter_edges_kernel(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                                         const typename Op::elem *__restrict__ w, int64_t m, typename Op::elem *D,
                                         Layout L, int64_t n, int *status) {
  int bad = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = src[e], v = dst[e];
    typename Op::elem x = w[e];
    if (u < 0 || u >= n || v < 0 || v >= n) { bad |= 1; continue; }
    if constexpr (Op::DTYPE == 2) {
      if (!(x >= 0.0f)) { bad |= 1; continue; }
      if (x == 0.0f) x = 0.0f;
    } else if constexpr (Op::DTYPE == 0) {
      if (x < 0) { bad |= 1; continue; }
    }
    if (x >= Op::inf_elem()) { if (!(Op::DTYPE == 2 && x == Op::inf_elem())) bad |= 2; continue; }
    if (u == v) continue;
    for (int k = 0; k < 2; ++k) {
      const int64_t a = k ? v : u, b = k ? u : v;
      if (!L.stored(a, b)) continue;
      typename Op::elem *p = D + L.off(a, b);
      if constexpr (Op::DTYPE == 1) atomic_min_u16(p, x);
      else if constexpr (Op::DTYPE == 2) atomicMin(reinterpret_cast<int *>(p), __float_as_int(x));
      else atomicMin(reinterpret_cast<int *>(p), (int)x);
    }
  }
  if (bad) atomicOr(status, bad);
}

// Dense out[r][c] for the stored elements with r, c < n (the lower triangle
// outside the diagonal super-tiles is filled afterwards by mirror_kernel).
template <class Op>
__global__ void tri_to_dense_kernel(const typename Op::elem *__restrict__ D, Layout L, int64_t n,
                                    typename Op::elem *__restrict__ out, int64_t ldo) {
  for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
    const int64_t c_first = (r >> L.sh) << L.sh;
    const int64_t o = L.off(r, c_first) - c_first;  // D[o + c] is element (r, c) for stored c
    for (int64_t c = c_first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x)
      out[r * ldo + c] = D[o + c];
  }
}

// out[i][c] = D(rows[i], c) for c < n: the stored element, or its mirror
// (c, rows[i]) below the diagonal super-tiles.  A row index outside [0, n)
// sets status |= 1 and its output row is left untouched.
template <class Op>
__global__ void tri_rows_kernel(const typename Op::elem *__restrict__ D, Layout L, int64_t n,
                                const int64_t *__restrict__ rows, int64_t k, typename Op::elem *__restrict__ out,
                                int64_t ldo, int *status) {
  for (int64_t i = blockIdx.y; i < k; i += gridDim.y) {
    const int64_t r = rows[i];
    if (r < 0 || r >= n) {
      if (threadIdx.x == 0 && blockIdx.x == 0 && status) atomicOr(status, 1);
      continue;
    }
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
      out[i * ldo + c] = L.stored(r, c) ? D[L.off(r, c)] : D[L.off(c, r)];
  }
}

// ---------------------------------------------------------------- host launchers
// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D row-major tensor map: dims {cols, rows}, row pitch in bytes, box {bx, by}.
static bool make_map(CUtensorMap *m, CUtensorMapDataType dt, const void *base, uint64_t cols, uint64_t rows,
                     uint64_t pitch, uint32_t bx, uint32_t by) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {pitch};
  cuuint32_t box[2] = {bx, by};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, dt, 2, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int sm_count() {
  int dev = 0, c = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
  return c > 0 ? c : 1;
}

static int *error_word() {
  // one device word per process and device for bounded-wait timeouts (rare)
  static int *w[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!w[dev]) {
    if (cudaMalloc(&w[dev], sizeof(int)) != cudaSuccess) return nullptr;
    cudaMemset(w[dev], 0, sizeof(int));
  }
  return w[dev];
}

static inline unsigned grid_rows(int64_t n) { return (unsigned)(n < 65535 ? (n > 0 ? n : 1) : 65535); }
static inline unsigned grid_cols(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return (unsigned)(g < 1 ? 1 : (g > 64 ? 64 : g));
}

// Launches kernel k on s with programmatic dependent launch (see pdl_trigger /
// pdl_wait): the per-round kernels' launch latency overlaps the previous
// kernel instead of adding to every round.
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);  // errors surface in cudaGetLastError
}

template <class Op, int BK>
static cudaError_t rounds_impl(void *Dv, Layout L, int64_t n, void *colTv, int64_t ldT, bool vec, int variant,
                               cudaStream_t s, int64_t *launches, PhaseTimer *tm, int *wait_err, bool sym,
                               void *rowPv, const int *sym_flag, const int *gate, uint32_t dep_spins,
                               int grid_cap) {
  const bool use_tma = variant != 0;
  const int sms = grid_cap > 0 ? std::min(sm_count(), grid_cap) : sm_count();
  using Elem = typename Op::elem;
  using E = Elem;
  E *D = static_cast<E *>(Dv);
  const int64_t ld = L.ld;
  const bool tri = L.tri();
  const int64_t q = (n + BK - 1) / BK;
  // lookahead rounds (the warp-specialized Phase 3 with the TMA path and more
  // than one round): two panel buffers used by round parity, then 4 counters
  // per round
  // kernel 4 (every round in one launch) when its conditions hold, else 3
  bool la_on = kLookaheadWidth<BK> && use_tma && vec && variant == 4 && q > 1 && !tri;
  if (variant == 4) variant = 3;
  // round width 128 runs the per-tile kernel or the warp-specialized one (its
  // tiles take two 64-step stages); the other TMA kernels hold a whole round
  // per stage, which does not fit
  if (BK > 64 && (variant == 1 || variant == 2)) variant = 3;
  // upper-triangular storage: symmetric mode on the warp-specialized Phase 3,
  // one launch per round
  if (tri && (!sym || !vec || variant != 3)) return cudaErrorNotSupported;
  // the device picks the symmetric mode (single launch only; otherwise the
  // general path, which is exact for any input)
  const bool dev_sym = la_on && !sym && sym_flag != nullptr;
  const bool any_sym = sym || dev_sym;
  uint32_t *colTb[2], *colT = static_cast<uint32_t *>(colTv);
  colTb[0] = colT;
  colTb[1] = la_on ? colT + (int64_t)kMaxRoundWidth * ldT : colT;
  // symmetric mode: the element panel (B operand of Phase 3) is colT itself
  // for 32-bit elements, a separate BK x ldT buffer for packed 16-bit
  Elem *rowP = any_sym ? (Op::EPW == 2 ? static_cast<Elem *>(rowPv) : nullptr) : nullptr;
  if (any_sym && Op::EPW == 2 && !rowP) return cudaErrorInvalidValue;
  Elem *rowPb[2] = {rowP, (la_on && rowP) ? rowP + (int64_t)kMaxRoundWidth * ldT : rowP};
  auto symB_of = [&](int b) -> const Elem * {
    return sym ? (Op::EPW == 2 ? rowPb[b] : reinterpret_cast<const Elem *>(colTb[b])) : nullptr;
  };
  auto symB_any = [&](int b) -> const Elem * {  // the symmetric-mode B when the device may pick it
    return Op::EPW == 2 ? rowPb[b] : reinterpret_cast<const Elem *>(colTb[b]);
  };
  using C2 = P2Cfg<Op, BK>;
  using C3 = P3Cfg<Op>;
  constexpr int SMEM3 = (BK * C3::BM + BK * C3::BNW) * 4;
  constexpr int KS = P3T<BK>::KS;  // k-steps per stage of the TMA Phase-3 kernels (box height of the A/B maps)
  // the attributes are per device, so they are set on every call (a cheap host call)
  cudaError_t e = cudaFuncSetAttribute(fw_phase2<Op, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2::SMEM);
  if (e != cudaSuccess) return e;
  if constexpr (BK > 64) {
    e = cudaFuncSetAttribute(fw_phase1_w128<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(P1Smem<Op, 128>));
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute(fw_phase3<Op, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM3);
  if (e != cudaSuccess) return e;
  // persistent TMA Phase 3 when D is 16-byte addressable (otherwise the
  // per-tile kernel with scalar edge handling); A (and B in symmetric mode)
  // maps for each panel buffer
  CUtensorMap mA[2], mB[2], mC, mBs[2];  // mBs: B of the symmetric mode when the device picks the mode
  bool tma = vec && use_tma;
  int *err = nullptr;
  if (tma) {
    constexpr CUtensorMapDataType dt = Op::DTYPE == 1   ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                       : Op::DTYPE == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                        : CU_TENSOR_MAP_DATA_TYPE_INT32;
    for (int b = 0; b < (la_on ? 2 : 1) && tma; ++b)
      tma = make_map(&mA[b], CU_TENSOR_MAP_DATA_TYPE_UINT32, colTb[b], (uint64_t)ldT, (uint64_t)BK,
                     (uint64_t)ldT * 4, 128, KS) &&
            (sym ? make_map(&mB[b], dt, symB_of(b), (uint64_t)ldT, (uint64_t)BK, (uint64_t)ldT * sizeof(E),
                            128 * Op::EPW, KS)
                 : make_map(&mB[b], dt, D, (uint64_t)n, (uint64_t)n, (uint64_t)ld * sizeof(E), 128 * Op::EPW, KS));
    for (int b = 0; b < 2 && dev_sym && tma; ++b)
      tma = make_map(&mBs[b], dt, symB_any(b), (uint64_t)ldT, (uint64_t)BK, (uint64_t)ldT * sizeof(E), 128 * Op::EPW,
                     KS);
    // int32 and fp32 (TMA min-reduction epilogue of variant 3): x extent
    // red_cols(n), and an int32 map (fp32 bits of non-negative values order
    // like int32); upper-triangular storage: the whole rectangle
    const bool red_map = kRedOp<Op> && variant == 3;
    const uint64_t cx = tri ? (uint64_t)ld : red_map ? (uint64_t)(n & ~(int64_t)3) : (uint64_t)n;
    const uint64_t cy = tri ? ((uint64_t)L.Th << L.sh) : (uint64_t)n;
    tma = tma && cx > 0 &&
          make_map(&mC, red_map ? CU_TENSOR_MAP_DATA_TYPE_INT32 : dt, D, cx, cy, (uint64_t)ld * sizeof(E),
                   128 * Op::EPW, 128);
    err = tma ? (wait_err ? wait_err : error_word()) : nullptr;
    tma = tma && err != nullptr;
    if (tma) {
      if constexpr (BK <= 64) {
        e = cudaFuncSetAttribute(fw_phase3_tma<Op, BK, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 P3T<BK>::SMEM);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(fw_phase3_tma<Op, BK, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   P3T<BK>::SMEM);
      }
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fw_phase3_ws<Op, BK, kRedOp<Op>>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 P3T<BK>::SMEM);
      if (e != cudaSuccess) return e;
    }
  }
  la_on = la_on && tma;
  if (!la_on) {
    colTb[1] = colT;
    rowPb[1] = rowP;
  }
  const int tiles_x = (int)((n + 128 * Op::EPW - 1) / (128 * Op::EPW));
  const int tiles_y = (int)((n + 127) / 128);
  int tiles_total = tiles_x * tiles_y;
  if (sym) {  // tiles with tx >= ty / EPW
    tiles_total = 0;
    for (int y = 0; y < tiles_y; ++y) tiles_total += tiles_x - std::min(tiles_x, y / Op::EPW);
  }
  const int grid_tma = std::min(sms, tiles_total);
  const int nrow = (int)((n + C2::ROW_BNW * Op::EPW - 1) / (C2::ROW_BNW * Op::EPW));
  const int ncol = (int)((n + C2::COL_BM - 1) / C2::COL_BM);
  const dim3 g3((unsigned)((n + C3::BNW * Op::EPW - 1) / (C3::BNW * Op::EPW)), (unsigned)((n + C3::BM - 1) / C3::BM));
  auto span = [&](int64_t k, int64_t &p0, int64_t &p1) {
    p0 = k * BK;
    p1 = (p0 + BK < n) ? p0 + BK : n;
  };
  // Phase 1 and Phase 2 of round k as their own launches, into panel cT / rP
  auto panels = [&](int64_t k, uint32_t *cT, Elem *rP) {
    int64_t p0, p1;
    span(k, p0, p1);
    const double w = (double)(p1 - p0), rest = (double)(n - (p1 - p0));
    if (tm) tm->before(0, s);
    if constexpr (BK > 64)
      launch_pdl(fw_phase1_w128<Op>, dim3(1), dim3(P1W_THREADS), sizeof(P1Smem<Op, 128>), s, D, L, n, p0, cT, ldT,
                 sym ? rP : nullptr);
    else if (sym && rP)
      launch_pdl(fw_phase1_sym<Op, BK>, dim3(1), dim3(P1_THREADS), 0, s, D, L, n, p0, cT, ldT, rP);
    else
      launch_pdl(fw_phase1<Op, BK>, dim3(1), dim3(P1_THREADS), 0, s, D, L, n, p0, cT, ldT);
    if (launches) *launches += 1;
    if (tm) tm->after(0, s, w * w * w);
    if (q == 1) return;
    if (tm) tm->before(1, s);
    SymPanel<Op> sp{rP, (p0 / (128 * Op::EPW)) * (128 * Op::EPW) + 128 * Op::EPW};
    int r_first = 0, r_count = nrow, c_count = ncol;
    if (sym) {  // row chunks that reach columns >= p1; column chunks with rows < p0
      r_first = (int)(p1 / (C2::ROW_BNW * Op::EPW));
      r_count = std::max(0, nrow - r_first);
      c_count = (int)((p0 + C2::COL_BM - 1) / C2::COL_BM);
    }
    if (r_count + c_count > 0) {
      launch_pdl(fw_phase2<Op, BK>, dim3(r_count + c_count), dim3(C2::THREADS), (size_t)C2::SMEM, s, D, L, n, p0, p1, cT,
                 ldT, r_count, vec ? 1 : 0, r_first, sym ? 1 : 0, sp);
      if (launches) *launches += 1;
    }
    if (sym && p0 > 0) {
      const int64_t band_start = (p0 / (128 * Op::EPW)) * (128 * Op::EPW);
      const int64_t xs = rP ? p0 : p0 - band_start;  // elements to visit per row
      const unsigned gx = (unsigned)std::min<int64_t>((xs + 255) / 256, 64);
      if (xs > 0) {
        launch_pdl(panel_finalize<Op>, dim3(gx, BK), dim3(256), 0, s, D, L, n, p0, (const uint32_t *)cT, ldT, rP,
                   band_start);
        if (launches) *launches += 1;
      }
    }
    if (tm) tm->after(1, s, sym ? rest * w * w : 2.0 * rest * w * w);
  };
  // relaxations of round k's Phase 3 actually performed: the processed tiles' share of (n - w)^2 w
  auto p3_work = [&](int64_t k) {
    int64_t p0, p1;
    span(k, p0, p1);
    const double w = (double)(p1 - p0), rest = (double)(n - (p1 - p0));
    const double frac = sym ? (double)tiles_total / ((double)tiles_x * tiles_y) : 1.0;
    return rest * rest * w * frac;
  };
  if (!la_on) {
    for (int64_t k = 0; k < q; ++k) {
      int64_t p0, p1;
      span(k, p0, p1);
      panels(k, colT, rowP);
      if (q == 1) break;
      if (tm) tm->before(2, s);
      if (tma && variant == 3)
        launch_pdl(fw_phase3_ws<Op, BK, kRedOp<Op>>, dim3(grid_tma), dim3(P3W_THREADS), (size_t)P3T<BK>::SMEM, s,
                   mA[0], mB[0], mC, D, L, n, p0, p1, tiles_x, tiles_total, err, sym ? 1 : 0, tiles_y);
      else if constexpr (BK <= 64) {
        if (tma && variant == 2)
          fw_phase3_tma<Op, BK, 4><<<grid_tma, TileMap<128, 128, 4>::THREADS, P3T<BK>::SMEM, s>>>(
              mA[0], mB[0], mC, D, ld, n, p0, p1, tiles_x, tiles_total, err, sym ? 1 : 0, tiles_y);
        else if (tma)
          fw_phase3_tma<Op, BK, 8><<<grid_tma, TileMap<128, 128, 8>::THREADS, P3T<BK>::SMEM, s>>>(
              mA[0], mB[0], mC, D, ld, n, p0, p1, tiles_x, tiles_total, err, sym ? 1 : 0, tiles_y);
        else
          fw_phase3<Op, BK><<<g3, C3::THREADS, SMEM3, s>>>(D, ld, n, p0, p1, colT, ldT, vec ? 1 : 0, symB_of(0));
      } else
        fw_phase3<Op, BK><<<g3, C3::THREADS, SMEM3, s>>>(D, ld, n, p0, p1, colT, ldT, vec ? 1 : 0, symB_of(0));
      if (launches) *launches += 1;
      if (tm) tm->after(2, s, p3_work(k));
    }
  } else if constexpr (kLookaheadWidth<BK>) {
    // every round in one persistent launch (fw_solve_ws)
    constexpr bool RED = kRedOp<Op>;
    int tiles_sym = 0;  // tiles with tx >= ty / EPW
    for (int y = 0; y < tiles_y; ++y) tiles_sym += tiles_x - std::min(tiles_x, y / Op::EPW);
    const int grid = std::min(sms, tiles_sym);  // one launch grid for either mode
    char *cbase = reinterpret_cast<char *>(colT) + lookahead_counter_offset(ldT);
    double work[2] = {0.0, 0.0};
    auto plan = [&](bool msym) {
      SolvePlan<Op> P{};
      P.n = n;
      P.ld = ld;
      P.ldT = ldT;
      P.q = (int)q;
      P.tiles_x = tiles_x;
      P.tiles_y = tiles_y;
      P.tiles_total = msym ? tiles_sym : tiles_x * tiles_y;
      P.grid = grid;
      P.sym = msym ? 1 : 0;
      P.vec = vec ? 1 : 0;
      P.colT[0] = colTb[0];
      P.colT[1] = colTb[1];
      P.rowP[0] = msym ? rowPb[0] : nullptr;
      P.rowP[1] = msym ? rowPb[1] : nullptr;
      P.items = reinterpret_cast<unsigned long long *>(cbase);
      P.cnt = reinterpret_cast<int *>(cbase + 16);
      P.tile_round = P.cnt + 6 * q;
      const bool has_rowP = P.rowP[0] != nullptr;
      P.base1 = solve_round<Op, BK>(n, P.q, tiles_x, tiles_y, P.tiles_total, grid, P.sym, has_rowP, 0).total;
      P.block = 0;
      double &wk = work[msym ? 1 : 0];
      const double frac = (double)P.tiles_total / ((double)tiles_x * tiles_y);
      for (int j = 1; j <= P.q; ++j) {
        P.block = std::max(P.block,
                           solve_round<Op, BK>(n, P.q, tiles_x, tiles_y, P.tiles_total, grid, P.sym, has_rowP, j).total);
        int64_t p0, p1;
        span(j - 1, p0, p1);
        const double w = (double)(p1 - p0), rest = (double)(n - (p1 - p0));
        wk += rest * rest * w * frac;  // the processed tiles' share of (n - w)^2 w
        wk += w * w * w + (msym ? rest * w * w : 2.0 * rest * w * w);  // the round's Phase 1 and Phase 2
      }
      return P;
    };
    SolvePlans<Op> PP{};
    PP.p[0] = plan(sym);
    PP.p[1] = dev_sym ? plan(true) : PP.p[0];
    PP.sym_flag = dev_sym ? sym_flag : nullptr;
    PP.abort = reinterpret_cast<int *>(cbase + 8);
    PP.gate = gate;
    PP.dep_spins = dep_spins ? dep_spins : P3T_WAIT_LIMIT / 4;
    // B maps: symmetric mode's element panels (by parity) and the general mode's D rows
    const CUtensorMap &b0 = dev_sym ? mBs[0] : mB[0], &b1 = dev_sym ? mBs[1] : mB[1];
    const CUtensorMap &bg = mB[0];  // D rows unless the host fixed the symmetric mode (then unused)
    e = cudaMemsetAsync(cbase, 0, 16 + sizeof(int) * (6 * (size_t)q + (RED ? 0 : (size_t)tiles_x * tiles_y)), s);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fw_solve_ws<Op, BK, RED>, cudaFuncAttributeMaxDynamicSharedMemorySize, P3T<BK>::SMEM);
    if (e != cudaSuccess) return e;
    if (tm) tm->before(2, s);
    fw_solve_ws<Op, BK, RED><<<grid, P3W_THREADS, P3T<BK>::SMEM, s>>>(mA[0], mA[1], b0, b1, bg, mC, D, err, PP);
    if (launches) *launches += 1;
    if (tm) {
      if (dev_sym) tm->after_choice(2, s, work[1], work[0], sym_flag);
      else tm->after(2, s, work[sym ? 1 : 0]);
    }
  }
  if ((sym || dev_sym) && q > 1 && !tri) {  // the lower triangle from the upper (not stored when tri)
    const dim3 gm((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
    mirror_kernel<Op><<<gm, dim3(32, 8), 0, s>>>(D, n, ld, dev_sym ? sym_flag : nullptr);
    if (launches) *launches += 1;
  }
  return cudaGetLastError();
}

static bool aligned16(const void *p, int64_t ld, size_t esz) {
  return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && ((ld * (int64_t)esz) % 16 == 0);
}

template <class Op>
static cudaError_t rounds_bk(const RoundConfig &cfg, void *D, Layout L, int64_t n, void *colT, int64_t ldT,
                             cudaStream_t s, int64_t *launches, PhaseTimer *tm, int *wait_err) {
  const bool vec = aligned16(D, L.ld, sizeof(typename Op::elem));
  if (cfg.bk == 32)
    return rounds_impl<Op, 32>(D, L, n, colT, ldT, vec, cfg.p3, s, launches, tm, wait_err, cfg.sym, cfg.rowP,
                               cfg.sym_flag, cfg.gate, cfg.dep_spins, cfg.grid_cap);
  if (cfg.bk == 64)
    return rounds_impl<Op, 64>(D, L, n, colT, ldT, vec, cfg.p3, s, launches, tm, wait_err, cfg.sym, cfg.rowP,
                               cfg.sym_flag, cfg.gate, cfg.dep_spins, cfg.grid_cap);
  if (cfg.bk == 128)
    return rounds_impl<Op, 128>(D, L, n, colT, ldT, vec, cfg.p3, s, launches, tm, wait_err, cfg.sym, cfg.rowP,
                                cfg.sym_flag, cfg.gate, cfg.dep_spins, cfg.grid_cap);
  return cudaErrorInvalidValue;
}

bool single_launch(int dtype, const void *D, int64_t ld, int64_t n, const RoundConfig &cfg) {
  const size_t es = dtype == 1 ? 2 : 4;
  return cfg.p3 == 4 && cfg.bk == 64 && n > 64 && aligned16(D, ld, es);
}

cudaError_t launch_symmetry_check(int dtype, const void *D, int64_t n, int64_t ld, int *flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const dim3 g((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
  switch (dtype) {
    case 0: symmetry_check_kernel<OpI32><<<g, dim3(32, 8), 0, s>>>(static_cast<const int32_t *>(D), n, ld, flag); break;
    case 1: symmetry_check_kernel<OpU16><<<g, dim3(32, 8), 0, s>>>(static_cast<const uint16_t *>(D), n, ld, flag); break;
    case 2: symmetry_check_kernel<OpF32><<<g, dim3(32, 8), 0, s>>>(static_cast<const float *>(D), n, ld, flag); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_rounds(int dtype, void *D, int64_t ld, int64_t n, void *colT, int64_t ldT, cudaStream_t s,
                          int64_t *launches, PhaseTimer *tm, const RoundConfig &cfg, int *wait_err) {
  if (n <= 0) return cudaSuccess;
  switch (dtype) {
    case 0: return rounds_bk<OpI32>(cfg, D, Layout(ld), n, colT, ldT, s, launches, tm, wait_err);
    case 1: return rounds_bk<OpU16>(cfg, D, Layout(ld), n, colT, ldT, s, launches, tm, wait_err);
    case 2: return rounds_bk<OpF32>(cfg, D, Layout(ld), n, colT, ldT, s, launches, tm, wait_err);
    default: return cudaErrorInvalidValue;
  }
}

void tri_shape(int64_t n, int dtype, int64_t *rows, int64_t *ld) {
  const Layout L = tri_layout(n, dtype == 1 ? 2 : 1, rows);
  if (ld) *ld = L.ld;
}

cudaError_t launch_rounds_tri(int dtype, void *T, int64_t n, void *colT, int64_t ldT, cudaStream_t s,
                              int64_t *launches, PhaseTimer *tm, RoundConfig cfg, int *wait_err) {
  if (n <= 0) return cudaSuccess;
  const Layout L = tri_layout(n, dtype == 1 ? 2 : 1, nullptr);
  cfg.sym = true;
  cfg.p3 = 3;
  cfg.sym_flag = nullptr;
  switch (dtype) {
    case 0: return rounds_bk<OpI32>(cfg, T, L, n, colT, ldT, s, launches, tm, wait_err);
    case 1: return rounds_bk<OpU16>(cfg, T, L, n, colT, ldT, s, launches, tm, wait_err);
    case 2: return rounds_bk<OpF32>(cfg, T, L, n, colT, ldT, s, launches, tm, wait_err);
    default: return cudaErrorInvalidValue;
  }
}

template <class Op>
static cudaError_t tri_fill_impl(const void *W, int64_t ldw, void *T, int64_t n, int *status, cudaStream_t s,
                                 int64_t *launches) {
  using E = typename Op::elem;
  const Layout L = tri_layout(n, Op::EPW, nullptr);
  const int64_t rows = (int64_t)L.T << L.sh;
  tri_fill_kernel<Op><<<dim3(grid_cols(rows, 256), grid_rows(rows)), 256, 0, s>>>(static_cast<const E *>(W), ldw,
                                                                                  static_cast<E *>(T), L, n, status);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_tri_fill(int dtype, const void *W, int64_t ldw, void *T, int64_t n, int *status, cudaStream_t s,
                            int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  if (W) {  // an asymmetric W has no upper-triangular form: status |= 1
    cudaError_t e = launch_symmetry_check(dtype, W, n, ldw, status, s);
    if (e != cudaSuccess) return e;
    if (launches) *launches += 1;
  }
  switch (dtype) {
    case 0: return tri_fill_impl<OpI32>(W, ldw, T, n, status, s, launches);
    case 1: return tri_fill_impl<OpU16>(W, ldw, T, n, status, s, launches);
    case 2: return tri_fill_impl<OpF32>(W, ldw, T, n, status, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

template <class Op>
static cudaError_t tri_scatter_impl(const int32_t *src, const int32_t *dst, const void *w, int64_t m, void *T,
                                    int64_t n, int *status, cudaStream_t s, int64_t *launches) {
  using E = typename Op::elem;
  cudaError_t e = tri_fill_impl<Op>(nullptr, 0, T, n, status, s, launches);
  if (e != cudaSuccess || m <= 0) return e;
  const Layout L = tri_layout(n, Op::EPW, nullptr);
  int64_t blocks = (m + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  tri_scatter_edges_kernel<Op><<<(unsigned)blocks, 256, 0, s>>>(src, dst, static_cast<const E *>(w), m,
                                                                static_cast<E *>(T), L, n, status);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_tri_from_edges(int dtype, const int32_t *src, const int32_t *dst, const void *w, int64_t m,
                                  void *T, int64_t n, int *status, cudaStream_t s, int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  switch (dtype) {
    case 0: return tri_scatter_impl<OpI32>(src, dst, w, m, T, n, status, s, launches);
    case 1: return tri_scatter_impl<OpU16>(src, dst, w, m, T, n, status, s, launches);
    case 2: return tri_scatter_impl<OpF32>(src, dst, w, m, T, n, status, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

template <class Op>
static cudaError_t tri_out_impl(const void *T, int64_t n, void *D, int64_t ld, const int64_t *rows, int64_t k,
                                int *status, cudaStream_t s, int64_t *launches) {
  using E = typename Op::elem;
  const Layout L = tri_layout(n, Op::EPW, nullptr);
  if (rows) {
    if (k <= 0) return cudaSuccess;
    tri_rows_kernel<Op><<<dim3(grid_cols(n, 256), grid_rows(k)), 256, 0, s>>>(
        static_cast<const E *>(T), L, n, rows, k, static_cast<E *>(D), ld, status);
    if (launches) *launches += 1;
    return cudaGetLastError();
  }
  tri_to_dense_kernel<Op><<<dim3(grid_cols(n, 256), grid_rows(n)), 256, 0, s>>>(static_cast<const E *>(T), L, n,
                                                                              static_cast<E *>(D), ld);
  const dim3 gm((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
  mirror_kernel<Op><<<gm, dim3(32, 8), 0, s>>>(static_cast<E *>(D), n, ld, nullptr);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_tri_to_dense(int dtype, const void *T, int64_t n, void *D, int64_t ld, cudaStream_t s,
                                int64_t *launches) {
  if (n <= 0) return cudaSuccess;
  switch (dtype) {
    case 0: return tri_out_impl<OpI32>(T, n, D, ld, nullptr, 0, nullptr, s, launches);
    case 1: return tri_out_impl<OpU16>(T, n, D, ld, nullptr, 0, nullptr, s, launches);
    case 2: return tri_out_impl<OpF32>(T, n, D, ld, nullptr, 0, nullptr, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tri_rows(int dtype, const void *T, int64_t n, const int64_t *rows, int64_t k, void *out,
                            int64_t ldo, int *status, cudaStream_t s, int64_t *launches) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  switch (dtype) {
    case 0: return tri_out_impl<OpI32>(T, n, out, ldo, rows, k, status, s, launches);
    case 1: return tri_out_impl<OpU16>(T, n, out, ldo, rows, k, status, s, launches);
    case 2: return tri_out_impl<OpF32>(T, n, out, ldo, rows, k, status, s, launches);
    default: return cudaErrorInvalidValue;
  }
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

cudaError_t launch_synth(int dtype, void *D, int64_t n, int64_t ld, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 g(grid_cols(n, 256), grid_rows(n));
  switch (dtype) {
    case 0: synth_kernel<OpI32><<<g, 256, 0, s>>>(static_cast<int32_t *>(D), n, ld); break;
    case 1: synth_kernel<OpU16><<<g, 256, 0, s>>>(static_cast<uint16_t *>(D), n, ld); break;
    case 2: synth_kernel<OpF32><<<g, 256, 0, s>>>(static_cast<float *>(D), n, ld); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
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

// The warp-specialized product (A^T in `scratch`); returns cudaErrorNotSupported
// when its preconditions do not hold (the caller then uses minplus_kernel).
template <class Op>
static cudaError_t minplus_ws_impl(const void *A, int64_t lda, const void *B, int64_t ldb, void *Cm, int64_t ldc,
                                   int64_t m, int64_t k, int64_t nn, cudaStream_t s, int64_t *launches,
                                   void *scratch, size_t scratch_bytes, int *wait_err) {
  using E = typename Op::elem;
  constexpr bool RED = Op::DTYPE == 0;
  const size_t es = sizeof(E);
  if (k <= 0 || !scratch || scratch_bytes < minplus_scratch_bytes(m, k)) return cudaErrorNotSupported;
  if (!aligned16(B, ldb, es) || !aligned16(Cm, ldc, es)) return cudaErrorNotSupported;
  const uint64_t cx = RED ? (uint64_t)(nn & ~(int64_t)3) : (uint64_t)nn;
  if (cx == 0) return cudaErrorNotSupported;
  int *err = wait_err ? wait_err : error_word();
  if (!err) return cudaErrorNotSupported;
  const int64_t k_pad = (k + 63) / 64 * 64, ldat = (m + 255) / 256 * 256;
  uint32_t *AT = static_cast<uint32_t *>(scratch);
  constexpr CUtensorMapDataType dt = Op::DTYPE == 1   ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                     : Op::DTYPE == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                      : CU_TENSOR_MAP_DATA_TYPE_INT32;
  CUtensorMap mA, mB, mC;
  if (!make_map(&mA, CU_TENSOR_MAP_DATA_TYPE_UINT32, AT, (uint64_t)ldat, (uint64_t)k_pad, (uint64_t)ldat * 4, 128,
                64) ||
      !make_map(&mB, dt, B, (uint64_t)nn, (uint64_t)k, (uint64_t)ldb * es, 128 * Op::EPW, 64) ||
      !make_map(&mC, dt, Cm, cx, (uint64_t)m, (uint64_t)ldc * es, 128 * Op::EPW, 128))
    return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(fw_minplus_ws<Op, RED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       P3T<64>::SMEM);
  if (e != cudaSuccess) return e;
  const dim3 gt((unsigned)(ldat / 32), (unsigned)(k_pad / 32));
  transpose_dup_kernel<Op><<<gt, dim3(32, 8), 0, s>>>(static_cast<const E *>(A), lda, m, k, AT, ldat, k_pad);
  const int tiles_x = (int)((nn + 128 * Op::EPW - 1) / (128 * Op::EPW));
  const int tiles_total = tiles_x * (int)((m + 127) / 128);
  const int grid = std::min(sm_count(), tiles_total);
  fw_minplus_ws<Op, RED><<<grid, P3W_THREADS, P3T<64>::SMEM, s>>>(mA, mB, mC, static_cast<E *>(Cm), ldc, m, nn,
                                                                   (int)(k_pad / 64), tiles_x, tiles_total, err);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

size_t minplus_scratch_bytes(int64_t m, int64_t k) {
  if (m <= 0 || k <= 0) return 0;
  return (size_t)((k + 63) / 64 * 64) * (size_t)((m + 255) / 256 * 256) * 4;
}

cudaError_t launch_minplus(int dtype, const void *A, int64_t lda, const void *B, int64_t ldb, void *Cm, int64_t ldc,
                           int64_t m, int64_t k, int64_t nn, cudaStream_t s, int64_t *launches, void *scratch,
                           size_t scratch_bytes, int *wait_err) {
  if (m <= 0 || nn <= 0) return cudaSuccess;
  cudaError_t e = cudaErrorNotSupported;
  switch (dtype) {
    case 0: e = minplus_ws_impl<OpI32>(A, lda, B, ldb, Cm, ldc, m, k, nn, s, launches, scratch, scratch_bytes, wait_err); break;
    case 1: e = minplus_ws_impl<OpU16>(A, lda, B, ldb, Cm, ldc, m, k, nn, s, launches, scratch, scratch_bytes, wait_err); break;
    case 2: e = minplus_ws_impl<OpF32>(A, lda, B, ldb, Cm, ldc, m, k, nn, s, launches, scratch, scratch_bytes, wait_err); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaErrorNotSupported) return e;
  switch (dtype) {
    case 0: return minplus_impl<OpI32>(A, lda, B, ldb, Cm, ldc, m, k, nn, s, launches);
    case 1: return minplus_impl<OpU16>(A, lda, B, ldb, Cm, ldc, m, k, nn, s, launches);
    case 2: return minplus_impl<OpF32>(A, lda, B, ldb, Cm, ldc, m, k, nn, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace apsp
