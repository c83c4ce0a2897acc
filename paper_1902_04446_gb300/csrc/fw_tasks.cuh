// Phase bodies of one round of blocked Floyd-Warshall (the paper's Sec. 4.4/4.5,
// Alg. 3 and 4), as device functions shared by the per-round kernels
// (fw_kernels.cu) and the batched persistent kernel (batch.cu).
//
// Round k covers vertices [p0, p1) = [k*BK, min(n, (k+1)*BK)); w = p1 - p0.
//   phase1_body   Floyd-Warshall closure of D_kk (Table 1 FloydWarshall); also
//                 writes D_kk transposed into the panel buffer colT.
//   p2_row_task   D_kJ = min(D_kJ, D_kk (x) D_kJ) for one column chunk J.
//   p2_col_task   D_Ik = min(D_Ik, D_Ik (x) D_kk) for one row chunk I; writes
//                 the updated block transposed into colT.
//   p3_task       D_IJ = min(D_IJ, D_Ik (x) D_kJ) for one output tile, rows and
//                 columns of the panel excluded (Table 1 MatProd + MatMin).
// CG = true reads everything through L2 (ld.global.cg), which is required when
// the producer of the data ran earlier in the same launch.
#pragma once
#include "fw_device.cuh"

namespace apsp {

// Barrier policy of the phase bodies: the whole CTA (the per-round and batch
// kernels), or, in the warp-specialized Phase-3 kernel that runs next-round
// tasks on its consumer warps while the producer warp goes on, a bounded
// barrier over those warps (GroupBar in fw_kernels.cu).
struct CtaBar {
  __device__ __forceinline__ static void sync() { __syncthreads(); }
};

template <bool CG, class T>
__device__ __forceinline__ T ld_elem(const T *p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// ---------------------------------------------------------------- Phase 1
// Needs blockDim.x == NT (NT = 256) and BK * (BK + 4) scalars of shared memory.
// Thread (by, bx) of a 16 x 16 grid owns the PT x PT block of rows by*PT + r,
// columns bx*PT + c (PT = BK / 16) in registers.
template <class Op, int BK>
struct P1Smem {
  typename Op::scalar s[BK][BK + 4];
};

template <class Op, int BK, int NT, bool CG, class Bar = CtaBar>
__device__ __forceinline__ void phase1_body(typename Op::elem *__restrict__ D, Layout L, int64_t n, int64_t p0,
                                            uint32_t *__restrict__ colT, int64_t ldT, P1Smem<Op, BK> &sm, int tid,
                                            typename Op::elem *__restrict__ rowP = nullptr) {
  using S = typename Op::scalar;
  constexpr int G = 16;
  constexpr int PT = BK / G;
  static_assert(BK % G == 0 && NT == G * G, "phase 1 layout");
  auto &s = sm.s;
  const int by = tid / G, bx = tid % G;
  const S INF = Op::to_s(Op::inf_elem());
  {
    // all of this thread's loads first, then the shared-memory stores
    constexpr int IT = BK * BK / NT;
    S tmp[IT];
#pragma unroll
    for (int k = 0; k < IT; ++k) {
      const int idx = tid + k * NT;
      const int64_t r = p0 + idx / BK, c = p0 + idx % BK;
      tmp[k] = (r < n && c < n) ? Op::to_s(ld_elem<CG>(D + L.off(r, c))) : INF;
    }
#pragma unroll
    for (int k = 0; k < IT; ++k) {
      const int idx = tid + k * NT;
      s[idx / BK][idx % BK] = tmp[k];
    }
  }
  Bar::sync();
  S v[PT][PT];
#pragma unroll
  for (int r = 0; r < PT; ++r)
#pragma unroll
    for (int c = 0; c < PT; ++c) v[r][c] = s[by * PT + r][bx * PT + c];
  // The pivots are taken PT at a time, t0 = p*PT .. t0+PT-1 (the rows and
  // columns of thread block p): the net effect of those PT Floyd-Warshall steps
  // on entry (i, j) is min(D_ij, min_{s,s'} D_i,t0+s + K*_ss' + D_t0+s',j), K*
  // the closure of the PT x PT corner at (t0, t0).  Every thread closes K itself
  // (PT^3 add-mins), forms a' = a (x) K* for its rows (a = its pivot-column
  // values, kept with a' >= a, so every sum has two terms and cannot overflow)
  // and applies a' (x) b (b = the pivot-row values of its columns).  Then the
  // owners of the next pivot block's rows and columns write their blocks back,
  // and one barrier per pivot block (not per pivot) orders the steps.  A
  // write-back that lands while another thread still reads this block's
  // pivot column only replaces a value by its own update a', which gives the
  // same a' again (K* is closed).
#pragma unroll 1
  for (int p = 0; p < G; ++p) {
    const int t0 = p * PT;
    S K[PT][PT], a[PT][PT], b[PT][PT];
#pragma unroll
    for (int i = 0; i < PT; ++i)
#pragma unroll
      for (int j = 0; j < PT; ++j) {
        K[i][j] = s[t0 + i][t0 + j];
        a[i][j] = s[by * PT + i][t0 + j];
        b[i][j] = s[t0 + i][bx * PT + j];
      }
#pragma unroll
    for (int m = 0; m < PT; ++m)
#pragma unroll
      for (int i = 0; i < PT; ++i)
#pragma unroll
        for (int j = 0; j < PT; ++j) K[i][j] = Op::s_addmin(K[i][m], K[m][j], K[i][j]);
    S a2[PT][PT];
#pragma unroll
    for (int r = 0; r < PT; ++r)
#pragma unroll
      for (int j = 0; j < PT; ++j) {
        S x = a[r][j];
#pragma unroll
        for (int i = 0; i < PT; ++i) x = Op::s_addmin(a[r][i], K[i][j], x);
        a2[r][j] = x;
      }
#pragma unroll
    for (int r = 0; r < PT; ++r)
#pragma unroll
      for (int c = 0; c < PT; ++c)
#pragma unroll
        for (int j = 0; j < PT; ++j) v[r][c] = Op::s_addmin(a2[r][j], b[j][c], v[r][c]);
    if (p + 1 < G && (by == p + 1 || bx == p + 1)) {
#pragma unroll
      for (int r = 0; r < PT; ++r)
#pragma unroll
        for (int c = 0; c < PT; ++c) s[by * PT + r][bx * PT + c] = v[r][c];
    }
    Bar::sync();
  }
#pragma unroll
  for (int r = 0; r < PT; ++r)
#pragma unroll
    for (int c = 0; c < PT; ++c) s[by * PT + r][bx * PT + c] = v[r][c];
  Bar::sync();
  for (int idx = tid; idx < BK * BK; idx += NT) {
    const int i = idx / BK, j = idx % BK;
    const int64_t r = p0 + i, c = p0 + j;
    if (r < n && c < n) D[L.off(r, c)] = Op::from_s(s[i][j]);
  }
  for (int idx = tid; idx < BK * BK; idx += NT) {
    const int t = idx / BK, i = idx % BK;
    colT[t * ldT + p0 + i] = Op::dup(Op::from_s(s[i][t]));
  }
  if (rowP) {  // symmetric mode: the panel as elements (row t = D[p0 + t][.])
    for (int idx = tid; idx < BK * BK; idx += NT) {
      const int t = idx / BK, j = idx % BK;
      rowP[t * ldT + p0 + j] = Op::from_s(s[t][j]);
    }
  }
}

// ---------------------------------------------------------------- Phase 2
// Row panel chunk: output rows [p0, p0+BK), words [col0/EPW, col0/EPW + BNW).
// A = D_kk (from colT), B = C = the chunk itself.  Shared memory: BK*BK + BK*BNW words.
//
// Symmetric mode (sym != nullptr, undirected input): only columns >= p1 are
// updated (the upper triangle); the results also go to the symmetric panel
// (colT words, and sym->rowP elements for packed 16-bit) and, for columns
// below sym->band_end, to the lower-triangle column-panel element D[x][p0+t]
// (those lie in diagonal-band Phase-3 tiles, which are updated in full).
template <class Op>
struct SymPanel {
  typename Op::elem *rowP;  // BK x ldT elements (packed 16-bit only; nullptr otherwise)
  int64_t band_end;         // end of the Phase-3 tile column band that holds the diagonal block
};

// Per-element publication of a chunk that straddles p1 or n (out of line: rare).
template <class Op>
__device__ __noinline__ void sym_publish_slow(typename Op::elem *D, Layout L, int64_t n, int64_t p0, int64_t p1,
                                              uint32_t *colT, int64_t ldT, const SymPanel<Op> *sym, int t,
                                              int64_t x0, uint4 w4) {
  constexpr int E = 4 * Op::EPW;
  for (int e = 0; e < E; ++e) {
    const int64_t x = x0 + e;
    if (x < p1 || x >= n) continue;
    const typename Op::elem v = bits_elem<Op>(chunk_get<Op>(w4, e));
    colT[(int64_t)t * ldT + x] = Op::dup(v);
    if (sym->rowP) sym->rowP[(int64_t)t * ldT + x] = v;
    if (x < sym->band_end && p0 + t < n) D[L.off(x, p0 + t)] = v;
  }
}

// Lower-triangle band elements D[x][p0+t] of a full chunk (out of line: only
// the chunks next to the diagonal block have any).
template <class Op>
__device__ __noinline__ void sym_band_store(typename Op::elem *D, Layout L, int64_t col, int64_t band_end, int64_t x0,
                                            uint4 w4) {
  constexpr int E = 4 * Op::EPW;
  for (int e = 0; e < E; ++e)
    if (x0 + e < band_end) D[L.off(x0 + e, col)] = bits_elem<Op>(chunk_get<Op>(w4, e));
}

template <class Op, int BK, int BNW, int NT, bool CG, int TN = 8, class Bar = CtaBar>
__device__ __forceinline__ void p2_row_task(typename Op::elem *__restrict__ D, Layout L, int64_t n, int64_t p0,
                                            int64_t p1, uint32_t *__restrict__ colT, int64_t ldT, int64_t col0,
                                            bool vec, uint32_t *smem, int tid, const SymPanel<Op> *sym = nullptr) {
  using Map = TileMap<BK, BNW, TN>;
  static_assert(Map::THREADS == NT, "row tile");
  uint32_t *As = smem;
  uint32_t *Bs = smem + BK * BK;
  const int tx = tid % Map::TX, ty = tid / Map::TX;
  uint32_t acc[8][TN];
  load_As_colT<BK, BK, NT, CG>(As, colT, ldT, p0, tid);
  load_Bs_rows<Op, BNW, BK, NT, CG>(Bs, D, L, n, n, p0, col0, vec, tid);
  load_acc<Op, BK, BNW, CG, TN>(D, L, n, n, p0, col0, vec, acc, ty, tx);
  Bar::sync();
  tile_minplus<Op, BK, BNW, BK, TN>(As, Bs, acc, ty, tx);
  if (!sym) {
    store_acc<Op, BK, BNW, TN>(D, L, n, n, p0, col0, 0, 0, p0, p1, vec, acc, ty, tx);
    return;
  }
  store_acc<Op, BK, BNW, TN>(D, L, n, n, p0, col0, 0, 0, 0, p1, vec, acc, ty, tx);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int t = Map::row(ty, r);
#pragma unroll
    for (int h = 0; h < Map::NH; ++h) {
      const int64_t x0 = col0 + (int64_t)Map::wcol(tx, h) * Op::EPW;  // first element of these 4 words
      constexpr int E = 4 * Op::EPW;
      const uint4 w4 = make_uint4(acc[r][4 * h + 0], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
      if (x0 >= p1 && x0 + E <= n) {
        // the whole chunk is right of the diagonal block: 16-byte panel stores
        uint32_t *cw = colT + (int64_t)t * ldT + x0;
        if constexpr (Op::EPW == 1) {
          *reinterpret_cast<uint4 *>(cw) = w4;
        } else {
          *reinterpret_cast<uint4 *>(cw) = make_uint4(Op::dup(w4.x & 0xFFFFu), Op::dup(w4.x >> 16),
                                                      Op::dup(w4.y & 0xFFFFu), Op::dup(w4.y >> 16));
          *reinterpret_cast<uint4 *>(cw + 4) = make_uint4(Op::dup(w4.z & 0xFFFFu), Op::dup(w4.z >> 16),
                                                          Op::dup(w4.w & 0xFFFFu), Op::dup(w4.w >> 16));
          *reinterpret_cast<uint4 *>(sym->rowP + (int64_t)t * ldT + x0) = w4;
        }
        if (x0 < sym->band_end && p0 + t < n) sym_band_store<Op>(D, L, p0 + t, sym->band_end, x0, w4);
      } else if (x0 + E > p1 && x0 < n) {
        sym_publish_slow<Op>(D, L, n, p0, p1, colT, ldT, sym, t, x0, w4);
      }
    }
  }
}

// Symmetric mode: only rows < p0 are updated (the upper triangle); the
// panel_finalize pass then copies colT[t][x < p0] to the element panel and to
// the row panel's lower-triangle elements in the diagonal band.
// Transposed colT store of 4 rows of which some lie in the panel (out of line: rare).
static __device__ __noinline__ void colT_store_partial(uint32_t *dst, int64_t rb, int64_t p0, int64_t xr1, uint32_t q0,
                                                uint32_t q1, uint32_t q2, uint32_t q3) {
  const uint32_t q4[4] = {q0, q1, q2, q3};
  for (int q = 0; q < 4; ++q)
    if (rb + q < p0 || rb + q >= xr1) dst[q] = q4[q];
}

template <class Op, int BK, int BM, int NT, bool CG, int TN = 8, class Bar = CtaBar>
__device__ __forceinline__ void p2_col_task(typename Op::elem *__restrict__ D, Layout L, int64_t n, int64_t p0,
                                            int64_t p1, uint32_t *__restrict__ colT, int64_t ldT, int64_t row0,
                                            bool vec, uint32_t *smem, int tid, const SymPanel<Op> *sym = nullptr) {
  constexpr int BNW = BK / Op::EPW;
  using Map = TileMap<BM, BNW, TN>;
  static_assert(Map::THREADS == NT, "col tile");
  uint32_t *As = smem;
  uint32_t *Bs = smem + BK * BM;
  const int tx = tid % Map::TX, ty = tid / Map::TX;
  uint32_t acc[8][TN];
  load_As_transposed<Op, BM, BK, NT, CG>(As, D, L, n, n, row0, p0, vec, tid);
  load_Bs_rows<Op, BNW, BK, NT, CG>(Bs, D, L, n, n, p0, p0, vec, tid);
  load_acc<Op, BM, BNW, CG, TN>(D, L, n, n, row0, p0, vec, acc, ty, tx);
  Bar::sync();
  tile_minplus<Op, BM, BNW, BK, TN>(As, Bs, acc, ty, tx);
  // symmetric mode stores rows < p0 only
  const int64_t xr1 = sym ? INT64_MAX : p1;
  store_acc<Op, BM, BNW, TN>(D, L, n, n, row0, p0, p0, xr1, 0, 0, vec, acc, ty, tx);
  // transposed copy: colT[t][row0 + i] = word(D_Ik[i][t]) for rows outside [p0, p1)
#pragma unroll
  for (int h = 0; h < Map::NH; ++h) {
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int ib = Map::row(ty, 4 * g);  // 4 consecutive rows ib .. ib+3
      const int64_t rb = row0 + ib;
      const bool all_out = (rb + 3 < p0) || (rb >= xr1);
#pragma unroll
      for (int cw = 0; cw < 4; ++cw) {
        const int w = Map::wcol(tx, h) + cw;
#pragma unroll
        for (int lane = 0; lane < Op::EPW; ++lane) {
          const int t = w * Op::EPW + lane;
          uint32_t q4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t word = acc[4 * g + q][4 * h + cw];
            q4[q] = (Op::EPW == 2) ? Op::dup(bits_elem<Op>(lane ? (word >> 16) : (word & 0xFFFFu))) : word;
          }
          uint32_t *dst = colT + (int64_t)t * ldT + rb;
          if (all_out) *reinterpret_cast<uint4 *>(dst) = make_uint4(q4[0], q4[1], q4[2], q4[3]);
          else colT_store_partial(dst, rb, p0, xr1, q4[0], q4[1], q4[2], q4[3]);

        }
      }
    }
  }
}

// ---------------------------------------------------------------- Phase 3 (one tile)
// Output tile rows [row0, row0+128), words [col0/EPW, +128); 256 threads;
// shared memory 2 * BK * 128 words.
// symB (nullable): symmetric mode, B rows come from this BK x ldT panel of
// elements instead of D's row panel.
template <class Op, int BK, bool CG>
__device__ __forceinline__ void p3_task(typename Op::elem *__restrict__ D, Layout L, int64_t n, int64_t p0,
                                        int64_t p1, const uint32_t *__restrict__ colT, int64_t ldT, int64_t row0,
                                        int64_t col0, bool vec, uint32_t *smem, int tid,
                                        const typename Op::elem *symB = nullptr) {
  constexpr int BM = 128, BNW = 128, NT = 256;
  using Map = TileMap<BM, BNW>;
  uint32_t *As = smem;
  uint32_t *Bs = smem + BK * BM;
  const int tx = tid % Map::TX, ty = tid / Map::TX;
  uint32_t acc[8][8];
  load_As_colT<BM, BK, NT, CG>(As, colT, ldT, row0, tid);
  if (symB)
    load_Bs_rows<Op, BNW, BK, NT, CG>(Bs, symB, ldT, BK, ldT, 0, col0, true, tid);
  else
    load_Bs_rows<Op, BNW, BK, NT, CG>(Bs, D, L, n, n, p0, col0, vec, tid);
  load_acc<Op, BM, BNW, CG>(D, L, n, n, row0, col0, vec, acc, ty, tx);
  __syncthreads();
  tile_minplus<Op, BM, BNW, BK>(As, Bs, acc, ty, tx);
  store_acc<Op, BM, BNW>(D, L, n, n, row0, col0, p0, p1, p0, p1, vec, acc, ty, tx);
}

}  // namespace apsp
