// Device-side building blocks of the blocked Floyd-Warshall kernels (sm_103a).
//
// Three storage modes share one code path through a "word" abstraction: every
// kernel moves and computes 32-bit words.
//   OpI32  one int32 distance per word, add-min = __viaddmin_s32
//   OpU16  two unsigned 16-bit distances per word (element 2w in the low half),
//          add-min = __viaddmin_u16x2 (two relaxations per lane-op)
//   OpF32  one fp32 distance per word, add-min = fminf(a + b, c)
// The relaxation is the min-plus step of the paper's Table 1 (MatProd followed
// by MatMin): c = min(c, a + b).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace apsp {

struct OpI32 {
  using elem = int32_t;
  static constexpr int EPW = 1;                 // elements per 32-bit word
  static constexpr uint32_t INF_WORD = 1073741823u;
  static constexpr int DTYPE = 0;
  __device__ __forceinline__ static uint32_t addmin(uint32_t a, uint32_t b, uint32_t c) {
    return (uint32_t)__viaddmin_s32((int)a, (int)b, (int)c);
  }
  // A-operand word for one element (same value in every lane of the word)
  __device__ __forceinline__ static uint32_t dup(elem e) { return (uint32_t)e; }
  __device__ __forceinline__ static elem inf_elem() { return (elem)1073741823; }
  // scalar arithmetic for the diagonal closure
  using scalar = int32_t;
  __device__ __forceinline__ static scalar to_s(elem e) { return e; }
  __device__ __forceinline__ static elem from_s(scalar s) { return s; }
  __device__ __forceinline__ static scalar s_addmin(scalar a, scalar b, scalar c) { return __viaddmin_s32(a, b, c); }
};

struct OpU16 {
  using elem = uint16_t;
  static constexpr int EPW = 2;
  static constexpr uint32_t INF_WORD = 0x7FFF7FFFu;
  static constexpr int DTYPE = 1;
  __device__ __forceinline__ static uint32_t addmin(uint32_t a, uint32_t b, uint32_t c) {
    return __viaddmin_u16x2(a, b, c);
  }
  __device__ __forceinline__ static uint32_t dup(elem e) { return (uint32_t)e | ((uint32_t)e << 16); }
  __device__ __forceinline__ static elem inf_elem() { return (elem)0x7FFF; }
  using scalar = int32_t;
  __device__ __forceinline__ static scalar to_s(elem e) { return (scalar)e; }
  __device__ __forceinline__ static elem from_s(scalar s) { return (elem)s; }
  // stored values are <= 0x7FFF, so a + b <= 0xFFFE and min() keeps <= 0x7FFF
  __device__ __forceinline__ static scalar s_addmin(scalar a, scalar b, scalar c) { return __viaddmin_s32(a, b, c); }
};

struct OpF32 {
  using elem = float;
  static constexpr int EPW = 1;
  static constexpr uint32_t INF_WORD = 0x7F800000u;
  static constexpr int DTYPE = 2;
  __device__ __forceinline__ static uint32_t addmin(uint32_t a, uint32_t b, uint32_t c) {
    return __float_as_uint(fminf(__uint_as_float(a) + __uint_as_float(b), __uint_as_float(c)));
  }
  __device__ __forceinline__ static uint32_t dup(elem e) { return __float_as_uint(e); }
  __device__ __forceinline__ static elem inf_elem() { return __int_as_float(0x7F800000); }
  using scalar = float;
  __device__ __forceinline__ static scalar to_s(elem e) { return e; }
  __device__ __forceinline__ static elem from_s(scalar s) { return s; }
  __device__ __forceinline__ static scalar s_addmin(scalar a, scalar b, scalar c) { return fminf(a + b, c); }
};

// ---------------------------------------------------------------------------
// Where element (r, c) of the distance matrix D lives.
//
// Dense (the default; an int64_t leading dimension converts to it): row-major,
// D[r * ld + c].
//
// Upper-triangular storage (the paper keeps only the upper triangle of blocks,
// Sec. 4; the lower blocks are transposes): the matrix is cut into S x S
// super-tiles, S = 128 * EPW elements (one Phase-3 tile column wide, one or two
// tile rows tall), T = ceil(n / S) per side, and only the super-tiles (I, J)
// with I <= J are stored -- the diagonal super-tiles in full.  They are folded
// into one rectangle of Th * S rows and (2 Th + 1) * S elements per row
// (Th = ceil(T / 2); about n^2 / 2 elements), so that every stored row is
// contiguous and the rectangle has one row pitch (one TMA tensor map covers
// it):
//   super-row I <  Th: rectangle rows I*S.., columns shifted right by S
//                      (logical columns [I S, T S) -> [(I+1) S, (T+1) S));
//   super-row I >= Th: rectangle rows (2 Th - 1 - I)*S.., columns shifted left
//                      by I S (logical [I S, T S) -> [0, (T - I) S)), in the
//                      part that the top super-row of that rectangle row
//                      leaves free.
// Element (r, c) is stored when c >= S * floor(r / S); rows and columns in
// [n, T S) are padding.
struct Layout {
  int64_t ld;  // dense: leading dimension; upper-triangular: the rectangle's row pitch (elements)
  int32_t sh;  // upper-triangular: log2(S)
  int32_t Th;  // upper-triangular: super-rows in the top half (0 = dense)
  int32_t T;   // upper-triangular: super-tiles per side
  __host__ __device__ Layout(int64_t ld_ = 0) : ld(ld_), sh(0), Th(0), T(0) {}
  __host__ __device__ __forceinline__ bool tri() const { return Th != 0; }
  // rectangle row and column of logical element (r, c) (dense: (r, c) itself)
  __host__ __device__ __forceinline__ void phys(int64_t r, int64_t c, int64_t &pr, int64_t &pc) const {
    if (Th == 0) {
      pr = r;
      pc = c;
      return;
    }
    const int64_t I = r >> sh;
    if (I < Th) {
      pr = r;
      pc = c + (int64_t(1) << sh);
    } else {
      pr = r + ((2 * (int64_t)Th - 1 - 2 * I) << sh);
      pc = c - (I << sh);
    }
  }
  __host__ __device__ __forceinline__ int64_t off(int64_t r, int64_t c) const {
    if (Th == 0) return r * ld + c;
    int64_t pr, pc;
    phys(r, c, pr, pc);
    return pr * ld + pc;
  }
  // one past the last stored logical column of every row
  __host__ __device__ __forceinline__ int64_t row_end() const { return Th == 0 ? ld : ((int64_t)T << sh); }
  // whether logical element (r, c) is stored
  __host__ __device__ __forceinline__ bool stored(int64_t r, int64_t c) const {
    return Th == 0 || (c >> sh) >= (r >> sh);
  }
};

// The upper-triangular layout of an n x n matrix with `epw` elements per
// 32-bit word; *rows = the rectangle's rows (its size is rows * L.ld elements).
inline Layout tri_layout(int64_t n, int epw, int64_t *rows) {
  const int sh = epw == 2 ? 8 : 7;
  const int64_t S = int64_t(1) << sh;
  const int64_t T = ((n > 0 ? n : 1) + S - 1) >> sh;
  const int64_t Th = (T + 1) / 2;
  Layout L((2 * Th + 1) * S);
  L.sh = sh;
  L.Th = (int32_t)Th;
  L.T = (int32_t)T;
  if (rows) *rows = Th * S;
  return L;
}

// ---------------------------------------------------------------------------
// element <-> word helpers
template <class Op>
__device__ __forceinline__ uint32_t elem_bits(typename Op::elem e) {
  if constexpr (Op::EPW == 2) return (uint32_t)e;
  else if constexpr (Op::DTYPE == 2) return __float_as_uint(e);
  else return (uint32_t)e;
}
template <class Op>
__device__ __forceinline__ typename Op::elem bits_elem(uint32_t b) {
  if constexpr (Op::EPW == 2) return (typename Op::elem)(b & 0xFFFFu);
  else if constexpr (Op::DTYPE == 2) return __uint_as_float(b);
  else return (typename Op::elem)b;
}

// Element e (0 .. 4*EPW-1) of a 4-word chunk.
template <class Op>
__device__ __forceinline__ uint32_t chunk_get(const uint4 &v, int e) {
  uint32_t w = (e / Op::EPW == 0) ? v.x : (e / Op::EPW == 1) ? v.y : (e / Op::EPW == 2) ? v.z : v.w;
  if constexpr (Op::EPW == 2) return (e & 1) ? (w >> 16) : (w & 0xFFFFu);
  else return w;
}
template <class Op>
__device__ __forceinline__ void chunk_set(uint4 &v, int e, uint32_t bits) {
  uint32_t *w = (e / Op::EPW == 0) ? &v.x : (e / Op::EPW == 1) ? &v.y : (e / Op::EPW == 2) ? &v.z : &v.w;
  if constexpr (Op::EPW == 2) {
    if (e & 1) *w = (*w & 0x0000FFFFu) | (bits << 16);
    else *w = (*w & 0xFFFF0000u) | (bits & 0xFFFFu);
  } else {
    *w = bits;
  }
}

// Loads 4 words (4*EPW elements) of row r starting at element column c0 of a
// row-major matrix with leading dimension ld.  Elements outside
// [0, nrows) x [0, ncols) read as INF.  `vec` says that the matrix base is
// 16-byte aligned and ld * sizeof(elem) is a multiple of 16, so that a chunk
// starting at a multiple of 4*EPW is one aligned 16-byte access inside row r
// (the row holds ld >= ncols elements).
// CG = true reads through L2 only (ld.global.cg): required for data that other
// CTAs of the same launch wrote (the batched persistent kernel); otherwise the
// read-only path is used.
template <bool CG>
__device__ __forceinline__ uint4 ld16(const void *p) {
  if constexpr (CG) return __ldcg(reinterpret_cast<const uint4 *>(p));
  else return __ldg(reinterpret_cast<const uint4 *>(p));
}

// Per-element path of load_chunk (a chunk that crosses the matrix edge, or an
// unaligned matrix).  Kept out of line: it is rare, and inlining it into every
// tile loop makes the kernels too large for the instruction cache.
template <class Op, bool CG>
__device__ __noinline__ uint4 load_chunk_slow(const typename Op::elem *M, Layout L, int64_t ncols, int64_t r,
                                              int64_t c0, bool vec) {
  constexpr int E = 4 * Op::EPW;
  uint4 v = make_uint4(Op::INF_WORD, Op::INF_WORD, Op::INF_WORD, Op::INF_WORD);
  const typename Op::elem *p = M + L.off(r, c0);
  if (vec && c0 + E <= L.row_end()) {
    v = ld16<CG>(p);
    for (int e = 0; e < E; ++e)
      if (c0 + e >= ncols) chunk_set<Op>(v, e, elem_bits<Op>(Op::inf_elem()));
  } else {
    for (int e = 0; e < E; ++e)
      if (c0 + e < ncols) {
        if constexpr (CG) chunk_set<Op>(v, e, elem_bits<Op>(__ldcg(p + e)));
        else chunk_set<Op>(v, e, elem_bits<Op>(p[e]));
      }
  }
  return v;
}

template <class Op, bool CG = false>
__device__ __forceinline__ uint4 load_chunk(const typename Op::elem *M, Layout L, int64_t nrows, int64_t ncols,
                                            int64_t r, int64_t c0, bool vec) {
  constexpr int E = 4 * Op::EPW;
  if (r < 0 || r >= nrows || c0 >= ncols)
    return make_uint4(Op::INF_WORD, Op::INF_WORD, Op::INF_WORD, Op::INF_WORD);
  if (vec && c0 + E <= ncols) return ld16<CG>(M + L.off(r, c0));  // the common case: one 16-byte load
  return load_chunk_slow<Op, CG>(M, L, ncols, r, c0, vec);
}

// Per-element path of store_chunk, out of line for the same reason.
template <class Op>
__device__ __noinline__ void store_chunk_slow(typename Op::elem *p, uint4 v, uint32_t mask) {
  constexpr int E = 4 * Op::EPW;
  for (int e = 0; e < E; ++e)
    if (mask & (1u << e)) p[e] = bits_elem<Op>(chunk_get<Op>(v, e));
}

// Stores the elements of a 4-word chunk whose mask bit is set (bit e for
// element e).  A full mask with `vec` is one 16-byte store.
template <class Op>
__device__ __forceinline__ void store_chunk(typename Op::elem *M, Layout L, int64_t r, int64_t c0, uint4 v,
                                            uint32_t mask, bool vec) {
  constexpr int E = 4 * Op::EPW;
  constexpr uint32_t FULL = (1u << E) - 1u;
  if (mask == 0) return;
  typename Op::elem *p = M + L.off(r, c0);
  if (vec && mask == FULL) *reinterpret_cast<uint4 *>(p) = v;
  else store_chunk_slow<Op>(p, v, mask);
}

// Mask of the elements c0 .. c0+E-1 that lie in [0, ncols) and outside the
// excluded column range [x0, x1).
template <class Op>
__device__ __forceinline__ uint32_t col_mask(int64_t c0, int64_t ncols, int64_t x0, int64_t x1) {
  constexpr int E = 4 * Op::EPW;
  uint32_t m = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    int64_t c = c0 + e;
    if (c < ncols && (c < x0 || c >= x1)) m |= 1u << e;
  }
  return m;
}

// ---------------------------------------------------------------------------
// Register-blocked min-plus tile.
//
// A CTA of (BM/8) x (BNW/8) threads owns a BM x BNW-word output tile; thread
// (ty, tx) holds an 8 x 8 word block: rows {ty*4 + 0..3} and
// {BM/2 + ty*4 + 0..3}, word columns {tx*4 + 0..3} and {BNW/2 + tx*4 + 0..3},
// so that every operand fetch is one 16-byte shared-memory load and a warp's
// B fetch covers 256 contiguous bytes (no bank conflicts).
//   As[t][i]  (BK x BM words)  A operand, transposed, each element duplicated
//                              over the lanes of its word
//   Bs[t][w]  (BK x BNW words) B operand
//   acc[r][c] += min-plus over t:  acc = min(acc, As[t][row r] + Bs[t][col c])
template <int BM, int BNW, int TN = 8>
struct TileMap {
  static_assert(TN == 8 || TN == 4, "8 or 4 words per thread and row");
  static constexpr int TX = BNW / TN;
  static constexpr int TY = BM / 8;
  static constexpr int THREADS = TX * TY;
  static constexpr int NH = TN / 4;  // 16-byte column chunks per thread and row
  __device__ __forceinline__ static int row(int ty, int r) { return (r < 4) ? (ty * 4 + r) : (BM / 2 + ty * 4 + r - 4); }
  __device__ __forceinline__ static int wcol(int tx, int h) { return h == 0 ? tx * 4 : BNW / 2 + tx * 4; }
};

// Three-input minimum of fp32 values (sm_100 and later).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
// fp32 min-plus tile, two k-steps at a time: acc = min(acc, a_t + b_t,
// a_t+1 + b_t+1) with one three-input minimum, the sums for two neighbouring
// columns formed by one packed pair add -- the same sums (each rounded to
// nearest) and the same minimum as one add and one minimum per relaxation,
// in fewer instructions.
// U = k-step pairs per unrolled loop trip, chosen per kernel (measured on
// GB300: every round in one launch 4, the per-round Phase 3 2, the min-plus
// product 1; their register use and schedules differ).
template <int BM, int BNW, int BK, int TN, int U>
__device__ __forceinline__ void tile_minplus_f32(const uint32_t *__restrict__ As, const uint32_t *__restrict__ Bs,
                                                 uint32_t (&acc)[8][TN], int ty, int tx) {
  static_assert(BK % 2 == 0, "k-steps in pairs");
  float f[8][TN];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) f[r][c] = __uint_as_float(acc[r][c]);
  constexpr int UNROLL = TN == 8 ? U : 2;
#pragma unroll UNROLL
  for (int t = 0; t < BK; t += 2) {
    float a[2][8];
    uint64_t b[2][TN / 2];  // neighbouring columns (c, c + 1) as one packed pair
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint4 a0 = *reinterpret_cast<const uint4 *>(As + (t + k) * BM + ty * 4);
      const uint4 a1 = *reinterpret_cast<const uint4 *>(As + (t + k) * BM + BM / 2 + ty * 4);
      a[k][0] = __uint_as_float(a0.x); a[k][1] = __uint_as_float(a0.y);
      a[k][2] = __uint_as_float(a0.z); a[k][3] = __uint_as_float(a0.w);
      a[k][4] = __uint_as_float(a1.x); a[k][5] = __uint_as_float(a1.y);
      a[k][6] = __uint_as_float(a1.z); a[k][7] = __uint_as_float(a1.w);
#pragma unroll
      for (int h = 0; h < TN / 4; ++h) {
        const ulonglong2 bv =
            *reinterpret_cast<const ulonglong2 *>(Bs + (t + k) * BNW + (h == 0 ? tx * 4 : BNW / 2 + tx * 4));
        b[k][2 * h + 0] = bv.x;
        b[k][2 * h + 1] = bv.y;
      }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      uint64_t ad[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) asm("mov.b64 %0, {%1, %1};" : "=l"(ad[k]) : "f"(a[k][r]));
#pragma unroll
      for (int p = 0; p < TN / 2; ++p) {
        uint64_t s0, s1;
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s0) : "l"(ad[0]), "l"(b[0][p]));
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s1) : "l"(ad[1]), "l"(b[1][p]));
        float x0, y0, x1, y1;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x0), "=f"(y0) : "l"(s0));
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x1), "=f"(y1) : "l"(s1));
        f[r][2 * p] = fmin3(f[r][2 * p], x0, x1);
        f[r][2 * p + 1] = fmin3(f[r][2 * p + 1], y0, y1);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[r][c] = __float_as_uint(f[r][c]);
}

template <class Op, int BM, int BNW, int BK, int TN = 8, int F32U = 2>
__device__ __forceinline__ void tile_minplus(const uint32_t *__restrict__ As, const uint32_t *__restrict__ Bs,
                                             uint32_t (&acc)[8][TN], int ty, int tx) {
  if constexpr (Op::DTYPE == 2) {
    tile_minplus_f32<BM, BNW, BK, TN, F32U>(As, Bs, acc, ty, tx);
    return;
  }
  // deeper unrolling for the 8 x 8 block (fewer loop instructions on the
  // add-min pipe): for the integer ops 16 k-steps per loop trip measured
  // fastest (8: 1.1 % slower on an n = 16384 int32 solve; 32 and 64: 1.5 % and
  // 4.7 % slower, the longer bodies costing instruction fetch); fp32, two
  // instructions per relaxation, was 2.7 % slower at 16 than at 8; the 8 x 4
  // block of the 512-thread kernel must stay within 128 registers
  constexpr int UNROLL = TN == 8 ? (Op::DTYPE == 2 ? 8 : 16) : 4;
#pragma unroll UNROLL
  for (int t = 0; t < BK; ++t) {
    const uint4 a0 = *reinterpret_cast<const uint4 *>(As + t * BM + ty * 4);
    const uint4 a1 = *reinterpret_cast<const uint4 *>(As + t * BM + BM / 2 + ty * 4);
    const uint32_t a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    uint32_t b[TN];
#pragma unroll
    for (int h = 0; h < TN / 4; ++h) {
      const uint4 bv = *reinterpret_cast<const uint4 *>(Bs + t * BNW + (h == 0 ? tx * 4 : BNW / 2 + tx * 4));
      b[4 * h + 0] = bv.x;
      b[4 * h + 1] = bv.y;
      b[4 * h + 2] = bv.z;
      b[4 * h + 3] = bv.w;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < TN; ++c) acc[r][c] = Op::addmin(a[r], b[c], acc[r][c]);
  }
}

// Loads the thread's 8 x 8 word block of the output tile whose top-left
// element is (row0, col0) from M (INF outside [0,nrows) x [0,ncols)).
template <class Op, int BM, int BNW, bool CG = false, int TN = 8>
__device__ __forceinline__ void load_acc(const typename Op::elem *M, Layout L, int64_t nrows, int64_t ncols,
                                         int64_t row0, int64_t col0, bool vec, uint32_t (&acc)[8][TN], int ty,
                                         int tx) {
  using Map = TileMap<BM, BNW, TN>;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
#pragma unroll
    for (int h = 0; h < Map::NH; ++h) {
      const uint4 v = load_chunk<Op, CG>(M, L, nrows, ncols, row0 + Map::row(ty, r),
                                         col0 + (int64_t)Map::wcol(tx, h) * Op::EPW, vec);
      acc[r][4 * h + 0] = v.x;
      acc[r][4 * h + 1] = v.y;
      acc[r][4 * h + 2] = v.z;
      acc[r][4 * h + 3] = v.w;
    }
  }
}

// Stores the thread's block: row r is written when it lies in [0, nrows) and
// outside [xr0, xr1); an element column when it lies in [0, ncols) and outside
// [xc0, xc1).
// Stores an interior tile (every element inside the matrix, none excluded)
// with unconditional 16-byte stores; needs `vec`.
template <class Op, int BM, int BNW, int TN = 8>
__device__ __forceinline__ void store_acc_interior(typename Op::elem *M, Layout L, int64_t row0, int64_t col0,
                                                   const uint32_t (&acc)[8][TN], int ty, int tx) {
  using Map = TileMap<BM, BNW, TN>;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    typename Op::elem *rowp = M + L.off(row0 + Map::row(ty, r), col0);
#pragma unroll
    for (int h = 0; h < Map::NH; ++h)
      *reinterpret_cast<uint4 *>(rowp + (int64_t)Map::wcol(tx, h) * Op::EPW) =
          make_uint4(acc[r][4 * h + 0], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
  }
}

template <class Op, int BM, int BNW, int TN = 8>
__device__ __forceinline__ void store_acc(typename Op::elem *M, Layout L, int64_t nrows, int64_t ncols,
                                          int64_t row0, int64_t col0, int64_t xr0, int64_t xr1, int64_t xc0,
                                          int64_t xc1, bool vec, const uint32_t (&acc)[8][TN], int ty, int tx) {
  using Map = TileMap<BM, BNW, TN>;
#pragma unroll
  for (int h = 0; h < Map::NH; ++h) {
    const int64_t c0 = col0 + (int64_t)Map::wcol(tx, h) * Op::EPW;
    const uint32_t cm = col_mask<Op>(c0, ncols, xc0, xc1);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int64_t row = row0 + Map::row(ty, r);
      if (row >= nrows || (row >= xr0 && row < xr1)) continue;
      const uint4 v = make_uint4(acc[r][4 * h + 0], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
      store_chunk<Op>(M, L, row, c0, v, cm, vec);
    }
  }
}

// The loaders below issue all of a thread's global loads before the first
// shared-memory store (compile-time trip counts, fully unrolled in batches of
// up to 8), so their latencies overlap instead of adding up.

// As[t][i] = colT[t][i0 + i] for t < BK, i < BM (colT rows are aligned words).
template <int BM, int BK, int NT, bool CG = false>
__device__ __forceinline__ void load_As_colT(uint32_t *As, const uint32_t *__restrict__ colT, int64_t ldT, int64_t i0,
                                             int tid) {
  constexpr int CH = BK * BM / 4;
  static_assert(CH % NT == 0, "chunk count");
  constexpr int IT = CH / NT, BATCH = IT < 8 ? IT : 8;
#pragma unroll
  for (int k0 = 0; k0 < IT; k0 += BATCH) {
    uint4 v[BATCH];
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int c = tid + (k0 + k) * NT;
      v[k] = ld16<CG>(colT + (c / (BM / 4)) * ldT + i0 + (c % (BM / 4)) * 4);
    }
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int c = tid + (k0 + k) * NT;
      *reinterpret_cast<uint4 *>(As + (c / (BM / 4)) * BM + (c % (BM / 4)) * 4) = v[k];
    }
  }
}

// Bs[t][w] = word w of row (r0 + t), element columns c0 .. c0 + BNW*EPW.
template <class Op, int BNW, int BK, int NT, bool CG = false>
__device__ __forceinline__ void load_Bs_rows(uint32_t *Bs, const typename Op::elem *__restrict__ M, Layout L,
                                             int64_t nrows, int64_t ncols, int64_t r0, int64_t c0, bool vec,
                                             int tid) {
  constexpr int CH = BK * BNW / 4;
  static_assert(CH % NT == 0, "chunk count");
  constexpr int IT = CH / NT, BATCH = IT < 8 ? IT : 8;
#pragma unroll
  for (int k0 = 0; k0 < IT; k0 += BATCH) {
    uint4 v[BATCH];
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int c = tid + (k0 + k) * NT;
      v[k] = load_chunk<Op, CG>(M, L, nrows, ncols, r0 + c / (BNW / 4), c0 + (int64_t)((c % (BNW / 4)) * 4) * Op::EPW,
                                vec);
    }
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int c = tid + (k0 + k) * NT;
      *reinterpret_cast<uint4 *>(Bs + (c / (BNW / 4)) * BNW + (c % (BNW / 4)) * 4) = v[k];
    }
  }
}

// As[t][i] = dup(M[i0 + i][c0 + t]) for t < BK, i < BM: a transposing load of a
// BM x BK block (consecutive threads take consecutive rows, so the scalar
// shared-memory stores hit consecutive banks).
template <class Op, int BM, int BK, int NT, bool CG = false>
__device__ __forceinline__ void load_As_transposed(uint32_t *As, const typename Op::elem *__restrict__ M, Layout L,
                                                   int64_t nrows, int64_t ncols, int64_t i0, int64_t c0, bool vec,
                                                   int tid) {
  constexpr int E = 4 * Op::EPW;
  constexpr int CH = BM * (BK / E);
  static_assert(CH % NT == 0, "chunk count");
  constexpr int IT = CH / NT, BATCH = IT < 8 ? IT : 8;
#pragma unroll
  for (int k0 = 0; k0 < IT; k0 += BATCH) {
    uint4 v[BATCH];
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int c = tid + (k0 + k) * NT;
      v[k] = load_chunk<Op, CG>(M, L, nrows, ncols, i0 + c % BM, c0 + (c / BM) * E, vec);
    }
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const int c = tid + (k0 + k) * NT;
      const int i = c % BM, tq = (c / BM) * E;
#pragma unroll
      for (int e = 0; e < E; ++e) As[(tq + e) * BM + i] = Op::dup(bits_elem<Op>(chunk_get<Op>(v[k], e)));
    }
  }
}

}  // namespace apsp
