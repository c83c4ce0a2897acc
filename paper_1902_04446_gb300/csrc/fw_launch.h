// Internal launchers shared by the C-ABI layer (not part of the public ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace apsp {

// Optional per-phase timing hook: launch_rounds calls before()/after() around
// every phase launch on the launch stream (phase 0, 1, 2 = Phase 1, 2, 3) and
// passes the phase's algorithmic relaxation count.
struct PhaseTimer {
  virtual void before(int phase, cudaStream_t s) = 0;
  virtual void after(int phase, cudaStream_t s, double relaxations) = 0;
  // the count depends on a mode decided on the device: relax_sym when the int
  // at dflag is 0 (symmetric), relax_gen otherwise
  virtual void after_choice(int phase, cudaStream_t s, double relax_sym, double relax_gen, const int *dflag) {
    (void)dflag;
    after(phase, s, relax_gen);
  }
  virtual ~PhaseTimer() {}
};

// Tunable shape of the rounds: round width Bk (32, 64 or 128) and the Phase-3
// kernel: 0 = one CTA per tile, 1 = persistent TMA kernel with 256 threads
// (8 x 8 words each), 2 = persistent TMA kernel with 512 threads (8 x 4 words
// each), 3 = warp-specialized persistent kernel (8 consumer warps with 8 x 8
// words each and a TMA producer warp; int32 results leave by a TMA
// min-reduction), one launch per round, 4 = the same kernel running every
// round in one launch, each round's Phase 1 and Phase 2 as tasks inside it
// (fw_solve_ws; round width 64, needs the double panel buffer of
// panel_buffer_bytes(n, ldT, true); otherwise it falls back to 3).  The TMA
// kernels need a 16-byte addressable matrix and fall back to 0 otherwise.
// Round width 128 runs kernels 0 and 3 (1 and 2 run as 3): kernel 3 then
// takes each tile's 128 k-steps as two 64-step stages.
// sym: symmetric mode for undirected (symmetric) inputs -- Phase 3 updates
// only the tiles that touch the upper triangle, both of its operands come from
// one symmetric panel, and a final pass mirrors the upper triangle into the
// lower; rowP is the BK x ldT element panel that packed 16-bit needs for it
// (row_panel_bytes(ldT, p3 == 4)).
// sym_flag (device int, kernel 4 only): the symmetric mode is decided on the
// device -- symmetric when the int is 0 (as left by launch_symmetry_check) --
// so the host need not wait for the check; rowP must then be allocated.
struct RoundConfig {
  int bk = 64;
  int p3 = 3;
  bool sym = false;
  void *rowP = nullptr;
  const int *sym_flag = nullptr;
  const int *gate = nullptr;  // kernel 4 only: round 0's Phase 1 also waits for *gate >= 1
  uint32_t dep_spins = 0;     // kernel 4 only: limit of each wait on another work item (0 = default)
  int grid_cap = 0;           // persistent Phase-3 kernels: at most this many CTAs (0 = one per SM), so that
                              // solves on other streams can run on the remaining SMs
};
// Whether launch_rounds would run every round in one launch for this call
// (kernel 4 with round width 64, a 16-byte addressable D and more than one round).
bool single_launch(int dtype, const void *D, int64_t ld, int64_t n, const RoundConfig &cfg);
// The default Phase-3 kernel for (n, dtype) when nothing was tuned: every round
// in one launch for mid-size n, one launch per round below and above (timed per
// n and dtype on GB300, the per-round kernels with programmatic dependent
// launch).  Below the lower cut a round is at most a few waves of tiles and the
// per-round launches are cheaper than the single launch's item scheduling;
// above the upper cut the per-round launches' fixed cost per round is small
// against the single launch's cost per tile.  Measured (symmetric mode, ms per
// solve, one launch per round / single launch): int32 n = 5120 6.52 / 6.89,
// 6144 9.89 / 8.62, 16384 128.4 / 125.6, 32768 954 / 975; packed 16-bit
// n = 5120 5.48 / 6.23, 6144 8.05 / 7.66, 65536 3922 / 3983 (its rounds have
// half the tiles); fp32 n = 5120 6.39 / 6.82, 6144 9.60 / 8.55.
inline int default_phase3(int64_t n, int dtype) {
  const int64_t hi = dtype == 1 ? 49152 : 24576;
  return n >= 6144 && n < hi ? 4 : 3;
}
// The default round width for (n, dtype): 128 where large n runs one launch
// per round in packed 16-bit or fp32 (each tile then takes 128 k-steps in two
// stages and stores its C block half as often), else 64.  Measured (symmetric
// mode, ms per solve, width 64 / 128): fp32 n = 65536 7177 / 6967, packed
// 16-bit n = 65536 3931 / 3910, n = 32768 528 / 519; int32 n = 65536 7486 /
// 7550 (its k-loop runs slower in the two-stage kernel than the epilogue
// saves), and every element type at small n, where the 128-wide Phase 1 on
// one SM is on the critical path (int32 n = 4096 4.07 / 5.24).
inline int default_round_width(int64_t n, int dtype) {
  return dtype != 0 && default_phase3(n, dtype) == 3 && n >= 6144 ? 128 : 64;
}

// flag |= 1 when D (n x n, leading dimension ld) is not symmetric.
cudaError_t launch_symmetry_check(int dtype, const void *D, int64_t n, int64_t ld, int *flag, cudaStream_t s);
constexpr int64_t kMaxRoundWidth = 128;  // panel buffers are sized for this (the widest round)

// Bytes of the colT panel buffer launch_rounds needs for n (ldT = its row
// pitch in words): one kMaxRoundWidth x ldT panel of 32-bit words, or for
// Phase-3 kernel 4 (every round in one launch, `all_rounds`) two of them, a
// 64-bit item counter, 6 counters per round (round width >= 32) and one per
// Phase-3 tile.
inline size_t lookahead_counter_offset(int64_t ldT) { return 2 * (size_t)kMaxRoundWidth * (size_t)ldT * 4; }
inline size_t panel_buffer_bytes(int64_t n, int64_t ldT, bool all_rounds) {
  const size_t one = (size_t)kMaxRoundWidth * (size_t)ldT * 4;
  if (!all_rounds) return one;
  const size_t rounds = (size_t)((n + 31) / 32) + 1;
  const size_t tiles = (size_t)((n + 127) / 128) * (size_t)((n + 127) / 128);
  return 2 * one + 16 + sizeof(int) * (6 * rounds + tiles);
}
// Bytes of the element panel (symmetric mode, packed 16-bit).
inline size_t row_panel_bytes(int64_t ldT, bool all_rounds) {
  return (all_rounds ? 2 : 1) * (size_t)kMaxRoundWidth * (size_t)ldT * 2;
}

// q rounds of Phase 1 -> Phase 2 -> Phase 3 on D (n x n, leading dimension ld).
// colT is the panel buffer (panel_buffer_bytes(n, ldT, cfg.p3 == 4) bytes),
// ldT a multiple of 256 and >= n; cfg.rowP the element panel when needed.
// wait_err: device word that the persistent Phase-3 kernel ORs 4 into when a
// bounded wait gives up; nullptr = a per-device word the library allocates on
// first use.
cudaError_t launch_rounds(int dtype, void *D, int64_t ld, int64_t n, void *colT, int64_t ldT, cudaStream_t s,
                          int64_t *launches, PhaseTimer *timer = nullptr, const RoundConfig &cfg = RoundConfig(),
                          int *wait_err = nullptr);
// Upper-triangular storage (the Layout of fw_device.cuh): only the S x S
// super-tiles (I, J) with I <= J of the n x n matrix are stored (S = 128
// elements per word lane: 128 for int32/fp32, 256 for packed 16-bit), folded
// into a rectangle of *rows rows with row pitch *ld elements.
void tri_shape(int64_t n, int dtype, int64_t *rows, int64_t *ld);
// q rounds on T in that layout, symmetric mode, warp-specialized Phase 3 one
// launch per round (cfg.bk and cfg.rowP are used; the other fields are set here).
cudaError_t launch_rounds_tri(int dtype, void *T, int64_t n, void *colT, int64_t ldT, cudaStream_t s,
                              int64_t *launches, PhaseTimer *timer, RoundConfig cfg, int *wait_err);
// T <- the stored part of the symmetric dense W (checked as launch_ingest, plus
// status |= 1 when W is not symmetric), or with W == nullptr 0 on the diagonal
// and INF elsewhere; the padding is INF.
cudaError_t launch_tri_fill(int dtype, const void *W, int64_t ldw, void *T, int64_t n, int *status, cudaStream_t s,
                            int64_t *launches);
// T <- the adjacency matrix of an undirected edge list (as launch_densify).
cudaError_t launch_tri_from_edges(int dtype, const int32_t *src, const int32_t *dst, const void *w, int64_t m,
                                  void *T, int64_t n, int *status, cudaStream_t s, int64_t *launches);
// Dense n x n D (leading dimension ld) from T, both triangles.
cudaError_t launch_tri_to_dense(int dtype, const void *T, int64_t n, void *D, int64_t ld, cudaStream_t s,
                                int64_t *launches);
// out[i][0..n) = row rows[i] of the matrix in T (rows: k device int64; a bad
// index sets status |= 1).
cudaError_t launch_tri_rows(int dtype, const void *T, int64_t n, const int64_t *rows, int64_t k, void *out,
                            int64_t ldo, int *status, cudaStream_t s, int64_t *launches);

// Copies W to D when they differ and checks the input (status |= 1 invalid, 2 range).
cudaError_t launch_ingest(int dtype, const void *W, void *D, int64_t n, int64_t ld, int *status, cudaStream_t s,
                          int64_t *launches);
// Fills D with a synthetic symmetric graph (autotuner input).
cudaError_t launch_synth(int dtype, void *D, int64_t n, int64_t ld, cudaStream_t s);
cudaError_t launch_pack(const int32_t *src, int64_t lds, uint16_t *dst, int64_t ldd, int64_t n, cudaStream_t s,
                        int64_t *launches);
cudaError_t launch_unpack(const uint16_t *src, int64_t lds, int32_t *dst, int64_t ldd, int64_t n, cudaStream_t s,
                          int64_t *launches);
cudaError_t launch_densify(int dtype, const int32_t *src, const int32_t *dst, const void *w, int64_t m, void *D,
                           int64_t n, int64_t ld, int *status, cudaStream_t s, int64_t *launches);
// C = min(C, A (x) B).  With scratch (>= minplus_scratch_bytes(m, k)) and
// 16-byte addressable B and C: A^T into scratch, then the warp-specialized TMA
// kernel (C may then alias A and B: every value read is a valid upper bound,
// so an in-place product only converges faster); otherwise one CTA per tile.
// wait_err as for launch_rounds.
size_t minplus_scratch_bytes(int64_t m, int64_t k);
cudaError_t launch_minplus(int dtype, const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc,
                           int64_t m, int64_t k, int64_t nn, cudaStream_t s, int64_t *launches,
                           void *scratch = nullptr, size_t scratch_bytes = 0, int *wait_err = nullptr);

// 16-bit enable test.  *bound = max over components of 2 * ecc(smallest vertex);
// *ok = bound < 0x7FFF.  Both synchronize `s`.
// Edge list: undirected edges (src[e], dst[e]) with weights of type wtype
// (0 int32, 1 uint16); entries with a bad id, a self loop or an INF weight are
// skipped.
cudaError_t bound_from_edges(const int32_t *src, const int32_t *dst, const void *w, int wtype, int64_t m, int64_t n,
                             cudaStream_t s, int64_t *bound, int *ok, int64_t *launches);
// Dense int32 matrix: the finite off-diagonal entries become the edge list;
// an asymmetric matrix (W_ij != W_ji) or more than `max_edges` finite entries
// gives *ok = 0.
cudaError_t bound_from_dense(const int32_t *W, int64_t n, int64_t ld, int64_t max_edges, cudaStream_t s,
                             int64_t *bound, int *ok, int64_t *launches);

}  // namespace apsp
