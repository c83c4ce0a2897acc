/*
 * apsp.h -- C ABI of the GB300 blocked Floyd-Warshall all-pairs shortest-path
 * library (libapsp.so).
 *
 * Problem (the paper, Sec. 3): an undirected weighted graph G = (V, E, w) with
 * n vertices and no negative cycles is given by its adjacency matrix A with
 * A_ij = A_ji = w_ij; the library returns the length of the shortest path
 * between every pair of vertices (no paths).  Conventions of this ABI:
 *   - A_ii = 0; a missing edge is INF (APSP_INF_I32, APSP_INF_U16, or +inf for
 *     fp32); weights are >= 0 (an undirected negative edge is a negative
 *     cycle).
 *   - Output entry D_ij = shortest-path length, INF exactly when i and j are in
 *     different components.
 * Method (Sec. 4.4 and 4.5, Alg. 3 and 4; Fig. 1 phases): the n x n matrix is
 * split into Bk x Bk blocks; for each round k = 0..q-1 (q = ceil(n/Bk)):
 *   Phase 1  closes the diagonal block D_kk by Floyd-Warshall (Table 1
 *            "FloydWarshall");
 *   Phase 2  updates the row panel D_kJ = min(D_kJ, D_kk (x) D_kJ) and the
 *            column panel D_Ik = min(D_Ik, D_Ik (x) D_kk) (Table 1 "MinPlus");
 *   Phase 3  updates every remaining block D_IJ = min(D_IJ, D_Ik (x) D_kJ)
 *            (Table 1 "MatProd" + "MatMin").
 * (x) is the min-plus product (X (x) Y)_ij = min_t X_it + Y_tj.  Directed
 * inputs are also solved exactly (the paper notes the method applies to them
 * once symmetry is not exploited; the library never assumes symmetry).
 *
 * Memory: every matrix argument is a caller-owned pointer to DEVICE memory
 * (unless a function says otherwise), row-major, n rows of `ld` elements
 * (ld >= n); only the first n elements of each row are read or written.
 * Calls that take a stream are asynchronous on it (a cudaStream_t passed as
 * void*, NULL = the legacy default stream) unless stated otherwise.  No C++
 * exception crosses this ABI; every call returns an apsp_status, 0 = success.
 */
#ifndef APSP_H_
#define APSP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- sentinels ---------------------------------------------------------- */
/* int32 INF = INT32_MAX / 2: any sum of two stored values stays <= INT32_MAX,
 * so the add-min never overflows and a pair in different components keeps
 * exactly INF (INF + x > INF >= the current value). */
#define APSP_INF_I32 1073741823
/* Packed unsigned 16-bit INF: stored values are <= 0x7FFF, so the sum of two
 * never exceeds 0xFFFE and the 16-bit add never wraps. */
#define APSP_INF_U16 0x7FFF

typedef enum {
  APSP_OK = 0,
  APSP_E_INVALID = 1,   /* bad argument (null, n < 0, ld < n, negative weight, non-zero diagonal) */
  APSP_E_CUDA = 2,      /* a CUDA runtime call failed; apsp_last_error() has the text */
  APSP_E_NOMEM = 3,     /* workspace or request does not fit the memory budget */
  APSP_E_RANGE = 4,     /* a finite weight >= INF, or the 16-bit bound does not hold */
  APSP_E_BUSY = 5,      /* request queue full */
  APSP_E_NOTFOUND = 6,  /* unknown ticket */
  APSP_E_TIMEOUT = 7,   /* a bounded device wait gave up */
  APSP_E_CANCELLED = 8, /* request cancelled, or the handle was destroyed */
  APSP_E_NOTREADY = 9,  /* poll: the request has not finished */
  APSP_E_UNSUPPORTED = 10
} apsp_status;

typedef enum {
  APSP_I32 = 0,  /* int32 distances, INF = APSP_INF_I32 */
  APSP_U16 = 1,  /* packed unsigned 16-bit distances, INF = APSP_INF_U16 */
  APSP_F32 = 2,  /* fp32 distances, INF = +inf */
  APSP_AUTO = 3  /* int32 in/out; solved in packed 16-bit when the bound allows */
} apsp_dtype;

typedef struct apsp_handle apsp_handle;

typedef struct {
  int device;            /* CUDA device ordinal (the handle makes it current in every call) */
  int dtype;             /* apsp_dtype used by apsp_solve (default APSP_I32) */
  int block_k;           /* round width Bk (32, 64 or 128); 0 = tuned (apsp_autotune), else by n and dtype
                            (128 for packed 16-bit from n = 49152 and fp32 from n = 24576, else 64) */
  int max_batch;         /* serving: graphs per persistent launch (default 64) */
  int queue_depth;       /* serving: pending requests before APSP_E_BUSY (default 4096) */
  int64_t memory_budget; /* serving: bytes of device memory for admitted requests (0 = free HBM - reserve) */
  int64_t spin_limit;    /* bounded device waits: iterations before APSP_E_TIMEOUT (0 = default) */
  int phase3_variant;    /* Phase-3 kernel: 0 = tuned, else by n and dtype (5 for 6144 <= n < 24576,
                            6144 <= n < 49152 for packed 16-bit; 4 otherwise), 1 = one
                            CTA per tile, 2 = persistent TMA kernel with 256 threads, 3 = persistent TMA
                            kernel with 512 threads, 4 = warp-specialized persistent kernel (TMA producer
                            warp; int32 results leave by a TMA min-reduction), one launch per round,
                            5 = the same kernel running every round in one launch with each round's
                            Phase 1 and Phase 2 as tasks inside it (round width 64).  At round width 128
                            variants 2, 3 and 5 run as 4, whose tiles then take two 64-step stages */
  int symmetric;         /* symmetric mode for undirected graphs (Sec. 3: A_ij = A_ji; the paper keeps
                            only the upper triangle): Phase 3 updates only the tiles touching the upper
                            triangle and the lower triangle is mirrored at the end -- same result, about
                            half the relaxations.  0 = use it when a device check finds W symmetric
                            (one stream synchronization per solve), 1 = the caller guarantees W is
                            symmetric, 2 = never.  Edge-list solves are symmetric by construction. */
  int64_t serving_large_n; /* serving: a request with n >= this runs alone in its own group on the per-round
                              kernels; smaller ones share the batched persistent kernel (0 = default 1536),
                              except one that finds the server idle, which also runs alone on the per-round
                              kernels */
  int serving_large_grid;  /* serving: CTAs of a large request's persistent Phase-3 kernel (0 = one per SM, and
                              one launch per round); a smaller grid lets several large requests run side by side
                              on disjoint SMs, each with its size's default round shape */
} apsp_config;

/* Fills *cfg with the defaults (library plumbing; no paper counterpart). */
void apsp_config_default(apsp_config *cfg);

/* Creates a handle on cfg->device (cfg == NULL: defaults; library plumbing, no
 * paper counterpart).  The library owns
 * the handle, its device workspace and its serving thread (started on the
 * first apsp_submit).  Errors: APSP_E_INVALID, APSP_E_CUDA. */
apsp_status apsp_create(apsp_handle **h, const apsp_config *cfg);

/* Frees everything the handle owns; pending requests end as
 * APSP_E_CANCELLED.  Safe on NULL. */
apsp_status apsp_destroy(apsp_handle *h);

/* ---- one-shot solve (Alg. 3/4 rounds on the caller's stream) ------------ */
/* Solves APSP for the n x n matrix W into D, element type = the handle's
 * dtype.  W and D are device pointers with the same leading dimension ld;
 * W == D (in place) is allowed.  Asynchronous on `stream`, except that
 * APSP_AUTO synchronizes the stream once to read the 16-bit bound.
 * Input checks that need the data (negative weight, non-zero diagonal,
 * finite weight >= INF) run on the device; read their result with
 * apsp_last_status().  Errors returned directly: APSP_E_INVALID (null pointer,
 * n < 0, ld < n), APSP_E_NOMEM (workspace), APSP_E_CUDA. */
apsp_status apsp_solve(apsp_handle *h, const void *W, int64_t n, int64_t ld, void *D, void *stream);

/* Same with an explicit element type. */
apsp_status apsp_solve_t(apsp_handle *h, int dtype, const void *W, int64_t n, int64_t ld, void *D,
                         void *stream);

/* Builds D from an edge list on the device and solves it in place: D_ii = 0,
 * D_uv = D_vu = min over duplicate edges of w, INF elsewhere (the adjacency
 * matrix A of Sec. 3, built on the device).
 * src/dst are int32 device arrays of m vertex ids, w holds m weights of the
 * element type (int32 for APSP_I32/APSP_AUTO, uint16 for APSP_U16, float for
 * APSP_F32).  For APSP_U16 and APSP_AUTO the 16-bit bound is computed from the
 * edge list first (this synchronizes `stream`); APSP_U16 returns APSP_E_RANGE
 * when it fails, APSP_AUTO then falls back to int32 (D must then be int32).
 * This is the path for sizes where a dense int32 W does not fit next to D. */
apsp_status apsp_solve_edges(apsp_handle *h, int dtype, const int32_t *src, const int32_t *dst, const void *w,
                             int64_t m, int64_t n, void *D, int64_t ld, void *stream);

/* Waits for `stream` and returns the device-side input check of the last
 * solve on this handle: APSP_OK, APSP_E_INVALID (negative weight or non-zero
 * diagonal), APSP_E_RANGE (a finite weight >= INF) or, after
 * apsp_solve_batch, APSP_E_TIMEOUT (a bounded device wait gave up). */
apsp_status apsp_last_status(apsp_handle *h, void *stream);

/* The 16-bit enable test by itself (the precision selection; no paper
 * counterpart, the paper's runs use one precision): for
 * every connected component c of the graph given by the int32 matrix W, the
 * single-source distances from the smallest vertex r_c of c give
 * ecc(r_c); every finite distance in c is <= 2 ecc(r_c) (triangle inequality
 * through r_c).  *bound = max_c 2 ecc(r_c) (saturated at INT64_MAX / 4), *ok =
 * (*bound < APSP_INF_U16).  Synchronizes `stream`. */
apsp_status apsp_int16_bound(apsp_handle *h, const int32_t *W, int64_t n, int64_t ld, int64_t *bound, int *ok,
                             void *stream);

/* ---- batched solve: many graphs in one launch ----------------------------- */
/* Solves `count` int32 graphs of uneven n in ONE persistent launch on
 * `stream`: the rounds of every graph (Alg. 3/4 phases) are cut into tasks
 * that resident CTAs pull from a device work queue in dependency order, so
 * rounds of different graphs overlap on the device.  W[i], D[i] are device
 * matrices (n[i] rows of ld[i] elements, W[i] == D[i] allowed).  Asynchronous;
 * apsp_last_status() reports the input checks of all graphs and
 * APSP_E_TIMEOUT if a bounded device wait gave up.  Errors: APSP_E_INVALID,
 * APSP_E_NOMEM (workspace), APSP_E_CUDA. */
apsp_status apsp_solve_batch(apsp_handle *h, int64_t count, const int32_t *const *W, const int64_t *n,
                             const int64_t *ld, int32_t *const *D, void *stream);

/* Diagnostic of the bounded device waits (no paper counterpart): runs two
 * launches over small built-in graphs (paths) whose first task waits on a
 * device flag that nothing sets, with the given spin limit (> 0) on each wait
 * for another work item: the batched kernel (96 nodes), then every round of a
 * 320-node solve in one persistent launch (phase3_variant 5).  Returns
 * APSP_E_TIMEOUT when both kernels gave up and reported it (the expected
 * outcome), APSP_OK if one of them did not wait, or another error.
 * Synchronizes the device; the context stays usable. */
apsp_status apsp_check_bounded_wait(apsp_handle *h, int64_t spin_limit);

/* ---- building blocks (Table 1) ------------------------------------------ */
/* C = min(C, A (x) B): the min-plus product ("MatProd") followed by the
 * element-wise minimum ("MatMin").  A is m x k (lda), B is k x n (ldb), C is
 * m x n (ldc), all device, row-major, of the given dtype (APSP_I32, APSP_U16 or
 * APSP_F32).  C must not overlap A or B.  Uses a handle-owned workspace of
 * about 4*m*k bytes (A transposed) for the TMA-fed kernel when it can be
 * allocated and B and C are 16-byte addressable; otherwise a kernel without
 * workspace.  Asynchronous on `stream`; a device wait that gave up is reported
 * by apsp_last_status (bit 4).  Errors: APSP_E_INVALID, APSP_E_CUDA. */
apsp_status apsp_minplus(apsp_handle *h, int dtype, const void *A, int64_t lda, const void *B, int64_t ldb,
                         void *C, int64_t ldc, int64_t m, int64_t k, int64_t n, void *stream);

/* All-pairs shortest paths by repeated min-plus squaring (Alg. 1): D = W, then
 * ceil(log2(n - 1)) times D = min(D, D (x) D), in place.  The same matrix as
 * apsp_solve_t (exact for APSP_I32 and APSP_U16; fp32 within rounding), for
 * about log2(n) times the work of Floyd-Warshall: the paper's first method, kept
 * as a second workload of the min-plus product.  Arguments, layout, input
 * checks and status as apsp_solve_t with an explicit dtype (no APSP_AUTO);
 * uses the apsp_minplus workspace (about 4*n*n bytes). */
apsp_status apsp_solve_squaring(apsp_handle *h, int dtype, const void *W, int64_t n, int64_t ld, void *D,
                                void *stream);

/* ---- upper-triangular storage ------------------------------------------- */
/* The paper stores only the upper triangle of blocks of the symmetric
 * distance matrix; a lower block is the transpose of an upper one (Sec. 4,
 * the block decomposition; Sec. 3: A_ij = A_ji).  These calls keep an
 * undirected graph's n x n matrix in about half the memory: it is cut into
 * S x S super-tiles (S = 128 elements for APSP_I32 / APSP_F32, 256 for
 * APSP_U16) and only the super-tiles (I, J) with I <= J are stored -- the
 * diagonal super-tiles in full -- folded into one rectangle of `rows` rows
 * with a row pitch of `ld` elements (about n^2 / 2 elements plus one
 * super-tile band; 68.8 GB instead of 137 GB for n = 262144 in packed
 * 16-bit).  Element (r, c) is stored when floor(c / S) >= floor(r / S);
 * rows and columns n .. S*ceil(n/S)-1 are padding, whose contents after a
 * solve are unspecified.  The rectangle ("T" below) is caller-owned device
 * memory of apsp_tri_layout's `bytes`, 16-byte aligned.
 * Placement of a super-row I (T = ceil(n / S) super-rows, Th = ceil(T / 2)):
 * I < Th in rectangle rows I*S.. with columns shifted right by S; I >= Th in
 * rectangle rows (2 Th - 1 - I)*S.. with columns shifted left by I*S.  This
 * mapping is the format's definition; apsp_tri_rows and apsp_tri_to_dense
 * read it back. */

/* Rectangle of the upper-triangular layout for n and dtype (APSP_I32,
 * APSP_U16 or APSP_F32): *rows, *ld (row pitch, elements) and *bytes (each
 * nullable, not all).  Host only.  Errors: APSP_E_INVALID. */
apsp_status apsp_tri_layout(int dtype, int64_t n, int64_t *rows, int64_t *ld, int64_t *bytes);

/* T <- the upper-triangular layout of the symmetric dense n x n matrix W
 * (device, leading dimension ldw; only its stored part is copied), padding
 * INF.  The input checks of apsp_solve_t run on the device, plus a symmetry
 * check (an asymmetric W is APSP_E_INVALID); read them with
 * apsp_last_status.  Asynchronous on `stream`.  Errors: APSP_E_INVALID,
 * APSP_E_CUDA. */
apsp_status apsp_tri_from_dense(apsp_handle *h, int dtype, const void *W, int64_t n, int64_t ldw, void *T,
                                void *stream);

/* T <- the adjacency matrix of an undirected edge list in the
 * upper-triangular layout (the conventions of apsp_solve_edges: min over
 * duplicate edges, 0 on the diagonal, INF elsewhere; checks read by
 * apsp_last_status).  For APSP_U16 the 16-bit bound is computed from the
 * edge list first (this synchronizes `stream`) and APSP_E_RANGE is returned
 * when it fails.  This is the path at sizes where even one dense matrix does
 * not fit.  Errors: APSP_E_INVALID, APSP_E_RANGE, APSP_E_CUDA. */
apsp_status apsp_tri_from_edges(apsp_handle *h, int dtype, const int32_t *src, const int32_t *dst, const void *w,
                                int64_t m, int64_t n, void *T, void *stream);

/* Solves APSP in place on T, which holds an undirected graph's adjacency
 * matrix in the upper-triangular layout (from apsp_tri_from_dense or
 * apsp_tri_from_edges): the q rounds of Phase 1 / 2 / 3 (Alg. 3/4) update only
 * stored super-tiles -- Phase 3 the tiles (I, J) with I <= J, both of its
 * operands from the round's symmetric panel -- with the warp-specialized
 * Phase-3 kernel launched once per round; the distances equal apsp_solve_t's
 * on the dense matrix.  Does not reset the status word: apsp_last_status then
 * reports the checks of the call that filled T and APSP_E_TIMEOUT if a bounded
 * device wait gave up.  Asynchronous on `stream`.  Errors: APSP_E_INVALID (T
 * not 16-byte aligned, bad arguments), APSP_E_NOMEM, APSP_E_CUDA. */
apsp_status apsp_solve_tri(apsp_handle *h, int dtype, void *T, int64_t n, void *stream);

/* D (dense n x n, device, leading dimension ld) <- the full matrix held in T:
 * the stored elements, and the lower triangle mirrored from the upper.
 * Asynchronous on `stream`.  Errors: APSP_E_INVALID, APSP_E_CUDA. */
apsp_status apsp_tri_to_dense(int dtype, const void *T, int64_t n, void *D, int64_t ld, void *stream);

/* out[i][0..n) <- row rows[i] of the full matrix held in T, for k row indices
 * (device int64 array, each in [0, n); an index outside is skipped, its output
 * row left as it was); out is device memory with leading dimension ldo >= n.
 * The way to read results of a matrix too large to hold densely.
 * Asynchronous on `stream`.  Errors: APSP_E_INVALID, APSP_E_CUDA. */
apsp_status apsp_tri_rows(int dtype, const void *T, int64_t n, const int64_t *rows, int64_t k, void *out, int64_t ldo,
                          void *stream);

/* int32 -> packed u16 (INF32 -> INF16) and back, n x n with separate leading
 * dimensions; the caller guarantees every finite entry is < APSP_INF_U16.
 * (The storage of the packed 16-bit precision; no paper counterpart -- the
 * paper's runs use one precision.) */
apsp_status apsp_pack_u16(const int32_t *src, int64_t lds, uint16_t *dst, int64_t ldd, int64_t n, void *stream);
apsp_status apsp_unpack_u16(const uint16_t *src, int64_t lds, int32_t *dst, int64_t ldd, int64_t n, void *stream);

/* ---- request loop (serving) ---------------------------------------------- */
/* A stream of independent solve requests (no paper counterpart: the paper's
 * Spark scheduler runs one solve; Sec. 5.3 tunes its task over-decomposition,
 * the nearest analogue of grouping requests into one launch). */
typedef enum {
  APSP_QUEUED = 0,   /* accepted, waiting for memory or a batch slot */
  APSP_ADMITTED = 1, /* device matrix allocated, the copy of W in flight: W must not change yet */
  APSP_RUNNING = 2,  /* W copied (the caller may reuse it); rounds in progress on the device */
  APSP_DONE = 3,
  APSP_ERROR = 4
} apsp_state;

typedef struct {
  const void *W;   /* int32 adjacency matrix, n rows of ld elements */
  int is_host;     /* 1: W is host memory (copied at admission), 0: device memory */
  int64_t n;
  int64_t ld;
  int dtype;       /* APSP_I32 (0, the default of a zeroed struct) or APSP_AUTO: the result is int32 either
                      way; APSP_AUTO solves a request with n >= 1536 in packed 16-bit when the 16-bit
                      bound holds (the bound synchronizes that request's stream in the serving thread),
                      smaller requests run in the batched int32 kernel (the same exact result) */
} apsp_request;

/* Queues a request; non-blocking.  The library copies W into a device matrix
 * it owns when the request is admitted (its n^2 * 4-byte footprint, plus its
 * share of workspace, fits the memory budget); the caller may reuse W once
 * apsp_poll reports APSP_RUNNING or later.  Errors: APSP_E_INVALID,
 * APSP_E_UNSUPPORTED (dtype other than APSP_I32 / APSP_AUTO), APSP_E_BUSY
 * (queue full), APSP_E_NOMEM (n^2 * 4 bytes exceeds the whole budget). */
apsp_status apsp_submit(apsp_handle *h, const apsp_request *r, uint64_t *ticket);

/* Non-blocking state query.  On APSP_DONE, *D_dev (if non-NULL) points at the
 * library-owned int32 n x n result (leading dimension n), valid until
 * apsp_release.  Returns APSP_OK, or the request's error (APSP_E_TIMEOUT,
 * APSP_E_CANCELLED, ...) with *st = APSP_ERROR, or APSP_E_NOTFOUND. */
apsp_status apsp_poll(apsp_handle *h, uint64_t ticket, apsp_state *st, const void **D_dev);

/* Blocks until the request is DONE or ERROR, or timeout_ms passes
 * (APSP_E_NOTREADY). */
apsp_status apsp_wait(apsp_handle *h, uint64_t ticket, int64_t timeout_ms);

/* Copies a finished result to dst (device or host, leading dimension ldd) on
 * `stream`. */
apsp_status apsp_fetch(apsp_handle *h, uint64_t ticket, void *dst, int64_t ldd, void *stream);

/* Frees a finished request's device matrix and forgets the ticket. */
apsp_status apsp_release(apsp_handle *h, uint64_t ticket);

/* Cancels a request that has not started running; running requests finish. */
apsp_status apsp_cancel(apsp_handle *h, uint64_t ticket);

/* ---- autotuner ---------------------------------------------------------- */
/* The paper picks its block size b per problem size (Sec. 3 "user-provided
 * (or auto-tuned)", Sec. 5.2-5.4, Table 3).  For `dtype` and every n bucket
 * (powers of two from 128 up to n_max) this times the candidate round shapes
 * -- round width Bk in {32, 64} x Phase-3 variant (the persistent TMA kernels,
 * per round or all rounds in one launch, or one CTA per tile), and Bk = 128
 * with the per-round warp-specialized kernel or one CTA per tile -- on a synthetic matrix generated on the device (the
 * kernels do the same work for any graph of a given n), and keeps the
 * fastest for later solves on this handle.  cache_path (nullable): a JSON
 * file keyed by GPU name; entries for this GPU are loaded instead of timing
 * when present, and new results are written back.  Synchronizes the device. */
apsp_status apsp_autotune(apsp_handle *h, int dtype, int64_t n_max, const char *cache_path);

/* The round shape the handle uses for (dtype, n): *block_k and *tma, the
 * Phase-3 kernel numbered as apsp_config.phase3_variant minus one (0 = one
 * CTA per tile, 1-3 = the persistent TMA kernels launched per round, 4 = every
 * round in one launch). */
apsp_status apsp_tuned_config(apsp_handle *h, int dtype, int64_t n, int *block_k, int *tma);

/* ---- solve without allocation -------------------------------------------- */
/* Largest n accepted by apsp_solve_i32_noalloc. */
#define APSP_NOALLOC_MAX_N 16384

/* An int32 solve (same result as apsp_solve_t with APSP_I32) that allocates
 * no memory of its own: no handle, no cudaMalloc, no allocating library call.
 * The paper has no counterpart; this exists for callers that cannot allocate
 * device memory where they solve -- code that runs inside another
 * framework's memory pool or allocator hooks and must not allocate behind its
 * back, or a latency-bound loop that cannot afford the device-wide
 * synchronization an allocation may cause.  The caller passes W and D
 * (device, n rows of ld elements, W == D allowed) and a stream (void*, NULL =
 * legacy default stream); the call is asynchronous on it.
 * Scratch memory: a fixed array in device global memory inside the library,
 * sized for n <= APSP_NOALLOC_MAX_N (about 4 MiB), which every GPU that loads
 * the library keeps until the process exits.  Every call shares that array:
 * calls that overlap on the GPU (different streams, or different host
 * threads) race on it and give wrong results -- order them on one stream.
 * First use on a device: CUDA loads the library's device code and globals
 * lazily, so the first call on each device (and the first call of a size that
 * runs a kernel not run before on that device) may load code and create the
 * array -- memory the driver allocates, possibly with a device
 * synchronization.  Make one call of each size class you will use (n <= 64,
 * n <= 128, larger) during set-up, outside the phase that must not allocate
 * and before any stream capture, or set CUDA_MODULE_LOADING=EAGER before the
 * process initializes CUDA.  The first call also looks up the array's device
 * address.  Inputs are not checked on the device (use apsp_solve for checked
 * solves).  The call returns before the solve has run: a bounded device wait
 * that gave up (D then incomplete) is reported by apsp_noalloc_status.
 * Errors: APSP_E_INVALID (n < 0, ld < n, null pointer), APSP_E_RANGE (n >
 * APSP_NOALLOC_MAX_N), APSP_E_CUDA (a CUDA call failed). */
apsp_status apsp_solve_i32_noalloc(const int32_t *W, int64_t n, int64_t ld, int32_t *D, void *stream);

/* Waits for `stream` and reports the device-side outcome of the last
 * apsp_solve_i32_noalloc on the current device: APSP_OK, or APSP_E_TIMEOUT
 * when a bounded wait of its Phase-3 kernel gave up (D is then incomplete).
 * Reads one word of the fixed scratch array into the caller's stack;
 * allocates nothing.  (Library plumbing; no paper counterpart.)  Errors:
 * APSP_E_CUDA. */
apsp_status apsp_noalloc_status(void *stream);

/* ---- the add-min step itself (measurement support) ----------------------- */
/* The relaxation c = min(c, a + b) is the min-plus step of Table 1 (MatProd
 * followed by MatMin); Phase 3 is bound by how many of them the SMs issue per
 * clock.  apsp_addmin_peak measures that rate on `device` for the add-min form
 * the library's Phase-3 tiles use for `dtype` (APSP_I32: __viaddmin_s32;
 * APSP_U16: __viaddmin_u16x2, two relaxations per 32-bit lane-op; APSP_F32:
 * two k-steps at a time, a packed pair add for two neighbouring columns and
 * one three-input minimum for each output's two sums): independent chains in
 * registers, one full wave of 4 CTAs x 256 threads per SM.
 * *relax_per_clk_per_sm = relaxations per SM clock (by clock64 of the slowest
 * CTA); *relax_per_s = relaxations per second by event time (at whatever
 * clock the GPU ran).  Allocates a few KB of device memory and synchronizes
 * the device.  Errors: APSP_E_INVALID, APSP_E_CUDA. */
apsp_status apsp_addmin_peak(int device, int dtype, double *relax_per_clk_per_sm, double *relax_per_s);

/* out[i] = the library's add-min of the 32-bit words (a[i], b[i], c[i]) for
 * `dtype`: APSP_I32 min(a + b, c) as int32; APSP_U16 per 16-bit lane
 * min(a + b, c) with the add taken modulo 2^16 (the stored values never reach
 * the wrap: they are <= APSP_INF_U16); APSP_F32 fminf(a + b, c) on the bit
 * patterns.  Device arrays of m words; asynchronous on `stream`.  Exposes the
 * primitive so that its lane semantics can be tested.  Errors: APSP_E_INVALID,
 * APSP_E_CUDA. */
apsp_status apsp_addmin_eval(int dtype, const uint32_t *a, const uint32_t *b, const uint32_t *c, uint32_t *out,
                             int64_t m, void *stream);

/* ---- diagnostics (library plumbing; no paper counterpart) ---------------- */
const char *apsp_strerror(apsp_status s);
/* Text of the last failure on this handle (thread-local per handle); never NULL. */
const char *apsp_last_error(apsp_handle *h);
/* Number of kernel launches this handle has issued (for launch accounting). */
int64_t apsp_launch_count(apsp_handle *h);

/* Per-phase device timing (measurement support; the paper has no counterpart
 * beyond its wall-clock times of Sec. 5).  enable = 1: every later solve on
 * this handle records a CUDA event pair around each Phase 1 / 2 / 3 launch on
 * the solve's stream; enable = 0 stops recording.  apsp_profile_read waits for
 * the recorded events and writes, for phases 0, 1, 2 (= Phase 1, 2, 3), the
 * number of timed launches, their summed device time in ms, and their summed
 * algorithmic relaxation counts (Phase 1: w^3, Phase 2: 2 (n-w) w^2, Phase 3:
 * (n-w)^2 w for a round of width w); then it clears the record.  Any of the
 * output arrays may be NULL. */
apsp_status apsp_profile(apsp_handle *h, int enable);
apsp_status apsp_profile_read(apsp_handle *h, int64_t launches[3], double ms[3], double relaxations[3]);

#ifdef __cplusplus
}
#endif
#endif /* APSP_H_ */
