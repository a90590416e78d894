/*
 * arrow.h -- C-ABI of the GB300 arrow-decomposition SpMM library (libarrow_gb300.so).
 *
 * The library computes the iterated product X_{t+1} = sigma(A X_t) of Section 2
 * ("Matrices") through an arrow matrix decomposition A = sum_i P_{pi_i} B_i P_{pi_i}^T
 * (Section 3, Eq. 1): each B_i has arrow-width b (non-zeros only in its first b rows,
 * its first b columns and its b x b diagonal tiles, Section 3.1 / Fig. 2), and the
 * P_{pi_i} are vertex permutations found by LA-Decompose (Section 4.1) with the random
 * spanning forest arrangement (Section 4.3) and smallest-first tree layout (Section 4.4).
 *
 * Conventions used by every call:
 *   - Matrices are square n x n.  Vertex v of the graph of A is row/column v.
 *   - Dense blocks (X, Y) are row-major n x k with row stride k elements.
 *   - Return codes: ARROW_OK (0) or a negative ARROW_E* code; after a failure
 *     arrow_last_error() returns a message for the calling thread.
 *   - Calls on one handle are not thread-safe; different handles are independent.
 *   - "stream" arguments are cudaStream_t values passed as void* (NULL = legacy default stream).
 */
#ifndef ARROW_GB300_H
#define ARROW_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------------------- */
#define ARROW_OK        0
#define ARROW_EINVAL   (-1)   /* invalid argument (bad CSR, b < 2, bad k, bad dtype, ...) */
#define ARROW_ENOMEM   (-2)   /* host or device allocation failed; no state was leaked   */
#define ARROW_ECUDA    (-3)   /* a CUDA runtime call failed (message has the CUDA error)  */
#define ARROW_ETIMEOUT (-4)   /* a bounded device-side wait ran out (status word set)      */
#define ARROW_ESTATE   (-5)   /* call not valid in the handle's state (e.g. not uploaded)  */

/* ---- element types ----------------------------------------------------------------- */
typedef enum { ARROW_F32 = 0, ARROW_BF16 = 1, ARROW_F16 = 2 } arrow_dtype;

/* ---- arrow predicates (shape of each B_i) ---------------------------------------- */
/* Block-diagonal arrow (Section 3.1, Fig. 2, Alg. 1): entry at positions (r, c) belongs
 * to B_i iff r < b or c < b or floor(r/b) == floor(c/b).  The default. */
#define ARROW_PRED_BLOCK 0
/* Banded arrow (Section 1 definition, 0-based): r < b or c < b or |r - c| <= b.  A band row
 * reaches into three consecutive b x b tiles (block-tridiagonal).  The device path runs it
 * through the same fused row program as the block form. */
#define ARROW_PRED_BAND  1

/* ---- input matrix ------------------------------------------------------------------ */
/* CSR in HOST memory, caller-owned, read during arrow_decompose only (copied).
 * rowptr[0] = 0, rowptr non-decreasing, rowptr[n] = nnz; colidx in [0, n) strictly
 * increasing inside each row; values are float64.  nnz must be < 2^31.
 * The matrix need not be symmetric: LA-Decompose works on the symmetric pattern of A
 * (Section 4.1 works on graphs), and every entry keeps its own value. */
typedef struct {
    int64_t        n;
    int64_t        nnz;
    const int64_t* rowptr;
    const int32_t* colidx;
    const double*  values;
} arrow_csr;

/* ---- decomposition options ------------------------------------------------------- */
#define ARROW_HOST_ONLY 0x1   /* opts.flags: build on the host, do not touch a GPU */
/* opts.flags: run the data-parallel steps of LA-Decompose on the GPU (opts.device, or the
 * current one): per level the degrees, the edges of G_i' with their random keys, the minimum
 * spanning forest (Boruvka; Section 4.3) and the split of the entries by the arrow shape
 * (steps 3-4 of Section 4.1).  The head choice and the tree layout (Section 4.4) stay on the
 * host.  The result is the host path's decomposition, bit for bit.  Needs device memory of
 * about 40 bytes per entry of the symmetric pattern while it runs.  Not with ARROW_HOST_ONLY. */
#define ARROW_DEVICE_DECOMPOSE 0x2

typedef struct {
    uint64_t seed;        /* seed of the random edge weights (Section 4.3 step 1)           */
    int32_t  value_dtype; /* arrow_dtype the device stores A's values in (RNE from float64) */
    int32_t  predicate;   /* ARROW_PRED_BLOCK (default) or ARROW_PRED_BAND                  */
    int32_t  flags;       /* ARROW_HOST_ONLY, ARROW_DEVICE_DECOMPOSE or 0                    */
    int32_t  nthreads;    /* host threads for the decomposition; 0 = all hardware threads   */
    int32_t  max_levels;  /* cap on the order l of the decomposition; 0 = 254               */
    int32_t  long_row;    /* rows with more entries than this are split; 0 = default (64)   */
    int32_t  segment;     /* entries per split segment; 0 = default (512)                   */
    int32_t  device;      /* CUDA device ordinal for the upload; -1 = current device.  The
                             caller's current device is restored after the upload; later
                             calls on the handle need its device current                  */
} arrow_opts;

/* Fill *o with defaults: seed 0, F32 values, block predicate, upload, all threads. */
int arrow_opts_default(arrow_opts* o);

/* ---- launch tuning -------------------------------------------------------------------- */
/* How the fused row program is cut and launched (not in the paper; a property of this GPU
 * path): rows per tile, entries per tile (>= 1024, so every unsplit row fits), resident CTAs
 * per SM of the persistent rows kernel (1..4, as far as shared memory allows), the
 * shared-memory carveout in percent, and
 * fold_permute_in = 1, which makes the first iteration gather straight from the caller's X
 * through a second copy of the column indices in vertex ids (4 bytes per entry of device
 * memory, set up when the setting is applied) instead of permuting X into pi_0 order first.
 * fused_small = 1 runs a whole arrow_spmm call as one cooperative launch (permute-in, every
 * iteration's phases separated by grid-wide barriers with a 2 s limit, permute-out) when the
 * problem is small (n <= 2^20, nnz <= 2^23) and k / (16 / sizeof(x_dtype)) <= 32, where kernel
 * start-up would dominate; identical results without ARROW_RESCALE, within rounding with it
 * (the FP64 column sums are grouped differently).  Larger problems ignore it.
 * Defaults: 256, 2048, 4, 70, 0, 0. */
typedef struct {
    int32_t tile_rows;
    int32_t tile_nnz;
    int32_t ctas_per_sm;
    int32_t carveout;
    int32_t fold_permute_in;
    int32_t fused_small;
} arrow_tuning;


/* ---- handle ------------------------------------------------------------------------ */
typedef struct arrow_handle_s* arrow_handle;   /* opaque, library-owned */

int arrow_get_tuning(arrow_handle h, arrow_tuning* t);

/* Re-tile the handle (host, O(n)) and, if uploaded, replace its device tile tables; waits for
 * the device first.  Errors: ARROW_EINVAL (out of range: 32 <= tile_rows <= 2048,
 * 1024 <= tile_nnz <= 16384, 1 <= ctas_per_sm <= 4, 0 <= carveout <= 100,
 * fold_permute_in and fused_small 0 or 1), ARROW_ENOMEM, ARROW_ECUDA. */
int arrow_set_tuning(arrow_handle h, const arrow_tuning* t);

/* arrow_autotune -- time a fixed set of tunings (tile shapes 128/1024, 256/2048, 384/3072,
 * 512/4096 rows/entries x 2..4 CTAs per SM that fit, carveout fitted to them; then, for a small
 * problem, the one-launch path (fused_small); then the best multi-launch shape with
 * fold_permute_in switched) with arrow_spmm on the caller's X, Y (as arrow_spmm) for
 * `iters` iterations each (one warm-up call, two timed), keep the fastest on the handle, and
 * return it with its milliseconds per call.  Synchronises `stream`.
 * Errors: as arrow_spmm and arrow_set_tuning. */
int arrow_autotune(arrow_handle h, const void* X, void* Y, int64_t k, int32_t iters, int32_t x_dtype,
                   int32_t flags, void* stream, arrow_tuning* best, double* best_ms);


/* arrow_decompose -- LA-Decompose(A, b) of Section 4.1 on the host, then (unless
 * opts->flags has ARROW_HOST_ONLY) upload of the decomposition to the device.
 *   A    : host CSR as above (copied; may be freed after return).
 *   b    : arrow width, b >= 2 (Section 4.1 requires b >= 2); b >= n gives one level.
 *   o    : options, or NULL for arrow_opts_default().
 *   out  : receives the handle; *out is set to NULL on failure.
 * Levels are built until no entry of A is left (the paper's stop rule "nnz(A_i) <= 2b"
 * read as "empty").  Errors: ARROW_EINVAL (bad CSR, b < 2, too many levels),
 * ARROW_ENOMEM, ARROW_ECUDA (upload).  On error nothing is leaked. */
int arrow_decompose(const arrow_csr* A, int64_t b, const arrow_opts* o, arrow_handle* out);

/* Upload a handle built with ARROW_HOST_ONLY to the current (or opts.device) GPU; the
 * caller's current device is left as it was.  No-op if already uploaded.
 * Errors: ARROW_ENOMEM, ARROW_ECUDA. */
int arrow_upload(arrow_handle h);

/* arrow_handle_copy -- a second handle with the same decomposition (no re-decomposition),
 * storing A's values in value_dtype; uploaded if h is.  *out is NULL on failure.
 * Errors: ARROW_EINVAL, ARROW_ENOMEM, ARROW_ECUDA. */
int arrow_handle_copy(arrow_handle h, int32_t value_dtype, arrow_handle* out);

/* arrow_save -- write the handle's host state (input copy, every level's permutation and
 * structure, the fused row program) to a binary file with a checksum, so that a
 * decomposition computed once (the expensive offline step, Section 6) can be reused.
 * Errors: ARROW_EINVAL (NULL, cannot write). */
int arrow_save(arrow_handle h, const char* path);

/* arrow_load -- read a file written by arrow_save.  o (may be NULL = as saved) overrides
 * value_dtype (-1 keeps the saved one), flags (ARROW_HOST_ONLY) and device; the handle is
 * uploaded unless host-only.
 * Errors: ARROW_EINVAL (missing, truncated, corrupt or inconsistent file), ARROW_ENOMEM,
 * ARROW_ECUDA. */
int arrow_load(const char* path, const arrow_opts* o, arrow_handle* out);

/* Release the handle and all host and device memory it owns.  NULL-safe.
 * Must not be called while work that uses the handle is still running on a stream. */
void arrow_free(arrow_handle h);

/* ---- the hot path ------------------------------------------------------------------ */
#define ARROW_RESCALE 0x1   /* spmm flags: sigma = per-column L2 normalisation (FP64 norms) */
#define ARROW_PROFILE 0x2   /* spmm flags: record CUDA events around every kernel launch  */
#define ARROW_RELU    0x8   /* spmm flags: sigma includes the rectifier max(0, y)          */
#define ARROW_ROWNORM 0x10  /* spmm flags: sigma includes the per-row L2 normalisation     */

/* arrow_spmm -- iters steps of X_{t+1} = sigma(A X_t), X_0 = X, result X_iters in Y.
 * A is applied as sum_i P_i B_i P_i^T X (Eq. 1, Alg. 1 / Alg. 2 computed on one GPU):
 * X is permuted into the first level's order once, every step runs the split head-row
 * reduction and the fused arrow-row kernel (all levels, fixed level order, no atomics),
 * and the result is permuted back once (Section 5.1: rows stay in pi_0 order between
 * iterations).  sigma (Section 2 leaves it to the application) is composed from three
 * optional parts in a fixed order, sigma(Y) = colnorm(rownorm(relu(Y))):
 *   ARROW_RELU    -- max(0, y) on every element (the non-linearity of a graph-network
 *                    layer, the use the introduction motivates), fused into the row store;
 *   ARROW_ROWNORM -- every row divided by its L2 norm (zero rows stay zero), fused into the
 *                    row store; needs k / (16 / sizeof(x_dtype)) <= 32;
 *   ARROW_RESCALE -- every column divided by its L2 norm, reduced in FP64 (power/Lanczos).
 * No flag: sigma is the identity.
 *   h       : uploaded handle.
 *   X, Y    : DEVICE pointers, row-major n x k, element type x_dtype, caller-owned.
 *             X and Y may be the same buffer.  Both must be 16-byte aligned.
 *   k       : columns; k * sizeof(x_dtype) must be a multiple of 16 and
 *             k / (16 / sizeof(x_dtype)) a power of two <= 32, or a multiple of 32.
 *   iters   : >= 0; iters = 0 copies X to Y.
 *   x_dtype : arrow_dtype of X and Y (FP32 accumulation in every case).
 *   flags   : 0 or any of ARROW_RESCALE, ARROW_RELU, ARROW_ROWNORM, ARROW_PROFILE.
 *   stream  : cudaStream_t; the call only enqueues work (no host synchronisation), except
 *             that the first call for a given (k, x_dtype) allocates the handle's workspace.
 * The handle's device must be the current device (ARROW_EINVAL otherwise, nothing launched).
 * Errors: ARROW_EINVAL, ARROW_ESTATE (not uploaded), ARROW_ENOMEM, ARROW_ECUDA. */
int arrow_spmm(arrow_handle h, const void* X, int64_t k, int32_t iters, void* Y,
               int32_t x_dtype, int32_t flags, void* stream);

/* Workspace bytes arrow_spmm_ws needs for (k, x_dtype, flags). */
int arrow_workspace_size(arrow_handle h, int64_t k, int32_t x_dtype, int32_t flags, size_t* bytes);

/* arrow_spmm with caller-provided DEVICE workspace (256-byte aligned, >= the size from
 * arrow_workspace_size).  Makes no allocation; calls with distinct workspaces on
 * distinct streams may overlap on one handle (the handle's device data is read-only). */
int arrow_spmm_ws(arrow_handle h, const void* X, int64_t k, int32_t iters, void* Y,
                  int32_t x_dtype, int32_t flags, void* workspace, size_t ws_bytes, void* stream);

/* arrow_spmm_static -- arrow_spmm for callers that cannot allocate device memory.
 * The paper has no counterpart; it exists for code that must not call cudaMalloc: plugins
 * running inside another framework or inference runtime that owns all device memory through
 * its own allocator, and latency-bound serving loops that forbid allocation after start-up
 * (cudaMalloc/cudaFree synchronise the device and can stall every stream).  Same arguments
 * and result as arrow_spmm (X, Y on the device, caller-owned), but the scratch lives in one
 * file-scope device array of 64 MiB that every GPU loading the library holds until the
 * process exits.  Problems whose scratch (two n x k feature buffers, split-row partials,
 * FP64 norm sums: the arrow_workspace_size value) exceeds 64 MiB -- about 500,000 rows at
 * k = 16 in FP32 -- are rejected with ARROW_EINVAL.  The call allocates nothing.  The
 * handle's device must be current.  The first call in each CUDA context looks up the
 * array's device address (cudaGetSymbolAddress) and caches it for that context: make that
 * first call before any stream capture.  All calls share the array and it keeps the last
 * call's contents, so calls whose work overlaps on the GPU (other streams, other threads,
 * other handles) race: serialise them.  ARROW_PROFILE is rejected (it creates events).
 * Errors: ARROW_EINVAL, ARROW_ESTATE, ARROW_ECUDA. */
int arrow_spmm_static(arrow_handle h, const void* X, int64_t k, int32_t iters, void* Y,
                      int32_t x_dtype, int32_t flags, void* stream);

/* ---- batches: many matrices advanced together --------------------------------------- */
#define ARROW_GRAPH 0x4   /* arrow_batch_spmm flags: capture the call once as a CUDA graph, replay it */

typedef struct arrow_batch_s* arrow_batch;   /* opaque, library-owned */

/* arrow_batch_create -- group count uploaded handles (same device, same value dtype) so that
 * one call advances all of them.  The handles must outlive the batch.  A member handle may be
 * re-tuned (arrow_set_tuning) or re-uploaded between batch calls: the next arrow_batch_spmm
 * sees it, waits for its stream and rebuilds the batch's work-unit tables, descriptors and
 * graph.  Not in the paper (its matrices are advanced by separate rank groups, Alg. 2); this
 * is the one-GPU batching of many independent problems.  Errors: ARROW_EINVAL, ARROW_ESTATE
 * (a handle not uploaded), ARROW_ECUDA. */
int arrow_batch_create(const arrow_handle* handles, int32_t count, arrow_batch* out);

/* arrow_batch_spmm -- for every matrix m: Y[m] = A_m^iters X[m] (sigma = identity), with
 * X[m], Y[m] DEVICE pointers (host arrays of count pointers), row-major n_m x k[m], 16-byte
 * aligned, element type x_dtype; k[m] = V * 2^j with V = 16 / sizeof(x_dtype) and k[m] / V <= 32.
 * Each iteration of the whole batch is one launch per kernel class (split-row segments,
 * rows, split-row combine) over the work units of all matrices; the permutes are one launch
 * each.  Results are bit-identical to arrow_spmm on each matrix alone.  flags: 0 or
 * ARROW_GRAPH (capture once, replay while X, Y, k, iters and dtype stay the same).  The call
 * allocates its workspace on first use or growth (outside any capture) and synchronises
 * the stream when X, Y, k or dtype change.  The batch's device must be current (ARROW_EINVAL
 * otherwise, nothing launched).  Errors: ARROW_EINVAL, ARROW_ECUDA. */
int arrow_batch_spmm(arrow_batch b, const void* const* X, void* const* Y, const int64_t* k, int32_t iters,
                     int32_t x_dtype, int32_t flags, void* stream);

/* arrow_batch_autotune -- arrow_autotune for a whole batch: each candidate tuning is applied to
 * every handle of the batch, the batch (as arrow_batch_spmm, ARROW_GRAPH) is timed, and the
 * fastest is kept on all handles.  Synchronises `stream`. */
int arrow_batch_autotune(arrow_batch b, const void* const* X, void* const* Y, const int64_t* k, int32_t iters,
                         int32_t x_dtype, void* stream, arrow_tuning* best, double* best_ms);

/* Read and clear the batch's device status word (see arrow_status). */
int arrow_batch_status(arrow_batch b, int32_t* status);

/* Release the batch (not its handles).  NULL-safe. */
void arrow_batch_free(arrow_batch b);

/* ---- serving: continuous batching of requests ---------------------------------------- */
/* Not in the paper.  A request is (decomposed matrix, X, Y, k, iters); the server keeps the
 * matrices and the requests' state on the device and advances every admitted request by one
 * iteration per step, all of them in the same launches (continuous batching). */
typedef struct arrow_server_s* arrow_server;   /* opaque, library-owned */

typedef struct {
    int64_t hbm_budget;    /* bytes of device memory for request state (allocated once, up front) */
    int32_t max_active;    /* slots: requests advanced together, 1..4096                          */
    int32_t x_dtype;       /* arrow_dtype of every request's X and Y                               */
    int32_t max_inflight;  /* steps queued on the GPU before a step waits for the oldest; 0 = 2    */
    int32_t device;        /* CUDA device ordinal; -1 = current                                    */
} arrow_server_opts;

typedef struct {
    int64_t queued, active, inflight_steps, completed, steps;
    int64_t bytes_in_use, peak_bytes;   /* request state in the budget (peak <= hbm_budget) */
    int32_t status;                     /* device status word (0 = no wait ran out)          */
    double  host_seconds;   /* time spent in arrow_server_step on the host, without the waits */
    double  wait_seconds;   /* time arrow_server_step spent waiting for the GPU (max_inflight) */
    double  gpu_seconds;    /* device time of the retired steps (event before to event after) */
} arrow_server_stats;

/* Create a server; allocates hbm_budget bytes of device memory and a few pinned staging
 * buffers.  Errors: ARROW_EINVAL (bad options), ARROW_ENOMEM, ARROW_ECUDA. */
int arrow_server_create(const arrow_server_opts* o, arrow_server* out);

/* Queue a request: Y = A^iters X for the uploaded handle h; X, Y DEVICE pointers (n x k,
 * 16-byte aligned, caller-owned, valid until the request completes); k as for
 * arrow_batch_spmm.  All handles served must store values in one dtype.  Its state needs
 * 2 n k sizeof(x_dtype) + (split-row segments) k 4 bytes of the budget while active.
 * *id identifies it in arrow_server_poll.  Errors: ARROW_EINVAL, ARROW_ESTATE. */
int arrow_server_submit(arrow_server s, arrow_handle h, const void* X, void* Y, int64_t k, int32_t iters,
                        int64_t* id);

/* One step: retire requests the GPU has finished, admit queued requests in arrival order
 * while a slot and budget are free, launch one iteration of every active request (plus the
 * permute-in of new ones and the permute-out of finishing ones) on `stream`, which must be
 * the same for every step.  Waits for the oldest step only when max_inflight steps are queued.
 * The server's device must be current (ARROW_EINVAL otherwise, nothing launched).
 * *active receives the number of active requests (may be NULL).  Errors: ARROW_EINVAL, ARROW_ECUDA. */
int arrow_server_step(arrow_server s, void* stream, int32_t* active);

/* Completed requests since the last poll: up to max (id, latency = device completion time -
 * submission time, seconds) pairs; *count receives how many.  Non-blocking. */
int arrow_server_poll(arrow_server s, int64_t* ids, double* latency_s, int32_t max, int32_t* count);

/* Step (on `stream`, as arrow_server_step) until every queued and active request has
 * completed, then wait for the GPU. */
int arrow_server_drain(arrow_server s, void* stream);

int arrow_server_get_stats(arrow_server s, arrow_server_stats* st);

/* Synchronise the server's stream and release everything it owns (not the handles).  NULL-safe. */
void arrow_server_free(arrow_server s);

/* ---- structure export (parity tests, reports) ------------------------------------ */
/* Number of levels l (order of the decomposition). */
int arrow_num_levels(arrow_handle h, int32_t* l);
/* Level i: active rows n_i (1 + largest position touched by an entry of B_i) and nnz(B_i). */
int arrow_level_info(arrow_handle h, int32_t i, int64_t* n_active, int64_t* nnz);
/* Level i: perm_out[v] = pi_i(v), the position of vertex v (host buffer of n int32). */
int arrow_level_perm(arrow_handle h, int32_t i, int32_t* perm_out);
/* Level i: B_i in CSR over positions 0..n-1 (host buffers: rowptr n+1, colidx and vals
 * nnz(B_i)); columns ascending in each row; values are A's float64 values. */
int arrow_level_csr(arrow_handle h, int32_t i, int64_t* rowptr, int32_t* colidx, double* vals);

/* Where the entries of B_i sit under the b x b tiling of Section 3.1 / Fig. 2: in the head
 * rows or head columns (position < b; the part pruned towards the top and left corners in
 * the discussion of the decomposition results, Section 6), or elsewhere (the diagonal tiles
 * for ARROW_PRED_BLOCK, the band for ARROW_PRED_BAND), and how many distinct b x b tiles hold
 * an entry.  head_nnz + band_nnz = nnz.  Host computation, O(nnz(A) + n). */
typedef struct {
    int64_t n_active;   /* as arrow_level_info */
    int64_t nnz;        /* nnz(B_i) */
    int64_t head_nnz;   /* entries (p, q) of B_i with p < b or q < b */
    int64_t band_nnz;   /* the other entries of B_i */
    int64_t tiles;      /* distinct (p / b, q / b) over the entries of B_i */
} arrow_level_shape;
/* Errors: ARROW_EINVAL (NULL argument, level out of range). */
int arrow_get_level_shape(arrow_handle h, int32_t i, arrow_level_shape* out);

/* The fused row program the device kernels run (host copy; read-only views that stay valid
 * until the handle is freed, re-tuned or reloaded).  Rows are pi_0 positions.  Every level's
 * entries of the vertex at position p sit in row p, in level order and, inside a level, in
 * increasing level position of the column (the write-back of Alg. 2 with destinations fixed
 * at preprocessing, Thm. 5.2); each entry names the pi_0 position of the X row it reads (the
 * level shuffle of Alg. 2 folded into the index) and the index of its value in A.  Rows with
 * more than long_row entries are split: their short range is empty and their entries sit in
 * the long stream, cut into segments of at most `segment` entries (Alg. 1's head-row
 * reduction in two fixed-order stages).  Tiles cut the short rows into the units the rows
 * kernel stages into shared memory.  Exported for tests and reports. */
typedef struct {
    int64_t n, n_short, n_long_entries, n_long_rows, n_segments, n_tiles;
    int32_t long_row;
    const int32_t* rowptr;      /* [n+1] short rows */
    const int32_t* col;         /* [n_short] pi_0 position read */
    const int32_t* src;         /* [n_short] index of the entry in A */
    const int32_t* lcol;        /* [n_long_entries] */
    const int32_t* lsrc;        /* [n_long_entries] */
    const int32_t* long_rows;   /* [n_long_rows] split rows, ascending */
    const int32_t* long_segptr; /* [n_long_rows+1] first segment of each split row */
    const int32_t* seg_begin;   /* [n_segments] entry range of each segment in the long stream */
    const int32_t* seg_end;     /* [n_segments] */
    const int32_t* tile_row;    /* [n_tiles+1] first row of each tile */
    const int32_t* tile_ent;    /* [n_tiles+1] first short entry of each tile */
} arrow_program;
/* Errors: ARROW_EINVAL (NULL argument). */
int arrow_get_program(arrow_handle h, arrow_program* out);

/* Number of distinct non-zero b x b tiles of A in its own row and column order: the equally
 * sized blocks a 1.5D distribution deals out, against which Section 6 counts the non-zero
 * blocks of the decomposition.  A as for arrow_decompose (host CSR, read only); b >= 1.
 * Errors: ARROW_EINVAL (bad CSR, b < 1, NULL tiles). */
int arrow_count_tiles(const arrow_csr* A, int64_t b, int64_t* tiles);

typedef struct {
    int64_t n, nnz, b;
    int32_t levels;
    int32_t value_dtype;
    int64_t long_rows;       /* rows split into segments (head rows of hubs)        */
    int64_t segments;        /* segments of the split rows                           */
    int64_t tiles;           /* row tiles of the fused row program                   */
    int64_t device_bytes;    /* bytes of device memory owned by the handle (no workspace) */
    double  decompose_seconds;
} arrow_stats;
int arrow_get_stats(arrow_handle h, arrow_stats* s);

/* Kernel classes reported by arrow_profile_get. */
#define ARROW_K_ROWS     0   /* fused arrow-row kernel (band rows, folded levels, write-back) */
#define ARROW_K_SEGMENTS 1   /* split-row segment kernel (first stage of the head-row reduction) */
#define ARROW_K_NORM     2   /* FP64 column-norm finalize                                    */
#define ARROW_K_PERMUTE  3   /* permute-in / permute-out gathers                             */
#define ARROW_K_FUSED    4   /* the one-launch path (whole call in one cooperative kernel)   */

/* arrow_profile_get -- device time of the launches recorded by arrow_spmm calls made with
 * ARROW_PROFILE since the last arrow_profile_get, for one kernel class: total milliseconds
 * and number of launches.  Synchronises on the recorded events, then forgets them.
 * The events are measured on the stream the kernels were launched on. */
int arrow_profile_get(arrow_handle h, int32_t kernel, double* total_ms, int64_t* launches);

/* arrow_status -- synchronously read and clear the handle's device status word.  Kernels
 * that wait on bulk copies give every wait a 2 s limit; when one runs out the kernel sets
 * the word, waits (bounded) for its copies in flight and returns, so the context stays
 * usable.  Returns ARROW_OK with *status = 0, or ARROW_ETIMEOUT with *status != 0. */
int arrow_status(arrow_handle h, int32_t* status);

/* arrow_selftest_timeout -- runs the bounded-wait path on purpose: a one-block kernel
 * waits on an mbarrier that nothing completes, gives up after limit_ns (0 < limit <= 10 s)
 * and sets its status word, which is copied to *status (1 = the wait ran out, as expected).
 * Touches no handle; the context stays usable.  Errors: ARROW_EINVAL, ARROW_ECUDA. */
int arrow_selftest_timeout(int64_t limit_ns, int32_t* status);

/* arrow_selftest_grid_timeout -- runs the one-launch path's grid-barrier timeout on purpose: a
 * cooperative launch of `blocks` blocks (2 <= blocks <= SMs) in which block 0 never arrives, so
 * every other block's barrier wait gives up after limit_ns (0 < limit <= 10 s) and returns;
 * *gave_up receives how many blocks gave up (blocks - 1 expected).  Touches no handle; the
 * context stays usable.  Errors: ARROW_EINVAL, ARROW_ECUDA. */
int arrow_selftest_grid_timeout(int64_t limit_ns, int32_t blocks, int32_t* gave_up);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* arrow_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ARROW_GB300_H */
