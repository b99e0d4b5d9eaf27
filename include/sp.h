/*
 * sp.h -- C ABI of the GB300 library for sparse matrix permutation, extraction and
 * assignment on CSR matrices (arXiv 2509.20776: HipPerm, HipExtract, HipAssign).
 *
 * Conventions for every entry point
 *  - Indices are 0-based (the paper writes them 1-based).
 *  - All array pointers are DEVICE pointers of the context's device unless a
 *    parameter says "host".  Scalars and descriptors (sp_csr) live in host memory.
 *  - Every call is stream-ordered on `stream` (a cudaStream_t; NULL is the legacy
 *    default stream) and returns without waiting for the GPU unless it says
 *    "synchronises".  Inputs must stay valid and unmodified until the work is done.
 *  - Host-detectable errors (null pointers, shapes, types, sizes) are returned
 *    immediately and nothing is launched.  Errors found on the device (index out of
 *    range, repeated index, p not a permutation, look-back timeout) are recorded in
 *    the context and returned by the next synchronising call on it (sp_ctx_sync,
 *    sp_extract_count, sp_assign_count, ...); the outputs of the failed call are then
 *    unspecified.
 *  - A context's workspace is shared by all calls made through it: calls through one
 *    context must be ordered (same stream, or synchronised between streams).  Use one
 *    context per concurrently used stream.
 *  - Matrices are canonical CSR: row pointer non-decreasing from 0 to nnz, column
 *    indices in [0, ncols) and strictly ascending within each row.  Inputs are
 *    assumed canonical (check with sp_csr_validate); outputs always are.
 *  - Values are moved as opaque 4- or 8-byte words: no arithmetic touches them
 *    (except SP_ASSIGN_PLUS), so -0.0, NaN payloads and stored zeros are preserved.
 */
#ifndef SP_H_
#define SP_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SP_API __attribute__((visibility("default")))
#else
#define SP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sp_stream_t; /* identical to cudaStream_t */

/* Width of row pointers, column indices and index vectors. */
typedef enum sp_itype { SP_I32 = 0, SP_I64 = 1 } sp_itype;
/* Width of values: fp32 or fp64 (moved as 4- or 8-byte words). */
typedef enum sp_vtype { SP_F32 = 0, SP_F64 = 1 } sp_vtype;

typedef enum sp_status {
  SP_OK = 0,
  SP_ERR_INVALID_ARG = 1,     /* null pointer, bad enum, inconsistent descriptor */
  SP_ERR_SHAPE = 2,           /* dimensions or vector lengths do not match */
  SP_ERR_INDEX_RANGE = 3,     /* an index vector entry lies outside its dimension */
  SP_ERR_DUPLICATE_INDEX = 4, /* an index vector that must be distinct repeats a value */
  SP_ERR_NOT_PERMUTATION = 5, /* p or q is not a permutation of its dimension */
  SP_ERR_NOT_CANONICAL = 6,   /* an input matrix is not canonical CSR (sp_csr_validate) */
  SP_ERR_OVERFLOW = 7,        /* a result does not fit the requested index width */
  SP_ERR_OOM = 8,             /* the allocator returned NULL */
  SP_ERR_TIMEOUT = 9,         /* a bounded device-side wait gave up (no hang) */
  SP_ERR_CUDA = 10,           /* a CUDA runtime call failed */
  SP_ERR_INTERNAL = 11        /* an internal invariant failed (a library bug) */
} sp_status;

/* How sp_assign combines B with the region A(I, J) (Sec. 2.3, "Variants of matrix
 * assignment"). */
typedef enum sp_assign_mode {
  SP_ASSIGN_REPLACE = 0,   /* overwrite: A(I,J) is cleared, then B is written; afterwards
                              A'(I,J) == B exactly */
  SP_ASSIGN_SELECT2ND = 1, /* A (+) P B Q^T with select-second: A's entries inside the
                              region that B does not store survive; B wins ties */
  SP_ASSIGN_PLUS = 2       /* A (+) P B Q^T with arithmetic add: where both store an
                              entry, one IEEE round-to-nearest add a + b in the value type */
} sp_assign_mode;

/* A CSR matrix descriptor (host struct, device arrays).
 *   rowptr: nrows+1 entries of rowptr_type; colidx: nnz entries of colidx_type;
 *   values: nnz entries of value_type. */
typedef struct sp_csr {
  int64_t nrows, ncols, nnz;
  sp_itype rowptr_type;
  sp_itype colidx_type;
  sp_vtype value_type;
  void* rowptr;
  void* colidx;
  void* values;
} sp_csr;

/* Device-memory allocator hook.  alloc returns device memory usable on `stream` (or
 * NULL on failure); free releases it after the work queued on `stream`.  A NULL
 * allocator in sp_ctx_create selects stream-ordered cudaMallocAsync/cudaFreeAsync. */
typedef struct sp_allocator {
  void* (*alloc)(void* user, size_t bytes, sp_stream_t stream);
  void (*free)(void* user, void* ptr, size_t bytes, sp_stream_t stream);
  void* user;
} sp_allocator;

typedef struct sp_ctx sp_ctx;   /* device, allocator, workspace, device error record */
typedef struct sp_plan sp_plan; /* state kept between a count call and its fill call */

/* Human-readable name of a status code (static string, never NULL). */
SP_API const char* sp_status_str(sp_status s);

/* Library ABI version (major*10000 + minor*100 + patch). */
SP_API int sp_version(void);

/* Create a context on CUDA device `device`.  `allocator` may be NULL (see
 * sp_allocator); it is copied.  *ctx receives the new context.  A context is used by
 * one host thread at a time (its workspace, options and per-call kernel shapes are not
 * locked); work from several threads or streams in parallel takes one context each.
 * Errors: SP_ERR_INVALID_ARG (ctx NULL), SP_ERR_CUDA (device unusable). */
SP_API sp_status sp_ctx_create(sp_ctx** ctx, int device, const sp_allocator* allocator);

/* Destroy a context: waits for the device, frees its workspace.  NULL is a no-op. */
SP_API sp_status sp_ctx_destroy(sp_ctx* ctx);

/* Synchronises `stream`, then returns and clears the first device-detected error
 * recorded since the last synchronising call (SP_OK if none). */
SP_API sp_status sp_ctx_sync(sp_ctx* ctx, sp_stream_t stream);

/* Host: detail of the last error returned by a synchronising call (for index errors
 * the offending position in the index vector; -1 if none). */
SP_API int64_t sp_ctx_error_detail(const sp_ctx* ctx);

/* Host: the CUDA runtime error code behind the calling thread's most recent
 * SP_ERR_CUDA (0 if there was none), and in *where (may be NULL) a static string
 * naming the library source line and the error ("file.cu:123 (cudaErrorXxx)"). */
SP_API int sp_last_cuda_error(const char** where);

/* Tuning and test knobs (values < 0 restore the default):
 *   SP_OPT_SPIN_LIMIT      polls a look-back wait makes before it gives up with
 *                          SP_ERR_TIMEOUT (default 1<<22, each poll sleeps ~100 ns);
 *   SP_OPT_SCAN_HOLD_TILE  test hook: the scan tile with this index never publishes
 *                          its status, so its successors' bounded waits run out and
 *                          the call reports SP_ERR_TIMEOUT (default -1 = off);
 *   SP_OPT_VALIDATE        1: every op first checks its input matrices are canonical
 *                          (SP_ERR_NOT_CANONICAL); default 0. */
/* Kernel shapes (the autotuner's knobs; every value gives the same output, bit for bit):
 *   SP_OPT_TILE_SHAPE      row sort of short rows: 0 = tiles of 1024 entries holding rows
 *                          of at most 512, 128 threads, 9 CTAs per SM (default);
 *                          1 = tiles of 2048 entries holding rows of at most 1024,
 *                          256 threads, 4 CTAs per SM;
 *   SP_OPT_HEAVY           a bucket of the row sort with more keys than this is written
 *                          in bucket order and sorted by a later pass: 128 (default) to
 *                          4096;
 *   SP_OPT_COUNT_ROWS      rows a warp takes per step in the kept-entry count of
 *                          assignment: 1 to 4 (default 4);
 *   SP_OPT_FILL_ROWS       the same for its compacting fill: 1 or 2 (default 2);
 *   SP_OPT_BATCH_ROWS      rows a warp serves at once in the batched extraction's count
 *                          and fill (32 / rows lanes per row): 1 (default), 2, 4 or 8;
 *   SP_OPT_IDENTIFY        how an extraction identifies the kept columns (general or
 *                          ascending J, and every request of a batch): 0 = rank map over
 *                          the columns (a membership bit and a rank per column, one
 *                          position per member of J: n/4 + |J| * idx bytes, two lookups
 *                          per entry; default; a batch whose maps would exceed 16 GB uses
 *                          1); 1 = J sorted once, binary search per stored entry
 *                          (Algorithm 5's search: |J| log |J| set-up, no column-sized
 *                          table). */
/* Scheduling (same output either way):
 *   SP_OPT_OVERLAP         1 (default): phases that write disjoint rows run side by side,
 *                          one of them on the context's own side stream (created with the
 *                          device's highest stream priority): a row sort's key-range
 *                          split of the rows longer than 4096 entries beside the tile sort
 *                          of its short rows, and an assignment's copy of the rows outside
 *                          I beside the merge of the rows of I (REPLACE); the side work is
 *                          forked from and joined back to the caller's stream with events,
 *                          so the call stays ordered on that stream and capturable;
 *                          0: every launch on the caller's stream. */
typedef enum sp_option {
  SP_OPT_SPIN_LIMIT = 0,
  SP_OPT_SCAN_HOLD_TILE = 1,
  SP_OPT_VALIDATE = 2,
  SP_OPT_TIMING = 3, /* 1: bracket every kernel launch with CUDA events (see below) */
  SP_OPT_TILE_SHAPE = 4,
  SP_OPT_HEAVY = 5,
  SP_OPT_COUNT_ROWS = 6,
  SP_OPT_FILL_ROWS = 7,
  SP_OPT_BATCH_ROWS = 8,
  SP_OPT_IDENTIFY = 9,
  SP_OPT_OVERLAP = 10
} sp_option;
SP_API sp_status sp_ctx_set_option(sp_ctx* ctx, sp_option key, int64_t value);

/* Tuning table (written by the autotuner, paper_2509_20776_gb300/autotune.py).  Each
 * call of an operation takes the first entry with its op whose size_max is at least the
 * call's size, and uses that entry's kernel shapes (fields < 0 keep the context's
 * option) for this call only.  Size: nnz(A) for permute / extract / assign (and the
 * fused assign + permute), the total number of selected rows (sum of |I|) for a batch.
 * The table is copied; n = 0 removes it.  Errors: SP_ERR_INVALID_ARG for a NULL ctx, a
 * NULL table with n > 0, n < 0, an unknown op or an out-of-range shape value. */
typedef enum sp_op { SP_OP_PERMUTE = 0, SP_OP_EXTRACT = 1, SP_OP_ASSIGN = 2, SP_OP_BATCH = 3 } sp_op;
typedef struct sp_tune_entry {
  int32_t op;        /* sp_op */
  int32_t tile_shape, heavy, count_rows, fill_rows, batch_rows, identify; /* as the options above */
  int64_t size_max;  /* the entry covers calls of size <= size_max */
} sp_tune_entry;
SP_API sp_status sp_ctx_set_tuning(sp_ctx* ctx, const sp_tune_entry* table, int n);
/* Host only (no device work): the entry of `table` (n entries) that a call of `op` with
 * size `size` takes — the first entry with that op and size_max >= size — copied to
 * *out; returns 1 if one applies, 0 if none (then *out is untouched), -1 for a NULL
 * table with n > 0, n < 0 or a NULL out.  sp_ctx_set_tuning's lookup is this one. */
SP_API int sp_tuning_lookup(const sp_tune_entry* table, int n, int op, int64_t size, sp_tune_entry* out);

/* Per-phase kernel statistics (tracing).  Every kernel the library launches belongs to
 * one phase; the context counts launches per phase always, and with SP_OPT_TIMING=1
 * also records CUDA events around each launch on the launching stream.
 * sp_ctx_phase_stats waits for the recorded events, then writes SP_NUM_PHASES entries
 * to ms[] (summed device milliseconds) and launches[] (host arrays, either may be
 * NULL); reset != 0 clears the totals afterwards. */
typedef enum sp_phase {
  SP_PHASE_MAP = 0,       /* inverse maps, membership bitmaps, range checks */
  SP_PHASE_COUNT = 1,     /* kept-entry counting passes */
  SP_PHASE_SCAN = 2,      /* exclusive scans (row pointers) */
  SP_PHASE_PARTITION = 3, /* tile partition / row classification */
  SP_PHASE_TILE = 4,      /* in-place sort of short rows, many per CTA */
  SP_PHASE_LONG = 5,      /* in-place sort of rows / runs of up to 4096 entries, one CTA each */
  SP_PHASE_HUGE = 6,      /* key-range split of longer rows into runs */
  SP_PHASE_GATHER = 7,    /* load-balanced row gather / compacting fill into the output */
  SP_PHASE_OTHER = 8,     /* row-pointer width conversion, validation */
  SP_NUM_PHASES = 9
} sp_phase;
SP_API sp_status sp_ctx_phase_stats(sp_ctx* ctx, double* ms, int64_t* launches, int reset);
/* Static name of a phase ("map", "count", ...; "?" when out of range). */
SP_API const char* sp_phase_name(int phase);

/* ------------------------------------------------------------------------------
 * Permutation  (Sec. 2.1; HipPerm, Algorithm 1)
 *   B[i, j] = A[p[i], q[j]], i.e. B = P A Q^T with P[i, p[i]] = 1, Q[j, q[j]] = 1.
 *   p: A->nrows entries (new row -> old row), q: A->ncols entries (new column -> old
 *   column), both of idx_type; NULL means the identity.  q == p (same pointer) with a
 *   square A is the symmetric reordering P A P^T.
 *   B (host descriptor): on entry B->rowptr_type selects the output row-pointer width;
 *   colidx_type/value_type are taken from A.  If B->rowptr, B->colidx and B->values
 *   are all NULL the library allocates them through the context allocator (release
 *   with sp_csr_free); otherwise all three must be caller-owned device buffers of at
 *   least nrows+1 / nnz / nnz entries.  On return B's shape fields are set.
 *   Errors: SP_ERR_INVALID_ARG, SP_ERR_SHAPE, SP_ERR_OVERFLOW (nnz does not fit an
 *   int32 B->rowptr); on the device SP_ERR_INDEX_RANGE / SP_ERR_NOT_PERMUTATION.
 * ------------------------------------------------------------------------------ */
SP_API sp_status sp_permute(sp_ctx* ctx, const sp_csr* A, const void* p, const void* q,
                     sp_itype idx_type, sp_csr* B, sp_stream_t stream);

/* ------------------------------------------------------------------------------
 * Extraction  (Sec. 2.2; HipExtract, Algorithms 3 and 5)
 *   B = A(I, J): B[i, j] = A[I[i], J[j]] for (i, j) in I x J; B is nI x nJ.
 *   I: nI row indices (may repeat, any order); J: nJ column indices (any order; unsorted
 *   J permutes the columns of the result; a repeated column is copied under each of its
 *   positions).  Both of idx_type.  Consecutive J (J[k] = J[0] + k) takes a per-row
 *   binary search of the kept segment; ascending J needs no row sort.
 *
 * sp_extract_count: builds the column map and the row pointer of B, and returns the
 *   number of stored entries of B in *nnz_out (host).  Synchronises.  *plan receives
 *   the state needed by sp_extract_fill; it borrows A, I and J, which must stay valid
 *   until the plan is destroyed.
 * sp_extract_fill: writes B (same allocation rule as sp_permute; B->nnz must be the
 *   counted value when caller-owned).  The plan can be filled more than once.
 * sp_extract: count + allocate + fill in one call (synchronises once).
 *   Errors: SP_ERR_INVALID_ARG, SP_ERR_SHAPE, SP_ERR_OVERFLOW; from the device
 *   SP_ERR_INDEX_RANGE.
 * ------------------------------------------------------------------------------ */
SP_API sp_status sp_extract_count(sp_ctx* ctx, const sp_csr* A, const void* I, int64_t nI,
                           const void* J, int64_t nJ, sp_itype idx_type, sp_plan** plan,
                           int64_t* nnz_out, sp_stream_t stream);
SP_API sp_status sp_extract_fill(sp_ctx* ctx, sp_plan* plan, sp_csr* B, sp_stream_t stream);
SP_API sp_status sp_extract(sp_ctx* ctx, const sp_csr* A, const void* I, int64_t nI, const void* J,
                     int64_t nJ, sp_itype idx_type, sp_csr* B, sp_stream_t stream);

/* ------------------------------------------------------------------------------
 * Assignment  (Sec. 2.3; HipAssign, Algorithm 4)
 *   A' = A with A'(I, J) = B (REPLACE), or A (+) P B Q^T (SELECT2ND, PLUS); A is not
 *   modified.  I: nI distinct rows of A, J: nJ distinct columns of A (any order), both
 *   of idx_type; B: nI x nJ, with A's colidx and value types.
 *   The count/fill/one-shot split, plan lifetime and output allocation rules are those
 *   of extraction (the plan also borrows B).
 *   Errors: SP_ERR_INVALID_ARG, SP_ERR_SHAPE, SP_ERR_OVERFLOW; from the device
 *   SP_ERR_INDEX_RANGE, SP_ERR_DUPLICATE_INDEX.
 * ------------------------------------------------------------------------------ */
SP_API sp_status sp_assign_count(sp_ctx* ctx, const sp_csr* A, const void* I, int64_t nI,
                          const void* J, int64_t nJ, sp_itype idx_type, const sp_csr* B,
                          sp_assign_mode mode, sp_plan** plan, int64_t* nnz_out,
                          sp_stream_t stream);
SP_API sp_status sp_assign_fill(sp_ctx* ctx, sp_plan* plan, sp_csr* Aprime, sp_stream_t stream);
SP_API sp_status sp_assign(sp_ctx* ctx, const sp_csr* A, const void* I, int64_t nI, const void* J,
                    int64_t nJ, sp_itype idx_type, const sp_csr* B, sp_assign_mode mode,
                    sp_csr* Aprime, sp_stream_t stream);

/* Fused assignment + permutation (Sec. 6.3: incremental updates of a randomly permuted
 * matrix; the fused HipAssign + HipPerm of the experiments):
 *   out = P (A (+) B') Q^T, i.e. out[i, j] = A'[p[i], q[j]] with A' = sp_assign(A, I, J, B,
 *   mode), computed without forming A'.
 *   sp_assign_permute_fill takes a plan from sp_assign_count (which fixes I, J, B, mode
 *   and the output nnz) and writes out; the plan stays valid.  p: nrows entries, q: ncols
 *   entries (permutations of the plan's idx_type, or NULL for the identity; q == p gives
 *   P A' P^T).  out: rowptr_type chosen by the caller, arrays caller-allocated (nnz from
 *   the count) or all NULL (library-allocated).  sp_assign_permute = count + fill and
 *   synchronises once.  Errors: those of sp_assign and sp_permute. */
SP_API sp_status sp_assign_permute_fill(sp_ctx* ctx, sp_plan* plan, const void* p, const void* q,
                                        sp_csr* out, sp_stream_t stream);
SP_API sp_status sp_assign_permute(sp_ctx* ctx, const sp_csr* A, const void* I, int64_t nI,
                                   const void* J, int64_t nJ, sp_itype idx_type, const sp_csr* B,
                                   sp_assign_mode mode, const void* p, const void* q, sp_csr* out,
                                   sp_stream_t stream);

/* ------------------------------------------------------------------------------
 * Batched extraction (the batching pattern for serving many small requests; no
 * counterpart in the paper, whose Algorithm 5 binary search per (i, j) it reuses for
 * identification)
 *   B_k = A_{mat}(I_k, J_k) for nreq requests over nmats device-resident matrices, all
 *   matrices of one type combination; I_k may repeat, J_k distinct (idx_type; device
 *   pointers).  Every step runs once for the whole batch (a fixed number of launches).
 * sp_extract_batch_count: validates the requests, sorts every J_k, counts the kept
 *   entries of every output row and returns the batch's total in *nnz_total (host).
 *   Synchronises once.  *batch keeps the sorted J's and the row pointer; it borrows the
 *   matrices and the index vectors until destroyed.
 * sp_extract_batch_fill: writes all results into one CSR `out`: the rows of request k
 *   are rows [sp_batch_row_offset(k), sp_batch_row_offset(k+1)) with column j meaning
 *   position j of J_k; out has sum(nI) rows and max(nJ) columns.  out's arrays must be
 *   caller-allocated (nnz from the count, A's colidx / value types, any rowptr type).
 *   Never synchronises and allocates nothing, so it can be captured in a CUDA graph
 *   and replayed while the inputs keep their addresses.
 *   Errors: SP_ERR_INVALID_ARG, SP_ERR_SHAPE, SP_ERR_OVERFLOW; from the device
 *   SP_ERR_INDEX_RANGE, SP_ERR_DUPLICATE_INDEX.
 * ------------------------------------------------------------------------------ */
typedef struct sp_extract_req {
  int64_t mat;    /* index of the matrix in mats */
  int64_t nI, nJ; /* lengths of I and J */
  const void* I;  /* device, nI row indices */
  const void* J;  /* device, nJ distinct column indices */
} sp_extract_req;
typedef struct sp_batch sp_batch;

SP_API sp_status sp_extract_batch_count(sp_ctx* ctx, const sp_csr* mats, int64_t nmats,
                                        const sp_extract_req* reqs, int64_t nreq, sp_itype idx_type,
                                        sp_batch** batch, int64_t* nnz_total, sp_stream_t stream);
SP_API sp_status sp_extract_batch_fill(sp_ctx* ctx, sp_batch* batch, sp_csr* out, sp_stream_t stream);
/* sp_extract_batch_run: the whole batch again on the device -- identification, kept
 *   counts, row pointer, fill and row sort -- into `out` (arrays as for the fill, the
 *   counted nnz being their capacity).  It reads I_k and J_k when it runs, allocates
 *   nothing (the count reserved its workspace) and never synchronises, so count, fill
 *   and sort replay together from one CUDA graph while the inputs keep their addresses
 *   and sizes.  If the inputs now select more entries than the counted nnz, the row
 *   pointer is clamped to it, SP_ERR_OVERFLOW is recorded for sp_ctx_sync and the
 *   output is not the extraction (no write leaves its arrays).  Errors: as the fill. */
SP_API sp_status sp_extract_batch_run(sp_ctx* ctx, sp_batch* batch, sp_csr* out, sp_stream_t stream);
/* First output row of request k (k = nreq gives the total); -1 for a bad k. */
SP_API int64_t sp_batch_row_offset(const sp_batch* batch, int64_t k);
/* Release a batch (stream-ordered on the stream of its count).  NULL is a no-op. */
SP_API sp_status sp_batch_destroy(sp_ctx* ctx, sp_batch* batch);

/* ------------------------------------------------------------------------------
 * Batched permutation (the same batching pattern; no counterpart in the paper)
 *   B_k = P_k A_{mat} Q_k^T, B_k[i, j] = A_{mat}[p_k[i], q_k[j]] (Sec. 2.1) for nreq
 *   requests over nmats device-resident matrices of one type combination; p_k (nrows
 *   entries) and q_k (ncols entries) of idx_type, device pointers, NULL = identity.
 * sp_permute_batch_plan: host only, no device synchronisation.  Lays out the batch
 *   (a permutation keeps every entry, so the output size is known: *nnz_total = the
 *   sum of the matrices' nnz over the requests) and allocates one device buffer
 *   (inverse column maps, row bitmaps, the row table, the row pointer, the row-sort
 *   workspace), whose request tables it writes on `stream` by small kernel launches
 *   (no copy from pageable memory, which would wait for the stream's earlier work): a
 *   fill on another stream must be ordered after it.  *plan borrows the matrices and p_k, q_k until
 *   destroyed; the fill reads p_k and q_k when it runs, so a replayed graph picks up
 *   new permutations written into the same buffers.
 * sp_permute_batch_fill: runs the whole batch on `stream` (per request the inverse
 *   column map and the row bitmap, which validate q_k and p_k; the row table; the row
 *   pointer; the partition, gather and row sort of sp_permute over the whole batch)
 *   into one CSR `out`:
 *   request k owns rows [sp_pbatch_row_offset(k), sp_pbatch_row_offset(k+1)) and its
 *   columns keep their meaning; out has the sum of nrows rows and the largest ncols as
 *   its column count.  out's arrays are caller-allocated (nnz_total entries, the
 *   matrices' colidx / value types, any rowptr type).  Never synchronises and allocates
 *   nothing, so the whole batch can be captured in a CUDA graph and replayed while the
 *   inputs keep their addresses.
 *   Errors: SP_ERR_INVALID_ARG, SP_ERR_OVERFLOW (int32 indices or rowptr too narrow,
 *   more than 2^23 requests, a matrix of 2^40 entries or more); from the device
 *   (sp_ctx_sync) SP_ERR_NOT_PERMUTATION, SP_ERR_INDEX_RANGE (under a column map, a
 *   stored column outside [0, ncols)), SP_ERR_NOT_CANONICAL (row lengths that do not
 *   add up to a matrix's nnz); on a device error the output is not the permutation but
 *   no write leaves its arrays.
 * ------------------------------------------------------------------------------ */
typedef struct sp_permute_req {
  int64_t mat;   /* index of the matrix in mats */
  const void* p; /* device, nrows entries (new row -> old row) or NULL */
  const void* q; /* device, ncols entries (new column -> old column) or NULL */
} sp_permute_req;
typedef struct sp_pbatch sp_pbatch;

SP_API sp_status sp_permute_batch_plan(sp_ctx* ctx, const sp_csr* mats, int64_t nmats,
                                       const sp_permute_req* reqs, int64_t nreq, sp_itype idx_type,
                                       sp_pbatch** plan, int64_t* nnz_total, sp_stream_t stream);
SP_API sp_status sp_permute_batch_fill(sp_ctx* ctx, sp_pbatch* plan, sp_csr* out, sp_stream_t stream);
/* First output row of request k (k = nreq gives the total); -1 for a bad k. */
SP_API int64_t sp_pbatch_row_offset(const sp_pbatch* plan, int64_t k);
/* Release a batch plan (stream-ordered on the stream of its plan call).  NULL is a no-op. */
SP_API sp_status sp_pbatch_destroy(sp_ctx* ctx, sp_pbatch* plan);

/* Release a plan (stream-ordered on the stream of its last call).  NULL is a no-op. */
SP_API sp_status sp_plan_destroy(sp_ctx* ctx, sp_plan* plan);

/* Release the arrays of a library-allocated matrix and zero its pointers. */
SP_API sp_status sp_csr_free(sp_ctx* ctx, sp_csr* M);

/* ------------------------------------------------------------------------------
 * Steps of the path, callable on their own
 * ------------------------------------------------------------------------------ */

/* Inverse index map (the index/value swap of the Identify step, Sec. 3.1 Step 1(a):
 * pvec[pvec_inv[i]] = i; with -1 for absent positions, the sparse form of Sec. 4):
 *   inv[idx[k]] = k for k < len, inv[x] = -1 for every other x in [0, n).
 *   idx: len entries, inv: n entries, both of idx_type.  require_permutation != 0 also
 *   demands len == n (host check) so that idx is a permutation.
 *   Errors: host SP_ERR_SHAPE; device SP_ERR_INDEX_RANGE, SP_ERR_DUPLICATE_INDEX or
 *   SP_ERR_NOT_PERMUTATION. */
SP_API sp_status sp_inverse_map(sp_ctx* ctx, const void* idx, int64_t len, int64_t n,
                         sp_itype idx_type, void* inv, int require_permutation,
                         sp_stream_t stream);

/* Exclusive prefix sum (the proc_pointer / thread_offset prefix sums of Algorithm 2,
 * Fig. 3(ii), which become the output row pointer on one GPU):
 *   out[i] = sum_{k<i} in[k] for i = 0..len (out has len+1 entries; out[len] = total).
 *   in: len entries of in_type (non-negative); out: of out_type.  Single-pass
 *   decoupled look-back scan; in and out must not overlap.
 *   Errors: host SP_ERR_INVALID_ARG; device SP_ERR_OVERFLOW (int32 out overflows),
 *   SP_ERR_TIMEOUT (a look-back wait exceeded SP_OPT_SPIN_LIMIT). */
SP_API sp_status sp_exclusive_scan(sp_ctx* ctx, const void* in, sp_itype in_type, int64_t len,
                            void* out, sp_itype out_type, sp_stream_t stream);

/* Exclusive prefix sum that allocates nothing (the paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory when they need the scan --
 * a device allocator doing its own bookkeeping, which cannot recurse into itself; a
 * service that reserved all device memory up front; a latency-critical loop that must
 * not pay for or synchronise on an allocation.  Such callers cannot create an sp_ctx,
 * whose error record is allocated, so no context is taken).
 *   Same result as sp_exclusive_scan: out[i] = sum_{k<i} in[k], i = 0..len.
 *   The scan's tile-status words, tile ticket and error record live in a fixed device
 *   array inside the library (about 512 KB, held by every GPU that loads the library
 *   until the process exits); no cudaMalloc, cudaFree or allocating routine is called.
 *   len must not exceed SP_SCAN_NOALLOC_MAX_LEN (else SP_ERR_SHAPE, nothing launched).
 *   The first call on a device looks up the array's device address (once per device,
 *   with that device current); make that first call before any stream capture.
 *   Every call reuses the same array: calls that overlap on the GPU (other streams,
 *   other host threads, the same device) race and must be serialised by the caller.
 *   Synchronises `stream` and returns the scan's device status (SP_ERR_OVERFLOW,
 *   SP_ERR_TIMEOUT) or SP_OK. */
#define SP_SCAN_NOALLOC_MAX_LEN (INT64_C(1) << 28)
SP_API sp_status sp_exclusive_scan_noalloc(const void* in, sp_itype in_type, int64_t len,
                                           void* out, sp_itype out_type, sp_stream_t stream);

/* Kept-entry counts of an extraction (the first, counting pass of Algorithm 5):
 *   counts[i] = #{ k in row I[i] of A : colidx[k] is an entry of J }  (int64, nI).
 *   J must be distinct.  Errors as sp_extract. */
SP_API sp_status sp_kept_counts(sp_ctx* ctx, const sp_csr* A, const void* I, int64_t nI,
                         const void* J, int64_t nJ, sp_itype idx_type, int64_t* counts,
                         sp_stream_t stream);

/* Sort every row of M by column, in place, moving values with their columns (the
 * Build step's sort, Sec. 3.1 Step 3).  Column indices must be distinct within each
 * row and in [0, M->ncols).  Errors: SP_ERR_INVALID_ARG, SP_ERR_OVERFLOW (ncols too
 * large for the 32-bit sort keys). */
SP_API sp_status sp_sort_rows(sp_ctx* ctx, sp_csr* M, sp_stream_t stream);

/* Check that A is canonical CSR.  Synchronises; returns SP_ERR_NOT_CANONICAL (detail:
 * offending row) or SP_OK. */
SP_API sp_status sp_csr_validate(sp_ctx* ctx, const sp_csr* A, sp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SP_H_ */
