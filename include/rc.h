/*
 * rc.h -- C ABI of the GB300 concrete-instance SIMT race checker.
 *
 * The question (paper, Abstract and Introduction): can two distinct GPU threads
 * touch the same array cell within one barrier interval, with at least one
 * write?  The paper answers it symbolically: it writes a kernel's Domain,
 * Read, Write and Schedule as ISCC integer sets and maps (Section "Using ISCC
 * in Formal Analysis/Verification") and tests the RaW / WaW / WaR relations
 * (same cell, at least one write) against the schedule (appendix listing of the
 * dependence test).  This library answers it concretely: for a model with a
 * fixed grid and fixed parameters it expands every access instance into a
 * 64-bit key, groups keys by cell (partition passes on a bijective hash of the
 * cell and a counting sort of every bucket; a radix sort where intervals must
 * stay in order; or a hash table), and reports whether any cell races, how
 * many cells race and the smallest racing pair.
 *
 * Race rule (the paper orders instances by a sequential Before relation; for
 * SIMT threads this library reads concurrency as the CUDA barrier rule):
 *   instances x, y race  iff  same (array, scope instance, element)
 *                          and gtid_x != gtid_y
 *                          and their kinds conflict
 *                          and they are concurrent:
 *     block_x != block_y:  grid_phase[phase_x] == grid_phase[phase_y]
 *     same block:          phase_x == phase_y and
 *                          (warp_x != warp_y or warp_phase_x == warp_phase_y),
 * with warp = thread / 32.  Without warp or grid barriers (every warp_phase and
 * grid_phase 0) this is: block_x != block_y or phase_x == phase_y.
 * where kinds are R (read), W (write) and A (atomic read-modify-write) and two
 * kinds conflict iff one is W, or one is A and the other R (two atomics on one
 * cell are ordered by the memory system).
 * A shared array has one instance per block (indexed block-locally), a global
 * array one for the grid.  The phase of an instance is the number of block
 * barriers its thread passed before it; blocks are never ordered against each
 * other except by grid-wide barriers (a grid interval per block interval,
 * rc_model_desc.grid_phase); the warp phase counts the warp barriers
 * (__syncwarp) a thread passed inside its block interval.  Count = number of
 * distinct racy cells.  Witness = the lexicographically smallest racing pair
 * (x, y), x < y, in the order (array, scope instance, element, block, phase,
 * thread, kind R<W<A, warp phase).
 *
 * Conventions for every entry point:
 *  - All calls return an rc_status; none aborts, throws or prints.
 *  - Pointers named *_dev are device pointers, others are host pointers.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Asynchronous calls only enqueue work on the stream; inputs they read on
 *    the device must stay valid until the work completes.
 */
#ifndef RC_H
#define RC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------- */
/* status codes                                                               */
/* ------------------------------------------------------------------------- */
typedef enum rc_status {
  RC_OK = 0,
  RC_E_INVALID = 1,       /* malformed descriptor or argument                          */
  RC_E_KEY_OVERFLOW = 2,  /* the model is too wide even for chunked checks (its cells
                             need more than 2^20 chunks), or a wide model (see
                             rc_layout.wide) was given to a call that takes one key
                             per instance: rc_check_batch, rc_tune, rc_expand_keys,
                             the hash path                                            */
  RC_E_OOB = 3,           /* an index outside its extent, or a phase outside [0, n_phases) */
  RC_E_NOMEM = 4,         /* workspace smaller than rc_workspace_size(), or host/device allocation failed */
  RC_E_TIMEOUT = 5,       /* a bounded device wait expired (the result is not valid)   */
  RC_E_CUDA = 6,          /* a CUDA runtime call failed                                 */
  RC_E_NOT_READY = 7,     /* rc_report(wait=0) on work that has not completed           */
  RC_E_UNSUPPORTED = 8    /* a valid model outside this build's limits (see rc_limits)  */
} rc_status;

/* Static text for a status code. */
const char* rc_status_str(rc_status s);

/* ------------------------------------------------------------------------- */
/* model descriptor                                                           */
/*                                                                            */
/* Follows the paper's statement of what a race model needs (Introduction:    */
/* thread/block ids, barriers and fences, shared-memory arrays, input/output   */
/* arrays; Methods: the same list as components (1)-(7)) and its ISCC          */
/* relations: a statement is a labelled code section (the paper's S, T, I, F)  */
/* with a Domain (loop nest + guards, the Presburger constraints of the Domain */
/* listings) and Read/Write access relations "Stmt[iters] -> Array[index]"     */
/* (the Read and Write listings).                                              */
/* ------------------------------------------------------------------------- */

/* Expression bytecode, evaluated in postfix order on a stack of int64 values
 * with two's-complement wrapping.  Quasi-affine: the paper's Ge-SpMM model
 * uses j % 32 (Section "Doing this for Ge-SpMM", Read listing).
 *   RC_OP_CONST  push imm
 *   RC_OP_TID    push threadIdx[arg]  (arg 0,1,2 = x,y,z)
 *   RC_OP_BID    push blockIdx[arg]
 *   RC_OP_PARAM  push params[arg]
 *   RC_OP_ITER   push the iterator of loop level arg of the statement (0 = outermost)
 *   RC_OP_ADD    pop b, pop a, push a + b
 *   RC_OP_MUL    pop a, push imm * a
 *   RC_OP_FDIV   pop a, push floor(a / imm)   (imm > 0; rounds toward minus infinity)
 *   RC_OP_MOD    pop a, push a mod imm        (imm > 0; Euclidean, result in [0, imm))
 *   RC_OP_LOAD   pop a, push tables[arg].data[a]: a data-dependent value such as
 *                the row bounds rowPtr[i], rowPtr[i + 1] of a sparse matrix (the
 *                paper's rs / re of Ge-SpMM, Section "Problems to deal with",
 *                made concrete; a table with superset = 1 over-approximates
 *                them instead, see rc_table).
 *                A table reads as 0 outside [0, len) (a total function, so a
 *                load needs no out-of-bounds report).
 * A well-formed expression leaves exactly one value. */
enum {
  RC_OP_CONST = 0, RC_OP_TID = 1, RC_OP_BID = 2, RC_OP_PARAM = 3, RC_OP_ITER = 4,
  RC_OP_ADD = 5, RC_OP_MUL = 6, RC_OP_FDIV = 7, RC_OP_MOD = 8, RC_OP_LOAD = 9
};
typedef struct rc_insn { int32_t op; int32_t arg; int64_t imm; } rc_insn;
typedef struct rc_expr { const rc_insn* code; uint32_t len; } rc_expr;

enum { RC_SCOPE_GLOBAL = 0, RC_SCOPE_SHARED = 1 };
enum { RC_READ = 0, RC_WRITE = 1, RC_ATOMIC = 2 };

/* for (v = lower; v < upper; v += step): bounds may use tid, bid, params and
 * the iterators of outer loops; step > 0. */
typedef struct rc_loop { rc_expr lower; rc_expr upper; int64_t step; } rc_loop;

/* One access relation: array[index[0]]...[index[ndims-1]], row-major. */
typedef struct rc_access {
  uint32_t array;          /* index into rc_model_desc.arrays                     */
  uint32_t kind;           /* RC_READ, RC_WRITE or RC_ATOMIC.  A model with atomic
                              accesses has a 2-bit kind field (R = 0, W = 1, A = 2);
                              with more than 16 barrier intervals it is checked
                              on the sort path only (RC_E_UNSUPPORTED on the hash
                              path)                                                */
  const rc_expr* index;    /* ndims expressions (ndims of the array)              */
} rc_access;

/* A statement instance exists for every thread and every point of the loop
 * nest at which all guards are >= 0.  phase may use bid, params and the
 * iterators of loops whose bounds do not depend on tid (a barrier interval is
 * uniform over the block); a phase that names tid is RC_E_INVALID. */
typedef struct rc_stmt {
  rc_expr phase;
  const rc_loop* loops;     uint32_t n_loops;
  const rc_expr* guards;    uint32_t n_guards;
  const rc_access* accesses; uint32_t n_accesses;
  rc_expr warp_phase;       /* warp barriers passed in the block interval, in
                               [0, n_warp_phases); len 0 = 0                     */
} rc_stmt;

typedef struct rc_array {
  const char* name;        /* informational, may be NULL                          */
  uint32_t scope;          /* RC_SCOPE_GLOBAL or RC_SCOPE_SHARED                  */
  uint32_t ndims;          /* 1..4                                                */
  int64_t extent[4];       /* sizes of the dimensions, each >= 1                  */
} rc_array;

/* A read-only integer table for RC_OP_LOAD (copied by rc_model_create).
 *
 * superset = 0: the loads read the values (concrete bounds).
 * superset = 1: the values are unknown, only their range [lo, hi] is stated:
 *   the paper's superset domain for bounds that depend on data (Section
 *   "Problems to deal with"; the free rs, re of the Ge-SpMM Domain).  In every
 *   statement each distinct load of this table (distinct by its expression:
 *   the same expression twice is one parameter) is replaced by a free
 *   parameter that ranges over [lo, hi], and the statement has an instance for
 *   every value of its free parameters.  The checked domain is a superset of
 *   every concrete one whose values lie in [lo, hi]: race-free means race-free
 *   for all such data, a race may be a false positive.  Different statements
 *   get independent parameters.  data may be NULL and len 0 (the values are
 *   not read).  Each free parameter takes one loop level (the statement's
 *   loops plus its free parameters <= max_loops, RC_E_UNSUPPORTED otherwise);
 *   lo > hi, or a bound outside [-2^62, 2^62], is RC_E_INVALID. */
typedef struct rc_table {
  const int64_t* data;     /* host memory, len values                             */
  uint64_t len;
  uint32_t superset;       /* 0 or 1 (above)                                      */
  int64_t lo, hi;          /* the stated value range (superset = 1 only)          */
} rc_table;

typedef struct rc_model_desc {
  uint32_t grid[3];        /* gridDim  (each >= 1)                                */
  uint32_t block[3];       /* blockDim (each >= 1)                                */
  const int64_t* params;   uint32_t n_params;
  uint32_t n_phases;       /* phases are in [0, n_phases); >= 1                   */
  const rc_array* arrays;  uint32_t n_arrays;
  const rc_stmt* stmts;    uint32_t n_stmts;
  const rc_table* tables;  uint32_t n_tables;   /* for RC_OP_LOAD; may be 0     */
  uint32_t n_warp_phases;  /* warp intervals per block interval; 0 or 1 = none   */
  const uint32_t* grid_phase;  /* n_phases entries, non-decreasing: the grid
                               interval of each block interval (grid-wide
                               barriers); NULL = none.  A model with warp or
                               grid barriers is checked on the sort path by
                               default (alone or in a batch, where it shares a
                               pack only with models of at most 16 barrier
                               intervals, and holds a pack alone when it has
                               more than 16 fine intervals n_phases *
                               n_warp_phases) or, with at most 16 fine
                               intervals, on the hash path on request
                               (RC_E_UNSUPPORTED beyond).
                               With more than one grid interval the witness
                               keeps a record per (block, fine interval), so
                               such a model needs bit_length(blocks - 1) +
                               bit_length(n_phases * n_warp_phases - 1) <= 20
                               (RC_E_UNSUPPORTED otherwise) and its workspace
                               grows by 68 bytes per record                    */
} rc_model_desc;

/* Build limits of this library (rc_model_create returns RC_E_UNSUPPORTED
 * beyond them). */
typedef struct rc_limits {
  uint32_t max_loops;        /* loop depth per statement                         */
  uint32_t max_terms;        /* distinct floor-div / mod terms per statement      */
  uint32_t max_stmts;
  uint32_t max_accesses;     /* per statement                                     */
  uint32_t max_phase_bits;
  uint32_t key_bits;         /* packed key width available                        */
} rc_limits;
void rc_get_limits(rc_limits* out);

/* ------------------------------------------------------------------------- */
/* models                                                                     */
/* ------------------------------------------------------------------------- */
typedef struct rc_model rc_model;   /* opaque */

/* Validate and lower a descriptor: compile every expression, compute the key
 * layout and the instance count, and upload the lowered program to the
 * current CUDA device.  For a model with at least 2^22 keys the expansion
 * kernel is generated for the model and compiled with NVRTC (cached per
 * device by source; environment RC_JIT=0 disables it, RC_JIT=1 forces it for
 * every model); if NVRTC is not available the interpreted expansion is used.  The descriptor is deep-copied: the caller may free it
 * on return.  Statements whose loop trip counts depend on the thread are
 * counted on the device (a synchronous count pass on an internal stream).
 * Errors: RC_E_INVALID (malformed), RC_E_KEY_OVERFLOW, RC_E_UNSUPPORTED,
 * RC_E_NOMEM, RC_E_CUDA.  On error *out is NULL. */
rc_status rc_model_create(const rc_model_desc* desc, rc_model** out);
/* Frees the model's host and device memory.  Work using the model must have
 * completed.  NULL is ignored. */
void rc_model_destroy(rc_model* m);

/* Key layout of a lowered model, MSB to LSB: [cell | phase | block | thread |
 * kind], each field `*_bits` wide at `*_shift`; cell = array_base[a] +
 * scope_instance * array_cells[a] + element.  Keys are grouped (sorted) on
 * bits [sort_lo, sort_hi): the cell alone when the model has at most 16
 * barrier intervals (the scan then groups a cell's phases itself), else
 * (cell, phase); the other fields ride along. */
typedef struct rc_layout {
  uint32_t kind_shift, thread_shift, block_shift, phase_shift, cell_shift;
  uint32_t thread_bits, block_bits, phase_bits, cell_bits;
  uint32_t sort_lo, sort_hi;
  uint64_t key_slots;        /* keys written by the expansion (valid + padding)  */
  uint64_t total_cells;
  uint32_t n_arrays;
  uint32_t n_threads_per_block;
  uint64_t n_blocks;
  uint64_t program_bytes;    /* bytes of the lowered program uploaded by rc_model_create */
  uint32_t expand_jit;       /* 1 = the expansion runs a kernel generated for this model   */
  uint32_t wide;             /* 1 = [cell | phase | block | thread | kind] needs more than
                                63 bits: rc_check runs the model in cell-range chunks
                                (RC_OPT_CHUNKED) whose cells are rebased to the chunk
                                start; cell_bits is then the rebased field's width     */
  uint64_t array_base[64];   /* first linear cell of each array (first 64 arrays) */
  uint64_t array_cells[64];  /* cells of one scope instance of each array         */
} rc_layout;
rc_status rc_model_layout(const rc_model* m, rc_layout* out);

/* Source text of the expansion kernel rc_model_create would generate for this
 * descriptor: up to cap-1 bytes and a terminating NUL go to buf (may be NULL
 * when cap is 0); *len receives the full length.  Host lowering only, no
 * device needed.  Errors: those of lowering (RC_E_INVALID, RC_E_KEY_OVERFLOW,
 * RC_E_UNSUPPORTED). */
rc_status rc_kernel_source(const rc_model_desc* desc, char* buf, size_t cap, size_t* len);

/* ------------------------------------------------------------------------- */
/* checking                                                                   */
/* ------------------------------------------------------------------------- */
enum { RC_PATH_AUTO = 0, RC_PATH_SORT = 1, RC_PATH_HASH = 2 };

typedef struct rc_check_opts {
  uint32_t path;           /* RC_PATH_*; AUTO = the tuner's choice                */
  uint32_t digit_bits;     /* radix digit width for the sort path, 0 = auto (<= 8) */
  uint32_t early_exit;     /* hash path: stop at the first racy cell; the count
                              is then a lower bound                               */
  uint32_t test_flags;     /* 0 in normal use; RC_TEST_STALL_LOOKBACK makes every
                              look-back wait for a status nothing publishes, so the
                              bounded wait runs out and the check reports
                              RC_E_TIMEOUT (exercises the timeout path)           */
  uint32_t flags;          /* RC_OPT_* bits                                       */
  uint32_t reserved;
  uint64_t spin_limit;     /* iterations of every bounded device wait, 0 = default */
  uint64_t cell_lo;        /* partial check: only cells in [cell_lo, cell_hi) of   */
  uint64_t cell_hi;        /* the key layout count (0 / 0 = all).  Instances of    */
                           /* other cells are still enumerated, bounds-checked and */
                           /* counted.  The racy cells of disjoint ranges add up;  */
                           /* the witness is the one of the lowest racy range      */
                           /* (a model split across processes or GPUs).  Ignored   */
                           /* by rc_check_batch.                                   */
  uint32_t part_count;     /* partial check by hash part (0 or 1 = none; else a
                              power of two 2^p, p <= 16): only the cells c whose
                              part
                                (((c * 0x9E3779B97F4A7C15) mod 2^cb) * 2^p) >> cb,
                              cb = rc_layout.cell_bits, equals part_index are
                              checked (with cell_lo / cell_hi both apply): the top
                              p bits of the cb-bit hash (if p > cb, only every
                              2^(p-cb)-th part holds cells).  The
                              multiplier is odd, so this is a bijection of the cell
                              field: every cell has exactly one part, and the parts
                              hold about equal shares of the keys whatever the
                              access pattern, so part_count ranks taking parts
                              0 .. part_count - 1 split one model evenly; their
                              racy cells add up and the model's witness is the
                              racy part's witness with the smallest cell.  (It is
                              also the bucket path's hash, whose remaining cb - p
                              bits the part groups by.)  Sort path of rc_check
                              only (RC_E_UNSUPPORTED on the hash path, for chunked
                              checks and wide models; ignored by rc_check_batch);
                              a part count that is not a power of two, or
                              part_index >= part_count, is RC_E_INVALID.          */
  uint32_t part_index;
} rc_check_opts;
enum { RC_TEST_STALL_LOOKBACK = 1,
       RC_TEST_FEW_SCAN_WARPS = 2   /* scan with 3 warps (long ranges per warp) */ };
/* RC_OPT_STAGE_TIMES: record CUDA events between the stages of rc_check on its
 * stream so rc_ticket_stage_times can report per-stage device times (not for
 * chunked checks).
 * RC_OPT_CHUNKED (rc_check; implied for wide models): a count pass expands the
 * model and histograms its keys by cell; rc_check then waits for it (one host
 * synchronisation on `stream`), cuts the checked cell range into chunks whose
 * keys fit the given workspace and whose rebased cells fit the key, and
 * enqueues one expansion (keeping and compacting only the chunk's keys), sort,
 * scan and witness per chunk.  The report merges the chunks: racy cells add
 * up, the witness is the first racy chunk's (chunks are in cell order).  Any
 * workspace that holds the keys of the fullest bucket of cells works
 * (RC_E_NOMEM otherwise); rc_workspace_size gives the size for one chunk of all
 * keys.  The sort path only (RC_PATH_HASH: RC_E_INVALID, wide: RC_E_KEY_OVERFLOW);
 * the expansion runs the interpreted kernels.
 * RC_OPT_GRAPH (rc_check_batch): the device work of a batch is captured once
 * as a CUDA graph per (models, options, workspace) and relaunched as that one
 * graph on later calls with the same arguments; rc_model_destroy drops the
 * captured graphs.  Not a library convenience of the paper: the paper has no
 * batching. */
enum { RC_OPT_STAGE_TIMES = 1, RC_OPT_GRAPH = 2, RC_OPT_CHUNKED = 4, RC_OPT_LSD = 8 };
/* Grouping step of the sort path.  By default a check (or a batch pack) whose
 * keys carry at most 16 barrier intervals groups its keys by cell with the
 * bucket path: two look-back-free partition passes on the top bits of a
 * bijective hash of the cell field, then a counting sort of every bucket in
 * shared memory on the hash's remaining bits, which leaves every cell's keys
 * together (cells in hash order), then the cell scan; its result is identical
 * to the radix-sorted check's.
 * RC_OPT_LSD (or a non-zero digit_bits, or any test flag) selects the stable
 * LSD radix sort followed by the ordered scan instead; models of more than 16
 * intervals, chunked checks and rc_sort_keys always take that path. */

typedef struct rc_inst {
  uint64_t block;          /* linear block index bx + gx*(by + gy*bz)             */
  uint32_t thread;         /* linear thread index in the block tx + bx*(ty + by*tz) */
  uint32_t kind;           /* RC_READ / RC_WRITE / RC_ATOMIC                       */
  int64_t phase;
  uint64_t gtid;           /* block * blockSize + thread                           */
  uint32_t warp_phase;
  uint32_t reserved;
} rc_inst;

typedef struct rc_result {
  int32_t status;          /* rc_status of this check                             */
  int32_t verdict;         /* 1 = some pair races                                 */
  uint64_t racy_cells;     /* distinct racy cells                                 */
  uint64_t instances;      /* access instances checked (guards true, duplicates counted) */
  /* witness (valid when verdict == 1): the racy cell and the smallest pair     */
  uint32_t w_array;
  uint32_t w_reserved;
  uint64_t w_scope;        /* block for a shared array, 0 for a global one        */
  uint64_t w_addr;         /* row-major element index inside the array            */
  rc_inst x, y;
  /* first offending instance when status == RC_E_OOB: the smallest
   * (stmt, access, gtid, dim) with dim 0 = the phase, d+1 = index dimension d */
  uint32_t oob_stmt, oob_access;
  uint64_t oob_gtid;
  int32_t oob_dim;
  int32_t reserved2;
} rc_result;

typedef struct rc_ticket_s* rc_ticket;   /* opaque handle of an enqueued check */

/* Bytes of device workspace rc_check needs for this model and options (for a
 * chunked check: the size that holds all keys in one chunk; smaller ones work,
 * see RC_OPT_CHUNKED).  Errors: RC_E_INVALID, RC_E_KEY_OVERFLOW. */
rc_status rc_workspace_size(const rc_model* m, const rc_check_opts* opts, size_t* bytes);

/* Enqueue one check on `stream`.  `workspace_dev` (>= rc_workspace_size bytes,
 * 256-byte aligned, caller-owned) is scratch for the keys, histograms and
 * look-back state; it may be reused by the next check on the same stream.
 * opts may be NULL (defaults).  *ticket receives a handle for rc_report.
 * A chunked check (RC_OPT_CHUNKED, wide models) blocks until its count pass
 * is done, then enqueues the chunks and returns.
 * Errors: RC_E_INVALID, RC_E_NOMEM (workspace too small), RC_E_KEY_OVERFLOW,
 * RC_E_CUDA. */
rc_status rc_check(rc_model* m, const rc_check_opts* opts, void* workspace_dev,
                   size_t workspace_bytes, void* stream, rc_ticket* ticket);

/* Bytes of workspace rc_check_batch needs for these n models. */
rc_status rc_batch_workspace_size(rc_model* const* models, size_t n,
                                  const rc_check_opts* opts, size_t* bytes);

/* Enqueue a check of n models as one batch; one ticket reports n results in
 * the order of `models`.  Same workspace and error rules as rc_check. */
rc_status rc_check_batch(rc_model* const* models, size_t n, const rc_check_opts* opts,
                         void* workspace_dev, size_t workspace_bytes, void* stream,
                         rc_ticket* ticket);

/* Autotuner (a library facility; the paper has no counterpart).  Times every
 * candidate configuration of checking these models -- the sort path with each
 * distinct number of radix passes (digits of 6..11 bits) and the hash path --
 * on `stream` with the given workspace (3 runs each, the first one a warm-up),
 * keeps the fastest whose check succeeded, and records it for the models'
 * shape class (single model or batch; log2 of the model count, of the key
 * count, and the width of the sorted key fields).  Later checks and workspace
 * queries with path = RC_PATH_AUTO use the recorded choice for that class
 * (else the sort path); a recorded choice that needs more workspace than a
 * check is given falls back to the sort path.  The call blocks until the timed
 * runs finish.  *best receives the chosen options (path and digit_bits set).
 * Candidates that need more workspace than given are skipped; RC_E_NOMEM if
 * none fits.  Batches (n > 1) time rc_check_batch's pipelines. */
rc_status rc_tune(rc_model* const* models, size_t n, const rc_check_opts* opts,
                  void* workspace_dev, size_t workspace_bytes, void* stream,
                  rc_check_opts* best);

/* ------------------------------------------------------------------------- */
/* request server (continuous batching; a library facility, the paper has no   */
/* counterpart)                                                                */
/* ------------------------------------------------------------------------- */

/* A server owns a pool of device memory and `slots` CUDA streams.  Its
 * scheduler thread admits queued requests whenever a slot is idle and the pool
 * has room: the oldest waiting requests, as many as fit the largest free block
 * (at most max_batch, 0 = 1024), are checked together as one rc_check_batch on
 * that slot, so batches of different slots overlap on the device.  Each
 * request's result is the one rc_check gives for its model (the batched
 * pipeline is exact).  Requests are served in arrival order.  A request that
 * cannot fit the pool even when it is empty completes with RC_E_NOMEM. */
typedef struct rc_server rc_server;
typedef struct rc_server_opts {
  uint64_t memory_bytes;   /* device pool for workspaces, allocated at creation */
  uint32_t slots;          /* batches in flight at once (1..64)                  */
  uint32_t max_batch;      /* requests per batch, 0 = 1024                       */
  uint32_t digit_bits;     /* radix digit width of the sort, 0 = auto            */
  uint32_t reserved;
} rc_server_opts;

typedef struct rc_server_done {
  uint64_t request;        /* id from rc_server_submit                           */
  rc_result result;
  double submit_s;         /* host steady-clock seconds: submission,             */
  double start_s;          /*   enqueue of its batch,                            */
  double done_s;           /*   completion seen by the scheduler                 */
  uint32_t batch_size;     /* requests in its batch                              */
  uint32_t pad;
} rc_server_done;

/* Create a server on the current device (allocates the pool, creates the
 * streams, starts the scheduler thread).  RC_E_INVALID for slots outside
 * 1..64 or memory_bytes < 256; RC_E_NOMEM if the pool cannot be allocated. */
rc_status rc_server_create(const rc_server_opts* opts, rc_server** out);

/* Queue a check of `model` (which must stay alive until its result is
 * polled); *request receives its id.  Thread-safe; does not block on the GPU. */
rc_status rc_server_submit(rc_server* server, rc_model* model, uint64_t* request);

/* Move up to `cap` finished requests into `out` (*n_out of them), waiting up to
 * wait_ms milliseconds for one if none is ready.  Returns RC_E_CUDA once a CUDA
 * error has been seen by the scheduler, else RC_OK. */
rc_status rc_server_poll(rc_server* server, rc_server_done* out, size_t cap, size_t* n_out,
                         int wait_ms);

/* Requests waiting for admission and requests in flight. */
rc_status rc_server_stats(rc_server* server, uint64_t* pending, uint64_t* in_flight);

/* Finish every queued and in-flight request, then free the server (results not
 * yet polled are dropped). */
rc_status rc_server_destroy(rc_server* server);

/* Copy out the result(s) of a ticket: `out` holds 1 (rc_check) or n
 * (rc_check_batch) records.  wait=1 blocks until the work completes; wait=0
 * returns RC_E_NOT_READY (ticket still valid) if it has not.  After any other
 * return the ticket is released.  The return value is RC_OK when the results
 * were produced; each record's own status tells how its check went. */
rc_status rc_report(rc_ticket ticket, rc_result* out, int wait);

/* Per-stage device times of a check enqueued with RC_OPT_STAGE_TIMES, in
 * milliseconds between events recorded on the check's stream.  Call after the
 * work completed (e.g. rc_report(wait=0) no longer returns RC_E_NOT_READY is
 * not required: this call waits) and before rc_report releases the ticket.
 * Errors: RC_E_INVALID (no stage times were recorded), RC_E_CUDA. */
typedef struct rc_stage_times {
  float expand_ms;         /* K1 expansion                                         */
  float histogram_ms;      /* digit histograms + digit offsets (bucket path: the
                              pass-A histogram and its offsets)                    */
  float sort_ms[16];       /* K2, one entry per pass (bucket path: partition
                              passes A and B)                                      */
  uint32_t n_sort_passes;
  float scan_ms;           /* K3 scan + fold (bucket path: the bucket fold)        */
  float witness_ms;        /* K4 witness                                           */
  float total_ms;          /* from the first to the last event                     */
  uint64_t n_keys;         /* keys sorted and scanned                              */
  float histogram2_ms;     /* bucket path: the pass-B histogram and its offsets    */
  uint32_t bucketed;       /* 1: bucket path, 0: LSD radix sort and ordered scan   */
  uint32_t histogram_fused;  /* 1: the generated expansion counted the pass-A
                              histogram while writing the keys (histogram_ms then
                              holds only its offsets)                              */
} rc_stage_times;
rc_status rc_ticket_stage_times(rc_ticket ticket, rc_stage_times* out);

/* ------------------------------------------------------------------------- */
/* stage entry points (the hot path one kernel family at a time)              */
/* ------------------------------------------------------------------------- */

/* Expansion only: writes the model's layout.key_slots keys to keys_dev
 * (padding slots hold 0xFFFF...FFFF) and the number of valid instances to
 * *count_dev (uint64).  Only accesses to arrays that some statement writes get
 * a key: a cell that is never written holds no conflicting pair (the race
 * needs a write: Abstract and Introduction), so
 * the instances of read-only arrays are bounds-checked and counted but not
 * emitted.  workspace as for rc_check. */
rc_status rc_expand_keys(rc_model* m, void* workspace_dev, size_t workspace_bytes,
                         uint64_t* keys_dev, uint64_t* count_dev, void* stream);

/* Bytes of workspace rc_sort_keys needs for n keys with digit width digit_bits
 * (0 = 8). */
rc_status rc_sort_workspace_size(uint64_t n, uint32_t digit_bits, size_t* bytes);

/* Stable LSD radix sort (onesweep) of n uint64 keys on bits [lo_bit, hi_bit):
 * reads keys_in_dev, writes keys_out_dev (distinct buffers, n keys each).
 * Keys with equal bits in the range keep their input order.  Asynchronous on
 * `stream`; the returned status covers the enqueue only (RC_E_INVALID,
 * RC_E_NOMEM, RC_E_CUDA).  Errors of the device work itself -- a bounded
 * look-back wait that ran out (RC_E_TIMEOUT: the keys are then in a wrong
 * order) or inconsistent digit counts because the input changed while the sort
 * ran (RC_E_INVALID: nothing was written outside keys_out_dev) -- are read
 * with rc_sort_status(workspace_dev, stream) after the call. */
rc_status rc_sort_keys(const uint64_t* keys_in_dev, uint64_t* keys_out_dev, uint64_t n,
                       uint32_t lo_bit, uint32_t hi_bit, uint32_t digit_bits,
                       void* workspace_dev, size_t workspace_bytes, void* stream);

/* Status of the device work of the last sort that used `workspace_dev`
 * (rc_sort_keys), or, with workspace_dev == NULL, of the last
 * rc_sort_keys_static call on the current device.  Synchronises `stream` (the
 * stream the sort ran on), then reads the sort's error word: RC_OK,
 * RC_E_TIMEOUT (a look-back wait ran out; the output order is wrong) or
 * RC_E_INVALID (the digit counts and the ranks disagreed: the input changed
 * during the sort; stores that would have left the output were skipped), or
 * RC_E_CUDA.  The paper has no counterpart (this is the sort stage's error
 * report, as rc_report is the check's). */
rc_status rc_sort_status(const void* workspace_dev, void* stream);

/* The same sort for callers that cannot allocate device memory when they sort:
 * code whose device memory is entirely reserved up front by another allocator
 * (a framework's caching allocator or a fixed pool), or whose hot path must
 * not pay the latency and synchronisation of cudaMalloc / cudaFree.  The
 * paper has no counterpart; this is a library convenience.
 *
 * The scratch (histograms, look-back words, second key buffer) lives in one
 * static device array of this library sized for RC_SORT_STATIC_MAX_KEYS keys
 * (about 12.8 MB); every GPU that loads the library holds it until the process
 * exits.  The call allocates nothing and calls no allocating routine; the
 * caller still passes the input and output buffers (device, n uint64 keys
 * each, distinct).  n > RC_SORT_STATIC_MAX_KEYS returns RC_E_UNSUPPORTED.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls on a device share the one array, which
 * keeps the last call's contents (the counters that must start at zero are
 * cleared on every call), so calls whose work overlaps on the GPU (different
 * streams, or host threads on one device) race: serialise them.
 * Errors of the enqueue: RC_E_INVALID, RC_E_UNSUPPORTED, RC_E_CUDA; errors of
 * the device work (RC_E_TIMEOUT, RC_E_INVALID, as for rc_sort_keys) are read
 * with rc_sort_status(NULL, stream) after the call. */
#define RC_SORT_STATIC_MAX_KEYS (1u << 20)
rc_status rc_sort_keys_static(const uint64_t* keys_in_dev, uint64_t* keys_out_dev, uint64_t n,
                              uint32_t lo_bit, uint32_t hi_bit, uint32_t digit_bits, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RC_H */
