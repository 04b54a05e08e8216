// Internal data structures of the race checker: the lowered model program that
// the expansion kernels interpret, the device-side result record, the
// workspace plan and the cell-piece algebra of the long-cell scan.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime_api.h>

#include "../../include/rc.h"

#ifdef __CUDACC__
#define RC_HD __host__ __device__ __forceinline__
#else
#define RC_HD inline
#endif

namespace rc {

constexpr int kMaxLoops = 8;      // loop depth per statement
constexpr int kMaxTerms = 16;     // distinct floor-div / mod terms per statement
constexpr int kMaxStmts = 4096;
constexpr int kMaxAccesses = 64;  // per statement
constexpr int kMaxDims = 4;
constexpr int kMaxPhaseBits = 16;
constexpr int kKeyBits = 63;      // bit 63 is reserved so 0xFFFF...FFFF is never a valid key
constexpr uint64_t kSentinel = ~0ull;
// Models with at most this many phase bits are sorted by cell only: the scan
// groups a cell's keys by phase with small per-part tables instead of relying
// on the sort order (scan.cu).
constexpr uint32_t kScanTablePhaseBits = 4;
constexpr int kFastCache = 16;    // per-thread cached thread-constant rows per statement
constexpr int kFastLoops = 4;     // loop depth of the compile-time loop nests of the expansion

// ---------------------------------------------------------------------------
// lowered program
//
// Every expression of a statement (loop bounds, guards, phase, indices and the
// operands of its floor-div / mod terms) becomes a *row*:
//     value = c0 + ct . (tid.x, tid.y, tid.z, bid.x, bid.y, bid.z)
//                + sum_k coef_k * var_k
// where var_k is an iterator (var < kMaxLoops) or a term (var - kMaxLoops);
// parameters are folded into the constants.  A term is
//     term_q = op_q(value(row_q), d_q),   op = floor division or Euclidean mod,
// evaluated once its iterators are bound (level_q = number of loop levels it
// needs).
// ---------------------------------------------------------------------------
struct LinTerm {
  int32_t var;
  int32_t pad;
  int64_t coef;
};

struct Row {
  int64_t c0;
  int64_t ct[6];
  int32_t off;   // first LinTerm of this row in the model's pool
  int32_t nnz;
  int32_t level; // loop levels whose iterators it needs (0 = constant per thread)
  int32_t cache; // slot of its per-thread cached value when level == 0 and used per point, else -1
};

enum TermOp : int32_t { kFdiv = 0, kMod = 1, kLoad = 2 };   // kLoad: d = table number

struct Term {
  int32_t row;
  int32_t op;
  int64_t d;
  int32_t level;   // iterators 0..level-1 must be bound
  int32_t pad;
  uint64_t magic;  // ceil(2^64 / d) for the multiply-high division (d >= 2), 0 for d == 1
};

struct DevAccess {
  int32_t array;
  int32_t kind;
  int32_t ndims;
  int32_t row0;    // first of ndims consecutive index rows
  int32_t key_idx; // slot of its key among the statement's keyed accesses, -1 when the
                   // array is never written (its cells cannot race: no key is made)
  int32_t pad;
};

struct DevArray {
  int64_t ext[kMaxDims];
  int32_t ndims;
  int32_t shared;
  uint64_t base;   // first linear cell
  uint64_t cells;  // cells of one scope instance
};

struct DevStmt {
  int32_t n_loops, n_guards, n_acc, n_terms;
  int32_t n_key;        // accesses that make keys (arrays some statement writes)
  int32_t pad_k;
  int32_t row_lower[kMaxLoops];
  int32_t row_upper[kMaxLoops];
  int64_t step[kMaxLoops];
  int32_t row_phase;
  int32_t row_wphase;   // warp interval row, -1 = 0
  int32_t pad_w;
  int32_t guard_row0;   // guards are rows [guard_row0, guard_row0 + n_guards)
  int32_t acc0;         // first DevAccess
  int32_t term0;        // first Term
  int32_t dense;        // 1 = every loop has a constant trip count
  int32_t n_cache;      // per-thread cached rows (level 0, used at every point)
  int64_t trips[kMaxLoops];
  uint64_t n_iter;      // product of trips (dense)
  uint64_t slot_base;   // dense: first key slot; general: index of its first unit offset
};

struct DevModel {
  uint32_t grid[3], block[3];
  uint32_t bs;            // threads per block
  uint32_t n_stmts;
  uint64_t n_blocks;
  uint64_t n_threads;     // n_blocks * bs
  int64_t n_phases;
  int64_t n_wphases;      // warp intervals per block interval (1 = no warp barriers)
  // key layout; the phase field holds phase * n_wphases + warp phase
  uint32_t kind_shift, thread_shift, block_shift, phase_shift, cell_shift;
  uint32_t thread_bits, block_bits, phase_bits, cell_bits;
  uint32_t sort_lo, sort_hi;
  uint64_t dense_slots;   // keys [0, dense_slots) are written by dense statements
  uint64_t general_slots; // keys [dense_slots, dense_slots + general_slots) by general ones
  // pointers into the uploaded program (device addresses)
  const DevStmt* stmts;
  const DevAccess* accs;
  const DevArray* arrays;
  const Row* rows;
  const LinTerm* lin;
  const Term* terms;
  const uint64_t* unit_offset;  // general statements: offset of each (stmt, gtid) unit
  const uint64_t* tables;       // per table: offset into tdata, length (2 words each)
  const int64_t* tdata;         // table values
  uint32_t n_tables, pad_t;
  // warp / grid barriers: block interval and grid interval of each fine
  // interval (4 bits per interval), warp intervals | their bit width << 32
  uint64_t sync_tab[3];
  // multiply-high reciprocals (fastdiv_magic) of bs, block.x, block.y,
  // block.x * block.y, grid.x, grid.y, grid.x * grid.y for thread_vars
  uint64_t div_magic[7];
};

// Value of a table load: tables read as 0 outside [0, len), so a load is a
// total function of its index and needs no out-of-bounds report.
RC_HD int64_t table_load(const DevModel& M, int64_t table, int64_t idx) {
  const uint64_t off = M.tables[2 * table], len = M.tables[2 * table + 1];
  return (idx < 0 || (uint64_t)idx >= len) ? 0 : M.tdata[off + (uint64_t)idx];
}

// ---------------------------------------------------------------------------
// device result record (head of the workspace)
// ---------------------------------------------------------------------------
struct DevResult {
  unsigned long long oob_code;     // min packed (stmt, access, gtid, dimcode); ~0 = none
  unsigned long long instances;    // guard-true access instances
  unsigned long long racy_cells;
  unsigned long long min_start;    // first key position of the first racy cell; ~0 = none
  unsigned long long seg_end;      // one past its last key
  unsigned long long cell;         // its cell value
  unsigned long long x_rank;       // witness x as (p, t, k) packed; ~0 = none
  unsigned long long y_rank;       // witness y as (b, p, t, k) packed; ~0 = none
  unsigned int minb, maxb, minWb, maxWb, anyW, err;
  // witness summary of atomic and plain-read instances (blocks holding each)
  unsigned int minAb, maxAb, anyA, minRb, maxRb, anyR;
  unsigned long long n_keys;       // keys in the sorted buffer
  unsigned long long sorted_buf;   // index (0/1) of the buffer that holds the sorted keys
  unsigned long long hash_cell;    // hash path: smallest racy cell found; ~0 = none
  unsigned int stop;               // hash path: early-exit flag
  unsigned int pad0;
  unsigned long long pad[2];
};
static_assert(sizeof(DevResult) <= 256, "result record must fit its slot");

// words of one witness phase-group record (scan.cu): [mint, maxt], per access
// kind (R, W, A) [min thread, max thread, any] in one block, and per kind
// [min block, max block] over all blocks
constexpr unsigned kWitnessGroupWords = 17;
// Models with more than one grid interval keep one record per (block, fine
// interval) -- the smallest racing instance may lie above the cell's lowest
// block -- so their block and phase bits are bounded: 2^20 records of 68 bytes.
constexpr uint32_t kWitnessBlockGroupBits = 20;

enum DevError : unsigned int {
  kErrLookbackTimeout = 1u,
  kErrHashTimeout = 2u,
  kErrHashFull = 4u,
  kErrScanLongFull = 8u,
  kErrChunkOverflow = 16u,   // a chunk produced more keys than its count pass planned
  kErrSortRange = 32u,       // a sort pass computed a destination outside the output (its digit
                             // counts and its ranks disagree: the input changed while it ran)
  kErrCopyTimeout = 64u,     // a bulk copy into shared memory did not complete within its wait bound
};

// packed out-of-bounds code: stmt (12 bits) | access (6) | gtid (42) | dimcode (3)
RC_HD unsigned long long oob_pack(uint32_t stmt, uint32_t acc, uint64_t gtid, uint32_t dimcode) {
  return ((unsigned long long)stmt << 51) | ((unsigned long long)acc << 45) |
         ((unsigned long long)(gtid & ((1ull << 42) - 1)) << 3) | (unsigned long long)dimcode;
}

// ---------------------------------------------------------------------------
// floor division / Euclidean modulo by a positive constant (int64)
// ---------------------------------------------------------------------------
RC_HD int64_t floor_div(int64_t a, int64_t d) {
  int64_t q = a / d;
  return ((a % d) != 0 && a < 0) ? q - 1 : q;
}
RC_HD int64_t euclid_mod(int64_t a, int64_t d) {
  int64_t r = a % d;
  return r < 0 ? r + d : r;
}
// Floor division / Euclidean modulo by a positive invariant divisor using the
// multiply-high method of Lemire, Kaser and Kurz ("Faster remainder by direct
// computation", Software: Practice and Experience, 2019): for 0 <= x < 2^32
// and 2 <= d < 2^32, floor(x / d) = floor(M * x / 2^64) with M = ceil(2^64 / d).
// Negative numerators use floor(a / d) = -1 - floor((-a - 1) / d).  Values
// outside [-2^32, 2^32) or divisors >= 2^32 take the plain 64-bit division.
constexpr int64_t kFastDivLimit = (int64_t)1 << 32;
inline uint64_t fastdiv_magic(int64_t d) { return d >= 2 && d < kFastDivLimit ? ~0ull / (uint64_t)d + 1 : 0; }

#ifdef __CUDACC__
__device__ __forceinline__ int64_t fast_floor_div(int64_t a, int64_t d, uint64_t magic) {
  if (d == 1) return a;
  if (magic != 0 && a >= -kFastDivLimit && a < kFastDivLimit) {
    if (a >= 0) return (int64_t)__umul64hi(magic, (uint64_t)a);
    return -1 - (int64_t)__umul64hi(magic, (uint64_t)(-a - 1));
  }
  return floor_div(a, d);
}
__device__ __forceinline__ int64_t fast_euclid_mod(int64_t a, int64_t d, uint64_t magic) {
  return a - fast_floor_div(a, d, magic) * d;
}
#endif

RC_HD int64_t wadd(int64_t a, int64_t b) { return (int64_t)((uint64_t)a + (uint64_t)b); }
RC_HD int64_t wmul(int64_t a, int64_t b) { return (int64_t)((uint64_t)a * (uint64_t)b); }

// ---------------------------------------------------------------------------
// cell pieces of the long-cell scan
//
// Sorted keys are grouped by cell and, inside a cell, by (cell, phase) "sub"
// groups.  A cell is racy iff
//     (min block != max block)  ? (some write in the cell)
//                               : (some sub group has min thread != max thread
//                                  and a write),
// the cell-level form of the pair rule (a multi-block cell races iff it has a
// write; a single-block cell races iff two threads meet in one barrier
// interval with a write).  A CellPiece describes a contiguous run of keys of
// one cell; piece_combine() concatenates two runs of the same cell.
// ---------------------------------------------------------------------------
struct SubAgg {
  uint32_t mint, maxt, anyW, pad;
};

RC_HD SubAgg sub_merge(SubAgg a, SubAgg b) {
  SubAgg r;
  r.mint = a.mint < b.mint ? a.mint : b.mint;
  r.maxt = a.maxt > b.maxt ? a.maxt : b.maxt;
  r.anyW = a.anyW | b.anyW;
  r.pad = 0;
  return r;
}
RC_HD bool sub_racy(SubAgg s) { return s.mint != s.maxt && s.anyW; }
RC_HD SubAgg sub_none() { SubAgg s; s.mint = 0; s.maxt = 0; s.anyW = 0; s.pad = 0; return s; }

// A run of keys that all lie in one cell.
struct CellPiece {
  uint64_t cell;
  uint64_t start;          // position of the run's first key
  uint32_t minb, maxb;
  uint32_t anyW;
  uint32_t first_p, last_p;
  uint32_t single_sub;     // the run holds one sub group (fs and ls are the same)
  uint32_t inner;          // OR of sub_racy over sub groups strictly between fs and ls
  uint32_t pad;
  SubAgg fs, ls;           // first and last sub group of the run
};

RC_HD bool piece_racy(const CellPiece& c) {
  if (c.minb != c.maxb) return c.anyW != 0;
  return c.inner || sub_racy(c.fs) || sub_racy(c.ls);
}

// X then Y, both pieces of the same cell.
RC_HD CellPiece piece_combine(const CellPiece& X, const CellPiece& Y) {
  CellPiece r;
  r.cell = X.cell;
  r.start = X.start;
  r.minb = X.minb < Y.minb ? X.minb : Y.minb;
  r.maxb = X.maxb > Y.maxb ? X.maxb : Y.maxb;
  r.anyW = X.anyW | Y.anyW;
  r.first_p = X.first_p;
  r.last_p = Y.last_p;
  r.pad = 0;
  if (X.last_p == Y.first_p) {
    SubAgg m = sub_merge(X.ls, Y.fs);
    if (X.single_sub && Y.single_sub) {
      r.single_sub = 1; r.fs = m; r.ls = m; r.inner = 0;
    } else if (X.single_sub) {
      r.single_sub = 0; r.fs = m; r.ls = Y.ls; r.inner = Y.inner;
    } else if (Y.single_sub) {
      r.single_sub = 0; r.fs = X.fs; r.ls = m; r.inner = X.inner;
    } else {
      r.single_sub = 0; r.fs = X.fs; r.ls = Y.ls;
      r.inner = X.inner | Y.inner | (sub_racy(m) ? 1u : 0u);
    }
  } else {
    r.single_sub = 0;
    r.fs = X.fs;
    r.ls = Y.ls;
    r.inner = X.inner | Y.inner | ((!X.single_sub && sub_racy(X.ls)) ? 1u : 0u) |
              ((!Y.single_sub && sub_racy(Y.fs)) ? 1u : 0u);
  }
  return r;
}

// ---------------------------------------------------------------------------
// host-side model and workspace plan
// ---------------------------------------------------------------------------
struct SortPlan {
  uint32_t n_pass;
  uint32_t shift[16];
  uint32_t bits[16];
};
// widest digit of a plan (for sizing the look-back words of its passes)
inline uint32_t plan_max_bits(const SortPlan& sp) {
  uint32_t b = 8;
  for (uint32_t p = 0; p < sp.n_pass; ++p) b = sp.bits[p] > b ? sp.bits[p] : b;
  return b;
}

// The bucket path of the grouping step (bucket.cu): see kernels.h.
constexpr uint32_t kSortThreadsHost = 256;
constexpr uint64_t kCellHashMul = 0x9E3779B97F4A7C15ull;

constexpr uint32_t kBucketMaxDigitBits = 10;        // per partition pass
constexpr uint32_t kBucketMaxBits = 2 * kBucketMaxDigitBits;
constexpr int kFoldCap = 7680;                      // keys of a bucket folded in shared memory
constexpr uint32_t kFoldBinBits = 12;               // counting-sort bins of a bucket (at most)
constexpr uint64_t kBucketTarget = kFoldCap / 2 + kFoldCap / 16;   // planned mean keys per bucket
constexpr int kBucketHistTile = 16384;              // keys per block of the pass-B histogram
constexpr int kPartTileHost = kSortThreadsHost * 16;    // keys per tile of the partition passes

struct BucketPlan {
  bool on = false;
  uint32_t cb = 0, dA = 0, dB = 0, D = 0, r = 0, rbin = 0;
  uint64_t n = 0;                 // key slots (padding included)
  uint64_t tiles_b = 0, tiles_h = 0;   // grid bounds of pass B and its histogram
  // workspace offsets (bytes) of the bucket section
  size_t hist_a = 0, off_a = 0, cur_a = 0, tpref_b = 0, tpref_h = 0, tile_a = 0;
  size_t hist_b = 0, boff = 0, cur_b = 0, temp = 0;
  size_t scan_ctr = 0;            // the ordered scan's long-cell counter (in the cleared range)
  size_t zero_lo = 0, zero_hi = 0;    // cleared at the start of a check (the two histograms)
  size_t end = 0;
};
// host (runtime.cu): whether the bucket path applies to n keys of cb cell bits
// (at most 2^kBucketMaxBits buckets of about kBucketTarget keys), its digit
// widths, and its workspace section laid out from byte offset `off`
bool plan_buckets(uint64_t n, uint64_t n_expect, uint32_t cb, size_t off, BucketPlan* bp);


struct WorkspacePlan {
  size_t result_off;      // DevResult
  size_t keys_off[2];     // ping-pong key buffers
  size_t hist_off;        // n_pass x 256 uint64 digit counts
  size_t digoff_off;      // n_pass x 256 uint64 digit offsets
  size_t cursor_off;      // partition pass: next output position per digit
  size_t lookback_off;    // n_tiles x 256 uint64 status words (one pass at a time)
  size_t tilectr_off;     // n_pass uint32 tile counters
  size_t long_off;        // scan: cells handed to the long-cell pass
  size_t scanctr_off;     // scan: count of those cells (in the cleared range)
  uint64_t long_cap;
  size_t group_off;       // witness per-phase group summaries
  size_t zero_lo, zero_hi;  // byte range cleared at the start of a check
  size_t total;
  uint64_t n_keys;
  uint64_t n_tiles;
  uint32_t scan_warps;
  SortPlan sort;
  BucketPlan bucket;      // bucket path (bucket.on) instead of the LSD sections
  // hash path
  bool hash;
  uint64_t hash_cap;      // slots per table (power of two)
  size_t gkey_off, gword_off, ckey_off, cword_off, filt_off, nfilt_off;
};

struct Model {
  DevModel host;                  // copy of the device header (device pointers inside)
  std::vector<uint8_t> program;   // host image of the uploaded program
  void* dev_program = nullptr;    // device allocation (program + unit offsets)
  size_t dev_bytes = 0;
  uint64_t key_slots = 0;
  uint64_t total_cells = 0;
  std::vector<uint64_t> array_base, array_cells;
  std::vector<uint32_t> array_shared;
  uint32_t n_general_stmts = 0;
  bool has_deep_loops = false;    // some statement has more than kFastLoops loops
  bool loop_free = true;          // no statement has a loop
  // the packed key [cell | phase | block | thread | kind] needs more than
  // kKeyBits: checks run in cell-range chunks whose rebased cell field has
  // host.cell_bits bits (the width left beside the other fields)
  bool wide = false;
  bool has_atomic = false;        // some access is atomic: 2-bit kind field
  bool sync_scopes = false;       // warp or grid barriers
  bool multi_grid = false;        // more than one grid interval (grid barriers)
  uint64_t coarse_tab = 0;        // fine interval q -> block interval (4 bits per q, q < 16)
  uint64_t grid_tab = 0;          // fine interval q -> grid interval (4 bits per q, q < 16)
  // sections of the program image (byte offsets), for the kernel generator
  size_t sec_arrays = 0, sec_stmts = 0, sec_accs = 0, sec_rows = 0, sec_lin = 0, sec_terms = 0, sec_tabidx = 0;
  // grid interval (dense numbering) of every block interval, uint32 each: the
  // phase-sorted scan of models with warp or grid barriers and more than 16
  // fine intervals (0 = no such section)
  size_t sec_gridof = 0;
  void* jit_fn = nullptr;         // generated expansion kernel (CUfunction), or null
  void* jit_chunk_fn = nullptr;   // wide models: generated count / route kernel, or null
  uint64_t max_iter_per_unit = 0;
};

// implemented in jit.cpp
constexpr uint64_t kJitMinKeys = 1ull << 22;   // models with fewer keys keep the interpreted expansion
// Arguments of the generated count / route kernel of chunked checks (the
// generated source declares the same struct).
struct ChunkJitArgs {
  unsigned long long* oob;
  unsigned long long* inst;
  const int64_t* tdata;
  int32_t mode;                       // 0 = count keys per bucket, 1 = route keys to chunk segments
  int32_t pad;
  unsigned long long* counts;
  uint64_t lo, span;
  uint32_t bshift, cell_shift;
  uint64_t* keys;
  const uint32_t* chunk_of;
  const uint64_t* c_lo;
  const uint64_t* c_base;
  const uint64_t* c_end;
  unsigned long long* c_ctr;
  uint64_t b0, n_buckets, low_mask;
  unsigned int* err;
};
std::string jit_expand_source(const Model& m);
std::string jit_chunk_source(const Model& m);
bool jit_expand_build(Model* m);
cudaError_t jit_chunk_launch(const Model& m, const ChunkJitArgs& a, cudaStream_t st);
// The bucket path's pass-A histogram counted by the generated expansion as it
// writes the keys: digit = ((cell * kCellHashMul) & cmask) >> shift, bins
// counters (at most kBucketMaxHistBins) added to hist.
struct ExpandHist {
  unsigned long long* hist;
  uint64_t cmask;
  uint32_t shift, bins;
};
constexpr int kBucketMaxHistBins = 1 << kBucketMaxDigitBits;
constexpr unsigned kExpandHistUnits = 8;   // 128-thread units per block of a histogram-counting expansion
// cells kept by a partial check: [lo, hi) and the hash part
// ((c * kCellHashMul) & pmask) == pval (pmask = pval = 0: every part)
struct CellFilter {
  uint64_t lo = 0, hi = ~0ull;
  uint64_t pmask = 0, pval = 0;
};
cudaError_t jit_expand_launch(const Model& m, uint64_t* keys, DevResult* res, cudaStream_t st,
                              const CellFilter& cf = CellFilter(), const ExpandHist* eh = nullptr);

// implemented in lower.cpp
rc_status lower_model(const rc_model_desc* d, Model* m, std::vector<int32_t>* general_stmt_ids);
void plan_workspace(const Model& m, const rc_check_opts* opts, WorkspacePlan* p);
// the sort-path plan for n keys whose cell field has cell_bits bits; the
// look-back region holds digits of at least min_lookback_bits bits (so that a
// narrower sort of fewer bits, whose widest digit may be wider, fits it)
void plan_workspace_keys(const Model& m, const rc_check_opts* opts, uint64_t n, uint32_t cell_bits, WorkspacePlan* p,
                         uint32_t min_lookback_bits = 0, bool allow_bucket = true);
// whether options and a key layout of phase_bits phase bits admit the bucket path
bool bucket_path_allowed(uint32_t phase_bits, const rc_check_opts* opts);
void plan_sort(uint32_t lo, uint32_t hi, uint32_t digit_bits, SortPlan* sp);
uint32_t bit_length(uint64_t v);

}  // namespace rc
