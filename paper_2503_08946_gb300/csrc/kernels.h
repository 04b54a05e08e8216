// Host launchers of the race-check kernels (one translation unit per family).
#pragma once

#include <cuda_runtime.h>

#include "rc_internal.h"

namespace rc {

// runtime.cu: sets a kernel's dynamic shared-memory limit to `smem_bytes` (and,
// with max_carveout, its preferred carveout to the largest shared-memory share)
// once per (device, kernel), with the current device; thread-safe; returns the
// first failing CUDA call's error (and retries on the next launch).
cudaError_t ensure_kernel_smem(const void* func, size_t smem_bytes, bool max_carveout = true);

// expand.cu
// has_deep: some statement has more than kFastLoops loops (runs the generic kernel too)
// keys of cells the filter does not keep (a partial check) are written as padding
cudaError_t launch_expand(const DevModel* dm, uint32_t n_stmts, uint64_t n_threads, bool has_deep, uint64_t* keys,
                          DevResult* res, cudaStream_t st, const CellFilter& cf = CellFilter());
// Count pass of a chunked check: counts[(cell - lo) >> bshift] += keys of the
// cells in [lo, lo + span) (instances and out-of-bounds reports go to res).
cudaError_t launch_expand_count(const DevModel* dm, uint32_t n_stmts, uint64_t n_threads, bool has_deep,
                                DevResult* res, unsigned long long* counts, uint64_t lo, uint64_t span,
                                uint32_t bshift, cudaStream_t st);
// Key pass of a chunked check for one wave of chunks: the keys of cells in the
// wave's chunks, cell field rebased to the chunk start, appended to their
// chunk's segment of `keys`.
struct RouteArgs {
  uint64_t* keys;
  const uint32_t* chunk_of;    // chunk (in the wave) of bucket b0 + i; ~0 = not in the wave
  const uint64_t* c_lo;        // per chunk: first cell
  const uint64_t* c_base;      // per chunk: first key position of its segment
  const uint64_t* c_end;       // per chunk: one past its segment
  unsigned long long* c_ctr;   // per chunk: keys appended (cleared before the pass)
  uint64_t lo, span;           // checked cell range [lo, lo + span)
  uint64_t b0, n_buckets;      // the wave's buckets [b0, b0 + n_buckets)
  uint64_t low_mask;           // key bits below the cell field
  uint32_t bshift, cell_shift;
};
cudaError_t launch_expand_route(const DevModel* dm, uint32_t n_stmts, uint64_t n_threads, bool has_deep,
                                const RouteArgs& r, DevResult* res, cudaStream_t st);
cudaError_t launch_count(const DevModel* dm, uint64_t n_units, uint64_t* counts, cudaStream_t st);
size_t scan_u64_temp_bytes(uint64_t n);
cudaError_t scan_u64_exclusive(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t add, uint64_t* temp,
                               uint64_t* total_dev, cudaStream_t st);

// batch.cu
constexpr int kExpandThreadsHost = 128;   // == kExpandThreads of expand_core.cuh
struct BatchModel {              // one model of a batch (device table entry)
  const DevModel* dm;
  uint64_t key_base;             // first slot of the model's keys in the batch key buffer
  uint64_t cell_base;            // first batch cell of the model
  uint64_t unit_base;            // first expansion unit of the model
  uint64_t n_threads;
  uint32_t n_stmts, n_chunks;    // statements, thread chunks (expansion units)
  uint32_t cell_shift, phase_shift, block_shift;   // the model's key layout
  uint32_t phase_bits, block_bits, thread_bits;
  uint32_t thread_shift;         // = the model's kind field bits
};
struct BatchArgs {
  const BatchModel* models;
  uint32_t n_models;
  uint64_t n_units;
  unsigned long long* queue;     // starts at 0
  uint64_t* keys;                // batch key buffer
  DevResult* res;                // one per model
  uint32_t cell_shift, phase_shift, block_shift;   // batch key layout
  uint32_t thread_shift;                           // = the batch's kind field bits
};
// loop_free: every statement of the pack's models has no loops
cudaError_t launch_batch_expand(const BatchArgs& a, bool loop_free, cudaStream_t st);
cudaError_t launch_batch_errors(const DevResult* pack, DevResult* res, uint32_t n, cudaStream_t st);

// hash.cu
struct HashArgs {
  unsigned long long* gkey;    // group table keys (cell, phase), kEmpty = free
  unsigned long long* gword;
  unsigned long long* ckey;    // cell table keys
  unsigned long long* cword;
  uint64_t gmask, cmask;       // table sizes - 1 (powers of two)
  DevResult* res;
  unsigned int early_exit;
  unsigned int* stop;
  uint64_t* filtered;          // keys of the smallest racy cell
  unsigned long long* n_filtered;
  uint64_t cell_lo, cell_hi;   // only cells in [cell_lo, cell_hi) are inserted
  uint32_t sync;               // warp or grid barriers: three groups per instance (see hash.cu)
};
cudaError_t launch_hash(const DevModel* dm, uint32_t n_stmts, uint64_t n_threads, const HashArgs& h,
                        cudaStream_t st);

// sort.cu
constexpr int kSortThreads = 256;
static_assert(kSortThreads == (int)kSortThreadsHost, "one block size for the sort kernels");
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;   // keys per onesweep tile
constexpr int kMaxRadixBits = 11;
constexpr int kMaxRadix = 1 << kMaxRadixBits;           // bins of the widest digit

struct SortArgs {
  const uint64_t* keys_in;
  uint64_t* keys_out;
  uint64_t n;
  uint32_t shift, bits;
  const unsigned long long* digit_offset;   // exclusive offsets of this pass's digits
  unsigned long long* lookback;             // n_tiles x 2^radix_bits status words
  unsigned int* tile_counter;
  unsigned int epoch;                       // distinct per pass within one check
  unsigned int wait_epoch;                  // epoch the look-back accepts (== epoch in normal use)
  unsigned long long spin_limit;
  unsigned int* err;
  unsigned long long* cursor;               // partition pass: next output position per digit
};
// digit counts of every pass (any number of passes, any key alignment)
cudaError_t launch_histogram(const uint64_t* keys, uint64_t n, const SortPlan& sp, unsigned long long* hist,
                             cudaStream_t st);
// histogram.cu: the same counts by a kernel compiled per pass count (plans of
// up to 6 passes over 16-byte aligned keys; others take launch_histogram)
cudaError_t launch_digit_counts(const uint64_t* keys, uint64_t n, const SortPlan& sp, unsigned long long* hist,
                                cudaStream_t st);
cudaError_t launch_digit_offsets(const unsigned long long* hist, unsigned long long* digoff, const SortPlan& sp,
                                 cudaStream_t st);
// radix_bits: counters of the onesweep kernel (radix_bits_for(pass bits))
cudaError_t launch_onesweep(const SortArgs& a, uint32_t radix_bits, cudaStream_t st);
// unstable pass (any order among equal digits); a.cursor starts at the digit offsets
cudaError_t launch_partition(const SortArgs& a, uint32_t radix_bits, cudaStream_t st);
uint32_t radix_bits_for(uint32_t bits);
// runtime.cu: byte ranges (offset, length) of a sort's scratch that must start
// at zero -- the digit counts of its passes, the look-back words of its tiles
// at its widest radix, its tile counters
void sort_clear_ranges(const SortPlan& sp, uint64_t n, size_t hist_off, size_t lookback_off, size_t tilectr_off,
                       size_t (*ranges)[2]);
// Test hook of the sort entry points: with RC_TEST_SORT_STALL=1 in the
// environment every look-back waits for a status epoch that no pass publishes,
// so its bounded wait runs out (after a short spin limit) and the error word is
// set; every access stays in bounds.
bool sort_stall_requested();
// sort_static.cu: device address of the static scratch's result record on the
// current device (looked up once per device)
rc_status sort_static_record(const void** rec);

// bucket.cu: the bucket path of the grouping step.  The cell field of a key is
// mapped by the bijection h(cell) = cell * kCellHashMul mod 2^cb (cb = cell
// bits); the keys are partitioned by the top dA bits of h (pass A, padding keys
// dropped), then each A-bucket by the next dB bits (pass B), without look-back;
// every resulting bucket (top D = dA + dB bits of h) holds all keys of its cells
// and is grouped by cell and folded in shared memory (bucket_fold_kernel).
struct BucketArgs {
  const uint64_t* keys_in;
  uint64_t* keys_out;
  uint64_t n;                       // keys of keys_in (pass A: padding included)
  uint32_t cell_shift, cb;
  uint64_t cmask;                   // 2^cb - 1
  uint32_t dA, dB;
  unsigned long long* hist_a;       // [2^dA] valid keys per A-bucket
  unsigned long long* off_a;        // [2^dA + 1] A-bucket offsets (exclusive, then the total)
  unsigned long long* cur_a;        // [2^dA] pass-A output cursors
  unsigned long long* tpref_b;      // [2^dA + 1] pass-B tiles before each A-bucket
  unsigned* tile_a;                 // [pass-B tiles] the A-bucket of each pass-B tile (written by the histogram)
  unsigned long long* tpref_h;      // [2^dA + 1] histogram tiles before each A-bucket
  unsigned long long* hist_b;       // [2^D] keys per bucket
  unsigned long long* boff;         // [2^D + 1] bucket offsets
  unsigned long long* cur_b;        // [2^D] pass-B output cursors
  unsigned long long* temp;         // scan scratch
  unsigned int* err;
};
cudaError_t launch_bucket_hist_a(const BucketArgs& a, cudaStream_t st);
cudaError_t launch_bucket_scan_a(const BucketArgs& a, cudaStream_t st);
cudaError_t launch_bucket_pass_a(const BucketArgs& a, cudaStream_t st);
cudaError_t launch_bucket_hist_b(const BucketArgs& a, uint64_t tiles_h, cudaStream_t st);
cudaError_t launch_bucket_scan_b(const BucketArgs& a, cudaStream_t st);
cudaError_t launch_bucket_pass_b(const BucketArgs& a, uint64_t tiles_b, cudaStream_t st);
// D == 0: the single bucket [0, n) of the unpartitioned keys (padding included)
cudaError_t launch_bucket_whole(unsigned long long* boff, uint64_t n, cudaStream_t st);

// scan.cu
constexpr int kScanRun = 32;          // keys per lane run (multiple of 2)
// at most four waves of 152 SMs x 6 resident blocks of 4 warps (measured a
// little faster than two: the per-warp ranges are shorter at the tail)
constexpr uint32_t kScanMaxWarps = 152 * 24 * 4;
struct ScanArgs {
  const uint64_t* keys;                // 16-byte aligned (the phase-table scan reads pairs)
  uint64_t n;
  uint32_t cell_shift, phase_shift, block_shift, thread_shift;
  uint32_t phase_bits, block_bits, thread_bits;
  uint32_t n_warps;                    // warps of the cell scan
  DevResult* res;                      // the result, or one per model of a batch
  unsigned int* err;                   // error flags of the whole check
  unsigned int* groups;                // per result: (1 << phase_bits) x kWitnessGroupWords for the witness
  unsigned long long* long_list;       // first positions of cells handed to the long-cell pass
  unsigned long long* long_count;      // starts at 0
  uint64_t long_cap;                   // scan_long_capacity(n, n_warps)
  const uint64_t* cell_base;           // batch: first batch cell of each model (ascending)
  uint32_t n_models;                   // batch: number of models (0 = single model)
  uint32_t phase_table;                // keys sorted by cell only (phase_bits <= kScanTablePhaseBits)
  // warp and grid barriers (null without them): the phase field is a fine
  // interval q; device words [block interval of q, grid interval of q (4 bits
  // per q each), warp intervals per block interval | their bit width << 32],
  // one triple per model of a batch (a model without such barriers: q = its
  // phase, one grid interval, one warp interval)
  const uint64_t* sync_tabs;
  // witness group records per result: 2^(wit_block_bits + phase_bits), indexed
  // (block, fine interval) when wit_block_bits > 0 (models with more than one
  // grid interval), else by fine interval for the cell's lowest block only
  uint32_t wit_block_bits;
  // keys grouped by cell but not in cell order (bucket path): the first racy
  // cell is kept by value in DevResult.hash_cell (phase-table scan only)
  uint32_t by_cell;
  // phase-table scan: the number of keys on the device (the bucket path's
  // kept keys, in front of the buffer), or null for n
  const unsigned long long* n_dev;
  // keys sorted by (cell, fine interval) with warp or grid barriers: the grid
  // interval of each block interval (null: the 4-bit table of sync_tabs,
  // which covers fine intervals below 16)
  const uint32_t* grid_of;
};
// the interval tables of a scan (no warp or grid barriers: q is the phase)
struct SyncTabs {
  uint64_t coarse = 0, grid = 0;
  uint32_t n_wp = 1, wp_bits = 0;
  bool on = false;
};
cudaError_t launch_scan(const ScanArgs& a, cudaStream_t st);
cudaError_t launch_witness(const ScanArgs& a, cudaStream_t st);
// bucket.cu: the local sort of the bucket path: every bucket b = keys
// [boff[b], boff[b+1]) of keys_in (b < 2^D) put in cell order by the remaining
// bits of h and written to the same positions of keys_out (padding dropped:
// a bucket's kept keys come first in its range, padding after them), so that
// the ordered cell scan can fold keys_out up to boff[2^D] (with
// ScanArgs.by_cell and ScanArgs.n_dev; nothing behind it is read).
struct LocalSortArgs {
  const uint64_t* keys_in;
  uint64_t* keys_out;
  uint64_t n;                       // key slots of both buffers
  const unsigned long long* boff;
  uint64_t cmask;
  uint32_t cell_shift, cb, D, rbin, r;
  unsigned int* err;
};
cudaError_t launch_bucket_local_sort(const LocalSortArgs& a, cudaStream_t st);
// per result: [min_start, seg_end) = the bucket of its smallest racy cell
// (DevResult.hash_cell) and `cell` = that cell, for the witness kernels
struct FinishArgs {
  DevResult* res;
  uint32_t n_models;                // 0: one result
  const unsigned long long* boff;
  uint64_t cmask;
  uint32_t cb, D;
};
cudaError_t launch_bucket_finish(const FinishArgs& a, cudaStream_t st);
cudaError_t launch_init_result(DevResult* res, cudaStream_t st, uint32_t n = 1);
uint64_t scan_long_capacity(uint64_t n, uint32_t n_warps);

}  // namespace rc
