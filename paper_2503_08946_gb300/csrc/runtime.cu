// C ABI of the race checker (include/rc.h): model creation, workspace plan,
// the enqueued check pipeline and result tickets.
//
// rc_check enqueues, on the caller's stream:
//   clear of the look-back / histogram region -> result init -> K1 expand ->
//   digit histograms -> per pass K2 onesweep -> K3 scan + fold -> K4 witness ->
//   device-to-host copy of the result record into the ticket's pinned buffer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdlib>
#include <map>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "kernels.h"
#include "rc_internal.h"

struct rc_model {
  rc::Model m;
};

// Events recorded between the stages of one check (RC_OPT_STAGE_TIMES).
struct StageTimer {
  static constexpr int kMax = 24;
  cudaEvent_t ev[kMax] = {};
  int n = 0;
  cudaStream_t st = nullptr;
  bool ok = true;
  void mark() {
    if (n >= kMax) { ok = false; return; }
    if (!ev[n] && cudaEventCreate(&ev[n]) != cudaSuccess) { ok = false; return; }
    if (cudaEventRecord(ev[n], st) != cudaSuccess) ok = false;
    ++n;
  }
};

struct rc_ticket_s {
  StageTimer timer;
  bool timed = false;
  int i_start = 0, i_expand = 0, i_hist = 0, i_scan = 0, i_wit = 0;
  uint32_t n_pass = 0;
  int i_pass_from[16] = {}, i_pass_to[16] = {};   // events around each sort / partition pass
  int i_hist2_from = -1, i_hist2_to = -1;        // bucket path: the pass-B histogram
  bool bucketed = false;
  bool hist_fused = false;                        // the expansion counted the pass-A histogram
  uint64_t n_keys = 0;
  cudaEvent_t done = nullptr;
  rc::DevResult* host = nullptr;   // pinned, `cap` records
  size_t cap = 0;
  size_t n = 0;
  std::vector<const rc_model*> models;
  rc_status enqueue_status = RC_OK;
  // batch: per model, the first batch cell and the batch thread / phase widths
  // (witness decoding); empty for single checks
  std::vector<uint64_t> cell_base;
  std::vector<uint32_t> field_bits;   // thread_bits | phase_bits << 8
  void* upload = nullptr;             // pinned staging of the batch tables
  size_t upload_cap = 0;
  // chunked check: host[0] is the count pass, host[1 + k] chunk k, whose
  // cells start at chunk_lo[k]; the report merges them into one result
  bool chunked = false;
  std::vector<uint64_t> chunk_lo;
};

namespace {

std::mutex g_pool_mu;
std::vector<rc_ticket_s*> g_pool;

rc_ticket_s* ticket_get(size_t n) {
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (size_t i = 0; i < g_pool.size(); ++i) {
      if (g_pool[i]->cap >= n) {
        rc_ticket_s* t = g_pool[i];
        g_pool.erase(g_pool.begin() + (long)i);
        t->n = n;
        t->models.assign(n, nullptr);
        t->enqueue_status = RC_OK;
        t->cell_base.clear();
        t->field_bits.clear();
        t->chunked = false;
        t->chunk_lo.clear();
        t->timed = false;
        t->timer.n = 0;
        t->timer.ok = true;
        t->i_hist2_from = t->i_hist2_to = -1;
        t->bucketed = false;
        t->hist_fused = false;
        return t;
      }
    }
  }
  rc_ticket_s* t = new (std::nothrow) rc_ticket_s();
  if (!t) return nullptr;
  size_t cap = n < 1 ? 1 : n;
  if (cudaEventCreateWithFlags(&t->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost((void**)&t->host, cap * sizeof(rc::DevResult)) != cudaSuccess) {
    if (t->done) cudaEventDestroy(t->done);
    delete t;
    return nullptr;
  }
  t->cap = cap;
  t->n = n;
  t->models.assign(n, nullptr);
  return t;
}

void ticket_put(rc_ticket_s* t) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pool.size() < 64) {
    g_pool.push_back(t);
  } else {
    cudaEventDestroy(t->done);
    for (auto& e : t->timer.ev)
      if (e) cudaEventDestroy(e);
    cudaFreeHost(t->host);
    if (t->upload) cudaFreeHost(t->upload);
    delete t;
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

rc_status cuda_status(cudaError_t e) { return e == cudaSuccess ? RC_OK : RC_E_CUDA; }

uint32_t scan_warps_for(uint64_t n) {
  // whole segments of 32 x kScanRun keys per warp, at most kScanMaxWarps warps
  uint64_t w = (n + 32 * rc::kScanRun - 1) / (32 * rc::kScanRun);
  const uint64_t cap = rc::kScanMaxWarps;
  if (w > cap) w = cap;
  if (w < 1) w = 1;
  return (uint32_t)w;
}

}  // namespace

namespace rc {

namespace {
struct SmemAttr {
  int device;
  const void* func;
};
std::mutex g_attr_mu;
std::vector<SmemAttr> g_attr_done;
}  // namespace

cudaError_t ensure_kernel_smem(const void* func, size_t smem_bytes, bool max_carveout) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  for (const SmemAttr& d : g_attr_done)
    if (d.device == dev && d.func == func) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e == cudaSuccess && max_carveout)
    e = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  g_attr_done.push_back({dev, func});
  return cudaSuccess;
}

// Witness group records of one check: one per fine interval of the cell's
// lowest block, or one per (block, fine interval) with more than one grid
// interval (the smallest racing instance may then lie in a later block).
size_t witness_group_bytes(const Model& m) {
  const uint32_t bits = m.host.phase_bits + (m.multi_grid ? m.host.block_bits : 0u);
  return ((size_t)1 << bits) * kWitnessGroupWords * sizeof(unsigned int);
}

// The path a check takes: RC_PATH_HASH on request, otherwise the sort path.
bool use_hash_path(const Model&, const rc_check_opts* opts) { return opts && opts->path == RC_PATH_HASH; }
// the hash path maps fine intervals through the 4-bit interval tables, so
// with warp or grid barriers, or atomics, it covers at most 16 of them
bool hash_path_fits(const Model& m) {
  return !(m.sync_scopes || m.has_atomic) || m.host.phase_bits <= (uint32_t)kScanTablePhaseBits;
}

void plan_workspace(const Model& m, const rc_check_opts* opts, WorkspacePlan* p) {
  std::memset(p, 0, sizeof(*p));
  const uint64_t n = m.key_slots;
  p->n_keys = n;
  if (use_hash_path(m, opts)) {
    // tables of at least 1.5x the instances (an upper bound on distinct groups
    // and cells; three groups per instance with warp or grid barriers), the
    // keys of the first racy cell, witness phase groups
    p->hash = true;
    const uint64_t groups = m.sync_scopes ? 3 * n : n;
    uint64_t cap = 1024;
    while (cap < groups + groups / 2) cap <<= 1;
    p->hash_cap = cap;
    size_t off = 0;
    p->result_off = off;
    off = align256(off + sizeof(DevResult));
    p->gkey_off = off;
    off = align256(off + cap * 8);
    p->gword_off = off;
    off = align256(off + cap * 8);
    p->ckey_off = off;
    off = align256(off + cap * 8);
    p->cword_off = off;
    off = align256(off + cap * 8);
    p->filt_off = off;
    off = align256(off + n * 8);
    p->nfilt_off = off;
    off = align256(off + 8);
    p->group_off = off;
    off = align256(off + witness_group_bytes(m));
    p->total = off;
    return;
  }
  plan_workspace_keys(m, opts, n, m.host.cell_bits, p);
}

bool bucket_path_allowed(uint32_t phase_bits, const rc_check_opts* opts) {
  if (phase_bits > kScanTablePhaseBits) return false;   // the fold keeps per-interval masks of 16 intervals
  if (opts && ((opts->flags & RC_OPT_LSD) || opts->digit_bits || opts->test_flags)) return false;
  return true;
}

// n key slots, of which about n_expect are kept (a hash-partitioned check keeps
// its share): the bucket count is chosen for n_expect, the tile bounds for n
bool plan_buckets(uint64_t n, uint64_t n_expect, uint32_t cb, size_t off, BucketPlan* bp) {
  *bp = BucketPlan();
  if (n == 0 || n >= (1ull << 32) || cb == 0 || cb > 62) return false;
  if (n_expect == 0 || n_expect > n) n_expect = n;
  uint32_t D = 0;
  while (D < cb && D < kBucketMaxBits && (n_expect >> D) > kBucketTarget) ++D;
  if (D == kBucketMaxBits && D < cb && (n_expect >> D) > kBucketTarget) return false;   // more keys than the buckets hold
  bp->on = true;
  bp->n = n;
  bp->cb = cb;
  bp->D = D;
  bp->dA = D <= kBucketMaxDigitBits ? D : (D + 1) / 2;
  bp->dB = D - bp->dA;
  bp->r = cb - D;
  bp->rbin = bp->r < kFoldBinBits ? bp->r : kFoldBinBits;
  const uint64_t na = 1ull << bp->dA, nb = 1ull << D;
  bp->tiles_b = n / kPartTileHost + na + 1;
  bp->tiles_h = n / kBucketHistTile + na + 1;
  bp->zero_lo = off;
  bp->hist_a = off;
  off = align256(off + na * 8);
  bp->hist_b = off;
  off = align256(off + nb * 8);
  bp->scan_ctr = off;
  off = align256(off + 8);
  bp->zero_hi = off;
  bp->off_a = off;
  off = align256(off + (na + 1) * 8);
  bp->cur_a = off;
  off = align256(off + na * 8);
  bp->tpref_b = off;
  off = align256(off + (na + 1) * 8);
  bp->tile_a = off;
  off = align256(off + bp->tiles_b * 4);
  bp->tpref_h = off;
  off = align256(off + (na + 1) * 8);
  bp->boff = off;
  off = align256(off + (nb + 1) * 8);
  bp->cur_b = off;
  off = align256(off + nb * 8);
  bp->temp = off;
  off = align256(off + scan_u64_temp_bytes(nb));
  bp->end = off;
  return true;
}

void plan_workspace_keys(const Model& m, const rc_check_opts* opts, uint64_t n, uint32_t cell_bits,
                         WorkspacePlan* p, uint32_t min_lookback_bits, bool allow_bucket) {
  std::memset(p, 0, sizeof(*p));
  p->n_keys = n;
  const uint32_t hi = m.host.cell_shift + cell_bits;
  plan_sort(m.host.sort_lo < hi ? m.host.sort_lo : hi, hi, opts ? opts->digit_bits : 0, &p->sort);
  p->n_tiles = (n + kSortTile - 1) / kSortTile;
  p->scan_warps = scan_warps_for(n);
  size_t off = 0;
  p->result_off = off;
  off = align256(off + sizeof(DevResult));
  p->keys_off[0] = off;
  off = align256(off + n * 8);
  p->keys_off[1] = off;
  off = align256(off + n * 8);
  // a hash part keeps about 1 / part_count of the keys (the parts are
  // near-equal; 1/16 more for the spread), all with the same top bits of the
  // cell hash: its buckets are cut from the hash's remaining bits
  const bool part = opts && opts->part_count > 1;
  const uint32_t part_bits = part ? bit_length(opts->part_count - 1) : 0u;
  const uint64_t n_expect = part ? n / opts->part_count + n / (16ull * opts->part_count) + 1 : n;
  if (allow_bucket && bucket_path_allowed(m.host.phase_bits, opts) && cell_bits > part_bits &&
      plan_buckets(n, n_expect, cell_bits - part_bits, off, &p->bucket)) {
    // the bucket path: its own section instead of the radix-sort sections
    p->zero_lo = p->bucket.zero_lo;
    p->zero_hi = p->bucket.zero_hi;
    off = p->bucket.end;
    p->scanctr_off = p->bucket.scan_ctr;
    p->long_cap = scan_long_capacity(n, p->scan_warps);
    p->long_off = off;
    off = align256(off + (size_t)p->long_cap * 8);
    p->group_off = off;
    off = align256(off + witness_group_bytes(m));
    p->total = off;
    return;
  }
  p->zero_lo = off;
  p->hist_off = off;
  off = align256(off + (size_t)16 * kMaxRadix * 8);
  p->lookback_off = off;
  off = align256(off + (size_t)p->n_tiles * ((size_t)1 << std::max(plan_max_bits(p->sort), min_lookback_bits)) * 8);
  p->tilectr_off = off;
  off = align256(off + 16 * sizeof(unsigned int));
  p->scanctr_off = off;
  off = align256(off + 8);
  p->zero_hi = off;
  p->digoff_off = off;
  off = align256(off + (size_t)16 * kMaxRadix * 8);
  p->cursor_off = off;
  off = align256(off + (size_t)kMaxRadix * 8);
  p->long_cap = scan_long_capacity(n, p->scan_warps);
  p->long_off = off;   // cells handed to the long-cell pass
  off = align256(off + (size_t)p->long_cap * 8);
  p->group_off = off;
  off = align256(off + witness_group_bytes(m));
  p->total = off;
}

}  // namespace rc

namespace {

rc::ScanArgs scan_args(const rc::Model& m, const rc::WorkspacePlan& p, uint8_t* ws, int sorted_buf) {
  rc::ScanArgs a;
  a.keys = reinterpret_cast<const uint64_t*>(ws + p.keys_off[sorted_buf]);
  a.n = p.n_keys;
  a.cell_shift = m.host.cell_shift;
  a.phase_shift = m.host.phase_shift;
  a.block_shift = m.host.block_shift;
  a.thread_shift = m.host.thread_shift;
  a.phase_bits = m.host.phase_bits;
  a.block_bits = m.host.block_bits;
  a.thread_bits = m.host.thread_bits;
  a.n_warps = p.scan_warps;
  a.res = reinterpret_cast<rc::DevResult*>(ws + p.result_off);
  a.err = &a.res->err;
  a.groups = reinterpret_cast<unsigned int*>(ws + p.group_off);
  a.long_list = reinterpret_cast<unsigned long long*>(ws + p.long_off);
  a.long_count = reinterpret_cast<unsigned long long*>(ws + p.scanctr_off);
  a.long_cap = p.long_cap;
  a.cell_base = nullptr;
  a.n_models = 0;
  a.phase_table = m.host.phase_bits <= rc::kScanTablePhaseBits ? 1u : 0u;
  // the interval tables live in the uploaded program header
  a.sync_tabs = m.sync_scopes ? reinterpret_cast<const uint64_t*>(static_cast<const uint8_t*>(m.dev_program) +
                                                                  offsetof(rc::DevModel, sync_tab))
                              : nullptr;
  a.wit_block_bits = m.multi_grid ? m.host.block_bits : 0u;
  a.by_cell = 0;
  a.n_dev = nullptr;
  a.grid_of = m.sec_gridof ? reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(m.dev_program) +
                                                               m.sec_gridof)
                           : nullptr;
  return a;
}

// Enqueue the sort of p.n_keys keys from buffer 0; returns the index of the
// buffer holding the sorted keys.
// unstable_first: the first pass may leave equal digits in any order (the
// input order of a check's keys carries no meaning), so it runs as the
// look-back-free partition pass.
rc_status enqueue_sort(const rc::WorkspacePlan& p, uint8_t* ws, uint64_t* buf0, uint64_t* buf1,
                       uint64_t spin_limit, uint32_t test_flags, cudaStream_t st, int* sorted_buf,
                       StageTimer* tm = nullptr, bool unstable_first = false) {
  uint64_t* bufs[2] = {buf0, buf1};
  auto* hist = reinterpret_cast<unsigned long long*>(ws + p.hist_off);
  auto* digoff = reinterpret_cast<unsigned long long*>(ws + p.digoff_off);
  auto* res = reinterpret_cast<rc::DevResult*>(ws + p.result_off);
  rc_status s = cuda_status(rc::launch_digit_counts(bufs[0], p.n_keys, p.sort, hist, st));
  if (s != RC_OK) return s;
  s = cuda_status(rc::launch_digit_offsets(hist, digoff, p.sort, st));
  if (s != RC_OK) return s;
  if (tm) tm->mark();
  const int i_first = tm ? tm->n - 1 : 0;
  int cur = 0;
  for (uint32_t k = 0; k < p.sort.n_pass; ++k) {
    rc::SortArgs a;
    a.keys_in = bufs[cur];
    a.keys_out = bufs[1 - cur];
    a.n = p.n_keys;
    a.shift = p.sort.shift[k];
    a.bits = p.sort.bits[k];
    a.digit_offset = digoff + (size_t)k * rc::kMaxRadix;
    a.lookback = reinterpret_cast<unsigned long long*>(ws + p.lookback_off);
    a.tile_counter = reinterpret_cast<unsigned int*>(ws + p.tilectr_off) + k;
    a.epoch = k + 1;
    // the stall test waits for an epoch no pass ever publishes
    a.wait_epoch = (test_flags & RC_TEST_STALL_LOOKBACK) ? (k + 1) ^ 0x8000u : k + 1;
    a.spin_limit = spin_limit;
    a.err = &res->err;
    a.cursor = nullptr;
    if (k == 0 && unstable_first && !(test_flags & RC_TEST_STALL_LOOKBACK)) {
      a.cursor = reinterpret_cast<unsigned long long*>(ws + p.cursor_off);
      s = cuda_status(cudaMemcpyAsync(a.cursor, a.digit_offset, ((size_t)1 << a.bits) * 8, cudaMemcpyDeviceToDevice, st));
      if (s == RC_OK) s = cuda_status(rc::launch_partition(a, rc::radix_bits_for(a.bits), st));
    } else {
      s = cuda_status(rc::launch_onesweep(a, rc::radix_bits_for(a.bits), st));
    }
    if (s != RC_OK) return s;
    if (tm) tm->mark();
    cur = 1 - cur;
  }
  (void)i_first;
  *sorted_buf = cur;
  return RC_OK;
}

// Enqueue the bucket path (bucket.cu) over p.n_keys keys in buf0: partition
// passes, bucket fold and the finish that points the witness at the smallest
// racy cell's bucket.  `sa` carries the key layout, results and tables; on
// return *final_keys is the buffer the witness reads.  Stage events: after the
// pass-A histogram (i_hist), around each pass, around the pass-B histogram.
rc_status enqueue_bucketed(const rc::WorkspacePlan& p, uint8_t* ws, uint64_t* buf0, uint64_t* buf1,
                           const rc::ScanArgs& sa, cudaStream_t st, const uint64_t** final_keys,
                           rc_ticket_s* timed = nullptr, bool hist_a_done = false) {
  const rc::BucketPlan& bp = p.bucket;
  StageTimer* tm = timed ? &timed->timer : nullptr;
  auto u64 = [&](size_t off) { return reinterpret_cast<unsigned long long*>(ws + off); };
  rc::BucketArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = p.n_keys;
  a.cell_shift = sa.cell_shift;
  a.cb = bp.cb;
  a.cmask = bp.cb >= 64 ? ~0ull : ((1ull << bp.cb) - 1ull);
  a.dA = bp.dA;
  a.dB = bp.dB;
  a.hist_a = u64(bp.hist_a);
  a.off_a = u64(bp.off_a);
  a.cur_a = u64(bp.cur_a);
  a.tpref_b = u64(bp.tpref_b);
  a.tile_a = reinterpret_cast<unsigned*>(ws + bp.tile_a);
  a.tpref_h = u64(bp.tpref_h);
  a.hist_b = u64(bp.hist_b);
  a.boff = u64(bp.boff);
  a.cur_b = u64(bp.cur_b);
  a.temp = u64(bp.temp);
  a.err = sa.err;
  uint64_t* fin = buf0;
  uint64_t* scratch = buf1;
  uint32_t n_pass = 0;
  rc_status s = RC_OK;
  if (bp.D == 0) {
    s = cuda_status(rc::launch_bucket_whole(a.boff, p.n_keys, st));
    if (tm) { timed->i_hist = tm->n; tm->mark(); }
  } else {
    a.keys_in = buf0;
    a.keys_out = buf1;
    // (the generated expansion may have counted the pass-A histogram already)
    if (!hist_a_done) s = cuda_status(rc::launch_bucket_hist_a(a, st));
    if (s == RC_OK) s = cuda_status(rc::launch_bucket_scan_a(a, st));
    if (tm) { timed->i_hist = tm->n; tm->mark(); }
    if (s == RC_OK) s = cuda_status(rc::launch_bucket_pass_a(a, st));
    if (tm) { timed->i_pass_from[0] = tm->n - 1; timed->i_pass_to[0] = tm->n; tm->mark(); }
    n_pass = 1;
    fin = buf1;
    scratch = buf0;
    if (bp.dB && s == RC_OK) {
      a.keys_in = buf1;
      a.keys_out = buf0;
      s = cuda_status(rc::launch_bucket_hist_b(a, bp.tiles_h, st));
      if (s == RC_OK) s = cuda_status(rc::launch_bucket_scan_b(a, st));
      if (tm) { timed->i_hist2_from = tm->n - 1; timed->i_hist2_to = tm->n; tm->mark(); }
      if (s == RC_OK) s = cuda_status(rc::launch_bucket_pass_b(a, bp.tiles_b, st));
      if (tm) { timed->i_pass_from[1] = tm->n - 1; timed->i_pass_to[1] = tm->n; tm->mark(); }
      n_pass = 2;
      fin = buf0;
      scratch = buf1;
    }
  }
  if (s != RC_OK) return s;
  // the local sort into the other buffer, then the ordered cell scan with the
  // first racy cell kept by value, then its bucket for the witness
  rc::LocalSortArgs ls;
  ls.keys_in = fin;
  ls.keys_out = scratch;
  ls.n = p.n_keys;
  ls.boff = a.boff;
  ls.cmask = a.cmask;
  ls.cell_shift = sa.cell_shift;
  ls.cb = bp.cb;
  ls.D = bp.D;
  ls.rbin = bp.rbin;
  ls.r = bp.r;
  ls.err = sa.err;
  s = cuda_status(rc::launch_bucket_local_sort(ls, st));
  if (tm) { timed->i_pass_from[n_pass] = tm->n - 1; timed->i_pass_to[n_pass] = tm->n; tm->mark(); }
  ++n_pass;
  rc::ScanArgs sc = sa;
  sc.keys = scratch;
  sc.n = p.n_keys;
  sc.n_dev = a.boff + ((size_t)1 << bp.D);   // the kept keys: the scan reads nothing behind them
  sc.by_cell = 1;
  sc.phase_table = 1;
  if (s == RC_OK) s = cuda_status(rc::launch_scan(sc, st));
  rc::FinishArgs fa;
  fa.res = sa.res;
  fa.n_models = sa.n_models;
  fa.boff = a.boff;
  fa.cmask = a.cmask;
  fa.cb = bp.cb;
  fa.D = bp.D;
  if (s == RC_OK) s = cuda_status(rc::launch_bucket_finish(fa, st));
  if (timed) {
    timed->n_pass = n_pass;
    timed->bucketed = true;
  }
  fin = scratch;
  *final_keys = fin;
  return s;
}

rc_status enqueue_check(rc_model* model, const rc_check_opts* opts, uint8_t* ws, size_t ws_bytes,
                        cudaStream_t st, rc::DevResult* host_out, rc_ticket_s* timed = nullptr) {
  const rc::Model& m = model->m;
  rc::WorkspacePlan p;
  rc::plan_workspace(m, opts, &p);
  if (!ws || ws_bytes < p.total) return RC_E_NOMEM;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return RC_E_INVALID;
  const uint64_t spin = (opts && opts->spin_limit) ? opts->spin_limit : (1ull << 20);
  const uint64_t cell_lo = opts ? opts->cell_lo : 0;
  const uint64_t cell_hi = (opts && opts->cell_hi) ? opts->cell_hi : ~0ull;
  auto* res = reinterpret_cast<rc::DevResult*>(ws + p.result_off);
  StageTimer* tm = nullptr;
  if (timed) {
    tm = &timed->timer;
    tm->st = st;
    tm->n = 0;
    tm->ok = true;
    timed->timed = true;
    timed->n_pass = p.sort.n_pass;
    timed->n_keys = p.n_keys;
  }
  const rc::DevModel* dm = reinterpret_cast<const rc::DevModel*>(m.dev_program);
  rc_status s = cuda_status(rc::launch_init_result(res, st));
  if (s != RC_OK) return s;
  if (p.hash) {
    rc::HashArgs h;
    h.gkey = reinterpret_cast<unsigned long long*>(ws + p.gkey_off);
    h.gword = reinterpret_cast<unsigned long long*>(ws + p.gword_off);
    h.ckey = reinterpret_cast<unsigned long long*>(ws + p.ckey_off);
    h.cword = reinterpret_cast<unsigned long long*>(ws + p.cword_off);
    h.gmask = h.cmask = p.hash_cap - 1;
    h.res = res;
    h.early_exit = opts && opts->early_exit ? 1u : 0u;
    h.stop = &res->stop;
    h.filtered = reinterpret_cast<uint64_t*>(ws + p.filt_off);
    h.n_filtered = reinterpret_cast<unsigned long long*>(ws + p.nfilt_off);
    h.cell_lo = cell_lo;
    h.cell_hi = cell_hi;
    h.sync = m.sync_scopes ? 1u : 0u;
    s = cuda_status(cudaMemsetAsync(h.gkey, 0xFF, p.hash_cap * 8, st));
    if (s == RC_OK) s = cuda_status(cudaMemsetAsync(h.ckey, 0xFF, p.hash_cap * 8, st));
    if (s == RC_OK) s = cuda_status(cudaMemsetAsync(h.gword, 0, p.hash_cap * 8, st));
    if (s == RC_OK) s = cuda_status(cudaMemsetAsync(h.cword, 0, p.hash_cap * 8, st));
    if (s == RC_OK) s = cuda_status(cudaMemsetAsync(h.n_filtered, 0, 8, st));
    if (s != RC_OK) return s;
    if (tm) { timed->i_start = tm->n; tm->mark(); }
    s = cuda_status(rc::launch_hash(dm, m.host.n_stmts, m.host.n_threads, h, st));
    if (s != RC_OK) return s;
    if (tm) {
      timed->i_expand = timed->i_hist = timed->i_scan = tm->n;
      timed->n_pass = 0;
      tm->mark();
    }
    rc::ScanArgs sa = scan_args(m, p, ws, 0);
    sa.keys = h.filtered;
    s = cuda_status(rc::launch_witness(sa, st));
    if (s != RC_OK) return s;
    if (tm) { timed->i_wit = tm->n; tm->mark(); }
    if (host_out)
      s = cuda_status(cudaMemcpyAsync(host_out, res, sizeof(rc::DevResult), cudaMemcpyDeviceToHost, st));
    return s;
  }
  s = cuda_status(cudaMemsetAsync(ws + p.zero_lo, 0, p.zero_hi - p.zero_lo, st));
  if (s != RC_OK) return s;
  if (tm) { timed->i_start = tm->n; tm->mark(); }
  // the bucket path's pass-A histogram is counted by the generated expansion
  // as it writes the keys (the interpreted expansion leaves it to its kernel)
  rc::ExpandHist eh{};
  const bool fuse_hist = p.bucket.on && p.bucket.D > 0 && m.jit_fn != nullptr && p.bucket.dA <= rc::kBucketMaxDigitBits;
  if (fuse_hist) {
    eh.hist = reinterpret_cast<unsigned long long*>(ws + p.bucket.hist_a);
    eh.cmask = p.bucket.cb >= 64 ? ~0ull : ((1ull << p.bucket.cb) - 1ull);
    eh.shift = p.bucket.cb - p.bucket.dA;
    eh.bins = 1u << p.bucket.dA;
  }
  if (timed) timed->hist_fused = fuse_hist;
  rc::CellFilter cf;
  cf.lo = cell_lo;
  cf.hi = cell_hi;
  if (opts && opts->part_count > 1) {
    // part = (h * 2^pb) >> cb of the cb-bit hash h: its top pb bits, or with
    // pb > cb the hash shifted up (a part with any of the low pb - cb bits set
    // is empty: a mask no hash meets)
    const uint32_t pb = rc::bit_length(opts->part_count - 1), cb = m.host.cell_bits;
    if (pb <= cb) {
      cf.pmask = ((uint64_t)opts->part_count - 1) << (cb - pb);
      cf.pval = (uint64_t)opts->part_index << (cb - pb);
    } else if ((opts->part_index & ((1u << (pb - cb)) - 1u)) != 0u) {
      cf.lo = cf.hi = 0;   // the part holds no cell: an empty range
    } else {
      cf.pmask = cb >= 64 ? ~0ull : (1ull << cb) - 1ull;
      cf.pval = (uint64_t)(opts->part_index >> (pb - cb));
    }
  }
  if (m.jit_fn)
    s = cuda_status(rc::jit_expand_launch(m, reinterpret_cast<uint64_t*>(ws + p.keys_off[0]), res, st, cf,
                                          fuse_hist ? &eh : nullptr));
  else
    s = cuda_status(rc::launch_expand(dm, m.host.n_stmts, m.host.n_threads, m.has_deep_loops,
                                      reinterpret_cast<uint64_t*>(ws + p.keys_off[0]), res, st, cf));
  if (s != RC_OK) return s;
  if (tm) { timed->i_expand = tm->n; tm->mark(); }
  if (p.bucket.on) {
    // the bucket path: partition passes and the bucket fold
    const uint64_t* fin = nullptr;
    rc::ScanArgs sa = scan_args(m, p, ws, 0);
    s = enqueue_bucketed(p, ws, reinterpret_cast<uint64_t*>(ws + p.keys_off[0]),
                         reinterpret_cast<uint64_t*>(ws + p.keys_off[1]), sa, st, &fin, timed, fuse_hist);
    if (s != RC_OK) return s;
    if (tm) { timed->i_scan = tm->n; tm->mark(); }
    sa.keys = fin;
    s = cuda_status(rc::launch_witness(sa, st));
    if (s != RC_OK) return s;
    if (tm) { timed->i_wit = tm->n; tm->mark(); }
    if (host_out) s = cuda_status(cudaMemcpyAsync(host_out, res, sizeof(rc::DevResult), cudaMemcpyDeviceToHost, st));
    return s;
  }
  int sorted = 0;
  if (tm) {
    timed->i_hist = tm->n;
    for (uint32_t k = 0; k < p.sort.n_pass && k < 16; ++k) {
      timed->i_pass_from[k] = tm->n + (int)k;
      timed->i_pass_to[k] = tm->n + (int)k + 1;
    }
  }
  s = enqueue_sort(p, ws, reinterpret_cast<uint64_t*>(ws + p.keys_off[0]),
                   reinterpret_cast<uint64_t*>(ws + p.keys_off[1]), spin,
                   opts ? opts->test_flags : 0u, st, &sorted, tm, true);
  if (s != RC_OK) return s;
  if (p.n_keys > 0) {
    rc::ScanArgs sa = scan_args(m, p, ws, sorted);
    if (opts && (opts->test_flags & RC_TEST_FEW_SCAN_WARPS) && sa.n_warps > 3) sa.n_warps = 3;
    s = cuda_status(rc::launch_scan(sa, st));
    if (s != RC_OK) return s;
    if (tm) { timed->i_scan = tm->n; tm->mark(); }
    s = cuda_status(rc::launch_witness(sa, st));
    if (s != RC_OK) return s;
    if (tm) { timed->i_wit = tm->n; tm->mark(); }
  } else if (tm) {
    timed->i_scan = tm->n; tm->mark();
    timed->i_wit = tm->n; tm->mark();
  }
  if (host_out) {
    s = cuda_status(cudaMemcpyAsync(host_out, res, sizeof(rc::DevResult), cudaMemcpyDeviceToHost, st));
    if (s != RC_OK) return s;
  }
  return RC_OK;
}

// cell_base: first batch cell of the model (0 for a single check); tb / pb /
// kb: thread, phase and kind widths of the keys the witness ranks were taken
// from.
void decode_result(const rc::DevResult& r, const rc::Model& m, rc_result* out, uint64_t cell_base, uint32_t tb,
                   uint32_t pb, uint32_t kb = 1, uint32_t wb = 0) {
  std::memset(out, 0, sizeof(*out));
  out->instances = r.instances;
  if (r.err & (rc::kErrLookbackTimeout | rc::kErrCopyTimeout)) {
    out->status = RC_E_TIMEOUT;
    return;
  }
  if (r.err & (rc::kErrHashFull | rc::kErrScanLongFull)) {
    out->status = RC_E_NOMEM;
    return;
  }
  if (r.err & rc::kErrSortRange) {   // (the sort's guard against an out-of-range store fired)
    out->status = RC_E_CUDA;
    return;
  }
  if (r.oob_code != ~0ull) {
    out->status = RC_E_OOB;
    out->oob_stmt = (uint32_t)(r.oob_code >> 51);
    out->oob_access = (uint32_t)((r.oob_code >> 45) & 63u);
    out->oob_gtid = (r.oob_code >> 3) & ((1ull << 42) - 1);
    out->oob_dim = (int32_t)(r.oob_code & 7u);
    return;
  }
  out->status = RC_OK;
  out->racy_cells = r.racy_cells;
  out->verdict = r.racy_cells > 0;
  if (!out->verdict || r.x_rank == ~0ull || r.y_rank == ~0ull) return;
  // cell -> (array, scope instance, element)
  const uint64_t cell = r.cell - cell_base;
  size_t a = 0;
  for (size_t k = 0; k < m.array_base.size(); ++k)
    if (m.array_base[k] <= cell) a = k;
  const uint64_t rem = cell - m.array_base[a];
  out->w_array = (uint32_t)a;
  out->w_scope = m.array_shared[a] ? rem / m.array_cells[a] : 0;
  out->w_addr = m.array_shared[a] ? rem % m.array_cells[a] : rem;
  // ranks of x and y: (block, phase, thread, kind, warp phase)
  const uint64_t tmask = (1ull << tb) - 1, pmask = (1ull << pb) - 1, kmask = (1ull << kb) - 1;
  const uint64_t wmask = (1ull << wb) - 1;
  const uint64_t bs = m.host.bs;
  out->x.block = r.x_rank >> (pb + tb + kb + wb);
  out->x.warp_phase = (uint32_t)(r.x_rank & wmask);
  out->x.kind = (uint32_t)((r.x_rank >> wb) & kmask);
  out->x.thread = (uint32_t)((r.x_rank >> (wb + kb)) & tmask);
  out->x.phase = (int64_t)((r.x_rank >> (wb + tb + kb)) & pmask);
  out->x.gtid = out->x.block * bs + out->x.thread;
  out->y.warp_phase = (uint32_t)(r.y_rank & wmask);
  out->y.kind = (uint32_t)((r.y_rank >> wb) & kmask);
  out->y.thread = (uint32_t)((r.y_rank >> (wb + kb)) & tmask);
  out->y.phase = (int64_t)((r.y_rank >> (wb + tb + kb)) & pmask);
  out->y.block = r.y_rank >> (pb + tb + kb + wb);
  out->y.gtid = out->y.block * bs + out->y.thread;
}

// ---------------------------------------------------------------------------
// chunked check: models wider than one key, and checks in a bounded workspace
// ---------------------------------------------------------------------------
// A count pass expands the whole model (all instances are counted and
// bounds-checked) and histograms its keys over buckets of 2^bshift cells of the
// checked range.  The host then cuts the range into chunks of whole buckets,
// each with a cell span that fits the key's cell field and at most `cap` keys
// (what the workspace holds), and groups consecutive chunks into waves whose
// keys fit the workspace together.  Per wave one expansion routes every key of
// the wave's chunks to its chunk's segment, with its cell rebased to the chunk
// start; then each chunk runs the ordinary sort, scan and witness stages on its
// segment.  A cell races or not on its own, so the chunk counts add up and the
// smallest racing pair is the one of the first chunk with a race.
constexpr uint64_t kMaxChunkBuckets = 1ull << 20;
constexpr size_t kMaxChunks = 1u << 16;

struct ChunkGeometry {
  uint64_t lo = 0, span = 0;   // checked cell range [lo, lo + span)
  uint32_t bshift = 0;         // bucket = (cell - lo) >> bshift
  uint64_t n_buckets = 0;
  uint64_t max_span = 0;       // cells one chunk may span
  // workspace: bucket counts | chunk of each bucket | per chunk (lo, base, end, counter) | region
  size_t counts_off = 0, table_off = 0, chunks_off = 0, region_off = 0;
};

rc_status chunk_geometry(const rc::Model& m, const rc_check_opts* opts, ChunkGeometry* g) {
  uint64_t lo = opts ? opts->cell_lo : 0;
  uint64_t hi = (opts && opts->cell_hi) ? opts->cell_hi : m.total_cells;
  if (hi > m.total_cells) hi = m.total_cells;
  if (lo > hi) lo = hi;
  g->lo = lo;
  g->span = hi - lo;
  const uint32_t cb = m.host.cell_bits;
  g->max_span = cb >= 63 ? (1ull << 62) : (1ull << cb) - 1ull;
  uint32_t bs = 0;
  while (bs < 63 && ((g->span + (1ull << bs) - 1) >> bs) > kMaxChunkBuckets) ++bs;
  if (bs > 0 && (1ull << bs) > g->max_span) return RC_E_KEY_OVERFLOW;   // would need too many chunks
  g->bshift = bs;
  g->n_buckets = g->span ? ((g->span - 1) >> bs) + 1 : 0;
  const size_t nb = g->n_buckets ? g->n_buckets : 1;
  g->counts_off = 0;
  g->table_off = align256(g->counts_off + nb * 8);
  g->chunks_off = align256(g->table_off + nb * 4);
  g->region_off = align256(g->chunks_off + kMaxChunks * 4 * 8);
  return RC_OK;
}

// widest digit any chunk's sort may use (plan_sort's clamp of the digit width)
uint32_t chunk_digit_bits(const rc_check_opts* opts) {
  const uint32_t d = (opts && opts->digit_bits) ? opts->digit_bits : 8u;
  return d < 4 ? 4u : (d > 11 ? 11u : d);
}

// the region's layout for n keys
void chunk_region_plan(const rc::Model& m, const rc_check_opts* opts, uint64_t n, rc::WorkspacePlan* p) {
  rc::plan_workspace_keys(m, opts, n, m.host.cell_bits, p, chunk_digit_bits(opts), false);
}

// keys one region can hold in `bytes` (~0 if not even its fixed part fits)
uint64_t chunk_capacity(const rc::Model& m, const rc_check_opts* opts, size_t bytes, uint64_t upper) {
  rc::WorkspacePlan p;
  uint64_t lo = 0, hi = upper;
  chunk_region_plan(m, opts, 0, &p);
  if (p.total > bytes) return ~0ull;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo + 1) / 2;
    chunk_region_plan(m, opts, mid, &p);
    if (p.total <= bytes) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

size_t chunked_workspace_size(const rc::Model& m, const rc_check_opts* opts) {
  ChunkGeometry g;
  if (chunk_geometry(m, opts, &g) != RC_OK) return 0;
  rc::WorkspacePlan p;
  chunk_region_plan(m, opts, m.key_slots, &p);
  return g.region_off + p.total;
}

bool use_chunked(const rc::Model& m, const rc_check_opts* opts) {
  return m.wide || (opts && (opts->flags & RC_OPT_CHUNKED));
}

// Count pass, planning (one host synchronisation) and the enqueued waves.
rc_status enqueue_chunked(rc_model* model, const rc_check_opts* opts, uint8_t* ws, size_t ws_bytes,
                          cudaStream_t st, rc_ticket_s** out) {
  const rc::Model& m = model->m;
  *out = nullptr;
  if (opts && opts->path == RC_PATH_HASH) return m.wide ? RC_E_KEY_OVERFLOW : RC_E_INVALID;
  if (!ws) return RC_E_NOMEM;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return RC_E_INVALID;
  ChunkGeometry g;
  rc_status s = chunk_geometry(m, opts, &g);
  if (s != RC_OK) return s;
  if (ws_bytes <= g.region_off) return RC_E_NOMEM;
  const uint64_t cap = chunk_capacity(m, opts, ws_bytes - g.region_off, m.key_slots);
  if (cap == ~0ull) return RC_E_NOMEM;
  uint8_t* region = ws + g.region_off;
  auto* counts = reinterpret_cast<unsigned long long*>(ws + g.counts_off);
  const rc::DevModel* dm = reinterpret_cast<const rc::DevModel*>(m.dev_program);
  // the region's layout for a full wave; each chunk uses a prefix of its scratch
  rc::WorkspacePlan pc;
  chunk_region_plan(m, opts, cap, &pc);
  auto* res = reinterpret_cast<rc::DevResult*>(region + pc.result_off);

  // count pass
  rc::DevResult r0;
  std::vector<unsigned long long> hc(g.n_buckets);
  s = cuda_status(rc::launch_init_result(res, st));
  if (s == RC_OK && g.n_buckets) s = cuda_status(cudaMemsetAsync(counts, 0, g.n_buckets * 8, st));
  rc::ChunkJitArgs ja;
  std::memset(&ja, 0, sizeof(ja));
  ja.oob = &res->oob_code;
  ja.inst = &res->instances;
  ja.tdata = m.host.tdata;
  ja.counts = counts;
  ja.lo = g.lo;
  ja.span = g.span;
  ja.bshift = g.bshift;
  ja.cell_shift = m.host.cell_shift;
  ja.err = &res->err;
  if (s == RC_OK) {
    if (m.jit_chunk_fn)
      s = cuda_status(rc::jit_chunk_launch(m, ja, st));
    else
      s = cuda_status(rc::launch_expand_count(dm, m.host.n_stmts, m.host.n_threads, m.has_deep_loops, res, counts,
                                              g.lo, g.span, g.bshift, st));
  }
  if (s == RC_OK) s = cuda_status(cudaMemcpyAsync(&r0, res, sizeof(r0), cudaMemcpyDeviceToHost, st));
  if (s == RC_OK && g.n_buckets)
    s = cuda_status(cudaMemcpyAsync(hc.data(), counts, g.n_buckets * 8, cudaMemcpyDeviceToHost, st));
  if (s == RC_OK) s = cuda_status(cudaStreamSynchronize(st));
  if (s != RC_OK) return s;

  // chunks of whole buckets (at most `cap` keys, `max_span` cells), then waves
  // of consecutive chunks with at most `cap` keys together
  struct Chunk { uint64_t lo, span, n, b0, b1, base; };
  struct Wave { size_t k0, k1; uint64_t b0, b1; };
  std::vector<Chunk> chunks;
  std::vector<Wave> waves;
  std::vector<uint32_t> chunk_of(g.n_buckets, 0xffffffffu);
  if (r0.oob_code == ~0ull && r0.err == 0) {
    const uint64_t per = g.max_span >> g.bshift;   // buckets one chunk may span (>= 1)
    uint64_t i = 0;
    while (i < g.n_buckets) {
      if (hc[i] == 0) { ++i; continue; }
      if (hc[i] > cap) return RC_E_NOMEM;   // one bucket's keys do not fit the workspace
      const uint64_t start = i;
      uint64_t n = 0;
      while (i < g.n_buckets && i - start < per && n + hc[i] <= cap) n += hc[i++];
      if (chunks.size() == kMaxChunks) return RC_E_NOMEM;
      const uint64_t clo = g.lo + (start << g.bshift);
      const uint64_t cend = std::min(g.lo + (i << g.bshift), g.lo + g.span);
      for (uint64_t b = start; b < i; ++b) chunk_of[b] = (uint32_t)chunks.size();
      chunks.push_back(Chunk{clo, cend - clo, n, start, i, 0});
    }
    // segments start at even key positions (the scan reads 16-byte pairs)
    uint64_t used = 0;
    for (size_t k = 0; k < chunks.size(); ++k) {
      if (waves.empty() || ((used + 1) & ~1ull) + chunks[k].n > cap) {
        waves.push_back(Wave{k, k, chunks[k].b0, chunks[k].b0});
        used = 0;
      }
      used = (used + 1) & ~1ull;
      chunks[k].base = used;
      used += chunks[k].n;
      waves.back().k1 = k + 1;
      waves.back().b1 = chunks[k].b1;
    }
  }
  rc_ticket_s* t = ticket_get(chunks.size() + 1);
  if (!t) return RC_E_NOMEM;
  t->models.assign(chunks.size() + 1, model);
  t->chunked = true;
  t->host[0] = r0;
  for (const Chunk& c : chunks) t->chunk_lo.push_back(c.lo);
  if (!chunks.empty()) {
    // tables of the route pass: chunk of each bucket; per chunk lo, base, end, counter
    const size_t K = chunks.size();
    std::vector<uint64_t> arr(4 * K, 0);
    for (size_t k = 0; k < K; ++k) {
      arr[k] = chunks[k].lo;
      arr[K + k] = chunks[k].base;
      arr[2 * K + k] = chunks[k].base + chunks[k].n;
    }
    s = cuda_status(cudaMemcpyAsync(ws + g.table_off, chunk_of.data(), g.n_buckets * 4, cudaMemcpyHostToDevice, st));
    if (s == RC_OK)
      s = cuda_status(cudaMemcpyAsync(ws + g.chunks_off, arr.data(), arr.size() * 8, cudaMemcpyHostToDevice, st));
  }
  const uint64_t spin = (opts && opts->spin_limit) ? opts->spin_limit : (1ull << 20);
  uint64_t* keys0 = reinterpret_cast<uint64_t*>(region + pc.keys_off[0]);
  uint64_t* keys1 = reinterpret_cast<uint64_t*>(region + pc.keys_off[1]);
  const size_t K = chunks.size();
  auto* c_lo = reinterpret_cast<const uint64_t*>(ws + g.chunks_off);
  for (const Wave& wv : waves) {
    if (s != RC_OK) break;
    rc::RouteArgs ra;
    ra.keys = keys0;
    ra.chunk_of = reinterpret_cast<const uint32_t*>(ws + g.table_off) + wv.b0;
    ra.c_lo = c_lo;
    ra.c_base = c_lo + K;
    ra.c_end = c_lo + 2 * K;
    ra.c_ctr = reinterpret_cast<unsigned long long*>(ws + g.chunks_off) + 3 * K;
    ra.lo = g.lo;
    ra.span = g.span;
    ra.b0 = wv.b0;
    ra.n_buckets = wv.b1 - wv.b0;
    ra.low_mask = (1ull << m.host.cell_shift) - 1ull;
    ra.bshift = g.bshift;
    ra.cell_shift = m.host.cell_shift;
    s = cuda_status(cudaMemsetAsync(ra.c_ctr + wv.k0, 0, (wv.k1 - wv.k0) * 8, st));
    if (s == RC_OK) s = cuda_status(rc::launch_init_result(res, st));
    if (s == RC_OK && m.jit_chunk_fn) {
      rc::ChunkJitArgs jr = ja;
      jr.mode = 1;
      jr.keys = ra.keys;
      jr.chunk_of = ra.chunk_of;
      jr.c_lo = ra.c_lo;
      jr.c_base = ra.c_base;
      jr.c_end = ra.c_end;
      jr.c_ctr = ra.c_ctr;
      jr.b0 = ra.b0;
      jr.n_buckets = ra.n_buckets;
      jr.low_mask = ra.low_mask;
      s = cuda_status(rc::jit_chunk_launch(m, jr, st));
    } else if (s == RC_OK) {
      s = cuda_status(rc::launch_expand_route(dm, m.host.n_stmts, m.host.n_threads, m.has_deep_loops, ra, res, st));
    }
    for (size_t k = wv.k0; k < wv.k1 && s == RC_OK; ++k) {
      const Chunk& c = chunks[k];
      rc::WorkspacePlan p = pc;
      p.n_keys = c.n;
      p.n_tiles = (c.n + rc::kSortTile - 1) / rc::kSortTile;
      p.scan_warps = scan_warps_for(c.n);
      const uint32_t hi = m.host.cell_shift + std::max<uint32_t>(1u, rc::bit_length(c.span - 1));
      rc::plan_sort(m.host.sort_lo < hi ? m.host.sort_lo : hi, hi, opts ? opts->digit_bits : 0, &p.sort);
      // clear the digit histograms, the look-back words this chunk uses and the counters
      const size_t lb_used = (size_t)p.n_tiles * ((size_t)1 << rc::plan_max_bits(p.sort)) * 8;
      if (p.lookback_off + lb_used > pc.tilectr_off) s = RC_E_INVALID;   // cannot happen: sized for the widest digit
      if (s == RC_OK) s = cuda_status(cudaMemsetAsync(region + p.hist_off, 0, p.lookback_off - p.hist_off + lb_used, st));
      if (s == RC_OK) s = cuda_status(cudaMemsetAsync(region + p.tilectr_off, 0, p.zero_hi - p.tilectr_off, st));
      // a fresh record per chunk; the first chunk of a wave keeps the route
      // pass's error bits, which the report checks in every record
      if (k > wv.k0 && s == RC_OK) s = cuda_status(rc::launch_init_result(res, st));
      int sorted = 0;
      if (s == RC_OK)
        s = enqueue_sort(p, region, keys0 + c.base, keys1 + c.base, spin, opts ? opts->test_flags : 0u, st, &sorted,
                         nullptr, true);
      if (s == RC_OK && c.n > 0) {
        rc::ScanArgs sa = scan_args(m, p, region, sorted);
        sa.keys = (sorted ? keys1 : keys0) + c.base;
        s = cuda_status(rc::launch_scan(sa, st));
        if (s == RC_OK) s = cuda_status(rc::launch_witness(sa, st));
      }
      if (s == RC_OK)
        s = cuda_status(cudaMemcpyAsync(t->host + 1 + k, res, sizeof(rc::DevResult), cudaMemcpyDeviceToHost, st));
    }
  }
  if (s == RC_OK) s = cuda_status(cudaEventRecord(t->done, st));
  if (s != RC_OK) {
    ticket_put(t);
    return s;
  }
  *out = t;
  return RC_OK;
}

// Merge of a chunked ticket's records into one result.
void decode_chunked(const rc_ticket_s* t, rc_result* out) {
  const rc::Model& m = t->models[0]->m;
  decode_result(t->host[0], m, out, 0, m.host.thread_bits, m.host.phase_bits, m.host.thread_shift,
                    rc::bit_length((uint64_t)m.host.n_wphases - 1));
  if (out->status != RC_OK) return;
  const uint64_t instances = out->instances;
  out->racy_cells = 0;
  out->verdict = 0;
  bool have_witness = false;
  for (size_t k = 0; k + 1 < t->n; ++k) {
    rc_result part;
    // cell_base = -chunk start: the scan's cells are relative to the chunk
    decode_result(t->host[1 + k], m, &part, (uint64_t)0 - t->chunk_lo[k], m.host.thread_bits, m.host.phase_bits,
                  m.host.thread_shift, rc::bit_length((uint64_t)m.host.n_wphases - 1));
    if (t->host[1 + k].err & rc::kErrChunkOverflow) part.status = RC_E_NOMEM;
    if (part.status != RC_OK) {
      std::memset(out, 0, sizeof(*out));
      out->status = part.status;
      out->instances = instances;
      return;
    }
    out->racy_cells += part.racy_cells;
    if (part.verdict && !have_witness) {
      const uint64_t racy = out->racy_cells;
      *out = part;
      out->racy_cells = racy;
      have_witness = true;
    }
  }
  out->instances = instances;
  out->verdict = out->racy_cells > 0;
}

// ---------------------------------------------------------------------------
// batched check (batch.cu holds the kernels)
// ---------------------------------------------------------------------------
struct BatchPack {
  size_t i0 = 0, i1 = 0;               // models [i0, i1)
  uint32_t tb = 0, bb = 0, pb = 0, cell_bits = 0;
  uint32_t kb = 1;                     // kind field bits (2 if some model has atomics)
  bool loop_free = true;               // every model of the pack is loop-free
  bool sy = false;                     // some model has warp or grid barriers
  bool mg = false;                     // its models have more than one grid interval (per-block witness groups)
  const uint32_t* grid_of = nullptr;   // phase-order scan with warp / grid barriers: its model's interval table
  uint64_t total_cells = 0, n_keys = 0, n_units = 0;
  rc::WorkspacePlan p;                 // sort / scan sections (offsets into the shared pack region)
};

struct BatchLayout {
  std::vector<BatchPack> packs;
  size_t res_off = 0, packres_off = 0, table_off = 0, cellbase_off = 0, synctab_off = 0, queue_off = 0;
  size_t upload_bytes = 0;             // table, cell bases, interval tables; staged through pinned memory
  size_t total = 0;
};

uint32_t chunks_of(const rc::Model& m) {
  return (uint32_t)((m.host.n_threads + rc::kExpandThreadsHost - 1) / rc::kExpandThreadsHost);
}

rc_status plan_batch(rc_model* const* models, size_t n, const rc_check_opts* opts, BatchLayout* L) {
  L->packs.clear();
  BatchPack cur;
  bool open = false;
  for (size_t i = 0; i < n; ++i) {
    const rc::Model& m = models[i]->m;
    const rc::DevModel& h = m.host;
    if (open) {
      const uint32_t tb = std::max(cur.tb, h.thread_bits), bb = std::max(cur.bb, h.block_bits);
      const uint32_t pb = std::max(cur.pb, h.phase_bits);
      const uint32_t kb = std::max(cur.kb, h.thread_shift);
      const uint64_t cells = cur.total_cells + m.total_cells;
      const uint32_t cb = rc::bit_length(cells);
      // a model with atomics or with warp / grid barriers joins only a pack
      // scanned with phase tables, and a pack holding one takes only models
      // that fit them
      const bool sy = cur.sy || m.sync_scopes;
      const bool table_ok = (kb == 1 && !sy) || pb <= (uint32_t)rc::kScanTablePhaseBits;
      // models with several grid intervals share a pack only with each other, and
      // its per-(model, block, fine interval) witness records stay bounded
      const bool mg_ok = cur.mg == m.multi_grid &&
                         (!cur.mg || ((uint64_t)(i + 1 - cur.i0) << (bb + pb)) <= (1ull << rc::kWitnessBlockGroupBits));
      if (cells >= cur.total_cells && table_ok && mg_ok && kb + tb + bb + pb + cb <= (uint32_t)rc::kKeyBits) {
        cur.tb = tb; cur.bb = bb; cur.pb = pb; cur.kb = kb; cur.total_cells = cells; cur.cell_bits = cb;
        cur.loop_free = cur.loop_free && m.loop_free;
        cur.sy = sy;
        cur.n_keys += m.key_slots;
        cur.n_units += chunks_of(m);
        cur.i1 = i + 1;
        continue;
      }
      L->packs.push_back(cur);
    }
    cur = BatchPack();
    cur.i0 = i;
    cur.i1 = i + 1;
    cur.tb = h.thread_bits; cur.bb = h.block_bits; cur.pb = h.phase_bits; cur.kb = h.thread_shift;
    cur.loop_free = m.loop_free;
    cur.sy = m.sync_scopes;
    cur.mg = m.multi_grid;
    // (a model scanned in phase order with warp or grid barriers holds its pack alone)
    cur.grid_of = m.sec_gridof ? reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(m.dev_program) +
                                                                   m.sec_gridof)
                               : nullptr;
    cur.total_cells = m.total_cells;
    cur.cell_bits = rc::bit_length(m.total_cells);
    cur.n_keys = m.key_slots;
    cur.n_units = chunks_of(m);
    open = true;
  }
  if (open) L->packs.push_back(cur);
  // per-model records and tables, then one pack region sized for the largest pack
  size_t off = 0;
  L->res_off = off;
  off = align256(off + n * sizeof(rc::DevResult));
  L->packres_off = off;
  off = align256(off + sizeof(rc::DevResult));
  L->table_off = off;
  off = align256(off + n * sizeof(rc::BatchModel));
  L->cellbase_off = off;
  off = align256(off + n * 8);
  L->synctab_off = off;
  off = align256(off + n * 24);
  L->upload_bytes = L->synctab_off + n * 24 - L->table_off;
  L->queue_off = off;
  off = align256(off + 8);
  const size_t region = off;
  size_t need = region;
  for (BatchPack& k : L->packs) {
    rc::WorkspacePlan& p = k.p;
    std::memset(&p, 0, sizeof(p));
    p.n_keys = k.n_keys;
    const uint32_t ps = k.kb + k.tb + k.bb;
    const uint32_t lo = k.pb <= rc::kScanTablePhaseBits ? ps + k.pb : ps;   // cell-only sort with phase tables
    plan_sort(lo, ps + k.pb + k.cell_bits, opts ? opts->digit_bits : 0, &p.sort);
    p.n_tiles = (k.n_keys + rc::kSortTile - 1) / rc::kSortTile;
    p.scan_warps = scan_warps_for(k.n_keys);
    size_t o = region;
    p.result_off = L->packres_off;
    p.keys_off[0] = o;
    o = align256(o + k.n_keys * 8);
    p.keys_off[1] = o;
    o = align256(o + k.n_keys * 8);
    if (rc::bucket_path_allowed(k.pb, opts) && rc::plan_buckets(k.n_keys, k.n_keys, k.cell_bits, o, &p.bucket)) {
      p.zero_lo = p.bucket.zero_lo;
      p.zero_hi = p.bucket.zero_hi;
      o = p.bucket.end;
      p.scan_warps = scan_warps_for(k.n_keys);
      p.scanctr_off = p.bucket.scan_ctr;
      p.long_cap = rc::scan_long_capacity(k.n_keys, p.scan_warps);
      p.long_off = o;
      o = align256(o + (size_t)p.long_cap * 8);
      p.group_off = o;
      o = align256(o + (k.i1 - k.i0) * ((size_t)1 << (k.pb + (k.mg ? k.bb : 0u))) * rc::kWitnessGroupWords *
                           sizeof(unsigned int));
      p.total = o;
      need = std::max(need, o);
      continue;
    }
    p.zero_lo = o;
    p.hist_off = o;
    o = align256(o + (size_t)16 * rc::kMaxRadix * 8);
    p.lookback_off = o;
    o = align256(o + (size_t)p.n_tiles * ((size_t)1 << rc::plan_max_bits(p.sort)) * 8);
    p.tilectr_off = o;
    o = align256(o + 16 * sizeof(unsigned int));
    p.scanctr_off = o;
    o = align256(o + 8);
    p.zero_hi = o;
    p.digoff_off = o;
    o = align256(o + (size_t)16 * rc::kMaxRadix * 8);
    p.cursor_off = o;
    o = align256(o + (size_t)rc::kMaxRadix * 8);
    p.long_cap = rc::scan_long_capacity(k.n_keys, p.scan_warps);
    p.long_off = o;
    o = align256(o + (size_t)p.long_cap * 8);
    p.group_off = o;
    o = align256(o + (k.i1 - k.i0) * ((size_t)1 << (k.pb + (k.mg ? k.bb : 0u))) * rc::kWitnessGroupWords *
                         sizeof(unsigned int));
    p.total = o;
    need = std::max(need, o);
  }
  L->total = need;
  return RC_OK;
}

// Model tables of a batch (pack-relative key, cell and unit bases) into
// `upload` (L.upload_bytes), and the per-model decoding data.
void fill_batch_tables(rc_model* const* models, const BatchLayout& L, void* upload, std::vector<uint64_t>* cell_base,
                       std::vector<uint32_t>* field_bits) {
  const size_t n = L.packs.empty() ? 0 : L.packs.back().i1;
  auto* table = static_cast<rc::BatchModel*>(upload);
  auto* cbase = reinterpret_cast<uint64_t*>(static_cast<uint8_t*>(upload) + (L.cellbase_off - L.table_off));
  auto* stabs = reinterpret_cast<uint64_t*>(static_cast<uint8_t*>(upload) + (L.synctab_off - L.table_off));
  cell_base->assign(n, 0);
  field_bits->assign(n, 0);
  for (const BatchPack& k : L.packs) {
    uint64_t key_base = 0, cb = 0, unit_base = 0;
    for (size_t i = k.i0; i < k.i1; ++i) {
      const rc::Model& m = models[i]->m;
      const rc::DevModel& h = m.host;
      rc::BatchModel& b = table[i];
      b.dm = reinterpret_cast<const rc::DevModel*>(m.dev_program);
      b.key_base = key_base;
      b.cell_base = cb;
      b.unit_base = unit_base;
      b.n_threads = h.n_threads;
      b.n_stmts = h.n_stmts;
      b.n_chunks = chunks_of(m);
      b.cell_shift = h.cell_shift;
      b.phase_shift = h.phase_shift;
      b.block_shift = h.block_shift;
      b.phase_bits = h.phase_bits;
      b.block_bits = h.block_bits;
      b.thread_bits = h.thread_bits;
      b.thread_shift = h.thread_shift;
      cbase[i] = cb;
      // interval tables (a model without warp or grid barriers: block interval
      // = phase, one grid interval, one warp interval)
      for (int q = 0; q < 3; ++q) stabs[3 * i + q] = h.sync_tab[q];
      (*cell_base)[i] = cb;
      (*field_bits)[i] = k.tb | (k.pb << 8) | (k.kb << 16);
      key_base += m.key_slots;
      cb += m.total_cells;
      unit_base += b.n_chunks;
    }
  }
}

// Device work of a batch: upload of the tables, then every pack's pipeline.
// The per-model result records stay in the workspace (L.res_off).
rc_status enqueue_batch_device(const BatchLayout& L, size_t n, const rc_check_opts* opts, uint8_t* ws,
                               const void* upload, cudaStream_t st) {
  auto* res = reinterpret_cast<rc::DevResult*>(ws + L.res_off);
  auto* pres = reinterpret_cast<rc::DevResult*>(ws + L.packres_off);
  const auto* dtable = reinterpret_cast<const rc::BatchModel*>(ws + L.table_off);
  const auto* dcbase = reinterpret_cast<const uint64_t*>(ws + L.cellbase_off);
  const auto* dstabs = reinterpret_cast<const uint64_t*>(ws + L.synctab_off);
  auto* queue = reinterpret_cast<unsigned long long*>(ws + L.queue_off);
  const uint64_t spin = (opts && opts->spin_limit) ? opts->spin_limit : (1ull << 20);
  rc_status s = cuda_status(cudaMemcpyAsync(ws + L.table_off, upload, L.upload_bytes, cudaMemcpyHostToDevice, st));
  if (s == RC_OK) s = cuda_status(rc::launch_init_result(res, st, (uint32_t)n));
  for (const BatchPack& k : L.packs) {
    if (s != RC_OK) break;
    const rc::WorkspacePlan& p = k.p;
    const uint32_t nm = (uint32_t)(k.i1 - k.i0);
    s = cuda_status(rc::launch_init_result(pres, st));
    if (s == RC_OK) s = cuda_status(cudaMemsetAsync(ws + p.zero_lo, 0, p.zero_hi - p.zero_lo, st));
    if (s == RC_OK) s = cuda_status(cudaMemsetAsync(queue, 0, 8, st));
    if (s != RC_OK) break;
    rc::BatchArgs ba;
    ba.models = dtable + k.i0;
    ba.n_models = nm;
    ba.n_units = k.n_units;
    ba.queue = queue;
    ba.keys = reinterpret_cast<uint64_t*>(ws + p.keys_off[0]);
    ba.res = res + k.i0;
    ba.thread_shift = k.kb;
    ba.phase_shift = k.kb + k.tb + k.bb;
    ba.block_shift = k.kb + k.tb;
    ba.cell_shift = ba.phase_shift + k.pb;
    s = cuda_status(rc::launch_batch_expand(ba, k.loop_free, st));
    if (s != RC_OK) break;
    int sorted = 0;
    if (!p.bucket.on) {
      s = enqueue_sort(p, ws, reinterpret_cast<uint64_t*>(ws + p.keys_off[0]),
                       reinterpret_cast<uint64_t*>(ws + p.keys_off[1]), spin, opts ? opts->test_flags : 0u, st,
                       &sorted, nullptr, true);
      if (s != RC_OK) break;
    }
    rc::ScanArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.keys = reinterpret_cast<const uint64_t*>(ws + p.keys_off[sorted]);
    sa.n = k.n_keys;
    sa.cell_shift = ba.cell_shift;
    sa.phase_shift = ba.phase_shift;
    sa.block_shift = ba.block_shift;
    sa.thread_shift = k.kb;
    sa.phase_bits = k.pb;
    sa.block_bits = k.bb;
    sa.thread_bits = k.tb;
    sa.n_warps = p.scan_warps;
    if (opts && (opts->test_flags & RC_TEST_FEW_SCAN_WARPS) && sa.n_warps > 3) sa.n_warps = 3;
    sa.res = res + k.i0;
    sa.err = &pres->err;
    sa.groups = reinterpret_cast<unsigned int*>(ws + p.group_off);
    sa.long_list = reinterpret_cast<unsigned long long*>(ws + p.long_off);
    sa.long_count = reinterpret_cast<unsigned long long*>(ws + p.scanctr_off);
    sa.long_cap = p.long_cap;
    sa.cell_base = dcbase + k.i0;
    sa.n_models = nm;
    sa.phase_table = k.pb <= rc::kScanTablePhaseBits ? 1u : 0u;
    sa.sync_tabs = k.sy ? dstabs + 3 * k.i0 : nullptr;
    sa.wit_block_bits = k.mg ? k.bb : 0u;
    sa.grid_of = k.grid_of;
    if (p.bucket.on) {
      const uint64_t* fin = nullptr;
      s = enqueue_bucketed(p, ws, reinterpret_cast<uint64_t*>(ws + p.keys_off[0]),
                           reinterpret_cast<uint64_t*>(ws + p.keys_off[1]), sa, st, &fin);
      sa.keys = fin;
    } else {
      s = cuda_status(rc::launch_scan(sa, st));
    }
    if (s == RC_OK) s = cuda_status(rc::launch_witness(sa, st));
    if (s == RC_OK) s = cuda_status(rc::launch_batch_errors(pres, res + k.i0, nm, st));
  }
  return s;
}

rc_status check_batch_layout(const BatchLayout& L, uint8_t* ws, size_t ws_bytes) {
  if (!ws || ws_bytes < L.total) return RC_E_NOMEM;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return RC_E_INVALID;
  return RC_OK;
}

rc_status enqueue_batch(rc_model* const* models, size_t n, const rc_check_opts* opts, uint8_t* ws,
                        size_t ws_bytes, cudaStream_t st, rc_ticket_s* t) {
  BatchLayout L;
  rc_status s = plan_batch(models, n, opts, &L);
  if (s == RC_OK) s = check_batch_layout(L, ws, ws_bytes);
  if (s != RC_OK || n == 0) return s;
  if (t->upload_cap < L.upload_bytes) {
    if (t->upload) cudaFreeHost(t->upload);
    t->upload = nullptr;
    t->upload_cap = 0;
    if (cudaMallocHost(&t->upload, L.upload_bytes) != cudaSuccess) return RC_E_NOMEM;
    t->upload_cap = L.upload_bytes;
  }
  fill_batch_tables(models, L, t->upload, &t->cell_base, &t->field_bits);
  s = enqueue_batch_device(L, n, opts, ws, t->upload, st);
  if (s == RC_OK)
    s = cuda_status(cudaMemcpyAsync(t->host, ws + L.res_off, n * sizeof(rc::DevResult), cudaMemcpyDeviceToHost,
                                    st));
  return s;
}

// ---------------------------------------------------------------------------
// CUDA-graph replay of a batch (RC_OPT_GRAPH): the device work of one batch
// signature (models, options, workspace) is captured once and relaunched as
// one graph; the tables it uploads live in the cache entry.
// ---------------------------------------------------------------------------
struct GraphEntry {
  std::vector<const void*> models;
  uint32_t digit_bits = 0, test_flags = 0;
  uint64_t spin = 0;
  uint8_t* ws = nullptr;
  size_t ws_bytes = 0;
  int device = -1;
  BatchLayout L;
  void* upload = nullptr;
  std::vector<uint64_t> cell_base;
  std::vector<uint32_t> field_bits;
  cudaGraphExec_t exec = nullptr;
};
std::mutex g_graph_mu;
std::vector<GraphEntry*> g_graphs;
constexpr size_t kMaxGraphs = 16;

void graph_entry_free(GraphEntry* e) {
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->upload) cudaFreeHost(e->upload);
  delete e;
}

void graph_cache_clear() {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (GraphEntry* e : g_graphs) graph_entry_free(e);
  g_graphs.clear();
}

cudaStream_t capture_stream(int device) {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  std::lock_guard<std::mutex> lk(mu);
  if (device < 0 || device >= 64) return nullptr;
  if (!streams[device] && cudaStreamCreateWithFlags(&streams[device], cudaStreamNonBlocking) != cudaSuccess)
    return nullptr;
  return streams[device];
}

rc_status enqueue_batch_graph(rc_model* const* models, size_t n, const rc_check_opts* opts, uint8_t* ws,
                              size_t ws_bytes, cudaStream_t st, rc_ticket_s* t) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return RC_E_CUDA;
  const uint32_t db = opts ? opts->digit_bits : 0, tf = opts ? opts->test_flags : 0;
  const uint64_t spin = opts ? opts->spin_limit : 0;
  std::lock_guard<std::mutex> lk(g_graph_mu);
  GraphEntry* hit = nullptr;
  for (GraphEntry* e : g_graphs) {
    if (e->device == dev && e->ws == ws && e->ws_bytes == ws_bytes && e->digit_bits == db && e->test_flags == tf &&
        e->spin == spin && e->models.size() == n &&
        std::equal(e->models.begin(), e->models.end(), models,
                   [](const void* a, rc_model* b) { return a == static_cast<const void*>(b); })) {
      hit = e;
      break;
    }
  }
  if (!hit) {
    auto* e = new (std::nothrow) GraphEntry();
    if (!e) return RC_E_NOMEM;
    e->models.assign(models, models + n);
    e->digit_bits = db;
    e->test_flags = tf;
    e->spin = spin;
    e->ws = ws;
    e->ws_bytes = ws_bytes;
    e->device = dev;
    rc_status s = plan_batch(models, n, opts, &e->L);
    if (s == RC_OK) s = check_batch_layout(e->L, ws, ws_bytes);
    if (s == RC_OK && cudaMallocHost(&e->upload, std::max<size_t>(e->L.upload_bytes, 256)) != cudaSuccess)
      s = RC_E_NOMEM;
    if (s != RC_OK) {
      graph_entry_free(e);
      return s;
    }
    fill_batch_tables(models, e->L, e->upload, &e->cell_base, &e->field_bits);
    cudaStream_t cs = capture_stream(dev);
    cudaGraph_t g = nullptr;
    if (!cs || cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      graph_entry_free(e);
      return RC_E_CUDA;
    }
    s = enqueue_batch_device(e->L, n, opts, ws, e->upload, cs);
    const cudaError_t ce = cudaStreamEndCapture(cs, &g);
    if (s == RC_OK && ce != cudaSuccess) s = RC_E_CUDA;
    if (s == RC_OK && cudaGraphInstantiate(&e->exec, g, 0) != cudaSuccess) s = RC_E_CUDA;
    if (g) cudaGraphDestroy(g);
    if (s != RC_OK) {
      graph_entry_free(e);
      return s;
    }
    if (g_graphs.size() >= kMaxGraphs) {
      graph_entry_free(g_graphs.front());
      g_graphs.erase(g_graphs.begin());
    }
    g_graphs.push_back(e);
    hit = e;
  }
  t->cell_base = hit->cell_base;
  t->field_bits = hit->field_bits;
  if (n == 0) return RC_OK;
  rc_status s = cuda_status(cudaGraphLaunch(hit->exec, st));
  if (s == RC_OK)
    s = cuda_status(cudaMemcpyAsync(t->host, ws + hit->L.res_off, n * sizeof(rc::DevResult),
                                    cudaMemcpyDeviceToHost, st));
  return s;
}

// ---------------------------------------------------------------------------
// autotuner: path (sort / hash) and radix digit width per shape class
// ---------------------------------------------------------------------------
struct TuneKey {
  uint32_t batch, n_log2, keys_log2, sort_bits;
  bool operator<(const TuneKey& o) const {
    if (batch != o.batch) return batch < o.batch;
    if (n_log2 != o.n_log2) return n_log2 < o.n_log2;
    if (keys_log2 != o.keys_log2) return keys_log2 < o.keys_log2;
    return sort_bits < o.sort_bits;
  }
};
struct TuneChoice {
  uint32_t path, digit_bits;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tuned;

TuneKey tune_key(rc_model* const* models, size_t n) {
  TuneKey k{};
  uint64_t keys = 0, cells = 0;
  uint32_t pb = 0;
  for (size_t i = 0; i < n; ++i) {
    keys += models[i]->m.key_slots;
    cells += models[i]->m.total_cells;
    pb = std::max(pb, models[i]->m.host.phase_bits);
  }
  k.batch = n > 1 ? 1u : 0u;
  k.n_log2 = rc::bit_length(n);
  k.keys_log2 = rc::bit_length(keys);
  k.sort_bits = rc::bit_length(cells) + (pb <= rc::kScanTablePhaseBits ? 0u : pb);
  return k;
}

// AUTO resolved: the tuned choice of the shape class, else the sort path.
rc_check_opts resolve_opts(rc_model* const* models, size_t n, const rc_check_opts* opts) {
  rc_check_opts o{};
  if (opts) o = *opts;
  if (o.path != RC_PATH_AUTO) return o;
  o.path = RC_PATH_SORT;
  for (size_t i = 0; i < n; ++i)   // warp / grid barriers, or a model the hash path cannot take: sort path
    if (models[i] && (models[i]->m.sync_scopes || !rc::hash_path_fits(models[i]->m))) return o;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(tune_key(models, n));
  if (it != g_tuned.end()) {
    o.path = it->second.path;
    if (o.digit_bits == 0) o.digit_bits = it->second.digit_bits;
  }
  return o;
}

}  // namespace

extern "C" {

const char* rc_status_str(rc_status s) {
  switch (s) {
    case RC_OK: return "ok";
    case RC_E_INVALID: return "invalid descriptor or argument";
    case RC_E_KEY_OVERFLOW: return "packed key exceeds 63 bits";
    case RC_E_OOB: return "index or phase out of bounds";
    case RC_E_NOMEM: return "workspace too small or allocation failed";
    case RC_E_TIMEOUT: return "bounded device wait expired";
    case RC_E_CUDA: return "CUDA runtime error";
    case RC_E_NOT_READY: return "not ready";
    case RC_E_UNSUPPORTED: return "model outside this build's limits";
  }
  return "unknown status";
}

void rc_get_limits(rc_limits* out) {
  if (!out) return;
  out->max_loops = rc::kMaxLoops;
  out->max_terms = rc::kMaxTerms;
  out->max_stmts = rc::kMaxStmts;
  out->max_accesses = rc::kMaxAccesses;
  out->max_phase_bits = rc::kMaxPhaseBits;
  out->key_bits = rc::kKeyBits;
}

rc_status rc_model_create(const rc_model_desc* desc, rc_model** out) {
  if (!out) return RC_E_INVALID;
  *out = nullptr;
  rc_model* mm = new (std::nothrow) rc_model();
  if (!mm) return RC_E_NOMEM;
  rc::Model& m = mm->m;
  std::vector<int32_t> general;
  rc_status s = rc::lower_model(desc, &m, &general);
  if (s != RC_OK) {
    delete mm;
    return s;
  }
  const uint64_t T = m.host.n_threads;
  const uint64_t n_units_general = (uint64_t)general.size() * T;
  const size_t prog = m.program.size();
  const size_t total = prog + (size_t)n_units_general * 8;
  if (cudaMalloc(&m.dev_program, total) != cudaSuccess) {
    delete mm;
    return RC_E_NOMEM;
  }
  m.dev_bytes = total;
  // relocate the section offsets to device addresses
  uint8_t* base = static_cast<uint8_t*>(m.dev_program);
  rc::DevModel& h = m.host;
  h.arrays = reinterpret_cast<const rc::DevArray*>(base + reinterpret_cast<uintptr_t>(h.arrays));
  h.stmts = reinterpret_cast<const rc::DevStmt*>(base + reinterpret_cast<uintptr_t>(h.stmts));
  h.accs = reinterpret_cast<const rc::DevAccess*>(base + reinterpret_cast<uintptr_t>(h.accs));
  h.rows = reinterpret_cast<const rc::Row*>(base + reinterpret_cast<uintptr_t>(h.rows));
  h.lin = reinterpret_cast<const rc::LinTerm*>(base + reinterpret_cast<uintptr_t>(h.lin));
  h.terms = reinterpret_cast<const rc::Term*>(base + reinterpret_cast<uintptr_t>(h.terms));
  h.unit_offset = reinterpret_cast<const uint64_t*>(base + reinterpret_cast<uintptr_t>(h.unit_offset));
  h.tables = reinterpret_cast<const uint64_t*>(base + reinterpret_cast<uintptr_t>(h.tables));
  h.tdata = reinterpret_cast<const int64_t*>(base + reinterpret_cast<uintptr_t>(h.tdata));
  std::memcpy(m.program.data(), &h, sizeof(h));
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(m.dev_program);
    delete mm;
    return RC_E_CUDA;
  }
  cudaError_t e = cudaMemcpyAsync(m.dev_program, m.program.data(), prog, cudaMemcpyHostToDevice, st);
  uint64_t general_slots = 0;
  if (e == cudaSuccess && n_units_general > 0) {
    // count the keys of each (statement, thread) unit, then scan them into offsets
    uint64_t* offs = reinterpret_cast<uint64_t*>(base + prog);
    void* tmp = nullptr;
    const size_t tmp_bytes = rc::scan_u64_temp_bytes(n_units_general) + 256;
    e = cudaMalloc(&tmp, tmp_bytes);
    if (e == cudaSuccess) {
      uint64_t* total_dev = reinterpret_cast<uint64_t*>(static_cast<uint8_t*>(tmp) + tmp_bytes - 256);
      e = rc::launch_count(reinterpret_cast<const rc::DevModel*>(m.dev_program),
                           (uint64_t)m.host.n_stmts * T, offs, st);
      if (e == cudaSuccess)
        e = rc::scan_u64_exclusive(offs, offs, n_units_general, h.dense_slots, static_cast<uint64_t*>(tmp),
                                   total_dev, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&general_slots, total_dev, 8, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      cudaFree(tmp);
    }
  }
  if (e == cudaSuccess) {
    h.general_slots = general_slots;
    std::memcpy(m.program.data(), &h, sizeof(h));
    e = cudaMemcpyAsync(m.dev_program, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaStreamDestroy(st);
  if (e != cudaSuccess) {
    cudaFree(m.dev_program);
    delete mm;
    return RC_E_CUDA;
  }
  m.key_slots = h.dense_slots + h.general_slots;
  // large models get a generated expansion kernel; failure keeps the interpreted one
  rc::jit_expand_build(&m);
  *out = mm;
  return RC_OK;
}

void rc_model_destroy(rc_model* m) {
  if (!m) return;
  graph_cache_clear();   // captured batches may hold this model's program
  if (m->m.dev_program) cudaFree(m->m.dev_program);
  delete m;
}

rc_status rc_model_layout(const rc_model* mm, rc_layout* out) {
  if (!mm || !out) return RC_E_INVALID;
  const rc::Model& m = mm->m;
  std::memset(out, 0, sizeof(*out));
  out->kind_shift = m.host.kind_shift;
  out->thread_shift = m.host.thread_shift;
  out->block_shift = m.host.block_shift;
  out->phase_shift = m.host.phase_shift;
  out->cell_shift = m.host.cell_shift;
  out->thread_bits = m.host.thread_bits;
  out->block_bits = m.host.block_bits;
  out->phase_bits = m.host.phase_bits;
  out->cell_bits = m.host.cell_bits;
  out->sort_lo = m.host.sort_lo;
  out->sort_hi = m.host.sort_hi;
  out->key_slots = m.key_slots;
  out->total_cells = m.total_cells;
  out->n_arrays = (uint32_t)m.array_base.size();
  out->n_threads_per_block = m.host.bs;
  out->n_blocks = m.host.n_blocks;
  out->program_bytes = m.dev_bytes;
  out->expand_jit = (m.jit_fn || m.jit_chunk_fn) ? 1u : 0u;
  out->wide = m.wide ? 1u : 0u;
  for (size_t a = 0; a < m.array_base.size() && a < 64; ++a) {
    out->array_base[a] = m.array_base[a];
    out->array_cells[a] = m.array_cells[a];
  }
  return RC_OK;
}

rc_status rc_kernel_source(const rc_model_desc* desc, char* buf, size_t cap, size_t* len) {
  if (!desc || !len || (cap && !buf)) return RC_E_INVALID;
  rc::Model m;
  std::vector<int32_t> general;
  const rc_status st = rc::lower_model(desc, &m, &general);
  if (st != RC_OK) return st;
  const std::string src = m.wide ? rc::jit_chunk_source(m) : rc::jit_expand_source(m);
  *len = src.size();
  if (cap) {
    const size_t n = src.size() < cap - 1 ? src.size() : cap - 1;
    std::memcpy(buf, src.data(), n);
    buf[n] = 0;
  }
  return RC_OK;
}

// A hash-partitioned check (rc_check_opts.part_count > 1) runs on the sort
// path of a single, unchunked check.
static rc_status partition_status(const rc::Model& m, const rc_check_opts& o) {
  if (o.part_count <= 1) return RC_OK;
  if ((o.part_count & (o.part_count - 1)) != 0 || o.part_index >= o.part_count) return RC_E_INVALID;
  if (o.part_count > (1u << 16)) return RC_E_INVALID;
  if (o.path == RC_PATH_HASH || use_chunked(m, &o)) return RC_E_UNSUPPORTED;
  return RC_OK;
}

rc_status rc_workspace_size(const rc_model* m, const rc_check_opts* opts, size_t* bytes) {
  if (!m || !bytes) return RC_E_INVALID;
  rc_model* mm = const_cast<rc_model*>(m);
  const rc_check_opts o = resolve_opts(&mm, 1, opts);
  if (o.path == RC_PATH_HASH && !rc::hash_path_fits(m->m)) return RC_E_UNSUPPORTED;
  {
    const rc_status ps = partition_status(m->m, o);
    if (ps != RC_OK) return ps;
  }
  if (use_chunked(m->m, &o)) {
    ChunkGeometry g;
    const rc_status s = chunk_geometry(m->m, &o, &g);
    if (s != RC_OK) return s;
    *bytes = chunked_workspace_size(m->m, &o);
    return RC_OK;
  }
  rc::WorkspacePlan p;
  rc::plan_workspace(m->m, &o, &p);
  *bytes = p.total;
  return RC_OK;
}

rc_status rc_check(rc_model* m, const rc_check_opts* opts, void* workspace, size_t ws_bytes, void* stream,
                   rc_ticket* ticket) {
  if (!m || !ticket) return RC_E_INVALID;
  *ticket = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc_check_opts o = resolve_opts(&m, 1, opts);
  if (o.path == RC_PATH_HASH && !rc::hash_path_fits(m->m)) return RC_E_UNSUPPORTED;
  {
    const rc_status ps = partition_status(m->m, o);
    if (ps != RC_OK) return ps;
  }
  // warp / grid barriers take the sort path unless the hash path is asked for
  if (m->m.sync_scopes && (!opts || opts->path != RC_PATH_HASH)) o.path = RC_PATH_SORT;
  if (use_chunked(m->m, &o)) {
    if (!opts || opts->path != RC_PATH_HASH) o.path = RC_PATH_SORT;   // chunks take the sort path
    return enqueue_chunked(m, &o, static_cast<uint8_t*>(workspace), ws_bytes, st, ticket);
  }
  rc_ticket_s* t = ticket_get(1);
  if (!t) return RC_E_NOMEM;
  const bool want_times = opts && (opts->flags & RC_OPT_STAGE_TIMES);
  if (opts && opts->path == RC_PATH_AUTO) {
    // a tuned choice that needs more workspace than given falls back to the sort path
    size_t need = 0;
    rc::WorkspacePlan p;
    rc::plan_workspace(m->m, &o, &p);
    need = p.total;
    if (need > ws_bytes) {
      o = *opts;
      o.path = RC_PATH_SORT;
    }
  }
  rc_status s = enqueue_check(m, &o, static_cast<uint8_t*>(workspace), ws_bytes, st, t->host,
                              want_times ? t : nullptr);
  if (s == RC_OK) s = cuda_status(cudaEventRecord(t->done, st));
  if (s != RC_OK) {
    ticket_put(t);
    return s;
  }
  t->models[0] = m;
  *ticket = t;
  return RC_OK;
}

// The batch takes the batched pipeline (batch.cu) unless the hash path is
// requested; the hash path checks the models one after another.
bool batch_is_sequential(const rc_check_opts* opts) { return opts && opts->path == RC_PATH_HASH; }

rc_status rc_batch_workspace_size(rc_model* const* models, size_t n, const rc_check_opts* opts_in, size_t* bytes) {
  if (!bytes || (n && !models)) return RC_E_INVALID;
  for (size_t i = 0; i < n; ++i) {
    if (!models[i]) return RC_E_INVALID;
    if (models[i]->m.wide) return RC_E_KEY_OVERFLOW;   // wide models are checked alone, in chunks
  }
  const rc_check_opts ro = resolve_opts(models, n, opts_in);
  const rc_check_opts* opts = &ro;
  if (ro.path == RC_PATH_HASH)
    for (size_t i = 0; i < n; ++i)
      if (!rc::hash_path_fits(models[i]->m)) return RC_E_UNSUPPORTED;
  if (batch_is_sequential(opts)) {
    size_t mx = 0;
    for (size_t i = 0; i < n; ++i) {
      size_t b;
      rc_workspace_size(models[i], opts, &b);
      if (b > mx) mx = b;
    }
    *bytes = mx;
    return RC_OK;
  }
  BatchLayout L;
  rc_status s = plan_batch(models, n, opts, &L);
  if (s != RC_OK) return s;
  *bytes = L.total;
  return RC_OK;
}

rc_status rc_check_batch(rc_model* const* models, size_t n, const rc_check_opts* opts_in, void* workspace,
                         size_t ws_bytes, void* stream, rc_ticket* ticket) {
  if (!ticket || (n && !models)) return RC_E_INVALID;
  *ticket = nullptr;
  for (size_t i = 0; i < n; ++i) {
    if (!models[i]) return RC_E_INVALID;
    if (models[i]->m.wide) return RC_E_KEY_OVERFLOW;   // wide models are checked alone, in chunks
  }
  rc_check_opts ro = resolve_opts(models, n, opts_in);
  if (ro.path == RC_PATH_HASH)
    for (size_t i = 0; i < n; ++i)
      if (!rc::hash_path_fits(models[i]->m)) return RC_E_UNSUPPORTED;
  if (opts_in && opts_in->path == RC_PATH_AUTO) {
    size_t need = 0;
    rc_batch_workspace_size(models, n, &ro, &need);
    if (need > ws_bytes) {
      ro = *opts_in;
      ro.path = RC_PATH_SORT;
    }
  }
  const rc_check_opts* opts = &ro;
  rc_ticket_s* t = ticket_get(n);
  if (!t) return RC_E_NOMEM;
  for (size_t i = 0; i < n; ++i) t->models[i] = models[i];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc_status s = RC_OK;
  if (batch_is_sequential(opts)) {
    for (size_t i = 0; i < n && s == RC_OK; ++i)
      s = enqueue_check(models[i], opts, static_cast<uint8_t*>(workspace), ws_bytes, st, t->host + i);
  } else if (opts && (opts->flags & RC_OPT_GRAPH)) {
    s = enqueue_batch_graph(models, n, opts, static_cast<uint8_t*>(workspace), ws_bytes, st, t);
  } else {
    s = enqueue_batch(models, n, opts, static_cast<uint8_t*>(workspace), ws_bytes, st, t);
  }
  if (s == RC_OK) s = cuda_status(cudaEventRecord(t->done, st));
  if (s != RC_OK) {
    ticket_put(t);
    return s;
  }
  *ticket = t;
  return RC_OK;
}

rc_status rc_tune(rc_model* const* models, size_t n, const rc_check_opts* opts, void* workspace, size_t ws_bytes,
                  void* stream, rc_check_opts* best) {
  if (!best || !models || n == 0) return RC_E_INVALID;
  for (size_t i = 0; i < n; ++i) {
    if (!models[i]) return RC_E_INVALID;
    if (models[i]->m.wide) return RC_E_KEY_OVERFLOW;   // a wide model has one path: chunked sort
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  rc_check_opts base{};
  if (opts) base = *opts;
  base.flags &= ~(uint32_t)(RC_OPT_STAGE_TIMES | RC_OPT_GRAPH);
  base.early_exit = 0;
  const TuneKey key = tune_key(models, n);
  const uint32_t sort_bits = n == 1 ? models[0]->m.host.sort_hi - models[0]->m.host.sort_lo : key.sort_bits;
  // candidates: the bucket path (where it applies), every distinct number of
  // LSD sort passes for digits of 6..11 bits, and the hash path
  std::vector<rc_check_opts> cands;
  std::vector<uint32_t> passes;
  if (!(base.flags & RC_OPT_LSD)) {
    rc_check_opts o = base;
    o.path = RC_PATH_SORT;
    o.digit_bits = 0;
    cands.push_back(o);
  }
  for (uint32_t d = 6; d <= 11; ++d) {
    rc::SortPlan sp;
    rc::plan_sort(0, sort_bits, d, &sp);
    if (std::find(passes.begin(), passes.end(), sp.n_pass) != passes.end()) continue;
    passes.push_back(sp.n_pass);
    rc_check_opts o = base;
    o.path = RC_PATH_SORT;
    o.digit_bits = d;
    cands.push_back(o);
  }
  bool hash_ok = !opts || opts->part_count <= 1;   // (a hash-partitioned check takes the sort path)
  for (size_t i = 0; i < n; ++i) hash_ok = hash_ok && rc::hash_path_fits(models[i]->m);
  if (hash_ok) {
    rc_check_opts o = base;
    o.path = RC_PATH_HASH;
    o.digit_bits = 0;
    cands.push_back(o);
  }
  rc_ticket_s* t = ticket_get(n);
  if (!t) return RC_E_NOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    ticket_put(t);
    return RC_E_CUDA;
  }
  float best_ms = 0.f;
  bool any = false;
  rc_check_opts bo = cands[0];
  rc_status fail = RC_OK;
  for (const rc_check_opts& c : cands) {
    size_t need = 0;
    if (n == 1) rc_workspace_size(models[0], &c, &need);
    else rc_batch_workspace_size(models, n, &c, &need);
    if (need > ws_bytes) continue;
    float ms_min = 0.f;
    bool ok = true;
    for (int r = 0; r < 3 && ok; ++r) {   // run 0 warms up
      rc_status s = cuda_status(cudaEventRecord(e0, st));
      if (s == RC_OK) {
        if (n == 1) {
          s = enqueue_check(models[0], &c, ws, ws_bytes, st, t->host);
        } else if (batch_is_sequential(&c)) {
          for (size_t i = 0; i < n && s == RC_OK; ++i) s = enqueue_check(models[i], &c, ws, ws_bytes, st, t->host + i);
        } else {
          s = enqueue_batch(models, n, &c, ws, ws_bytes, st, t);
        }
      }
      if (s == RC_OK) s = cuda_status(cudaEventRecord(e1, st));
      if (s == RC_OK) s = cuda_status(cudaEventSynchronize(e1));
      if (s != RC_OK) {
        ok = false;
        if (s == RC_E_CUDA) fail = s;
        break;
      }
      for (size_t i = 0; i < n; ++i)
        if (t->host[i].err) ok = false;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r == 1 || (r > 1 && ms < ms_min)) ms_min = ms;
    }
    if (ok && (!any || ms_min < best_ms)) {
      best_ms = ms_min;
      bo = c;
      any = true;
    }
    if (fail != RC_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ticket_put(t);
  if (fail != RC_OK) return fail;
  if (!any) return RC_E_NOMEM;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = TuneChoice{bo.path, bo.digit_bits};
  }
  *best = bo;
  if (opts) best->flags = opts->flags;
  return RC_OK;
}

rc_status rc_report(rc_ticket t, rc_result* out, int wait) {
  if (!t || !out) return RC_E_INVALID;
  if (wait) {
    if (cudaEventSynchronize(t->done) != cudaSuccess) {
      ticket_put(t);
      return RC_E_CUDA;
    }
  } else {
    cudaError_t q = cudaEventQuery(t->done);
    if (q == cudaErrorNotReady) return RC_E_NOT_READY;
    if (q != cudaSuccess) {
      ticket_put(t);
      return RC_E_CUDA;
    }
  }
  if (t->chunked) {
    decode_chunked(t, out);
    ticket_put(t);
    return RC_OK;
  }
  for (size_t i = 0; i < t->n; ++i) {
    const rc::Model& m = t->models[i]->m;
    if (t->cell_base.empty())
      decode_result(t->host[i], m, &out[i], 0, m.host.thread_bits, m.host.phase_bits, m.host.thread_shift,
                    rc::bit_length((uint64_t)m.host.n_wphases - 1));
    else
      decode_result(t->host[i], m, &out[i], t->cell_base[i], t->field_bits[i] & 0xFFu, (t->field_bits[i] >> 8) & 0xFFu,
                    t->field_bits[i] >> 16, rc::bit_length((uint64_t)m.host.n_wphases - 1));
  }
  ticket_put(t);
  return RC_OK;
}

rc_status rc_ticket_stage_times(rc_ticket t, rc_stage_times* out) {
  if (!t || !out || !t->timed || !t->timer.ok) return RC_E_INVALID;
  if (cudaEventSynchronize(t->done) != cudaSuccess) return RC_E_CUDA;
  std::memset(out, 0, sizeof(*out));
  auto ms = [&](int a, int b) {
    float v = 0.f;
    cudaEventElapsedTime(&v, t->timer.ev[a], t->timer.ev[b]);
    return v;
  };
  out->expand_ms = ms(t->i_start, t->i_expand);
  out->histogram_ms = ms(t->i_expand, t->i_hist);
  out->n_sort_passes = t->n_pass;
  int prev = t->i_hist;
  for (uint32_t k = 0; k < t->n_pass && k < 16; ++k) {
    out->sort_ms[k] = ms(t->i_pass_from[k], t->i_pass_to[k]);
    prev = t->i_pass_to[k];
  }
  if (t->i_hist2_from >= 0) out->histogram2_ms = ms(t->i_hist2_from, t->i_hist2_to);
  out->bucketed = t->bucketed ? 1u : 0u;
  out->histogram_fused = t->hist_fused ? 1u : 0u;
  out->scan_ms = ms(prev, t->i_scan);
  out->witness_ms = ms(t->i_scan, t->i_wit);
  out->total_ms = ms(t->i_start, t->i_wit);
  out->n_keys = t->n_keys;
  return RC_OK;
}

rc_status rc_expand_keys(rc_model* mm, void* workspace, size_t ws_bytes, uint64_t* keys_dev, uint64_t* count_dev,
                         void* stream) {
  if (!mm || !keys_dev || !count_dev) return RC_E_INVALID;
  const rc::Model& m = mm->m;
  if (m.wide) return RC_E_KEY_OVERFLOW;   // its cells do not fit one key
  rc::WorkspacePlan p;
  rc::plan_workspace(m, nullptr, &p);
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  if (!ws || ws_bytes < p.total) return RC_E_NOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto* res = reinterpret_cast<rc::DevResult*>(ws + p.result_off);
  rc_status s = cuda_status(rc::launch_init_result(res, st));
  if (s != RC_OK) return s;
  if (m.jit_fn)
    s = cuda_status(rc::jit_expand_launch(m, keys_dev, res, st));
  else
    s = cuda_status(rc::launch_expand(reinterpret_cast<const rc::DevModel*>(m.dev_program),
                                      m.host.n_stmts, m.host.n_threads, m.has_deep_loops, keys_dev, res, st));
  if (s != RC_OK) return s;
  return cuda_status(cudaMemcpyAsync(count_dev, &res->instances, 8, cudaMemcpyDeviceToDevice, st));
}

rc_status rc_sort_workspace_size(uint64_t n, uint32_t digit_bits, size_t* bytes) {
  if (!bytes) return RC_E_INVALID;
  rc::SortPlan sp;
  rc::plan_sort(0, 64, digit_bits, &sp);
  const uint64_t n_tiles = (n + rc::kSortTile - 1) / rc::kSortTile;
  size_t off = align256(sizeof(rc::DevResult));
  off = align256(off + (size_t)16 * rc::kMaxRadix * 8);                                    // histograms
  off = align256(off + (size_t)n_tiles * ((size_t)1 << rc::kMaxRadixBits) * 8);             // look-back
  off = align256(off + 16 * sizeof(unsigned int));                                         // tile counters
  off = align256(off + (size_t)16 * rc::kMaxRadix * 8);                                    // digit offsets
  off = align256(off + n * 8);                             // ping-pong buffer
  *bytes = off;
  return RC_OK;
}

}  // extern "C"

namespace rc {
bool sort_stall_requested() {
  const char* v = std::getenv("RC_TEST_SORT_STALL");
  return v && v[0] == '1';
}

// The byte ranges of a sort's scratch that must start at zero: the digit
// counts of its passes, the look-back words of its tiles at the widest radix of
// its passes, and its tile counters.
void sort_clear_ranges(const SortPlan& sp, uint64_t n, size_t hist_off, size_t lookback_off, size_t tilectr_off,
                       size_t (*ranges)[2]) {
  uint32_t rb = 0;
  for (uint32_t k = 0; k < sp.n_pass; ++k) rb = std::max(rb, radix_bits_for(sp.bits[k]));
  const uint64_t n_tiles = (n + kSortTile - 1) / kSortTile;
  ranges[0][0] = hist_off;
  ranges[0][1] = (size_t)sp.n_pass * kMaxRadix * 8;
  ranges[1][0] = lookback_off;
  ranges[1][1] = (size_t)n_tiles * ((size_t)1 << rb) * 8;
  ranges[2][0] = tilectr_off;
  ranges[2][1] = 16 * sizeof(unsigned int);
}
}  // namespace rc

extern "C" {

rc_status rc_sort_keys(const uint64_t* keys_in, uint64_t* keys_out, uint64_t n, uint32_t lo_bit, uint32_t hi_bit,
                       uint32_t digit_bits, void* workspace, size_t ws_bytes, void* stream) {
  if (hi_bit > 64 || lo_bit > hi_bit || (n && (!keys_in || !keys_out || keys_in == keys_out))) return RC_E_INVALID;
  size_t need;
  rc_sort_workspace_size(n, digit_bits, &need);
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  if (!ws || ws_bytes < need) return RC_E_NOMEM;
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return RC_E_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc::WorkspacePlan p;
  std::memset(&p, 0, sizeof(p));
  rc::plan_sort(lo_bit, hi_bit, digit_bits, &p.sort);
  p.n_keys = n;
  p.n_tiles = (n + rc::kSortTile - 1) / rc::kSortTile;
  size_t off = 0;
  p.result_off = off;
  off = align256(off + sizeof(rc::DevResult));
  p.zero_lo = off;
  p.hist_off = off;
  off = align256(off + (size_t)16 * rc::kMaxRadix * 8);
  p.lookback_off = off;
  off = align256(off + (size_t)p.n_tiles * ((size_t)1 << rc::kMaxRadixBits) * 8);
  p.tilectr_off = off;
  off = align256(off + 16 * sizeof(unsigned int));
  p.zero_hi = off;
  p.digoff_off = off;
  off = align256(off + (size_t)16 * rc::kMaxRadix * 8);
  const size_t pong = off;
  rc_status s = cuda_status(rc::launch_init_result(reinterpret_cast<rc::DevResult*>(ws + p.result_off), st));
  if (s != RC_OK || n == 0) return s;
  size_t clear[3][2];
  rc::sort_clear_ranges(p.sort, n, p.hist_off, p.lookback_off, p.tilectr_off, clear);
  for (int r = 0; r < 3 && s == RC_OK; ++r) s = cuda_status(cudaMemsetAsync(ws + clear[r][0], 0, clear[r][1], st));
  if (s != RC_OK) return s;
  // Stage the input in the output buffer and ping-pong with the workspace
  // buffer; with an odd number of passes the result lands in the workspace
  // buffer and is copied back.
  s = cuda_status(cudaMemcpyAsync(keys_out, keys_in, n * 8, cudaMemcpyDeviceToDevice, st));
  if (s != RC_OK) return s;
  int sorted = 0;
  const bool stall = rc::sort_stall_requested();
  s = enqueue_sort(p, ws, keys_out, reinterpret_cast<uint64_t*>(ws + pong), stall ? 4096ull : (1ull << 20),
                   stall ? (uint32_t)RC_TEST_STALL_LOOKBACK : 0u, st, &sorted);
  if (s != RC_OK) return s;
  if (sorted == 1) s = cuda_status(cudaMemcpyAsync(keys_out, ws + pong, n * 8, cudaMemcpyDeviceToDevice, st));
  return s;
}

rc_status rc_sort_status(const void* workspace, void* stream) {
  const void* rec = workspace;
  if (!rec) {
    rc_status s = rc::sort_static_record(&rec);
    if (s != RC_OK) return s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return RC_E_CUDA;
  unsigned int err = 0;
  if (cudaMemcpy(&err, static_cast<const uint8_t*>(rec) + offsetof(rc::DevResult, err), sizeof(err),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return RC_E_CUDA;
  if (err & rc::kErrLookbackTimeout) return RC_E_TIMEOUT;
  if (err & rc::kErrSortRange) return RC_E_INVALID;
  return RC_OK;
}

}  // extern "C"
