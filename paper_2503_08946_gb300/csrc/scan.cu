// K3: scan of the sorted keys -> racy-cell count and first racy cell;
// K4: witness (smallest racing pair) inside that cell.
//
// The paper's RaW / WaW / WaR relations (appendix listing of the dependence
// test) pair instances on the same cell with at least one write.  After the
// sort, the instances of a cell are contiguous and grouped by phase.  A cell is
// racy iff it has a write and (two blocks meet in it, or inside one block some
// phase group holds two threads and a write) -- the cell-level form of the
// pair rule in include/rc.h.  With atomic accesses (models with a 2-bit kind
// field, phase-table scan only) "a write" widens to "a conflict": a write, or
// an atomic and a plain read.
//
// K3a (scan_cells_kernel): each warp owns a contiguous range of segments of
//      32 x kScanRun keys, staged through shared memory with coalesced loads.
//      Every lane folds its run of kScanRun keys in one pass: the keys that
//      continue the cell open before the run into a prefix part, the cells
//      that begin in the run into a fold state (closed ones are counted at
//      once).  The cell open at a run's end is then completed by merging the
//      prefix parts of the following lanes (usually one), and a cell open at
//      the segment end is carried into the next segment.  A cell carried over
//      more than kCarryMaxSegs segments, or still open at the end of the
//      warp's range, is handed to K3b by its first position.
// K3b (scan_long_kernel): one block per handed-over cell folds it from its
//      first key, 2048 keys at a time, as an ordered reduction of CellPieces
//      (rc_internal.h).
// Counts are added and the first racy cell is the minimum start, so the
// result does not depend on which lane or block folds a cell.  In a batch
// (several models' keys sorted together, each model in its own cell range),
// a racy cell is charged to the model whose range holds it.
// K3c: one warp per result finds the end of its first racy cell.
// K4:  four grid-wide reductions over that one segment: the cell summary
//      (blocks, write blocks), per-phase groups of its lowest block, the
//      smallest instance that has a partner (x), and x's smallest partner (y).
//      The smallest participating instance always lies in the lowest block of a
//      racy cell, so only that block's phase groups are needed.
#include <cuda_runtime.h>

#include "fold.cuh"
#include "kernels.h"

namespace rc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// 32-way galloping search by one full warp: first position >= start whose key
// is not in `cell` (keys[start] is in it).
__device__ uint64_t warp_cell_end(const uint64_t* keys, uint64_t n, uint32_t cs, uint64_t start, uint64_t cell) {
  const int lane = threadIdx.x & 31;
  uint64_t lo = start, stride = 1;
  while (true) {
    const uint64_t q = lo + (uint64_t)(lane + 1) * stride;
    const bool f = q >= n || (keys[q] >> cs) != cell;
    const unsigned F = __ballot_sync(FULL, f);
    if (F) {
      lo += (uint64_t)(__ffs(F) - 1) * stride;
      break;
    }
    lo += 32 * stride;
    stride *= 32;
  }
  // keys[lo] is in the cell and keys[lo + stride] is not (or is past the end)
  while (stride > 1) {
    const uint64_t s2 = (stride + 31) / 32;
    const uint64_t q = lo + (uint64_t)(lane + 1) * s2;
    const bool f = q >= lo + stride || q >= n || (keys[q] >> cs) != cell;
    const unsigned F = __ballot_sync(FULL, f);
    lo += (uint64_t)(__ffs(F) - 1) * s2;
    stride = s2;
  }
  return lo + 1;
}

// Fold state of a run of keys of one cell (a whole cell, or a part of one).
// Keys are compared through masks: same cell iff ((k ^ k') & cell_mask) == 0,
// same phase group iff ((k ^ k') & group_mask) == 0.  bt = the (block, thread)
// bits of a key.  The first phase group is kept apart until it closes, so that
// a part that continues another can be merged into it (merge below).
struct Fold {
  uint64_t fk;       // first key
  uint64_t gk;       // a key of the current (last) phase group
  uint64_t start;    // position of the first key
  unsigned bt0;      // bt of the first key
  unsigned gbt0;     // bt of the current group's first key
  unsigned f;        // flags below
};
constexpr unsigned kFW = 1u;        // some write
constexpr unsigned kFMB = 2u;       // two blocks
constexpr unsigned kFGM = 4u;       // current group: two (block, thread)
constexpr unsigned kFGW = 8u;       // current group: a write
constexpr unsigned kFIn = 16u;      // a closed group other than the first is racy
constexpr unsigned kFFO = 32u;      // the first group is still the current group
constexpr unsigned kFFM = 64u;      // closed first group: two (block, thread)
constexpr unsigned kFFW = 128u;     // closed first group: a write

struct FoldCtx {
  uint64_t group_mask;   // bits of (cell, phase)
  unsigned btm;          // mask of the (block, thread) bits after >> 1
  uint32_t tb;           // thread bits
};

__device__ __forceinline__ unsigned key_bt(const FoldCtx& c, uint64_t k) { return (unsigned)(k >> 1) & c.btm; }

__device__ __forceinline__ void fold_start(Fold& s, uint64_t k, uint64_t pos, unsigned bt) {
  s.fk = s.gk = k;
  s.start = pos;
  s.bt0 = s.gbt0 = bt;
  s.f = kFFO | ((k & 1ull) ? (kFW | kFGW) : 0u);
}
// close the current group, whose flags are gm / gw
__device__ __forceinline__ unsigned close_group(unsigned f, bool gm, bool gw) {
  if (f & kFFO) return (f & ~kFFO) | (gm ? kFFM : 0u) | (gw ? kFFW : 0u);
  return (gm && gw) ? (f | kFIn) : f;
}
// add a key of the same cell
__device__ __forceinline__ void fold_add(const FoldCtx& c, Fold& s, uint64_t k, unsigned bt) {
  unsigned f = s.f;
  if (((bt ^ s.bt0) >> c.tb) != 0u) f |= kFMB;
  if (((k ^ s.gk) & c.group_mask) != 0ull) {
    f = close_group(f, (f & kFGM) != 0u, (f & kFGW) != 0u) & ~(kFGM | kFGW);
    s.gk = k;
    s.gbt0 = bt;
  } else if (bt != s.gbt0) {
    f |= kFGM;
  }
  if (k & 1ull) f |= kFW | kFGW;
  s.f = f;
}
__device__ __forceinline__ bool fold_racy(const Fold& s) {
  const unsigned f = s.f;
  if (!(f & kFW)) return false;
  if (f & (kFMB | kFIn)) return true;
  if ((f & (kFGM | kFGW)) == (kFGM | kFGW)) return true;
  return !(f & kFFO) && (f & (kFFM | kFFW)) == (kFFM | kFFW);
}
// s followed by p, a part that continues s's cell
__device__ __forceinline__ void fold_merge(const FoldCtx& c, Fold& s, const Fold& p) {
  unsigned f = s.f | (p.f & kFW);
  if ((p.f & kFMB) || ((p.bt0 ^ s.bt0) >> c.tb) != 0u) f |= kFMB;
  const bool p_single = (p.f & kFFO) != 0u;       // p holds one group
  const bool pfm = p_single ? (p.f & kFGM) != 0u : (p.f & kFFM) != 0u;
  const bool pfw = p_single ? (p.f & kFGW) != 0u : (p.f & kFFW) != 0u;
  if (((p.fk ^ s.gk) & c.group_mask) == 0ull) {
    // p's first group continues s's current group
    const bool gm = (f & kFGM) || pfm || p.bt0 != s.gbt0;
    const bool gw = (f & kFGW) || pfw;
    if (p_single) {
      f = (f & ~(kFGM | kFGW)) | (gm ? kFGM : 0u) | (gw ? kFGW : 0u);
    } else {
      f = close_group(f, gm, gw) | (p.f & kFIn);
      f = (f & ~(kFGM | kFGW)) | (p.f & (kFGM | kFGW));
      s.gk = p.gk;
      s.gbt0 = p.gbt0;
    }
  } else {
    f = close_group(f, (f & kFGM) != 0u, (f & kFGW) != 0u);
    if (!p_single && pfm && pfw) f |= kFIn;
    f = (f & ~(kFGM | kFGW)) | (p.f & (kFGM | kFGW)) | (p.f & kFIn);
    s.gk = p.gk;
    s.gbt0 = p.gbt0;
  }
  s.f = f;
}
__device__ __forceinline__ Fold fold_shfl(const Fold& s, int src) {
  Fold r;
  r.fk = __shfl_sync(FULL, s.fk, src);
  r.gk = __shfl_sync(FULL, s.gk, src);
  r.start = __shfl_sync(FULL, s.start, src);
  r.bt0 = __shfl_sync(FULL, s.bt0, src);
  r.gbt0 = __shfl_sync(FULL, s.gbt0, src);
  r.f = __shfl_sync(FULL, s.f, src);
  return r;
}

__device__ __forceinline__ void hand_over(const ScanArgs& a, uint64_t start) {
  const unsigned long long i = atomicAdd(a.long_count, 1ull);
  if (i < a.long_cap) a.long_list[i] = start;
  else atomicOr(a.err, (unsigned int)kErrScanLongFull);
}

constexpr int kScanWarps = 4;                 // warps per block of scan_cells_kernel
constexpr int kRunPad = kScanRun + 1;         // padded per-lane stride in shared memory
constexpr int kSegKeys = 32 * kScanRun;       // keys per warp segment
constexpr int kCarryMaxSegs = 8;              // longer carried cells go to scan_long_kernel

__device__ __forceinline__ int seg_slot(int j) { return (j / kScanRun) * kRunPad + (j % kScanRun); }

__global__ void __launch_bounds__(kScanWarps * 32) scan_cells_kernel(ScanArgs a) {
  __shared__ uint64_t sk[kScanWarps][32 * kRunPad];
  FoldCtx c;
  c.group_mask = ~((1ull << a.phase_shift) - 1ull);
  c.btm = (unsigned)((1ull << (a.block_bits + a.thread_bits)) - 1ull);
  c.tb = a.thread_bits;
  const uint64_t cell_mask = ~((1ull << a.cell_shift) - 1ull);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t* my = sk[w];
  const uint64_t n_seg = (a.n + kSegKeys - 1) / kSegKeys;
  const uint64_t gw = (uint64_t)blockIdx.x * kScanWarps + w;
  const uint64_t per = (n_seg + a.n_warps - 1) / a.n_warps;
  const uint64_t seg0 = gw * per, seg1 = min(n_seg, seg0 + per);
  unsigned long long count = 0, minstart = ~0ull;
  auto report = [&](const Fold& x) {
    if (!fold_racy(x)) return;
    if (a.n_models) {
      DevResult* r = result_of(a, x.fk >> a.cell_shift);
      atomicAdd(&r->racy_cells, 1ull);
      atomicMin(&r->min_start, (unsigned long long)x.start);
    } else {
      ++count;
      minstart = min(minstart, (unsigned long long)x.start);
    }
  };
  // key just before the current segment (kSentinel: none before the range)
  uint64_t k_before = kSentinel;
  if (seg0 > 0 && seg0 < seg1) k_before = a.keys[seg0 * kSegKeys - 1];
  bool carry = false;    // warp-uniform: a cell begun in an earlier segment is still open
  int carried = 0;
  Fold cc;
  cc.fk = cc.gk = 0; cc.start = 0; cc.bt0 = cc.gbt0 = 0; cc.f = 0;
  for (uint64_t seg = seg0; seg < seg1; ++seg) {
    const uint64_t S = seg * kSegKeys;
#pragma unroll
    for (int i = 0; i < kSegKeys / 64; ++i) {
      const int j = 2 * (i * 32 + lane);
      const uint64_t pos = S + j;
      uint64_t x = kSentinel, y = kSentinel;
      if (pos + 1 < a.n) {
        const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(a.keys + pos));
        x = v.x;
        y = v.y;
      } else if (pos < a.n) {
        x = a.keys[pos];
      }
      const int o = seg_slot(j);
      my[o] = x;
      my[o + 1] = y;
    }
    __syncwarp();
    // (1) fold the run in one pass, with selects rather than branches so that
    // the lanes of a warp stay converged.  `cur` is the part being folded: first
    // the keys that continue the cell open before the run (the prefix part P),
    // then each cell that begins in the run (closed ones are reported at once;
    // the last one stays open as O).
    const uint64_t s = S + (uint64_t)lane * kScanRun;
    const uint64_t* run = my + lane * kRunPad;
    const uint64_t kp = lane > 0 ? my[(lane - 1) * kRunPad + kScanRun - 1] : k_before;
    Fold P, cur;
    P.fk = P.gk = 0; P.start = 0; P.bt0 = P.gbt0 = 0; P.f = 0;
    cur = P;
    cur.fk = kp;                      // compared against for the prefix
    bool hasP = false, term = false, cur_empty = true, cur_prefix = true;
#pragma unroll 8
    for (int q = 0; q < kScanRun; ++q) {
      const uint64_t k = run[q];
      term |= k == kSentinel;
      const bool valid = !term;
      const unsigned bt = key_bt(c, k);
      const bool same_cell = ((k ^ cur.fk) & cell_mask) == 0ull;
      const bool do_start = !same_cell || cur_empty;
      const bool do_close = valid && !same_cell && !cur_empty;
      if (do_close) {
        if (cur_prefix) {
          P = cur;
          hasP = true;
        } else {
          report(cur);
        }
      }
      // add to cur (same cell)
      unsigned f = cur.f;
      const bool ng = ((k ^ cur.gk) & c.group_mask) != 0ull;
      const bool gm = (f & kFGM) != 0u, gw = (f & kFGW) != 0u;
      const unsigned fc = (f & kFFO) ? ((f & ~kFFO) | (gm ? kFFM : 0u) | (gw ? kFFW : 0u))
                                     : ((gm && gw) ? (f | kFIn) : f);
      f = ng ? (fc & ~(kFGM | kFGW)) : f;
      if (((bt ^ cur.bt0) >> c.tb) != 0u) f |= kFMB;
      if (!ng && bt != cur.gbt0) f |= kFGM;
      const unsigned wf = (k & 1ull) ? (kFW | kFGW) : 0u;
      f |= wf;
      const unsigned fs = kFFO | wf;
      if (valid) {
        cur.f = do_start ? fs : f;
        cur.gk = (do_start || ng) ? k : cur.gk;
        cur.gbt0 = (do_start || ng) ? bt : cur.gbt0;
        cur.fk = do_start ? k : cur.fk;
        cur.bt0 = do_start ? bt : cur.bt0;
        cur.start = do_start ? s + q : cur.start;
        cur_prefix = cur_prefix && same_cell;
        cur_empty = false;
      }
    }
    bool hasO = false;
    Fold O = cur;
    if (!cur_empty) {
      if (cur_prefix) {
        P = cur;
        hasP = true;
      } else {
        hasO = true;
      }
    }
    const bool pfull = hasP && !hasO && !term;   // the prefix fills the whole run
    // (2) the carried cell continues through the leading prefixes
    if (carry) {
      bool open = true;
      for (int src = 0; src < 32 && open; ++src) {
        const bool h = __shfl_sync(FULL, hasP, src);
        const bool full = __shfl_sync(FULL, pfull, src);
        const Fold ps = fold_shfl(P, src);
        if (h) fold_merge(c, cc, ps);
        if (!full) open = false;
      }
      if (!open) {
        if (lane == 0) report(cc);
        carry = false;
      } else if (++carried > kCarryMaxSegs) {
        if (lane == 0) hand_over(a, cc.start);
        carry = false;
      }
    }
    // (3) each lane's last cell continues through the following prefixes
    bool open = hasO;
    bool open_end = false;
    if (open && (term || S + (uint64_t)(lane + 1) * kScanRun >= a.n)) {   // the keys end in this run
      report(O);
      open = false;
    }
    for (int d = 1; __any_sync(FULL, open); ++d) {
      const int src = lane + d < 32 ? lane + d : 31;
      const bool h = __shfl_sync(FULL, hasP, src);
      const bool full = __shfl_sync(FULL, pfull, src);
      const Fold ps = fold_shfl(P, src);
      if (open) {
        if (lane + d >= 32) {
          open = false;
          open_end = true;
        } else {
          if (h) fold_merge(c, O, ps);
          if (!full) {
            report(O);
            open = false;
          }
        }
      }
    }
    // (4) the cell open at the segment end (at most one lane) becomes the carry
    const unsigned OE = __ballot_sync(FULL, open_end);
    if (OE) {
      cc = fold_shfl(O, __ffs(OE) - 1);
      carry = true;
      carried = 0;
    }
    k_before = my[31 * kRunPad + kScanRun - 1];
    __syncwarp();
  }
  // a cell still open at the range end continues past it
  if (carry && lane == 0) hand_over(a, cc.start);
  if (a.n_models == 0) {
    count = __reduce_add_sync(FULL, (unsigned)count);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(FULL, minstart, o);
      minstart = y < minstart ? y : minstart;
    }
    if (lane == 0) {
      if (count) atomicAdd(&a.res->racy_cells, count);
      if (minstart != ~0ull) atomicMin(&a.res->min_start, minstart);
    }
  }
}

// Keys of the scanned buffer: a.n, or fewer when the grouping step counted
// them on the device (the bucket path keeps only guard-true keys of the
// checked cell range, in front).
__device__ __forceinline__ uint64_t scan_key_count(const ScanArgs& a) {
  return a.n_dev ? min(a.n, (uint64_t)*a.n_dev) : a.n;
}

// One key as a CellPiece.
__device__ __forceinline__ CellPiece key_piece(const ScanArgs& a, uint64_t k, uint64_t cell, uint64_t pos) {
  CellPiece c;
  c.cell = cell;
  c.start = pos;
  const unsigned b = (unsigned)(k >> a.block_shift) & ((1u << a.block_bits) - 1u);
  const unsigned t = (unsigned)(k >> a.thread_shift) & ((1u << a.thread_bits) - 1u);
  const unsigned p = (unsigned)(k >> a.phase_shift) & ((1u << a.phase_bits) - 1u);
  const unsigned w = (unsigned)(k & 1ull);
  c.minb = c.maxb = b;
  c.anyW = w;
  c.first_p = c.last_p = p;
  c.single_sub = 1;
  c.inner = 0;
  c.pad = 0;
  c.fs.mint = c.fs.maxt = t;
  c.fs.anyW = w;
  c.fs.pad = 0;
  c.ls = c.fs;
  return c;
}

constexpr int kLongThreads = 256;
constexpr int kLongItems = 8;

// One block per handed-over cell: fold it from its first key.
__global__ void __launch_bounds__(kLongThreads) scan_long_kernel(ScanArgs a) {
  __shared__ CellPiece part[kLongThreads];
  __shared__ int part_empty[kLongThreads];
  const unsigned long long n_long = min(*a.long_count, (unsigned long long)a.long_cap);
  for (unsigned long long i = blockIdx.x; i < n_long; i += gridDim.x) {
    const uint64_t start = a.long_list[i];
    const uint64_t cell = a.keys[start] >> a.cell_shift;
    CellPiece acc{};
    bool acc_empty = true;
    for (uint64_t base = start;; base += (uint64_t)kLongThreads * kLongItems) {
      CellPiece p{};
      bool empty = true, end = false;
      for (int j = 0; j < kLongItems; ++j) {
        const uint64_t pos = base + (uint64_t)threadIdx.x * kLongItems + j;
        if (pos >= a.n) { end = true; break; }
        const uint64_t k = a.keys[pos];
        if (k == kSentinel || (k >> a.cell_shift) != cell) { end = true; break; }
        const CellPiece kp = key_piece(a, k, cell, pos);
        p = empty ? kp : piece_combine(p, kp);
        empty = false;
      }
      part[threadIdx.x] = p;
      part_empty[threadIdx.x] = empty ? 1 : 0;
      const bool any_end = __syncthreads_or(end) != 0;
      for (int width = 1; width < kLongThreads; width <<= 1) {
        if ((threadIdx.x % (2 * width)) == 0 && !part_empty[threadIdx.x + width]) {
          part[threadIdx.x] = part_empty[threadIdx.x] ? part[threadIdx.x + width]
                                                      : piece_combine(part[threadIdx.x], part[threadIdx.x + width]);
          part_empty[threadIdx.x] = 0;
        }
        __syncthreads();
      }
      if (threadIdx.x == 0 && !part_empty[0]) {
        acc = acc_empty ? part[0] : piece_combine(acc, part[0]);
        acc_empty = false;
      }
      __syncthreads();
      if (any_end) break;
    }
    if (threadIdx.x == 0 && !acc_empty && piece_racy(acc)) {
      DevResult* r = result_of(a, cell);
      atomicAdd(&r->racy_cells, 1ull);
      atomicMin(&r->min_start, (unsigned long long)start);
    }
  }
}

// ---------------------------------------------------------------------------
// Phase-order scan of models with warp or grid barriers, or atomics, and more
// than 16 fine intervals: the keys are sorted by (cell, fine interval q), so
// inside a cell the keys of each fine interval, of each block interval
// c = q / n_wp and of each grid interval g(c) are contiguous (all three are
// non-decreasing in q).  Per interval the fold keeps the smallest and largest
// (block, thread) and the kinds present.  A cell is racy iff a fine interval
// holds two (block, thread) and a conflict, a block interval holds two warps
// of one block and a conflict (its smallest and largest (block, thread) lie in
// one block and in different warps; two blocks there are caught by the grid
// test, a block interval lying in one grid interval), or a grid interval
// holds two blocks and a conflict.  Without warp or grid barriers (atomics
// only) every block interval is its fine interval and all lie in one grid
// interval, which is the plain rule.  Conflict: a write, or an atomic and a
// plain read.
// K3s (scan_sorted_sync_kernel): each thread folds, one after another, the
//      cells that begin in its 32 positions; a cell longer than
//      kSyncSeqMax keys is handed to K3t by its first position.
// K3t (scan_sorted_sync_long_kernel): one block per handed-over cell, folded
//      as an ordered reduction of SyncPieces (below).
// ---------------------------------------------------------------------------
struct ISeg {
  unsigned mn, mx;   // smallest and largest (block, thread)
  unsigned f;        // kinds present: bit 0 R, bit 1 W, bit 2 A
};
struct SyncCtx {
  uint32_t cs, ps, ts, tb;
  unsigned pmask, btmask, kmask;
  uint32_t n_wp;
  const uint32_t* grid_of;   // per block interval (null: the 4-bit table, q < 16)
  uint64_t grid_tab;
};
__device__ __forceinline__ SyncCtx sync_ctx(const ScanArgs& a, uint32_t mi) {
  SyncCtx c;
  c.cs = a.cell_shift;
  c.ps = a.phase_shift;
  c.ts = a.thread_shift;
  c.tb = a.thread_bits;
  c.pmask = (1u << a.phase_bits) - 1u;
  c.btmask = (unsigned)((1ull << (a.block_bits + a.thread_bits)) - 1ull);
  c.kmask = (1u << a.thread_shift) - 1u;
  const SyncTabs t = sync_tabs_of(a, mi);
  c.n_wp = t.on ? t.n_wp : 1u;
  c.grid_of = t.on ? a.grid_of : nullptr;
  c.grid_tab = t.on ? t.grid : 0ull;
  return c;
}
// the interval ids of a key at the three levels (fine, block, grid)
__device__ __forceinline__ void sync_ids(const SyncCtx& c, uint64_t k, unsigned id[3]) {
  const unsigned q = (unsigned)(k >> c.ps) & c.pmask;
  const unsigned p = q / c.n_wp;
  id[0] = q;
  id[1] = p;
  id[2] = c.grid_of ? __ldg(c.grid_of + p) : (q < 16u ? (unsigned)(c.grid_tab >> (4 * q)) & 15u : 0u);
}
__device__ __forceinline__ ISeg iseg_of(const SyncCtx& c, uint64_t k) {
  ISeg s;
  s.mn = s.mx = (unsigned)(k >> c.ts) & c.btmask;
  s.f = 1u << ((unsigned)k & c.kmask);
  return s;
}
__device__ __forceinline__ ISeg iseg_join(const ISeg& a, const ISeg& b) {
  ISeg s;
  s.mn = min(a.mn, b.mn);
  s.mx = max(a.mx, b.mx);
  s.f = a.f | b.f;
  return s;
}
__device__ __forceinline__ bool iseg_hot(const SyncCtx& c, int level, const ISeg& s) {
  const bool conf = (s.f & 2u) || ((s.f & 5u) == 5u);
  if (!conf) return false;
  if (level == 0) return s.mn != s.mx;
  const bool one_block = (s.mn >> c.tb) == (s.mx >> c.tb);
  if (level == 2) return !one_block;
  const unsigned tmask = (1u << c.tb) - 1u;
  return one_block && ((s.mn & tmask) >> 5) != ((s.mx & tmask) >> 5);
}

// a contiguous piece of one cell's keys: per level its first and last interval
// (bit L of `one`: the piece lies in one level-L interval), and whether an
// interval closed on both sides inside it is racy
struct SyncPiece {
  uint64_t fk, lk;
  ISeg first[3], last[3];
  unsigned one, racy;
};
__device__ __forceinline__ SyncPiece sync_piece_of(const SyncCtx& c, uint64_t k) {
  SyncPiece p;
  p.fk = p.lk = k;
  const ISeg s = iseg_of(c, k);
#pragma unroll
  for (int L = 0; L < 3; ++L) p.first[L] = p.last[L] = s;
  p.one = 7u;
  p.racy = 0u;
  return p;
}
// a followed by b (both of one cell)
__device__ __forceinline__ SyncPiece sync_piece_merge(const SyncCtx& c, const SyncPiece& a, const SyncPiece& b) {
  SyncPiece r;
  r.fk = a.fk;
  r.lk = b.lk;
  r.one = 0u;
  r.racy = a.racy | b.racy;
  unsigned ia[3], ib[3];
  sync_ids(c, a.lk, ia);
  sync_ids(c, b.fk, ib);
#pragma unroll
  for (int L = 0; L < 3; ++L) {
    const bool ao = (a.one >> L) & 1u, bo = (b.one >> L) & 1u;
    if (ia[L] == ib[L]) {
      const ISeg j = iseg_join(a.last[L], b.first[L]);
      r.first[L] = ao ? j : a.first[L];
      r.last[L] = bo ? j : b.last[L];
      if (ao && bo) r.one |= 1u << L;
      if (!ao && !bo && iseg_hot(c, L, j)) r.racy = 1u;
    } else {
      if (!ao && iseg_hot(c, L, a.last[L])) r.racy = 1u;
      if (!bo && iseg_hot(c, L, b.first[L])) r.racy = 1u;
      r.first[L] = a.first[L];
      r.last[L] = b.last[L];
    }
  }
  return r;
}
__device__ __forceinline__ bool sync_piece_racy(const SyncCtx& c, const SyncPiece& p) {
  bool r = p.racy != 0u;
#pragma unroll
  for (int L = 0; L < 3; ++L) r = r || iseg_hot(c, L, p.first[L]) || iseg_hot(c, L, p.last[L]);
  return r;
}

constexpr int kSyncChunk = 32;                 // positions per thread of K3s
constexpr uint64_t kSyncSeqMax = 8192;         // longer cells go to K3t (at most n / 8192 of them)
static_assert(kSyncSeqMax >= (uint64_t)kCarryMaxSegs * kSegKeys, "the long-cell list is sized for this");

__device__ __forceinline__ void sync_record(const ScanArgs& a, uint64_t cell, uint64_t start) {
  DevResult* r = result_of(a, cell);
  atomicAdd(&r->racy_cells, 1ull);
  atomicMin(&r->min_start, (unsigned long long)start);
}

__global__ void __launch_bounds__(256) scan_sorted_sync_kernel(ScanArgs a) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * kSyncChunk;
  for (uint64_t c0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * kSyncChunk; c0 < a.n; c0 += stride) {
    const uint64_t c1 = min(c0 + (uint64_t)kSyncChunk, a.n);
    uint64_t prev = c0 ? (a.keys[c0 - 1] >> a.cell_shift) : ~0ull;
    for (uint64_t i = c0; i < c1; ++i) {
      const uint64_t k = a.keys[i];
      if (k == kSentinel) break;                 // padding sorts last
      const uint64_t cell = k >> a.cell_shift;
      if (cell == prev) continue;                // not the first key of its cell
      prev = cell;
      const SyncCtx c = sync_ctx(a, model_of(a, cell));
      // one open interval per level; an interval is decided when it closes
      unsigned id[3];
      ISeg cur[3];
      sync_ids(c, k, id);
      cur[0] = cur[1] = cur[2] = iseg_of(c, k);
      bool racy = false;
      uint64_t j = i + 1;
      for (; j < a.n && j - i < kSyncSeqMax; ++j) {
        const uint64_t kj = a.keys[j];
        if ((kj >> a.cell_shift) != cell) break;
        unsigned idj[3];
        sync_ids(c, kj, idj);
        const ISeg sj = iseg_of(c, kj);
#pragma unroll
        for (int L = 0; L < 3; ++L) {
          if (idj[L] != id[L]) {
            racy = racy || iseg_hot(c, L, cur[L]);
            id[L] = idj[L];
            cur[L] = sj;
          } else {
            cur[L] = iseg_join(cur[L], sj);
          }
        }
      }
      if (j < a.n && j - i >= kSyncSeqMax && (a.keys[j] >> a.cell_shift) == cell) {
        hand_over(a, i);
        continue;
      }
#pragma unroll
      for (int L = 0; L < 3; ++L) racy = racy || iseg_hot(c, L, cur[L]);
      if (racy) sync_record(a, cell, i);
    }
  }
}

// One block per handed-over cell: each thread folds kLongItems keys into a
// piece, the block merges the pieces in order.
__global__ void __launch_bounds__(kLongThreads) scan_sorted_sync_long_kernel(ScanArgs a) {
  __shared__ SyncPiece part[kLongThreads];
  __shared__ int part_empty[kLongThreads];
  const unsigned long long n_long = min(*a.long_count, (unsigned long long)a.long_cap);
  for (unsigned long long i = blockIdx.x; i < n_long; i += gridDim.x) {
    const uint64_t start = a.long_list[i];
    const uint64_t cell = a.keys[start] >> a.cell_shift;
    const SyncCtx c = sync_ctx(a, model_of(a, cell));
    SyncPiece acc;
    bool acc_empty = true;
    for (uint64_t base = start;; base += (uint64_t)kLongThreads * kLongItems) {
      SyncPiece p;
      bool empty = true, end = false;
      for (int j = 0; j < kLongItems; ++j) {
        const uint64_t pos = base + (uint64_t)threadIdx.x * kLongItems + j;
        if (pos >= a.n) { end = true; break; }
        const uint64_t k = a.keys[pos];
        if (k == kSentinel || (k >> a.cell_shift) != cell) { end = true; break; }
        const SyncPiece kp = sync_piece_of(c, k);
        p = empty ? kp : sync_piece_merge(c, p, kp);
        empty = false;
      }
      if (!empty) part[threadIdx.x] = p;
      part_empty[threadIdx.x] = empty ? 1 : 0;
      const bool any_end = __syncthreads_or(end) != 0;
      for (int width = 1; width < kLongThreads; width <<= 1) {
        if ((threadIdx.x % (2 * width)) == 0 && !part_empty[threadIdx.x + width]) {
          part[threadIdx.x] = part_empty[threadIdx.x] ? part[threadIdx.x + width]
                                                      : sync_piece_merge(c, part[threadIdx.x], part[threadIdx.x + width]);
          part_empty[threadIdx.x] = 0;
        }
        __syncthreads();
      }
      if (threadIdx.x == 0 && !part_empty[0]) {
        acc = acc_empty ? part[0] : sync_piece_merge(c, acc, part[0]);
        acc_empty = false;
      }
      __syncthreads();
      if (any_end) break;
    }
    if (threadIdx.x == 0 && !acc_empty && sync_piece_racy(c, acc)) sync_record(a, cell, start);
  }
}

// ---------------------------------------------------------------------------
// Phase-table variants: keys sorted by cell only.  With at most
// 2^kScanTablePhaseBits barrier intervals the sort leaves out the phase bits,
// and the phase groups of a cell are tracked in a small table per part
// instead: for each phase, whether it was seen, the (block, thread) of its
// first key, whether two (block, thread) met in it and whether it has a write.
// A cell is racy iff it has a write and (two blocks, or some phase with two
// (block, thread) and a write) -- the same rule as above, order-free inside
// the cell.
// ---------------------------------------------------------------------------
template <bool AT, bool SY>
__device__ __forceinline__ typename FoldOf<SY>::type tfold_shfl(const typename FoldOf<SY>::type& s, int src) {
  typename FoldOf<SY>::type r;
  r.fk = __shfl_sync(FULL, s.fk, src);
  r.start = __shfl_sync(FULL, s.start, src);
  r.bt0 = __shfl_sync(FULL, s.bt0, src);
  r.f = __shfl_sync(FULL, s.f, src);
  r.vmask = __shfl_sync(FULL, s.vmask, src);
  r.gm = __shfl_sync(FULL, s.gm, src);
  r.gw = __shfl_sync(FULL, s.gw, src);
  if (AT) {
    r.ga = __shfl_sync(FULL, s.ga, src);
    r.gr = __shfl_sync(FULL, s.gr, src);
  } else {
    r.ga = r.gr = 0;
  }
  if constexpr (SY) {
    r.gmb = __shfl_sync(FULL, s.gmb, src);
    r.gmw = __shfl_sync(FULL, s.gmw, src);
  }
  return r;
}
// o (table otab) followed by p (table ptab), a part of the same cell; one lane
template <bool AT, bool SY>
__device__ __forceinline__ void tfold_merge(typename FoldOf<SY>::type& o, unsigned* otab,
                                            const typename FoldOf<SY>::type& p, const unsigned* ptab, uint32_t tb) {
  unsigned f = o.f | p.f;
  if (((p.bt0 ^ o.bt0) >> tb) != 0u) f |= kTMB;
  unsigned m = p.vmask;
  while (m) {
    const int ph = __ffs(m) - 1;
    const unsigned bit = 1u << ph;
    m &= m - 1;
    const unsigned pv = ptab[ph];
    if (o.vmask & bit) {
      if ((p.gm & bit) || pv != otab[ph]) o.gm |= bit;
      if constexpr (SY) {
        if (pv != otab[ph]) mark_pair(pv, otab[ph], bit, tb, o.gmb, o.gmw);
      }
    } else {
      otab[ph] = pv;
      o.vmask |= bit;
      o.gm |= p.gm & bit;
    }
  }
  o.gw |= p.gw;
  if (AT) {
    o.ga |= p.ga;
    o.gr |= p.gr;
  }
  if constexpr (SY) {
    o.gmb |= p.gmb;
    o.gmw |= p.gmw;
  }
  o.f = f;
}
// the warp's carried cell (warp-uniform state, table ctab) followed by p of
// lane src (table ptab); all lanes, one phase per lane
template <bool AT, bool SY>
__device__ __forceinline__ void tfold_merge_warp(typename FoldOf<SY>::type& o, unsigned* ctab,
                                                 const typename FoldOf<SY>::type& p, const unsigned* ptab, uint32_t tb) {
  const int lane = threadIdx.x & 31;
  unsigned f = o.f | p.f;
  if (((p.bt0 ^ o.bt0) >> tb) != 0u) f |= kTMB;
  bool g = false;
  unsigned mb = 0, mw = 0;
  if (lane < kTabPhases && (p.vmask >> lane) & 1u) {
    const unsigned pv = ptab[lane];
    if ((o.vmask >> lane) & 1u) {
      g = ((p.gm >> lane) & 1u) || pv != ctab[lane];
      if constexpr (SY) {
        if (pv != ctab[lane]) mark_pair(pv, ctab[lane], 1u, tb, mb, mw);
      }
    } else {
      ctab[lane] = pv;
      g = (p.gm >> lane) & 1u;
    }
  }
  o.gm |= __ballot_sync(FULL, g);
  if constexpr (SY) {
    o.gmb |= __ballot_sync(FULL, mb != 0u) | p.gmb;
    o.gmw |= __ballot_sync(FULL, mw != 0u) | p.gmw;
  }
  o.vmask |= p.vmask;
  o.gw |= p.gw;
  if (AT) {
    o.ga |= p.ga;
    o.gr |= p.gr;
  }
  o.f = f;
  __syncwarp();
}

// AT: the model has atomic accesses (2-bit kind field: R = 0, W = 1, A = 2);
// SY: it has warp or grid barriers (fine intervals, tfold_racy_sync);
// MC: the first racy cell is the smallest by cell value (DevResult.hash_cell),
// for keys grouped by cell but not in cell order (the bucket path), else the
// one at the smallest position (min_start, keys in cell order)
template <bool AT, bool SY, bool MC>
__global__ void __launch_bounds__(kScanWarps * 32, 6) scan_cells_table_kernel(ScanArgs a) {
  const uint64_t n = scan_key_count(a);
  constexpr uint32_t kKindBits = AT ? 2 : 1;
  __shared__ unsigned tabs[kScanWarps][32 * kTabStride];
  __shared__ unsigned ctabs[kScanWarps][kTabPhases];
  const uint32_t ps = a.phase_shift, tb = a.thread_bits;
  const unsigned pm = (1u << a.phase_bits) - 1u;
  const unsigned btm = (unsigned)((1ull << (a.block_bits + a.thread_bits)) - 1ull);
  const uint64_t cell_mask = ~((1ull << a.cell_shift) - 1ull);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned* mytab = tabs[w] + lane * kTabStride;     // [0, 16): prefix part, [16, 32): own cells
  unsigned* ctab = ctabs[w];
  const uint64_t n_seg = (n + kSegKeys - 1) / kSegKeys;
  const uint64_t gw = (uint64_t)blockIdx.x * kScanWarps + w;
  const uint64_t per = (n_seg + a.n_warps - 1) / a.n_warps;
  const uint64_t seg0 = gw * per, seg1 = min(n_seg, seg0 + per);
  unsigned long long count = 0, minstart = ~0ull;
  using TF = typename FoldOf<SY>::type;
  SyncTabs syt;
  if constexpr (SY) syt = sync_tabs_of(a);
  // count a racy cell and keep the first
  auto record = [&](const TF& x, const uint64_t start) {
    const unsigned long long first = MC ? (unsigned long long)(x.fk >> a.cell_shift) : (unsigned long long)start;
    if (a.n_models) {
      DevResult* r = result_of(a, x.fk >> a.cell_shift);
      atomicAdd(&r->racy_cells, 1ull);
      atomicMin(MC ? &r->hash_cell : &r->min_start, first);
    } else {
      ++count;
      minstart = min(minstart, first);
    }
  };
  auto report = [&](const TF& x, const unsigned* xtab, const uint64_t start) {
    if constexpr (SY) {
      if (a.n_models) {
        // a batch: the tables of the cell's model
        const uint32_t mi = model_of(a, x.fk >> a.cell_shift);
        const SyncTabs mt = sync_tabs_of(a, mi);
        if (!tfold_racy_sync<AT>(x, xtab, mt.coarse, mt.grid, tb)) return;
        DevResult* r = a.res + mi;
        atomicAdd(&r->racy_cells, 1ull);
        if (MC) atomicMin(&r->hash_cell, (unsigned long long)(x.fk >> a.cell_shift));
        else atomicMin(&r->min_start, (unsigned long long)start);
        return;
      }
      if (!tfold_racy_sync<AT>(x, xtab, syt.coarse, syt.grid, tb)) return;
    } else {
      (void)xtab;
      if (!tfold_racy<AT>(x)) return;
    }
    record(x, start);
  };
  bool carry = false;
  int carried = 0;
  TF cc;
  tfold_clear(cc);
  for (uint64_t seg = seg0; seg < seg1; ++seg) {
    const uint64_t S = seg * kSegKeys;
    // (1) fold the run (prefix part in table 0, own cells in table 1)
    // each lane reads its own run of kScanRun consecutive keys directly (the
    // lines of a run are shared by its consecutive loads through L1)
    const uint64_t s = S + (uint64_t)lane * kScanRun;
    const uint64_t kp = (s > 0 && s - 1 < n) ? __ldg(a.keys + s - 1) : kSentinel;
    TF P, cur;
    tfold_clear(P);
    cur = P;
    cur.fk = kp;
    bool hasP = false, term = false, cur_empty = true, cur_prefix = true;
    unsigned q0 = 0;   // run position of the current cell's first key
    // first: the run's first key (it starts the current part); check: the run
    // may end past n or hold sentinels (keys are ascending and a sentinel is
    // above every key, so a run whose last key is below it holds none)
    auto fold_key = [&](const uint64_t k, const int q, const bool first, const bool check) {
      if (check) term |= k == kSentinel;
      const bool valid = !check || !term;
      const unsigned bt = (unsigned)(k >> kKindBits) & btm;
      const unsigned ph = (unsigned)(k >> ps) & pm;
      const bool same_cell = ((k ^ cur.fk) & cell_mask) == 0ull;
      const bool do_start = first || !same_cell;
      const bool close = !first && valid && !same_cell;
      if (close && cur_prefix) {
        P = cur;
        hasP = true;
      }
      if constexpr (SY) {
        if (close && !cur_prefix) report(cur, mytab + kTabPhases, s + q0);
      } else {
        // the racy test without a branch; only a racy cell branches
        if (close && !cur_prefix && tfold_racy<AT>(cur)) record(cur, s + q0);
      }
      const bool np = cur_prefix && same_cell;
      unsigned* tab = mytab + (np ? 0 : kTabPhases);
      const unsigned bit = 1u << ph;
      const unsigned old = tab[ph];
      const bool seen = !do_start && (cur.vmask & bit);
      if (valid) {
        if (!seen) tab[ph] = bt;
        const unsigned wb = (unsigned)(k & 1ull) << ph;
        cur.gm = (do_start ? 0u : cur.gm) | ((seen && old != bt) ? bit : 0u);
        if constexpr (SY) {
          cur.gmb = do_start ? 0u : cur.gmb;
          cur.gmw = do_start ? 0u : cur.gmw;
          if (seen && old != bt) mark_pair(old, bt, bit, tb, cur.gmb, cur.gmw);
        }
        cur.vmask = (do_start ? 0u : cur.vmask) | bit;
        cur.gw = (do_start ? 0u : cur.gw) | wb;
        cur.f = do_start ? 0u : (((bt ^ cur.bt0) >> tb) != 0u ? kTMB : cur.f);
        if (AT) {
          const bool at = (k & 2ull) != 0ull, rd = (k & 3ull) == 0ull;
          cur.ga = (do_start ? 0u : cur.ga) | (at ? bit : 0u);
          cur.gr = (do_start ? 0u : cur.gr) | (rd ? bit : 0u);
        }
        cur.fk = do_start ? k : cur.fk;
        cur.bt0 = do_start ? bt : cur.bt0;
        q0 = do_start ? (unsigned)q : q0;
        cur_prefix = np;
        if (first) cur_empty = false;
      }
    };
    // pairs of keys by 16-byte loads (the key array is 16-byte aligned and runs
    // start at even positions; launch_scan checks the alignment)
    const bool full_run = s + kScanRun <= n && __ldg(a.keys + s + kScanRun - 1) != kSentinel;
    if (full_run) {
      const ulonglong2 k0 = __ldg(reinterpret_cast<const ulonglong2*>(a.keys + s));
      fold_key(k0.x, 0, true, false);
      fold_key(k0.y, 1, false, false);
#pragma unroll 3
      for (int q = 2; q < kScanRun; q += 2) {
        const ulonglong2 kk = __ldg(reinterpret_cast<const ulonglong2*>(a.keys + s + q));
        fold_key(kk.x, q, false, false);
        fold_key(kk.y, q + 1, false, false);
      }
    } else {
      fold_key(s < n ? __ldg(a.keys + s) : kSentinel, 0, true, true);
#pragma unroll 1
      for (int q = 1; q < kScanRun; ++q) fold_key(s + q < n ? __ldg(a.keys + s + q) : kSentinel, q, false, true);
    }
    bool hasO = false;
    TF O = cur;
    O.start = s + q0;
    if (!cur_empty) {
      if (cur_prefix) {
        P = cur;
        hasP = true;
      } else {
        hasO = true;
      }
    }
    const bool pfull = hasP && !hasO && !term;
    __syncwarp();
    // (2) the carried cell continues through the leading prefixes
    if (carry) {
      bool open = true;
      for (int src = 0; src < 32 && open; ++src) {
        const bool h = __shfl_sync(FULL, hasP, src);
        const bool full = __shfl_sync(FULL, pfull, src);
        const TF pp = tfold_shfl<AT, SY>(P, src);
        if (h) tfold_merge_warp<AT, SY>(cc, ctab, pp, tabs[w] + src * kTabStride, tb);
        if (!full) open = false;
      }
      if (!open) {
        if (lane == 0) report(cc, ctab, cc.start);
        carry = false;
      } else if (++carried > kCarryMaxSegs) {
        if (lane == 0) hand_over(a, cc.start);
        carry = false;
      }
    }
    // (3) each lane's last cell continues through the following prefixes
    bool open = hasO;
    bool open_end = false;
    if (open && (term || S + (uint64_t)(lane + 1) * kScanRun >= n)) {
      report(O, mytab + kTabPhases, O.start);
      open = false;
    }
    for (int d = 1; __any_sync(FULL, open); ++d) {
      const int src = lane + d < 32 ? lane + d : 31;
      const bool h = __shfl_sync(FULL, hasP, src);
      const bool full = __shfl_sync(FULL, pfull, src);
      const TF pp = tfold_shfl<AT, SY>(P, src);
      if (open) {
        if (lane + d >= 32) {
          open = false;
          open_end = true;
        } else {
          if (h) tfold_merge<AT, SY>(O, mytab + kTabPhases, pp, tabs[w] + src * kTabStride, tb);
          if (!full) {
            report(O, mytab + kTabPhases, O.start);
            open = false;
          }
        }
      }
    }
    // (4) the cell open at the segment end (at most one lane) becomes the carry
    const unsigned OE = __ballot_sync(FULL, open_end);
    if (OE) {
      const int src = __ffs(OE) - 1;
      cc = tfold_shfl<AT, SY>(O, src);
      if (lane < kTabPhases) ctab[lane] = tabs[w][src * kTabStride + kTabPhases + lane];
      carry = true;
      carried = 0;
    }
    __syncwarp();
  }
  if (carry && lane == 0) hand_over(a, cc.start);
  if (a.n_models == 0) {
    count = __reduce_add_sync(FULL, (unsigned)count);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(FULL, minstart, o);
      minstart = y < minstart ? y : minstart;
    }
    if (lane == 0) {
      if (count) atomicAdd(&a.res->racy_cells, count);
      if (minstart != ~0ull) atomicMin(MC ? &a.res->hash_cell : &a.res->min_start, minstart);
    }
  }
}

// One block per handed-over cell, order-free: per-phase min / max (block,
// thread) and write flags in shared memory.
__global__ void __launch_bounds__(kLongThreads) scan_long_table_kernel(ScanArgs a) {
  const uint64_t n = scan_key_count(a);
  __shared__ unsigned mn[kTabPhases], mx[kTabPhases];
  __shared__ unsigned s_gw, s_ga, s_gr, s_minb, s_maxb, s_w;
  const uint32_t kb = a.thread_shift;   // kind field bits (R = 0, W = 1, A = 2)
  const uint64_t kmask = (1ull << kb) - 1ull;
  const unsigned pm = (1u << a.phase_bits) - 1u;
  const unsigned btm = (unsigned)((1ull << (a.block_bits + a.thread_bits)) - 1ull);
  const unsigned long long n_long = min(*a.long_count, (unsigned long long)a.long_cap);
  for (unsigned long long i = blockIdx.x; i < n_long; i += gridDim.x) {
    const uint64_t start = a.long_list[i];
    const uint64_t cell = a.keys[start] >> a.cell_shift;
    const SyncTabs syt = sync_tabs_of(a, model_of(a, cell));
    if (threadIdx.x < kTabPhases) {
      mn[threadIdx.x] = 0xffffffffu;
      mx[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) {
      s_gw = s_ga = s_gr = 0;
      s_minb = 0xffffffffu;
      s_maxb = 0;
      s_w = 0;
    }
    __syncthreads();
    for (uint64_t base = start;; base += kLongThreads) {
      const uint64_t pos = base + threadIdx.x;
      bool end = pos >= n;
      if (!end) {
        const uint64_t k = a.keys[pos];
        end = k == kSentinel || (k >> a.cell_shift) != cell;
        if (!end) {
          const unsigned bt = (unsigned)(k >> kb) & btm;
          const unsigned ph = (unsigned)(k >> a.phase_shift) & pm;
          const unsigned kd = (unsigned)(k & kmask);
          atomicMin(&mn[ph], bt);
          atomicMax(&mx[ph], bt);
          atomicMin(&s_minb, bt >> a.thread_bits);
          atomicMax(&s_maxb, bt >> a.thread_bits);
          if (kd == 1u) {
            atomicOr(&s_gw, 1u << ph);
            s_w = 1;
          } else if (kd == 2u) {
            atomicOr(&s_ga, 1u << ph);
          } else {
            atomicOr(&s_gr, 1u << ph);
          }
        }
      }
      if (__syncthreads_or(end)) break;
    }
    if (threadIdx.x == 0) {
      const bool racy = summary_racy(mn, mx, s_gw, s_ga, s_gr, s_w != 0u, s_minb, s_maxb, syt, a.thread_bits);
      if (racy) {
        DevResult* r = result_of(a, cell);
        atomicAdd(&r->racy_cells, 1ull);
        if (a.by_cell) atomicMin(&r->hash_cell, (unsigned long long)cell);
        else atomicMin(&r->min_start, (unsigned long long)start);
      }
    }
    __syncthreads();
  }
}

// One warp per result: the end of its first racy cell.
__global__ void scan_finish_kernel(ScanArgs a) {
  DevResult* r = a.res + blockIdx.x;
  const unsigned long long s = r->min_start;
  if (s == ~0ull) return;
  const uint64_t cell = a.keys[s] >> a.cell_shift;
  const uint64_t e = warp_cell_end(a.keys, a.n, a.cell_shift, s, cell);
  if (threadIdx.x == 0) {
    r->seg_end = e;
    r->cell = cell;
  }
}

// ---------------------------------------------------------------------------
// K4 witness passes over [min_start, seg_end)
// ---------------------------------------------------------------------------
// Kind field (a.thread_shift bits): R = 0, W = 1, A = 2 (atomic).  Two kinds
// conflict iff one is W, or one is A and the other R.
struct Fields {
  unsigned b, p, t, k;
};
__device__ __forceinline__ Fields fields(const ScanArgs& a, uint64_t key) {
  Fields f;
  f.k = (unsigned)(key & ((1ull << a.thread_shift) - 1ull));
  f.t = (unsigned)(key >> a.thread_shift) & ((1u << a.thread_bits) - 1u);
  f.b = (unsigned)(key >> a.block_shift) & ((1u << a.block_bits) - 1u);
  f.p = (unsigned)(key >> a.phase_shift) & ((1u << a.phase_bits) - 1u);
  return f;
}
// block interval and grid interval of fine interval q (warp or grid barriers)
__device__ __forceinline__ unsigned coarse_q(const SyncTabs& t, unsigned q) { return q / t.n_wp; }
__device__ __forceinline__ unsigned grid_q(const ScanArgs& a, const SyncTabs& t, unsigned q) {
  return a.grid_of ? __ldg(a.grid_of + q / t.n_wp) : (unsigned)(t.grid >> (4 * q)) & 15u;
}
__device__ __forceinline__ bool kinds_conflict(unsigned kx, unsigned ky) {
  return kx == 1u || ky == 1u || (kx ^ ky) == 2u;
}

// group record of one fine interval q of one block: [mint, maxt] over all its
// instances, then per kind K (R, W, A) [minKt, maxKt, anyK]; words 11.. of the
// record (block 0, q) hold per kind the [min, max] block holding K in q (warp or
// grid barriers).  Without per-block records (a.wit_block_bits == 0) the thread
// words describe the cell's lowest block only: with at most one grid interval
// the smallest racing instance always lies there (a block barrier orders
// nothing across blocks, so the lowest block's instances meet every other
// block's).  With several grid intervals the lowest block's instances may all
// be ordered before the racing ones, so every block keeps its records.
constexpr unsigned kGroupWords = kWitnessGroupWords;
// Each kernel handles result blockIdx.y (one per model of a batch) with the
// blocks of its x dimension.
__device__ __forceinline__ unsigned* groups_of(const ScanArgs& a) {
  return a.groups + (size_t)blockIdx.y * kGroupWords * ((size_t)1 << (a.phase_bits + a.wit_block_bits));
}
// the record of (block b, fine interval q)
__device__ __forceinline__ unsigned* group_rec(const ScanArgs& a, unsigned* groups, unsigned b, unsigned q) {
  const size_t i = a.wit_block_bits ? (((size_t)b << a.phase_bits) | q) : q;
  return groups + i * kGroupWords;
}
__device__ __forceinline__ const unsigned* group_rec(const ScanArgs& a, const unsigned* groups, unsigned b,
                                                     unsigned q) {
  const size_t i = a.wit_block_bits ? (((size_t)b << a.phase_bits) | q) : q;
  return groups + i * kGroupWords;
}

// the cell summary: blocks of all instances and of each kind
__global__ void __launch_bounds__(256) witness_cell_kernel(ScanArgs a) {
  DevResult* r = a.res + blockIdx.y;
  const uint64_t s = r->min_start;
  const uint32_t n_groups = 1u << (a.phase_bits + a.wit_block_bits);
  unsigned* groups = groups_of(a);
  if (s == ~0ull) return;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n_groups; g += gridDim.x * blockDim.x) {
    unsigned* gr = groups + g * kGroupWords;
    gr[0] = 0xffffffffu;
    gr[1] = 0;
    for (int k = 0; k < 3; ++k) {
      gr[2 + 3 * k] = 0xffffffffu;
      gr[3 + 3 * k] = 0;
      gr[4 + 3 * k] = 0;
      gr[11 + 2 * k] = 0xffffffffu;
      gr[12 + 2 * k] = 0;
    }
  }
  const uint64_t e = r->seg_end;
  const uint64_t wcell = r->cell;
  unsigned minb = 0xffffffffu, maxb = 0;
  unsigned kmin[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, kmax[3] = {0, 0, 0}, kany[3] = {0, 0, 0};
  for (uint64_t i = s + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < e; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t key = a.keys[i];
    if ((key >> a.cell_shift) != wcell) continue;   // the bucket path's range holds other cells too
    const Fields f = fields(a, key);
    minb = min(minb, f.b);
    maxb = max(maxb, f.b);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (f.k == (unsigned)k) {
        kmin[k] = min(kmin[k], f.b);
        kmax[k] = max(kmax[k], f.b);
        kany[k] = 1;
      }
  }
  minb = __reduce_min_sync(FULL, minb);
  maxb = __reduce_max_sync(FULL, maxb);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    kmin[k] = __reduce_min_sync(FULL, kmin[k]);
    kmax[k] = __reduce_max_sync(FULL, kmax[k]);
    kany[k] = __reduce_or_sync(FULL, kany[k]);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&r->minb, minb);
    atomicMax(&r->maxb, maxb);
    unsigned* mn[3] = {&r->minRb, &r->minWb, &r->minAb};
    unsigned* mx[3] = {&r->maxRb, &r->maxWb, &r->maxAb};
    unsigned* an[3] = {&r->anyR, &r->anyW, &r->anyA};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicMin(mn[k], kmin[k]);
      atomicMax(mx[k], kmax[k]);
      if (kany[k]) atomicOr(an[k], 1u);
    }
  }
}

__global__ void __launch_bounds__(256) witness_group_kernel(ScanArgs a) {
  DevResult* r = a.res + blockIdx.y;
  const SyncTabs syt = sync_tabs_of(a, blockIdx.y);
  unsigned* groups = groups_of(a);
  const uint64_t s = r->min_start;
  if (s == ~0ull) return;
  const uint64_t e = r->seg_end;
  const uint64_t wcell = r->cell;
  const unsigned b0 = r->minb;
  for (uint64_t i = s + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < e; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t key = a.keys[i];
    if ((key >> a.cell_shift) != wcell) continue;   // the bucket path's range holds other cells too
    const Fields f = fields(a, key);
    if (syt.on) {
      // blocks holding each kind per fine interval (cross-block partners of one grid interval)
      unsigned* g0 = group_rec(a, groups, 0u, f.p);
      atomicMin(&g0[11 + 2 * f.k], f.b);
      atomicMax(&g0[12 + 2 * f.k], f.b);
    }
    if (!a.wit_block_bits && f.b != b0) continue;
    unsigned* g = group_rec(a, groups, f.b, f.p);
    atomicMin(&g[0], f.t);
    atomicMax(&g[1], f.t);
    unsigned* gk = g + 2 + 3 * f.k;
    atomicMin(&gk[0], f.t);
    atomicMax(&gk[1], f.t);
    atomicOr(&gk[2], 1u);
  }
}

__global__ void __launch_bounds__(256) witness_x_kernel(ScanArgs a) {
  DevResult* r = a.res + blockIdx.y;
  const SyncTabs syt = sync_tabs_of(a, blockIdx.y);
  const unsigned* groups = groups_of(a);
  const uint64_t s = r->min_start;
  if (s == ~0ull) return;
  const uint64_t e = r->seg_end;
  const uint64_t wcell = r->cell;
  const unsigned b0 = r->minb;
  const unsigned kminb[3] = {r->minRb, r->minWb, r->minAb}, kmaxb[3] = {r->maxRb, r->maxWb, r->maxAb};
  const unsigned kany[3] = {r->anyR, r->anyW, r->anyA};
  const uint32_t kb = a.thread_shift;
  unsigned long long best = ~0ull;
  for (uint64_t i = s + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < e; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t key = a.keys[i];
    if ((key >> a.cell_shift) != wcell) continue;   // the bucket path's range holds other cells too
    const Fields f = fields(a, key);
    // candidates: the lowest block's instances, or every block's with per-block records
    if (!a.wit_block_bits && f.b != b0) continue;
    const unsigned xb = f.b;
    const unsigned* g = group_rec(a, groups, xb, f.p);
    bool cross = false, same = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (!kinds_conflict(f.k, (unsigned)k)) continue;
      // a conflicting instance of another thread in the same block and (fine) phase
      const unsigned* gk = g + 2 + 3 * k;
      same |= gk[2] && (gk[0] != f.t || gk[1] != f.t);
      if (!syt.on) {
        // a conflicting instance in another block (global cells; a shared cell has one block)
        cross |= kany[k] && (kminb[k] != b0 || kmaxb[k] != b0);
        continue;
      }
      // warp / grid barriers: another block of the same grid interval, or another
      // warp of this block in the same block interval
      const unsigned xc = coarse_q(syt, f.p), xg = grid_q(a, syt, f.p);
      for (unsigned q = 0; q < (1u << a.phase_bits); ++q) {
        const unsigned* gq = group_rec(a, groups, 0u, q);
        // (a record with a key of kind k: q is a fine interval of the model)
        if (gq[11 + 2 * k] != 0xffffffffu && (gq[11 + 2 * k] != xb || gq[12 + 2 * k] != xb) &&
            grid_q(a, syt, q) == xg)
          cross = true;
        if (q != f.p && coarse_q(syt, q) == xc) {
          const unsigned* gqk = group_rec(a, groups, xb, q) + 2 + 3 * k;
          if (gqk[2] && ((gqk[0] >> 5) != (f.t >> 5) || (gqk[1] >> 5) != (f.t >> 5))) same = true;
        }
      }
    }
    if (cross || same) {
      // rank in the tuple order (block, phase, thread, kind, warp phase)
      const unsigned p = syt.on ? coarse_q(syt, f.p) : f.p;
      const unsigned wv = f.p - p * syt.n_wp;
      const unsigned long long rank =
          ((((unsigned long long)xb << (a.phase_bits + a.thread_bits + kb)) |
            ((unsigned long long)p << (a.thread_bits + kb)) | ((unsigned long long)f.t << kb) | f.k) << syt.wp_bits) |
          wv;
      best = rank < best ? rank : best;
    }
  }
  // 64-bit min across the warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(FULL, best, o);
    best = y < best ? y : best;
  }
  if ((threadIdx.x & 31) == 0 && best != ~0ull) atomicMin(&r->x_rank, best);
}

__global__ void __launch_bounds__(256) witness_y_kernel(ScanArgs a) {
  DevResult* r = a.res + blockIdx.y;
  const SyncTabs syt = sync_tabs_of(a, blockIdx.y);
  const uint64_t s = r->min_start;
  if (s == ~0ull || r->x_rank == ~0ull) return;
  const uint64_t e = r->seg_end;
  const uint64_t wcell = r->cell;
  const uint32_t kb = a.thread_shift;
  const unsigned long long xr = r->x_rank;
  const uint32_t wb = syt.wp_bits;
  const unsigned xw = (unsigned)(xr & ((1ull << wb) - 1ull));
  const unsigned xk = (unsigned)(xr >> wb) & ((1u << kb) - 1u);
  const unsigned xt = (unsigned)(xr >> (wb + kb)) & ((1u << a.thread_bits) - 1u);
  const unsigned xp = (unsigned)(xr >> (wb + kb + a.thread_bits)) & ((1u << a.phase_bits) - 1u);
  const unsigned b0 = (unsigned)(xr >> (wb + kb + a.thread_bits + a.phase_bits));   // x's block
  const unsigned xq = xp * syt.n_wp + xw;
  const unsigned xg = syt.on ? grid_q(a, syt, xq) : 0u;
  unsigned long long best = ~0ull;
  for (uint64_t i = s + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < e; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t key = a.keys[i];
    if ((key >> a.cell_shift) != wcell) continue;   // the bucket path's range holds other cells too
    const Fields f = fields(a, key);
    const unsigned yp = syt.on ? coarse_q(syt, f.p) : f.p;
    const unsigned yw = f.p - yp * syt.n_wp;
    const bool other_thread = f.b != b0 || f.t != xt;
    bool concurrent;
    if (!syt.on) concurrent = f.b != b0 || f.p == xp;
    else if (f.b != b0) concurrent = grid_q(a, syt, f.p) == xg;
    else concurrent = yp == xp && ((f.t >> 5) != (xt >> 5) || yw == xw);
    if (other_thread && kinds_conflict(xk, f.k) && concurrent) {
      const unsigned long long rank =
          ((((unsigned long long)f.b << (a.phase_bits + a.thread_bits + kb)) |
            ((unsigned long long)yp << (a.thread_bits + kb)) | ((unsigned long long)f.t << kb) | f.k) << wb) | yw;
      best = rank < best ? rank : best;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(FULL, best, o);
    best = y < best ? y : best;
  }
  if ((threadIdx.x & 31) == 0 && best != ~0ull) atomicMin(&r->y_rank, best);
}

__global__ void init_result_kernel(DevResult* res, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    DevResult* r = res + i;
    r->oob_code = ~0ull;
    r->instances = 0;
    r->racy_cells = 0;
    r->min_start = ~0ull;
    r->seg_end = 0;
    r->cell = 0;
    r->x_rank = ~0ull;
    r->y_rank = ~0ull;
    r->minb = 0xffffffffu;
    r->maxb = 0;
    r->minWb = 0xffffffffu;
    r->maxWb = 0;
    r->anyW = 0;
    r->minAb = r->minRb = 0xffffffffu;
    r->maxAb = r->maxRb = 0;
    r->anyA = r->anyR = 0;
    r->err = 0;
    r->n_keys = 0;
    r->sorted_buf = 0;
    r->hash_cell = ~0ull;
    r->stop = 0;
  }
}

}  // namespace

cudaError_t launch_init_result(DevResult* res, cudaStream_t st, uint32_t n) {
  if (n == 0) return cudaSuccess;
  init_result_kernel<<<(n + 127) / 128, 128, 0, st>>>(res, n);
  return cudaGetLastError();
}

// keys sorted by (cell, fine interval) of a check with warp or grid barriers
// or atomics: the phase-order scan with interval summaries
static bool phase_order_sync(const ScanArgs& a) { return !a.phase_table && (a.sync_tabs != nullptr || a.thread_shift == 2); }

cudaError_t launch_scan(const ScanArgs& a, cudaStream_t st) {
  // the phase-table scan reads keys in 16-byte pairs
  if (a.phase_table && (reinterpret_cast<uintptr_t>(a.keys) & 15u) != 0u) return cudaErrorMisalignedAddress;
  if (a.n > 0) {
    const unsigned blocks = (a.n_warps + kScanWarps - 1) / kScanWarps;
    if (a.phase_table) {
      const bool at = a.thread_shift == 2, sy = a.sync_tabs != nullptr;
      const bool mc = a.by_cell != 0;
      if (mc) {
        if (at && sy) scan_cells_table_kernel<true, true, true><<<blocks, kScanWarps * 32, 0, st>>>(a);
        else if (at) scan_cells_table_kernel<true, false, true><<<blocks, kScanWarps * 32, 0, st>>>(a);
        else if (sy) scan_cells_table_kernel<false, true, true><<<blocks, kScanWarps * 32, 0, st>>>(a);
        else scan_cells_table_kernel<false, false, true><<<blocks, kScanWarps * 32, 0, st>>>(a);
      } else {
        if (at && sy) scan_cells_table_kernel<true, true, false><<<blocks, kScanWarps * 32, 0, st>>>(a);
        else if (at) scan_cells_table_kernel<true, false, false><<<blocks, kScanWarps * 32, 0, st>>>(a);
        else if (sy) scan_cells_table_kernel<false, true, false><<<blocks, kScanWarps * 32, 0, st>>>(a);
        else scan_cells_table_kernel<false, false, false><<<blocks, kScanWarps * 32, 0, st>>>(a);
      }
    }
    else if (phase_order_sync(a)) {
      const uint64_t want = (a.n + 256ull * kSyncChunk - 1) / (256ull * kSyncChunk);
      scan_sorted_sync_kernel<<<(unsigned)min(want, (uint64_t)152 * 16), 256, 0, st>>>(a);
    }
    else scan_cells_kernel<<<blocks, kScanWarps * 32, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.phase_table) scan_long_table_kernel<<<152 * 2, kLongThreads, 0, st>>>(a);
    else if (phase_order_sync(a)) scan_sorted_sync_long_kernel<<<152 * 2, kLongThreads, 0, st>>>(a);
    else scan_long_kernel<<<152 * 2, kLongThreads, 0, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const unsigned nr = a.n_models ? a.n_models : 1u;
  scan_finish_kernel<<<nr, 32, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_witness(const ScanArgs& a, cudaStream_t st) {
  const dim3 g(a.n_models ? 1u : 152u * 2u, a.n_models ? a.n_models : 1u);
  witness_cell_kernel<<<g, 256, 0, st>>>(a);
  witness_group_kernel<<<g, 256, 0, st>>>(a);
  witness_x_kernel<<<g, 256, 0, st>>>(a);
  witness_y_kernel<<<g, 256, 0, st>>>(a);
  return cudaGetLastError();
}

uint64_t scan_long_capacity(uint64_t n, uint32_t n_warps) {
  return n / ((uint64_t)kCarryMaxSegs * kSegKeys) + n_warps + 16;
}

}  // namespace rc
