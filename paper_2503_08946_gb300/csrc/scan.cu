// K3: scan of the sorted keys -> racy-cell count and first racy cell;
// K4: witness (smallest racing pair) inside that cell.
//
// The paper's RaW / WaW / WaR relations (appendix listing of the dependence
// test) pair instances on the same cell with at least one write.  After the
// sort, the instances of a cell are contiguous and grouped by phase.  A cell is
// racy iff (two blocks meet in it and it has a write) or (inside one block,
// some phase group has two threads and a write) -- the cell-level form of the
// pair rule in include/rc.h.
//
// K3a: each warp scans a contiguous range of the sorted keys, 32 keys per
//      lane per segment, staged through shared memory with coalesced loads.  A
//      lane folds its run in order: keys that continue the cell open before the
//      run form its prefix piece, cells that begin and end in the run are
//      counted at once, and the cell open at the run's end is finished by a
//      segmented suffix scan of the lanes' prefix pieces (5 shuffle rounds).
//      The warp's first cell and the cell open at its end go to a Summary
//      (rc_internal.h).
// K3b: one block folds the warp summaries in order (count, first racy cell);
//      one warp finds that cell's end with a 32-way galloping search.
// K4:  four grid-wide reductions over that one segment: the cell summary
//      (blocks, write blocks), per-phase groups of its lowest block, the
//      smallest instance that has a partner (x), and x's smallest partner (y).
//      The smallest participating instance always lies in the lowest block of a
//      racy cell, so only that block's phase groups are needed.
#include <cuda_runtime.h>

#include "kernels.h"

namespace rc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(FULL, v, o);
    v = y < v ? y : v;
  }
  return v;
}

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

// Compact piece of a cell for the lane-level scan: block range, write flag, and
// the first / last phase group with the OR of the racy groups in between
// (the same information as CellPiece in rc_internal.h, packed in 8 words).
struct Piece {
  unsigned minb, maxb;
  unsigned flags;     // bit0 anyW, bit1 single group, bit2 inner racy, bit3 fs write, bit4 ls write, bit5 empty
  unsigned ps;        // first phase | last phase << 16
  unsigned fs_min, fs_max, ls_min, ls_max;
};
constexpr unsigned kPW = 1u, kPSingle = 2u, kPInner = 4u, kPFsW = 8u, kPLsW = 16u, kPEmpty = 32u;

__device__ __forceinline__ Piece piece_empty() {
  Piece p;
  p.minb = p.maxb = 0;
  p.flags = kPEmpty;
  p.ps = 0;
  p.fs_min = p.fs_max = p.ls_min = p.ls_max = 0;
  return p;
}
__device__ __forceinline__ void piece_start(Piece& P, unsigned ph, unsigned t, unsigned b, bool w) {
  P.minb = P.maxb = b;
  P.flags = kPSingle | (w ? (kPW | kPFsW | kPLsW) : 0u);
  P.ps = ph | (ph << 16);
  P.fs_min = P.fs_max = P.ls_min = P.ls_max = t;
}
__device__ __forceinline__ bool ls_racy(const Piece& P) { return P.ls_min != P.ls_max && (P.flags & kPLsW); }
__device__ __forceinline__ bool fs_racy(const Piece& P) { return P.fs_min != P.fs_max && (P.flags & kPFsW); }
__device__ __forceinline__ bool cpiece_racy(const Piece& P) {
  if (P.minb != P.maxb) return (P.flags & kPW) != 0;
  return (P.flags & kPInner) || fs_racy(P) || ls_racy(P);
}
// Add one key.  keep_fs: the piece's first group may continue a group on its
// left, so it is kept apart instead of folding into `inner` when it closes.
__device__ __forceinline__ void piece_add(Piece& P, unsigned ph, unsigned t, unsigned b, bool w, bool keep_fs) {
  if (ph != (P.ps >> 16)) {
    if ((P.flags & kPSingle) && !keep_fs) {
      if (fs_racy(P)) P.flags |= kPInner;
      P.fs_min = P.fs_max = 0;
      P.flags &= ~kPFsW;
    } else if (!(P.flags & kPSingle) && ls_racy(P)) {
      P.flags |= kPInner;
    }
    P.flags &= ~(kPSingle | kPLsW);
    P.ps = (P.ps & 0xFFFFu) | (ph << 16);
    P.ls_min = P.ls_max = t;
    if (w) P.flags |= kPLsW;
  } else {
    P.ls_min = min(P.ls_min, t);
    P.ls_max = max(P.ls_max, t);
    if (w) P.flags |= kPLsW;
    if (P.flags & kPSingle) {
      P.fs_min = P.ls_min;
      P.fs_max = P.ls_max;
      P.flags = (P.flags & ~kPFsW) | ((P.flags & kPLsW) ? kPFsW : 0u);
    }
  }
  P.minb = min(P.minb, b);
  P.maxb = max(P.maxb, b);
  if (w) P.flags |= kPW;
}
// X then Y, pieces of one cell (either may be empty).
__device__ __forceinline__ Piece piece_cat(const Piece& X, const Piece& Y) {
  if (X.flags & kPEmpty) return Y;
  if (Y.flags & kPEmpty) return X;
  Piece r;
  r.minb = min(X.minb, Y.minb);
  r.maxb = max(X.maxb, Y.maxb);
  const unsigned xs = X.flags & kPSingle, ys = Y.flags & kPSingle;
  unsigned inner = ((X.flags | Y.flags) & kPInner);
  r.ps = (X.ps & 0xFFFFu) | (Y.ps & 0xFFFF0000u);
  // merged group when X's last group continues into Y's first group
  const bool join = (X.ps >> 16) == (Y.ps & 0xFFFFu);
  unsigned m_min = 0, m_max = 0;
  bool m_w = false;
  if (join) {
    m_min = min(X.ls_min, Y.fs_min);
    m_max = max(X.ls_max, Y.fs_max);
    m_w = (X.flags & kPLsW) || (Y.flags & kPFsW);
  }
  unsigned fsw, lsw;
  if (join) {
    if (xs && ys) {
      r.fs_min = r.ls_min = m_min; r.fs_max = r.ls_max = m_max; fsw = lsw = m_w;
    } else if (xs) {
      r.fs_min = m_min; r.fs_max = m_max; fsw = m_w;
      r.ls_min = Y.ls_min; r.ls_max = Y.ls_max; lsw = (Y.flags & kPLsW) != 0;
    } else if (ys) {
      r.fs_min = X.fs_min; r.fs_max = X.fs_max; fsw = (X.flags & kPFsW) != 0;
      r.ls_min = m_min; r.ls_max = m_max; lsw = m_w;
    } else {
      r.fs_min = X.fs_min; r.fs_max = X.fs_max; fsw = (X.flags & kPFsW) != 0;
      r.ls_min = Y.ls_min; r.ls_max = Y.ls_max; lsw = (Y.flags & kPLsW) != 0;
      if (m_min != m_max && m_w) inner = kPInner;
    }
  } else {
    r.fs_min = X.fs_min; r.fs_max = X.fs_max; fsw = (X.flags & kPFsW) != 0;
    r.ls_min = Y.ls_min; r.ls_max = Y.ls_max; lsw = (Y.flags & kPLsW) != 0;
    if (!xs && ls_racy(X)) inner = kPInner;
    if (!ys && fs_racy(Y)) inner = kPInner;
  }
  const bool single = join && xs && ys;
  r.flags = ((X.flags | Y.flags) & kPW) | (single ? kPSingle : 0u) | inner | (fsw ? kPFsW : 0u) | (lsw ? kPLsW : 0u);
  return r;
}

__device__ __forceinline__ CellPiece to_cellpiece(const Piece& P, uint64_t cell, uint64_t start) {
  CellPiece c;
  c.cell = cell;
  c.start = start;
  c.minb = P.minb;
  c.maxb = P.maxb;
  c.anyW = (P.flags & kPW) ? 1u : 0u;
  c.first_p = P.ps & 0xFFFFu;
  c.last_p = P.ps >> 16;
  c.single_sub = (P.flags & kPSingle) ? 1u : 0u;
  c.inner = (P.flags & kPInner) ? 1u : 0u;
  c.pad = 0;
  c.fs.mint = P.fs_min; c.fs.maxt = P.fs_max; c.fs.anyW = (P.flags & kPFsW) ? 1u : 0u; c.fs.pad = 0;
  c.ls.mint = P.ls_min; c.ls.maxt = P.ls_max; c.ls.anyW = (P.flags & kPLsW) ? 1u : 0u; c.ls.pad = 0;
  return c;
}

template <class T>
__device__ __forceinline__ T shfl_down_T(const T& v, int delta) {
  static_assert(sizeof(T) % 4 == 0, "shuffle of 4-byte words");
  T r;
  const unsigned* pv = reinterpret_cast<const unsigned*>(&v);
  unsigned* pr = reinterpret_cast<unsigned*>(&r);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) / 4); ++i) pr[i] = __shfl_down_sync(FULL, pv[i], delta);
  return r;
}
template <class T>
__device__ __forceinline__ T shfl_idx_T(const T& v, int src) {
  T r;
  const unsigned* pv = reinterpret_cast<const unsigned*>(&v);
  unsigned* pr = reinterpret_cast<unsigned*>(&r);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) / 4); ++i) pr[i] = __shfl_sync(FULL, pv[i], src);
  return r;
}

constexpr int kScanWarps = 4;                 // warps per block of scan_runs_kernel
constexpr int kRunPad = kScanRun + 1;         // padded per-lane stride in shared memory
constexpr int kSegKeys = 32 * kScanRun;       // keys per warp segment

// Each warp scans a contiguous range of segments of kSegKeys keys, in order.
// Per segment every lane folds its run of kScanRun keys: the keys that continue
// the cell open before the run form its prefix piece; cells that begin and end
// in the run are counted at once; the cell open at the run's end is finished
// by a segmented suffix scan over the lanes' prefix pieces (5 shuffle rounds).
// A cell still open at the segment end is carried to the next segment.  The
// first cell of the warp's range (it may continue the previous warp's range)
// and the cell open at its end go to the warp's Summary for the ordered fold.
__global__ void __launch_bounds__(kScanWarps * 32) scan_runs_kernel(ScanArgs a) {
  __shared__ uint64_t sk[kScanWarps][32 * kRunPad];
  const unsigned tm = (1u << a.thread_bits) - 1u;
  const unsigned bm = (1u << a.block_bits) - 1u;
  const unsigned pm = (1u << a.phase_bits) - 1u;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t* my = sk[w];
  const uint64_t n_seg = (a.n + kSegKeys - 1) / kSegKeys;
  const uint64_t gw = (uint64_t)blockIdx.x * kScanWarps + w;
  const uint64_t per = (n_seg + a.n_warps - 1) / a.n_warps;
  const uint64_t seg0 = gw * per, seg1 = min(n_seg, seg0 + per);
  const uint64_t range_start = seg0 * kSegKeys;
  unsigned count = 0;
  unsigned long long minstart = ~0ull;
  // warp-uniform state
  bool carry_valid = false;
  Piece carry = piece_empty();
  uint64_t carry_cell = 0, carry_start = 0;
  bool first_closed = false;
  Piece Lw = piece_empty();
  uint64_t Lw_cell = 0;
  for (uint64_t seg = seg0; seg < seg1; ++seg) {
    const uint64_t S = seg * kSegKeys;
#pragma unroll
    for (int i = 0; i < kSegKeys / 64; ++i) {
      const int j = 2 * (i * 32 + lane);
      const uint64_t pos = S + j;
      uint64_t x = ~0ull, y = ~0ull;
      if (pos + 1 < a.n) {
        const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(a.keys + pos));
        x = v.x;
        y = v.y;
      } else if (pos < a.n) {
        x = a.keys[pos];
      }
      const int o = (j / kScanRun) * kRunPad + (j % kScanRun);
      my[o] = x;
      my[o + 1] = y;
    }
    __syncwarp();
    const uint64_t s = S + (uint64_t)lane * kScanRun;
    const int len = s < a.n ? (int)min((uint64_t)kScanRun, a.n - s) : 0;
    const uint64_t* run = my + lane * kRunPad;
    // cell of the key just before the run (none before the warp's range)
    uint64_t c_prev = ~0ull;
    if (lane > 0) c_prev = my[(lane - 1) * kRunPad + kScanRun - 1] >> a.cell_shift;
    else if (seg != seg0) c_prev = a.keys[S - 1] >> a.cell_shift;
    Piece PP = piece_empty();       // keys continuing the cell open before the run
    Piece OC = piece_empty();       // the cell open at the current key
    uint64_t oc_cell = 0, oc_start = 0;
    bool has_head = false;
    bool got_L = false;             // this lane closed the warp range's first cell
    Piece Lc = piece_empty();
    uint64_t Lc_cell = 0;
    for (int q = 0; q < len; ++q) {
      const uint64_t k = run[q];
      const uint64_t cc = k >> a.cell_shift;
      const unsigned ph = (unsigned)(k >> a.phase_shift) & pm;
      const unsigned t = (unsigned)(k >> a.thread_shift) & tm;
      const unsigned b = (unsigned)(k >> a.block_shift) & bm;
      const bool wr = (k & 1ull) != 0;
      const uint64_t pos = s + q;
      if (!has_head && cc == c_prev) {
        if (PP.flags & kPEmpty) piece_start(PP, ph, t, b, wr);
        else piece_add(PP, ph, t, b, wr, true);
      } else if (!has_head || cc != oc_cell) {
        if (has_head) {
          if (oc_start == range_start) { got_L = true; Lc = OC; Lc_cell = oc_cell; }
          else if (cpiece_racy(OC)) { ++count; minstart = min(minstart, (unsigned long long)oc_start); }
        }
        has_head = true;
        piece_start(OC, ph, t, b, wr);
        oc_cell = cc;
        oc_start = pos;
      } else {
        piece_add(OC, ph, t, b, wr, oc_start == range_start);
      }
    }
    // suffix scan of the prefix pieces: C = continuation from this lane onward,
    // stop = it ends in this segment (at a lane that has a head)
    Piece C = PP;
    bool stop = has_head || len == 0;
    bool dead = len == 0;                 // the chain ran into lanes past the end of the keys
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const Piece Cn = shfl_down_T(C, d);
      const bool sn = __shfl_down_sync(FULL, stop, d);
      const bool dn = __shfl_down_sync(FULL, dead, d);
      if (!stop && lane + d < 32) {
        C = piece_cat(C, Cn);
        stop = sn;
        dead = dn;
      }
    }
    const Piece Cn1 = shfl_down_T(C, 1);
    const bool stop1 = __shfl_down_sync(FULL, stop, 1);
    const bool dead1 = __shfl_down_sync(FULL, dead, 1);
    // the lane's open cell: finished if its continuation ends inside the segment
    bool open_at_end = false;
    Piece total = OC;
    if (has_head) {
      const bool has_next = lane < 31;
      if (has_next) total = piece_cat(OC, Cn1);
      const bool ended = has_next && stop1 && !dead1;
      if (ended) {
        if (oc_start == range_start) { got_L = true; Lc = total; Lc_cell = oc_cell; }
        else if (cpiece_racy(total)) { ++count; minstart = min(minstart, (unsigned long long)oc_start); }
      } else {
        open_at_end = true;
      }
    }
    // the warp's carried cell continues into lane 0's prefix chain
    const Piece C0 = shfl_idx_T(C, 0);
    const bool stop0 = __shfl_sync(FULL, stop, 0);
    const bool dead0 = __shfl_sync(FULL, dead, 0);
    if (carry_valid && !(C0.flags & kPEmpty)) {
      carry = piece_cat(carry, C0);
      if (stop0 && !dead0) {
        // the carried cell ends in this segment
        if (carry_start == range_start) { first_closed = true; Lw = carry; Lw_cell = carry_cell; }
        else if (cpiece_racy(carry) && lane == 0) { ++count; minstart = min(minstart, (unsigned long long)carry_start); }
        carry_valid = false;
      }
    } else if (carry_valid && C0.flags & kPEmpty) {
      // lane 0 begins a new cell (or there are no keys): the carried cell ended at the segment start
      const bool lane0_has_keys = __shfl_sync(FULL, len, 0) > 0;
      if (lane0_has_keys) {
        if (carry_start == range_start) { first_closed = true; Lw = carry; Lw_cell = carry_cell; }
        else if (cpiece_racy(carry) && lane == 0) { ++count; minstart = min(minstart, (unsigned long long)carry_start); }
        carry_valid = false;
      }
    }
    // the range's first cell closed inside a lane
    const unsigned GL = __ballot_sync(FULL, got_L);
    if (GL) {
      const int src = __ffs(GL) - 1;
      Lw = shfl_idx_T(Lc, src);
      Lw_cell = __shfl_sync(FULL, Lc_cell, src);
      first_closed = true;
    }
    // new carry: the open cell whose continuation reaches the segment end
    const unsigned OE = __ballot_sync(FULL, open_at_end);
    if (OE) {
      const int src = 31 - __clz(OE);
      carry = shfl_idx_T(total, src);
      carry_cell = __shfl_sync(FULL, oc_cell, src);
      carry_start = __shfl_sync(FULL, oc_start, src);
      carry_valid = true;
    }
    __syncwarp();
  }
  // warp summary for the ordered fold
  count = __reduce_add_sync(FULL, count);
  minstart = warp_min_u64(minstart);
  if (lane == 0 && gw < a.n_warps) {
    Summary S = summary_empty();
    if (carry_valid || first_closed) {
      S.empty = 0;
      S.count = count;
      S.minstart = minstart;
      if (first_closed) {
        S.single_cell = 0;
        S.L = to_cellpiece(Lw, Lw_cell, range_start);
        S.R = to_cellpiece(carry, carry_cell, carry_start);
      } else {
        S.single_cell = 1;
        S.L = S.R = to_cellpiece(carry, carry_cell, carry_start);
      }
    }
    a.summaries[gw] = S;
  }
}

// One block: fold the warp summaries in order; count and first racy cell.
constexpr int kFoldThreads = 128;

__global__ void __launch_bounds__(kFoldThreads) scan_fold_kernel(ScanArgs a) {
  __shared__ Summary part[kFoldThreads];
  const uint32_t per = (a.n_warps + kFoldThreads - 1) / kFoldThreads;
  const uint32_t b0 = threadIdx.x * per;
  const uint32_t b1 = min(a.n_warps, b0 + per);
  Summary s = summary_empty();
  for (uint32_t k = b0; k < b1; ++k) s = summary_combine(s, a.summaries[k]);
  part[threadIdx.x] = s;
  __syncthreads();
  for (int width = 1; width < kFoldThreads; width <<= 1) {
    if ((threadIdx.x % (2 * width)) == 0)
      part[threadIdx.x] = summary_combine(part[threadIdx.x], part[threadIdx.x + width]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    uint64_t cnt, ms;
    summary_finish(part[0], &cnt, &ms);
    a.res->racy_cells = cnt;
    a.res->min_start = ms;
  }
}

// One warp: the end of the first racy cell.
__global__ void scan_finish_kernel(ScanArgs a) {
  const unsigned long long s = a.res->min_start;
  if (s == ~0ull) return;
  const uint64_t cell = a.keys[s] >> a.cell_shift;
  const uint64_t e = warp_cell_end(a.keys, a.n, a.cell_shift, s, cell);
  if (threadIdx.x == 0) {
    a.res->seg_end = e;
    a.res->cell = cell;
  }
}

// ---------------------------------------------------------------------------
// K4 witness passes over [min_start, seg_end)
// ---------------------------------------------------------------------------
struct Fields {
  unsigned b, p, t, k;
};
__device__ __forceinline__ Fields fields(const ScanArgs& a, uint64_t key) {
  Fields f;
  f.k = (unsigned)(key & 1ull);
  f.t = (unsigned)(key >> a.thread_shift) & ((1u << a.thread_bits) - 1u);
  f.b = (unsigned)(key >> a.block_shift) & ((1u << a.block_bits) - 1u);
  f.p = (unsigned)(key >> a.phase_shift) & ((1u << a.phase_bits) - 1u);
  return f;
}

// group record: [mint, maxt, minWt, maxWt, anyW]
__global__ void __launch_bounds__(256) witness_cell_kernel(ScanArgs a) {
  DevResult* r = a.res;
  const uint64_t s = r->min_start;
  const uint32_t n_groups = 1u << a.phase_bits;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n_groups; g += gridDim.x * blockDim.x) {
    a.groups[g * 5 + 0] = 0xffffffffu;
    a.groups[g * 5 + 1] = 0;
    a.groups[g * 5 + 2] = 0xffffffffu;
    a.groups[g * 5 + 3] = 0;
    a.groups[g * 5 + 4] = 0;
  }
  if (s == ~0ull) return;
  const uint64_t e = r->seg_end;
  unsigned minb = 0xffffffffu, maxb = 0, minWb = 0xffffffffu, maxWb = 0, anyW = 0;
  for (uint64_t i = s + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < e; i += (uint64_t)gridDim.x * blockDim.x) {
    const Fields f = fields(a, a.keys[i]);
    minb = min(minb, f.b);
    maxb = max(maxb, f.b);
    if (f.k) {
      minWb = min(minWb, f.b);
      maxWb = max(maxWb, f.b);
      anyW = 1;
    }
  }
  minb = __reduce_min_sync(FULL, minb);
  maxb = __reduce_max_sync(FULL, maxb);
  minWb = __reduce_min_sync(FULL, minWb);
  maxWb = __reduce_max_sync(FULL, maxWb);
  anyW = __reduce_or_sync(FULL, anyW);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&r->minb, minb);
    atomicMax(&r->maxb, maxb);
    atomicMin(&r->minWb, minWb);
    atomicMax(&r->maxWb, maxWb);
    if (anyW) atomicOr(&r->anyW, 1u);
  }
}

__global__ void __launch_bounds__(256) witness_group_kernel(ScanArgs a) {
  DevResult* r = a.res;
  const uint64_t s = r->min_start;
  if (s == ~0ull) return;
  const uint64_t e = r->seg_end;
  const unsigned b0 = r->minb;
  for (uint64_t i = s + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < e; i += (uint64_t)gridDim.x * blockDim.x) {
    const Fields f = fields(a, a.keys[i]);
    if (f.b != b0) continue;
    unsigned* g = a.groups + f.p * 5;
    atomicMin(&g[0], f.t);
    atomicMax(&g[1], f.t);
    if (f.k) {
      atomicMin(&g[2], f.t);
      atomicMax(&g[3], f.t);
      atomicOr(&g[4], 1u);
    }
  }
}

__global__ void __launch_bounds__(256) witness_x_kernel(ScanArgs a) {
  DevResult* r = a.res;
  const uint64_t s = r->min_start;
  if (s == ~0ull) return;
  const uint64_t e = r->seg_end;
  const unsigned b0 = r->minb, maxb = r->maxb, minWb = r->minWb, maxWb = r->maxWb, anyW = r->anyW;
  unsigned long long best = ~0ull;
  for (uint64_t i = s + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < e; i += (uint64_t)gridDim.x * blockDim.x) {
    const Fields f = fields(a, a.keys[i]);
    if (f.b != b0) continue;
    // a partner in another block (global cells; a shared cell has one block)
    const bool cross = f.k ? (b0 != maxb) : (anyW && (minWb != f.b || maxWb != f.b));
    // a partner of another thread in the same block and phase
    const unsigned* g = a.groups + f.p * 5;
    const bool same = f.k ? (g[0] != g[1]) : (g[4] && (g[2] != f.t || g[3] != f.t));
    if (cross || same) {
      const unsigned long long rank = ((unsigned long long)f.p << (a.thread_bits + 1)) |
                                      ((unsigned long long)f.t << 1) | f.k;
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
  DevResult* r = a.res;
  const uint64_t s = r->min_start;
  if (s == ~0ull || r->x_rank == ~0ull) return;
  const uint64_t e = r->seg_end;
  const unsigned b0 = r->minb;
  const unsigned long long xr = r->x_rank;
  const unsigned xk = (unsigned)(xr & 1ull);
  const unsigned xt = (unsigned)(xr >> 1) & ((1u << a.thread_bits) - 1u);
  const unsigned xp = (unsigned)(xr >> (a.thread_bits + 1));
  unsigned long long best = ~0ull;
  for (uint64_t i = s + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < e; i += (uint64_t)gridDim.x * blockDim.x) {
    const Fields f = fields(a, a.keys[i]);
    const bool other_thread = f.b != b0 || f.t != xt;
    const bool write = xk || f.k;
    const bool concurrent = f.b != b0 || f.p == xp;
    if (other_thread && write && concurrent) {
      const unsigned long long rank =
          ((unsigned long long)f.b << (a.phase_bits + a.thread_bits + 1)) |
          ((unsigned long long)f.p << (a.thread_bits + 1)) | ((unsigned long long)f.t << 1) | f.k;
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

__global__ void init_result_kernel(DevResult* r) {
  if (threadIdx.x == 0) {
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
    r->err = 0;
    r->n_keys = 0;
    r->sorted_buf = 0;
    r->hash_cell = ~0ull;
    r->stop = 0;
  }
}

}  // namespace

cudaError_t launch_init_result(DevResult* res, cudaStream_t st) {
  init_result_kernel<<<1, 32, 0, st>>>(res);
  return cudaGetLastError();
}

cudaError_t launch_scan(const ScanArgs& a, cudaStream_t st) {
  scan_runs_kernel<<<(a.n_warps + kScanWarps - 1) / kScanWarps, kScanWarps * 32, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scan_fold_kernel<<<1, kFoldThreads, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scan_finish_kernel<<<1, 32, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_witness(const ScanArgs& a, cudaStream_t st) {
  const unsigned g = 152 * 2;
  witness_cell_kernel<<<g, 256, 0, st>>>(a);
  witness_group_kernel<<<g, 256, 0, st>>>(a);
  witness_x_kernel<<<g, 256, 0, st>>>(a);
  witness_y_kernel<<<g, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace rc
