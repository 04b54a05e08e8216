// K3: segmented scan of the sorted keys -> racy-cell count and first racy cell;
// K4: witness (smallest racing pair) inside that cell.
//
// The paper's RaW / WaW / WaR relations (appendix listing of the dependence
// test) pair instances on the same cell with at least one write.  After the
// sort, the instances of a cell are contiguous and grouped by phase.  A cell is
// racy iff (two blocks meet in it and it has a write) or (inside one block,
// some phase group has two threads and a write) -- the cell-level form of the
// pair rule in include/rc.h.
//
// K3a: each warp walks a contiguous range 32 keys per step.  Cell and
//      (cell, phase) group boundaries come from ballots of head flags; per-group
//      min/max thread and min/max block come from redux.sync over the lanes of
//      the group (__reduce_min/max_sync with the group's lane mask); a warp-
//      uniform carry holds the group open at the end of a step.  Cells that
//      close inside the warp's range are counted there; the range's first and
//      last cell pieces go to a Summary (rc_internal.h).
// K3b: one block folds the warp summaries in order, finishes the count and the
//      first racy cell, and finds that cell's end with a 32-way galloping search.
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

__device__ __forceinline__ unsigned lane_range_mask(int lo, int hi) {
  // lanes lo..hi inclusive (0 <= lo <= hi <= 31)
  const unsigned upto = hi >= 31 ? FULL : ((2u << hi) - 1u);
  return upto & ~((1u << lo) - 1u);
}

template <class T>
__device__ __forceinline__ T shfl_T(const T& v, int src) {
  static_assert(sizeof(T) % 4 == 0, "shuffle of 4-byte words");
  T r;
  const unsigned* pv = reinterpret_cast<const unsigned*>(&v);
  unsigned* pr = reinterpret_cast<unsigned*>(&r);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(T) / 4); ++i) pr[i] = __shfl_sync(FULL, pv[i], src);
  return r;
}

__device__ __forceinline__ CellPiece piece_none() {
  CellPiece c;
  c.cell = 0; c.start = 0; c.minb = 0; c.maxb = 0; c.anyW = 0; c.first_p = 0; c.last_p = 0;
  c.single_sub = 1; c.inner = 0; c.pad = 0; c.fs = sub_none(); c.ls = sub_none();
  return c;
}

__global__ void __launch_bounds__(256) scan_warps_kernel(ScanArgs a) {
  const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= a.n_warps) return;
  const uint64_t lo = (uint64_t)wid * a.per_warp;
  const uint64_t hi = lo + a.per_warp < a.n ? lo + a.per_warp : a.n;
  if (lo >= hi) {
    if (lane == 0) a.summaries[wid] = summary_empty();
    return;
  }
  const unsigned tmask = (1u << a.thread_bits) - 1u;
  const unsigned bmask = (1u << a.block_bits) - 1u;
  const unsigned pmask = (1u << a.phase_bits) - 1u;

  bool have = false;
  uint64_t prev_key = 0;
  CellPiece cur = piece_none();
  bool cur_is_L = false;
  bool L_done = false;
  CellPiece Lp = piece_none();
  SubAgg L_fs = sub_none();
  uint64_t count = 0, minstart = ~0ull;

  for (uint64_t base = lo; base < hi; base += 32) {
    const uint64_t i = base + lane;
    const bool valid = i < hi;
    const uint64_t key = valid ? a.keys[i] : 0ull;
    const uint64_t up = __shfl_up_sync(FULL, key, 1);
    const uint64_t pk = lane == 0 ? prev_key : up;
    const bool first = !have && lane == 0;
    const uint64_t cellv = key >> a.cell_shift;
    const bool ch = valid && (first || cellv != (pk >> a.cell_shift));
    const bool sh = valid && (first || (key >> a.phase_shift) != (pk >> a.phase_shift));
    const unsigned V = __ballot_sync(FULL, valid);
    const int last = 31 - __clz(V);
    const unsigned CH = __ballot_sync(FULL, ch);
    const unsigned SH = __ballot_sync(FULL, sh);
    const unsigned WB = __ballot_sync(FULL, valid && (key & 1ull));
    // groups carried from the previous step that end exactly at the step boundary
    if (have && (SH & 1u)) {
      const bool was_single = cur.single_sub != 0;
      if (was_single && cur_is_L) {
        L_fs = cur.ls;          // first sub group of the warp's first cell: kept apart
        cur.fs = L_fs;
      } else if (sub_racy(cur.ls)) {
        cur.inner = 1;
      }
      cur.single_sub = 0;
      if (CH & 1u) {
        if (cur_is_L) {
          Lp = cur;
          Lp.single_sub = was_single ? 1u : 0u;
          Lp.fs = L_fs;
          Lp.ls = was_single ? L_fs : sub_none();
          L_done = true;
        } else {
          const bool racy = (cur.minb != cur.maxb) ? (cur.anyW != 0) : (cur.inner != 0);
          if (racy) {
            count += 1;
            if (cur.start < minstart) minstart = cur.start;
          }
        }
        cur_is_L = false;
      }
    }
    const unsigned t = (unsigned)(key >> a.thread_shift) & tmask;
    const unsigned b = (unsigned)(key >> a.block_shift) & bmask;
    const unsigned p = (unsigned)(key >> a.phase_shift) & pmask;
    const unsigned le = lane == 31 ? FULL : ((2u << lane) - 1u);

    const unsigned sle = SH & le;
    const int s_start = sle ? 31 - __clz(sle) : 0;
    const bool s_cont = sle == 0;
    const unsigned sgt = SH & ~le;
    const int s_end = sgt ? __ffs(sgt) - 2 : last;
    const unsigned cle = CH & le;
    const int c_start = cle ? 31 - __clz(cle) : 0;
    const bool c_cont = cle == 0;
    const unsigned cgt = CH & ~le;
    const int c_end = cgt ? __ffs(cgt) - 2 : last;

    SubAgg sa = sub_none();
    unsigned minb = 0, maxb = 0, cW = 0;
    if (valid) {
      const unsigned smask = lane_range_mask(s_start, s_end);
      const unsigned cmask = lane_range_mask(c_start, c_end);
      sa.mint = __reduce_min_sync(smask, t);
      sa.maxt = __reduce_max_sync(smask, t);
      sa.anyW = (WB & smask) != 0;
      minb = __reduce_min_sync(cmask, b);
      maxb = __reduce_max_sync(cmask, b);
      cW = (WB & cmask) != 0;
    }
    if (valid && s_cont) sa = sub_merge(cur.ls, sa);
    if (valid && c_cont) {
      minb = min(minb, cur.minb);
      maxb = max(maxb, cur.maxb);
      cW |= cur.anyW;
    }
    const bool cell_is_L = c_cont ? cur_is_L : (!have && c_start == 0);
    const bool sub_is_first = s_cont ? (cur.single_sub != 0) : (((CH >> s_start) & 1u) != 0);
    const bool s_closes = valid && lane == s_end && s_end < last;
    const bool keep_fs = s_closes && sub_is_first && cell_is_L;
    const unsigned RS = __ballot_sync(FULL, s_closes && sub_racy(sa) && !keep_fs);
    const unsigned cmask_all = valid ? lane_range_mask(c_start, c_end) : 0u;
    const bool inner = ((RS & cmask_all) != 0) || (c_cont && cur.inner);
    const bool c_closes = valid && lane == c_end && c_end < last;
    const bool racy_c = (minb != maxb) ? (cW != 0) : inner;
    const uint64_t my_start = c_cont ? cur.start : base + (uint64_t)c_start;

    // cells that close here (not the warp's first cell)
    const unsigned RC = __ballot_sync(FULL, c_closes && !cell_is_L && racy_c);
    count += __popc(RC);
    if (RC) {
      const uint64_t s0 = __shfl_sync(FULL, my_start, __ffs(RC) - 1);
      if (s0 < minstart) minstart = s0;
    }
    // the first sub group of the warp's first cell closes here: keep it apart
    const unsigned KF = __ballot_sync(FULL, keep_fs);
    if (KF) L_fs = shfl_T(sa, __ffs(KF) - 1);
    // the warp's first cell closes here
    const unsigned LC = __ballot_sync(FULL, c_closes && cell_is_L);
    const unsigned pf = __shfl_sync(FULL, p, c_start);   // phase of the first key of my cell in this step
    if (LC) {
      const int f = __ffs(LC) - 1;
      const bool single = KF && (__ffs(KF) - 1) == f;
      Lp.cell = __shfl_sync(FULL, cellv, f);
      Lp.start = lo;
      Lp.minb = __shfl_sync(FULL, minb, f);
      Lp.maxb = __shfl_sync(FULL, maxb, f);
      Lp.anyW = __shfl_sync(FULL, cW, f);
      const unsigned my_first_p = c_cont ? cur.first_p : pf;
      Lp.first_p = __shfl_sync(FULL, my_first_p, f);
      Lp.last_p = __shfl_sync(FULL, p, f);
      Lp.inner = __shfl_sync(FULL, (unsigned)inner, f);
      Lp.single_sub = single ? 1u : 0u;
      Lp.fs = L_fs;
      Lp.ls = single ? L_fs : sub_none();
      Lp.pad = 0;
      L_done = true;
    }
    // carry: the cell and sub group open at the last valid lane
    {
      const uint64_t c_cell = __shfl_sync(FULL, cellv, last);
      const uint64_t c_st = __shfl_sync(FULL, my_start, last);
      const unsigned c_minb = __shfl_sync(FULL, minb, last);
      const unsigned c_maxb = __shfl_sync(FULL, maxb, last);
      const unsigned c_w = __shfl_sync(FULL, cW, last);
      const unsigned c_inner = __shfl_sync(FULL, (unsigned)inner, last);
      const unsigned c_single = __shfl_sync(FULL, (unsigned)sub_is_first, last);
      const SubAgg c_ls = shfl_T(sa, last);
      const unsigned c_lastp = __shfl_sync(FULL, p, last);
      const unsigned c_cont_last = __shfl_sync(FULL, (unsigned)c_cont, last);
      const unsigned pf_last = __shfl_sync(FULL, pf, last);
      const unsigned c_firstp = c_cont_last ? cur.first_p : pf_last;
      const unsigned c_isL = __shfl_sync(FULL, (unsigned)cell_is_L, last);
      cur.cell = c_cell;
      cur.start = c_st;
      cur.minb = c_minb;
      cur.maxb = c_maxb;
      cur.anyW = c_w;
      cur.inner = c_inner;
      cur.single_sub = c_single;
      cur.ls = c_ls;
      cur.last_p = c_lastp;
      cur.first_p = c_firstp;
      cur_is_L = c_isL != 0;
      cur.fs = c_single ? c_ls : (cur_is_L ? L_fs : sub_none());
      prev_key = __shfl_sync(FULL, key, last);
      have = true;
    }
  }
  if (lane == 0) {
    Summary S;
    S.empty = 0;
    S.count = count;
    S.minstart = minstart;
    if (L_done) {
      S.single_cell = 0;
      S.L = Lp;
      S.R = cur;
    } else {
      S.single_cell = 1;
      S.L = cur;
      S.R = cur;
    }
    a.summaries[wid] = S;
  }
}

// One block: fold the warp summaries in order, then locate the first racy cell.
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
    if ((threadIdx.x % (2 * width)) == 0) part[threadIdx.x] = summary_combine(part[threadIdx.x], part[threadIdx.x + width]);
    __syncthreads();
  }
  __shared__ unsigned long long s_start;
  if (threadIdx.x == 0) {
    uint64_t cnt, ms;
    summary_finish(part[0], &cnt, &ms);
    a.res->racy_cells = cnt;
    a.res->min_start = ms;
    s_start = ms;
  }
  __syncthreads();
  // end of the first racy cell: 32-way galloping then refinement, warp 0
  if (threadIdx.x < 32 && s_start != ~0ull) {
    const int lane = threadIdx.x;
    const uint64_t target = a.keys[s_start] >> a.cell_shift;
    uint64_t lo = s_start, stride = 1;
    auto fails = [&](uint64_t q) { return q >= a.n || (a.keys[q] >> a.cell_shift) != target; };
    while (true) {
      const uint64_t q = lo + (uint64_t)(lane + 1) * stride;
      const unsigned F = __ballot_sync(FULL, fails(q));
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
      const unsigned F = __ballot_sync(FULL, q >= lo + stride || fails(q));
      lo += (uint64_t)(__ffs(F) - 1) * s2;
      stride = s2;
    }
    if (lane == 0) {
      a.res->seg_end = lo + 1;
      a.res->cell = target;
    }
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
  }
}

}  // namespace

cudaError_t launch_init_result(DevResult* res, cudaStream_t st) {
  init_result_kernel<<<1, 32, 0, st>>>(res);
  return cudaGetLastError();
}

cudaError_t launch_scan(const ScanArgs& a, cudaStream_t st) {
  const unsigned blocks = (a.n_warps * 32 + 255) / 256;
  scan_warps_kernel<<<blocks, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scan_fold_kernel<<<1, kFoldThreads, 0, st>>>(a);
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
