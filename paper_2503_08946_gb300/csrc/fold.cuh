// Per-cell fold state of the cell scans (scan.cu): the keys of one cell, taken
// in any order, reduce to
// per-barrier-interval masks (seen, two (block, thread), write, atomic, plain
// read) plus the (block, thread) of each interval's first key, from which the
// cell-level race rule of include/rc.h is decided.  A cell is racy iff it has a
// conflict (a write, or an atomic and a plain read) and two blocks meet in it,
// or some barrier interval holds two (block, thread) and a conflict; with warp
// or grid barriers the block-interval and grid-interval tests of
// tfold_racy_sync below apply.
#pragma once

#include "kernels.h"

namespace rc {
namespace {

struct TFold {
  uint64_t fk;       // first key
  uint64_t start;    // its position
  unsigned bt0;      // its (block, thread)
  unsigned f;        // kTMB: two blocks (writes, atomics and reads are the masks below)
  unsigned vmask;    // phases seen
  unsigned gm;       // phases with two (block, thread)
  unsigned gw;       // phases with a write
  unsigned ga, gr;   // phases with an atomic / a plain read (atomic models only)
};
// the fold of models with warp or grid barriers
struct TFoldSync : TFold {
  unsigned gmb, gmw; // phases with two blocks / two warps of one block
};
template <bool SY> struct FoldOf { using type = TFold; };
template <> struct FoldOf<true> { using type = TFoldSync; };
constexpr unsigned kTMB = 2u;
constexpr int kTabPhases = 1 << kScanTablePhaseBits;
constexpr int kTabStride = 2 * kTabPhases + 1;     // per lane: prefix table, own table, pad

template <class F>
__device__ __forceinline__ void tfold_clear(F& x) {
  x.fk = 0; x.start = 0; x.bt0 = 0; x.f = 0; x.vmask = x.gm = x.gw = x.ga = x.gr = 0;
  if constexpr (sizeof(F) != sizeof(TFold)) x.gmb = x.gmw = 0;
}
template <bool AT>
__device__ __forceinline__ bool tfold_racy(const TFold& x) {
  if (!AT) return x.gw != 0u && ((x.f & kTMB) || (x.gm & x.gw) != 0u);
  // a conflict across blocks, or in a phase group with two (block, thread)
  const bool conf = x.gw != 0u || (x.ga != 0u && x.gr != 0u);
  return (conf && (x.f & kTMB)) || (x.gm & (x.gw | (x.ga & x.gr))) != 0u;
}

// With warp or grid barriers the phase field is a fine interval q (block
// interval c(q), warp interval, grid interval g(q)).  A cell races iff some
// fine interval holds two (block, thread) and a conflict, some block interval
// holds two warps of one block and a conflict, or some grid interval holds two
// blocks and a conflict.  The two coarser tests combine the fine intervals'
// masks with their first (block, thread) in `tab` (a difference between two
// fine intervals of one block interval in the block is covered by the grid
// test, as the block interval lies in one grid interval).
// (tab[q * TS] is the first (block, thread) of fine interval q)
template <bool AT, int TS = 1>
__device__ bool tfold_racy_sync(const TFoldSync& x, const unsigned* tab, uint64_t coarse_tab, uint64_t grid_tab,
                                uint32_t tb) {
  const unsigned confq = x.gw | (AT ? (x.ga & x.gr) : 0u);
  if (x.gm & confq) return true;
  unsigned cseen = 0, cmw = 0, cw = 0, ca = 0, cr = 0, gseen = 0, gmb = 0, gw = 0, ga = 0, gr = 0;
  unsigned cfirst[kTabPhases], gfirst[kTabPhases];
  const unsigned tmask = (1u << tb) - 1u;
  unsigned m = x.vmask;
  while (m) {
    const int q = __ffs(m) - 1;
    m &= m - 1;
    const unsigned qb = 1u << q;
    const unsigned c = (unsigned)(coarse_tab >> (4 * q)) & 15u, g = (unsigned)(grid_tab >> (4 * q)) & 15u;
    const unsigned cb = 1u << c, gb = 1u << g;
    const unsigned bt = tab[q * TS];
    const unsigned blk = bt >> tb, wrp = (bt & tmask) >> 5;
    if (!(cseen & cb)) {
      cseen |= cb;
      cfirst[c] = bt;
    } else if ((cfirst[c] >> tb) == blk && ((cfirst[c] & tmask) >> 5) != wrp) {
      cmw |= cb;
    }
    if (x.gmw & qb) cmw |= cb;
    if (!(gseen & gb)) {
      gseen |= gb;
      gfirst[g] = blk;
    } else if (gfirst[g] != blk) {
      gmb |= gb;
    }
    if (x.gmb & qb) gmb |= gb;
    if (x.gw & qb) { cw |= cb; gw |= gb; }
    if (AT) {
      if (x.ga & qb) { ca |= cb; ga |= gb; }
      if (x.gr & qb) { cr |= cb; gr |= gb; }
    }
  }
  return (cmw & (cw | (ca & cr))) != 0u || (gmb & (gw | (ga & gr))) != 0u;
}
// two first (block, thread) of one fine interval: mark two blocks / two warps
__device__ __forceinline__ void mark_pair(unsigned a, unsigned b, unsigned bit, uint32_t tb, unsigned& gmb,
                                          unsigned& gmw) {
  if ((a ^ b) >> tb) gmb |= bit;
  else if ((((a ^ b) & ((1u << tb) - 1u)) >> 5) != 0u) gmw |= bit;
}

// Result record of the model whose cell range holds `cell` (batch), else the
// single result.
// the model of a batch cell (binary search of the models' first cells); 0 for one model
__device__ __forceinline__ uint32_t model_of(const ScanArgs& a, uint64_t cell) {
  if (a.n_models == 0) return 0;
  uint32_t lo = 0, hi = a.n_models;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(&a.cell_base[mid]) <= cell) lo = mid;
    else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ DevResult* result_of(const ScanArgs& a, uint64_t cell) {
  return a.res + model_of(a, cell);
}

// The interval tables of model mi (one model: mi = 0) when the check has warp
// or grid barriers (see ScanArgs).
__device__ __forceinline__ SyncTabs sync_tabs_of(const ScanArgs& a, uint32_t mi = 0) {
  SyncTabs t;
  if (a.sync_tabs) {
    const uint64_t* w = a.sync_tabs + 3 * (size_t)mi;
    t.coarse = w[0];
    t.grid = w[1];
    t.n_wp = (uint32_t)w[2];
    t.wp_bits = (uint32_t)(w[2] >> 32);
    t.on = true;
  }
  return t;
}


// Order-free summary of one cell: per fine interval q the smallest and largest
// (block, thread) of its keys (mn[q] == 0xffffffff: no key in q), the intervals
// holding a write / an atomic / a plain read, whether the cell has a write, and
// its smallest and largest block.  A cell is racy iff some interval holds two
// (block, thread) and a conflict, or the cell has a conflict and two blocks
// (without warp or grid barriers), or -- with them -- some block interval holds
// two warps of one block and a conflict, or some grid interval two blocks and a
// conflict (fine intervals mapped by the interval tables).
__device__ __forceinline__ bool summary_racy(const unsigned* mn, const unsigned* mx, unsigned s_gw, unsigned s_ga,
                                             unsigned s_gr, bool s_w, unsigned s_minb, unsigned s_maxb,
                                             const SyncTabs& syt, uint32_t thread_bits) {
  // a conflict across blocks, or in a phase group with two (block, thread)
  const bool conf = s_w || (s_ga && s_gr);
  const unsigned gconf = s_gw | (s_ga & s_gr);
  bool racy = false;
  for (int ph = 0; ph < kTabPhases; ++ph)
    if (((gconf >> ph) & 1u) && mn[ph] != mx[ph]) racy = true;
  if (!syt.on) {
    racy = racy || (conf && s_minb != s_maxb);
  } else {
    // warp / grid barriers: two warps of one block in a block interval, or
    // two blocks in a grid interval, each with a conflict (fine intervals q
    // mapped by the interval tables; mn / mx are (block, thread) extremes)
    const unsigned tmask = (1u << thread_bits) - 1u;
    unsigned cmin[kTabPhases], cmax[kTabPhases], gmin[kTabPhases], gmax[kTabPhases];
    unsigned cseen = 0, gseen = 0, cc = 0, gc = 0, cwm = 0, cam = 0, crm = 0, gwm = 0, gam = 0, grm = 0;
    for (int q = 0; q < kTabPhases; ++q) {
      if (mn[q] == 0xffffffffu) continue;
      const unsigned c = (unsigned)(syt.coarse >> (4 * q)) & 15u, g = (unsigned)(syt.grid >> (4 * q)) & 15u;
      if (!((cseen >> c) & 1u)) { cseen |= 1u << c; cmin[c] = mn[q]; cmax[c] = mx[q]; }
      else { cmin[c] = min(cmin[c], mn[q]); cmax[c] = max(cmax[c], mx[q]); }
      if (!((gseen >> g) & 1u)) { gseen |= 1u << g; gmin[g] = mn[q] >> thread_bits; gmax[g] = mx[q] >> thread_bits; }
      else { gmin[g] = min(gmin[g], mn[q] >> thread_bits); gmax[g] = max(gmax[g], mx[q] >> thread_bits); }
      if ((s_gw >> q) & 1u) { cwm |= 1u << c; gwm |= 1u << g; }
      if ((s_ga >> q) & 1u) { cam |= 1u << c; gam |= 1u << g; }
      if ((s_gr >> q) & 1u) { crm |= 1u << c; grm |= 1u << g; }
    }
    cc = cwm | (cam & crm);
    gc = gwm | (gam & grm);
    for (int c = 0; c < kTabPhases; ++c)
      if (((cc >> c) & 1u) && (cmin[c] >> thread_bits) == (cmax[c] >> thread_bits) &&
          ((cmin[c] & tmask) >> 5) != ((cmax[c] & tmask) >> 5))
        racy = true;
    for (int g = 0; g < kTabPhases; ++g)
      if (((gc >> g) & 1u) && gmin[g] != gmax[g]) racy = true;
  }
  return racy;
}

}  // namespace
}  // namespace rc
