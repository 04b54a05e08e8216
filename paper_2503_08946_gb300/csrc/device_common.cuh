// Device-side evaluation of a lowered statement: rows (linear forms over tid,
// bid, iterators and floor-div/mod terms) and the walk over a statement's loop
// nest in lexicographic order (the paper's Domain: loop bounds as Presburger
// constraints, Section "Using ISCC in Formal Analysis/Verification").
#pragma once

#include <cuda_runtime.h>

#include "rc_internal.h"

namespace rc {

struct ThreadVars {
  int64_t v[6];    // tid.x, tid.y, tid.z, bid.x, bid.y, bid.z
  uint64_t b;      // linear block
  uint32_t t;      // linear thread in block
  uint64_t gtid;
};

// a / d for a < 2^32 by the multiply-high reciprocal of d (magic 0: d = 1)
__device__ __forceinline__ uint64_t div_small(uint64_t a, uint64_t magic) {
  return magic ? __umul64hi(magic, a) : a;
}

__device__ __forceinline__ ThreadVars thread_vars(const DevModel& M, uint64_t gtid) {
  ThreadVars tv;
  tv.gtid = gtid;
  if (M.n_threads < (1ull << 32)) {
    // every quotient and remainder below has operands under 2^32
    const uint64_t* mg = M.div_magic;
    const uint64_t b = div_small(gtid, mg[0]);
    const uint32_t t = (uint32_t)(gtid - b * M.bs);
    tv.b = b;
    tv.t = t;
    const uint64_t bx = M.block[0], by = M.block[1], gx = M.grid[0], gy = M.grid[1];
    const uint64_t q1 = div_small(t, mg[1]);
    tv.v[0] = (int64_t)(t - q1 * bx);
    tv.v[1] = (int64_t)(q1 - div_small(q1, mg[2]) * by);
    tv.v[2] = (int64_t)div_small(t, mg[3]);
    const uint64_t q2 = div_small(b, mg[4]);
    tv.v[3] = (int64_t)(b - q2 * gx);
    tv.v[4] = (int64_t)(q2 - div_small(q2, mg[5]) * gy);
    tv.v[5] = (int64_t)div_small(b, mg[6]);
    return tv;
  }
  uint64_t b = gtid / M.bs;
  uint32_t t = (uint32_t)(gtid - b * M.bs);
  tv.b = b;
  tv.t = t;
  uint32_t bx = M.block[0], by = M.block[1];
  tv.v[0] = t % bx;
  tv.v[1] = (t / bx) % by;
  tv.v[2] = t / (bx * by);
  uint64_t gx = M.grid[0], gy = M.grid[1];
  tv.v[3] = (int64_t)(b % gx);
  tv.v[4] = (int64_t)((b / gx) % gy);
  tv.v[5] = (int64_t)(b / (gx * gy));
  return tv;
}

__device__ __forceinline__ int64_t eval_row(const DevModel& M, int r, const ThreadVars& tv,
                                            const int64_t* it, const int64_t* term) {
  const Row& R = M.rows[r];
  int64_t x = R.c0;
#pragma unroll
  for (int i = 0; i < 6; ++i) x = wadd(x, wmul(R.ct[i], tv.v[i]));
  for (int k = 0; k < R.nnz; ++k) {
    const LinTerm lt = M.lin[R.off + k];
    const int64_t val = lt.var < kMaxLoops ? it[lt.var] : term[lt.var - kMaxLoops];
    x = wadd(x, wmul(lt.coef, val));
  }
  return x;
}

__device__ __forceinline__ void eval_terms(const DevModel& M, const DevStmt& S, int level,
                                           const ThreadVars& tv, const int64_t* it, int64_t* term) {
  for (int q = 0; q < S.n_terms; ++q) {
    const Term T = M.terms[S.term0 + q];
    if (T.level == level) {
      const int64_t a = eval_row(M, T.row, tv, it, term);
      term[q] = T.op == kFdiv ? floor_div(a, T.d) : T.op == kMod ? euclid_mod(a, T.d) : table_load(M, T.d, a);
    }
  }
}

// Calls body(it, term) for every point of the statement's loop nest, in
// lexicographic order, with the terms of the innermost level evaluated.
// Guards are the body's business.
template <class Body>
__device__ __forceinline__ void walk_nest(const DevModel& M, const DevStmt& S, const ThreadVars& tv,
                                          Body&& body) {
  int64_t it[kMaxLoops];
  int64_t hi[kMaxLoops];
  int64_t term[kMaxTerms];
  const int L = S.n_loops;
  eval_terms(M, S, 0, tv, it, term);
  if (L == 0) {
    body(it, term);
    return;
  }
  int l = 0;
  it[0] = eval_row(M, S.row_lower[0], tv, it, term);
  hi[0] = eval_row(M, S.row_upper[0], tv, it, term);
  while (true) {
    if (it[l] >= hi[l]) {
      if (l == 0) break;
      --l;
      it[l] += S.step[l];
      continue;
    }
    if (l == L - 1) {
      eval_terms(M, S, L, tv, it, term);
      body(it, term);
      it[l] += S.step[l];
      continue;
    }
    ++l;
    eval_terms(M, S, l, tv, it, term);
    it[l] = eval_row(M, S.row_lower[l], tv, it, term);
    hi[l] = eval_row(M, S.row_upper[l], tv, it, term);
  }
}

// true iff every guard of the statement is >= 0 at this point
__device__ __forceinline__ bool guards_hold(const DevModel& M, const DevStmt& S, const ThreadVars& tv,
                                            const int64_t* it, const int64_t* term) {
  for (int g = 0; g < S.n_guards; ++g)
    if (eval_row(M, S.guard_row0 + g, tv, it, term) < 0) return false;
  return true;
}

// The key of access `a` of statement `s` at this point, or kSentinel when the
// instance is out of bounds (the smallest offending code is folded into *oob).
// The fine interval of a statement instance (phase * n_wphases + warp phase),
// or -1 if its block or warp interval is out of range.
__device__ __forceinline__ int64_t fine_phase(const DevModel& M, const DevStmt& S, const ThreadVars& tv,
                                              const int64_t* it, const int64_t* term) {
  const int64_t p = eval_row(M, S.row_phase, tv, it, term);
  const int64_t w = S.row_wphase >= 0 ? eval_row(M, S.row_wphase, tv, it, term) : 0;
  return (p < 0 || p >= M.n_phases || w < 0 || w >= M.n_wphases) ? -1 : p * M.n_wphases + w;
}

// The key of one access instance (kSentinel if it is out of bounds); *cell_out
// receives its linear cell (all ones if out of bounds), which the key's cell
// field may not hold whole when the model is wider than one key.
__device__ __forceinline__ uint64_t make_key(const DevModel& M, const DevStmt& S, uint32_t s, int a,
                                             int64_t phase, const ThreadVars& tv, const int64_t* it,
                                             const int64_t* term, unsigned long long* oob, uint64_t* cell_out) {
  const DevAccess A = M.accs[S.acc0 + a];
  const DevArray& arr = M.arrays[A.array];
  bool bad = false;
  if (phase < 0 || phase >= M.n_phases * M.n_wphases) {
    atomicMin(oob, oob_pack(s, (uint32_t)a, tv.gtid, 0));
    bad = true;
  }
  uint64_t e = 0;
  for (int d = 0; d < A.ndims; ++d) {
    const int64_t v = eval_row(M, A.row0 + d, tv, it, term);
    if (v < 0 || v >= arr.ext[d]) {
      atomicMin(oob, oob_pack(s, (uint32_t)a, tv.gtid, (uint32_t)d + 1));
      bad = true;
    }
    e = e * (uint64_t)arr.ext[d] + (uint64_t)v;
  }
  *cell_out = ~0ull;
  if (bad) return kSentinel;
  const uint64_t cell = arr.base + (arr.shared ? tv.b : 0ull) * arr.cells + e;
  *cell_out = cell;
  return (cell << M.cell_shift) | ((uint64_t)phase << M.phase_shift) | (tv.b << M.block_shift) |
         ((uint64_t)tv.t << M.thread_shift) | (uint64_t)A.kind;
}

}  // namespace rc
