// Expansion core shared by the sort path (keys written to slots) and the hash
// path (keys inserted into tables): evaluation of a lowered statement for one
// (statement, thread) unit, handing every access instance's key to a sink.
//
// Fast path (loop depth <= kFastLoops): the loop nest is a compile-time nest
// with the iterators in registers; terms and the thread-constant rows used at
// every point are kept per thread in shared-memory columns; floor division and
// modulo by the invariant divisors use the multiply-high method.  Deeper nests
// take the interpreted walk of device_common.cuh.
#pragma once

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace rc {

constexpr int kExpandThreads = 128;

// Per-thread evaluation state of one statement in the fast path.  Terms and
// cached thread-constant rows live in shared memory columns (stride
// kExpandThreads); iterators live in registers (compile-time loop nest).
struct FastCtx {
  const DevModel* M;
  const DevStmt* S;
  ThreadVars tv;
  int64_t* tval;    // tval[q * kExpandThreads]
  int64_t* cache;   // cache[slot * kExpandThreads]
};

template <int L>
__device__ __forceinline__ int64_t it_sel(const int64_t (&it)[L], int var) {
  int64_t v = 0;
#pragma unroll
  for (int l = 0; l < L; ++l)
    if (var == l) v = it[l];
  return v;
}

template <int L>
__device__ __forceinline__ int64_t row_eval(const FastCtx& c, int r, const int64_t (&it)[L]) {
  const Row* R = c.M->rows + r;
  int64_t x = __ldg(&R->c0);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const int64_t k = __ldg(&R->ct[i]);
    if (k) x = wadd(x, wmul(k, c.tv.v[i]));
  }
  const int off = __ldg(&R->off), nnz = __ldg(&R->nnz);
  for (int k = 0; k < nnz; ++k) {
    const LinTerm* lt = c.M->lin + off + k;
    const int var = __ldg(&lt->var);
    const int64_t v = var < kMaxLoops ? it_sel<L>(it, var) : c.tval[(var - kMaxLoops) * kExpandThreads];
    x = wadd(x, wmul(__ldg(&lt->coef), v));
  }
  return x;
}

// value of a row evaluated at every point: cached if thread-constant (NC: a
// statement without loops has one point, so its rows are evaluated directly)
template <int L, bool NC = false>
__device__ __forceinline__ int64_t point_row(const FastCtx& c, int r, const int64_t (&it)[L]) {
  if (NC) return row_eval<L>(c, r, it);
  const int slot = __ldg(&c.M->rows[r].cache);
  return slot >= 0 ? c.cache[slot * kExpandThreads] : row_eval<L>(c, r, it);
}

template <int L>
__device__ __forceinline__ void terms_at_level(const FastCtx& c, int level, const int64_t (&it)[L]) {
  const Term* T = c.M->terms + c.S->term0;
  for (int q = 0; q < c.S->n_terms; ++q) {
    if (__ldg(&T[q].level) != level) continue;
    const int64_t a = row_eval<L>(c, __ldg(&T[q].row), it);
    const int64_t d = __ldg(&T[q].d);
    const uint64_t mg = __ldg(&T[q].magic);
    const int32_t op = __ldg(&T[q].op);
    c.tval[q * kExpandThreads] = op == kFdiv ? fast_floor_div(a, d, mg)
                                 : op == kMod ? fast_euclid_mod(a, d, mg)
                                              : table_load(*c.M, d, a);
  }
}

// Loop nest of depth L over iterators held in registers (array of LA = max(L, 1)).
template <int D, int L, int LA, class Body>
__device__ __forceinline__ void nest(const FastCtx& c, int64_t (&it)[LA], Body& body) {
  if constexpr (D == L) {
    if (L > 0) terms_at_level<LA>(c, L, it);
    body(it);
  } else {
    if (D > 0) terms_at_level<LA>(c, D, it);
    const int64_t lo = row_eval<LA>(c, c.S->row_lower[D], it);
    const int64_t hi = row_eval<LA>(c, c.S->row_upper[D], it);
    const int64_t step = c.S->step[D];
    for (int64_t v = lo; v < hi; v += step) {
      it[D] = v;
      nest<D + 1, L, LA>(c, it, body);
    }
  }
}

// One statement instance point: guards, phase, and one key per access, each
// handed to sink(a, key, cell) (key = kSentinel and cell = all ones for an
// out-of-bounds instance).
template <int L, bool NC, class Sink>
__device__ __forceinline__ bool point_keys(const FastCtx& c, uint32_t s, const int64_t (&it)[L], uint64_t low,
                                           unsigned long long* oob, Sink& sink) {
  const DevModel& M = *c.M;
  const DevStmt& S = *c.S;
  for (int g = 0; g < S.n_guards; ++g)
    if (point_row<L, NC>(c, S.guard_row0 + g, it) < 0) return false;
  // the key's phase field: the fine interval phase * n_wphases + warp phase
  const int64_t bphase = point_row<L, NC>(c, S.row_phase, it);
  const int64_t wphase = S.row_wphase >= 0 ? point_row<L, NC>(c, S.row_wphase, it) : 0;
  const bool phase_bad = bphase < 0 || bphase >= M.n_phases || wphase < 0 || wphase >= M.n_wphases;
  const int64_t phase = bphase * M.n_wphases + wphase;
  for (int a = 0; a < S.n_acc; ++a) {
    const DevAccess* A = M.accs + S.acc0 + a;
    const int arr_i = __ldg(&A->array), nd = __ldg(&A->ndims), row0 = __ldg(&A->row0), kind = __ldg(&A->kind);
    const DevArray* arr = M.arrays + arr_i;
    bool bad = phase_bad;
    if (phase_bad) atomicMin(oob, oob_pack(s, (uint32_t)a, c.tv.gtid, 0));
    uint64_t e = 0;
    for (int d = 0; d < nd; ++d) {
      const int64_t v = point_row<L, NC>(c, row0 + d, it);
      const int64_t ext = __ldg(&arr->ext[d]);
      if (v < 0 || v >= ext) {
        atomicMin(oob, oob_pack(s, (uint32_t)a, c.tv.gtid, (uint32_t)d + 1));
        bad = true;
      }
      e = e * (uint64_t)ext + (uint64_t)v;
    }
    const int kidx = __ldg(&A->key_idx);
    if (kidx < 0) continue;   // array never written: bounds-checked and counted, no key
    uint64_t key = kSentinel, cell = ~0ull;
    if (!bad) {
      cell = __ldg(&arr->base) + (__ldg(&arr->shared) ? c.tv.b : 0ull) * __ldg(&arr->cells) + e;
      key = (cell << M.cell_shift) | ((uint64_t)phase << M.phase_shift) | low | (uint64_t)kind;
    }
    sink(kidx, key, cell);
  }
  return true;
}

// Expansion of one (statement, thread) unit with loop depth L.  Sink:
//   put(slot, key, cell)  -- one access instance of a guard-true point
//   pad(slot)             -- a key slot of a guard-false point (dense statements)
// where slot is the dense slot (dense statements) or the running offset
// (others); the sink decides where keys go.
template <int L, class Sink>
__device__ void expand_unit_fast(const FastCtx& c, uint32_t s, uint64_t g, DevResult* res,
                                 unsigned long long& count, Sink& sink) {
  constexpr int LA = L > 0 ? L : 1;
  const DevModel& M = *c.M;
  const DevStmt& S = *c.S;
  int64_t it[LA];
#pragma unroll
  for (int l = 0; l < LA; ++l) it[l] = 0;
  // thread-constant terms and rows
  terms_at_level<LA>(c, 0, it);
  constexpr bool NC = L == 0;   // one point: rows are evaluated where used, not cached
  if (!NC) {
    const Row* rows = M.rows;
    auto cache_row = [&](int r) {
      const int slot = __ldg(&rows[r].cache);
      if (slot >= 0) c.cache[slot * kExpandThreads] = row_eval<LA>(c, r, it);
    };
    for (int g2 = 0; g2 < S.n_guards; ++g2) cache_row(S.guard_row0 + g2);
    cache_row(S.row_phase);
    if (S.row_wphase >= 0) cache_row(S.row_wphase);
    for (int a = 0; a < S.n_acc; ++a) {
      const DevAccess* A = M.accs + S.acc0 + a;
      const int nd = __ldg(&A->ndims), row0 = __ldg(&A->row0);
      for (int d = 0; d < nd; ++d) cache_row(row0 + d);
    }
  }
  const uint64_t low = (c.tv.b << M.block_shift) | ((uint64_t)c.tv.t << M.thread_shift);
  const uint64_t T = M.n_threads;
  if (S.dense) {
    uint64_t slot = S.slot_base + g;
    const uint64_t step_pt = (uint64_t)S.n_key * T;
    auto body = [&](const int64_t (&itv)[LA]) {
      auto put = [&](int kidx, uint64_t key, uint64_t cell) { sink.put(slot + (uint64_t)kidx * T, key, cell); };
      if (point_keys<LA, NC>(c, s, itv, low, &res->oob_code, put)) {
        count += (unsigned long long)S.n_acc;
      } else {
        for (int kq = 0; kq < S.n_key; ++kq) sink.pad(slot + (uint64_t)kq * T);
      }
      slot += step_pt;
    };
    nest<0, L, LA>(c, it, body);
  } else {
    uint64_t off = M.unit_offset[S.slot_base + g];
    auto body = [&](const int64_t (&itv)[LA]) {
      auto put = [&](int kidx, uint64_t key, uint64_t cell) { sink.put(off + (uint64_t)kidx, key, cell); };
      if (point_keys<LA, NC>(c, s, itv, low, &res->oob_code, put)) {
        off += (uint64_t)S.n_key;
        count += (unsigned long long)S.n_acc;
      }
    };
    nest<0, L, LA>(c, it, body);
  }
}

template <class Sink>
__device__ __forceinline__ void expand_unit_dispatch(const FastCtx& c, uint32_t s, uint64_t g, DevResult* res,
                                                     unsigned long long& count, Sink& sink) {
  switch (c.S->n_loops) {
    case 0: expand_unit_fast<0>(c, s, g, res, count, sink); break;
    case 1: expand_unit_fast<1>(c, s, g, res, count, sink); break;
    case 2: expand_unit_fast<2>(c, s, g, res, count, sink); break;
    case 3: expand_unit_fast<3>(c, s, g, res, count, sink); break;
    default: expand_unit_fast<4>(c, s, g, res, count, sink); break;
  }
}

// Generic path for loop nests deeper than kFastLoops: interpreted nest with
// local arrays, same sink interface.
template <class Sink>
__device__ void expand_unit_generic(const DevModel& M, uint32_t s, uint64_t g, DevResult* res,
                                    unsigned long long& count, Sink& sink) {
  const uint64_t T = M.n_threads;
  const DevStmt& S = M.stmts[s];
  const ThreadVars tv = thread_vars(M, g);
  if (S.dense) {
    uint64_t j = 0;
    walk_nest(M, S, tv, [&](const int64_t* it, const int64_t* term) {
      const uint64_t slot = S.slot_base + j * (uint64_t)S.n_key * T + g;
      if (guards_hold(M, S, tv, it, term)) {
        const int64_t phase = fine_phase(M, S, tv, it, term);
        for (int a = 0; a < S.n_acc; ++a) {
          uint64_t cell;
          const uint64_t key = make_key(M, S, s, a, phase, tv, it, term, &res->oob_code, &cell);
          const int kidx = M.accs[S.acc0 + a].key_idx;
          if (kidx >= 0) sink.put(slot + (uint64_t)kidx * T, key, cell);
        }
        count += (unsigned long long)S.n_acc;
      } else {
        for (int kq = 0; kq < S.n_key; ++kq) sink.pad(slot + (uint64_t)kq * T);
      }
      ++j;
    });
  } else {
    uint64_t off = M.unit_offset[S.slot_base + g];
    walk_nest(M, S, tv, [&](const int64_t* it, const int64_t* term) {
      if (!guards_hold(M, S, tv, it, term)) return;
      const int64_t phase = fine_phase(M, S, tv, it, term);
      for (int a = 0; a < S.n_acc; ++a) {
        uint64_t cell;
        const uint64_t key = make_key(M, S, s, a, phase, tv, it, term, &res->oob_code, &cell);
        const int kidx = M.accs[S.acc0 + a].key_idx;
        if (kidx >= 0) sink.put(off + (uint64_t)kidx, key, cell);
      }
      off += (uint64_t)S.n_key;
      count += (unsigned long long)S.n_acc;
    });
  }
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace rc
