// Host lowering of a model descriptor (include/rc.h) into the program the
// expansion kernels interpret.
//
// The descriptor holds the paper's Domain / Read / Write relations made
// concrete (Section "Using ISCC in Formal Analysis/Verification": labelled code
// sections, their loop-bound Presburger constraints, and the access relations
// "Stmt[iters] -> Array[index]"), with quasi-affine floor division / modulo as
// in the Ge-SpMM model (Section "Doing this for Ge-SpMM", "j % 32").  Lowering
// folds the parameters into constants, rewrites every expression as a linear
// row over (tid, bid, iterators, floor-div/mod terms), checks that barrier
// phases do not depend on the thread, decides per statement whether every loop
// has a constant trip count ("dense": keys go to fixed slots) and computes the
// 64-bit key layout [cell | phase | block | thread | kind].
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <tuple>

#include "rc_internal.h"

namespace rc {

uint32_t bit_length(uint64_t v) {
  uint32_t n = 0;
  while (v) { n++; v >>= 1; }
  return n;
}

namespace {

// Linear form over tid/bid/iterators/terms with a constant.
struct Lin {
  int64_t c0 = 0;
  int64_t ct[6] = {0, 0, 0, 0, 0, 0};
  std::map<int32_t, int64_t> v;   // var -> coefficient (var < kMaxLoops: iterator; else term)

  void add(const Lin& o, int64_t k) {
    c0 = wadd(c0, wmul(k, o.c0));
    for (int i = 0; i < 6; ++i) ct[i] = wadd(ct[i], wmul(k, o.ct[i]));
    for (auto& kv : o.v) {
      int64_t c = wadd(v[kv.first], wmul(k, kv.second));
      if (c == 0) v.erase(kv.first); else v[kv.first] = c;
    }
  }
  bool is_const() const {
    for (int i = 0; i < 6; ++i) if (ct[i]) return false;
    return v.empty();
  }
  bool operator<(const Lin& o) const {
    if (c0 != o.c0) return c0 < o.c0;
    for (int i = 0; i < 6; ++i) if (ct[i] != o.ct[i]) return ct[i] < o.ct[i];
    return v < o.v;
  }
};

struct TermKey {
  Lin inner;
  int32_t op;
  int64_t d;
  bool operator<(const TermKey& o) const {
    if (op != o.op) return op < o.op;
    if (d != o.d) return d < o.d;
    return inner < o.inner;
  }
};

struct StmtBuilder {
  const rc_model_desc* desc;
  std::vector<TermKey> terms;
  std::map<TermKey, int> term_ids;
  std::vector<int> term_level;      // iterators needed
  std::vector<bool> term_tid;       // depends on tid
  std::vector<bool> loop_tid;       // loop l's iterator varies with tid
  rc_status err = RC_OK;

  int level_of(const Lin& l) const {
    int lev = 0;
    for (auto& kv : l.v) {
      if (kv.first < kMaxLoops) lev = std::max(lev, kv.first + 1);
      else lev = std::max(lev, term_level[kv.first - kMaxLoops]);
    }
    return lev;
  }
  bool depends_on_tid(const Lin& l) const {
    if (l.ct[0] || l.ct[1] || l.ct[2]) return true;
    for (auto& kv : l.v) {
      if (kv.first < kMaxLoops) { if (loop_tid[kv.first]) return true; }
      else if (term_tid[kv.first - kMaxLoops]) return true;
    }
    return false;
  }

  // Compile one postfix expression; `n_iters` iterators are in scope.
  bool compile(const rc_expr& e, int n_iters, Lin* out) {
    if (e.len == 0 || e.code == nullptr) { err = RC_E_INVALID; return false; }
    std::vector<Lin> st;
    for (uint32_t i = 0; i < e.len; ++i) {
      const rc_insn& in = e.code[i];
      Lin x;
      switch (in.op) {
        case RC_OP_CONST: x.c0 = in.imm; st.push_back(x); break;
        case RC_OP_TID:
        case RC_OP_BID:
          if (in.arg < 0 || in.arg > 2) { err = RC_E_INVALID; return false; }
          x.ct[(in.op == RC_OP_TID ? 0 : 3) + in.arg] = 1;
          st.push_back(x);
          break;
        case RC_OP_PARAM:
          if (in.arg < 0 || (uint32_t)in.arg >= desc->n_params || !desc->params) { err = RC_E_INVALID; return false; }
          x.c0 = desc->params[in.arg];
          st.push_back(x);
          break;
        case RC_OP_ITER:
          if (in.arg < 0 || in.arg >= n_iters) { err = RC_E_INVALID; return false; }
          x.v[in.arg] = 1;
          st.push_back(x);
          break;
        case RC_OP_ADD: {
          if (st.size() < 2) { err = RC_E_INVALID; return false; }
          Lin b = st.back(); st.pop_back();
          st.back().add(b, 1);
          break;
        }
        case RC_OP_MUL: {
          if (st.empty()) { err = RC_E_INVALID; return false; }
          Lin a = st.back();
          Lin r;
          r.add(a, in.imm);
          st.back() = r;
          break;
        }
        case RC_OP_FDIV:
        case RC_OP_MOD: {
          if (st.empty() || in.imm <= 0) { err = RC_E_INVALID; return false; }
          Lin a = st.back();
          Lin r;
          if (a.is_const()) {
            r.c0 = in.op == RC_OP_FDIV ? floor_div(a.c0, in.imm) : euclid_mod(a.c0, in.imm);
          } else {
            TermKey k{a, in.op == RC_OP_FDIV ? kFdiv : kMod, in.imm};
            auto it = term_ids.find(k);
            int id;
            if (it == term_ids.end()) {
              if ((int)terms.size() >= kMaxTerms) { err = RC_E_UNSUPPORTED; return false; }
              id = (int)terms.size();
              terms.push_back(k);
              term_ids[k] = id;
              term_level.push_back(level_of(a));
              term_tid.push_back(depends_on_tid(a));
            } else {
              id = it->second;
            }
            r.v[kMaxLoops + id] = 1;
          }
          st.back() = r;
          break;
        }
        case RC_OP_LOAD: {
          // a data-dependent value: always a term (never folded), so that an
          // index outside the table is reported for the thread that reads it
          if (st.empty() || in.arg < 0 || (uint32_t)in.arg >= desc->n_tables || !desc->tables) {
            err = RC_E_INVALID;
            return false;
          }
          Lin a = st.back();
          TermKey k{a, kLoad, (int64_t)in.arg};
          auto it = term_ids.find(k);
          int id;
          if (it == term_ids.end()) {
            if ((int)terms.size() >= kMaxTerms) { err = RC_E_UNSUPPORTED; return false; }
            id = (int)terms.size();
            terms.push_back(k);
            term_ids[k] = id;
            term_level.push_back(level_of(a));
            term_tid.push_back(depends_on_tid(a));
          } else {
            id = it->second;
          }
          Lin r;
          r.v[kMaxLoops + id] = 1;
          st.back() = r;
          break;
        }
        default: err = RC_E_INVALID; return false;
      }
    }
    if (st.size() != 1) { err = RC_E_INVALID; return false; }
    *out = st.back();
    return true;
  }
};

void put_row(const Lin& l, std::vector<Row>* rows, std::vector<LinTerm>* lin, int level = 0) {
  Row r;
  r.level = level;
  r.cache = -1;
  r.c0 = l.c0;
  for (int i = 0; i < 6; ++i) r.ct[i] = l.ct[i];
  r.off = (int32_t)lin->size();
  r.nnz = (int32_t)l.v.size();
  for (auto& kv : l.v) {
    LinTerm t;
    t.var = kv.first;
    t.pad = 0;
    t.coef = kv.second;
    lin->push_back(t);
  }
  rows->push_back(r);
}

bool mul_ok(uint64_t a, uint64_t b, uint64_t* r) {
  if (a != 0 && b > UINT64_MAX / a) return false;
  *r = a * b;
  return true;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------------
// The superset domain (Section "Problems to deal with"; the free rs, re of the
// Ge-SpMM Domain): every distinct load of a table flagged superset becomes a
// free parameter of its statement, ranging over the table's stated [lo, hi].
// The rewrite makes each parameter an outermost loop of the statement (lower
// lo, upper hi + 1, step 1) and replaces the load's whole subexpression by
// that loop's iterator; the statement's own loops move inward.  Where in the
// nest a parameter's loop sits does not change the instance set: an instance
// is fixed by its loop point and the one value of each parameter it uses.
// ---------------------------------------------------------------------------
struct SupersetDesc {
  rc_model_desc desc;
  std::vector<rc_table> tables;
  std::vector<rc_stmt> stmts;
  std::deque<std::vector<rc_insn>> code;      // owned expression code (stable addresses)
  std::deque<std::vector<rc_loop>> loops;
  std::deque<std::vector<rc_expr>> exprs;     // guards and access indices
  std::deque<std::vector<rc_access>> accs;
};

int insn_inputs(int32_t op) {
  switch (op) {
    case RC_OP_ADD: return 2;
    case RC_OP_MUL: case RC_OP_FDIV: case RC_OP_MOD: case RC_OP_LOAD: return 1;
    default: return 0;
  }
}

bool insn_equal(const rc_insn& a, const rc_insn& b) {
  if (a.op != b.op) return false;
  switch (a.op) {
    case RC_OP_CONST: return a.imm == b.imm;
    case RC_OP_MUL: case RC_OP_FDIV: case RC_OP_MOD: return a.imm == b.imm;
    default: return a.arg == b.arg;
  }
}

// First instruction of the subexpression that ends at position p (postfix
// code), or -1 for malformed code.
int64_t subexpr_start(const rc_expr& e, int64_t p) {
  int64_t need = 1;
  for (int64_t q = p; q >= 0; --q) {
    need += insn_inputs(e.code[q].op) - 1;
    if (need == 0) return q;
  }
  return -1;
}

struct FreeParams {
  const rc_model_desc* d;
  std::vector<std::vector<rc_insn>> keys;   // the distinct load subexpressions, first-appearance order
  std::vector<uint32_t> table;              // their tables

  bool is_free_load(const rc_insn& in) const {
    return in.op == RC_OP_LOAD && in.arg >= 0 && (uint32_t)in.arg < d->n_tables && d->tables[in.arg].superset;
  }
  // The outermost free loads of e: (start, end) ranges, none inside another.
  bool segments(const rc_expr& e, std::vector<std::pair<int64_t, int64_t>>* out) const {
    out->clear();
    for (int64_t p = (int64_t)e.len - 1; p >= 0; --p) {
      if (!is_free_load(e.code[p])) continue;
      const int64_t st = subexpr_start(e, p);
      if (st < 0) return false;
      out->push_back({st, p});
      p = st;   // the loop's --p moves before this subexpression: inner loads are part of it
    }
    std::reverse(out->begin(), out->end());
    return true;
  }
  int id_of(const rc_insn* c, int64_t n) {
    for (size_t k = 0; k < keys.size(); ++k) {
      if ((int64_t)keys[k].size() != n) continue;
      bool eq = true;
      for (int64_t i = 0; i < n && eq; ++i) eq = insn_equal(keys[k][i], c[i]);
      if (eq) return (int)k;
    }
    keys.emplace_back(c, c + n);
    table.push_back((uint32_t)c[n - 1].arg);
    return (int)keys.size() - 1;
  }
  bool collect(const rc_expr& e) {
    if (e.len == 0) return true;
    if (!e.code) return false;
    std::vector<std::pair<int64_t, int64_t>> seg;
    if (!segments(e, &seg)) return false;
    for (auto& sg : seg) id_of(e.code + sg.first, sg.second - sg.first + 1);
    return true;
  }
  // e with every outermost free load replaced by its parameter's iterator and
  // every other iterator moved inward past the parameters
  rc_expr rewrite(const rc_expr& e, SupersetDesc* sd) {
    if (e.len == 0) return e;
    std::vector<std::pair<int64_t, int64_t>> seg;
    segments(e, &seg);
    std::vector<rc_insn> out;
    size_t next = 0;
    for (int64_t i = 0; i < (int64_t)e.len; ++i) {
      if (next < seg.size() && seg[next].first == i) {
        rc_insn it{RC_OP_ITER, id_of(e.code + i, seg[next].second - i + 1), 0};
        out.push_back(it);
        i = seg[next].second;
        ++next;
        continue;
      }
      rc_insn in = e.code[i];
      if (in.op == RC_OP_ITER) in.arg += (int32_t)keys.size();
      out.push_back(in);
    }
    sd->code.push_back(std::move(out));
    return rc_expr{sd->code.back().data(), (uint32_t)sd->code.back().size()};
  }
};

// Fills sd with the rewritten descriptor when some table is flagged superset;
// *used = false (and d stays as it is) otherwise.
rc_status superset_rewrite(const rc_model_desc* d, SupersetDesc* sd, bool* used) {
  *used = false;
  if (d->n_tables && !d->tables) return RC_E_INVALID;
  const int64_t kLim = (int64_t)1 << 62;
  for (uint32_t t = 0; t < d->n_tables; ++t) {
    const rc_table& T = d->tables[t];
    if (T.superset > 1) return RC_E_INVALID;
    if (!T.superset) continue;
    if (T.lo > T.hi || T.lo < -kLim || T.hi > kLim) return RC_E_INVALID;
    *used = true;
  }
  if (!*used) return RC_OK;
  if (d->n_stmts && !d->stmts) return RC_E_INVALID;
  sd->desc = *d;
  sd->tables.assign(d->tables, d->tables + d->n_tables);
  for (rc_table& T : sd->tables)
    if (T.superset) { T.data = nullptr; T.len = 0; T.superset = 0; }   // no load reads it any more
  sd->desc.tables = sd->tables.data();
  sd->stmts.assign(d->stmts, d->stmts + d->n_stmts);
  for (uint32_t s = 0; s < d->n_stmts; ++s) {
    const rc_stmt& S = d->stmts[s];
    if ((S.n_loops && !S.loops) || (S.n_guards && !S.guards) || (S.n_accesses && !S.accesses)) return RC_E_INVALID;
    FreeParams fp;
    fp.d = d;
    bool ok = true;
    for (uint32_t l = 0; l < S.n_loops; ++l) ok = ok && fp.collect(S.loops[l].lower) && fp.collect(S.loops[l].upper);
    for (uint32_t g = 0; g < S.n_guards; ++g) ok = ok && fp.collect(S.guards[g]);
    ok = ok && fp.collect(S.phase) && fp.collect(S.warp_phase);
    for (uint32_t a = 0; a < S.n_accesses && ok; ++a) {
      const rc_access& A = S.accesses[a];
      if (A.array >= d->n_arrays || !A.index || !d->arrays) return RC_E_INVALID;
      for (uint32_t k = 0; k < d->arrays[A.array].ndims && k < (uint32_t)kMaxDims; ++k) ok = ok && fp.collect(A.index[k]);
    }
    if (!ok) return RC_E_INVALID;
    if (fp.keys.empty()) continue;
    const size_t nf = fp.keys.size();
    if (nf + S.n_loops > (size_t)kMaxLoops) return RC_E_UNSUPPORTED;
    rc_stmt& D = sd->stmts[s];
    std::vector<rc_loop> loops;
    for (size_t f = 0; f < nf; ++f) {
      const rc_table& T = d->tables[fp.table[f]];
      sd->code.push_back({rc_insn{RC_OP_CONST, 0, T.lo}});
      const rc_expr lo{sd->code.back().data(), 1};
      sd->code.push_back({rc_insn{RC_OP_CONST, 0, T.hi + 1}});
      const rc_expr hi{sd->code.back().data(), 1};
      loops.push_back(rc_loop{lo, hi, 1});
    }
    for (uint32_t l = 0; l < S.n_loops; ++l)
      loops.push_back(rc_loop{fp.rewrite(S.loops[l].lower, sd), fp.rewrite(S.loops[l].upper, sd), S.loops[l].step});
    sd->loops.push_back(std::move(loops));
    D.loops = sd->loops.back().data();
    D.n_loops = (uint32_t)sd->loops.back().size();
    std::vector<rc_expr> guards;
    for (uint32_t g = 0; g < S.n_guards; ++g) guards.push_back(fp.rewrite(S.guards[g], sd));
    sd->exprs.push_back(std::move(guards));
    D.guards = sd->exprs.back().data();
    D.phase = fp.rewrite(S.phase, sd);
    D.warp_phase = fp.rewrite(S.warp_phase, sd);
    std::vector<rc_access> accs(S.accesses, S.accesses + S.n_accesses);
    for (uint32_t a = 0; a < S.n_accesses; ++a) {
      std::vector<rc_expr> idx;
      for (uint32_t k = 0; k < d->arrays[accs[a].array].ndims && k < (uint32_t)kMaxDims; ++k)
        idx.push_back(fp.rewrite(S.accesses[a].index[k], sd));
      sd->exprs.push_back(std::move(idx));
      accs[a].index = sd->exprs.back().data();
    }
    sd->accs.push_back(std::move(accs));
    D.accesses = sd->accs.back().data();
  }
  sd->desc.stmts = sd->stmts.data();
  return RC_OK;
}

}  // namespace

rc_status lower_model(const rc_model_desc* d, Model* m, std::vector<int32_t>* general_ids) {
  if (!d || !m) return RC_E_INVALID;
  SupersetDesc sd;
  bool superset = false;
  {
    const rc_status st = superset_rewrite(d, &sd, &superset);
    if (st != RC_OK) return st;
  }
  if (superset) d = &sd.desc;
  for (int i = 0; i < 3; ++i)
    if (d->grid[i] == 0 || d->block[i] == 0) return RC_E_INVALID;
  if (d->n_phases == 0) return RC_E_INVALID;
  if (d->n_stmts > (uint32_t)kMaxStmts) return RC_E_UNSUPPORTED;
  if (d->n_stmts && !d->stmts) return RC_E_INVALID;
  if (d->n_arrays && !d->arrays) return RC_E_INVALID;
  if (d->n_params && !d->params) return RC_E_INVALID;
  if (d->n_tables && !d->tables) return RC_E_INVALID;
  for (uint32_t t = 0; t < d->n_tables; ++t)
    if (d->tables[t].len && !d->tables[t].data) return RC_E_INVALID;

  DevModel& h = m->host;
  std::memset(&h, 0, sizeof(h));
  for (int i = 0; i < 3; ++i) { h.grid[i] = d->grid[i]; h.block[i] = d->block[i]; }
  uint64_t bs = 0, nb = 0, nt = 0;
  if (!mul_ok((uint64_t)d->block[0] * d->block[1], d->block[2], &bs)) return RC_E_UNSUPPORTED;
  if (!mul_ok((uint64_t)d->grid[0] * d->grid[1], d->grid[2], &nb)) return RC_E_UNSUPPORTED;
  if (bs > (1u << 20) || !mul_ok(bs, nb, &nt) || nt >= (1ull << 42)) return RC_E_UNSUPPORTED;
  h.bs = (uint32_t)bs;
  h.n_blocks = nb;
  h.n_threads = nt;
  {
    const uint64_t dv[7] = {bs, d->block[0], d->block[1], (uint64_t)d->block[0] * d->block[1], d->grid[0],
                            d->grid[1], (uint64_t)d->grid[0] * d->grid[1]};
    for (int i = 0; i < 7; ++i) h.div_magic[i] = fastdiv_magic((int64_t)dv[i]);
  }
  h.n_stmts = d->n_stmts;
  h.n_phases = d->n_phases;
  // warp and grid barriers: the key's phase field holds the fine interval
  // q = phase * n_wphases + warp_phase; the scan maps q to its block interval
  // and its grid interval through two 16-entry tables
  const uint32_t n_wp = d->n_warp_phases ? d->n_warp_phases : 1u;
  h.n_wphases = n_wp;
  bool grid_sync = false;
  if (d->grid_phase) {
    for (uint32_t p = 0; p < d->n_phases; ++p) {
      if (p && d->grid_phase[p] < d->grid_phase[p - 1]) return RC_E_INVALID;   // a grid barrier ends a block interval
      grid_sync |= d->grid_phase[p] != 0;
    }
  }
  m->sync_scopes = n_wp > 1 || grid_sync;

  // arrays and the linear cell space
  std::vector<DevArray> arrays(d->n_arrays);
  uint64_t cells_total = 0;
  m->array_base.assign(d->n_arrays, 0);
  m->array_cells.assign(d->n_arrays, 0);
  m->array_shared.assign(d->n_arrays, 0);
  for (uint32_t a = 0; a < d->n_arrays; ++a) {
    const rc_array& A = d->arrays[a];
    if (A.ndims < 1 || A.ndims > (uint32_t)kMaxDims) return RC_E_INVALID;
    if (A.scope != RC_SCOPE_GLOBAL && A.scope != RC_SCOPE_SHARED) return RC_E_INVALID;
    DevArray& D = arrays[a];
    std::memset(&D, 0, sizeof(D));
    uint64_t c = 1;
    for (uint32_t k = 0; k < A.ndims; ++k) {
      if (A.extent[k] < 1) return RC_E_INVALID;
      if (!mul_ok(c, (uint64_t)A.extent[k], &c) || c >= (1ull << 62)) return RC_E_KEY_OVERFLOW;
      D.ext[k] = A.extent[k];
    }
    D.ndims = (int32_t)A.ndims;
    D.shared = A.scope == RC_SCOPE_SHARED;
    D.base = cells_total;
    D.cells = c;
    uint64_t span;
    if (!mul_ok(c, D.shared ? nb : 1, &span) || cells_total + span < cells_total ||
        cells_total + span >= (1ull << 62))
      return RC_E_KEY_OVERFLOW;
    m->array_base[a] = cells_total;
    m->array_cells[a] = c;
    m->array_shared[a] = D.shared;
    cells_total += span;
  }
  m->total_cells = cells_total;

  // key layout [cell | phase | block | thread | kind]; the kind field is 2 bits
  // (R = 0, W = 1, A = 2) when some access is atomic, else 1 bit
  bool has_atomic = false;
  for (uint32_t s = 0; s < d->n_stmts; ++s)
    for (uint32_t a = 0; a < d->stmts[s].n_accesses && d->stmts[s].accesses; ++a)
      if (d->stmts[s].accesses[a].kind == RC_ATOMIC) has_atomic = true;
  m->has_atomic = has_atomic;
  h.kind_shift = 0;
  h.thread_shift = has_atomic ? 2 : 1;
  h.thread_bits = bit_length(bs - 1);
  h.block_shift = h.thread_shift + h.thread_bits;
  h.block_bits = bit_length(nb - 1);
  h.phase_shift = h.block_shift + h.block_bits;
  uint64_t n_fine = 0;
  if (!mul_ok((uint64_t)d->n_phases, (uint64_t)n_wp, &n_fine)) return RC_E_UNSUPPORTED;
  h.phase_bits = bit_length(n_fine - 1);
  if (h.phase_bits > (uint32_t)kMaxPhaseBits) return RC_E_UNSUPPORTED;
  // up to 16 fine intervals the keys are sorted by cell only and scanned with
  // phase tables; beyond, sorted by (cell, fine interval) and scanned in that
  // order (block and grid intervals are then contiguous inside a cell)
  // grid intervals are compared only for equality, so they are numbered
  // densely (0, 1, ... in block-interval order, the descriptor's numbers being
  // non-decreasing): a grid interval is then below n_phases and fits the
  // phase field (the hash path packs it there)
  m->coarse_tab = m->grid_tab = 0;
  std::vector<uint32_t> grid_of(d->n_phases, 0);   // dense grid interval of each block interval
  if (d->grid_phase)
    for (uint32_t p = 1; p < d->n_phases; ++p) grid_of[p] = grid_of[p - 1] + (d->grid_phase[p] != d->grid_phase[p - 1] ? 1u : 0u);
  for (uint64_t q = 0; q < n_fine && q < 16; ++q) {
    const uint64_t p = q / n_wp;
    m->coarse_tab |= (p & 15u) << (4 * q);
    m->grid_tab |= ((uint64_t)grid_of[p] & 15u) << (4 * q);
  }
  h.sync_tab[0] = m->coarse_tab;
  h.sync_tab[1] = m->grid_tab;
  // more than one grid interval: the witness keeps per-block group records
  // (2^(block bits + phase bits) of them), so the grid is bounded
  m->multi_grid = grid_of.back() != 0;
  if (m->multi_grid && h.block_bits + h.phase_bits > kWitnessBlockGroupBits) return RC_E_UNSUPPORTED;
  h.sync_tab[2] = (uint64_t)n_wp | ((uint64_t)bit_length((uint64_t)n_wp - 1) << 32);
  h.cell_shift = h.phase_shift + h.phase_bits;
  // one more value than the cells so the all-ones cell field is never a valid cell
  h.cell_bits = bit_length(cells_total);
  m->wide = h.cell_shift + h.cell_bits > (uint32_t)kKeyBits;
  if (m->wide) {
    // checked in cell-range chunks; each chunk's cells are rebased to fit the
    // field left beside the other fields (at least 2 bits: one cell per chunk)
    if (h.cell_shift + 2 > (uint32_t)kKeyBits) return RC_E_KEY_OVERFLOW;
    h.cell_bits = (uint32_t)kKeyBits - h.cell_shift;
  }
  h.sort_lo = h.phase_bits <= kScanTablePhaseBits ? h.cell_shift : h.phase_shift;
  h.sort_hi = h.cell_shift + h.cell_bits;

  // arrays that some statement writes or updates atomically; a cell of any
  // other array is only read and cannot race, so its instances are counted and
  // bounds-checked but make no key
  std::vector<bool> written(d->n_arrays, false);
  for (uint32_t s = 0; s < d->n_stmts; ++s)
    for (uint32_t a = 0; a < d->stmts[s].n_accesses && d->stmts[s].accesses; ++a)
      if (d->stmts[s].accesses[a].kind != RC_READ && d->stmts[s].accesses[a].array < d->n_arrays)
        written[d->stmts[s].accesses[a].array] = true;

  // statements
  std::vector<DevStmt> stmts(d->n_stmts);
  std::vector<DevAccess> accs;
  std::vector<Row> rows;
  std::vector<LinTerm> lin;
  std::vector<Term> terms;
  uint64_t dense_slots = 0;
  general_ids->clear();
  for (uint32_t s = 0; s < d->n_stmts; ++s) {
    const rc_stmt& S = d->stmts[s];
    DevStmt& D = stmts[s];
    std::memset(&D, 0, sizeof(D));
    if (S.n_loops > (uint32_t)kMaxLoops || S.n_accesses > (uint32_t)kMaxAccesses) return RC_E_UNSUPPORTED;
    if ((S.n_loops && !S.loops) || (S.n_guards && !S.guards) || (S.n_accesses && !S.accesses))
      return RC_E_INVALID;
    StmtBuilder b;
    b.desc = d;
    b.loop_tid.assign(kMaxLoops, false);
    std::vector<Lin> lo(S.n_loops), hi(S.n_loops), guards(S.n_guards);
    Lin phase, wphase;
    bool dense = true;
    for (uint32_t l = 0; l < S.n_loops; ++l) {
      if (S.loops[l].step <= 0) return RC_E_INVALID;
      if (!b.compile(S.loops[l].lower, (int)l, &lo[l])) return b.err;
      if (!b.compile(S.loops[l].upper, (int)l, &hi[l])) return b.err;
      b.loop_tid[l] = b.depends_on_tid(lo[l]) || b.depends_on_tid(hi[l]);
      Lin diff = hi[l];
      diff.add(lo[l], -1);
      if (diff.is_const()) {
        int64_t span = diff.c0;
        D.trips[l] = span <= 0 ? 0 : (int64_t)(((uint64_t)span + (uint64_t)S.loops[l].step - 1) /
                                               (uint64_t)S.loops[l].step);
      } else {
        dense = false;
      }
      D.step[l] = S.loops[l].step;
    }
    int nl = (int)S.n_loops;
    if (nl > kFastLoops) m->has_deep_loops = true;
    if (nl > 0) m->loop_free = false;
    for (uint32_t g = 0; g < S.n_guards; ++g)
      if (!b.compile(S.guards[g], nl, &guards[g])) return b.err;
    if (!b.compile(S.phase, nl, &phase)) return b.err;
    if (b.depends_on_tid(phase)) return RC_E_INVALID;   // a barrier interval is block-uniform
    const bool has_wp = S.warp_phase.len > 0;
    if (has_wp && !b.compile(S.warp_phase, nl, &wphase)) return b.err;
    std::vector<std::vector<Lin>> idx(S.n_accesses);
    for (uint32_t a = 0; a < S.n_accesses; ++a) {
      const rc_access& A = S.accesses[a];
      if (A.array >= d->n_arrays || (A.kind != RC_READ && A.kind != RC_WRITE && A.kind != RC_ATOMIC) || !A.index)
        return RC_E_INVALID;
      idx[a].resize(d->arrays[A.array].ndims);
      for (uint32_t k = 0; k < d->arrays[A.array].ndims; ++k)
        if (!b.compile(A.index[k], nl, &idx[a][k])) return b.err;
    }
    // emit rows
    D.n_loops = nl;
    D.n_guards = (int32_t)S.n_guards;
    D.n_acc = (int32_t)S.n_accesses;
    for (int l = 0; l < nl; ++l) {
      D.row_lower[l] = (int32_t)rows.size(); put_row(lo[l], &rows, &lin, b.level_of(lo[l]));
      D.row_upper[l] = (int32_t)rows.size(); put_row(hi[l], &rows, &lin, b.level_of(hi[l]));
    }
    // rows evaluated at every point: guards, phase, indices; the thread-constant
    // ones (level 0) get a per-thread cache slot
    int n_cache = 0;
    auto put_point_row = [&](const Lin& e) {
      const int lev = b.level_of(e);
      put_row(e, &rows, &lin, lev);
      if (lev == 0 && n_cache < kFastCache) rows.back().cache = n_cache++;
    };
    D.guard_row0 = (int32_t)rows.size();
    for (auto& g : guards) put_point_row(g);
    D.row_phase = (int32_t)rows.size();
    put_point_row(phase);
    D.row_wphase = -1;
    if (has_wp) {
      D.row_wphase = (int32_t)rows.size();
      put_point_row(wphase);
    }
    D.acc0 = (int32_t)accs.size();
    int n_key = 0;
    for (uint32_t a = 0; a < S.n_accesses; ++a) {
      DevAccess da;
      da.array = (int32_t)S.accesses[a].array;
      da.kind = (int32_t)S.accesses[a].kind;
      da.ndims = (int32_t)idx[a].size();
      da.row0 = (int32_t)rows.size();
      da.key_idx = written[da.array] ? n_key++ : -1;
      da.pad = 0;
      for (auto& e : idx[a]) put_point_row(e);
      accs.push_back(da);
    }
    D.n_cache = n_cache;
    D.n_key = n_key;
    D.term0 = (int32_t)terms.size();
    D.n_terms = (int32_t)b.terms.size();
    for (size_t q = 0; q < b.terms.size(); ++q) {
      Term t;
      t.row = (int32_t)rows.size();
      put_row(b.terms[q].inner, &rows, &lin, b.term_level[q]);
      t.op = b.terms[q].op;
      t.d = b.terms[q].d;
      t.level = b.term_level[q];
      t.pad = 0;
      t.magic = t.op == kLoad ? 0 : fastdiv_magic(t.d);
      terms.push_back(t);
    }
    D.dense = dense ? 1 : 0;
    if (dense) {
      uint64_t it = 1;
      for (int l = 0; l < nl; ++l)
        if (!mul_ok(it, (uint64_t)D.trips[l], &it)) return RC_E_UNSUPPORTED;
      D.n_iter = it;
      uint64_t slots;
      if (!mul_ok(it, (uint64_t)n_key, &slots) || !mul_ok(slots, nt, &slots) ||
          dense_slots + slots < dense_slots)
        return RC_E_UNSUPPORTED;
      D.slot_base = dense_slots;
      dense_slots += slots;
    } else {
      D.n_iter = 0;
      D.slot_base = (uint64_t)general_ids->size() * nt;   // index of its first unit offset
      general_ids->push_back((int32_t)s);
    }
  }
  h.dense_slots = dense_slots;
  h.general_slots = 0;   // filled in after the device count pass
  m->n_general_stmts = (uint32_t)general_ids->size();

  // program image: header | arrays | stmts | accs | rows | lin | terms (256-aligned sections)
  size_t off_arrays = align256(sizeof(DevModel));
  size_t off_stmts = align256(off_arrays + arrays.size() * sizeof(DevArray));
  size_t off_accs = align256(off_stmts + stmts.size() * sizeof(DevStmt));
  size_t off_rows = align256(off_accs + accs.size() * sizeof(DevAccess));
  size_t off_lin = align256(off_rows + rows.size() * sizeof(Row));
  size_t off_terms = align256(off_lin + lin.size() * sizeof(LinTerm));
  // tables: (offset, length) per table, then the values
  std::vector<uint64_t> tab_index;
  uint64_t tab_words = 0;
  for (uint32_t t = 0; t < d->n_tables; ++t) {
    tab_index.push_back(tab_words);
    tab_index.push_back(d->tables[t].len);
    if (tab_words + d->tables[t].len < tab_words || d->tables[t].len > (1ull << 40)) return RC_E_UNSUPPORTED;
    tab_words += d->tables[t].len;
  }
  size_t off_tabidx = align256(off_terms + terms.size() * sizeof(Term));
  size_t off_tdata = align256(off_tabidx + tab_index.size() * 8);
  // the grid interval of each block interval (models scanned in phase order
  // with warp or grid barriers)
  const bool want_gridof = m->sync_scopes && h.phase_bits > (uint32_t)kScanTablePhaseBits;
  size_t off_gridof = align256(off_tdata + (size_t)tab_words * 8);
  size_t off_units = want_gridof ? align256(off_gridof + grid_of.size() * 4) : off_gridof;
  size_t total = off_units;
  m->program.assign(total, 0);
  auto put = [&](size_t off, const void* src, size_t n) {
    if (n) std::memcpy(m->program.data() + off, src, n);
  };
  put(off_arrays, arrays.data(), arrays.size() * sizeof(DevArray));
  put(off_stmts, stmts.data(), stmts.size() * sizeof(DevStmt));
  put(off_accs, accs.data(), accs.size() * sizeof(DevAccess));
  put(off_rows, rows.data(), rows.size() * sizeof(Row));
  put(off_lin, lin.data(), lin.size() * sizeof(LinTerm));
  put(off_terms, terms.data(), terms.size() * sizeof(Term));
  put(off_tabidx, tab_index.data(), tab_index.size() * 8);
  for (uint32_t t = 0; t < d->n_tables; ++t)
    put(off_tdata + (size_t)tab_index[2 * t] * 8, d->tables[t].data, (size_t)d->tables[t].len * 8);
  if (want_gridof) put(off_gridof, grid_of.data(), grid_of.size() * 4);
  m->sec_gridof = want_gridof ? off_gridof : 0;
  // device pointers are stored as offsets here and relocated at upload
  h.arrays = reinterpret_cast<const DevArray*>(off_arrays);
  h.stmts = reinterpret_cast<const DevStmt*>(off_stmts);
  h.accs = reinterpret_cast<const DevAccess*>(off_accs);
  h.rows = reinterpret_cast<const Row*>(off_rows);
  h.lin = reinterpret_cast<const LinTerm*>(off_lin);
  h.terms = reinterpret_cast<const Term*>(off_terms);
  h.unit_offset = reinterpret_cast<const uint64_t*>(off_units);
  h.tables = reinterpret_cast<const uint64_t*>(off_tabidx);
  h.tdata = reinterpret_cast<const int64_t*>(off_tdata);
  h.n_tables = d->n_tables;
  m->sec_arrays = off_arrays;
  m->sec_stmts = off_stmts;
  m->sec_accs = off_accs;
  m->sec_rows = off_rows;
  m->sec_lin = off_lin;
  m->sec_terms = off_terms;
  m->sec_tabidx = off_tabidx;
  return RC_OK;
}

void plan_sort(uint32_t lo, uint32_t hi, uint32_t digit_bits, SortPlan* sp) {
  std::memset(sp, 0, sizeof(*sp));
  uint32_t dbits = digit_bits == 0 ? 8 : digit_bits;
  if (dbits > 11) dbits = 11;
  if (dbits < 4) dbits = 4;
  if (hi <= lo) return;
  uint32_t n = hi - lo;
  uint32_t passes = (n + dbits - 1) / dbits;
  uint32_t base = n / passes, extra = n % passes;
  uint32_t sh = lo;
  for (uint32_t p = 0; p < passes; ++p) {
    uint32_t w = base + (p < extra ? 1 : 0);
    sp->shift[p] = sh;
    sp->bits[p] = w;
    sh += w;
  }
  sp->n_pass = passes;
}

}  // namespace rc
