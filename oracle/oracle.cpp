// CPU oracle for the concrete-instance SIMT race check.
//
// TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's CPU
// baseline may load this library; the product path never does.  It shares no
// code, header, table or helper with the CUDA path: it reads its own text
// description of a model (written by oracle/__init__.py) and computes the
// result from the definitions below with plain loops and std::sort.
//
// What is computed (the paper gives the ingredients, the concurrency rule is the
// reading adopted for SIMT):
//
//  * The model: the paper's Domain / Read / Write relations (Section "Using ISCC
//    in Formal Analysis", listings of the Domain, Read and Write sets) made
//    concrete: for every thread of a fixed grid, every statement, every point of
//    its loop nest whose guards hold, and every access, one *access instance*
//        x = (array a, scope instance s, element e, block b, phase p, thread t, kind k)
//    with s = b for shared arrays and s = 0 for global arrays, e the row-major
//    element index, p the value of the statement's barrier-interval expression
//    and k in {R=0, W=1, A=2} (A: an atomic read-modify-write).  gtid = b *
//    blockSize + t.  Each instance also carries its warp interval w (the
//    number of warp barriers, __syncwarp, its thread passed inside the current
//    block interval) and, through a table of the model, the grid interval
//    g(p) of its block interval (the number of grid-wide barriers before it;
//    a grid barrier also ends a block interval, so g is non-decreasing in p).
//    The full tuple is (a, s, e, b, p, t, k, w), ordered in that order.
//  * Dependences: the paper's RaW / WaW / WaR relations (Section "Using ISCC in
//    Formal Analysis", the dependence test of the appendix listing) pair two
//    instances that touch the same array cell with at least one write.  The
//    paper orders them by a sequential Before relation; for SIMT threads the
//    reading adopted here is: two instances are *concurrent* iff they belong to
//    different threads and (different blocks, or the same barrier interval).
//    Hence x, y race iff
//        (a, s, e) equal  and  gtid_x != gtid_y  and  conflict(k_x, k_y)
//        and (b_x != b_y ? g(p_x) = g(p_y)
//                        : p_x = p_y and (warp_x != warp_y or w_x = w_y)),
//    with warp = t / 32: blocks are ordered only by grid barriers, two warps of
//    one block only by block barriers, the threads of one warp also by warp
//    barriers.  Without warp or grid barriers (w = 0, g = 0) this is
//    (b_x != b_y or p_x = p_y).
//    where two kinds conflict iff one is W, or one is A and the other R: an
//    atomic modifies the cell (so it conflicts with plain reads and writes), and
//    two atomics on one cell are ordered by the memory system (no race).
//    Shared cells have s = b, so they can only race inside one block and one
//    interval; global cells also race across blocks in any interval.
//  * Result: verdict = some pair races; count = number of distinct racy cells
//    (a, s, e); witness = the lexicographically smallest racing pair (x, y),
//    x < y, under tuple order (a, s, e, b, p, t, k).  Identical tuples are one
//    instance.  Quasi-affine floor division rounds toward minus infinity and
//    modulo is Euclidean (result in [0, d)), as in the Presburger
//    floor/mod of the paper's Ge-SpMM model (j % 32).
//  * Data-dependent values: a load reads an integer table of the model (0
//    outside it).  A table whose values are unknown and only bounded, lo <= v
//    <= hi, gives the paper's superset domain (Section "Problems to deal
//    with"; the free rs, re, ptr of the Ge-SpMM Domain listing): each of its
//    loads in a statement is a free parameter of that statement, loads with
//    the same expression being one parameter, and the statement has an
//    instance for every value in [lo, hi] of every free parameter.
//  * Errors: an index outside its extent, or an interval outside
//    [0, n_phases), makes the status OUT_OF_BOUNDS; the smallest
//    (statement, access, gtid, dimcode) over the offending instances is reported
//    (dimcode 0 = the interval, d+1 = index dimension d).
//
// Per cell the oracle uses the equivalent cell-level test
//     racy(cell) <=> (some grid interval G has >= 2 distinct blocks and conf(G))
//                 or (some (b, p) group has >= 2 distinct warps and conf)
//                 or (some (b, p, w) group has >= 2 distinct threads and conf),
//     conf(S) = (S has a W) or (S has an A and an R),
// (without warp and grid barriers: >= 2 blocks and conf(cell), or some (b, p)
// group with >= 2 threads and conf).  The three kinds of groups are exactly the
// sets whose members are pairwise concurrent across blocks, across warps, and
// within one warp interval,
// which follows from the pair predicate: a W in a multi-block cell races with an
// instance of any other block, and a W in a (b, p) group with >= 2 threads races
// with an instance of another thread of that group.  Without a W, if a set
// spread over two blocks (threads) holds an A and an R, some A and some R lie in
// different blocks (threads): if all A and all R sat in one block, the other
// block's instances could only be W.  Conversely every racing pair is of one of
// the two kinds.  oracle_brute() applies the pair predicate to every pair
// instead, so the two can be compared on small models.
#include <algorithm>
#include <cctype>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <stdexcept>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

namespace {

// ----------------------------------------------------------------------------
// model
// ----------------------------------------------------------------------------
enum Op { C_CONST, C_TID, C_BID, C_PARAM, C_ITER, C_ADD, C_MUL, C_FDIV, C_MOD, C_LOAD, C_FREE };

struct Node {
  Op op;
  int64_t v;   // constant, axis, parameter number, loop level, multiplier, divisor, table or free parameter
  int a, b;    // operand node indices (or -1)
};

struct Expr {
  std::vector<Node> nodes;
  int root = -1;
};

struct Loop { Expr lower, upper; int64_t step; };
struct Access { int kind; int array; std::vector<Expr> index; };
struct Stmt {
  Expr phase;
  Expr wphase;          // warp interval (empty: 0)
  std::vector<Loop> loops;
  std::vector<Expr> guards;
  std::vector<Access> accesses;
  std::vector<int64_t> free_lo, free_hi;   // ranges of the statement's free parameters (superset tables)
};
struct Array { bool shared; std::vector<int64_t> ext; };
struct Model {
  int64_t grid[3], block[3];
  std::vector<int64_t> params;
  int64_t n_phases = 1;
  int64_t n_wphases = 1;                      // warp intervals per block interval
  std::vector<int64_t> grid_phase;            // grid interval of each block interval
  std::vector<std::vector<int64_t>> tables;   // integer tables read by loads (0 outside)
  std::vector<bool> table_free;               // superset tables: values unknown, in [lo, hi]
  std::vector<int64_t> table_lo, table_hi;
  std::vector<Array> arrays;
  std::vector<Stmt> stmts;
};

// ----------------------------------------------------------------------------
// parsing of the oracle's text format (see oracle/__init__.py)
// ----------------------------------------------------------------------------
struct Parser {
  std::vector<std::string> tok;
  size_t pos = 0;
  size_t n_tables = 0;
  explicit Parser(const char* s) {
    std::string cur;
    for (const char* p = s; *p; ++p) {
      if (std::isspace((unsigned char)*p)) {
        if (!cur.empty()) { tok.push_back(cur); cur.clear(); }
      } else {
        cur.push_back(*p);
      }
    }
    if (!cur.empty()) tok.push_back(cur);
  }
  const std::string& next() {
    if (pos >= tok.size()) throw std::runtime_error("unexpected end of model text");
    return tok[pos++];
  }
  void expect(const char* w) {
    if (next() != w) throw std::runtime_error(std::string("expected ") + w);
  }
  int64_t integer() {
    const std::string& t = next();
    char* end = nullptr;
    long long v = std::strtoll(t.c_str(), &end, 10);
    if (end == t.c_str() || *end) throw std::runtime_error("expected integer, got " + t);
    return (int64_t)v;
  }
  int expr_node(Expr& e) {
    const std::string t = next();
    Node n{C_CONST, 0, -1, -1};
    if (t == "(") {
      const std::string o = next();
      if (o == "+") {
        n.op = C_ADD; n.a = expr_node(e); n.b = expr_node(e);
      } else if (o == "*") {
        n.op = C_MUL; n.v = integer(); n.a = expr_node(e);
      } else if (o == "/") {
        n.op = C_FDIV; n.a = expr_node(e); n.v = integer();
        if (n.v <= 0) throw std::runtime_error("divisor must be positive");
      } else if (o == "%") {
        n.op = C_MOD; n.a = expr_node(e); n.v = integer();
        if (n.v <= 0) throw std::runtime_error("modulus must be positive");
      } else if (o == "L") {
        n.op = C_LOAD; n.v = integer(); n.a = expr_node(e);
        if (n.v < 0 || n.v >= (int64_t)n_tables) throw std::runtime_error("bad table");
      } else {
        throw std::runtime_error("bad operator " + o);
      }
      expect(")");
    } else if (t == "tx" || t == "ty" || t == "tz") {
      n.op = C_TID; n.v = t[1] - 'x';
    } else if (t == "bx" || t == "by" || t == "bz") {
      n.op = C_BID; n.v = t[1] - 'x';
    } else if (t[0] == 'p') {
      n.op = C_PARAM; n.v = std::atoll(t.c_str() + 1);
    } else if (t[0] == 'i') {
      n.op = C_ITER; n.v = std::atoll(t.c_str() + 1);
    } else {
      pos--;
      n.op = C_CONST; n.v = integer();
    }
    e.nodes.push_back(n);
    return (int)e.nodes.size() - 1;
  }
  Expr expr() { Expr e; e.root = expr_node(e); return e; }

  Model model() {
    Model m;
    expect("rcmodel");
    if (integer() != 1) throw std::runtime_error("unknown model text version");
    expect("grid");
    for (int i = 0; i < 3; ++i) m.grid[i] = integer();
    expect("block");
    for (int i = 0; i < 3; ++i) m.block[i] = integer();
    expect("params");
    int64_t np = integer();
    for (int64_t i = 0; i < np; ++i) m.params.push_back(integer());
    expect("phases");
    m.n_phases = integer();
    expect("wphases");
    m.n_wphases = integer();
    expect("gridphase");
    const int64_t ng = integer();
    for (int64_t i = 0; i < ng; ++i) m.grid_phase.push_back(integer());
    if (m.n_wphases < 1 || (ng != 0 && ng != m.n_phases)) throw std::runtime_error("bad sync description");
    if (ng == 0) m.grid_phase.assign((size_t)m.n_phases, 0);
    expect("tables");
    int64_t nt = integer();
    for (int64_t t = 0; t < nt; ++t) {
      std::vector<int64_t> v;
      if (next() == "free") {
        const int64_t lo = integer(), hi = integer();
        if (lo > hi) throw std::runtime_error("empty superset range");
        m.tables.push_back(v);
        m.table_free.push_back(true);
        m.table_lo.push_back(lo);
        m.table_hi.push_back(hi);
        continue;
      }
      pos--;
      int64_t len = integer();
      for (int64_t k = 0; k < len; ++k) v.push_back(integer());
      m.tables.push_back(v);
      m.table_free.push_back(false);
      m.table_lo.push_back(0);
      m.table_hi.push_back(0);
    }
    n_tables = m.tables.size();
    expect("arrays");
    int64_t na = integer();
    for (int64_t i = 0; i < na; ++i) {
      Array a;
      const std::string sc = next();
      if (sc != "G" && sc != "S") throw std::runtime_error("bad scope");
      a.shared = sc == "S";
      int64_t nd = integer();
      for (int64_t d = 0; d < nd; ++d) a.ext.push_back(integer());
      m.arrays.push_back(a);
    }
    expect("stmts");
    int64_t ns = integer();
    for (int64_t i = 0; i < ns; ++i) {
      Stmt s;
      expect("stmt");
      expect("phase");
      s.phase = expr();
      expect("wphase");
      s.wphase = expr();
      expect("loops");
      int64_t nl = integer();
      for (int64_t l = 0; l < nl; ++l) {
        Loop lp;
        lp.lower = expr();
        lp.upper = expr();
        lp.step = integer();
        if (lp.step <= 0) throw std::runtime_error("loop step must be positive");
        s.loops.push_back(lp);
      }
      expect("guards");
      int64_t ng = integer();
      for (int64_t g = 0; g < ng; ++g) s.guards.push_back(expr());
      expect("accesses");
      int64_t nacc = integer();
      for (int64_t k = 0; k < nacc; ++k) {
        Access a;
        const std::string kd = next();
        if (kd != "R" && kd != "W" && kd != "A") throw std::runtime_error("bad access kind");
        a.kind = kd == "W" ? 1 : (kd == "A" ? 2 : 0);
        a.array = (int)integer();
        if (a.array < 0 || a.array >= (int)m.arrays.size()) throw std::runtime_error("bad array");
        int64_t nd = integer();
        if (nd != (int64_t)m.arrays[a.array].ext.size()) throw std::runtime_error("index rank");
        for (int64_t d = 0; d < nd; ++d) a.index.push_back(expr());
        s.accesses.push_back(a);
      }
      free_parameters(m, s);
      m.stmts.push_back(s);
    }
    expect("end");
    return m;
  }

  // The superset domain (Section "Problems to deal with"): a load of a table
  // whose values are unknown is a free parameter of the statement, ranging
  // over the table's stated [lo, hi].  Loads written the same way (the same
  // expression) are one parameter; the node of each outermost such load
  // becomes a reference to its parameter.
  static std::string text_of(const Expr& e, int n) {
    const Node& x = e.nodes[n];
    std::string r = "(" + std::to_string((int)x.op) + ":" + std::to_string(x.v);
    if (x.a >= 0) r += " " + text_of(e, x.a);
    if (x.b >= 0) r += " " + text_of(e, x.b);
    return r + ")";
  }
  static void free_in(const Model& m, Expr& e, int n, std::vector<std::string>& seen, Stmt& s) {
    if (n < 0) return;
    Node& x = e.nodes[n];
    if (x.op == C_LOAD && m.table_free[(size_t)x.v]) {
      const std::string key = text_of(e, n);
      size_t id = 0;
      while (id < seen.size() && seen[id] != key) ++id;
      if (id == seen.size()) {
        seen.push_back(key);
        s.free_lo.push_back(m.table_lo[(size_t)x.v]);
        s.free_hi.push_back(m.table_hi[(size_t)x.v]);
      }
      x.op = C_FREE;
      x.v = (int64_t)id;
      return;
    }
    const int a = x.a, b = x.b;
    free_in(m, e, a, seen, s);
    free_in(m, e, b, seen, s);
  }
  static void free_parameters(const Model& m, Stmt& s) {
    std::vector<std::string> seen;
    auto one = [&](Expr& e) { free_in(m, e, e.root, seen, s); };
    one(s.phase);
    one(s.wphase);
    for (Loop& l : s.loops) { one(l.lower); one(l.upper); }
    for (Expr& g : s.guards) one(g);
    for (Access& a : s.accesses)
      for (Expr& x : a.index) one(x);
    if (s.free_lo.size() > 16) throw std::runtime_error("too many free parameters");
  }
};

// ----------------------------------------------------------------------------
// expression evaluation: two's-complement wrapping int64, floor division and
// Euclidean modulo by positive constants
// ----------------------------------------------------------------------------
struct Env {
  int64_t tid[3], bid[3];
  const std::vector<int64_t>* params;
  const std::vector<std::vector<int64_t>>* tables;
  int64_t iter[16];
  int64_t free[16];   // values of the statement's free parameters
};

int64_t wrap_add(int64_t a, int64_t b) { return (int64_t)((uint64_t)a + (uint64_t)b); }
int64_t wrap_mul(int64_t a, int64_t b) { return (int64_t)((uint64_t)a * (uint64_t)b); }

int64_t floor_div(int64_t a, int64_t d) {
  int64_t q = a / d;
  if ((a % d) != 0 && a < 0) q -= 1;
  return q;
}
int64_t euclid_mod(int64_t a, int64_t d) {
  int64_t r = a % d;
  if (r < 0) r += d;
  return r;
}

int64_t eval(const Expr& e, int n, const Env& env) {
  const Node& x = e.nodes[n];
  switch (x.op) {
    case C_CONST: return x.v;
    case C_TID: return env.tid[x.v];
    case C_BID: return env.bid[x.v];
    case C_PARAM:
      if (x.v < 0 || x.v >= (int64_t)env.params->size()) throw std::runtime_error("bad parameter");
      return (*env.params)[x.v];
    case C_ITER: return env.iter[x.v];
    case C_ADD: return wrap_add(eval(e, x.a, env), eval(e, x.b, env));
    case C_MUL: return wrap_mul(x.v, eval(e, x.a, env));
    case C_FDIV: return floor_div(eval(e, x.a, env), x.v);
    case C_MOD: return euclid_mod(eval(e, x.a, env), x.v);
    case C_LOAD: {
      // a table reads as 0 outside its values
      const std::vector<int64_t>& t = (*env.tables)[x.v];
      const int64_t i = eval(e, x.a, env);
      return (i < 0 || i >= (int64_t)t.size()) ? 0 : t[i];
    }
    case C_FREE: return env.free[x.v];
  }
  return 0;
}
int64_t eval(const Expr& e, const Env& env) { return eval(e, e.root, env); }

// ----------------------------------------------------------------------------
// instances
// ----------------------------------------------------------------------------
struct Inst {
  int64_t a, s, e, b, p, t, k, w;
  bool operator<(const Inst& o) const {
    if (a != o.a) return a < o.a;
    if (s != o.s) return s < o.s;
    if (e != o.e) return e < o.e;
    if (b != o.b) return b < o.b;
    if (p != o.p) return p < o.p;
    if (t != o.t) return t < o.t;
    if (k != o.k) return k < o.k;
    return w < o.w;
  }
  bool operator==(const Inst& o) const {
    return a == o.a && s == o.s && e == o.e && b == o.b && p == o.p && t == o.t && k == o.k && w == o.w;
  }
  bool same_cell(const Inst& o) const { return a == o.a && s == o.s && e == o.e; }
};

struct OobRecord {
  bool any = false;
  int64_t stmt = 0, access = 0, gtid = 0, dimcode = 0;
  void offer(int64_t st, int64_t ac, int64_t g, int64_t dc) {
    if (!any || std::make_tuple(st, ac, g, dc) < std::make_tuple(stmt, access, gtid, dimcode)) {
      any = true; stmt = st; access = ac; gtid = g; dimcode = dc;
    }
  }
};

// Linear cell number used only to select a range of cells (chunked mode):
// arrays in order, then scope instance, then element.
struct CellRange {
  bool all = true;
  int64_t lo = 0, hi = 0;
  // hash part (part_count = 2^p > 1): the cells whose part, by the definition
  // of the check options, (((cell * 0x9E3779B97F4A7C15) mod 2^cb) * 2^p) >> cb
  // with cb = bit_length(number of cells), is part_index
  uint64_t part_count = 0, part_index = 0;
  uint32_t cb = 0;
};

struct Enumerator {
  const Model& m;
  CellRange range;
  std::vector<int64_t> cell_base, cell_size;   // per array
  std::vector<Inst> out;
  uint64_t enumerated = 0;
  OobRecord oob;

  Enumerator(const Model& mm, CellRange r) : m(mm), range(r) {
    int64_t nblocks = m.grid[0] * m.grid[1] * m.grid[2];
    int64_t base = 0;
    for (const Array& a : m.arrays) {
      int64_t sz = 1;
      for (int64_t e : a.ext) sz *= e;
      cell_base.push_back(base);
      cell_size.push_back(sz);
      base += sz * (a.shared ? nblocks : 1);
    }
  }

  void emit(int64_t si, const Stmt& st, Env& env, int64_t b, int64_t t, int64_t gtid) {
    int64_t phase = eval(st.phase, env);
    const int64_t wphase = st.wphase.root < 0 ? 0 : eval(st.wphase, env);
    for (size_t ai = 0; ai < st.accesses.size(); ++ai) {
      const Access& ac = st.accesses[ai];
      const Array& arr = m.arrays[ac.array];
      enumerated++;
      bool bad = false;
      // an interval outside its range (block or warp interval) has dimcode 0
      if (phase < 0 || phase >= m.n_phases || wphase < 0 || wphase >= m.n_wphases) {
        oob.offer(si, (int64_t)ai, gtid, 0);
        bad = true;
      }
      int64_t e = 0;
      for (size_t d = 0; d < ac.index.size(); ++d) {
        int64_t v = eval(ac.index[d], env);
        if (v < 0 || v >= arr.ext[d]) { oob.offer(si, (int64_t)ai, gtid, (int64_t)d + 1); bad = true; }
        e = e * arr.ext[d] + v;
      }
      if (bad) continue;
      Inst x;
      x.a = ac.array;
      x.s = arr.shared ? b : 0;
      x.e = e;
      x.b = b;
      x.p = phase;
      x.t = t;
      x.k = ac.kind;
      x.w = wphase;
      if (!range.all) {
        int64_t lin = cell_base[x.a] + x.s * cell_size[x.a] + x.e;
        if (lin < range.lo || lin >= range.hi) continue;
        if (range.part_count > 1) {
          uint32_t p = 0;
          while ((1ull << p) < range.part_count) ++p;
          uint64_t hsh = (uint64_t)lin * 0x9E3779B97F4A7C15ull;
          if (range.cb < 64) hsh &= (1ull << range.cb) - 1ull;
          const uint64_t part = p <= range.cb ? hsh >> (range.cb - p) : hsh << (p - range.cb);
          if (part != range.part_index) continue;
        }
      }
      out.push_back(x);
    }
  }

  void loops(int64_t si, const Stmt& st, size_t level, Env& env, int64_t b, int64_t t, int64_t gtid) {
    if (level == st.loops.size()) {
      for (const Expr& g : st.guards)
        if (eval(g, env) < 0) return;
      emit(si, st, env, b, t, gtid);
      return;
    }
    const Loop& lp = st.loops[level];
    int64_t lo = eval(lp.lower, env), hi = eval(lp.upper, env);
    for (int64_t v = lo; v < hi; v += lp.step) {
      env.iter[level] = v;
      loops(si, st, level + 1, env, b, t, gtid);
    }
  }

  // every value of every free parameter, then the loop nest
  void frees(int64_t si, const Stmt& st, size_t k, Env& env, int64_t b, int64_t t, int64_t gtid) {
    if (k == st.free_lo.size()) {
      loops(si, st, 0, env, b, t, gtid);
      return;
    }
    for (int64_t v = st.free_lo[k]; v <= st.free_hi[k]; ++v) {
      env.free[k] = v;
      frees(si, st, k + 1, env, b, t, gtid);
    }
  }

  void run() {
    const int64_t bsize = m.block[0] * m.block[1] * m.block[2];
    Env env;
    env.params = &m.params;
    env.tables = &m.tables;
    for (int64_t bz = 0; bz < m.grid[2]; ++bz)
      for (int64_t by = 0; by < m.grid[1]; ++by)
        for (int64_t bx = 0; bx < m.grid[0]; ++bx) {
          const int64_t b = bx + m.grid[0] * (by + m.grid[1] * bz);
          env.bid[0] = bx; env.bid[1] = by; env.bid[2] = bz;
          for (int64_t tz = 0; tz < m.block[2]; ++tz)
            for (int64_t ty = 0; ty < m.block[1]; ++ty)
              for (int64_t tx = 0; tx < m.block[0]; ++tx) {
                const int64_t t = tx + m.block[0] * (ty + m.block[1] * tz);
                env.tid[0] = tx; env.tid[1] = ty; env.tid[2] = tz;
                for (size_t si = 0; si < m.stmts.size(); ++si)
                  frees((int64_t)si, m.stmts[si], 0, env, b, t, b * bsize + t);
              }
        }
  }
};

// ----------------------------------------------------------------------------
// result record (all fields int64, see oracle/__init__.py for the names)
// ----------------------------------------------------------------------------
enum {
  F_STATUS, F_VERDICT, F_RACY_CELLS, F_INSTANCES, F_DISTINCT,
  F_W_ARRAY, F_W_SCOPE, F_W_ADDR,
  F_X_BLOCK, F_X_THREAD, F_X_PHASE, F_X_KIND,
  F_Y_BLOCK, F_Y_THREAD, F_Y_PHASE, F_Y_KIND,
  F_OOB_STMT, F_OOB_ACCESS, F_OOB_GTID, F_OOB_DIM,
  F_X_WPHASE, F_Y_WPHASE,
  F_COUNT
};
enum { ST_OK = 0, ST_INVALID = 1, ST_OOB = 3 };

void put_witness(int64_t* out, const Inst& x, const Inst& y) {
  out[F_W_ARRAY] = x.a; out[F_W_SCOPE] = x.s; out[F_W_ADDR] = x.e;
  out[F_X_BLOCK] = x.b; out[F_X_THREAD] = x.t; out[F_X_PHASE] = x.p; out[F_X_KIND] = x.k;
  out[F_Y_BLOCK] = y.b; out[F_Y_THREAD] = y.t; out[F_Y_PHASE] = y.p; out[F_Y_KIND] = y.k;
  out[F_X_WPHASE] = x.w; out[F_Y_WPHASE] = y.w;
}

enum { K_R = 0, K_W = 1, K_A = 2 };

bool conflict(int64_t kx, int64_t ky) {
  return kx == K_W || ky == K_W || (kx == K_A && ky == K_R) || (kx == K_R && ky == K_A);
}

constexpr int64_t kWarpSize = 32;

// concurrency of two instances of distinct threads (see the header)
bool concurrent(const Inst& x, const Inst& y, const Model& m) {
  if (x.b != y.b) return m.grid_phase[x.p] == m.grid_phase[y.p];
  return x.p == y.p && (x.t / kWarpSize != y.t / kWarpSize || x.w == y.w);
}

bool races(const Inst& x, const Inst& y, int64_t bsize, const Model& m) {
  if (!x.same_cell(y)) return false;
  if (x.b * bsize + x.t == y.b * bsize + y.t) return false;
  if (!conflict(x.k, y.k)) return false;
  return concurrent(x, y, m);
}

// kinds present in a set of instances
struct Kinds {
  bool r = false, w = false, a = false;
  void add(int64_t k) { r |= k == K_R; w |= k == K_W; a |= k == K_A; }
  bool conf() const { return w || (a && r); }
};

// Cell-level test without warp or grid barriers: two blocks and a conflict in
// the cell, or a (b, p) group with two threads and a conflict.
bool cell_racy_plain(const std::vector<Inst>& v, size_t lo, size_t hi) {
  bool two_blocks = false;
  Kinds all;
  for (size_t i = lo; i < hi; ++i) { two_blocks |= v[i].b != v[lo].b; all.add(v[i].k); }
  if (two_blocks && all.conf()) return true;
  // (b, p) groups are contiguous because the instances are sorted by (b, p, t, k)
  size_t g = lo;
  while (g < hi) {
    size_t h = g;
    bool two_threads = false;
    Kinds gk;
    while (h < hi && v[h].b == v[g].b && v[h].p == v[g].p) {
      two_threads |= v[h].t != v[g].t;
      gk.add(v[h].k);
      ++h;
    }
    if (two_threads && gk.conf()) return true;
    g = h;
  }
  return false;
}

bool has_sync_scopes(const Model& m) {
  if (m.n_wphases > 1) return true;
  for (int64_t g : m.grid_phase) if (g != 0) return true;
  return false;
}

// Cell-level test on one cell's sorted, duplicate-free instances [lo, hi).
bool cell_racy(const std::vector<Inst>& v, size_t lo, size_t hi, const Model& m) {
  if (!has_sync_scopes(m)) return cell_racy_plain(v, lo, hi);
  // grid intervals: two blocks and a conflict
  std::map<int64_t, std::set<int64_t>> g_blocks;
  std::map<int64_t, Kinds> g_kinds;
  // (b, p) groups: two warps and a conflict; (b, p, w) groups: two threads and a conflict
  std::map<std::pair<int64_t, int64_t>, std::set<int64_t>> bp_warps;
  std::map<std::pair<int64_t, int64_t>, Kinds> bp_kinds;
  std::map<std::tuple<int64_t, int64_t, int64_t>, std::set<int64_t>> bpw_threads;
  std::map<std::tuple<int64_t, int64_t, int64_t>, Kinds> bpw_kinds;
  for (size_t i = lo; i < hi; ++i) {
    const Inst& x = v[i];
    const int64_t g = m.grid_phase[x.p];
    g_blocks[g].insert(x.b);
    g_kinds[g].add(x.k);
    bp_warps[{x.b, x.p}].insert(x.t / kWarpSize);
    bp_kinds[{x.b, x.p}].add(x.k);
    bpw_threads[std::make_tuple(x.b, x.p, x.w)].insert(x.t);
    bpw_kinds[std::make_tuple(x.b, x.p, x.w)].add(x.k);
  }
  for (auto& kv : g_blocks)
    if (kv.second.size() >= 2 && g_kinds[kv.first].conf()) return true;
  for (auto& kv : bp_warps)
    if (kv.second.size() >= 2 && bp_kinds[kv.first].conf()) return true;
  for (auto& kv : bpw_threads)
    if (kv.second.size() >= 2 && bpw_kinds[kv.first].conf()) return true;
  return false;
}

// Smallest racing pair inside one racy cell [lo, hi).
void cell_witness(const std::vector<Inst>& v, size_t lo, size_t hi, int64_t bsize, const Model& m, Inst& x,
                  Inst& y) {
  const size_t n = hi - lo;
  if (n <= 4096) {
    // by the definition: first x with any partner, then its first partner
    for (size_t i = lo; i < hi; ++i)
      for (size_t j = lo; j < hi; ++j)
        if (races(v[i], v[j], bsize, m)) {
          // v[i] is the smallest instance with a partner; every partner of the
          // smallest participant is larger than it, so the first j found is y.
          x = v[i];
          y = v[j];
          return;
        }
    throw std::runtime_error("cell_witness called on a race-free cell");
  }
  // large cells: decide "x has a partner" from the blocks holding each kind
  // per grid interval and the (thread, warp interval) pairs holding each kind
  // per (b, p) group
  std::map<int64_t, std::set<int64_t>> kblocks[3];
  std::map<std::pair<int64_t, int64_t>, std::set<std::pair<int64_t, int64_t>>> kthreads[3];
  for (size_t i = lo; i < hi; ++i) {
    kblocks[v[i].k][m.grid_phase[v[i].p]].insert(v[i].b);
    kthreads[v[i].k][{v[i].b, v[i].p}].insert({v[i].t, v[i].w});
  }
  for (size_t i = lo; i < hi; ++i) {
    const Inst& c = v[i];
    bool cross = false, same = false;
    for (int k = 0; k < 3; ++k) {
      if (!conflict(c.k, k)) continue;
      // a partner in another block of the same grid interval
      auto bt = kblocks[k].find(m.grid_phase[c.p]);
      if (bt != kblocks[k].end())
        for (int64_t b : bt->second) if (b != c.b) { cross = true; break; }
      // another thread of the (b, p) group in another warp or in the same warp interval
      auto it = kthreads[k].find({c.b, c.p});
      if (it != kthreads[k].end())
        for (const auto& tw : it->second)
          if (tw.first != c.t && (tw.first / kWarpSize != c.t / kWarpSize || tw.second == c.w)) { same = true; break; }
    }
    if (cross || same) {
      x = c;
      for (size_t j = lo; j < hi; ++j)
        if (races(c, v[j], bsize, m)) { y = v[j]; return; }
      throw std::runtime_error("inconsistent partner summary");
    }
  }
  throw std::runtime_error("cell_witness called on a race-free cell");
}

void clear(int64_t* out) { for (int i = 0; i < F_COUNT; ++i) out[i] = 0; }

int check_model(const Model& m, CellRange range, int64_t* out) {
  clear(out);
  Enumerator en(m, range);
  en.run();
  out[F_INSTANCES] = (int64_t)en.enumerated;
  if (en.oob.any) {
    out[F_STATUS] = ST_OOB;
    out[F_OOB_STMT] = en.oob.stmt;
    out[F_OOB_ACCESS] = en.oob.access;
    out[F_OOB_GTID] = en.oob.gtid;
    out[F_OOB_DIM] = en.oob.dimcode;
    return ST_OOB;
  }
  std::vector<Inst>& v = en.out;
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
  out[F_DISTINCT] = (int64_t)v.size();
  const int64_t bsize = m.block[0] * m.block[1] * m.block[2];
  uint64_t racy = 0;
  bool have_witness = false;
  size_t i = 0;
  while (i < v.size()) {
    size_t j = i;
    while (j < v.size() && v[j].same_cell(v[i])) ++j;
    if (cell_racy(v, i, j, m)) {
      racy++;
      if (!have_witness) {
        Inst x{}, y{};
        cell_witness(v, i, j, bsize, m, x, y);
        put_witness(out, x, y);
        have_witness = true;
      }
    }
    i = j;
  }
  out[F_RACY_CELLS] = (int64_t)racy;
  out[F_VERDICT] = racy > 0;
  out[F_STATUS] = ST_OK;
  return ST_OK;
}

}  // namespace

extern "C" {

// Full check of one model given in the oracle's text format.  `out` receives
// F_COUNT int64 fields.  Returns the status (0 ok, 1 invalid text, 3 out of bounds).
int oracle_check(const char* text, int64_t* out) {
  try {
    Parser p(text);
    Model m = p.model();
    return check_model(m, CellRange{}, out);
  } catch (const std::exception&) {
    clear(out);
    out[F_STATUS] = ST_INVALID;
    return ST_INVALID;
  }
}

// Same check restricted to the linear cells [lo, hi) (arrays in order, then
// scope instance, then element): the racy-cell count of the range and the
// smallest racing pair whose cell lies in it.  Instance counts still cover the
// whole model.  Used to bound memory on large models.
int oracle_check_cells(const char* text, int64_t lo, int64_t hi, int64_t* out) {
  try {
    Parser p(text);
    Model m = p.model();
    CellRange r;
    r.all = false; r.lo = lo; r.hi = hi;
    return check_model(m, r, out);
  } catch (const std::exception&) {
    clear(out);
    out[F_STATUS] = ST_INVALID;
    return ST_INVALID;
  }
}

// The same check restricted to the cells of one hash part (the partition of a
// model over ranks by the check options' part_count / part_index).
int oracle_check_part(const char* text, int64_t part_count, int64_t part_index, int64_t* out) {
  try {
    Parser p(text);
    Model m = p.model();
    CellRange r;
    r.all = false;
    r.lo = 0;
    r.hi = INT64_MAX;
    r.part_count = (uint64_t)part_count;
    r.part_index = (uint64_t)part_index;
    // cb: the bits of the number of cells (arrays in order, shared arrays once per block)
    int64_t total = 0;
    const int64_t nblocks = m.grid[0] * m.grid[1] * m.grid[2];
    for (const Array& a : m.arrays) {
      int64_t sz = 1;
      for (int64_t e : a.ext) sz *= e;
      total += sz * (a.shared ? nblocks : 1);
    }
    while (r.cb < 63 && (1ull << r.cb) <= (uint64_t)total) ++r.cb;
    return check_model(m, r, out);
  } catch (const std::exception&) {
    clear(out);
    out[F_STATUS] = ST_INVALID;
    return ST_INVALID;
  }
}

// The same check as oracle_check on n_threads host threads (std::thread): the
// linear cells are cut into n_threads ranges of equal length, each thread runs
// the cell-range check of its range (every thread enumerates the whole model
// and keeps the instances of its own cells), and the partial results merge by
// the decomposition the cell-range check is pinned to: racy cells and distinct
// instances add up (a cell races or not on its own), and the witness is that of
// the lowest range that holds a racy cell (ranges ascend in cell order).
int oracle_check_parallel(const char* text, int n_threads, int64_t* out) {
  try {
    Parser p(text);
    Model m = p.model();
    if (n_threads < 1) n_threads = 1;
    Enumerator en(m, CellRange{});
    const int64_t nblocks = m.grid[0] * m.grid[1] * m.grid[2];
    int64_t total = 0;
    if (!m.arrays.empty()) {
      const size_t last = m.arrays.size() - 1;
      total = en.cell_base[last] + en.cell_size[last] * (m.arrays[last].shared ? nblocks : 1);
    }
    std::vector<std::vector<int64_t>> part(n_threads, std::vector<int64_t>(F_COUNT, 0));
    std::vector<int> status(n_threads, ST_OK);
    std::vector<std::thread> pool;
    const int64_t per = (total + n_threads - 1) / n_threads;
    for (int k = 0; k < n_threads; ++k)
      pool.emplace_back([&, k] {
        try {
          CellRange r;
          r.all = false;
          r.lo = std::min(total, (int64_t)k * per);
          r.hi = std::min(total, r.lo + per);
          status[k] = check_model(m, r, part[k].data());
        } catch (const std::exception&) {
          status[k] = ST_INVALID;
        }
      });
    for (std::thread& t : pool) t.join();
    clear(out);
    for (int k = 0; k < n_threads; ++k)
      if (status[k] != ST_OK) {
        for (int f = 0; f < F_COUNT; ++f) out[f] = part[k][f];
        out[F_STATUS] = status[k];
        return status[k];
      }
    out[F_INSTANCES] = part[0][F_INSTANCES];
    bool have = false;
    for (int k = 0; k < n_threads; ++k) {
      out[F_RACY_CELLS] += part[k][F_RACY_CELLS];
      out[F_DISTINCT] += part[k][F_DISTINCT];
      if (!have && part[k][F_RACY_CELLS] > 0) {
        for (int f = F_W_ARRAY; f < F_COUNT; ++f) out[f] = part[k][f];
        have = true;
      }
    }
    out[F_VERDICT] = out[F_RACY_CELLS] > 0;
    out[F_STATUS] = ST_OK;
    return ST_OK;
  } catch (const std::exception&) {
    clear(out);
    out[F_STATUS] = ST_INVALID;
    return ST_INVALID;
  }
}

// Total number of linear cells of the model (the upper end for oracle_check_cells).
int64_t oracle_cell_count(const char* text) {
  try {
    Parser p(text);
    Model m = p.model();
    Enumerator en(m, CellRange{});
    int64_t nblocks = m.grid[0] * m.grid[1] * m.grid[2];
    if (m.arrays.empty()) return 0;
    size_t last = m.arrays.size() - 1;
    return en.cell_base[last] + en.cell_size[last] * (m.arrays[last].shared ? nblocks : 1);
  } catch (const std::exception&) {
    return -1;
  }
}

// Pairwise check: the racing predicate applied to every pair of distinct
// instances (O(n^2), small models only).  Same output record.
int oracle_brute(const char* text, int64_t* out) {
  try {
    Parser p(text);
    Model m = p.model();
    clear(out);
    Enumerator en(m, CellRange{});
    en.run();
    out[F_INSTANCES] = (int64_t)en.enumerated;
    if (en.oob.any) {
      out[F_STATUS] = ST_OOB;
      out[F_OOB_STMT] = en.oob.stmt; out[F_OOB_ACCESS] = en.oob.access;
      out[F_OOB_GTID] = en.oob.gtid; out[F_OOB_DIM] = en.oob.dimcode;
      return ST_OOB;
    }
    std::vector<Inst> v = en.out;
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    out[F_DISTINCT] = (int64_t)v.size();
    const int64_t bsize = m.block[0] * m.block[1] * m.block[2];
    std::set<std::tuple<int64_t, int64_t, int64_t>> racy_cells;
    bool have = false;
    Inst bx{}, by{};
    for (size_t i = 0; i < v.size(); ++i)
      for (size_t j = i + 1; j < v.size(); ++j)
        if (races(v[i], v[j], bsize, m)) {
          racy_cells.insert(std::make_tuple(v[i].a, v[i].s, v[i].e));
          // v is sorted, so (i, j) pairs come in lexicographic order
          if (!have) { bx = v[i]; by = v[j]; have = true; }
        }
    out[F_RACY_CELLS] = (int64_t)racy_cells.size();
    out[F_VERDICT] = !racy_cells.empty();
    if (have) put_witness(out, bx, by);
    out[F_STATUS] = ST_OK;
    return ST_OK;
  } catch (const std::exception&) {
    clear(out);
    out[F_STATUS] = ST_INVALID;
    return ST_INVALID;
  }
}

// All in-bounds instances, sorted by (a, s, e, b, p, t, k), duplicates kept, as
// 7 int64 per instance.  Returns the number of instances (which may exceed
// `cap`; only the first `cap` are written), or -1 on invalid text.
int64_t oracle_expand(const char* text, int64_t* out, int64_t cap) {
  try {
    Parser p(text);
    Model m = p.model();
    Enumerator en(m, CellRange{});
    en.run();
    std::sort(en.out.begin(), en.out.end());
    int64_t n = (int64_t)en.out.size();
    for (int64_t i = 0; i < n && i < cap; ++i) {
      const Inst& x = en.out[i];
      int64_t* o = out + 7 * i;
      o[0] = x.a; o[1] = x.s; o[2] = x.e; o[3] = x.b; o[4] = x.p; o[5] = x.t; o[6] = x.k;
    }
    return n;
  } catch (const std::exception&) {
    return -1;
  }
}

int oracle_result_fields(void) { return F_COUNT; }

}  // extern "C"
