// Per-model expansion kernel generated as CUDA C and compiled at run time with
// NVRTC for sm_103a.
//
// The interpreted expansion (expand.cu) reads every coefficient, divisor and
// array constant from the lowered program at every access instance.  For a
// large model the same lowered rows are instead written out as source code:
// each statement becomes a real loop nest with its coefficients, extents and
// divisors as literals, so the compiler folds constants, hoists the
// thread-constant expressions out of the loops and turns floor division and
// modulo by constants into multiply-shift sequences (or masks and shifts for
// powers of two).  The generated kernel writes exactly the keys of the
// interpreted one (same slots, same padding, same out-of-bounds report).
//
// NVRTC and the CUDA driver entry points are resolved at run time (dlopen and
// cudaGetDriverEntryPointByVersion), so the library loads on machines without
// them; rc_model_create then keeps the interpreted expansion.  Compiled
// kernels are cached per device by their source text.
#include <cuda.h>
#include <cuda_runtime_api.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "rc_internal.h"

namespace rc {

namespace {

// ---------------------------------------------------------------------------
// run-time loaded NVRTC and driver entry points
// ---------------------------------------------------------------------------
struct Nvrtc {
  bool ok = false;
  nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*);
  nvrtcResult (*compile)(nvrtcProgram, int, const char* const*);
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t*);
  nvrtcResult (*cubin)(nvrtcProgram, char*);
  nvrtcResult (*destroy)(nvrtcProgram*);
};

struct Driver {
  bool ok = false;
  CUresult (*load)(CUmodule*, const void*);
  CUresult (*get)(CUfunction*, CUmodule, const char*);
  CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, CUstream,
                     void**, void**);
};

std::mutex g_jit_mu;

// The NVRTC entry points, looked up once per process (a function-local static
// is initialised once even when several host threads get here together).
Nvrtc load_nvrtc() {
  Nvrtc n;
  const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                         "/usr/local/cuda/lib64/libnvrtc.so"};
  void* h = nullptr;
  for (const char* nm : names)
    if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
  if (!h) return n;
  n.create = reinterpret_cast<decltype(n.create)>(dlsym(h, "nvrtcCreateProgram"));
  n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(h, "nvrtcCompileProgram"));
  n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
  n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
  n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
  n.ok = n.create && n.compile && n.cubin_size && n.cubin && n.destroy;
  return n;
}
Nvrtc& nvrtc() {
  static Nvrtc n = load_nvrtc();
  return n;
}

Driver load_driver() {
  Driver d;
  auto get = [](const char* sym, void** fn) {
    cudaDriverEntryPointQueryResult q;
    return cudaGetDriverEntryPointByVersion(sym, fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
           q == cudaDriverEntryPointSuccess && *fn != nullptr;
  };
  void *a = nullptr, *b = nullptr, *c = nullptr;
  d.ok = get("cuModuleLoadData", &a) && get("cuModuleGetFunction", &b) && get("cuLaunchKernel", &c);
  d.load = reinterpret_cast<decltype(d.load)>(a);
  d.get = reinterpret_cast<decltype(d.get)>(b);
  d.launch = reinterpret_cast<decltype(d.launch)>(c);
  return d;
}
Driver& driver() {
  static Driver d = load_driver();
  return d;
}

std::map<std::string, void*> g_cache;   // (device, source) -> CUfunction

// ---------------------------------------------------------------------------
// code generation
// ---------------------------------------------------------------------------
std::string lit(int64_t v) {
  if (v == INT64_MIN) return "((long long)0x8000000000000000ull)";
  return "(" + std::to_string(v) + "LL)";
}
std::string ulit(uint64_t v) { return std::to_string(v) + "ull"; }

bool is_pow2(int64_t d) { return d > 0 && (d & (d - 1)) == 0; }
int log2i(int64_t d) {
  int k = 0;
  while ((1ll << k) < d) ++k;
  return k;
}

struct Gen {
  const Model& m;
  bool chunked = false;   // count / route kernel of chunked checks instead of the slot kernel
  const uint8_t* img;
  const DevStmt* stmts;
  const DevAccess* accs;
  const DevArray* arrays;
  const Row* rows;
  const LinTerm* lin;
  const Term* terms;
  std::ostringstream o;

  explicit Gen(const Model& mm) : m(mm), img(mm.program.data()) {
    stmts = reinterpret_cast<const DevStmt*>(img + m.sec_stmts);
    accs = reinterpret_cast<const DevAccess*>(img + m.sec_accs);
    arrays = reinterpret_cast<const DevArray*>(img + m.sec_arrays);
    rows = reinterpret_cast<const Row*>(img + m.sec_rows);
    lin = reinterpret_cast<const LinTerm*>(img + m.sec_lin);
    terms = reinterpret_cast<const Term*>(img + m.sec_terms);
  }

  std::string row(int r) {
    static const char* tv[6] = {"tx", "ty", "tz", "bx", "by", "bz"};
    const Row& R = rows[r];
    std::string e = lit(R.c0);
    for (int i = 0; i < 6; ++i)
      if (R.ct[i]) e += " + " + lit(R.ct[i]) + " * " + tv[i];
    for (int k = 0; k < R.nnz; ++k) {
      const LinTerm& t = lin[R.off + k];
      const std::string v = t.var < kMaxLoops ? "i" + std::to_string(t.var) : "q" + std::to_string(t.var - kMaxLoops);
      e += " + " + lit(t.coef) + " * " + v;
    }
    return "(" + e + ")";
  }

  void emit_terms(const DevStmt& S, int level, const std::string& ind) {
    for (int q = 0; q < S.n_terms; ++q) {
      const Term& T = terms[S.term0 + q];
      if (T.level != level) continue;
      const std::string a = row(T.row);
      std::string v;
      if (T.op == kLoad) {
        const uint64_t* tidx = reinterpret_cast<const uint64_t*>(img + m.sec_tabidx);
        v = "tload_c(tdata, " + ulit(tidx[2 * T.d]) + ", " + ulit(tidx[2 * T.d + 1]) + ", " + a + ")";
      } else if (T.op == kFdiv) {
        v = is_pow2(T.d) ? "(" + a + " >> " + std::to_string(log2i(T.d)) + ")" : "fdiv_c(" + a + ", " + lit(T.d) + ")";
      } else {
        v = is_pow2(T.d) ? "(" + a + " & " + lit(T.d - 1) + ")" : "mod_c(" + a + ", " + lit(T.d) + ")";
      }
      o << ind << "const long long q" << q << " = " << v << ";\n";
    }
  }

  void emit_stmt(uint32_t s) {
    const DevStmt& S = stmts[s];
    const uint64_t T = m.host.n_threads;
    o << "    case " << s << ": {\n";
    if (chunked) {
      // keys go to chunk_put; no slots
    } else if (S.dense) {
      o << "      unsigned long long slot = " << ulit(S.slot_base) << " + g;\n";
    } else {
      o << "      unsigned long long off = unit_offset[" << ulit(S.slot_base) << " + g];\n";
    }
    emit_terms(S, 0, "      ");
    std::string ind = "      ";
    for (int l = 0; l < S.n_loops; ++l) {
      o << ind << "for (long long i" << l << " = " << row(S.row_lower[l]) << "; i" << l << " < " << row(S.row_upper[l])
        << "; i" << l << " += " << lit(S.step[l]) << ") {\n";
      ind += "  ";
      emit_terms(S, l + 1, ind);
    }
    // guards
    std::string gcond = "true";
    for (int gi = 0; gi < S.n_guards; ++gi) gcond += " && " + row(S.guard_row0 + gi) + " >= 0";
    o << ind << "if (" << gcond << ") {\n";
    const std::string in2 = ind + "  ";
    const bool fine = S.row_wphase >= 0 || m.host.n_wphases > 1;
    if (fine) {
      // the fine interval phase * n_wphases + warp phase; -1 if either is out of range
      o << in2 << "const long long ph0 = " << row(S.row_phase) << ";\n";
      o << in2 << "const long long wph = " << (S.row_wphase >= 0 ? row(S.row_wphase) : std::string("0LL")) << ";\n";
      o << in2 << "const long long ph = (ph0 < 0 || ph0 >= " << lit(m.host.n_phases) << " || wph < 0 || wph >= "
        << lit(m.host.n_wphases) << ") ? -1LL : ph0 * " << lit(m.host.n_wphases) << " + wph;\n";
    } else {
      o << in2 << "const long long ph = " << row(S.row_phase) << ";\n";
    }
    for (int a = 0; a < S.n_acc; ++a) {
      const DevAccess& A = accs[S.acc0 + a];
      const DevArray& arr = arrays[A.array];
      o << in2 << "{\n";
      const std::string in3 = in2 + "  ";
      for (int d = 0; d < A.ndims; ++d) o << in3 << "const long long v" << d << " = " << row(A.row0 + d) << ";\n";
      o << in3 << "unsigned dc = 0xFFFFFFFFu;\n";
      o << in3 << "if (ph < 0 || ph >= " << lit(m.host.n_phases * m.host.n_wphases) << ") dc = 0u;\n";
      for (int d = 0; d < A.ndims; ++d)
        o << in3 << "else if (v" << d << " < 0 || v" << d << " >= " << lit(arr.ext[d]) << ") dc = " << d + 1 << "u;\n";
      // row-major element index
      std::string e;
      for (int d = 0; d < A.ndims; ++d) {
        int64_t stride = 1;
        for (int d2 = d + 1; d2 < A.ndims; ++d2) stride *= arr.ext[d2];
        if (!e.empty()) e += " + ";
        e += "v" + std::to_string(d) + " * " + lit(stride);
      }
      std::string cell = ulit(arr.base) + " + (unsigned long long)(" + e + ")";
      if (arr.shared) cell += " + b * " + ulit(arr.cells);
      const uint64_t pack = ((unsigned long long)s << 51) | ((unsigned long long)a << 45);
      if (chunked) {
        // the whole cell goes to the sink beside the key, whose cell field may not hold it
        o << in3 << "unsigned long long key = ~0ull, cl = ~0ull;\n";
        o << in3 << "if (dc != 0xFFFFFFFFu) atomicMin(oob, " << ulit(pack) << " | ((g & 0x3FFFFFFFFFFull) << 3) | dc);\n";
        o << in3 << "else { cl = " << cell << ";\n";
        o << in3 << "  key = (cl << " << m.host.cell_shift << ") | ((unsigned long long)ph << " << m.host.phase_shift
          << ") | low | " << ulit((uint64_t)A.kind) << "; }\n";
        if (A.key_idx < 0) o << in3 << "(void)key; (void)cl;\n";
        else o << in3 << "chunk_put(a, key, cl);\n";
        o << in2 << "}\n";
        continue;
      }
      o << in3 << "unsigned long long key;\n";
      o << in3 << "if (dc != 0xFFFFFFFFu) { atomicMin(oob, " << ulit(pack)
        << " | ((g & 0x3FFFFFFFFFFull) << 3) | dc); key = ~0ull; }\n";
      o << in3 << "else { const unsigned long long cl = " << cell << ";\n";
      o << in3 << "  key = (cl >= cell_lo && cl < cell_hi && (part_mask == 0ull || ((cl * " << ulit(kCellHashMul)
        << ") & part_mask) == part_val)) ? ((cl << " << m.host.cell_shift
        << ") | ((unsigned long long)ph << " << m.host.phase_shift << ") | low | " << ulit((uint64_t)A.kind)
        << ") : ~0ull; }\n";
      if (A.key_idx < 0) {
        o << in3 << "(void)key;\n";   // array never written: checked, no key
      } else {
        // the pass-A histogram of the bucket path, counted as the keys are written
        o << in3 << "if (hist_a != nullptr && key != ~0ull) atomicAdd(&hA[(unsigned)((((key >> "
          << m.host.cell_shift << ") * " << ulit(kCellHashMul) << ") & hmask) >> hsh)], 1u);\n";
        if (S.dense) o << in3 << "keys[slot + " << ulit((uint64_t)A.key_idx * T) << "] = key;\n";
        else o << in3 << "keys[off + " << A.key_idx << "] = key;\n";
      }
      o << in2 << "}\n";
    }
    o << in2 << "cnt += " << S.n_acc << ";\n";
    if (!S.dense && !chunked) o << in2 << "off += " << S.n_key << ";\n";
    o << ind << "}";
    if (chunked) {
      o << "\n";
    } else if (S.dense) {
      o << " else {\n";
      for (int kq = 0; kq < S.n_key; ++kq) o << in2 << "keys[slot + " << ulit((uint64_t)kq * T) << "] = ~0ull;\n";
      o << ind << "}\n";
      o << ind << "slot += " << ulit((uint64_t)S.n_key * T) << ";\n";
    } else {
      o << "\n";
    }
    for (int l = S.n_loops - 1; l >= 0; --l) {
      ind.resize(ind.size() - 2);
      o << ind << "}\n";
    }
    o << "    } break;\n";
  }

  std::string source() {
    const DevModel& h = m.host;
    o << "// generated expansion kernel\n";
    o << "__device__ __forceinline__ long long fdiv_c(long long a, long long d) {\n"
         "  return a >= 0 ? a / d : -1 - (-(a + 1)) / d;\n}\n";
    o << "__device__ __forceinline__ long long mod_c(long long a, long long d) { return a - fdiv_c(a, d) * d; }\n";
    o << "__device__ __forceinline__ long long tload_c(const long long* t, unsigned long long off, "
         "unsigned long long len, long long i) {\n"
         "  return (i < 0 || (unsigned long long)i >= len) ? 0LL : t[off + (unsigned long long)i];\n}\n";
    if (chunked) {
      // same layout as rc::ChunkJitArgs
      o << "struct ChunkJitArgs {\n"
           "  unsigned long long* oob; unsigned long long* inst; const long long* tdata;\n"
           "  int mode; int pad;\n"
           "  unsigned long long* counts; unsigned long long lo, span; unsigned bshift, cell_shift;\n"
           "  unsigned long long* keys; const unsigned* chunk_of; const unsigned long long* c_lo;\n"
           "  const unsigned long long* c_base; const unsigned long long* c_end; unsigned long long* c_ctr;\n"
           "  unsigned long long b0, n_buckets, low_mask; unsigned* err;\n};\n";
      // mode 0: count keys per bucket; mode 1: route keys to their chunk's segment
      o << "__device__ __forceinline__ void chunk_put(const ChunkJitArgs& a, unsigned long long key, "
           "unsigned long long cell) {\n"
           "  if (key == ~0ull) return;\n"
           "  const unsigned long long rel = cell - a.lo;\n"
           "  if (rel >= a.span) return;\n"
           "  const unsigned long long bucket = rel >> a.bshift;\n"
           "  const unsigned lane = threadIdx.x & 31u;\n"
           "  if (a.mode == 0) {\n"
           "    const unsigned act = __activemask();\n"
           "    const int leader = __ffs(act) - 1;\n"
           "    const unsigned long long b0 = __shfl_sync(act, bucket, leader);\n"
           "    if (__all_sync(act, bucket == b0)) {\n"
           "      if ((int)lane == leader) atomicAdd(a.counts + b0, (unsigned long long)__popc(act));\n"
           "    } else {\n"
           "      atomicAdd(a.counts + bucket, 1ull);\n"
           "    }\n"
           "    return;\n"
           "  }\n"
           "  const unsigned long long bk = bucket - a.b0;\n"
           "  if (bk >= a.n_buckets) return;\n"
           "  const unsigned k = a.chunk_of[bk];\n"
           "  if (k == 0xffffffffu) return;\n"
           "  const unsigned long long out = ((cell - a.c_lo[k]) << a.cell_shift) | (key & a.low_mask);\n"
           "  const unsigned act = __activemask();\n"
           "  const int leader = __ffs(act) - 1;\n"
           "  const unsigned k0 = __shfl_sync(act, k, leader);\n"
           "  unsigned long long pos;\n"
           "  if (__all_sync(act, k == k0)) {\n"
           "    unsigned long long base = 0;\n"
           "    if ((int)lane == leader) base = atomicAdd(a.c_ctr + k0, (unsigned long long)__popc(act));\n"
           "    pos = __shfl_sync(act, base, leader) + __popc(act & ((1u << lane) - 1u));\n"
           "  } else {\n"
           "    pos = atomicAdd(a.c_ctr + k, 1ull);\n"
           "  }\n"
           "  pos += a.c_base[k];\n"
           "  if (pos < a.c_end[k]) a.keys[pos] = out;\n"
           "  else atomicOr(a.err, " + std::to_string((unsigned)kErrChunkOverflow) + "u);\n"
           "}\n";
      o << "extern \"C\" __global__ void __launch_bounds__(128) rc_chunk_jit(const ChunkJitArgs a) {\n";
      o << "  unsigned long long* oob = a.oob;\n  const long long* tdata = a.tdata;\n  (void)tdata;\n";
    } else {
      // hist_a: the bucket path's pass-A digit counts (null: not counted here);
      // each block expands `units` consecutive 128-thread units of its
      // statement, so that its shared histogram is flushed once for them all
      o << "extern \"C\" __global__ void __launch_bounds__(128) rc_expand_jit(unsigned long long* __restrict__ keys, "
           "unsigned long long* oob, unsigned long long* inst, const unsigned long long* __restrict__ unit_offset, "
           "unsigned long long cell_lo, unsigned long long cell_hi, unsigned long long part_mask, unsigned long long part_val, "
           "const long long* __restrict__ tdata, "
           "unsigned long long* hist_a, unsigned long long hmask, unsigned hsh, unsigned hbins, unsigned units) {\n";
      o << "  __shared__ unsigned hA[" << kBucketMaxHistBins << "];\n";
      o << "  if (hist_a != nullptr) {\n"
           "    for (unsigned i = threadIdx.x; i < hbins; i += 128u) hA[i] = 0u;\n"
           "    __syncthreads();\n  }\n";
    }
    o << "  unsigned long long cnt = 0;\n";
    if (!chunked) o << "  for (unsigned u = 0; u < units; ++u) {\n";
    o << "  const unsigned long long g = " << (chunked ? "(unsigned long long)blockIdx.x" :
                                                   "((unsigned long long)blockIdx.x * units + u)")
      << " * 128ull + threadIdx.x;\n";
    o << "  if (g < " << ulit(h.n_threads) << ") {\n";
    o << "    const unsigned long long b = g / " << ulit(h.bs) << ";\n";
    o << "    const unsigned t = (unsigned)(g - b * " << ulit(h.bs) << ");\n";
    o << "    const long long tx = t % " << h.block[0] << "u, ty = (t / " << h.block[0] << "u) % " << h.block[1]
      << "u, tz = t / " << (uint64_t)h.block[0] * h.block[1] << "u;\n";
    o << "    const long long bx = (long long)(b % " << ulit(h.grid[0]) << "), by = (long long)((b / " << ulit(h.grid[0])
      << ") % " << ulit(h.grid[1]) << "), bz = (long long)(b / " << ulit((uint64_t)h.grid[0] * h.grid[1]) << ");\n";
    o << "    (void)tx; (void)ty; (void)tz; (void)bx; (void)by; (void)bz;\n";
    o << "    const unsigned long long low = (b << " << h.block_shift << ") | ((unsigned long long)t << "
      << h.thread_shift << ");\n";
    o << "    switch (blockIdx.y) {\n";
    for (uint32_t s = 0; s < h.n_stmts; ++s) emit_stmt(s);
    o << "    default: break;\n    }\n  }\n";
    if (!chunked) o << "  }\n";
    o << "  for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);\n";
    o << "  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(" << (chunked ? "a.inst" : "inst") << ", cnt);\n";
    if (!chunked)
      o << "  if (hist_a != nullptr) {\n"
           "    __syncthreads();\n"
           "    for (unsigned i = threadIdx.x; i < hbins; i += 128u)\n"
           "      if (hA[i]) atomicAdd(&hist_a[i], (unsigned long long)hA[i]);\n  }\n";
    o << "}\n";
    return o.str();
  }
};

}  // namespace

std::string jit_expand_source(const Model& m) {
  Gen g(m);
  return g.source();
}

std::string jit_chunk_source(const Model& m) {
  Gen g(m);
  g.chunked = true;
  return g.source();
}

namespace {

// Compile `src` for the current device (or fetch it from the cache) and return
// its kernel `name`, or null if NVRTC, the driver or the compile fails.
void* jit_compile(const std::string& src, const char* name) {
  std::lock_guard<std::mutex> lk(g_jit_mu);
  Nvrtc& nv = nvrtc();
  Driver& dr = driver();
  if (!nv.ok || !dr.ok) return nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  const std::string key = std::to_string(dev) + "\n" + name + "\n" + src;
  auto it = g_cache.find(key);
  if (it != g_cache.end()) return it->second;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return nullptr;
  const std::string arch = "--gpu-architecture=sm_" + std::to_string(prop.major) + std::to_string(prop.minor) + "a";
  nvrtcProgram prog;
  if (nv.create(&prog, src.c_str(), "rc_expand_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) return nullptr;
  const char* opts[] = {arch.c_str(), "--std=c++17"};
  bool ok = nv.compile(prog, 2, opts) == NVRTC_SUCCESS;
  std::vector<char> cubin;
  if (ok) {
    size_t n = 0;
    ok = nv.cubin_size(prog, &n) == NVRTC_SUCCESS && n > 0;
    if (ok) {
      cubin.resize(n);
      ok = nv.cubin(prog, cubin.data()) == NVRTC_SUCCESS;
    }
  }
  nv.destroy(&prog);
  if (!ok) return nullptr;
  CUmodule mod;
  CUfunction fn;
  if (dr.load(&mod, cubin.data()) != CUDA_SUCCESS) return nullptr;
  if (dr.get(&fn, mod, name) != CUDA_SUCCESS) return nullptr;
  g_cache[key] = reinterpret_cast<void*>(fn);
  return reinterpret_cast<void*>(fn);
}

// RC_JIT=0 disables generated kernels, RC_JIT=1 forces them for every model
bool jit_wanted(const Model& m) {
  const char* env = std::getenv("RC_JIT");
  if (env && env[0] == '0') return false;
  const bool force = env && env[0] == '1';
  if (!force && m.key_slots < kJitMinKeys) return false;
  return m.host.n_stmts != 0 && m.host.n_threads != 0;
}

}  // namespace

// The model's generated kernel: the slot kernel of the ordinary check, or for
// a wide model the count / route kernel of its chunked checks.  Returns false
// (the interpreted kernels stay in use) if NVRTC, the driver or the compile fails.
bool jit_expand_build(Model* m) {
  if (!jit_wanted(*m)) return false;
  if (m->wide) {
    m->jit_chunk_fn = jit_compile(jit_chunk_source(*m), "rc_chunk_jit");
    return m->jit_chunk_fn != nullptr;
  }
  m->jit_fn = jit_compile(jit_expand_source(*m), "rc_expand_jit");
  return m->jit_fn != nullptr;
}

cudaError_t jit_chunk_launch(const Model& m, const ChunkJitArgs& a, cudaStream_t st) {
  Driver& dr = driver();
  CUfunction fn = reinterpret_cast<CUfunction>(m.jit_chunk_fn);
  ChunkJitArgs args = a;
  void* params[] = {&args};
  const unsigned gx = (unsigned)((m.host.n_threads + 127) / 128);
  const CUresult r = dr.launch(fn, gx, m.host.n_stmts, 1, 128, 1, 1, 0, reinterpret_cast<CUstream>(st), params, nullptr);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

cudaError_t jit_expand_launch(const Model& m, uint64_t* keys, DevResult* res, cudaStream_t st, const CellFilter& cf,
                              const ExpandHist* eh) {
  Driver& dr = driver();
  CUfunction fn = reinterpret_cast<CUfunction>(m.jit_fn);
  unsigned long long* oob = &res->oob_code;
  unsigned long long* inst = &res->instances;
  const uint64_t* uo = m.host.unit_offset;
  unsigned long long lo = cf.lo, hi = cf.hi;
  unsigned long long pmask = cf.pmask, pval = cf.pval;
  const int64_t* td = m.host.tdata;
  unsigned long long* hist = eh ? eh->hist : nullptr;
  unsigned long long hmask = eh ? eh->cmask : 0ull;
  unsigned hsh = eh ? eh->shift : 0u, hbins = eh ? eh->bins : 0u;
  if (hbins > (unsigned)kBucketMaxHistBins) return cudaErrorInvalidValue;
  const uint64_t units_total = (m.host.n_threads + 127) / 128;
  // with the histogram, blocks of up to kExpandHistUnits units (one flush per
  // block), as long as the grid keeps about 64 blocks per SM
  uint64_t units = 1;
  if (eh) {
    units = units_total * m.host.n_stmts / (152ull * 64ull);
    units = units < 1 ? 1 : (units > kExpandHistUnits ? kExpandHistUnits : units);
  }
  unsigned units32 = (unsigned)units;
  void* params[] = {&keys, &oob, &inst, &uo, &lo, &hi, &pmask, &pval, &td, &hist, &hmask, &hsh, &hbins, &units32};
  const unsigned gx = (unsigned)((units_total + units - 1) / units);
  const CUresult r = dr.launch(fn, gx, m.host.n_stmts, 1, 128, 1, 1, 0, reinterpret_cast<CUstream>(st), params, nullptr);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

}  // namespace rc
