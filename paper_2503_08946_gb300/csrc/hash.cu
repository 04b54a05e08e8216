// K5: the hash path -- expansion fused with open-addressing hash tables, no key
// materialisation, optional early exit at the first racy cell.
//
// Every access instance (cell, phase, block, thread, kind) updates two
// lock-free tables (linear probing, keys claimed by atomicCAS):
//   group table, keyed by (cell, phase):  word = [gtid0 | R | A | RACY | W | MULTI | VALID]
//   cell table,  keyed by cell:           word = [block0 | R | A | RACY | W | MULTI_B | VALID]
// Words only gain bits, by atomicCAS, so the instance whose CAS first makes a
// group "two threads and a conflict" (MULTI and (W, or A and R)) or a cell "two
// blocks and a conflict" sees that transition, and it alone sets the cell's
// RACY bit with atomicOr and counts the cell.  This is the cell-level form of
// the pair rule (include/rc.h); it gives the same verdict as the sort path, and
// without early exit the same count.  The smallest racy cell is kept with
// atomicMin; its instances are then collected by a filtered re-expansion and
// the K4 witness reductions run on them.
//
// With warp or grid barriers the phase field is a fine interval q, and an
// instance updates three groups of the group table, one per kind of set whose
// members are pairwise concurrent: (cell, q) with the gtid as identity (two
// threads of one fine interval), (cell, grid interval of q) with the block as
// identity (two blocks of one grid interval; tag bit 62), and (cell, block
// interval of q, block) with the warp as identity (two warps of one block in
// one block interval; tag bit 63, only for blocks of more than 32 threads).
// The untagged keys are below 2^62 (the key's cell and phase fields shifted
// down by at least one bit), the grid keys too before their tag, and the warp
// keys below 2^62 before theirs (cell, block interval and block fields of a
// key without its thread and kind fields); none is all ones, as the all-ones
// cell field is never a cell.  The cell table then only holds the RACY bit.
//
// No wait in these kernels depends on another thread: a probe sequence is at
// most the table size, and a CAS loop retries only after another thread
// changed the word, which happens a bounded number of times per word.
#include <cuda_runtime.h>

#include "expand_core.cuh"
#include "kernels.h"

namespace rc {

namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr unsigned long long kValid = 1ull, kMulti = 2ull, kWrite = 4ull, kRacy = 8ull, kAtomic = 16ull,
                             kRead = 32ull;
constexpr int kIdShift = 6;   // identity (gtid or block) above the flags

// two identities and a conflict: a write, or an atomic and a plain read
__device__ __forceinline__ bool word_racy(unsigned long long w) {
  return (w & kMulti) && ((w & kWrite) || ((w & kAtomic) && (w & kRead)));
}

// SplitMix64 finalizer as the table hash (Steele, Lea, Flood 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ int64_t find_slot(unsigned long long* keys, uint64_t mask, uint64_t x,
                                             unsigned int* err) {
  uint64_t h = mix64(x) & mask;
  for (uint64_t probes = 0; probes <= mask; ++probes) {
    const unsigned long long cur = __ldcg(keys + h);
    if (cur == x) return (int64_t)h;
    if (cur == kEmpty) {
      const unsigned long long prev = atomicCAS(keys + h, kEmpty, (unsigned long long)x);
      if (prev == kEmpty || prev == x) return (int64_t)h;
    }
    h = (h + 1) & mask;
  }
  atomicOr(err, (unsigned int)kErrHashFull);
  return -1;
}

// Fold identity `id` and the kind flag kf (kWrite, kAtomic or kRead) into a
// word; true if this call made the word racy (word_racy).
__device__ __forceinline__ bool word_update(unsigned long long* word, uint64_t id, unsigned long long kf) {
  unsigned long long old = __ldcg(word);
  while (true) {
    unsigned long long nw;
    if (!(old & kValid)) nw = kValid | ((unsigned long long)id << kIdShift) | kf;
    else nw = old | (((old >> kIdShift) != id) ? kMulti : 0ull) | kf;
    if (nw == old) return false;
    const unsigned long long prev = atomicCAS(word, old, nw);
    if (prev == old) return word_racy(nw) && !word_racy(old);
    old = prev;
  }
}

struct HashSink {
  const DevModel* M;
  HashArgs h;
  __device__ __forceinline__ void put(uint64_t, uint64_t key, uint64_t cell) {
    if (key == kSentinel) return;
    const DevModel& m = *M;
    if (cell < h.cell_lo || cell >= h.cell_hi) return;
    const uint64_t cp = key >> m.phase_shift;
    const uint64_t b = (key >> m.block_shift) & ((1ull << m.block_bits) - 1ull);
    const uint64_t t = (key >> m.thread_shift) & ((1ull << m.thread_bits) - 1ull);
    // kind field: R = 0, W = 1, A = 2 (thread_shift bits wide)
    const unsigned kd = (unsigned)(key & ((1ull << m.thread_shift) - 1ull));
    const unsigned long long kf = kd == 1u ? kWrite : (kd == 2u ? kAtomic : kRead);
    const int64_t gs = find_slot(h.gkey, h.gmask, cp, &h.res->err);
    const int64_t cs = find_slot(h.ckey, h.cmask, cell, &h.res->err);
    if (gs < 0 || cs < 0) return;
    // group identity: gtid
    const bool bg = word_update(h.gword + gs, b * m.bs + t, kf);
    bool bc;
    if (h.sync) {
      const uint64_t q = cp & ((1ull << m.phase_bits) - 1ull);
      const uint64_t c = (m.sync_tab[0] >> (4 * q)) & 15u, g = (m.sync_tab[1] >> (4 * q)) & 15u;
      const uint64_t cq = cp >> m.phase_bits;   // the cell
      const uint64_t kgrid = (1ull << 62) | (cq << m.phase_bits) | g;
      const int64_t s2 = find_slot(h.gkey, h.gmask, kgrid, &h.res->err);
      if (s2 < 0) return;
      bc = word_update(h.gword + s2, b, kf);
      if (m.bs > 32u) {
        const uint64_t kwarp = (1ull << 63) | ((((cq << m.phase_bits) | c) << m.block_bits) | b);
        const int64_t s3 = find_slot(h.gkey, h.gmask, kwarp, &h.res->err);
        if (s3 < 0) return;
        bc = word_update(h.gword + s3, t >> 5, kf) || bc;
      }
    } else {
      // cell identity: block
      bc = word_update(h.cword + cs, b, kf);
    }
    if (bg || bc) {
      const unsigned long long old = atomicOr(h.cword + cs, kRacy);
      if (!(old & kRacy)) {
        atomicAdd(&h.res->racy_cells, 1ull);
        atomicMin(&h.res->hash_cell, (unsigned long long)cell);
        if (h.early_exit) atomicExch(h.stop, 1u);
      }
    }
  }
  __device__ __forceinline__ void pad(uint64_t) {}
};

// Filtered re-expansion: keys of one cell are appended to a buffer.
struct FilterSink {
  const DevModel* M;
  uint64_t target;
  uint64_t* out;
  unsigned long long* n_out;
  __device__ __forceinline__ void put(uint64_t, uint64_t key, uint64_t cell) {
    if (key == kSentinel || cell != target) return;
    const unsigned long long i = atomicAdd(n_out, 1ull);
    out[i] = key;
  }
  __device__ __forceinline__ void pad(uint64_t) {}
};

template <class Sink>
__device__ __forceinline__ void run_unit(const DevModel* Mp, uint32_t s, uint64_t g, DevResult* res,
                                         unsigned long long& count, Sink& sink, int64_t* s_tval, int64_t* s_cache) {
  const DevModel& M = *Mp;
  const DevStmt& S = M.stmts[s];
  if (S.n_loops <= kFastLoops) {
    FastCtx c;
    c.M = Mp;
    c.S = &S;
    c.tv = thread_vars(M, g);
    c.tval = s_tval + threadIdx.x;
    c.cache = s_cache + threadIdx.x;
    expand_unit_dispatch(c, s, g, res, count, sink);
  } else {
    expand_unit_generic(M, s, g, res, count, sink);
  }
}

// grid (ceil(T / kExpandThreads), n_stmts)
__global__ void __launch_bounds__(kExpandThreads, 4) hash_expand_kernel(const DevModel* __restrict__ Mp, HashArgs h) {
  __shared__ int64_t s_tval[kMaxTerms * kExpandThreads];
  __shared__ int64_t s_cache[kFastCache * kExpandThreads];
  if (h.early_exit && *reinterpret_cast<volatile unsigned int*>(h.stop)) return;
  const uint32_t s = blockIdx.y;
  const uint64_t g = (uint64_t)blockIdx.x * kExpandThreads + threadIdx.x;
  unsigned long long count = 0;
  if (g < Mp->n_threads) {
    HashSink sink{Mp, h};
    run_unit(Mp, s, g, h.res, count, sink, s_tval, s_cache);
  }
  count = warp_sum(count);
  if ((threadIdx.x & 31) == 0 && count) atomicAdd(&h.res->instances, count);
}

__global__ void __launch_bounds__(kExpandThreads, 4) filter_expand_kernel(const DevModel* __restrict__ Mp, HashArgs h) {
  __shared__ int64_t s_tval[kMaxTerms * kExpandThreads];
  __shared__ int64_t s_cache[kFastCache * kExpandThreads];
  const unsigned long long target = h.res->hash_cell;
  if (target == ~0ull) return;
  const uint32_t s = blockIdx.y;
  const uint64_t g = (uint64_t)blockIdx.x * kExpandThreads + threadIdx.x;
  unsigned long long count = 0;   // the instances were counted by the hash pass
  if (g < Mp->n_threads) {
    // bounds errors fold into the same result record again (atomicMin of equal codes)
    FilterSink sink{Mp, target, h.filtered, h.n_filtered};
    run_unit(Mp, s, g, h.res, count, sink, s_tval, s_cache);
  }
}

// Point the witness reductions at the filtered keys of the racy cell.
__global__ void hash_finish_kernel(HashArgs h) {
  if (threadIdx.x == 0) {
    DevResult* r = h.res;
    if (r->hash_cell != ~0ull) {
      r->min_start = 0;
      r->seg_end = *h.n_filtered;
      r->cell = r->hash_cell;
    }
  }
}

}  // namespace

cudaError_t launch_hash(const DevModel* dm, uint32_t n_stmts, uint64_t n_threads, const HashArgs& h,
                        cudaStream_t st) {
  if (n_stmts == 0 || n_threads == 0) return cudaSuccess;
  const dim3 grid((unsigned)((n_threads + kExpandThreads - 1) / kExpandThreads), n_stmts);
  hash_expand_kernel<<<grid, kExpandThreads, 0, st>>>(dm, h);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  filter_expand_kernel<<<grid, kExpandThreads, 0, st>>>(dm, h);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  hash_finish_kernel<<<1, 32, 0, st>>>(h);
  return cudaGetLastError();
}

}  // namespace rc
