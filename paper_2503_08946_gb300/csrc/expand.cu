// K1: expansion of access instances into packed 64-bit keys.
//
// One work unit = (statement, thread).  For a statement whose loops all have
// constant trip counts ("dense") the key of iteration j, access a and thread g
// goes to slot  slot_base + (j * n_key + k) * T + g  (k = the access's key index
// among the accesses to written arrays),  so the 32 lanes of a warp
// (consecutive g) store 32 consecutive keys; guard-false and out-of-bounds
// instances leave the all-ones padding key.  Other statements are first counted
// per unit (expand_count_kernel, run once when the model is created), and then
// write their keys contiguously at the scanned unit offsets.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "expand_core.cuh"
#include "kernels.h"

namespace rc {

namespace cg = cooperative_groups;

namespace {

// Sort-path sink: keys go to their slot; guard-false dense slots get padding,
// and so do keys whose cell lies outside [cell_lo, cell_hi) or outside the
// hash part of a partial check.
struct SlotSink {
  uint64_t* keys;
  uint64_t cell_lo, cell_hi;
  uint64_t pmask, pval;
  __device__ __forceinline__ void put(uint64_t i, uint64_t key, uint64_t cell) {
    const bool part_ok = pmask == 0ull || ((cell * kCellHashMul) & pmask) == pval;
    keys[i] = (cell >= cell_lo && cell < cell_hi && part_ok) ? key : kSentinel;
  }
  __device__ __forceinline__ void pad(uint64_t i) { keys[i] = kSentinel; }
};

// Count pass of a chunked check: keys per bucket of 2^bshift cells of the
// range [lo, lo + span).  The lanes that reach the add together and share the
// bucket add once.
struct CountSink {
  unsigned long long* counts;
  uint64_t lo, span;
  uint32_t bshift;
  __device__ __forceinline__ void put(uint64_t, uint64_t key, uint64_t cell) {
    if (key == kSentinel || cell - lo >= span) return;
    const uint64_t bucket = (cell - lo) >> bshift;
    cg::coalesced_group g = cg::coalesced_threads();
    const uint64_t b0 = g.shfl(bucket, 0);
    if (g.all(bucket == b0)) {
      if (g.thread_rank() == 0) atomicAdd(counts + b0, (unsigned long long)g.size());
    } else {
      atomicAdd(counts + bucket, 1ull);
    }
  }
  __device__ __forceinline__ void pad(uint64_t) {}
};

// Key pass of a chunked check, for one wave of chunks (consecutive chunks
// whose keys fit the workspace together): the key of a cell in a chunk of the
// wave is appended to that chunk's segment with its cell field rebased to the
// chunk start, which fits the field even when the model's cells do not.  The
// chunk of a cell comes from its bucket (chunks are whole buckets).  The lanes
// that append to one chunk together reserve their positions with one atomic
// add; a position past the chunk's segment is not written and flags
// kErrChunkOverflow.
struct RouteSink {
  RouteArgs r;
  unsigned int* err;
  __device__ __forceinline__ void put(uint64_t, uint64_t key, uint64_t cell) {
    if (key == kSentinel) return;
    const uint64_t rel = cell - r.lo;
    if (rel >= r.span) return;
    const uint64_t bk = (rel >> r.bshift) - r.b0;
    if (bk >= r.n_buckets) return;
    const uint32_t k = r.chunk_of[bk];
    if (k == 0xffffffffu) return;
    const uint64_t out = ((cell - r.c_lo[k]) << r.cell_shift) | (key & r.low_mask);
    cg::coalesced_group g = cg::coalesced_threads();
    const uint32_t k0 = g.shfl(k, 0);
    unsigned long long pos;
    if (g.all(k == k0)) {
      unsigned long long base = 0;
      if (g.thread_rank() == 0) base = atomicAdd(r.c_ctr + k0, (unsigned long long)g.size());
      pos = g.shfl(base, 0) + g.thread_rank();
    } else {
      pos = atomicAdd(r.c_ctr + k, 1ull);
    }
    pos += r.c_base[k];
    if (pos < r.c_end[k]) r.keys[pos] = out;
    else atomicOr(err, (unsigned int)kErrChunkOverflow);
  }
  __device__ __forceinline__ void pad(uint64_t) {}
};

// grid: (ceil(T / kExpandThreads), n_stmts); one statement per grid row.
// Statements with at most kFastLoops loops.
template <class Sink>
__global__ void __launch_bounds__(kExpandThreads, 4) expand_kernel(const DevModel* __restrict__ Mp, DevResult* res,
                                                                Sink sink) {
  __shared__ int64_t s_tval[kMaxTerms * kExpandThreads];
  __shared__ int64_t s_cache[kFastCache * kExpandThreads];
  const DevModel& M = *Mp;
  const uint32_t s = blockIdx.y;
  const DevStmt& S = M.stmts[s];
  if (S.n_loops > kFastLoops) return;
  const uint64_t g = (uint64_t)blockIdx.x * kExpandThreads + threadIdx.x;
  unsigned long long count = 0;
  if (g < M.n_threads) {
    FastCtx c;
    c.M = Mp;
    c.S = &S;
    c.tv = thread_vars(M, g);
    c.tval = s_tval + threadIdx.x;
    c.cache = s_cache + threadIdx.x;
    expand_unit_dispatch(c, s, g, res, count, sink);
  }
  count = warp_sum(count);
  if ((threadIdx.x & 31) == 0 && count) atomicAdd(&res->instances, count);
}

// Statements with more than kFastLoops loops: interpreted nest.
template <class Sink>
__global__ void __launch_bounds__(kExpandThreads) expand_generic_kernel(const DevModel* __restrict__ Mp,
                                                                        DevResult* res, Sink sink) {
  const DevModel& M = *Mp;
  const uint32_t s = blockIdx.y;
  if (M.stmts[s].n_loops <= kFastLoops) return;
  const uint64_t g = (uint64_t)blockIdx.x * kExpandThreads + threadIdx.x;
  unsigned long long count = 0;
  if (g < M.n_threads) expand_unit_generic(M, s, g, res, count, sink);
  count = warp_sum(count);
  if ((threadIdx.x & 31) == 0 && count) atomicAdd(&res->instances, count);
}

template <class Sink>
cudaError_t launch_expand_sink(const DevModel* dm, uint32_t n_stmts, uint64_t n_threads, bool has_deep,
                               DevResult* res, const Sink& sink, cudaStream_t st) {
  if (n_stmts == 0 || n_threads == 0) return cudaSuccess;
  const dim3 grid((unsigned)((n_threads + kExpandThreads - 1) / kExpandThreads), n_stmts);
  expand_kernel<Sink><<<grid, kExpandThreads, 0, st>>>(dm, res, sink);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (has_deep) {
    expand_generic_kernel<Sink><<<grid, kExpandThreads, 0, st>>>(dm, res, sink);
    e = cudaGetLastError();
  }
  return e;
}

// Keys per (statement, thread) unit of the statements with thread-dependent trip
// counts: counts[S.slot_base + g] = guard-true points * accesses.
__global__ void __launch_bounds__(256) count_kernel(const DevModel* __restrict__ Mp, uint64_t n_units,
                                                    uint64_t* __restrict__ counts) {
  const DevModel& M = *Mp;
  const uint64_t T = M.n_threads;
  for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < n_units;
       u += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = (uint32_t)(u / T);
    const uint64_t g = u - (uint64_t)s * T;
    const DevStmt& S = M.stmts[s];
    if (S.dense) continue;
    const ThreadVars tv = thread_vars(M, g);
    uint64_t c = 0;
    walk_nest(M, S, tv, [&](const int64_t* it, const int64_t* term) {
      if (guards_hold(M, S, tv, it, term)) c += (uint64_t)S.n_key;
    });
    counts[S.slot_base + g] = c;
  }
}

// ---------------------------------------------------------------------------
// exclusive scan of uint64 counts (three kernels: tile sums, scan of the tile
// sums in one block, tile scans plus base)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t* total) {
  __shared__ uint64_t warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  uint64_t wbase = 0, tot = 0;
  for (int i = 0; i < kScanThreads / 32; ++i) {
    if (i < w) wbase += warp_tot[i];
    tot += warp_tot[i];
  }
  __syncthreads();
  *total = tot;
  return wbase + x - v;
}

__global__ void scan_tile_sums(const uint64_t* __restrict__ in, uint64_t n, uint64_t* __restrict__ sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  uint64_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    uint64_t i = base + (uint64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  uint64_t tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_sums_single(uint64_t* __restrict__ sums, uint64_t n, uint64_t* __restrict__ total_out) {
  // one block: sequential chunks of kScanThreads
  uint64_t carry = 0;
  for (uint64_t base = 0; base < n; base += kScanThreads) {
    uint64_t i = base + threadIdx.x;
    uint64_t v = i < n ? sums[i] : 0;
    uint64_t tot;
    uint64_t ex = block_excl_scan(v, &tot);
    if (i < n) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void scan_tile_apply(const uint64_t* __restrict__ in, uint64_t n, const uint64_t* __restrict__ sums,
                                uint64_t add, uint64_t* __restrict__ out) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint64_t v[kScanItems];
  uint64_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    uint64_t i = base + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  uint64_t tot;
  uint64_t ex = block_excl_scan(s, &tot) + sums[blockIdx.x] + add;
  for (int k = 0; k < kScanItems; ++k) {
    uint64_t i = base + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
}

int grid_for(uint64_t n_units) {
  uint64_t g = (n_units + 255) / 256;
  const uint64_t cap = 152ull * 64;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

cudaError_t launch_expand(const DevModel* dm, uint32_t n_stmts, uint64_t n_threads, bool has_deep, uint64_t* keys,
                          DevResult* res, cudaStream_t st, const CellFilter& cf) {
  return launch_expand_sink(dm, n_stmts, n_threads, has_deep, res, SlotSink{keys, cf.lo, cf.hi, cf.pmask, cf.pval}, st);
}

cudaError_t launch_expand_count(const DevModel* dm, uint32_t n_stmts, uint64_t n_threads, bool has_deep,
                                DevResult* res, unsigned long long* counts, uint64_t lo, uint64_t span,
                                uint32_t bshift, cudaStream_t st) {
  return launch_expand_sink(dm, n_stmts, n_threads, has_deep, res, CountSink{counts, lo, span, bshift}, st);
}

cudaError_t launch_expand_route(const DevModel* dm, uint32_t n_stmts, uint64_t n_threads, bool has_deep,
                                const RouteArgs& r, DevResult* res, cudaStream_t st) {
  return launch_expand_sink(dm, n_stmts, n_threads, has_deep, res, RouteSink{r, &res->err}, st);
}

cudaError_t launch_count(const DevModel* dm, uint64_t n_units, uint64_t* counts, cudaStream_t st) {
  if (n_units == 0) return cudaSuccess;
  count_kernel<<<grid_for(n_units), 256, 0, st>>>(dm, n_units, counts);
  return cudaGetLastError();
}

size_t scan_u64_temp_bytes(uint64_t n) {
  uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  return (size_t)(tiles + 1) * sizeof(uint64_t);
}

cudaError_t scan_u64_exclusive(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t add, uint64_t* temp,
                               uint64_t* total_dev, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, temp);
  scan_sums_single<<<1, kScanThreads, 0, st>>>(temp, tiles, total_dev);
  scan_tile_apply<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, temp, add, out);
  return cudaGetLastError();
}

}  // namespace rc
