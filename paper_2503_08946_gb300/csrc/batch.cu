// Batched check: many models in one pipeline.
//
// The models of a batch are checked together instead of one pipeline per
// model.  Every model keeps its own lowered program; the batch gives each model
// its own range of cells, so that the keys of all models can be sorted and
// scanned as one array:
//
//   batch key = [model's first batch cell + cell | phase | block | thread | kind]
//
// with the phase, block and thread fields as wide as the widest model's.  A
// racy cell of the shared scan is charged to the model whose cell range holds
// it, and the witness kernels run once per model (blockIdx.y), on the first
// racy cell of that model.  Models whose combined fields would not fit in 63
// bits go to separate packs, each checked by its own pipeline in turn.
//
// Expansion is one persistent kernel over a work queue: a unit is (model,
// chunk of kExpandThreads threads) with all the model's statements, and blocks
// take units in groups from an atomic counter until the queue is empty.
#include <cuda_runtime.h>

#include "expand_core.cuh"
#include "kernels.h"

namespace rc {

namespace {

constexpr int kUnitsPerGrab = 16;
static_assert(kExpandThreadsHost == kExpandThreads, "host and device chunk sizes agree");

// Keys are re-packed from the model's layout into the batch layout.
struct BatchSink {
  uint64_t* keys;
  uint64_t cell_base;
  uint32_t mcs, mps, mbs, mts;       // model field shifts (thread field at mts = its kind bits)
  uint64_t pm, bm, tm;               // model field masks
  uint32_t bcs, bps, bbs, bts;       // batch field shifts
  __device__ __forceinline__ void put(uint64_t i, uint64_t key, uint64_t) {
    if (key != kSentinel) {
      const uint64_t cell = key >> mcs;
      const uint64_t ph = (key >> mps) & pm, b = (key >> mbs) & bm, t = (key >> mts) & tm;
      key = ((cell_base + cell) << bcs) | (ph << bps) | (b << bbs) | (t << bts) | (key & ((1ull << mts) - 1ull));
    }
    keys[i] = key;
  }
  __device__ __forceinline__ void pad(uint64_t i) { keys[i] = kSentinel; }
};

// LF: every statement of the pack is loop-free -- only the one-point
// expansion is compiled (fewer registers, no row cache: more resident warps)
template <bool LF>
__global__ void __launch_bounds__(kExpandThreads, LF ? 6 : 4) batch_expand_kernel(BatchArgs a) {
  __shared__ int64_t s_tval[kMaxTerms * kExpandThreads];
  __shared__ int64_t s_cache[LF ? 1 : kFastCache * kExpandThreads];
  __shared__ unsigned long long s_u;
  __shared__ uint32_t s_model;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_u = atomicAdd(a.queue, (unsigned long long)kUnitsPerGrab);
      // the model of the grab's first unit (binary search once per grab)
      uint32_t lo = 0, hi = a.n_models;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a.models[mid].unit_base <= s_u) lo = mid;
        else hi = mid;
      }
      s_model = lo;
    }
    __syncthreads();
    const uint64_t u0 = s_u;
    if (u0 >= a.n_units) break;
    const uint64_t u1 = min(a.n_units, u0 + kUnitsPerGrab);
    for (uint64_t u = u0; u < u1; ++u) {
      // the model of unit u: the grab's units are consecutive, so step forward
      if (threadIdx.x == 0) {
        uint32_t m = s_model;
        while (m + 1 < a.n_models && a.models[m + 1].unit_base <= u) ++m;
        s_model = m;
      }
      __syncthreads();
      const uint32_t lo = s_model;
      const BatchModel& B = a.models[lo];
      // one unit = one chunk of kExpandThreads threads of the model, all its statements
      const uint64_t g = (u - B.unit_base) * kExpandThreads + threadIdx.x;
      const DevModel& M = *B.dm;
      DevResult* res = a.res + lo;
      unsigned long long count = 0;
      if (g < B.n_threads) {
        BatchSink sink;
        sink.keys = a.keys + B.key_base;
        sink.cell_base = B.cell_base;
        sink.mcs = B.cell_shift;
        sink.mps = B.phase_shift;
        sink.mbs = B.block_shift;
        sink.mts = B.thread_shift;
        sink.pm = (1ull << B.phase_bits) - 1;
        sink.bm = (1ull << B.block_bits) - 1;
        sink.tm = (1ull << B.thread_bits) - 1;
        sink.bcs = a.cell_shift;
        sink.bps = a.phase_shift;
        sink.bbs = a.block_shift;
        sink.bts = a.thread_shift;
        const ThreadVars tv = thread_vars(M, g);
        for (uint32_t s = 0; s < B.n_stmts; ++s) {
          const DevStmt& S = M.stmts[s];
          if (LF) {
            FastCtx c;
            c.M = B.dm;
            c.S = &S;
            c.tv = tv;
            c.tval = s_tval + threadIdx.x;
            c.cache = s_cache;   // not read: a loop-free statement evaluates its rows where used
            expand_unit_fast<0>(c, s, g, res, count, sink);
          } else if (S.n_loops > kFastLoops) {
            expand_unit_generic(M, s, g, res, count, sink);
          } else {
            FastCtx c;
            c.M = B.dm;
            c.S = &S;
            c.tv = tv;
            c.tval = s_tval + threadIdx.x;
            c.cache = s_cache + threadIdx.x;
            expand_unit_dispatch(c, s, g, res, count, sink);
          }
        }
      }
      count = warp_sum(count);
      if ((threadIdx.x & 31) == 0 && count) atomicAdd(&res->instances, count);
      __syncthreads();   // s_model is rewritten for the next unit
    }
  }
}

// Errors of a pack's shared stages (sort look-back, scan) reach every model.
__global__ void batch_errors_kernel(const DevResult* pack, DevResult* res, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned e = pack->err;
  if (i < n && e) res[i].err |= e;
}

}  // namespace

cudaError_t launch_batch_errors(const DevResult* pack, DevResult* res, uint32_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  batch_errors_kernel<<<(n + 127) / 128, 128, 0, st>>>(pack, res, n);
  return cudaGetLastError();
}

cudaError_t launch_batch_expand(const BatchArgs& a, bool loop_free, cudaStream_t st) {
  if (a.n_units == 0) return cudaSuccess;
  int dev = 0, sms = 152, per_sm = 4;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (loop_free) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_expand_kernel<true>, kExpandThreads, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_expand_kernel<false>, kExpandThreads, 0);
  if (per_sm < 1) per_sm = 1;
  uint64_t grid = (uint64_t)sms * per_sm;
  const uint64_t need = (a.n_units + kUnitsPerGrab - 1) / kUnitsPerGrab;
  if (grid > need) grid = need;
  if (loop_free) batch_expand_kernel<true><<<(unsigned)grid, kExpandThreads, 0, st>>>(a);
  else batch_expand_kernel<false><<<(unsigned)grid, kExpandThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace rc
