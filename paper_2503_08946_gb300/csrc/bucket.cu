// The bucket path of the grouping step: the keys are grouped by cell without a
// stable sort.
//
// The scan of a race check needs the keys of each cell together, in any order
// (its per-cell fold keeps per-barrier-interval masks, so the order of phases,
// blocks and threads inside a cell does not matter).  The cell field is mapped
// by the bijection h(c) = c * kCellHashMul mod 2^cb (an odd multiplier is
// invertible modulo a power of two), which spreads any set of cells evenly over
// the top bits of h, and the keys are moved by their top bits of h:
//   pass A  partition of all keys by the top dA bits of h (padding keys of
//           guard-false slots dropped); tiles claim their output ranges per
//           digit with one atomic add each on per-digit cursors: no look-back;
//   pass B  partition of every A-bucket by the next dB bits, tiles lying inside
//           one A-bucket;
//   local   every bucket (top D = dA + dB bits of h: all keys of its cells, on
//   sort    average kBucketTarget) is counting-sorted by the remaining bits of
//           h in shared memory and written back, so that the keys of every
//           cell are contiguous (the cells are in h order, not in cell order).
// The ordered cell scan (scan.cu) then folds the cells; it needs each cell's
// keys together, in any order, and with `by_cell` keeps the smallest racy cell
// by value (DevResult.hash_cell); bucket_finish points the witness kernels at
// its bucket, whose keys they filter by cell.
#include <cuda_runtime.h>

#include "kernels.h"

namespace rc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint64_t cell_hash_of(uint64_t cell, uint64_t cmask) {
  return (cell * kCellHashMul) & cmask;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned int d = static_cast<unsigned int>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned int d = static_cast<unsigned int>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One bulk copy global -> shared memory (the TMA engine; 16-byte aligned
// addresses, a size that is a multiple of 16) completing on an mbarrier.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
// the wait for a bulk copy, bounded: on running out the error word is flagged
// and the copy still in flight is waited for once more (bounded again) before
// the block goes on
constexpr unsigned kBulkWaitTries = 1u << 20;
__device__ __forceinline__ void mbar_wait_bounded(unsigned long long* bar, unsigned parity, unsigned int* err) {
  for (unsigned i = 0; i < kBulkWaitTries; ++i)
    if (mbar_try_wait(bar, parity)) return;
  atomicOr(err, (unsigned int)kErrCopyTimeout);
  for (unsigned i = 0; i < kBulkWaitTries; ++i)
    if (mbar_try_wait(bar, parity)) return;
}
// pass-B tiles by one bulk copy (pass B's tiles start at any key position; pass A's
// start at even ones, where 16-byte cp.async per thread measured a little faster)
constexpr bool kPartBulkCopy = true;

// ---------------------------------------------------------------------------
// pass-A histogram: valid keys per top-dA-bit digit of h
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) bucket_hist_a_kernel(BucketArgs a) {
  __shared__ unsigned h[1 << kBucketMaxDigitBits];
  const unsigned nd = 1u << a.dA;
  const uint32_t sh = a.cb - a.dA;
  for (unsigned i = threadIdx.x; i < nd; i += blockDim.x) h[i] = 0;
  __syncthreads();
  auto count = [&](uint64_t k) {
    if (k != kSentinel) atomicAdd(&h[(unsigned)(cell_hash_of(k >> a.cell_shift, a.cmask) >> sh)], 1u);
  };
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if ((reinterpret_cast<uintptr_t>(a.keys_in) & 15u) == 0u) {
    const uint64_t np = a.n / 2;
    const ulonglong2* kp = reinterpret_cast<const ulonglong2*>(a.keys_in);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < np; i += stride) {
      const ulonglong2 k = __ldg(kp + i);
      count(k.x);
      count(k.y);
    }
    if ((a.n & 1u) && blockIdx.x == 0 && threadIdx.x == 0) count(__ldg(a.keys_in + a.n - 1));
  } else {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n; i += stride) count(__ldg(a.keys_in + i));
  }
  __syncthreads();
  for (unsigned d = threadIdx.x; d < nd; d += blockDim.x)
    if (h[d]) atomicAdd(&a.hist_a[d], (unsigned long long)h[d]);
}

// Exclusive scan by 1024 threads of one value per thread (block-wide); returns
// the thread's exclusive prefix and sets *total.
__device__ __forceinline__ unsigned long long block_excl_1024(unsigned long long v, unsigned long long* total) {
  __shared__ unsigned long long wsum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned long long s = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s += y;
    }
    wsum[lane] = s;   // inclusive over warps
  }
  __syncthreads();
  const unsigned long long before = w ? wsum[w - 1] : 0ull;
  *total = wsum[31];
  __syncthreads();
  return before + x - v;
}

// A-bucket offsets and cursors, the tile prefixes of pass B and of its
// histogram, and (one partition pass) the bucket offsets of the fold
__global__ void __launch_bounds__(1024) bucket_scan_a_kernel(BucketArgs a) {
  const unsigned nd = 1u << a.dA;
  const unsigned d = threadIdx.x;
  const unsigned long long c = d < nd ? a.hist_a[d] : 0ull;
  const unsigned long long tb = (c + kPartTileHost - 1) / kPartTileHost;
  const unsigned long long th = (c + kBucketHistTile - 1) / kBucketHistTile;
  unsigned long long tot_c, tot_b, tot_h;
  const unsigned long long ec = block_excl_1024(c, &tot_c);
  const unsigned long long eb = block_excl_1024(tb, &tot_b);
  const unsigned long long eh = block_excl_1024(th, &tot_h);
  if (d < nd) {
    a.off_a[d] = ec;
    a.cur_a[d] = ec;
    a.tpref_b[d] = eb;
    a.tpref_h[d] = eh;
    if (a.dB == 0) a.boff[d] = ec;
  }
  if (d == 0) {
    a.off_a[nd] = tot_c;
    a.tpref_b[nd] = tot_b;
    a.tpref_h[nd] = tot_h;
    if (a.dB == 0) a.boff[nd] = tot_c;
  }
}

__global__ void bucket_whole_kernel(unsigned long long* boff, uint64_t n) {
  boff[0] = 0;
  boff[1] = n;
}

// ---------------------------------------------------------------------------
// partition passes (unstable: equal digits in any order).  Per tile of
// kPTile keys: ranks from one shared atomic per key (one per warp when the
// warp holds one digit), per-digit output ranges claimed from the cursors,
// keys staged in digit order in shared memory, then stored so that the keys
// of one digit go to consecutive addresses.
//   B = false: pass A over all keys (tile t = keys [t * kPTile, ...)), digit =
//              top dA bits of h, padding keys dropped;
//   B = true:  pass B, tiles inside one A-bucket (tpref_b), digit = next dB
//              bits, cursors of that A-bucket's buckets.
// ---------------------------------------------------------------------------
constexpr int kPThreads = kSortThreads;
constexpr int kPItems = 16;
constexpr int kPTile = kPThreads * kPItems;
static_assert(kPTile == kPartTileHost, "pass-B tiles are planned with the host's tile size");
// pass-B tiles per pass-B histogram tile (the histogram writes their A-bucket)
constexpr int kHistPassTiles = kBucketHistTile / kPTile;
static_assert(kHistPassTiles * kPTile == kBucketHistTile && kHistPassTiles <= 256, "whole pass-B tiles per histogram tile");

template <int RB>
constexpr size_t bpart_smem() {
  return (size_t)(kPTile + 2) * 8 + (size_t)(1 << RB) * (4 + 4 + 8);
}

// H32: the cell field has at most 32 bits, so h is computed in 32-bit
// arithmetic (the product modulo 2^cb depends only on the low 32 bits of each
// factor).
// 4 blocks per SM, without spills (5 blocks, 48 registers, spill in both passes)
template <int RB, bool B, bool H32>
__global__ void __launch_bounds__(kPThreads, 4) bucket_partition_kernel(BucketArgs a) {
  constexpr int R = 1 << RB;
  constexpr int DPT = (R + kPThreads - 1) / kPThreads;
  constexpr int kWarps = kPThreads / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(smem);                            // [kPTile + 2]
  unsigned int* cnt = reinterpret_cast<unsigned int*>(s_keys + kPTile + 2);       // [R]
  unsigned int* excl = cnt + R;                                                     // [R]
  unsigned long long* delta = reinterpret_cast<unsigned long long*>(excl + R);      // [R]
  __shared__ unsigned int s_wt[kWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;

  // tile geometry (block-uniform)
  uint64_t t0, len;
  unsigned long long* cursor;
  uint32_t sh, dbits;
  if (!B) {
    t0 = (uint64_t)blockIdx.x * kPTile;
    if (t0 >= a.n) return;
    len = min((uint64_t)kPTile, a.n - t0);
    cursor = a.cur_a;
    sh = a.cb - a.dA;
    dbits = a.dA;
  } else {
    const unsigned nd = 1u << a.dA;
    const uint64_t t = blockIdx.x;
    if (t >= a.tpref_b[nd]) return;
    const uint32_t d1 = a.tile_a[t];
    // (every entry below tpref_b[nd] was written by the histogram of this check)
    if (d1 >= nd) {
      if (threadIdx.x == 0) atomicOr(a.err, (unsigned int)kErrSortRange);
      return;
    }
    t0 = a.off_a[d1] + (t - a.tpref_b[d1]) * kPTile;
    len = min((uint64_t)kPTile, (uint64_t)(a.off_a[d1 + 1] - t0));
    cursor = a.cur_b + ((uint64_t)d1 << a.dB);
    sh = a.cb - a.dA - a.dB;
    dbits = a.dB;
  }
  const unsigned dmask = (1u << dbits) - 1u;
  const uint32_t cs = a.cell_shift;
  auto digit = [&](uint64_t k) -> unsigned {
    if constexpr (H32) return (((uint32_t)(k >> cs) * (uint32_t)kCellHashMul) >> sh) & dmask;
    return (unsigned)(cell_hash_of(k >> cs, a.cmask) >> sh) & dmask;
  };

  for (int i = threadIdx.x; i < R; i += kPThreads) cnt[i] = 0;
  // the tile into shared memory by 16-byte copies where it can be: a full tile
  // of a 16-byte aligned buffer at an even key position, or at an odd one
  // widened by a key on each side (kept inside the buffer: the key after the
  // tile exists); else 8-byte copies.  Key j of the tile is s_keys[off + j].
  const bool full = len == (uint64_t)kPTile;
  const bool al16 = (reinterpret_cast<uintptr_t>(a.keys_in) & 15u) == 0u;
  int off = 0;
  __shared__ __align__(8) unsigned long long s_bar;
  if (kPartBulkCopy && B && full && al16 && ((t0 & 1u) == 0u || t0 + kPTile < a.n)) {
    // one bulk copy by the TMA engine (the widened tile for an odd start)
    off = (int)(t0 & 1u);
    if (threadIdx.x == 0) {
      mbar_init(&s_bar, 1u);
      bulk_load(s_keys, a.keys_in + (t0 - (uint64_t)off), (unsigned)((kPTile + 2 * off) * 8), &s_bar);
    }
    __syncthreads();   // the barrier is initialised before anyone waits on it
    mbar_wait_bounded(&s_bar, 0u, a.err);
  } else if (full && al16 && (t0 & 1u) == 0u) {
#pragma unroll
    for (int m = 0; m < kPTile / 2 / kPThreads; ++m) {
      const int j = m * kPThreads + (int)threadIdx.x;
      cp_async16(s_keys + 2 * j, a.keys_in + t0 + 2 * j);
    }
  } else if (full && al16 && t0 + kPTile < a.n) {
    off = 1;
    for (int j = threadIdx.x; j < kPTile / 2 + 1; j += kPThreads)
      cp_async16(s_keys + 2 * j, a.keys_in + (t0 - 1) + 2 * j);
  } else {
    for (int j = threadIdx.x; j < (int)len; j += kPThreads) cp_async8(s_keys + j, a.keys_in + t0 + j);
  }
  cp_async_wait_all();
  __syncthreads();

  const int lpos = w * (32 * kPItems) + lane;
  unsigned short r[kPItems];   // rank inside the digit (0xffff: no key)
#pragma unroll
  for (int i = 0; i < kPItems; ++i) {
    const int j = lpos + i * 32;
    const uint64_t k = j < (int)len ? s_keys[off + j] : kSentinel;
    const bool valid = j < (int)len && (B || k != kSentinel);
    const unsigned d = valid ? digit(k) : 0u;
    const unsigned d0 = __shfl_sync(FULL, d, 0);
    unsigned rank = 0;
    if (__all_sync(FULL, valid && d == d0)) {
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(&cnt[d0], 32u);
      rank = __shfl_sync(FULL, base, 0) + (unsigned)lane;
    } else if (valid) {
      rank = atomicAdd(&cnt[d], 1u);
    }
    r[i] = valid ? (unsigned short)rank : (unsigned short)0xffffu;
  }
  __syncthreads();
  // per digit: claim the output range, tile offsets
  unsigned carry = 0;
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    const int dg = q * kPThreads + threadIdx.x;
    const unsigned c = dg < R ? cnt[dg] : 0u;
    const unsigned long long claim = c ? atomicAdd(&cursor[dg], (unsigned long long)c) : 0ull;
    unsigned x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wt[w] = x;
    __syncthreads();
    unsigned base = carry, tot = 0;
    for (int i = 0; i < kWarps; ++i) {
      if (i < w) base += s_wt[i];
      tot += s_wt[i];
    }
    __syncthreads();
    if (dg < R) {
      const unsigned e = base + x - c;
      excl[dg] = e;
      delta[dg] = claim - e;
    }
    carry += tot;
  }
  __syncthreads();
  uint64_t kk[kPItems];
#pragma unroll
  for (int i = 0; i < kPItems; ++i) {
    const int j = lpos + i * 32;
    kk[i] = j < (int)len ? s_keys[off + j] : kSentinel;
  }
  __syncthreads();   // every key read before any is overwritten
#pragma unroll
  for (int i = 0; i < kPItems; ++i)
    if (r[i] != 0xffffu) s_keys[excl[digit(kk[i])] + r[i]] = kk[i];
  __syncthreads();
  // carry = valid keys of the tile
  for (int pos = threadIdx.x; pos < (int)carry; pos += kPThreads) {
    const uint64_t key = s_keys[pos];
    const unsigned long long dst = delta[digit(key)] + (unsigned long long)pos;
    // in range whenever the histogram and the ranks agree (see sort.cu)
    if (dst < a.n) a.keys_out[dst] = key;
    else atomicOr(a.err, (unsigned int)kErrSortRange);
  }
}

template <int RB, bool B>
cudaError_t launch_bpart_rb(const BucketArgs& a, uint64_t grid, cudaStream_t st) {
  constexpr size_t smem = bpart_smem<RB>();
  const bool h32 = a.cb <= 32;
  const void* fn = h32 ? reinterpret_cast<const void*>(bucket_partition_kernel<RB, B, true>)
                       : reinterpret_cast<const void*>(bucket_partition_kernel<RB, B, false>);
  const cudaError_t e = ensure_kernel_smem(fn, smem);
  if (e != cudaSuccess) return e;
  if (h32) bucket_partition_kernel<RB, B, true><<<(unsigned)grid, kPThreads, smem, st>>>(a);
  else bucket_partition_kernel<RB, B, false><<<(unsigned)grid, kPThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <bool B>
cudaError_t launch_bpart(const BucketArgs& a, uint32_t bits, uint64_t grid, cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
  if (grid > 0x7fffffffull) return cudaErrorInvalidValue;
  if (bits <= 7) return launch_bpart_rb<7, B>(a, grid, st);
  if (bits == 8) return launch_bpart_rb<8, B>(a, grid, st);
  if (bits == 9) return launch_bpart_rb<9, B>(a, grid, st);
  if (bits == 10) return launch_bpart_rb<10, B>(a, grid, st);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// pass-B histogram: keys per (A-bucket, next dB bits), tiles inside A-buckets
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) bucket_hist_b_kernel(BucketArgs a) {
  __shared__ unsigned h[1 << kBucketMaxDigitBits];
  const unsigned nd = 1u << a.dA, nb = 1u << a.dB;
  const uint64_t t = blockIdx.x;
  if (t >= a.tpref_h[nd]) return;
  uint32_t d1 = 0;
  {
    uint32_t hi = nd;
    while (hi - d1 > 1) {
      const uint32_t mid = (d1 + hi) >> 1;
      if (a.tpref_h[mid] <= t) d1 = mid;
      else hi = mid;
    }
  }
  const uint64_t s = a.off_a[d1] + (t - a.tpref_h[d1]) * kBucketHistTile;
  const uint64_t e = min(s + kBucketHistTile, (uint64_t)a.off_a[d1 + 1]);
  // the A-bucket of the pass-B tiles inside this one (both tilings start at
  // the A-bucket's first key), so that a pass-B block finds it with one load
  if (threadIdx.x < (unsigned)kHistPassTiles) {
    const uint64_t tb = (uint64_t)a.tpref_b[d1] + (t - a.tpref_h[d1]) * kHistPassTiles + threadIdx.x;
    if (tb < a.tpref_b[d1 + 1]) a.tile_a[tb] = d1;
  }
  const uint32_t sh = a.cb - a.dA - a.dB;
  const uint32_t cs = a.cell_shift;
  const bool h32 = a.cb <= 32;
  for (unsigned i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
  __syncthreads();
  auto count = [&](uint64_t k) {
    const unsigned d = h32 ? (((uint32_t)(k >> cs) * (uint32_t)kCellHashMul) >> sh)
                           : (unsigned)(cell_hash_of(k >> cs, a.cmask) >> sh);
    atomicAdd(&h[d & (nb - 1u)], 1u);
  };
  // eight loads of each thread in flight together
  constexpr int kU = 8;
  uint64_t i = s + threadIdx.x;
  for (; i + (kU - 1) * 256 < e; i += kU * 256) {
    uint64_t k[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) k[u] = __ldg(a.keys_in + i + u * 256);
#pragma unroll
    for (int u = 0; u < kU; ++u) count(k[u]);
  }
  for (; i < e; i += 256) count(__ldg(a.keys_in + i));
  __syncthreads();
  for (unsigned d = threadIdx.x; d < nb; d += blockDim.x)
    if (h[d]) atomicAdd(&a.hist_b[((uint64_t)d1 << a.dB) | d], (unsigned long long)h[d]);
}

// ---------------------------------------------------------------------------
// local sort: every bucket put in cell order (by the remaining bits of h)
// ---------------------------------------------------------------------------
constexpr int kLocThreads = 512;
constexpr int kLocKPT = (kFoldCap + kLocThreads - 1) / kLocThreads;   // keys per thread of a bucket in registers

size_t local_smem(uint32_t rbin) { return (size_t)kFoldCap * 8 + ((size_t)8 << rbin); }   // keys, bins, cursors

// Exclusive scan in place of n counters by a block of NT threads (each thread
// a run of consecutive counters, read and written 16 bytes at a time when the
// run is a multiple of 4); *total receives the sum, bin2 (if given) the same
// exclusive prefix (the scatter's cursors).
template <int NT>
__device__ __forceinline__ void bin_scan(unsigned* bin, unsigned n, unsigned* total, unsigned* bin2 = nullptr) {
  static_assert(NT % 32 == 0 && NT <= 1024, "whole warps, at most 32");
  __shared__ unsigned wsum[NT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned per = (n + NT - 1) / NT;
  const unsigned b0 = threadIdx.x * per;
  const bool vec = (per & 3u) == 0u && b0 + per <= n;
  unsigned v[8];
  unsigned s = 0;
  if (vec && per <= 8) {
#pragma unroll
    for (unsigned i = 0; i < 8; i += 4)
      if (i < per) {
        const uint4 x = *reinterpret_cast<const uint4*>(bin + b0 + i);
        v[i] = x.x; v[i + 1] = x.y; v[i + 2] = x.z; v[i + 3] = x.w;
        s += x.x + x.y + x.z + x.w;
      }
  } else {
    for (unsigned i = 0; i < per; ++i)
      if (b0 + i < n) s += bin[b0 + i];
  }
  unsigned x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned t = lane < NT / 32 ? wsum[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(FULL, t, o);
      if (lane >= o) t += y;
    }
    if (lane < NT / 32) wsum[lane] = t;   // inclusive over warps
    if (lane == NT / 32 - 1) *total = t;
  }
  __syncthreads();
  unsigned run = (w ? wsum[w - 1] : 0u) + x - s;
  if (vec && per <= 8) {
#pragma unroll
    for (unsigned i = 0; i < 8; i += 4)
      if (i < per) {
        uint4 o;
        o.x = run; run += v[i];
        o.y = run; run += v[i + 1];
        o.z = run; run += v[i + 2];
        o.w = run; run += v[i + 3];
        *reinterpret_cast<uint4*>(bin + b0 + i) = o;
        if (bin2) *reinterpret_cast<uint4*>(bin2 + b0 + i) = o;
      }
  } else {
    for (unsigned i = 0; i < per; ++i)
      if (b0 + i < n) {
        const unsigned c = bin[b0 + i];
        bin[b0 + i] = run;
        if (bin2) bin2[b0 + i] = run;
        run += c;
      }
  }
}

// Each bucket [boff[b], boff[b+1]) of keys_in is counting-sorted by the rbin
// bits of h below the bucket bits (cells with equal h are equal, so a bin holds
// one cell when rbin == r; otherwise a bin holding several cells is put in cell
// order by insertion sort) and written to the same positions of keys_out.  A
// bucket of at most kFoldCap keys is read once into registers and sorted in
// shared memory; a larger one is read twice and scattered to keys_out.
// Padding keys (the unpartitioned single bucket holds them) are dropped and the
// bucket's tail becomes padding; keys_out behind boff[nb] is left as it is (the
// scan reads up to boff[nb]).  Each thread's key slots past the bucket's length
// are skipped as a block (nq, block-uniform).
// H32: cb <= 32, so h is computed in 32-bit arithmetic (the same value: the
// product modulo 2^cb depends only on the low 32 bits of each factor).
template <bool H32>
__global__ void __launch_bounds__(kLocThreads, 2) bucket_local_sort_kernel(LocalSortArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(smem);
  unsigned* s_bin = reinterpret_cast<unsigned*>(s_keys + kFoldCap);
  const unsigned nbins = 1u << a.rbin;
  const uint32_t bin_shift = a.r - a.rbin;
  const bool multi = a.rbin < a.r;
  const uint32_t cs = a.cell_shift;
  const uint64_t nb = 1ull << a.D;
  const int tid = threadIdx.x;
  __shared__ unsigned s_total;
  auto bin_of = [&](uint64_t k) -> unsigned {
    if constexpr (H32) {
      const uint32_t h = (uint32_t)(k >> cs) * (uint32_t)kCellHashMul;
      return (h >> bin_shift) & (nbins - 1u);
    }
    return (unsigned)(cell_hash_of(k >> cs, a.cmask) >> bin_shift) & (nbins - 1u);
  };
  // bin g's keys after the scatter: [bin_start(g), bin_end(g))
  auto bin_start = [&](unsigned g) { return s_bin[g]; };
  auto bin_end = [&](unsigned g) { return g + 1 < nbins ? s_bin[g + 1] : s_total; };
  // The keys of a bucket that fits in shared memory are held in registers
  // (kLocKPT slots a thread, nq of them used).  The next bucket's loads are
  // issued as soon as the scatter has consumed this one's, so that they are in
  // flight while the sorted bucket is copied out.
  uint64_t kr[kLocKPT];
  uint64_t lo = 0, hi = 0;
  int nq = 0;   // block-uniform; 0 for an empty bucket or one read from global memory
  auto fetch = [&](uint64_t bb) {
    lo = bb < nb ? a.boff[bb] : 0ull;
    hi = bb < nb ? a.boff[bb + 1] : 0ull;
    const uint64_t len = hi > lo ? hi - lo : 0ull;
    nq = len <= (uint64_t)kFoldCap ? (int)((len + kLocThreads - 1) / kLocThreads) : 0;
    const uint64_t* src = a.keys_in + lo;
#pragma unroll
    for (int q = 0; q < kLocKPT; ++q) {
      if (q >= nq) break;
      const unsigned i = (unsigned)q * kLocThreads + (unsigned)tid;
      kr[q] = i < len ? __ldg(src + i) : kSentinel;
    }
  };
  auto clear_bins = [&]() {
    if ((nbins & 3u) == 0u) {
      for (unsigned i = 4 * tid; i < nbins; i += 4 * kLocThreads) *reinterpret_cast<uint4*>(s_bin + i) = make_uint4(0, 0, 0, 0);
    } else {
      for (unsigned i = tid; i < nbins; i += kLocThreads) s_bin[i] = 0;
    }
  };
  clear_bins();
  fetch(blockIdx.x);
  __syncthreads();
  for (uint64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    if (hi <= lo) {
      // empty: the bins stay clear
      fetch(b + gridDim.x);
      continue;
    }
    const uint64_t blo = lo, len = hi - lo;   // (lo and hi move on to the next bucket below)
    const bool in_smem = len <= (uint64_t)kFoldCap;
    const uint64_t* src = a.keys_in + blo;
    uint64_t* out = a.keys_out + blo;
    uint64_t* dst = in_smem ? s_keys : out;
    if (in_smem) {
#pragma unroll
      for (int q = 0; q < kLocKPT; ++q) {
        if (q >= nq) break;
        if (kr[q] != kSentinel) atomicAdd(&s_bin[bin_of(kr[q])], 1u);
      }
      __syncthreads();
      // the scatter cursors: the bins themselves when each holds one cell, else
      // a copy (the starts stay in s_bin for the in-bin ordering below)
      unsigned* cur = multi ? s_bin + nbins : s_bin;
      bin_scan<kLocThreads>(s_bin, nbins, &s_total, multi ? cur : nullptr);
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kLocKPT; ++q) {
        if (q >= nq) break;
        if (kr[q] != kSentinel) s_keys[atomicAdd(&cur[bin_of(kr[q])], 1u)] = kr[q];
      }
    } else {
      // read twice from global memory; the cursors live in the (unused) key buffer
      unsigned* cur = reinterpret_cast<unsigned*>(s_keys);
      for (uint64_t i = tid; i < len; i += kLocThreads) {
        const uint64_t k = src[i];
        if (k != kSentinel) atomicAdd(&s_bin[bin_of(k)], 1u);
      }
      __syncthreads();
      bin_scan<kLocThreads>(s_bin, nbins, &s_total);
      __syncthreads();
      for (unsigned i = tid; i < nbins; i += kLocThreads) cur[i] = s_bin[i];
      __syncthreads();
      for (uint64_t i = tid; i < len; i += kLocThreads) {
        const uint64_t k = src[i];
        if (k != kSentinel) dst[atomicAdd(&cur[bin_of(k)], 1u)] = k;
      }
    }
    __syncthreads();
    const unsigned total = s_total;
    if (multi) {
      for (unsigned g = tid; g < nbins; g += kLocThreads) {
        const unsigned s = bin_start(g), e = bin_end(g);
        bool one = true;
        for (unsigned i = s + 1; i < e && one; ++i) one = (dst[i] >> cs) == (dst[s] >> cs);
        if (one) continue;
        for (unsigned i = s + 1; i < e; ++i) {
          const uint64_t v = dst[i];
          unsigned j = i;
          while (j > s && (dst[j - 1] >> cs) > (v >> cs)) {
            dst[j] = dst[j - 1];
            --j;
          }
          dst[j] = v;
        }
      }
      __syncthreads();
    }
    // the bins are no longer read: the next bucket's loads and the cleared bins
    // go ahead of this bucket's copy out
    fetch(b + gridDim.x);
    clear_bins();
    if (in_smem) {
      // coalesced copy out (16-byte stores where the bucket starts at an even position)
      if ((blo & 1u) == 0u && (reinterpret_cast<uintptr_t>(a.keys_out) & 15u) == 0u) {
        const unsigned np = total / 2;
        for (unsigned i = tid; i < np; i += kLocThreads)
          reinterpret_cast<ulonglong2*>(out)[i] = reinterpret_cast<const ulonglong2*>(s_keys)[i];
        if ((total & 1u) && tid == 0) out[total - 1] = s_keys[total - 1];
      } else {
        for (unsigned i = tid; i < total; i += kLocThreads) out[i] = s_keys[i];
      }
    }
    // padding keys dropped from the bucket: its tail becomes padding (only the
    // unpartitioned single bucket, the last one, holds any)
    for (uint64_t i = total + tid; i < len; i += kLocThreads) out[i] = kSentinel;
    __syncthreads();
  }
}


// one thread per result: the bucket of its smallest racy cell
__global__ void bucket_finish_kernel(FinishArgs fa) {
  const uint32_t nr = fa.n_models ? fa.n_models : 1u;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  DevResult* r = fa.res + i;
  const unsigned long long c = r->hash_cell;
  if (c == ~0ull) return;
  const uint64_t b = fa.D ? (cell_hash_of(c, fa.cmask) >> (fa.cb - fa.D)) : 0ull;
  r->min_start = fa.boff[b];
  r->seg_end = fa.boff[b + 1];
  r->cell = c;
}

}  // namespace

cudaError_t launch_bucket_hist_a(const BucketArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  uint64_t g = (a.n / 2 + 255) / 256;
  if (g < 1) g = 1;
  if (g > 152ull * 8) g = 152ull * 8;
  bucket_hist_a_kernel<<<(unsigned)g, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bucket_scan_a(const BucketArgs& a, cudaStream_t st) {
  bucket_scan_a_kernel<<<1, 1024, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bucket_pass_a(const BucketArgs& a, cudaStream_t st) {
  return launch_bpart<false>(a, a.dA, (a.n + kPTile - 1) / kPTile, st);
}

cudaError_t launch_bucket_hist_b(const BucketArgs& a, uint64_t tiles_h, cudaStream_t st) {
  if (tiles_h == 0) return cudaSuccess;
  if (tiles_h > 0x7fffffffull) return cudaErrorInvalidValue;
  bucket_hist_b_kernel<<<(unsigned)tiles_h, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bucket_scan_b(const BucketArgs& a, cudaStream_t st) {
  const uint64_t nb = 1ull << (a.dA + a.dB);
  cudaError_t e = scan_u64_exclusive(reinterpret_cast<const uint64_t*>(a.hist_b), reinterpret_cast<uint64_t*>(a.boff),
                                     nb, 0, reinterpret_cast<uint64_t*>(a.temp),
                                     reinterpret_cast<uint64_t*>(a.boff + nb), st);
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(a.cur_b, a.boff, nb * 8, cudaMemcpyDeviceToDevice, st);
}

cudaError_t launch_bucket_pass_b(const BucketArgs& a, uint64_t tiles_b, cudaStream_t st) {
  return launch_bpart<true>(a, a.dB, tiles_b, st);
}

cudaError_t launch_bucket_whole(unsigned long long* boff, uint64_t n, cudaStream_t st) {
  bucket_whole_kernel<<<1, 1, 0, st>>>(boff, n);
  return cudaGetLastError();
}

cudaError_t launch_bucket_local_sort(const LocalSortArgs& a, cudaStream_t st) {
  const bool h32 = a.cb <= 32;
  const void* fn = h32 ? reinterpret_cast<const void*>(bucket_local_sort_kernel<true>)
                       : reinterpret_cast<const void*>(bucket_local_sort_kernel<false>);
  cudaError_t e = ensure_kernel_smem(fn, local_smem(kFoldBinBits));
  if (e != cudaSuccess) return e;
  const uint64_t nb = 1ull << a.D;
  const unsigned grid = (unsigned)(nb < 152ull * 2 ? nb : 152ull * 2);
  const size_t smem = local_smem(a.rbin);
  if (h32) bucket_local_sort_kernel<true><<<grid, kLocThreads, smem, st>>>(a);
  else bucket_local_sort_kernel<false><<<grid, kLocThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bucket_finish(const FinishArgs& fa, cudaStream_t st) {
  const uint32_t nr = fa.n_models ? fa.n_models : 1u;
  bucket_finish_kernel<<<(nr + 127) / 128, 128, 0, st>>>(fa);
  return cudaGetLastError();
}

}  // namespace rc
