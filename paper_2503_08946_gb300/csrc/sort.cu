// K2: LSD radix sort of 64-bit keys, one "onesweep" kernel per digit pass.
//
// The paper has no sort: its dependence relations (Write . Read^-1 composed with
// the schedule, appendix listing) join instances on the array cell; here that
// join is a grouping of keys by (cell, phase), done by sorting on those bits.
// Design (after Adinets & Merrill, "Onesweep: a faster least significant digit
// radix sort for GPUs", 2022): one upfront pass counts the digits of every pass;
// then each pass is a single kernel in which a tile of kSortTile keys
//   (1) ranks its keys per digit, stably: per item (32 keys of a warp) the
//       lanes sharing a digit are found with one ballot per digit bit, and the
//       lowest of them reads the warp's 16-bit digit counter (the group's base
//       rank) and adds the group size to it;
//   (2) publishes its per-digit counts, (3) obtains the exclusive per-digit
//       prefix of all earlier tiles by decoupled look-back over their status
//       words, and (4) scatters the keys, staged in shared memory in digit
//       order so the stores of one digit are contiguous.
// The kernel is templated on the radix (2^8 .. 2^11 bins) so that wide digits
// take fewer passes.  Tiles are taken in launch order from an atomic counter,
// so every tile waited on is already running or finished; every wait is
// bounded by spin_limit and reports kErrLookbackTimeout instead of hanging.
#include <cuda_runtime.h>

#include "kernels.h"

namespace rc {

namespace {

constexpr unsigned long long kFlagAggregate = 1ull;
constexpr unsigned long long kFlagPrefix = 2ull;
constexpr unsigned long long kCountMask = (1ull << 46) - 1;

__device__ __forceinline__ unsigned long long status_word(unsigned long long flag, unsigned int epoch,
                                                          unsigned long long count) {
  return (flag << 62) | ((unsigned long long)(epoch & 0xFFFFu) << 46) | (count & kCountMask);
}

__device__ __forceinline__ unsigned int lanemask_lt() {
  unsigned int m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Lanes of the warp whose digit equals this lane's (among lanes with `valid`
// set; an invalid lane gets only itself): one ballot per digit bit, ANDed with
// the bit's sense -- measured cheaper than __match_any_sync on this GPU.  In a
// full tile (block-uniform `full`) every lane is valid and the validity ballot
// is skipped.
template <int RB>
__device__ __forceinline__ unsigned int digit_peers(unsigned int d, bool valid, bool full) {
  // (the skip costs the 256-counter kernel a register spill, so it takes it only
  // for narrower digits)
  unsigned int m = (RB <= 7 && full) ? 0xffffffffu : __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    const bool bit = (d >> b) & 1u;
    const unsigned int bal = __ballot_sync(0xffffffffu, bit);
    m &= bit ? bal : ~bal;
  }
  return valid ? m : (1u << (threadIdx.x & 31));
}

// ---------------------------------------------------------------------------
// upfront digit histograms of every pass (shared-memory counters, one section
// of 2^bits[p] per pass)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) histogram_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                        SortPlan sp, unsigned long long* __restrict__ hist) {
  extern __shared__ unsigned int h[];
  unsigned base[16];
  unsigned tot = 0;
  for (uint32_t p = 0; p < sp.n_pass; ++p) {
    base[p] = tot;
    tot += 1u << sp.bits[p];
  }
  for (unsigned i = threadIdx.x; i < tot; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    for (uint32_t p = 0; p < sp.n_pass; ++p) {
      const unsigned int d = (unsigned int)(k >> sp.shift[p]) & ((1u << sp.bits[p]) - 1u);
      atomicAdd(&h[base[p] + d], 1u);
    }
  }
  __syncthreads();
  for (uint32_t p = 0; p < sp.n_pass; ++p)
    for (unsigned d = threadIdx.x; d < (1u << sp.bits[p]); d += blockDim.x)
      if (h[base[p] + d]) atomicAdd(&hist[p * kMaxRadix + d], (unsigned long long)h[base[p] + d]);
}

// Exclusive scan of up to kMaxRadix counts by 256 threads (contiguous digits per thread).
__device__ __forceinline__ void block_excl_scan_digits(const unsigned long long* in, unsigned long long* out,
                                                       int n_digits) {
  __shared__ unsigned long long wt[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int dpt = (n_digits + 255) / 256;
  const int d0 = threadIdx.x * dpt;
  unsigned long long s = 0;
  for (int k = 0; k < dpt; ++k)
    if (d0 + k < n_digits) s += in[d0 + k];
  unsigned long long x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[w] = x;
  __syncthreads();
  unsigned long long base = 0;
  for (int i = 0; i < w; ++i) base += wt[i];
  unsigned long long run = base + x - s;
  for (int k = 0; k < dpt; ++k)
    if (d0 + k < n_digits) {
      out[d0 + k] = run;
      run += in[d0 + k];
    }
}

__global__ void __launch_bounds__(256) digit_offsets_kernel(const unsigned long long* __restrict__ hist,
                                                            unsigned long long* __restrict__ digoff, SortPlan sp) {
  const int p = blockIdx.x;
  block_excl_scan_digits(hist + p * kMaxRadix, digoff + p * kMaxRadix, 1 << sp.bits[p]);
}

// ---------------------------------------------------------------------------
// one onesweep pass with 2^RB counters per warp
// ---------------------------------------------------------------------------
template <int RB>
constexpr size_t onesweep_smem() {
  // keys | per-warp 16-bit counters | per-digit scatter delta (u64) | per-digit tile offset (u32)
  return (size_t)kSortTile * 8 + (size_t)(kSortThreads / 32) * (1 << RB) * 2 + (size_t)(1 << RB) * 8 +
         (size_t)(1 << RB) * 4;
}

// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned int d = static_cast<unsigned int>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// SK (staged keys): the tile is first copied into shared memory (cp.async), the
// ranking reads its digits from there and the keys come back into registers
// only to be staged in digit order, so 16 keys per thread fit in 64 registers
// and 4 blocks stay resident per SM (instead of 80 registers and 3 blocks)
template <int RB, bool SK>
__global__ void __launch_bounds__(kSortThreads, SK ? 4 : (RB <= 9 ? 3 : 2)) onesweep_kernel(SortArgs a) {
  constexpr int R = 1 << RB;
  // digits per thread in the per-digit phases (fewer digits than threads: one
  // digit for each of the first R threads)
  constexpr bool kAllThreads = R >= kSortThreads;
  constexpr int DPT = kAllThreads ? R / kSortThreads : 1;
  constexpr int kWarps = kSortThreads / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(smem);
  unsigned short* cnt16 = reinterpret_cast<unsigned short*>(s_keys + kSortTile);   // [kWarps][R]
  unsigned int* cnt32 = reinterpret_cast<unsigned int*>(cnt16);
  unsigned long long* delta = reinterpret_cast<unsigned long long*>(cnt16 + kWarps * R);   // [R]
  unsigned int* tile_excl = reinterpret_cast<unsigned int*>(delta + R);                    // [R]
  __shared__ unsigned int s_tile;
  __shared__ unsigned int s_wt[kWarps];

  const uint64_t n_tiles = (a.n + kSortTile - 1) / kSortTile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_counter, 1u);
  for (int i = threadIdx.x; i < kWarps * R / 2; i += kSortThreads) cnt32[i] = 0;
  __syncthreads();
  const uint64_t tile = s_tile;
  if (tile >= n_tiles) return;

  const unsigned int dmask = (1u << a.bits) - 1u;
  const uint64_t wbase = tile * kSortTile + (uint64_t)w * (32 * kSortItems);
  const bool full_tile = (tile + 1) * (uint64_t)kSortTile <= a.n;
  uint64_t k[SK ? 1 : kSortItems];
  // item i of this lane in the tile (and in the staged copy)
  const int lpos = w * (32 * kSortItems) + lane;
  if constexpr (SK) {
    const uint64_t t0 = tile * kSortTile;
    if (full_tile && (reinterpret_cast<uintptr_t>(a.keys_in) & 15u) == 0u) {
#pragma unroll
      for (int m = 0; m < kSortTile / 2 / kSortThreads; ++m) {
        const int j = m * kSortThreads + (int)threadIdx.x;   // pair j: keys 2j, 2j + 1
        cp_async16(s_keys + 2 * j, a.keys_in + t0 + 2 * j);
      }
      cp_async_wait_all();
    } else {
      for (int j = threadIdx.x; j < kSortTile; j += kSortThreads)
        s_keys[j] = t0 + (uint64_t)j < a.n ? a.keys_in[t0 + j] : ~0ull;
    }
    __syncthreads();
  } else {
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      const uint64_t pos = wbase + (uint64_t)i * 32 + lane;
      k[i] = (full_tile || pos < a.n) ? a.keys_in[pos] : ~0ull;
    }
  }
  auto key_of = [&](int i) -> uint64_t {
    if constexpr (SK) return s_keys[lpos + i * 32];
    else return k[i];
  };

  // (1) ranking: per item the peer mask, then the rank through the warp's counters
  unsigned short r[kSortItems];
  const unsigned int lt = lanemask_lt();
  unsigned short* my_cnt = cnt16 + w * R;
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const unsigned int d = (unsigned int)(key_of(i) >> a.shift) & dmask;
    const bool valid = full_tile || wbase + (uint64_t)i * 32 + lane < a.n;
    const unsigned int peers = digit_peers<RB>(d, valid, full_tile);
    const unsigned int leader = __ffs(peers) - 1;
    unsigned int prev = 0;
    if (lane == leader && valid) {
      // the leaders of one item hold distinct digits, so their 16-bit
      // counters are distinct and plain loads and stores suffice
      prev = my_cnt[d];
      my_cnt[d] = (unsigned short)(prev + __popc(peers));
    }
    prev = __shfl_sync(0xffffffffu, prev, leader);
    r[i] = (unsigned short)(prev + __popc(peers & lt));
    __syncwarp();
  }
  __syncthreads();

  // (2) per digit: tile count, publication, and the tile's exclusive digit offsets
  const bool has_digits = kAllThreads || (int)threadIdx.x < R;
  unsigned int cnt[DPT];
  unsigned int tsum = 0;
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    const int dg = threadIdx.x * DPT + q;
    unsigned int c = 0;
    if (has_digits) {
#pragma unroll
      for (int ww = 0; ww < kWarps; ++ww) c += cnt16[ww * R + dg];
    }
    cnt[q] = c;
    tsum += c;
  }
  volatile unsigned long long* lb = a.lookback;
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    const int dg = threadIdx.x * DPT + q;
    if (has_digits) lb[tile * R + dg] = status_word(tile == 0 ? kFlagPrefix : kFlagAggregate, a.epoch, cnt[q]);
  }
  {
    unsigned int x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wt[w] = x;
    __syncthreads();
    unsigned int base = 0;
    for (int i = 0; i < w; ++i) base += s_wt[i];
    unsigned int run = base + x - tsum;
#pragma unroll
    for (int q = 0; q < DPT && has_digits; ++q) {
      const int dg = threadIdx.x * DPT + q;
      tile_excl[dg] = run;
      // staging offset of warp ww's keys of digit dg = tile offset + earlier warps' counts
      unsigned int wrun = run;
#pragma unroll
      for (int ww = 0; ww < kWarps; ++ww) {
        const unsigned int c = cnt16[ww * R + dg];
        cnt16[ww * R + dg] = (unsigned short)wrun;
        wrun += c;
      }
      run += cnt[q];
    }
  }
  __syncthreads();

  // stage the keys in digit order (stable); with SK the keys come back from
  // the tile copy first, and all are read before any is overwritten
  const unsigned short* my_off = cnt16 + w * R;
  uint64_t kk[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) kk[i] = key_of(i);
  if constexpr (SK) __syncthreads();
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    if (full_tile || wbase + (uint64_t)i * 32 + lane < a.n) {
      const unsigned int d = (unsigned int)(kk[i] >> a.shift) & dmask;
      s_keys[my_off[d] + r[i]] = kk[i];
    }
  }

  // (3) decoupled look-back for this thread's digits
#pragma unroll
  for (int q = 0; q < DPT && has_digits; ++q) {
    const int dg = threadIdx.x * DPT + q;
    unsigned long long excl = 0;
    if (tile > 0) {
      uint64_t j = tile - 1;
      unsigned long long spins = 0;
      while (true) {
        const unsigned long long s = lb[j * R + dg];
        const unsigned long long flag = s >> 62;
        const unsigned int ep = (unsigned int)((s >> 46) & 0xFFFFu);
        if (flag == 0 || ep != (a.wait_epoch & 0xFFFFu)) {
          if (++spins > a.spin_limit) {
            atomicOr(a.err, (unsigned int)kErrLookbackTimeout);
            break;
          }
          continue;
        }
        excl += s & kCountMask;
        if (flag == kFlagPrefix || j == 0) break;
        --j;
      }
      lb[tile * R + dg] = status_word(kFlagPrefix, a.epoch, excl + cnt[q]);
    }
    // output position of a staged key = delta[digit] + staged position
    delta[dg] = a.digit_offset[dg] + excl - tile_excl[dg];
  }
  __syncthreads();

  // (4) scatter: consecutive staged keys of one digit go to consecutive addresses
  const uint64_t t0 = tile * kSortTile;
  const int n_here = full_tile ? kSortTile : (int)(a.n - t0);
  for (int pos = threadIdx.x; pos < n_here; pos += kSortThreads) {
    const uint64_t key = s_keys[pos];
    const unsigned int dd = (unsigned int)(key >> a.shift) & dmask;
    const unsigned long long dst = delta[dd] + (unsigned long long)pos;
    // in range whenever the digit counts match the ranks; a mismatch (input
    // changed under the sort) is reported instead of written out of bounds
    if (dst < a.n) a.keys_out[dst] = key;
    else atomicOr(a.err, (unsigned int)kErrSortRange);
  }
}

// ---------------------------------------------------------------------------
// unstable partition pass (the first pass of a check's sort: its input is the
// expansion order, which carries no meaning, so equal digits may come out in
// any order).  Each tile ranks its keys with block-wide digit counters (one
// shared atomic per key, or per warp when the warp holds a single digit),
// claims each digit's output range from a global cursor (started at the
// digit's offset), stages the keys in digit order and scatters them.  No
// look-back and no waiting: tiles are independent.
// ---------------------------------------------------------------------------
// The partition pass's tile: 12 keys per thread.  It has no look-back, so its
// tile size is free of the stable passes'; at 12 keys a thread fits in 64
// registers and 4 blocks stay resident per SM (measured on the 4096 x 256 model:
// 4.24 ms against 5.35 ms for 16 keys at 3 blocks).
constexpr int kPartItems = 12;
constexpr int kPartTile = kSortThreads * kPartItems;

template <int RB>
constexpr size_t partition_smem() {
  return (size_t)kPartTile * 8 + (size_t)(1 << RB) * (4 + 4 + 8);
}

template <int RB>
__global__ void __launch_bounds__(kSortThreads, 5) partition_kernel(SortArgs a) {
  constexpr int R = 1 << RB;
  constexpr int DPT = (R + kSortThreads - 1) / kSortThreads;
  constexpr int kWarps = kSortThreads / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* s_keys = reinterpret_cast<uint64_t*>(smem);
  unsigned int* cnt = reinterpret_cast<unsigned int*>(s_keys + kPartTile);           // [R]
  unsigned int* excl = cnt + R;                                                       // [R]
  unsigned long long* delta = reinterpret_cast<unsigned long long*>(excl + R);        // [R]
  __shared__ unsigned int s_wt[kWarps];
  const uint64_t tile = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned int dmask = (1u << a.bits) - 1u;
  for (int i = threadIdx.x; i < R; i += kSortThreads) cnt[i] = 0;
  __syncthreads();
  const uint64_t wbase = tile * kPartTile + (uint64_t)w * (32 * kPartItems);
  const bool full_tile = (tile + 1) * (uint64_t)kPartTile <= a.n;
  // the tile is copied into shared memory (cp.async for full tiles of a
  // 16-byte aligned key array) and ranked from there; the keys come back into
  // registers only to be staged
  {
    const uint64_t t0 = tile * kPartTile;
    if (full_tile && (reinterpret_cast<uintptr_t>(a.keys_in) & 15u) == 0u) {
#pragma unroll
      for (int m = 0; m < kPartTile / 2 / kSortThreads; ++m) {
        const int j = m * kSortThreads + (int)threadIdx.x;   // pair j: keys 2j, 2j + 1
        cp_async16(s_keys + 2 * j, a.keys_in + t0 + 2 * j);
      }
      cp_async_wait_all();
    } else {
      for (int j = threadIdx.x; j < kPartTile; j += kSortThreads)
        s_keys[j] = t0 + (uint64_t)j < a.n ? a.keys_in[t0 + j] : ~0ull;
    }
  }
  __syncthreads();
  const int lpos = w * (32 * kPartItems) + lane;
  // ranks within the tile's digit buckets in any order: one shared atomic per
  // lane, or one per warp when the whole warp holds one digit (frequent: the 32
  // keys of a warp come from one access of 32 consecutive threads)
  unsigned short r[kPartItems];
#pragma unroll
  for (int i = 0; i < kPartItems; ++i) {
    const unsigned int d = (unsigned int)(s_keys[lpos + i * 32] >> a.shift) & dmask;
    const bool valid = full_tile || wbase + (uint64_t)i * 32 + lane < a.n;
    const unsigned int d0 = __shfl_sync(0xffffffffu, d, 0);
    unsigned int rank = 0;
    if (__all_sync(0xffffffffu, valid && d == d0)) {
      unsigned int base = 0;
      if (lane == 0) base = atomicAdd(&cnt[d0], 32u);
      rank = __shfl_sync(0xffffffffu, base, 0) + (unsigned int)lane;
    } else if (valid) {
      rank = atomicAdd(&cnt[d], 1u);
    }
    r[i] = (unsigned short)rank;
  }
  __syncthreads();
  // per digit dg = q * kSortThreads + tid: claim the output range, tile offsets
  unsigned int carry = 0;
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    const int dg = q * kSortThreads + threadIdx.x;
    const unsigned int c = dg < R ? cnt[dg] : 0u;
    const unsigned long long claim = c ? atomicAdd(&a.cursor[dg], (unsigned long long)c) : 0ull;
    unsigned int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wt[w] = x;
    __syncthreads();
    unsigned int base = carry, tot = 0;
    for (int i = 0; i < kWarps; ++i) {
      if (i < w) base += s_wt[i];
      tot += s_wt[i];
    }
    __syncthreads();
    if (dg < R) {
      const unsigned int e = base + x - c;
      excl[dg] = e;
      delta[dg] = claim - e;
    }
    carry += tot;
  }
  __syncthreads();
  uint64_t kk[kPartItems];
#pragma unroll
  for (int i = 0; i < kPartItems; ++i) kk[i] = s_keys[lpos + i * 32];
  __syncthreads();   // every key read before any is overwritten
#pragma unroll
  for (int i = 0; i < kPartItems; ++i) {
    if (full_tile || wbase + (uint64_t)i * 32 + lane < a.n) {
      const unsigned int d = (unsigned int)(kk[i] >> a.shift) & dmask;
      s_keys[excl[d] + r[i]] = kk[i];
    }
  }
  __syncthreads();
  const uint64_t t0 = tile * kPartTile;
  const int n_here = full_tile ? kPartTile : (int)(a.n - t0);
  for (int pos = threadIdx.x; pos < n_here; pos += kSortThreads) {
    const uint64_t key = s_keys[pos];
    const unsigned int dd = (unsigned int)(key >> a.shift) & dmask;
    const unsigned long long dst = delta[dd] + (unsigned long long)pos;
    if (dst < a.n) a.keys_out[dst] = key;   // (see the onesweep scatter)
    else atomicOr(a.err, (unsigned int)kErrSortRange);
  }
}

template <int RB>
cudaError_t launch_partition_rb(const SortArgs& a, cudaStream_t st) {
  constexpr size_t smem = partition_smem<RB>();
  const cudaError_t e = ensure_kernel_smem(reinterpret_cast<const void*>(partition_kernel<RB>), smem);
  if (e != cudaSuccess) return e;
  const uint64_t n_tiles = (a.n + kPartTile - 1) / kPartTile;
  partition_kernel<RB><<<(unsigned)n_tiles, kSortThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int RB>
cudaError_t launch_rb(const SortArgs& a, cudaStream_t st) {
  constexpr size_t smem = onesweep_smem<RB>();
  constexpr bool SK = RB <= 8;   // staged keys for the 7- and 8-bit kernels
  const cudaError_t e = ensure_kernel_smem(reinterpret_cast<const void*>(onesweep_kernel<RB, SK>), smem);
  if (e != cudaSuccess) return e;
  const uint64_t n_tiles = (a.n + kSortTile - 1) / kSortTile;
  onesweep_kernel<RB, SK><<<(unsigned)n_tiles, kSortThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

// 7-bit digits take the 128-counter kernel (7 ballots per key instead of 8)
uint32_t radix_bits_for(uint32_t bits) { return bits <= 7 ? 7 : (bits <= 8 ? 8 : bits); }

cudaError_t launch_histogram(const uint64_t* keys, uint64_t n, const SortPlan& sp, unsigned long long* hist,
                             cudaStream_t st) {
  if (n == 0 || sp.n_pass == 0) return cudaSuccess;
  size_t smem = 0;
  for (uint32_t p = 0; p < sp.n_pass; ++p) smem += (size_t)4 << sp.bits[p];
  const cudaError_t e = ensure_kernel_smem(reinterpret_cast<const void*>(histogram_kernel), 16 * kMaxRadix * 4, false);
  if (e != cudaSuccess) return e;
  uint64_t g = (n + 255) / 256;
  if (g > 152ull * 8) g = 152ull * 8;
  histogram_kernel<<<(unsigned)g, 256, smem, st>>>(keys, n, sp, hist);
  return cudaGetLastError();
}

cudaError_t launch_digit_offsets(const unsigned long long* hist, unsigned long long* digoff, const SortPlan& sp,
                                 cudaStream_t st) {
  if (sp.n_pass == 0) return cudaSuccess;
  digit_offsets_kernel<<<sp.n_pass, 256, 0, st>>>(hist, digoff, sp);
  return cudaGetLastError();
}

cudaError_t launch_partition(const SortArgs& a, uint32_t radix_bits, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  switch (radix_bits) {
    case 7: return launch_partition_rb<7>(a, st);
    case 8: return launch_partition_rb<8>(a, st);
    case 9: return launch_partition_rb<9>(a, st);
    case 10: return launch_partition_rb<10>(a, st);
    case 11: return launch_partition_rb<11>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_onesweep(const SortArgs& a, uint32_t radix_bits, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  switch (radix_bits) {
    case 7: return launch_rb<7>(a, st);
    case 8: return launch_rb<8>(a, st);
    case 9: return launch_rb<9>(a, st);
    case 10: return launch_rb<10>(a, st);
    case 11: return launch_rb<11>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rc
