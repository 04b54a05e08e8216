// K2: LSD radix sort of 64-bit keys, one "onesweep" kernel per digit pass.
//
// The paper has no sort: its dependence relations (Write . Read^-1 composed with
// the schedule, appendix listing) join instances on the array cell; here that
// join is a grouping of keys by (cell, phase), done by sorting on those bits.
// Design (after Adinets & Merrill, "Onesweep: a faster least significant digit
// radix sort for GPUs", 2022): one upfront pass counts the digits of every pass;
// then each pass is a single kernel in which a tile of kSortTile keys (1) ranks
// its keys per digit with warp-level __match_any_sync multi-split into per-warp
// shared-memory histograms, (2) publishes its per-digit counts, (3) obtains the
// exclusive per-digit prefix of all earlier tiles by decoupled look-back over
// their published status words, and (4) scatters the keys, staged in shared
// memory in digit order so stores of one digit are contiguous.  Tiles are taken
// in launch order from an atomic counter, so every tile waited on is already
// running or finished; every wait is bounded by spin_limit and reports
// kErrLookbackTimeout instead of hanging.
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

// ---------------------------------------------------------------------------
// upfront digit histograms of every pass
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) histogram_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                        SortPlan sp, unsigned long long* __restrict__ hist) {
  __shared__ unsigned int h[16][kRadix];
  for (int i = threadIdx.x; i < 16 * kRadix; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    for (uint32_t p = 0; p < sp.n_pass; ++p) {
      const unsigned int d = (unsigned int)(k >> sp.shift[p]) & ((1u << sp.bits[p]) - 1u);
      atomicAdd(&h[p][d], 1u);
    }
  }
  __syncthreads();
  for (uint32_t p = 0; p < sp.n_pass; ++p)
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
      if (h[p][d]) atomicAdd(&hist[p * kRadix + d], (unsigned long long)h[p][d]);
}

__device__ __forceinline__ unsigned long long block_excl_scan256(unsigned long long v, unsigned long long* total) {
  __shared__ unsigned long long wt[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[w] = x;
  __syncthreads();
  unsigned long long base = 0, tot = 0;
  for (int i = 0; i < 8; ++i) {
    if (i < w) base += wt[i];
    tot += wt[i];
  }
  __syncthreads();
  if (total) *total = tot;
  return base + x - v;
}

__global__ void __launch_bounds__(256) digit_offsets_kernel(const unsigned long long* __restrict__ hist,
                                                            unsigned long long* __restrict__ digoff) {
  const int p = blockIdx.x;
  const unsigned long long v = hist[p * kRadix + threadIdx.x];
  digoff[p * kRadix + threadIdx.x] = block_excl_scan256(v, nullptr);
}

// ---------------------------------------------------------------------------
// one onesweep pass
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads, 3) onesweep_kernel(SortArgs a) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ unsigned int s_tile;
  __shared__ unsigned int warp_hist[kWarps][kRadix];
  __shared__ unsigned int tile_excl[kRadix];
  __shared__ unsigned long long g_base[kRadix];
  __shared__ uint64_t s_keys[kSortTile];

  const uint64_t n_tiles = (a.n + kSortTile - 1) / kSortTile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_counter, 1u);
  for (int i = threadIdx.x; i < kWarps * kRadix; i += kSortThreads) (&warp_hist[0][0])[i] = 0;
  __syncthreads();
  const uint64_t tile = s_tile;
  if (tile >= n_tiles) return;

  const unsigned int dmask = (1u << a.bits) - 1u;
  const uint64_t wbase = tile * kSortTile + (uint64_t)w * (32 * kSortItems);
  uint64_t k[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint64_t pos = wbase + (uint64_t)i * 32 + lane;
    k[i] = pos < a.n ? a.keys_in[pos] : ~0ull;
  }

  // Warp-level multi-split ranking, stable in (item, lane) order.  First the
  // peer masks of all items (independent __match_any_sync, so their latencies
  // overlap; an out-of-range lane gets a digit no other lane has), then one
  // pass over the items that turns the masks into ranks through the warp's
  // shared-memory digit counters (the lowest peer updates the counter).
  const bool full_tile = (tile + 1) * (uint64_t)kSortTile <= a.n;
  unsigned int peers[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    unsigned int d = (unsigned int)(k[i] >> a.shift) & dmask;
    if (!full_tile && wbase + (uint64_t)i * 32 + lane >= a.n) d = 0x100u | lane;
    peers[i] = __match_any_sync(0xffffffffu, d);
  }
  unsigned int r[kSortItems];
  const unsigned int lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const unsigned int d = (unsigned int)(k[i] >> a.shift) & dmask;
    const bool valid = full_tile || wbase + (uint64_t)i * 32 + lane < a.n;
    const unsigned int leader = __ffs(peers[i]) - 1;
    unsigned int prev = 0;
    if (lane == leader && valid) {
      prev = warp_hist[w][d];
      warp_hist[w][d] = prev + __popc(peers[i]);
    }
    prev = __shfl_sync(0xffffffffu, prev, leader);
    r[i] = prev + __popc(peers[i] & lt);
    __syncwarp();
  }
  __syncthreads();

  // per digit: exclusive offsets of the warps, the tile's count, and its publication
  const int dg = threadIdx.x;   // kSortThreads == kRadix
  unsigned int cnt = 0;
#pragma unroll
  for (int ww = 0; ww < kWarps; ++ww) {
    const unsigned int c = warp_hist[ww][dg];
    warp_hist[ww][dg] = cnt;
    cnt += c;
  }
  volatile unsigned long long* lb = a.lookback;
  if (tile == 0) lb[dg] = status_word(kFlagPrefix, a.epoch, cnt);
  else lb[tile * kRadix + dg] = status_word(kFlagAggregate, a.epoch, cnt);
  {
    unsigned long long tot;
    tile_excl[dg] = (unsigned int)block_excl_scan256(cnt, &tot);
  }
  __syncthreads();

  // stage the keys in digit order (stable)
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint64_t pos = wbase + (uint64_t)i * 32 + lane;
    if (pos < a.n) {
      const unsigned int d = (unsigned int)(k[i] >> a.shift) & dmask;
      s_keys[tile_excl[d] + warp_hist[w][d] + r[i]] = k[i];
    }
  }

  // decoupled look-back for digit dg
  unsigned long long excl = 0;
  if (tile > 0) {
    uint64_t j = tile - 1;
    unsigned long long spins = 0;
    while (true) {
      const unsigned long long s = lb[j * kRadix + dg];
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
    lb[tile * kRadix + dg] = status_word(kFlagPrefix, a.epoch, excl + cnt);
  }
  g_base[dg] = a.digit_offset[dg] + excl;
  __syncthreads();

  // scatter: consecutive staged keys of one digit go to consecutive addresses
  const uint64_t t0 = tile * kSortTile;
  const int n_here = (int)((a.n - t0) < (uint64_t)kSortTile ? (a.n - t0) : (uint64_t)kSortTile);
  for (int pos = threadIdx.x; pos < n_here; pos += kSortThreads) {
    const uint64_t key = s_keys[pos];
    const unsigned int dd = (unsigned int)(key >> a.shift) & dmask;
    a.keys_out[g_base[dd] + (unsigned long long)(pos - (int)tile_excl[dd])] = key;
  }
}

}  // namespace

cudaError_t launch_histogram(const uint64_t* keys, uint64_t n, const SortPlan& sp, unsigned long long* hist,
                             cudaStream_t st) {
  if (n == 0 || sp.n_pass == 0) return cudaSuccess;
  uint64_t g = (n + 255) / 256;
  if (g > 152ull * 8) g = 152ull * 8;
  histogram_kernel<<<(unsigned)g, 256, 0, st>>>(keys, n, sp, hist);
  return cudaGetLastError();
}

cudaError_t launch_digit_offsets(const unsigned long long* hist, unsigned long long* digoff, uint32_t n_pass,
                                 cudaStream_t st) {
  if (n_pass == 0) return cudaSuccess;
  digit_offsets_kernel<<<n_pass, 256, 0, st>>>(hist, digoff);
  return cudaGetLastError();
}

cudaError_t launch_onesweep(const SortArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  static bool carveout_set = false;
  if (!carveout_set) {
    // as much shared memory as possible: 3 resident blocks of ~44 KB per SM
    cudaFuncSetAttribute(onesweep_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    carveout_set = true;
  }
  const uint64_t n_tiles = (a.n + kSortTile - 1) / kSortTile;
  onesweep_kernel<<<(unsigned)n_tiles, kSortThreads, 0, st>>>(a);
  return cudaGetLastError();
}

size_t sort_workspace_bytes(uint64_t n, uint32_t n_pass) {
  const uint64_t n_tiles = (n + kSortTile - 1) / kSortTile;
  return (size_t)n_pass * kRadix * 8 * 2 + (size_t)n_tiles * kRadix * 8 + 256;
}

}  // namespace rc
