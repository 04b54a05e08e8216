// Digit counts of all passes of a radix sort plan, for plans of at most
// kHistMaxPasses passes: the pass count is a template parameter, so each
// pass's shift, mask and counter base stay in registers and a key costs one
// shift, one mask and one shared atomic per pass.  Each thread reads two
// independent 16-byte pairs of keys per step (the warp's pairs contiguous).
#include <cstdint>

#include "kernels.h"

namespace rc {
namespace {

constexpr int kHistMaxPasses = 6;     // plans with more passes take launch_histogram

template <int NP>
__global__ void __launch_bounds__(256) histogram_np_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                           SortPlan sp, unsigned long long* __restrict__ hist) {
  extern __shared__ unsigned int h[];
  unsigned base[NP], shift[NP], mask[NP];
  unsigned tot = 0;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    base[p] = tot;
    shift[p] = sp.shift[p];
    mask[p] = (1u << sp.bits[p]) - 1u;
    tot += 1u << sp.bits[p];
  }
  for (unsigned i = threadIdx.x; i < tot; i += blockDim.x) h[i] = 0;
  __syncthreads();
  auto count = [&](const uint64_t k) {
#pragma unroll
    for (int p = 0; p < NP; ++p) atomicAdd(&h[base[p] + ((unsigned)(k >> shift[p]) & mask[p])], 1u);
  };
  // the key array is 16-byte aligned (checked by the launcher)
  const ulonglong2* k2 = reinterpret_cast<const ulonglong2*>(keys);
  const uint64_t n2 = n / 2;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + stride < n2; i += 2 * stride) {
    const ulonglong2 a = __ldg(k2 + i), b = __ldg(k2 + i + stride);
    count(a.x);
    count(a.y);
    count(b.x);
    count(b.y);
  }
  if (i < n2) {
    const ulonglong2 a = __ldg(k2 + i);
    count(a.x);
    count(a.y);
  }
  if ((n & 1u) && blockIdx.x == 0 && threadIdx.x == 0) count(__ldg(keys + n - 1));
  __syncthreads();
#pragma unroll
  for (int p = 0; p < NP; ++p)
    for (unsigned d = threadIdx.x; d <= mask[p]; d += blockDim.x)
      if (h[base[p] + d]) atomicAdd(&hist[p * kMaxRadix + d], (unsigned long long)h[base[p] + d]);
}

template <int NP>
cudaError_t launch_np(const uint64_t* keys, uint64_t n, const SortPlan& sp, unsigned long long* hist, size_t smem,
                      cudaStream_t st) {
  const cudaError_t e =
      ensure_kernel_smem(reinterpret_cast<const void*>(histogram_np_kernel<NP>), NP * kMaxRadix * 4, false);
  if (e != cudaSuccess) return e;
  uint64_t g = (n / 2 + 255) / 256;
  if (g < 1) g = 1;
  if (g > 152ull * 8) g = 152ull * 8;
  histogram_np_kernel<NP><<<(unsigned)g, 256, smem, st>>>(keys, n, sp, hist);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_digit_counts(const uint64_t* keys, uint64_t n, const SortPlan& sp, unsigned long long* hist,
                                cudaStream_t st) {
  if (n == 0 || sp.n_pass == 0) return cudaSuccess;
  if (sp.n_pass > (uint32_t)kHistMaxPasses || (reinterpret_cast<uintptr_t>(keys) & 15u) != 0u)
    return launch_histogram(keys, n, sp, hist, st);
  size_t smem = 0;
  for (uint32_t p = 0; p < sp.n_pass; ++p) smem += (size_t)4 << sp.bits[p];
  switch (sp.n_pass) {
    case 1: return launch_np<1>(keys, n, sp, hist, smem, st);
    case 2: return launch_np<2>(keys, n, sp, hist, smem, st);
    case 3: return launch_np<3>(keys, n, sp, hist, smem, st);
    case 4: return launch_np<4>(keys, n, sp, hist, smem, st);
    case 5: return launch_np<5>(keys, n, sp, hist, smem, st);
    default: return launch_np<6>(keys, n, sp, hist, smem, st);
  }
}

}  // namespace rc
