// rc_sort_keys_static: the radix sort of rc_sort_keys with its scratch in a
// file-scope device array instead of a caller-provided workspace, for callers
// that must not allocate device memory when they sort (see include/rc.h).
//
// The scratch array is a static __device__ object of this translation unit.
// Host code cannot pass the array's name to a kernel (on the host it is only a
// stand-in symbol, not a device address), so the device address is looked up
// with cudaGetSymbolAddress once per device, with that device current, and
// cached.  All calls on a device share the array.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "kernels.h"

namespace {

constexpr uint64_t kStaticMaxKeys = RC_SORT_STATIC_MAX_KEYS;
constexpr size_t kStaticTiles = (kStaticMaxKeys + rc::kSortTile - 1) / rc::kSortTile;
// layout: result record | digit histograms | look-back words | tile counters | digit offsets | second key buffer
constexpr size_t kOffResult = 0;
constexpr size_t kOffHist = 256;
constexpr size_t kOffLookback = kOffHist + (size_t)16 * rc::kMaxRadix * 8;
constexpr size_t kOffTileCtr = kOffLookback + kStaticTiles * ((size_t)1 << rc::kMaxRadixBits) * 8;
constexpr size_t kOffDigoff = kOffTileCtr + 256;
constexpr size_t kOffPong = kOffDigoff + (size_t)16 * rc::kMaxRadix * 8;
constexpr size_t kScratchBytes = kOffPong + kStaticMaxKeys * 8;
static_assert(kOffLookback % 256 == 0 && kOffTileCtr % 256 == 0 && kOffDigoff % 256 == 0 &&
                  kOffPong % 256 == 0,
              "scratch sections are 256-byte aligned");

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of this device's scratch array (looked up once per device).
rc_status scratch_for_current_device(uint8_t** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return RC_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return RC_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return RC_E_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<uint8_t*>(g_scratch_addr[dev]);
  return RC_OK;
}

rc_status as_status(cudaError_t e) { return e == cudaSuccess ? RC_OK : RC_E_CUDA; }

}  // namespace

namespace rc {
rc_status sort_static_record(const void** rec) {
  uint8_t* s = nullptr;
  const rc_status st = scratch_for_current_device(&s);
  if (st == RC_OK) *rec = s + kOffResult;
  return st;
}
}  // namespace rc

extern "C" rc_status rc_sort_keys_static(const uint64_t* keys_in, uint64_t* keys_out, uint64_t n, uint32_t lo_bit,
                                         uint32_t hi_bit, uint32_t digit_bits, void* stream) {
  if (hi_bit > 64 || lo_bit > hi_bit || (n && (!keys_in || !keys_out || keys_in == keys_out))) return RC_E_INVALID;
  if (n > kStaticMaxKeys) return RC_E_UNSUPPORTED;
  uint8_t* s = nullptr;
  rc_status st = scratch_for_current_device(&s);
  if (st != RC_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  auto* res = reinterpret_cast<rc::DevResult*>(s + kOffResult);
  // the error word read by rc_sort_status starts clear for every call
  st = as_status(rc::launch_init_result(res, cs));
  if (st != RC_OK || n == 0) return st;
  rc::SortPlan sp;
  rc::plan_sort(lo_bit, hi_bit, digit_bits, &sp);
  auto* hist = reinterpret_cast<unsigned long long*>(s + kOffHist);
  auto* digoff = reinterpret_cast<unsigned long long*>(s + kOffDigoff);
  uint64_t* pong = reinterpret_cast<uint64_t*>(s + kOffPong);
  // the array keeps the previous call's contents: clear what must start at
  // zero (this call's digit counts, look-back words and tile counters)
  size_t clear[3][2];
  rc::sort_clear_ranges(sp, n, kOffHist, kOffLookback, kOffTileCtr, clear);
  for (int r = 0; r < 3 && st == RC_OK; ++r) st = as_status(cudaMemsetAsync(s + clear[r][0], 0, clear[r][1], cs));
  if (st == RC_OK) st = as_status(cudaMemcpyAsync(keys_out, keys_in, n * 8, cudaMemcpyDeviceToDevice, cs));
  if (st == RC_OK) st = as_status(rc::launch_digit_counts(keys_out, n, sp, hist, cs));
  if (st == RC_OK) st = as_status(rc::launch_digit_offsets(hist, digoff, sp, cs));
  uint64_t* bufs[2] = {keys_out, pong};
  const bool stall = rc::sort_stall_requested();
  int cur = 0;
  for (uint32_t k = 0; k < sp.n_pass && st == RC_OK; ++k) {
    rc::SortArgs a;
    a.keys_in = bufs[cur];
    a.keys_out = bufs[1 - cur];
    a.n = n;
    a.shift = sp.shift[k];
    a.bits = sp.bits[k];
    a.digit_offset = digoff + (size_t)k * rc::kMaxRadix;
    a.lookback = reinterpret_cast<unsigned long long*>(s + kOffLookback);
    a.tile_counter = reinterpret_cast<unsigned int*>(s + kOffTileCtr) + k;
    a.epoch = k + 1;
    a.wait_epoch = stall ? (k + 1) ^ 0x8000u : k + 1;   // (the test hook: a wait nothing ends)
    a.spin_limit = stall ? 4096ull : (1ull << 20);
    a.err = &res->err;
    a.cursor = nullptr;
    st = as_status(rc::launch_onesweep(a, rc::radix_bits_for(a.bits), cs));
    cur = 1 - cur;
  }
  if (st == RC_OK && cur == 1) st = as_status(cudaMemcpyAsync(keys_out, pong, n * 8, cudaMemcpyDeviceToDevice, cs));
  return st;
}
