// Request server: continuous batching of race-check requests on one GPU.
//
// A scheduler thread admits queued requests as soon as a slot (a CUDA stream
// with one batch in flight) and device memory are free: it takes the waiting
// requests in arrival order, as many as fit the largest free block of the
// server's memory pool (at most max_batch), and enqueues them as one batched
// check (rc_check_batch) on the free slot.  Work of different slots overlaps on
// the device.  Finished batches are reported per request with host timestamps
// (submission, start, completion), and their pool blocks return to the pool.
//
// The pool is one device allocation made when the server is created; the
// scheduler sub-allocates workspaces from it (first fit, 256-byte aligned,
// neighbours coalesced on release), so serving allocates no device memory per
// request.  A request whose workspace cannot fit the pool even when it is empty
// completes at once with status RC_E_NOMEM.
#include <cuda_runtime_api.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "rc.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing.
class Pool {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  // offset of a block of `bytes` (rounded to 256), or SIZE_MAX
  size_t alloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t largest() const {
    size_t m = 0;
    for (auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }

 private:
  std::map<size_t, size_t> free_;   // offset -> length
};

struct Request {
  uint64_t id;
  rc_model* model;
  double submit_s;
};

struct Slot {
  cudaStream_t stream = nullptr;
  bool busy = false;
  rc_ticket ticket = nullptr;
  std::vector<Request> reqs;
  size_t ws_off = 0, ws_bytes = 0;
  double start_s = 0;
};

}  // namespace

struct rc_server {
  rc_server_opts opts{};
  int device = 0;
  uint8_t* pool_base = nullptr;
  Pool pool;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> pending;
  std::deque<rc_server_done> done;
  uint64_t next_id = 1;
  uint64_t in_flight = 0;
  bool stop = false;
  rc_status fatal = RC_OK;
  std::thread th;

  void finish(Slot& sl) {
    std::vector<rc_result> out(sl.reqs.size());
    const rc_status st = rc_report(sl.ticket, out.data(), 1);
    const double t = now_s();
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
      rc_server_done d;
      std::memset(&d, 0, sizeof(d));
      d.request = sl.reqs[i].id;
      d.result = out[i];
      if (st != RC_OK) d.result.status = st;
      d.submit_s = sl.reqs[i].submit_s;
      d.start_s = sl.start_s;
      d.done_s = t;
      d.batch_size = (uint32_t)sl.reqs.size();
      done.push_back(d);
    }
    pool.release(sl.ws_off, sl.ws_bytes);
    in_flight -= sl.reqs.size();
    sl.reqs.clear();
    sl.ticket = nullptr;
    sl.busy = false;
  }

  void fail_now(const Request& r, rc_status st) {
    rc_server_done d;
    std::memset(&d, 0, sizeof(d));
    d.request = r.id;
    d.result.status = st;
    d.submit_s = r.submit_s;
    d.start_s = d.done_s = now_s();
    d.batch_size = 1;
    done.push_back(d);
  }

  size_t need_for(const std::vector<rc_model*>& ms) {
    size_t b = 0;
    rc_check_opts o{};
    o.path = RC_PATH_SORT;
    o.digit_bits = opts.digit_bits;
    if (rc_batch_workspace_size(ms.data(), ms.size(), &o, &b) != RC_OK) return SIZE_MAX;
    return b;
  }

  // Admit waiting requests into free slots.  Called with mu held.
  void admit() {
    for (Slot& sl : slots) {
      if (sl.busy || pending.empty()) continue;
      // the longest prefix of the queue (at most max_batch) whose batch fits the
      // largest free block, by binary search over the prefix length
      const size_t room = pool.largest();
      const size_t cap = std::min<size_t>(pending.size(), opts.max_batch ? opts.max_batch : 1024);
      std::vector<rc_model*> all;
      all.reserve(cap);
      for (size_t i = 0; i < cap; ++i) all.push_back(pending[i].model);
      size_t lo = 0, hi = cap, need = 0;
      while (lo < hi) {
        const size_t mid = (lo + hi + 1) / 2;
        std::vector<rc_model*> pre(all.begin(), all.begin() + (long)mid);
        const size_t b = need_for(pre);
        if (b <= room) {
          lo = mid;
          need = b;
        } else {
          hi = mid - 1;
        }
      }
      std::vector<rc_model*> ms(all.begin(), all.begin() + (long)lo);
      if (ms.empty()) {
        // the oldest request does not fit now; if it cannot fit at all, fail it
        std::vector<rc_model*> one{pending.front().model};
        if (need_for(one) > opts.memory_bytes) {
          fail_now(pending.front(), RC_E_NOMEM);
          pending.pop_front();
          cv_done.notify_all();
        }
        return;
      }
      const size_t off = pool.alloc(need);
      if (off == SIZE_MAX) return;
      sl.reqs.assign(pending.begin(), pending.begin() + (long)ms.size());
      pending.erase(pending.begin(), pending.begin() + (long)ms.size());
      rc_check_opts o{};
      o.path = RC_PATH_SORT;
      o.digit_bits = opts.digit_bits;
      rc_ticket t = nullptr;
      const rc_status st = rc_check_batch(ms.data(), ms.size(), &o, pool_base + off, need, sl.stream, &t);
      if (st != RC_OK) {
        pool.release(off, need);
        for (const Request& r : sl.reqs) fail_now(r, st);
        sl.reqs.clear();
        cv_done.notify_all();
        continue;
      }
      sl.ticket = t;
      sl.ws_off = off;
      sl.ws_bytes = need;
      sl.start_s = now_s();
      sl.busy = true;
      in_flight += sl.reqs.size();
    }
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      bool progressed = false;
      for (Slot& sl : slots) {
        if (!sl.busy) continue;
        const cudaError_t q = cudaStreamQuery(sl.stream);
        if (q == cudaSuccess) {
          finish(sl);
          progressed = true;
        } else if (q != cudaErrorNotReady) {
          fatal = RC_E_CUDA;
          finish(sl);
          progressed = true;
        }
      }
      if (progressed) cv_done.notify_all();
      admit();
      bool any_busy = false;
      for (Slot& sl : slots) any_busy |= sl.busy;
      if (stop && !any_busy && pending.empty()) break;
      if (any_busy) {
        // poll the streams again shortly
        cv_work.wait_for(lk, std::chrono::microseconds(20));
      } else {
        cv_work.wait(lk, [&] { return stop || !pending.empty(); });
      }
    }
  }
};

extern "C" {

rc_status rc_server_create(const rc_server_opts* opts, rc_server** out) {
  if (!opts || !out || opts->memory_bytes < 256 || opts->slots == 0 || opts->slots > 64) return RC_E_INVALID;
  *out = nullptr;
  rc_server* s = new (std::nothrow) rc_server();
  if (!s) return RC_E_NOMEM;
  s->opts = *opts;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return RC_E_CUDA;
  }
  if (cudaMalloc(reinterpret_cast<void**>(&s->pool_base), opts->memory_bytes) != cudaSuccess) {
    delete s;
    return RC_E_NOMEM;
  }
  s->pool.reset(opts->memory_bytes);
  s->slots.resize(opts->slots);
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (Slot& x : s->slots)
        if (x.stream) cudaStreamDestroy(x.stream);
      cudaFree(s->pool_base);
      delete s;
      return RC_E_CUDA;
    }
  }
  try {
    s->th = std::thread([s] { s->loop(); });
  } catch (...) {
    for (Slot& x : s->slots) cudaStreamDestroy(x.stream);
    cudaFree(s->pool_base);
    delete s;
    return RC_E_NOMEM;
  }
  *out = s;
  return RC_OK;
}

rc_status rc_server_submit(rc_server* s, rc_model* m, uint64_t* request) {
  if (!s || !m || !request) return RC_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return RC_E_INVALID;
  Request r{s->next_id++, m, now_s()};
  *request = r.id;
  s->pending.push_back(r);
  s->cv_work.notify_one();
  return RC_OK;
}

rc_status rc_server_poll(rc_server* s, rc_server_done* out, size_t cap, size_t* n_out, int wait_ms) {
  if (!s || !n_out || (cap && !out)) return RC_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  size_t n = 0;
  while (n < cap && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  *n_out = n;
  return s->fatal;
}

rc_status rc_server_stats(rc_server* s, uint64_t* pending, uint64_t* in_flight) {
  if (!s) return RC_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (pending) *pending = s->pending.size();
  if (in_flight) *in_flight = s->in_flight;
  return RC_OK;
}

rc_status rc_server_destroy(rc_server* s) {
  if (!s) return RC_E_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  const rc_status st = s->fatal;
  for (Slot& sl : s->slots) cudaStreamDestroy(sl.stream);
  cudaFree(s->pool_base);
  delete s;
  return st;
}

}  // extern "C"
