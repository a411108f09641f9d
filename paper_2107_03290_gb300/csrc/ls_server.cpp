// Serving loop of the learned sort: continuous batching of sort requests.
//
// A dispatcher thread admits queued requests, in arrival order, while the
// bytes of the admitted requests (keys + scratch) stay within the HBM budget
// and the number on the GPU stays below max_inflight.  Whatever has arrived is
// launched together: the small requests of one key type go through one
// batched launch sequence (ls_sort_batch), larger ones through the full
// learned sort, on the server's streams in turn, so requests overlap on the
// device.  Completion is detected with CUDA events; waiters get queue /
// device / total latency.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ls.h"
#include "ls_call.h"

namespace ls {
constexpr uint32_t ERR_TIMEOUT_BIT = 1u, ERR_BOUNDS_BIT = 2u;
}

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t SERVER_BATCH_MAX = LS_SERVER_BATCH_MAX;  // requests this small are batched

struct Request {
  uint64_t ticket;
  void* keys;
  const void* src;       // optional device source copied into keys first
  size_t n;
  ls_dtype dt;
  uint64_t bytes;
  Clock::time_point t_submit, t_launch, t_done;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  int stream = -1;
  int slot = -1;          // the request's status block (device) and pinned word (host)
  bool done = false;
  ls_request_stats st{};
};

}  // namespace

struct ls_server {
  ls_server_config cfg{};
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::vector<Request*> inflight;
  std::unordered_map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  uint64_t inflight_bytes = 0;
  uint32_t rr = 0;
  ls::CallStatus* dstat = nullptr;   // device, max_inflight blocks (one per request slot)
  uint32_t* hstat = nullptr;         // pinned, max_inflight words
  std::vector<int> free_slots;
  bool stop = false;
  std::thread th;
};

static uint64_t request_bytes(size_t n, ls_dtype dt, bool in_place) {
  const uint64_t w = (dt == LS_F64 || dt == LS_U64) ? 8 : 4;
  if (in_place && n > SERVER_BATCH_MAX) {  // keys + the in-place workspace
    ls_params p;
    ls_default_params(&p);
    p.flags |= LS_FLAG_IN_PLACE;
    return n * w + ls_workspace_bytes(n, dt, &p);
  }
  return 2 * n * w + (64ull << 20);  // keys + scratch + model/job space
}

static void dispatcher(ls_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // retire finished requests
    for (size_t i = 0; i < s->inflight.size();) {
      Request* r = s->inflight[i];
      if (cudaEventQuery(r->ev_end) == cudaSuccess) {
        r->t_done = Clock::now();
        float ms = 0;
        cudaEventElapsedTime(&ms, r->ev_start, r->ev_end);
        r->st.device_ms = ms;
        r->st.queue_ms = std::chrono::duration<double, std::milli>(r->t_launch - r->t_submit).count();
        r->st.total_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
        // device status copied behind the sort (no stream synchronization)
        if (r->st.status == LS_OK && r->slot >= 0) {
          const uint32_t w = s->hstat[r->slot];
          r->st.status = (w & ls::ERR_TIMEOUT_BIT) ? LS_ERR_TIMEOUT
                         : ((w & ls::ERR_BOUNDS_BIT) ? LS_ERR_CUDA : LS_OK);
        }
        if (r->slot >= 0) s->free_slots.push_back(r->slot);
        r->done = true;
        s->inflight_bytes -= r->bytes;
        s->inflight[i] = s->inflight.back();
        s->inflight.pop_back();
        s->cv_done.notify_all();
      } else {
        ++i;
      }
    }
    // admit while budget and slots allow (arrival order)
    std::vector<Request*> adm;
    while (!s->queue.empty() && s->inflight.size() + adm.size() < s->cfg.max_inflight &&
           s->inflight_bytes + s->queue.front()->bytes <= s->cfg.hbm_budget_bytes) {
      Request* r = s->queue.front();
      s->queue.pop_front();
      s->inflight_bytes += r->bytes;
      r->slot = s->free_slots.back();  // max_inflight slots for max_inflight requests
      s->free_slots.pop_back();
      adm.push_back(r);
    }
    if (!adm.empty()) {
      // the admitted requests belong to this thread now: launch them without
      // holding the lock, so that submit() and wait() are not held up
      lk.unlock();
      const auto now = Clock::now();
      auto prologue = [&](Request* r, cudaStream_t st, int si) {
        r->stream = si;
        r->t_launch = now;
        if (r->src && r->n)
          cudaMemcpyAsync(r->keys, r->src, r->n * ((r->dt == LS_F64 || r->dt == LS_U64) ? 8 : 4),
                          cudaMemcpyDeviceToDevice, st);
        cudaEventRecord(r->ev_start, st);
      };
      // each launch reports into the status block of its (first) request,
      // cleared on the stream first; its word is copied to every request it
      // served, behind the sort
      auto opts = [&](int slot, cudaStream_t st) {
        cudaMemsetAsync(&s->dstat[slot], 0, sizeof(ls::CallStatus), st);
        ls::CallOpts o;
        o.fold_to = &s->dstat[slot];
        o.stall = s->cfg.debug_stall;
        o.spin_limit = s->cfg.debug_spin_limit;
        return o;
      };
      for (int dt = LS_F64; dt <= LS_U32; ++dt) {  // one batched launch per key type
        std::vector<Request*> grp;
        for (Request* r : adm)
          if (r->dt == dt && r->n <= SERVER_BATCH_MAX) grp.push_back(r);
        if (grp.empty()) continue;
        const int si = (int)(s->rr++ % s->streams.size());
        cudaStream_t st = s->streams[si];
        std::vector<void*> ptrs;
        std::vector<size_t> ns;
        for (Request* r : grp) { prologue(r, st, si); ptrs.push_back(r->keys); ns.push_back(r->n); }
        const int lead = grp[0]->slot;
        const ls::CallOpts o = opts(lead, st);
        const ls_status rc = ls::batch_call(ptrs.data(), ns.data(), grp.size(), (ls_dtype)dt, st, &o);
        for (Request* r : grp)  // every copy before any completion event, so that
          cudaMemcpyAsync(&s->hstat[r->slot], &s->dstat[lead].word, sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, st);  // the lead's block outlives them
        for (Request* r : grp) {
          cudaEventRecord(r->ev_end, st);
          if (rc != LS_OK) r->st.status = rc;
        }
      }
      for (Request* r : adm) {  // larger requests: the full learned sort each
        if (r->n <= SERVER_BATCH_MAX) continue;
        const int si = (int)(s->rr++ % s->streams.size());
        cudaStream_t st = s->streams[si];
        prologue(r, st, si);
        const ls::CallOpts o = opts(r->slot, st);
        ls_params prm;
        ls_default_params(&prm);
        if (s->cfg.in_place) prm.flags |= LS_FLAG_IN_PLACE;
        const ls_status rc = ls::sort_call(r->keys, r->n, r->dt, st, &prm, nullptr, &o);
        cudaMemcpyAsync(&s->hstat[r->slot], &s->dstat[r->slot].word, sizeof(uint32_t),
                        cudaMemcpyDeviceToHost, st);
        cudaEventRecord(r->ev_end, st);
        if (rc != LS_OK) r->st.status = rc;
      }
      lk.lock();
      for (Request* r : adm) s->inflight.push_back(r);
    }
    if (s->stop && s->queue.empty() && s->inflight.empty()) break;
    if (s->inflight.empty() && s->queue.empty()) {
      s->cv_work.wait(lk);
    } else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

extern "C" {

ls_status ls_server_create(const ls_server_config* cfg, ls_server** out) {
  if (!out) return LS_ERR_INVALID;
  ls_server* s = new ls_server();
  if (cfg) s->cfg = *cfg;
  if (!s->cfg.hbm_budget_bytes) s->cfg.hbm_budget_bytes = 120ull << 30;
  if (!s->cfg.max_inflight) s->cfg.max_inflight = 64;
  if (!s->cfg.max_queue) s->cfg.max_queue = 4096;
  if (!s->cfg.streams) s->cfg.streams = 8;
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return LS_ERR_CUDA; }
  if (cudaMalloc((void**)&s->dstat, s->cfg.max_inflight * sizeof(ls::CallStatus)) != cudaSuccess) {
    delete s;
    return LS_ERR_NOMEM;
  }
  if (cudaHostAlloc((void**)&s->hstat, s->cfg.max_inflight * sizeof(uint32_t), cudaHostAllocDefault) != cudaSuccess) {
    cudaFree(s->dstat);
    delete s;
    return LS_ERR_NOMEM;
  }
  std::memset(s->hstat, 0, s->cfg.max_inflight * sizeof(uint32_t));
  for (int i = (int)s->cfg.max_inflight - 1; i >= 0; --i) s->free_slots.push_back(i);
  for (uint32_t i = 0; i < s->cfg.streams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : s->streams) cudaStreamDestroy(x);
      cudaFreeHost(s->hstat);
      cudaFree(s->dstat);
      delete s;
      return LS_ERR_CUDA;
    }
    s->streams.push_back(st);
  }
  s->th = std::thread(dispatcher, s);
  *out = s;
  return LS_OK;
}

ls_status ls_server_submit(ls_server* s, void* keys, size_t n, ls_dtype dtype, uint64_t* ticket) {
  return ls_server_submit_from(s, nullptr, keys, n, dtype, ticket);
}

ls_status ls_server_submit_from(ls_server* s, const void* src, void* keys, size_t n,
                                ls_dtype dtype, uint64_t* ticket) {
  if (!s || !ticket || dtype < LS_F64 || dtype > LS_U32 || (n > 0 && !keys)) return LS_ERR_INVALID;
  const uint64_t bytes = request_bytes(n, dtype, s && s->cfg.in_place != 0);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return LS_ERR_CANCELLED;
  if (bytes > s->cfg.hbm_budget_bytes || s->queue.size() >= s->cfg.max_queue) return LS_ERR_BUSY;
  Request* r = new Request();
  r->ticket = s->next_ticket++;
  r->keys = keys;
  r->src = src;
  r->n = n;
  r->dt = dtype;
  r->bytes = bytes;
  r->t_submit = Clock::now();
  cudaEventCreate(&r->ev_start);
  cudaEventCreate(&r->ev_end);
  s->all[r->ticket] = r;
  s->queue.push_back(r);
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return LS_OK;
}

ls_status ls_server_wait(ls_server* s, uint64_t ticket, uint32_t timeout_ms, ls_request_stats* st) {
  if (!s) return LS_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return LS_ERR_INVALID;
  Request* r = it->second;
  auto pred = [&] { return r->done; };
  if (timeout_ms == UINT32_MAX) s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return LS_ERR_TIMEOUT;
  if (st) *st = r->st;
  const ls_status rc = r->st.status;
  cudaEventDestroy(r->ev_start);
  cudaEventDestroy(r->ev_end);
  s->all.erase(it);
  delete r;
  return rc;
}

ls_status ls_server_destroy(ls_server* s) {
  if (!s) return LS_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  s->th.join();
  for (auto& kv : s->all) {
    cudaEventDestroy(kv.second->ev_start);
    cudaEventDestroy(kv.second->ev_end);
    delete kv.second;
  }
  for (auto x : s->streams) cudaStreamDestroy(x);
  if (s->hstat) cudaFreeHost(s->hstat);
  if (s->dstat) cudaFree(s->dstat);
  delete s;
  return LS_OK;
}

}  // extern "C"
