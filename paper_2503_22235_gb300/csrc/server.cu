// Forecast server: continuous batching of latent rollouts on one context.
//
// Requests (a host latent + a lead time) wait in a bounded queue. A worker
// thread admits them into device-resident latent slots while the slot memory
// fits the HBM budget, then runs ticks: in every tick each admitted request
// with steps left takes exactly one processor step (six-hour steps first,
// then one-hour steps, the greedy schedule of Section 2.1). The requests due
// for the same processor are gathered into one contiguous batch (at most
// max_batch latents per launch), stepped together -- the step replayed from
// a CUDA graph captured once per batch size and processor -- and scattered
// back, so a request that arrives while others run joins at the next tick. Kernels are
// row independent, so a result does not depend on what it was batched with.
// A finished request keeps its result in its slot until it is collected by
// wm_server_poll, which frees the slot for the next admission.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wm_internal.cuh"

namespace {

using clk = std::chrono::steady_clock;

// COLLECTING: a poller has taken the finished result and is copying it out;
// every other poll of that id already sees it as collected.
enum ReqState { PENDING = 0, ACTIVE = 1, DONE = 2, COLLECTING = 3 };

struct Req {
  std::vector<float> input;  // host copy of the initial latent until admission
  int n6 = 0, n1 = 0, steps_done = 0;
  int slot = -1;
  ReqState state = PENDING;
  clk::time_point t_arrive, t_done;
};

}  // namespace

struct wm_server {
  wm_ctx* ctx = nullptr;
  int device = 0;
  size_t latent_floats = 0;
  int nslots = 0, max_batch = 1;
  size_t max_pending = 1 << 16;
  float* slab = nullptr;    // nslots latents
  float* stage = nullptr;   // max_batch latents
  cudaStream_t stream = nullptr, io_stream = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, Req> reqs;
  std::vector<int> free_slots;
  std::vector<uint64_t> active;
  std::thread worker;
  bool stopping = false;
  uint64_t next_id = 1;
  wm_status worker_error = WM_OK;
  std::string worker_msg;
  // statistics
  std::vector<double> latencies_ms;
  clk::time_point t_first_arrival, t_last_done;
  bool any_arrival = false;
  long ticks = 0, batched_steps = 0;
  long multi_request_steps = 0;   // batched steps that advanced two or more requests together
  int max_active = 0;
  int max_step_batch = 0;         // most requests advanced by one batched step
};

namespace {

wm_status run_tick(wm_server* s, const std::vector<uint64_t>& ids, const std::vector<int>& slots,
                   const std::vector<int>& which) {
  const size_t lat = s->latent_floats;
  for (int w = 0; w < 2; ++w) {
    std::vector<int> due;
    for (size_t i = 0; i < ids.size(); ++i)
      if (which[i] == w) due.push_back(slots[i]);
    for (size_t b0 = 0; b0 < due.size(); b0 += s->max_batch) {
      const int g = (int)std::min<size_t>(s->max_batch, due.size() - b0);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->max_step_batch = std::max(s->max_step_batch, g);
        if (g >= 2) ++s->multi_request_steps;
      }
      if (wm::processor_step_inplace_ok(s->ctx, g)) {
        // narrow latent: one whole-rollout launch reads and writes the slots in place
        std::vector<float*> xs(g);
        for (int j = 0; j < g; ++j) xs[j] = s->slab + (size_t)due[b0 + j] * lat;
        wm_status st = wm::processor_step_inplace(s->ctx, xs.data(), g, w, s->stream);
        if (st != WM_OK) return st;
      } else {
        // gather into the staging batch, one graph-replayed step, scatter back
        for (int j = 0; j < g; ++j)
          WM_CUDA(cudaMemcpyAsync(s->stage + (size_t)j * lat, s->slab + (size_t)due[b0 + j] * lat, lat * 4,
                                  cudaMemcpyDeviceToDevice, s->stream));
        wm_status st = wm::processor_step_graphed(s->ctx, s->stage, g, w, s->stream);
        if (st != WM_OK) return st;
        for (int j = 0; j < g; ++j)
          WM_CUDA(cudaMemcpyAsync(s->slab + (size_t)due[b0 + j] * lat, s->stage + (size_t)j * lat, lat * 4,
                                  cudaMemcpyDeviceToDevice, s->stream));
      }
      ++s->batched_steps;
    }
  }
  WM_CUDA(cudaStreamSynchronize(s->stream));
  return WM_OK;
}

void worker_main(wm_server* s) {
  cudaSetDevice(s->device);
  const size_t lat = s->latent_floats;
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv.wait(lk, [&] { return s->stopping || !s->active.empty() || (!s->pending.empty() && !s->free_slots.empty()); });
    if (s->stopping) break;
    // ---- admission: pending requests into free slots
    std::vector<std::pair<uint64_t, int>> admitted;
    while (!s->pending.empty() && !s->free_slots.empty()) {
      const uint64_t id = s->pending.front();
      s->pending.pop_front();
      Req& r = s->reqs[id];
      r.slot = s->free_slots.back();
      s->free_slots.pop_back();
      r.state = ACTIVE;
      admitted.push_back({id, r.slot});
      s->active.push_back(id);
    }
    s->max_active = std::max<int>(s->max_active, (int)s->active.size());
    // host -> slot copies (the input vectors are not touched by clients once queued)
    std::vector<const float*> srcs;
    for (auto& a : admitted) srcs.push_back(s->reqs[a.first].input.data());
    lk.unlock();
    wm_status st = WM_OK;
    for (size_t i = 0; i < admitted.size() && st == WM_OK; ++i) {
      cudaError_t e = cudaMemcpyAsync(s->slab + (size_t)admitted[i].second * lat, srcs[i], lat * 4,
                                      cudaMemcpyHostToDevice, s->stream);
      if (e != cudaSuccess) st = wm::cuda_fail(e, "server admission copy");
    }
    if (st == WM_OK && !admitted.empty()) {
      cudaError_t e = cudaStreamSynchronize(s->stream);
      if (e != cudaSuccess) st = wm::cuda_fail(e, "server admission copy");
    }
    lk.lock();
    for (auto& a : admitted) {
      std::vector<float>().swap(s->reqs[a.first].input);
    }
    // ---- one tick over the active requests
    std::vector<uint64_t> ids;
    std::vector<int> slots, which;
    const auto now0 = clk::now();
    for (uint64_t id : s->active) {
      Req& r = s->reqs[id];
      if (r.steps_done >= r.n6 + r.n1) continue;  // lead 0: finishes below without a step
      ids.push_back(id);
      slots.push_back(r.slot);
      which.push_back(r.steps_done < r.n6 ? WM_P6 : WM_P1);
    }
    (void)now0;
    if (st == WM_OK && !ids.empty()) {
      lk.unlock();
      st = run_tick(s, ids, slots, which);
      lk.lock();
      ++s->ticks;
    }
    if (st != WM_OK) {
      s->worker_error = st;
      s->worker_msg = wm_last_error();
      s->stopping = true;
      s->cv.notify_all();
      break;
    }
    const auto now = clk::now();
    for (uint64_t id : ids) s->reqs[id].steps_done++;
    std::vector<uint64_t> still;
    for (uint64_t id : s->active) {
      Req& r = s->reqs[id];
      if (r.steps_done >= r.n6 + r.n1) {
        r.state = DONE;
        r.t_done = now;
        s->t_last_done = now;
        s->latencies_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_arrive).count());
      } else {
        still.push_back(id);
      }
    }
    s->active.swap(still);
    s->cv.notify_all();
  }
}

}  // namespace

extern "C" {

wm_status wm_server_start(wm_ctx* ctx, size_t hbm_budget_bytes, int max_batch, wm_server** out) {
  if (!ctx || !out || max_batch < 1) return wm::fail(WM_ERR_INVALID_ARG, "bad server arguments");
  *out = nullptr;
  size_t lat = 0, ws_bytes = 0;
  wm_status st = wm_ctx_sizes(ctx, max_batch, &lat, &ws_bytes);
  if (st != WM_OK) return st;
  const size_t lat_bytes = lat * 4;
  const size_t fixed = ws_bytes + (size_t)max_batch * lat_bytes;  // workspace + staging batch
  if (hbm_budget_bytes < fixed + lat_bytes)
    return wm::fail(WM_ERR_INVALID_ARG, "HBM budget too small: need at least " + std::to_string(fixed + lat_bytes) +
                                            " bytes for max_batch " + std::to_string(max_batch) + " and one slot");
  wm_server* s = new wm_server();
  s->ctx = ctx;
  cudaGetDevice(&s->device);
  s->latent_floats = lat;
  s->max_batch = max_batch;
  s->nslots = (int)std::min<size_t>((hbm_budget_bytes - fixed) / lat_bytes, 1 << 20);
  cudaError_t e = cudaMalloc(&s->slab, (size_t)s->nslots * lat_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->stage, (size_t)max_batch * lat_bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->io_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->slab);
    cudaFree(s->stage);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->io_stream) cudaStreamDestroy(s->io_stream);
    delete s;
    return wm::fail(WM_ERR_OOM, "server slot allocation failed");
  }
  st = wm_ctx_reserve(ctx, max_batch);
  if (st != WM_OK) {
    cudaFree(s->slab);
    cudaFree(s->stage);
    cudaStreamDestroy(s->stream);
    cudaStreamDestroy(s->io_stream);
    delete s;
    return st;
  }
  for (int i = s->nslots - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return WM_OK;
}

wm_status wm_server_submit(wm_server* s, const float* host_latent, int lead_hours, uint64_t* req_id) {
  if (!s || !host_latent || !req_id) return wm::fail(WM_ERR_INVALID_ARG, "bad submit arguments");
  if (lead_hours < 0) return wm::fail(WM_ERR_INVALID_ARG, "lead time must be >= 0");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->worker_error != WM_OK) return wm::fail(s->worker_error, "server stopped: " + s->worker_msg);
  if (s->stopping) return wm::fail(WM_ERR_INVALID_ARG, "server is stopping");
  if (s->pending.size() >= s->max_pending) return wm::fail(WM_ERR_BUSY, "server queue is full");
  const uint64_t id = s->next_id++;
  Req& r = s->reqs[id];
  r.input.assign(host_latent, host_latent + s->latent_floats);
  wm_schedule(lead_hours, &r.n6, &r.n1);
  r.t_arrive = clk::now();
  if (!s->any_arrival) {
    s->any_arrival = true;
    s->t_first_arrival = r.t_arrive;
  }
  s->pending.push_back(id);
  *req_id = id;
  s->cv.notify_all();
  return WM_OK;
}

wm_status wm_server_poll(wm_server* s, uint64_t req_id, float* host_out, int* done, double* latency_ms) {
  if (!s || !done) return wm::fail(WM_ERR_INVALID_ARG, "bad poll arguments");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end() || it->second.state == COLLECTING)
    return wm::fail(WM_ERR_NOT_FOUND, "unknown or already collected request id");
  *done = 0;
  if (it->second.state != DONE) {
    if (s->worker_error != WM_OK) return wm::fail(s->worker_error, "server stopped: " + s->worker_msg);
    return WM_OK;
  }
  // Claim the result under the lock: a concurrent poll of the same id now
  // gets WM_ERR_NOT_FOUND, so the slot is copied out and released once.
  it->second.state = COLLECTING;
  const int slot = it->second.slot;
  const double lat_ms = std::chrono::duration<double, std::milli>(it->second.t_done - it->second.t_arrive).count();
  if (host_out) {
    lk.unlock();
    cudaError_t e = cudaMemcpyAsync(host_out, s->slab + (size_t)slot * s->latent_floats, s->latent_floats * 4,
                                    cudaMemcpyDeviceToHost, s->io_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->io_stream);
    lk.lock();
    if (e != cudaSuccess) {
      // the result is still in its slot: leave it collectable
      auto again = s->reqs.find(req_id);
      if (again != s->reqs.end()) again->second.state = DONE;
      return wm::cuda_fail(e, "server result copy");
    }
  }
  if (latency_ms) *latency_ms = lat_ms;
  s->free_slots.push_back(slot);
  s->reqs.erase(req_id);
  *done = 1;
  s->cv.notify_all();
  return WM_OK;
}

wm_status wm_server_stats(wm_server* s, double* out) {
  if (!s || !out) return wm::fail(WM_ERR_INVALID_ARG, "bad stats arguments");
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> v = s->latencies_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double q) -> double {
    if (v.empty()) return 0.0;
    const double pos = q * (v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
  };
  double mean = 0;
  for (double x : v) mean += x;
  if (!v.empty()) mean /= v.size();
  const double span_s =
      s->any_arrival && !v.empty() ? std::chrono::duration<double>(s->t_last_done - s->t_first_arrival).count() : 0.0;
  out[0] = (double)v.size();
  out[1] = pct(0.50);
  out[2] = pct(0.99);
  out[3] = mean;
  out[4] = span_s > 0 ? v.size() / span_s : 0.0;
  out[5] = (double)s->max_active;
  out[6] = (double)s->ticks;
  out[7] = (double)s->batched_steps;
  out[8] = (double)s->nslots;
  out[9] = (double)s->max_step_batch;
  out[10] = (double)s->multi_request_steps;
  return WM_OK;
}

wm_status wm_server_stop(wm_server* s) {
  if (!s) return WM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  const wm_status err = s->worker_error;
  const std::string msg = s->worker_msg;
  cudaStreamSynchronize(s->stream);
  cudaFree(s->slab);
  cudaFree(s->stage);
  cudaStreamDestroy(s->stream);
  cudaStreamDestroy(s->io_stream);
  delete s;
  if (err != WM_OK) return wm::fail(err, "server worker failed: " + msg);
  return WM_OK;
}

}  // extern "C"
