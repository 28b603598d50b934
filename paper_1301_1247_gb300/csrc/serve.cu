// A serving loop over built solvers: requests (geometry, incidence angle) arrive at any
// time from any thread; `slots` worker threads, each with its own CUDA stream, take every
// request queued for one geometry at the moment they become free and solve them with
// one hbs_solve call (which groups the angles by Bloch phase, Remark 3.1).  Requests that
// arrive while other batches are on the device join the next batch a slot takes, so
// under load the batches grow and several of them overlap on the GPU.  Geometries are
// admitted against a device-memory budget.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "handle.hpp"

namespace hbs {

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id;
  int64_t geometry;
  double theta;
  Clock::time_point t_submit;
};

struct Done {
  hbs_status status = HBS_OK;
  AngleResult angle;
  bool illcond = false;
};

}  // namespace

struct Server {
  size_t budget = 0, resident = 0;
  int slots = 1, max_batch = 256, device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::map<int64_t, const hbs_handle*> geoms;
  std::map<int64_t, size_t> geom_bytes;
  std::map<int64_t, int> geom_busy;
  std::deque<Request> queue;
  std::map<int64_t, Done> done;
  int64_t next_geom = 1, next_req = 1;
  int64_t submitted = 0, completed = 0, batches = 0, batched_requests = 0;
  std::vector<double> latencies;
  Clock::time_point t_first{}, t_last{};
  bool any = false;
  std::vector<std::thread> workers;

  void worker() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
      std::vector<Request> batch;
      const hbs_handle* h = nullptr;
      int64_t g = 0;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || !queue.empty(); });
        if (queue.empty()) break;  // stopping and nothing left
        g = queue.front().geometry;
        for (auto it = queue.begin(); it != queue.end() && (int)batch.size() < max_batch;) {
          if (it->geometry == g) {
            batch.push_back(*it);
            it = queue.erase(it);
          } else {
            ++it;
          }
        }
        h = geoms.count(g) ? geoms[g] : nullptr;
        ++geom_busy[g];
      }
      std::vector<double> th(batch.size());
      for (size_t i = 0; i < batch.size(); ++i) th[i] = batch[i].theta;
      hbs_result* res = nullptr;
      hbs_status stt = h ? hbs_solve(const_cast<hbs_handle*>(h), th.data(), (int64_t)th.size(), st, &res)
                         : HBS_ERR_INVALID_ARG;
      const auto t_end = Clock::now();
      {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t i = 0; i < batch.size(); ++i) {
          Done d;
          d.status = stt;
          if (res && (stt == HBS_OK || stt == HBS_WARN_ILLCOND)) {
            d.angle = res->r.angles[i];
            d.illcond = res->r.illcond;
          }
          done[batch[i].id] = std::move(d);
          latencies.push_back(std::chrono::duration<double>(t_end - batch[i].t_submit).count());
        }
        completed += (int64_t)batch.size();
        ++batches;
        batched_requests += (int64_t)batch.size();
        t_last = t_end;
        --geom_busy[g];
      }
      if (res) hbs_result_free(res);
      cv_done.notify_all();
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
};

}  // namespace hbs

struct hbs_server {
  hbs::Server s;
};

using namespace hbs;

extern "C" {

hbs_status hbs_server_create(size_t hbm_budget_bytes, int slots, int max_batch, hbs_server** out) {
  if (!out || slots < 1 || slots > 64 || max_batch < 1) {
    set_last_error("bad arguments to hbs_server_create");
    return HBS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  hbs_server* sv = new (std::nothrow) hbs_server();
  if (!sv) {
    set_last_error("host allocation failed");
    return HBS_ERR_OOM;
  }
  Server& S = sv->s;
  S.budget = hbm_budget_bytes;
  S.slots = slots;
  S.max_batch = max_batch;
  if (cudaGetDevice(&S.device) != cudaSuccess) {
    cudaGetLastError();
    delete sv;
    set_last_error("no CUDA device");
    return HBS_ERR_CUDA;
  }
  for (int i = 0; i < slots; ++i) S.workers.emplace_back([&S] { S.worker(); });
  *out = sv;
  return HBS_OK;
}

hbs_status hbs_server_add(hbs_server* sv, const hbs_handle* h, int64_t* geometry_id) {
  if (!sv || !h || !geometry_id) {
    set_last_error("bad arguments to hbs_server_add");
    return HBS_ERR_INVALID_ARG;
  }
  Server& S = sv->s;
  const size_t bytes = h->h.device_bytes();
  std::lock_guard<std::mutex> lk(S.mu);
  if (S.budget && S.resident + bytes > S.budget) {
    set_last_error("geometry does not fit in the server's device-memory budget");
    return HBS_ERR_OOM;
  }
  const int64_t id = S.next_geom++;
  S.geoms[id] = h;
  S.geom_bytes[id] = bytes;
  S.geom_busy[id] = 0;
  S.resident += bytes;
  *geometry_id = id;
  return HBS_OK;
}

hbs_status hbs_server_remove(hbs_server* sv, int64_t geometry_id) {
  if (!sv) return HBS_ERR_INVALID_ARG;
  Server& S = sv->s;
  std::unique_lock<std::mutex> lk(S.mu);
  if (!S.geoms.count(geometry_id)) {
    set_last_error("unknown geometry id");
    return HBS_ERR_INVALID_ARG;
  }
  // wait until no queued or running request refers to it
  S.cv_done.wait(lk, [&] {
    if (S.geom_busy[geometry_id] > 0) return false;
    for (const auto& r : S.queue)
      if (r.geometry == geometry_id) return false;
    return true;
  });
  S.resident -= S.geom_bytes[geometry_id];
  S.geoms.erase(geometry_id);
  S.geom_bytes.erase(geometry_id);
  S.geom_busy.erase(geometry_id);
  return HBS_OK;
}

hbs_status hbs_server_submit(hbs_server* sv, int64_t geometry_id, double theta, int64_t* request_id) {
  if (!sv || !request_id || !(theta > -M_PI && theta < 0.0)) {
    set_last_error("bad arguments to hbs_server_submit");
    return HBS_ERR_INVALID_ARG;
  }
  Server& S = sv->s;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    if (!S.geoms.count(geometry_id)) {
      set_last_error("unknown geometry id");
      return HBS_ERR_INVALID_ARG;
    }
    const auto now = Clock::now();
    if (!S.any) {
      S.t_first = now;
      S.any = true;
    }
    const int64_t id = S.next_req++;
    S.queue.push_back({id, geometry_id, theta, now});
    ++S.submitted;
    *request_id = id;
  }
  S.cv_work.notify_one();
  return HBS_OK;
}

hbs_status hbs_server_wait(hbs_server* sv, int64_t request_id, double timeout_s, hbs_result** out) {
  if (!sv || !out) return HBS_ERR_INVALID_ARG;
  *out = nullptr;
  Server& S = sv->s;
  std::unique_lock<std::mutex> lk(S.mu);
  const bool ok = S.cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                     [&] { return S.done.count(request_id) > 0; });
  if (!ok) {
    set_last_error("request not finished within the timeout");
    return HBS_ERR_TIMEOUT;
  }
  Done d = std::move(S.done[request_id]);
  S.done.erase(request_id);
  lk.unlock();
  if (d.status != HBS_OK && d.status != HBS_WARN_ILLCOND) return d.status;
  hbs_result* r = new (std::nothrow) hbs_result();
  if (!r) return HBS_ERR_OOM;
  r->r.angles.push_back(std::move(d.angle));
  r->r.illcond = d.illcond;
  *out = r;
  return d.status;
}

hbs_status hbs_server_stats(hbs_server* sv, hbs_server_stats_t* st) {
  if (!sv || !st) return HBS_ERR_INVALID_ARG;
  Server& S = sv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = S.submitted;
  st->completed = S.completed;
  st->batches = S.batches;
  st->mean_batch = S.batches ? (double)S.batched_requests / S.batches : 0.0;
  st->resident_bytes = S.resident;
  if (!S.latencies.empty()) {
    std::vector<double> v = S.latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    st->p50_latency_s = pct(0.50);
    st->p99_latency_s = pct(0.99);
    st->max_latency_s = v.back();
    const double span = std::chrono::duration<double>(S.t_last - S.t_first).count();
    st->solves_per_s = span > 0 ? (double)S.completed / span : 0.0;
  }
  return HBS_OK;
}

void hbs_server_free(hbs_server* sv) {
  if (!sv) return;
  Server& S = sv->s;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    S.stop = true;
  }
  S.cv_work.notify_all();
  for (auto& t : S.workers) t.join();
  delete sv;
}

}  // extern "C"
