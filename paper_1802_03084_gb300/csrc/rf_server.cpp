// rf_server.cpp -- serving: segments of mixed shapes searched as they arrive,
// with plans kept resident on the device, admission by HBM budget and
// several segments in flight on their own streams (continuous batching).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "realfast_gb300.h"
#include "rf_engine.h"

namespace {

double now_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// A deep copy of a plan description; `key` identifies equal descriptions.
struct DescCopy {
  rf_plan_desc d{};
  std::vector<double> ant, freq, dm;
  std::vector<int32_t> dt;
  std::string key;

  explicit DescCopy(const rf_plan_desc& in) : d(in) {
    ant.assign(in.ant_uvw_m, in.ant_uvw_m + 3 * in.nant);
    freq.assign(in.freq_hz, in.freq_hz + in.nchan);
    dm.assign(in.dm_list, in.dm_list + in.ndm);
    dt.assign(in.dt_list, in.dt_list + in.ndt);
    d.ant_uvw_m = ant.data();
    d.freq_hz = freq.data();
    d.dm_list = dm.data();
    d.dt_list = dt.data();
    auto put = [this](const void* p, size_t n) { key.append(static_cast<const char*>(p), n); };
    put(&d.nant, 4);
    put(&d.nchan, 4);
    put(&d.npol, 4);
    put(&d.inttime_s, 8);
    put(&d.npix, 4);
    put(&d.cell_rad, 8);
    put(&d.ndm, 4);
    put(&d.ndt, 4);
    put(&d.threshold_sigma, 8);
    put(&d.flags, 4);
    put(&d.max_nint, 4);
    put(ant.data(), ant.size() * 8);
    put(freq.data(), freq.size() * 8);
    put(dm.data(), dm.size() * 8);
    put(dt.data(), dt.size() * 4);
  }
};

struct Request {
  int64_t id = 0;
  std::unique_ptr<DescCopy> desc;
  const void* vis = nullptr;
  int32_t nint = 0;
  uint64_t need_bytes = 0;
  rf_request_info info{};
  std::vector<rf_candidate> cands;
  std::string err;  // message of a failed search
};

struct PlanEntry {
  std::string key;
  rf_plan* plan = nullptr;
  uint64_t bytes = 0;
  bool busy = false;
  double last_used = 0.0;
};

}  // namespace

struct rf_server {
  int device = 0;
  int slots = 1;
  uint64_t budget = 0;
  int64_t wave_images = 0;
  std::chrono::steady_clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv_work;  // workers: a request may be admissible
  std::condition_variable cv_done;  // waiters: a request finished
  std::deque<Request*> pending;
  std::map<int64_t, std::unique_ptr<Request>> requests;
  std::vector<std::unique_ptr<PlanEntry>> plans;
  uint64_t resident = 0;
  int64_t next_id = 1;
  bool stopping = false;
  std::vector<std::thread> workers;

  // With `mu` held: a plan for the head request, if it can start now.  An
  // idle resident plan of the same description is reused; otherwise, if the
  // budget (after evicting idle plans) has room, a slot is reserved and the
  // plan is created by the worker outside the lock.
  PlanEntry* admit(Request* r, bool* create) {
    *create = false;
    for (auto& e : plans)
      if (!e->busy && e->key == r->desc->key) return e.get();
    // evict idle plans, least recently used first, until the new one fits
    while (resident + r->need_bytes > budget) {
      PlanEntry* lru = nullptr;
      for (auto& e : plans)
        if (!e->busy && e->plan && (!lru || e->last_used < lru->last_used)) lru = e.get();
      if (!lru) return nullptr;
      rf_plan_destroy(lru->plan);
      resident -= lru->bytes;
      plans.erase(std::find_if(plans.begin(), plans.end(), [lru](const auto& e) { return e.get() == lru; }));
    }
    plans.push_back(std::make_unique<PlanEntry>());
    PlanEntry* e = plans.back().get();
    e->key = r->desc->key;
    e->bytes = r->need_bytes;
    resident += e->bytes;
    *create = true;
    return e;
  }

  void worker_loop();
};

void rf_server::worker_loop() {
  cudaSetDevice(device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    Request* r = nullptr;
    PlanEntry* pe = nullptr;
    bool create = false;
    for (;;) {
      if (!pending.empty()) {
        // the budget is also checked against what the device has free
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        Request* head = pending.front();
        bool fits_now = true;
        bool reusable = false;
        for (auto& e : plans) reusable = reusable || (!e->busy && e->key == head->desc->key);
        if (!reusable && head->need_bytes + (512ull << 20) > free_b) {
          // evicting idle plans may free enough; admit() evicts within the budget
          uint64_t idle = 0;
          for (auto& e : plans)
            if (!e->busy) idle += e->bytes;
          fits_now = head->need_bytes + (512ull << 20) <= free_b + idle;
        }
        if (fits_now) pe = admit(head, &create);
        if (pe) {
          r = head;
          pending.pop_front();
          pe->busy = true;
          break;
        }
      }
      if (stopping && pending.empty()) {
        lk.unlock();
        cudaStreamDestroy(st);
        return;
      }
      cv_work.wait(lk);
    }
    r->info.start_s = now_since(t0);
    r->info.plan_reused = create ? 0 : 1;
    lk.unlock();

    rf_status s = RF_OK;
    std::string err;
    if (create) {
      s = rf_plan_create(&r->desc->d, &pe->plan);
      if (s == RF_OK && wave_images > 0) s = rf_plan_set_tuning(pe->plan, RF_TUNE_WAVE_IMAGES, wave_images);
      if (s != RF_OK) err = rf_last_error();
    }
    if (s == RF_OK) {
      int64_t nimg = 0;
      rf_count_images(pe->plan, r->nint, &nimg);
      r->info.n_images = nimg;
      r->cands.resize((size_t)std::max<int64_t>(nimg, 1));
      size_t n = 0;
      s = rf_search_segment(pe->plan, r->vis, r->nint, st, r->cands.data(), r->cands.size(), &n);
      if (s != RF_OK) err = rf_last_error();
      r->cands.resize(std::min(n, r->cands.size()));
      r->info.n_candidates = n;
    }

    lk.lock();
    if (!pe->plan) {  // creation failed: give the reservation back
      resident -= pe->bytes;
      plans.erase(std::find_if(plans.begin(), plans.end(), [pe](const auto& e) { return e.get() == pe; }));
    } else {
      pe->busy = false;
      pe->last_used = now_since(t0);
    }
    r->info.status = s;
    r->info.done = 1;
    r->info.done_s = now_since(t0);
    if (s != RF_OK) r->cands.clear();
    r->err = err;
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" {

rf_status rf_server_create(const rf_server_desc* desc, rf_server** out) {
  if (!desc || !out) {
    rf::set_last_error("rf_server_create: NULL argument");
    return RF_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (desc->slots < 1 || desc->slots > 16 || desc->hbm_budget_bytes == 0 || desc->wave_images < 0) {
    rf::set_last_error("rf_server_create: slots must be 1..16 and the HBM budget > 0");
    return RF_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    rf::set_last_error("rf_server_create: no CUDA device");
    return RF_ERR_NO_DEVICE;
  }
  if (desc->device < 0 || desc->device >= ndev) {
    rf::set_last_error("rf_server_create: device out of range");
    return RF_ERR_INVALID_ARG;
  }
  rf_server* sv = new rf_server();
  sv->device = desc->device;
  sv->slots = desc->slots;
  sv->budget = desc->hbm_budget_bytes;
  sv->wave_images = desc->wave_images;
  sv->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < sv->slots; ++i) sv->workers.emplace_back([sv] { sv->worker_loop(); });
  *out = sv;
  return RF_OK;
}

rf_status rf_server_submit(rf_server* sv, const rf_plan_desc* desc, const void* vis, int32_t nint, int64_t* ticket) {
  if (!sv || !desc || !vis || !ticket) {
    rf::set_last_error("rf_server_submit: NULL argument");
    return RF_ERR_INVALID_ARG;
  }
  if (nint < 1 || nint > desc->max_nint) {
    rf::set_last_error("rf_server_submit: nint out of [1, desc->max_nint]");
    return RF_ERR_SHAPE;
  }
  rf_plan_desc d = *desc;
  d.device = sv->device;
  d.flags &= ~RF_HOST_ONLY;
  auto r = std::make_unique<Request>();
  r->desc = std::make_unique<DescCopy>(d);
  uint64_t need = 0;
  rf_status s = rf_plan_estimate_bytes(&r->desc->d, sv->wave_images, &need);
  if (s != RF_OK) return s;
  if (need > sv->budget) {
    rf::set_last_error("rf_server_submit: the plan for this segment does not fit in the server's HBM budget");
    return RF_ERR_NO_MEMORY;
  }
  r->need_bytes = need;
  r->vis = vis;
  r->nint = nint;
  std::lock_guard<std::mutex> lk(sv->mu);
  r->id = sv->next_id++;
  r->info.submit_s = now_since(sv->t0);
  *ticket = r->id;
  sv->pending.push_back(r.get());
  sv->requests[r->id] = std::move(r);
  sv->cv_work.notify_all();
  return RF_OK;
}

rf_status rf_server_wait(rf_server* sv, int64_t ticket, int32_t timeout_ms, rf_request_info* info) {
  if (!sv || !info) {
    rf::set_last_error("rf_server_wait: NULL argument");
    return RF_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->requests.find(ticket);
  if (it == sv->requests.end()) {
    rf::set_last_error("rf_server_wait: unknown ticket");
    return RF_ERR_INVALID_ARG;
  }
  Request* r = it->second.get();
  auto done = [r] { return r->info.done != 0; };
  if (timeout_ms < 0) {
    sv->cv_done.wait(lk, done);
  } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    *info = r->info;
    rf::set_last_error("rf_server_wait: request still running");
    return RF_ERR_TIMEOUT;
  }
  *info = r->info;
  if (r->info.status != RF_OK) rf::set_last_error(r->err.c_str());
  return RF_OK;
}

rf_status rf_server_results(rf_server* sv, int64_t ticket, rf_candidate* out, size_t cap, size_t* n_out) {
  if (!sv || !n_out || (cap > 0 && !out)) {
    rf::set_last_error("rf_server_results: NULL argument");
    return RF_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->requests.find(ticket);
  if (it == sv->requests.end() || !it->second->info.done) {
    rf::set_last_error("rf_server_results: unknown or unfinished ticket");
    return RF_ERR_INVALID_ARG;
  }
  Request* r = it->second.get();
  *n_out = r->cands.size();
  const size_t n = std::min(cap, r->cands.size());
  if (n) std::memcpy(out, r->cands.data(), n * sizeof(rf_candidate));
  if (r->cands.size() > cap) {
    rf::set_last_error("rf_server_results: capacity too small");
    return RF_ERR_CAPACITY;
  }
  const rf_status st = (rf_status)r->info.status;
  sv->requests.erase(it);
  return st;
}

rf_status rf_server_destroy(rf_server* sv) {
  if (!sv) return RF_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stopping = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->workers) t.join();
  for (auto& e : sv->plans)
    if (e->plan) rf_plan_destroy(e->plan);
  delete sv;
  return RF_OK;
}

}  // extern "C"
