// pa_server.cu -- continuous-batching request server over the plan ABI.
//
// One scheduler thread issues every batch: device buffers (a stream-ordered
// memory pool), the H2D copy, pa_beamform and the D2H copy, and completion
// polling.  A builder thread creates new plans on a stream of its own, so a
// request with a new descriptor does not hold up batches whose plans are
// resident: the scheduler reserves the plan's memory, queues the build and
// goes on with other requests; a finished build is handed back to the
// scheduler, which alone inserts plans into (and destroys them from) its
// cache.  Callers only enqueue requests and wait for results, so each plan
// object (not thread-safe) is touched by one thread at a time.
//
// Scheduling: requests become visible at their arrival time.  Whenever a
// slot (stream) is free, the oldest visible request whose plan is not busy
// in another slot is taken, with up to max_batch - 1 later visible requests
// of the same descriptor; the batch is admitted if its buffers (and a new
// plan's tables) fit in the device budget next to the batches in flight.
// Completion is detected by polling each slot's event; the request's latency
// is the server-clock time of that detection minus its arrival time.
//
// Tensor memory: compensated plans keep their Kahan totals in TMEM (512
// columns per SM).  Blocks whose columns stay within their register share of
// an SM can share it with any other such blocks; a TMEM-dense plan (see
// pa::plan_tmem) is never in flight together with another compensated batch,
// so no block waits in tcgen05.alloc for another kernel's columns.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pa_internal.cuh"

namespace {

using clock_type = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  pa_plan_desc desc{};
  std::string key;
  size_t key_hash = 0;  // hash of key, compared first
  const void* rf = nullptr;
  float* out = nullptr;
  size_t rf_bytes = 0, out_bytes = 0;
  double arrival = 0, start = 0, done = 0;
  pa_status status = PA_OK;
  int batch = 0;
  float device_ms = 0.f;  // its batch's device time
  bool finished = false;
};

// Idle gaps shorter than this before the next arrival are spun, not slept.
constexpr double kSpinWindow = 1e-3;

struct PlanEntry {
  pa_plan_t plan = nullptr;
  size_t bytes = 0;
  bool busy = false;
  bool building = false;  // queued for, or in, the builder thread
  int tmem_cols = 0;      // > 0: compensated plan (Kahan totals in TMEM)
  bool tmem_dense = false;
  uint64_t last_used = 0;
  int timeouts_seen = 0;  // timed-out waits of this plan already charged to a batch
};

// A plan the builder thread finished (or failed to build).
struct Built {
  std::string key;
  pa_plan_t plan = nullptr;
  pa_status status = PA_OK;
  std::string error;
  size_t bytes = 0;
  int tmem_cols = 0;
  bool tmem_dense = false;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  cudaEvent_t ev_start = nullptr;  // timing pair around the batch's stream work
  cudaEvent_t ev_end = nullptr;
  int* h_timeouts = nullptr;  // pinned copy of the plan's timed-out-wait count after the batch
  bool busy = false;
  std::vector<Request*> reqs;
  size_t bytes = 0;
  PlanEntry* pe = nullptr;
};

std::string plan_key(const pa_plan_desc& d) {
  char buf[640];
  snprintf(buf, sizeof buf,
           "%d|%.17g|%.17g|%.17g|%.17g|%d|%d|%d|%.17g|%.17g|%.17g|%.17g|%d|%u|%d|%.17g|%.17g|%.17g|"
           "%.17g|%.17g|%d|%d|%d",
           d.n_elem, d.pitch_m, d.c_m_s, d.fs_hz, d.t0_s, d.n_samples, d.nx, d.nz, d.x0_m, d.x1_m,
           d.z0_m, d.z1_m, d.order_k, d.outputs, (int)d.rf_dtype, d.f_number, d.f0_hz,
           d.band_lo_hz, d.band_hi_hz, d.dyn_range_db, d.compensated, (int)d.interp,
           (int)d.delay_table);
  return buf;
}

int popc3(uint32_t m) { return (int)((m & 1u) + ((m >> 1) & 1u) + ((m >> 2) & 1u)); }

size_t align_up(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

struct pa_server_s {
  pa_server_config cfg{};
  int device = 0;
  clock_type::time_point t0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::multimap<double, Request*> pending;  // submitted, by arrival time
  std::unordered_map<uint64_t, Request*> by_ticket;
  uint64_t next_ticket = 1;
  bool stop = false;
  // scheduler-thread state
  std::list<Request*> visible;  // arrived, not yet issued, in arrival order
  std::map<std::string, PlanEntry> plans;
  std::vector<Slot> slots;
  cudaMemPool_t pool = nullptr;
  cudaStream_t plan_stream = nullptr;
  uint64_t use_clock = 0;
  int comp_in_flight = 0, dense_in_flight = 0;  // compensated / TMEM-dense batches in flight
  int plans_count = 0;  // plans.size(), kept under mu for pa_server_get_stats
  // builder thread (queue and results guarded by mu)
  std::deque<std::pair<std::string, pa_plan_desc>> build_q;
  std::vector<Built> built;
  std::condition_variable cv_build;
  bool stop_build = false;
  std::thread builder;
  // statistics (guarded by mu)
  uint64_t submitted = 0, completed = 0, failed = 0, batches = 0;
  size_t in_use = 0, peak = 0;
  std::thread th;

  double now() const {
    return std::chrono::duration<double>(clock_type::now() - t0).count();
  }

  void finish(Request* r, pa_status st, double t) {
    // caller holds mu
    r->status = st;
    r->done = t;
    r->finished = true;
    if (st == PA_OK) ++completed;
    else ++failed;
  }

  // Poll slots; returns true if any batch completed.
  bool reap() {
    bool any = false;
    for (auto& s : slots) {
      if (!s.busy) continue;
      cudaError_t e = cudaEventQuery(s.ev);
      if (e == cudaErrorNotReady) continue;
      const double t = now();
      pa_status done = e == cudaSuccess ? PA_OK : PA_ECUDA;
      if (done == PA_OK && *s.h_timeouts > s.pe->timeouts_seen) {
        s.pe->timeouts_seen = *s.h_timeouts;
        done = PA_ETIMEOUT;  // the fused kernel gave up waiting for its staging copies
      }
      float dev_ms = 0.f;
      if (done == PA_OK && cudaEventElapsedTime(&dev_ms, s.ev_start, s.ev_end) != cudaSuccess) {
        cudaGetLastError();
        dev_ms = 0.f;
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        for (Request* r : s.reqs) {
          r->device_ms = dev_ms;
          finish(r, done, t);
        }
        in_use -= s.bytes;
      }
      if (e != cudaSuccess) cudaGetLastError();
      if (s.pe->tmem_cols > 0) {
        --comp_in_flight;
        if (s.pe->tmem_dense) --dense_in_flight;
      }
      s.pe->busy = false;
      s.busy = false;
      s.reqs.clear();
      s.bytes = 0;
      any = true;
    }
    if (any) cv_done.notify_all();
    return any;
  }

  // Destroy least recently used idle plans until `need` more bytes fit and,
  // when a plan is about to be added, the resident plans stay within
  // max_plans.
  void evict_for(size_t need, bool adding_plan) {
    for (;;) {
      size_t cur;
      {
        std::lock_guard<std::mutex> lk(mu);
        cur = in_use;
      }
      const bool over_count =
          (int)plans.size() + (adding_plan ? 1 : 0) > std::max(1, cfg.max_plans);
      if (cur + need <= cfg.device_budget_bytes && !over_count) return;
      auto victim = plans.end();
      for (auto it = plans.begin(); it != plans.end(); ++it) {
        if (it->second.busy || it->second.building) continue;
        if (victim == plans.end() || it->second.last_used < victim->second.last_used) victim = it;
      }
      if (victim == plans.end()) return;
      pa_destroy(victim->second.plan);
      const size_t freed = victim->second.bytes;
      plans.erase(victim);
      {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= freed;
        plans_count = (int)plans.size();
      }
    }
  }

  // Try to issue one batch on slot s; returns true if something was issued
  // or failed (the visible list changed).  The scan walks the queue in
  // arrival order; a request whose plan was already found unable to run in
  // this scan (being built, in flight, held back by the TMEM rule, or
  // waiting for memory for its build) is passed over by comparing its key
  // with those plans' keys, without another lookup in the plan map: with
  // many requests queued behind a few busy plans, a lookup per request made
  // each scheduler pass, and so the reaping of finished batches, slower.
  bool issue(Slot& s) {
    // a TMEM-dense request waiting for the compensated batches in flight to
    // drain holds back later compensated requests, so it is not starved
    bool hold_comp = false;
    std::vector<const Request*> blocked;  // one request per plan that cannot run now
    auto is_blocked = [&](const Request* r) {
      for (const Request* b : blocked)
        if (b->key_hash == r->key_hash && b->key == r->key) return true;
      return false;
    };
    for (auto it = visible.begin(); it != visible.end(); ++it) {
      Request* head = *it;
      if (is_blocked(head)) continue;
      blocked.push_back(head);  // taken back out below if the request runs
      auto pit = plans.find(head->key);
      if (pit == plans.end()) {
        // new descriptor: reserve the plan's memory and queue its build;
        // requests of resident plans go on meanwhile
        pa_plan_desc d = head->desc;
        d.max_batch = cfg.max_batch;
        size_t plan_bytes = 0;
        if (pa_plan_footprint(&d, 0, &plan_bytes) != PA_OK) plan_bytes = 0;
        evict_for(plan_bytes, true);
        {
          std::lock_guard<std::mutex> lk(mu);
          if (in_use + plan_bytes > cfg.device_budget_bytes) continue;  // wait for memory
          in_use += plan_bytes;
          peak = std::max(peak, in_use);
          build_q.emplace_back(head->key, d);
        }
        PlanEntry pe;
        pe.building = true;
        pe.bytes = plan_bytes;
        plans.emplace(head->key, pe);
        {
          std::lock_guard<std::mutex> lk(mu);
          plans_count = (int)plans.size();
        }
        cv_build.notify_one();
        continue;
      }
      if (pit->second.building || pit->second.busy) continue;  // being built / in flight
      if (pit->second.tmem_cols > 0) {
        // TMEM: a dense plan never shares the GPU with another compensated batch
        if (hold_comp) continue;
        if (pit->second.tmem_dense ? comp_in_flight > 0 : dense_in_flight > 0) {
          if (pit->second.tmem_dense) hold_comp = true;
          continue;
        }
      }
      blocked.pop_back();
      std::vector<std::list<Request*>::iterator> pick{it};
      for (auto jt = std::next(it); jt != visible.end() && (int)pick.size() < cfg.max_batch; ++jt)
        if ((*jt)->key_hash == head->key_hash && (*jt)->key == head->key) pick.push_back(jt);
      const int nf = (int)pick.size();
      const size_t buf_rf = align_up(head->rf_bytes * nf), buf_out = align_up(head->out_bytes * nf);
      const size_t need = buf_rf + buf_out;
      evict_for(need, false);
      {
        std::lock_guard<std::mutex> lk(mu);
        if (in_use + need > cfg.device_budget_bytes) return false;  // wait for memory
      }
      PlanEntry& pe = pit->second;
      void* rf_dev = nullptr;
      void* out_dev = nullptr;
      cudaError_t e = cudaEventRecord(s.ev_start, s.st);
      if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&rf_dev, buf_rf, pool, s.st);
      if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&out_dev, buf_out, pool, s.st);
      pa_status st = PA_OK;
      if (e == cudaSuccess) {
        for (int q = 0; q < nf && e == cudaSuccess; ++q) {
          Request* r = *pick[q];
          e = cudaMemcpyAsync((char*)rf_dev + q * r->rf_bytes, r->rf, r->rf_bytes,
                              cudaMemcpyHostToDevice, s.st);
        }
      }
      if (e == cudaSuccess) {
        st = pa_beamform(pe.plan, rf_dev, nf, (float*)out_dev, cfg.stages, s.st);
        for (int q = 0; q < nf && st == PA_OK && e == cudaSuccess; ++q) {
          Request* r = *pick[q];
          e = cudaMemcpyAsync(r->out, (char*)out_dev + q * r->out_bytes, r->out_bytes,
                              cudaMemcpyDeviceToHost, s.st);
        }
      }
      if (rf_dev) cudaFreeAsync(rf_dev, s.st);
      if (out_dev) cudaFreeAsync(out_dev, s.st);
      // a bounded wait that ran out inside the batch shows in the plan's count
      if (e == cudaSuccess && st == PA_OK) {
        *s.h_timeouts = pe.timeouts_seen;
        const int* cnt = pa::plan_timeout_counter(pe.plan);
        if (cnt) e = cudaMemcpyAsync(s.h_timeouts, cnt, sizeof(int), cudaMemcpyDeviceToHost, s.st);
      }
      if (e == cudaSuccess && st == PA_OK) e = cudaEventRecord(s.ev_end, s.st);
      if (e == cudaSuccess && st == PA_OK) e = cudaEventRecord(s.ev, s.st);
      const double t = now();
      std::lock_guard<std::mutex> lk(mu);
      if (e != cudaSuccess || st != PA_OK) {
        cudaGetLastError();
        for (auto& p : pick) finish(*p, st != PA_OK ? st : PA_ECUDA, t);
        for (auto& p : pick) visible.erase(p);
        cv_done.notify_all();
        return true;
      }
      s.busy = true;
      s.pe = &pe;
      if (pe.tmem_cols > 0) {
        ++comp_in_flight;
        if (pe.tmem_dense) ++dense_in_flight;
      }
      s.bytes = buf_rf + buf_out;
      in_use += s.bytes;
      peak = std::max(peak, in_use);
      pe.busy = true;
      pe.last_used = ++use_clock;
      ++batches;
      for (auto& p : pick) {
        (*p)->start = t;
        (*p)->batch = nf;
        s.reqs.push_back(*p);
      }
      for (auto& p : pick) visible.erase(p);
      return true;
    }
    return false;
  }

  // Plans the builder finished: resident from now on (or, if the build
  // failed, every waiting request with that descriptor completes with the
  // build's status).
  bool adopt_built() {
    std::vector<Built> done;
    {
      std::lock_guard<std::mutex> lk(mu);
      done.swap(built);
    }
    if (done.empty()) return false;
    for (Built& b : done) {
      auto pit = plans.find(b.key);
      if (pit == plans.end()) {  // cannot happen: entries being built are never evicted
        if (b.plan) pa_destroy(b.plan);
        continue;
      }
      PlanEntry& pe = pit->second;
      std::lock_guard<std::mutex> lk(mu);
      in_use -= pe.bytes;  // the reservation, replaced by what the plan holds
      if (b.status != PA_OK) {
        const double t = now();
        for (auto it = visible.begin(); it != visible.end();) {
          if ((*it)->key == b.key) {
            finish(*it, b.status, t);
            it = visible.erase(it);
          } else {
            ++it;
          }
        }
        plans.erase(pit);
        plans_count = (int)plans.size();
        cv_done.notify_all();
        continue;
      }
      pe.plan = b.plan;
      pe.bytes = b.bytes;
      pe.building = false;
      pe.tmem_cols = b.tmem_cols;
      pe.tmem_dense = b.tmem_dense;
      in_use += pe.bytes;
      peak = std::max(peak, in_use);
    }
    return true;
  }

  void build_loop() {
    cudaSetDevice(device);
    for (;;) {
      std::pair<std::string, pa_plan_desc> job;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_build.wait(lk, [&] { return stop_build || !build_q.empty(); });
        if (stop_build) return;
        job = build_q.front();
        build_q.pop_front();
      }
      Built b;
      b.key = job.first;
      b.status = pa_plan(&job.second, plan_stream, &b.plan);
      // Batches are launched kernel by kernel: with batch sizes 1..max_batch
      // per plan, graph launch would instantiate a new graph on the
      // scheduler thread for every new (plan, batch size), each a stall of
      // all slots' issue.
      if (b.status == PA_OK) b.status = pa_plan_use_graph(b.plan, 0);
      if (b.status == PA_OK) {
        b.bytes = pa::plan_device_bytes(b.plan);
        pa::plan_tmem(b.plan, &b.tmem_cols, &b.tmem_dense);
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        built.push_back(std::move(b));
      }
      cv_sched.notify_one();
    }
  }

  void loop() {
    cudaSetDevice(device);
    for (;;) {
      double next_arrival = -1;
      {
        std::unique_lock<std::mutex> lk(mu);
        const double t = now();
        while (!pending.empty() && pending.begin()->first <= t) {
          visible.push_back(pending.begin()->second);
          pending.erase(pending.begin());
        }
        if (!pending.empty()) next_arrival = pending.begin()->first;
        bool busy = false;
        for (auto& s : slots) busy = busy || s.busy;
        if (stop && !busy) break;
        if (!busy && visible.empty() && built.empty()) {
          // Nothing to run or poll.  Sleep until shortly before the next
          // arrival (or a submit); the last stretch is spun, since a timed
          // wake-up of the thread comes tens of microseconds late.
          if (next_arrival < 0) {
            cv_sched.wait_for(lk, std::chrono::milliseconds(50));
          } else if (next_arrival - t > kSpinWindow) {
            cv_sched.wait_for(lk, std::chrono::duration<double>(next_arrival - t - kSpinWindow));
          } else {
            lk.unlock();
            std::this_thread::yield();
          }
          continue;
        }
      }
      bool progress = adopt_built();
      progress = reap() || progress;
      if (!stop) {
        for (auto& s : slots) {
          if (s.busy || visible.empty()) continue;
          // what one free slot cannot issue, no other free slot can in this pass
          if (!issue(s)) break;
          progress = true;
        }
      }
      if (!progress) {
        // slots busy or waiting for memory: poll again at once (completion is
        // seen within a yield of the thread, not a timed wake-up later)
        std::this_thread::yield();
      }
    }
  }
};

extern "C" {

pa_status pa_server_create(const pa_server_config* cfg, pa_server_t* out) {
  if (!cfg || !out) {
    pa::set_error_message("pa_server_create: null argument");
    return PA_EINVAL;
  }
  *out = nullptr;
  if (cfg->slots < 1 || cfg->max_batch < 1 || cfg->device_budget_bytes == 0 ||
      (cfg->stages & 7u) == 0 || (cfg->stages & ~7u)) {
    pa::set_error_message("pa_server_create: slots, max_batch, budget and stages must be set");
    return PA_EINVAL;
  }
  pa_server_s* S = new pa_server_s();
  S->cfg = *cfg;
  if (S->cfg.max_plans < 1) S->cfg.max_plans = 1 << 20;
  cudaError_t e = cudaGetDevice(&S->device);
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = S->device;
  if (e == cudaSuccess) e = cudaMemPoolCreate(&S->pool, &props);
  if (e == cudaSuccess) {
    uint64_t keep = UINT64_MAX;  // keep freed blocks cached in the pool
    e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->plan_stream, cudaStreamNonBlocking);
  // Reserve the pool's memory up front (up to the budget, at most three
  // quarters of what is free): growing the pool while batches are in flight
  // stalls the scheduler thread, which showed up as multi-millisecond p99
  // latencies the first time a trace reached a new peak of buffers in flight.
  if (e == cudaSuccess) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
      const size_t want = std::min(cfg->device_budget_bytes, free_b / 4 * 3) & ~(size_t)((1 << 21) - 1);
      void* blk = nullptr;
      if (want > 0 && cudaMallocFromPoolAsync(&blk, want, S->pool, S->plan_stream) == cudaSuccess) {
        cudaFreeAsync(blk, S->plan_stream);
        e = cudaStreamSynchronize(S->plan_stream);
      } else {
        cudaGetLastError();  // a failed reservation only costs the warm-up
      }
    }
  }
  S->slots.resize(cfg->slots);
  for (auto& s : S->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&s.ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&s.ev_end);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_timeouts, sizeof(int));
    if (e == cudaSuccess) *s.h_timeouts = 0;
  }
  if (e != cudaSuccess) {
    pa::set_error_message(cudaGetErrorString(e));
    for (auto& s : S->slots) {
      if (s.st) cudaStreamDestroy(s.st);
      if (s.ev) cudaEventDestroy(s.ev);
      if (s.ev_start) cudaEventDestroy(s.ev_start);
      if (s.ev_end) cudaEventDestroy(s.ev_end);
      if (s.h_timeouts) cudaFreeHost(s.h_timeouts);
    }
    if (S->plan_stream) cudaStreamDestroy(S->plan_stream);
    if (S->pool) cudaMemPoolDestroy(S->pool);
    delete S;
    return PA_ECUDA;
  }
  S->t0 = clock_type::now();
  S->builder = std::thread([S] { S->build_loop(); });
  S->th = std::thread([S] { S->loop(); });
  *out = S;
  return PA_OK;
}

double pa_server_now(pa_server_t S) { return S ? S->now() : 0.0; }

pa_status pa_server_submit(pa_server_t S, const pa_plan_desc* desc, const void* rf_host,
                           float* out_host, double arrival_s, uint64_t* ticket) {
  if (!S || !desc || !rf_host || !out_host || !ticket) {
    pa::set_error_message("pa_server_submit: null argument");
    return PA_EINVAL;
  }
  pa_plan_desc d = *desc;
  d.max_batch = S->cfg.max_batch;
  size_t one = 0;
  pa_status st = pa_plan_footprint(&d, 1, &one);
  if (st != PA_OK) return st;  // message already set
  Request* r = new Request();
  r->desc = d;
  r->key = plan_key(d);
  r->key_hash = std::hash<std::string>{}(r->key);
  r->rf = rf_host;
  r->out = out_host;
  r->rf_bytes = (size_t)d.n_elem * d.n_samples * (d.rf_dtype == PA_RF_F32 ? 4 : 2);
  r->out_bytes = (size_t)popc3(S->cfg.stages) * popc3(d.outputs) * d.nx * d.nz * sizeof(float);
  size_t plan_bytes = 0;
  pa_plan_footprint(&d, 0, &plan_bytes);
  if (plan_bytes + align_up(r->rf_bytes) + align_up(r->out_bytes) > S->cfg.device_budget_bytes) {
    delete r;
    pa::set_error_message("pa_server_submit: one frame needs more device memory than the budget");
    return PA_ENOMEM;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      delete r;
      pa::set_error_message("pa_server_submit: server is stopping");
      return PA_EBUSY;
    }
    r->ticket = S->next_ticket++;
    r->arrival = arrival_s > 0 ? arrival_s : S->now();
    S->pending.emplace(r->arrival, r);
    S->by_ticket[r->ticket] = r;
    ++S->submitted;
    *ticket = r->ticket;
  }
  S->cv_sched.notify_one();
  return PA_OK;
}

pa_status pa_server_wait(pa_server_t S, uint64_t ticket, int32_t timeout_ms,
                         pa_request_result* res) {
  if (!S || !res) {
    pa::set_error_message("pa_server_wait: null argument");
    return PA_EINVAL;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->by_ticket.find(ticket);
  if (it == S->by_ticket.end()) {
    pa::set_error_message("pa_server_wait: unknown ticket (or result already read)");
    return PA_EINVAL;
  }
  Request* r = it->second;
  auto ready = [&] { return r->finished; };
  if (timeout_ms < 0) S->cv_done.wait(lk, ready);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    pa::set_error_message("pa_server_wait: request still pending");
    return PA_ETIMEOUT;
  }
  res->ticket = r->ticket;
  res->status = r->status;
  res->arrival_s = r->arrival;
  res->start_s = r->start;
  res->done_s = r->done;
  res->latency_ms = (r->done - r->arrival) * 1e3;
  res->batch_frames = r->batch;
  res->device_ms = r->device_ms;
  S->by_ticket.erase(it);
  delete r;
  return PA_OK;
}

pa_status pa_server_get_stats(pa_server_t S, pa_server_stats* st) {
  if (!S || !st) {
    pa::set_error_message("pa_server_get_stats: null argument");
    return PA_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  st->submitted = S->submitted;
  st->completed = S->completed;
  st->failed = S->failed;
  st->batches = S->batches;
  st->bytes_in_use = S->in_use;
  st->bytes_peak = S->peak;
  st->plans_resident = S->plans_count;
  return PA_OK;
}

pa_status pa_server_destroy(pa_server_t S) {
  if (!S) return PA_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_sched.notify_all();
  if (S->th.joinable()) S->th.join();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop_build = true;
  }
  S->cv_build.notify_all();
  if (S->builder.joinable()) S->builder.join();
  for (auto& b : S->built)
    if (b.plan) pa_destroy(b.plan);
  S->built.clear();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    const double t = S->now();
    for (auto& p : S->pending) S->finish(p.second, PA_EBUSY, t);
    for (Request* r : S->visible) S->finish(r, PA_EBUSY, t);
    S->pending.clear();
    S->visible.clear();
    for (auto& kv : S->by_ticket) delete kv.second;
    S->by_ticket.clear();
  }
  S->cv_done.notify_all();
  for (auto& kv : S->plans)
    if (kv.second.plan) pa_destroy(kv.second.plan);
  for (auto& s : S->slots) {
    cudaStreamSynchronize(s.st);
    cudaStreamDestroy(s.st);
    cudaEventDestroy(s.ev);
    cudaEventDestroy(s.ev_start);
    cudaEventDestroy(s.ev_end);
    cudaFreeHost(s.h_timeouts);
  }
  cudaStreamDestroy(S->plan_stream);
  cudaMemPoolDestroy(S->pool);
  delete S;
  return PA_OK;
}

}  // extern "C"
