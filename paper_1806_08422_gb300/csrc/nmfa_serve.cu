// nmfa_serve.cu -- a serving loop for NMFA requests on one GPU (C ABI in nmfa.h).
//
// A request is an Ising instance (h, J) to anneal with R replicas until some
// replica's Eq. (1) energy reaches the request's target.  The server:
//   - copies each submitted request and queues it (arrival time = submit time);
//   - admits queued requests in arrival order while the device memory they will
//     hold (couplings, run scratch, outputs) fits the configured budget: a loader
//     thread creates the request's problem (upload, validation, row norms);
//   - continuously batches: whenever fewer than `max_inflight` launches are on the
//     GPU, every admitted request that is not running goes into one new batch (one
//     persistent tensor-core launch on its own stream), so requests that arrive
//     while others run start as soon as a launch slot frees, and the GPU work of
//     different launches overlaps;
//   - on completion reads the energies, and either finishes the request (target
//     met: time-to-target = completion - arrival) or reruns it with the next noise
//     stream id, up to `max_attempts` runs; finished requests release their memory;
//   - a launch whose requests all rerun, and are launched again together, reuses its
//     batch (plan and workspace) with the next noise stream ids instead of planning
//     a new one.
// Results depend only on each request (instance, schedule, seed, attempt), never on
// what it was batched with: batches are bit-identical to solo runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "nmfa_internal.h"

using namespace nmfa;

namespace {

struct Request {
  uint64_t ticket = 0;
  int32_t n = 0;
  std::vector<double> h, J, T;
  int32_t precision = NMFA_BF16_FP8J;
  int32_t t_f = 0;
  double sigma = 0.15, alpha = 0.15;
  int32_t replicas = 1;
  uint64_t seed = 0;
  double target = 0.0;
  // progress
  nmfa_result res{};
  std::vector<int8_t> best_signs;
  nmfa_problem* prob = nullptr;
  int64_t footprint = 0;
  double* T_dev = nullptr;
  int8_t* signs_dev = nullptr;
  double* energy_dev = nullptr;
  std::vector<double> energy_host;
};

struct InFlight {
  nmfa_batch* batch = nullptr;
  std::vector<Request*> reqs;
  int slot = 0;
  cudaEvent_t ev = nullptr;
};

// A finished launch whose requests all rerun: its batch, kept for their next launch.
struct Reusable {
  nmfa_batch* batch = nullptr;
  std::vector<Request*> reqs;  // in the batch's job order
};

}  // namespace

struct nmfa_server {
  nmfa_server_config cfg{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> pending;   // submitted, not admitted
  std::deque<Request*> ready;     // admitted, waiting for a launch
  std::vector<Request*> graveyard; // finished, memory to release
  std::vector<nmfa_batch*> dead_batches;
  std::map<uint64_t, Request*> all;
  int64_t mem_used = 0;
  uint64_t next_ticket = 1;
  int outstanding = 0;            // submitted and not finished
  bool stop = false;
  std::thread loader, worker, reaper;
  std::vector<cudaStream_t> streams;
  std::vector<bool> slot_busy;
  std::atomic<int64_t> launches{0};
  std::atomic<int64_t> reused{0};  // launches that reused a batch
  int32_t max_batch = 0;          // most requests one launch has carried
  std::vector<Reusable> reusable;  // worker thread only

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Device memory a request holds while admitted: its couplings as stored, the BF16
// copy a batch makes of FP8-stored couplings of n_pad <= 4096 (larger ones are read
// as stored by the kernel), the creation-time FP64 copy, the tensor kernel's scratch
// and its inputs/outputs.  The state is counted for the widest tile
// the library may pick (256 replicas), so admission never under-counts it.
int64_t request_footprint(const Request* r) {
  const int64_t n = r->n, n_pad = (n + 127) / 128 * 128;
  const int64_t bn = r->replicas <= 64 ? 64 : 256;
  const int64_t r_pad = (r->replicas + bn - 1) / bn * bn;
  const int64_t jq = (r->precision == NMFA_BF16 ? 2 : 1) * n_pad * n_pad;
  // FP8-stored couplings of small and mid-size problems are widened once per batch
  const int64_t widened = (r->precision == NMFA_BF16_FP8J && n_pad <= kFp8WidenOnceMaxNpad) ? 2 * n_pad * n_pad : 0;
  const int64_t creation = 8 * n * n;                      // FP64 staging copy held by the problem
  const int64_t scratch = 4 * r_pad * n_pad + (1 << 20);
  const int64_t io = r->replicas * (n + 16) + 8 * r->t_f;
  return jq + widened + n * n + creation + scratch + io;
}

// Finished requests are handed to the reaper thread, which destroys their problems
// (nmfa_destroy waits for the problem's runs) and returns their buffers to the
// memory pool, so that the scheduler never blocks on a release.
void release(nmfa_server* s, Request* r) {
  std::lock_guard<std::mutex> g(s->mu);
  s->graveyard.push_back(r);
  s->cv.notify_all();
}

void reaper_main(nmfa_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    std::vector<Request*> batch;
    std::vector<nmfa_batch*> dead;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || !s->graveyard.empty() || !s->dead_batches.empty(); });
      if (s->graveyard.empty() && s->dead_batches.empty() && s->stop) return;
      batch.swap(s->graveyard);
      dead.swap(s->dead_batches);
    }
    for (nmfa_batch* b : dead) nmfa_batch_destroy(b);
    for (Request* r : batch) {
      if (r->prob) nmfa_destroy(r->prob);
      pool_free(r->T_dev);
      pool_free(r->signs_dev);
      pool_free(r->energy_dev);
      r->prob = nullptr;
      r->T_dev = nullptr;
      r->signs_dev = nullptr;
      r->energy_dev = nullptr;
      std::lock_guard<std::mutex> g(s->mu);
      s->mem_used -= r->footprint;
      s->cv.notify_all();
    }
  }
}

void finish(nmfa_server* s, Request* r, int32_t error) {
  {
    std::lock_guard<std::mutex> g(s->mu);
    r->res.t_done = s->now();
    r->res.error = error;
    r->res.state = error ? -1 : 3;
    --s->outstanding;
  }
  release(s, r);
}

// Admission: create problems in arrival order while the budget allows.
void loader_main(nmfa_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] {
        return s->stop || (!s->pending.empty() &&
                           (s->mem_used + s->pending.front()->footprint <= s->cfg.memory_budget_bytes ||
                            s->mem_used == 0));
      });
      if (s->stop) return;
      r = s->pending.front();
      s->pending.pop_front();
      s->mem_used += r->footprint;
    }
    int rc = nmfa_create(r->n, r->h.empty() ? nullptr : r->h.data(), r->J.data(), r->precision, &r->prob);
    if (rc == NMFA_OK) {
      bool ok = pool_alloc(reinterpret_cast<void**>(&r->T_dev), sizeof(double) * std::max(r->t_f, 1)) == NMFA_OK &&
                pool_alloc(reinterpret_cast<void**>(&r->signs_dev), static_cast<size_t>(r->replicas) * r->n) ==
                    NMFA_OK &&
                pool_alloc(reinterpret_cast<void**>(&r->energy_dev), sizeof(double) * r->replicas) == NMFA_OK &&
                cudaMemcpy(r->T_dev, r->T.data(), sizeof(double) * r->t_f, cudaMemcpyHostToDevice) == cudaSuccess;
      if (!ok) rc = NMFA_ENOMEM;
    }
    std::vector<double>().swap(r->J);  // the host copy is no longer needed
    if (rc != NMFA_OK) {
      cudaGetLastError();
      finish(s, r, rc);
      continue;
    }
    std::lock_guard<std::mutex> g(s->mu);
    r->res.state = 1;
    r->res.t_admit = s->now();
    s->ready.push_back(r);
    s->cv.notify_all();
  }
}

// Launches batch b (jobs in the order of reqs) on the slot's stream.
int launch_created(nmfa_server* s, nmfa_batch* b, const std::vector<Request*>& reqs, int slot, InFlight* out) {
  int rc;
  if ((rc = nmfa_batch_launch(b, s->streams[slot]))) return rc;
  cudaEvent_t ev = nullptr;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, s->streams[slot]);
  out->batch = b;
  out->reqs = reqs;
  out->slot = slot;
  out->ev = ev;
  const double t = s->now();
  for (Request* r : reqs) {
    r->res.state = 2;
    if (r->res.attempts == 0) r->res.t_first_start = t;
    r->res.attempts += 1;
    r->res.spin_updates += static_cast<int64_t>(r->replicas) * r->n * r->t_f;
  }
  s->launches += 1;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->max_batch = std::max<int32_t>(s->max_batch, static_cast<int32_t>(reqs.size()));
  }
  return NMFA_OK;
}

// Reuses a kept batch whose requests are exactly `take` (in any order): its jobs get
// the requests' next noise streams.  Kept batches that do not match are released.
bool launch_reused(nmfa_server* s, const std::vector<Request*>& take, int slot, InFlight* out) {
  std::vector<Request*> want(take);
  std::sort(want.begin(), want.end());
  bool done = false;
  for (Reusable& k : s->reusable) {
    std::vector<Request*> have(k.reqs);
    std::sort(have.begin(), have.end());
    if (!done && have == want) {
      std::vector<uint32_t> ids;
      for (Request* r : k.reqs) ids.push_back(static_cast<uint32_t>(r->res.attempts));  // attempt k: stream k
      if (nmfa_batch_set_stream_ids(k.batch, ids.data(), static_cast<int32_t>(ids.size())) == NMFA_OK &&
          launch_created(s, k.batch, k.reqs, slot, out) == NMFA_OK) {
        s->reused += 1;
        k.batch = nullptr;
        done = true;
        continue;
      }
    }
  }
  {
    std::lock_guard<std::mutex> g(s->mu);
    for (Reusable& k : s->reusable)
      if (k.batch) s->dead_batches.push_back(k.batch);
    s->cv.notify_all();
  }
  s->reusable.clear();
  return done;
}

int launch_batch(nmfa_server* s, std::vector<Request*>& reqs, int slot, InFlight* out) {
  std::vector<nmfa_problem*> probs;
  std::vector<nmfa_job> jobs;
  for (Request* r : reqs) {
    nmfa_job j{};
    j.T_dev = r->T_dev;
    j.t_f = r->t_f;
    j.sigma = r->sigma;
    j.alpha = r->alpha;
    j.replicas = r->replicas;
    j.seed = r->seed;
    j.stream_id = static_cast<uint32_t>(r->res.attempts);  // attempt k draws noise stream k
    j.signs_dev = r->signs_dev;
    j.energy_dev = r->energy_dev;
    probs.push_back(r->prob);
    jobs.push_back(j);
  }
  nmfa_batch* b = nullptr;
  int rc = nmfa_batch_create(probs.data(), jobs.data(), static_cast<int32_t>(jobs.size()), 0, &b);
  if (rc) return rc;
  if ((rc = launch_created(s, b, reqs, slot, out))) {
    nmfa_batch_destroy(b);
    return rc;
  }
  return NMFA_OK;
}

void complete(nmfa_server* s, InFlight& f) {
  const int rc = nmfa_batch_sync(f.batch);
  bool all_rerun = rc == NMFA_OK;
  for (Request* r : f.reqs) {
    if (rc != NMFA_OK) {
      finish(s, r, rc);
      continue;
    }
    r->energy_host.resize(r->replicas);
    cudaMemcpy(r->energy_host.data(), r->energy_dev, sizeof(double) * r->replicas, cudaMemcpyDeviceToHost);
    int best = 0;
    for (int k = 1; k < r->replicas; ++k)
      if (r->energy_host[k] < r->energy_host[best]) best = k;
    const double e = r->energy_host[best];
    if (r->res.attempts == 1 || e < r->res.best_energy) {
      r->res.best_energy = e;
      r->best_signs.resize(r->n);
      cudaMemcpy(r->best_signs.data(), r->signs_dev + static_cast<int64_t>(best) * r->n, r->n, cudaMemcpyDeviceToHost);
    }
    if (e <= r->target) {
      r->res.success = 1;
      r->res.time_to_target = s->now() - r->res.t_submit;
      all_rerun = false;
      finish(s, r, NMFA_OK);
    } else if (r->res.attempts >= s->cfg.max_attempts) {
      r->res.time_to_target = -1.0;
      all_rerun = false;
      finish(s, r, NMFA_OK);
    } else {
      std::lock_guard<std::mutex> g(s->mu);
      r->res.state = 1;
      s->ready.push_front(r);  // reruns go first
    }
  }
  if (all_rerun) {
    s->reusable.push_back(Reusable{f.batch, f.reqs});  // for their next launch
  } else {
    std::lock_guard<std::mutex> g(s->mu);
    s->dead_batches.push_back(f.batch);  // its workspace is released by the reaper
    s->cv.notify_all();
  }
  cudaEventDestroy(f.ev);
  s->slot_busy[f.slot] = false;
}

void worker_main(nmfa_server* s) {
  cudaSetDevice(s->device);
  std::vector<InFlight> inflight;
  while (true) {
    // retire finished launches
    for (size_t k = 0; k < inflight.size();) {
      if (cudaEventQuery(inflight[k].ev) == cudaSuccess) {
        complete(s, inflight[k]);
        inflight.erase(inflight.begin() + k);
      } else {
        ++k;
      }
    }
    cudaGetLastError();
    // start a new launch with everything admitted, if a slot is free
    int slot = -1;
    for (int k = 0; k < static_cast<int>(s->slot_busy.size()); ++k)
      if (!s->slot_busy[k]) {
        slot = k;
        break;
      }
    std::vector<Request*> take;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop && inflight.empty()) return;
      if (slot >= 0) {
        while (!s->ready.empty()) {
          take.push_back(s->ready.front());
          s->ready.pop_front();
        }
      }
      if (take.empty()) {
        // nothing to launch: wait briefly for an arrival, an admission or a completion
        s->cv.wait_for(lk, std::chrono::microseconds(inflight.empty() ? 2000 : 50));
        continue;
      }
    }
    InFlight f;
    const int rc = launch_reused(s, take, slot, &f) ? NMFA_OK : launch_batch(s, take, slot, &f);
    if (rc != NMFA_OK) {
      for (Request* r : take) finish(s, r, rc);
      continue;
    }
    s->slot_busy[slot] = true;
    inflight.push_back(f);
  }
}

}  // namespace

extern "C" {

int nmfa_server_create(const nmfa_server_config* cfg, nmfa_server** out) {
  if (out == nullptr) return set_error(NMFA_EINVAL, "out is NULL");
  *out = nullptr;
  nmfa_server* s = new nmfa_server();
  if (cfg) s->cfg = *cfg;
  if (s->cfg.max_inflight < 1) s->cfg.max_inflight = 2;
  if (s->cfg.max_attempts < 1) s->cfg.max_attempts = 4;
  int rc;
  if ((rc = cuda_error(cudaGetDevice(&s->device), "cudaGetDevice"))) {
    delete s;
    return rc;
  }
  if (s->cfg.memory_budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    if ((rc = cuda_error(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo"))) {
      delete s;
      return rc;
    }
    s->cfg.memory_budget_bytes = static_cast<int64_t>(fr * 0.8);
  }
  s->streams.resize(s->cfg.max_inflight);
  s->slot_busy.assign(s->cfg.max_inflight, false);
  for (auto& st : s->streams) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  s->t0 = std::chrono::steady_clock::now();
  s->loader = std::thread(loader_main, s);
  s->worker = std::thread(worker_main, s);
  s->reaper = std::thread(reaper_main, s);
  *out = s;
  return NMFA_OK;
}

int nmfa_server_submit(nmfa_server* s, const nmfa_request* q, uint64_t* ticket) {
  if (s == nullptr || q == nullptr || ticket == nullptr) return set_error(NMFA_EINVAL, "NULL argument");
  if (q->n < 1 || q->J == nullptr || q->T == nullptr || q->t_f < 1 || q->replicas < 1)
    return set_error(NMFA_EINVAL, "bad request");
  if (q->precision != NMFA_BF16 && q->precision != NMFA_BF16_FP8J)
    return set_error(NMFA_EUNSUPPORTED, "the server runs NMFA_BF16 / NMFA_BF16_FP8J problems");
  Request* r = new Request();
  r->n = q->n;
  r->J.assign(q->J, q->J + static_cast<int64_t>(q->n) * q->n);
  if (q->h) r->h.assign(q->h, q->h + q->n);
  r->T.assign(q->T, q->T + q->t_f);
  r->precision = q->precision;
  r->t_f = q->t_f;
  r->sigma = q->sigma;
  r->alpha = q->alpha;
  r->replicas = q->replicas;
  r->seed = q->seed;
  r->target = q->target_energy;
  r->footprint = request_footprint(r);
  std::lock_guard<std::mutex> g(s->mu);
  r->ticket = s->next_ticket++;
  r->res.t_submit = s->now();
  r->res.time_to_target = -1.0;
  s->all[r->ticket] = r;
  s->pending.push_back(r);
  ++s->outstanding;
  *ticket = r->ticket;
  s->cv.notify_all();
  return NMFA_OK;
}

int nmfa_server_poll(nmfa_server* s, uint64_t ticket, nmfa_result* out, int8_t* best_signs) {
  if (s == nullptr || out == nullptr) return set_error(NMFA_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return set_error(NMFA_EINVAL, "unknown ticket");
  *out = it->second->res;
  if (best_signs && (out->state == 3) && !it->second->best_signs.empty())
    std::memcpy(best_signs, it->second->best_signs.data(), it->second->best_signs.size());
  return NMFA_OK;
}

int nmfa_server_drain(nmfa_server* s, double timeout_s) {
  if (s == nullptr) return set_error(NMFA_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  const bool done = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return s->outstanding == 0; });
  return done ? NMFA_OK : set_error(NMFA_ETIMEOUT, "requests still outstanding");
}

int nmfa_server_stats(nmfa_server* s, int64_t* launches, int64_t* mem_used, int32_t* outstanding,
                      int32_t* max_requests_per_launch, int64_t* batches_reused) {
  if (s == nullptr) return set_error(NMFA_EINVAL, "NULL server");
  std::lock_guard<std::mutex> g(s->mu);
  if (batches_reused) *batches_reused = s->reused.load();
  if (max_requests_per_launch) *max_requests_per_launch = s->max_batch;
  if (launches) *launches = s->launches.load();
  if (mem_used) *mem_used = s->mem_used;
  if (outstanding) *outstanding = s->outstanding;
  return NMFA_OK;
}

void nmfa_server_destroy(nmfa_server* s) {
  if (s == nullptr) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->loader.joinable()) s->loader.join();
  if (s->worker.joinable()) s->worker.join();
  if (s->reaper.joinable()) s->reaper.join();
  for (Reusable& k : s->reusable)
    if (k.batch) nmfa_batch_destroy(k.batch);
  for (nmfa_batch* b : s->dead_batches) nmfa_batch_destroy(b);
  for (auto& kv : s->all) {
    Request* r = kv.second;
    if (r->prob) nmfa_destroy(r->prob);
    pool_free(r->T_dev);
    pool_free(r->signs_dev);
    pool_free(r->energy_dev);
    delete r;
  }
  for (auto& st : s->streams) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
