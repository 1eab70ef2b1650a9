// brng_serve.cu -- continuous batching of Gibbs sampling jobs (the paper's
// "BatchRNG as asynchronous service", Sec. 3 item 3, grown into a request
// loop).
//
// Clients submit jobs (model, chains, sweeps, seed, host inputs) at any time.
// One scheduler thread owned by the server, round after round:
//   1. admits queued jobs in arrival order while their device memory fits the
//      budget: one stream-ordered allocation per job, start state and inputs
//      uploaded on the admission stream;
//   2. when admitted jobs wait and one of `max_inflight` batch slots is free,
//      launches them (in arrival order, up to about `batch_cost_s` of
//      estimated GPU time, at least one job) as one batch (brng_batch.cu) on
//      that slot's stream, ordered after the admission uploads;
//   3. polls the slots' completion events and marks their jobs done.
// Several batches are in flight at once on different streams, so jobs that
// arrive while others run are admitted and start at once, their work
// overlapping on the device with the earlier batches.  The server mutex only
// guards bookkeeping; every CUDA call is made outside it, so submitting never
// waits for the device.  Chain, ring and generator state stay on the device
// until the client collects the results, which also returns the job's memory
// to the budget.  A job gives the same results served in any mix as alone (a
// batch runs each unit with the same code on the same streams).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "brng.h"
#include "brng_internal.h"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

enum Stage { kQueued = 0, kAdmitting = 1, kAdmitted = 2, kLaunched = 3, kDone = 4, kFailed = 5 };

constexpr size_t kInitialTableJobs = 4096;

struct ServeJob {
  uint64_t id = 0;
  brng_request_t req{};
  std::vector<float> in0, in1, in2;  // host copies (unless the inputs are borrowed)
  size_t bytes = 0;                  // device bytes (one allocation)
  unsigned char* dev = nullptr;
  size_t off_state = 0, off_mom = 0, off_in0 = 0, off_in1 = 0, off_in2 = 0, off_pos = 0;
  size_t state_bytes = 0, mom_bytes = 0;
  brng_normal_gamma_params_t ngp{};
  brng_lda_params_t ldap{};
  brng_lda_state_t ldas{};
  int stage = kQueued;
  int status = BRNG_OK;
  int64_t t_submit = 0, t_admit = 0, t_launch = 0, t_done = 0;
};

// device layout of a job: [state | moments | inputs... | positions (LDA)]
void layout(ServeJob* j) {
  const brng_request_t& r = j->req;
  const size_t n = r.n_chains;
  size_t o = 0;
  switch (r.model) {
    case BRNG_MODEL_TRIANGLE:
      j->state_bytes = n * sizeof(brng_triangle_state_t);
      j->mom_bytes = n * 5 * sizeof(double);
      j->off_state = o; o = align256(o + j->state_bytes);
      j->off_mom = o; o = align256(o + j->mom_bytes);
      break;
    case BRNG_MODEL_NORMAL_GAMMA:
      j->state_bytes = n * sizeof(brng_normal_gamma_state_t);
      j->mom_bytes = n * 4 * sizeof(double);
      j->off_state = o; o = align256(o + j->state_bytes);
      j->off_mom = o; o = align256(o + j->mom_bytes);
      j->off_in0 = o; o = align256(o + n * 4);
      j->off_in1 = o; o = align256(o + n * 4);
      j->off_in2 = o; o = align256(o + n * 4);
      break;
    default: {
      const size_t nk = n * r.K;
      j->state_bytes = nk * sizeof(float);  // theta
      j->mom_bytes = nk * sizeof(double);
      j->off_state = o; o = align256(o + j->state_bytes);
      j->off_mom = o; o = align256(o + j->mom_bytes);
      j->off_in0 = o; o = align256(o + nk * 4);   // alpha
      j->off_pos = o; o = align256(o + nk * 16);  // (N, U) positions
      break;
    }
  }
  j->bytes = o;
}

// Rough GPU time of a job on a whole GB300, for batch sizing only (per
// triangle chain-sweep, per normal-gamma chain-sweep, per LDA Gamma draw).
double est_seconds(const brng_request_t& r) {
  const double cs = static_cast<double>(r.n_chains) * r.n_sweeps;
  switch (r.model) {
    case BRNG_MODEL_TRIANGLE: return 1.5e-11 * cs;
    case BRNG_MODEL_NORMAL_GAMMA: return 2.0e-11 * cs;
    default: return 4.7e-11 * cs * r.K;
  }
}

// Allocates and fills a job's device memory on `st` (no lock held).
int upload_job(ServeJob* j, cudaStream_t st) {
  void* p = nullptr;
  if (cudaMallocAsync(&p, j->bytes, st) != cudaSuccess) return BRNG_ENOMEM;
  j->dev = static_cast<unsigned char*>(p);
  const brng_request_t& r = j->req;
  const size_t n = r.n_chains;
  const bool borrow = r.flags & BRNG_SERVE_BORROW_INPUTS;
  cudaError_t e = cudaMemsetAsync(j->dev + j->off_mom, 0, j->mom_bytes, st);
  if (r.model == BRNG_MODEL_TRIANGLE) {
    std::vector<brng_triangle_state_t> init(n, brng_triangle_state_t{0.5, 0.5, 0, 0});
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(j->dev + j->off_state, init.data(), j->state_bytes, cudaMemcpyHostToDevice, st);
  } else if (r.model == BRNG_MODEL_NORMAL_GAMMA) {
    std::vector<brng_normal_gamma_state_t> init(n, brng_normal_gamma_state_t{r.mu0, 0.0f, 0, 0});
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(j->dev + j->off_state, init.data(), j->state_bytes, cudaMemcpyHostToDevice, st);
    const size_t nb = n * 4;
    const float* s0 = borrow ? r.nobs : j->in0.data();
    const float* s1 = borrow ? r.xbar : j->in1.data();
    const float* s2 = borrow ? r.sc : j->in2.data();
    if (e == cudaSuccess) e = cudaMemcpyAsync(j->dev + j->off_in0, s0, nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(j->dev + j->off_in1, s1, nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(j->dev + j->off_in2, s2, nb, cudaMemcpyHostToDevice, st);
    j->ngp = brng_normal_gamma_params_t{r.a0, r.b0, r.mu0, r.prec0,
                                        reinterpret_cast<const float*>(j->dev + j->off_in0),
                                        reinterpret_cast<const float*>(j->dev + j->off_in1),
                                        reinterpret_cast<const float*>(j->dev + j->off_in2)};
  } else {
    const size_t nk = n * r.K;
    const float* s0 = borrow ? r.alpha : j->in0.data();
    if (e == cudaSuccess) e = cudaMemsetAsync(j->dev + j->off_state, 0, j->state_bytes, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(j->dev + j->off_in0, s0, nk * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(j->dev + j->off_pos, 0, nk * 16, st);
    j->ldap = brng_lda_params_t{r.K, reinterpret_cast<const float*>(j->dev + j->off_in0)};
    j->ldas = brng_lda_state_t{reinterpret_cast<float*>(j->dev + j->off_state),
                               reinterpret_cast<uint64_t*>(j->dev + j->off_pos)};
  }
  // pageable sources are staged before the copies return: the host copies may go
  j->in0 = std::vector<float>();
  j->in1 = std::vector<float>();
  j->in2 = std::vector<float>();
  return e == cudaSuccess ? BRNG_OK : BRNG_ECUDA;
}

brng_job_t batch_entry(ServeJob* j) {
  const brng_request_t& r = j->req;
  brng_job_t b{};
  b.model = r.model;
  b.n_chains = r.n_chains;
  b.n_sweeps = r.n_sweeps;
  b.seed = r.seed;
  b.chain_offset = r.chain_offset;
  b.moments = reinterpret_cast<double*>(j->dev + j->off_mom);
  if (r.model == BRNG_MODEL_TRIANGLE) {
    b.state = j->dev + j->off_state;
  } else if (r.model == BRNG_MODEL_NORMAL_GAMMA) {
    b.params = &j->ngp;
    b.state = j->dev + j->off_state;
  } else {
    b.params = &j->ldap;
    b.state = &j->ldas;
  }
  return b;
}

}  // namespace

struct brng_server {
  brng_t* h = nullptr;  // tuning and counters
  uint64_t budget = 0, used = 0;
  uint32_t max_inflight = 1;
  double batch_cost_s = 0.05;
  cudaStream_t admit_stream = nullptr;
  cudaEvent_t admit_event = nullptr;
  cudaStream_t result_stream = nullptr;
  std::mutex result_mu;
  struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<uint64_t> jobs;
    brng::BatchJob* d_table = nullptr;
    size_t cap = 0;
    unsigned long long* d_counter = nullptr;
  };
  std::vector<Slot> slots;
  std::mutex mu;  // guards everything below and every job's stage/status/times
  std::condition_variable cv;
  std::deque<uint64_t> queue;  // submitted, waiting for memory
  std::vector<uint64_t> ready; // admitted, waiting for a slot
  std::unordered_map<uint64_t, std::unique_ptr<ServeJob>> jobs;
  uint64_t next_id = 1;
  bool stop = false;
  int fatal = BRNG_OK;
  brng_serve_stats_t st{};
  std::thread thr;
  int device = 0;

  void run();
};

void brng_server::run() {
  cudaSetDevice(device);
  while (true) {
    std::vector<ServeJob*> admit;
    std::vector<std::pair<Slot*, std::vector<uint64_t>>> done_slots;
    Slot* launch_slot = nullptr;
    std::vector<uint64_t> launch_ids;
    std::vector<ServeJob*> launch_jobs;
    std::vector<Slot*> busy;
    {
      std::unique_lock<std::mutex> lock(mu);
      if (stop) {  // closing: jobs waiting for memory or for a launch are cancelled
        const int64_t t = now_ns();
        for (uint64_t id : queue) {
          ServeJob* j = jobs[id].get();
          j->stage = kFailed;
          j->status = BRNG_EAGAIN;
          j->t_done = t;
          st.cancelled++;
        }
        queue.clear();
        // admitted but not launched: their device blocks are freed with the
        // other uncollected jobs' once the launched batches have finished
        for (uint64_t id : ready) {
          ServeJob* j = jobs[id].get();
          j->stage = kFailed;
          j->status = BRNG_EAGAIN;
          j->t_done = t;
          st.cancelled++;
        }
        ready.clear();
      }
      bool inflight = false;
      for (auto& s : slots)
        if (s.busy) {
          inflight = true;
          busy.push_back(&s);
        }
      if (stop && ready.empty() && !inflight) break;
      // admission: arrival order, while the budget allows
      while (!queue.empty()) {
        ServeJob* j = jobs[queue.front()].get();
        if (j->bytes > budget) {  // can never fit
          j->stage = kFailed;
          j->status = BRNG_ENOMEM;
          j->t_done = now_ns();
          st.refused++;
          queue.pop_front();
          continue;
        }
        if (used + j->bytes > budget) break;
        used += j->bytes;
        j->stage = kAdmitting;
        admit.push_back(j);
        queue.pop_front();
      }
      // a launch: the waiting jobs in arrival order up to batch_cost_s
      if (!ready.empty()) {
        for (auto& s : slots)
          if (!s.busy) {
            launch_slot = &s;
            break;
          }
        if (launch_slot) {
          double cost = 0.0;
          size_t k = 0;
          for (; k < ready.size(); ++k) {
            ServeJob* j = jobs[ready[k]].get();
            const double c = est_seconds(j->req);
            if (k > 0 && cost + c > batch_cost_s) break;
            cost += c;
            launch_ids.push_back(ready[k]);
            launch_jobs.push_back(j);
          }
          ready.erase(ready.begin(), ready.begin() + k);
          launch_slot->busy = true;  // reserved
        }
      }
      if (admit.empty() && !launch_slot && busy.empty() && !stop) {
        cv.wait_for(lock, std::chrono::milliseconds(1));
        continue;
      }
    }
    // ---- CUDA work, no lock held ----
    bool progress = false;
    // completions
    std::vector<std::pair<Slot*, cudaError_t>> finished;
    for (Slot* s : busy) {
      const cudaError_t q = cudaEventQuery(s->done);
      if (q != cudaErrorNotReady) finished.emplace_back(s, q);
    }
    // admissions
    std::vector<int> admit_rc(admit.size());
    if (!admit.empty()) {
      const brng::TraceRange trace("brng_serve admit");
      for (size_t i = 0; i < admit.size(); ++i) admit_rc[i] = upload_job(admit[i], admit_stream);
    }
    if (!admit.empty()) cudaEventRecord(admit_event, admit_stream);
    // launch
    int launch_rc = BRNG_OK;
    if (launch_slot) {
      const brng::TraceRange trace("brng_serve launch batch");
      std::vector<brng_job_t> batch;
      batch.reserve(launch_jobs.size());
      for (ServeJob* j : launch_jobs) batch.push_back(batch_entry(j));
      cudaStreamWaitEvent(launch_slot->stream, admit_event, 0);
      launch_rc = brng::batch_launch_into(h, batch.data(), static_cast<uint32_t>(batch.size()),
                                          &launch_slot->d_table, &launch_slot->cap,
                                          &launch_slot->d_counter, launch_slot->stream);
      if (launch_rc == BRNG_OK) cudaEventRecord(launch_slot->done, launch_slot->stream);
    }
    // ---- bookkeeping ----
    {
      std::lock_guard<std::mutex> lock(mu);
      const int64_t t = now_ns();
      for (auto& f : finished) {
        for (uint64_t id : f.first->jobs) {
          ServeJob* j = jobs[id].get();
          j->stage = f.second == cudaSuccess ? kDone : kFailed;
          j->status = f.second == cudaSuccess ? BRNG_OK : BRNG_ECUDA;
          j->t_done = t;
          st.completed++;
        }
        if (f.second != cudaSuccess) fatal = BRNG_ECUDA;
        f.first->jobs.clear();
        f.first->busy = false;
        progress = true;
      }
      for (size_t i = 0; i < admit.size(); ++i) {
        ServeJob* j = admit[i];
        if (admit_rc[i] == BRNG_OK) {
          j->stage = kAdmitted;
          j->t_admit = t;
          st.admitted++;
          ready.push_back(j->id);
        } else {
          if (j->dev) cudaFreeAsync(j->dev, admit_stream);
          j->dev = nullptr;
          used -= j->bytes;
          j->stage = kFailed;
          j->status = admit_rc[i];
          j->t_done = t;
          st.refused++;
        }
        progress = true;
      }
      if (launch_slot) {
        for (ServeJob* j : launch_jobs) {
          if (launch_rc == BRNG_OK) {
            j->stage = kLaunched;
            j->t_launch = t;
          } else {
            j->stage = kFailed;
            j->status = launch_rc;
            j->t_done = t;
          }
        }
        if (launch_rc == BRNG_OK) {
          launch_slot->jobs.swap(launch_ids);
          st.batches++;
        } else {
          launch_slot->busy = false;
        }
        progress = true;
      }
    }
    if (progress) cv.notify_all();
    else std::this_thread::sleep_for(std::chrono::microseconds(20));  // batches running: poll again
  }
}

extern "C" {

int brng_serve_open(uint64_t mem_budget, uint32_t max_inflight, const brng_tuning_t* tuning,
                    brng_server_t** out) {
  if (!out || mem_budget == 0 || max_inflight == 0 || max_inflight > 64) return BRNG_EINVAL;
  std::unique_ptr<brng_server_t> s(new (std::nothrow) brng_server_t());
  if (!s) return BRNG_ENOMEM;
  int rc = brng_create(0, 1, 0, &s->h);
  if (rc != BRNG_OK) return rc;
  if (tuning && (rc = brng_set_tuning(s->h, tuning)) != BRNG_OK) {
    brng_destroy(s->h);
    return rc;
  }
  cudaGetDevice(&s->device);
  s->budget = mem_budget;
  s->max_inflight = max_inflight;
  s->slots.resize(max_inflight);
  cudaError_t e = cudaStreamCreateWithFlags(&s->admit_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->result_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->admit_event, cudaEventDisableTiming);
  for (auto& sl : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    // batch tables sized up front: growing one later waits for the device
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_table, sizeof(brng::BatchJob) * kInitialTableJobs);
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_counter, sizeof(unsigned long long));
    sl.cap = kInitialTableJobs;
  }
  if (e != cudaSuccess) {
    brng_destroy(s->h);
    return BRNG_ECUDA;
  }
  brng_server_t* raw = s.release();
  raw->thr = std::thread([raw] { raw->run(); });
  *out = raw;
  return BRNG_OK;
}

int brng_serve_submit(brng_server_t* s, const brng_request_t* r, uint64_t* id) {
  if (!s || !r || !id) return BRNG_EINVAL;
  if (r->n_chains == 0) return BRNG_EINVAL;
  std::unique_ptr<ServeJob> j(new (std::nothrow) ServeJob());
  if (!j) return BRNG_ENOMEM;
  j->req = *r;
  const size_t n = r->n_chains;
  const bool borrow = r->flags & BRNG_SERVE_BORROW_INPUTS;
  switch (r->model) {
    case BRNG_MODEL_TRIANGLE:
      break;
    case BRNG_MODEL_NORMAL_GAMMA:
      if (!r->nobs || !r->xbar || !r->sc) return BRNG_EINVAL;
      if (!borrow) {
        j->in0.assign(r->nobs, r->nobs + n);
        j->in1.assign(r->xbar, r->xbar + n);
        j->in2.assign(r->sc, r->sc + n);
      }
      break;
    case BRNG_MODEL_LDA:
      if (!r->alpha || r->K == 0 || r->K > 128) return BRNG_EINVAL;
      if (!borrow) j->in0.assign(r->alpha, r->alpha + n * r->K);
      break;
    default:
      return BRNG_EINVAL;
  }
  if (!borrow) j->req.nobs = j->req.xbar = j->req.sc = j->req.alpha = nullptr;
  layout(j.get());
  j->t_submit = now_ns();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return BRNG_EINVAL;
    j->id = s->next_id++;
    *id = j->id;
    s->queue.push_back(j->id);
    s->jobs.emplace(j->id, std::move(j));
    s->st.submitted++;
  }
  s->cv.notify_all();
  return BRNG_OK;
}

int brng_serve_poll(brng_server_t* s, uint64_t id, int* done) {
  if (!s || !done) return BRNG_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return BRNG_ENOTFOUND;
  *done = it->second->stage >= kDone;
  return it->second->stage == kFailed ? it->second->status : BRNG_OK;
}

int brng_serve_wait(brng_server_t* s, uint64_t id, double timeout_s) {
  if (!s) return BRNG_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::nanoseconds(static_cast<int64_t>(timeout_s * 1e9));
  while (true) {
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return BRNG_ENOTFOUND;
    if (it->second->stage == kFailed) return it->second->status;
    if (it->second->stage == kDone) return BRNG_OK;
    if (std::chrono::steady_clock::now() >= deadline) return BRNG_EAGAIN;
    s->cv.wait_until(lock, deadline);  // re-checked at the top, also after a timeout
  }
}

int brng_serve_result(brng_server_t* s, uint64_t id, void* host_state, double* host_moments,
                      brng_job_info_t* info) {
  if (!s) return BRNG_EINVAL;
  std::unique_ptr<ServeJob> j;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return BRNG_ENOTFOUND;
    if (it->second->stage != kDone && it->second->stage != kFailed) return BRNG_EAGAIN;
    j = std::move(it->second);
    s->jobs.erase(it);
  }
  int rc = j->status;
  if (info) {
    info->submitted_ns = static_cast<uint64_t>(j->t_submit);
    info->admitted_ns = static_cast<uint64_t>(j->t_admit);
    info->launched_ns = static_cast<uint64_t>(j->t_launch);
    info->completed_ns = static_cast<uint64_t>(j->t_done);
    info->device_bytes = j->bytes;
    info->status = j->status;
  }
  if (j->dev) {
    // the job's kernel has finished (its batch event fired); copy on the
    // server's result stream and return the memory there (stream-ordered, no
    // device-wide synchronisation while other batches run)
    std::lock_guard<std::mutex> rl(s->result_mu);
    // the job's uploads ran on the admission stream: a job that failed before
    // its batch event fired has no launch ordering them before this stream,
    // so wait for the admission work recorded so far before reusing the block
    cudaError_t e = cudaStreamWaitEvent(s->result_stream, s->admit_event, 0);
    if (e == cudaSuccess && rc == BRNG_OK && host_state)
      e = cudaMemcpyAsync(host_state, j->dev + j->off_state, j->state_bytes, cudaMemcpyDeviceToHost,
                          s->result_stream);
    if (e == cudaSuccess && rc == BRNG_OK && host_moments)
      e = cudaMemcpyAsync(host_moments, j->dev + j->off_mom, j->mom_bytes, cudaMemcpyDeviceToHost,
                          s->result_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->result_stream);
    cudaFreeAsync(j->dev, s->result_stream);
    if (e != cudaSuccess && rc == BRNG_OK) rc = BRNG_ECUDA;
    std::lock_guard<std::mutex> lock(s->mu);
    s->used -= j->bytes;
  }
  s->cv.notify_all();
  return rc;
}

int brng_serve_stats(brng_server_t* s, brng_serve_stats_t* out) {
  if (!s || !out) return BRNG_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->st;
  out->queued = s->queue.size();
  out->device_bytes_in_use = s->used;
  return s->fatal;
}

int brng_serve_cancel(brng_server_t* s, uint64_t id) {
  if (!s) return BRNG_EINVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return BRNG_ENOTFOUND;
    if (it->second->stage != kQueued) return BRNG_EAGAIN;  // admitted: it runs to the end
    auto q = std::find(s->queue.begin(), s->queue.end(), id);
    if (q != s->queue.end()) s->queue.erase(q);
    s->jobs.erase(it);
    s->st.cancelled++;
  }
  s->cv.notify_all();  // a waiter on the id sees BRNG_ENOTFOUND
  return BRNG_OK;
}

int brng_serve_close(brng_server_t* s) {
  if (!s) return BRNG_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->thr.joinable()) s->thr.join();
  cudaDeviceSynchronize();
  for (auto& kv : s->jobs)
    if (kv.second->dev) cudaFree(kv.second->dev);  // uncollected results
  for (auto& sl : s->slots) {
    cudaFree(sl.d_table);
    cudaFree(sl.d_counter);
    cudaEventDestroy(sl.done);
    cudaStreamDestroy(sl.stream);
  }
  cudaEventDestroy(s->admit_event);
  cudaStreamDestroy(s->admit_stream);
  cudaStreamDestroy(s->result_stream);
  brng_destroy(s->h);
  const int rc = s->fatal;
  delete s;
  return rc;
}

}  // extern "C"
