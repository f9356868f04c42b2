// Serving: a request loop that admits refinement jobs by device-memory
// footprint and runs several at once, each on its own stream, so that jobs
// arriving while others are on the GPU are admitted as soon as a slot and
// enough of the memory budget are free (continuous batching), and their
// kernels overlap on the device.  A job is one jet_refine_host call (upload,
// Algorithm 1 as one graph, download); its inputs and output stay in the
// caller's host memory until the job is reported done.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "jet_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  int64_t id = 0;
  jet_hypergraph hg{};
  jet_params params{};
  std::vector<int32_t> tau;
  int32_t limit = 0;
  int32_t *part = nullptr;
  size_t bytes = 0;
  Clock::time_point t_submit, t_admit;
};

}  // namespace

struct jet_server {
  size_t budget = 0;
  size_t reserved = 0;
  int max_active = 1;
  int active = 0;
  int64_t next_id = 1;
  bool stopping = false;
  std::mutex mu;
  std::condition_variable cv_work;  // workers: a job was admitted, or stop
  std::condition_variable cv_done;  // waiters: a job finished
  std::deque<Job> pending;          // submitted, not yet admitted (FIFO)
  std::deque<Job> admitted;         // admitted, waiting for a worker
  std::deque<jet_job_done> done;
  std::vector<std::thread> workers;
  int device = 0;
  cudaEvent_t ev_ref = nullptr;     // origin of the jobs' GPU-timeline intervals
  std::mutex err_mu;                // guards err (calls from several threads may fail at once)
  char err[256] = {0};
};

namespace {

int sfail(jet_server *s, int code, const char *msg) {
  if (s) {
    std::lock_guard<std::mutex> lk(s->err_mu);
    snprintf(s->err, sizeof(s->err), "%s", msg);
  }
  jet::set_global_error("%s", msg);
  return code;
}

// Moves jobs from `pending` to `admitted` in submission order while a slot
// and enough of the budget are free (caller holds the lock).
void admit_locked(jet_server *s) {
  while (!s->pending.empty() && s->active + (int)s->admitted.size() < s->max_active &&
         s->reserved + s->pending.front().bytes <= s->budget) {
    Job j = std::move(s->pending.front());
    s->pending.pop_front();
    s->reserved += j.bytes;
    j.t_admit = Clock::now();
    s->admitted.push_back(std::move(j));
    s->cv_work.notify_one();
  }
}

void worker_main(jet_server *s) {
  cudaSetDevice(s->device);
  // one stream and one pair of timing events per worker, reused by its jobs
  cudaStream_t stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  const bool timed = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess &&
                     cudaEventCreate(&ev0) == cudaSuccess && cudaEventCreate(&ev1) == cudaSuccess;
  for (;;) {
    Job j;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stopping || !s->admitted.empty(); });
      if (s->admitted.empty()) break;  // stopping and nothing left
      j = std::move(s->admitted.front());
      s->admitted.pop_front();
      s->active += 1;
    }
    jet_job_done d;
    memset(&d, 0, sizeof(d));
    d.id = j.id;
    if (timed) {
      d.status = jet::refine_host_on(&j.hg, &j.params, j.tau.data(), (int32_t)(j.tau.size() / 2), j.limit, j.part,
                                     &d.result, stream, ev0, ev1);
    } else {
      d.status = jet_refine_host(&j.hg, &j.params, j.tau.data(), (int32_t)(j.tau.size() / 2), j.limit, j.part,
                                 &d.result);
    }
    const Clock::time_point t_end = Clock::now();
    d.latency_ms = std::chrono::duration<double, std::milli>(t_end - j.t_submit).count();
    d.queue_ms = std::chrono::duration<double, std::milli>(j.t_admit - j.t_submit).count();
    d.device_start_ms = d.device_end_ms = -1.0;
    if (d.status != JET_OK) {
      snprintf(d.message, sizeof(d.message), "%s", jet_last_error(nullptr));  // this worker thread's error text
    } else if (timed && s->ev_ref) {
      float a = 0.f, b = 0.f;
      if (cudaEventElapsedTime(&a, s->ev_ref, ev0) == cudaSuccess &&
          cudaEventElapsedTime(&b, s->ev_ref, ev1) == cudaSuccess) {
        d.device_start_ms = a;
        d.device_end_ms = b;
      }
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->active -= 1;
      s->reserved -= j.bytes;
      s->done.push_back(d);
      admit_locked(s);
    }
    s->cv_done.notify_all();
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

size_t jet_job_footprint(int32_t n, int32_t m, int64_t P, int32_t k) {
  if (n < 0 || m < 0 || P < 0 || k < 2) return 0;
  const size_t N = (size_t)n, M = (size_t)m, Pz = (size_t)P, K = (size_t)k;
  const size_t kw = (K + 31) / 32, kwp = kw <= 1 ? 1 : kw <= 2 ? 2 : kw <= 4 ? 4 : 8;
  size_t b = 8 * (M + 1) + 8 * (N + 1) + 8 * Pz + 4 * N + 4 * M;  // CSR views and weights
  b += 4 * N + 4 * M * K + 8 * K;                                 // partition, phi, block weights
  b += 8 * M * kwp;                                               // edge bitmasks
  b += N * (8 + 4 + 4 + 4 + 8 + 4 + 4 + 4 + 1 + 1 + 4) + 4 * M;   // per-vertex workspace, class lists
  b += 16 * N + 4 * M;                                            // set-up temporaries of the context
  b += 64 * K + 4096 + 8 * std::max((size_t)4 * N, 2048 * K);      // per-block state, counters, histograms
  return b + b / 16;                                              // allocator rounding
}

int jet_server_create(jet_server **out, size_t hbm_budget, int32_t max_active) {
  if (!out) return sfail(nullptr, JET_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (max_active < 1 || max_active > 64) return sfail(nullptr, JET_ERR_INVALID_ARG, "max_active must be in [1, 64]");
  if (hbm_budget == 0) return sfail(nullptr, JET_ERR_INVALID_ARG, "the memory budget is 0");
  jet_server *s = new (std::nothrow) jet_server;
  if (!s) return sfail(nullptr, JET_ERR_OOM, "host allocation failed");
  s->budget = hbm_budget;
  s->max_active = max_active;
  cudaGetDevice(&s->device);
  if (cudaEventCreate(&s->ev_ref) == cudaSuccess) {  // the origin of the jobs' GPU-timeline intervals
    if (cudaEventRecord(s->ev_ref, nullptr) != cudaSuccess || cudaEventSynchronize(s->ev_ref) != cudaSuccess) {
      cudaEventDestroy(s->ev_ref);
      s->ev_ref = nullptr;
    }
  } else {
    s->ev_ref = nullptr;
  }
  try {
    for (int i = 0; i < max_active; ++i) s->workers.emplace_back(worker_main, s);
  } catch (...) {
    jet_server_destroy(s);
    return sfail(nullptr, JET_ERR_OOM, "could not start the worker threads");
  }
  *out = s;
  return JET_OK;
}

int jet_server_submit(jet_server *s, const jet_hypergraph *hg_host, const jet_params *params, const int32_t *tau_pairs,
                      int32_t n_tau, int32_t limit, int32_t *part_host, int64_t *id_out) {
  if (!s) return sfail(nullptr, JET_ERR_INVALID_ARG, "server is NULL");
  if (!hg_host || !params || !part_host || !id_out) return sfail(s, JET_ERR_INVALID_ARG, "NULL argument");
  if (hg_host->n < 0 || hg_host->m < 0 || hg_host->P < 0 || params->k < 2 || params->k > jet::kMaxK)
    return sfail(s, JET_ERR_INVALID_ARG, "bad sizes or k");
  if (n_tau < 0 || (n_tau > 0 && !tau_pairs) || limit < 1) return sfail(s, JET_ERR_INVALID_ARG, "bad schedule");
  Job j;
  j.hg = *hg_host;
  j.params = *params;
  j.tau.assign(tau_pairs, tau_pairs + 2 * n_tau);
  j.limit = limit;
  j.part = part_host;
  j.bytes = jet_job_footprint(hg_host->n, hg_host->m, hg_host->P, params->k);
  if (j.bytes > s->budget) return sfail(s, JET_ERR_OOM, "the job's device footprint exceeds the whole budget");
  j.t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return sfail(s, JET_ERR_INVALID_ARG, "the server is shutting down");
  j.id = s->next_id++;
  *id_out = j.id;
  s->pending.push_back(std::move(j));
  admit_locked(s);
  return JET_OK;
}

int jet_server_wait(jet_server *s, jet_job_done *done, int32_t max_done, int32_t *n_done, int32_t timeout_ms) {
  if (!s || !n_done || (max_done > 0 && !done)) return sfail(s, JET_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && timeout_ms != 0) {
    auto ready = [&] { return !s->done.empty(); };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  }
  int32_t k = 0;
  while (k < max_done && !s->done.empty()) {
    done[k++] = s->done.front();
    s->done.pop_front();
  }
  *n_done = k;
  return JET_OK;
}

int jet_server_load(jet_server *s, int32_t *pending, int32_t *running, size_t *reserved_bytes) {
  if (!s) return sfail(nullptr, JET_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  if (pending) *pending = (int32_t)s->pending.size();
  if (running) *running = s->active + (int32_t)s->admitted.size();
  if (reserved_bytes) *reserved_bytes = s->reserved;
  return JET_OK;
}

const char *jet_server_last_error(const jet_server *s) { return s ? s->err : jet_last_error(nullptr); }

void jet_server_destroy(jet_server *s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // every submitted job still runs to completion: wait until nothing is pending
    s->cv_done.wait(lk, [&] { return s->pending.empty() && s->admitted.empty() && s->active == 0; });
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (std::thread &t : s->workers)
    if (t.joinable()) t.join();
  if (s->ev_ref) cudaEventDestroy(s->ev_ref);
  delete s;
}

}  // extern "C"
