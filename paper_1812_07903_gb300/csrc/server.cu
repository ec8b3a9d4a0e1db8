// Continuous-batching server for leverage-score and sketched-SVD jobs (C ABI: slso_server_*).
//
// A worker thread owns the device side.  Jobs are submitted without blocking and queue in
// arrival order.  A job is admitted when a slot is free and its device footprint (its scratch
// plan, measured exactly like slso_workspace_size) fits in the memory budget next to the jobs
// already running; admission is FIFO, so a large job is not overtaken.  Each slot has its own
// stream and its own device status words, so admitted jobs run concurrently on the GPU and
// jobs arriving while others run are admitted as slots and memory free up.  Scratch is
// allocated stream-ordered (cudaMallocAsync / cudaFreeAsync on the slot's stream), which never
// synchronises the device.  Every kernel on the path is deterministic, so a job's result is
// the same alone and in any mix.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace slso {
namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
  int64_t ticket = 0;
  slso_job desc{};
  size_t bytes = 0;
  slso_status status = SLSO_OK;
  slso_info info{};
  double t_submit = 0, t_admit = 0, t_done = 0;
  bool done = false;
};

struct Slot {
  Handle h;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  Job* job = nullptr;
  void* ws = nullptr;
};

}  // namespace

struct Server {
  int device = 0;
  std::vector<Slot> slots;
  size_t budget = 0, in_use = 0;
  std::deque<Job*> queue;
  std::unordered_map<int64_t, Job*> jobs;
  int64_t next_ticket = 1;
  int64_t n_submitted = 0, n_admitted = 0, n_completed = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
};

namespace {

// Scratch plan of a job; measured with a null arena (nothing is launched).
slso_status job_plan(Handle& h, Arena& ar, const slso_job& j, cudaStream_t st) {
  if (j.job == SLSO_JOB_LEVERAGE) {
    SLSO_TRY(leverage_plan(h, ar, j.X, j.n, j.d, j.ldx, j.xdt, &j.params, j.scores, st));
    if (j.order) {
      const int32_t sdt = j.params.compute == SLSO_F64 ? SLSO_F64 : SLSO_F32;
      SLSO_TRY(order_scores(h, ar, j.scores, sdt, j.n, j.order, st));
    }
    return SLSO_OK;
  }
  const double tau = j.params.tau < 0 ? default_tau(j.n, j.d) : j.params.tau;
  SolveOut so;
  SLSO_TRY(run_solve(h, ar, static_cast<const double*>(j.X), j.n, j.d, tau, 0, 0, 1, &so, st));
  if (!ar.measure()) {
    SLSO_CHECK_CUDA(cudaMemcpyAsync(j.sigma, so.sigma, sizeof(double) * j.d, cudaMemcpyDeviceToDevice, st));
    SLSO_CHECK_CUDA(cudaMemcpyAsync(j.V, so.V, sizeof(double) * j.d * j.d, cudaMemcpyDeviceToDevice, st));
    if (j.R) SLSO_CHECK_CUDA(cudaMemcpyAsync(j.R, so.R, sizeof(double) * j.d * j.d, cudaMemcpyDeviceToDevice, st));
  }
  return SLSO_OK;
}

slso_status check_job(const slso_job* j) {
  if (!j) return fail(SLSO_ERR_INVALID_ARG, "job is NULL");
  if (j->job == SLSO_JOB_LEVERAGE) {
    SLSO_TRY(check_x(j->X, j->n, j->d, j->ldx, j->xdt));
    SLSO_TRY(check_params(&j->params, j->n, j->d));
    if (!j->scores) return fail(SLSO_ERR_INVALID_ARG, "job scores is NULL");
    return SLSO_OK;
  }
  if (j->job == SLSO_JOB_SKETCHED_SVD) {
    if (!j->X || !j->sigma || !j->V) return fail(SLSO_ERR_INVALID_ARG, "sketched SVD job needs SX, sigma and V");
    if (j->d < 1 || j->n < j->d || j->d > 8192 || j->n >= (int64_t(1) << 31))
      return fail(SLSO_ERR_SHAPE, "sketched SVD job needs 1 <= d <= s (s=%lld, d=%lld)", (long long)j->n,
                  (long long)j->d);
    return SLSO_OK;
  }
  return fail(SLSO_ERR_INVALID_ARG, "unknown job kind %d", j->job);
}

// Enqueue a job's work on its slot (worker thread, lock not held).
void start_job(Slot& sl, Job* j) {
  slso_status stt = SLSO_OK;
  if (cudaMemsetAsync(sl.h.state, 0, sizeof(DevState), sl.st) != cudaSuccess) stt = SLSO_ERR_CUDA;
  if (stt == SLSO_OK && cudaMallocAsync(&sl.ws, j->bytes + 256, sl.st) != cudaSuccess) {
    cudaGetLastError();
    sl.ws = nullptr;
    stt = SLSO_ERR_OOM;
  }
  if (stt == SLSO_OK) {
    Arena ar(static_cast<char*>(sl.ws), j->bytes + 256, false);
    stt = job_plan(sl.h, ar, j->desc, sl.st);
  }
  if (sl.ws) cudaFreeAsync(sl.ws, sl.st);
  sl.ws = nullptr;
  j->status = stt;
  cudaEventRecord(sl.done, sl.st);
}

// Collect a finished job (worker thread, lock held).
void finish_job(Server& s, Slot& sl) {
  Job* j = sl.job;
  if (j->status == SLSO_OK) {
    if (cudaMemcpy(sl.h.state_host, sl.h.state, sizeof(DevState), cudaMemcpyDeviceToHost) != cudaSuccess) {
      j->status = SLSO_ERR_CUDA;
    } else {
      const DevState& d = *sl.h.state_host;
      j->info.rank = d.rank;
      j->info.sigma_max = d.sigma_max;
      j->info.sigma_min_kept = d.sigma_min_kept;
      j->info.score_sum = d.score_sum;
      j->info.tau = d.tau;
      j->info.nonfinite = d.nonfinite;
      j->info.svd_sweeps = d.sweeps;
      j->info.svd_route = d.need_svd;
      if (d.timeout) j->status = SLSO_ERR_TIMEOUT;
      else if (d.nonfinite) j->status = SLSO_ERR_NONFINITE;
    }
  }
  j->t_done = now_ms();
  j->done = true;
  s.in_use -= j->bytes;
  ++s.n_completed;
  sl.job = nullptr;
  s.cv_done.notify_all();
}

void worker_main(Server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool progressed = false;
    for (Slot& sl : s->slots) {
      if (!sl.job) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) sl.job->status = SLSO_ERR_CUDA;
      finish_job(*s, sl);
      progressed = true;
    }
    while (!s->queue.empty()) {
      Job* j = s->queue.front();
      Slot* free_slot = nullptr;
      for (Slot& sl : s->slots)
        if (!sl.job) {
          free_slot = &sl;
          break;
        }
      if (!free_slot || s->in_use + j->bytes > s->budget) break;  // FIFO: no overtaking
      s->queue.pop_front();
      s->in_use += j->bytes;
      j->t_admit = now_ms();
      ++s->n_admitted;
      free_slot->job = j;
      lk.unlock();
      start_job(*free_slot, j);
      lk.lock();
      progressed = true;
    }
    bool busy = false;
    for (Slot& sl : s->slots) busy |= sl.job != nullptr;
    if (s->stop && !busy) break;
    if (!progressed) s->cv_work.wait_for(lk, std::chrono::microseconds(busy ? 20 : 2000));
  }
}

}  // namespace
}  // namespace slso

using namespace slso;

extern "C" slso_status slso_server_create(slso_server** out, int device, int nslots, size_t mem_budget_bytes) {
  if (!out) return fail(SLSO_ERR_INVALID_ARG, "server out-pointer is NULL");
  *out = nullptr;
  if (nslots < 1 || nslots > 64) return fail(SLSO_ERR_INVALID_ARG, "slots must be in [1, 64]");
  if (mem_budget_bytes == 0) return fail(SLSO_ERR_INVALID_ARG, "memory budget is 0");
  int count = 0;
  SLSO_CHECK_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return fail(SLSO_ERR_INVALID_ARG, "device %d out of range", device);
  SLSO_CHECK_CUDA(cudaSetDevice(device));
  Server* s = new Server();
  s->device = device;
  s->budget = mem_budget_bytes;
  s->slots.resize(nslots);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  for (Slot& sl : s->slots) {
    sl.h.device = device;
    sl.h.num_sms = sms;
    cudaError_t e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sl.h.state), sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&sl.h.state_host), sizeof(DevState));
    if (e != cudaSuccess) {
      for (Slot& t : s->slots) {
        if (t.st) cudaStreamDestroy(t.st);
        if (t.done) cudaEventDestroy(t.done);
        if (t.h.state) cudaFree(t.h.state);
        if (t.h.state_host) cudaFreeHost(t.h.state_host);
      }
      delete s;
      return fail(SLSO_ERR_CUDA, "slso_server_create: %s", cudaGetErrorString(e));
    }
  }
  s->worker = std::thread(worker_main, s);
  *out = reinterpret_cast<slso_server*>(s);
  return SLSO_OK;
}

extern "C" slso_status slso_server_destroy(slso_server* srv) {
  if (!srv) return SLSO_OK;
  Server* s = reinterpret_cast<Server*>(srv);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Job* j : s->queue) {  // not admitted: fail them
      j->status = SLSO_ERR_BUSY;
      j->done = true;
    }
    s->queue.clear();
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->worker.join();
  cudaSetDevice(s->device);
  for (Slot& sl : s->slots) {
    cudaStreamSynchronize(sl.st);
    cudaStreamDestroy(sl.st);
    cudaEventDestroy(sl.done);
    cudaFree(sl.h.state);
    cudaFreeHost(sl.h.state_host);
  }
  for (auto& kv : s->jobs) delete kv.second;
  delete s;
  return SLSO_OK;
}

extern "C" slso_status slso_server_submit(slso_server* srv, const slso_job* job, int64_t* ticket) {
  if (!srv || !ticket) return fail(SLSO_ERR_INVALID_ARG, "server and ticket must be non-NULL");
  SLSO_TRY(check_job(job));
  Server* s = reinterpret_cast<Server*>(srv);
  Handle probe;
  probe.num_sms = s->slots[0].h.num_sms;
  Arena m(nullptr, ~size_t(0), true);
  SLSO_TRY(job_plan(probe, m, *job, nullptr));
  const size_t bytes = m.used();
  if (bytes > s->budget)
    return fail(SLSO_ERR_BUSY, "job needs %zu bytes of scratch, more than the server's budget %zu", bytes,
                s->budget);
  Job* j = new Job();
  j->desc = *job;
  j->bytes = bytes;
  j->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete j;
      return fail(SLSO_ERR_BUSY, "server is shutting down");
    }
    j->ticket = s->next_ticket++;
    s->jobs[j->ticket] = j;
    s->queue.push_back(j);
    ++s->n_submitted;
    *ticket = j->ticket;
  }
  s->cv_work.notify_all();
  return SLSO_OK;
}

extern "C" slso_status slso_server_poll(slso_server* srv, int64_t ticket, int timeout_ms, slso_status* job_status,
                                        slso_info* info, double* times_ms) {
  if (!srv || !job_status) return fail(SLSO_ERR_INVALID_ARG, "server and job_status must be non-NULL");
  Server* s = reinterpret_cast<Server*>(srv);
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return fail(SLSO_ERR_NOT_FOUND, "unknown ticket %lld", (long long)ticket);
  Job* j = it->second;
  if (!j->done) {
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), [&] { return j->done; });
    if (!j->done) return fail(SLSO_ERR_TIMEOUT, "job %lld not finished within %d ms", (long long)ticket, timeout_ms);
  }
  *job_status = j->status;
  if (info) *info = j->info;
  if (times_ms) {
    times_ms[0] = (j->t_admit > 0 ? j->t_admit : j->t_done) - j->t_submit;  // queued
    times_ms[1] = j->t_admit > 0 ? j->t_done - j->t_admit : 0.0;            // admitted -> done
    times_ms[2] = j->t_done - j->t_submit;                                   // latency
  }
  s->jobs.erase(it);
  delete j;
  return SLSO_OK;
}

extern "C" slso_status slso_server_cancel(slso_server* srv, int64_t ticket) {
  if (!srv) return fail(SLSO_ERR_INVALID_ARG, "server is NULL");
  Server* s = reinterpret_cast<Server*>(srv);
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return fail(SLSO_ERR_NOT_FOUND, "unknown ticket %lld", (long long)ticket);
  Job* j = it->second;
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q) {
    if (*q != j) continue;
    s->queue.erase(q);
    j->status = SLSO_ERR_CANCELLED;
    j->t_done = now_ms();
    j->done = true;
    s->cv_done.notify_all();
    s->cv_work.notify_all();  // the job behind it may now fit
    return SLSO_OK;
  }
  return fail(SLSO_ERR_BUSY, "job %lld is already %s", (long long)ticket, j->done ? "finished" : "running");
}

extern "C" slso_status slso_server_stats(slso_server* srv, int64_t* counters, size_t* mem_in_use) {
  if (!srv || !counters) return fail(SLSO_ERR_INVALID_ARG, "server and counters must be non-NULL");
  Server* s = reinterpret_cast<Server*>(srv);
  std::lock_guard<std::mutex> lk(s->mu);
  counters[0] = s->n_submitted;
  counters[1] = s->n_admitted;
  counters[2] = s->n_completed;
  counters[3] = static_cast<int64_t>(s->queue.size());
  if (mem_in_use) *mem_in_use = s->in_use;
  return SLSO_OK;
}
