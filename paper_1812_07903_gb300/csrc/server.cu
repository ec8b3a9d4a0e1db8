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
//
// Captured graphs: from the second job of a shape on (n, d, ldx, dtype, parameters, with or
// without the order), a leverage job's launches are recorded by stream capture into a CUDA graph
// and replayed with one cudaGraphLaunch.  Each slot keeps the instantiated graphs of recent job
// shapes together with their workspace, so a later job of the same shape only re-records its
// launches against that workspace and updates the instantiated graph in place
// (cudaGraphExecUpdate: new X, scores and order pointers) instead of instantiating again.  Cached workspaces count against a quarter of
// the memory budget (least recently used shapes are dropped); a job whose launches cannot be
// captured runs them directly.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "tmap.cuh"

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

// An instantiated graph of one job shape and the workspace its launches were recorded against.
struct GraphEntry {
  std::vector<int64_t> key;
  cudaGraphExec_t exec = nullptr;
  void* ws = nullptr;
  size_t bytes = 0;
  uint64_t last_use = 0;
};

struct Slot {
  Handle h;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  Job* job = nullptr;
  void* ws = nullptr;
  std::vector<GraphEntry> graphs;
  // a grouped launch: the slot's jobs (job == group[0]), each with its own device status words,
  // scratch, and descriptor of its score product (pinned on the host, copied to the device)
  std::vector<Job*> group;
  DevState* gstate = nullptr;
  DevState* gstate_host = nullptr;
  ScoreGroupJob* gdesc_host = nullptr;
  ScoreGroupJob* gdesc_dev = nullptr;
  void* gws[kMaxScoreGroup] = {};
};

constexpr int64_t kGroupMaxRows = int64_t(1) << 17;  // jobs of at most this many rows are grouped

constexpr size_t kGraphsPerSlot = 8;
constexpr size_t kSeenShapes = 256;

}  // namespace

struct Server {
  int device = 0;
  std::vector<Slot> slots;
  size_t budget = 0, in_use = 0;
  std::deque<Job*> queue;
  std::unordered_map<int64_t, Job*> jobs;
  int64_t next_ticket = 1;
  int64_t n_submitted = 0, n_admitted = 0, n_completed = 0;
  // graph statistics: new instantiations, in-place updates, direct (uncaptured) leverage runs
  int64_t n_graph_new = 0, n_graph_update = 0, n_graph_direct = 0;
  int64_t n_group_launches = 0, n_grouped_jobs = 0;  // grouped score launches and the jobs they ran
  size_t graph_bytes = 0;  // workspaces held by cached graphs (all slots)
  uint64_t use_clock = 0;
  bool capture_ok = true;  // cleared if the CUDA driver refuses to capture the launches
  std::deque<std::vector<int64_t>> seen;  // recent leverage shapes (a shape's first job runs direct)
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
    if (j->d < 1 || j->n < j->d || j->d > kMaxD || j->n >= (int64_t(1) << 31))
      return fail(SLSO_ERR_SHAPE, "sketched SVD job needs 1 <= d <= s (s=%lld, d=%lld)", (long long)j->n,
                  (long long)j->d);
    return SLSO_OK;
  }
  return fail(SLSO_ERR_INVALID_ARG, "unknown job kind %d", j->job);
}

// Shape key of a leverage job: everything the launch sequence depends on except the X, scores
// and order addresses (an X address of different alignment may change it; then the update is
// refused and the graph instantiated again).
std::vector<int64_t> graph_key(const slso_job& d) {
  const slso_params& p = d.params;
  int64_t tau_bits = 0, frac_bits = 0;
  std::memcpy(&tau_bits, &p.tau, sizeof(double));
  std::memcpy(&frac_bits, &p.correct_frac, sizeof(double));
  return {d.n, d.d, d.ldx, d.xdt, p.kind, p.s, p.k, static_cast<int64_t>(p.seed_S), static_cast<int64_t>(p.seed_Pi),
          tau_bits, p.compute, frac_bits, p.nnz, d.order ? 1 : 0};
}

// Record the job's launches on the slot's stream into a graph against workspace ws.
slso_status capture_job(Slot& sl, const Job* j, void* ws, cudaGraph_t* g) {
  *g = nullptr;
  SLSO_CHECK_CUDA(cudaStreamBeginCapture(sl.st, cudaStreamCaptureModeThreadLocal));
  Arena ar(static_cast<char*>(ws), j->bytes + 256, false);
  const slso_status stt = job_plan(sl.h, ar, j->desc, sl.st);
  const cudaError_t e = cudaStreamEndCapture(sl.st, g);  // always ends the capture
  cudaGetLastError();
  if (stt != SLSO_OK || e != cudaSuccess) {
    if (*g) cudaGraphDestroy(*g);
    *g = nullptr;
    return stt != SLSO_OK ? stt : fail(SLSO_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
  }
  return SLSO_OK;
}

// Run a leverage job through the slot's graph cache (worker thread only: the slots' graph lists,
// graph_bytes and capture_ok are touched by no other thread).  Returns 0 when the job must run
// uncaptured (nothing was enqueued), 1 after a new instantiation, 2 after an in-place update.
int start_job_graph(Server& s, Slot& sl, Job* j) {
  if (!s.capture_ok || j->desc.job != SLSO_JOB_LEVERAGE) return 0;
  const std::vector<int64_t> key = graph_key(j->desc);
  int outcome = 0;
  GraphEntry* e = nullptr;
  for (GraphEntry& g : sl.graphs)
    if (g.key == key) e = &g;
  if (!e) {
    // a shape's first job runs direct: instantiating a graph costs more than launching once
    bool seen = false;
    for (const auto& k : s.seen) seen |= k == key;
    if (!seen) {
      s.seen.push_back(key);
      if (s.seen.size() > kSeenShapes) s.seen.pop_front();
      return 0;
    }
    // room for one more cached workspace: drop least recently used entries of this slot
    const size_t cap = s.budget / 4;
    while (!sl.graphs.empty() && (sl.graphs.size() >= kGraphsPerSlot || s.graph_bytes + j->bytes + 256 > cap)) {
      size_t lru = 0;
      for (size_t i = 1; i < sl.graphs.size(); ++i)
        if (sl.graphs[i].last_use < sl.graphs[lru].last_use) lru = i;
      GraphEntry& v = sl.graphs[lru];
      cudaGraphExecDestroy(v.exec);
      cudaFreeAsync(v.ws, sl.st);
      s.graph_bytes -= v.bytes + 256;
      sl.graphs.erase(sl.graphs.begin() + static_cast<std::ptrdiff_t>(lru));
    }
    if (s.graph_bytes + j->bytes + 256 > cap) return 0;
    GraphEntry ne;
    ne.key = key;
    ne.bytes = j->bytes;
    if (cudaMallocAsync(&ne.ws, j->bytes + 256, sl.st) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaGraph_t g = nullptr;
    if (capture_job(sl, j, ne.ws, &g) != SLSO_OK || cudaGraphInstantiate(&ne.exec, g, 0) != cudaSuccess) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      cudaFreeAsync(ne.ws, sl.st);
      s.capture_ok = false;  // the plan is the same kind of launch sequence for every job: stop trying
      return 0;
    }
    cudaGraphDestroy(g);
    s.graph_bytes += ne.bytes + 256;
    sl.graphs.push_back(ne);
    e = &sl.graphs.back();
    outcome = 1;
  } else {
    cudaGraph_t g = nullptr;
    if (capture_job(sl, j, e->ws, &g) != SLSO_OK) return 0;
    cudaGraphExecUpdateResultInfo res{};
    if (cudaGraphExecUpdate(e->exec, g, &res) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(e->exec);
      e->exec = nullptr;
      if (cudaGraphInstantiate(&e->exec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        cudaFreeAsync(e->ws, sl.st);
        s.graph_bytes -= e->bytes + 256;
        sl.graphs.erase(sl.graphs.begin() + (e - sl.graphs.data()));
        return 0;
      }
      outcome = 1;
    } else {
      outcome = 2;
    }
    cudaGraphDestroy(g);
  }
  e->last_use = ++s.use_clock;
  j->status = SLSO_OK;
  if (cudaMemsetAsync(sl.h.state, 0, sizeof(DevState), sl.st) != cudaSuccess ||
      cudaGraphLaunch(e->exec, sl.st) != cudaSuccess) {
    cudaGetLastError();
    j->status = SLSO_ERR_CUDA;
  }
  cudaEventRecord(sl.done, sl.st);
  return outcome;
}

// Enqueue a job's work on its slot (worker thread, lock not held).
void start_job(Server& srv, Slot& sl, Job* j) {
  const int outcome = start_job_graph(srv, sl, j);
  {
    std::lock_guard<std::mutex> lk(srv.mu);
    if (outcome == 1) ++srv.n_graph_new;
    else if (outcome == 2) ++srv.n_graph_update;
    else if (j->desc.job == SLSO_JOB_LEVERAGE) ++srv.n_graph_direct;
  }
  if (outcome) return;
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

// A leverage job whose scores can share a grouped launch: float32 X and compute, k <= 128,
// d <= 2048, at most kGroupMaxRows rows, no correction pass.  Jobs group with those of the same
// JL width (rounded up to 32).
bool group_eligible(const Slot& sl, const Job* j) {
  const slso_job& d = j->desc;
  return d.job == SLSO_JOB_LEVERAGE && d.n <= kGroupMaxRows &&
         score_group_eligible(sl.h, d.X, d.d, d.ldx, d.xdt, d.params.k, d.params.compute, d.params.correct_frac);
}
int64_t group_width(const Job* j) { return (j->desc.params.k + 31) / 32; }

// Enqueue a group's work on its slot (worker thread, lock not held): every job's sketch and solve
// with its own status words and scratch, one grouped score launch over all of them, then every
// job's score sum and order.  A job that fails before the launch is left out of it.
void start_group(Server& srv, Slot& sl) {
  const int m = static_cast<int>(sl.group.size());
  std::vector<Arena> ars;
  std::vector<double*> sums(m, nullptr);
  std::vector<int> in(m, 0);
  ars.reserve(m);
  int nd = 0;
  for (int i = 0; i < m; ++i) {
    Job* j = sl.group[i];
    const slso_job& d = j->desc;
    Handle hj = sl.h;
    hj.state = sl.gstate + i;
    hj.state_host = sl.gstate_host + i;
    sl.gws[i] = nullptr;
    slso_status stt = SLSO_OK;
    if (cudaMemsetAsync(hj.state, 0, sizeof(DevState), sl.st) != cudaSuccess) stt = SLSO_ERR_CUDA;
    if (stt == SLSO_OK && cudaMallocAsync(&sl.gws[i], j->bytes + 256, sl.st) != cudaSuccess) {
      cudaGetLastError();
      sl.gws[i] = nullptr;
      stt = SLSO_ERR_OOM;
    }
    ars.emplace_back(static_cast<char*>(sl.gws[i]), j->bytes + 256, false);
    const double* M = nullptr;
    int64_t kk = 0;
    const unsigned int* colmax = nullptr;
    if (stt == SLSO_OK) stt = leverage_solve(hj, ars[i], d.X, d.n, d.d, d.ldx, d.xdt, &d.params, sl.st, &M, &kk, &colmax);
    if (stt == SLSO_OK)
      stt = score_group_add(hj, ars[i], d.X, d.n, d.d, d.ldx, M, kk, static_cast<float*>(d.scores),
                            &sl.gdesc_host[nd], &sums[i], sl.st);
    j->status = stt;
    if (stt == SLSO_OK) {
      in[i] = 1;
      ++nd;
    }
  }
  if (nd > 0 && score_group_launch(sl.h, sl.gdesc_host, sl.gdesc_dev, nd, sl.st) != SLSO_OK)
    for (int i = 0; i < m; ++i)
      if (in[i]) {
        sl.group[i]->status = SLSO_ERR_CUDA;
        in[i] = 0;
      }
  for (int i = 0; i < m; ++i) {
    if (!in[i]) continue;
    Job* j = sl.group[i];
    const slso_job& d = j->desc;
    Handle hj = sl.h;
    hj.state = sl.gstate + i;
    hj.state_host = sl.gstate_host + i;
    slso_status stt = score_group_sum(hj, static_cast<const float*>(d.scores), d.n, sums[i], sl.st);
    if (stt == SLSO_OK && d.order) stt = order_scores(hj, ars[i], d.scores, SLSO_F32, d.n, d.order, sl.st);
    j->status = stt;
  }
  for (int i = 0; i < m; ++i)
    if (sl.gws[i]) cudaFreeAsync(sl.gws[i], sl.st);
  cudaEventRecord(sl.done, sl.st);
  std::lock_guard<std::mutex> lk(srv.mu);
  ++srv.n_group_launches;
  srv.n_grouped_jobs += nd;
}

// Collect a finished group (worker thread, lock held): every job's status words.
void finish_group(Server& s, Slot& sl) {
  const int m = static_cast<int>(sl.group.size());
  const bool copied =
      cudaMemcpy(sl.gstate_host, sl.gstate, sizeof(DevState) * m, cudaMemcpyDeviceToHost) == cudaSuccess;
  for (int i = 0; i < m; ++i) {
    Job* j = sl.group[i];
    if (j->status == SLSO_OK) {
      if (!copied) {
        j->status = SLSO_ERR_CUDA;
      } else {
        const DevState& d = sl.gstate_host[i];
        info_from_state(d, &j->info);
        if (d.timeout) j->status = SLSO_ERR_TIMEOUT;
        else if (d.nonfinite) j->status = SLSO_ERR_NONFINITE;
      }
    }
    j->t_done = now_ms();
    j->done = true;
    s.in_use -= j->bytes;
    ++s.n_completed;
  }
  sl.group.clear();
  sl.job = nullptr;
  s.cv_done.notify_all();
}

// Collect a finished job (worker thread, lock held).
void finish_job(Server& s, Slot& sl) {
  Job* j = sl.job;
  if (j->status == SLSO_OK) {
    if (cudaMemcpy(sl.h.state_host, sl.h.state, sizeof(DevState), cudaMemcpyDeviceToHost) != cudaSuccess) {
      j->status = SLSO_ERR_CUDA;
    } else {
      const DevState& d = *sl.h.state_host;
      info_from_state(d, &j->info);
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
      if (q != cudaSuccess) {
        sl.job->status = SLSO_ERR_CUDA;
        for (Job* g : sl.group) g->status = SLSO_ERR_CUDA;
      }
      if (sl.group.empty()) finish_job(*s, sl);
      else finish_group(*s, sl);
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
      // consecutive queued jobs that can share one grouped score launch go to this slot together
      if (free_slot->gstate && group_eligible(*free_slot, j)) {
        size_t bytes = j->bytes;
        size_t cnt = 1;
        while (cnt < s->queue.size() && cnt < static_cast<size_t>(kMaxScoreGroup)) {
          Job* nx = s->queue[cnt];
          if (!group_eligible(*free_slot, nx) || group_width(nx) != group_width(j) ||
              s->in_use + bytes + nx->bytes > s->budget)
            break;
          bytes += nx->bytes;
          ++cnt;
        }
        if (cnt >= 2) {
          free_slot->group.assign(s->queue.begin(), s->queue.begin() + static_cast<std::ptrdiff_t>(cnt));
          for (size_t c = 0; c < cnt; ++c) s->queue.pop_front();
          const double t = now_ms();
          for (Job* g : free_slot->group) g->t_admit = t;
          s->in_use += bytes;
          s->n_admitted += static_cast<int64_t>(cnt);
          free_slot->job = j;
          lk.unlock();
          start_group(*s, *free_slot);
          lk.lock();
          progressed = true;
          continue;
        }
      }
      s->queue.pop_front();
      s->in_use += j->bytes;
      j->t_admit = now_ms();
      ++s->n_admitted;
      free_slot->job = j;
      lk.unlock();
      start_job(*s, *free_slot, j);
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
    if (e == cudaSuccess) e = side_stream_create(sl.h);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sl.gstate), sizeof(DevState) * kMaxScoreGroup);
    if (e == cudaSuccess)
      e = cudaMallocHost(reinterpret_cast<void**>(&sl.gstate_host), sizeof(DevState) * kMaxScoreGroup);
    if (e == cudaSuccess)
      e = cudaMallocHost(reinterpret_cast<void**>(&sl.gdesc_host), sizeof(ScoreGroupJob) * kMaxScoreGroup);
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&sl.gdesc_dev), sizeof(ScoreGroupJob) * kMaxScoreGroup);
    if (e != cudaSuccess) {
      for (Slot& t : s->slots) {
        side_stream_release(t.h);
        if (t.gstate) cudaFree(t.gstate);
        if (t.gstate_host) cudaFreeHost(t.gstate_host);
        if (t.gdesc_host) cudaFreeHost(t.gdesc_host);
        if (t.gdesc_dev) cudaFree(t.gdesc_dev);
        if (t.st) cudaStreamDestroy(t.st);
        if (t.done) cudaEventDestroy(t.done);
        if (t.h.state) cudaFree(t.h.state);
        if (t.h.state_host) cudaFreeHost(t.h.state_host);
      }
      delete s;
      return fail(SLSO_ERR_CUDA, "slso_server_create: %s", cudaGetErrorString(e));
    }
  }
  encode_fn();  // resolve the CUDA driver entry point now, not while a capture is recording
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
    for (GraphEntry& g : sl.graphs) {
      cudaGraphExecDestroy(g.exec);
      cudaFree(g.ws);
    }
    sl.graphs.clear();
    side_stream_release(sl.h);
    if (sl.gstate) cudaFree(sl.gstate);
    if (sl.gstate_host) cudaFreeHost(sl.gstate_host);
    if (sl.gdesc_host) cudaFreeHost(sl.gdesc_host);
    if (sl.gdesc_dev) cudaFree(sl.gdesc_dev);
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

extern "C" slso_status slso_server_counters(slso_server* srv, int64_t* counters, int32_t count) {
  if (!srv || !counters || count < 0) return fail(SLSO_ERR_INVALID_ARG, "server and counters must be non-NULL");
  Server* s = reinterpret_cast<Server*>(srv);
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t v[] = {s->n_submitted, s->n_admitted, s->n_completed, static_cast<int64_t>(s->queue.size()),
                       static_cast<int64_t>(s->in_use), s->n_graph_new, s->n_graph_update, s->n_graph_direct,
                       s->n_group_launches, s->n_grouped_jobs};
  for (int32_t i = 0; i < count; ++i) counters[i] = i < static_cast<int32_t>(sizeof(v) / sizeof(v[0])) ? v[i] : 0;
  return SLSO_OK;
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
