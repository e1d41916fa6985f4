// Job server: continuous batching of contraction jobs on one GPU.
//
// A scheduler thread owns `slots` execution slots.  Each slot is a sub-context (its own
// workspace, phase-table cache and device error word) with its own non-blocking stream, so
// jobs admitted to different slots overlap on the device.  Jobs wait in a queue; the
// scheduler admits the first queued job that fits, as soon as a slot is free and the HBM
// budget allows: resident propagators + the workspace every slot holds + the job's
// additional need (an upper bound from the call shapes) must stay within the budget.
// Completion is detected with an event on the slot's stream, then the slot's device error
// word is read, so a job that hit a bounded device wait ends in LHC_JOB_FAILED.
//
// Kernels are deterministic (fixed summation order, no atomics), so a job's result does
// not depend on what runs beside it.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "lhc_internal.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Prop {
  const void *ptr;
  lhc_lattice lat;
  size_t bytes;
};

struct Job {
  uint64_t id;
  lhc_job spec;
  std::vector<int> k;   // copied momentum list
  int state = LHC_JOB_QUEUED;
  int status = LHC_OK;
  std::string msg;      // error text of a failed job
  size_t need = 0;      // workspace upper bound
  int slot = -1;
  double t_submit = 0, t_start = 0, t_done = 0;
  // device times (ms after the server's epoch event) at which the slot's stream reached
  // the job's first launch and finished its last, from timing events on that stream
  double d_start = -1, d_done = -1;
  cudaEvent_t ev0 = nullptr, ev = nullptr;
};

struct Slot {
  lhc_ctx sub = nullptr;
  cudaStream_t stream = nullptr;
  size_t reserved = 0;   // workspace this slot may hold (largest admitted need)
  Job *job = nullptr;
};

size_t esize(int dtype) { return dtype == LHC_C128 ? 16 : 8; }

}  // namespace

struct lhc_server_s {
  lhc_ctx ctx;
  size_t budget;
  std::vector<Slot> slots;
  std::deque<Job *> queue;
  std::map<uint64_t, Job *> jobs;
  std::map<uint64_t, Prop> props;
  size_t prop_bytes = 0;
  uint64_t next_id = 1, next_prop = 1;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::thread worker;
  bool stop = false;
  cudaEvent_t epoch = nullptr;   // recorded once at start: the origin of the jobs' device times
};

namespace {

std::mutex g_servers_mu;
std::map<lhc_ctx, lhc_server_s *> g_servers;

lhc_server_s *server_of(lhc_ctx ctx) {
  std::lock_guard<std::mutex> g(g_servers_mu);
  auto it = g_servers.find(ctx);
  return it == g_servers.end() ? nullptr : it->second;
}

size_t in_use(lhc_server_s *s) {
  size_t b = s->prop_bytes;
  for (auto &sl : s->slots) b += sl.reserved;
  return b;
}

// upper bound of the workspace a job needs in its slot
size_t job_need(const lhc_job &j, const Prop &p) {
  const int V3 = p.lat.L * p.lat.L * p.lat.L;
  size_t ins = 0, spec = 0;
  const bool fp64 = j.prec == LHC_FP64;
  // a slot's context projects in the automatic mode: the transform for half the momenta or more
  const bool dft = 2 * (long long)j.nq >= V3;
  if (j.type != LHC_JOB_SPECTATOR) {
    int nt = j.t_hi - j.t_lo + 1;
    ins = dft    ? lhc::fft_call_bytes(lhc::PART_INS, j.prec, p.lat.L, j.n_r, j.nq)
          : fp64 ? ((size_t)1 << 30) + (size_t)j.nq * V3 * 16 + 4096
                 : lhc::mixed_call_bytes(lhc::PART_INS, p.lat.dtype, V3, j.n_r, nt, j.nq);
  }
  if (j.type != LHC_JOB_INSERTION) {
    auto part = j.kind == LHC_BARYON ? lhc::PART_SPEC_BARYON : lhc::PART_SPEC_MESON;
    spec = dft    ? lhc::fft_call_bytes(part, j.prec, p.lat.L, j.n_r, j.nq)
           : fp64 ? ((size_t)1 << 30) + (size_t)j.nq * V3 * 16 + 4096
                  : lhc::mixed_call_bytes(part, p.lat.dtype, V3, j.n_r, 1, j.nq);
  }
  // one workspace (the larger call) plus both phase tables, with 25 % growth slack
  return (size_t)((std::max(ins, spec) + std::min(ins, spec) / 4) * 1.25);
}

int launch_job(lhc_server_s *s, Slot &sl, Job *jb) {
  const lhc_job &j = jb->spec;
  lhc_set_gamma5(sl.sub, s->ctx->g5);
  const Prop &p = s->props.at(j.prop);
  const void *gb = j.prop_b ? s->props.at(j.prop_b).ptr : nullptr;
  int st = LHC_OK;
  if (cudaEventRecord(jb->ev0, sl.stream) != cudaSuccess) st = LHC_ECUDA;
  if (st == LHC_OK && j.type != LHC_JOB_SPECTATOR)
    st = lhc_insertion(sl.sub, &p.lat, p.ptr, j.psi, j.n_r, j.t_lo, j.t_hi, j.r, jb->k.data(), j.nq, j.prec,
                       j.out_ins, sl.stream);
  if (st == LHC_OK && j.type != LHC_JOB_INSERTION)
    st = lhc_spectator(sl.sub, &p.lat, j.kind, p.ptr, gb, j.eta, j.n_r, j.t_sink, j.r, jb->k.data(), j.nq, j.prec,
                       j.out_spec, sl.stream);
  if (st == LHC_OK && cudaEventRecord(jb->ev, sl.stream) != cudaSuccess) st = LHC_ECUDA;
  return st;
}

void worker_main(lhc_server_s *s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    // completions
    for (auto &sl : s->slots) {
      if (!sl.job) continue;
      if (cudaEventQuery(sl.job->ev) == cudaErrorNotReady) continue;
      Job *jb = sl.job;
      int st = lhc_sync(sl.sub, sl.stream);   // the stream is idle; reads the device error word
      float a = 0.f, b = 0.f;
      if (cudaEventElapsedTime(&a, s->epoch, jb->ev0) == cudaSuccess &&
          cudaEventElapsedTime(&b, s->epoch, jb->ev) == cudaSuccess) {
        jb->d_start = a;
        jb->d_done = b;
      } else {
        cudaGetLastError();
      }
      jb->status = st;
      if (st != LHC_OK) jb->msg = lhc_last_error();
      jb->state = st == LHC_OK ? LHC_JOB_DONE : LHC_JOB_FAILED;
      jb->t_done = now_s();
      sl.job = nullptr;
      s->done_cv.notify_all();
    }
    // admissions: first queued job that fits a free slot within the budget
    for (auto &sl : s->slots) {
      if (sl.job || s->queue.empty()) continue;
      Job *pick = nullptr;
      for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        Job *jb = *it;
        size_t extra = jb->need > sl.reserved ? jb->need - sl.reserved : 0;
        if (!s->budget || in_use(s) + extra <= s->budget) {
          pick = jb;
          s->queue.erase(it);
          break;
        }
      }
      if (!pick) {
        // release the workspaces of idle slots and try again on the next pass
        for (auto &o : s->slots)
          if (!o.job && o.reserved) {
            lhc_release_workspace(o.sub);
            o.reserved = 0;
          }
        break;
      }
      sl.reserved = std::max(sl.reserved, pick->need);
      sl.job = pick;
      pick->slot = (int)(&sl - s->slots.data());
      pick->state = LHC_JOB_RUNNING;
      pick->t_start = now_s();
      lk.unlock();
      int st = launch_job(s, sl, pick);
      lk.lock();
      if (st != LHC_OK) {
        pick->status = st;
        pick->msg = lhc_last_error();
        pick->state = LHC_JOB_FAILED;
        pick->t_done = now_s();
        sl.job = nullptr;
        s->done_cv.notify_all();
      }
    }
    bool busy = false;
    for (auto &sl : s->slots) busy |= sl.job != nullptr;
    s->cv.wait_for(lk, std::chrono::microseconds(busy ? 20 : 2000));
  }
}

}  // namespace

extern "C" {

int lhc_serve_start(lhc_ctx ctx, int slots) {
  if (!ctx || slots < 1 || slots > 64) {
    lhc::set_error("lhc_serve_start: bad arguments");
    return LHC_EINVAL;
  }
  std::lock_guard<std::mutex> g(g_servers_mu);
  if (g_servers.count(ctx)) return LHC_OK;
  auto *s = new lhc_server_s();
  s->ctx = ctx;
  s->budget = ctx->budget;
  LHC_CHECK_CUDA(cudaSetDevice(ctx->device));
  s->slots.resize(slots);
  for (auto &sl : s->slots) {
    int st = lhc_create(&sl.sub, ctx->device, 0);
    if (st != LHC_OK) return st;
    lhc_set_gamma5(sl.sub, ctx->g5);
    LHC_CHECK_CUDA(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
  }
  LHC_CHECK_CUDA(cudaEventCreate(&s->epoch));
  LHC_CHECK_CUDA(cudaEventRecord(s->epoch, s->slots[0].stream));
  LHC_CHECK_CUDA(cudaEventSynchronize(s->epoch));
  g_servers[ctx] = s;
  s->worker = std::thread(worker_main, s);
  return LHC_OK;
}

int lhc_serve_stop(lhc_ctx ctx) {
  lhc_server_s *s;
  {
    std::lock_guard<std::mutex> g(g_servers_mu);
    auto it = g_servers.find(ctx);
    if (it == g_servers.end()) return LHC_OK;
    s = it->second;
    g_servers.erase(it);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  s->worker.join();
  for (auto &sl : s->slots) {
    cudaStreamSynchronize(sl.stream);
    cudaStreamDestroy(sl.stream);
    lhc_destroy(sl.sub);
  }
  for (auto &kv : s->jobs) {
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    if (kv.second->ev0) cudaEventDestroy(kv.second->ev0);
    delete kv.second;
  }
  if (s->epoch) cudaEventDestroy(s->epoch);
  delete s;
  return LHC_OK;
}

int lhc_prop_register(lhc_ctx ctx, const void *dev_ptr, const lhc_lattice *lat, uint64_t *handle) {
  lhc_server_s *s = server_of(ctx);
  if (!s) {
    lhc::set_error("lhc_prop_register: call lhc_serve_start first");
    return LHC_EINVAL;
  }
  if (!dev_ptr || !lat || !handle || lat->L < 1 || lat->T < 1 || (lat->dtype != LHC_C128 && lat->dtype != LHC_C64) ||
      ((uintptr_t)dev_ptr & 15)) {
    lhc::set_error("lhc_prop_register: bad arguments (NULL, bad lattice, or not 16-byte aligned)");
    return LHC_EINVAL;
  }
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, dev_ptr) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    lhc::set_error("lhc_prop_register: the propagator must be resident device memory");
    return LHC_EINVAL;
  }
  size_t bytes = (size_t)lat->T * lat->L * lat->L * lat->L * 144 * esize(lat->dtype);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->budget && in_use(s) + bytes > s->budget) {
    lhc::set_error("registering %zu bytes of propagator exceeds the HBM budget", bytes);
    return LHC_EBUDGET;
  }
  *handle = s->next_prop++;
  s->props[*handle] = Prop{dev_ptr, *lat, bytes};
  s->prop_bytes += bytes;
  return LHC_OK;
}

int lhc_prop_release(lhc_ctx ctx, uint64_t handle) {
  lhc_server_s *s = server_of(ctx);
  if (!s) return LHC_ENOTFOUND;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->props.find(handle);
  if (it == s->props.end()) return LHC_ENOTFOUND;
  for (auto &kv : s->jobs) {
    Job *j = kv.second;
    if ((j->state == LHC_JOB_QUEUED || j->state == LHC_JOB_RUNNING) &&
        (j->spec.prop == handle || j->spec.prop_b == handle)) {
      lhc::set_error("propagator %llu is used by an unfinished job", (unsigned long long)handle);
      return LHC_EBUSY;
    }
  }
  s->prop_bytes -= it->second.bytes;
  s->props.erase(it);
  return LHC_OK;
}

int lhc_submit(lhc_ctx ctx, const lhc_job *job, uint64_t *job_id) {
  lhc_server_s *s = server_of(ctx);
  if (!s) {
    lhc::set_error("lhc_submit: call lhc_serve_start first");
    return LHC_EINVAL;
  }
  if (!job || !job_id || job->type < LHC_JOB_INSERTION || job->type > LHC_JOB_THREEPT || job->n_r < 1 ||
      job->nq < 1 || !job->k || (job->prec != LHC_FP64 && job->prec != LHC_MIXED) ||
      (((uintptr_t)job->psi | (uintptr_t)job->eta | (uintptr_t)job->out_ins | (uintptr_t)job->out_spec) & 15)) {
    lhc::set_error("lhc_submit: bad job description (sizes, precision, or a buffer not 16-byte aligned)");
    return LHC_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto pit = s->props.find(job->prop);
  if (pit == s->props.end() || (job->kind == LHC_BARYON && job->type != LHC_JOB_INSERTION &&
                                !s->props.count(job->prop_b))) {
    lhc::set_error("lhc_submit: unknown propagator handle");
    return LHC_ENOTFOUND;
  }
  const lhc_lattice &lat = pit->second.lat;
  if (job->type != LHC_JOB_SPECTATOR &&
      (!job->psi || !job->out_ins || job->t_hi < job->t_lo || job->t_hi - job->t_lo >= lat.T)) {
    lhc::set_error("lhc_submit: bad insertion part");
    return LHC_EINVAL;
  }
  if (job->type != LHC_JOB_INSERTION && (!job->eta || !job->out_spec)) {
    lhc::set_error("lhc_submit: bad spectator part");
    return LHC_EINVAL;
  }
  auto *jb = new Job();
  jb->spec = *job;
  jb->k.assign(job->k, job->k + 3 * job->nq);
  jb->spec.k = nullptr;
  jb->need = job_need(*job, pit->second);
  if (s->budget && s->prop_bytes + jb->need > s->budget) {
    delete jb;
    lhc::set_error("job needs %zu bytes of workspace; with %zu bytes of resident propagators it can never fit "
                   "the %zu-byte HBM budget",
                   job_need(*job, pit->second), s->prop_bytes, s->budget);
    return LHC_EBUDGET;
  }
  if (cudaEventCreate(&jb->ev0) != cudaSuccess || cudaEventCreate(&jb->ev) != cudaSuccess) {
    cudaGetLastError();
    if (jb->ev0) cudaEventDestroy(jb->ev0);
    delete jb;
    lhc::set_error("cannot create the job's timing events");
    return LHC_ECUDA;
  }
  jb->id = s->next_id++;
  jb->t_submit = now_s();
  s->jobs[jb->id] = jb;
  s->queue.push_back(jb);
  *job_id = jb->id;
  lk.unlock();
  s->cv.notify_all();
  return LHC_OK;
}

int lhc_poll(lhc_ctx ctx, uint64_t job_id, int *state) {
  lhc_server_s *s = server_of(ctx);
  if (!s) return LHC_ENOTFOUND;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return LHC_ENOTFOUND;
  if (state) *state = it->second->state;
  int st = it->second->state;
  return (st == LHC_JOB_QUEUED || st == LHC_JOB_RUNNING) ? LHC_EBUSY : LHC_OK;
}

int lhc_wait(lhc_ctx ctx, uint64_t job_id, int timeout_ms) {
  lhc_server_s *s = server_of(ctx);
  if (!s) return LHC_ENOTFOUND;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return LHC_ENOTFOUND;
  Job *jb = it->second;
  auto finished = [&] { return jb->state != LHC_JOB_QUEUED && jb->state != LHC_JOB_RUNNING; };
  if (!s->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), finished)) {
    lhc::set_error("job %llu not finished after %d ms", (unsigned long long)job_id, timeout_ms);
    return LHC_ETIMEOUT;
  }
  if (jb->state == LHC_JOB_CANCELED) return LHC_ECANCELED;
  if (jb->status != LHC_OK)
    lhc::set_error("job %llu failed: %s", (unsigned long long)job_id, jb->msg.c_str());
  return jb->status;
}

int lhc_cancel(lhc_ctx ctx, uint64_t job_id) {
  lhc_server_s *s = server_of(ctx);
  if (!s) return LHC_ENOTFOUND;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return LHC_ENOTFOUND;
  Job *jb = it->second;
  if (jb->state != LHC_JOB_QUEUED) {
    lhc::set_error("job %llu is no longer queued", (unsigned long long)job_id);
    return LHC_EBUSY;
  }
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
    if (*q == jb) {
      s->queue.erase(q);
      break;
    }
  jb->state = LHC_JOB_CANCELED;
  jb->status = LHC_ECANCELED;
  jb->t_done = now_s();
  s->done_cv.notify_all();
  return LHC_OK;
}

int lhc_job_times(lhc_ctx ctx, uint64_t job_id, double *t_submit, double *t_start, double *t_done) {
  lhc_server_s *s = server_of(ctx);
  if (!s) return LHC_ENOTFOUND;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return LHC_ENOTFOUND;
  if (t_submit) *t_submit = it->second->t_submit;
  if (t_start) *t_start = it->second->t_start;
  if (t_done) *t_done = it->second->t_done;
  return LHC_OK;
}

int lhc_job_device_times(lhc_ctx ctx, uint64_t job_id, double *ms_start, double *ms_done) {
  lhc_server_s *s = server_of(ctx);
  if (!s) return LHC_ENOTFOUND;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return LHC_ENOTFOUND;
  const Job *jb = it->second;
  if (jb->state != LHC_JOB_DONE) {
    lhc::set_error("job %llu has no device times (not finished, or not run)", (unsigned long long)job_id);
    return LHC_EBUSY;
  }
  if (ms_start) *ms_start = jb->d_start;
  if (ms_done) *ms_done = jb->d_done;
  return LHC_OK;
}

int lhc_serve_stats(lhc_ctx ctx, size_t *bytes_in_use, int *queued, int *running) {
  lhc_server_s *s = server_of(ctx);
  if (!s) return LHC_ENOTFOUND;
  std::lock_guard<std::mutex> lk(s->mu);
  if (bytes_in_use) *bytes_in_use = in_use(s);
  if (queued) *queued = (int)s->queue.size();
  if (running) {
    int n = 0;
    for (auto &sl : s->slots) n += sl.job != nullptr;
    *running = n;
  }
  return LHC_OK;
}

}  // extern "C"
