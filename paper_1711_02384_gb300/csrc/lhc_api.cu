// C ABI of liblhc: argument checks, memory, host staging, phase-table cache and
// dispatch to the kernels.  Every entry point returns an lhc_status.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>

#include "lhc_internal.h"

namespace lhc {

std::atomic<unsigned long long> g_launches{0};

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

static int fail(int status, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return status;
}

bool PhaseKey::operator<(const PhaseKey &o) const {
  if (L != o.L) return L < o.L;
  if (nq != o.nq) return nq < o.nq;
  if (sign != o.sign) return sign < o.sign;
  if (fmt != o.fmt) return fmt < o.fmt;
  if (rx != o.rx) return rx < o.rx;
  if (ry != o.ry) return ry < o.ry;
  if (rz != o.rz) return rz < o.rz;
  return khash < o.khash;
}

uint64_t hash_k(const int *k, int nq) {
  uint64_t h = 1469598103934665603ull;   // FNV-1a over the integers
  for (int j = 0; j < 3 * nq; ++j) {
    uint32_t v = (uint32_t)k[j];
    for (int b = 0; b < 4; ++b) {
      h ^= (v >> (8 * b)) & 0xffu;
      h *= 1099511628211ull;
    }
  }
  return h;
}

int g5mask_of(const lhc_ctx ctx) {
  int m = 0;
  for (int s = 0; s < 4; ++s)
    if (ctx->g5[s] < 0) m |= 1 << s;
  return m;
}

// Frees the least recently used phase table that the current call has not taken; false
// when there is none.  Only earlier calls of this context can still read the table, and
// the current call's stream is ordered after all of them, so synchronizing that stream
// suffices: other contexts (the job server's slots) keep running.
static bool evict_one_phase(lhc_ctx ctx) {
  for (auto k = ctx->phase_lru.rbegin(); k != ctx->phase_lru.rend(); ++k) {
    auto it = ctx->phases.find(*k);
    if (it != ctx->phases.end() && it->second.used_in == ctx->call_seq) continue;
    if (it != ctx->phases.end()) {
      cudaStreamSynchronize(ctx->cur_stream);
      dev_free(ctx, it->second.buf);
      ctx->phases.erase(it);
    }
    ctx->phase_lru.erase(std::next(k).base());
    return true;
  }
  return false;
}

const PhaseEntry *phase_take(lhc_ctx ctx, const PhaseKey &key) {
  auto it = ctx->phases.find(key);
  if (it == ctx->phases.end()) return nullptr;
  ctx->phase_lru.remove(key);
  ctx->phase_lru.push_front(key);
  it->second.used_in = ctx->call_seq;
  return &it->second;
}

void phase_insert(lhc_ctx ctx, const PhaseKey &key, const PhaseEntry &e) {
  PhaseEntry &d = ctx->phases[key];
  d = e;
  d.used_in = ctx->call_seq;
  ctx->phase_lru.push_front(key);
}

int dev_alloc(lhc_ctx ctx, DevBuf &b, size_t bytes) {
  b = DevBuf{};
  if (bytes == 0) return LHC_OK;
  while (ctx->budget && ctx->used + bytes > ctx->budget && evict_one_phase(ctx)) {
  }
  if (ctx->budget && ctx->used + bytes > ctx->budget)
    return fail(LHC_EBUDGET, "allocation of %zu bytes exceeds the HBM budget (%zu of %zu in use)",
                bytes, ctx->used, ctx->budget);
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(LHC_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  b.bytes = bytes;
  ctx->used += bytes;
  return LHC_OK;
}

void dev_free(lhc_ctx ctx, DevBuf &b) {
  if (b.p) {
    cudaFree(b.p);
    ctx->used -= b.bytes;
  }
  b = DevBuf{};
}

int ensure(lhc_ctx ctx, DevBuf &b, size_t bytes) {
  if (b.bytes >= bytes) return LHC_OK;
  // nothing in flight may still use the old buffer: this context's work is ordered on the
  // current call's stream (see begin_call), so that stream, not the device, is waited for
  LHC_CHECK_CUDA(cudaStreamSynchronize(ctx->cur_stream));
  dev_free(ctx, b);
  return dev_alloc(ctx, b, bytes + bytes / 4);
}

int get_phase_f64(lhc_ctx ctx, int L, const int *k, int nq, const int r[4], int sign,
                  cudaStream_t st, const double2 **out) {
  PhaseKey key{L, nq, sign, 0, ((r[0] % L) + L) % L, ((r[1] % L) + L) % L, ((r[2] % L) + L) % L,
                hash_k(k, nq)};
  if (const PhaseEntry *hit = phase_take(ctx, key)) {
    *out = static_cast<const double2 *>(hit->buf.p);
    return LHC_OK;
  }
  size_t V3 = (size_t)L * L * L;
  size_t tbytes = (size_t)nq * V3 * sizeof(double2);
  size_t kbytes = (size_t)3 * nq * sizeof(int);
  size_t off_roots = (tbytes + kbytes + 255) & ~(size_t)255;
  size_t off_k = tbytes;
  PhaseEntry e;
  LHC_TRY(dev_alloc(ctx, e.buf, off_roots + (size_t)L * sizeof(double2)));
  std::vector<double2> roots(L);
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < L; ++m) roots[m] = make_double2(std::cos(two_pi * m / L), std::sin(two_pi * m / L));
  char *base = static_cast<char *>(e.buf.p);
  // synchronous copies: the host vectors go out of scope at return
  LHC_CHECK_CUDA(cudaMemcpy(base + off_k, k, kbytes, cudaMemcpyHostToDevice));
  LHC_CHECK_CUDA(cudaMemcpy(base + off_roots, roots.data(), (size_t)L * sizeof(double2),
                            cudaMemcpyHostToDevice));
  launch_phase_f64(reinterpret_cast<double2 *>(base), reinterpret_cast<const int *>(base + off_k), nq,
                   L, key.rx, key.ry, key.rz, sign, reinterpret_cast<const double2 *>(base + off_roots),
                   st);
  LHC_CHECK_CUDA(cudaGetLastError());
  phase_insert(ctx, key, e);
  *out = reinterpret_cast<const double2 *>(base);
  return LHC_OK;
}

ProfScope::ProfScope(lhc_ctx c, cudaStream_t s, int k, double w) : ctx(c), st(s), kernel(k), work(w) {
  if (!ctx->prof_on) return;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    a = b = nullptr;
    return;
  }
  cudaEventRecord(a, st);
}

ProfScope::~ProfScope() {
  if (!a) return;
  cudaEventRecord(b, st);
  ctx->prof.push_back(ProfRecord{kernel, a, b, work});
}

}  // namespace lhc

using namespace lhc;

namespace {

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t esize(int dtype) { return dtype == LHC_C128 ? 16 : 8; }

int check_lattice(const lhc_lattice *lat) {
  if (!lat) return fail(LHC_EINVAL, "lattice is NULL");
  if (lat->L < 1 || lat->L > 128 || lat->T < 1 || lat->T > 4096)
    return fail(LHC_EINVAL, "lattice extent out of range (L=%d, T=%d)", lat->L, lat->T);
  if (lat->dtype != LHC_C128 && lat->dtype != LHC_C64)
    return fail(LHC_EINVAL, "unknown dtype %d", lat->dtype);
  return LHC_OK;
}

}  // namespace

// per-context event ordering the shared workspace between streams
struct CtxSync {
  cudaEvent_t ev = nullptr;
  cudaStream_t last = nullptr;
  bool used = false;
};
static std::map<lhc_ctx, CtxSync> g_sync;
static std::mutex g_sync_mu;

// ---------------------------------------------------------------- host staging
// A call with host buffers takes the next of kStageSlots staging slots.  Its input
// copies run on the context's H2D stream once the slot is free (the call kStageSlots
// back has finished with it) and any output copy in flight into the same host memory has
// landed; the caller's stream waits for them, runs the kernels, and the D2H stream
// copies the output back, which the caller's stream waits for in turn.  So the copies of
// one call overlap the kernels of the ones before, and a stream or device synchronize
// still covers all.  One H2D stream, not one per slot: the calls' copies then land in
// call order at the full link rate, and each call's kernels start as soon as its own
// inputs are in, instead of all calls' inputs arriving together at the end of a shared
// transfer.
static int stage_streams(lhc_ctx ctx) {
  if (ctx->d2h) return LHC_OK;
  LHC_CHECK_CUDA(cudaStreamCreateWithFlags(&ctx->h2d, cudaStreamNonBlocking));
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = ctx->device;
  LHC_CHECK_CUDA(cudaMemPoolCreate(&ctx->stage_pool, &props));
  uint64_t keep = UINT64_MAX;   // freed slot memory stays mapped for the next growth
  LHC_CHECK_CUDA(cudaMemPoolSetAttribute(ctx->stage_pool, cudaMemPoolAttrReleaseThreshold, &keep));
  for (int s = 0; s < lhc_ctx_s::kStageSlots; ++s) {
    LHC_CHECK_CUDA(cudaEventCreateWithFlags(&ctx->slot_free[s], cudaEventDisableTiming));
    LHC_CHECK_CUDA(cudaEventCreateWithFlags(&ctx->in_ready[s], cudaEventDisableTiming));
  }
  LHC_CHECK_CUDA(cudaEventCreateWithFlags(&ctx->comp_done, cudaEventDisableTiming));
  LHC_CHECK_CUDA(cudaStreamCreateWithFlags(&ctx->d2h, cudaStreamNonBlocking));
  return LHC_OK;
}

// Grows every staging slot to `bytes` plus a quarter, in stream order on the H2D stream:
// the stream first waits for each slot's last call, then the old buffers go back with
// cudaFreeAsync and the new ones come from the context's pool with
// cudaMallocFromPoolAsync.  No device synchronization (cudaFree would be one), and since
// all slots grow together, calls of different sizes rotating over the slots grow nothing
// once the largest has been seen.
static int stage_grow(lhc_ctx ctx, size_t bytes) {
  if (ctx->stage_bytes >= bytes) return LHC_OK;
  const size_t want = bytes + bytes / 4;
  const size_t held = ctx->stage_bytes * (size_t)lhc_ctx_s::kStageSlots;
  const size_t need = want * (size_t)lhc_ctx_s::kStageSlots;
  while (ctx->budget && ctx->used - held + need > ctx->budget && evict_one_phase(ctx)) {
  }
  if (ctx->budget && ctx->used - held + need > ctx->budget)
    return fail(LHC_EBUDGET, "%d staging slots of %zu bytes exceed the HBM budget (%zu of %zu in use)",
                lhc_ctx_s::kStageSlots, want, ctx->used - held, ctx->budget);
  for (int s = 0; s < lhc_ctx_s::kStageSlots; ++s) {
    DevBuf &b = ctx->stage[s];
    if (ctx->slot_used[s]) LHC_CHECK_CUDA(cudaStreamWaitEvent(ctx->h2d, ctx->slot_free[s], 0));
    if (b.p) {
      LHC_CHECK_CUDA(cudaFreeAsync(b.p, ctx->h2d));
      ctx->used -= b.bytes;
      b = DevBuf{};
    }
    cudaError_t e = cudaMallocFromPoolAsync(&b.p, want, ctx->stage_pool, ctx->h2d);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b = DevBuf{};
      return fail(LHC_ENOMEM, "cudaMallocFromPoolAsync(%zu): %s", want, cudaGetErrorString(e));
    }
    b.bytes = want;
    ctx->used += want;
  }
  ctx->stage_bytes = want;
  return LHC_OK;
}

// Takes a staging slot of at least `bytes`; *base is its device address.
static int stage_begin(lhc_ctx ctx, size_t bytes, int *slot, char **base) {
  LHC_TRY(stage_streams(ctx));
  const int s = ctx->next_slot;
  ctx->next_slot = (s + 1) % lhc_ctx_s::kStageSlots;
  if (ctx->slot_used[s]) LHC_CHECK_CUDA(cudaStreamWaitEvent(ctx->h2d, ctx->slot_free[s], 0));
  LHC_TRY(stage_grow(ctx, bytes));
  *slot = s;
  *base = static_cast<char *>(ctx->stage[s].p);
  return LHC_OK;
}

// The H2D stream waits for any output copy still writing host memory in [a, a + bytes).
static int wait_pending_out(lhc_ctx ctx, const char *a, size_t bytes) {
  for (auto it = ctx->pending_out.begin(); it != ctx->pending_out.end();) {
    if (cudaEventQuery(it->ev) == cudaSuccess) {   // landed: forget it
      ctx->event_pool.push_back(it->ev);
      it = ctx->pending_out.erase(it);
      continue;
    }
    cudaGetLastError();   // cudaErrorNotReady is not an error here
    if (a < it->p + it->n && it->p < a + bytes) LHC_CHECK_CUDA(cudaStreamWaitEvent(ctx->h2d, it->ev, 0));
    ++it;
  }
  return LHC_OK;
}

// Host -> slot copy on the H2D stream, after any output copy still writing that memory.
static int stage_in(lhc_ctx ctx, int slot, void *dst, const void *src, size_t bytes) {
  (void)slot;
  LHC_TRY(wait_pending_out(ctx, static_cast<const char *>(src), bytes));
  LHC_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->h2d));
  return LHC_OK;
}

// The same for `rows` equal pieces of `width` bytes, `spitch` apart in host memory and
// `dpitch` apart in the slot: one strided copy instead of one copy per piece (the noises
// of a solution tensor), so the link does not idle between many medium copies.
static int stage_in_rows(lhc_ctx ctx, int slot, void *dst, size_t dpitch, const void *src, size_t spitch,
                         size_t width, size_t rows) {
  if (rows == 0) return LHC_OK;
  int max_pitch = 0;
  LHC_CHECK_CUDA(cudaDeviceGetAttribute(&max_pitch, cudaDevAttrMaxPitch, ctx->device));
  if (spitch > (size_t)max_pitch || dpitch > (size_t)max_pitch) {   // beyond a strided copy's pitch: one per piece
    for (size_t r = 0; r < rows; ++r)
      LHC_TRY(stage_in(ctx, slot, static_cast<char *>(dst) + r * dpitch, static_cast<const char *>(src) + r * spitch,
                       width));
    return LHC_OK;
  }
  LHC_TRY(wait_pending_out(ctx, static_cast<const char *>(src), (rows - 1) * spitch + width));
  LHC_CHECK_CUDA(cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, cudaMemcpyHostToDevice, ctx->h2d));
  return LHC_OK;
}

// The kernels on `st` may start once the inputs have landed.
static int stage_ready(lhc_ctx ctx, int slot, cudaStream_t st) {
  LHC_CHECK_CUDA(cudaEventRecord(ctx->in_ready[slot], ctx->h2d));
  LHC_CHECK_CUDA(cudaStreamWaitEvent(st, ctx->in_ready[slot], 0));
  return LHC_OK;
}

// After the kernels: copy the output back (if it is host memory) and release the slot.
static int stage_end(lhc_ctx ctx, int slot, cudaStream_t st, void *host_out, const void *dev_out, size_t bytes) {
  if (host_out) {
    LHC_CHECK_CUDA(cudaEventRecord(ctx->comp_done, st));
    LHC_CHECK_CUDA(cudaStreamWaitEvent(ctx->d2h, ctx->comp_done, 0));
    LHC_CHECK_CUDA(cudaMemcpyAsync(host_out, dev_out, bytes, cudaMemcpyDeviceToHost, ctx->d2h));
    LHC_CHECK_CUDA(cudaEventRecord(ctx->slot_free[slot], ctx->d2h));
    LHC_CHECK_CUDA(cudaStreamWaitEvent(st, ctx->slot_free[slot], 0));   // the caller's stream covers the copy
    cudaEvent_t ev;
    if (ctx->event_pool.empty()) {
      LHC_CHECK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    } else {
      ev = ctx->event_pool.back();
      ctx->event_pool.pop_back();
    }
    LHC_CHECK_CUDA(cudaEventRecord(ev, ctx->d2h));
    ctx->pending_out.push_back({static_cast<const char *>(host_out), bytes, ev});
  } else {
    LHC_CHECK_CUDA(cudaEventRecord(ctx->slot_free[slot], st));
  }
  ctx->slot_used[slot] = true;
  return LHC_OK;
}

static void stage_release(lhc_ctx ctx) {   // the device is synchronized
  for (int s = 0; s < lhc_ctx_s::kStageSlots; ++s) {
    DevBuf &b = ctx->stage[s];
    if (b.p) {
      cudaFreeAsync(b.p, ctx->h2d);   // pool memory, returned in the H2D stream's order
      ctx->used -= b.bytes;
    }
    b = DevBuf{};
  }
  ctx->stage_bytes = 0;
  if (ctx->h2d) cudaStreamSynchronize(ctx->h2d);
  if (ctx->stage_pool) cudaMemPoolTrimTo(ctx->stage_pool, 0);
}

static void stage_destroy(lhc_ctx ctx) {
  stage_release(ctx);
  for (auto &po : ctx->pending_out) cudaEventDestroy(po.ev);
  for (auto ev : ctx->event_pool) cudaEventDestroy(ev);
  ctx->pending_out.clear();
  ctx->event_pool.clear();
  if (ctx->d2h) {
    cudaStreamDestroy(ctx->h2d);
    ctx->h2d = nullptr;
    for (int s = 0; s < lhc_ctx_s::kStageSlots; ++s) {
      cudaEventDestroy(ctx->slot_free[s]);
      cudaEventDestroy(ctx->in_ready[s]);
    }
    cudaStreamDestroy(ctx->d2h);
    cudaEventDestroy(ctx->comp_done);
    ctx->d2h = nullptr;
  }
  if (ctx->stage_pool) {
    cudaMemPoolDestroy(ctx->stage_pool);
    ctx->stage_pool = nullptr;
  }
}

static int begin_call(lhc_ctx ctx, cudaStream_t st) {
  LHC_CHECK_CUDA(cudaSetDevice(ctx->device));
  std::lock_guard<std::mutex> g(g_sync_mu);
  ++ctx->call_seq;   // the caller holds ctx->mu
  ctx->cur_stream = st;
  CtxSync &s = g_sync[ctx];
  if (!s.ev) LHC_CHECK_CUDA(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
  if (s.used && s.last != st) LHC_CHECK_CUDA(cudaStreamWaitEvent(st, s.ev, 0));
  return LHC_OK;
}

static int end_call(lhc_ctx ctx, cudaStream_t st) {
  std::lock_guard<std::mutex> g(g_sync_mu);
  CtxSync &s = g_sync[ctx];
  LHC_CHECK_CUDA(cudaEventRecord(s.ev, st));
  s.last = st;
  s.used = true;
  return LHC_OK;
}

extern "C" {

const char *lhc_strerror(int status) {
  switch (status) {
    case LHC_OK: return "success";
    case LHC_EINVAL: return "invalid argument";
    case LHC_ENOMEM: return "out of device memory";
    case LHC_EBUDGET: return "request exceeds the HBM budget";
    case LHC_ETIMEOUT: return "timed out";
    case LHC_ECUDA: return "CUDA error";
    case LHC_EBUSY: return "busy";
    case LHC_ENOTFOUND: return "not found";
    case LHC_ECANCELED: return "canceled";
    default: return "unknown status";
  }
}

const char *lhc_last_error(void) { return g_err; }

int lhc_version(void) { return 100; }

unsigned long long lhc_launch_count(void) { return lhc::g_launches.load(std::memory_order_relaxed); }

int lhc_create(lhc_ctx *out, int device, size_t hbm_budget_bytes) {
  if (!out) return fail(LHC_EINVAL, "ctx pointer is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(LHC_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
  if (device < 0 || device >= n) return fail(LHC_EINVAL, "device %d out of range (%d devices)", device, n);
  LHC_CHECK_CUDA(cudaSetDevice(device));
  cudaDeviceProp prop;
  LHC_CHECK_CUDA(cudaGetDeviceProperties(&prop, device));
  if (prop.major * 10 + prop.minor < 100)
    return fail(LHC_ECUDA, "device %d is sm_%d%d; this library is built for sm_103a", device, prop.major,
                prop.minor);
  lhc_ctx c = new lhc_ctx_s();
  c->device = device;
  c->budget = hbm_budget_bytes;
  c->num_sms = prop.multiProcessorCount;
  if (cudaMalloc(&c->dev_err, 256) != cudaSuccess || cudaMemset(c->dev_err, 0, 256) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return fail(LHC_ENOMEM, "cannot allocate the device error word");
  }
  *out = c;
  return LHC_OK;
}

int lhc_destroy(lhc_ctx ctx) {
  if (!ctx) return fail(LHC_EINVAL, "ctx is NULL");
  lhc_serve_stop(ctx);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  release_staged(ctx);
  dev_free(ctx, ctx->ws);
  stage_destroy(ctx);
  if (ctx->dev_err) cudaFree(ctx->dev_err);
  for (auto &kv : ctx->phases) dev_free(ctx, kv.second.buf);
  for (auto &r : ctx->prof) {
    cudaEventDestroy(r.start);
    cudaEventDestroy(r.stop);
  }
  {
    std::lock_guard<std::mutex> g(g_sync_mu);
    auto it = g_sync.find(ctx);
    if (it != g_sync.end()) {
      if (it->second.ev) cudaEventDestroy(it->second.ev);
      g_sync.erase(it);
    }
  }
  delete ctx;
  return LHC_OK;
}

int lhc_release_workspace(lhc_ctx ctx) {
  if (!ctx) return fail(LHC_EINVAL, "ctx is NULL");
  std::lock_guard<std::mutex> g(ctx->mu);
  LHC_CHECK_CUDA(cudaSetDevice(ctx->device));
  LHC_CHECK_CUDA(cudaDeviceSynchronize());
  dev_free(ctx, ctx->ws);
  stage_release(ctx);
  for (auto &kv : ctx->phases) dev_free(ctx, kv.second.buf);
  ctx->phases.clear();
  ctx->phase_lru.clear();
  return LHC_OK;
}

int lhc_sync(lhc_ctx ctx, void *stream) {
  if (!ctx) return fail(LHC_EINVAL, "ctx is NULL");
  LHC_CHECK_CUDA(cudaSetDevice(ctx->device));
  LHC_CHECK_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int code = 0;
  LHC_CHECK_CUDA(cudaMemcpy(&code, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (code) {
    LHC_CHECK_CUDA(cudaMemset(ctx->dev_err, 0, sizeof(int)));
    return fail(LHC_ETIMEOUT, "a bounded device wait gave up (site %d); results of the affected calls are invalid",
                code);
  }
  return LHC_OK;
}

int lhc_set_gamma5(lhc_ctx ctx, const int g5[4]) {
  if (!ctx || !g5) return fail(LHC_EINVAL, "NULL argument");
  for (int s = 0; s < 4; ++s)
    if (g5[s] != 1 && g5[s] != -1) return fail(LHC_EINVAL, "gamma5 diagonal entries must be +1 or -1");
  std::lock_guard<std::mutex> g(ctx->mu);
  for (int s = 0; s < 4; ++s) ctx->g5[s] = g5[s];
  return LHC_OK;
}

int lhc_profile(lhc_ctx ctx, int enable) {
  if (!ctx) return fail(LHC_EINVAL, "ctx is NULL");
  std::lock_guard<std::mutex> g(ctx->mu);
  if (enable) {
    for (auto &r : ctx->prof) {
      cudaEventSynchronize(r.stop);
      cudaEventDestroy(r.start);
      cudaEventDestroy(r.stop);
    }
    ctx->prof.clear();
  }
  ctx->prof_on = enable != 0;
  return LHC_OK;
}

int lhc_profile_read(lhc_ctx ctx, int kernel, double *total_ms, long long *launches, double *work) {
  if (!ctx || !total_ms || !launches || !work) return fail(LHC_EINVAL, "NULL argument");
  if (kernel < 0 || kernel >= LHC_KERNEL_COUNT) return fail(LHC_EINVAL, "unknown kernel id %d", kernel);
  std::lock_guard<std::mutex> g(ctx->mu);
  double ms = 0, w = 0;
  long long n = 0;
  for (auto &r : ctx->prof) {
    if (r.kernel != kernel) continue;
    LHC_CHECK_CUDA(cudaEventSynchronize(r.stop));
    float e = 0;
    LHC_CHECK_CUDA(cudaEventElapsedTime(&e, r.start, r.stop));
    ms += e;
    w += r.work;
    ++n;
  }
  *total_ms = ms;
  *launches = n;
  *work = w;
  return LHC_OK;
}

int lhc_momenta(int n2max, int cmax, int *k, int cap, int *nq) {
  if (n2max < 0 || !nq || cap < 0 || (cap > 0 && !k)) return fail(LHC_EINVAL, "bad momentum arguments");
  int c = cmax >= 0 ? cmax : (int)std::floor(std::sqrt((double)n2max) + 1e-9);
  struct K { int n2, x, y, z; };
  std::vector<K> v;
  for (int x = -c; x <= c; ++x)
    for (int y = -c; y <= c; ++y)
      for (int z = -c; z <= c; ++z) {
        int n2 = x * x + y * y + z * z;
        if (n2 <= n2max) v.push_back({n2, x, y, z});
      }
  std::sort(v.begin(), v.end(), [](const K &a, const K &b) {
    if (a.n2 != b.n2) return a.n2 < b.n2;
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    return a.z < b.z;
  });
  *nq = (int)v.size();
  for (int j = 0; j < (int)v.size() && j < cap; ++j) {
    k[3 * j] = v[j].x;
    k[3 * j + 1] = v[j].y;
    k[3 * j + 2] = v[j].z;
  }
  return LHC_OK;
}

}  // extern "C"

namespace {

// Common driver of the insertion and spectator calls.
struct PartCall {
  Part part;
  const lhc_lattice *lat;
  const void *S, *SB, *vec;
  int n_r;
  int t0, nt;          // slices t0 .. t0+nt-1 (mod T)
  bool vec_has_time;   // psi carries a time axis, eta does not
  const int *r, *k;
  int nq, prec;
  void *out;
  int sign;
};

int run_part(lhc_ctx ctx, const PartCall &c, cudaStream_t st) {
  const int L = c.lat->L, T = c.lat->T, V3 = L * L * L;
  const size_t es = esize(c.lat->dtype);
  const int cols = (c.part == PART_SPEC_BARYON ? kBarCols : 192);
  const size_t slice_elems = (size_t)V3 * 144;
  const size_t vec_slice = (size_t)V3 * 12;
  const size_t out_bytes = (size_t)c.nt * c.nq * c.n_r * cols * sizeof(double2);

  bool hS = !is_device_ptr(c.S), hSB = c.SB && !is_device_ptr(c.SB), hV = !is_device_ptr(c.vec);
  bool hO = !is_device_ptr(c.out);
  bool any_host = hS || hSB || hV || hO;

  // staging layout: [S slices][SB slices][vec][out]
  size_t bS = hS ? c.nt * slice_elems * es : 0;
  size_t bSB = hSB ? c.nt * slice_elems * es : 0;
  size_t nvt = c.vec_has_time ? c.nt : 1;
  size_t bV = hV ? (size_t)c.n_r * nvt * vec_slice * es : 0;
  size_t bO = hO ? out_bytes : 0;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  int slot = -1;
  char *sp = nullptr;
  if (any_host) LHC_TRY(stage_begin(ctx, al(bS) + al(bSB) + al(bV) + al(bO), &slot, &sp));
  const char *S = static_cast<const char *>(c.S), *SB = static_cast<const char *>(c.SB),
             *V = static_cast<const char *>(c.vec);
  size_t S_tstride = slice_elems * es;   // bytes between slices
  // runs of consecutive t among the call's slices j0 .. j1-1 (t = t0 + j mod T): one copy
  // per run
  auto runs_of = [&](int j0, int j1) {
    std::vector<std::pair<int, int>> runs;   // (first j, length)
    for (int j = j0; j < j1;) {
      const int t = (c.t0 + j) % T, len = std::min(j1 - j, T - t);
      runs.emplace_back(j, len);
      j += len;
    }
    return runs;
  };
  const char *Sd = hS ? sp : S;
  const char *SBd = hSB ? sp + al(bS) : SB;
  // vec layout on device: noise stride and slice base
  const char *Vd = hV ? sp + al(bS) + al(bSB) : V;
  const size_t v_noise_stride = hV ? nvt * vec_slice : (c.vec_has_time ? (size_t)T * vec_slice : vec_slice);
  double2 *Od = hO ? reinterpret_cast<double2 *>(sp + al(bS) + al(bSB) + al(bV))
                   : static_cast<double2 *>(c.out);

  const bool dft = use_fft(ctx, c.prec, V3, c.nq);   // all-momenta mode: the projection as a DFT
  const double2 *phase = nullptr;
  if (c.prec == LHC_FP64 && !dft) LHC_TRY(get_phase_f64(ctx, L, c.k, c.nq, c.r, c.sign, st, &phase));

  std::vector<SliceJob> jobs(c.nt);
  for (int j = 0; j < c.nt; ++j) {
    int t = (c.t0 + j) % T;
    SliceJob &job = jobs[j];
    job.part = c.part;
    job.dtype = c.lat->dtype;
    job.L = L;
    job.V3 = V3;
    job.n_r = c.n_r;
    job.nq = c.nq;
    job.S = Sd + (hS ? (size_t)j : (size_t)t) * S_tstride;
    job.SB = c.SB ? SBd + (hSB ? (size_t)j : (size_t)t) * S_tstride : nullptr;
    size_t vt = c.vec_has_time ? (hV ? (size_t)j : (size_t)t) : 0;
    job.vec = Vd + vt * vec_slice * es;
    job.vec_stride = v_noise_stride;
    job.g5mask = g5mask_of(ctx);
    job.out = Od + (size_t)j * c.nq * c.n_r * cols;
  }
  // With host inputs the slices go in up to four groups: each group's copies are followed
  // by its kernels, which start as soon as that group has landed, so a call's own
  // transfer overlaps its kernels (one group per call would leave all of them after it).
  const bool host_in = hS || hSB || hV;
  const int ngroups = host_in ? std::min(c.nt, 4) : 1;
  const int gsz = (c.nt + ngroups - 1) / ngroups;
  for (int g0 = 0; g0 < c.nt; g0 += gsz) {
    const int g1 = std::min(c.nt, g0 + gsz);
    const auto runs = runs_of(g0, g1);
    for (const auto &rn : runs) {   // the group's slices of S (and SB), as [nt][V3][144]
      const size_t t = (size_t)((c.t0 + rn.first) % T), n = (size_t)rn.second * S_tstride;
      if (hS) LHC_TRY(stage_in(ctx, slot, sp + rn.first * S_tstride, S + t * S_tstride, n));
      if (hSB) LHC_TRY(stage_in(ctx, slot, sp + al(bS) + rn.first * S_tstride, SB + t * S_tstride, n));
    }
    if (hV) {
      char *dst = sp + al(bS) + al(bSB);
      if (!c.vec_has_time) {   // eta: [n_r][V3][12], one block (a spectator call has one slice)
        if (g0 == 0) LHC_TRY(stage_in(ctx, slot, dst, V, (size_t)c.n_r * vec_slice * es));
      } else {   // psi: the group's runs of slices, every noise in one strided copy per run
        for (const auto &rn : runs) {
          const size_t t = (size_t)((c.t0 + rn.first) % T);
          LHC_TRY(stage_in_rows(ctx, slot, dst + (size_t)rn.first * vec_slice * es, (size_t)nvt * vec_slice * es,
                                V + t * vec_slice * es, (size_t)T * vec_slice * es,
                                (size_t)rn.second * vec_slice * es, (size_t)c.n_r));
        }
      }
    }
    if (any_host) LHC_TRY(stage_ready(ctx, slot, st));
    if (dft) {
      LHC_TRY(run_part_fft(ctx, jobs.data() + g0, g1 - g0, c.k, c.nq, c.r, c.sign, c.prec, st));
    } else if (c.prec == LHC_MIXED) {
      // the call's launch shape for every group: each slice computed as in one launch
      LHC_TRY(run_part_mixed(ctx, jobs.data() + g0, g1 - g0, c.k, c.nq, c.r, c.sign, st, c.nt));
    } else {
      for (int j = g0; j < g1; ++j) LHC_TRY(run_slice_f64(ctx, jobs[j], phase, st));
    }
  }
  if (any_host) LHC_TRY(stage_end(ctx, slot, st, hO ? c.out : nullptr, Od, out_bytes));
  return LHC_OK;
}

int common_checks(lhc_ctx ctx, const lhc_lattice *lat, const void *S, const void *vec, int n_r,
                  const int r[4], const int *k, int nq, int prec, void *out) {
  if (!ctx) return fail(LHC_EINVAL, "ctx is NULL");
  LHC_TRY(check_lattice(lat));
  if (!S || !vec || !out || !r || !k) return fail(LHC_EINVAL, "NULL buffer argument");
  if (((uintptr_t)S | (uintptr_t)vec | (uintptr_t)out) & 15)
    return fail(LHC_EINVAL, "propagator, vector and output buffers must be 16-byte aligned");
  if (n_r < 1 || n_r > 4096) return fail(LHC_EINVAL, "n_r=%d out of range", n_r);
  if (nq < 1 || nq > 65536) return fail(LHC_EINVAL, "nq=%d out of range", nq);
  if (prec != LHC_FP64 && prec != LHC_MIXED) return fail(LHC_EINVAL, "unknown precision %d", prec);
  return LHC_OK;
}

}  // namespace

extern "C" {

int lhc_insertion(lhc_ctx ctx, const lhc_lattice *lat, const void *S3, const void *psi, int n_r,
                  int t_lo, int t_hi, const int r[4], const int *k, int nq, int prec, void *out,
                  void *stream) {
  LHC_TRY(common_checks(ctx, lat, S3, psi, n_r, r, k, nq, prec, out));
  if (t_hi < t_lo || t_hi - t_lo >= lat->T) return fail(LHC_EINVAL, "bad slice range %d..%d", t_lo, t_hi);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(ctx->mu);
  LHC_TRY(begin_call(ctx, st));
  PartCall c{PART_INS, lat, S3, nullptr, psi, n_r, ((t_lo % lat->T) + lat->T) % lat->T,
             t_hi - t_lo + 1, true, r, k, nq, prec, out, +1};
  int s = run_part(ctx, c, st);
  int e = end_call(ctx, st);
  return s != LHC_OK ? s : e;
}

int lhc_spectator(lhc_ctx ctx, const lhc_lattice *lat, int kind, const void *S1_or_GA, const void *GB,
                  const void *eta, int n_r, int t_sink, const int r[4], const int *k, int nq, int prec,
                  void *out, void *stream) {
  LHC_TRY(common_checks(ctx, lat, S1_or_GA, eta, n_r, r, k, nq, prec, out));
  if (kind != LHC_MESON && kind != LHC_BARYON) return fail(LHC_EINVAL, "unknown kind %d", kind);
  if ((kind == LHC_MESON) != (GB == nullptr))
    return fail(LHC_EINVAL, "GB must be NULL for mesons and given for baryons");
  if ((uintptr_t)GB & 15) return fail(LHC_EINVAL, "GB must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(ctx->mu);
  LHC_TRY(begin_call(ctx, st));
  PartCall c{kind == LHC_MESON ? PART_SPEC_MESON : PART_SPEC_BARYON, lat, S1_or_GA, GB, eta, n_r,
             ((t_sink % lat->T) + lat->T) % lat->T, 1, false, r, k, nq, prec, out, -1};
  int s = run_part(ctx, c, st);
  int e = end_call(ctx, st);
  return s != LHC_OK ? s : e;
}

int lhc_combine(lhc_ctx ctx, int kind, const void *spec, int np, const void *ins, int nq, int n_r, int nt,
                const void *snk, const void *ins_g, const void *src, int ng, int prec, void *out, void *stream) {
  if (!ctx) return fail(LHC_EINVAL, "ctx is NULL");
  if (kind != LHC_MESON && kind != LHC_BARYON) return fail(LHC_EINVAL, "unknown kind %d", kind);
  if (!spec || !ins || !snk || !ins_g || !src || !out) return fail(LHC_EINVAL, "NULL buffer argument");
  if (np < 1 || nq < 1 || n_r < 1 || ng < 1 || nt < 1) return fail(LHC_EINVAL, "sizes must be positive");
  if (prec != LHC_FP64 && prec != LHC_MIXED) return fail(LHC_EINVAL, "unknown precision %d", prec);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(ctx->mu);
  LHC_TRY(begin_call(ctx, st));
  const int scols = kind == LHC_MESON ? 192 : kBarCols;
  const size_t nw = kind == LHC_MESON ? 16 : 64;
  size_t b_spec = (size_t)np * n_r * scols * 16, b_ins = (size_t)nt * nq * n_r * 192 * 16;
  size_t b_snk = (size_t)ng * nw * 16, b_g = (size_t)ng * 16 * 16, b_src = (size_t)ng * nw * 16;
  size_t b_out = (size_t)nt * ng * np * nq * 16;
  const void *ptr[6] = {spec, ins, snk, ins_g, src, out};
  size_t bytes[6] = {b_spec, b_ins, b_snk, b_g, b_src, b_out};
  bool host[6];
  bool any = false;
  size_t need = 0;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  for (int j = 0; j < 6; ++j) {
    host[j] = !is_device_ptr(ptr[j]);
    any |= host[j];
    if (host[j]) need += al(bytes[j]);
  }
  int s = LHC_OK, slot = -1;
  const void *dev[6];
  char *sp = nullptr;
  if (any) s = stage_begin(ctx, need, &slot, &sp);
  if (s == LHC_OK) {
    size_t off = 0;
    for (int j = 0; j < 6 && s == LHC_OK; ++j) {
      if (host[j]) {
        dev[j] = sp + off;
        if (j < 5) s = stage_in(ctx, slot, sp + off, ptr[j], bytes[j]);
        off += al(bytes[j]);
      } else {
        dev[j] = ptr[j];
      }
    }
  }
  if (s == LHC_OK && any) s = stage_ready(ctx, slot, st);
  if (s == LHC_OK)
    s = run_combine(ctx, kind, (const double2 *)dev[0], np, (const double2 *)dev[1], nq, n_r, nt,
                    (const double2 *)dev[2], (const double2 *)dev[3], (const double2 *)dev[4], ng, prec,
                    (double2 *)dev[5], st);
  if (s == LHC_OK && any) s = stage_end(ctx, slot, st, host[5] ? out : nullptr, dev[5], b_out);
  int e2 = end_call(ctx, st);
  return s != LHC_OK ? s : e2;
}

namespace {
int combine_open(lhc_ctx ctx, int kind, const char *name, const void *spec, int np, const void *ins, int nq,
                 int n_r, int nt, const void *snk, int ngs, const void *ins_g, int ngi, int prec, void *out,
                 void *stream) {
  if (!ctx) return fail(LHC_EINVAL, "ctx is NULL");
  if (!spec || !ins || !snk || !ins_g || !out) return fail(LHC_EINVAL, "NULL buffer argument");
  if (np < 1 || nq < 1 || n_r < 1 || nt < 1 || ngs < 1 || ngi < 1) return fail(LHC_EINVAL, "sizes must be positive");
  if (prec != LHC_FP64 && prec != LHC_MIXED) return fail(LHC_EINVAL, "unknown precision %d", prec);
  const void *ptr[5] = {spec, ins, snk, ins_g, out};
  for (const void *p : ptr)
    if (!is_device_ptr(p)) return fail(LHC_EINVAL, "%s takes device buffers only", name);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(ctx->mu);
  LHC_TRY(begin_call(ctx, st));
  int s = run_combine_open(ctx, kind, static_cast<const double2 *>(spec), np, static_cast<const double2 *>(ins), nq,
                           n_r, nt, static_cast<const double2 *>(snk), ngs, static_cast<const double2 *>(ins_g), ngi,
                           prec, static_cast<double2 *>(out), st);
  int e = end_call(ctx, st);
  return s != LHC_OK ? s : e;
}
}  // namespace

int lhc_combine_open(lhc_ctx ctx, const void *spec, int np, const void *ins, int nq, int n_r, int nt,
                     const void *snk, int ngs, const void *ins_g, int ngi, int prec, void *out, void *stream) {
  return combine_open(ctx, LHC_MESON, "lhc_combine_open", spec, np, ins, nq, n_r, nt, snk, ngs, ins_g, ngi, prec, out,
                      stream);
}

int lhc_combine_open_baryon(lhc_ctx ctx, const void *spec, int np, const void *ins, int nq, int n_r, int nt,
                            const void *wsnk, int ngs, const void *ins_g, int ngi, int prec, void *out,
                            void *stream) {
  return combine_open(ctx, LHC_BARYON, "lhc_combine_open_baryon", spec, np, ins, nq, n_r, nt, wsnk, ngs, ins_g, ngi,
                      prec, out, stream);
}

int lhc_prop_stage(lhc_ctx ctx, const lhc_lattice *lat, const void *S, int t_lo, int t_hi, void *stream) {
  if (!ctx) return fail(LHC_EINVAL, "ctx is NULL");
  LHC_TRY(check_lattice(lat));
  if (lat->dtype != LHC_C128) return fail(LHC_EINVAL, "lhc_prop_stage: complex128 propagators only");
  if (!S || ((uintptr_t)S & 15)) return fail(LHC_EINVAL, "lhc_prop_stage: S must be 16-byte aligned");
  if (!is_device_ptr(S)) return fail(LHC_EINVAL, "lhc_prop_stage: S must be device memory");
  if (t_hi < t_lo || t_hi - t_lo >= lat->T) return fail(LHC_EINVAL, "bad slice range %d..%d", t_lo, t_hi);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(ctx->mu);
  LHC_TRY(begin_call(ctx, st));
  int s = stage_propagator(ctx, lat, S, ((t_lo % lat->T) + lat->T) % lat->T, t_hi - t_lo + 1, st);
  int e = end_call(ctx, st);
  return s != LHC_OK ? s : e;
}

int lhc_prop_unstage(lhc_ctx ctx, const void *S) {
  if (!ctx || !S) return fail(LHC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(ctx->mu);
  LHC_CHECK_CUDA(cudaSetDevice(ctx->device));
  return unstage_propagator(ctx, S);
}

int lhc_set_projection(lhc_ctx ctx, int mode) {
  if (!ctx) return fail(LHC_EINVAL, "ctx is NULL");
  if (mode != LHC_PROJ_AUTO && mode != LHC_PROJ_GEMM && mode != LHC_PROJ_DFT)
    return fail(LHC_EINVAL, "unknown projection mode %d", mode);
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->proj_mode = mode;
  return LHC_OK;
}

int lhc_batch(lhc_ctx ctx, const lhc_call *calls, int ncalls, void *stream) {
  if (!ctx) return fail(LHC_EINVAL, "ctx is NULL");
  if (ncalls < 1 || !calls) return fail(LHC_EINVAL, "lhc_batch: no calls");
  std::vector<lhc::BatchCall> bcs(ncalls);
  const int g5m = g5mask_of(ctx);
  for (int c = 0; c < ncalls; ++c) {
    const lhc_call &a = calls[c];
    const lhc_lattice *lat = &a.lat;
    LHC_TRY(common_checks(ctx, lat, a.S, a.vec, a.n_r, a.r, a.k, a.nq, LHC_MIXED, a.out));
    if (a.part < PART_INS || a.part > PART_SPEC_BARYON) return fail(LHC_EINVAL, "call %d: unknown part %d", c, a.part);
    if ((a.part == PART_SPEC_BARYON) != (a.GB != nullptr))
      return fail(LHC_EINVAL, "call %d: GB must be given for baryons only", c);
    if ((uintptr_t)a.GB & 15) return fail(LHC_EINVAL, "call %d: GB must be 16-byte aligned", c);
    const bool ins = a.part == PART_INS;
    if (a.t_hi < a.t_lo || a.t_hi - a.t_lo >= lat->T || (!ins && a.t_hi != a.t_lo))
      return fail(LHC_EINVAL, "call %d: bad slice range %d..%d", c, a.t_lo, a.t_hi);
    const void *ptrs[4] = {a.S, a.vec, a.out, a.GB ? a.GB : a.S};
    for (const void *p : ptrs)
      if (!is_device_ptr(p)) return fail(LHC_EINVAL, "call %d: lhc_batch takes device buffers only", c);
    const int T = lat->T, V3 = lat->L * lat->L * lat->L;
    const size_t es = esize(lat->dtype), slice = (size_t)V3 * 144 * es, vslice = (size_t)V3 * 12;
    const int cols = a.part == PART_SPEC_BARYON ? kBarCols : 192;
    lhc::BatchCall &bc = bcs[c];
    bc.k = a.k;
    bc.nq = a.nq;
    for (int e = 0; e < 4; ++e) bc.r[e] = a.r[e];
    bc.sign = ins ? +1 : -1;
    const int nt = a.t_hi - a.t_lo + 1, t0 = ((a.t_lo % T) + T) % T;
    bc.jobs.resize(nt);
    for (int j = 0; j < nt; ++j) {
      const int t = (t0 + j) % T;
      SliceJob &job = bc.jobs[j];
      job.part = static_cast<Part>(a.part);
      job.dtype = lat->dtype;
      job.L = lat->L;
      job.V3 = V3;
      job.n_r = a.n_r;
      job.nq = a.nq;
      job.S = static_cast<const char *>(a.S) + (size_t)t * slice;
      job.SB = a.GB ? static_cast<const char *>(a.GB) + (size_t)t * slice : nullptr;
      job.vec = static_cast<const char *>(a.vec) + (ins ? (size_t)t * vslice * es : 0);
      job.vec_stride = ins ? (size_t)T * vslice : vslice;
      job.g5mask = g5m;
      job.out = static_cast<double2 *>(a.out) + (size_t)j * a.nq * a.n_r * cols;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(ctx->mu);
  LHC_TRY(begin_call(ctx, st));
  int s = lhc::run_batch_mixed(ctx, bcs, st);
  int e = end_call(ctx, st);
  return s != LHC_OK ? s : e;
}

}  // extern "C"
