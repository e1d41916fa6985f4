// Internal declarations of liblhc (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lhc.h"

namespace lhc {

// ---------------------------------------------------------------- launch accounting
// Every kernel launch site calls note_launch() right after the launch.
extern std::atomic<unsigned long long> g_launches;
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
#define LHC_CHECK_CUDA(call)                                                     \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      ::lhc::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                 \
                       cudaGetErrorString(e_));                                  \
      return LHC_ECUDA;                                                          \
    }                                                                            \
  } while (0)
#define LHC_TRY(expr)                 \
  do {                                \
    int s_ = (expr);                  \
    if (s_ != LHC_OK) return s_;      \
  } while (0)

// Raises a kernel's dynamic shared-memory limit to `bytes` once per device.  `done` holds
// one bit per device ordinal; it is atomic, so calls from several host threads (the job
// server's scheduler and a caller) are safe, and a repeated call from a racing thread is
// harmless.
template <typename K>
int ensure_smem_limit(K *kernel, int bytes, std::atomic<unsigned long long> &done) {
  int dev = 0;
  LHC_CHECK_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return LHC_OK;
  LHC_CHECK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.fetch_or(bit, std::memory_order_acq_rel);
  return LHC_OK;
}

// ---------------------------------------------------------------- problem shapes
constexpr int kInsCols = 192;       // (alpha~, beta~, beta, a) per noise
constexpr int kMesCols = 192;       // (beta', alpha', alpha, a) per noise
constexpr int kBarCols = 3072;      // (alpha1', alpha1, alpha2', alpha2, beta', c) per noise
// site splits per slice of a mixed launch: the autotuner's largest candidate, the bound of
// a tuning-table entry and of the workspace estimate of the job server's admission
constexpr int kMaxSplits = 16;

enum Part { PART_INS = 0, PART_SPEC_MESON = 1, PART_SPEC_BARYON = 2 };

// One slice worth of contraction + projection.  Pointers are device pointers.
struct SliceJob {
  Part part;
  int dtype;            // lhc_dtype of the inputs
  int L, V3, n_r, nq;
  const void *S;        // propagator slice [V3][144] (S3, S1 or GA)
  const void *SB;       // baryon: GB slice [V3][144]
  const void *vec;      // psi slice of noise 0 (ins) or eta (spec): [V3][12]
  size_t vec_stride;    // elements between consecutive noises of vec
  int g5mask;           // bit s set when g5(s) = -1
  double2 *out;         // [nq][n_r * cols]
};

// ---------------------------------------------------------------- context
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

struct PhaseKey {
  int L, nq, sign, fmt, rx, ry, rz;
  uint64_t khash;
  bool operator<(const PhaseKey &o) const;
  bool operator==(const PhaseKey &o) const { return !(*this < o) && !(o < *this); }
};

struct ProfRecord {
  int kernel;
  cudaEvent_t start, stop;
  double work;
};

// Records CUDA events around one kernel launch when profiling is on.
struct ProfScope {
  lhc_ctx ctx;
  cudaStream_t st;
  int kernel;
  double work;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(lhc_ctx c, cudaStream_t s, int k, double w);
  ~ProfScope();
};

struct PhaseEntry {
  DevBuf buf;
  int nq_pad = 0;
  unsigned long long used_in = 0;   // the last call (lhc_ctx_s::call_seq) that took this table
};

}  // namespace lhc

struct lhc_ctx_s {
  int device = 0;
  size_t budget = 0;   // 0 = unbounded
  size_t used = 0;     // bytes the library holds
  int g5[4] = {1, 1, -1, -1};
  std::mutex mu;
  lhc::DevBuf ws;                         // general workspace (grown on demand)
  // Host-buffer staging: kStageSlots device slots used by successive calls in turn, one
  // H2D copy stream (copies land in call order; a slot's reuse waits for the call
  // kStageSlots back, which with 8 slots is normally long done), one D2H copy stream,
  // and the host ranges that output copies still in flight will write (a later call
  // reading such a range waits for that copy).  All slots have one size, grown together
  // (in stream order, from a memory pool of the context that keeps freed memory mapped)
  // when a call needs more, so a rotation of differently sized calls over the slots
  // grows nothing once the largest call has been seen.
  static constexpr int kStageSlots = 8;
  lhc::DevBuf stage[kStageSlots];
  size_t stage_bytes = 0;                 // the size of every allocated slot
  cudaMemPool_t stage_pool = nullptr;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t slot_free[kStageSlots] = {}, in_ready[kStageSlots] = {}, comp_done = nullptr;
  bool slot_used[kStageSlots] = {};
  int next_slot = 0;
  struct PendingOut {
    const char *p;
    size_t n;
    cudaEvent_t ev;
  };
  std::vector<PendingOut> pending_out;
  std::vector<cudaEvent_t> event_pool;
  std::map<lhc::PhaseKey, lhc::PhaseEntry> phases;
  std::list<lhc::PhaseKey> phase_lru;     // front = most recent
  unsigned long long call_seq = 0;        // counts calls; the current call's tables are never evicted
  // the stream of the current call; the context's calls are ordered across streams (each
  // call's stream waits for the previous call), so it covers all earlier work of the context
  cudaStream_t cur_stream = nullptr;
  int num_sms = 0;
  bool prof_on = false;
  int *dev_err = nullptr;                 // sticky device error word (bounded waits that gave up)
  int tune_mode = 0;                      // lhc_tune_mode: time launch shapes of new shapes
  int proj_mode = 0;                      // lhc_projection: auto, GEMM or DFT momentum projection
  std::vector<lhc::ProfRecord> prof;
};

namespace lhc {

// memory accounting
int dev_alloc(lhc_ctx ctx, DevBuf &b, size_t bytes);
void dev_free(lhc_ctx ctx, DevBuf &b);
int ensure(lhc_ctx ctx, DevBuf &b, size_t bytes);   // grows b (synchronizes the current call's stream first)

int g5mask_of(const lhc_ctx ctx);
uint64_t hash_k(const int *k, int nq);

// phase tables.  phase_take() marks a cached entry as used by the current call (LRU
// front); phase_insert() adds a new one the same way.  Eviction under the HBM budget skips
// every entry the current call has taken: its pointers are already in the call's launches.
const PhaseEntry *phase_take(lhc_ctx ctx, const PhaseKey &key);
void phase_insert(lhc_ctx ctx, const PhaseKey &key, const PhaseEntry &e);
// fmt 0: complex128 [nq][V3], P[q][x] = exp(sign*2*pi*i*((k.(x-r)) mod L)/L)
int get_phase_f64(lhc_ctx ctx, int L, const int *k, int nq, const int r[4], int sign,
                  cudaStream_t st, const double2 **out);

// FP64 path: contraction into a workspace, then projection (k_f64.cu)
int run_slice_f64(lhc_ctx ctx, const SliceJob &job, const double2 *phase, cudaStream_t st);

// FP64 site contraction of sites s0 .. s0+ns-1 into U[site - s0][i][cols] (k_f64.cu)
int contract_f64(const SliceJob &j, int s0, int ns, double2 *U, cudaStream_t st);
int contract_f32(const SliceJob &j, int s0, int ns, float2 *U, cudaStream_t st);

// all-momenta mode: FP64 contraction, three line DFTs over the slice, gather (k_fft.cu)
bool use_fft(lhc_ctx ctx, int prec, int V3, int nq);
size_t fft_call_bytes(Part part, int prec, int L, int n_r, int nq);   // its allocation bound
int run_part_fft(lhc_ctx ctx, const SliceJob *jobs, int nt, const int *k, int nq, const int r[4], int sign,
                 int prec, cudaStream_t st);

// mixed path: all slices of one call in one set of launches (k_mixed.cu)
int run_part_mixed(lhc_ctx ctx, const SliceJob *jobs, int nt, const int *k, int nq, const int r[4], int sign,
                   cudaStream_t st, int shape_nt = 0);

size_t mixed_call_bytes(Part part, int dtype, int V3, int n_r, int nt, int nq);

// complex64 copies of complex128 propagator slices shared by later mixed calls (k_mixed.cu)
int stage_propagator(lhc_ctx ctx, const lhc_lattice *lat, const void *S, int t_lo, int nt, cudaStream_t st);
int unstage_propagator(lhc_ctx ctx, const void *S);
void release_staged(lhc_ctx ctx);   // the copies the context holds (the device is synchronized)

// a batch of mixed calls with one fused launch per part kind and chunk width (k_mixed.cu)
struct BatchCall {
  std::vector<SliceJob> jobs;
  const int *k;
  int nq;
  int r[4];
  int sign;
};
int run_batch_mixed(lhc_ctx ctx, const std::vector<BatchCall> &calls, cudaStream_t st);

// launch-shape table of the mixed path (lhc_tune.cu): process-wide, guarded by a mutex
struct TuneKey {
  int part, dtype, V3, n_r, nt, nrep;   // nt: slices per launch
  bool operator<(const TuneKey &o) const;
};
struct TuneChoice {
  int NH, nsplit;   // representatives per CTA, site splits per slice
  float us;         // measured time of one call with this shape
};
bool tune_lookup(const TuneKey &key, TuneChoice *out);
void tune_store(const TuneKey &key, const TuneChoice &c);   // and rewrites the table file, if one is set

// combine (k_combine.cu)
int run_combine(lhc_ctx ctx, int kind, const double2 *spec, int np, const double2 *ins, int nq,
                int n_r, int nt, const double2 *snk, const double2 *ins_g, const double2 *src, int ng,
                int prec, double2 *out, cudaStream_t st);

// open-source-spin combine, meson or baryon (k_combine.cu)
int run_combine_open(lhc_ctx ctx, int kind, const double2 *spec, int np, const double2 *ins, int nq, int n_r, int nt,
                     const double2 *snk, int ngs, const double2 *ins_g, int ngi, int prec, double2 *out,
                     cudaStream_t st);

// combine on caller-provided scratch, no allocation (k_combine.cu)
int run_combine_scratch(int kind, const double2 *spec, int np, const double2 *ins, int nq, int n_r, int nt,
                        const double2 *snk, const double2 *ins_g, const double2 *src, int ng, int prec,
                        double2 *Xs, double2 *Xi, double2 *out, cudaStream_t st);

// kernels' launch wrappers
void launch_phase_f64(double2 *P, const int *k_dev, int nq, int L, int rx, int ry, int rz,
                      int sign, const double2 *roots_dev, cudaStream_t st);

}  // namespace lhc
