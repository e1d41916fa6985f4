/*
 * liblhc -- factorized stochastic three-point contractions with open spin indices
 * (Bali et al., "Baryonic and mesonic 3-point functions with open spin indices",
 * Lattice 2017, arXiv:1711.02384), for one NVIDIA GB300 (sm_103a).
 *
 * The correlator of Eq. 1 is split (Eq. 8) into a spectator part (Eq. 9), living
 * on the sink timeslice, and an insertion part (Eq. 10), living on every
 * insertion timeslice.  Both keep every spin index and the source colour open and
 * are Fourier-projected onto many momenta; the correlator for any Gamma structure
 * and any momentum pair is then the cheap noise average of Eq. 5 (the combine).
 *
 * Conventions shared by every call
 * --------------------------------
 * complex numbers   interleaved (re, im); LHC_C128 = 2 x double, LHC_C64 = 2 x float.
 * timeslice         L^3 sites, site = (z*L + y)*L + x.
 * propagator        S[T][L^3][12][12] = G(x, r): row = sink spin*3 + colour at x,
 *                   column = source spin*3 + colour at r (a point-to-all propagator).
 * solution psi      psi[n_r][T][L^3][12]: s_i of Eq. 5 (D s_i = eta_i).
 * noise eta         eta[n_r][L^3][12] on the sink slice only (Eq. 5, time-partitioned).
 * momenta k         host int[nq][3]; p = 2*pi*k/L (Sec. 3).  Any order, any values.
 * source r          host int[4] = (x, y, z, t).  Spatial phases use x - r (the rule
 *                   stated after Eq. 10), wrapped periodically; r[3] is not used
 *                   (timeslices are passed as absolute indices, taken mod T).
 * gamma5            diagonal, set per context (default chiral basis diag(1,1,-1,-1)).
 * output            always complex128, in caller memory.
 *
 * Memory: every buffer argument may be device memory or host memory (pinned or
 * pageable), and must be 16-byte aligned (the kernels move complex64 data in 16-byte
 * copies); misaligned buffers return LHC_EINVAL.  Every call is asynchronous on `stream`
 * (a cudaStream_t; NULL = legacy default stream), with device or host buffers alike.
 * Host buffers are staged through eight device slots that successive calls take in
 * turn: the input copies run in call order on a copy stream of the context and overlap
 * the kernels of earlier calls (a call with several slices copies them in up to four
 * groups, each followed by its kernels), and the output copy runs on a second copy
 * stream that `stream` waits for.  So once `stream` (or the device) is synchronized after a call, its host output
 * is written and its host inputs have been read; until then the caller must not change
 * the inputs or read the output.  A later call may take an earlier call's host output
 * as its input: the library tracks host ranges that output copies in flight will write
 * and orders the copies.  Pinned host memory gives overlap; pageable memory is copied
 * synchronously by CUDA.  The caller owns every buffer it passes; the library never
 * frees them.  The first call with a new momentum list, lattice extent or source
 * position builds its phase table (or, in the all-momenta mode, its device copy of the
 * list) with blocking copies; later calls with the same list copy nothing from the host
 * but their host buffers.  The library owns its workspace, its cached phase tables and the
 * staging slots, all counted against the context's HBM budget.  The eight slots share
 * one size, 1.25 times the largest host-buffer call so far (its staged inputs and
 * output), and grow together when a larger call arrives: with a tight budget, prefer
 * device buffers for the largest calls.
 *
 * Errors: every call returns an lhc_status; nothing is thrown across the ABI.
 * Invalid arguments return LHC_EINVAL before anything is launched.
 * lhc_last_error() gives a human-readable description of the last failure on
 * the calling thread.
 */
#ifndef LHC_H
#define LHC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lhc_ctx_s *lhc_ctx;

typedef enum {
  LHC_OK = 0,
  LHC_EINVAL = 1,     /* bad argument (shape, pointer, enum)                        */
  LHC_ENOMEM = 2,     /* device allocation failed                                    */
  LHC_EBUDGET = 3,    /* request does not fit the context's HBM budget               */
  LHC_ETIMEOUT = 4,   /* a bounded wait ran out                                      */
  LHC_ECUDA = 5,      /* a CUDA runtime call failed (see lhc_last_error)             */
  LHC_EBUSY = 6,      /* job still running                                           */
  LHC_ENOTFOUND = 7,  /* unknown handle or job id                                    */
  LHC_ECANCELED = 8   /* job was cancelled                                           */
} lhc_status;

typedef enum {
  LHC_FP64 = 0,   /* plain FP64 GPU path: FP64 site contraction and projection          */
  LHC_MIXED = 1   /* FP32 site contraction, split-FP16 tensor-core projection with
                     FP32 accumulation, FP64 cross-block reduction                       */
} lhc_precision;

typedef enum { LHC_C128 = 0, LHC_C64 = 1 } lhc_dtype;
typedef enum { LHC_MESON = 0, LHC_BARYON = 1 } lhc_kind;

typedef struct {
  int L;       /* spatial extent (sites per direction), 1 <= L <= 128 */
  int T;       /* temporal extent                                     */
  int dtype;   /* lhc_dtype of the propagator, solution and noise     */
} lhc_lattice;

/* Status text (static string). */
const char *lhc_strerror(int status);

/* Description of the last failure on the calling thread (static per thread). */
const char *lhc_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int lhc_version(void);

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the device
 * memory the library itself allocates (workspace, phase tables, staging slots);
 * 0 = no bound. */
int lhc_create(lhc_ctx *ctx, int device, size_t hbm_budget_bytes);

/* Destroy a context: synchronizes the device, then frees everything it owns. */
int lhc_destroy(lhc_ctx ctx);

/* Wait for `stream`, then report whether any kernel of this context gave up a
 * bounded wait since the last check (LHC_ETIMEOUT; results of the affected calls
 * are invalid).  Kernels never spin without limit: a wait that exceeds about two
 * seconds raises this flag and the kernel returns. */
int lhc_sync(lhc_ctx ctx, void *stream);

/* Diagonal of gamma5 (each entry +1 or -1) used by every later call on ctx. */
int lhc_set_gamma5(lhc_ctx ctx, const int g5[4]);

/* Momentum set of Sec. 3: every integer k with |k|^2 <= n2max and, if cmax >= 0,
 * |k_j| <= cmax, ordered by (|k|^2, kx, ky, kz).  Writes min(count, cap) vectors
 * to k (host int[cap][3], may be NULL when cap = 0) and the full count to *nq. */
int lhc_momenta(int n2max, int cmax, int *k, int cap, int *nq);

/* Insertion part, Eq. 10, on every slice t = t_lo .. t_hi (taken mod T):
 *
 *   out[t - t_lo][q][i][(at*4 + bt)*12 + b*3 + a]
 *     = sum_y e^{+i p_q.(y - r)} sum_{a~} g5(at) conj(psi_i(y)[at*3 + a~])
 *                                   S3(y)[(bt*3 + a~)*12 + b*3 + a]
 *
 * (at = alpha~, bt = beta~, b = beta, a = source colour).  S3: propagator
 * G3(y, r); psi: solutions; out: complex128 [t_hi - t_lo + 1][nq][n_r][192].
 * prec: lhc_precision.  Requires 1 <= n_r, 1 <= nq, 0 <= t_hi - t_lo < T. */
int lhc_insertion(lhc_ctx ctx, const lhc_lattice *lat, const void *S3, const void *psi,
                  int n_r, int t_lo, int t_hi, const int r[4], const int *k, int nq,
                  int prec, void *out, void *stream);

/* Spectator part on the sink slice t_sink.
 *
 * kind = LHC_MESON, Eq. 9 with G1(r, x') = gamma5 S1(x')^dagger gamma5:
 *   out[q][i][(bp*4 + ap)*12 + al*3 + a]
 *     = sum_x' e^{-i p_q.(x' - r)} sum_{a'} g5(bp) g5(ap) g5(al) eta_i(x')[bp*3 + a']
 *                                      conj(S1(x')[(ap*3 + a')*12 + al*3 + a])
 *   (bp = beta', ap = alpha', al = alpha); out: complex128 [nq][n_r][192].
 *
 * kind = LHC_BARYON (the paper states the baryon case without a formula; this is
 * the eps-eps reading in which the third quark's sink end is the same stochastic
 * (gamma5 eta_i) as the meson's, so the insertion part is shared):
 *   out[q][i][((((a1p*4 + a1)*4 + a2p)*4 + a2)*4 + bp)*3 + c]
 *     = sum_x' e^{-i p_q.(x' - r)} sum eps_{a' b' c'} eps_{a b c}
 *         GA(x')[(a1p*3 + a')*12 + a1*3 + a] GB(x')[(a2p*3 + b')*12 + a2*3 + b]
 *         g5(bp) eta_i(x')[bp*3 + c']
 *   GA, GB: the two spectator propagators G(x', r); out: complex128 [nq][n_r][3072].
 * GB must be NULL for LHC_MESON and non-NULL for LHC_BARYON. */
int lhc_spectator(lhc_ctx ctx, const lhc_lattice *lat, int kind, const void *S1_or_GA,
                  const void *GB, const void *eta, int n_r, int t_sink, const int r[4],
                  const int *k, int nq, int prec, void *out, void *stream);

/* Noise-averaged combine (Eqs. 5 and 8) for ng spin structures and nt insertion
 * slices (index t):
 *
 * LHC_MESON:  out[t][g][p][q] = (1/n_r) sum_i sum Gsnk[g][ap][bp] Gins[g][at][bt] Gsrc[g][b][al]
 *                               spec[p][i][(bp, ap, al, a)] ins[t][q][i][(at, bt, b, a)]
 *             snk, src: complex128 [ng][4][4]
 * LHC_BARYON: out[t][g][p][q] = (1/n_r) sum_{i,c} sum Wsnk[g][a1p][a2p][bp] Wsrc[g][a1][a2][b]
 *                               Gins[g][at][bt] spec[p][i][(a1p,a1,a2p,a2,bp,c)] ins[t][q][i][(at,bt,b,c)]
 *             snk, src: complex128 [ng][4][4][4]
 * ins_g: complex128 [ng][4][4]; spec: [np][n_r][192 | 3072]; ins: [nt][nq][n_r][192] (the
 * output of lhc_insertion); out: complex128 [nt][ng][np][nq].
 * prec LHC_FP64: everything in FP64.  LHC_MIXED: the Gamma contractions and the 12-term
 * spin-colour sum of each noise in FP32, the sum over noises (the noise average) in FP64. */
int lhc_combine(lhc_ctx ctx, int kind, const void *spec, int np, const void *ins, int nq,
                int n_r, int nt, const void *snk, const void *ins_g, const void *src, int ng,
                int prec, void *out, void *stream);

/* Free the context's workspace and cached phase tables (they are re-created on demand). */
int lhc_release_workspace(lhc_ctx ctx);

/* Failure-detection self-test: launches a kernel that waits on a barrier nothing will
 * complete, with a limit of limit_us microseconds (1..2000000).  The wait gives up, sets
 * the context's device error word and the kernel returns; lhc_sync then reports
 * LHC_ETIMEOUT and the context stays usable.  Returns the lhc_sync status. */
int lhc_selftest_timeout(lhc_ctx ctx, int limit_us, void *stream);

/* The same bounded wait without the report: on return (asynchronously, on `stream`) the
 * context's device error word is set, as after a kernel that gave up a wait, until the
 * next lhc_sync reports it.  Meanwhile the context's kernels give up their waits at once,
 * and an autotuning call stops with LHC_ETIMEOUT instead of recording a shape.  For tests
 * of failure handling; limit_us as above. */
int lhc_selftest_flag(lhc_ctx ctx, int limit_us, void *stream);

/* ---------------------------------------------------------------- job server
 * Continuous batching of contraction jobs (the serving form of the hot path; the paper
 * runs measurements as batch jobs and has no counterpart).  lhc_serve_start starts a
 * scheduler thread with `slots` execution slots, each with its own stream and workspace,
 * so admitted jobs overlap on the GPU.  Propagators are registered once and stay resident
 * on the device.  A job is admitted as soon as a slot is free and the context's HBM budget
 * (lhc_create) covers the resident propagators, the workspace every slot holds and the
 * job's additional workspace (an upper bound from its shapes); jobs that can never fit are
 * refused at submission with LHC_EBUDGET.  Admission is first-fit in submission order.
 * Slots project in the automatic mode (lhc_set_projection): a job with nq >= L^3 / 2
 * takes the all-momenta transform, and its bound is that of the transform.
 * Results do not depend on what else runs: the kernels sum in a fixed order.  Timestamps
 * (steady clock, seconds) give submit -> start -> poll-visible completion latencies. */
typedef enum { LHC_JOB_INSERTION = 0, LHC_JOB_SPECTATOR = 1, LHC_JOB_THREEPT = 2 } lhc_job_type;
typedef enum {
  LHC_JOB_QUEUED = 0,
  LHC_JOB_RUNNING = 1,
  LHC_JOB_DONE = 2,
  LHC_JOB_FAILED = 3,
  LHC_JOB_CANCELED = 4
} lhc_job_state;

typedef struct {
  int type;           /* lhc_job_type; THREEPT = insertion + spectator                    */
  int kind;           /* LHC_MESON or LHC_BARYON (spectator part)                          */
  int prec;           /* lhc_precision                                                     */
  uint64_t prop;      /* registered propagator: S3 for the insertion, S1 / GA for the
                         spectator (one source position, the lattice of the handle)      */
  uint64_t prop_b;    /* registered GB for baryons, else 0                                 */
  const void *psi;    /* device, [n_r][T][V3][12] (insertion)                             */
  const void *eta;    /* device, [n_r][V3][12] on t_sink (spectator)                      */
  int n_r;
  int t_lo, t_hi;     /* insertion slices                                                  */
  int t_sink;         /* spectator slice                                                   */
  int r[4];           /* source position                                                   */
  const int *k;       /* host [nq][3]; copied at submission                               */
  int nq;
  void *out_ins;      /* device, [t_hi - t_lo + 1][nq][n_r][192]                           */
  void *out_spec;     /* device, [nq][n_r][192 | 3072]                                     */
} lhc_job;

int lhc_serve_start(lhc_ctx ctx, int slots);
int lhc_serve_stop(lhc_ctx ctx);   /* waits for running jobs; lhc_destroy calls it */
int lhc_prop_register(lhc_ctx ctx, const void *dev_ptr, const lhc_lattice *lat, uint64_t *handle);
int lhc_prop_release(lhc_ctx ctx, uint64_t handle);   /* LHC_EBUSY while jobs use it */
int lhc_submit(lhc_ctx ctx, const lhc_job *job, uint64_t *job_id);
/* non-blocking: LHC_EBUSY while queued or running, LHC_OK once finished (any outcome);
 * *state receives the lhc_job_state */
int lhc_poll(lhc_ctx ctx, uint64_t job_id, int *state);
/* the job's final status, or LHC_ETIMEOUT if it has not finished within timeout_ms */
int lhc_wait(lhc_ctx ctx, uint64_t job_id, int timeout_ms);
int lhc_cancel(lhc_ctx ctx, uint64_t job_id);   /* queued jobs only, else LHC_EBUSY */
int lhc_job_times(lhc_ctx ctx, uint64_t job_id, double *t_submit, double *t_start, double *t_done);
/* Device times of a finished job, in ms after an event the server recorded when it started:
 * when its slot's stream reached the job's first launch and when it finished the last, from
 * CUDA timing events on that stream.  Jobs whose intervals intersect had work in flight on
 * the device at the same time.  LHC_EBUSY until the job is done (LHC_JOB_DONE). */
int lhc_job_device_times(lhc_ctx ctx, uint64_t job_id, double *ms_start, double *ms_done);
int lhc_serve_stats(lhc_ctx ctx, size_t *bytes_in_use, int *queued, int *running);

/* Allocation-free variant of lhc_combine (the paper has no counterpart; this is a
 * library service).  For callers that cannot let a library allocate device memory:
 * a process whose device memory is owned by another allocator (for example an analysis
 * framework's caching pool that has reserved almost all of HBM), or host code that must
 * not stall, since cudaMalloc/cudaFree can synchronize the device.  Same arguments and
 * results as lhc_combine, but no context, and every buffer must be device memory of
 * the current device or managed memory (host buffers and buffers of another GPU give
 * LHC_EINVAL).  The intermediate tensors live in a fixed 32 MiB
 * scratch array inside the library image, which every GPU that loads the library
 * holds until the process exits; the call itself never allocates.  A call needs
 * ng*(np+nq)*12*n_r*16 + 4*ng bytes of it for one insertion slice (larger combines give
 * LHC_EINVAL with the size; nt is processed in chunks that fit).  The first call on a
 * device looks up the scratch's device address (cudaGetSymbolAddress), so make that
 * first call before any stream capture.  All calls on a device share the scratch and
 * it keeps the last call's contents (nothing in it needs clearing); calls whose kernels
 * may overlap on the GPU race on it, so order them on one stream or with events. */
int lhc_combine_noalloc(int kind, const void *spec, int np, const void *ins, int nq, int n_r, int nt,
                        const void *snk, const void *ins_g, const void *src, int ng, int prec,
                        void *out, void *stream);

/* Kernel-level timing with CUDA events recorded on the launching stream, for
 * roofline measurements.  lhc_profile(ctx, 1) clears the records and starts
 * recording around every launch of the listed kernels; lhc_profile(ctx, 0) stops.
 * lhc_profile_read waits for the recorded launches and returns, for one kernel
 * class, the summed device time in ms, the number of launches, and the
 * algorithmic work of those launches (flops for LHC_KERNEL_PROJECT and
 * LHC_KERNEL_FUSED: 8 per complex multiply-add of the direct sum; bytes of input
 * read plus output written for LHC_KERNEL_CONTRACT).  Timing adds two event
 * records per launch; leave it off outside measurements. */
typedef enum {
  LHC_KERNEL_PROJECT = 0,    /* FP64 projection GEMM                                   */
  LHC_KERNEL_CONTRACT = 1,   /* FP64 site contraction                                  */
  LHC_KERNEL_FUSED = 2,      /* mixed path: fused contraction + tensor-core projection */
  LHC_KERNEL_REDUCE = 3,     /* mixed path: FP64 cross-block reduction                 */
  LHC_KERNEL_COMBINE = 4,    /* FP64 combine (all of its kernels)                      */
  LHC_KERNEL_COUNT = 5
} lhc_kernel_id;

int lhc_profile(lhc_ctx ctx, int enable);
int lhc_profile_read(lhc_ctx ctx, int kernel, double *total_ms, long long *launches,
                     double *work);

/* Number of CUDA kernel launches this library has issued since it was loaded, over
 * all contexts and threads (launches replayed from a captured CUDA graph are not
 * counted again).  Never fails; reading it costs one atomic load. */
unsigned long long lhc_launch_count(void);

/* Open-source-spin combine (meson): Eq. 8 with the source Gamma left open,
 *
 *   out[t][gs][gi][p][q][al*4 + be]
 *     = (1/N) sum_i sum_a Shat_i[gs](p)[al*3 + a] Ihat_i[t][gi](q)[be*3 + a],
 *   Shat_i[gs] = sum_{ap,bp} Gsnk[gs][ap][bp] spec_i[(bp*4 + ap)*12 + al*3 + a],
 *   Ihat_i[gi] = sum_{at,bt} Gins[gi][at][bt] ins_i[(at*4 + bt)*12 + be*3 + a],
 *
 * the quantities of lhc_combine before Gamma_src is applied. For any source structure,
 *   C = sum_{al,be} Gsrc[be][al] out[...][al*4 + be]
 * equals lhc_combine's result. So one call serves every (Gamma_snk, Gamma_ins) pair of
 * the two lists and, after a 4x4 contraction per (p, q), every Gamma_src: with
 * 16-entry lists that is the whole 16 x 16 x 16 sweep over the Dirac basis (Sec. 3).
 * spec: [np][n_r][192], ins: [nt][nq][n_r][192], snk: [ngs][4][4], ins_g: [ngi][4][4];
 * out: complex128 [nt][ngs][ngi][np][nq][16]; nt*ngs*ngi <= 65535. Device buffers only
 * (LHC_EINVAL otherwise). prec as for lhc_combine. */
int lhc_combine_open(lhc_ctx ctx, const void *spec, int np, const void *ins, int nq, int n_r, int nt,
                     const void *snk, int ngs, const void *ins_g, int ngi, int prec, void *out, void *stream);

/* Open-source-spin combine (baryon): Eq. 8 for the baryon with the source structure
 * W_src left open (Sec. 2: with open indices every spin structure, parity projector or
 * diquark, follows after the expensive contractions),
 *
 *   out[t][gs][gi][p][q][(a1*4 + a2)*4 + b]
 *     = (1/N) sum_i sum_c Bhat_i[gs](p)[(a1*4 + a2)*3 + c] Ihat_i[t][gi](q)[b*3 + c],
 *   Bhat_i[gs] = sum_{a1p,a2p,bp} Wsnk[gs][a1p][a2p][bp]
 *                  spec_i[((((a1p*4 + a1)*4 + a2p)*4 + a2)*4 + bp)*3 + c],
 *   Ihat_i[gi] = sum_{at,bt} Gins[gi][at][bt] ins_i[(at*4 + bt)*12 + b*3 + c],
 *
 * lhc_combine's baryon quantities before W_src is applied. For any source structure,
 *   C = sum_{a1,a2,b} Wsrc[a1][a2][b] out[...][(a1*4 + a2)*4 + b]
 * equals lhc_combine's LHC_BARYON result for (Wsnk[gs], Gins[gi], Wsrc).
 * spec: [np][n_r][3072] (lhc_spectator, LHC_BARYON), ins: [nt][nq][n_r][192],
 * wsnk: [ngs][4][4][4], ins_g: [ngi][4][4]; out: complex128 [nt][ngs][ngi][np][nq][64];
 * nt*ngs*ngi <= 65535, ngs <= 150 (shared memory). Device buffers only (LHC_EINVAL
 * otherwise). prec as for lhc_combine: LHC_MIXED sums each group of four noises in
 * FP32 and the groups exactly. */
int lhc_combine_open_baryon(lhc_ctx ctx, const void *spec, int np, const void *ins, int nq, int n_r, int nt,
                            const void *wsnk, int ngs, const void *ins_g, int ngi, int prec, void *out,
                            void *stream);

/* ---- Batched calls: one fused launch for many calls.
 * One call of lhc_insertion or lhc_spectator (LHC_MIXED): part 0 insertion (Eq. 10),
 * 1 meson spectator (Eq. 9), 2 baryon spectator. S is S3, S1 or GA; GB is the second
 * baryon propagator (else NULL); vec is psi [n_r][T][L^3][12] (insertion) or eta
 * [n_r][L^3][12]. Slices t_lo..t_hi (mod T, at most 64) for the insertion, and
 * t_lo = t_hi = t_sink for the spectators. out as for the single call. */
typedef struct {
  int part;
  lhc_lattice lat;
  const void *S, *GB, *vec;
  int n_r, t_lo, t_hi;
  int r[4];
  const int *k;
  int nq;
  void *out;
} lhc_call;
/* Runs ncalls calls in precision LHC_MIXED with one persistent fused-kernel launch per
 * part kind and momentum-chunk width, for up to 64 calls per launch: one CTA per SM takes
 * the calls' tasks (tile, site split, slice, momentum chunk), longest first, from a device
 * counter until none is left. The per-call staging and
 * reduce kernels stay separate launches. A batch always projects on the tensor cores,
 * whatever lhc_set_projection says. The results are bitwise those of the same calls
 * made one by one in LHC_PROJ_GEMM mode: each CTA does the work it does in its call's
 * own launch, with the same launch shape, taken from the tuning table or the heuristic
 * (a batch never tunes; tune its shapes with single calls first). A call that asks
 * for at least half of a slice's momenta takes the transform when made alone in
 * LHC_PROJ_AUTO mode; the two agree within the mixed path's tolerance. Device buffers only. The calls'
 * outputs must not overlap their inputs or each other. Asynchronous on `stream`;
 * capturable in a CUDA graph once the phase tables exist (after a first run). The
 * paper has no counterpart: it ran one contraction at a time. */
int lhc_batch(lhc_ctx ctx, const lhc_call *calls, int ncalls, void *stream);

/* ---- Staged propagator slices (mixed path).
 * A mixed-precision call with complex128 inputs first narrows them to complex64 (the
 * contraction runs in FP32). Calls that share a propagator (the insertion calls of
 * several sink times over slices t0..t_f, the spectators on their sink slices) would each
 * narrow it again. lhc_prop_stage narrows slices t_lo..t_hi (mod T) of the complex128
 * propagator S [T][L^3][12][12] once, into a complex64 copy held by the library (counted
 * against ctx's HBM budget) together with each slice's largest |re| or |im|. Every later
 * LHC_MIXED insertion or meson spectator call, of any context on the same device, whose
 * propagator slices are consecutive slices of one staged range reads the copy instead of
 * narrowing S; its results are bitwise the same. Other calls (baryon spectators, FP64,
 * complex64 inputs, host buffers, slices outside the range) are not affected.
 * The caller must not change the staged slices of S while they are staged, or must stage
 * them again (staging the same range of the same S again rewrites the copy in stream
 * order, with no allocation); the staging context must outlive the calls that read the
 * copy. The copy is found by S's address: S must stay allocated while staged (unstage it,
 * or destroy the staging context, before freeing it), or memory later allocated at that
 * address would be read through the stale copy. Asynchronous on `stream`: calls on other
 * streams must wait for it (an event).
 * Staging another range of the same S, and lhc_prop_unstage, synchronize the device
 * before the old copy is freed. Errors: LHC_EINVAL (not complex128, not device memory,
 * bad range), LHC_ENOTFOUND (unstage of a pointer not staged). The paper has no
 * counterpart: its propagators stay in double precision. */
int lhc_prop_stage(lhc_ctx ctx, const lhc_lattice *lat, const void *S, int t_lo, int t_hi, void *stream);
int lhc_prop_unstage(lhc_ctx ctx, const void *S);

/* ---- Momentum projection by discrete Fourier transform (all-momenta mode).
 * The projection of Eqs. 9 and 10 over every momentum of a slice is a 3-D discrete
 * Fourier transform of the contracted values. In this mode the library contracts and
 * transforms along x, y and z with L-point sums (3L complex multiply-adds per value,
 * against nq for the direct projection, for any L). It then gathers the
 * requested momenta (any list, order or duplicates), each times exp(-+i p.r) for the
 * source position. LHC_FP64 calls contract and transform in FP64 (within 1e-12);
 * LHC_MIXED calls contract and transform in FP32 (within 1e-6 per correlator). The
 * output is complex128 either way.
 * LHC_PROJ_AUTO (the default) uses it for calls with nq >= L^3 / 2, where it is far
 * cheaper than the direct projection in either precision. LHC_PROJ_GEMM never uses
 * the transform, LHC_PROJ_DFT always. The mode governs single calls (and the job
 * server's slots use LHC_PROJ_AUTO); lhc_batch always projects on the tensor cores.
 * Asynchronous on `stream` once the call's momentum
 * list has been seen (its device copy is cached with the phase tables); the first call
 * with a list uploads it with blocking copies, so make that call before any stream
 * capture. The paper projects directly (it uses at most 93 momenta). */
typedef enum { LHC_PROJ_AUTO = 0, LHC_PROJ_GEMM = 1, LHC_PROJ_DFT = 2 } lhc_projection;
int lhc_set_projection(lhc_ctx ctx, int mode);

/* ---- Free-field Wilson-Dirac operator and solver: inputs for end-to-end checks.
 *
 * The paper computes propagators and solutions on gauge configurations with a
 * multigrid solver (Sec. 3). With unit gauge links the Wilson-Dirac operator
 * (Wilson parameter 1, bare mass m) is
 *   (D psi)(x) = (m + 4) psi(x)
 *                - 1/2 sum_mu [ (1 - gamma_mu) psi(x + mu) + (1 + gamma_mu) psi(x - mu) ],
 * colour-diagonal and periodic in all four directions (mu = x, y, z, t). Its inverse
 * has a closed form, so point-to-all propagators G(x, r) (Eq. 1) and solutions
 * s_i = D^{-1} eta_i (Eq. 5) made with it let the whole path be checked against an
 * independent momentum-space evaluation.
 *
 * Fields are complex128 device arrays [nrhs][T][L^3][12] (spin*3 + colour), lat->dtype
 * = LHC_C128. gammas: host double[4][4][4][2], gamma_mu[s][s'] (re, im) for
 * mu = x, y, z, t. They must be Hermitian, and with gamma5 = g1 g2 g3 g4 diagonal, as
 * in the default chiral basis, the results feed the other calls directly.
 * Asynchronous on `stream`. Returns LHC_EINVAL for host fields or bad shapes. */
/* out = D in (dagger = 0) or D^dagger in (dagger != 0: gamma_mu -> -gamma_mu). */
int lhc_wilson_apply(lhc_ctx ctx, const lhc_lattice *lat, double mass, const double *gammas, int dagger,
                     const void *in, void *out, int nrhs, void *stream);
/* sol = D^{-1} src for nrhs right-hand sides: conjugate gradients on
 * D^dagger D sol = D^dagger src, in FP64, until |D^dagger r| <= tol |D^dagger src| for
 * every right-hand side or maxiter iterations. Synchronizes `stream` once per
 * iteration; allocates its three work fields from the context's budget.
 * *iters = iterations, *relres = max over right-hand sides of |src - D sol| / |src|
 * (either may be NULL). */
int lhc_wilson_solve(lhc_ctx ctx, const lhc_lattice *lat, double mass, const double *gammas, const void *src,
                     void *sol, int nrhs, double tol, int maxiter, int *iters, double *relres, void *stream);

/* ---- Launch-shape autotuning of the LHC_MIXED path.  The paper has no counterpart:
 * its kernels were tuned by hand for one machine.
 *
 * The fused kernel's launch shape has two parameters: how many momentum
 * representatives (one per pair k, -k) one CTA projects (8..48, a multiple of 8), and
 * into how many site ranges each slice is split.  Without tuning a heuristic picks
 * them: the widest chunks, and splits that fill whole waves of one CTA per SM.
 *
 * With mode LHC_TUNE_ON, the first LHC_MIXED call of every new shape (part, dtype, L^3,
 * n_r, slices per launch, representatives) times up to 30 candidate shapes on its own
 * inputs. It synchronizes its stream meanwhile, and the fastest shape is kept for every
 * later call of that shape in the process, from any context. Calls whose stream is
 * being captured into a CUDA graph never tune, so tune before capturing. A tuned
 * call's results equal those of any other shape within the mixed path's error bound:
 * the site split changes the summation order. Calls of the same shape always use the
 * same launch shape, so they are bitwise reproducible.
 *
 * path (may be NULL) names a text file. Entries already in it are loaded now, and the
 * whole table is rewritten after each new entry, one line per shape:
 *   part dtype V3 n_r nt nrep  NH nsplit  microseconds
 * Returns LHC_EINVAL for an unknown mode or a malformed file. */
typedef enum { LHC_TUNE_OFF = 0, LHC_TUNE_ON = 1 } lhc_tune_mode;
int lhc_set_tuning(lhc_ctx ctx, int mode, const char *path);

/* The process-wide launch-shape table: writes min(count, cap) entries as int[cap][8]
 * (part, dtype, V3, n_r, nt, nrep, NH, nsplit; part 0 insertion, 1 meson spectator,
 * 2 baryon spectator) and the number of entries to *count. */
int lhc_tuning_table(int *entries, int cap, int *count);

/* Loads the entries of a table file into the process-wide table without touching a
 * GPU; *count = entries read (0 when the file does not exist).  LHC_EINVAL on a
 * malformed line, which leaves the lines before it loaded. */
int lhc_tuning_load(const char *path, int *count);

#ifdef __cplusplus
}
#endif

#endif /* LHC_H */
