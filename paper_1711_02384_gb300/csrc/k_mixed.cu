// Mixed-precision path for the meson insertion (Eq. 10) and spectator (Eq. 9): one
// fused kernel per call that performs the site contraction in FP32 and the momentum
// projection on tcgen05 tensor cores, plus an FP64 cross-block reduction.
//
// GEMM view: out[q][col] = sum_x P[q][x] U[x][col], x over the sites of a timeslice,
// P[q][x] = exp(i sign phi_q(x)), phi_q(x) = 2 pi k_q.(x - r) / L.
//
// Momentum pairs.  phi_{-k} = -phi_k, so the phases of k and -k are complex conjugates.
// The momenta are grouped into representatives k_rho (one per pair {k, -k}, or per
// momentum whose partner is not requested), and the tensor cores compute only the two
// real projections
//   C_rho = sum_x cos(phi_rho(x)) U(x),   S_rho = sum_x sin(phi_rho(x)) U(x)   (U complex),
// from which every requested momentum follows as out[q] = C_rho + i sigma_q S_rho with
// sigma_q = sign * (+1 if k_q = k_rho, -1 if k_q = -k_rho).  A symmetric momentum set
// (all |k|^2 <= n^2) therefore costs half the tensor-core work of the direct complex
// projection; an asymmetric one costs the same.
//
// A CTA owns one tile of 128 columns (2 noises x 4 "vector" spins x 16 "matrix"
// indices s), one chunk of NH <= 48 representatives and one range of sites:
//
//   warp 0      bulk-copies the phase tiles (FP16 hi/lo of [cos | sin], K-major) into
//               the A/B ring, whose stages the MMA frees
//   warp 22     loads the contraction inputs of each k-step with TMA tensor copies (the
//               propagator or diquark box and the two noises' vector box) into the input
//               ring, whose stages the producers free
//   warp 1      allocates tensor memory and issues the MMAs
//   warps 2-9   drain the accumulator every KD k-steps into an FP32 running sum, which
//               starts again after every group of at most 64 chunks
//   warps 10-21 producers, four per k-step and three k-steps in flight: contract the
//               inputs in FP32, split each value into fp16 hi + lo and write the four A
//               tiles (Ur hi/lo, Ui hi/lo), MN-major
//
// Per k-step (16 sites) the accumulator D (128 x 4NH, FP32, tensor memory) receives
//   D[:, 0:2NH]   += Ur_h [cos|sin]_h + Ur_h [cos|sin]_l + Ur_l [cos|sin]_h
//   D[:, 2NH:4NH] += Ui_h [cos|sin]_h + Ui_h [cos|sin]_l + Ui_l [cos|sin]_h
// (the lo*lo term dropped), i.e. Re C, Re S, Im C, Im S.  Tensor memory accumulation
// truncates, so the products with a lo factor go first within each pair of k-steps, and D
// is double-buffered and drained every KD k-steps into a two-level FP32 sum (a running
// sum over groups of at most 64 chunks, whose group sums add up in tensor memory or, for
// the widest chunks, in the CTA's partial sums in global memory); reduce_f64 adds the
// partials of all CTAs exactly, rounds to FP64 and forms out[q] = C + i sigma_q S.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <memory>
#include <type_traits>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "conv.cuh"
#include "lhc_internal.h"
#include "tc_ptx.cuh"

namespace lhc {
namespace {

constexpr int MT = 128;                  // GEMM M tile: output columns per CTA
constexpr int KSTEP = 16;                // sites per MMA k-step
constexpr int RCHUNK = 48;               // momentum representatives per CTA (tensor memory bounds this)
// one 128 x 16 fp16 operand tile, MN-major with 16 B of padding per 8-row group
// (row groups 144 B apart, the two 8-site k blocks 2304 B apart)
constexpr int ATILE = 2 * 16 * 144;
constexpr int ASTAGE = 4 * ATILE;        // Ur hi, Ur lo, Ui hi, Ui lo
constexpr int NSTAGE = 6;                // A/B ring (freed by the MMA), used as pairs of stages
constexpr int NPAIR = NSTAGE / 2;
constexpr int NIN = 6;                   // input ring (freed by the producers)
constexpr int NPK = 3;                   // k-steps in flight in the producers (4 warps each)
// warp roles: 0 phase-tile loader, 1 MMA issue, 2-9 drain, 10-21 producers, 22 input loader
constexpr int kWarps = 23;
constexpr int kThreads = kWarps * 32;
constexpr int kDrainWarp0 = 2;
constexpr int kMaxGroup = 64;            // drained chunks per running sum before it goes out
constexpr int kProdWarp0 = 10;
constexpr int kInWarp = kProdWarp0 + 4 * NPK;
constexpr uint32_t kTmemCols = 512;

// Threads per block of the staging, maximum and diquark kernels (memory- or
// instruction-bound elementwise work) and of the reduce.
constexpr int kSmallThreads = 256;
constexpr int kReduceThreads = 128;

// K-major, no swizzle: (row, k) -> core matrices of 8 rows x 16 B; 16 k per row block
__host__ __device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
  return (uint32_t)((row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

struct SlicePtrs {
  const void *S;
  const void *vec;
};



// ------------------------------------------------------------ phase table (FP16 split)
// layout [rc][kb][hl][2 NH rows: cos | sin][16 sites], each (rc, kb, hl) block K-major;
// row n < NH holds cos(phi_rho), row NH + n sin(phi_rho) for rho = rc NH + n, with
// phi_rho(x) = 2 pi ((k_rho.(x - r)) mod L) / L taken from the L-entry root table.
__global__ void phase_cs_kernel(__half *out, const int *krep, int nrep, int NH, int nrc, int nkb, int L, int rx,
                                int ry, int rz, const double2 *roots) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int rows = 2 * NH;
  size_t total = (size_t)nrc * nkb * 2 * rows * KSTEP;
  if (idx >= total) return;
  int kk = (int)(idx % KSTEP);
  size_t rest = idx / KSTEP;
  int n = (int)(rest % rows);
  rest /= rows;
  int hl = (int)(rest % 2);
  rest /= 2;
  int kb = (int)(rest % nkb);
  int rc = (int)(rest / nkb);
  int g = n / NH, rho = rc * NH + n % NH;
  int V3 = L * L * L;
  int x = kb * KSTEP + kk;
  double v = 0.0;
  if (rho < nrep && x < V3) {
    int cx = x % L, cy = (x / L) % L, cz = x / (L * L);
    long long m = (long long)krep[3 * rho] * (cx - rx) + (long long)krep[3 * rho + 1] * (cy - ry) +
                  (long long)krep[3 * rho + 2] * (cz - rz);
    m %= L;
    if (m < 0) m += L;
    v = g == 0 ? roots[m].x : roots[m].y;
  }
  __half hi = __double2half(v);
  __half lo = __double2half(v - (double)__half2float(hi));
  size_t block = ((size_t)rc * nkb + kb) * 2 + hl;
  char *base = reinterpret_cast<char *>(out) + block * (size_t)rows * 32;
  *reinterpret_cast<__half *>(base + kmajor_off(n, kk)) = hl ? lo : hi;
}

// ------------------------------------------------------------ fused kernel
constexpr int kMaxSlices = 64;   // slices per launch (time coordinates travel as kernel parameters)

// Tensor maps (built on the host per launch) of the two contraction inputs, both complex64
// viewed as 8-byte elements:
//   tmM  meson/insertion: the propagator as [T][V3][4 bt][3 c][12 ba] (column index
//        (bt*3 + c)*12 + ba of the 144 per site), box [1][16][2][3][12]: 16 sites, two
//        consecutive bt blocks (every 16-column tile lies within two), all colours;
//        baryon: the diquark as [V3][3 c'][768 s], box [16][3][16].
//   tmV  the vector (psi or eta) as [n_r][T][V3][12], box [2][1][16][12]: the tile's two
//        noises on 16 sites (noises past n_r and sites past V3 read as zero).
struct FusedCore {
  CUtensorMap tmM;   // (CUtensorMap carries its own 64-byte alignment)
  CUtensorMap tmV;
  const __half *B;                      // phase table
  // per CTA (slice j, split, chunk rc, tile ct; in that order, ct fastest) a block of
  // [half h][column quad m < NH / 2][row < 128] float4s (columns 4m .. 4m + 3): the
  // thread of (row, h) owns one float4 of every quad, so a warp's accesses are 512-byte
  // runs
  float *partial;
  int *err;
  // per slice of the launch: the largest |re| or |im| of the matrix operand and of the
  // vector operand (as float bits), from which the CTA picks its power-of-two scale
  const unsigned *maxM, *maxV;
  int maxM_per_slice;                   // 1: maxM[j]; 0: maxM[0] for every slice (diquark)
  int n_r, V3, nct, nkb, nrc, nrep, ncols, nsplit, kd, g5mask;
  // batched launches: slice j's time coordinates are (tm0 + j) % tmT, (tv0 + j) % tvT
  // (these fit in the structure's alignment padding)
  int tm0, tmT, tv0, tvT;
  int NH;     // representatives per CTA (a multiple of 8, at most RCHUNK)
  int mode;   // the part: 0 insertion, 1 meson spectator, 2 baryon spectator
};

// One call's launch: the core parameters and, per slice, the time coordinates of its
// matrix and vector boxes in the tensor maps.
struct FusedParams {
  FusedCore c;
  int tM[kMaxSlices], tV[kMaxSlices];
};

// Power-of-two scale of the contracted values before their FP16 split.  Every value is a
// sum over 3 colours of (vector x matrix) products, so |re|, |im| <= 6 mV mM with mV, mM
// the largest real or imaginary parts of the operands.  The scale 2^e puts that bound at
// 2^14: far below the FP16 maximum (65504), and typical values, which lie well below the
// bound, keep their lo parts (2^-11 of the value) out of the FP16 subnormal range.  A bound
// already in [2^6, 2^14] (unit-scale data) is left unscaled (e = 0), which spares the
// producers the multiplications; a lo part that falls subnormal there is off by at most
// 2^-25, below 2^-31 of the bound.  The drain multiplies the sums by 2^-e, which is exact.
__device__ __forceinline__ int split_scale_exp(unsigned mM_bits, unsigned mV_bits) {
  const float b = 6.f * __uint_as_float(mM_bits) * __uint_as_float(mV_bits);
  if (!(b > 0.f) || !(b < 3.0e38f)) return 0;
  int x;
  frexpf(b, &x);   // b = f 2^x, f in [0.5, 1): b <= 2^x
  const int e = 14 - x;
  return e >= 0 && e <= 8 ? 0 : max(-100, min(100, e));
}

// (a0, a1) += (b0, b1) as one packed FP32 instruction: two IEEE round-to-nearest additions,
// bitwise those of two scalar adds, in one issue slot (the drain runs on the same SM
// sub-partitions as the producers, whose instruction issue bounds the kernel)
__device__ __forceinline__ void add2(float &a0, float &a1, float b0, float b1) {
  unsigned long long a, b;
  asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(a0), "f"(a1));
  asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(b0), "f"(b1));
  asm("add.rn.f32x2 %0, %0, %1;" : "+l"(a) : "l"(b));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a0), "=f"(a1) : "l"(a));
}

// Packed FP32 pairs for fma.rn.f32x2: (lo, hi) in one 64-bit register pair.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
// d = a * b + d elementwise on the two FP32 lanes, each rounded once
__device__ __forceinline__ void fma2(unsigned long long &d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

// fp16 hi/lo split of two floats, packed as half2 pairs
__device__ __forceinline__ void split2(float v0, float v1, uint32_t &hi, uint32_t &lo) {
  __half2 h = __floats2half2_rn(v0, v1);
  float2 hf = __half22float2(h);
  __half2 l = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
  hi = *reinterpret_cast<uint32_t *>(&h);
  lo = *reinterpret_cast<uint32_t *>(&l);
}

// Shared memory: NSTAGE stages of the A tiles (Ur hi, Ur lo, Ui hi, Ui lo) and the phase
// tile B (hi and lo of 2 NH rows x 16 sites; room for NH = RCHUNK), then NIN stages of the
// matrix box M and the vector box V.  Every region size is a multiple of 1024 bytes.
template <int MODE>
struct Stage {
  static constexpr int A = ASTAGE;
  static constexpr int B = 2 * 2 * RCHUNK * 32;
  static constexpr int M = MODE == 2 ? 16 * 48 * 8 : 16 * 72 * 8;
  static constexpr int V = 2 * 16 * 12 * 8;
  static constexpr int ab = A + B;
  static constexpr int in = M + V;
  static constexpr int bytes = NSTAGE * ab + NIN * in;
};

// Running-sum columns per half in registers when a chunk has the most representatives
// (NH = RCHUNK): tensor memory holds the two accumulator buffers (8 NH columns) and 64
// columns of each half's running sum.
constexpr int kNRMax = 2 * RCHUNK - (kTmemCols - 8 * RCHUNK) / 2;
static_assert(kNRMax == 32 && (kTmemCols - 8 * RCHUNK) / 2 == 64, "tensor-memory split at the widest chunk");

// The work of one CTA: tile ct (noise pair, 16 matrix columns), site split `split`,
// slice j and representative chunk rc of the call described by p; tm, tv are slice j's
// time coordinates in the tensor maps; tbase is the CTA's tensor memory (all 512 columns,
// allocated by the kernel).  NH is the chunk width (p.NH, compiled in).  Every width uses
// the same shared-memory layout and order of operations.  On return every barrier of the
// body is invalidated, so a persistent CTA can run the body again.
template <typename CT, int MODE, int NH>
__device__ __forceinline__ void fused_body(const FusedCore &p, const int ct, const int split, const int j,
                                           const int rc, const int tm, const int tv, const uint32_t tbase) {
  static_assert(NH % 8 == 0 && NH >= 8 && NH <= RCHUNK, "representative chunk");
  using St = Stage<MODE>;
  // NP accumulator columns per half: [cos | sin] x NH representatives; half 0 takes the
  // products with Ur, half 1 those with Ui.
  const int NP = 2 * NH;
  // tensor memory: D buffers [0, 2NP) and [2NP, 4NP); the rest holds NT columns of each
  // half's running sum (a multiple of 16, at most NP).  Only the widest chunk (NH = 48,
  // NP = 96) leaves columns over: NT = 64, and NR = kNRMax = 32 columns of each half stay
  // in registers.  Narrower chunks keep the whole running sum in tensor memory.
  const int NT = min(((int)kTmemCols - 4 * NP) / 2 / 16 * 16, NP);
  const bool wide = NT < NP;
  const int Bbytes = 2 * 2 * NH * 32;   // the phase tile of one k-step
  extern __shared__ __align__(1024) char smem_raw[];
  // TMA destinations want 128-byte alignment: align the stage ring to 1024 explicitly
  char *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + St::bytes);
  // The A/B stages go in pairs (two k-steps): full[pair] completes when both phase tiles
  // have landed (transaction bytes) and the eight producer warps of the two k-steps have
  // written their A tiles; empty[pair] when the pair's twelve MMAs have completed.  One
  // wait and one commit per two k-steps keeps the MMA thread's gaps short.
  uint64_t *full = bars, *empty = bars + NPAIR, *inFull = bars + 2 * NPAIR, *inEmpty = bars + 2 * NPAIR + NIN,
           *tfull = bars + 2 * NPAIR + 2 * NIN, *tempty = tfull + 2, *done = tfull + 4;
  // Verdicts of waits that one leader thread performs for a group of warps, which block on
  // a named barrier meanwhile: [0, 2) drain (by chunk parity), then four slots per
  // producer group (k-step offset), of which the first two hold the verdict of the
  // joint input and A-stage wait (by iteration parity).
  volatile int *verdict = reinterpret_cast<volatile int *>(done + 1) + 1;
  auto stA = [&](int s) { return smem + s * St::ab; };
  auto stB = [&](int s) { return smem + s * St::ab + St::A; };
  auto stM = [&](int s) { return smem + NSTAGE * St::ab + s * St::in; };
  auto stV = [&](int s) { return smem + NSTAGE * St::ab + s * St::in + St::M; };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sc_e = split_scale_exp(p.maxM[p.maxM_per_slice ? j : 0], p.maxV[j]);
  // site range in k-steps; splits start on even k-steps so producer iterations align
  const int npair = (p.nkb + 1) / 2;
  const int kb0 = 2 * (int)((long long)npair * split / p.nsplit);
  const int kb1 = min(p.nkb, 2 * (int)((long long)npair * (split + 1) / p.nsplit));
  const int nk = kb1 - kb0;
  const int nchunks = (nk + p.kd - 1) / p.kd;
  volatile int *err = p.err;
  // tile = (noise pair, block of 16 matrix columns s), noise pairs fastest so that CTAs
  // sharing the same matrix columns run together (the baryon diquark is reused via L2)
  const int npairs = (p.n_r + 1) / 2;
  const int i0 = 2 * (ct % npairs), s0 = 16 * (ct / npairs);   // first noise and first s of this tile
  const int bt0 = s0 / 12;                                     // first bt block of the matrix box

  if (threadIdx.x == 0) {
    for (int s = 0; s < NPAIR; ++s) {
      tc::mbar_init(&full[s], 10);   // two phase-tile arrivals + the eight producer warps
      tc::mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < NIN; ++s) {
      tc::mbar_init(&inFull[s], 1);
      tc::mbar_init(&inEmpty[s], 4);   // the four producer warps that read a k-step
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 8);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();

  if (warp == 0) {
    // ---------------------------------------------------- phase tiles (A/B ring)
    if (lane == 0 && nk > 0) {
      const char *Bsrc = reinterpret_cast<const char *>(p.B) + ((size_t)rc * p.nkb + kb0) * Bbytes;
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % NSTAGE, pr = s >> 1, u = i / NSTAGE;
        if (u > 0 && !tc::mbar_wait(&empty[pr], (u - 1) & 1, err, 1)) break;
        tc::mbar_arrive_expect_tx(&full[pr], Bbytes);
        tc::bulk_g2s(stB(s), Bsrc + (size_t)i * Bbytes, Bbytes, &full[pr]);
        issued = i + 1;
      }
      for (int i = max(0, issued - NSTAGE); i < issued; i += 2) {   // nothing may still be landing
        const int pr = (i % NSTAGE) >> 1, u = i / NSTAGE;
        long long t0 = clock64();
        while (!tc::mbar_try_wait(&full[pr], u & 1) && clock64() - t0 < tc::kSpinLimit && !*err) {
        }
      }
    }
  } else if (warp == kInWarp) {
    // ---------------------------------------------------- contraction inputs (input ring, TMA)
    if (lane == 0 && nk > 0) {
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % NIN, u = i / NIN;
        if (u > 0 && !tc::mbar_wait(&inEmpty[s], (u - 1) & 1, err, 7)) break;
        const int x0 = 16 * (kb0 + i);
        tc::mbar_arrive_expect_tx(&inFull[s], St::in);
        if (MODE == 2)
          tc::tma_load_3d(stM(s), &p.tmM, s0, 0, x0, &inFull[s]);
        else
          tc::tma_load_5d(stM(s), &p.tmM, 0, 0, bt0, x0, tm, &inFull[s]);
        tc::tma_load_4d(stV(s), &p.tmV, 0, x0, tv, i0, &inFull[s]);
        issued = i + 1;
      }
      for (int i = max(0, issued - NIN); i < issued; ++i) {   // nothing may still be landing
        const int s = i % NIN, u = i / NIN;
        long long t0 = clock64();
        while (!tc::mbar_try_wait(&inFull[s], u & 1) && clock64() - t0 < tc::kSpinLimit) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------- MMA issue
    if (lane == 0 && nk > 0) {
      // A: MN-major (row m = s*8 + noise*4 + spin), core matrices 8 k x 16 B: the 16 row
      // groups s lie 144 B apart (SBO; the 16 B of padding per group keep the producers'
      // stores free of bank conflicts), the two 8-site k blocks 2304 B apart (LBO)
      const uint32_t idesc = tc::idesc_f16(MT, NP) | (1u << 15);
      // Everything between two k-steps' MMAs is on the tensor pipe's critical path (it
      // queues few MMAs), so the loop does no division and builds no descriptor: the
      // descriptors of stage 0 are offset by immediates (the start-address field is
      // bytes / 16 and cannot carry out for shared-memory addresses).
      const uint64_t dA0 = tc::smem_desc(tc::smem_u32(stA(0)), 2304, 144);
      const uint64_t dB0 = tc::smem_desc(tc::smem_u32(stB(0)), 128, 256);
      constexpr uint64_t kStageStep = St::ab >> 4, kATile = ATILE >> 4;
      const uint64_t kBHalf = (uint64_t)(NP * 32) >> 4;
      // k-steps come in pairs (nk is even): stage pair pr holds stages 2 pr and 2 pr + 1
      int i = 0, pr = 0;
      uint32_t ph = 0;   // phase of full[pr] for the pair starting at k-step i
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int b = c & 1, ub = c >> 1;
        // the chunk's accumulator buffer must have been drained (chunk c - 2)
        if (ub > 0 && !tc::mbar_wait(&tempty[b], (ub - 1) & 1, err, 2)) break;
        const uint32_t d = tbase + (uint32_t)(b * 2 * NP);
        const int iend = min(nk, (c + 1) * p.kd);
        for (uint32_t acc0 = 0; i < iend; i += 2, acc0 = 1) {
          if (!tc::mbar_wait(&full[pr], ph, err, 3)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          // Per half (Ur: columns [0, NP), Ui: [NP, 2NP)) the products with one lo factor
          // of both k-steps come first and the hi x hi products last.  Every MMA
          // truncates the accumulator, by up to one unit in its last place; the small
          // products then meet a small accumulator at the start of a chunk, so a drain
          // interval of two k-steps takes two full-size truncations instead of six.
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            const uint32_t dd = d + part * NP;
            const uint64_t ah = dA0 + 2 * part * kATile, al = ah + kATile;   // U hi, U lo of stage 0
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const uint64_t so = (2 * pr + h) * kStageStep;
              tc::mma_f16(dd, ah + so, dB0 + so + kBHalf, idesc, h ? 1u : acc0);   // U_h [cos|sin]_l
              tc::mma_f16(dd, al + so, dB0 + so, idesc, 1u);                       // U_l [cos|sin]_h
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const uint64_t so = (2 * pr + h) * kStageStep;
              tc::mma_f16(dd, ah + so, dB0 + so, idesc, 1u);                       // U_h [cos|sin]_h
            }
          }
          tc::mma_commit(&empty[pr]);
          if (++pr == NPAIR) {
            pr = 0;
            ph ^= 1u;
          }
        }
        tc::mma_commit(&tfull[b]);
      }
      tc::mma_commit(done);
      long long t0 = clock64();
      while (!tc::mbar_try_wait(done, 0) && clock64() - t0 < tc::kSpinLimit) {
      }
    }
  } else if (warp < kProdWarp0) {
    // ---------------------------------------------------- drain (quadrant = warp % 4)
    const int qd = warp & 3, h = (warp - kDrainWarp0) >> 2;
    const int row = qd * 32 + lane;
    const uint32_t lane_base = tbase + ((uint32_t)(qd * 32) << 16);
    const uint32_t rsum = lane_base + (uint32_t)(4 * NP + h * NT);   // this half's running sum in TMEM
    // Two-level sum over the CTA's chunks.  The running sum takes up to kMaxGroup chunks
    // (the chunks split into equal groups) and restarts; the group sums add up in tensor
    // memory or in the CTA's block of partial sums in global memory.  A long site range
    // (a 48^3 slice split 8 ways has 432 chunks of 2 k-steps per CTA) would otherwise add
    // FP32 roundings of a growing sum above the tensor-memory truncation; shorter ranges
    // (up to 64 chunks) make one group.  The group length is recomputed where needed
    // (one register fewer across the chunk loop).
    auto ngrp = [&]() {
      const int ng = (nchunks + kMaxGroup - 1) / kMaxGroup;
      return (nchunks + ng - 1) / max(ng, 1);
    };
    // Chunks of at most 32 representatives (NP <= 64) leave tensor-memory columns for the
    // second level as well: the group sums of this half, NT columns after both running
    // sums.  Wider chunks add each group into global memory.
    constexpr bool kGroupInTmem = 8 * 2 * NH <= (int)kTmemCols;
    const uint32_t gsum = rsum + (uint32_t)(2 * NT);
    float acc[kNRMax];   // columns NT .. NP - 1 of the running sum (widest chunk only)
#pragma unroll
    for (int n = 0; n < kNRMax; ++n) acc[n] = 0.f;
    // tcgen05.ld is warp-collective: every lane executes it and stores its own row
    auto flush = [&](bool first, bool last) {
      // this thread's row of the block (computed here so that none of it stays live
      // across the chunk loop; the empty asm keeps the compiler from hoisting it)
      int rw = row;
      asm volatile("" : "+r"(rw));
      // gamma5 signs of this row: g5(v) for the insertion and the baryon spectator,
      // g5(v) g5(bt) g5(b) for the meson spectator (s = bt*12 + b*3 + a), row = (s - s0)*8
      // + noise*4 + v; the projection is linear, so they act on the finished sums
      const int v = rw & 3, sidx = s0 + (rw >> 3);
      const int smask = MODE != 1 ? (p.g5mask >> v)
                                  : ((p.g5mask >> v) ^ (p.g5mask >> (sidx / 12)) ^ (p.g5mask >> ((sidx % 12) / 3)));
      const float sgn = ldexpf((smask & 1) ? -1.f : 1.f, -sc_e);   // the sign and the inverse split scale
      // column quad m (columns 4m .. 4m + 3) of this half at out[m * MT]
      float4 *out = reinterpret_cast<float4 *>(p.partial) +
                    ((((size_t)j * p.nsplit + split) * p.nrc + rc) * p.nct + ct) * (NH * MT) + (size_t)h * (NH / 2) * MT +
                    rw;
      if constexpr (kGroupInTmem) {
        // the group sums add up in tensor memory; only the last group writes, once
#pragma unroll 1
        for (int n0 = 0; n0 < NT; n0 += 8) {
          float r[8], g[8];
          tc::tmem_ld8(rsum + n0, r);
          if (!first) tc::tmem_ld8(gsum + n0, g);
          tc::tmem_wait_ld();
          if (!first)
#pragma unroll
            for (int e = 0; e < 8; e += 2) add2(r[e], r[e + 1], g[e], g[e + 1]);
          if (last) {
#pragma unroll
            for (int e = 0; e < 8; e += 4)
              out[(size_t)(n0 + e) / 4 * MT] = make_float4(sgn * r[e], sgn * r[e + 1], sgn * r[e + 2], sgn * r[e + 3]);
          } else {
            tc::tmem_st8(gsum + n0, r);
          }
        }
        if (!last) tc::tmem_wait_st();
      } else {
        // the first group stores; later groups add with fire-and-forget vector reductions
        // (one thread per address, so they apply in program order: the sum is
        // deterministic)
        auto put = [&](int m, float x0, float x1, float x2, float x3) {
          const float4 x = make_float4(sgn * x0, sgn * x1, sgn * x2, sgn * x3);
          if (first)
            out[(size_t)m * MT] = x;
          else
            atomicAdd(out + (size_t)m * MT, x);
        };
#pragma unroll 1
        for (int n0 = 0; n0 < NT; n0 += 16) {
          float r[16];
          tc::tmem_ld16(rsum + n0, r);
          tc::tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 16; e += 4) put((n0 + e) / 4, r[e], r[e + 1], r[e + 2], r[e + 3]);
        }
        if (wide) {   // NP - NT == kNRMax
#pragma unroll
          for (int e = 0; e < kNRMax; e += 4) {
            put((NT + e) / 4, acc[e], acc[e + 1], acc[e + 2], acc[e + 3]);
            acc[e] = acc[e + 1] = acc[e + 2] = acc[e + 3] = 0.f;
          }
        }
      }
    };
    bool ok = true;
    for (int c0 = 0; c0 < nchunks && ok; c0 += ngrp()) {
     const int c1 = min(nchunks, c0 + ngrp());
     for (int c = c0; c < c1; ++c) {
      int b = c & 1, ub = c >> 1;
      const bool restart = c == c0;   // the chunk opens a group: it replaces the running sum
      // one thread waits, the eight drain warps block on named barrier 1 and follow its
      // verdict together (the tensor-memory loads below are warp-collective and must
      // never see a split warp; every drain warp reaches the barrier in every chunk)
      if (warp == kDrainWarp0 && lane == 0) verdict[b] = tc::mbar_wait(&tfull[b], ub & 1, err, 5) ? 1 : 0;
      tc::named_bar_sync(1, 256);
      if (!verdict[b]) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
      const uint32_t t = lane_base + (uint32_t)(b * 2 * NP + h * NP);
#pragma unroll
      for (int n0 = 0; n0 < 2 * RCHUNK; n0 += 16) {
        if (n0 >= NP) break;   // uniform over the CTA
        float v[16];
        tc::tmem_ld16(t + n0, v);
        if (n0 < NT) {
          float r[16];
          if (!restart) tc::tmem_ld16(rsum + n0, r);
          tc::tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 16; e += 2) {
            if (!restart) {
              add2(r[e], r[e + 1], v[e], v[e + 1]);
            } else {
              r[e] = v[e];
              r[e + 1] = v[e + 1];
            }
          }
          tc::tmem_st16(rsum + n0, r);
        } else if (n0 >= 2 * RCHUNK - kNRMax) {   // register part (NT = 2 RCHUNK - kNRMax here)
          tc::tmem_wait_ld();
          constexpr int kNT = 2 * RCHUNK - kNRMax;
#pragma unroll
          for (int e = 0; e < 16; e += 2) add2(acc[n0 - kNT + e], acc[n0 - kNT + e + 1], v[e], v[e + 1]);
        }
      }
      tc::tmem_wait_st();
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[b]);
     }
     // the buffer is free again: the group's sum goes out while the next chunk accumulates
     if (ok) flush(c0 == 0, c1 == nchunks);
    }
  } else {
    // ---------------------------------------------------- producers
    // Producer warp pw computes k-step kofs of every NPK k-steps for 4 of its 16 sites
    // (quarter wq), all 128 rows (s, noise, spin): lane = (column sp in 0..7, site
    // xq in 0..3) handles the columns s = sp and sp + 8 for 8 (noise, spin) rows.  A
    // quarter-warp holds 8 consecutive columns of one site, so its 16-byte A-tile stores
    // land 144 B apart (distinct banks) and its matrix reads are contiguous.
    const int pw = warp - kProdWarp0;                    // 0 .. 4 NPK - 1
    const int kofs = pw >> 2, wq = pw & 3;
    const int sp = lane & 7, x = 4 * wq + (lane >> 3);   // column and site within the k-step
    const int nit = (nk + NPK - 1) / NPK;
    const float sc = ldexpf(1.f, sc_e);
    // matrix-box offsets of this lane's two columns (colour 0; colour c adds c*12 or c*16)
    int mo[2];
#pragma unroll
    for (int jx = 0; jx < 2; ++jx) {
      const int sv = s0 + sp + 8 * jx;
      mo[jx] = MODE == 2 ? x * 48 + sp + 8 * jx : ((x * 2 + (sv / 12 - bt0)) * 3) * 12 + sv % 12;
    }
    static_assert(NIN == 2 * NPK && NSTAGE == 2 * NPK, "stage indices from the iteration count");
    // The loop is compiled twice: with the split scale and, for unit-scale data (e = 0),
    // without its multiplications.
    auto produce = [&](auto scaled) {
      for (int it = 0; it < nit; ++it) {
        const int kstep = NPK * it + kofs;
        if (kstep >= nk) break;
        // k-step kstep = NPK it + kofs uses input stage and A stage kstep % 6 = kofs + 3 (it & 1),
        // in round kstep / 6 = it / 2
        const int si = kofs + NPK * (it & 1), ui = it >> 1;
        // The first warp of the group waits for the input stage and, after the first round,
        // for the MMA to be done with the A stage (its k-step NSTAGE back); the four warps
        // block on the group's named barrier and follow its verdict together, so a wait
        // that gives up (a loader stopped, or the limit ran out) ends the loop of all four
        // at once.
        volatile int *vin = verdict + 2 + 4 * kofs;
        const int pr = si >> 1;
        if (wq == 0 && lane == 0)
          vin[it & 1] = (tc::mbar_wait(&inFull[si], ui & 1, err, 6) &&
                         (ui == 0 || tc::mbar_wait(&empty[pr], (ui - 1) & 1, err, 8)))
                            ? 1
                            : 0;
        tc::named_bar_sync(2 + kofs, 128);
        if (!vin[it & 1]) break;
        const float2 *Ms = reinterpret_cast<const float2 *>(stM(si));
        const float2 *Vs = reinterpret_cast<const float2 *>(stV(si)) + x * 12;
        char *a_st = stA(si);
        // One column at a time.  The colour sum of each (noise, spin) row runs on packed
        // FP32 pairs: with the vector value p in its natural pair (p.x, p.y) and the
        // matrix value m,
        //   A += p * (m.x, ±m.x),  B += p * (±m.y, ±m.y),  Re = A.x + B.y,  Im = A.y + B.x.
        // The one minus sign sits in A.y for conj(psi) S, in B.x for eta conj(S) and in
        // B.y for eta D.  The matrix pairs are formed once per column and k-step (and carry
        // the split scale); each accumulator sums the colours in the order 0, 1, 2.
  #pragma unroll
        for (int jx = 0; jx < 2; ++jx) {
          unsigned long long ma[3], mb[3];
  #pragma unroll
          for (int c = 0; c < 3; ++c) {
            float2 m = Ms[mo[jx] + c * (MODE == 2 ? 16 : 12)];
            if constexpr (decltype(scaled)::value) m = make_float2(m.x * sc, m.y * sc);
            ma[c] = pack2(m.x, MODE == 0 ? -m.x : m.x);
            mb[c] = MODE == 1 ? pack2(-m.y, m.y) : pack2(m.y, MODE == 2 ? -m.y : m.y);
          }
          unsigned long long A[8], B[8];
  #pragma unroll
          for (int iv = 0; iv < 8; ++iv) A[iv] = B[iv] = 0ull;
          // the four spins of one noise at a time (rows iv .. iv + 3): the colour step c of
          // all eight accumulators is issued together, so eight independent FMAs separate
          // two steps of one accumulator chain (the order of each chain is unchanged)
  #pragma unroll
          for (int i4 = 0; i4 < 8; i4 += 4) {
            unsigned long long pv[4][3];
  #pragma unroll
            for (int r = 0; r < 4; ++r) {
              // noise (i4 + r) / 4, spin r: the three colours with one 16-byte and one 8-byte load
              const unsigned long long *pb =
                  reinterpret_cast<const unsigned long long *>(Vs + (i4 >> 2) * 16 * 12 + r * 3);
              if ((r & 1) == 0) {   // colours 0, 1 start on a 16-byte boundary
                const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(pb);
                pv[r][0] = q.x;
                pv[r][1] = q.y;
                pv[r][2] = pb[2];
              } else {              // colours 1, 2 do
                pv[r][0] = pb[0];
                const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(pb + 1);
                pv[r][1] = q.x;
                pv[r][2] = q.y;
              }
            }
  #pragma unroll
            for (int c = 0; c < 3; ++c) {
  #pragma unroll
              for (int r = 0; r < 4; ++r) fma2(A[i4 + r], pv[r][c], ma[c]);
  #pragma unroll
              for (int r = 0; r < 4; ++r) fma2(B[i4 + r], pv[r][c], mb[c]);
            }
          }
          if (jx == 1) {   // the input stage is read: hand it back to the input loader
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&inEmpty[si]);
          }
          uint32_t rh[4], rl[4], ih[4], il[4];
  #pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 a0 = unpack2(A[2 * q]), b0 = unpack2(B[2 * q]);
            const float2 a1 = unpack2(A[2 * q + 1]), b1 = unpack2(B[2 * q + 1]);
            split2(a0.x + b0.y, a1.x + b1.y, rh[q], rl[q]);
            split2(a0.y + b0.x, a1.y + b1.x, ih[q], il[q]);
          }
          // row group s = sp + 8 jx, its 8 rows (noise, spin) contiguous at k = site x
          const uint32_t off = (uint32_t)((sp + 8 * jx) * 144 + (x >> 3) * 2304 + (x & 7) * 16);
          *reinterpret_cast<uint4 *>(a_st + 0 * ATILE + off) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
          *reinterpret_cast<uint4 *>(a_st + 1 * ATILE + off) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
          *reinterpret_cast<uint4 *>(a_st + 2 * ATILE + off) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
          *reinterpret_cast<uint4 *>(a_st + 3 * ATILE + off) = make_uint4(il[0], il[1], il[2], il[3]);
        }
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&full[pr]);
      }
    };
    if (sc_e == 0)
      produce(std::false_type{});
    else
      produce(std::true_type{});
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  // every copy has landed and every MMA has completed (the loaders and the MMA thread
  // waited for that): nothing arrives on the barriers any more
  if (threadIdx.x == 0)
    for (uint64_t *b = bars; b <= done; ++b) tc::mbar_inval(b);
}

// Tensor memory for the whole CTA: warp 1 allocates all 512 columns (one CTA per SM) and
// gives up the right to allocate again; the address reaches every thread through shared
// memory.
__device__ __forceinline__ uint32_t cta_tmem_alloc(uint32_t *slot) {
  if ((threadIdx.x >> 5) == 1) tc::tmem_alloc(slot, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  return *slot;
}

template <typename CT, int MODE, int NH>
__global__ void __launch_bounds__(kThreads, 1) fused_meson(const __grid_constant__ FusedParams p) {
  __shared__ uint32_t tslot;
  const uint32_t tbase = cta_tmem_alloc(&tslot);
  const int j = blockIdx.z / p.c.nrc, rc = blockIdx.z % p.c.nrc;
  fused_body<CT, MODE, NH>(p.c, blockIdx.x, blockIdx.y, j, rc, p.tM[j], p.tV[j], tbase);
  if ((threadIdx.x >> 5) == 1) tc::tmem_dealloc(tbase, kTmemCols);
}

// Many calls in one persistent launch.  The parameters of up to kMaxBatch calls of one part
// kind and chunk width travel in the kernel's parameter space (a captured graph keeps
// them), and every call's work is numbered as tasks (tile, site split, slice,
// representative chunk), call c owning tasks first[c] .. first[c+1]-1.  One CTA per SM
// takes the next task from a device counter (an atomic add, no waiting) until none is
// left, so an SM that finishes a short task takes the next one at once.  Each task does
// exactly what the CTA with its coordinates does in its call's own launch.  (The width is
// a compile-time parameter: a kernel body that handles several widths, by a runtime
// width or by a switch over compiled widths, needs more than the 80 registers a thread
// has and spills, and measured slower than the calls one by one.)
constexpr int kMaxBatch = 64;
struct BatchParams {
  FusedCore item[kMaxBatch];
  int first[kMaxBatch + 1];
  int n;
  int *cursor;   // the next task; set to zero before the launch
};
static_assert(sizeof(BatchParams) <= 32764, "kernel parameter space");

template <typename CT, int MODE, int NH>
__global__ void __launch_bounds__(kThreads, 1) fused_persistent(const __grid_constant__ BatchParams b) {
  __shared__ int next;
  __shared__ uint32_t tslot;
  const uint32_t tbase = cta_tmem_alloc(&tslot);   // once: the permit to allocate is given up
  const int ntasks = b.first[b.n];
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(b.cursor, 1);
    __syncthreads();
    const int task = next;
    __syncthreads();   // every thread has read the task before thread 0 takes another
    if (task >= ntasks) break;
    int lo = 0, hi = b.n;   // the call: first[lo] <= task < first[lo + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (b.first[mid] <= task)
        lo = mid;
      else
        hi = mid;
    }
    const FusedCore &it = b.item[lo];
    int local = task - b.first[lo];
    const int ct = local % it.nct;
    local /= it.nct;
    const int split = local % it.nsplit;
    local /= it.nsplit;
    const int j = local / it.nrc, rc = local % it.nrc;
    const int tm = (it.tm0 + j) % it.tmT, tv = (it.tv0 + j) % it.tvT;
    fused_body<CT, MODE, NH>(it, ct, split, j, rc, tm, tv, tbase);
  }
  if ((threadIdx.x >> 5) == 1) tc::tmem_dealloc(tbase, kTmemCols);
}

// out[j][q][col] = sum over splits of the FP32 partials.  The partials are added without
// error (Knuth's TwoSum keeps the exact sum as an unevaluated FP32 pair hi + lo) and the
// pair is rounded once to FP64: no less accurate than FP64 accumulation of the partials,
// with a few FP64 operations per output instead of two per partial.
__device__ __forceinline__ void two_sum(float &hi, float &lo, float v) {
  float s = hi + v;
  float bp = s - hi;
  float e = (hi - (s - bp)) + (v - bp);
  hi = s;
  lo += e;
}

// One thread per (slice j, chunk rc, tile ct, quad m of representatives of the chunk,
// row of the tile), rows fastest, so that the float4 loads of the CTA blocks are 512-byte
// runs: for each representative rho = rc NH + 4m + i (i < 4) the four sums (Re C, Re S,
// Im C, Im S) over the site splits are each kept exactly as an unevaluated FP32 pair
// (TwoSum).  The row is the output column col of noise i0 + ii, spin v and matrix index
// s0 + sl (row = sl*8 + ii*4 + v; meson col = (noise, v, s), baryon col = (noise,
// alpha = s/3, beta' = v, c = s%3)); rows of a missing second noise and representatives
// past the last are skipped.  Every requested momentum q of rho (rep_q[rep_first[rho]
// ..], entry 2 q + 1 when k_q = -k_rho) receives out[j][q][col] = C + i sigma_q S with
// sigma_q = sign * (+1 or -1): Re = Re C - sigma Im S and Im = Im C + sigma Re S are
// formed as FP32 pairs too (TwoSum of the leading parts, the trailing parts added), and
// each pair is rounded once to FP64 with one FP64 addition; the FP64 pipe of GB300 does
// nothing else here.
struct ReduceArgs {
  const float *part;
  size_t per_split;   // floats per site split of a slice (nrc * nct blocks of 4 NH * MT)
  const int *rep_first, *rep_q;
  double2 *out;
  size_t out_stride;  // between slices
  int nsplit, nrep, sign, ncols, nt, nrc, nct, NH, n_r, mode;
};

__global__ void __launch_bounds__(kReduceThreads) reduce_f64(const ReduceArgs a) {
  const int nm = a.NH / 4;
  const size_t n_in = (size_t)a.nrc * a.nct * nm * MT;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_in * a.nt) return;
  const int j = (int)(idx / n_in);
  size_t e = idx % n_in;
  const int row = (int)(e % MT);
  e /= MT;
  const int m = (int)(e % nm);
  e /= nm;
  const int ct = (int)(e % a.nct), rc = (int)(e / a.nct);
  const int rg0 = rc * a.NH + 4 * m;
  const int npairs = (a.n_r + 1) / 2;
  const int noise = 2 * (ct % npairs) + ((row >> 2) & 1), sidx = 16 * (ct / npairs) + (row >> 3), v = row & 3;
  if (rg0 >= a.nrep || noise >= a.n_r) return;
  const int col = a.mode == 2 ? noise * 3072 + (sidx / 3) * 12 + v * 3 + sidx % 3 : noise * 192 + v * 48 + sidx;
  // quads of the block: Re C at m, Re S at NH/4 + m (half 0), Im C at NH/2 + m, Im S at
  // 3NH/4 + m (half 1)
  const float4 *pj = reinterpret_cast<const float4 *>(a.part + (size_t)j * a.nsplit * a.per_split) +
                     ((size_t)rc * a.nct + ct) * (a.NH * MT) + (size_t)m * MT + row;
  const size_t o1 = (size_t)nm * MT, o2 = 2 * o1, o3 = 3 * o1, sp = a.per_split / 4;
  float h[4][4], l[4][4];   // [component][representative of the quad]
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int i = 0; i < 4; ++i) h[c][i] = l[c][i] = 0.f;
  // the four loads of a split are in flight together (the order of the sums is fixed)
#pragma unroll 1
  for (int s = 0; s < a.nsplit; ++s) {
    const float4 *q = pj + (size_t)s * sp;
    const float4 x[4] = {__ldcs(q), __ldcs(q + o1), __ldcs(q + o2), __ldcs(q + o3)};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      two_sum(h[c][0], l[c][0], x[c].x);
      two_sum(h[c][1], l[c][1], x[c].y);
      two_sum(h[c][2], l[c][2], x[c].z);
      two_sum(h[c][3], l[c][3], x[c].w);
    }
  }
  double2 *oj = a.out + (size_t)j * a.out_stride + col;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rg = rg0 + i;
    if (rg >= a.nrep) break;
    for (int u = __ldg(a.rep_first + rg), u1 = __ldg(a.rep_first + rg + 1); u < u1; ++u) {
      const int qe = __ldg(a.rep_q + u);
      const float sg = (qe & 1) ? -(float)a.sign : (float)a.sign;
      // Re = (h0 + l0) - sg (h3 + l3), Im = (h2 + l2) + sg (h1 + l1): sg = +-1 is exact
      float rh = h[0][i], rl = l[0][i] - sg * l[3][i], ih = h[2][i], il = l[2][i] + sg * l[1][i];
      two_sum(rh, rl, -sg * h[3][i]);
      two_sum(ih, il, sg * h[1][i]);
      oj[(size_t)(qe >> 1) * a.ncols] =
          make_double2(f32_to_f64(rh) + f32_to_f64(rl), f32_to_f64(ih) + f32_to_f64(il));
    }
  }
}

template <int MODE>
constexpr size_t fused_smem() {
  // rings + barriers + tensor-memory slot + up to 1023 B to align the rings
  return (size_t)Stage<MODE>::bytes + (2 * NPAIR + 2 * NIN + 5) * 8 + 16 + 4 * (2 + 4 * NPK) + 1024;
}
static_assert(fused_smem<0>() <= 232448 && fused_smem<1>() <= 232448 && fused_smem<2>() <= 232448,
              "shared memory per CTA");

// One call's fused launch, compiled for its chunk width; the shared memory (over 120 KB)
// keeps one CTA per SM, which the whole-tensor-memory allocation needs.
template <int MODE, int NH>
int launch_fused_t(const FusedParams &p, int nt, cudaStream_t st) {
  constexpr size_t smem = fused_smem<MODE>();
  static_assert(smem > 120 * 1024, "one CTA per SM");
  static std::atomic<unsigned long long> done{0};
  LHC_TRY(ensure_smem_limit(fused_meson<float2, MODE, NH>, (int)smem, done));
  dim3 grid(p.c.nct, p.c.nsplit, nt * p.c.nrc);
  fused_meson<float2, MODE, NH><<<grid, kThreads, smem, st>>>(p);
  note_launch();
  return LHC_OK;
}

template <int MODE>
int launch_fused(const FusedParams &p, int nt, cudaStream_t st) {
  switch (p.c.NH) {
    case 8: return launch_fused_t<MODE, 8>(p, nt, st);
    case 16: return launch_fused_t<MODE, 16>(p, nt, st);
    case 24: return launch_fused_t<MODE, 24>(p, nt, st);
    case 32: return launch_fused_t<MODE, 32>(p, nt, st);
    case 40: return launch_fused_t<MODE, 40>(p, nt, st);
    case 48: return launch_fused_t<MODE, 48>(p, nt, st);
    default: set_error("unsupported representative chunk %d", p.c.NH); return LHC_EINVAL;
  }
}

template <int MODE, int NH>
int launch_persistent_t(const BatchParams &b, int nctas, cudaStream_t st) {
  constexpr size_t smem = fused_smem<MODE>();
  static std::atomic<unsigned long long> done{0};
  LHC_TRY(ensure_smem_limit(fused_persistent<float2, MODE, NH>, (int)smem, done));
  fused_persistent<float2, MODE, NH><<<nctas, kThreads, smem, st>>>(b);
  note_launch();
  return LHC_OK;
}

template <int MODE>
int launch_persistent(int NH, const BatchParams &b, int nctas, cudaStream_t st) {
  switch (NH) {
    case 8: return launch_persistent_t<MODE, 8>(b, nctas, st);
    case 16: return launch_persistent_t<MODE, 16>(b, nctas, st);
    case 24: return launch_persistent_t<MODE, 24>(b, nctas, st);
    case 32: return launch_persistent_t<MODE, 32>(b, nctas, st);
    case 40: return launch_persistent_t<MODE, 40>(b, nctas, st);
    case 48: return launch_persistent_t<MODE, 48>(b, nctas, st);
    default: set_error("unsupported representative chunk %d", NH); return LHC_EINVAL;
  }
}

// number of site splits: fill whole waves of one CTA per SM as well as possible
int choose_nsplit(int base_ctas, int nk_pairs, int sms) {
  int best = 1;
  double best_eff = 0.0;
  for (int s = 1; s <= 8 && s <= std::max(1, nk_pairs / 2); ++s) {
    long long w = (long long)base_ctas * s;
    long long waves = (w + sms - 1) / sms;
    double eff = (double)w / (double)(waves * sms);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = s;
    }
  }
  return best;
}

// complex128 -> complex64 staging of the slices one launch touches: propagator slices
// to Sst[j][V3*144], noise vectors to Vst[i][j][V3*12] (the contraction runs in FP32)
struct NarrowParams {
  SlicePtrs slices[kMaxSlices];
  const void *SB;      // baryon: second propagator slice (one slice), else nullptr
  size_t vec_stride;   // source elements between noises
  float2 *Sst, *SBst, *Vst;
  unsigned *maxS, *maxV;   // per slice: largest |re| or |im| of the propagator and of the vectors
  int nb, V3;
  int withS;           // 0: the propagator slices are staged already (only the vectors here)
};

// Largest |re| or |im| over a block's values, folded into *m with an atomic max on the
// float bits (non-negative floats order like their bit patterns).
__device__ __forceinline__ void block_max_to(unsigned *m, float v) {
  __shared__ float wmax[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0 && m) atomicMax(m, __float_as_uint(v));
  }
}

// One block per chunk of 1024 complex numbers of one part (propagator slices first, then
// the second baryon propagator, then the noise vectors noise-major); every thread issues
// its four 16-byte loads before converting, so each SM keeps many loads in flight.  The
// conversion is the integer one (f64_to_f32_rne): with the hardware conversion this
// copy is bound by the FP64 pipe.
constexpr int kNarrowChunk = 4 * kSmallThreads;
__global__ void __launch_bounds__(kSmallThreads) narrow_c128(NarrowParams p) {
  const size_t nS = (size_t)p.V3 * 144, nV = (size_t)p.V3 * 12;
  const size_t cS = (nS + kNarrowChunk - 1) / kNarrowChunk, cV = (nV + kNarrowChunk - 1) / kNarrowChunk;
  size_t b = blockIdx.x;
  const double2 *src;
  float2 *dst;
  size_t n;
  unsigned *mx;
  const size_t nSb = p.withS ? (size_t)p.nb * cS : 0;
  if (b < nSb) {
    const int j = (int)(b / cS);
    src = static_cast<const double2 *>(p.slices[j].S);
    dst = p.Sst + (size_t)j * nS;
    n = nS;
    b %= cS;
    mx = p.maxS + j;
  } else if (p.SB && b < nSb + cS) {
    src = static_cast<const double2 *>(p.SB);
    dst = p.SBst;
    n = nS;
    b -= nSb;
    mx = nullptr;   // the baryon's matrix operand is the diquark, bounded separately
  } else {
    b -= nSb + (p.SB ? cS : 0);
    const size_t iv = b / cV;   // noise * nb + slice
    const int i = (int)(iv / p.nb), j = (int)(iv % p.nb);
    src = static_cast<const double2 *>(p.slices[j].vec) + (size_t)i * p.vec_stride;
    dst = p.Vst + iv * nV;
    n = nV;
    b %= cV;
    mx = p.maxV + j;
  }
  const size_t e0 = b * kNarrowChunk + threadIdx.x;
  double2 v[4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (e0 + u * kSmallThreads < n) v[u] = __ldcs(src + e0 + u * kSmallThreads);
  float m = 0.f;
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (e0 + u * kSmallThreads < n) {
      const float2 w = make_float2(f64_to_f32_rne(v[u].x), f64_to_f32_rne(v[u].y));
      dst[e0 + u * kSmallThreads] = w;
      m = fmaxf(m, fmaxf(fabsf(w.x), fabsf(w.y)));
    }
  block_max_to(mx, m);
}

// The same per-slice maxima for complex64 inputs, which are read in place (no copy).
struct MaxParams {
  SlicePtrs slices[kMaxSlices];
  size_t vec_stride;
  unsigned *maxS, *maxV;
  int nb, V3, n_r, with_S;
};

__global__ void __launch_bounds__(kSmallThreads) max_c64(MaxParams p) {
  const size_t nS = (size_t)p.V3 * 144, nV = (size_t)p.V3 * 12;
  const size_t cS = (nS + kNarrowChunk - 1) / kNarrowChunk, cV = (nV + kNarrowChunk - 1) / kNarrowChunk;
  size_t b = blockIdx.x;
  const float4 *src;   // two complex64 per float4 (sizes are multiples of 2 complex numbers)
  size_t n;
  unsigned *mx;
  const size_t nSb = p.with_S ? (size_t)p.nb * cS : 0;
  if (b < nSb) {
    const int j = (int)(b / cS);
    src = static_cast<const float4 *>(p.slices[j].S);
    n = nS / 2;
    b %= cS;
    mx = p.maxS + j;
  } else {
    b -= nSb;
    const size_t iv = b / cV;
    const int i = (int)(iv / p.nb), j = (int)(iv % p.nb);
    src = reinterpret_cast<const float4 *>(static_cast<const float2 *>(p.slices[j].vec) + (size_t)i * p.vec_stride);
    n = nV / 2;
    b %= cV;
    mx = p.maxV + j;
  }
  const size_t e0 = b * (kNarrowChunk / 2) + threadIdx.x;
  float m = 0.f;
#pragma unroll
  for (int u = 0; u < 2; ++u)
    if (e0 + u * kSmallThreads < n) {
      const float4 w = __ldcs(src + e0 + u * kSmallThreads);
      m = fmaxf(m, fmaxf(fmaxf(fabsf(w.x), fabsf(w.y)), fmaxf(fabsf(w.z), fabsf(w.w))));
    }
  block_max_to(mx, m);
}

// Noise-independent baryon diquark, FP32: D[x][c'][(alpha, c)] with
// alpha = ((a1p*4 + a1)*4 + a2p)*4 + a2 and D = sum eps_{a'b'c'} eps_{abc} GA[(a1p,a'),(a1,a)] GB[(a2p,b'),(a2,b)];
// with p = c'+1, q = c'+2, u = c+1, v = c+2 (mod 3) the four nonzero terms are
// GA[p,u]GB[q,v] - GA[p,v]GB[q,u] - GA[q,u]GB[p,v] + GA[q,v]GB[p,u].
// One CTA per site: the two 12x12 propagators are staged in shared memory.
__global__ void __launch_bounds__(kSmallThreads)
    baryon_diquark(const float2 *__restrict__ GA, const float2 *__restrict__ GB, int V3, float2 *__restrict__ D,
                   unsigned *maxD) {
  __shared__ float2 a[144], bm[144];
  const int x = blockIdx.x;
  for (int e = threadIdx.x; e < 144; e += kSmallThreads) {
    a[e] = GA[(size_t)x * 144 + e];
    bm[e] = GB[(size_t)x * 144 + e];
  }
  __syncthreads();
  float2 *out = D + (size_t)x * 2304;
  float m = 0.f;   // largest |re| or |im| of D (the bound of the fused kernel's split scale)
  for (int e = threadIdx.x; e < 2304; e += kSmallThreads) {
    const int cp = e / 768, sidx = e % 768, c = sidx % 3, al = sidx / 3;
    const int a2 = al & 3, a2p = (al >> 2) & 3, a1 = (al >> 4) & 3, a1p = al >> 6;
    const int pp = (cp + 1) % 3, qq = (cp + 2) % 3, u = (c + 1) % 3, v = (c + 2) % 3;
    auto A = [&](int r, int s2) { return a[(a1p * 3 + r) * 12 + a1 * 3 + s2]; };
    auto B = [&](int r, int s2) { return bm[(a2p * 3 + r) * 12 + a2 * 3 + s2]; };
    auto mul = [](float2 x1, float2 y1) { return make_float2(x1.x * y1.x - x1.y * y1.y, x1.x * y1.y + x1.y * y1.x); };
    float2 t1 = mul(A(pp, u), B(qq, v)), t2 = mul(A(pp, v), B(qq, u)), t3 = mul(A(qq, u), B(pp, v)),
           t4 = mul(A(qq, v), B(pp, u));
    const float2 d = make_float2(t1.x - t2.x - t3.x + t4.x, t1.y - t2.y - t3.y + t4.y);
    out[e] = d;
    m = fmaxf(m, fmaxf(fabsf(d.x), fabsf(d.y)));
  }
  block_max_to(maxD, m);
}

}  // namespace

// Representatives of a momentum list: one k_rho per pair {k, -k} (the lexicographically
// larger of the two), in order of first appearance.  The momenta of representative rho
// are q_list[first[rho] .. first[rho + 1]), each entry 2 q + (1 if k_q = -k_rho).
struct MomentumReps {
  std::vector<int> k;       // [nrep][3]
  std::vector<int> first;   // [nrep + 1]
  std::vector<int> q_list;  // [nq]
  int nrep() const { return (int)k.size() / 3; }
};

static MomentumReps momentum_reps(const int *k, int nq) {
  MomentumReps m;
  std::map<std::array<int, 3>, int> index;
  std::vector<int> map(nq);
  for (int q = 0; q < nq; ++q) {
    const std::array<int, 3> a{k[3 * q], k[3 * q + 1], k[3 * q + 2]}, b{-a[0], -a[1], -a[2]};
    const bool neg = b > a;
    const std::array<int, 3> &c = neg ? b : a;
    auto it = index.find(c);
    int rho;
    if (it == index.end()) {
      rho = (int)index.size();
      index.emplace(c, rho);
      m.k.insert(m.k.end(), c.begin(), c.end());
    } else {
      rho = it->second;
    }
    map[q] = 2 * rho + (neg ? 1 : 0);
  }
  const int nrep = m.nrep();
  m.first.assign(nrep + 1, 0);
  for (int q = 0; q < nq; ++q) ++m.first[(map[q] >> 1) + 1];
  for (int r = 0; r < nrep; ++r) m.first[r + 1] += m.first[r];
  m.q_list.resize(nq);
  std::vector<int> fill(m.first.begin(), m.first.end() - 1);
  for (int q = 0; q < nq; ++q) m.q_list[fill[map[q] >> 1]++] = 2 * q + (map[q] & 1);
  return m;
}

// Chunks of representatives per CTA: as few chunks as the tensor memory allows, balanced,
// each a multiple of 8 representatives (the accumulator width 2 NH is a multiple of 16).
static void rep_chunks(int nrep, int *nrc, int *NH) {
  *nrc = (nrep + RCHUNK - 1) / RCHUNK;
  *NH = ((nrep + *nrc - 1) / *nrc + 7) / 8 * 8;
}

// Phase table (cos | sin of the representatives, FP16 hi/lo) and the device copy of the
// momentum map, cached per (L, momentum list, source position, chunk width NH, which the
// key carries in its sign field); the sign of the phase does not enter the table, so
// insertion and spectator share it.
static int get_phase_cs(lhc_ctx ctx, int L, const int *k, int nq, const int r[4], const MomentumReps &reps, int NH,
                        int nrc, int nkb, cudaStream_t st, const __half **table, const int **rmap) {
  PhaseKey key{L, nq, NH, 2, ((r[0] % L) + L) % L, ((r[1] % L) + L) % L, ((r[2] % L) + L) % L, hash_k(k, nq)};
  const int nrep = reps.nrep();
  const size_t tbytes = (size_t)nrc * nkb * 2 * 2 * NH * 32;
  // rmap: first[nrep + 1] followed by q_list[nq]
  const size_t off_map = (tbytes + 255) & ~(size_t)255;
  if (const PhaseEntry *hit = phase_take(ctx, key)) {
    *table = static_cast<const __half *>(hit->buf.p);
    *rmap = reinterpret_cast<const int *>(static_cast<const char *>(hit->buf.p) + off_map);
    return LHC_OK;
  }
  const size_t off_k = (off_map + sizeof(int) * (size_t)(nrep + 1 + nq) + 255) & ~(size_t)255;
  const size_t off_roots = (off_k + (size_t)12 * nrep + 255) & ~(size_t)255;
  PhaseEntry e;
  LHC_TRY(dev_alloc(ctx, e.buf, off_roots + (size_t)L * sizeof(double2)));
  std::vector<double2> roots(L);
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < L; ++m) roots[m] = make_double2(std::cos(two_pi * m / L), std::sin(two_pi * m / L));
  char *base = static_cast<char *>(e.buf.p);
  LHC_CHECK_CUDA(cudaMemcpy(base + off_map, reps.first.data(), sizeof(int) * (size_t)(nrep + 1), cudaMemcpyHostToDevice));
  LHC_CHECK_CUDA(cudaMemcpy(base + off_map + sizeof(int) * (size_t)(nrep + 1), reps.q_list.data(),
                            sizeof(int) * (size_t)nq, cudaMemcpyHostToDevice));
  LHC_CHECK_CUDA(cudaMemcpy(base + off_k, reps.k.data(), (size_t)12 * nrep, cudaMemcpyHostToDevice));
  LHC_CHECK_CUDA(cudaMemcpy(base + off_roots, roots.data(), (size_t)L * sizeof(double2), cudaMemcpyHostToDevice));
  const size_t total = (size_t)nrc * nkb * 2 * 2 * NH * KSTEP;
  phase_cs_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<__half *>(base), reinterpret_cast<const int *>(base + off_k), nrep, NH, nrc, nkb, L, key.rx,
      key.ry, key.rz, reinterpret_cast<const double2 *>(base + off_roots));
  note_launch();
  LHC_CHECK_CUDA(cudaGetLastError());
  e.nq_pad = nrc * NH;
  phase_insert(ctx, key, e);
  *table = reinterpret_cast<const __half *>(base);
  *rmap = reinterpret_cast<const int *>(base + off_map);
  return LHC_OK;
}

// Upper bound of the device memory one mixed-precision call takes beyond its caller's
// buffers: workspace (partials at the largest site split, narrowed inputs, diquark) and
// the phase table of its momentum set.  Used for admission control by the job server.
size_t mixed_call_bytes(Part part, int dtype, int V3, int n_r, int nt, int nq) {
  const bool baryon = part == PART_SPEC_BARYON;
  // partial sums are kept per tile of two noises: an odd count is padded by one
  const size_t ncols = (size_t)(n_r + 1) / 2 * 2 * (baryon ? kBarCols : 192);
  const size_t ntl = (size_t)std::min(nt, kMaxSlices);
  // at most nq representatives: at most ceil(nq / RCHUNK) chunks of at most RCHUNK
  const size_t nrep_pad = (size_t)(nq + RCHUNK - 1) / RCHUNK * RCHUNK;
  const size_t nkb = (V3 + 2 * KSTEP - 1) / (2 * KSTEP) * 2;
  size_t b = ntl * kMaxSplits * nrep_pad * ncols * sizeof(float4);
  if (dtype == LHC_C128) b += ntl * V3 * 144 * 8 + (baryon ? (size_t)V3 * 144 * 8 : 0) + (size_t)n_r * ntl * V3 * 12 * 8;
  if (baryon) b += (size_t)V3 * 2304 * 8;
  b += nkb * 2 * 2 * nrep_pad * 32 + 4 * (size_t)(2 * nq + 1) + 12 * (size_t)nq + 4096;
  b += (2 * kMaxSlices + 1) * sizeof(unsigned) + 256;   // operand maxima of the split scale
  return b + 4 * 256;
}

// Tiled tensor map over complex64 data viewed as 8-byte elements (innermost dimension
// first; strides in bytes for dimensions 1..rank-1).
static int encode_map(CUtensorMap *m, int rank, const void *base, const uint64_t *dims, const uint64_t *strides,
                      const uint32_t *box) {
  cuuint64_t d[5], sb[4];
  cuuint32_t b[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    es[i] = 1;
  }
  for (int i = 0; i + 1 < rank; ++i) sb[i] = strides[i];
  // the driver function is looked up through the runtime, so that the library itself
  // loads on machines without a driver (and links no libcuda); the lookup runs once, and
  // the static's initialization is thread-safe
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) {
    set_error("the driver does not provide cuTensorMapEncodeTiled");
    return LHC_ECUDA;
  }
  CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, (cuuint32_t)rank, const_cast<void *>(base), d, sb, b, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for a rank-%d map", (int)r, rank);
    return LHC_ECUDA;
  }
  return LHC_OK;
}

// Time coordinates of slices that lie in one tensor at multiples of slice_bytes from the
// lowest of them (slices wrap around the time extent, so the order is not monotonic).
static int slice_coords(const void *const *ptrs, int nb, size_t slice_bytes, const char **base, int *coord,
                        int *extent) {
  const char *lo = static_cast<const char *>(ptrs[0]);
  for (int j = 1; j < nb; ++j) lo = std::min(lo, static_cast<const char *>(ptrs[j]));
  int hi = 0;
  for (int j = 0; j < nb; ++j) {
    const size_t d = static_cast<const char *>(ptrs[j]) - lo;
    if (d % slice_bytes != 0 || d / slice_bytes > (size_t)1 << 30) {
      set_error("slices of one call must lie in one tensor");
      return LHC_EINVAL;
    }
    coord[j] = (int)(d / slice_bytes);
    hi = std::max(hi, coord[j]);
  }
  *base = lo;
  *extent = hi + 1;
  return LHC_OK;
}

// ---------------------------------------------------------------- staged propagators
// Complex64 copies of complex128 propagator slices made once by lhc_prop_stage and read by
// every later mixed call whose propagator slices all lie in one staged range (any context
// on the device): the insertion calls of several sink times and the spectators on their
// sink slices share the propagator, and each would otherwise narrow it again.  Process-
// wide, keyed by the device and the caller's base pointer.
struct StagedProp {
  int device = 0, V3 = 0, T = 0, t_lo = 0, nt = 0;
  const char *base = nullptr;   // the caller's propagator [T][V3][144] complex128
  DevBuf copy, maxS;            // [nt][V3][144] complex64; [nt] largest |re| or |im| (float bits)
  lhc_ctx owner = nullptr;      // the context whose budget holds the copy
};
static std::mutex g_staged_mu;
static std::vector<StagedProp> g_staged;

// The staged copy of slices jobs[0..nb) if they are consecutive slices of one staged range
// (in the range's order), else no copy.
struct StagedView {
  const float2 *copy = nullptr;
  const unsigned *maxS = nullptr;
  int idx0 = 0, nt = 0;
};
static StagedView find_staged(int device, const SliceJob *jobs, int nb) {
  StagedView v;
  const size_t slice = (size_t)jobs[0].V3 * 144 * sizeof(double2);
  std::lock_guard<std::mutex> g(g_staged_mu);
  for (const StagedProp &e : g_staged) {
    if (e.device != device || e.V3 != jobs[0].V3) continue;
    const char *p0 = static_cast<const char *>(jobs[0].S);
    if (p0 < e.base || (size_t)(p0 - e.base) % slice != 0 || (size_t)(p0 - e.base) / slice >= (size_t)e.T) continue;
    const int t0 = (int)((size_t)(p0 - e.base) / slice);
    const int idx0 = ((t0 - e.t_lo) % e.T + e.T) % e.T;
    if (idx0 + nb > e.nt) continue;
    bool ok = true;
    for (int j = 1; j < nb && ok; ++j)
      ok = jobs[j].S == e.base + (size_t)((e.t_lo + idx0 + j) % e.T) * slice;
    if (!ok) continue;
    v.copy = static_cast<const float2 *>(e.copy.p);
    v.maxS = static_cast<const unsigned *>(e.maxS.p);
    v.idx0 = idx0;
    v.nt = e.nt;
    return v;
  }
  return v;
}

int stage_propagator(lhc_ctx ctx, const lhc_lattice *lat, const void *S, int t_lo, int nt, cudaStream_t st) {
  const int V3 = lat->L * lat->L * lat->L, T = lat->T;
  const char *base = static_cast<const char *>(S);
  std::lock_guard<std::mutex> g(g_staged_mu);
  StagedProp *e = nullptr;
  for (StagedProp &x : g_staged)
    if (x.device == ctx->device && x.base == base) e = &x;
  if (e && (e->V3 != V3 || e->T != T || e->t_lo != t_lo || e->nt != nt || e->owner != ctx)) {
    // another range of the same tensor: the old copy goes (after all work that may read it)
    LHC_CHECK_CUDA(cudaDeviceSynchronize());
    dev_free(e->owner, e->copy);
    dev_free(e->owner, e->maxS);
    g_staged.erase(g_staged.begin() + (e - g_staged.data()));
    e = nullptr;
  }
  if (!e) {
    StagedProp x;
    x.device = ctx->device;
    x.V3 = V3;
    x.T = T;
    x.t_lo = t_lo;
    x.nt = nt;
    x.base = base;
    x.owner = ctx;
    LHC_TRY(dev_alloc(ctx, x.copy, (size_t)nt * V3 * 144 * sizeof(float2)));
    int s = dev_alloc(ctx, x.maxS, (size_t)nt * sizeof(unsigned));
    if (s != LHC_OK) {
      dev_free(ctx, x.copy);
      return s;
    }
    g_staged.push_back(x);
    e = &g_staged.back();
  }
  // narrow the slices (in stream order: calls that read the copy must follow on `st`, or
  // wait for it)
  LHC_CHECK_CUDA(cudaMemsetAsync(e->maxS.p, 0, (size_t)nt * sizeof(unsigned), st));
  const size_t cS = ((size_t)V3 * 144 + kNarrowChunk - 1) / kNarrowChunk;
  const size_t slice = (size_t)V3 * 144 * sizeof(double2);
  for (int j0 = 0; j0 < nt; j0 += kMaxSlices) {
    NarrowParams np{};
    np.nb = std::min(kMaxSlices, nt - j0);
    for (int j = 0; j < np.nb; ++j) np.slices[j] = SlicePtrs{base + (size_t)((t_lo + j0 + j) % T) * slice, nullptr};
    np.SB = nullptr;
    np.vec_stride = 0;
    np.Sst = static_cast<float2 *>(e->copy.p) + (size_t)j0 * V3 * 144;
    np.SBst = np.Vst = nullptr;
    np.maxS = static_cast<unsigned *>(e->maxS.p) + j0;
    np.maxV = nullptr;
    np.V3 = V3;
    np.withS = 1;
    ProfScope ps(ctx, st, LHC_KERNEL_CONTRACT, (double)np.nb * V3 * 144.0 * 24);
    narrow_c128<<<(unsigned)(np.nb * cS), kSmallThreads, 0, st>>>(np);
    note_launch();
  }
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

int unstage_propagator(lhc_ctx ctx, const void *S) {
  std::lock_guard<std::mutex> g(g_staged_mu);
  for (size_t i = 0; i < g_staged.size(); ++i) {
    StagedProp &e = g_staged[i];
    if (e.device == ctx->device && e.base == static_cast<const char *>(S)) {
      LHC_CHECK_CUDA(cudaDeviceSynchronize());   // nothing in flight may still read the copy
      dev_free(e.owner, e.copy);
      dev_free(e.owner, e.maxS);
      g_staged.erase(g_staged.begin() + i);
      return LHC_OK;
    }
  }
  set_error("lhc_prop_unstage: this propagator is not staged on device %d", ctx->device);
  return LHC_ENOTFOUND;
}

// The copies a context holds go with it (its destruction has synchronized the device).
void release_staged(lhc_ctx ctx) {
  std::lock_guard<std::mutex> g(g_staged_mu);
  for (size_t i = 0; i < g_staged.size();) {
    if (g_staged[i].owner == ctx) {
      dev_free(ctx, g_staged[i].copy);
      dev_free(ctx, g_staged[i].maxS);
      g_staged.erase(g_staged.begin() + i);
    } else {
      ++i;
    }
  }
}

// ---------------------------------------------------------------- one call, in steps
// A mixed call runs, per chunk of at most kMaxSlices slices: sizing, prepare (operand
// maxima, the complex128 narrowing or the complex64 maximum pass, the baryon diquark, the
// tensor maps and the fused kernel's parameters), the fused launch, and finish (the
// reduce).  A batch prepares all its calls, launches the fused kernel once per part kind
// and chunk width, and finishes all calls.

struct ChunkLayout {
  size_t off_s, off_sb, off_v, off_d, off_m, bytes;
};

// floats of the partial sums per site split of one slice: nrc chunks x nct tiles, each
// a CTA block of 4 NH x MT floats
static size_t split_floats(const SliceJob &j0, int NH, int nrc) {
  const int nct = (j0.part == PART_SPEC_BARYON ? 48 : 3) * ((j0.n_r + 1) / 2);
  return (size_t)nrc * nct * 4 * NH * MT;
}

static ChunkLayout chunk_layout(const SliceJob &j0, int ntl, int nsplit, size_t per_split) {
  const bool baryon = j0.part == PART_SPEC_BARYON, narrow = j0.dtype == LHC_C128;
  const int V3 = j0.V3, n_r = j0.n_r;
  const size_t p_bytes = (size_t)ntl * nsplit * per_split * sizeof(float);
  const size_t s_bytes = narrow ? (size_t)ntl * V3 * 144 * sizeof(float2) : 0;
  const size_t sb_bytes = narrow && baryon ? (size_t)V3 * 144 * sizeof(float2) : 0;
  const size_t v_bytes = narrow ? (size_t)n_r * ntl * V3 * 12 * sizeof(float2) : 0;
  const size_t d_bytes = baryon ? (size_t)V3 * 2304 * sizeof(float2) : 0;   // diquark (one sink slice)
  auto al256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
  ChunkLayout c;
  c.off_s = al256(p_bytes);
  c.off_sb = c.off_s + al256(s_bytes);
  c.off_v = c.off_sb + al256(sb_bytes);
  c.off_d = c.off_v + al256(v_bytes);
  c.off_m = c.off_d + al256(d_bytes);
  c.bytes = al256(c.off_m + (2 * kMaxSlices + 1) * sizeof(unsigned));   // maxS, maxV per slice, maxD
  return c;
}

// one launch chunk of one call, ready for the fused launch and the reduce
struct Prepared {
  FusedParams fp;
  int nb, sign, nrep, ncols, nsplit, NH, mode;
  size_t per_split, n_out;
  const int *rmap;
  double2 *out;
  int tm0, tmT, tv0, tvT;   // slice j's coordinates: (tm0 + j) % tmT, (tv0 + j) % tvT
};

static int prepare_chunk(lhc_ctx ctx, const SliceJob *jobs, int nb, int nq, int sign, const MomentumReps &reps,
                         const __half *phase, const int *rmap, int NH, int nsplit, int kd, char *ws,
                         const ChunkLayout &lay, cudaStream_t st, Prepared *pc) {
  const SliceJob &j0 = jobs[0];
  const bool baryon = j0.part == PART_SPEC_BARYON, narrow = j0.dtype == LHC_C128;
  const int V3 = j0.V3, n_r = j0.n_r;
  const int ncols = n_r * (baryon ? kBarCols : 192);
  const int nrc = (reps.nrep() + NH - 1) / NH;
  unsigned *maxS = reinterpret_cast<unsigned *>(ws + lay.off_m), *maxV = maxS + kMaxSlices, *maxD = maxV + kMaxSlices;
  FusedParams &fp = pc->fp;
  fp.c.B = phase;
  fp.c.partial = reinterpret_cast<float *>(ws);
  fp.c.err = ctx->dev_err;
  fp.c.n_r = n_r;
  fp.c.V3 = V3;
  fp.c.nct = (baryon ? 48 : 3) * ((n_r + 1) / 2);
  // site blocks, rounded up to an even number: the kernel consumes k-steps in pairs (the
  // pad block's phases are zero and its sites lie past the slice, which TMA reads as zero)
  fp.c.nkb = ((V3 + 2 * KSTEP - 1) / (2 * KSTEP)) * 2;
  if (NH < 8 || NH > RCHUNK || NH % 8 != 0) {
    set_error("unsupported representative chunk %d", NH);
    return LHC_EINVAL;
  }
  fp.c.nrc = nrc;
  fp.c.NH = NH;
  fp.c.mode = (int)j0.part;
  fp.c.nrep = reps.nrep();
  fp.c.ncols = ncols;
  fp.c.nsplit = nsplit;
  fp.c.kd = kd;
  fp.c.g5mask = j0.g5mask;
  fp.c.maxM = baryon ? maxD : maxS;
  fp.c.maxM_per_slice = baryon ? 0 : 1;
  fp.c.maxV = maxV;
  pc->nb = nb;
  pc->sign = sign;
  pc->nrep = reps.nrep();
  pc->ncols = ncols;
  pc->nsplit = nsplit;
  pc->NH = NH;
  pc->mode = (int)j0.part;
  pc->per_split = split_floats(j0, NH, nrc);
  pc->n_out = (size_t)nq * ncols;
  pc->rmap = rmap;
  pc->out = j0.out;
  // the operand maxima of this chunk of slices (for the split scale) start at zero
  LHC_CHECK_CUDA(cudaMemsetAsync(maxS, 0, (2 * kMaxSlices + 1) * sizeof(unsigned), st));
  const size_t cS = ((size_t)V3 * 144 + kNarrowChunk - 1) / kNarrowChunk;
  const size_t cV = ((size_t)V3 * 12 + kNarrowChunk - 1) / kNarrowChunk;
  // propagator slices staged by lhc_prop_stage replace the narrowing of the propagator
  const StagedView sv = narrow && !baryon ? find_staged(ctx->device, jobs, nb) : StagedView{};
  if (narrow) {
    NarrowParams np;
    np.withS = sv.copy ? 0 : 1;
    for (int j = 0; j < nb; ++j) np.slices[j] = SlicePtrs{jobs[j].S, jobs[j].vec};
    np.SB = baryon ? j0.SB : nullptr;
    np.vec_stride = j0.vec_stride;
    np.Sst = reinterpret_cast<float2 *>(ws + lay.off_s);
    np.SBst = reinterpret_cast<float2 *>(ws + lay.off_sb);
    np.Vst = reinterpret_cast<float2 *>(ws + lay.off_v);
    np.maxS = maxS;
    np.maxV = maxV;
    np.nb = nb;
    np.V3 = V3;
    ProfScope ps(ctx, st, LHC_KERNEL_CONTRACT,
                 (double)nb * V3 * ((baryon ? 288.0 : sv.copy ? 0.0 : 144.0) + 12.0 * n_r) * 24);
    const size_t blocks = (size_t)((sv.copy ? 0 : nb) + (baryon ? 1 : 0)) * cS + (size_t)n_r * nb * cV;
    narrow_c128<<<(unsigned)blocks, kSmallThreads, 0, st>>>(np);
    note_launch();
  } else {
    // complex64 inputs are read in place; one read-only pass finds their maxima
    MaxParams mp;
    for (int j = 0; j < nb; ++j) mp.slices[j] = SlicePtrs{jobs[j].S, jobs[j].vec};
    mp.vec_stride = j0.vec_stride;
    mp.maxS = maxS;
    mp.maxV = maxV;
    mp.nb = nb;
    mp.V3 = V3;
    mp.n_r = n_r;
    mp.with_S = baryon ? 0 : 1;   // the baryon's matrix operand is the diquark
    ProfScope ps(ctx, st, LHC_KERNEL_CONTRACT, (double)nb * V3 * ((baryon ? 0.0 : 144.0) + 12.0 * n_r) * 8);
    const size_t blocks = (size_t)(baryon ? 0 : nb) * cS + (size_t)n_r * nb * cV;
    max_c64<<<(unsigned)blocks, kSmallThreads, 0, st>>>(mp);
    note_launch();
  }
  // tensor maps of the matrix operand and the vector of this chunk of slices
  const char *Mbase, *Vbase;
  int Tm, Tv;
  size_t vstride_bytes;
  if (narrow) {
    Mbase = sv.copy ? reinterpret_cast<const char *>(sv.copy) : ws + lay.off_s;
    Vbase = ws + lay.off_v;
    for (int j = 0; j < nb; ++j) {
      fp.tM[j] = sv.copy ? sv.idx0 + j : j;
      fp.tV[j] = j;
    }
    Tm = sv.copy ? sv.nt : nb;
    Tv = nb;
    if (sv.copy) fp.c.maxM = sv.maxS + sv.idx0;   // the slice maxima were taken when staging
    vstride_bytes = (size_t)nb * V3 * 12 * sizeof(float2);
  } else {
    const void *mp[kMaxSlices], *vp[kMaxSlices];
    for (int j = 0; j < nb; ++j) {
      mp[j] = jobs[j].S;
      vp[j] = jobs[j].vec;
    }
    LHC_TRY(slice_coords(mp, nb, (size_t)V3 * 144 * sizeof(float2), &Mbase, fp.tM, &Tm));
    LHC_TRY(slice_coords(vp, nb, (size_t)V3 * 12 * sizeof(float2), &Vbase, fp.tV, &Tv));
    vstride_bytes = j0.vec_stride * sizeof(float2);
  }
  pc->tm0 = fp.tM[0];
  pc->tmT = Tm;
  pc->tv0 = fp.tV[0];
  pc->tvT = Tv;
  if (baryon) {   // the matrix operand becomes the diquark of the (single) sink slice
    const float2 *GA = reinterpret_cast<const float2 *>(Mbase) + (size_t)fp.tM[0] * V3 * 144;
    const float2 *GB = narrow ? reinterpret_cast<const float2 *>(ws + lay.off_sb) : static_cast<const float2 *>(j0.SB);
    float2 *D = reinterpret_cast<float2 *>(ws + lay.off_d);
    ProfScope ps(ctx, st, LHC_KERNEL_CONTRACT, (double)V3 * (288.0 + 2304.0) * 8);
    baryon_diquark<<<V3, kSmallThreads, 0, st>>>(GA, GB, V3, D, maxD);
    note_launch();
    const uint64_t dims[3] = {768, 3, (uint64_t)V3}, strides[2] = {768 * 8, 2304 * 8};
    const uint32_t box[3] = {16, 3, 16};
    LHC_TRY(encode_map(&fp.c.tmM, 3, D, dims, strides, box));
  } else {
    const uint64_t dims[5] = {12, 3, 4, (uint64_t)V3, (uint64_t)Tm};
    const uint64_t strides[4] = {96, 288, 1152, (uint64_t)V3 * 1152};
    const uint32_t box[5] = {12, 3, 2, 16, 1};
    LHC_TRY(encode_map(&fp.c.tmM, 5, Mbase, dims, strides, box));
  }
  const uint64_t dims[4] = {12, (uint64_t)V3, (uint64_t)Tv, (uint64_t)n_r};
  const uint64_t strides[3] = {96, (uint64_t)V3 * 96, vstride_bytes};
  const uint32_t box[4] = {12, 16, 1, 2};
  LHC_TRY(encode_map(&fp.c.tmV, 4, Vbase, dims, strides, box));
  return LHC_OK;
}

static int finish_chunk(lhc_ctx ctx, const Prepared &pc, cudaStream_t st) {
  const size_t n_in = (size_t)pc.nrep * pc.ncols;
  ProfScope ps(ctx, st, LHC_KERNEL_REDUCE, (double)pc.nb * pc.nsplit * n_in * 16 + (double)pc.nb * pc.n_out * 16);
  ReduceArgs a;
  a.part = pc.fp.c.partial;
  a.per_split = pc.per_split;
  a.rep_first = pc.rmap;
  a.rep_q = pc.rmap + pc.nrep + 1;
  a.out = pc.out;
  a.out_stride = pc.n_out;
  a.nsplit = pc.nsplit;
  a.nrep = pc.nrep;
  a.sign = pc.sign;
  a.ncols = pc.ncols;
  a.nt = pc.nb;
  a.nrc = pc.fp.c.nrc;
  a.nct = pc.fp.c.nct;
  a.NH = pc.NH;
  a.n_r = pc.fp.c.n_r;
  a.mode = pc.mode;
  const size_t threads = (size_t)pc.nb * a.nrc * a.nct * (a.NH / 4) * MT;
  reduce_f64<<<(unsigned)((threads + kReduceThreads - 1) / kReduceThreads), kReduceThreads, 0, st>>>(a);
  note_launch();
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

static int kd_for(Part part) {
  // k-steps accumulated in tensor memory between drains.  The accumulation truncates, so
  // the error grows with the interval.  Measured against the oracle on the 24^3 chain (16
  // noises, 93 momenta): the insertion gives 1.6e-7 per block at interval 2 and 2.5e-7 at
  // 4, for 13% more fused-kernel time at 2; the meson and baryon spectators 1.6e-7 and
  // 1.4e-7 at 2, 2.5e-7 and 2.4e-7 at 4, for 11% and 10% more time at 2.  The combine adds
  // the errors of both parts: the meson spectator (a tenth of the meson step) drains every
  // 2, the insertion and the baryon spectator (most of the baryon step) every 4, which
  // leaves every correlator of those chains within 6.5e-7 (meson) and 7.5e-7 (baryon) of
  // the oracle, relative to its row.  LHC_KD sets every part's interval, LHC_KD_INS,
  // LHC_KD_SPEC and LHC_KD_BAR one part's; intervals are even, since k-steps come in pairs.
  static const int defaults[3] = {4, 2, 4};   // insertion, meson spectator, baryon spectator
  static const char *names[3] = {"LHC_KD_INS", "LHC_KD_SPEC", "LHC_KD_BAR"};
  int kd = defaults[(int)part];
  const char *e = getenv(names[(int)part]);
  if (!e) e = getenv("LHC_KD");
  if (e) kd = std::max(2, (atoi(e) + 1) / 2 * 2);
  return kd;
}

// One mixed-precision call with a given launch shape: NH representatives per CTA (a
// multiple of 8, at most RCHUNK) and nsplit site ranges per slice.
static int run_mixed_shape(lhc_ctx ctx, const SliceJob *jobs, int nt, const int *k, int nq, const int r[4],
                           int sign, cudaStream_t st, const MomentumReps &reps, int NH, int nsplit) {
  const SliceJob &j0 = jobs[0];
  const int nrc = (reps.nrep() + NH - 1) / NH;
  const int nkb = ((j0.V3 + 2 * KSTEP - 1) / (2 * KSTEP)) * 2;
  const __half *phase = nullptr;
  const int *rmap = nullptr;
  LHC_TRY(get_phase_cs(ctx, j0.L, k, nq, r, reps, NH, nrc, nkb, st, &phase, &rmap));
  const int ncols = j0.n_r * (j0.part == PART_SPEC_BARYON ? kBarCols : 192);
  const ChunkLayout lay = chunk_layout(j0, std::min(nt, kMaxSlices), nsplit, split_floats(j0, NH, nrc));
  LHC_TRY(ensure(ctx, ctx->ws, lay.bytes));
  char *ws = static_cast<char *>(ctx->ws.p);
  const int kd = kd_for(j0.part);
  for (int jb = 0; jb < nt; jb += kMaxSlices) {
    const int nb = std::min(kMaxSlices, nt - jb);
    Prepared pc;
    LHC_TRY(prepare_chunk(ctx, jobs + jb, nb, nq, sign, reps, phase, rmap, NH, nsplit, kd, ws, lay, st, &pc));
    {
      ProfScope ps(ctx, st, LHC_KERNEL_FUSED, 8.0 * nb * (double)nq * ncols * j0.V3);
      if (j0.part == PART_INS)
        LHC_TRY(launch_fused<0>(pc.fp, nb, st));
      else if (j0.part == PART_SPEC_MESON)
        LHC_TRY(launch_fused<1>(pc.fp, nb, st));
      else
        LHC_TRY(launch_fused<2>(pc.fp, nb, st));
    }
    LHC_TRY(finish_chunk(ctx, pc, st));
  }
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

// Candidate launch shapes of the autotuner: the distinct chunk widths NH that split the
// representatives evenly (at least 16 unless fewer are needed; at most three, widest
// first) and site splits from 1 to 16 that leave every split at least two k-step pairs.
static void tune_candidates(int nrep, int npairs, std::vector<std::pair<int, int>> *out) {
  std::vector<int> widths;
  for (int w = RCHUNK; w >= 8 && (int)widths.size() < 3; w -= 8) {
    const int nrc = (nrep + w - 1) / w, nh = ((nrep + nrc - 1) / nrc + 7) / 8 * 8;
    if (nh < 16 && nrep > 8 && !widths.empty()) break;
    if (std::find(widths.begin(), widths.end(), nh) == widths.end()) widths.push_back(nh);
  }
  static const int kSplits[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, kMaxSplits};
  for (int nh : widths)
    for (int ns : kSplits)
      if (ns == 1 || ns <= npairs / 2) out->emplace_back(nh, ns);
}

// Times every candidate shape on this call's own inputs (each run rewrites the outputs;
// the last run uses the chosen shape) and stores the fastest.  Runs only outside stream
// capture: it synchronizes the stream.
static int autotune(lhc_ctx ctx, const SliceJob *jobs, int nt, const int *k, int nq, const int r[4], int sign,
                    cudaStream_t st, const MomentumReps &reps, const TuneKey &key, TuneChoice *best) {
  const int nkb = ((jobs[0].V3 + 2 * KSTEP - 1) / (2 * KSTEP)) * 2;
  std::vector<std::pair<int, int>> cand;
  tune_candidates(reps.nrep(), (nkb + 1) / 2, &cand);
  cudaEvent_t e0, e1;
  LHC_CHECK_CUDA(cudaEventCreate(&e0));
  LHC_CHECK_CUDA(cudaEventCreate(&e1));
  best->us = -1.f;
  int status = LHC_OK;
  for (const auto &c : cand) {
    int s = run_mixed_shape(ctx, jobs, nt, k, nq, r, sign, st, reps, c.first, c.second);   // warm-up
    if (s == LHC_EBUDGET || s == LHC_ENOMEM) continue;   // this shape does not fit: skip it
    if (s != LHC_OK) {
      status = s;
      break;
    }
    cudaEventRecord(e0, st);
    for (int rep = 0; rep < 2 && s == LHC_OK; ++rep) s = run_mixed_shape(ctx, jobs, nt, k, nq, r, sign, st, reps, c.first, c.second);
    cudaEventRecord(e1, st);
    if (s != LHC_OK || cudaEventSynchronize(e1) != cudaSuccess) {
      status = s != LHC_OK ? s : LHC_ECUDA;
      break;
    }
    // a candidate whose kernels gave up a bounded wait would time as the fastest (every
    // later wait gives up at once): stop and report instead of choosing it
    int code = 0;
    if (cudaMemcpy(&code, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || code != 0) {
      set_error("autotune: shape NH %d, %d splits: a bounded device wait gave up (site %d)", c.first, c.second, code);
      status = LHC_ETIMEOUT;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const float us = ms * 500.f;   // per run
    if (best->us < 0.f || us < best->us) *best = TuneChoice{c.first, c.second, us};
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != LHC_OK) return status;
  if (best->us < 0.f) {
    set_error("no launch shape of this call fits the memory budget");
    return LHC_EBUDGET;
  }
  tune_store(key, *best);
  return LHC_OK;
}

// Launch shape of a call: the tuned one if the table has its key, else the heuristic
// (widest chunks; site splits that fill whole waves of one CTA per SM).
static bool call_shape(lhc_ctx ctx, const SliceJob &j0, int nt, const MomentumReps &reps, int *NH, int *nsplit,
                       TuneKey *key) {
  const bool baryon = j0.part == PART_SPEC_BARYON;
  const int nkb = ((j0.V3 + 2 * KSTEP - 1) / (2 * KSTEP)) * 2;
  const int nct = (baryon ? 48 : 3) * ((j0.n_r + 1) / 2);
  int nrc;
  rep_chunks(reps.nrep(), &nrc, NH);
  *nsplit = choose_nsplit(nct * nt * nrc, (nkb + 1) / 2, ctx->num_sms);
  *key = TuneKey{(int)j0.part, j0.dtype, j0.V3, j0.n_r, std::min(nt, kMaxSlices), reps.nrep()};
  TuneChoice ch;
  const bool tuned = tune_lookup(*key, &ch);
  if (tuned) {
    *NH = ch.NH;
    *nsplit = ch.nsplit;
  }
  if (const char *e = getenv("LHC_NSPLIT")) *nsplit = std::max(1, std::min((nkb + 1) / 2, atoi(e)));
  return tuned;
}

// shape_nt > 0: the launch shape (and its tuning key) is that of a call of shape_nt slices,
// of which these nt are a group; every slice is then computed exactly as in that call.
int run_part_mixed(lhc_ctx ctx, const SliceJob *jobs, int nt, const int *k, int nq, const int r[4], int sign,
                   cudaStream_t st, int shape_nt) {
  const SliceJob &j0 = jobs[0];
  const MomentumReps reps = momentum_reps(k, nq);
  int NH, nsplit;
  TuneKey key;
  const bool tuned = call_shape(ctx, j0, shape_nt > 0 ? shape_nt : nt, reps, &NH, &nsplit, &key);
  if (!tuned && ctx->tune_mode == LHC_TUNE_ON) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LHC_CHECK_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      TuneChoice ch;
      LHC_TRY(autotune(ctx, jobs, nt, k, nq, r, sign, st, reps, key, &ch));
      NH = ch.NH;
      nsplit = ch.nsplit;
      if (const char *e = getenv("LHC_NSPLIT")) nsplit = std::max(1, atoi(e));
    }
  }
  return run_mixed_shape(ctx, jobs, nt, k, nq, r, sign, st, reps, NH, nsplit);
}

// A batch of mixed calls: every call is prepared (in its own workspace region), the fused
// work of up to kMaxBatch calls of one part kind and chunk width runs in one persistent
// launch, and every call is reduced.  Each task does what the CTA with its
// coordinates does in its call's own launch, with the same launch shape, so the results
// are bitwise those of the calls made one by one.  Within a launch the calls are ordered
// by the length of their tasks (k-steps per site split), longest first, so that the short
// tasks fill the end.
int run_batch_mixed(lhc_ctx ctx, const std::vector<BatchCall> &calls, cudaStream_t st) {
  const int n = (int)calls.size();
  std::vector<MomentumReps> reps(n);
  std::vector<int> NH(n), nsplit(n);
  std::vector<const __half *> phase(n);
  std::vector<const int *> rmap(n);
  std::vector<ChunkLayout> lay(n);
  std::vector<size_t> off(n + 1, 0);
  for (int c = 0; c < n; ++c) {
    const BatchCall &bc = calls[c];
    const SliceJob &j0 = bc.jobs[0];
    const int nt = (int)bc.jobs.size();
    if (nt > kMaxSlices) {
      set_error("batch: a call spans %d slices; at most %d", nt, kMaxSlices);
      return LHC_EINVAL;
    }
    reps[c] = momentum_reps(bc.k, bc.nq);
    TuneKey key;
    call_shape(ctx, j0, nt, reps[c], &NH[c], &nsplit[c], &key);
    const int nrc = (reps[c].nrep() + NH[c] - 1) / NH[c];
    const int nkb = ((j0.V3 + 2 * KSTEP - 1) / (2 * KSTEP)) * 2;
    LHC_TRY(get_phase_cs(ctx, j0.L, bc.k, bc.nq, bc.r, reps[c], NH[c], nrc, nkb, st, &phase[c], &rmap[c]));
    lay[c] = chunk_layout(j0, nt, nsplit[c], split_floats(j0, NH[c], nrc));
    off[c + 1] = off[c] + lay[c].bytes;
  }
  // persistent launches: at most one per (part, chunk width) and kMaxBatch calls
  int nlaunch = 0;
  {
    std::map<std::pair<int, int>, int> count;
    for (int c = 0; c < n; ++c) ++count[{(int)calls[c].jobs[0].part, NH[c]}];
    for (const auto &kv : count) nlaunch += (kv.second + kMaxBatch - 1) / kMaxBatch;
  }
  const size_t off_cursor = (off[n] + 255) & ~(size_t)255;   // one task counter per launch
  LHC_TRY(ensure(ctx, ctx->ws, off_cursor + sizeof(int) * (size_t)nlaunch));
  char *ws = static_cast<char *>(ctx->ws.p);
  int *cursor = reinterpret_cast<int *>(ws + off_cursor);
  std::vector<Prepared> pc(n);
  for (int c = 0; c < n; ++c) {
    const BatchCall &bc = calls[c];
    LHC_TRY(prepare_chunk(ctx, bc.jobs.data(), (int)bc.jobs.size(), bc.nq, bc.sign, reps[c], phase[c], rmap[c], NH[c],
                          nsplit[c], kd_for(bc.jobs[0].part), ws + off[c], lay[c], st, &pc[c]));
    const Prepared &q = pc[c];
    for (int j = 0; j < q.nb; ++j)
      if (q.fp.tM[j] != (q.tm0 + j) % q.tmT || q.fp.tV[j] != (q.tv0 + j) % q.tvT) {
        set_error("batch: the slices of a call must be consecutive (mod T) in its tensors");
        return LHC_EINVAL;
      }
  }
  // A call whose own launch fills at least kOwnWaves waves of one CTA per SM gains
  // nothing from sharing a launch (its tail is a small part of it; measured on 144 calls of
  // 32^3 x 64: 359 ms in persistent launches against 348 ms one by one), so it keeps its own
  // fused launch.  The others go to the persistent launches: by part kind and chunk width,
  // longest tasks first (k-steps per site split), ties in call order.
  constexpr int kOwnWaves = 4;
  std::vector<int> order;
  for (int c = 0; c < n; ++c) {
    const long long ctas = (long long)pc[c].fp.c.nct * pc[c].fp.c.nsplit * pc[c].nb * pc[c].fp.c.nrc;
    if (ctas >= (long long)kOwnWaves * ctx->num_sms) {
      ProfScope ps(ctx, st, LHC_KERNEL_FUSED, 8.0 * pc[c].nb * (double)calls[c].nq * pc[c].ncols * pc[c].fp.c.V3);
      if (pc[c].mode == 0)
        LHC_TRY(launch_fused<0>(pc[c].fp, pc[c].nb, st));
      else if (pc[c].mode == 1)
        LHC_TRY(launch_fused<1>(pc[c].fp, pc[c].nb, st));
      else
        LHC_TRY(launch_fused<2>(pc[c].fp, pc[c].nb, st));
    } else {
      order.push_back(c);
    }
  }
  const int nper = (int)order.size();
  auto task_len = [&](int c) { return (pc[c].fp.c.nkb + pc[c].nsplit - 1) / pc[c].nsplit; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (pc[a].mode != pc[b].mode) return pc[a].mode < pc[b].mode;
    if (pc[a].NH != pc[b].NH) return pc[a].NH > pc[b].NH;
    return task_len(a) > task_len(b);
  });
  if (nper > 0) LHC_CHECK_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * (size_t)nlaunch, st));
  for (int c0 = 0, l = 0; c0 < nper; ++l) {
    const int mode = pc[order[c0]].mode, nh = pc[order[c0]].NH;
    int c1 = c0;
    while (c1 < nper && c1 - c0 < kMaxBatch && pc[order[c1]].mode == mode && pc[order[c1]].NH == nh) ++c1;
    std::unique_ptr<BatchParams> bpp(new BatchParams());   // 25 KB: kept off the stack
    BatchParams &bp = *bpp;
    bp.n = c1 - c0;
    bp.cursor = cursor + l;
    bp.first[0] = 0;
    double w = 0.0;
    for (int e = 0; e < bp.n; ++e) {
      const Prepared &q = pc[order[c0 + e]];
      bp.item[e] = q.fp.c;
      bp.item[e].tm0 = q.tm0;
      bp.item[e].tmT = q.tmT;
      bp.item[e].tv0 = q.tv0;
      bp.item[e].tvT = q.tvT;
      bp.first[e + 1] = bp.first[e] + q.fp.c.nct * q.fp.c.nsplit * q.nb * q.fp.c.nrc;
      w += 8.0 * q.nb * (double)(q.n_out / q.ncols) * q.ncols * q.fp.c.V3;
    }
    ProfScope ps(ctx, st, LHC_KERNEL_FUSED, w);
    const int nctas = std::min(bp.first[bp.n], ctx->num_sms);
    if (mode == 0)
      LHC_TRY(launch_persistent<0>(nh, bp, nctas, st));
    else if (mode == 1)
      LHC_TRY(launch_persistent<1>(nh, bp, nctas, st));
    else
      LHC_TRY(launch_persistent<2>(nh, bp, nctas, st));
    c0 = c1;
  }
  for (int c = 0; c < n; ++c) LHC_TRY(finish_chunk(ctx, pc[c], st));
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

}  // namespace lhc
