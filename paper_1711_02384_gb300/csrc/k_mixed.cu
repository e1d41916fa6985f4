// Mixed-precision path (meson insertion and spectator):
//
//   1. contract_split: the site contraction (Eq. 10 / Eq. 9) in FP32, each value split
//      into an FP16 pair hi + lo (hi = fp16(u), lo = fp16(u - hi)), written as the
//      K-major operand tiles of the tensor-core GEMM (core matrices of 8 rows x 16 B).
//   2. proj_mma: the momentum projection out[q][col] = sum_x P[q][x] U[x][col] as a
//      complex GEMM on tcgen05 tensor cores.  Real and imaginary parts are two halves
//      of one accumulator: D[:, 0:Np] = Ur Re - Ui Im, D[:, Np:2Np] = Ur Im + Ui Re, with
//      three products per split pair (hi*hi + hi*lo + lo*hi), FP32 accumulation in
//      tensor memory, drained every few k-steps into FP32 registers.  Operand tiles
//      arrive by 1-D bulk copies into a ring of shared-memory stages.
//   3. reduce_f64: FP64 sum of the per-site-range FP32 partials into complex128.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "lhc_internal.h"
#include "tc_ptx.cuh"

namespace lhc {
namespace {

constexpr int MT = 128;            // GEMM M tile: output columns per CTA
constexpr int KSTEP = 16;          // sites per MMA k-step
constexpr int ATILE = MT * KSTEP * 2;   // bytes of one 128x16 fp16 operand tile
constexpr int ASTAGE = 4 * ATILE;  // Ur hi, Ur lo, Ui hi, Ui lo
constexpr int NSTAGE = 4;
constexpr int kThreads = 320;      // warp 0 bulk copies, warp 1 MMA, warps 2..9 drain

// byte offset of element (row, k) in a K-major no-swizzle tile with 16 k per row block
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)((row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

struct SlicePtrs {
  const void *S;
  const void *vec;
};

__device__ __forceinline__ float2 ldc(const double2 *p) {
  double2 v = *p;
  return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ float2 ldc(const float2 *p) { return *p; }

// ------------------------------------------------------------ phase table (FP16 split)
// layout [qc][kb][hl][3*Np rows: -Im | Re | Im][16 sites], each (qc,kb,hl) block in core order
__global__ void phase_split_kernel(__half *out, const int *k, int nq, int Np, int nqc, int nkb, int L,
                                   int rx, int ry, int rz, int sign, const double2 *roots) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int rows = 3 * Np;
  size_t total = (size_t)nqc * nkb * 2 * rows * KSTEP;
  if (idx >= total) return;
  int kk = (int)(idx % KSTEP);
  size_t rest = idx / KSTEP;
  int n = (int)(rest % rows);
  rest /= rows;
  int hl = (int)(rest % 2);
  rest /= 2;
  int kb = (int)(rest % nkb);
  int qc = (int)(rest / nkb);
  int g = n / Np, qi = n % Np;
  int q = qc * 128 + qi;
  int qend = min(nq, (qc + 1) * 128);
  int V3 = L * L * L;
  int x = kb * KSTEP + kk;
  double v = 0.0;
  if (q < qend && x < V3) {
    int cx = x % L, cy = (x / L) % L, cz = x / (L * L);
    long long m = (long long)k[3 * q] * (cx - rx) + (long long)k[3 * q + 1] * (cy - ry) +
                  (long long)k[3 * q + 2] * (cz - rz);
    m %= L;
    if (m < 0) m += L;
    double re = roots[m].x, im = sign * roots[m].y;
    v = g == 0 ? -im : (g == 1 ? re : im);
  }
  __half hi = __double2half(v);
  __half lo = __double2half(v - (double)__half2float(hi));
  size_t block = ((size_t)qc * nkb + kb) * 2 + hl;
  char *base = reinterpret_cast<char *>(out) + block * (size_t)rows * 32;
  *reinterpret_cast<__half *>(base + core_off(n, kk)) = hl ? lo : hi;
}

// ------------------------------------------------------------ contraction + split
// One thread per (slice, column tile, site block, row, 8-site half): computes U for
// column ct*128 + row on 8 sites and writes 16 bytes into each of the 4 tiles.
template <typename CT, int MODE>
__global__ void contract_split(const SlicePtrs *__restrict__ sl, size_t vec_stride, int n_r, int V3,
                               int nct, int nkb, int g5mask, char *__restrict__ ws) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)gridDim.x * blockDim.x) return;
  int kc = (int)(idx & 1);
  size_t rest = idx >> 1;
  int row = (int)(rest % MT);
  rest /= MT;
  int kb = (int)(rest % nkb);
  rest /= nkb;
  int ct = (int)(rest % nct);
  int j = (int)(rest / nct);
  const int ncols = n_r * 192;
  int col = ct * MT + row;
  const CT *S = static_cast<const CT *>(sl[j].S);
  const CT *vec = static_cast<const CT *>(sl[j].vec);
  uint32_t pk[4][4];   // [tile][packed pairs]
  int i = col / 192, c = col % 192, v = c / 48, s = c % 48;
  int srow = (s / 12) * 3, scol = s % 12;
  float g;
  if (MODE == 0)
    g = ((g5mask >> v) & 1) ? -1.f : 1.f;
  else
    g = (((g5mask >> v) ^ (g5mask >> (s / 12)) ^ (g5mask >> ((s % 12) / 3))) & 1) ? -1.f : 1.f;
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    __half h[2][4];
#pragma unroll
    for (int e2 = 0; e2 < 2; ++e2) {
      int x = kb * KSTEP + kc * 8 + e + e2;
      float2 u = make_float2(0.f, 0.f);
      if (col < ncols && x < V3) {
        const CT *Sx = S + (size_t)x * 144;
        const CT *vx = vec + (size_t)i * vec_stride + (size_t)x * 12 + v * 3;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          float2 a = ldc(vx + cc);
          float2 b = ldc(Sx + (srow + cc) * 12 + scol);
          if (MODE == 0) {   // conj(psi) * S
            u.x += a.x * b.x + a.y * b.y;
            u.y += a.x * b.y - a.y * b.x;
          } else {           // eta * conj(S)
            u.x += a.x * b.x + a.y * b.y;
            u.y += a.y * b.x - a.x * b.y;
          }
        }
        u.x *= g;
        u.y *= g;
      }
      __half rh = __float2half_rn(u.x), ih = __float2half_rn(u.y);
      h[e2][0] = rh;
      h[e2][1] = __float2half_rn(u.x - __half2float(rh));
      h[e2][2] = ih;
      h[e2][3] = __float2half_rn(u.y - __half2float(ih));
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      __half2 p = __halves2half2(h[0][t], h[1][t]);
      pk[t][e / 2] = *reinterpret_cast<uint32_t *>(&p);
    }
  }
  char *tile = ws + (((size_t)j * nct + ct) * nkb + kb) * ASTAGE;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    *reinterpret_cast<uint4 *>(tile + t * ATILE + core_off(row, kc * 8)) =
        make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
}

// ------------------------------------------------------------ tensor-core projection
struct MmaParams {
  const char *A;        // [nt][nct][nkb][ASTAGE]
  const __half *B;      // [nqc][nkb][2][3Np][16]
  float2 *partial;      // [nt][nsplit][nq][ncols]
  int *err;
  int nct, nkb, nqc, nq, ncols, nsplit, kd;
};

template <int NP>
__global__ void __launch_bounds__(kThreads, 1) proj_mma(MmaParams p) {
  constexpr int BSTAGE = 2 * 3 * NP * 32;                 // hi and lo blocks of [-Im|Re|Im]
  constexpr uint32_t TMEM_COLS = (4 * NP <= 32) ? 32 : (4 * NP <= 64) ? 64 : (4 * NP <= 128) ? 128
                                 : (4 * NP <= 256) ? 256 : 512;
  extern __shared__ __align__(1024) char smem[];
  char *sA = smem;
  char *sB = smem + NSTAGE * ASTAGE;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sB + NSTAGE * BSTAGE);
  uint64_t *full = bars, *empty = bars + NSTAGE, *tfull = bars + 2 * NSTAGE, *tempty = bars + 2 * NSTAGE + 2,
           *done = bars + 2 * NSTAGE + 4;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NSTAGE + 5);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ct = blockIdx.x, split = blockIdx.y;
  const int j = blockIdx.z / p.nqc, qc = blockIdx.z % p.nqc;
  const int kb0 = (int)((long long)p.nkb * split / p.nsplit);
  const int kb1 = (int)((long long)p.nkb * (split + 1) / p.nsplit);
  const int nk = kb1 - kb0;
  const int nchunks = (nk + p.kd - 1) / p.kd;
  volatile int *err = p.err;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 8);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, TMEM_COLS);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      const char *Asrc = p.A + (((size_t)j * p.nct + ct) * p.nkb + kb0) * ASTAGE;
      const char *Bsrc = reinterpret_cast<const char *>(p.B) + ((size_t)qc * p.nkb + kb0) * BSTAGE;
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        int s = i % NSTAGE, u = i / NSTAGE;
        if (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1, err, 1)) break;
        tc::mbar_arrive_expect_tx(&full[s], ASTAGE + BSTAGE);
        tc::bulk_g2s(sA + s * ASTAGE, Asrc + (size_t)i * ASTAGE, ASTAGE, &full[s]);
        tc::bulk_g2s(sB + s * BSTAGE, Bsrc + (size_t)i * BSTAGE, BSTAGE, &full[s]);
        issued = i + 1;
      }
      // never leave the CTA with copies still landing in shared memory
      for (int i = max(0, issued - NSTAGE); i < issued; ++i) {
        int s = i % NSTAGE, u = i / NSTAGE;
        long long t0 = clock64();
        while (!tc::mbar_try_wait(&full[s], u & 1) && clock64() - t0 < tc::kSpinLimit) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_f16(MT, 2 * NP);
      const uint32_t aBase = tc::smem_u32(sA), bBase = tc::smem_u32(sB);
      int i = 0;
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        int b = c & 1, ub = c >> 1;
        if (ub > 0 && !tc::mbar_wait(&tempty[b], (ub - 1) & 1, err, 2)) break;
        tc::tc_fence_after();
        const uint32_t d = tbase + (uint32_t)(b * 2 * NP);
        int iend = min(nk, (c + 1) * p.kd);
        for (; i < iend; ++i) {
          int s = i % NSTAGE, u = i / NSTAGE;
          if (!tc::mbar_wait(&full[s], u & 1, err, 3)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          uint32_t a = aBase + s * ASTAGE, bb = bBase + s * BSTAGE;
          // A tiles: 0 Ur hi, 1 Ur lo, 2 Ui hi, 3 Ui lo; B: hl block h at bb + h*3*NP*32,
          // rows [0,NP) = -Im, [NP,2NP) = Re, [2NP,3NP) = Im
          auto dA = [&](int t) { return tc::smem_desc(a + t * ATILE, 128, 256); };
          auto dB = [&](int h, int row0) { return tc::smem_desc(bb + h * 3 * NP * 32 + row0 * 32, 128, 256); };
          uint32_t acc0 = (i == c * p.kd) ? 0u : 1u;
          tc::mma_f16(d, dA(0), dB(0, NP), idesc, acc0);   // Ur_h [Re|Im]_h
          tc::mma_f16(d, dA(0), dB(1, NP), idesc, 1u);     // Ur_h [Re|Im]_l
          tc::mma_f16(d, dA(1), dB(0, NP), idesc, 1u);     // Ur_l [Re|Im]_h
          tc::mma_f16(d, dA(2), dB(0, 0), idesc, 1u);      // Ui_h [-Im|Re]_h
          tc::mma_f16(d, dA(2), dB(1, 0), idesc, 1u);      // Ui_h [-Im|Re]_l
          tc::mma_f16(d, dA(3), dB(0, 0), idesc, 1u);      // Ui_l [-Im|Re]_h
          tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(&tfull[b]);
      }
      tc::mma_commit(done);
      long long t0 = clock64();
      while (!tc::mbar_try_wait(done, 0) && clock64() - t0 < tc::kSpinLimit) {
      }
    }
  } else {
    // drain warps: quadrant = warp % 4 (TMEM lane access rule), half 0 = real, 1 = imag
    const int qd = warp & 3, h = (warp - 2) >> 2;
    const int row = qd * 32 + lane;
    float acc[NP];
#pragma unroll
    for (int n = 0; n < NP; ++n) acc[n] = 0.f;
    for (int c = 0; c < nchunks; ++c) {
      int b = c & 1, ub = c >> 1;
      if (!tc::mbar_wait(&tfull[b], ub & 1, err, 4)) break;
      tc::tc_fence_after();
      const uint32_t t = tbase + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * 2 * NP + h * NP);
#pragma unroll
      for (int n0 = 0; n0 < NP; n0 += 16) {
        float v[16];
        tc::tmem_ld16(t + n0, v);
        tc::tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[n0 + e] += v[e];
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[b]);
    }
    const int col = ct * MT + row;
    const int qend = min(p.nq - qc * 128, NP);
    if (col < p.ncols && !*err) {
      float *out = reinterpret_cast<float *>(p.partial + ((size_t)j * p.nsplit + split) * p.nq * p.ncols);
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (n < qend) out[((size_t)(qc * 128 + n) * p.ncols + col) * 2 + h] = acc[n];
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, TMEM_COLS);
}

// out[j][q][col] = sum over splits of the FP32 partials, in FP64
__global__ void reduce_f64(const float2 *__restrict__ part, int nsplit, size_t per_split,
                           double2 *__restrict__ out, size_t n_out, int nt, size_t out_stride) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_out * nt) return;
  int j = (int)(idx / n_out);
  size_t e = idx % n_out;
  const float2 *pj = part + (size_t)j * nsplit * per_split + e;
  double sx = 0.0, sy = 0.0;
  for (int s = 0; s < nsplit; ++s) {
    float2 v = pj[(size_t)s * per_split];
    sx += v.x;
    sy += v.y;
  }
  out[(size_t)j * out_stride + e] = make_double2(sx, sy);
}

template <int NP>
int launch_mma(const MmaParams &p, int nt, cudaStream_t st) {
  constexpr int BSTAGE = 2 * 3 * NP * 32;
  size_t smem = (size_t)NSTAGE * (ASTAGE + BSTAGE) + 2 * NSTAGE * 8 + 5 * 8 + 16;
  smem = std::max<size_t>(smem, 120 * 1024);   // one CTA per SM: tensor memory is never contended
  static bool attr = false;
  if (!attr) {
    LHC_CHECK_CUDA(cudaFuncSetAttribute(proj_mma<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  dim3 grid(p.nct, p.nsplit, nt * p.nqc);
  proj_mma<NP><<<grid, kThreads, smem, st>>>(p);
  return LHC_OK;
}

int launch_mma_np(int Np, const MmaParams &p, int nt, cudaStream_t st) {
  switch (Np) {
    case 16: return launch_mma<16>(p, nt, st);
    case 32: return launch_mma<32>(p, nt, st);
    case 48: return launch_mma<48>(p, nt, st);
    case 64: return launch_mma<64>(p, nt, st);
    case 80: return launch_mma<80>(p, nt, st);
    case 96: return launch_mma<96>(p, nt, st);
    case 112: return launch_mma<112>(p, nt, st);
    case 128: return launch_mma<128>(p, nt, st);
    default: set_error("unsupported Np %d", Np); return LHC_EINVAL;
  }
}

}  // namespace

// Mixed phase table: cached like the FP64 one (fmt 1).
static int get_phase_split(lhc_ctx ctx, int L, const int *k, int nq, const int r[4], int sign, int Np, int nqc,
                           int nkb, cudaStream_t st, const __half **out) {
  PhaseKey key{L, nq, sign, 1, ((r[0] % L) + L) % L, ((r[1] % L) + L) % L, ((r[2] % L) + L) % L, hash_k(k, nq)};
  auto it = ctx->phases.find(key);
  if (it != ctx->phases.end()) {
    ctx->phase_lru.remove(key);
    ctx->phase_lru.push_front(key);
    *out = static_cast<const __half *>(it->second.buf.p);
    return LHC_OK;
  }
  size_t tbytes = (size_t)nqc * nkb * 2 * 3 * Np * 32;
  size_t off_k = (tbytes + 255) & ~(size_t)255;
  size_t off_roots = (off_k + (size_t)12 * nq + 255) & ~(size_t)255;
  PhaseEntry e;
  LHC_TRY(dev_alloc(ctx, e.buf, off_roots + (size_t)L * sizeof(double2)));
  std::vector<double2> roots(L);
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < L; ++m) roots[m] = make_double2(std::cos(two_pi * m / L), std::sin(two_pi * m / L));
  char *base = static_cast<char *>(e.buf.p);
  LHC_CHECK_CUDA(cudaMemcpy(base + off_k, k, (size_t)12 * nq, cudaMemcpyHostToDevice));
  LHC_CHECK_CUDA(cudaMemcpy(base + off_roots, roots.data(), (size_t)L * sizeof(double2), cudaMemcpyHostToDevice));
  size_t total = (size_t)nqc * nkb * 2 * 3 * Np * KSTEP;
  phase_split_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<__half *>(base), reinterpret_cast<const int *>(base + off_k), nq, Np, nqc, nkb, L, key.rx,
      key.ry, key.rz, sign, reinterpret_cast<const double2 *>(base + off_roots));
  LHC_CHECK_CUDA(cudaGetLastError());
  e.nq_pad = Np;
  ctx->phases[key] = e;
  ctx->phase_lru.push_front(key);
  *out = reinterpret_cast<const __half *>(base);
  return LHC_OK;
}

int run_part_mixed(lhc_ctx ctx, const SliceJob *jobs, int nt, const int *k, int nq, const int r[4], int sign,
                   cudaStream_t st) {
  const SliceJob &j0 = jobs[0];
  if (j0.part == PART_SPEC_BARYON) {
    set_error("mixed baryon spectator not available in this build");
    return LHC_EINVAL;
  }
  const int V3 = j0.V3, n_r = j0.n_r;
  const int ncols = n_r * 192;
  const int nct = (ncols + MT - 1) / MT;
  const int nkb = (V3 + KSTEP - 1) / KSTEP;
  const int nqc = (nq + 127) / 128;
  const int nq_max_chunk = std::min(nq, 128);
  const int Np = ((nq_max_chunk + 15) / 16) * 16;
  const __half *phase = nullptr;
  LHC_TRY(get_phase_split(ctx, j0.L, k, nq, r, sign, Np, nqc, nkb, st, &phase));

  // site-range split so that the grid covers the GPU about twice
  int ctas = nct * nt * nqc;
  int nsplit = std::max(1, std::min(nkb / 8, (2 * ctx->num_sms + ctas - 1) / ctas));
  int kd = 4;   // k-steps accumulated in tensor memory between drains
  // tuning overrides (benchmarks and accuracy studies)
  if (const char *e = getenv("LHC_KD")) kd = std::max(1, atoi(e));
  if (const char *e = getenv("LHC_NSPLIT")) nsplit = std::max(1, std::min(nkb, atoi(e)));

  size_t a_bytes = (size_t)nt * nct * nkb * ASTAGE;
  size_t p_bytes = (size_t)nt * nsplit * nq * ncols * sizeof(float2);
  size_t s_bytes = (size_t)nt * sizeof(SlicePtrs);
  size_t off_p = (a_bytes + 255) & ~(size_t)255;
  size_t off_s = (off_p + p_bytes + 255) & ~(size_t)255;
  size_t off_e = (off_s + s_bytes + 255) & ~(size_t)255;
  LHC_TRY(ensure(ctx, ctx->ws, off_e + 256));
  char *ws = static_cast<char *>(ctx->ws.p);
  std::vector<SlicePtrs> sp(nt);
  for (int j = 0; j < nt; ++j) sp[j] = SlicePtrs{jobs[j].S, jobs[j].vec};
  LHC_CHECK_CUDA(cudaMemcpyAsync(ws + off_s, sp.data(), s_bytes, cudaMemcpyHostToDevice, st));
  int *err = ctx->dev_err;

  {
    size_t threads = (size_t)nt * nct * nkb * MT * 2;
    unsigned grid = (unsigned)((threads + 255) / 256);
    size_t es = j0.dtype == LHC_C128 ? 16 : 8;
    ProfScope ps(ctx, st, LHC_KERNEL_CONTRACT,
                 (double)nt * V3 * (144.0 + 12.0 * n_r) * es + (double)a_bytes);
    const SlicePtrs *spd = reinterpret_cast<const SlicePtrs *>(ws + off_s);
    bool ins = j0.part == PART_INS;
    if (j0.dtype == LHC_C128) {
      if (ins)
        contract_split<double2, 0><<<grid, 256, 0, st>>>(spd, j0.vec_stride, n_r, V3, nct, nkb, j0.g5mask, ws);
      else
        contract_split<double2, 1><<<grid, 256, 0, st>>>(spd, j0.vec_stride, n_r, V3, nct, nkb, j0.g5mask, ws);
    } else {
      if (ins)
        contract_split<float2, 0><<<grid, 256, 0, st>>>(spd, j0.vec_stride, n_r, V3, nct, nkb, j0.g5mask, ws);
      else
        contract_split<float2, 1><<<grid, 256, 0, st>>>(spd, j0.vec_stride, n_r, V3, nct, nkb, j0.g5mask, ws);
    }
  }
  MmaParams mp;
  mp.A = ws;
  mp.B = phase;
  mp.partial = reinterpret_cast<float2 *>(ws + off_p);
  mp.err = err;
  mp.nct = nct;
  mp.nkb = nkb;
  mp.nqc = nqc;
  mp.nq = nq;
  mp.ncols = ncols;
  mp.nsplit = nsplit;
  mp.kd = kd;
  {
    ProfScope ps(ctx, st, LHC_KERNEL_FUSED, 8.0 * nt * (double)nq * ncols * V3);
    LHC_TRY(launch_mma_np(Np, mp, nt, st));
  }
  {
    size_t n_out = (size_t)nq * ncols;
    ProfScope ps(ctx, st, LHC_KERNEL_REDUCE, (double)p_bytes + (double)nt * n_out * 16);
    reduce_f64<<<(unsigned)((n_out * nt + 255) / 256), 256, 0, st>>>(
        mp.partial, nsplit, n_out, j0.out, n_out, nt, n_out);
  }
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

}  // namespace lhc
