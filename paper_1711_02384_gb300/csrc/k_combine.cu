// Noise-averaged combine (Eqs. 5 and 8).
//
// Both cases reduce to  out[t][g][p][q] = (1/N) sum_K Xs[g][p][K] Xi[t][u(g)][q][K]  with
// K = (noise i, spin b, colour c) (12 N values):
//   meson   Xs[g][p][i,b,a] = sum_al Gsrc[b][al] sum_{ap,bp} Gsnk[ap][bp] S[p][i][bp,ap,al,a]
//   baryon  Xs[g][p][i,b,c] = sum Wsnk[a1p][a2p][bp] Wsrc[a1][a2][b] B[p][i][a1p,a1,a2p,a2,bp,c]
//   both    Xi[t][g][q][i,b,c] = sum_{at,bt} Gins[at][bt] I[t][q][i][at,bt,b,c]
// The meson's source structure sits on the spectator side (Eq. 8's sum over the source
// spins regrouped), so the insertion side depends on g only through Gins: it is formed
// for the first g of each distinct Gins matrix, u(g) (gamma_reps), and shared.
// Precision: LHC_FP64 does everything in double.  LHC_MIXED does the Gamma contractions and
// the spin-colour sums of each pair of noises in FP32; the sum over those (the noise
// average of Eq. 5) is exact: each pair's term is added with Knuth's TwoSum into an
// unevaluated FP32 pair hi + lo, rounded once to FP64 (no less accurate than FP64
// accumulation of those terms, and it keeps GB300's slow FP64 pipe out of the inner loop).
#include <algorithm>
#include <type_traits>

#include "conv.cuh"
#include "lhc_internal.h"

namespace lhc {
namespace {

template <typename R>
struct cplx {
  R x, y;
};

template <typename R>
__device__ __forceinline__ cplx<R> ld(const double2 *p) {
  double2 v = *p;
  if constexpr (std::is_same<R, float>::value)
    return {f64_to_f32_rne(v.x), f64_to_f32_rne(v.y)};   // integer conversion, off the FP64 pipe
  else
    return {v.x, v.y};
}
template <typename R>
__device__ __forceinline__ void cfma(cplx<R> &acc, cplx<R> a, cplx<R> b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
template <typename R>
__device__ __forceinline__ void st(double2 *p, cplx<R> v) {
  *p = make_double2((double)v.x, (double)v.y);
}

// Stage one [n_r][cols] block (and the Gamma matrices) of an input in shared memory and
// let the CTA's threads serve all (g, i, colour) tasks of that block from there.  Each
// thread issues its loads four at a time before converting and storing any of them, so
// a thread waits for one memory latency per four values instead of one per value.
template <typename R, typename Dst>
__device__ __forceinline__ void stage_batched(const double2 *src, int n, Dst dst_index, cplx<R> *dst) {
  constexpr int U = 4;
  const int step = blockDim.x;
  for (int e0 = threadIdx.x; e0 < n; e0 += U * step) {
    double2 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e0 + u * step < n) v[u] = src[e0 + u * step];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * step;
      if (e < n) {
        if constexpr (std::is_same<R, float>::value)
          dst[dst_index(e)] = cplx<R>{f64_to_f32_rne(v[u].x), f64_to_f32_rne(v[u].y)};
        else
          dst[dst_index(e)] = cplx<R>{v[u].x, v[u].y};
      }
    }
  }
}
template <typename R>
__device__ __forceinline__ void stage(cplx<R> *dst, const double2 *src, int n) {
  stage_batched<R>(src, n, [](int e) { return e; }, dst);
}
// The per-noise blocks of 192 values are staged 193 apart: consecutive tasks belong to
// different noises, and a stride of 192 complex numbers would put them in one bank.
constexpr int SROW = 193;
template <typename R>
__device__ __forceinline__ void stage_rows(cplx<R> *dst, const double2 *src, int n_r) {
  stage_batched<R>(src, n_r * 192, [](int e) { return (e / 192) * SROW + e % 192; }, dst);
}

// Distinct Gamma_ins matrices: umap[g] = the first g' <= g whose matrix equals Gins[g]
// entry for entry.  The insertion part with Gamma_ins applied is formed once per distinct
// matrix, and every g reads that of umap[g] (the 16 structures of a sweep at sink and
// source often share one insertion current).
__global__ void gamma_reps(const double2 *__restrict__ G, int ng, int *__restrict__ umap) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ng) return;
  int rep = g;
  for (int h = 0; h < g && rep == g; ++h) {
    bool same = true;
    for (int e = 0; e < 16 && same; ++e) {
      const double2 x = G[h * 16 + e], y = G[g * 16 + e];
      same = x.x == y.x && x.y == y.y;
    }
    if (same) rep = h;
  }
  umap[g] = rep;
}
constexpr int kMaxGamma = 512;

// CTA per (t, q): Xi[t][g][q][i,b,c] = sum_{at,bt} Gins[g][at][bt] I[t][q][i][at,bt,b,c] for
// the representatives g (umap[g] == g) only: the insertion part with Gamma_ins applied,
// spins (b, c) left for the spectator side
// (FP32: at most 64 registers, so that four CTAs share an SM; the kernel spends its time
// staging the insertion part, and more CTAs keep more of those loads in flight)
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1)
    comb_ins_gamma(const double2 *__restrict__ I, int nq, int n_r, int nch, const double2 *__restrict__ Gins,
                   const int *__restrict__ umap, int ng, cplx<R> *__restrict__ Xi) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int reps[kMaxGamma];
  __shared__ int nrep;
  cplx<R> *sGi = reinterpret_cast<cplx<R> *>(sm_raw), *sI = sGi + 2 * ng * 16;
  const int tq = blockIdx.x, t = tq / nq, q = tq % nq;
  if (threadIdx.x < 32) {   // the representatives in order, by ballot
    int n = 0;
    for (int g0 = 0; g0 < ng; g0 += 32) {
      const int g = g0 + (int)threadIdx.x;
      const bool r = g < ng && umap[g] == g;
      const unsigned m = __ballot_sync(0xffffffffu, r);
      if (r) reps[n + __popc(m & ((1u << threadIdx.x) - 1u))] = g;
      n += __popc(m);
    }
    if (threadIdx.x == 0) nrep = n;
  }
  stage(sGi, Gins, ng * 16);
  for (int i0 = 0; i0 < n_r; i0 += nch) {
  const int nc = min(nch, n_r - i0);
  __syncthreads();
  stage_rows(sI, I + ((size_t)tq * n_r + i0) * 192, nc);
  __syncthreads();
  for (int task = threadIdx.x; task < nrep * nc * 3; task += blockDim.x) {
    const int c = task % 3, ii = (task / 3) % nc, g = reps[task / (3 * nc)], i = i0 + ii;
    const cplx<R> *v = sI + ii * SROW, *Gi = sGi + g * 16;
    cplx<R> *o = Xi + (((size_t)t * ng + g) * nq + q) * 12 * n_r + i * 12 + c;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      cplx<R> acc{0, 0};
#pragma unroll
      for (int at = 0; at < 4; ++at)
#pragma unroll
        for (int bt = 0; bt < 4; ++bt) cfma(acc, Gi[at * 4 + bt], v[at * 48 + bt * 12 + b * 3 + c]);
      o[b * 3] = acc;
    }
  }
  }
}

// CTA per p: Xs[g][p][i,al,a] = sum_{ap,bp} Gsnk[g][ap][bp] S[p][i][bp,ap,al,a]; with
// Gsrc given, the source structure is applied here too, on the spectator's side:
// Xs[g][p][i,b,a] = sum_al Gsrc[g][b][al] (the sum above), so that the insertion part needs
// Gamma_ins only (sum_{al,b} Xs_al Gsrc[b][al] Ins_b regrouped)
template <typename R>
__global__ void comb_spec_meson(const double2 *__restrict__ S, int np, int n_r, int nch, const double2 *__restrict__ Gsnk,
                                const double2 *__restrict__ Gsrc, int ng, cplx<R> *__restrict__ Xs) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<R> *sG = reinterpret_cast<cplx<R> *>(sm_raw), *sGc = sG + ng * 16, *sS = sG + 2 * ng * 16;
  const int p = blockIdx.x;
  stage(sG, Gsnk, ng * 16);
  if (Gsrc) stage(sGc, Gsrc, ng * 16);
  for (int i0 = 0; i0 < n_r; i0 += nch) {
  const int nc = min(nch, n_r - i0);
  __syncthreads();
  stage_rows(sS, S + ((size_t)p * n_r + i0) * 192, nc);
  __syncthreads();
  for (int task = threadIdx.x; task < ng * nc * 3; task += blockDim.x) {
    const int a = task % 3, ii = (task / 3) % nc, g = task / (3 * nc), i = i0 + ii;
    const cplx<R> *s = sS + ii * SROW, *G = sG + g * 16;
    cplx<R> *o = Xs + ((size_t)g * np + p) * 12 * n_r + i * 12 + a;
    cplx<R> x[4];
#pragma unroll
    for (int al = 0; al < 4; ++al) {
      x[al] = {0, 0};
#pragma unroll
      for (int ap = 0; ap < 4; ++ap)
#pragma unroll
        for (int bp = 0; bp < 4; ++bp) cfma(x[al], G[ap * 4 + bp], s[bp * 48 + ap * 12 + al * 3 + a]);
    }
    if (Gsrc) {
      const cplx<R> *Gc = sGc + g * 16;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        cplx<R> acc{0, 0};
#pragma unroll
        for (int al = 0; al < 4; ++al) cfma(acc, Gc[b * 4 + al], x[al]);
        o[b * 3] = acc;
      }
    } else {
#pragma unroll
      for (int al = 0; al < 4; ++al) o[al * 3] = x[al];
    }
  }
  }
}

// one thread per (g, p, i, c): Bhat[a1][a2] = sum Wsnk B, then the four b values.  The sums
// (64 terms, then 16) run in FP64 in both precisions and are rounded once to R: in FP32
// their rounding would be the largest error of the mixed baryon combine, and the kernel
// is small beside the GEMM.
template <typename R>
__global__ void comb_spec_baryon(const double2 *__restrict__ B, int np, int n_r, const double2 *__restrict__ Wsnk,
                                 const double2 *__restrict__ Wsrc, int ng, cplx<R> *__restrict__ Xs) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)ng * np * n_r * 3) return;
  int c = (int)(idx % 3);
  size_t rest = idx / 3;
  int i = (int)(rest % n_r);
  rest /= n_r;
  int p = (int)(rest % np), g = (int)(rest / np);
  const double2 *s = B + ((size_t)p * n_r + i) * 3072;
  const double2 *Ws = Wsnk + (size_t)g * 64;
  const double2 *Wc = Wsrc + (size_t)g * 64;
  cplx<double> out[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
#pragma unroll 1
  for (int a1 = 0; a1 < 4; ++a1)
#pragma unroll 1
    for (int a2 = 0; a2 < 4; ++a2) {
      cplx<double> h{0, 0};
#pragma unroll 1
      for (int a1p = 0; a1p < 4; ++a1p)
#pragma unroll
        for (int a2p = 0; a2p < 4; ++a2p)
#pragma unroll
          for (int bp = 0; bp < 4; ++bp)
            cfma(h, ld<double>(Ws + (a1p * 4 + a2p) * 4 + bp),
                 ld<double>(s + ((((a1p * 4 + a1) * 4 + a2p) * 4 + a2) * 4 + bp) * 3 + c));
#pragma unroll
      for (int b = 0; b < 4; ++b) cfma(out[b], ld<double>(Wc + (a1 * 4 + a2) * 4 + b), h);
    }
  cplx<R> *o = Xs + ((size_t)g * np + p) * 12 * n_r + i * 12 + c;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    if constexpr (std::is_same<R, float>::value)
      o[b * 3] = cplx<R>{f64_to_f32_rne(out[b].x), f64_to_f32_rne(out[b].y)};
    else
      o[b * 3] = out[b];
  }
}

// CTA per (p, i), the source spins left open:
//   Xs[g][p][i][(a1*4 + a2)*3 + c] = sum_{a1p,a2p,bp} Wsnk[g][a1p][a2p][bp] B[p][i][a1p,a1,a2p,a2,bp,c]
// The noise's 3072 values and the ng Wsnk tensors are staged in shared memory; a task is
// one (g, a1, a2, c).
// As in the closed form, the 64-term sums run in FP64 in both precisions (the noise's
// values and the W tensors staged in double) and are rounded once to R.
template <typename R>
__global__ void comb_spec_baryon_open(const double2 *__restrict__ B, int np, int n_r, const double2 *__restrict__ Wsnk,
                                      int ng, cplx<R> *__restrict__ Xs) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<double> *sW = reinterpret_cast<cplx<double> *>(sm_raw), *sB = sW + ng * 64;
  const int pi = blockIdx.x, p = pi / n_r, i = pi % n_r;
  stage(sW, Wsnk, ng * 64);
  stage(sB, B + (size_t)pi * 3072, 3072);
  __syncthreads();
  for (int task = threadIdx.x; task < ng * 48; task += blockDim.x) {
    const int c = task % 3, a2 = (task / 3) % 4, a1 = (task / 12) % 4, g = task / 48;
    const cplx<double> *W = sW + g * 64;
    cplx<double> h{0, 0};
#pragma unroll
    for (int a1p = 0; a1p < 4; ++a1p)
#pragma unroll
      for (int a2p = 0; a2p < 4; ++a2p)
#pragma unroll
        for (int bp = 0; bp < 4; ++bp)
          cfma(h, W[(a1p * 4 + a2p) * 4 + bp], sB[((((a1p * 4 + a1) * 4 + a2p) * 4 + a2) * 4 + bp) * 3 + c]);
    cplx<R> *o = Xs + (((size_t)g * np + p) * n_r + i) * 48 + task % 48;
    if constexpr (std::is_same<R, float>::value)
      *o = cplx<R>{f64_to_f32_rne(h.x), f64_to_f32_rne(h.y)};
    else
      *o = h;
  }
}

// Sum over noises of the per-noise terms: in double for R = double; for R = float an
// unevaluated pair hi + lo per component, each term added with Knuth's TwoSum (the pair
// holds the sum exactly up to the rounding of lo), rounded once to double at the end.
template <typename R>
struct NoiseSum {
  double x = 0.0, y = 0.0;
  __device__ __forceinline__ void add(cplx<R> v) {
    x += (double)v.x;
    y += (double)v.y;
  }
  __device__ __forceinline__ double2 get(double scale, float) const { return make_double2(x * scale, y * scale); }
};
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float v) {
  const float s = hi + v, bp = s - hi;
  lo += (hi - (s - bp)) + (v - bp);
  hi = s;
}
template <>
struct NoiseSum<float> {
  float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
  __device__ __forceinline__ void add(cplx<float> v) {
    two_sum_acc(hx, lx, v.x);
    two_sum_acc(hy, ly, v.y);
  }
  // (hi + lo) * scale rounded once to FP64; a power-of-two scale (1/N for N = 2^m) is
  // applied to hi and lo in FP32 without error (barring underflow), which leaves one
  // FP64 addition per component
  __device__ __forceinline__ double2 get(double scale, float scale_pow2) const {
    if (scale_pow2 != 0.f)
      return make_double2(f32_to_f64(hx * scale_pow2) + f32_to_f64(lx * scale_pow2),
                          f32_to_f64(hy * scale_pow2) + f32_to_f64(ly * scale_pow2));
    return make_double2((f32_to_f64(hx) + f32_to_f64(lx)) * scale, (f32_to_f64(hy) + f32_to_f64(ly)) * scale);
  }
};

// out[t][g][p][q] = (1/N) sum_i sum_{j<12} Xs[g][p][12i+j] Xi[t][g][q][12i+j]: a tiled complex
// GEMM whose 24-term sums over two noises run in R (float or double) and whose sum of
// those over the noise pairs is the NoiseSum above.  A CTA computes a TP x TQ tile of (p, q) for one (t, g);
// thread (ty, tx) of 16 x 16 holds p = p0 + ty + 16 a (a < 2) and q = q0 + tx + 16 b
// (b < 3).  KN noises (12 KN values of K) are staged per pass (4 in FP32, 2 in FP64: the
// static shared memory stays below 48 KB); rows are padded by one element so that the
// 16 q rows a warp reads fall into distinct banks.
constexpr int TP = 32, TQ = 48;

// Rows r0 .. r0 + ROWS - 1 (those below nrow), columns k0 .. k0 + kw - 1 of a row-major
// [nrow][ldk] matrix into a [ROWS][KW] shared tile (zeros outside); a thread issues its
// loads in groups of three before storing them.
template <typename R, int ROWS, int COLS, int KW>
__device__ __forceinline__ void stage_tile(cplx<R> *dst, const cplx<R> *src, size_t ldk, int k0, int r0, int nrow,
                                           int kw) {
  constexpr int N = ROWS * COLS, G = 3;
  for (int e0 = threadIdx.x; e0 < N; e0 += G * 256) {
    cplx<R> v[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int e = e0 + 256 * u, r = e / COLS, k = e % COLS;
      v[u] = (e < N && r0 + r < nrow && k < kw) ? src[(size_t)(r0 + r) * ldk + k0 + k] : cplx<R>{0, 0};
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int e = e0 + 256 * u;
      if (e < N) dst[(e / COLS) * KW + e % COLS] = v[u];
    }
  }
}
template <typename R>
__global__ void __launch_bounds__(256) comb_gemm(const cplx<R> *__restrict__ Xs, const cplx<R> *__restrict__ Xi,
                                                 const int *__restrict__ umap, int np, int nq, int n_r, int ng,
                                                 double inv_n, float inv_n_pow2, double2 *__restrict__ out) {
  constexpr int KN = sizeof(R) == 4 ? 4 : 2, KW = 12 * KN + 1;
  __shared__ cplx<R> As[TP * KW];
  __shared__ cplx<R> Bs[TQ * KW];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int q0 = blockIdx.x * TQ, p0 = blockIdx.y * TP;
  const int tg = blockIdx.z;   // t * ng + g
  const int g = tg % ng;
  const size_t K = (size_t)12 * n_r;
  const cplx<R> *A = Xs + ((size_t)g * np) * K;
  const cplx<R> *B = Xi + ((size_t)(tg - g + umap[g]) * nq) * K;   // the insertion part of g's Gamma_ins
  NoiseSum<R> acc[2][3];
  for (int i0 = 0; i0 < n_r; i0 += KN) {
    const int kw = 12 * min(KN, n_r - i0);
    // all of a thread's loads of the pass are issued before any is stored (one memory
    // latency per pass, not one per value)
    stage_tile<R, TP, 12 * KN, KW>(As, A, K, 12 * i0, p0, np, kw);
    stage_tile<R, TQ, 12 * KN, KW>(Bs, B, K, 12 * i0, q0, nq, kw);
    __syncthreads();
    // two noises (24 terms) per partial sum; a missing second noise is staged as zeros
    for (int ii = 0; ii < kw / 12; ii += 2) {
      cplx<R> pa[2][3];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) pa[a][b] = cplx<R>{0, 0};
      const cplx<R> *ar = As + ty * KW + 12 * ii, *br = Bs + tx * KW + 12 * ii;
#pragma unroll
      for (int k = 0; k < 24; ++k) {
        const cplx<R> a0 = ar[k], a1 = ar[16 * KW + k];
        const cplx<R> b0 = br[k], b1 = br[16 * KW + k], b2 = br[32 * KW + k];
        cfma(pa[0][0], a0, b0);
        cfma(pa[0][1], a0, b1);
        cfma(pa[0][2], a0, b2);
        cfma(pa[1][0], a1, b0);
        cfma(pa[1][1], a1, b1);
        cfma(pa[1][2], a1, b2);
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) acc[a][b].add(pa[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int p = p0 + ty + 16 * a, q = q0 + tx + 16 * b;
      if (p < np && q < nq) out[((size_t)tg * np + p) * nq + q] = acc[a][b].get(inv_n, inv_n_pow2);
    }
}

// Open-source-spin combine:
//   O[t][gs][gi][p][q][e][be] = (1/N) sum_{i,a} Xs[gs][p][i,e,a] Xi[t][gi][q][i,be,a]
// with Xi the insertion part with Gamma_ins applied (comb_ins_gamma, which applies
// Gamma_ins only) and Xs the spectator part with the sink structure applied: for a
// meson e = al (RS = 4 open row spins, comb_spec_meson), for a baryon e = (a1, a2)
// (RS = 16, comb_spec_baryon_open).  Rows are (p, e), columns (q, be); the tiling is
// comb_gemm's, with KN noises of three colours staged per pass and four noises (12
// terms) per partial sum.
template <typename R, int RS>
__global__ void __launch_bounds__(256) comb_gemm_open(const cplx<R> *__restrict__ Xs, const cplx<R> *__restrict__ Xi,
                                                      const int *__restrict__ umap, int np, int nq, int n_r, int ngs,
                                                      int ngi, double inv_n, float inv_n_pow2,
                                                      double2 *__restrict__ out) {
  constexpr int KN = sizeof(R) == 4 ? 8 : 4, KW = 3 * KN + 1;
  __shared__ cplx<R> As[TP * KW];
  __shared__ cplx<R> Bs[TQ * KW];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int c0 = blockIdx.x * TQ, r0 = blockIdx.y * TP;
  const int z = blockIdx.z, gi = z % ngi, gs = (z / ngi) % ngs, t = z / (ngi * ngs);
  const cplx<R> *A = Xs + (size_t)gs * np * 3 * RS * n_r;             // [p][i][e][a]
  const cplx<R> *B = Xi + ((size_t)t * ngi + umap[gi]) * nq * 12 * n_r;   // [q][i][be][a]
  NoiseSum<R> acc[2][3];
  for (int i0 = 0; i0 < n_r; i0 += KN) {
    const int kn = min(KN, n_r - i0);
    for (int e = threadIdx.x; e < TP * 3 * KN; e += 256) {
      const int r = e / (3 * KN), k = e % (3 * KN), ii = k / 3, a = k % 3, R_ = r0 + r;
      As[r * KW + k] = (R_ < RS * np && ii < kn) ? A[((size_t)(R_ / RS) * n_r + i0 + ii) * 3 * RS + (R_ % RS) * 3 + a]
                                                 : cplx<R>{0, 0};
    }
    for (int e = threadIdx.x; e < TQ * 3 * KN; e += 256) {
      const int r = e / (3 * KN), k = e % (3 * KN), ii = k / 3, a = k % 3, C_ = c0 + r;
      Bs[r * KW + k] = (C_ < 4 * nq && ii < kn) ? B[((size_t)(C_ >> 2) * n_r + i0 + ii) * 12 + (C_ & 3) * 3 + a]
                                                : cplx<R>{0, 0};
    }
    __syncthreads();
    for (int ii = 0; ii < kn; ii += 4) {   // missing noises of a group of four are staged as zeros
      cplx<R> pa[2][3];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) pa[a][b] = cplx<R>{0, 0};
      const cplx<R> *ar = As + ty * KW + 3 * ii, *br = Bs + tx * KW + 3 * ii;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const cplx<R> a0 = ar[k], a1 = ar[16 * KW + k];
        const cplx<R> b0 = br[k], b1 = br[16 * KW + k], b2 = br[32 * KW + k];
        cfma(pa[0][0], a0, b0);
        cfma(pa[0][1], a0, b1);
        cfma(pa[0][2], a0, b2);
        cfma(pa[1][0], a1, b0);
        cfma(pa[1][1], a1, b1);
        cfma(pa[1][2], a1, b2);
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) acc[a][b].add(pa[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int R_ = r0 + ty + 16 * a, C_ = c0 + tx + 16 * b;
      if (R_ < RS * np && C_ < 4 * nq)
        out[(((size_t)z * np + R_ / RS) * nq + (C_ >> 2)) * 4 * RS + (R_ % RS) * 4 + (C_ & 3)] =
            acc[a][b].get(inv_n, inv_n_pow2);
    }
}

unsigned blocks(size_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

// The staging kernels may take up to 200 KB of dynamic shared memory (set once per device).
template <typename R>
int staging_smem_limits() {
  static std::atomic<unsigned long long> d1{0}, d2{0};
  LHC_TRY(ensure_smem_limit(comb_ins_gamma<R>, 200 * 1024, d1));
  LHC_TRY(ensure_smem_limit(comb_spec_meson<R>, 200 * 1024, d2));
  return LHC_OK;
}

// Noises staged per pass by the staging kernels, and their shared memory: as many as fit
// 96 KB next to the 2 ng Gamma matrices (two CTAs per SM), at least one.
template <typename R>
int noise_chunk(int ng, int n_r, int *nch, size_t *smem) {
  const size_t g_bytes = (size_t)2 * ng * 16 * sizeof(cplx<R>), row = (size_t)SROW * sizeof(cplx<R>);
  if (g_bytes + row > 200 * 1024 || ng > kMaxGamma) {
    set_error("combine: %d Gamma structures do not fit shared memory", ng);
    return LHC_EINVAL;
  }
  *nch = (int)std::min<size_t>((size_t)n_r, g_bytes + row <= 96 * 1024 ? (96 * 1024 - g_bytes) / row : 1);
  *smem = g_bytes + (size_t)*nch * row;
  if (*smem > 48 * 1024) LHC_TRY(staging_smem_limits<R>());
  return LHC_OK;
}

// Shared memory of comb_spec_baryon_open: one noise's 3072 values and ng Wsnk tensors.
template <typename R>
int spec_open_smem(int ng, size_t *smem) {
  *smem = ((size_t)ng * 64 + 3072) * sizeof(cplx<double>);   // staged in double in both precisions
  if (*smem > 200 * 1024) {
    set_error("combine_open: %d sink structures do not fit shared memory", ng);
    return LHC_EINVAL;
  }
  if (*smem > 48 * 1024) {
    static std::atomic<unsigned long long> done{0};
    LHC_TRY(ensure_smem_limit(comb_spec_baryon_open<R>, 200 * 1024, done));
  }
  return LHC_OK;
}

// The distinct Gamma_ins matrices (umap, gamma_reps), then the spectator part with the
// sink (and, closed, the source) structures applied, the insertion part with Gamma_ins
// applied once per distinct matrix, and the GEMM.  Scratch: Xs, Xi, then ng ints of umap.
template <typename R>
int launch_combine_open(int kind, const double2 *spec, int np, const double2 *ins, int nq, int n_r, int nt,
                        const double2 *snk, int ngs, const double2 *ins_g, int ngi, void *scratch, double2 *out,
                        cudaStream_t st) {
  const int RS = kind == LHC_MESON ? 4 : 16;
  cplx<R> *Xs = static_cast<cplx<R> *>(scratch);
  cplx<R> *Xi = Xs + (size_t)ngs * np * 3 * RS * n_r;
  int *umap = reinterpret_cast<int *>(Xi + (size_t)nt * ngi * nq * 12 * n_r);
  int nch;
  size_t smem;
  gamma_reps<<<blocks(ngi, 128), 128, 0, st>>>(ins_g, ngi, umap);
  note_launch();
  if (kind == LHC_MESON) {
    LHC_TRY(noise_chunk<R>(ngs, n_r, &nch, &smem));
    comb_spec_meson<R><<<np, 256, smem, st>>>(spec, np, n_r, nch, snk, nullptr, ngs, Xs);
  } else {
    LHC_TRY(spec_open_smem<R>(ngs, &smem));
    comb_spec_baryon_open<R><<<np * n_r, 256, smem, st>>>(spec, np, n_r, snk, ngs, Xs);
  }
  note_launch();
  LHC_TRY(noise_chunk<R>(ngi, n_r, &nch, &smem));
  comb_ins_gamma<R><<<nt * nq, 256, smem, st>>>(ins, nq, n_r, nch, ins_g, umap, ngi, Xi);   // Gamma_ins only
  note_launch();
  const dim3 grid((4 * nq + TQ - 1) / TQ, (RS * np + TP - 1) / TP, nt * ngs * ngi);
  const float inv_pow2 = (n_r & (n_r - 1)) == 0 ? 1.0f / (float)n_r : 0.0f;   // exact for N = 2^m
  if (kind == LHC_MESON)
    comb_gemm_open<R, 4><<<grid, 256, 0, st>>>(Xs, Xi, umap, np, nq, n_r, ngs, ngi, 1.0 / n_r, inv_pow2, out);
  else
    comb_gemm_open<R, 16><<<grid, 256, 0, st>>>(Xs, Xi, umap, np, nq, n_r, ngs, ngi, 1.0 / n_r, inv_pow2, out);
  note_launch();
  return LHC_OK;
}

template <typename R>
int launch_combine(int kind, const double2 *spec, int np, const double2 *ins, int nq, int n_r, int nt,
                   const double2 *snk, const double2 *ins_g, const double2 *src, int ng, void *scratch,
                   double2 *out, cudaStream_t st) {
  cplx<R> *Xs = static_cast<cplx<R> *>(scratch);
  cplx<R> *Xi = Xs + (size_t)ng * np * 12 * n_r;
  int *umap = reinterpret_cast<int *>(Xi + (size_t)nt * ng * nq * 12 * n_r);
  int nch;
  size_t smem;
  LHC_TRY(noise_chunk<R>(ng, n_r, &nch, &smem));
  gamma_reps<<<blocks(ng, 128), 128, 0, st>>>(ins_g, ng, umap);
  note_launch();
  if (kind == LHC_MESON) {
    comb_spec_meson<R><<<np, 256, smem, st>>>(spec, np, n_r, nch, snk, src, ng, Xs);
  } else {
    size_t ns = (size_t)ng * np * n_r * 3;
    comb_spec_baryon<R><<<blocks(ns, 128), 128, 0, st>>>(spec, np, n_r, snk, src, ng, Xs);
  }
  note_launch();
  comb_ins_gamma<R><<<nt * nq, 256, smem, st>>>(ins, nq, n_r, nch, ins_g, umap, ng, Xi);
  note_launch();
  dim3 grid((nq + TQ - 1) / TQ, (np + TP - 1) / TP, nt * ng);
  const float inv_pow2 = (n_r & (n_r - 1)) == 0 ? 1.0f / (float)n_r : 0.0f;   // exact for N = 2^m
  comb_gemm<R><<<grid, 256, 0, st>>>(Xs, Xi, umap, np, nq, n_r, ng, 1.0 / n_r, inv_pow2, out);
  note_launch();
  return LHC_OK;
}

}  // namespace

int run_combine(lhc_ctx ctx, int kind, const double2 *spec, int np, const double2 *ins, int nq, int n_r, int nt,
                const double2 *snk, const double2 *ins_g, const double2 *src, int ng, int prec, double2 *out,
                cudaStream_t st) {
  const size_t es = prec == LHC_MIXED ? sizeof(cplx<float>) : sizeof(cplx<double>);
  const size_t K = (size_t)12 * n_r;
  LHC_TRY(ensure(ctx, ctx->ws, ((size_t)ng * np * K + (size_t)nt * ng * nq * K) * es + (size_t)ng * sizeof(int)));
  ProfScope ps(ctx, st, LHC_KERNEL_COMBINE, 8.0 * nt * ng * (double)np * nq * K);
  if (prec == LHC_MIXED)
    LHC_TRY(launch_combine<float>(kind, spec, np, ins, nq, n_r, nt, snk, ins_g, src, ng, ctx->ws.p, out, st));
  else
    LHC_TRY(launch_combine<double>(kind, spec, np, ins, nq, n_r, nt, snk, ins_g, src, ng, ctx->ws.p, out, st));
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

// The same kernels on caller-provided scratch (room for ng*np*12*n_r + nt*ng*nq*12*n_r
// complex values of the precision, then ng ints); no allocation and no context.
int run_combine_scratch(int kind, const double2 *spec, int np, const double2 *ins, int nq, int n_r, int nt,
                        const double2 *snk, const double2 *ins_g, const double2 *src, int ng, int prec,
                        double2 *Xs, double2 *Xi, double2 *out, cudaStream_t st) {
  (void)Xi;   // the intermediates are laid out from Xs on
  if (prec == LHC_MIXED)
    LHC_TRY(launch_combine<float>(kind, spec, np, ins, nq, n_r, nt, snk, ins_g, src, ng, Xs, out, st));
  else
    LHC_TRY(launch_combine<double>(kind, spec, np, ins, nq, n_r, nt, snk, ins_g, src, ng, Xs, out, st));
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

int run_combine_open(lhc_ctx ctx, int kind, const double2 *spec, int np, const double2 *ins, int nq, int n_r, int nt,
                     const double2 *snk, int ngs, const double2 *ins_g, int ngi, int prec, double2 *out,
                     cudaStream_t st) {
  if ((size_t)nt * ngs * ngi > 65535) {
    set_error("combine_open: nt * ngs * ngi = %lld exceeds 65535", (long long)nt * ngs * ngi);
    return LHC_EINVAL;
  }
  const int RS = kind == LHC_MESON ? 4 : 16;
  if ((size_t)RS * np > 65535u * TP) {
    set_error("combine_open: %d sink momenta exceed the grid", np);
    return LHC_EINVAL;
  }
  const size_t es = prec == LHC_MIXED ? sizeof(cplx<float>) : sizeof(cplx<double>);
  const size_t K = (size_t)3 * n_r;   // (noise, colour)
  LHC_TRY(ensure(ctx, ctx->ws, ((size_t)ngs * np * RS * K + (size_t)nt * ngi * nq * 4 * K) * es + (size_t)ngi * sizeof(int)));
  ProfScope ps(ctx, st, LHC_KERNEL_COMBINE, 8.0 * nt * ngs * ngi * (double)RS * np * 4.0 * nq * K);
  if (prec == LHC_MIXED)
    LHC_TRY(launch_combine_open<float>(kind, spec, np, ins, nq, n_r, nt, snk, ngs, ins_g, ngi, ctx->ws.p, out, st));
  else
    LHC_TRY(launch_combine_open<double>(kind, spec, np, ins, nq, n_r, nt, snk, ngs, ins_g, ngi, ctx->ws.p, out, st));
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

}  // namespace lhc
