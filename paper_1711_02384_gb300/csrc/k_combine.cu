// Noise-averaged combine (Eqs. 5 and 8) in FP64.
//
// Both cases reduce to  out[g][p][q] = (1/N) sum_K Xs[g][p][K] Xi[g][q][K]  with
// K = (noise i, spin j, colour c) (12 N values):
//   meson   Xs[g][p][i,al,a] = sum_{ap,bp} Gsnk[ap][bp] S[p][i][bp,ap,al,a]
//           Xi[g][q][i,al,a] = sum_b Gsrc[b][al] sum_{at,bt} Gins[at][bt] I[q][i][at,bt,b,a]
//   baryon  Xs[g][p][i,b,c]  = sum Wsnk[a1p][a2p][bp] Wsrc[a1][a2][b] B[p][i][a1p,a1,a2p,a2,bp,c]
//           Xi[g][q][i,b,c]  = sum_{at,bt} Gins[at][bt] I[q][i][at,bt,b,c]
// for every insertion slice t of the call.
#include <type_traits>

#include "lhc_internal.h"

namespace lhc {
namespace {

__device__ __forceinline__ void cfma(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}

// one thread per (g, p, K)
__global__ void comb_spec_meson(const double2 *__restrict__ S, int np, int n_r,
                                const double2 *__restrict__ Gsnk, int ng, double2 *__restrict__ Xs) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t K = (size_t)12 * n_r;
  if (idx >= (size_t)ng * np * K) return;
  int kk = (int)(idx % K);
  size_t rest = idx / K;
  int p = (int)(rest % np), g = (int)(rest / np);
  int i = kk / 12, al = (kk / 3) & 3, a = kk % 3;
  const double2 *s = S + ((size_t)p * n_r + i) * 192;
  const double2 *G = Gsnk + (size_t)g * 16;
  double2 acc = make_double2(0.0, 0.0);
  for (int ap = 0; ap < 4; ++ap)
    for (int bp = 0; bp < 4; ++bp) cfma(acc, G[ap * 4 + bp], s[bp * 48 + ap * 12 + al * 3 + a]);
  Xs[idx] = acc;
}

__global__ void comb_ins_meson(const double2 *__restrict__ I, int nq, int n_r,
                               const double2 *__restrict__ Gins, const double2 *__restrict__ Gsrc,
                               int ng, double2 *__restrict__ Xi) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t K = (size_t)12 * n_r;
  if (idx >= (size_t)ng * nq * K) return;
  int kk = (int)(idx % K);
  size_t rest = idx / K;
  int q = (int)(rest % nq), g = (int)(rest / nq);
  int i = kk / 12, al = (kk / 3) & 3, a = kk % 3;
  const double2 *v = I + ((size_t)q * n_r + i) * 192;
  const double2 *Gi = Gins + (size_t)g * 16;
  const double2 *Gc = Gsrc + (size_t)g * 16;
  double2 acc = make_double2(0.0, 0.0);
  for (int b = 0; b < 4; ++b) {
    double2 t = make_double2(0.0, 0.0);
    for (int at = 0; at < 4; ++at)
      for (int bt = 0; bt < 4; ++bt) cfma(t, Gi[at * 4 + bt], v[at * 48 + bt * 12 + b * 3 + a]);
    cfma(acc, Gc[b * 4 + al], t);
  }
  Xi[idx] = acc;
}

__global__ void comb_spec_baryon(const double2 *__restrict__ B, int np, int n_r,
                                 const double2 *__restrict__ Wsnk, const double2 *__restrict__ Wsrc,
                                 int ng, double2 *__restrict__ Xs) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t K = (size_t)12 * n_r;
  if (idx >= (size_t)ng * np * K) return;
  int kk = (int)(idx % K);
  size_t rest = idx / K;
  int p = (int)(rest % np), g = (int)(rest / np);
  int i = kk / 12, b = (kk / 3) & 3, c = kk % 3;
  const double2 *s = B + ((size_t)p * n_r + i) * 3072;
  const double2 *Ws = Wsnk + (size_t)g * 64;
  const double2 *Wc = Wsrc + (size_t)g * 64;
  double2 acc = make_double2(0.0, 0.0);
  for (int a1 = 0; a1 < 4; ++a1)
    for (int a2 = 0; a2 < 4; ++a2) {
      double2 t = make_double2(0.0, 0.0);
      for (int a1p = 0; a1p < 4; ++a1p)
        for (int a2p = 0; a2p < 4; ++a2p)
          for (int bp = 0; bp < 4; ++bp)
            cfma(t, Ws[(a1p * 4 + a2p) * 4 + bp],
                 s[((((a1p * 4 + a1) * 4 + a2p) * 4 + a2) * 4 + bp) * 3 + c]);
      cfma(acc, Wc[(a1 * 4 + a2) * 4 + b], t);
    }
  Xs[idx] = acc;
}

__global__ void comb_ins_baryon(const double2 *__restrict__ I, int nq, int n_r,
                                const double2 *__restrict__ Gins, int ng, double2 *__restrict__ Xi) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t K = (size_t)12 * n_r;
  if (idx >= (size_t)ng * nq * K) return;
  int kk = (int)(idx % K);
  size_t rest = idx / K;
  int q = (int)(rest % nq), g = (int)(rest / nq);
  int i = kk / 12, b = (kk / 3) & 3, c = kk % 3;
  const double2 *v = I + ((size_t)q * n_r + i) * 192;
  const double2 *Gi = Gins + (size_t)g * 16;
  double2 acc = make_double2(0.0, 0.0);
  for (int at = 0; at < 4; ++at)
    for (int bt = 0; bt < 4; ++bt) cfma(acc, Gi[at * 4 + bt], v[at * 48 + bt * 12 + b * 3 + c]);
  Xi[idx] = acc;
}

// out[t][g][p][q] = (1/N) sum_i sum_{j<12} Xs[g][p][12i+j] Xi[t][g][q][12i+j]: a tiled complex
// GEMM.  FP64: all in double.  MIXED: the 12-term spin-colour sum of each noise in FP32,
// the sum over noises (the noise average of Eq. 5) in FP64.
constexpr int CT = 32;
template <bool MIXED>
__global__ void __launch_bounds__(256) comb_gemm(const double2 *__restrict__ Xs, const double2 *__restrict__ Xi,
                                                 int np, int nq, int n_r, int ng, double inv_n,
                                                 double2 *__restrict__ out) {
  using E = typename std::conditional<MIXED, float2, double2>::type;
  __shared__ E As[CT][13];
  __shared__ E Bs[CT][13];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int q0 = blockIdx.x * CT, p0 = blockIdx.y * CT;
  const int tg = blockIdx.z;                 // t * ng + g
  const int g = tg % ng;
  const size_t K = (size_t)12 * n_r;
  const double2 *A = Xs + ((size_t)g * np) * K;
  const double2 *B = Xi + ((size_t)tg * nq) * K;
  double2 acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = make_double2(0.0, 0.0);
  for (int i = 0; i < n_r; ++i) {
    for (int e = threadIdx.x; e < CT * 12; e += 256) {
      int r = e / 12, k = e % 12;
      double2 va = (p0 + r < np) ? A[(size_t)(p0 + r) * K + 12 * i + k] : make_double2(0.0, 0.0);
      double2 vb = (q0 + r < nq) ? B[(size_t)(q0 + r) * K + 12 * i + k] : make_double2(0.0, 0.0);
      if constexpr (MIXED) {
        As[r][k] = make_float2((float)va.x, (float)va.y);
        Bs[r][k] = make_float2((float)vb.x, (float)vb.y);
      } else {
        As[r][k] = va;
        Bs[r][k] = vb;
      }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        E pa;
        pa.x = 0;
        pa.y = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          E x = As[ty + 16 * a][k], y = Bs[tx + 16 * b][k];
          pa.x = fma(x.x, y.x, fma(-x.y, y.y, pa.x));
          pa.y = fma(x.x, y.y, fma(x.y, y.x, pa.y));
        }
        acc[a][b].x += (double)pa.x;
        acc[a][b].y += (double)pa.y;
      }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int p = p0 + ty + 16 * a, q = q0 + tx + 16 * b;
      if (p < np && q < nq)
        out[((size_t)tg * np + p) * nq + q] = make_double2(acc[a][b].x * inv_n, acc[a][b].y * inv_n);
    }
}

unsigned blocks(size_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int run_combine(lhc_ctx ctx, int kind, const double2 *spec, int np, const double2 *ins, int nq,
                int n_r, int nt, const double2 *snk, const double2 *ins_g, const double2 *src, int ng,
                int prec, double2 *out, cudaStream_t st) {
  size_t K = (size_t)12 * n_r;
  size_t ns = (size_t)ng * np * K, ni = (size_t)nt * ng * nq * K;
  LHC_TRY(ensure(ctx, ctx->ws, (ns + ni) * sizeof(double2)));
  double2 *Xs = static_cast<double2 *>(ctx->ws.p);
  double2 *Xi = Xs + ns;
  ProfScope ps(ctx, st, LHC_KERNEL_COMBINE, 8.0 * nt * ng * (double)np * nq * K);
  if (kind == LHC_MESON) {
    comb_spec_meson<<<blocks(ns, 256), 256, 0, st>>>(spec, np, n_r, snk, ng, Xs);
    // the insertion slices are consecutive [nq][n_r][192] blocks: treat them as nt*nq momenta
    // with the Gamma sets repeated per slice (index g of slice t is t*ng + g)
    for (int t = 0; t < nt; ++t)
      comb_ins_meson<<<blocks((size_t)ng * nq * K, 256), 256, 0, st>>>(ins + (size_t)t * nq * n_r * 192, nq, n_r,
                                                                       ins_g, src, ng, Xi + (size_t)t * ng * nq * K);
  } else {
    comb_spec_baryon<<<blocks(ns, 256), 256, 0, st>>>(spec, np, n_r, snk, src, ng, Xs);
    for (int t = 0; t < nt; ++t)
      comb_ins_baryon<<<blocks((size_t)ng * nq * K, 256), 256, 0, st>>>(ins + (size_t)t * nq * n_r * 192, nq, n_r,
                                                                        ins_g, ng, Xi + (size_t)t * ng * nq * K);
  }
  dim3 grid((nq + CT - 1) / CT, (np + CT - 1) / CT, nt * ng);
  if (prec == LHC_MIXED)
    comb_gemm<true><<<grid, 256, 0, st>>>(Xs, Xi, np, nq, n_r, ng, 1.0 / n_r, out);
  else
    comb_gemm<false><<<grid, 256, 0, st>>>(Xs, Xi, np, nq, n_r, ng, 1.0 / n_r, out);
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

}  // namespace lhc
