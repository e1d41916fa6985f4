// Noise-averaged combine (Eqs. 5 and 8) in FP64.
//
// Both cases reduce to  out[g][p][q] = (1/N) sum_K Xs[g][p][K] Xi[g][q][K]  with
// K = (noise i, spin j, colour c) (12 N values):
//   meson   Xs[g][p][i,al,a] = sum_{ap,bp} Gsnk[ap][bp] S[p][i][bp,ap,al,a]
//           Xi[g][q][i,al,a] = sum_b Gsrc[b][al] sum_{at,bt} Gins[at][bt] I[q][i][at,bt,b,a]
//   baryon  Xs[g][p][i,b,c]  = sum Wsnk[a1p][a2p][bp] Wsrc[a1][a2][b] B[p][i][a1p,a1,a2p,a2,bp,c]
//           Xi[g][q][i,b,c]  = sum_{at,bt} Gins[at][bt] I[q][i][at,bt,b,c]
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

// out[g][p][q] = (1/N) sum_K Xs[g][p][K] Xi[g][q][K]; one warp per output, fixed order
__global__ void comb_dot(const double2 *__restrict__ Xs, const double2 *__restrict__ Xi, int np,
                         int nq, int K, int ng, double inv_n, double2 *__restrict__ out) {
  size_t w = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= (size_t)ng * np * nq) return;
  int q = (int)(w % nq);
  size_t rest = w / nq;
  int p = (int)(rest % np), g = (int)(rest / np);
  const double2 *a = Xs + ((size_t)g * np + p) * K;
  const double2 *b = Xi + ((size_t)g * nq + q) * K;
  double2 acc = make_double2(0.0, 0.0);
  for (int k = lane; k < K; k += 32) cfma(acc, a[k], b[k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) out[w] = make_double2(acc.x * inv_n, acc.y * inv_n);
}

unsigned blocks(size_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int run_combine(lhc_ctx ctx, int kind, const double2 *spec, int np, const double2 *ins, int nq,
                int n_r, const double2 *snk, const double2 *ins_g, const double2 *src, int ng,
                double2 *out, cudaStream_t st) {
  size_t K = (size_t)12 * n_r;
  size_t ns = (size_t)ng * np * K, ni = (size_t)ng * nq * K;
  LHC_TRY(ensure(ctx, ctx->ws, (ns + ni) * sizeof(double2)));
  double2 *Xs = static_cast<double2 *>(ctx->ws.p);
  double2 *Xi = Xs + ns;
  if (kind == LHC_MESON) {
    comb_spec_meson<<<blocks(ns, 256), 256, 0, st>>>(spec, np, n_r, snk, ng, Xs);
    comb_ins_meson<<<blocks(ni, 256), 256, 0, st>>>(ins, nq, n_r, ins_g, src, ng, Xi);
  } else {
    comb_spec_baryon<<<blocks(ns, 256), 256, 0, st>>>(spec, np, n_r, snk, src, ng, Xs);
    comb_ins_baryon<<<blocks(ni, 256), 256, 0, st>>>(ins, nq, n_r, ins_g, ng, Xi);
  }
  size_t nout = (size_t)ng * np * nq;
  comb_dot<<<blocks(nout * 32, 256), 256, 0, st>>>(Xs, Xi, np, nq, (int)K, ng, 1.0 / n_r, out);
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

}  // namespace lhc
