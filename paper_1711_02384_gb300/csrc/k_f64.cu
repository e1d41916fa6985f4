// Plain FP64 GPU path: site contractions (Eqs. 9, 10 and the baryon eps-eps
// reading) in FP64, written to a workspace in site chunks, then the momentum
// projection sum_x P[q][x] U[x][col] as an FP64 complex GEMM on CUDA cores.
// This is the comparator path and the 1e-12 parity reference on the GPU.
#include "conv.cuh"
#include "lhc_internal.h"

namespace lhc {
namespace {

__device__ __forceinline__ double2 ld2(const double2 *p) { return *p; }
__device__ __forceinline__ double2 ld2(const float2 *p) {
  float2 v = *p;
  return make_double2(v.x, v.y);
}
// acc += a * b
__device__ __forceinline__ void cfma(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
// acc += a * conj(b)
__device__ __forceinline__ void cfma_cb(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.y, b.x, fma(-a.x, b.y, acc.y));
}
// The same in FP32, for the contractions of the mixed path's all-momenta mode: inputs
// are rounded to FP32 (complex128 by the integer IEEE conversion, off the FP64 pipe)
// and the three-colour sums run in FP32.
__device__ __forceinline__ float2 ldf(const float2 *p) { return *p; }
__device__ __forceinline__ float2 ldf(const double2 *p) {
  const double2 v = *p;
  return make_float2(f64_to_f32_rne(v.x), f64_to_f32_rne(v.y));
}
__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
__device__ __forceinline__ void cfmac(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}
__device__ __forceinline__ void cfma_cb(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.y, b.x, fmaf(-a.x, b.y, acc.y));
}
// load with conversion to the accumulation type OT (double2 or float2)
template <typename OT, typename CT>
__device__ __forceinline__ OT ldo(const CT *p) {
  if constexpr (sizeof(OT) == sizeof(double2))
    return ld2(p);
  else
    return ldf(p);
}

// Insertion (Eq. 10) before the momentum sum:
// U[x][i][(at,bt,b,a)] = g5(at) sum_{a~} conj(psi_i(x)[at,a~]) S3(x)[(bt,a~),(b,a)]
template <typename CT, typename OT>
__global__ void ins_contract(const CT *__restrict__ S, const CT *__restrict__ psi,
                             size_t psi_stride, int n_r, int s0, int ns, int g5mask,
                             OT *__restrict__ U) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)ns * n_r * 192;
  if (idx >= total) return;
  int col = (int)(idx % 192);
  size_t rest = idx / 192;
  int i = (int)(rest % n_r);
  int x = s0 + (int)(rest / n_r);
  int at = col / 48, bt = (col / 12) & 3, b = (col / 3) & 3, a = col % 3;
  const CT *s = S + (size_t)x * 144;
  const CT *p = psi + (size_t)i * psi_stride + (size_t)x * 12;
  OT acc{0, 0};
#pragma unroll
  for (int ac = 0; ac < 3; ++ac) cfmac(acc, ldo<OT>(p + at * 3 + ac), ldo<OT>(s + (bt * 3 + ac) * 12 + b * 3 + a));
  if ((g5mask >> at) & 1) acc = OT{-acc.x, -acc.y};
  U[idx] = acc;
}

// Meson spectator (Eq. 9) before the momentum sum, G1(r,x') = g5 S1(x')^dagger g5:
// V[x][i][(bp,ap,al,a)] = g5(bp) g5(ap) g5(al) sum_{a'} eta_i(x)[bp,a'] conj(S1(x)[(ap,a'),(al,a)])
template <typename CT, typename OT>
__global__ void spec_meson_contract(const CT *__restrict__ S, const CT *__restrict__ eta,
                                    size_t eta_stride, int n_r, int s0, int ns, int g5mask,
                                    OT *__restrict__ U) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)ns * n_r * 192;
  if (idx >= total) return;
  int col = (int)(idx % 192);
  size_t rest = idx / 192;
  int i = (int)(rest % n_r);
  int x = s0 + (int)(rest / n_r);
  int bp = col / 48, ap = (col / 12) & 3, al = (col / 3) & 3, a = col % 3;
  const CT *s = S + (size_t)x * 144;
  const CT *e = eta + (size_t)i * eta_stride + (size_t)x * 12;
  OT acc{0, 0};
#pragma unroll
  for (int ac = 0; ac < 3; ++ac) cfma_cb(acc, ldo<OT>(e + bp * 3 + ac), ldo<OT>(s + (ap * 3 + ac) * 12 + al * 3 + a));
  if (((g5mask >> bp) ^ (g5mask >> ap) ^ (g5mask >> al)) & 1) acc = OT{-acc.x, -acc.y};
  U[idx] = acc;
}

// Baryon spectator before the momentum sum:
// B[x][i][(a1p,a1,a2p,a2,bp,c)] = g5(bp) sum_{c'} eta_i(x)[bp,c'] D[a1p,a1,a2p,a2,c',c],
// D = sum eps_{a'b'c'} eps_{abc} GA[(a1p,a'),(a1,a)] GB[(a2p,b'),(a2,b)]; with
// p=c'+1, q=c'+2, u=c+1, v=c+2 (mod 3) the four nonzero terms are
// GA[p,u]GB[q,v] - GA[p,v]GB[q,u] - GA[q,u]GB[p,v] + GA[q,v]GB[p,u].
template <typename CT, typename OT>
__global__ void spec_baryon_contract(const CT *__restrict__ GA, const CT *__restrict__ GB,
                                     const CT *__restrict__ eta, size_t eta_stride, int n_r,
                                     int s0, int ns, int g5mask, OT *__restrict__ U) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)ns * n_r * 3072;
  if (idx >= total) return;
  int col = (int)(idx % 3072);
  size_t rest = idx / 3072;
  int i = (int)(rest % n_r);
  int x = s0 + (int)(rest / n_r);
  int c = col % 3, bp = (col / 3) & 3, a2 = (col / 12) & 3, a2p = (col / 48) & 3,
      a1 = (col / 192) & 3, a1p = col / 768;
  const CT *A = GA + (size_t)x * 144;
  const CT *B = GB + (size_t)x * 144;
  const CT *e = eta + (size_t)i * eta_stride + (size_t)x * 12;
  int u = (c + 1) % 3, v = (c + 2) % 3;
  OT acc{0, 0};
#pragma unroll
  for (int cp = 0; cp < 3; ++cp) {
    int p = (cp + 1) % 3, q = (cp + 2) % 3;
    auto ga = [&](int r, int s) { return ldo<OT>(A + (a1p * 3 + r) * 12 + a1 * 3 + s); };
    auto gb = [&](int r, int s) { return ldo<OT>(B + (a2p * 3 + r) * 12 + a2 * 3 + s); };
    OT d{0, 0}, t{0, 0};
    cfma(d, ga(p, u), gb(q, v));
    cfma(t, ga(p, v), gb(q, u));
    cfma(t, ga(q, u), gb(p, v));
    d.x -= t.x;
    d.y -= t.y;
    cfma(d, ga(q, v), gb(p, u));
    cfma(acc, ldo<OT>(e + bp * 3 + cp), d);
  }
  if ((g5mask >> bp) & 1) acc = OT{-acc.x, -acc.y};
  U[idx] = acc;
}

// out[q][col] (+)= sum_{x < ns} P[q][s0 + x] U[x][col]   (complex FP64 GEMM)
constexpr int PBM = 32, PBN = 64, PBK = 16;
__global__ void __launch_bounds__(256) project_f64(const double2 *__restrict__ P, int V3, int s0,
                                                   int ns, int nq, const double2 *__restrict__ U,
                                                   int ncols, double2 *__restrict__ out,
                                                   int accumulate) {
  __shared__ double2 Ps[PBK][PBM + 1];
  __shared__ double2 Us[PBK][PBN];
  int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  int q0 = blockIdx.y * PBM, c0 = blockIdx.x * PBN;
  double2 acc[4][2];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int l = 0; l < 2; ++l) acc[j][l] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < ns; k0 += PBK) {
#pragma unroll
    for (int e = tid; e < PBK * PBM; e += 256) {
      int kk = e % PBK, qq = e / PBK;
      int q = q0 + qq, x = k0 + kk;
      Ps[kk][qq] = (q < nq && x < ns) ? P[(size_t)q * V3 + s0 + x] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int e = tid; e < PBK * PBN; e += 256) {
      int cc = e % PBN, kk = e / PBN;
      int c = c0 + cc, x = k0 + kk;
      Us[kk][cc] = (c < ncols && x < ns) ? U[(size_t)x * ncols + c] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < PBK; ++kk) {
      double2 u0 = Us[kk][tx], u1 = Us[kk][tx + 32];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        double2 p = Ps[kk][ty + 8 * j];
        cfma(acc[j][0], p, u0);
        cfma(acc[j][1], p, u1);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int q = q0 + ty + 8 * j;
    if (q >= nq) continue;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      int c = c0 + tx + 32 * l;
      if (c >= ncols) continue;
      double2 *o = out + (size_t)q * ncols + c;
      double2 v = acc[j][l];
      if (accumulate) {
        double2 w = *o;
        v.x += w.x;
        v.y += w.y;
      }
      *o = v;
    }
  }
}

__global__ void phase_f64_kernel(double2 *P, const int *k, int nq, int L, int rx, int ry, int rz,
                                 int sign, const double2 *roots) {
  int V3 = L * L * L;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nq * V3) return;
  int q = (int)(idx / V3), s = (int)(idx % V3);
  int x = s % L, y = (s / L) % L, z = s / (L * L);
  long long m = (long long)k[3 * q] * (x - rx) + (long long)k[3 * q + 1] * (y - ry) +
                (long long)k[3 * q + 2] * (z - rz);
  m %= L;
  if (m < 0) m += L;
  double2 w = roots[m];
  P[idx] = make_double2(w.x, sign * w.y);
}

template <typename CT, typename OT>
void launch_contract(const SliceJob &j, int s0, int ns, OT *U, cudaStream_t st) {
  const CT *S = static_cast<const CT *>(j.S);
  const CT *v = static_cast<const CT *>(j.vec);
  int cols = j.part == PART_SPEC_BARYON ? kBarCols : 192;
  size_t total = (size_t)ns * j.n_r * cols;
  unsigned grid = (unsigned)((total + 255) / 256);
  if (j.part == PART_INS)
    ins_contract<CT, OT><<<grid, 256, 0, st>>>(S, v, j.vec_stride, j.n_r, s0, ns, j.g5mask, U);
  else if (j.part == PART_SPEC_MESON)
    spec_meson_contract<CT, OT><<<grid, 256, 0, st>>>(S, v, j.vec_stride, j.n_r, s0, ns, j.g5mask, U);
  else
    spec_baryon_contract<CT, OT><<<grid, 256, 0, st>>>(S, static_cast<const CT *>(j.SB), v, j.vec_stride, j.n_r,
                                                       s0, ns, j.g5mask, U);
  note_launch();
}

}  // namespace

int contract_f64(const SliceJob &j, int s0, int ns, double2 *U, cudaStream_t st) {
  if (j.dtype == LHC_C128)
    launch_contract<double2, double2>(j, s0, ns, U, st);
  else
    launch_contract<float2, double2>(j, s0, ns, U, st);
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

int contract_f32(const SliceJob &j, int s0, int ns, float2 *U, cudaStream_t st) {
  if (j.dtype == LHC_C128)
    launch_contract<double2, float2>(j, s0, ns, U, st);
  else
    launch_contract<float2, float2>(j, s0, ns, U, st);
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

void launch_phase_f64(double2 *P, const int *k_dev, int nq, int L, int rx, int ry, int rz, int sign,
                      const double2 *roots_dev, cudaStream_t st) {
  size_t total = (size_t)nq * L * L * L;
  phase_f64_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, k_dev, nq, L, rx, ry, rz,
                                                                    sign, roots_dev);
  note_launch();
}

int run_slice_f64(lhc_ctx ctx, const SliceJob &j, const double2 *phase, cudaStream_t st) {
  int cols = (j.part == PART_SPEC_BARYON ? kBarCols : 192) * j.n_r;
  // site chunk so that the FP64 intermediate stays within 1 GiB of workspace
  size_t per_site = (size_t)cols * sizeof(double2);
  size_t cap = (size_t)1 << 30;
  int chunk = (int)std::min<size_t>((size_t)j.V3, std::max<size_t>(16, cap / per_site));
  LHC_TRY(ensure(ctx, ctx->ws, (size_t)chunk * per_site));
  double2 *U = static_cast<double2 *>(ctx->ws.p);
  for (int s0 = 0; s0 < j.V3; s0 += chunk) {
    int ns = std::min(chunk, j.V3 - s0);
    {
      size_t es = j.dtype == LHC_C128 ? 16 : 8;
      int nS = j.part == PART_SPEC_BARYON ? 2 : 1;
      double bytes = (double)ns * (144.0 * nS + 12.0 * j.n_r) * es + (double)ns * cols * 16.0;
      ProfScope ps(ctx, st, LHC_KERNEL_CONTRACT, bytes);
      if (j.dtype == LHC_C128)
        launch_contract<double2, double2>(j, s0, ns, U, st);
      else
        launch_contract<float2, double2>(j, s0, ns, U, st);
    }
    {
      ProfScope ps(ctx, st, LHC_KERNEL_PROJECT, 8.0 * j.nq * (double)cols * ns);
      dim3 grid((cols + PBN - 1) / PBN, (j.nq + PBM - 1) / PBM);
      project_f64<<<grid, 256, 0, st>>>(phase, j.V3, s0, ns, j.nq, U, cols, j.out, s0 > 0);
      note_launch();
    }
  }
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

}  // namespace lhc
