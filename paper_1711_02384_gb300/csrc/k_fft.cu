// All-momenta mode of the momentum projection (Eqs. 9, 10): when the momentum list is a
// large part of the L^3 momenta of a slice, the projection sum_x e^{+-i p.(x - r)} U(x)
// is a discrete Fourier transform of U over the slice, evaluated for every momentum at
// once and then gathered in the requested order:
//
//   F(k) = sum_x exp(s 2 pi i k.x / L) U(x)          (s = +1 insertion, -1 spectator)
//   out[q] = exp(-s 2 pi i k_q.r / L) F(k_q mod L),
//
// which is the phase of the direct sum, exp(s 2 pi i k.(x - r)/L), split in two.  F is
// computed as three passes of L-point transforms along x, y and z, each in place on the
// contracted values; a pass costs L complex multiply-adds per value, so the whole
// transform costs 3L per value against nq for the direct projection.  Any L works (the
// transforms are direct sums over a root table, not a radix factorization).
// Precision: LHC_FP64 contracts and transforms in FP64.  LHC_MIXED contracts in FP32 and
// transforms in FP32 with FP32 roots (each output a sum of L terms per pass, about 1e-7
// relative per correlator); the gather rounds the result to FP64.  GB300's FP64 pipe
// makes the FP32 transform the faster one by far.
#include <algorithm>
#include <cmath>
#include <vector>

#include "conv.cuh"
#include "lhc_internal.h"

namespace lhc {
namespace {

constexpr int kDftCols = 32;   // columns per block of a line transform

// One block per (line, group of kDftCols columns): the L values of the line for those
// columns are staged in shared memory, transformed, and written back in place.  Lines
// along direction d (0 = x, 1 = y, 2 = z); the site stride along the line is L^d.
template <typename T>   // double2 or float2
__global__ void __launch_bounds__(256) dft_line_kernel(T *__restrict__ U, int L, size_t ncols, int d, int sign,
                                                       const T *__restrict__ roots) {
  using R = decltype(T::x);
  extern __shared__ __align__(16) unsigned char sm_raw[];   // [L][kDftCols] values, then [L] roots
  T *line = reinterpret_cast<T *>(sm_raw), *w = line + (size_t)L * kDftCols;
  const size_t ngroups = (ncols + kDftCols - 1) / kDftCols;
  const size_t b = blockIdx.x;
  const size_t grp = b % ngroups, ln = b / ngroups;   // ln: index of the line among L^2
  const size_t stride = d == 0 ? 1 : (d == 1 ? (size_t)L : (size_t)L * L);
  // the line's first site: the two other coordinates from ln
  size_t base;
  {
    const size_t u = ln % L, v = ln / L;
    base = d == 0 ? (v * L + u) * L : (d == 1 ? v * L * L + u : v * L + u);
  }
  const size_t c0 = grp * kDftCols;
  const int nc = (int)min((size_t)kDftCols, ncols - c0);
  for (int e = threadIdx.x; e < L; e += blockDim.x) w[e] = roots[e];
  for (int e = threadIdx.x; e < L * kDftCols; e += blockDim.x) {
    const int x = e / kDftCols, c = e % kDftCols;
    line[e] = c < nc ? U[(base + x * stride) * ncols + c0 + c] : T{0, 0};
  }
  __syncthreads();
  T res[(128 * kDftCols + 255) / 256];   // L <= 128: at most 16 outputs per thread
  int nres = 0;
  for (int e = threadIdx.x; e < L * kDftCols; e += blockDim.x) {
    const int k = e / kDftCols, c = e % kDftCols;
    T acc{0, 0};
    for (int x = 0, m = 0; x < L; ++x, m = m + k >= L ? m + k - L : m + k) {   // m = (k x) mod L, 0 <= k < L
      const T a = line[x * kDftCols + c], z = w[m];
      const R zi = sign > 0 ? z.y : -z.y;
      acc.x = fma(a.x, z.x, fma(-a.y, zi, acc.x));
      acc.y = fma(a.x, zi, fma(a.y, z.x, acc.y));
    }
    res[nres++] = acc;
  }
  __syncthreads();   // every thread has read the line before anyone writes it back
  nres = 0;
  for (int e = threadIdx.x; e < L * kDftCols; e += blockDim.x) {
    const int k = e / kDftCols, c = e % kDftCols;
    if (c < nc) U[(base + k * stride) * ncols + c0 + c] = res[nres];
    ++nres;
  }
}

__device__ __forceinline__ double2 to_f64(double2 v) { return v; }
__device__ __forceinline__ double2 to_f64(float2 v) { return make_double2(f32_to_f64(v.x), f32_to_f64(v.y)); }

// out[q][i0 + i][col] = exp(-s 2 pi i k_q.r / L) F[site(k_q mod L)][i][col], formed in the
// transform's precision and widened to complex128
template <typename T>
__global__ void dft_gather_kernel(const T *__restrict__ F, const int *__restrict__ kq, int nq, int L, int rx,
                                  int ry, int rz, int sign, const T *__restrict__ roots, size_t ncols_chunk,
                                  size_t out_row, size_t col0, double2 *__restrict__ out) {
  using R = decltype(T::x);
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nq * ncols_chunk) return;
  const int q = (int)(idx / ncols_chunk);
  const size_t c = idx % ncols_chunk;
  const int kx = kq[3 * q], ky = kq[3 * q + 1], kz = kq[3 * q + 2];
  const int mx = ((kx % L) + L) % L, my = ((ky % L) + L) % L, mz = ((kz % L) + L) % L;
  long long m = ((long long)kx * rx + (long long)ky * ry + (long long)kz * rz) % L;
  if (m < 0) m += L;
  const T z = roots[m];
  const R zi = sign > 0 ? -z.y : z.y;   // exp(-s 2 pi i k.r / L)
  const T f = F[((size_t)(mz * L + my) * L + mx) * ncols_chunk + c];
  out[(size_t)q * out_row + col0 + c] = to_f64(T{f.x * z.x - f.y * zi, f.x * zi + f.y * z.x});
}

}  // namespace

// Automatic choice: the transform replaces the direct projection once a call asks for at
// least half of the slice's momenta.  In FP64 the direct projection is the slowest part
// there (GB300's FP64 rate); in the mixed path the FP32 transform's 3L multiply-adds per
// value cost less than the tensor-core projection with its split and drain at that size.
bool use_fft(lhc_ctx ctx, int prec, int V3, int nq) {
  (void)prec;   // both precisions switch at half of the slice's momenta
  if (ctx->proj_mode == LHC_PROJ_DFT) return true;
  if (ctx->proj_mode == LHC_PROJ_GEMM) return false;
  return 2 * (long long)nq >= V3;
}

// Upper bound of the device memory one all-momenta call allocates: the workspace of a
// noise chunk (the values of a whole slice for as many noises as fit 2 GiB, at least one)
// and the cached momentum list with its roots.
size_t fft_call_bytes(Part part, int prec, int L, int n_r, int nq) {
  const size_t V3 = (size_t)L * L * L, cols = part == PART_SPEC_BARYON ? kBarCols : 192;
  const size_t per_noise = V3 * cols * (prec == LHC_MIXED ? sizeof(float2) : sizeof(double2));
  const size_t nch = std::max<size_t>(1, std::min<size_t>(n_r, ((size_t)2 << 30) / per_noise));
  return nch * per_noise + 12 * (size_t)nq + (size_t)L * sizeof(double2) + 2 * 256;
}

namespace {

// The device copies of a call's momentum list and of the L-th roots of unity (rounded
// once from FP64 to T), cached with the phase tables per (L, momentum list, precision).
// Built with synchronous copies on first use; later calls with the same list copy
// nothing from the host, so they stay asynchronous and can be captured in a graph.
template <typename T>
int get_dft_table(lhc_ctx ctx, int L, const int *k, int nq, const int **kd, const T **roots) {
  const PhaseKey key{L, nq, 0, sizeof(T) == sizeof(double2) ? 4 : 3, 0, 0, 0, hash_k(k, nq)};
  const size_t off_roots = (12 * (size_t)nq + 255) & ~(size_t)255;
  const PhaseEntry *hit = phase_take(ctx, key);
  if (!hit) {
    PhaseEntry e;
    LHC_TRY(dev_alloc(ctx, e.buf, off_roots + (size_t)L * sizeof(T)));
    std::vector<T> hroots(L);
    const double two_pi = 6.283185307179586476925286766559;
    for (int m = 0; m < L; ++m)
      hroots[m] = T{static_cast<decltype(T::x)>(std::cos(two_pi * m / L)),
                    static_cast<decltype(T::x)>(std::sin(two_pi * m / L))};
    char *base = static_cast<char *>(e.buf.p);
    cudaError_t c = cudaMemcpy(base, k, 12 * (size_t)nq, cudaMemcpyHostToDevice);
    if (c == cudaSuccess) c = cudaMemcpy(base + off_roots, hroots.data(), (size_t)L * sizeof(T), cudaMemcpyHostToDevice);
    if (c != cudaSuccess) {
      dev_free(ctx, e.buf);
      set_error("DFT table upload: %s", cudaGetErrorString(c));
      return LHC_ECUDA;
    }
    phase_insert(ctx, key, e);
    hit = phase_take(ctx, key);
  }
  *kd = static_cast<const int *>(hit->buf.p);
  *roots = reinterpret_cast<const T *>(static_cast<const char *>(hit->buf.p) + off_roots);
  return LHC_OK;
}

template <typename T>
int run_fft_t(lhc_ctx ctx, const SliceJob *jobs, int nt, const int *k, int nq, const int r[4], int sign,
              cudaStream_t st) {
  const SliceJob &j0 = jobs[0];
  const int L = j0.L, V3 = j0.V3;
  const int cols = j0.part == PART_SPEC_BARYON ? kBarCols : 192;
  // noises per chunk: the values of a whole slice for that many noises within 2 GiB
  const size_t per_noise = (size_t)V3 * cols * sizeof(T);
  const int nch = (int)std::max<size_t>(1, std::min<size_t>(j0.n_r, ((size_t)2 << 30) / per_noise));
  const int *kd = nullptr;
  const T *roots = nullptr;
  LHC_TRY(get_dft_table(ctx, L, k, nq, &kd, &roots));   // before the workspace: it may allocate
  LHC_TRY(ensure(ctx, ctx->ws, (size_t)nch * per_noise));
  T *U = static_cast<T *>(ctx->ws.p);
  const int rx = ((r[0] % L) + L) % L, ry = ((r[1] % L) + L) % L, rz = ((r[2] % L) + L) % L;
  const size_t smem = ((size_t)L * kDftCols + L) * sizeof(T);
  if (smem > 48 * 1024)
    LHC_CHECK_CUDA(cudaFuncSetAttribute(dft_line_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int jt = 0; jt < nt; ++jt) {
    const SliceJob &j = jobs[jt];
    for (int i0 = 0; i0 < j.n_r; i0 += nch) {
      SliceJob jc = j;
      jc.n_r = std::min(nch, j.n_r - i0);
      const size_t esz = j.dtype == LHC_C128 ? 16 : 8;
      jc.vec = static_cast<const char *>(j.vec) + (size_t)i0 * j.vec_stride * esz;
      const size_t ncc = (size_t)jc.n_r * cols;
      {
        const int nS = j.part == PART_SPEC_BARYON ? 2 : 1;
        ProfScope ps(ctx, st, LHC_KERNEL_CONTRACT,
                     (double)V3 * (144.0 * nS + 12.0 * jc.n_r) * esz + (double)V3 * ncc * sizeof(T));
        if constexpr (sizeof(T) == sizeof(double2))
          LHC_TRY(contract_f64(jc, 0, V3, U, st));
        else
          LHC_TRY(contract_f32(jc, 0, V3, U, st));
      }
      {
        ProfScope ps(ctx, st, LHC_KERNEL_PROJECT, 3.0 * 8.0 * L * (double)V3 * ncc);
        const size_t blocks = (size_t)L * L * ((ncc + kDftCols - 1) / kDftCols);
        for (int d = 0; d < 3; ++d) {
          dft_line_kernel<T><<<(unsigned)blocks, 256, smem, st>>>(U, L, ncc, d, sign, roots);
          note_launch();
        }
      }
      const size_t n = (size_t)nq * ncc;
      dft_gather_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U, kd, nq, L, rx, ry, rz, sign, roots, ncc,
                                                                        (size_t)j.n_r * cols, (size_t)i0 * cols, j.out);
      note_launch();
    }
  }
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}

}  // namespace

int run_part_fft(lhc_ctx ctx, const SliceJob *jobs, int nt, const int *k, int nq, const int r[4], int sign,
                 int prec, cudaStream_t st) {
  return prec == LHC_MIXED ? run_fft_t<float2>(ctx, jobs, nt, k, nq, r, sign, st)
                           : run_fft_t<double2>(ctx, jobs, nt, k, nq, r, sign, st);
}

}  // namespace lhc
