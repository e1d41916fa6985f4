// Free-field Wilson-Dirac operator and solver: real solutions s_i = D^{-1} eta_i and
// point-to-all propagators from unit links, so the whole path can be checked on the GPU
// against the closed-form free correlator.  The paper solves on gauge configurations
// with a multigrid solver (Sec. 3); with unit links the operator is (Wilson parameter 1)
//
//   (D psi)(x) = (m + 4) psi(x) - 1/2 sum_mu [ (1 - gamma_mu) psi(x + mu) + (1 + gamma_mu) psi(x - mu) ],
//
// colour-diagonal, periodic in all four directions, mu = x, y, z, t.  gamma_mu are
// Hermitian, so D^dagger is the same stencil with gamma_mu -> -gamma_mu.  The solver is
// conjugate gradients on the normal equations D^dagger D x = D^dagger b, in FP64, one
// independent recursion per right-hand side.  It produces test inputs, not hot-path work.
#include <cmath>
#include <vector>

#include "lhc_internal.h"

namespace lhc {
namespace {

struct Gammas {
  double2 g[4][16];   // gamma_mu[s][s'] row-major, mu = x, y, z, t
  // The same matrices when every row has a single entry, a unit phase (any chiral or
  // Dirac-Pauli basis): row s of gamma_mu is i^ph[mu][s] in column col[mu][s].
  bool sparse;
  int col[4][4], ph[4][4];
};

// One thread per (rhs, t, site, colour): the four spins of one colour at one site.
__global__ void wilson_kernel(const double2 *__restrict__ in, double2 *__restrict__ out, int L, int T, int nrhs,
                              double m, double sigma, Gammas gm) {
  const size_t V3 = (size_t)L * L * L, n = (size_t)nrhs * T * V3 * 3;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int c = (int)(idx % 3);
  size_t rest = idx / 3;
  const size_t site = rest % V3;
  rest /= V3;
  const int t = (int)(rest % T);
  const size_t rhs = rest / T;
  const int x = (int)(site % L), y = (int)((site / L) % L), z = (int)(site / ((size_t)L * L));
  const double2 *f = in + rhs * T * V3 * 12;
  auto at = [&](int tt, int xx, int yy, int zz) {
    return f + ((size_t)tt * V3 + ((size_t)zz * L + yy) * L + xx) * 12 + c;
  };
  double2 acc[4];
  const double2 *h = at(t, x, y, z);
#pragma unroll
  for (int s = 0; s < 4; ++s) acc[s] = make_double2((m + 4.0) * h[3 * s].x, (m + 4.0) * h[3 * s].y);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int d[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
    const double2 *fw = at((t + d[mu][3]) % T, (x + d[mu][0]) % L, (y + d[mu][1]) % L, (z + d[mu][2]) % L);
    const double2 *bw =
        at((t - d[mu][3] + T) % T, (x - d[mu][0] + L) % L, (y - d[mu][1] + L) % L, (z - d[mu][2] + L) % L);
    double2 pf[4], pb[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      pf[s] = fw[3 * s];
      pb[s] = bw[3 * s];
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      // -1/2 [ (psi_f + psi_b) - sigma gamma (psi_f - psi_b) ]
      double2 v = make_double2(pf[s].x + pb[s].x, pf[s].y + pb[s].y);
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2) {
        const double2 gg = gm.g[mu][s * 4 + s2];
        const double2 dd = make_double2(pf[s2].x - pb[s2].x, pf[s2].y - pb[s2].y);
        v.x -= sigma * (gg.x * dd.x - gg.y * dd.y);
        v.y -= sigma * (gg.x * dd.y + gg.y * dd.x);
      }
      acc[s].x -= 0.5 * v.x;
      acc[s].y -= 0.5 * v.y;
    }
  }
  double2 *o = out + rhs * T * V3 * 12 + ((size_t)t * V3 + site) * 12 + c;
#pragma unroll
  for (int s = 0; s < 4; ++s) o[3 * s] = acc[s];
}

// i^ph * (x + i y) for ph in 0..3: exact (sign changes and a swap)
__device__ __forceinline__ double2 unit_phase(int ph, double2 v) {
  switch (ph & 3) {
    case 0: return v;
    case 1: return make_double2(-v.y, v.x);
    case 2: return make_double2(-v.x, -v.y);
    default: return make_double2(v.y, -v.x);
  }
}

// The same stencil for gamma matrices with one unit-phase entry per row: each spin row
// takes one difference, multiplied by a phase without FP64 multiplications.  GB300's
// FP64 pipe runs at a small fraction of the FP32 rate, and the dense 4x4 complex products
// above cost about 7 times the FP64 instructions.
__global__ void wilson_sparse_kernel(const double2 *__restrict__ in, double2 *__restrict__ out, int L, int T,
                                     int nrhs, double m, double sigma, Gammas gm) {
  const size_t V3 = (size_t)L * L * L, n = (size_t)nrhs * T * V3 * 3;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int c = (int)(idx % 3);
  size_t rest = idx / 3;
  const size_t site = rest % V3;
  rest /= V3;
  const int t = (int)(rest % T);
  const size_t rhs = rest / T;
  const int x = (int)(site % L), y = (int)((site / L) % L), z = (int)(site / ((size_t)L * L));
  const double2 *f = in + rhs * T * V3 * 12;
  auto at = [&](int tt, int xx, int yy, int zz) {
    return f + ((size_t)tt * V3 + ((size_t)zz * L + yy) * L + xx) * 12 + c;
  };
  double2 acc[4];
  const double2 *h = at(t, x, y, z);
#pragma unroll
  for (int s = 0; s < 4; ++s) acc[s] = make_double2((m + 4.0) * h[3 * s].x, (m + 4.0) * h[3 * s].y);
  // sigma = +1 (D) or -1 (D^dagger) flips every phase by i^2
  const int flip = sigma < 0.0 ? 2 : 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int d[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
    const double2 *fw = at((t + d[mu][3]) % T, (x + d[mu][0]) % L, (y + d[mu][1]) % L, (z + d[mu][2]) % L);
    const double2 *bw =
        at((t - d[mu][3] + T) % T, (x - d[mu][0] + L) % L, (y - d[mu][1] + L) % L, (z - d[mu][2] + L) % L);
    double2 pf[4], pb[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      pf[s] = fw[3 * s];
      pb[s] = bw[3 * s];
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      // -1/2 [ (psi_f + psi_b)_s - sigma i^ph (psi_f - psi_b)_col ]
      const int cs = gm.col[mu][s];
      double2 dd = make_double2(0.0, 0.0);
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2)   // register select, no dynamic indexing
        if (s2 == cs) dd = make_double2(pf[s2].x - pb[s2].x, pf[s2].y - pb[s2].y);
      const double2 g = unit_phase(gm.ph[mu][s] + flip, dd);
      acc[s].x -= 0.5 * ((pf[s].x + pb[s].x) - g.x);
      acc[s].y -= 0.5 * ((pf[s].y + pb[s].y) - g.y);
    }
  }
  double2 *o = out + rhs * T * V3 * 12 + ((size_t)t * V3 + site) * 12 + c;
#pragma unroll
  for (int s = 0; s < 4; ++s) o[3 * s] = acc[s];
}

// partial[rhs][block] = sum over this block's share of Re(conj(a) b) for one rhs
__global__ void dot_kernel(const double2 *__restrict__ a, const double2 *__restrict__ b, size_t n, double *partial) {
  const size_t rhs = blockIdx.y;
  const double2 *pa = a + rhs * n, *pb = b + rhs * n;
  double s = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    s += pa[e].x * pb[e].x + pa[e].y * pb[e].y;
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[rhs * gridDim.x + blockIdx.x] = red[0];
}

// y[rhs] = a[rhs] * x[rhs] + b[rhs] * y[rhs] (scalars per right-hand side)
__global__ void axpby_kernel(const double *__restrict__ a, const double2 *__restrict__ x, const double *__restrict__ b,
                             double2 *__restrict__ y, size_t n, int nrhs) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  const size_t rhs = idx / n;
  const double2 xv = x[idx], yv = y[idx];
  y[idx] = make_double2(a[rhs] * xv.x + b[rhs] * yv.x, a[rhs] * xv.y + b[rhs] * yv.y);
}

// The same with the scalars in the kernel's parameters (up to kParamRhs right-hand
// sides): no copy, and no wait for one before the host reuses its scalars.
constexpr int kParamRhs = 64;
struct AxpbyCoef {
  double a[kParamRhs], b[kParamRhs];
};
__global__ void axpby_param_kernel(const __grid_constant__ AxpbyCoef cf, const double2 *__restrict__ x,
                                   double2 *__restrict__ y, size_t n, int nrhs) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  const size_t rhs = idx / n;
  const double2 xv = x[idx], yv = y[idx];
  y[idx] = make_double2(cf.a[rhs] * xv.x + cf.b[rhs] * yv.x, cf.a[rhs] * xv.y + cf.b[rhs] * yv.y);
}

constexpr int kDotBlocks = 64;

struct Solver {
  lhc_ctx ctx;
  cudaStream_t st;
  int L, T, nrhs;
  size_t n;   // complex numbers per right-hand side
  double m;
  Gammas gm;
  double *partial = nullptr, *coef = nullptr;   // device: [nrhs][kDotBlocks], [4][nrhs]
  std::vector<double> hpart;

  int apply(const double2 *in, double2 *out, double sigma) {
    const size_t threads = (size_t)nrhs * T * L * L * L * 3;
    if (gm.sparse)
      wilson_sparse_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(in, out, L, T, nrhs, m, sigma, gm);
    else
      wilson_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(in, out, L, T, nrhs, m, sigma, gm);
    note_launch();
    LHC_CHECK_CUDA(cudaGetLastError());
    return LHC_OK;
  }
  int dot(const double2 *a, const double2 *b, std::vector<double> &res) {
    dot_kernel<<<dim3(kDotBlocks, nrhs), 256, 0, st>>>(a, b, n, partial);
    note_launch();
    LHC_CHECK_CUDA(cudaMemcpyAsync(hpart.data(), partial, sizeof(double) * hpart.size(), cudaMemcpyDeviceToHost, st));
    LHC_CHECK_CUDA(cudaStreamSynchronize(st));
    res.assign(nrhs, 0.0);
    for (int r = 0; r < nrhs; ++r)
      for (int b = 0; b < kDotBlocks; ++b) res[r] += hpart[(size_t)r * kDotBlocks + b];
    return LHC_OK;
  }
  // y = a x + b y with per-rhs host scalars
  int axpby(const std::vector<double> &a, const double2 *x, const std::vector<double> &b, double2 *y) {
    if (nrhs <= kParamRhs) {
      AxpbyCoef cf{};
      for (int r = 0; r < nrhs; ++r) cf.a[r] = a[r], cf.b[r] = b[r];
      axpby_param_kernel<<<(unsigned)((n * nrhs + 255) / 256), 256, 0, st>>>(cf, x, y, n, nrhs);
      note_launch();
      LHC_CHECK_CUDA(cudaGetLastError());
      return LHC_OK;
    }
    std::vector<double> ab(2 * (size_t)nrhs);
    for (int r = 0; r < nrhs; ++r) ab[r] = a[r], ab[nrhs + r] = b[r];
    LHC_CHECK_CUDA(cudaMemcpyAsync(coef, ab.data(), sizeof(double) * ab.size(), cudaMemcpyHostToDevice, st));
    axpby_kernel<<<(unsigned)((n * nrhs + 255) / 256), 256, 0, st>>>(coef, x, coef + nrhs, y, n, nrhs);
    note_launch();
    LHC_CHECK_CUDA(cudaGetLastError());
    // the scalars are read by the kernel: keep them alive until it has run
    LHC_CHECK_CUDA(cudaStreamSynchronize(st));
    return LHC_OK;
  }
};

int load_gammas(const double *g, Gammas *out) {
  for (int mu = 0; mu < 4; ++mu)
    for (int e = 0; e < 16; ++e) {
      const double re = g[(mu * 16 + e) * 2], im = g[(mu * 16 + e) * 2 + 1];
      if (!std::isfinite(re) || !std::isfinite(im)) {
        set_error("gamma matrices must be finite");
        return LHC_EINVAL;
      }
      out->g[mu][e] = make_double2(re, im);
    }
  // one unit-phase entry per row?  (exact comparisons: the basis matrices hold 0, +-1)
  out->sparse = true;
  for (int mu = 0; mu < 4 && out->sparse; ++mu)
    for (int s = 0; s < 4 && out->sparse; ++s) {
      int nz = 0;
      for (int s2 = 0; s2 < 4; ++s2) {
        const double2 v = out->g[mu][s * 4 + s2];
        if (v.x == 0.0 && v.y == 0.0) continue;
        ++nz;
        out->col[mu][s] = s2;
        if (v.x == 1.0 && v.y == 0.0)
          out->ph[mu][s] = 0;
        else if (v.x == 0.0 && v.y == 1.0)
          out->ph[mu][s] = 1;
        else if (v.x == -1.0 && v.y == 0.0)
          out->ph[mu][s] = 2;
        else if (v.x == 0.0 && v.y == -1.0)
          out->ph[mu][s] = 3;
        else
          nz = 2;   // not a unit phase: dense
      }
      if (nz != 1) out->sparse = false;
    }
  return LHC_OK;
}

bool is_device(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_args(lhc_ctx ctx, const lhc_lattice *lat, double mass, const double *gammas, const void *a, const void *b,
               int nrhs) {
  if (!ctx || !lat || !gammas || !a || !b || nrhs < 1 || lat->L < 1 || lat->L > 128 || lat->T < 1 ||
      lat->dtype != LHC_C128 || !(mass > -4.0) || !std::isfinite(mass)) {
    set_error("wilson: bad arguments (complex128 fields, 1 <= L <= 128, T >= 1, nrhs >= 1, mass > -4)");
    return LHC_EINVAL;
  }
  if (!is_device(a) || !is_device(b)) {
    set_error("wilson: the fields must be device memory");
    return LHC_EINVAL;
  }
  return LHC_OK;
}

}  // namespace
}  // namespace lhc

extern "C" int lhc_wilson_apply(lhc_ctx ctx, const lhc_lattice *lat, double mass, const double *gammas, int dagger,
                                const void *in, void *out, int nrhs, void *stream) {
  using namespace lhc;
  LHC_TRY(check_args(ctx, lat, mass, gammas, in, out, nrhs));
  Solver sv{ctx, static_cast<cudaStream_t>(stream), lat->L, lat->T, nrhs, 0, mass, {}};
  LHC_TRY(load_gammas(gammas, &sv.gm));
  LHC_CHECK_CUDA(cudaSetDevice(ctx->device));
  return sv.apply(static_cast<const double2 *>(in), static_cast<double2 *>(out), dagger ? -1.0 : 1.0);
}

extern "C" int lhc_wilson_solve(lhc_ctx ctx, const lhc_lattice *lat, double mass, const double *gammas,
                                const void *src, void *sol, int nrhs, double tol, int maxiter, int *iters,
                                double *relres, void *stream) {
  using namespace lhc;
  LHC_TRY(check_args(ctx, lat, mass, gammas, src, sol, nrhs));
  if (!(tol > 0.0) || maxiter < 1) {
    set_error("wilson_solve: tol > 0 and maxiter >= 1 required");
    return LHC_EINVAL;
  }
  LHC_CHECK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Solver sv{ctx, st, lat->L, lat->T, nrhs, (size_t)lat->T * lat->L * lat->L * lat->L * 12, mass, {}};
  LHC_TRY(load_gammas(gammas, &sv.gm));
  const size_t nf = sv.n * nrhs;
  DevBuf work;
  LHC_TRY(dev_alloc(ctx, work, 3 * nf * sizeof(double2) + sizeof(double) * ((size_t)nrhs * (kDotBlocks + 2)) + 256));
  double2 *r = static_cast<double2 *>(work.p), *p = r + nf, *t = p + nf;
  sv.partial = reinterpret_cast<double *>(t + nf);
  sv.coef = sv.partial + (size_t)nrhs * kDotBlocks;
  sv.hpart.resize((size_t)nrhs * kDotBlocks);
  double2 *x = static_cast<double2 *>(sol);
  const double2 *b = static_cast<const double2 *>(src);
  const std::vector<double> one(nrhs, 1.0);
  int status = LHC_OK, it = 0;
  std::vector<double> rr, rr_new, pAp, bnorm, alpha(nrhs), beta(nrhs), nalpha(nrhs);
  DevBuf work2;   // D^dagger D p
  LHC_TRY(dev_alloc(ctx, work2, nf * sizeof(double2)));
  double2 *Ap = static_cast<double2 *>(work2.p);
  do {
    cudaError_t e = cudaMemsetAsync(x, 0, nf * sizeof(double2), st);
    if (e != cudaSuccess) {
      set_error("wilson_solve: %s", cudaGetErrorString(e));
      status = LHC_ECUDA;
      break;
    }
    if ((status = sv.apply(b, r, -1.0)) != LHC_OK) break;   // r = D^dagger b - D^dagger D 0
    if (cudaMemcpyAsync(p, r, nf * sizeof(double2), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      status = LHC_ECUDA;
      break;
    }
    if ((status = sv.dot(r, r, rr)) != LHC_OK) break;
    bnorm = rr;
    for (it = 0; it < maxiter; ++it) {
      bool done = true;
      for (int k = 0; k < nrhs; ++k) done = done && rr[k] <= tol * tol * bnorm[k];
      if (done) break;
      if ((status = sv.apply(p, t, 1.0)) != LHC_OK) break;     // t = D p
      if ((status = sv.apply(t, Ap, -1.0)) != LHC_OK) break;   // Ap = D^dagger D p
      if ((status = sv.dot(p, Ap, pAp)) != LHC_OK) break;
      for (int k = 0; k < nrhs; ++k) {
        const bool active = rr[k] > tol * tol * bnorm[k] && pAp[k] > 0.0;
        alpha[k] = active ? rr[k] / pAp[k] : 0.0;
        nalpha[k] = -alpha[k];
      }
      if ((status = sv.axpby(alpha, p, one, x)) != LHC_OK) break;     // x += alpha p
      if ((status = sv.axpby(nalpha, Ap, one, r)) != LHC_OK) break;   // r -= alpha Ap
      if ((status = sv.dot(r, r, rr_new)) != LHC_OK) break;
      for (int k = 0; k < nrhs; ++k) beta[k] = rr[k] > 0.0 ? rr_new[k] / rr[k] : 0.0;
      if ((status = sv.axpby(one, r, beta, p)) != LHC_OK) break;      // p = r + beta p
      rr = rr_new;
    }
    if (status != LHC_OK) break;
    // true residual of D x = b, relative to |b|
    std::vector<double> b2, res2;
    if ((status = sv.apply(x, t, 1.0)) != LHC_OK) break;
    if ((status = sv.axpby(one, b, std::vector<double>(nrhs, -1.0), t)) != LHC_OK) break;   // t = b - D x
    if ((status = sv.dot(t, t, res2)) != LHC_OK) break;
    if ((status = sv.dot(b, b, b2)) != LHC_OK) break;
    double worst = 0.0;
    for (int k = 0; k < nrhs; ++k) worst = std::max(worst, b2[k] > 0.0 ? std::sqrt(res2[k] / b2[k]) : std::sqrt(res2[k]));
    if (relres) *relres = worst;
    if (iters) *iters = it;
  } while (false);
  dev_free(ctx, work2);
  dev_free(ctx, work);
  return status;
}
