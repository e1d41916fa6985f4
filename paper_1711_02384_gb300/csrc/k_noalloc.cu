// Allocation-free combine: lhc_combine_noalloc.
//
// Some callers cannot let a library allocate device memory: a process whose device memory
// is already owned by another allocator (an analysis framework's caching pool that has
// reserved almost all of HBM, so a further cudaMalloc fails or fragments its pool), and
// host code that must not stall, since cudaMalloc and cudaFree can synchronize the whole
// device.  For them this entry point runs the combine with its intermediate tensors in a
// fixed scratch array that is part of the library image: a file-scope __device__ array of
// kNoallocScratchBytes (32 MiB).  Every GPU that loads the library holds that array until
// the process exits; the entry point itself never calls cudaMalloc, cudaFree or any
// allocating routine, and it needs no context.
//
// The scratch is shared by every call on a device and keeps the last call's contents.
// Every element the kernels read is written earlier in the same call, so nothing needs
// clearing; but two calls whose kernels overlap on the GPU (different streams, no
// ordering between them) race on the scratch and give wrong results.  Order such calls
// on one stream or with events.
#include <algorithm>
#include <mutex>

#include "lhc_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(32) << 20;

// the scratch: only host code below needs its device address
static __device__ __align__(256) double2 g_noalloc_scratch[kNoallocScratchBytes / sizeof(double2)];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double2 *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch for the current device.  In host code the symbol
// g_noalloc_scratch is only a host-side stand-in, never a device address, so the address
// is looked up once per device (with that device current) and cached.
int scratch_for_current_device(double2 **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    lhc::set_error("cudaGetDevice: %s", cudaGetErrorString(e));
    return LHC_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    lhc::set_error("device %d out of range", dev);
    return LHC_EINVAL;
  }
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      lhc::set_error("cudaGetSymbolAddress of the combine scratch: %s", cudaGetErrorString(e));
      return LHC_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double2 *>(p);
  }
  *out = g_scratch_ptr[dev];
  return LHC_OK;
}

// Device memory of the current device, or managed memory.  A buffer of another GPU is
// refused: the scratch address belongs to the current device, and the kernels would
// otherwise read the buffer as peer memory (or fail where peer access is off).
bool on_device(const void *p, int dev) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int lhc_combine_noalloc(int kind, const void *spec, int np, const void *ins, int nq, int n_r, int nt,
                                   const void *snk, const void *ins_g, const void *src, int ng, int prec, void *out,
                                   void *stream) {
  if (kind != LHC_MESON && kind != LHC_BARYON) {
    lhc::set_error("unknown kind %d", kind);
    return LHC_EINVAL;
  }
  if (np < 1 || nq < 1 || n_r < 1 || ng < 1 || nt < 1) {
    lhc::set_error("sizes must be positive");
    return LHC_EINVAL;
  }
  if (prec != LHC_FP64 && prec != LHC_MIXED) {
    lhc::set_error("unknown precision %d", prec);
    return LHC_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    lhc::set_error("cudaGetDevice failed");
    return LHC_ECUDA;
  }
  const void *bufs[6] = {spec, ins, snk, ins_g, src, out};
  for (const void *b : bufs)
    if (!on_device(b, dev)) {
      lhc::set_error("lhc_combine_noalloc takes buffers of the current device only (it cannot stage host "
                     "memory or read another GPU's)");
      return LHC_EINVAL;
    }
  // scratch use: Xs (ng*np*12*n_r) once, then Xi (ng*nq*12*n_r) per insertion slice of a
  // chunk, then the ng ints that map each Gamma_ins to its first equal one
  const size_t K = (size_t)12 * n_r;
  const size_t xs = (size_t)ng * np * K, xi_slice = (size_t)ng * nq * K;
  const size_t cap = kNoallocScratchBytes / sizeof(double2) - ((size_t)ng * sizeof(int) + 15) / 16;
  if (xs + xi_slice > cap) {
    lhc::set_error("combine too large for the %zu-byte allocation-free scratch: needs %zu bytes for one "
                   "insertion slice (ng*(np+nq)*12*n_r*16 + 4*ng); use lhc_combine",
                   kNoallocScratchBytes, (xs + xi_slice) * sizeof(double2));
    return LHC_EINVAL;
  }
  double2 *scratch = nullptr;
  int s = scratch_for_current_device(&scratch);
  if (s != LHC_OK) return s;
  const int chunk = (int)std::min<size_t>((size_t)nt, (cap - xs) / xi_slice);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int t0 = 0; t0 < nt; t0 += chunk) {
    const int n = std::min(chunk, nt - t0);
    s = lhc::run_combine_scratch(kind, static_cast<const double2 *>(spec), np,
                                 static_cast<const double2 *>(ins) + (size_t)t0 * nq * n_r * 192, nq, n_r, n,
                                 static_cast<const double2 *>(snk), static_cast<const double2 *>(ins_g),
                                 static_cast<const double2 *>(src), ng, prec, scratch, scratch + xs,
                                 static_cast<double2 *>(out) + (size_t)t0 * ng * np * nq, st);
    if (s != LHC_OK) return s;
  }
  return LHC_OK;
}
