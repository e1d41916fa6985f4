// Failure-detection self-test: a kernel that waits on an mbarrier nothing completes.  The
// wait is bounded (limit in microseconds); when it gives up it sets the context's device
// error word and returns, leaving the context usable.  lhc_sync then reports LHC_ETIMEOUT.
#include "lhc_internal.h"
#include "tc_ptx.cuh"

namespace {

__global__ void never_completed_wait(int *err, long long limit_cycles) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    lhc::tc::mbar_init(&bar, 1);
    lhc::tc::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t0 = clock64();
    while (!lhc::tc::mbar_try_wait(&bar, 0)) {   // phase 0 never completes: nobody arrives
      if (clock64() - t0 > limit_cycles) {
        atomicExch(err, 99);
        break;
      }
    }
  }
  __syncthreads();
}

}  // namespace

extern "C" int lhc_selftest_timeout(lhc_ctx ctx, int limit_us, void *stream) {
  if (!ctx || limit_us < 1 || limit_us > 2000000) {
    lhc::set_error("lhc_selftest_timeout: bad arguments");
    return LHC_EINVAL;
  }
  LHC_CHECK_CUDA(cudaSetDevice(ctx->device));
  int clk_khz = 0;
  LHC_CHECK_CUDA(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, ctx->device));
  long long cycles = (long long)limit_us * (long long)clk_khz / 1000;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  never_completed_wait<<<1, 32, 0, st>>>(ctx->dev_err, cycles);
  lhc::note_launch();
  LHC_CHECK_CUDA(cudaGetLastError());
  return lhc_sync(ctx, stream);
}

extern "C" int lhc_selftest_flag(lhc_ctx ctx, int limit_us, void *stream) {
  if (!ctx || limit_us < 1 || limit_us > 2000000) {
    lhc::set_error("lhc_selftest_flag: bad arguments");
    return LHC_EINVAL;
  }
  LHC_CHECK_CUDA(cudaSetDevice(ctx->device));
  int clk_khz = 0;
  LHC_CHECK_CUDA(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, ctx->device));
  const long long cycles = (long long)limit_us * (long long)clk_khz / 1000;
  never_completed_wait<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(ctx->dev_err, cycles);
  lhc::note_launch();
  LHC_CHECK_CUDA(cudaGetLastError());
  return LHC_OK;
}
