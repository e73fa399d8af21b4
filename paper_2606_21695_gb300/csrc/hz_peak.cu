// FMA-pipe peak of the current device, measured (not part of the method).
//
// The subdomain sweep is bound by FP32 FMA issue and the outer Krylov work by
// the FP64 pipe, so the roofline fractions the library's users report need
// the rate those pipes actually reach on their part and clock.  This kernel
// runs nothing but independent fused multiply-adds: every thread carries
// kChains dependent chains a = a * s + t (kChains independent FMAs in flight
// per thread, enough to cover the pipe latency at 32 resident warps per SM),
// over a grid of 4 blocks of 256 threads per SM.  The result is stored only
// when a run-time flag that the host never sets is true, so the compiler
// cannot drop the arithmetic.
#include <cuda_runtime.h>

#include "hz_internal.h"

namespace hz {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(int iters, T s, T t, int store, T* out) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], s, t);
    }
  }
  T sum = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) sum += a[k];
  if (store) out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

template <typename T>
hz_status time_peak(int iters, double* tflops, double* ms_out) {
  const int blocks = sm_count() * kPeakBlocksPerSm;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HZ_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  hz_status s = HZ_OK;
  float ms = 0.0f;
  auto chk = [&](cudaError_t e, const char* what) {
    if (s == HZ_OK && e != cudaSuccess) s = cuda_fail(e, what);
  };
  chk(cudaEventCreate(&e0), "cudaEventCreate");
  chk(cudaEventCreate(&e1), "cudaEventCreate");
  // s < 1, t small: the chains converge to t / (1 - s) and stay normal
  const T sc = (T)0.999, tc = (T)1e-3;
  if (s == HZ_OK) {
    fma_peak_kernel<T><<<blocks, kPeakThreads, 0, st>>>(iters / 4 + 1, sc, tc, 0, nullptr);  // warm-up
    note_launch();
    chk(cudaGetLastError(), "fma_peak_kernel launch");
  }
  if (s == HZ_OK) {
    chk(cudaEventRecord(e0, st), "cudaEventRecord");
    fma_peak_kernel<T><<<blocks, kPeakThreads, 0, st>>>(iters, sc, tc, 0, nullptr);
    note_launch();
    chk(cudaGetLastError(), "fma_peak_kernel launch");
    chk(cudaEventRecord(e1, st), "cudaEventRecord");
    chk(cudaEventSynchronize(e1), "cudaEventSynchronize");
    chk(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (s != HZ_OK) return s;
  const double fmas = (double)blocks * kPeakThreads * kChains * 16.0 * (double)iters;
  *ms_out = ms;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return HZ_OK;
}

}  // namespace
}  // namespace hz

using namespace hz;

extern "C" hz_status hz_fma_peak(int32_t precision, int32_t iters, double* tflops, double* ms) {
  if (!tflops || !ms) return fail(HZ_ERR_INVALID_ARG, "null argument");
  if (iters < 1) return fail(HZ_ERR_INVALID_ARG, "iters must be >= 1");
  if (precision == HZ_FP32_REFINE) return time_peak<float>(iters, tflops, ms);
  if (precision == HZ_FP64) return time_peak<double>(iters, tflops, ms);
  return fail(HZ_ERR_INVALID_ARG, "precision must be HZ_FP64 or HZ_FP32_REFINE");
}
