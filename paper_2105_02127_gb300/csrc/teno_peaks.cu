// teno_peaks.cu -- arithmetic pipe peaks of the GPU the library runs on
// (measurement support; the paper has no counterpart).
//
// The FP64 reconstruction runs on the FP64 pipe, whose rate bounds it (it is
// far below the HBM bound on this part); the double-float and FP32-mixed
// kernels issue FP32 instructions.  teno_fma_peak measures the sustained rate
// of independent fused multiply-adds on every SM, so that the roofline
// fractions of those kernels are taken against measured peaks rather than
// nominal ones.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/teno.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;  // independent FMA chains per thread (hides the pipe latency)

static __device__ double g_peak_sink[2];

// Each thread runs kChains independent chains x = x * a + b for `iters`
// rounds (a, b are kernel arguments, so nothing folds at compile time); the
// result is stored only when it equals `never`, which keeps every FMA live.
template <typename T>
__global__ void __launch_bounds__(kThreads) fma_kernel(T a, T b, int iters, T never) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == never) g_peak_sink[sizeof(T) == 8] = (double)s;
}

template <typename T>
int run(cudaStream_t st, int blocks, int iters, double* rate) {
  // a, b keep the chains bounded (x -> b / (1 - a))
  const T a = (T)0.999, b = (T)1e-3, never = (T)-12345.0;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TENO_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return TENO_ECUDA;
  }
  int rc = TENO_OK;
  fma_kernel<T><<<blocks, kThreads, 0, st>>>(a, b, iters / 8, never);  // warm-up
  cudaEventRecord(e0, st);
  fma_kernel<T><<<blocks, kThreads, 0, st>>>(a, b, iters, never);
  cudaEventRecord(e1, st);
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
      cudaGetLastError() != cudaSuccess || !(ms > 0.f)) {
    cudaGetLastError();
    rc = TENO_ECUDA;
  } else {
    const double flops = 2.0 * kChains * (double)iters * kThreads * (double)blocks;
    *rate = flops / (ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace

extern "C" int teno_fma_peak(int device, void* cuda_stream, int precision, double* flops_per_s) {
  if (!flops_per_s || (precision != 0 && precision != 1)) return TENO_EINVAL;
  int saved = -1;
  if (cudaGetDevice(&saved) != cudaSuccess) saved = -1;
  cudaGetLastError();
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return TENO_ECUDA;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // 8 blocks of 256 threads per SM; about 100 ms of FP64 and 20 ms of FP32 work
  const int blocks = (sms > 0 ? sms : 1) * 8;
  const int rc = precision == 1 ? run<double>(st, blocks, 4096, flops_per_s)
                                : run<float>(st, blocks, 1 << 16, flops_per_s);
  if (saved >= 0) cudaSetDevice(saved);
  return rc;
}
