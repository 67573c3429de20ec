// teno_noalloc.cu -- CFL time step with no device allocation.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework whose caching allocator owns the GPU (a cudaMalloc behind its
// back fragments or exhausts the pool it manages), drivers that work to a
// fixed device-memory budget decided at start-up, and real-time loops where
// an allocation's implicit synchronisation is not acceptable.
// teno_cfl_dt_noalloc gives them the step-size reduction of the solver
// without any allocation: the per-block partial maxima live in a file-scope
// device array of fixed size that every GPU loading this library holds until
// the process exits, and the caller passes every input and the output.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>

#include "../../include/teno.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 8;
constexpr int kCellsPerBlock = kThreads * kCellsPerThread;       // 2048
constexpr int kMaxBlocks = TENO_NOALLOC_MAX_CELLS / kCellsPerBlock;  // 4096
static_assert(kMaxBlocks * kCellsPerBlock == TENO_NOALLOC_MAX_CELLS, "block split");

// [0, kMaxBlocks): partial maxima of pass 1; [kMaxBlocks]: the resulting dt
static __device__ __align__(256) double g_cfl_scratch[kMaxBlocks + 1];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// pass 1: block b writes max over its cells of (|v| + c) / len into scratch[b]
__global__ void __launch_bounds__(kThreads) cfl_partial(const double* __restrict__ U,
                                                        const double* __restrict__ len,
                                                        int64_t n, int n_var, double gamma,
                                                        double adv_speed,
                                                        double* __restrict__ scratch) {
  double lam = 0.0;
  const int64_t base = (int64_t)blockIdx.x * kCellsPerBlock + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kCellsPerThread; ++k) {
    const int64_t c = base + (int64_t)k * kThreads;
    if (c >= n) break;
    double s;
    if (n_var == 1) {
      s = adv_speed;
    } else {
      const double rho = U[c], u = U[n + c] / rho, v = U[2 * n + c] / rho;
      const double p = (gamma - 1.0) * (U[3 * n + c] - 0.5 * rho * (u * u + v * v));
      s = sqrt(u * u + v * v) + sqrt(gamma * p / rho);
      // a non-physical cell (rho <= 0, p <= 0 or NaN) makes the maximum infinite
      // (fmax would drop a NaN speed)
      if (!(rho > 0.0) || !(p > 0.0)) s = __longlong_as_double(0x7ff0000000000000LL);
    }
    lam = fmax(lam, s / len[c]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  __shared__ double red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lam;
  __syncthreads();
  if (threadIdx.x < 32) {
    lam = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
    if (threadIdx.x == 0) scratch[blockIdx.x] = lam;
  }
}

// pass 2: one block reduces the nb partial maxima and writes dt
__global__ void __launch_bounds__(kThreads) cfl_final(const double* __restrict__ scratch, int nb,
                                                      double cfl, double* __restrict__ dt_out) {
  double lam = 0.0;
  for (int i = threadIdx.x; i < nb; i += kThreads) lam = fmax(lam, scratch[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  __shared__ double red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lam;
  __syncthreads();
  if (threadIdx.x < 32) {
    lam = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
    // no finite positive maximum speed (a non-physical cell, or every speed
    // zero): the documented NaN sentinel
    if (threadIdx.x == 0)
      *dt_out = (lam > 0.0 && lam < __longlong_as_double(0x7ff0000000000000LL))
                    ? cfl / lam
                    : __longlong_as_double(0x7ff8000000000000LL);
  }
}

// device address of the scratch array on `device` (looked up once per device,
// with that device current)
int scratch_for(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return TENO_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_cfl_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return TENO_ECUDA;
    }
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return TENO_OK;
}

// restores the calling thread's current device on every return
struct DeviceGuard {
  int saved = -1;
  DeviceGuard() {
    if (cudaGetDevice(&saved) != cudaSuccess) {
      saved = -1;
      cudaGetLastError();
    }
  }
  ~DeviceGuard() {
    if (saved >= 0) cudaSetDevice(saved);
  }
};

}  // namespace

extern "C" int teno_cfl_dt_noalloc(int device, void* cuda_stream, int32_t n_var, int64_t n_cell,
                                   const double* U, const double* cell_len, double gamma,
                                   double adv_x, double adv_y, double cfl, double* dt,
                                   int dt_on_device) {
  if (n_var != 1 && n_var != 4) return TENO_EINVAL;
  if (n_cell < 1 || n_cell > TENO_NOALLOC_MAX_CELLS) return TENO_EINVAL;
  if (!U || !cell_len || !dt || !(cfl > 0.0) || (n_var == 4 && !(gamma > 1.0)))
    return TENO_EINVAL;
  // an error left by earlier, unrelated work is not this call's
  cudaGetLastError();
  DeviceGuard guard;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return TENO_ECUDA;
  }
  double* scratch = nullptr;
  int rc = scratch_for(device, &scratch);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nb = (int)((n_cell + kCellsPerBlock - 1) / kCellsPerBlock);
  const double adv = sqrt(adv_x * adv_x + adv_y * adv_y);
  cfl_partial<<<nb, kThreads, 0, st>>>(U, cell_len, n_cell, n_var, gamma, adv, scratch);
  double* out = dt_on_device ? dt : scratch + kMaxBlocks;
  cfl_final<<<1, kThreads, 0, st>>>(scratch, nb, cfl, out);
  if (cudaGetLastError() != cudaSuccess) return TENO_ECUDA;
  if (!dt_on_device) {
    double h = 0.0;
    if (cudaMemcpyAsync(&h, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return TENO_ECUDA;
    }
    if (!(h > 0.0) || !std::isfinite(h)) return TENO_ENONPHYS;
    *dt = h;
  }
  return TENO_OK;
}
