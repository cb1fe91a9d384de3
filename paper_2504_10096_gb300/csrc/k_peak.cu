// FP64 FMA throughput of the device, measured (bse_measure_fp64_peak).
//
// The FP64 path's structured product is bound by the FP64 pipe on this GPU,
// so its roofline needs the pipe's rate.  This kernel keeps 8 independent
// FMA chains per thread (enough to cover the pipe latency), runs a fixed
// number of iterations, and is timed with CUDA events; no memory traffic
// besides one store per thread (so the compiler keeps the chains).
#include "../../include/bse.h"
#include "bse_internal.cuh"

namespace bse {
namespace {

constexpr int PK_CHAINS = 8;
constexpr int PK_THREADS = 256;

__global__ void __launch_bounds__(PK_THREADS)
k_fp64_fma(double* __restrict__ out, int iters, double a, double b) {
  double x[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace bse

extern "C" int bse_measure_fp64_peak(int iters, double* tflops_out, double* ms_out) {
  if (iters < 1 || iters > (1 << 24) || !tflops_out) return BSE_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return BSE_ECUDA;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bse::k_fp64_fma, bse::PK_THREADS, 0) != cudaSuccess)
    return BSE_ECUDA;
  const int grid = sms * (occ > 0 ? occ : 1);
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * (size_t)grid * bse::PK_THREADS) != cudaSuccess) {
    cudaGetLastError();
    return BSE_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // a = 1 - 2^-40, b = 2^-30: the chains stay finite and are not constant-folded
  const double a = 1.0 - 0x1p-40, b = 0x1p-30;
  bse::k_fp64_fma<<<grid, bse::PK_THREADS>>>(out, iters / 8 + 1, a, b);    // warm-up
  cudaEventRecord(e0);
  bse::k_fp64_fma<<<grid, bse::PK_THREADS>>>(out, iters, a, b);
  cudaEventRecord(e1);
  const cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || cudaGetLastError() != cudaSuccess || !(ms > 0.f)) return BSE_ECUDA;
  const double flops = 2.0 * bse::PK_CHAINS * (double)iters * grid * bse::PK_THREADS;
  *tflops_out = flops / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return BSE_OK;
}
