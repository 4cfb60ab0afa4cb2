// weno_peak.cu -- measured FMA throughput of the GPU the library runs on: the
// denominator of the stage kernels' roofline.  The stage kernels are bound by
// FP64 instruction issue (no step of the method is a dense contraction, and
// their HBM traffic is two orders of magnitude below the memory roof), so
// their peak is the FP64 FMA rate, which on GB300 also depends on the
// operands: chains whose values have full mantissas run slower than chains
// that settle on short ones.  Three kinds are timed:
//   0  FP64 FMA chains that settle on a full-mantissa fixed point (the data
//      of a real solve),
//   1  FP64 FMA chains that settle on 1.0 (mantissa of zeros),
//   2  FP32 FMA chains.
// Every thread runs 8 independent chains so the figure is throughput, not
// latency; the grid holds 8 blocks of 256 threads per SM.
#include <cstring>
#include <string>

#include "../../include/weno.h"
#include "weno_internal.h"

namespace {

// Never written in practice (every chain stays positive); it keeps the
// chains from being removed as dead code.
__device__ double g_sink64;
__device__ float g_sink32;

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fma64(int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) x[q] = 1.0 + 0.001 * (threadIdx.x & 7) + 0.01 * q;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = fma(x[q], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += x[q];
  if (s < 0.0) g_sink64 = s;
}

__global__ void __launch_bounds__(256) k_fma32(int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) x[q] = 1.0f + 0.001f * (threadIdx.x & 7) + 0.01f * q;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = fmaf(x[q], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += x[q];
  if (s < 0.0f) g_sink32 = s;
}

weno_status fail(weno_status s, const std::string &m) {
  weno::set_last_error(m);
  return s;
}

cudaError_t launch(int kind, int blocks, int iters, cudaStream_t s) {
  if (kind == 0)  // fixed point b / (1 - a) = 1.2345678901234...: full mantissa
    k_fma64<<<blocks, 256, 0, s>>>(iters, 0.99900000000001234, 1.2345678901234567e-3);
  else if (kind == 1)  // x <- x/2 + 1/2 settles on 1.0 exactly
    k_fma64<<<blocks, 256, 0, s>>>(iters, 0.5, 0.5);
  else
    k_fma32<<<blocks, 256, 0, s>>>(iters, 0.999f, 1.2345678e-3f);
  return cudaGetLastError();
}

}  // namespace

extern "C" weno_status weno_fma_rate(int kind, int iters, double *flops_per_s, void *stream) {
  if (kind < 0 || kind > 2) return fail(WENO_ERR_ARG, "kind must be 0, 1 or 2");
  if (iters < 1 || iters > (1 << 24)) return fail(WENO_ERR_ARG, "iters must be in [1, 2^24]");
  if (!flops_per_s) return fail(WENO_ERR_ARG, "flops_per_s is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(WENO_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
  const int blocks = 8 * sms;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch(kind, blocks, iters < 64 ? iters : 64, s);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = launch(kind, blocks, iters, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(WENO_ERR_CUDA, std::string("fma rate: ") + cudaGetErrorString(e));
  const double fmas = (double)blocks * 256.0 * kChains * (double)iters;
  *flops_per_s = 2.0 * fmas / (ms * 1e-3);
  weno::set_last_error("");
  return WENO_OK;
}
