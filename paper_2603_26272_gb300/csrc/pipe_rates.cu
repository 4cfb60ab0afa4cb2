// pipe_rates.cu -- throughput of the FP64 operations the stage kernels use,
// and of FP32 FMA, on the GPU it runs on (a diagnostic for the roofline
// denominators; not part of libweno.so).
//
// Every thread runs 8 independent dependency chains of one operation, so the
// measured rate is the pipe's throughput, not its latency.  Prints thread
// operations per SM per clock at the SM clock the driver reports.  The FMA
// chains are run on three kinds of data -- converging to 1.0 (a mantissa of
// zeros), converging to a value with a full mantissa, and never converging --
// to show whether the FP64 rate depends on the operands' bit patterns.
#include <cstdio>

#include <cuda_runtime.h>

__device__ __forceinline__ double fma_regs(double a, double b, double c) {
  double d;  // an FMA whose three operands are registers
  asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(d) : "d"(a), "d"(b), "d"(c));
  return d;
}

template <int OP>
__global__ void chains(double *out, int iters, double a, double b) {
  double x[8];
  for (int q = 0; q < 8; ++q) x[q] = 1.0 + 1e-3 * (threadIdx.x + q);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (OP == 0) x[q] = fma(x[q], a, b);
      if (OP == 1) x[q] = fma_regs(x[q], a, b);
      if (OP == 2) x[q] = x[q] + b;
      if (OP == 3) x[q] = x[q] * a;
      if (OP == 4) x[q] = b / x[q];
      if (OP == 5) x[q] = sqrt(x[q]) + b;
      if (OP == 6) x[q] = rsqrt(x[q]) + b;
      if (OP == 7) x[q] = (double)((float)x[q] * 1.0001f);
      if (OP == 8) x[q] = fma(x[q], a, 1.2345678901234567e-3);  // -> 1.2345678901234567
      if (OP == 9) x[q] = fma(x[q], 1.0000000001234567, 1.2345678901234567e-9);  // grows
      if (OP == 10) x[q] = x[q] * 0.99999998765432101;  // decays, full mantissa
    }
  }
  double s = 0;
  for (int q = 0; q < 8; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void chains_f32(float *out, int iters, float a, float b) {
  float x[8];
  for (int q = 0; q < 8; ++q) x[q] = 1.0f + 1e-3f * (threadIdx.x + q);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fmaf(x[q], a, b);
  }
  float s = 0;
  for (int q = 0; q < 8; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

static double g_clk_ghz = 0, g_sms = 0;

static void report(const char *name, float ms, double ops) {
  const double rate = ops / (ms * 1e-3);
  printf("%-28s %9.3f ms  %11.4g op/s  %7.3f op/SM/clk\n", name, ms, rate,
         rate / g_sms / (g_clk_ghz * 1e9));
}

template <int OP>
static int run(const char *name, double *d, int blocks, int threads, int iters) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  chains<OP><<<blocks, threads>>>(d, 16, 0.999, 1e-3);  // warm-up
  cudaEventRecord(e0);
  chains<OP><<<blocks, threads>>>(d, iters, 0.999, 1e-3);
  cudaEventRecord(e1);
  if (cudaEventSynchronize(e1) != cudaSuccess) return 1;
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  report(name, ms, (double)blocks * threads * iters * 8);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return 0;
}

int main() {
  int sms = 0, clk_khz = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
  g_sms = sms;
  g_clk_ghz = clk_khz * 1e-6;
  printf("SMs %d, SM clock %.3f GHz (driver attribute)\n", sms, g_clk_ghz);
  const int threads = 128, blocks = sms * 16;
  double *d = nullptr;
  float *f = nullptr;
  if (cudaMalloc(&d, sizeof(double) * blocks * threads) != cudaSuccess) return 1;
  if (cudaMalloc(&f, sizeof(float) * blocks * threads) != cudaSuccess) return 1;
  int bad = 0;
  bad |= run<0>("DFMA (constant operands) ->1.0", d, blocks, threads, 1024);
  bad |= run<1>("DFMA (register operands) ->1.0", d, blocks, threads, 1024);
  bad |= run<8>("DFMA -> full-mantissa value", d, blocks, threads, 1024);
  bad |= run<9>("DFMA, never converging", d, blocks, threads, 1024);
  bad |= run<10>("DMUL, full-mantissa factor", d, blocks, threads, 1024);
  bad |= run<2>("DADD", d, blocks, threads, 1024);
  bad |= run<3>("DMUL", d, blocks, threads, 1024);
  bad |= run<4>("DDIV", d, blocks, threads, 128);
  bad |= run<5>("DSQRT + DADD", d, blocks, threads, 128);
  bad |= run<6>("DRSQRT + DADD", d, blocks, threads, 128);
  bad |= run<7>("F2F f64->f32->f64 + FMUL", d, blocks, threads, 1024);
  {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    chains_f32<<<blocks, threads>>>(f, 16, 0.999f, 1e-3f);
    cudaEventRecord(e0);
    chains_f32<<<blocks, threads>>>(f, 32768, 0.999f, 1e-3f);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) bad = 1;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    report("FFMA", ms, (double)blocks * threads * 32768 * 8);
  }
  const cudaError_t e = cudaDeviceSynchronize();
  printf("status %s\n", cudaGetErrorString(e));
  cudaFree(d);
  cudaFree(f);
  return (bad || e != cudaSuccess) ? 1 : 0;
}
