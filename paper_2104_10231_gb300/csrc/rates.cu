// Device rates that the design of this library rests on, measured on the GPU
// it runs on (relres_measure_rates): FP32 and FP64 fused multiply-adds,
// conversions between 64-bit integers and FP32, and the bandwidth of a plain
// copy between two halves of a caller-provided buffer.  The FP32 rate is the
// FLOP side of the pair kernel's roofline; the FP64 and conversion rates are
// why the FP32 path keeps FP64 arithmetic and 64-bit conversions out of every
// per-atom and per-pair kernel.  Each kernel runs a fixed number of
// independent chains per thread so that latency is hidden and the issue rate
// of the measured instruction decides the time.
#include <cuda_runtime.h>

#include "common.cuh"
#include "relres_internal.h"

namespace relres {
namespace {

constexpr int kRateIters = 2048;
constexpr int kRateThreads = 256;

__global__ void k_rate_ffma(float seed, float* out) {
  float a = seed + threadIdx.x, b = a * 0.5f, c = a * 0.25f, d = a * 0.125f;
  float e = a + 1.f, f = b + 1.f, g = c + 1.f, h = d + 1.f;
  const float m = 0.9999f, k = 1e-7f;
  for (int i = 0; i < kRateIters; ++i) {
    a = fmaf(a, m, k);
    b = fmaf(b, m, k);
    c = fmaf(c, m, k);
    d = fmaf(d, m, k);
    e = fmaf(e, m, k);
    f = fmaf(f, m, k);
    g = fmaf(g, m, k);
    h = fmaf(h, m, k);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a + b + c + d + e + f + g + h;
}

__global__ void k_rate_dfma(double seed, double* out) {
  double a = seed + threadIdx.x, b = a * 0.5, c = a * 0.25, d = a * 0.125;
  const double m = 0.9999, k = 1e-7;
  for (int i = 0; i < kRateIters / 8; ++i) {
    a = fma(a, m, k);
    b = fma(b, m, k);
    c = fma(c, m, k);
    d = fma(d, m, k);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a + b + c + d;
}

__global__ void k_rate_conv64(long long seed, float* out) {
  long long a = seed + threadIdx.x, b = a * 3, c = a * 5, d = a * 7;
  float s = 0.f;
  for (int i = 0; i < kRateIters / 8; ++i) {
    s += __ll2float_rn(a) + __ll2float_rn(b) + __ll2float_rn(c) + __ll2float_rn(d);
    a += 17;
    b += 19;
    c += 23;
    d += 29;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_rate_copy(const float4* __restrict__ src, float4* __restrict__ dst, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    dst[i] = src[i];
}

__global__ void k_eval_recip(const double* __restrict__ x, float* __restrict__ out32,
                             double* __restrict__ out64, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const double v = x[k];
    out32[k] = rcp_nr(float(v));
    out64[k] = rcp_d(v);
    out64[n + k] = rsqrt_d(v);
  }
}

// milliseconds of one launch (after one warm-up launch)
template <class L>
cudaError_t time_ms(cudaStream_t st, L launch, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace
}  // namespace relres

using namespace relres;

extern "C" relres_status relres_measure_rates(void* d_scratch, size_t scratch_bytes, void* cuda_stream,
                                              relres_rates* out) {
  if (!d_scratch || !out || scratch_bytes < (size_t(1) << 20) ||
      (reinterpret_cast<size_t>(d_scratch) & 15) != 0)
    return RELRES_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0, clk_khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev) != cudaSuccess)
    return RELRES_ERR_CUDA;
  const int blocks = sms * 8;
  const size_t threads = size_t(blocks) * kRateThreads;
  // the arithmetic kernels write one value per thread at the start of the buffer
  if (scratch_bytes < threads * sizeof(double)) return RELRES_ERR_ARG;
  const double per_sm_clk = double(sms) * double(clk_khz) * 1e3;  // SM-clocks per second
  float ms = 0.f;
  cudaError_t e = time_ms(st, [&]() {
    k_rate_ffma<<<blocks, kRateThreads, 0, st>>>(1.5f, static_cast<float*>(d_scratch));
    return cudaGetLastError();
  }, &ms);
  if (e != cudaSuccess) return RELRES_ERR_CUDA;
  out->ffma_per_clk_sm = double(threads) * kRateIters * 8 / (ms * 1e-3) / per_sm_clk;
  e = time_ms(st, [&]() {
    k_rate_dfma<<<blocks, kRateThreads, 0, st>>>(1.5, static_cast<double*>(d_scratch));
    return cudaGetLastError();
  }, &ms);
  if (e != cudaSuccess) return RELRES_ERR_CUDA;
  out->dfma_per_clk_sm = double(threads) * (kRateIters / 8) * 4 / (ms * 1e-3) / per_sm_clk;
  e = time_ms(st, [&]() {
    k_rate_conv64<<<blocks, kRateThreads, 0, st>>>(12345ll, static_cast<float*>(d_scratch));
    return cudaGetLastError();
  }, &ms);
  if (e != cudaSuccess) return RELRES_ERR_CUDA;
  out->conv64_per_clk_sm = double(threads) * (kRateIters / 8) * 4 / (ms * 1e-3) / per_sm_clk;
  // copy: first half of the buffer to the second half
  const size_t n4 = scratch_bytes / 2 / sizeof(float4);
  const float4* src = static_cast<const float4*>(d_scratch);
  float4* dst = static_cast<float4*>(d_scratch) + n4;
  e = time_ms(st, [&]() {
    k_rate_copy<<<sms * 4, 512, 0, st>>>(src, dst, n4);
    return cudaGetLastError();
  }, &ms);
  if (e != cudaSuccess) return RELRES_ERR_CUDA;
  out->copy_gbs = 2.0 * double(n4) * sizeof(float4) / (ms * 1e-3) / 1e9;
  out->sm_count = sms;
  out->clock_mhz = clk_khz / 1000;
  out->fp32_tflops = out->ffma_per_clk_sm * 2.0 * per_sm_clk / 1e12;
  out->fp64_tflops = out->dfma_per_clk_sm * 2.0 * per_sm_clk / 1e12;
  return RELRES_OK;
}

extern "C" relres_status relres_eval_recip(const double* d_x, float* d_out32, double* d_out64, int n,
                                           void* cuda_stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_out32 || !d_out64))) return RELRES_ERR_ARG;
  if (n == 0) return RELRES_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int blocks = (n + kRateThreads - 1) / kRateThreads;
  k_eval_recip<<<blocks < 1024 ? blocks : 1024, kRateThreads, 0, st>>>(d_x, d_out32, d_out64, n);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return RELRES_ERR_CUDA;
  return RELRES_OK;
}
