// peaks.cu — FP32 FMA and special-function-unit throughput probes (a measurement aid with no
// counterpart in the paper).  The compositing kernels are bound by FP32 arithmetic and by the
// special-function unit (one ex2 and one reciprocal per response evaluation), so their roofline
// fractions divide by peaks measured on the same GPU, in the same run, with these kernels.
//
// Every thread runs `iters` iterations of kChains independent dependency chains of one
// operation; with enough resident warps the chains keep the pipe busy and the launch time gives
// the pipe's throughput.  The chains converge to finite values (|a| < 1 for the FMA, 2^-x on
// (0, 1] for ex2) and each thread writes its sum so the work stays live.
#include "ut3d_device.cuh"
#include "ut3d_internal.h"

namespace ut3d {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_probe_fma(int iters, float a, float b, float *__restrict__ out) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 1e-3f * (float)threadIdx.x + (float)j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_neg(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
  return y;
}

__global__ void __launch_bounds__(256) k_probe_ex2(int iters, float *__restrict__ out) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = 1e-3f * (float)threadIdx.x + 0.1f * (float)j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = ex2_neg(x[j]);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace ut3d

using namespace ut3d;

extern "C" ut_status ut_peak_probe(int32_t kind, int32_t blocks, int32_t threads, int32_t iters, float *out,
                                   ut_stream stream) {
  if ((kind != UT_PROBE_FMA && kind != UT_PROBE_EX2) || blocks < 1 || threads < 32 || threads > 256 ||
      (threads & 31) || iters < 1 || !out)
    return UT_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (kind == UT_PROBE_FMA) k_probe_fma<<<blocks, threads, 0, s>>>(iters, 0.999f, 1e-3f, out);
  else k_probe_ex2<<<blocks, threads, 0, s>>>(iters, out);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? UT_OK : UT_ERR_CUDA;
}
