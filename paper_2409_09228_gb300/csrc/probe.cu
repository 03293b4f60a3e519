// libfit: the FP32 throughput probe of fit_probe.h.  Each thread runs 16
// independent FMA chains, so that one warp alone has enough independent work
// to cover the FMA latency and the probe measures the pipe's throughput, not
// its latency; the multiplier and addend are kernel arguments, so nothing
// folds at compile time.
#include <cuda_runtime.h>

#include <string>

#include "fit_probe.h"
#include "internal.h"

namespace fitimpl {
namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(FIT_PROBE_THREADS)
    probe_ffma(float* __restrict__ out, int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (float)threadIdx.x + (float)k;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[(int64_t)blockIdx.x * FIT_PROBE_THREADS + threadIdx.x] = s;
}

__global__ void __launch_bounds__(FIT_PROBE_THREADS)
    probe_ffma2(float* __restrict__ out, int iters, float b, float c) {
  float2 a[kChains];
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
  for (int k = 0; k < kChains; ++k)
    a[k] = make_float2(1e-3f * (float)threadIdx.x + (float)k, (float)k - 1e-3f * (float)threadIdx.x);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
  out[(int64_t)blockIdx.x * FIT_PROBE_THREADS + threadIdx.x] = s;
}

}  // namespace
}  // namespace fitimpl

using namespace fitimpl;

extern "C" int fit_probe_fp32(int packed, int blocks, int iters, float* out, void* stream,
                              double* flops) {
  g_last_error.clear();
  if ((packed != 0 && packed != 1) || blocks < 1 || iters < 1 || !out || !flops)
    return fail(FIT_ERR_ARG, "fit_probe_fp32: bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // b and c keep the chains bounded: a -> a b + c converges to c / (1 - b).
  const float b = 0.999999f, c = 1e-6f;
  if (packed)
    probe_ffma2<<<blocks, FIT_PROBE_THREADS, 0, s>>>(out, iters, b, c);
  else
    probe_ffma<<<blocks, FIT_PROBE_THREADS, 0, s>>>(out, iters, b, c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fit_probe_fp32: launch");
  *flops = (double)blocks * FIT_PROBE_THREADS * (double)iters * kChains * 2.0 * (packed ? 2.0 : 1.0);
  return FIT_OK;
}
