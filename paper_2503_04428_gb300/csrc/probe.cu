// probe.cu -- measured arithmetic peak of the current GPU (include/hydro.h:
// hydro_fma_rate).  The FP64 forms of the step are bound by the FP64 FMA
// rate of the device rather than by HBM, so their roofline needs that rate
// measured on the machine at hand, as the HBM roofline uses a measured copy
// bandwidth.
#include <cuda_runtime.h>

#include <algorithm>

#include "runtime.h"

namespace hydro {

// Eight independent FMA chains per thread, a <- a*b + c with |b| < 1, so the
// values stay bounded and normal; the sink store is never taken but keeps the
// chains live.
template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(T* sink, int iters, T b, T c) {
  T a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == T(-1)) sink[blockIdx.x] = s;
}

// The same with paired FP32 operands: each step of a chain is one
// __ffma2_rn on a float2 (two FMAs in one instruction, the f32x2 form of
// this architecture).
__global__ void __launch_bounds__(256) fma2_rate_kernel(float* sink, int iters, float b, float c) {
  float2 a[8];
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = make_float2(float(threadIdx.x + k) * 1e-3f, float(threadIdx.x + 2 * k) * 1e-3f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k].x + a[k].y;
  if (s == -1.f) sink[blockIdx.x] = s;
}

template <typename T, bool PAIRED = false>
static int fma_rate(double* tflops) {
  int dev = 0, nsm = 0;
  HCK(cudaGetDevice(&dev));
  HCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * 8, threads = 256;
  T* sink = nullptr;
  HCK(cudaMalloc(&sink, sizeof(T) * blocks));
  cudaEvent_t e0, e1;
  HCK(cudaEventCreate(&e0));
  HCK(cudaEventCreate(&e1));
  const T b = T(0.999), c = T(1e-4);
  int iters = 64;
  double best = 0.0;
  for (int rep = 0; rep < 6; ++rep) {
    HCK(cudaEventRecord(e0, 0));
    if constexpr (PAIRED) fma2_rate_kernel<<<blocks, threads>>>(sink, iters, b, c);
    else fma_rate_kernel<T><<<blocks, threads>>>(sink, iters, b, c);
    HCK(cudaGetLastError());
    HCK(cudaEventRecord(e1, 0));
    HCK(cudaEventSynchronize(e1));
    float ms = 0.f;
    HCK(cudaEventElapsedTime(&ms, e0, e1));
    const double flops = (PAIRED ? 4.0 : 2.0) * 8 * 16 * (double)iters * blocks * threads;
    if (rep >= 2) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    // grow the launch to about 20 ms after the first, short calibration runs
    if (rep < 2 && ms > 0.f) iters = std::max(64, (int)std::min(1e8, iters * 20.0 / ms));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  *tflops = best;
  return HYDRO_OK;
}

}  // namespace hydro

extern "C" int hydro_fma_rate(int precision, double* tflops_out) {
  using namespace hydro;
  if (!tflops_out || (precision != 32 && precision != 64 && precision != HYDRO_FMA_F32X2)) {
    set_error("hydro_fma_rate: precision must be 32, 64 or HYDRO_FMA_F32X2 and tflops_out non-null");
    return HYDRO_ERR_ARG;
  }
  if (precision == 64) return fma_rate<double>(tflops_out);
  if (precision == 32) return fma_rate<float>(tflops_out);
  return fma_rate<float, true>(tflops_out);
}
