// FMA-throughput probe used to measure the FP64 and FP32 pipe peaks that the
// roofline of the face sweep is reported against.  Each thread runs eight
// independent dependent chains x <- fma(x, a, b), enough to hide the FMA
// latency at full occupancy.
#include <cuda_runtime.h>

#include "ws_internal.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma(T a, T b, int iters, T* out) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)12345.678) out[0] = s;  // keeps the chains live; never true in practice
}

template <typename T>
int probe(int blocks, double* tflops) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (blocks <= 0) blocks = 8 * sms;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return WS_ECUDA;
  cudaStream_t s;
  cudaEvent_t e0, e1;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int iters = sizeof(T) == 8 ? 2048 : 65536;
  k_fma<T><<<blocks, 256, 0, s>>>((T)0.999, (T)1e-4, iters / 16, out);
  cudaEventRecord(e0, s);
  k_fma<T><<<blocks, 256, 0, s>>>((T)0.999, (T)1e-4, iters, out);
  cudaEventRecord(e1, s);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  cudaFree(out);
  if (err != cudaSuccess || cudaGetLastError() != cudaSuccess) return WS_ECUDA;
  double fmas = (double)blocks * 256.0 * 8.0 * (double)iters;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return WS_OK;
}

}  // namespace

extern "C" WS_API int ws_peak_probe(int kind, int blocks, double* tflops) {
  if (!tflops || (kind != 0 && kind != 1)) return WS_EINVAL;
  return kind == 0 ? probe<double>(blocks, tflops) : probe<float>(blocks, tflops);
}

// ---- conversion probe: the integer-pipe FP64 <-> FP32 conversions of the
// mixed-precision kernels, exposed so that tests can compare them with the
// hardware conversions ----
#include "face_fp32.cuh"

namespace {
__global__ void k_convert(int64_t n, const double* __restrict__ in, float* __restrict__ o32,
                          double* __restrict__ o64) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float f = ws::fp32::f64_to_f32(in[i]);
    o32[i] = f;
    o64[i] = ws::fp32::f32_to_f64(f);
  }
}
}  // namespace

extern "C" WS_API int ws_convert_probe(int64_t n, const double* in, float* out32, double* out64) {
  if (n < 0 || (n > 0 && (!in || !out32 || !out64))) return WS_EINVAL;
  if (n == 0) return WS_OK;
  int64_t b = (n + 255) / 256;
  if (b > 65535) b = 65535;
  k_convert<<<(int)b, 256>>>(n, in, out32, out64);
  return cudaDeviceSynchronize() == cudaSuccess ? WS_OK : WS_ECUDA;
}
