// Arithmetic peak microbenchmark: the rates the roofline of the sweep
// kernels divides by.  Every thread runs NACC independent fused multiply-add
// chains of a register-resident accumulator, so the FMA pipe of the chosen
// type is the only limit; the grid fills every SM.  Rates count 2 flops per
// multiply-add (4 per packed FP32 pair).
#include <cuda_runtime.h>

#include "enoao.h"

namespace {

constexpr int NACC = 8;     // independent chains per thread (covers the FMA latency)
constexpr int UNROLL = 64;  // multiply-adds per chain per loop trip

template <typename T>
struct FmaOp;

template <>
struct FmaOp<float> {
  static __device__ __forceinline__ float step(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float seed(int k) { return 1.0f + 1e-3f * k; }
  static __device__ __forceinline__ float sum(float a) { return a; }
  static constexpr int kFlops = 2;
};

template <>
struct FmaOp<float2> {
  static __device__ __forceinline__ float2 step(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, c);
  }
  static __device__ __forceinline__ float2 seed(int k) {
    return make_float2(1.0f + 1e-3f * k, 1.0f - 1e-3f * k);
  }
  static __device__ __forceinline__ float sum(float2 a) { return a.x + a.y; }
  static constexpr int kFlops = 4;
};

template <>
struct FmaOp<double> {
  static __device__ __forceinline__ double step(double a, double b, double c) { return __fma_rn(a, b, c); }
  static __device__ __forceinline__ double seed(int k) { return 1.0 + 1e-3 * k; }
  static __device__ __forceinline__ float sum(double a) { return (float)a; }
  static constexpr int kFlops = 2;
};

// b and c come from the host, so the compiler cannot fold the chains; the
// sum is stored so that they are not dead.
template <typename T>
__global__ void __launch_bounds__(256) fma_kernel(T b, T c, int trips, float* out) {
  T acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = FmaOp<T>::seed(k + threadIdx.x);
  for (int t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
      for (int k = 0; k < NACC; ++k) acc[k] = FmaOp<T>::step(acc[k], b, c);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < NACC; ++k) s += FmaOp<T>::sum(acc[k]);
  if (s == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // practically never
}

template <typename T>
cudaError_t time_one(T b, T c, int trips, cudaStream_t s, float* out, double* tflops, float* ms) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int block = 256, grid = sms * 8;  // 64 warps per SM
  cudaEvent_t t0, t1;
  e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e != cudaSuccess) return e;
  fma_kernel<T><<<grid, block, 0, s>>>(b, c, trips, out);  // warm-up
  e = cudaEventRecord(t0, s);
  fma_kernel<T><<<grid, block, 0, s>>>(b, c, trips, out);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(t1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(t1);
  float m = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&m, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (e != cudaSuccess) return e;
  const double fmas = (double)grid * block * NACC * UNROLL * (double)trips;
  *tflops = fmas * FmaOp<T>::kFlops / (m * 1e-3) / 1e12;
  *ms = m;
  return cudaSuccess;
}

}  // namespace

extern "C" enoao_status enoao_measure_fma_peak(int kind, int trips, void* cuda_stream,
                                               double* tflops, float* ms) {
  if (!tflops || !ms || trips < 1) return ENOAO_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  float* out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(float) * 256 * 8 * 1024);
  if (e != cudaSuccess) return ENOAO_ENOMEM;
  if (kind == ENOAO_PEAK_FP32)
    e = time_one<float>(1.0000001f, 1e-7f, trips, s, out, tflops, ms);
  else if (kind == ENOAO_PEAK_FP32X2)
    e = time_one<float2>(make_float2(1.0000001f, 0.9999999f), make_float2(1e-7f, -1e-7f), trips, s,
                         out, tflops, ms);
  else if (kind == ENOAO_PEAK_FP64)
    e = time_one<double>(1.0000000001, 1e-10, trips, s, out, tflops, ms);
  else
    e = cudaErrorInvalidValue;
  cudaFree(out);
  if (e == cudaErrorInvalidValue) return ENOAO_EINVAL;
  return e == cudaSuccess ? ENOAO_OK : ENOAO_ECUDA;
}
