// Throughput microbenchmarks for the roofline of the step kernels (no
// counterpart in the paper).  The step kernels are bound by FP32 CUDA-core
// arithmetic, shared-memory traffic and per-step latency, never by HBM, so
// the denominators they are reported against are measured here on the same
// device: FP32 fused multiply-add throughput, FP64 fused multiply-add
// throughput (the adjoint recursion runs in FP64) and shared-memory load
// bandwidth.  Each is one short kernel timed with CUDA events after a
// warm-up launch; the result is the best of a few repetitions.
#include <cuda_runtime.h>

#include "sfd.h"

namespace {

constexpr int kChains = 16;      // independent FMA chains per thread (latency x issue width)
constexpr int kFmaIters = 32768; // FMAs per chain
constexpr int kThreads = 512;
constexpr int kSmemFloats = 8192;   // 32 KiB of shared memory per block
constexpr int kSmemIters = 16384;   // float4 loads per thread

template <class T>
__global__ void __launch_bounds__(kThreads) fma_kernel(T* out, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = static_cast<T>(threadIdx.x + k) * static_cast<T>(1e-3);
  for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Conflict-free 16-byte shared-memory loads: in every load instruction the
// warp's 32 lanes read 32 consecutive float4 (512 bytes).
__global__ void __launch_bounds__(kThreads) smem_kernel(float* out, int salt) {
  __shared__ float4 buf[kSmemFloats / 4];
  for (int i = threadIdx.x; i < kSmemFloats / 4; i += blockDim.x)
    buf[i] = make_float4(i + salt, i - salt, 2.f * i, 0.5f * i);
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int base = (warp * 32) & (kSmemFloats / 4 - 1);
#pragma unroll 4
  for (int it = 0; it < kSmemIters; ++it) {
    const float4 v = buf[(base + lane) & (kSmemFloats / 4 - 1)];
    acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    base += 32 * 5;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc.x + acc.y + acc.z + acc.w;
}

template <class K>
cudaError_t best_ms(K launch, float* best) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    launch();   // warm-up
    e = cudaGetLastError();
  }
  *best = 0.f;
  for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, 0);
    launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (*best == 0.f || ms < *best)) *best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" sfd_status sfd_measure_peaks(int device, double* fp32_tflops, double* fp64_tflops, double* smem_tbs) {
  if (!fp32_tflops || !fp64_tflops || !smem_tbs) return SFD_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  cudaError_t e = cudaSetDevice(device);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  // two blocks of 16 warps per SM: 8 warps per scheduler, 16 chains each
  const int blocks = 2 * sms;
  void* buf = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&buf, sizeof(double) * blocks * kThreads);
  float ms32 = 0.f, ms64 = 0.f, mss = 0.f;
  if (e == cudaSuccess)
    e = best_ms([&] { fma_kernel<float><<<blocks, kThreads>>>(static_cast<float*>(buf), 0.999f, 1e-4f); }, &ms32);
  // FP64 on a quarter of the threads: its pipe is far narrower than FP32's
  if (e == cudaSuccess)
    e = best_ms([&] { fma_kernel<double><<<blocks / 2, kThreads / 4>>>(static_cast<double*>(buf), 0.999, 1e-4); },
                &ms64);
  if (e == cudaSuccess)
    e = best_ms([&] { smem_kernel<<<4 * sms, kThreads>>>(static_cast<float*>(buf), 3); }, &mss);
  if (buf) cudaFree(buf);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess || ms32 <= 0.f || ms64 <= 0.f || mss <= 0.f) return SFD_ECUDA;
  const double f32 = 2.0 * kChains * static_cast<double>(kFmaIters) * kThreads * blocks;
  const double f64 = 2.0 * kChains * static_cast<double>(kFmaIters) * (kThreads / 4) * (blocks / 2);
  const double sb = 16.0 * kSmemIters * static_cast<double>(kThreads) * 4 * sms;
  *fp32_tflops = f32 / (ms32 * 1e-3) / 1e12;
  *fp64_tflops = f64 / (ms64 * 1e-3) / 1e12;
  *smem_tbs = sb / (mss * 1e-3) / 1e12;
  return SFD_OK;
}
