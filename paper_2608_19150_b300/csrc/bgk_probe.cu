// Measured FMA rate of the current device, the denominator of the ALU roofline of the
// FP64 sweeps (B300 has no FP64 tensor path; its FP64 FMA pipe is a small fraction of the
// FP32 one, so FP64 kernels here are bound by it, not by HBM).
#include <cuda_runtime.h>

#include "bgk.h"

namespace {

// Eight independent FMA chains per thread (enough to cover the pipe latency); the result
// is written only when it takes a value it cannot take, so the chains stay live.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* out, int iters, T a, T b) {
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
  if (s == (T)-12345.0) out[blockIdx.x] = s;
}

template <typename T>
int probe(int iters, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return BGK_E_CUDA;
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = BGK_OK;
  if (cudaMalloc(&out, sizeof(T) * blocks) != cudaSuccess) return BGK_E_OOM;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = BGK_E_CUDA;
  float best = 0.0f;
  // (a, b) keep |x| bounded: x -> 0.999999 x + 1e-6 converges to 1 from below
  const T a = (T)0.999999, b = (T)1e-6;
  for (int rep = 0; rc == BGK_OK && rep < 4; ++rep) {
    cudaEventRecord(e0, st);
    k_fma_probe<T><<<blocks, threads, 0, st>>>(out, iters, a, b);
    cudaEventRecord(e1, st);
    float ms = 0.0f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      rc = BGK_E_CUDA;
    else if (rep > 0 && (best == 0.0f || ms < best))
      best = ms;  // the first launch is a warm-up
  }
  if (rc == BGK_OK && best > 0.0f)
    *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
  else if (rc == BGK_OK)
    rc = BGK_E_CUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  return rc;
}

}  // namespace

extern "C" int bgk_probe_fma_tflops(int dtype, double* tflops) {
  if (!tflops || (dtype != BGK_DTYPE_F64 && dtype != BGK_DTYPE_F32)) return BGK_E_INVALID;
  return dtype == BGK_DTYPE_F64 ? probe<double>(1 << 12, tflops) : probe<float>(1 << 16, tflops);
}
