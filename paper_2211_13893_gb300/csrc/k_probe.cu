// Arithmetic throughput probe (msgfem_probe_fma): the rate of dependent-chain
// FMA loops in FP64 or FP32 over every SM, the measured counterpart of the
// ALU peaks that bound the factorisation (FP64 DFMA in the plain path, FP32
// FFMA in the mixed path).  Not part of the method.
#include "internal.h"

namespace {

constexpr int PROBE_CHAINS = 8;     // independent FMA chains per thread
constexpr int PROBE_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(int iters, T seed, T* out) {
  T a[PROBE_CHAINS];
  const T m = seed * (T)1e-3 + (T)0.999, c = (T)1e-7;
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = seed + (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = fma(a[i], m, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i];
  if (s == (T)-1.2345) out[blockIdx.x] = s;   // never true; keeps the loop alive
}

template <typename T>
cudaError_t run_probe(int blocks, int iters, T* out, float* ms) {
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&b);
  if (e != cudaSuccess) { cudaEventDestroy(a); return e; }
  k_fma_probe<T><<<blocks, PROBE_THREADS>>>(iters, (T)1, out);   // warm-up (clocks ramp up)
  *ms = 0.0f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {   // best of three
    cudaEventRecord(a);
    k_fma_probe<T><<<blocks, PROBE_THREADS>>>(iters, (T)1, out);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (e == cudaSuccess && (*ms == 0.0f || t < *ms)) *ms = t;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  g_launch_count += 4;
  return e;
}

}  // namespace

extern "C" msgfem_status msgfem_probe_fma(int precision, double* tflops, double* sm_count_out) {
  if (!tflops || (precision != MSGFEM_FP64 && precision != MSGFEM_MIXED)) return MSGFEM_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MSGFEM_ECUDA;
  const int blocks = sms * 8;                 // 8 resident CTAs of 256 threads per SM
  const int iters = precision == MSGFEM_FP64 ? 4096 : 131072;   // ~0.2 s (FP64), ~0.1 s (FP32) per launch
  void* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * sizeof(double)) != cudaSuccess) return MSGFEM_ENOMEM;
  float ms = 0.0f;
  const cudaError_t e = precision == MSGFEM_FP64 ? run_probe<double>(blocks, iters, (double*)out, &ms)
                                                 : run_probe<float>(blocks, iters, (float*)out, &ms);
  cudaFree(out);
  if (e != cudaSuccess || !(ms > 0.0f)) return MSGFEM_ECUDA;
  const double flops = 2.0 * PROBE_CHAINS * 16.0 * (double)iters * (double)blocks * PROBE_THREADS;
  *tflops = flops / (ms * 1e-3) / 1e12;
  if (sm_count_out) *sm_count_out = sms;
  return MSGFEM_OK;
}
