// Measurement hook: the arithmetic throughput the FP64 path is bound by.
//
// On this part the FP64 pipe, not HBM, bounds the plain FP64 path (its
// transforms do about 1.1 kflop per voxel per operator application), so its
// roofline fraction is taken against a measured FP64 FMA rate.  The probe
// runs independent FMA chains (eight accumulators per thread, no memory
// traffic in the loop) on every SM and reports FLOP/s (2 per FMA).
#include "../../include/mixfft.h"
#include "launch.h"

namespace {

// sinks of the probe's results (written only if a chain hit an impossible
// value: they keep the compiler from dropping the chains)
__device__ double g_fma_sink64[1];
__device__ float g_fma_sink32[1];
template <typename T> const void* fma_sink();
template <> const void* fma_sink<double>() { return (const void*)&g_fma_sink64; }
template <> const void* fma_sink<float>() { return (const void*)&g_fma_sink32; }

template <typename T>
__global__ void __launch_bounds__(256) k_fma(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)-1.2345e37) out[blockIdx.x] = s;   // keeps the chains live; never true
}

template <typename T>
cudaError_t time_fma(int blocks, int iters, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  T* out = nullptr;
  e = cudaGetSymbolAddress((void**)&out, fma_sink<T>());
  // a, b keep x bounded (|a| < 1)
  if (e == cudaSuccess) { k_fma<T><<<blocks, 256>>>(out, iters, (T)0.999, (T)0.001); e = cudaGetLastError(); }
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
    k_fma<T><<<blocks, 256>>>(out, iters, (T)0.999, (T)0.001);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms /= 3.0f;
  g_mf_launches += 4;
  return e;
}

}  // namespace

extern "C" int mf_probe_fma(int precision, double* tflops_out) {
  if (!tflops_out || (precision != MF_FP64 && precision != MF_FP32_INNER)) return MF_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MF_CUDA_ERROR;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MF_CUDA_ERROR;
  const int blocks = sms * 8;
  const int iters = precision == MF_FP64 ? 4096 : 65536;
  float ms = 0.f;
  const cudaError_t e = precision == MF_FP64 ? time_fma<double>(blocks, iters, &ms) : time_fma<float>(blocks, iters, &ms);
  if (e != cudaSuccess) return MF_CUDA_ERROR;
  const double flops = 2.0 * 8.0 * (double)iters * 256.0 * (double)blocks;
  *tflops_out = flops / (ms * 1e-3) / 1e12;
  return MF_OK;
}

// Self-test of the debug build's bounds checks: one thread evaluates a check
// whose index (7) lies outside its 4-element array; the check records it and
// redirects the write to element 0, inside the array.  Release builds have no
// checks (the index would be used as is), so there the call launches nothing
// and returns MF_INVALID_ARG.
#ifdef MF_DEBUG
namespace {
__device__ int g_dbg_probe[4];
__global__ void k_debug_selftest() { g_dbg_probe[MF_AT(7, 4)] = 1; }
}  // namespace
#endif

extern "C" int mf_debug_selftest(void) {
#ifdef MF_DEBUG
  k_debug_selftest<<<1, 1>>>();
  ++g_mf_launches;
  const cudaError_t e = cudaDeviceSynchronize();
  return e == cudaSuccess ? MF_OK : MF_CUDA_ERROR;
#else
  return MF_INVALID_ARG;
#endif
}
