// Arithmetic peak probe (instrumentation for the roofline of the FP64- and
// FP32-pipe-bound kernels; the paper has no counterpart): every thread of a
// grid of 8 CTAs per SM runs 8 independent FMA chains, and the rate is taken
// from CUDA events around the launch.
#include <string>

#include "tpp_internal.cuh"

namespace tpp {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T* out, int iters, T a, T b) {
  T v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fma(v[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += v[k];
  if (s < (T)0) out[blockIdx.x] = s;     // keeps the chains live; never true (all v > 0)
}

template <typename T>
tpp_status probe(int iters, double* flops, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_check(e, "probe device");
  const int blocks = 8 * sms, threads = 256;
  T* sink = nullptr;   // never written: the chains stay positive
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_check(e, "event");
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_check(e, "event");
  }
  k_fma_chain<T><<<blocks, threads, 0, s>>>(sink, iters / 8, (T)0.999999, (T)1e-7);   // warm-up
  cudaEventRecord(e0, s);
  k_fma_chain<T><<<blocks, threads, 0, s>>>(sink, iters, (T)0.999999, (T)1e-7);
  cudaEventRecord(e1, s);
  count_launch(2);
  e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_check(e, "probe timing");
  *flops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
  return TPP_OK;
}

}  // namespace
}  // namespace tpp

extern "C" tpp_status tpp_probe_fma_rate(int32_t prec, int32_t iters, double* flops,
                                         void* stream) {
  if (!flops || iters < 1 || (prec != TPP_FP64 && prec != TPP_FP32)) {
    tpp::set_error("tpp_probe_fma_rate: prec TPP_FP64 or TPP_FP32, iters >= 1, flops non-NULL");
    return TPP_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return prec == TPP_FP64 ? tpp::probe<double>(iters, flops, s)
                          : tpp::probe<float>(iters, flops, s);
}
