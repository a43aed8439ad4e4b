// Measurement: the fused multiply-add rate of this GPU's FP64 and FP32 pipes.
//
// The roofline fractions of the integral kernels are taken against these rates.  Every thread of a
// grid that fills each SM runs eight independent multiply-add chains (so neither the FMA latency nor
// the issue of one warp limits the pipe); the operands stay near 1 so no chain overflows or becomes
// subnormal, and each thread stores its sum so the compiler keeps every chain.
#include <cuda_runtime.h>

#include <string>

#include "shgo_internal.h"

namespace shgo {
void set_last_error(const std::string& msg);  // shgo_api.cpp
}

namespace {

constexpr int kUnroll = 4;
constexpr int kThreads = 256;

template <typename T, int CHAINS>
__global__ void __launch_bounds__(kThreads) k_fma_rate(int64_t iters, T m, T c, T* __restrict__ sink) {
  T a[CHAINS];
#pragma unroll
  for (int i = 0; i < CHAINS; ++i) a[i] = T(1) + T(i) * T(1e-3) + T(threadIdx.x) * T(1e-6);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < CHAINS; ++i) a[i] = fma(a[i], m, c);
    }
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < CHAINS; ++i) s += a[i];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, int CHAINS>
shgo_status run(int64_t iters, int threads_per_sm, cudaStream_t stream, double* flops_per_s, double* ms_out,
                std::string* err) {
  constexpr int kChains = CHAINS;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  const int blocks = nsm * (threads_per_sm / kThreads);  // threads_per_sm threads on every SM
  T* sink = nullptr;
  e = cudaMallocAsync(&sink, sizeof(T) * (size_t)blocks * kThreads, stream);
  if (e != cudaSuccess) {
    *err = std::string("sink: ") + cudaGetErrorString(e);
    return SHGO_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const T m = T(0.9999999), c = T(1e-7);
  // one short warm-up launch (clocks up, code loaded), then the timed launch
  if (e == cudaSuccess) {
    k_fma_rate<T, CHAINS><<<blocks, kThreads, 0, stream>>>(iters / 16 + 1, m, c, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
  if (e == cudaSuccess) {
    k_fma_rate<T, CHAINS><<<blocks, kThreads, 0, stream>>>(iters, m, c, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(sink, stream);
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return SHGO_ERR_CUDA;
  }
  const double fmas = (double)blocks * kThreads * (double)iters * kUnroll * kChains;
  *ms_out = ms;
  *flops_per_s = 2.0 * fmas / (ms * 1e-3);
  return SHGO_OK;
}

}  // namespace

template <typename T>
shgo_status run_chains(int chains, int64_t iters, int threads_per_sm, cudaStream_t stream, double* rate, double* ms,
                       std::string* err) {
  switch (chains) {
    case 4: return run<T, 4>(iters, threads_per_sm, stream, rate, ms, err);
    case 8: return run<T, 8>(iters, threads_per_sm, stream, rate, ms, err);
    default: return run<T, 16>(iters, threads_per_sm, stream, rate, ms, err);
  }
}

extern "C" shgo_status shgo_measure_fma_rate_shape(int32_t precision, int64_t iters, int32_t chains,
                                                   int32_t threads_per_sm, void* stream, double* flops_per_s,
                                                   double* ms) {
  shgo::set_last_error("");
  if (!flops_per_s || !ms || iters <= 0 || iters > (int64_t)1 << 32 || (chains != 4 && chains != 8 && chains != 16) ||
      threads_per_sm < kThreads || threads_per_sm > 2048 || threads_per_sm % kThreads) {
    shgo::set_last_error("shgo_measure_fma_rate_shape: NULL output, iters outside 1..2^32, chains not 4/8/16 or "
                         "threads per SM not a multiple of 256 in 256..2048");
    return SHGO_ERR_INVALID_ARG;
  }
  std::string err;
  shgo_status st;
  if (precision == SHGO_PREC_FP64)
    st = run_chains<double>(chains, iters, threads_per_sm, (cudaStream_t)stream, flops_per_s, ms, &err);
  else if (precision == SHGO_PREC_FP32_BULK || precision == SHGO_PREC_FP32_PLAIN)
    st = run_chains<float>(chains, iters, threads_per_sm, (cudaStream_t)stream, flops_per_s, ms, &err);
  else {
    shgo::set_last_error("shgo_measure_fma_rate_shape: unknown precision");
    return SHGO_ERR_INVALID_ARG;
  }
  if (st != SHGO_OK) shgo::set_last_error("shgo_measure_fma_rate_shape: " + err);
  return st;
}

extern "C" shgo_status shgo_measure_fma_rate(int32_t precision, int64_t iters, void* stream, double* flops_per_s,
                                             double* ms) {
  const shgo_status st = shgo_measure_fma_rate_shape(precision, iters, 8, 2048, stream, flops_per_s, ms);
  if (st != SHGO_OK) {
    const std::string m = shgo_last_error();
    shgo::set_last_error("shgo_measure_fma_rate" + m.substr(m.find(':')));
  }
  return st;
}
