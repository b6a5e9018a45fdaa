// Arithmetic throughput probe: the FP32 and FP64 fused multiply-add rate of
// the GPU this library runs on, measured with the library's own kernel.  The
// real-space pair sum and the FP64 operator are bound by these rates, so
// their rooflines are reported against the measured figure instead of a
// nominal one.  Not part of the method.
#include "fsd_internal.cuh"

#include <algorithm>

namespace fsd {
namespace {

constexpr int kChains = 8;    // independent FMA chains per thread
constexpr int kUnroll = 16;   // FMAs per chain per loop trip

// Every thread runs kChains independent chains a <- a * m + c; the sum is
// stored only when it equals an impossible value, which keeps the work alive
// without memory traffic.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(int iters, T m, T c, T *sink) {
  T a[kChains];
#pragma unroll
  for (int u = 0; u < kChains; ++u) a[u] = (T)(threadIdx.x + u) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kUnroll; ++k)
#pragma unroll
      for (int u = 0; u < kChains; ++u) a[u] = fma(a[u], m, c);
  }
  T s = 0;
#pragma unroll
  for (int u = 0; u < kChains; ++u) s += a[u];
  if (s == (T)-12345.678) sink[0] = s;
}

template <typename T>
double fma_rate(int iters, cudaStream_t st) {
  int dev = 0, sms = 0;
  FSD_CUDA(cudaGetDevice(&dev));
  FSD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DBuf<T> sink;
  sink.alloc(1);
  const int blocks = 8 * sms, threads = 256;
  cudaEvent_t e0, e1;
  FSD_CUDA(cudaEventCreate(&e0));
  FSD_CUDA(cudaEventCreate(&e1));
  const T m = (T)0.9999999, c = (T)1e-7;
  k_fma_chain<T><<<blocks, threads, 0, st>>>(iters / 8 + 1, m, c, sink.p);  // warm-up
  FSD_CUDA(cudaGetLastError());
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    FSD_CUDA(cudaEventRecord(e0, st));
    k_fma_chain<T><<<blocks, threads, 0, st>>>(iters, m, c, sink.p);
    FSD_CUDA(cudaEventRecord(e1, st));
    FSD_CUDA(cudaEventSynchronize(e1));
    FSD_CUDA(cudaGetLastError());
    float ms = 0.f;
    FSD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double fmas = (double)blocks * threads * iters * kUnroll * kChains;
  return 2.0 * fmas / (best * 1e-3);
}

}  // namespace
}  // namespace fsd

extern "C" fsd_status fsd_fma_throughput(int fp_bits, double *flop_per_s, void *cuda_stream) {
  using namespace fsd;
  if (!flop_per_s || (fp_bits != 32 && fp_bits != 64)) return FSD_EINVAL;
  try {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    *flop_per_s = fp_bits == 32 ? fma_rate<float>(2048, st) : fma_rate<double>(64, st);
  } catch (const CudaError &) {
    return FSD_ECUDA;
  }
  return FSD_OK;
}
