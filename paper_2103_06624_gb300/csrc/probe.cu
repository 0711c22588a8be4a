// Peak-rate probes for the rooflines of the SIMT kernels: FP32 (FFMA) and FP64 (DFMA) throughput
// of this GPU, measured with independent fused multiply-add chains in every thread.
#include <atomic>

#include "bcrown_internal.cuh"

namespace bcrown {

extern std::atomic<long long> g_launches;

namespace {

// Written only when the chains end in a value they cannot reach, so the work is not removed.
__device__ double g_probe_sink;

constexpr int kChains = 8;       // independent FMA chains per thread (hides the FMA latency)
constexpr int kUnroll = 16;

template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-1.2345e30) g_probe_sink = (double)s;
}

}  // namespace
}  // namespace bcrown

using namespace bcrown;

// kind 0: FP32 FFMA, kind 1: FP64 DFMA.  Launches one grid of 8 blocks x 256 threads per SM on
// `stream`, times it with CUDA events (synchronising the stream) and returns TFLOP/s (2 flops
// per FMA).
extern "C" int bcrown_peak_probe(int kind, int iters, double* tflops, void* stream) {
  if ((kind != 0 && kind != 1) || iters < 1 || !tflops) return fail(BCROWN_ERR_ARG, "peak_probe: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  BC_CUDA(cudaGetDevice(&dev));
  BC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  BC_CUDA(cudaEventCreate(&e0));
  BC_CUDA(cudaEventCreate(&e1));
  auto launch = [&](int n) {
    if (kind == 0)
      k_fma_probe<float><<<blocks, threads, 0, s>>>(n, 0.999999f, 1e-7f);
    else
      k_fma_probe<double><<<blocks, threads, 0, s>>>(n, 0.999999999, 1e-12);
    ++g_launches;
  };
  launch(std::max(1, iters / 10));   // warm-up (clocks, instruction cache)
  BC_CUDA(cudaEventRecord(e0, s));
  launch(iters);
  BC_CUDA(cudaEventRecord(e1, s));
  BC_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  BC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BC_CUDA(cudaGetLastError());
  const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * threads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return BCROWN_OK;
}
