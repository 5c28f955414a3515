// Measured FMA throughput of the current device: the roofline the matvec is held against.
// The matvec does one complex multiply-add (4 real FMA) per nonzero of H per state, so its
// ceiling is the FP32 (complex64) or FP64 (complex128) FMA rate, not HBM.  The kernel runs
// CH independent FMA chains per thread (enough to hide the pipe latency) on 4 blocks of 256
// threads per SM; the result is stored only under a condition the chains never meet, so the
// work cannot be dropped.
#include <cuda_runtime.h>

#include "syk_internal.h"

namespace syk {
namespace {

constexpr int kChains = 8;
__device__ double g_fma_sink[256];  // written only if the chains ever sum to -12345
constexpr int kUnroll = 16;

template <typename R>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, R a, R b) {
  R x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = R(threadIdx.x + c) * R(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  R s = R(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == R(-12345.0)) g_fma_sink[threadIdx.x] = double(s);  // never true for the chains' values
}

template <typename R>
int run(int iters, double* tflops, double* ms_out, cudaStream_t st) {
  const int sms = sm_count();
  const int blocks = 4 * sms, threads = 256;
  cudaEvent_t e0, e1;
  SYK_CUDA_CHECK(cudaEventCreate(&e0));
  SYK_CUDA_CHECK(cudaEventCreate(&e1));
  // x -> a x + b with |a| < 1 converges to b / (1 - a): bounded values, no overflow
  const R a = R(0.999), b = R(1e-4);
  k_fma_chains<R><<<blocks, threads, 0, st>>>(iters / 8 + 1, a, b);  // warm-up (clocks, module load)
  cudaEventRecord(e0, st);
  k_fma_chains<R><<<blocks, threads, 0, st>>>(iters, a, b);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    set_error("syk_fma_peak: %s", cudaGetErrorString(e));
    return SYK_ECUDA;
  }
  const double fmas = double(blocks) * threads * double(iters) * kUnroll * kChains;
  if (tflops) *tflops = 2.0 * fmas / (double(ms) * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return SYK_OK;
}

}  // namespace
}  // namespace syk

extern "C" int syk_fma_peak(int bits, int iters, double* tflops, int* sms, double* ms, void* stream) {
  syk::clear_error();
  if ((bits != 32 && bits != 64) || iters < 1 || iters > (1 << 24)) {
    syk::set_error("syk_fma_peak: bits must be 32 or 64 and 1 <= iters <= 2^24 (got %d, %d)", bits, iters);
    return SYK_EINVAL;
  }
  if (sms) *sms = syk::sm_count();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return bits == 32 ? syk::run<float>(iters, tflops, ms, st) : syk::run<double>(iters, tflops, ms, st);
}
