// Measured arithmetic peaks of the device for the rooflines of the stage
// kernel: fused multiply-add throughput of FP32 (scalar and packed pairs) and
// FP64 on the CUDA cores.  Every thread runs eight independent FMA chains
// (enough independent work to hide the pipeline latency); the grid fills every
// SM several times over.  Results go to a file-scope device word that the
// host never reads (it keeps the chains from being optimised away).
#include <cstdio>

#include "../../include/icarus.h"
#include "icarus_internal.h"

namespace {

__device__ double g_peak_sink;

template <typename real>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, real b, real c) {
  real a[8];
#pragma unroll
  for (int k = 0; k < 8; k++) a[k] = real(threadIdx.x) * real(1e-3) + real(k);
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = fma(a[k], b, c);
  real s = real(0);
#pragma unroll
  for (int k = 0; k < 8; k++) s += a[k];
  if (s == real(-1.2345e30)) g_peak_sink = (double)s;
}

// packed pairs: four float2 chains (eight lanes of work per thread)
__global__ void __launch_bounds__(256) k_fma2_chains(int iters, float b, float c) {
  float2 a[4];
#pragma unroll
  for (int k = 0; k < 4; k++) a[k] = make_float2(threadIdx.x * 1e-3f + k, threadIdx.x * 2e-3f + k);
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int k = 0; k < 4; k++) a[k] = __ffma2_rn(a[k], bb, cc);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 4; k++) s += a[k].x + a[k].y;
  if (s == -1.2345e30f) g_peak_sink = (double)s;
}

}  // namespace

extern "C" icarus_status icarus_alu_peak(int kind, void *stream, double *flops_per_s) {
  if (!flops_per_s || kind < 0 || kind > 2) return ICARUS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ICARUS_ERR_CUDA;
  const int blocks = nsm * 8, threads = 256;
  const int iters = kind == 0 ? 4096 : 65536;   // FP64 runs far fewer FMAs per second
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return ICARUS_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ICARUS_ERR_CUDA;
  }
  auto launch = [&]() {
    if (kind == 0) k_fma_chains<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7);
    else if (kind == 1) k_fma_chains<float><<<blocks, threads, 0, s>>>(iters, 0.9999f, 1e-4f);
    else k_fma2_chains<<<blocks, threads, 0, s>>>(iters, 0.9999f, 1e-4f);
  };
  launch();   // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; r++) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 0.f && ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || !(best < 1e30f)) return ICARUS_ERR_CUDA;
  // two flops per FMA, eight chains per thread
  *flops_per_s = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3);
  return ICARUS_OK;
}
