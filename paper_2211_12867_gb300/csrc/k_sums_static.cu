// Conservation sums that use no caller-provided or allocated scratch.
//
// Some programs that drive this library cannot allocate device memory once
// they are running: a host framework that hands every byte of the GPU to its
// own pool at start-up (so the footprint never grows and never fragments), or
// a service that must not stall on an allocation in the middle of a run.
// icarus_conservation_sums_static gives them the per-member sums of V * U
// without any allocation: its scratch is a fixed array in this file's device
// memory, kept on the device until the process exits.
//
// When the array comes into being: with CUDA's lazy module loading (the
// default) this file's module, with the array and its kernels, is loaded on a
// device the first time something in it is used.  icarus_init_grid does that
// on purpose (static_sums_prepare below, with the context's device current):
// it looks up the array's address, forces this file's kernels to load and caches
// the address per device.  So the array is in place once a context exists, and
// a caller that afterwards gives the rest of the GPU to its own pool can still
// call this entry point.
//
// Limits and rules, for users:
//   * at most ICARUS_STATIC_SUM_BLOCKS leaves per member; larger members are
//     rejected with ICARUS_ERR_CAPACITY and a message on stderr;
//   * the address is taken while the context is created; create contexts
//     before any stream capture begins;
//   * every call, on every context and stream, shares the one array: calls
//     that overlap on the GPU race and may return each other's sums.  Each call
//     overwrites every scratch entry it reads, so no clearing is needed, and
//     the array keeps the last call's partial sums afterwards.
//   * a cudaDeviceReset destroys the array with the rest of the device's
//     memory, and with it every context's arena: contexts do not outlive it.
// The result equals icarus_conservation_sums: the same per-block partial sums
// added in the same order, in FP64.
#include <cstdio>

#include "../../include/icarus.h"
#include "icarus_internal.h"

#define ICARUS_STATIC_SUM_BLOCKS 16384
#define ICARUS_MAX_DEVICES 64

namespace {

// [block][v] partial sums, then the 8 totals
__device__ __align__(256) double g_sum_scratch[(ICARUS_STATIC_SUM_BLOCKS + 1) * NVAR];

double *g_scratch_addr[ICARUS_MAX_DEVICES] = {nullptr};

template <typename real>
__global__ void k_block_sums_static(const KParams kp, const real *U, int slot0, double *partial) {
  __shared__ double sh[NVAR][256];
  const int slot = slot0 + blockIdx.x;
  const DevBlock B = kp.blk[slot];
  const LevelGeo<double> &GD = kp.geo->d[B.level];
  double acc[NVAR];
  for (int v = 0; v < NVAR; v++) acc[v] = 0.0;
  for (int c = threadIdx.x; c < kp.icells; c += blockDim.x) {
    const int k = c % kp.nb[2], j = (c / kp.nb[2]) % kp.nb[1], i = c / (kp.nb[2] * kp.nb[1]);
    const int I = B.ix[0] * kp.nb[0] + i + NGH, J = B.ix[1] * kp.nb[1] + j + NGH;
    const double V = GD.dr3[I] * GD.dcos[J] * GD.dphi;
    for (int v = 0; v < NVAR; v++) {
      const size_t idx = ((((size_t)slot * kp.nvs + v) * kp.P[0] + i + NGH) * kp.P[1] + j + NGH) * kp.P[2] + k + NGH;
      acc[v] += V * (double)U[idx];
    }
  }
  for (int v = 0; v < NVAR; v++) sh[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int v = 0; v < NVAR; v++) sh[v][threadIdx.x] += sh[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < NVAR) partial[(size_t)blockIdx.x * NVAR + threadIdx.x] = sh[threadIdx.x][0];
}

// totals in block order (one thread per variable), written after the partials
__global__ void k_total_static(const double *partial, int nblocks, double *total) {
  const int v = threadIdx.x;
  if (v >= NVAR) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; b++) s += partial[(size_t)b * NVAR + v];
  total[v] = s;
}

}  // namespace

// Look up the scratch array's device address on device `dev` (which must be
// the current device) and load this file's kernels there; cached per device.
// Called by icarus_init_grid.  Returns 0 on success.
int static_sums_prepare(int dev) {
  if (dev < 0 || dev >= ICARUS_MAX_DEVICES) return -1;
  if (g_scratch_addr[dev]) return 0;
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_sum_scratch);
  if (e != cudaSuccess || !p) {
    fprintf(stderr, "libicarus: cudaGetSymbolAddress of the static sum scratch failed: %s\n", cudaGetErrorString(e));
    return -1;
  }
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_block_sums_static<float>) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_block_sums_static<double>) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_total_static) != cudaSuccess)
    return -1;
  g_scratch_addr[dev] = static_cast<double *>(p);
  return 0;
}

extern "C" icarus_status icarus_conservation_sums_static(icarus_ctx *ctx, int member, double *out8) {
  if (!ctx || !out8) return ICARUS_ERR_ARG;
  KParams kp;
  const void *U = nullptr;
  int prec = 0, slot0 = 0, nl = 0;
  cudaStream_t s = nullptr;
  if (ctx_member_view(ctx, member, &kp, &U, &prec, &slot0, &nl, &s) != 0) return ICARUS_ERR_ARG;
  if (nl > ICARUS_STATIC_SUM_BLOCKS) {
    fprintf(stderr,
            "libicarus: icarus_conservation_sums_static supports at most %d leaves per member (member %d has %d); "
            "use icarus_conservation_sums\n",
            ICARUS_STATIC_SUM_BLOCKS, member, nl);
    return ICARUS_ERR_CAPACITY;
  }
  // the address was taken on the context's device when it was created
  const int dev = ctx_device(ctx);
  if (dev < 0 || dev >= ICARUS_MAX_DEVICES || !g_scratch_addr[dev]) return ICARUS_ERR_STATE;
  double *partial = g_scratch_addr[dev];
  double *total = partial + (size_t)ICARUS_STATIC_SUM_BLOCKS * NVAR;
  if (nl > 0) {
    if (prec)
      k_block_sums_static<float><<<nl, 256, 0, s>>>(kp, static_cast<const float *>(U), slot0, partial);
    else
      k_block_sums_static<double><<<nl, 256, 0, s>>>(kp, static_cast<const double *>(U), slot0, partial);
  }
  k_total_static<<<1, 32, 0, s>>>(partial, nl, total);
  if (cudaPeekAtLastError() != cudaSuccess) return ICARUS_ERR_CUDA;
  if (cudaMemcpyAsync(out8, total, NVAR * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return ICARUS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return ICARUS_ERR_CUDA;
  return ICARUS_OK;
}
