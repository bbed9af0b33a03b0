// diag.cu -- the FP64 velocity-error reduction over macroscopic fields, the
// fixed-order reduction of block partials (shared with the diagnostics passes
// of each lattice/storage unit) and the streaming copy kernel used as the
// measured bandwidth ceiling.
//
// The reductions are deterministic: a fixed grid of blocks accumulates nodes in
// grid-stride order, reduces warp by warp with shuffles (fixed tree) and writes
// one partial per block; a single block then sums the partials in a fixed order.
// Repeated calls on the same state therefore give bit-identical results.
#include <math.h>

#include "dispatch.h"

namespace lbm {

constexpr int DIAG_THREADS = 256;
constexpr int NVAL = 8;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of NVAL values into partials[blockIdx.x][*].
__device__ __forceinline__ void block_store(double (&acc)[NVAL], double* partials) {
  __shared__ double sh[DIAG_THREADS / 32][NVAL];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NVAL; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < NVAL) {
    double s = 0.0;
    for (int w = 0; w < DIAG_THREADS / 32; ++w) s += sh[w][threadIdx.x];
    partials[blockIdx.x * NVAL + threadIdx.x] = s;
  }
}

// Sums of |u - u_ref|^2 and |u_ref|^2 over fluid nodes.
__global__ void __launch_bounds__(DIAG_THREADS)
    k_diag_l2(GeoH G, int D, const double* u, const double* uref, const uint8_t* mask,
              double* partials) {
  const long long N = (long long)G.nx * G.ny * G.nz;
  double acc[NVAL] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    if (mask && mask[n]) continue;
    for (int a = 0; a < D; ++a) {
      const double d = u[a * N + n] - uref[a * N + n];
      acc[0] += d * d;
      acc[1] += uref[a * N + n] * uref[a * N + n];
    }
  }
  block_store(acc, partials);
}

// out[k] = sum over blocks of partials[b][k] in block order; the flag slot (6)
// takes the maximum.
__global__ void __launch_bounds__(DIAG_THREADS)
    k_reduce_partials(const double* partials, int blocks, double* out) {
  __shared__ double sh[DIAG_THREADS];
  for (int k = 0; k < NVAL; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < blocks; b += blockDim.x) {
      const double v = partials[b * NVAL + k];
      s = (k == 6) ? fmax(s, v) : s + v;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o)
        sh[threadIdx.x] = (k == 6) ? fmax(sh[threadIdx.x], sh[threadIdx.x + o])
                                   : sh[threadIdx.x] + sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
    __syncthreads();
  }
}

cudaError_t reduce_partials(const double* partials, int blocks, double* out, cudaStream_t st) {
  k_reduce_partials<<<1, DIAG_THREADS, 0, st>>>(partials, blocks, out);
  return cudaGetLastError();
}

cudaError_t diag_l2(const DiagLaunch& d) {
  k_diag_l2<<<d.blocks, DIAG_THREADS, 0, d.stream>>>(d.g, d.D, d.u, d.uref, d.mask, d.partials);
  k_reduce_partials<<<1, DIAG_THREADS, 0, d.stream>>>(d.partials, d.blocks, d.out);
  return cudaGetLastError();
}

// Grid-stride 128-bit copy: the same load/store pattern as a plane of the
// fused update without the collision, i.e. the practical bandwidth ceiling.
__global__ void __launch_bounds__(256) k_copy(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                              long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    dst[k] = __ldg(src + k);
}

cudaError_t copy_ceiling(const void* src, void* dst, size_t bytes, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long n = (long long)(bytes / 16);
  long long blocks = (n + 255) / 256;
  const long long cap = (long long)sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_copy<<<(unsigned)blocks, 256, 0, st>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst), n);
  return cudaGetLastError();
}

}  // namespace lbm
