// batch.cuh -- persistent kernel that advances many independent lattices.
//
// One cooperative launch runs all steps.  Each step the blocks sweep a tile
// list covering every lattice (tile = one block's rows x warp-aligned columns of
// one lattice, one node per thread, so any extent works), then meet at a grid
// barrier before the next step reads what the previous one wrote.  Loads use the
// L2-only path (ld.global.cg) because other SMs of the same launch wrote the
// data and L1 is not coherent.  The barrier is a bounded wait on %globaltimer:
// when the limit runs out the kernel records an error word and every block
// returns, so a missing arrival can never hang the GPU.
#pragma once
#include "dispatch.h"
#include "kernels.cuh"

namespace lbm {

struct BarrierWords {
  unsigned int count;  // arrivals in the current generation
  unsigned int gen;    // generation, bumped by the last arrival
  int err;             // 1: a wait ran out of time
  int pad;
};

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded grid-wide barrier.  Returns false (in every thread of the block) when
// this block's wait ran out or another block reported a timeout.
__device__ __forceinline__ bool grid_sync(BarrierWords* b, unsigned int expected,
                                          long long timeout_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    ok = 1;
    volatile unsigned int* vgen = &b->gen;
    volatile int* verr = &b->err;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&b->count, 1u) + 1u;
    if (arrived == expected) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const long long t0 = global_ns();
      while (*vgen == g) {
        if (*verr) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > timeout_ns) {
          atomicExch(&b->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(200);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <class L, int COLL, class S>
__global__ void __launch_bounds__(256)
    k_batch(const BatchDesc* __restrict__ desc, const BatchTile* __restrict__ tiles, int ntiles,
            char* A, char* B, int nsteps, int parity0, unsigned int step0, unsigned int* flags,
            BarrierWords* bar, unsigned int expected, long long timeout_ns) {
  using R = typename S::R;
  const int lane = threadIdx.x & 31;
  for (int s = 0; s < nsteps; ++s) {
    char* src = ((parity0 + s) & 1) ? B : A;
    char* dst = ((parity0 + s) & 1) ? A : B;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const BatchTile tl = tiles[t];
      const BatchDesc& d = desc[tl.lat];
      StepArgs<R> a;
      a.g.nx = d.g.nx;
      a.g.ny = d.g.ny;
      a.g.nz = d.g.nz;
      a.g.pitch = d.g.pitch;
      a.g.plane = d.g.plane;
      for (int k = 0; k < 3; ++k) a.g.per[k] = d.g.per[k];
      if constexpr (sizeof(R) == sizeof(double)) {
        a.c = d.cd;
      } else {
        a.c = d.cf;
      }
      a.src = src + d.off;
      a.dst = dst + d.off;
      a.mask = nullptr;
      a.flag = flags + tl.lat;
      a.step = step0 + (unsigned int)s;
      const int y = tl.y0 + threadIdx.y;
      if (y < a.g.ny) update_chunk<L, COLL, S, 1, false, LD_CG>(a, tl.x0 + threadIdx.x, y, tl.z, lane);
    }
    if (s + 1 < nsteps && !grid_sync(bar, expected, timeout_ns)) return;
  }
}

}  // namespace lbm
