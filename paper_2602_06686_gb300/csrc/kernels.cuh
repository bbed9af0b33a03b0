// kernels.cuh -- argument blocks, the pull gather and the fused stream-collide
// kernels shared by the per-(lattice, storage) translation units.
//
// Storage layout in HBM (structure of arrays): population plane i holds
// df_i = f_i - w_i rho0 for all nodes as [z][y][x] rows of `pitch` elements
// (pitch = nx rounded up to 16 bytes); planes are `plane` elements apart
// (a multiple of 256 bytes).  A/B layout: the buffer read at step t holds the
// post-collision state f*(., t-1); the kernel gathers f_i(x, t) = f*_i(x - e_i)
// (pull streaming, Sec. 2.1 / Eq. TRT-RLB left-hand side), collides and writes
// f*(x, t) to the other buffer at x, so every write is aligned and coalesced and
// only reads are shifted by one element in x.
//
// Thread mapping: a warp covers 32 consecutive chunks of NV nodes along x of
// one row; x-shifted planes are read as aligned NV-element vectors and shifted
// by one element with a warp shuffle; only the first / last lane of a warp
// fetches its outside neighbour with a scalar load (an L1 hit).  Rows shifted in
// y/z are simply other rows (each element is read exactly once per step, so
// there is no reuse for shared-memory staging to capture).
//
// Halfway bounce-back (Sec. 3.3): when x - e_i is solid or outside a
// non-periodic axis, f_i(x, t) = f*_ibar(x, t-1), read from the node's own slot.
#pragma once
#include <stdint.h>

#include "collide_v.cuh"
#include "lattice.cuh"
#include "storage.cuh"

namespace lbm {

struct Geo {
  int nx, ny, nz;
  int pitch;           // elements per row
  long long plane;     // elements per population plane
  int per[3];          // periodic flags
};

template <typename R>
struct StepArgs {
  Geo g;
  CoefV<R> c;
  const void* src;
  void* dst;
  const uint8_t* mask;  // [nz][ny][nx] or null
  unsigned int* flag;   // divergence: earliest step index seen (atomicMin; 0xffffffff = none)
  unsigned int step;    // index of the step being computed
};

__device__ __forceinline__ unsigned lane_id() {
  unsigned l;
  asm("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}

// Records `step` as a divergence step: one atomic per warp, and none once the
// flag already holds an earlier (or equal) step.
__device__ __forceinline__ void record_bad(unsigned int* flag, unsigned int step, bool bad) {
  const unsigned m = __activemask();
  const unsigned b = __ballot_sync(m, bad);
  if (b != 0u && lane_id() == (unsigned)(__ffs(b) - 1)) {
    if (*reinterpret_cast<volatile unsigned int*>(flag) > step) atomicMin(flag, step);
  }
}

template <typename R>
__device__ __forceinline__ R shfl_up1(R v) {
  return __shfl_up_sync(0xffffffffu, v, 1);
}
template <typename R>
__device__ __forceinline__ R shfl_down1(R v) {
  return __shfl_down_sync(0xffffffffu, v, 1);
}

// Pre-collision populations of the NV nodes [x0, x0 + NV) of row (y, z).
// Must be called by all 32 lanes of a warp (shuffles); `active` lanes load.
template <class L, class S, int NV, bool MASK, int LD = LD_NC>
__device__ __forceinline__ void gather(const Geo& G, const typename S::T* __restrict__ src,
                                       const uint8_t* __restrict__ mask, int x0, int y, int z,
                                       int lane, bool active, typename S::R (&f)[L::Q][NV]) {
  using T = typename S::T;
  using R = typename S::R;
  const long long own_row = ((long long)z * G.ny + y) * G.pitch;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int ex = L::cx(i), ey = L::cy(i), ez = L::cz(i);
    const T* opp_own = src + L::opp(i) * G.plane + own_row;  // bounce-back source row
    int ys = y - ey, zs = z - ez;
    bool wall = false;
    if (ey != 0 && (ys < 0 || ys >= G.ny)) {
      if (G.per[1]) ys = ys < 0 ? ys + G.ny : ys - G.ny;
      else wall = true;
    }
    if (ez != 0 && (zs < 0 || zs >= G.nz)) {
      if (G.per[2]) zs = zs < 0 ? zs + G.nz : zs - G.nz;
      else wall = true;
    }
    if (wall) {  // uniform across the warp: whole row bounces
      if (active) ld_dec<S, NV, LD>(opp_own + x0, f[i]);
      continue;
    }
    const long long srow = ((long long)zs * G.ny + ys) * G.pitch;
    const T* row = src + i * G.plane + srow;
    R v[NV];
    if (active) {
      ld_dec<S, NV, LD>(row + x0, v);
    } else {
#pragma unroll
      for (int k = 0; k < NV; ++k) v[k] = R(0);
    }
    if (ex == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) f[i][k] = v[k];
    } else if (ex == 1) {  // source x - 1
      const R left = shfl_up1(v[NV - 1]);
#pragma unroll
      for (int k = NV - 1; k >= 1; --k) f[i][k] = v[k - 1];
      if (lane > 0) {
        f[i][0] = left;
      } else if (active) {
        const int xs = x0 - 1;
        if (xs >= 0) f[i][0] = ld1<S, LD>(row + xs);
        else if (G.per[0]) f[i][0] = ld1<S, LD>(row + G.nx - 1);
        else f[i][0] = ld1<S, LD>(opp_own + x0);
      }
    } else {  // ex == -1: source x + 1
      const R right = shfl_down1(v[0]);
#pragma unroll
      for (int k = 0; k < NV - 1; ++k) f[i][k] = v[k + 1];
      const int xs = x0 + NV;
      if (active) {
        if (xs < G.nx) f[i][NV - 1] = lane < 31 ? right : ld1<S, LD>(row + xs);
        else if (G.per[0]) f[i][NV - 1] = ld1<S, LD>(row);
        else f[i][NV - 1] = ld1<S, LD>(opp_own + x0 + NV - 1);
      }
    }
    if constexpr (MASK) {
      // halfway bounce-back at solid neighbours: the source node x - e_i is solid
      if (active) {
        const uint8_t* mrow = mask + ((long long)zs * G.ny + ys) * G.nx;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          int xs = x0 + k - ex;
          if (xs < 0 || xs >= G.nx) {
            if (!G.per[0]) continue;  // already bounced at the x wall
            xs = xs < 0 ? xs + G.nx : xs - G.nx;
          }
          if (mrow[xs]) f[i][k] = ld1<S, LD>(opp_own + x0 + k);
        }
      }
    }
  }
}

// One fused update of a tile of rows: gather, collide, store.
template <class L, int COLL, class S, int NV, bool MASK, int LD = LD_NC>
__device__ __forceinline__ void update_chunk(const StepArgs<typename S::R>& a, int x0, int y, int z,
                                             int lane) {
  using T = typename S::T;
  using R = typename S::R;
  const Geo& G = a.g;
  const bool active = x0 < G.nx;
  const T* __restrict__ src = static_cast<const T*>(a.src);
  T* __restrict__ dst = static_cast<T*>(a.dst);
  R f[L::Q][NV];
  gather<L, S, NV, MASK, LD>(G, src, a.mask, x0, y, z, lane, active, f);
  if (!active) return;
  bool anybad = false;
  bool solid[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    solid[k] = false;
    if constexpr (MASK) solid[k] = a.mask[((long long)z * G.ny + y) * G.nx + x0 + k] != 0;
  }
  if constexpr (sizeof(R) == 4 && NV % 2 == 0) {
    // FP32 arithmetic, two nodes at a time with the packed f32x2 instructions
#pragma unroll
    for (int k = 0; k < NV; k += 2) {
      F2 g[L::Q];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) g[i] = F2{f[i][k], f[i][k + 1]};
      const unsigned bad = collide_v<L, COLL, true, F2>(g, a.c);
      anybad |= ((bad & 1u) && !solid[k]) || ((bad & 2u) && !solid[k + 1]);
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        f[i][k] = g[i].x;
        f[i][k + 1] = g[i].y;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      R g[L::Q];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) g[i] = f[i][k];
      const bool bad = collide_v<L, COLL, true, R>(g, a.c) != 0u;
      anybad |= bad && !solid[k];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) f[i][k] = g[i];
    }
  }
  const long long own = ((long long)z * G.ny + y) * G.pitch + x0;
  if constexpr (MASK) {
    bool anysolid = false;
#pragma unroll
    for (int k = 0; k < NV; ++k) anysolid |= solid[k];
    if (anysolid) {  // solid nodes keep their (never read) slots untouched
#pragma unroll
      for (int i = 0; i < L::Q; ++i)
#pragma unroll
        for (int k = 0; k < NV; ++k)
          if (!solid[k]) dst[i * G.plane + own + k] = S::enc(f[i][k]);
      record_bad(a.flag, a.step, anybad);
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < L::Q; ++i) st_enc<S, NV>(dst + i * G.plane + own, f[i]);
  record_bad(a.flag, a.step, anybad);
}

// Grid: x = ceil(nx / (NV * blockDim.x)) chunks-blocks, y = ceil(ny / blockDim.y), z = nz.
template <class L, int COLL, class S, int NV, bool MASK>
__global__ void __launch_bounds__(256) k_step_ab(const StepArgs<typename S::R> a) {
  const int lane = threadIdx.x & 31;
  const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * NV;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= a.g.ny) return;  // whole warps (blockDim.x is a multiple of 32)
  update_chunk<L, COLL, S, NV, MASK>(a, x0, y, z, lane);
}

}  // namespace lbm
