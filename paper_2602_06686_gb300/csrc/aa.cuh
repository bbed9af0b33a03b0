// aa.cuh -- AA-pattern in-place update (one population buffer).
//
// With an even number of completed steps the buffer holds f_i(x, t) in its
// natural slot (i, x).  Even step: every node reads its own Q slots, collides
// and writes f*_i(x) back into the opposite slot (ibar, x).  After it, f_i(x,t+1)
// = f*_i(x - e_i) sits in slot (ibar, x - e_i), or -- halfway bounce-back when
// x - e_i is solid or beyond a non-periodic edge -- f*_ibar(x) in slot (i, x).
// Odd step: every node gathers from those slots, collides and writes f*_i(x) to
// the natural slot (i, x + e_i) of its downstream neighbour, or to (ibar, x)
// when x + e_i is solid / outside, restoring natural order.  In both steps each
// node reads and writes exactly the same set of slots, so the update is race
// free in place.  One node per thread (x-shifted loads and stores are merged in
// L1/L2).
#pragma once
#include "kernels.cuh"

namespace lbm {

// One element through the L2-only path (the line may have been written by
// another SM earlier in the same launch).
template <typename T>
__device__ __forceinline__ T ldcg_elem(const T* p) {
  using Raw = typename RawT<sizeof(T)>::type;
  const Raw r = __ldcg(reinterpret_cast<const Raw*>(p));
  T t;
  memcpy(&t, &r, sizeof(T));
  return t;
}

__device__ __forceinline__ int aa_wrap(int s, int n, int per, bool& wall) {
  if (s < 0 || s >= n) {
    if (per) return s < 0 ? s + n : s - n;
    wall = true;
  }
  return s;
}

// Slot holding f_i(x, t) given the parity of the number of completed steps.
template <class L>
__device__ __forceinline__ long long aa_state_slot(const Geo& G, const uint8_t* mask, int parity,
                                                   int x, int y, int z, int i) {
  const long long own = ((long long)z * G.ny + y) * G.pitch + x;
  if (parity == 0) return i * G.plane + own;
  bool wall = false;
  const int xs = aa_wrap(x - L::cx(i), G.nx, G.per[0], wall);
  const int ys = aa_wrap(y - L::cy(i), G.ny, G.per[1], wall);
  const int zs = aa_wrap(z - L::cz(i), G.nz, G.per[2], wall);
  if (!wall && mask && mask[((long long)zs * G.ny + ys) * G.nx + xs]) wall = true;
  if (wall) return i * G.plane + own;
  return L::opp(i) * G.plane + ((long long)zs * G.ny + ys) * G.pitch + xs;
}

// Slot that receives f*_i(x) in an odd step.
template <class L>
__device__ __forceinline__ long long aa_odd_dst(const Geo& G, const uint8_t* mask, int x, int y,
                                                int z, int i) {
  bool wall = false;
  const int xd = aa_wrap(x + L::cx(i), G.nx, G.per[0], wall);
  const int yd = aa_wrap(y + L::cy(i), G.ny, G.per[1], wall);
  const int zd = aa_wrap(z + L::cz(i), G.nz, G.per[2], wall);
  if (!wall && mask && mask[((long long)zd * G.ny + yd) * G.nx + xd]) wall = true;
  if (wall) return L::opp(i) * G.plane + ((long long)z * G.ny + y) * G.pitch + x;
  return i * G.plane + ((long long)zd * G.ny + yd) * G.pitch + xd;
}

template <class L, int COLL, class S, bool MASK>
__device__ __forceinline__ void aa_node(const StepArgs<typename S::R>& a, int x, int y, int z,
                                        int parity) {
  using T = typename S::T;
  using R = typename S::R;
  const Geo& G = a.g;
  T* __restrict__ buf = static_cast<T*>(a.dst);
  const uint8_t* mask = MASK ? a.mask : nullptr;
  if (MASK && mask[((long long)z * G.ny + y) * G.nx + x]) return;
  long long slot[L::Q];
  R g[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    slot[i] = aa_state_slot<L>(G, mask, parity, x, y, z, i);
    g[i] = S::dec(buf[slot[i]]);
  }
  const bool bad = collide_v<L, COLL, true, R>(g, a.c) != 0u;
  if (parity == 0) {
    const long long own = ((long long)z * G.ny + y) * G.pitch + x;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) buf[L::opp(i) * G.plane + own] = S::enc(g[i]);
  } else {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) buf[aa_odd_dst<L>(G, mask, x, y, z, i)] = S::enc(g[i]);
  }
  record_bad(a.flag, a.step, bad);
}

template <class L, int COLL, class S, int NV, bool MASK>
__global__ void __launch_bounds__(256) k_step_aa_even(const StepArgs<typename S::R> a) {
  if constexpr (NV == 1) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x < a.g.nx && y < a.g.ny) aa_node<L, COLL, S, MASK>(a, x, y, blockIdx.z, 0);
  }
}

template <class L, int COLL, class S, int NV, bool MASK>
__global__ void __launch_bounds__(256) k_step_aa_odd(const StepArgs<typename S::R> a) {
  if constexpr (NV == 1) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x < a.g.nx && y < a.g.ny) aa_node<L, COLL, S, MASK>(a, x, y, blockIdx.z, 1);
  }
}

}  // namespace lbm
