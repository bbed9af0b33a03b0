// tma.cuh -- warp-specialised fused update fed by bulk asynchronous copies.
//
// A persistent block owns a ring of `stages` shared-memory buffers.  Warp 0
// (one elected lane) is the producer: for each tile -- one row segment
// [x0, x0 + X) of row (y, z) -- it issues, per population plane i, one
// cp.async.bulk copy of the source row (y - ey_i, z - ez_i) over
// [x0 - H, x0 + X + H) into the stage (H = 16 bytes of halo), plus 16-byte
// wrap copies at periodic row ends; completion is tracked by the stage's
// "full" mbarrier (expect_tx).  The consumer warps wait on "full", read each
// node's Q pre-collision populations from shared memory at the x offset -e_x
// (so the shift costs nothing), collide, store the post-collision values to
// their own aligned slots in HBM and release the stage through its "empty"
// mbarrier.  Loads never occupy consumer registers while in flight, so the
// bytes in flight per SM are set by the ring size, not by occupancy.
//
// FP32 / FP16 / BF16 storage: each consumer thread advances two nodes (x and
// x + X/2) with the packed f32x2 arithmetic (collide_v<..., F2>).
//
// Rows whose source lies beyond a non-periodic wall (halfway bounce-back) are
// replaced by the node's own row of the opposite plane; x-walls read the
// opposite plane's own value from HBM (rare, per node).  Masked lattices use
// the register kernel.
//
// Every mbarrier wait is bounded by %globaltimer: on time-out the block sets
// an error word, lets its issued copies land, and returns.
#pragma once
#include <stdint.h>

#include <type_traits>

#include "collide_v.cuh"
#include "kernels.cuh"
#include "storage.cuh"

namespace lbm {

constexpr int kTmaConsumerWarps = 4;
constexpr int kTmaThreads = 32 * (1 + kTmaConsumerWarps);

template <typename R>
struct TmaArgs {
  Geo g;
  CoefV<R> c;
  const void* src;
  void* dst;
  unsigned int* flag;  // divergence: earliest step (atomicMin)
  int* err;            // set to 1 when a bounded wait runs out
  unsigned int step;
  int X;       // tile width (nodes), a multiple of 2H
  int H;       // halo (elements) = 16 bytes
  int stages;  // ring depth
  int ntx;     // tiles per row
  long long ntiles;
  int slot;    // elements per plane slot = X + 2H
  long long timeout_ns;
  int extra_tx;  // test hook: extra bytes every stage waits for (never delivered)
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ long long tma_now() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait.  Returns false if the wait ran out (then the abort flag and the
// global error word are set) or another warp aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, long long timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = tma_now();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (tma_now() - t0 > timeout_ns) {
      *abort_flag = 1;
      atomicExch(err, 1);
      return false;
    }
  }
}

// Warp-uniform bounded wait (all 32 lanes call it and get the same answer).
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity,
                                               volatile int* abort_flag, int* err,
                                               long long timeout_ns) {
  const unsigned full = 0xffffffffu;
  if (__all_sync(full, mbar_try_wait(bar, parity))) return true;
  const long long t0 = tma_now();
  for (;;) {
    if (__all_sync(full, mbar_try_wait(bar, parity))) return true;
    int stop = 0;
    if ((threadIdx.x & 31) == 0) {
      if (*abort_flag) {
        stop = 1;
      } else if (tma_now() - t0 > timeout_ns) {
        *abort_flag = 1;
        atomicExch(err, 1);
        stop = 1;
      }
    }
    if (__shfl_sync(full, stop, 0)) return false;
  }
}

template <class L>
__device__ __forceinline__ void tma_source_row(const Geo& G, int i, int y, int z, int& ys, int& zs,
                                               bool& wall) {
  ys = y - L::cy(i);
  zs = z - L::cz(i);
  wall = false;
  if (ys < 0 || ys >= G.ny) {
    if (G.per[1]) ys = ys < 0 ? ys + G.ny : ys - G.ny;
    else wall = true;
  }
  if (zs < 0 || zs >= G.nz) {
    if (G.per[2]) zs = zs < 0 ? zs + G.nz : zs - G.nz;
    else wall = true;
  }
}

template <class L, int COLL, class S, bool FORCE, bool PACK>
__global__ void __launch_bounds__(kTmaThreads) k_step_tma(const TmaArgs<typename S::R> a) {
  using T = typename S::T;
  using R = typename S::R;
  using V = typename std::conditional<PACK, F2, R>::type;
  extern __shared__ __align__(128) unsigned char smem[];
  const Geo& G = a.g;
  const int ST = a.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + ST;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + ST);
  T* ring = reinterpret_cast<T*>(smem + 128 * ((2 * ST * 8 + 4 + 127) / 128));
  const long long stage_elems = (long long)L::Q * a.slot;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_addr(full + s), 1);
      mbar_init(smem_addr(empty + s), kTmaConsumerWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* __restrict__ src = static_cast<const T*>(a.src);
  T* __restrict__ dst = static_cast<T*>(a.dst);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane != 0) return;
    long long k = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
      const int s = (int)(k % ST);
      const long long u = k / ST;
      if (u > 0 && !mbar_wait(smem_addr(empty + s), (uint32_t)((u - 1) & 1), abort_flag, a.err,
                               a.timeout_ns)) {
        ok = false;
        break;
      }
      const int tx = (int)(t % a.ntx);
      const long long row = t / a.ntx;
      const int y = (int)(row % G.ny), z = (int)(row / G.ny);
      const int x0 = tx * a.X;
      const int xe = min(x0 + a.X, G.nx);  // end of the tile's nodes
      // copy window [lo, hi) of every source row, plus wrap halos at row ends
      const int lo = max(x0 - a.H, 0);
      const int hi = min(xe + a.H, G.nx);
      const bool lwrap = G.per[0] && x0 == 0;
      const bool rwrap = G.per[0] && xe == G.nx;
      const uint32_t main_bytes = (uint32_t)(hi - lo) * sizeof(T);
      const uint32_t halo_bytes = (uint32_t)a.H * sizeof(T);
      uint32_t total = 0;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        int ys, zs;
        bool wall;
        tma_source_row<L>(G, i, y, z, ys, zs, wall);
        total += main_bytes;
        if (!wall) total += (lwrap ? halo_bytes : 0u) + (rwrap ? halo_bytes : 0u);
      }
      const uint32_t fb = smem_addr(full + s);
      mbar_arrive_expect_tx(fb, total + (uint32_t)a.extra_tx);
      T* st = ring + s * stage_elems;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        int ys, zs;
        bool wall;
        tma_source_row<L>(G, i, y, z, ys, zs, wall);
        T* slot = st + i * a.slot;  // slot[k] holds x = x0 - H + k
        const T* rowp = wall ? src + L::opp(i) * G.plane + ((long long)z * G.ny + y) * G.pitch
                             : src + i * G.plane + ((long long)zs * G.ny + ys) * G.pitch;
        bulk_g2s(smem_addr(slot + (lo - (x0 - a.H))), rowp + lo, main_bytes, fb);
        if (!wall) {
          if (lwrap) bulk_g2s(smem_addr(slot), rowp + G.nx - a.H, halo_bytes, fb);
          if (rwrap) bulk_g2s(smem_addr(slot + a.H + (G.nx - x0)), rowp, halo_bytes, fb);
        }
      }
    }
    if (!ok) {
      // let every issued copy land before the block's shared memory is released
      for (long long kk = (k > ST ? k - ST : 0); kk < k; ++kk) {
        const int s = (int)(kk % ST);
        const long long u = kk / ST;
        volatile int dummy = 0;
        mbar_wait(smem_addr(full + s), (uint32_t)(u & 1), &dummy, a.err, a.timeout_ns);
      }
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  const int ct = threadIdx.x - 32;
  constexpr int NCT = 32 * kTmaConsumerWarps;
  long long k = 0;
  for (long long t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
    const int s = (int)(k % ST);
    const long long u = k / ST;
    if (!mbar_wait_warp(smem_addr(full + s), (uint32_t)(u & 1), abort_flag, a.err, a.timeout_ns))
      break;
    const int tx = (int)(t % a.ntx);
    const long long row = t / a.ntx;
    const int y = (int)(row % G.ny), z = (int)(row / G.ny);
    const int x0 = tx * a.X;
    const int wdt = min(a.X, G.nx - x0);
    const T* st = ring + s * stage_elems;
    const long long own = ((long long)z * G.ny + y) * G.pitch;
    bool wallrow[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      int ys, zs;
      tma_source_row<L>(G, i, y, z, ys, zs, wallrow[i]);
    }
    unsigned anybad = 0;
    constexpr int NPT = PACK ? 2 : 1;
    const int half = a.X / 2;
    const int nwork = PACK ? half : a.X;
    for (int p = ct; p < nwork; p += NCT) {
      int jn[NPT];
      jn[0] = p;
      if (PACK) jn[NPT - 1] = p + half;
      bool act[NPT];
#pragma unroll
      for (int n = 0; n < NPT; ++n) act[n] = jn[n] < wdt;
      V g[L::Q];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const int ex = L::cx(i);
        const T* slot = st + i * a.slot + a.H;
        R v[NPT];
#pragma unroll
        for (int n = 0; n < NPT; ++n) {
          const int j = jn[n];
          const int x = x0 + j;
          if (wallrow[i]) {
            v[n] = S::dec(slot[j]);
          } else if (!G.per[0] && ((ex == 1 && x == 0) || (ex == -1 && x == G.nx - 1))) {
            v[n] = act[n] ? S::dec(src[L::opp(i) * G.plane + own + x]) : R(0);
          } else {
            v[n] = S::dec(slot[j - ex]);
          }
        }
        if constexpr (PACK) {
          g[i] = F2{v[0], v[NPT - 1]};
        } else {
          g[i] = v[0];
        }
      }
      const unsigned bad = collide_v<L, COLL, FORCE, V>(g, a.c);
      if (act[0] && (bad & 1u)) anybad = 1;
      if (PACK && act[NPT - 1] && (bad & 2u)) anybad = 1;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        T* outp = dst + i * G.plane + own + x0;
        if constexpr (PACK) {
          if (act[0]) outp[jn[0]] = S::enc(g[i].x);
          if (act[NPT - 1]) outp[jn[NPT - 1]] = S::enc(g[i].y);
        } else {
          if (act[0]) outp[jn[0]] = S::enc(g[i]);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_addr(empty + s));
    record_bad(a.flag, a.step, anybad != 0u);
  }
}

}  // namespace lbm
