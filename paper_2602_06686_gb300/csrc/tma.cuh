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
// x + X/2) with the packed f32x2 arithmetic (collide_v<..., F2>).  The tile
// width X is a compile-time constant, so in tiles without walls every shared
// read is a single load at a fixed offset; consumers release the stage as soon
// as their populations are in registers, before colliding.
//
// Rows whose source lies beyond a non-periodic wall (halfway bounce-back) are
// replaced by the node's own row of the opposite plane; x-walls read the
// opposite plane's own value from HBM (rare, per node).  Masked lattices use
// the register kernel.
//
// Every mbarrier wait is bounded by %globaltimer: on time-out the block sets
// an error word, lets its issued copies land, and returns.
//
// MODE selects what the consumers do with the gathered populations: 0 the
// update; 1 the first pass of forcing Scheme II (Eq. source_simple, Eq. Gi):
// store Phi_a = rho u_a^3 of every node, no update; 2 the update followed by
// the cubic correction G_i from the differences of the stored Phi.  In MODE 2
// the producer also stages the Phi rows a tile's differences need -- Phi_x of
// the tile's own row with an x halo, Phi_y of rows y-1, y, y+1 and, on D3Q19,
// Phi_z of rows z-1, z, z+1, wrapped across periodic axes and skipped beyond
// walls -- so that they arrive with the populations (TmaPhi).  MODE 3 is the
// update with the staged bulk stores of a store warp; MODE 4 the update with
// four adjacent nodes per consumer thread (16-bit storage).
#pragma once
#include <stdint.h>

#include <type_traits>

#include "collide_v.cuh"
#include "dispatch.h"
#include "kernels.cuh"
#include "storage.cuh"

namespace lbm {

// One producer warp plus X / NPT consumer threads (NPT = 2 nodes per thread with
// the packed arithmetic, 1 otherwise): every consumer thread owns one node pair
// (x0 + j, x0 + j + X/2) -- or one node -- of each tile.
// SW = 1 adds a store warp (warp 1) between the producer and the consumers;
// NQ = 4 gives every consumer four adjacent nodes (two packed pairs).
template <int X, bool PACK, int SW = 0, int NQ = 0>
struct TmaShape {
  static constexpr int kNPT = NQ ? NQ : (PACK ? 2 : 1);
  static constexpr int kConsumers = X / kNPT;
  static constexpr int kConsumerWarps = kConsumers / 32;
  static constexpr int kBase = 32 * (1 + SW);  // first consumer thread
  static constexpr int kThreads = kBase + kConsumers;
  static_assert(kConsumers % 32 == 0, "tile width must give whole consumer warps");
};

template <typename R>
struct TmaArgs {
  Geo g;
  CoefV<R> c;
  const void* src;
  void* dst;
  unsigned int* flag;  // divergence: earliest step (atomicMin)
  int* err;            // set to 1 when a bounded wait runs out
  unsigned int step;
  int stages;  // ring depth
  int ntx;     // tiles per row (tile width is the kernel's compile-time X)
  int ntiles;  // ntx * ny * nz (< 2^31)
  long long timeout_ns;
  int extra_tx;  // test hook: extra bytes every stage waits for (never delivered)
  void* phi;     // MODE 1 / 2: rho u_a^3, [D][nx * ny * nz] (dense node index), precision R
  R gk;          // MODE 2: -(1 - w+/2) / (6 cs^6)
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
// try_wait with a suspend-time hint: a warp whose phase is not complete sleeps
// (up to kSuspendNs) instead of re-issuing, leaving the issue slots to others.
constexpr uint32_t kSuspendNs = 20000;
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendNs)
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
// shared -> global bulk copy (both addresses 16-byte aligned, bytes a multiple
// of 16), tracked by the issuing thread's bulk-async groups
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the sources of every committed group have been read (the shared memory may be reused)
__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// every committed group has completed
__device__ __forceinline__ void bulk_wait_all0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// orders this thread's shared-memory writes before later bulk copies that read them
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ long long tma_now() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait.  Returns false if the wait ran out (then the abort flag and the
// global error word are set) or another warp aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, long long timeout_ns, bool heed_abort = true) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = tma_now();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (heed_abort && *abort_flag) return false;
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

// The contiguous chunk of tiles [begin, end) owned by this block, walked with
// incremental (tx, y, z) coordinates (no divisions inside the loop).  Tiles are
// numbered ((z * ny) + y) * ntx + tx.
struct TileWalk {
  int t, end, tx, y, z, ntx, ny;
  __device__ __forceinline__ TileWalk(int ntiles, int ntx_, int ny_) : ntx(ntx_), ny(ny_) {
    t = (int)(((long long)ntiles * blockIdx.x) / gridDim.x);
    end = (int)(((long long)ntiles * (blockIdx.x + 1)) / gridDim.x);
    tx = t % ntx;
    const int row = t / ntx;
    y = row % ny;
    z = row / ny;
  }
  __device__ __forceinline__ bool more() const { return t < end; }
  __device__ __forceinline__ void next() {
    ++t;
    if (++tx == ntx) {
      tx = 0;
      if (++y == ny) {
        y = 0;
        ++z;
      }
    }
  }
};

template <class L>
__device__ __forceinline__ int opp_dyn(int i) {
  int r = 0;
#pragma unroll
  for (int k = 0; k < L::Q; ++k)
    if (k == i) r = L::opp(k);
  return r;
}

// tma_source_row for a plane index known only at run time.
template <class L>
__device__ __forceinline__ void tma_source_row_dyn(const Geo& G, int i, int y, int z, int& ys,
                                                   int& zs, bool& wall) {
  int ey = 0, ez = 0;
#pragma unroll
  for (int k = 0; k < L::Q; ++k)
    if (k == i) {
      ey = L::cy(k);
      ez = L::cz(k);
    }
  ys = y - ey;
  zs = z - ez;
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

// Shared-memory rows of the staged Phi in MODE 2 (after the Q population slots
// of a stage): row 0 Phi_x of the own row over [x0 - HR, x0 + X + HR), rows
// 1..3 Phi_y and 4..6 Phi_z of the rows at offsets -1, 0, +1, each over
// [x0, x0 + X) starting at element HR.  HR = 16 bytes of halo.
template <class L, typename R, int XT>
struct TmaPhi {
  static constexpr int kHR = 16 / (int)sizeof(R);
  static constexpr int kSlot = XT + 2 * kHR;
  static constexpr int kRows = 1 + 3 * (L::D - 1);
  static constexpr int kBytes = kRows * kSlot * (int)sizeof(R);
};

// One-sided / central difference from the neighbour flags and values.
template <typename R>
__device__ __forceinline__ R diff3(bool okm, bool okp, R vm, R v0, R vp) {
  if (okm && okp) return R(0.5) * (vp - vm);
  if (okp) return vp - v0;
  if (okm) return v0 - vm;
  return R(0);
}

// d_a Phi_a at node (x, y, z), dense index n, for forcing Scheme II: central
// difference where both neighbours along axis a are fluid nodes (a periodic
// axis wraps), one-sided where one is solid or beyond a non-periodic edge,
// zero where both are.
template <class L, typename R>
__device__ __forceinline__ R phi_grad(const Geo& G, const uint8_t* mask, const R* __restrict__ phi,
                                      int d, int x, int y, int z, long long n) {
  const int c = d == 0 ? x : (d == 1 ? y : z);
  const int ext = d == 0 ? G.nx : (d == 1 ? G.ny : G.nz);
  const long long stride = d == 0 ? 1LL : (d == 1 ? (long long)G.nx : (long long)G.nx * G.ny);
  const long long N = (long long)G.nx * G.ny * G.nz;
  bool okm = true, okp = true;
  long long nm = n - stride, np = n + stride;
  if (c == 0) {
    if (G.per[d]) nm = n + (long long)(ext - 1) * stride;
    else okm = false;
  }
  if (c == ext - 1) {
    if (G.per[d]) np = n - (long long)(ext - 1) * stride;
    else okp = false;
  }
  if (mask) {
    if (okm && mask[nm]) okm = false;
    if (okp && mask[np]) okp = false;
  }
  const R* p = phi + d * N;
  if (okm && okp) return R(0.5) * (p[np] - p[nm]);
  if (okp) return p[np] - p[n];
  if (okm) return p[n] - p[nm];
  return R(0);
}

// Resident blocks per SM the register allocation is asked to allow: 4 for
// 16-bit storage (the collision is then the limiter and more warps hide it), 2
// for FP32, none for FP64 (whose collision needs the registers).  Measured on
// GB300: +6% (D3Q19 FP16) and +11% (D2Q9 FP32) over no hint.
// D3Q27 FP32 asks for 3: at two blocks its 160-thread blocks leave the SM
// short of consumer warps (occupancy, not registers, limits it).
// With the staged bulk stores (MODE 3, one more warp) 16-bit storage asks for
// 3: at 4 blocks of 256 threads the 64-register cap spills.  Four nodes per
// thread (MODE 4) hold two pairs of populations and keep the 16-bit request
// of 4 (D3Q19 at tile 384: 128 threads, 128 registers, no spill); on D3Q27
// they keep its 3 (166 registers).  D3Q27 tiles wider than 256 with two nodes
// per thread (224 threads and more) ask for 2: three would cap them at 97
// registers and spill.
template <class L, class S, int MODE = 0, int XT = 0>
constexpr int tma_min_blocks() {
  if (L::Q == 27) return sizeof(typename S::T) == 8 ? 1 : (XT > 256 && MODE != 4 ? 2 : 3);
  if (MODE == 3 && sizeof(typename S::T) == 2) return 3;
  if (MODE == 4 && sizeof(typename S::T) == 2) return 4;
  return sizeof(typename S::T) == 2 ? 4 : (sizeof(typename S::T) == 4 ? 2 : 1);
}

template <class L, int COLL, class S, bool FORCE, bool PACK, int XT, int MODE = 0>
__global__ void __launch_bounds__(TmaShape<XT, PACK, MODE == 3 ? 1 : 0, MODE == 4 ? 4 : 0>::kThreads,
                                  tma_min_blocks<L, S, MODE, XT>())
    k_step_tma(const TmaArgs<typename S::R> a) {
  using T = typename S::T;
  using R = typename S::R;
  using V = typename std::conditional<PACK, F2, R>::type;
  using Sh = TmaShape<XT, PACK, MODE == 3 ? 1 : 0, MODE == 4 ? 4 : 0>;
  constexpr int HT = 16 / (int)sizeof(T);  // halo (elements)
  constexpr int SLOT = XT + 2 * HT;        // elements per plane slot
  extern __shared__ __align__(128) unsigned char smem[];
  const Geo& G = a.g;
  const int ST = a.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + ST;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + ST);
  unsigned char* ringb = smem + 128 * ((2 * ST * 8 + 4 + 127) / 128);
  using Ph = TmaPhi<L, R, XT>;
  constexpr long long pop_bytes = (long long)L::Q * SLOT * sizeof(T);
  constexpr long long stage_bytes = pop_bytes + (MODE == 2 ? Ph::kBytes : 0);
  // MODE 3: after the ring (128-byte aligned) the staging region of
  // tma_bs_smem: ob_full[2], ob_free[2], then staging buffers 0 and 1 of Q
  // rows of XT elements (row i holds plane i of the tile's nodes)
  constexpr long long kOutElems = ((long long)L::Q * XT * sizeof(T) + 127) / 128 * 128 / sizeof(T);
  unsigned char* oreg = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(ringb + ST * stage_bytes) + 127) & ~uintptr_t(127));
  uint64_t* ob_full = reinterpret_cast<uint64_t*>(oreg);
  uint64_t* ob_free = ob_full + 2;
  T* outs = reinterpret_cast<T*>(oreg + 128);

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_addr(full + s), 1);
      mbar_init(smem_addr(empty + s), Sh::kConsumerWarps);
    }
    if (MODE == 3) {
      for (int b = 0; b < 2; ++b) {
        mbar_init(smem_addr(ob_full + b), Sh::kConsumerWarps);
        mbar_init(smem_addr(ob_free + b), 1);
      }
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
    // Lane i (< Q) copies population plane i; lane 0 sets the expected byte
    // count.  The warp waits for the stage together, so it stays converged.
    const unsigned full_mask = 0xffffffffu;
    TileWalk w(a.ntiles, a.ntx, G.ny);
    int k = 0;
    int s = 0;       // stage of tile k
    uint32_t u = 0;  // use count of stage s
    bool ok = true;
    for (; w.more(); w.next(), ++k) {
      // every lane observes the stage's release itself before writing into it
      if (u > 0 && !mbar_wait_warp(smem_addr(empty + s), (u - 1) & 1u, abort_flag, a.err,
                                   a.timeout_ns)) {
        ok = false;
        break;
      }
      const int y = w.y, z = w.z;
      const int x0 = w.tx * XT;
      const int xe = min(x0 + XT, G.nx);  // end of the tile's nodes
      // copy window [lo, hi) of every source row, plus wrap halos at row ends
      const int lo = max(x0 - HT, 0);
      const int hi = min(xe + HT, G.nx);
      const bool lwrap = G.per[0] && x0 == 0;
      const bool rwrap = G.per[0] && xe == G.nx;
      const uint32_t main_bytes = (uint32_t)(hi - lo) * sizeof(T);
      constexpr uint32_t halo_bytes = (uint32_t)HT * sizeof(T);
      int ys = 0, zs = 0;
      bool wall = false;
      const int i = lane;
      if (i < L::Q) tma_source_row_dyn<L>(G, i, y, z, ys, zs, wall);
      const unsigned walls = __ballot_sync(full_mask, i < L::Q && wall);
      const uint32_t fb = smem_addr(full + s);
      // MODE 2: lane Q + k copies Phi row k of TmaPhi (phr: source row, or -1)
      long long phr = -1;
      int phd = 0;
      uint32_t phbytes = 0;
      if constexpr (MODE == 2) {
        const int k = lane - L::Q;
        if (k >= 0 && k < Ph::kRows) {
          constexpr uint32_t hrb = (uint32_t)Ph::kHR * sizeof(R);
          if (k == 0) {
            phd = 0;
            phr = (long long)z * G.ny + y;
            const int plo = max(x0 - Ph::kHR, 0), phi_ = min(xe + Ph::kHR, G.nx);
            phbytes = (uint32_t)(phi_ - plo) * sizeof(R) + ((lwrap ? hrb : 0u) + (rwrap ? hrb : 0u));
          } else {
            phd = (k - 1) / 3 + 1;          // 1: y rows, 2: z rows
            const int off = (k - 1) % 3 - 1;  // -1, 0, +1
            int yy = y, zz = z;
            bool ok = true;
            if (phd == 1) {
              yy = y + off;
              if (yy < 0 || yy >= G.ny) {
                if (G.per[1]) yy = yy < 0 ? yy + G.ny : yy - G.ny;
                else ok = false;
              }
            } else {
              zz = z + off;
              if (zz < 0 || zz >= G.nz) {
                if (G.per[2]) zz = zz < 0 ? zz + G.nz : zz - G.nz;
                else ok = false;
              }
            }
            if (ok) {
              phr = (long long)zz * G.ny + yy;
              phbytes = (uint32_t)(xe - x0) * sizeof(R);
            }
          }
        }
        phbytes = __reduce_add_sync(full_mask, phbytes);
      }
      if (lane == 0) {
        const uint32_t nwrap = (uint32_t)(L::Q - __popc(walls)) * ((lwrap ? 1u : 0u) + (rwrap ? 1u : 0u));
        mbar_arrive_expect_tx(fb, main_bytes * L::Q + nwrap * halo_bytes + phbytes + (uint32_t)a.extra_tx);
      }
      __syncwarp();
      if constexpr (MODE == 2) {
        if (phr >= 0) {
          const int k = lane - L::Q;
          R* prow = reinterpret_cast<R*>(ringb + s * stage_bytes + pop_bytes) + k * Ph::kSlot;
          const R* gsrc = static_cast<const R*>(a.phi) + (long long)phd * ((long long)G.nx * G.ny * G.nz) +
                          phr * G.nx;
          if (k == 0) {
            constexpr uint32_t hrb = (uint32_t)Ph::kHR * sizeof(R);
            const int plo = max(x0 - Ph::kHR, 0), phi_ = min(xe + Ph::kHR, G.nx);
            bulk_g2s(smem_addr(prow + (plo - (x0 - Ph::kHR))), gsrc + plo, (uint32_t)(phi_ - plo) * sizeof(R), fb);
            if (lwrap) bulk_g2s(smem_addr(prow), gsrc + G.nx - Ph::kHR, hrb, fb);
            if (rwrap) bulk_g2s(smem_addr(prow + Ph::kHR + (G.nx - x0)), gsrc, hrb, fb);
          } else {
            bulk_g2s(smem_addr(prow + Ph::kHR), gsrc + x0, (uint32_t)(xe - x0) * sizeof(R), fb);
          }
        }
      }
      if (i < L::Q) {
        T* slot = reinterpret_cast<T*>(ringb + s * stage_bytes) + i * SLOT;  // slot[k] holds x = x0 - HT + k
        const int pi = wall ? opp_dyn<L>(i) : i;
        const long long r = wall ? ((long long)z * G.ny + y) : ((long long)zs * G.ny + ys);
        const T* rowp = src + pi * G.plane + r * G.pitch;
        bulk_g2s(smem_addr(slot + (lo - (x0 - HT))), rowp + lo, main_bytes, fb);
        if (!wall) {
          if (lwrap) bulk_g2s(smem_addr(slot), rowp + G.nx - HT, halo_bytes, fb);
          if (rwrap) bulk_g2s(smem_addr(slot + HT + (G.nx - x0)), rowp, halo_bytes, fb);
        }
      }
      if (++s == ST) {
        s = 0;
        ++u;
      }
    }
    if (!ok && lane == 0) {
      // let every issued copy land before the block's shared memory is released
      for (int kk = (k > ST ? k - ST : 0); kk < k; ++kk)
        mbar_wait(smem_addr(full + kk % ST), (uint32_t)((kk / ST) & 1), abort_flag, a.err,
                  a.timeout_ns, false);
    }
    return;
  }

  if constexpr (MODE == 3) {
    if (warp == 1) {
      // ---------------------------------------------------------- store warp
      // Tile k's post-collision rows wait in staging buffer k & 1; lane i copies
      // row i to plane i of the tile's row segment with one bulk copy (the
      // 16-byte multiple; a ragged tile's remaining elements one by one), then
      // hands the buffer back once its rows have been read.
      TileWalk w(a.ntiles, a.ntx, G.ny);
      for (int k = 0; w.more(); w.next(), ++k) {
        const int b = k & 1;
        if (!mbar_wait_warp(smem_addr(ob_full + b), (uint32_t)((k >> 1) & 1), abort_flag, a.err,
                            a.timeout_ns))
          break;
        if (lane < L::Q) {
          const int x0 = w.tx * XT;
          const int wdt = min(XT, G.nx - x0);
          const T* so = outs + b * kOutElems + lane * XT;
          T* gd = dst + (long long)lane * G.plane + ((long long)w.z * G.ny + w.y) * G.pitch + x0;
          const int nb = (wdt * (int)sizeof(T)) & ~15;
          if (nb > 0) bulk_s2g(gd, smem_addr(so), (uint32_t)nb);
          for (int e = nb / (int)sizeof(T); e < wdt; ++e) gd[e] = so[e];
          bulk_commit();
          bulk_wait_read0();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(ob_free + b));
      }
      if (lane < L::Q) bulk_wait_all0();
      return;
    }
  }

  if constexpr (MODE == 4) {
    // ------------------------------------------- consumers, four nodes each
    // 16-bit storage: nodes x0 + j0 .. x0 + j0 + 3 (j0 = 4 ct) as two packed
    // pairs.  Unshifted planes load the four as one 64-bit word, shifted
    // planes element by element; full tiles store one 64-bit word per plane.
    static_assert(PACK && sizeof(T) == 2, "four nodes per thread: 16-bit storage");
    const int j0 = 4 * (threadIdx.x - Sh::kBase);
    TileWalk w(a.ntiles, a.ntx, G.ny);
    int s = 0;
    uint32_t u = 0;
    for (; w.more(); w.next()) {
      if (!mbar_wait_warp(smem_addr(full + s), u & 1u, abort_flag, a.err, a.timeout_ns)) break;
      const int y = w.y, z = w.z;
      const int x0 = w.tx * XT;
      const int wdt = min(XT, G.nx - x0);
      const T* st = reinterpret_cast<const T*>(ringb + s * stage_bytes);
      const long long own = ((long long)z * G.ny + y) * G.pitch;
      const bool anywall = (!G.per[1] && (y == 0 || y == G.ny - 1)) ||
                           (L::D == 3 && !G.per[2] && (z == 0 || z == G.nz - 1));
      const bool xwall = !G.per[0] && (x0 == 0 || x0 + XT >= G.nx);
      bool act[4];
#pragma unroll
      for (int n = 0; n < 4; ++n) act[n] = j0 + n < wdt;
      F2 ga[L::Q], gb[L::Q];
      if (!anywall && !xwall) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
          const T* slot = st + i * SLOT + HT - L::cx(i);
          if (L::cx(i) == 0) {
            // slot + HT is 16-byte aligned and j0 a multiple of 4: one 8-byte word
            const uint2 wv = *reinterpret_cast<const uint2*>(slot + j0);
            float a0, a1, a2, a3;
            S::dec2(wv.x, a0, a1);
            S::dec2(wv.y, a2, a3);
            ga[i] = F2{a0, a1};
            gb[i] = F2{a2, a3};
          } else {
            ga[i] = F2{S::dec(slot[j0]), S::dec(slot[j0 + 1])};
            gb[i] = F2{S::dec(slot[j0 + 2]), S::dec(slot[j0 + 3])};
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
          const int ex = L::cx(i);
          const T* slot = st + i * SLOT + HT;
          int ys, zs;
          bool wallrow;
          tma_source_row<L>(G, i, y, z, ys, zs, wallrow);
          float v[4];
#pragma unroll
          for (int n = 0; n < 4; ++n) {
            const int j = j0 + n;
            const int x = x0 + j;
            if (wallrow) {
              v[n] = S::dec(slot[j]);
            } else if (!G.per[0] && ((ex == 1 && x == 0) || (ex == -1 && x == G.nx - 1))) {
              v[n] = act[n] ? S::dec(src[L::opp(i) * G.plane + own + x]) : 0.f;
            } else {
              v[n] = S::dec(slot[j - ex]);
            }
          }
          ga[i] = F2{v[0], v[1]};
          gb[i] = F2{v[2], v[3]};
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(empty + s));
      if (++s == ST) {
        s = 0;
        ++u;
      }
      const unsigned ba = collide_v<L, COLL, FORCE, F2>(ga, a.c);
      const unsigned bb = collide_v<L, COLL, FORCE, F2>(gb, a.c);
      const bool anybad = (act[0] && (ba & 1u)) || (act[1] && (ba & 2u)) || (act[2] && (bb & 1u)) ||
                          (act[3] && (bb & 2u));
      T* op = dst + own + x0 + j0;
      if (wdt == XT) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
          uint2 wv;
          wv.x = S::enc2(ga[i].x, ga[i].y);
          wv.y = S::enc2(gb[i].x, gb[i].y);
          *reinterpret_cast<uint2*>(op) = wv;  // 8-byte aligned: 16-byte rows, j0 a multiple of 4
          op += G.plane;
        }
      } else {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
          const float o[4] = {ga[i].x, ga[i].y, gb[i].x, gb[i].y};
#pragma unroll
          for (int n = 0; n < 4; ++n)
            if (act[n]) op[n] = S::enc(o[n]);
          op += G.plane;
        }
      }
      record_bad(a.flag, a.step, anybad);
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  constexpr int NPT = Sh::kNPT;
  // 16-bit storage: a thread's node pair is adjacent (x0 + 2j, x0 + 2j + 1), so
  // unshifted planes load, and every plane stores, one 32-bit word per pair.
  // 32-bit storage keeps the split pair (x0 + j, x0 + j + X/2), whose scalar
  // shared reads are free of bank conflicts for every x shift.
  constexpr bool ADJ = PACK && sizeof(T) == 2;
  const int ct = threadIdx.x - Sh::kBase;  // 0 .. kConsumers-1: this thread's node (pair)
  int jn[NPT];
  jn[0] = ADJ ? 2 * ct : ct;
  if (PACK) jn[NPT - 1] = ADJ ? 2 * ct + 1 : ct + XT / 2;
  TileWalk w(a.ntiles, a.ntx, G.ny);
  int s = 0;
  uint32_t u = 0;
  int kt = 0;  // MODE 3: tiles done by this block
  for (; w.more(); w.next()) {
    if (!mbar_wait_warp(smem_addr(full + s), u & 1u, abort_flag, a.err, a.timeout_ns)) break;
    const int y = w.y, z = w.z;
    const int x0 = w.tx * XT;
    const int wdt = min(XT, G.nx - x0);
    const T* st = reinterpret_cast<const T*>(ringb + s * stage_bytes);
    const long long own = ((long long)z * G.ny + y) * G.pitch;
    // tile-uniform: does any plane's source row lie beyond a wall (|e| <= 1, so
    // only boundary rows of a non-periodic axis), or does the tile touch an x
    // wall?  If neither, every read is one shared load at a fixed offset.
    const bool anywall = (!G.per[1] && (y == 0 || y == G.ny - 1)) ||
                         (L::D == 3 && !G.per[2] && (z == 0 || z == G.nz - 1));
    const bool xwall = !G.per[0] && (x0 == 0 || x0 + XT >= G.nx);
    bool act[NPT];
#pragma unroll
    for (int n = 0; n < NPT; ++n) act[n] = jn[n] < wdt;
    V g[L::Q];
    if (!anywall && !xwall) {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const T* slot = st + i * SLOT + HT - L::cx(i);
        if constexpr (ADJ) {
          if (L::cx(i) == 0) {
            // slot + HT is 16-byte aligned and jn[0] even: one aligned word
            float a0, a1;
            S::dec2(*reinterpret_cast<const uint32_t*>(slot + jn[0]), a0, a1);
            g[i] = F2{a0, a1};
          } else {
            g[i] = F2{S::dec(slot[jn[0]]), S::dec(slot[jn[NPT - 1]])};
          }
        } else if constexpr (PACK) {
          g[i] = F2{S::dec(slot[jn[0]]), S::dec(slot[jn[NPT - 1]])};
        } else {
          g[i] = S::dec(slot[jn[0]]);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const int ex = L::cx(i);
        const T* slot = st + i * SLOT + HT;
        int ys, zs;
        bool wallrow;
        tma_source_row<L>(G, i, y, z, ys, zs, wallrow);
        R v[NPT];
#pragma unroll
        for (int n = 0; n < NPT; ++n) {
          const int j = jn[n];
          const int x = x0 + j;
          if (wallrow) {
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
    }
    R dn[NPT][3];  // MODE 2: d_a Phi_a of this thread's nodes, from the staged rows
    if constexpr (MODE == 2) {
      const R* pst = reinterpret_cast<const R*>(reinterpret_cast<const unsigned char*>(st) + pop_bytes);
      const bool ym = G.per[1] || y > 0, yp = G.per[1] || y < G.ny - 1;
      const bool zm = G.per[2] || z > 0, zp = G.per[2] || z < G.nz - 1;
      constexpr int HR = Ph::kHR, SR = Ph::kSlot;
#pragma unroll
      for (int n = 0; n < NPT; ++n) {
        const int j = jn[n];
        const int x = x0 + j;
        const R* px = pst + HR + j;
        const R* py = pst + SR + HR + j;
        dn[n][0] = act[n] ? diff3<R>(G.per[0] || x > 0, G.per[0] || x < G.nx - 1, px[-1], px[0], px[1]) : R(0);
        dn[n][1] = act[n] ? diff3<R>(ym, yp, py[0], py[SR], py[2 * SR]) : R(0);
        dn[n][2] = R(0);
        if constexpr (L::D == 3) {
          const R* pz = pst + 4 * SR + HR + j;
          dn[n][2] = act[n] ? diff3<R>(zm, zp, pz[0], pz[SR], pz[2 * SR]) : R(0);
        }
      }
    }
    // the stage is no longer read: release it before computing
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_addr(empty + s));
    if (++s == ST) {
      s = 0;
      ++u;
    }
    const long long rowd = ((long long)z * G.ny + y) * G.nx + x0;  // dense index of x0
    const long long Nd = (long long)G.nx * G.ny * G.nz;
    if constexpr (MODE == 1) {
      // rho and the half-force u (Eq. macro), then Phi_a = rho u_a^3
      using A = Ar<V>;
      V drho = g[0];
      V j[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) j[d] = A::c(0.0);
#pragma unroll
      for (int i = 1; i < L::Q; ++i) {
        drho = A::add(drho, g[i]);
#pragma unroll
        for (int d = 0; d < L::D; ++d) {
          const int e = d == 0 ? L::cx(i) : (d == 1 ? L::cy(i) : L::cz(i));
          if (e == 1) j[d] = A::add(j[d], g[i]);
          if (e == -1) j[d] = A::sub(j[d], g[i]);
        }
      }
      const V rho = A::add(A::c(a.c.rho0), drho);
      const V inv = A::rcp(rho);
      R* ph = static_cast<R*>(a.phi);
#pragma unroll
      for (int d = 0; d < L::D; ++d) {
        const V ud = FORCE ? A::mul(A::add(j[d], A::c(a.c.Fh[d])), inv) : A::mul(j[d], inv);
        const V p = A::mul(A::mul(rho, ud), A::mul(ud, ud));
        R* pd = ph + d * Nd + rowd;
        if constexpr (PACK) {
          if (act[0]) pd[jn[0]] = p.x;
          if (act[NPT - 1]) pd[jn[NPT - 1]] = p.y;
        } else {
          if (act[0]) pd[jn[0]] = p;
        }
      }
      continue;
    }
    const unsigned bad = collide_v<L, COLL, FORCE, V>(g, a.c);
    if constexpr (MODE == 2) {
      // G_i = gk w_i (sum_a e_ia^2 D_a - (1/3) sum_a D_a), D_a = d_a Phi_a
      using A = Ar<V>;
      V dv[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if constexpr (PACK) dv[d] = F2{dn[0][d], dn[NPT - 1][d]};
        else dv[d] = dn[0][d];
      }
      const V third = A::mul(A::add(A::add(dv[0], dv[1]), dv[2]), A::c(1.0 / 3.0));
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        V h = A::sub(A::c(0.0), third);
        if (L::cx(i)) h = A::add(h, dv[0]);
        if (L::cy(i)) h = A::add(h, dv[1]);
        if (L::cz(i)) h = A::add(h, dv[2]);
        g[i] = A::fma(A::c(R(a.gk * R(L::w(i)))), h, g[i]);
      }
    }
    bool anybad = act[0] && (bad & 1u);
    if (PACK) anybad = anybad || (act[NPT - 1] && (bad & 2u));
    if constexpr (MODE == 3) {
      // into staging buffer kt & 1 (free once the store warp has read tile kt - 2)
      const int b = kt & 1;
      if (kt >= 2 && !mbar_wait_warp(smem_addr(ob_free + b), (uint32_t)(((kt >> 1) - 1) & 1), abort_flag,
                                     a.err, a.timeout_ns))
        break;
      T* ob = outs + b * kOutElems;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        T* orow = ob + i * XT;
        if constexpr (ADJ) {
          if (act[NPT - 1]) *reinterpret_cast<uint32_t*>(orow + jn[0]) = S::enc2(g[i].x, g[i].y);
          else if (act[0]) orow[jn[0]] = S::enc(g[i].x);
        } else if constexpr (PACK) {
          if (act[0]) orow[jn[0]] = S::enc(g[i].x);
          if (act[NPT - 1]) orow[jn[NPT - 1]] = S::enc(g[i].y);
        } else {
          if (act[0]) orow[jn[0]] = S::enc(g[i]);
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(ob_full + b));
      record_bad(a.flag, a.step, anybad);
      ++kt;
      continue;
    }
    T* op = dst + own + x0;
    if (wdt == XT) {
      // a full tile: every node is active, the stores need no per-plane test
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        if constexpr (ADJ) {
          *reinterpret_cast<uint32_t*>(op + jn[0]) = S::enc2(g[i].x, g[i].y);
        } else if constexpr (PACK) {
          op[jn[0]] = S::enc(g[i].x);
          op[jn[NPT - 1]] = S::enc(g[i].y);
        } else {
          op[jn[0]] = S::enc(g[i]);
        }
        op += G.plane;
      }
      record_bad(a.flag, a.step, anybad);
      continue;
    }
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      if constexpr (ADJ) {
        // op + jn[0] is 4-byte aligned (16-byte row pitch, even x0 + jn[0])
        if (act[NPT - 1]) {
          *reinterpret_cast<uint32_t*>(op + jn[0]) = S::enc2(g[i].x, g[i].y);
        } else if (act[0]) {
          op[jn[0]] = S::enc(g[i].x);
        }
      } else if constexpr (PACK) {
        if (act[0]) op[jn[0]] = S::enc(g[i].x);
        if (act[NPT - 1]) op[jn[NPT - 1]] = S::enc(g[i].y);
      } else {
        if (act[0]) op[jn[0]] = S::enc(g[i]);
      }
      op += G.plane;
    }
    record_bad(a.flag, a.step, anybad);
  }
}

}  // namespace lbm
