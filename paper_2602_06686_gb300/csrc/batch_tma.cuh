// batch_tma.cuh -- persistent batched update fed by bulk asynchronous copies.
//
// The same warp-specialised pipeline as k_step_tma (tma.cuh), run over ALL
// lattices of a batch and over all steps in one cooperative launch:
//   * a tile is a row segment [x0, x0 + X) of one row (y, z) of one lattice;
//     tiles are numbered lattice by lattice (ntx * ny * nz tiles each, the
//     first one at the lattice's tile0), and block b owns the contiguous chunk
//     [T b / G, T (b + 1) / G) of the T tiles, the same chunk every step;
//   * per step, warp 0 copies each tile's Q source rows into the ring and the
//     consumer warps collide the nodes of the tile with the rates and force of
//     the tile's lattice (read from its descriptor) and store them;
//   * between steps every block meets at the bounded grid barrier; the ring's
//     mbarrier phases run on across steps.
// Extents need not be multiples of the 16-byte halo: a row copy is rounded up
// into the row's pitch padding (never read back), and where a periodic row end
// is not 16-byte aligned the producer also copies, per plane, the aligned
// 16 bytes that hold the wrap neighbour (x = nx - 1 for the row's first tile,
// x = 0 for its last) into two side slots of the stage, from which the end
// nodes read it.
// Data written in one step by generic stores is read in the next by the bulk
// copies (the async proxy): the grid barrier orders the two at GPU scope and
// a proxy fence on both sides of it orders them across the proxies.
#pragma once
#include "aa.cuh"
#include "batch.cuh"
#include "tma.cuh"

namespace lbm {

struct BatchTmaArgs {
  const BatchDesc* desc;
  int nlat;
  int ntiles;
  char* A;
  char* B;
  int nsteps;
  int parity0;
  unsigned int step0;
  unsigned int* flags;
  BarrierWords* bar;
  unsigned int expected;
  long long timeout_ns;
  int stages;
};

// Position of a block in the batch's tile sequence, with the geometry of the
// current lattice.
struct BatchWalk {
  int lat, tx, y, z;
  int nx, ny, nz, pitch, ntx;
  long long plane, off;
  int per0, per1, per2;

  __device__ __forceinline__ void load(const BatchDesc* __restrict__ desc, int l) {
    const BatchDesc& d = desc[l];
    lat = l;
    nx = d.g.nx;
    ny = d.g.ny;
    nz = d.g.nz;
    pitch = d.g.pitch;
    plane = d.g.plane;
    per0 = d.g.per[0];
    per1 = d.g.per[1];
    per2 = d.g.per[2];
    off = d.off;
    ntx = d.ntx;
  }
  // Tile t of the sequence: binary search of the lattices' first tiles.
  __device__ __forceinline__ void seek(const BatchDesc* __restrict__ desc, int nlat, int t) {
    int lo = 0, hi = nlat - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (desc[mid].tile0 <= t) lo = mid;
      else hi = mid - 1;
    }
    load(desc, lo);
    const int r = t - desc[lo].tile0;
    tx = r % ntx;
    const int row = r / ntx;
    y = row % ny;
    z = row / ny;
  }
  __device__ __forceinline__ void next(const BatchDesc* __restrict__ desc, int nlat) {
    if (++tx < ntx) return;
    tx = 0;
    if (++y < ny) return;
    y = 0;
    if (++z < nz) return;
    z = 0;
    if (lat + 1 < nlat) load(desc, lat + 1);
  }
};

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

template <class L, int COLL, class S, bool FORCE, int XT>
__global__ void __launch_bounds__(TmaShape<XT, true>::kThreads)
    k_batch_tma(const BatchTmaArgs a) {
  using T = typename S::T;
  using Sh = TmaShape<XT, true>;
  static_assert(sizeof(typename S::R) == 4, "the batched pipeline runs the packed FP32 arithmetic");
  constexpr int HT = 16 / (int)sizeof(T);  // halo (elements)
  constexpr int SLOT = XT + 2 * HT;        // elements per plane slot
  constexpr bool ADJ = sizeof(T) == 2;     // adjacent node pairs (see k_step_tma)
  extern __shared__ __align__(128) unsigned char smem[];
  const BatchDesc* __restrict__ desc = a.desc;
  const int ST = a.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + ST;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + ST);
  T* ring = reinterpret_cast<T*>(smem + 128 * ((2 * ST * 8 + 4 + 127) / 128));
  // Q plane slots, then per plane two HT-element side slots (unaligned wraps)
  constexpr long long stage_elems = (long long)L::Q * SLOT + (long long)L::Q * 2 * HT;
  int* err = &a.bar->err;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_addr(full + s), 1);
      mbar_init(smem_addr(empty + s), Sh::kConsumerWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t_begin = (int)(((long long)a.ntiles * blockIdx.x) / gridDim.x);
  const int t_end = (int)(((long long)a.ntiles * (blockIdx.x + 1)) / gridDim.x);
  const unsigned full_mask = 0xffffffffu;
  // ring position, running across steps (producer: next stage to fill;
  // consumers: next stage to read)
  int s = 0;
  uint32_t u = 0;
  long long issued = 0;  // producer: tiles issued so far

  for (int step = 0; step < a.nsteps; ++step) {
    const char* srcb = ((a.parity0 + step) & 1) ? a.B : a.A;
    char* dstb = ((a.parity0 + step) & 1) ? a.A : a.B;
    bool ok = true;
    BatchWalk w;
    if (t_begin < t_end) w.seek(desc, a.nlat, t_begin);
    if (warp == 0) {
      // -------------------------------------------------------- producer
      for (int t = t_begin; t < t_end; ++t, w.next(desc, a.nlat)) {
        if (u > 0 && !mbar_wait_warp(smem_addr(empty + s), (u - 1) & 1u, abort_flag, err,
                                     a.timeout_ns)) {
          ok = false;
          break;
        }
        const int x0 = w.tx * XT;
        const int xe = min(x0 + XT, w.nx);
        const int nxr = (w.nx + HT - 1) / HT * HT;  // row end rounded into the pitch padding
        const int lo = max(x0 - HT, 0);
        const int hi = min(xe + HT, nxr);
        const bool aligned = (w.nx % HT) == 0;
        const bool lwrap = w.per0 && aligned && x0 == 0;
        const bool rwrap = w.per0 && aligned && xe == w.nx;
        const bool lwrap_u = w.per0 && !aligned && x0 == 0;   // side slot copies
        const bool rwrap_u = w.per0 && !aligned && xe == w.nx;
        const uint32_t main_bytes = (uint32_t)(hi - lo) * sizeof(T);
        constexpr uint32_t halo_bytes = (uint32_t)HT * sizeof(T);
        const int i = lane;
        int ys = 0, zs = 0;
        bool wall = false;
        if (i < L::Q) {
          int ey = 0, ez = 0;
#pragma unroll
          for (int k = 0; k < L::Q; ++k)
            if (k == i) {
              ey = L::cy(k);
              ez = L::cz(k);
            }
          ys = w.y - ey;
          zs = w.z - ez;
          if (ys < 0 || ys >= w.ny) {
            if (w.per1) ys = ys < 0 ? ys + w.ny : ys - w.ny;
            else wall = true;
          }
          if (zs < 0 || zs >= w.nz) {
            if (w.per2) zs = zs < 0 ? zs + w.nz : zs - w.nz;
            else wall = true;
          }
        }
        const unsigned walls = __ballot_sync(full_mask, i < L::Q && wall);
        const uint32_t fb = smem_addr(full + s);
        if (lane == 0) {
          const uint32_t nwrap =
              (uint32_t)(L::Q - __popc(walls)) * ((lwrap || lwrap_u ? 1u : 0u) + (rwrap || rwrap_u ? 1u : 0u));
          mbar_arrive_expect_tx(fb, main_bytes * L::Q + nwrap * halo_bytes);
        }
        __syncwarp();
        if (i < L::Q) {
          const T* base = reinterpret_cast<const T*>(srcb + w.off);
          T* slot = ring + s * stage_elems + i * SLOT;  // slot[k] holds x = x0 - HT + k
          const int pi = wall ? opp_dyn<L>(i) : i;
          const long long r = wall ? ((long long)w.z * w.ny + w.y) : ((long long)zs * w.ny + ys);
          const T* rowp = base + pi * w.plane + r * w.pitch;
          bulk_g2s(smem_addr(slot + (lo - (x0 - HT))), rowp + lo, main_bytes, fb);
          if (!wall) {
            if (lwrap) bulk_g2s(smem_addr(slot), rowp + w.nx - HT, halo_bytes, fb);
            if (rwrap) bulk_g2s(smem_addr(slot + HT + (w.nx - x0)), rowp, halo_bytes, fb);
            // side slots: [0, HT) the aligned chunk holding x = nx - 1, [HT, 2 HT) x = 0..HT-1
            T* side = ring + s * stage_elems + (long long)L::Q * SLOT + i * 2 * HT;
            if (lwrap_u) bulk_g2s(smem_addr(side), rowp + (w.nx - 1) / HT * HT, halo_bytes, fb);
            if (rwrap_u) bulk_g2s(smem_addr(side + HT), rowp, halo_bytes, fb);
          }
        }
        ++issued;
        if (++s == ST) {
          s = 0;
          ++u;
        }
      }
    } else {
      // -------------------------------------------------------- consumers
      constexpr int NPT = 2;
      const int ct = threadIdx.x - 32;
      int jn[NPT];
      jn[0] = ADJ ? 2 * ct : ct;
      jn[1] = ADJ ? 2 * ct + 1 : ct + XT / 2;
      for (int t = t_begin; t < t_end; ++t, w.next(desc, a.nlat)) {
        if (!mbar_wait_warp(smem_addr(full + s), u & 1u, abort_flag, err, a.timeout_ns)) {
          ok = false;
          break;
        }
        const int x0 = w.tx * XT;
        const int wdt = min(XT, w.nx - x0);
        const T* st = ring + s * stage_elems;
        const long long own = ((long long)w.z * w.ny + w.y) * w.pitch;
        const T* src = reinterpret_cast<const T*>(srcb + w.off);
        T* dst = reinterpret_cast<T*>(dstb + w.off);
        const bool anywall = (!w.per1 && (w.y == 0 || w.y == w.ny - 1)) ||
                             (L::D == 3 && !w.per2 && (w.z == 0 || w.z == w.nz - 1));
        // tile touches a row end at an x wall (per-element path), or an
        // unaligned periodic row end (fast path, the end nodes then take their
        // wrap neighbours from the side slots)
        const bool rowend = x0 == 0 || x0 + XT >= w.nx;
        const bool xedge = rowend && !w.per0;
        const bool uwrap = rowend && w.per0 && (w.nx % HT) != 0;
        bool act[NPT];
#pragma unroll
        for (int n = 0; n < NPT; ++n) act[n] = jn[n] < wdt;
        F2 g[L::Q];
        if (!anywall && !xedge) {
#pragma unroll
          for (int i = 0; i < L::Q; ++i) {
            const T* slot = st + i * SLOT + HT - L::cx(i);
            if constexpr (ADJ) {
              if (L::cx(i) == 0) {
                float a0, a1;
                S::dec2(*reinterpret_cast<const uint32_t*>(slot + jn[0]), a0, a1);
                g[i] = F2{a0, a1};
              } else {
                g[i] = F2{S::dec(slot[jn[0]]), S::dec(slot[jn[1]])};
              }
            } else {
              g[i] = F2{S::dec(slot[jn[0]]), S::dec(slot[jn[1]])};
            }
          }
          if (uwrap) {
            const int jend = w.nx - 1 - x0;  // the row's last node, if in this tile
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
              const int ex = L::cx(i);
              if (ex == 0) continue;
              const T* side = st + (long long)L::Q * SLOT + i * 2 * HT;
              const T* src_w = ex == 1 ? side + (w.nx - 1) % HT : side + HT;
#pragma unroll
              for (int n = 0; n < NPT; ++n) {
                const bool end = ex == 1 ? (x0 + jn[n] == 0) : (jn[n] == jend);
                if (end) {
                  if (n == 0) g[i].x = S::dec(*src_w);
                  else g[i].y = S::dec(*src_w);
                }
              }
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < L::Q; ++i) {
            const int ex = L::cx(i);
            const T* slot = st + i * SLOT + HT;
            int ys = w.y - L::cy(i), zs = w.z - L::cz(i);
            bool wallrow = false;
            if (ys < 0 || ys >= w.ny) {
              if (w.per1) ys = ys < 0 ? ys + w.ny : ys - w.ny;
              else wallrow = true;
            }
            if (zs < 0 || zs >= w.nz) {
              if (w.per2) zs = zs < 0 ? zs + w.nz : zs - w.nz;
              else wallrow = true;
            }
            float v[NPT];
#pragma unroll
            for (int n = 0; n < NPT; ++n) {
              const int j = jn[n];
              const int x = x0 + j;
              const bool leaves = (ex == 1 && x == 0) || (ex == -1 && x == w.nx - 1);
              if (wallrow) {
                v[n] = S::dec(slot[j]);
              } else if (leaves && !w.per0) {
                // halfway bounce-back at an x wall: the node's own opposite population
                v[n] = act[n] ? S::dec(ldcg_elem(src + L::opp(i) * w.plane + own + x)) : 0.f;
              } else if (leaves && (w.nx % HT) != 0) {
                // unaligned periodic wrap: from the plane's side slots
                const T* side = st + (long long)L::Q * SLOT + i * 2 * HT;
                v[n] = S::dec(ex == 1 ? side[(w.nx - 1) % HT] : side[HT]);
              } else {
                v[n] = S::dec(slot[j - ex]);
              }
            }
            g[i] = F2{v[0], v[1]};
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(empty + s));
        if (++s == ST) {
          s = 0;
          ++u;
        }
        const unsigned bad = collide_v<L, COLL, FORCE, F2>(g, desc[w.lat].cf);
        const bool anybad = (act[0] && (bad & 1u)) || (act[1] && (bad & 2u));
        T* op = dst + own + x0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
          if constexpr (ADJ) {
            if (act[1]) {
              *reinterpret_cast<uint32_t*>(op + jn[0]) = S::enc2(g[i].x, g[i].y);
            } else if (act[0]) {
              op[jn[0]] = S::enc(g[i].x);
            }
          } else {
            if (act[0]) op[jn[0]] = S::enc(g[i].x);
            if (act[1]) op[jn[1]] = S::enc(g[i].y);
          }
          op += w.plane;
        }
        record_bad(a.flags + w.lat, a.step0 + (unsigned int)step, anybad);
      }
    }
    // ---- end of step: the whole block, then the whole grid
    if (!ok) *abort_flag = 1;
    __syncthreads();
    if (*abort_flag) {
      if (warp == 0 && lane == 0) {
        // let every issued copy land before the block's shared memory is released
        const long long k0 = issued > ST ? issued - ST : 0;
        for (long long kk = k0; kk < issued; ++kk)
          mbar_wait(smem_addr(full + (int)(kk % ST)), (uint32_t)((kk / ST) & 1), abort_flag, err,
                    a.timeout_ns, false);
      }
      return;
    }
    if (step + 1 < a.nsteps) {
      fence_proxy_async_global();
      if (!grid_sync(a.bar, a.expected, a.timeout_ns)) return;
      fence_proxy_async_global();
    }
  }
}

}  // namespace lbm
