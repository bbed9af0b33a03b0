// aa_tma.cuh -- the in-place AA update (aa.cuh) fed by the bulk-copy pipeline
// of tma.cuh: one population buffer, read and written by the same launch.
//
// Even step (an even number of completed steps): node x reads its own slots
// (i, x) and writes f*_i(x) to (ibar, x).  The producer copies, per plane i,
// the tile's own row segment [x0, x0 + X) (no halo); consumers store to the
// opposite plane of the same row.
// Odd step: node x reads f_i(x, t) from slot (ibar, x - e_i) -- or (i, x) when
// x - e_i is beyond a non-periodic edge -- and writes f*_i(x) to (i, x + e_i) --
// or (ibar, x) when x + e_i is beyond one.  Per plane and tile that is one
// source row, (y - e_iy, z - e_iz) of plane ibar (or the own row of plane i at a
// wall), copied with the 16-byte halo exactly like the A/B pull, and one
// destination row, (y + e_iy, z + e_iz) of plane i shifted by e_ix.  Stored
// thread by thread, such a shifted row makes every warp store span two
// 128-byte lines, so the odd step stages the tile's destination rows in shared
// memory (row i holds destination x at element HT + x - x0) and a store warp
// (warp 1) writes each row's 16-byte aligned interior with one bulk
// shared-to-global copy and its few end elements one by one.  Values that
// leave the tile's window (the neighbour tile's first or last slot), wrap
// across a periodic row end or bounce at an x wall are stored directly by the
// consumer thread that holds the tile's first or last node.
//
// In place is race free: the slots node x reads in a step are exactly the slots
// it writes (its own set, disjoint from every other node's), every one of them
// has landed in shared memory before the node's values are stored (by its
// consumer or the store warp), and the halo elements a copy brings along that
// belong to other nodes are never used.  Masked lattices use the register
// kernels of aa.cuh.
#pragma once
#include "aa.cuh"
#include "dispatch.h"
#include "tma.cuh"

namespace lbm {

// Destination row of plane i for the odd step at tile row (y, z): the row
// offset (elements) of plane i shifted by e_iy, e_iz with the periodic wrap,
// or kAaWall when that row lies beyond a non-periodic wall.
constexpr long long kAaWall = -(1LL << 62);
__device__ __forceinline__ long long aa_row_delta(const Geo& G, int y, int z, int ey, int ez) {
  const long long pitch = G.pitch, zstride = (long long)G.ny * G.pitch;
  long long d = 0;
  if (ey == 1) d = y + 1 < G.ny ? pitch : (G.per[1] ? -(long long)(G.ny - 1) * pitch : kAaWall);
  if (ey == -1) d = y > 0 ? -pitch : (G.per[1] ? (long long)(G.ny - 1) * pitch : kAaWall);
  if (d == kAaWall) return d;
  if (ez == 1) {
    const long long e = z + 1 < G.nz ? zstride : (G.per[2] ? -(long long)(G.nz - 1) * zstride : kAaWall);
    return e == kAaWall ? e : d + e;
  }
  if (ez == -1) {
    const long long e = z > 0 ? -zstride : (G.per[2] ? (long long)(G.nz - 1) * zstride : kAaWall);
    return e == kAaWall ? e : d + e;
  }
  return d;
}

template <class L, int COLL, class S, bool FORCE, bool PACK, int XT, bool ODD>
__global__ void __launch_bounds__(TmaShape<XT, PACK, ODD ? 1 : 0>::kThreads,
                                  tma_min_blocks<L, S, ODD ? 3 : 0>())
    k_step_aa_tma(const TmaArgs<typename S::R> a) {
  using T = typename S::T;
  using R = typename S::R;
  using V = typename std::conditional<PACK, F2, R>::type;
  using Sh = TmaShape<XT, PACK, ODD ? 1 : 0>;
  constexpr int HT = 16 / (int)sizeof(T);
  constexpr int SLOT = XT + 2 * HT;
  extern __shared__ __align__(128) unsigned char smem[];
  const Geo& G = a.g;
  const int ST = a.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + ST;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + ST);
  T* ring = reinterpret_cast<T*>(smem + 128 * ((2 * ST * 8 + 4 + 127) / 128));
  constexpr long long stage_elems = (long long)L::Q * SLOT;
  // odd step: after the ring (128-byte aligned) the staging region of
  // aa_odd_smem: mbarriers ob_full[NB] / ob_free[NB], then NB staging buffers
  // of one row of SLOT elements per plane (tile k uses buffer k % NB)
  constexpr int NB = aa_odd_buffers(L::Q);
  constexpr long long kStageElems = ((long long)L::Q * SLOT * sizeof(T) + 127) / 128 * 128 / sizeof(T);
  unsigned char* oreg = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(ring + ST * stage_elems) + 127) & ~uintptr_t(127));
  uint64_t* ob_full = reinterpret_cast<uint64_t*>(oreg);
  uint64_t* ob_free = ob_full + NB;
  T* ostages = reinterpret_cast<T*>(oreg + 128);

  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(smem_addr(full + s), 1);
      mbar_init(smem_addr(empty + s), Sh::kConsumerWarps);
    }
    if (ODD) {
      for (int b = 0; b < NB; ++b) {
        mbar_init(smem_addr(ob_full + b), Sh::kConsumerWarps);
        mbar_init(smem_addr(ob_free + b), 1);
      }
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* buf = static_cast<T*>(a.dst);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    const unsigned full_mask = 0xffffffffu;
    TileWalk w(a.ntiles, a.ntx, G.ny);
    int k = 0;
    int s = 0;
    uint32_t u = 0;
    bool ok = true;
    for (; w.more(); w.next(), ++k) {
      if (u > 0 && !mbar_wait_warp(smem_addr(empty + s), (u - 1) & 1u, abort_flag, a.err,
                                   a.timeout_ns)) {
        ok = false;
        break;
      }
      const int y = w.y, z = w.z;
      const int x0 = w.tx * XT;
      const int xe = min(x0 + XT, G.nx);
      const int lo = ODD ? max(x0 - HT, 0) : x0;
      const int hi = ODD ? min(xe + HT, G.nx) : xe;
      const bool lwrap = ODD && G.per[0] && x0 == 0;
      const bool rwrap = ODD && G.per[0] && xe == G.nx;
      const uint32_t main_bytes = (uint32_t)(hi - lo) * sizeof(T);
      constexpr uint32_t halo_bytes = (uint32_t)HT * sizeof(T);
      int ys = y, zs = z;
      bool wall = false;
      const int i = lane;
      if (ODD && i < L::Q) tma_source_row_dyn<L>(G, i, y, z, ys, zs, wall);
      const unsigned walls = __ballot_sync(full_mask, i < L::Q && wall);
      const uint32_t fb = smem_addr(full + s);
      if (lane == 0) {
        const uint32_t nwrap =
            (uint32_t)(L::Q - __popc(walls)) * ((lwrap ? 1u : 0u) + (rwrap ? 1u : 0u));
        mbar_arrive_expect_tx(fb, main_bytes * L::Q + nwrap * halo_bytes + (uint32_t)a.extra_tx);
      }
      __syncwarp();
      if (i < L::Q) {
        T* slot = ring + s * stage_elems + i * SLOT;  // slot[k] holds x = x0 - HT + k
        // odd: plane ibar of the source row, or at a wall the own slot (i, x);
        // even: the own slot (i, x)
        const int pi = (ODD && !wall) ? opp_dyn<L>(i) : i;
        const long long r = wall ? ((long long)z * G.ny + y) : ((long long)zs * G.ny + ys);
        const T* rowp = buf + pi * G.plane + r * G.pitch;
        bulk_g2s(smem_addr(slot + (lo - (x0 - HT))), rowp + lo, main_bytes, fb);
        if (ODD && !wall) {
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

  if constexpr (ODD) {
    if (warp == 1) {
      // ---------------------------------------------------------- store warp
      // The staging rows of tile k hold the destinations [lo, hi) of every
      // plane (row i: destination x at element HT + x - x0).  Lane i writes
      // plane i: the 16-byte aligned interior by one bulk copy, the few
      // elements at either end one by one; then the rows are handed back.
      constexpr int VE = 16 / (int)sizeof(T);
      TileWalk w(a.ntiles, a.ntx, G.ny);
      for (int k = 0; w.more(); w.next(), ++k) {
        const int b = k % NB;
        if (!mbar_wait_warp(smem_addr(ob_full + b), (uint32_t)((k / NB) & 1), abort_flag, a.err,
                            a.timeout_ns))
          break;
        const T* ostage = ostages + b * kStageElems;
        if (lane < L::Q) {
          const int y = w.y, z = w.z;
          const int x0 = w.tx * XT;
          const int wdt = min(XT, G.nx - x0);
          const long long own = ((long long)z * G.ny + y) * G.pitch;
          int ex = 0, ey = 0, ez = 0;
#pragma unroll
          for (int kk = 0; kk < L::Q; ++kk)
            if (kk == lane) {
              ex = L::cx(kk);
              ey = L::cy(kk);
              ez = L::cz(kk);
            }
          const long long dr = aa_row_delta(G, y, z, ey, ez);
          const bool rw = dr == kAaWall;
          const int sh = rw ? 0 : ex;
          T* drow = buf + (rw ? (long long)opp_dyn<L>(lane) * G.plane + own
                              : (long long)lane * G.plane + own + dr);
          const T* orow = ostage + lane * SLOT + HT - x0;  // orow[x]: destination x
          const int lo = max(x0 + sh, x0), hi = min(min(x0 + wdt + sh, G.nx), x0 + XT);
          const int ca = min(hi, (lo + VE - 1) / VE * VE), cb = max(ca, hi / VE * VE);
          if (cb > ca) bulk_s2g(drow + ca, smem_addr(orow + ca), (uint32_t)((cb - ca) * sizeof(T)));
          for (int e = lo; e < ca; ++e) drow[e] = orow[e];
          for (int e = cb; e < hi; ++e) drow[e] = orow[e];
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

  // -------------------------------------------------------------- consumers
  constexpr int NPT = Sh::kNPT;
  constexpr bool ADJ = PACK && sizeof(T) == 2;
  const int ct = threadIdx.x - Sh::kBase;
  int jn[NPT];
  jn[0] = ADJ ? 2 * ct : ct;
  if (PACK) jn[NPT - 1] = ADJ ? 2 * ct + 1 : ct + XT / 2;
  TileWalk w(a.ntiles, a.ntx, G.ny);
  int s = 0;
  uint32_t u = 0;
  int kt = 0;  // tiles done by this block
  for (; w.more(); w.next()) {
    if (!mbar_wait_warp(smem_addr(full + s), u & 1u, abort_flag, a.err, a.timeout_ns)) break;
    const int y = w.y, z = w.z;
    const int x0 = w.tx * XT;
    const int wdt = min(XT, G.nx - x0);
    const T* st = ring + s * stage_elems;
    const long long own = ((long long)z * G.ny + y) * G.pitch;
    // odd step: does the tile touch a wall row / plane, or an x wall?
    const bool anywall = ODD && ((!G.per[1] && (y == 0 || y == G.ny - 1)) ||
                                 (L::D == 3 && !G.per[2] && (z == 0 || z == G.nz - 1)));
    const bool xwall = ODD && !G.per[0] && (x0 == 0 || x0 + XT >= G.nx);
    bool act[NPT];
#pragma unroll
    for (int n = 0; n < NPT; ++n) act[n] = jn[n] < wdt;
    V g[L::Q];
    if (!anywall && !xwall) {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const int sh = ODD ? L::cx(i) : 0;
        const T* slot = st + i * SLOT + HT - sh;
        if constexpr (ADJ) {
          if (sh == 0) {
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
            v[n] = S::dec(slot[j]);  // the own slot (i, x) was copied
          } else if (!G.per[0] && ((ex == 1 && x == 0) || (ex == -1 && x == G.nx - 1))) {
            // x - e_i beyond an x wall: the own slot (i, x), which only this node touches
            v[n] = act[n] ? S::dec(ldcg_elem(buf + i * G.plane + own + x)) : R(0);
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
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_addr(empty + s));
    if (++s == ST) {
      s = 0;
      ++u;
    }
    const unsigned bad = collide_v<L, COLL, FORCE, V>(g, a.c);
    bool anybad = act[0] && (bad & 1u);
    if (PACK) anybad = anybad || (act[NPT - 1] && (bad & 2u));
    R out[NPT];
    if constexpr (!ODD) {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        if constexpr (PACK) {
          out[0] = g[i].x;
          out[NPT - 1] = g[i].y;
        } else {
          out[0] = g[i];
        }
        // even: f*_i(x) into the opposite slot of the node's own row
        T* op = buf + L::opp(i) * G.plane + own + x0;
        if constexpr (ADJ) {
          if (act[NPT - 1]) *reinterpret_cast<uint32_t*>(op + jn[0]) = S::enc2(out[0], out[NPT - 1]);
          else if (act[0]) op[jn[0]] = S::enc(out[0]);
        } else {
#pragma unroll
          for (int n = 0; n < NPT; ++n)
            if (act[n]) op[jn[n]] = S::enc(out[n]);
        }
      }
    } else {
      // odd: f*_i(x) goes to slot (i, x + e_i), or to (ibar, x) where x + e_i is
      // beyond a wall.  Destination row deltas (elements) for e_y = +1 / -1 and
      // e_z = +1 / -1 with the periodic wrap folded in; kWall marks a wall.
      constexpr long long kWall = kAaWall;
      const long long pitch = G.pitch, zstride = (long long)G.ny * G.pitch;
      const long long yp = y + 1 < G.ny ? pitch : (G.per[1] ? -(long long)(G.ny - 1) * pitch : kWall);
      const long long ym = y > 0 ? -pitch : (G.per[1] ? (long long)(G.ny - 1) * pitch : kWall);
      long long zp = 0, zm = 0;
      if (L::D == 3) {
        zp = z + 1 < G.nz ? zstride : (G.per[2] ? -(long long)(G.nz - 1) * zstride : kWall);
        zm = z > 0 ? -zstride : (G.per[2] ? (long long)(G.nz - 1) * zstride : kWall);
      }
      // (1) staging buffer kt % NB is free once the store warp has read the
      // rows of tile kt - NB
      const int ob = kt % NB;
      if (kt >= NB && !mbar_wait_warp(smem_addr(ob_free + ob), (uint32_t)((kt / NB - 1) & 1), abort_flag,
                                      a.err, a.timeout_ns))
        break;
      T* ostage = ostages + ob * kStageElems;
      // (2) the staged values: staging row i holds destination x at element
      // HT + (x - x0), so each node's value lands at HT + j + sh_i with
      // sh_i = e_ix (0 beyond a wall)
      // a thread that holds the tile's first or last node may have values for
      // outside the tile's window or the row (wraps, x walls): stored directly
      bool tend = false;
#pragma unroll
      for (int n = 0; n < NPT; ++n) tend |= act[n] && (jn[n] == 0 || jn[n] == wdt - 1);
      if (!anywall && wdt == XT) {
        // no destination row lies beyond a wall (that needs a wall row) and
        // every node exists: fixed offsets, no per-plane test
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
          T* orow = ostage + i * SLOT + HT + L::cx(i);
          if constexpr (ADJ) {
            if (L::cx(i) == 0) {
              *reinterpret_cast<uint32_t*>(orow + jn[0]) = S::enc2(g[i].x, g[i].y);
            } else {
              orow[jn[0]] = S::enc(g[i].x);
              orow[jn[1]] = S::enc(g[i].y);
            }
          } else if constexpr (PACK) {
            orow[jn[0]] = S::enc(g[i].x);
            orow[jn[1]] = S::enc(g[i].y);
          } else {
            orow[jn[0]] = S::enc(g[i]);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
          if constexpr (PACK) {
            out[0] = g[i].x;
            out[NPT - 1] = g[i].y;
          } else {
            out[0] = g[i];
          }
          const int ex = L::cx(i);
          const long long dy = L::cy(i) == 1 ? yp : (L::cy(i) == -1 ? ym : 0);
          const long long dz = L::cz(i) == 1 ? zp : (L::cz(i) == -1 ? zm : 0);
          const bool rw = dy == kWall || dz == kWall;
          T* orow = ostage + i * SLOT + HT;
          bool staged = false;
          if constexpr (ADJ) {
            if (ex == 0) {  // the pair's word, 4-byte aligned (HT and jn[0] even)
              if (act[NPT - 1]) *reinterpret_cast<uint32_t*>(orow + jn[0]) = S::enc2(out[0], out[NPT - 1]);
              else if (act[0]) orow[jn[0]] = S::enc(out[0]);
              staged = true;
            }
          }
          if (!staged) {
            const int sh = rw ? 0 : ex;
#pragma unroll
            for (int n = 0; n < NPT; ++n)
              if (act[n]) orow[jn[n] + sh] = S::enc(out[n]);
          }
        }
      }
      // a thread that holds the tile's first or last node may have values for
      // outside the tile's window or the row (wraps, x walls): stored directly
      if (tend) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
          const int ex = L::cx(i);
          if (ex == 0) continue;
          if constexpr (PACK) {
            out[0] = g[i].x;
            out[NPT - 1] = g[i].y;
          } else {
            out[0] = g[i];
          }
          const long long dy = L::cy(i) == 1 ? yp : (L::cy(i) == -1 ? ym : 0);
          const long long dz = L::cz(i) == 1 ? zp : (L::cz(i) == -1 ? zm : 0);
          if (dy == kWall || dz == kWall) continue;
#pragma unroll
          for (int n = 0; n < NPT; ++n) {
            const int x = x0 + jn[n];
            const int xd = x + ex;
            if (!act[n] || (xd >= x0 && xd < min(x0 + XT, G.nx))) continue;
            if (xd >= 0 && xd < G.nx) {
              buf[i * G.plane + own + dy + dz + xd] = S::enc(out[n]);  // next / previous tile's window
            } else if (G.per[0]) {
              buf[i * G.plane + own + dy + dz + (xd < 0 ? xd + G.nx : xd - G.nx)] = S::enc(out[n]);
            } else {
              buf[L::opp(i) * G.plane + own + x] = S::enc(out[n]);  // x wall: own opposite slot
            }
          }
        }
      }
      // (3) hand the rows to the store warp (its bulk copies read them through
      // the async proxy)
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(ob_full + ob));
    }
    ++kt;
    record_bad(a.flag, a.step, anybad);
  }
}

}  // namespace lbm
