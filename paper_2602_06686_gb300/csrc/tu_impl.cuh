// tu_impl.cuh -- instantiates the fused update and the auxiliary kernels for one
// (lattice, storage) pair; included by the step_<lattice>_<storage>.cu files.
#pragma once
#include "dispatch.h"
#include "kernels.cuh"
#include "aa.cuh"
#include "batch.cuh"
#include "tma.cuh"
#include "batch_tma.cuh"
#include "aa_tma.cuh"

namespace lbm {

// Shifted third-order equilibrium df_eq_i = f_eq_i - w_i rho0 (Eq. feq).
template <class L, typename R>
__device__ __forceinline__ void feq_shifted(R drho, R ux, R uy, R uz, R (&out)[L::Q], R rho0) {
  const R rho = rho0 + drho;
  const R usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const R eu = R(L::cx(i)) * ux + R(L::cy(i)) * uy + R(L::cz(i)) * uz;
    out[i] = R(L::w(i)) *
             (drho + rho * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * usq +
                            R(4.5) * eu * (eu * eu - usq)));
  }
}

__device__ __forceinline__ int wrap_or_wall(int s, int n, int per, bool& wall) {
  if (s < 0 || s >= n) {
    if (per) return s < 0 ? s + n : s - n;
    wall = true;
  }
  return s;
}

// Storage slot that carries f_i(x, t) at the start of a step (A/B layout, and AA
// after an even number of steps is handled in aa.cuh): slot (i, x - e_i), or
// (ibar, x) when x - e_i is solid or beyond a non-periodic edge.
template <class L>
__device__ __forceinline__ long long ab_slot(const Geo& G, const uint8_t* mask, int x, int y, int z,
                                             int i) {
  bool wall = false;
  const int xs = wrap_or_wall(x - L::cx(i), G.nx, G.per[0], wall);
  const int ys = wrap_or_wall(y - L::cy(i), G.ny, G.per[1], wall);
  const int zs = wrap_or_wall(z - L::cz(i), G.nz, G.per[2], wall);
  if (!wall && mask && mask[((long long)zs * G.ny + ys) * G.nx + xs]) wall = true;
  if (wall) return L::opp(i) * G.plane + ((long long)z * G.ny + y) * G.pitch + x;
  return i * G.plane + ((long long)zs * G.ny + ys) * G.pitch + xs;
}

template <class L>
__device__ __forceinline__ long long state_slot(const Geo& G, const uint8_t* mask, int layout,
                                                int parity, int x, int y, int z, int i) {
  if (layout == 1) return aa_state_slot<L>(G, mask, parity, x, y, z, i);
  return ab_slot<L>(G, mask, x, y, z, i);
}

// The per-node helper kernels run on a grid of (lattice row, x block): row
// r = z * ny + y is blockIdx.x, x = blockIdx.y * blockDim.x + threadIdx.x, so
// no thread divides a 64-bit node index.
struct RowNode {
  int x, y, z;
  long long n;
  bool valid;
  __device__ __forceinline__ RowNode(const Geo& G) {
    const int r = blockIdx.x;
    x = blockIdx.y * blockDim.x + threadIdx.x;
    y = r % G.ny;
    z = r / G.ny;
    n = (long long)r * G.nx + x;
    valid = x < G.nx;
  }
};

// Open boundaries of the square-cylinder benchmark (Sec. 3.4, D2Q9), applied
// to the shifted pre-collision populations g of node x as gathered with x
// non-periodic (a population from beyond either x edge then holds the node's
// own opposite slot):
//   inlet  (x = 0): bounce-back from a wall moving with (u_in, 0) adds
//          6 w_i rho0 u_in to every population with e_x = +1;
//   outlet (x = nx - 1): Zou-He, density rho_out and zero transverse velocity:
//          u_x = (sum_{e_x=0} f + 2 sum_{e_x=+1} f) / rho_out - 1 and, for e_x = -1,
//          f_i = f_ibar + 6 w_i rho_out e_x u_x - (e_y / 2)(f_{+y} - f_{-y}).
// In shifted variables the rest weights cancel: sum_{e_x=0} w + 2 sum_{e_x=+1} w = 1.
template <class L, typename R>
__device__ __forceinline__ void open_fix(int x, int nx, R (&g)[L::Q], R rho0, R u_in, R rho_out) {
  if (x == 0) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      if (L::cx(i) == 1) g[i] += R(6.0 * L::w(i)) * rho0 * u_in;
  }
  if (x == nx - 1) {
    R s0 = R(0), sp = R(0), gyp = R(0), gym = R(0);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      if (L::cx(i) == 0) s0 += g[i];
      if (L::cx(i) == 1) sp += g[i];
      if (L::cx(i) == 0 && L::cy(i) == 1 && L::cz(i) == 0) gyp = g[i];
      if (L::cx(i) == 0 && L::cy(i) == -1 && L::cz(i) == 0) gym = g[i];
    }
    const R ux = (s0 + R(2) * sp + rho0 - rho_out) / rho_out;
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      if (L::cx(i) == -1)
        g[i] = g[L::opp(i)] - R(6.0 * L::w(i)) * rho_out * ux - R(0.5 * L::cy(i)) * (gyp - gym);
  }
}

// One fused update with the open boundaries (A/B layout, one node per thread,
// grid of (row, x block) as the helper kernels).
template <class L, int COLL, class S>
__global__ void __launch_bounds__(256) k_step_open(const StepArgs<typename S::R> a, int fix,
                                                   typename S::R u_in, typename S::R rho_out) {
  using R = typename S::R;
  using T = typename S::T;
  const Geo& G = a.g;
  const RowNode q(G);
  if (!q.valid || (a.mask && a.mask[q.n])) return;
  const T* __restrict__ src = static_cast<const T*>(a.src);
  T* __restrict__ dst = static_cast<T*>(a.dst);
  R g[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) g[i] = S::dec(src[ab_slot<L>(G, a.mask, q.x, q.y, q.z, i)]);
  if (fix) open_fix<L, R>(q.x, G.nx, g, a.c.rho0, u_in, rho_out);
  const bool bad = collide_v<L, COLL, true, R>(g, a.c) != 0u;
  const long long own = ((long long)q.z * G.ny + q.y) * G.pitch + q.x;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) dst[i * G.plane + own] = S::enc(g[i]);
  record_bad(a.flag, a.step, bad);
}

// ---- Scheme II forcing (Eq. source_simple, Eq. Gi), two launches per step.
// The cubic correction G_i needs d_g Phi_abg of the pre-collision state, whose
// only non-zero entries are d_a (rho u_a^3); a node's derivative needs its
// neighbours' rho and u at the same time level, which the fused pull kernel of
// one node does not have.  So k_phi first stores Phi_a = rho u_a^3 of every
// fluid node ([D][N], arithmetic precision R), then k_step_s2 gathers, takes
// the differences, collides with the F_i projection in place of the Guo
// source and adds G_i.  Differences along axis a: central where both
// neighbours are fluid nodes (a periodic axis wraps), one-sided where one is
// solid or beyond a non-periodic edge, zero where both are.
template <class L, class S>
__global__ void __launch_bounds__(256) k_phi(const StepArgs<typename S::R> a, int layout,
                                             int parity, typename S::R* phi) {
  using R = typename S::R;
  using T = typename S::T;
  const Geo& G = a.g;
  const RowNode q(G);
  if (!q.valid || (a.mask && a.mask[q.n])) return;
  const T* __restrict__ src = static_cast<const T*>(a.src);
  R drho = R(0), j[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const R v = S::dec(src[state_slot<L>(G, a.mask, layout, parity, q.x, q.y, q.z, i)]);
    drho += v;
    if (L::cx(i)) j[0] += R(L::cx(i)) * v;
    if (L::cy(i)) j[1] += R(L::cy(i)) * v;
    if (L::cz(i)) j[2] += R(L::cz(i)) * v;
  }
  const R rho = a.c.rho0 + drho;
  const R inv = R(1) / rho;
  const long long N = (long long)G.nx * G.ny * G.nz;
#pragma unroll
  for (int d = 0; d < L::D; ++d) {
    const R u = (j[d] + a.c.Fh[d]) * inv;
    phi[d * N + q.n] = rho * u * u * u;
  }
}

// The step with the Scheme II source.  a.c carries no symmetric Guo terms
// (fe = fu = 0), so collide_v leaves f_eq + (1 - w+) R2 + (1 - w-) R3 plus the
// antisymmetric force content F_i/2 + (1 - w-) F_i/2, which is what
// (1 - w+) R1 + (1 - w+/2) F_i + (1 - w-) F_i/2 amounts to; then
//   G_i = gk w_i (sum_a e_ia^2 D_a - (1/3) sum_a D_a),  gk = -(1 - w+/2) / (6 cs^6) = -4.5 (1 - w+/2),
// i.e. -(1 - w+/2) w_i H2_i:dPhi / (6 cs^6) for the diagonal dPhi = diag(D_a).
template <class L, int COLL, bool FORCE, class S>
__global__ void __launch_bounds__(256) k_step_s2(const StepArgs<typename S::R> a,
                                                 const typename S::R* __restrict__ phi,
                                                 typename S::R gk) {
  using R = typename S::R;
  using T = typename S::T;
  const Geo& G = a.g;
  const RowNode q(G);
  if (!q.valid || (a.mask && a.mask[q.n])) return;
  const T* __restrict__ src = static_cast<const T*>(a.src);
  T* __restrict__ dst = static_cast<T*>(a.dst);
  R g[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) g[i] = S::dec(src[ab_slot<L>(G, a.mask, q.x, q.y, q.z, i)]);
  R Dg[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int d = 0; d < L::D; ++d) Dg[d] = phi_grad<L, R>(G, a.mask, phi, d, q.x, q.y, q.z, q.n);
  const bool bad = collide_v<L, COLL, FORCE, R>(g, a.c) != 0u;
  const R third = (Dg[0] + Dg[1] + Dg[2]) * R(1.0 / 3.0);
  const long long own = ((long long)q.z * G.ny + q.y) * G.pitch + q.x;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    R h = -third;
    if (L::cx(i)) h += Dg[0];
    if (L::cy(i)) h += Dg[1];
    if (L::cz(i)) h += Dg[2];
    dst[i * G.plane + own] = S::enc(g[i] + gk * R(L::w(i)) * h);
  }
  record_bad(a.flag, a.step, bad);
}

// The Scheme II update on the AA layout, in place as aa_node: the node reads
// its slot set through aa_state_slot and writes f*_i + G_i back into it.
template <class L, int COLL, bool FORCE, class S>
__global__ void __launch_bounds__(256) k_step_s2_aa(const StepArgs<typename S::R> a, int parity,
                                                    const typename S::R* __restrict__ phi,
                                                    typename S::R gk) {
  using R = typename S::R;
  using T = typename S::T;
  const Geo& G = a.g;
  const RowNode q(G);
  if (!q.valid || (a.mask && a.mask[q.n])) return;
  T* buf = static_cast<T*>(a.dst);
  R g[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    g[i] = S::dec(buf[aa_state_slot<L>(G, a.mask, parity, q.x, q.y, q.z, i)]);
  R Dg[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int d = 0; d < L::D; ++d) Dg[d] = phi_grad<L, R>(G, a.mask, phi, d, q.x, q.y, q.z, q.n);
  const bool bad = collide_v<L, COLL, FORCE, R>(g, a.c) != 0u;
  const R third = (Dg[0] + Dg[1] + Dg[2]) * R(1.0 / 3.0);
  const long long own = ((long long)q.z * G.ny + q.y) * G.pitch + q.x;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    R h = -third;
    if (L::cx(i)) h += Dg[0];
    if (L::cy(i)) h += Dg[1];
    if (L::cz(i)) h += Dg[2];
    const long long slot = parity == 0 ? L::opp(i) * G.plane + own
                                       : aa_odd_dst<L>(G, a.mask, q.x, q.y, q.z, i);
    buf[slot] = S::enc(g[i] + gk * R(L::w(i)) * h);
  }
  record_bad(a.flag, a.step, bad);
}

template <class L, class S>
__global__ void __launch_bounds__(256) k_init_eq(Geo G, const uint8_t* mask, int layout, int parity,
                                                 typename S::T* pop, const double* rho,
                                                 const double* u, double rho0) {
  using R = typename S::R;
  const long long N = (long long)G.nx * G.ny * G.nz;
  const RowNode q(G);
  if (!q.valid || (mask && mask[q.n])) return;
  const long long n = q.n;
  R f[L::Q];
  const R ux = R(u[n]), uy = R(u[N + n]), uz = L::D == 3 ? R(u[2 * N + n]) : R(0);
  feq_shifted<L, R>(R(rho[n] - rho0), ux, uy, uz, f, R(rho0));
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    pop[state_slot<L>(G, mask, layout, parity, q.x, q.y, q.z, i)] = S::enc(f[i]);
}

template <class L, class S>
__global__ void __launch_bounds__(256) k_set_pop(Geo G, const uint8_t* mask, int layout, int parity,
                                                 typename S::T* pop, const double* f, double rho0) {
  const long long N = (long long)G.nx * G.ny * G.nz;
  const RowNode q(G);
  if (!q.valid || (mask && mask[q.n])) return;
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    pop[state_slot<L>(G, mask, layout, parity, q.x, q.y, q.z, i)] =
        S::enc(typename S::R(f[i * N + q.n] - L::w(i) * rho0));
}

// mode 0: decoded populations f [Q][N]; mode 1: rho [N] and u [D][N] (FP64).
template <class L, class S>
__global__ void __launch_bounds__(256) k_get(Geo G, const uint8_t* mask, int layout, int parity,
                                             const typename S::T* pop, double rho0, double Fx,
                                             double Fy, double Fz, int mode, double* out0,
                                             double* out1, OpenBC open) {
  const long long N = (long long)G.nx * G.ny * G.nz;
  const RowNode q(G);
  if (!q.valid) return;
  const long long n = q.n;
  const bool solid = mask && mask[n];
  double g[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
    g[i] = solid ? 0.0 : double(S::dec(pop[state_slot<L>(G, mask, layout, parity, q.x, q.y, q.z, i)]));
  if (open.on && !solid) open_fix<L, double>(q.x, G.nx, g, rho0, open.u_in, open.rho_out);
  if (mode == 0) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) out0[i * N + n] = g[i] + L::w(i) * rho0;
  } else {
    double drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      drho += g[i];
      jx += L::cx(i) * g[i];
      jy += L::cy(i) * g[i];
      jz += L::cz(i) * g[i];
    }
    const double rho = rho0 + drho;
    out0[n] = rho;
    out1[n] = solid ? 0.0 : (jx + 0.5 * Fx) / rho;
    out1[N + n] = solid ? 0.0 : (jy + 0.5 * Fy) / rho;
    if (L::D == 3) out1[2 * N + n] = solid ? 0.0 : (jz + 0.5 * Fz) / rho;
  }
}

// ---- diagnostics (two passes and a fixed-order reduction of block partials)
//
// Per node, rho and u are formed in the arithmetic precision R of the update
// (FP32 for FP32/FP16/BF16 storage, FP64 for FP64), from the shifted
// populations as the collision forms them; every sum over nodes is carried in
// FP64 across threads and blocks.  Within a thread, FP32 terms are first
// accumulated with an error-free transformation (TwoSum, Knuth): the running
// sum s and its rounding error c together carry the exact sum of the terms to
// within about 2^-48 relative, so nothing is lost before the FP64 stage, and a
// thread converts to FP64 once instead of once per node (FP64 throughput on
// GB300 is about 1/60 of FP32).  Blocks own contiguous row ranges, so the
// result is deterministic.
template <typename R>
struct CompSum {
  R s = R(0), c = R(0);
  __device__ __forceinline__ void add(R v) {
    if constexpr (sizeof(R) == 8) {
      s += v;
    } else {
      const R t = __fadd_rn(s, v);
      const R bp = __fsub_rn(t, s);
      const R e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
      c = __fadd_rn(c, e);
      s = t;
    }
  }
  __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of K values into partials[blockIdx.x * 8 + k0 + k] (256 threads).
template <int K>
__device__ __forceinline__ void block_partials(const double (&acc)[K], double* partials, int k0) {
  __shared__ double sh[8][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double v = warp_sum_d(acc[k]);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w][threadIdx.x];
    partials[blockIdx.x * 8 + k0 + threadIdx.x] = t;
  }
}

__device__ __forceinline__ void block_rows(const Geo& G, int& r0, int& r1) {
  const long long rows = (long long)G.ny * G.nz;
  r0 = (int)(rows * blockIdx.x / gridDim.x);
  r1 = (int)(rows * (blockIdx.x + 1) / gridDim.x);
}

// Pass 1: drho and u into the field scratch (R precision; solid nodes u = 0),
// and the partial sums of mass, momentum, kinetic energy and the flag.
template <class L, class S>
__global__ void __launch_bounds__(256) k_diag_fields(Geo G, const uint8_t* mask, int layout,
                                                     int parity, const typename S::T* pop,
                                                     double rho0d, typename S::R Fhx,
                                                     typename S::R Fhy, typename S::R Fhz,
                                                     typename S::R* fld, double* partials,
                                                     OpenBC open) {
  using R = typename S::R;
  const long long N = (long long)G.nx * G.ny * G.nz;
  const R rho0 = R(rho0d);
  int r0, r1;
  block_rows(G, r0, r1);
  CompSum<R> sm, sx, sy, sz, sk;
  long long cnt = 0;
  bool bad = false;
  // A/B layout without a mask: the source row of every plane is fixed for a
  // row, so it is resolved once per row instead of once per node and plane
  const bool rowwise = layout == 0 && mask == nullptr;
  int y = r0 % G.ny, z = r0 / G.ny;
  for (int r = r0; r < r1; ++r) {
    const long long own = ((long long)z * G.ny + y) * G.pitch;
    const typename S::T* rowp[L::Q];
    unsigned wallrows = 0u;
    if (rowwise) {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        int ys, zs;
        bool wall;
        tma_source_row<L>(G, i, y, z, ys, zs, wall);
        rowp[i] = wall ? pop + L::opp(i) * G.plane + own
                       : pop + i * G.plane + ((long long)zs * G.ny + ys) * G.pitch;
        if (wall) wallrows |= 1u << i;
      }
    }
    for (int x = threadIdx.x; x < G.nx; x += blockDim.x) {
      const long long n = (long long)r * G.nx + x;
      if (mask && mask[n]) {
        fld[n] = R(0);
#pragma unroll
        for (int a = 0; a < L::D; ++a) fld[(1 + a) * N + n] = R(0);
        continue;
      }
      R gq[L::Q];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        R g;
        if (rowwise) {
          if (wallrows & (1u << i)) {
            g = S::dec(rowp[i][x]);  // beyond a wall: the node's own opposite slot
          } else {
            int xs = x - L::cx(i);
            if (xs < 0 || xs >= G.nx) {
              if (G.per[0]) {
                xs = xs < 0 ? xs + G.nx : xs - G.nx;
                g = S::dec(rowp[i][xs]);
              } else {
                g = S::dec(pop[L::opp(i) * G.plane + own + x]);
              }
            } else {
              g = S::dec(rowp[i][xs]);
            }
          }
        } else {
          g = S::dec(pop[state_slot<L>(G, mask, layout, parity, x, y, z, i)]);
        }
        gq[i] = g;
      }
      if (open.on) open_fix<L, R>(x, G.nx, gq, rho0, R(open.u_in), R(open.rho_out));
      R drho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const R g = gq[i];
        drho += g;
        if (L::cx(i) == 1) jx += g;
        if (L::cx(i) == -1) jx -= g;
        if (L::cy(i) == 1) jy += g;
        if (L::cy(i) == -1) jy -= g;
        if (L::cz(i) == 1) jz += g;
        if (L::cz(i) == -1) jz -= g;
      }
      const R rho = rho0 + drho;
      const R inv = R(1) / rho;
      const R ux = (jx + Fhx) * inv, uy = (jy + Fhy) * inv, uz = L::D == 3 ? (jz + Fhz) * inv : R(0);
      fld[n] = drho;
      fld[N + n] = ux;
      fld[2 * N + n] = uy;
      if (L::D == 3) fld[3 * N + n] = uz;
      sm.add(drho);
      sx.add(rho * ux);
      sy.add(rho * uy);
      sz.add(rho * uz);
      sk.add(R(0.5) * rho * (ux * ux + uy * uy + uz * uz));
      ++cnt;
      bad |= !isfinite(rho) || !(rho > R(0)) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz);
    }
    if (++y == G.ny) {
      y = 0;
      ++z;
    }
  }
  const double acc[8] = {double(cnt) * rho0d + sm.value(), sx.value(), sy.value(), sz.value(),
                         sk.value(), 0.0, bad ? 1.0 : 0.0, 0.0};
  block_partials<8>(acc, partials, 0);
}

// Pass 2: enstrophy 1/2 |curl u|^2 with second-order central differences
// (across a periodic axis the neighbour wraps; across a non-periodic edge or
// at a solid node it counts as u = 0), into partial slot 5.
template <typename R, int D>
__global__ void __launch_bounds__(256) k_diag_enstrophy(Geo G, const uint8_t* mask, const R* fld,
                                                        double* partials) {
  const long long N = (long long)G.nx * G.ny * G.nz;
  const R* u = fld + N;
  int r0, r1;
  block_rows(G, r0, r1);
  CompSum<R> se;
  int y = r0 % G.ny, z = r0 / G.ny;
  for (int r = r0; r < r1; ++r) {
    for (int x = threadIdx.x; x < G.nx; x += blockDim.x) {
      const long long n = (long long)r * G.nx + x;
      if (mask && mask[n]) continue;
      R du[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) du[a][b] = R(0);
#pragma unroll
      for (int b = 0; b < D; ++b) {
        R val[2][3];
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
          int c3[3] = {x, y, z};
          const int ext = b == 0 ? G.nx : (b == 1 ? G.ny : G.nz);
          c3[b] += sgn ? 1 : -1;
          bool zero = false;
          if (c3[b] < 0 || c3[b] >= ext) {
            if (G.per[b]) c3[b] = c3[b] < 0 ? c3[b] + ext : c3[b] - ext;
            else zero = true;
          }
          const long long m = zero ? 0 : ((long long)c3[2] * G.ny + c3[1]) * G.nx + c3[0];
          if (!zero && mask && mask[m]) zero = true;
#pragma unroll
          for (int a = 0; a < 3; ++a) val[sgn][a] = (zero || a >= D) ? R(0) : u[a * N + m];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) du[a][b] = R(0.5) * (val[1][a] - val[0][a]);
      }
      const R wx = du[2][1] - du[1][2], wy = du[0][2] - du[2][0], wz = du[1][0] - du[0][1];
      se.add(R(0.5) * (wx * wx + wy * wy + wz * wz));
    }
    if (++y == G.ny) {
      y = 0;
      ++z;
    }
  }
  const double acc[1] = {se.value()};
  block_partials<1>(acc, partials, 5);
}

// Force on the solid nodes by momentum exchange (Sec. 3.4): with halfway
// bounce-back from resting solid nodes every link from a fluid node x_f to a
// solid neighbour x_f + e_i returns f*_i(x_f) as f_ibar(x_f), so it transfers
// 2 e_i f*_i(x_f); f* is the collision of the current pre-collision state (the
// force of the coming streaming step).  Neighbours beyond a non-periodic edge
// are walls, not part of the body.  Partial sums per block into slots 0..2.
template <class L, int COLL, class S>
__global__ void __launch_bounds__(256) k_momentum(Geo G, const uint8_t* mask, int layout,
                                                  int parity, const typename S::T* pop,
                                                  const CoefV<typename S::R> c, OpenBC open,
                                                  double* partials) {
  using R = typename S::R;
  int r0, r1;
  block_rows(G, r0, r1);
  double fx = 0.0, fy = 0.0, fz = 0.0;
  int y = r0 % G.ny, z = r0 / G.ny;
  for (int r = r0; r < r1; ++r) {
    for (int x = threadIdx.x; x < G.nx; x += blockDim.x) {
      const long long n = (long long)r * G.nx + x;
      if (!mask || mask[n]) continue;
      unsigned links = 0u;
#pragma unroll
      for (int i = 1; i < L::Q; ++i) {
        bool out = false;
        const int xd = aa_wrap(x + L::cx(i), G.nx, G.per[0], out);
        const int yd = aa_wrap(y + L::cy(i), G.ny, G.per[1], out);
        const int zd = aa_wrap(z + L::cz(i), G.nz, G.per[2], out);
        if (!out && mask[((long long)zd * G.ny + yd) * G.nx + xd]) links |= 1u << i;
      }
      if (!links) continue;
      R g[L::Q];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) g[i] = S::dec(pop[state_slot<L>(G, mask, layout, parity, x, y, z, i)]);
      if (open.on) open_fix<L, R>(x, G.nx, g, c.rho0, R(open.u_in), R(open.rho_out));
      collide_v<L, COLL, true, R>(g, c);
#pragma unroll
      for (int i = 1; i < L::Q; ++i) {
        if (!(links & (1u << i))) continue;
        const double fs = 2.0 * (double(g[i]) + L::w(i) * double(c.rho0));
        fx += L::cx(i) * fs;
        fy += L::cy(i) * fs;
        fz += L::cz(i) * fs;
      }
    }
    if (++y == G.ny) {
      y = 0;
      ++z;
    }
  }
  const double acc[8] = {fx, fy, fz, 0.0, 0.0, 0.0, 0.0, 0.0};
  block_partials<8>(acc, partials, 0);
}

template <class L, class S>
struct TU {
  using R = typename S::R;
  using T = typename S::T;

  static Geo geo(const GeoH& h) {
    Geo g;
    g.nx = h.nx;
    g.ny = h.ny;
    g.nz = h.nz;
    g.pitch = h.pitch;
    g.plane = h.plane;
    for (int a = 0; a < 3; ++a) g.per[a] = h.per[a];
    return g;
  }

  static StepArgs<R> args(const StepLaunch& s) {
    StepArgs<R> a;
    a.g = geo(s.g);
    a.c = coef_cast<R>(s.c);
    a.src = s.src;
    a.dst = s.dst;
    a.mask = s.mask;
    a.flag = s.flag;
    a.step = s.step;
    return a;
  }

  template <int COLL, int NV, bool MASK>
  static cudaError_t go(const StepLaunch& s) {
    const dim3 block(s.v.bx, s.v.by, 1);
    const int chunks = (s.g.nx + NV - 1) / NV;
    const dim3 grid((chunks + s.v.bx - 1) / s.v.bx, (s.g.ny + s.v.by - 1) / s.v.by, s.g.nz);
    if (s.layout == 1) {
      if constexpr (NV != 1) {
        return cudaErrorInvalidValue;  // the AA update runs one node per thread
      } else {
        if (s.parity == 0)
          k_step_aa_even<L, COLL, S, NV, MASK><<<grid, block, 0, s.stream>>>(args(s));
        else
          k_step_aa_odd<L, COLL, S, NV, MASK><<<grid, block, 0, s.stream>>>(args(s));
      }
    } else {
      k_step_ab<L, COLL, S, NV, MASK><<<grid, block, 0, s.stream>>>(args(s));
    }
    return cudaGetLastError();
  }

  // ---- pipelined bulk-copy kernel (kind 1)
  static constexpr bool kPack = sizeof(R) == 4;
  // D3Q27 compiles fewer tile widths (256 and 384 packed, 128 FP64): its
  // 27-plane kernels are the slowest to compile.
  static constexpr bool kOneTile = L::Q == 27;
  // register kernels: at most 2 nodes per thread on D3Q27 (54 populations in
  // flight per thread already)
  static constexpr int kMaxNV = L::Q == 27 ? 2 : 8;
  static constexpr int kTile27 = kPack ? 256 : 128;
  // Packed D3Q27 also offers 384.  Where nx is a multiple of 384 (the 384^3
  // Taylor-Green) 256-wide tiles leave every second tile of a row half empty,
  // a quarter of the consumer threads idle, and the four-node FP16 update is
  // bound by its consumer warps (166 registers each), not by bytes: 384-wide
  // tiles ran it at 0.87 of the measured HBM peak against 0.67 on GB300
  // (FP32, closer to its bytes: 0.90 against 0.88).
  static constexpr bool kWide27 = kOneTile && kPack;
  static bool tma_width_ok(int X) {
    if (kOneTile) return X == kTile27 || (kWide27 && X == 384);
    return kPack ? (X == 256 || X == 384 || X == 512) : (X == 128 || X == 192 || X == 256);
  }
  static size_t tma_smem(int X, int stages) {
    const int H = 16 / (int)sizeof(T);
    if (!tma_width_ok(X) || stages < 2) return 0;
    const size_t head = 128 * ((2 * (size_t)stages * 8 + 4 + 127) / 128);
    return head + (size_t)stages * L::Q * (size_t)(X + 2 * H) * sizeof(T);
  }

  template <int COLL, bool FORCE, int XT, int MODE = 0>
  static cudaError_t go_tma_x(const StepLaunch& s) {
    using Sh = TmaShape<XT, kPack>;
    TmaArgs<R> a;
    a.g = geo(s.g);
    a.c = coef_cast<R>(s.c);
    a.src = s.src;
    a.dst = s.dst;
    a.flag = s.flag;
    a.err = s.err;
    a.step = s.step;
    a.ntx = (s.g.nx + XT - 1) / XT;
    a.stages = s.v.stages;
    const long long ntiles = (long long)a.ntx * s.g.ny * s.g.nz;
    if (ntiles >= (1LL << 31)) return cudaErrorInvalidValue;
    a.ntiles = (int)ntiles;
    a.timeout_ns = s.wait_ns > 0 ? s.wait_ns : 2000000000LL;
    a.extra_tx = s.extra_tx;
    a.phi = s.phi;
    a.gk = R(0);
    if (MODE == 2) {
      CoefV<double> c = s.c;  // the F_i projection: no symmetric Guo terms
      for (int i = 0; i < kQMax; ++i) c.fe[i] = c.fu[i] = 0.0;
      a.c = coef_cast<R>(c);
      a.gk = R(-4.5 * (1.0 - 0.5 * (1.0 - s.c.cp)));
    }
    size_t smem = tma_smem(XT, a.stages);
    if (MODE == 2 && smem > 0) smem += (size_t)a.stages * TmaPhi<L, R, XT>::kBytes;
    // 0: A/B, 1: AA even step, 2: AA odd step, 3: A/B with the staged bulk
    // stores (MODE 0 only, packed arithmetic); MODE 1 / 2: A/B only
    int kind = MODE != 0 ? 0 : (s.layout == 1 ? 1 + (s.parity & 1) : 0);
    if (kind == 0 && MODE == 0 && kPack && s.v.by == 1) kind = 3;
    if (kind == 0 && MODE == 0 && kPack && sizeof(T) == 2 && s.v.nv == 4) kind = 4;
    if (kind == 2 && smem > 0) smem += aa_odd_smem(L::Q, (int)sizeof(T), XT);
    if (kind == 3 && smem > 0) smem += tma_bs_smem(L::Q, (int)sizeof(T), XT);
    if (smem == 0 || smem > 227 * 1024 || a.stages > 8) return cudaErrorInvalidValue;
    void (*kern)(TmaArgs<R>);
    int threads = Sh::kThreads;
    if constexpr (MODE != 0) {
      kern = &k_step_tma<L, COLL, S, FORCE, kPack, XT, MODE>;
    } else {
      kern = kind == 0   ? &k_step_tma<L, COLL, S, FORCE, kPack, XT>
             : kind == 1 ? &k_step_aa_tma<L, COLL, S, FORCE, kPack, XT, false>
             : kind == 2 ? &k_step_aa_tma<L, COLL, S, FORCE, kPack, XT, true>
             : kind == 3 ? &k_step_tma<L, COLL, S, FORCE, kPack, XT, kPack ? 3 : 0>
                         : &k_step_tma<L, COLL, S, FORCE, kPack, XT, kPack && sizeof(T) == 2 ? 4 : 0>;
      if (kind == 2 || kind == 3) threads = TmaShape<XT, kPack, 1>::kThreads;
      if (kind == 4) threads = TmaShape<XT, kPack, 0, kPack && sizeof(T) == 2 ? 4 : 0>::kThreads;
    }
    // per instantiation and kind: the shared-memory opt-in (once) and the
    // resident blocks per SM for each ring depth (cached)
    static bool attr_set[5] = {false, false, false, false, false};
    static int per_sm_cache[5][9] = {};
    if (!attr_set[kind]) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      if (e != cudaSuccess) return e;
      attr_set[kind] = true;
    }
    int per_sm = per_sm_cache[kind][a.stages];
    if (per_sm == 0) {
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
      if (e != cudaSuccess) return e;
      if (per_sm < 1) return cudaErrorInvalidConfiguration;
      per_sm_cache[kind][a.stages] = per_sm;
    }
    const int resident = s.v.bx > 0 && s.v.bx < per_sm ? s.v.bx : per_sm;
    long long blocks = (long long)resident * (s.sms > 0 ? s.sms : 1);
    if (blocks > a.ntiles) blocks = a.ntiles;
    kern<<<(unsigned)blocks, threads, smem, s.stream>>>(a);
    return cudaGetLastError();
  }

  template <int COLL, bool FORCE>
  static cudaError_t go_tma(const StepLaunch& s) {
    if constexpr (kOneTile) {
      if (s.v.X == kTile27) return go_tma_x<COLL, FORCE, kTile27>(s);
      if constexpr (kWide27) {
        if (s.v.X == 384) return go_tma_x<COLL, FORCE, 384>(s);
      }
    } else if constexpr (kPack) {
      switch (s.v.X) {
        case 256:
          return go_tma_x<COLL, FORCE, 256>(s);
        case 384:
          return go_tma_x<COLL, FORCE, 384>(s);
        case 512:
          return go_tma_x<COLL, FORCE, 512>(s);
      }
    } else {
      switch (s.v.X) {
        case 128:
          return go_tma_x<COLL, FORCE, 128>(s);
        case 192:
          return go_tma_x<COLL, FORCE, 192>(s);
        case 256:
          return go_tma_x<COLL, FORCE, 256>(s);
      }
    }
    return cudaErrorInvalidValue;
  }

  template <int COLL>
  static cudaError_t tma_coll(const StepLaunch& s) {
    return s.force ? go_tma<COLL, true>(s) : go_tma<COLL, false>(s);
  }

  static cudaError_t step_tma(const StepLaunch& s) {
    if (s.mask != nullptr) return cudaErrorInvalidValue;
    switch (s.collision) {
      case C_TRT:
        return tma_coll<C_TRT>(s);
      case C_TRT_RLB:
        return tma_coll<C_TRT_RLB>(s);
      case C_P_TRT:
        return tma_coll<C_P_TRT>(s);
    }
    return cudaErrorInvalidValue;
  }

  template <int NV>
  static cudaError_t step_nv(const StepLaunch& s) {
    const bool m = s.mask != nullptr;
    switch (s.collision) {
      case C_TRT:
        return m ? go<C_TRT, NV, true>(s) : go<C_TRT, NV, false>(s);
      case C_TRT_RLB:
        return m ? go<C_TRT_RLB, NV, true>(s) : go<C_TRT_RLB, NV, false>(s);
      case C_P_TRT:
        return m ? go<C_P_TRT, NV, true>(s) : go<C_P_TRT, NV, false>(s);
    }
    return cudaErrorInvalidValue;
  }

  template <int COLL>
  static cudaError_t go_open(const StepLaunch& s) {
    const dim3 grid((unsigned)((long long)s.g.ny * s.g.nz), (unsigned)((s.g.nx + 255) / 256));
    k_step_open<L, COLL, S><<<grid, 256, 0, s.stream>>>(args(s), s.open.fix, R(s.open.u_in),
                                                        R(s.open.rho_out));
    return cudaGetLastError();
  }
  static cudaError_t step_open(const StepLaunch& s) {
    if (s.layout != 0) return cudaErrorInvalidValue;
    switch (s.collision) {
      case C_TRT:
        return go_open<C_TRT>(s);
      case C_TRT_RLB:
        return go_open<C_TRT_RLB>(s);
      case C_P_TRT:
        return go_open<C_P_TRT>(s);
    }
    return cudaErrorInvalidValue;
  }

  template <int COLL>
  static cudaError_t go_momentum(const AuxLaunch& a, const CoefV<double>& c, double* partials,
                                 int blocks) {
    k_momentum<L, COLL, S><<<blocks, 256, 0, a.stream>>>(geo(a.g), a.mask, a.layout, a.parity,
                                                         static_cast<const T*>(a.pop),
                                                         coef_cast<R>(c), a.open, partials);
    return cudaGetLastError();
  }
  static cudaError_t momentum(const AuxLaunch& a, int collision, const CoefV<double>& c,
                              double* partials, int blocks, double* out) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (collision) {
      case C_TRT:
        e = go_momentum<C_TRT>(a, c, partials, blocks);
        break;
      case C_TRT_RLB:
        e = go_momentum<C_TRT_RLB>(a, c, partials, blocks);
        break;
      case C_P_TRT:
        e = go_momentum<C_P_TRT>(a, c, partials, blocks);
        break;
    }
    if (e != cudaSuccess) return e;
    return reduce_partials(partials, blocks, out, a.stream);
  }

  // Scheme II on the pipelined kernel (no solid mask, rows of whole 16-byte
  // units): the tile width and ring depth of the chosen pipelined variant, the
  // update's ring reduced until it holds the staged Phi rows within 200 KB;
  // under a register variant the widest tile with a two-deep ring (four for FP64).
  template <int COLL, bool FORCE, int XT>
  static cudaError_t go_s2_tma_x(const StepLaunch& s, int st) {
    StepLaunch t = s;
    t.v = Variant{1, 0, 0, 0, XT, st};
    cudaError_t e = go_tma_x<C_TRT, FORCE, XT, 1>(t);
    if (e != cudaSuccess) return e;
    while (st > 2 && tma_smem(XT, st) + (size_t)st * TmaPhi<L, R, XT>::kBytes > 200 * 1024) --st;
    t.v.stages = st;
    return go_tma_x<COLL, FORCE, XT, 2>(t);
  }
  template <int COLL, bool FORCE>
  static cudaError_t go_s2_tma(const StepLaunch& s) {
    const int X = s.v.kind == 1 ? s.v.X : (kPack ? 512 : 128);
    const int st = s.v.kind == 1 ? s.v.stages : (kPack ? 2 : 4);
    if constexpr (kPack) {
      switch (X) {
        case 256:
          return go_s2_tma_x<COLL, FORCE, 256>(s, st);
        case 384:
          return go_s2_tma_x<COLL, FORCE, 384>(s, st);
        case 512:
          return go_s2_tma_x<COLL, FORCE, 512>(s, st);
      }
    } else {
      switch (X) {
        case 128:
          return go_s2_tma_x<COLL, FORCE, 128>(s, st);
        case 192:
          return go_s2_tma_x<COLL, FORCE, 192>(s, st);
        case 256:
          return go_s2_tma_x<COLL, FORCE, 256>(s, st);
      }
    }
    return cudaErrorInvalidValue;
  }
  static bool s2_tma_ok(const StepLaunch& s) {
    constexpr int H = 16 / (int)sizeof(T);
    // the producer warp copies one plane or Phi row per lane
    constexpr bool lanes = L::Q + TmaPhi<L, R, 128>::kRows <= 32;
    return lanes && s.mask == nullptr && s.g.nx % H == 0 && s.g.nx >= 2 * H;
  }

  template <int COLL, bool FORCE>
  static cudaError_t go_s2(const StepLaunch& s) {
    if constexpr (L::Q + TmaPhi<L, R, 128>::kRows <= 32) {
      if (s.layout == 0 && s2_tma_ok(s)) return go_s2_tma<COLL, FORCE>(s);
    }
    const dim3 grid((unsigned)((long long)s.g.ny * s.g.nz), (unsigned)((s.g.nx + 255) / 256));
    R* phi = static_cast<R*>(s.phi);
    StepArgs<R> a = args(s);
    k_phi<L, S><<<grid, 256, 0, s.stream>>>(a, s.layout, s.parity, phi);
    CoefV<double> c = s.c;  // the F_i projection: no symmetric Guo terms
    for (int i = 0; i < kQMax; ++i) c.fe[i] = c.fu[i] = 0.0;
    a.c = coef_cast<R>(c);
    const R gk = R(-4.5 * (1.0 - 0.5 * (1.0 - s.c.cp)));
    if (s.layout == 1)
      k_step_s2_aa<L, COLL, FORCE, S><<<grid, 256, 0, s.stream>>>(a, s.parity, phi, gk);
    else
      k_step_s2<L, COLL, FORCE, S><<<grid, 256, 0, s.stream>>>(a, phi, gk);
    return cudaGetLastError();
  }
  template <int COLL>
  static cudaError_t s2_coll(const StepLaunch& s) {
    return s.force ? go_s2<COLL, true>(s) : go_s2<COLL, false>(s);
  }
  static cudaError_t step_s2(const StepLaunch& s) {
    if (s.phi == nullptr || s.open.on) return cudaErrorInvalidValue;
    switch (s.collision) {
      case C_TRT:
        return s2_coll<C_TRT>(s);
      case C_TRT_RLB:
        return s2_coll<C_TRT_RLB>(s);
      case C_P_TRT:
        return s2_coll<C_P_TRT>(s);
    }
    return cudaErrorInvalidValue;
  }

  static cudaError_t step(const StepLaunch& s) {
    if (s.scheme == 2) return step_s2(s);
    if (s.open.on) return step_open(s);
    if (s.v.kind == 1) return step_tma(s);
    switch (s.v.nv) {
      case 1:
        return step_nv<1>(s);
      case 2:
        if constexpr (2 * sizeof(T) <= 16) return step_nv<2>(s);
        break;
      case 4:
        if constexpr (4 * sizeof(T) <= 16 && 4 <= kMaxNV) return step_nv<4>(s);
        break;
      case 8:
        if constexpr (8 * sizeof(T) <= 16 && 8 <= kMaxNV) return step_nv<8>(s);
        break;
    }
    return cudaErrorInvalidValue;
  }

  static dim3 aux_grid(const GeoH& g) {
    return dim3((unsigned)((long long)g.ny * g.nz), (unsigned)((g.nx + 255) / 256));
  }

  static cudaError_t diag(const AuxLaunch& a, void* fields, double* partials, int blocks, double* out) {
    const Geo G = geo(a.g);
    R* fld = static_cast<R*>(fields);
    k_diag_fields<L, S><<<blocks, 256, 0, a.stream>>>(G, a.mask, a.layout, a.parity,
                                                      static_cast<const T*>(a.pop), a.rho0,
                                                      R(0.5 * a.F[0]), R(0.5 * a.F[1]),
                                                      R(0.5 * a.F[2]), fld, partials, a.open);
    k_diag_enstrophy<R, L::D><<<blocks, 256, 0, a.stream>>>(G, a.mask, fld, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce_partials(partials, blocks, out, a.stream);
  }

  static cudaError_t init_eq(const AuxLaunch& a, const double* rho, const double* u) {
    k_init_eq<L, S><<<aux_grid(a.g), 256, 0, a.stream>>>(geo(a.g), a.mask, a.layout, a.parity,
                                                         static_cast<T*>(a.pop), rho, u, a.rho0);
    return cudaGetLastError();
  }
  static cudaError_t set_pop(const AuxLaunch& a, const double* f) {
    k_set_pop<L, S><<<aux_grid(a.g), 256, 0, a.stream>>>(geo(a.g), a.mask, a.layout, a.parity,
                                                         static_cast<T*>(a.pop), f, a.rho0);
    return cudaGetLastError();
  }
  static cudaError_t get_pop(const AuxLaunch& a, double* f) {
    k_get<L, S><<<aux_grid(a.g), 256, 0, a.stream>>>(geo(a.g), a.mask, a.layout, a.parity,
                                                     static_cast<const T*>(a.pop), a.rho0,
                                                     a.F[0], a.F[1], a.F[2], 0, f, nullptr, a.open);
    return cudaGetLastError();
  }
  static cudaError_t macros(const AuxLaunch& a, double* rho, double* u) {
    k_get<L, S><<<aux_grid(a.g), 256, 0, a.stream>>>(geo(a.g), a.mask, a.layout, a.parity,
                                                     static_cast<const T*>(a.pop), a.rho0,
                                                     a.F[0], a.F[1], a.F[2], 1, rho, u, a.open);
    return cudaGetLastError();
  }

  template <int COLL>
  static void* batch_fn() {
    return reinterpret_cast<void*>(&k_batch<L, COLL, S>);
  }
  static void* batch_kernel(int coll) {
    switch (coll) {
      case C_TRT:
        return batch_fn<C_TRT>();
      case C_TRT_RLB:
        return batch_fn<C_TRT_RLB>();
      case C_P_TRT:
        return batch_fn<C_P_TRT>();
    }
    return nullptr;
  }
  static int batch_blocks_per_sm(int coll, int threads) {
    void* fn = batch_kernel(coll);
    int n = 0;
    if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0) != cudaSuccess)
      return 0;
    return n;
  }
  static cudaError_t batch(const BatchLaunch& b) {
    void* fn = batch_kernel(b.collision);
    if (!fn) return cudaErrorInvalidValue;
    BarrierWords* bar = static_cast<BarrierWords*>(b.bar);
    void* args[] = {(void*)&b.desc,  (void*)&b.tiles,    (void*)&b.ntiles, (void*)&b.A,
                    (void*)&b.B,     (void*)&b.nsteps,   (void*)&b.parity0, (void*)&b.step0,
                    (void*)&b.flags, (void*)&bar,        (void*)&b.expected, (void*)&b.timeout_ns};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b.blocks);
    cfg.blockDim = dim3(b.bx, b.by);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
  }

  // ---- pipelined persistent batched kernel (FP32 arithmetic storages)
  static size_t batch_tma_smem(int X, int stages) {
    const int H = 16 / (int)sizeof(T);
    if ((X != 128 && X != 256) || stages < 2) return 0;
    const size_t head = 128 * ((2 * (size_t)stages * 8 + 4 + 127) / 128);
    // per stage: Q plane slots and 2 HT-element side slots per plane
    return head + (size_t)stages * L::Q * (size_t)(X + 4 * H) * sizeof(T);
  }
  // Dynamic shared-memory limit set on the batched kernel: enough for the
  // deepest ring of the variant list (4 stages), and below the opt-in maximum
  // net of the kernel's static shared memory (grid barrier), so that graphs
  // captured with any listed depth stay launchable.
  static int batch_tma_smem_cap(int X) { return (int)batch_tma_smem(X, 4); }
  template <int COLL, bool FORCE>
  static void* batch_tma_kernel_cf(int X) {
    if constexpr (kPack) {
      if constexpr (!kOneTile) {
        if (X == 128) return (void*)&k_batch_tma<L, COLL, S, FORCE, 128>;
      }
      if (X == 256) return (void*)&k_batch_tma<L, COLL, S, FORCE, 256>;
    }
    return nullptr;
  }
  template <int COLL>
  static void* batch_tma_kernel_c(bool force, int X) {
    return force ? batch_tma_kernel_cf<COLL, true>(X) : batch_tma_kernel_cf<COLL, false>(X);
  }
  static void* batch_tma_kernel(int coll, bool force, int X) {
    switch (coll) {
      case C_TRT:
        return batch_tma_kernel_c<C_TRT>(force, X);
      case C_TRT_RLB:
        return batch_tma_kernel_c<C_TRT_RLB>(force, X);
      case C_P_TRT:
        return batch_tma_kernel_c<C_P_TRT>(force, X);
    }
    return nullptr;
  }
  static int batch_tma_blocks_per_sm(int coll, bool force, int X, int stages) {
    void* fn = batch_tma_kernel(coll, force, X);
    const size_t smem = batch_tma_smem(X, stages);
    if (!fn || smem == 0 || smem > 227 * 1024) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_tma_smem_cap(X)) !=
        cudaSuccess)
      return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 32 + X / 2, smem) != cudaSuccess) return 0;
    return n;
  }
  static cudaError_t batch_tma(const BatchLaunch& b) {
    void* fn = batch_tma_kernel(b.collision, b.force, b.X);
    const size_t smem = batch_tma_smem(b.X, b.stages);
    if (!fn || smem == 0 || smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_tma_smem_cap(b.X));
    if (e != cudaSuccess) return e;
    BatchTmaArgs a;
    a.desc = b.desc;
    a.nlat = b.nlat;
    a.ntiles = b.ntiles;
    a.A = b.A;
    a.B = b.B;
    a.nsteps = b.nsteps;
    a.parity0 = b.parity0;
    a.step0 = b.step0;
    a.flags = b.flags;
    a.bar = static_cast<BarrierWords*>(b.bar);
    a.expected = b.expected;
    a.timeout_ns = b.timeout_ns;
    a.stages = b.stages;
    void* args[] = {(void*)&a};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b.blocks);
    cfg.blockDim = dim3(32 + b.X / 2);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = b.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
  }

  static const Ops* ops() {
    static Ops o = [] {
      Ops r{};
      r.Q = L::Q;
      r.D = L::D;
      r.esize = sizeof(T);
      int n = 0;
      for (int nv = 1; nv <= kMaxNV; nv *= 2)
        if (nv * (int)sizeof(T) <= 16) r.nvs[n++] = nv;
      r.n_nv = n;
      r.step = &step;
      r.init_eq = &init_eq;
      r.set_pop = &set_pop;
      r.get_pop = &get_pop;
      r.macros = &macros;
      r.diag = &diag;
      r.momentum = &momentum;
      r.batch = &batch;
      r.batch_blocks_per_sm = &batch_blocks_per_sm;
      if (kPack) {
        r.batch_tma = &batch_tma;
        r.batch_tma_blocks_per_sm = &batch_tma_blocks_per_sm;
      }
      r.tma_smem = &tma_smem;
      return r;
    }();
    return &o;
  }
};

}  // namespace lbm

#define LBM_DEFINE_OPS(NAME, LAT, STORE) \
  namespace lbm {                        \
  const Ops* NAME() { return TU<LAT, STORE>::ops(); } \
  }
