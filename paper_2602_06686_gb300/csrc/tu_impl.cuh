// tu_impl.cuh -- instantiates the fused update and the auxiliary kernels for one
// (lattice, storage) pair; included by the step_<lattice>_<storage>.cu files.
#pragma once
#include "dispatch.h"
#include "kernels.cuh"
#include "aa.cuh"
#include "batch.cuh"
#include "tma.cuh"

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

template <class L, class S>
__global__ void k_init_eq(Geo G, const uint8_t* mask, int layout, int parity,
                          typename S::T* pop, const double* rho, const double* u, double rho0) {
  using R = typename S::R;
  const long long N = (long long)G.nx * G.ny * G.nz;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    if (mask && mask[n]) continue;
    const int x = n % G.nx, y = (n / G.nx) % G.ny, z = n / ((long long)G.nx * G.ny);
    R f[L::Q];
    const R ux = R(u[n]), uy = R(u[N + n]), uz = L::D == 3 ? R(u[2 * N + n]) : R(0);
    feq_shifted<L, R>(R(rho[n] - rho0), ux, uy, uz, f, R(rho0));
#pragma unroll
    for (int i = 0; i < L::Q; ++i) pop[state_slot<L>(G, mask, layout, parity, x, y, z, i)] = S::enc(f[i]);
  }
}

template <class L, class S>
__global__ void k_set_pop(Geo G, const uint8_t* mask, int layout, int parity,
                          typename S::T* pop, const double* f, double rho0) {
  const long long N = (long long)G.nx * G.ny * G.nz;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    if (mask && mask[n]) continue;
    const int x = n % G.nx, y = (n / G.nx) % G.ny, z = n / ((long long)G.nx * G.ny);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      pop[state_slot<L>(G, mask, layout, parity, x, y, z, i)] =
          S::enc(typename S::R(f[i * N + n] - L::w(i) * rho0));
  }
}

// mode 0: decoded populations f [Q][N]; mode 1: rho [N] and u [D][N].
template <class L, class S>
__global__ void k_get(Geo G, const uint8_t* mask, int layout, int parity, const typename S::T* pop,
                      double rho0, double Fx, double Fy, double Fz, int mode, double* out0,
                      double* out1) {
  const long long N = (long long)G.nx * G.ny * G.nz;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = n % G.nx, y = (n / G.nx) % G.ny, z = n / ((long long)G.nx * G.ny);
    const bool solid = mask && mask[n];
    double g[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      g[i] = solid ? 0.0 : double(S::dec(pop[state_slot<L>(G, mask, layout, parity, x, y, z, i)]));
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
  static bool tma_width_ok(int X) {
    return kPack ? (X == 256 || X == 384 || X == 512) : (X == 128 || X == 192 || X == 256);
  }
  static size_t tma_smem(int X, int stages) {
    const int H = 16 / (int)sizeof(T);
    if (!tma_width_ok(X) || stages < 2) return 0;
    const size_t head = 128 * ((2 * (size_t)stages * 8 + 4 + 127) / 128);
    return head + (size_t)stages * L::Q * (size_t)(X + 2 * H) * sizeof(T);
  }

  template <int COLL, bool FORCE, int XT>
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
    const size_t smem = tma_smem(XT, a.stages);
    if (smem == 0 || smem > 227 * 1024) return cudaErrorInvalidValue;
    auto kern = &k_step_tma<L, COLL, S, FORCE, kPack, XT>;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      if (e != cudaSuccess) return e;
      attr_set = true;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Sh::kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long blocks = (long long)per_sm * (s.sms > 0 ? s.sms : 1);
    if (blocks > a.ntiles) blocks = a.ntiles;
    kern<<<(unsigned)blocks, Sh::kThreads, smem, s.stream>>>(a);
    return cudaGetLastError();
  }

  template <int COLL, bool FORCE>
  static cudaError_t go_tma(const StepLaunch& s) {
    if constexpr (kPack) {
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
    if (s.mask != nullptr || s.layout != 0) return cudaErrorInvalidValue;
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

  static cudaError_t step(const StepLaunch& s) {
    if (s.v.kind == 1) return step_tma(s);
    switch (s.v.nv) {
      case 1:
        return step_nv<1>(s);
      case 2:
        if constexpr (2 * sizeof(T) <= 16) return step_nv<2>(s);
        break;
      case 4:
        if constexpr (4 * sizeof(T) <= 16) return step_nv<4>(s);
        break;
      case 8:
        if constexpr (8 * sizeof(T) <= 16) return step_nv<8>(s);
        break;
    }
    return cudaErrorInvalidValue;
  }

  static dim3 aux_grid(const GeoH& g) {
    const long long N = (long long)g.nx * g.ny * g.nz;
    long long b = (N + 255) / 256;
    if (b > 65536) b = 65536;
    return dim3((unsigned)b);
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
                                                     a.F[0], a.F[1], a.F[2], 0, f, nullptr);
    return cudaGetLastError();
  }
  static cudaError_t macros(const AuxLaunch& a, double* rho, double* u) {
    k_get<L, S><<<aux_grid(a.g), 256, 0, a.stream>>>(geo(a.g), a.mask, a.layout, a.parity,
                                                     static_cast<const T*>(a.pop), a.rho0,
                                                     a.F[0], a.F[1], a.F[2], 1, rho, u);
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

  static const Ops* ops() {
    static Ops o = [] {
      Ops r{};
      r.Q = L::Q;
      r.D = L::D;
      r.esize = sizeof(T);
      int n = 0;
      for (int nv = 1; nv <= 8; nv *= 2)
        if (nv * (int)sizeof(T) <= 16) r.nvs[n++] = nv;
      r.n_nv = n;
      r.step = &step;
      r.init_eq = &init_eq;
      r.set_pop = &set_pop;
      r.get_pop = &get_pop;
      r.macros = &macros;
      r.batch = &batch;
      r.batch_blocks_per_sm = &batch_blocks_per_sm;
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
