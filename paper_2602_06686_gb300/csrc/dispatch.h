// dispatch.h -- host-side launch descriptors and the per-(lattice, storage)
// operation tables that each translation unit exports.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "collide_v.cuh"

namespace lbm {

struct GeoH {
  int nx, ny, nz;
  int pitch;
  long long plane;
  int per[3];
};

struct Variant {
  int kind;    // 0: register kernel (one warp row per block row), 1: bulk-copy pipelined kernel
  int nv;      // kind 0: nodes per thread along x; kind 1: 4 for four nodes per consumer
               // thread (16-bit storage, A/B), else 0
  int bx;      // kind 0: threads per block along x (multiple of 32); kind 1: at most this
               // many resident blocks per SM (0: as many as fit)
  int by;      // kind 0: rows per block; kind 1: 1 for the staged bulk stores (A/B)
  int X;       // kind 1: tile width (nodes)
  int stages;  // kind 1: shared-memory ring depth
};

// Open boundaries of the square-cylinder benchmark (D2Q9, A/B, x non-periodic):
// a wall moving with (u_in, 0) half a spacing left of x = 0, and a Zou-He
// constant-density outlet (rho_out) at x = nx - 1.
// `fix` (step launches): apply the boundary rules to the gathered state; off
// for the first step after the state was written directly (lbm_init_equilibrium,
// lbm_set_populations), which holds f(t) as given, not a streamed state.
// For the helper kernels `on` already carries that condition.
struct OpenBC {
  int on, fix;
  double u_in, rho_out;
};

struct StepLaunch {
  OpenBC open;
  GeoH g;
  int collision;  // 0 TRT, 1 TRT-RLB, 2 P-TRT (BGK / RLB mapped by the caller)
  bool force;     // any force component non-zero
  CoefV<double> c;
  int* err;       // bounded-wait error word
  long long wait_ns;  // limit of each bounded wait (pipelined kernel)
  int extra_tx;       // test hook: bytes a stage waits for that never arrive
  int sms;        // multiprocessors of the device
  const void* src;
  void* dst;
  const uint8_t* mask;
  unsigned int* flag;
  unsigned int step;
  int layout;     // 0 A/B, 1 AA
  int parity;     // AA: 0 even (local) step, 1 odd (neighbour) step
  Variant v;
  // forcing: 1 Guo (Eq. source_guo), 2 simplified projection + G_i (Eq. source_simple,
  // Eq. Gi; two launches, phi = [D][N] values of the arithmetic precision)
  int scheme;
  void* phi;
  cudaStream_t stream;
};

struct AuxLaunch {
  OpenBC open;
  GeoH g;
  double rho0, F[3];
  void* pop;            // buffer holding the current state
  const uint8_t* mask;
  int layout;
  int parity;           // AA: parity of the number of completed steps
  cudaStream_t stream;
};

// Per-lattice descriptor and tile of the persistent batched kernel.
struct BatchDesc {
  GeoH g;
  CoefV<double> cd;
  CoefV<float> cf;
  long long off;  // byte offset of the lattice in each population arena
  int ntx;        // pipelined kernel: tiles per row at the variant's tile width
  int tile0;      // pipelined kernel: index of the lattice's first tile
};
struct BatchTile {
  int lat, x0, y0, z;
};
struct BatchLaunch {
  const BatchDesc* desc;
  const BatchTile* tiles;
  int ntiles;
  char* A;
  char* B;
  int nsteps;
  int parity0;          // 0: state in A, 1: state in B
  unsigned int step0;   // index of the first step (divergence records)
  unsigned int* flags;  // per-lattice divergence flags
  void* bar;            // BarrierWords
  unsigned int expected;
  long long timeout_ns;
  int collision;
  int bx, by, blocks;
  // pipelined variant (kind 1): tile width, ring depth, lattices, any force
  int kind, X, stages, nlat;
  bool force;
  cudaStream_t stream;
};

struct Ops {
  int Q, D, esize;
  // vector widths this storage supports for the fused kernel
  int nvs[4];
  int n_nv;
  cudaError_t (*step)(const StepLaunch&);
  cudaError_t (*init_eq)(const AuxLaunch&, const double* rho, const double* u);
  cudaError_t (*set_pop)(const AuxLaunch&, const double* f);
  cudaError_t (*get_pop)(const AuxLaunch&, double* f);
  cudaError_t (*macros)(const AuxLaunch&, double* rho, double* u);
  // FP64 diagnostics of the current state: drho and u staged in `fields` in the
  // arithmetic precision ((1 + D) * N values), block partials [blocks][8]
  // (blocks <= rows), the eight sums in out[8] (mass, momentum, kinetic energy,
  // enstrophy, flag, 0)
  cudaError_t (*diag)(const AuxLaunch&, void* fields, double* partials, int blocks, double* out);
  // force on the solid nodes by momentum exchange (sum over fluid-to-solid links
  // of 2 e_i f*_i), partials [blocks][8] (slots 0..2), out[8] (slots 0..2)
  cudaError_t (*momentum)(const AuxLaunch&, int collision, const CoefV<double>& c, double* partials,
                          int blocks, double* out);
  // persistent batched kernel (cooperative launch) and its occupancy
  cudaError_t (*batch)(const BatchLaunch&);
  int (*batch_blocks_per_sm)(int collision, int threads);
  // pipelined persistent batched kernel (FP32 arithmetic storages only; else null)
  cudaError_t (*batch_tma)(const BatchLaunch&);
  int (*batch_tma_blocks_per_sm)(int collision, bool force, int X, int stages);
  // shared-memory bytes of the pipelined kernel for a tile width and ring depth (0: unsupported)
  size_t (*tma_smem)(int X, int stages);
};

// Staging buffers of the pipelined AA kernel's odd step: two on D2Q9 (its
// short collision would otherwise wait for the store warp), one on the 3-D
// lattices (whose staging rows are large).
inline constexpr int aa_odd_buffers(int Q) { return Q == 9 ? 2 : 1; }

// Shared memory the odd step of the pipelined AA kernel needs beyond its ring:
// the mbarriers (padded to 128 bytes) and aa_odd_buffers staging buffers of one
// row per plane of X + 2 * (16 / esize) elements, each rounded to 128 bytes;
// plus 128 bytes of alignment slack for where the ring ends.
inline constexpr size_t aa_odd_smem(int Q, int esize, int X) {
  return 128 + 128 +
         (size_t)aa_odd_buffers(Q) *
             (((size_t)Q * (size_t)(X + 2 * (16 / esize)) * (size_t)esize + 127) / 128 * 128);
}

// Shared memory the staged bulk stores of the pipelined A/B kernel (MODE 3)
// need beyond its ring: 128 bytes of alignment slack, four mbarriers (padded to
// 128 bytes) and two staging buffers of Q rows of X elements, each rounded to
// 128 bytes.
inline constexpr size_t tma_bs_smem(int Q, int esize, int X) {
  return 128 + 128 + 2 * (((size_t)Q * (size_t)X * (size_t)esize + 127) / 128 * 128);
}

// Per-direction collision constants from the rates and the force (host, FP64).
template <class L>
inline void fill_coef(double rho0, double wp, double wm_run, int collision, const double F[3],
                      CoefV<double>* c) {
  *c = CoefV<double>{};
  c->rho0 = rho0;
  c->cp = 1.0 - wp;
  c->cm = 1.0 - wm_run;
  const double hg = 1.0 - 0.5 * wp;
  for (int a = 0; a < 3; ++a) {
    c->Fh[a] = 0.5 * F[a];
    c->F[a] = F[a];
  }
  for (int i = 0; i < L::Q; ++i) {
    const double eF = L::cx(i) * F[0] + L::cy(i) * F[1] + L::cz(i) * F[2];
    const double w = L::w(i);
    c->fe[i] = 9.0 * w * eF * hg;
    c->fu[i] = -3.0 * w * hg;
    c->fa[i] = collision == 1 ? 1.5 * w * eF : 1.5 * w * eF * (2.0 - wm_run);
  }
}

template <typename R>
inline CoefV<R> coef_cast(const CoefV<double>& d) {
  CoefV<R> c;
  c.rho0 = R(d.rho0);
  c.cp = R(d.cp);
  c.cm = R(d.cm);
  for (int a = 0; a < 3; ++a) {
    c.Fh[a] = R(d.Fh[a]);
    c.F[a] = R(d.F[a]);
  }
  for (int i = 0; i < kQMax; ++i) {
    c.fe[i] = R(d.fe[i]);
    c.fu[i] = R(d.fu[i]);
    c.fa[i] = R(d.fa[i]);
  }
  return c;
}

const Ops* ops_d2q9_f64();
const Ops* ops_d2q9_f32();
const Ops* ops_d2q9_f16();
const Ops* ops_d2q9_bf16();
const Ops* ops_d3q19_f64();
const Ops* ops_d3q19_f32();
const Ops* ops_d3q19_f16();
const Ops* ops_d3q19_bf16();
const Ops* ops_d3q27_f64();
const Ops* ops_d3q27_f32();
const Ops* ops_d3q27_f16();
const Ops* ops_d3q27_bf16();

// Generic FP64 reductions over macroscopic fields (diag.cu).
struct DiagLaunch {
  GeoH g;
  int D;
  const double* rho;   // [N]
  const double* u;     // [D][N]
  const double* uref;  // [D][N] for the L2 error, else null
  const uint8_t* mask;
  double* partials;    // [blocks][8]
  double* out;         // [8]
  int blocks;
  cudaStream_t stream;
};
// out[k] = sum over blocks of partials[b][k] in block order (slot 6: maximum).
cudaError_t reduce_partials(const double* partials, int blocks, double* out, cudaStream_t st);
cudaError_t diag_l2(const DiagLaunch&);
cudaError_t copy_ceiling(const void* src, void* dst, size_t bytes, cudaStream_t st);

}  // namespace lbm
