// dispatch.h -- host-side launch descriptors and the per-(lattice, storage)
// operation tables that each translation unit exports.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

struct GeoH {
  int nx, ny, nz;
  int pitch;
  long long plane;
  int per[3];
};

struct Variant {
  int nv;  // nodes per thread along x
  int bx;  // threads per block along x (multiple of 32)
  int by;  // rows per block
};

struct StepLaunch {
  GeoH g;
  int collision;  // 0 TRT, 1 TRT-RLB, 2 P-TRT (BGK / RLB mapped by the caller)
  double rho0, cp, cm, hg, F[3];
  const void* src;
  void* dst;
  const uint8_t* mask;
  unsigned int* flag;
  unsigned int step;
  int layout;     // 0 A/B, 1 AA
  int parity;     // AA: 0 even (local) step, 1 odd (neighbour) step
  Variant v;
  cudaStream_t stream;
};

struct AuxLaunch {
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
  double rho0, cp, cm, hg, F[3];
  long long off;  // byte offset of the lattice in each population arena
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
  // persistent batched kernel (cooperative launch) and its occupancy
  cudaError_t (*batch)(const BatchLaunch&);
  int (*batch_blocks_per_sm)(int collision, int threads);
};

const Ops* ops_d2q9_f64();
const Ops* ops_d2q9_f32();
const Ops* ops_d2q9_f16();
const Ops* ops_d2q9_bf16();
const Ops* ops_d3q19_f64();
const Ops* ops_d3q19_f32();
const Ops* ops_d3q19_f16();
const Ops* ops_d3q19_bf16();

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
cudaError_t diag_sums(const DiagLaunch&);
cudaError_t diag_l2(const DiagLaunch&);
cudaError_t copy_ceiling(const void* src, void* dst, size_t bytes, cudaStream_t st);

}  // namespace lbm
