// noalloc.cu -- diagnostics for callers that cannot provide a scratch buffer.
//
// lbm_diagnostics needs the scratch buffer bound to a context: it writes the
// FP64 density and velocity fields there and then the per-block partial sums.
// Some callers cannot hand the library such a buffer: a host program whose
// device memory is entirely owned by another framework's pool, a plugin that
// is given population buffers but no right to allocate, or a monitoring tool
// attached to a running simulation that must not change its memory footprint.
// lbm_diagnostics_noalloc computes the same eight numbers for them without
// allocating anything: its working memory is the file-scope array below,
// created with the library and held by every GPU that loads it until the
// process exits.
//
// The array holds the staged fields of at most kNoAllocMaxNodes nodes (plus the
// block partials); larger lattices are rejected.  Nothing in it is
// read before the same call has written it, so it needs no clearing between
// calls; it keeps the contents of the last call.  All calls on a device share
// it, so calls whose work overlaps on the GPU (on different streams) race.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "internal.h"

using namespace lbm;

namespace {

constexpr long long kNoAllocMaxNodes = 1LL << 18;  // 262144 nodes, e.g. 512 x 512 or 64^3
constexpr int kNoAllocBlocks = 1024;               // block partials of the reduction
constexpr long long kNoAllocDoubles =
    4 * kNoAllocMaxNodes + (long long)kNoAllocBlocks * 8 + 32;  // rho, u[<=3], partials, result

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {nullptr};

// Device address of the array on the current device, looked up once per device
// (cudaGetSymbolAddress) with that device current.
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ctx_fail(LBM_ERR_CUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return ctx_fail(LBM_ERR_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      char buf[256];
      snprintf(buf, sizeof(buf), "cudaGetSymbolAddress of the static scratch failed: %s",
               cudaGetErrorString(e));
      return ctx_fail(LBM_ERR_CUDA, buf);
    }
    g_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ptr[dev];
  return LBM_OK;
}

// Turns the reduction's raw flag into 0/1 and stores the step counter.
__global__ void k_noalloc_finish(double* out, long long step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    out[6] = out[6] > 0.0 ? 1.0 : 0.0;
    out[7] = (double)step;
  }
}

const Ops* ops_for(int lattice, int storage) {
  static const Ops* (*table[3][4])() = {{ops_d2q9_f64, ops_d2q9_f32, ops_d2q9_f16, ops_d2q9_bf16},
                                       {ops_d3q19_f64, ops_d3q19_f32, ops_d3q19_f16, ops_d3q19_bf16},
                                       {ops_d3q27_f64, ops_d3q27_f32, ops_d3q27_f16, ops_d3q27_bf16}};
  return table[lattice][storage]();
}

}  // namespace

extern "C" int lbm_diagnostics_noalloc(const lbm_params* p, const void* pop_state,
                                       const uint8_t* solid_mask, long long steps_done, double* out,
                                       void* cuda_stream) {
  Plan pl;
  int rc = plan(p, &pl);
  if (rc) return rc;
  if (!pop_state || !out) return ctx_fail(LBM_ERR_ARG, "pop_state and out are required");
  if (steps_done < 0) return ctx_fail(LBM_ERR_ARG, "steps_done must be >= 0");
  if (pl.N > kNoAllocMaxNodes) {
    char buf[160];
    snprintf(buf, sizeof(buf),
             "lattice of %lld nodes exceeds the %lld-node limit of the static diagnostics scratch",
             pl.N, kNoAllocMaxNodes);
    return ctx_fail(LBM_ERR_ARG, buf);
  }
  double* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void* fields = base;  // drho [N] and u [D][N] in the arithmetic precision
  double* partials = base + 4 * kNoAllocMaxNodes;

  AuxLaunch a{};
  a.g = pl.g;
  a.rho0 = pl.p.rho0;
  for (int k = 0; k < 3; ++k) a.F[k] = pl.p.force[k];
  a.pop = const_cast<void*>(pop_state);
  a.mask = solid_mask;
  a.layout = pl.p.layout;
  a.parity = (int)(steps_done & 1);
  a.stream = st;
  const Ops* ops = ops_for(pl.p.lattice, pl.p.storage);
  long long blocks = (long long)pl.p.ny * pl.p.nz;
  if (blocks > kNoAllocBlocks) blocks = kNoAllocBlocks;
  cudaError_t e = ops->diag(a, fields, partials, (int)blocks, out);
  if (e != cudaSuccess) return ctx_fail(LBM_ERR_CUDA, "diagnostics launch failed");
  k_noalloc_finish<<<1, 32, 0, st>>>(out, steps_done);
  e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_fail(LBM_ERR_CUDA, "finish launch failed");
  return LBM_OK;
}
