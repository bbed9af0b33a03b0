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
//
// The reduction uses the block count of lbm_diagnostics (one block per row, at
// most 8 per multiprocessor and kMaxPartials), so that for the same state both
// entry points sum in the same order and return the same bits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "internal.h"

using namespace lbm;

namespace {

constexpr long long kNoAllocMaxNodes = 1LL << 18;  // 262144 nodes, e.g. 512 x 512 or 64^3
constexpr int kNoAllocBlocks = kMaxPartials;       // block partials of the reduction
constexpr long long kNoAllocDoubles =
    4 * kNoAllocMaxNodes + (long long)kNoAllocBlocks * 8 + 32;  // rho, u[<=3], partials, result

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// The array's device address belongs to the CUDA context that loaded the
// library's module; after a context is destroyed (cudaDeviceReset) and created
// again the module is loaded anew.  The address is therefore cached per
// context, keyed by the driver's context id (unique for the process lifetime),
// and looked up again for a context it has not seen.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

constexpr int kCacheSlots = 64;
struct CacheSlot {
  unsigned long long ctx_id;
  double* ptr;
};
std::mutex g_mu;
CacheSlot g_cache[kCacheSlots];
int g_cache_used = 0;
int g_cache_next = 0;  // slot replaced next once the cache is full
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;

int driver_entry_points() {
  if (g_get_current && g_get_id) return LBM_OK;
  void* a = nullptr;
  void* b = nullptr;
  cudaDriverEntryPointQueryResult qa, qb;
  cudaError_t ea = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa);
  cudaError_t eb = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
  if (ea != cudaSuccess || eb != cudaSuccess || qa != cudaDriverEntryPointSuccess ||
      qb != cudaDriverEntryPointSuccess || !a || !b)
    return ctx_fail(LBM_ERR_CUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId unavailable");
  g_get_current = reinterpret_cast<CtxGetCurrentFn>(a);
  g_get_id = reinterpret_cast<CtxGetIdFn>(b);
  return LBM_OK;
}

// Device address of the array in the current context, looked up
// (cudaGetSymbolAddress) once per context with that context's device current.
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ctx_fail(LBM_ERR_CUDA, "cudaGetDevice failed");
  std::lock_guard<std::mutex> lk(g_mu);
  int rc = driver_entry_points();
  if (rc) return rc;
  CUcontext ctx = nullptr;
  if (g_get_current(&ctx) != CUDA_SUCCESS)
    return ctx_fail(LBM_ERR_CUDA, "cannot query the current CUDA context");
  if (!ctx) {
    // no context current in this thread yet: make the device's primary one current
    e = cudaSetDevice(dev);
    if (e != cudaSuccess || g_get_current(&ctx) != CUDA_SUCCESS || !ctx)
      return ctx_fail(LBM_ERR_CUDA, "no CUDA context on the current device");
  }
  unsigned long long id = 0;
  if (g_get_id(ctx, &id) != CUDA_SUCCESS)
    return ctx_fail(LBM_ERR_CUDA, "cannot identify the current CUDA context");
  for (int k = 0; k < g_cache_used; ++k)
    if (g_cache[k].ctx_id == id) {
      *out = g_cache[k].ptr;
      return LBM_OK;
    }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    char buf[256];
    snprintf(buf, sizeof(buf), "cudaGetSymbolAddress of the static scratch failed: %s",
             cudaGetErrorString(e));
    return ctx_fail(LBM_ERR_CUDA, buf);
  }
  int slot = g_cache_used;
  if (slot < kCacheSlots) {
    ++g_cache_used;
  } else {
    slot = g_cache_next;
    g_cache_next = (g_cache_next + 1) % kCacheSlots;
  }
  g_cache[slot] = CacheSlot{id, static_cast<double*>(p)};
  *out = static_cast<double*>(p);
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
                                       const uint8_t* solid_mask, const double* open_bc,
                                       long long steps_done, double* out, void* cuda_stream) {
  Plan pl;
  int rc = plan(p, &pl);
  if (rc) return rc;
  if (!pop_state || !out) return ctx_fail(LBM_ERR_ARG, "pop_state and out are required");
  // the alignment lbm_bind_buffers asks of the state and the mask; out is FP64
  const uintptr_t ps = reinterpret_cast<uintptr_t>(pop_state);
  const uintptr_t ms = reinterpret_cast<uintptr_t>(solid_mask);
  if ((ps & 255u) || (ms & 255u) || (reinterpret_cast<uintptr_t>(out) & 7u))
    return ctx_fail(LBM_ERR_ALIGN, "pop_state and solid_mask must be 256-byte aligned, out 8-byte");
  if (steps_done < 0) return ctx_fail(LBM_ERR_ARG, "steps_done must be >= 0");
  if (pl.N > kNoAllocMaxNodes) {
    char buf[160];
    snprintf(buf, sizeof(buf),
             "lattice of %lld nodes exceeds the %lld-node limit of the static diagnostics scratch",
             pl.N, kNoAllocMaxNodes);
    return ctx_fail(LBM_ERR_ARG, buf);
  }
  OpenBC open{};
  if (open_bc) {
    // the same conditions as lbm_set_open_boundaries
    if (pl.p.lattice != LBM_D2Q9 || pl.p.layout != LBM_LAYOUT_AB)
      return ctx_fail(LBM_ERR_UNSUPPORTED, "open boundaries: D2Q9 with the A/B layout");
    if (pl.g.per[0] || pl.p.nx < 2)
      return ctx_fail(LBM_ERR_ARG, "open boundaries need a non-periodic x axis with nx >= 2");
    if (!(fabs(open_bc[0]) < 1.0) || !(open_bc[1] > 0.0))
      return ctx_fail(LBM_ERR_ARG, "open_bc needs |u_in| < 1 and rho_out > 0");
    open.on = 1;
    open.u_in = open_bc[0];
    open.rho_out = open_bc[1];
  }
  double* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ctx_fail(LBM_ERR_CUDA, "cannot query the multiprocessor count");
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
  a.open = open;
  const Ops* ops = ops_for(pl.p.lattice, pl.p.storage);
  // the block rule of lbm_diagnostics
  long long blocks = (long long)pl.p.ny * pl.p.nz;
  const long long cap = sms > 0 ? 8LL * sms : 1024;
  if (blocks > cap) blocks = cap;
  if (blocks > kNoAllocBlocks) blocks = kNoAllocBlocks;
  cudaError_t e = ops->diag(a, fields, partials, (int)blocks, out);
  if (e != cudaSuccess) return ctx_fail(LBM_ERR_CUDA, "diagnostics launch failed");
  k_noalloc_finish<<<1, 32, 0, st>>>(out, steps_done);
  e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_fail(LBM_ERR_CUDA, "finish launch failed");
  return LBM_OK;
}
