// capi.cu -- the C ABI declared in include/lbm.h: parameter validation, the
// buffer plan, dispatch to the per-(lattice, storage) kernels, diagnostics and
// the autotuner.  Host code only; every step of the path runs in the kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lbm.h"
#include "dispatch.h"
#include "internal.h"

using namespace lbm;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* what, cudaError_t e = cudaSuccess) {
  char buf[512];
  if (e != cudaSuccess)
    snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  else
    snprintf(buf, sizeof(buf), "%s", what);
  g_last_error = buf;
  return code;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LBM_OK;
  return fail(LBM_ERR_CUDA, what, e);
}

bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

const Ops* pick_ops(int lattice, int storage) {
  static const Ops* (*table[3][4])() = {{ops_d2q9_f64, ops_d2q9_f32, ops_d2q9_f16, ops_d2q9_bf16},
                                       {ops_d3q19_f64, ops_d3q19_f32, ops_d3q19_f16, ops_d3q19_bf16},
                                       {ops_d3q27_f64, ops_d3q27_f32, ops_d3q27_f16, ops_d3q27_bf16}};
  return table[lattice][storage]();
}

int storage_bytes(int storage) { return storage == LBM_F64 ? 8 : (storage == LBM_F32 ? 4 : 2); }

}  // namespace

namespace lbm {

int plan(const lbm_params* p, Plan* out) {
  if (!p) return fail(LBM_ERR_ARG, "params is NULL");
  if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19 && p->lattice != LBM_D3Q27)
    return fail(LBM_ERR_ARG, "bad lattice");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(LBM_ERR_ARG, "extent must be >= 1");
  if (p->lattice == LBM_D2Q9 && p->nz != 1) return fail(LBM_ERR_ARG, "D2Q9 needs nz == 1");
  if (p->ny > 65535 * 8 || p->nz > 65535) return fail(LBM_ERR_ARG, "extent too large");
  if (p->collision < LBM_TRT || p->collision > LBM_RLB) return fail(LBM_ERR_ARG, "bad collision");
  if (p->storage < LBM_F64 || p->storage > LBM_BF16_SHIFTED) return fail(LBM_ERR_ARG, "bad storage");
  if (p->layout != LBM_LAYOUT_AB && p->layout != LBM_LAYOUT_AA) return fail(LBM_ERR_ARG, "bad layout");
  if (!(p->rho0 > 0.0) || !isfinite(p->rho0)) return fail(LBM_ERR_ARG, "rho0 must be > 0");
  for (int a = 0; a < 3; ++a) {
    if (p->periodic[a] != 0 && p->periodic[a] != 1) return fail(LBM_ERR_ARG, "periodic flags are 0/1");
    if (!isfinite(p->force[a])) return fail(LBM_ERR_ARG, "force must be finite");
  }
  if (p->lattice == LBM_D2Q9 && p->force[2] != 0.0) return fail(LBM_ERR_ARG, "D2Q9 has no z force");
  // Rates: tau+ = 1/2 + nu/cs^2, tau- = 1/2 + Lambda / (tau+ - 1/2).
  if ((p->nu > 0) == (p->tau_plus > 0)) return fail(LBM_ERR_ARG, "give exactly one of nu, tau_plus");
  if ((p->Lambda > 0) == (p->tau_minus > 0))
    return fail(LBM_ERR_ARG, "give exactly one of Lambda, tau_minus");
  const double tp = p->tau_plus > 0 ? p->tau_plus : 0.5 + 3.0 * p->nu;
  if (!(tp > 0.5) || !isfinite(tp)) return fail(LBM_ERR_ARG, "tau_plus must be > 1/2");
  const double tm = p->tau_minus > 0 ? p->tau_minus : 0.5 + p->Lambda / (tp - 0.5);
  if (!(tm > 0.5) || !isfinite(tm)) return fail(LBM_ERR_ARG, "tau_minus must be > 1/2");
  Plan r{};
  r.p = *p;
  r.Q = p->lattice == LBM_D2Q9 ? 9 : (p->lattice == LBM_D3Q19 ? 19 : 27);
  r.D = p->lattice == LBM_D2Q9 ? 2 : 3;
  r.esize = storage_bytes(p->storage);
  const int per_vec = 16 / r.esize;
  r.g.nx = p->nx;
  r.g.ny = p->ny;
  r.g.nz = p->nz;
  r.g.pitch = (p->nx + per_vec - 1) / per_vec * per_vec;
  const long long per256 = 256 / r.esize;
  const long long cells = (long long)r.g.pitch * p->ny * p->nz;
  r.g.plane = (cells + per256 - 1) / per256 * per256;
  for (int a = 0; a < 3; ++a) r.g.per[a] = p->periodic[a];
  r.N = (long long)p->nx * p->ny * p->nz;
  r.pop_bytes = (size_t)r.Q * (size_t)r.g.plane * (size_t)r.esize;
  r.field_off = kFieldOffset;
  r.scratch_bytes = kFieldOffset + (size_t)(1 + r.D) * (size_t)r.N * sizeof(double);
  r.scratch_bytes = (r.scratch_bytes + 255) / 256 * 256;
  const double wp = 1.0 / tp, wm = 1.0 / tm;
  r.omega_plus = wp;
  r.omega_minus = wm;
  // BGK is TRT with equal rates; second-order RLB is P-TRT with w- = 1.
  double wmk = wm;
  r.kernel_collision = p->collision;
  if (p->collision == LBM_BGK) {
    r.kernel_collision = LBM_TRT;
    wmk = wp;
  } else if (p->collision == LBM_RLB) {
    r.kernel_collision = LBM_P_TRT;
    wmk = 1.0;
  }
  r.cp = 1.0 - wp;
  r.cm = 1.0 - wmk;
  r.hg = 1.0 - 0.5 * wp;
  r.force = p->force[0] != 0.0 || p->force[1] != 0.0 || p->force[2] != 0.0;
  if (p->lattice == LBM_D2Q9)
    fill_coef<D2Q9>(p->rho0, wp, wmk, r.kernel_collision, p->force, &r.coef);
  else if (p->lattice == LBM_D3Q19)
    fill_coef<D3Q19>(p->rho0, wp, wmk, r.kernel_collision, p->force, &r.coef);
  else
    fill_coef<D3Q27>(p->rho0, wp, wmk, r.kernel_collision, p->force, &r.coef);
  *out = r;
  return LBM_OK;
}

std::vector<Variant> variants_for(const Plan& pl, const Ops* ops, bool masked) {
  static const int shapes[][2] = {{32, 8}, {64, 4}, {128, 2}, {256, 1}, {32, 4}, {64, 2}, {128, 1}};
  std::vector<Variant> v;
  // pipelined bulk-copy kernel (A/B or AA): no solid mask, rows a multiple of 16 bytes
  const int H = 16 / pl.esize;
  if (!masked && pl.p.nx % H == 0 && pl.p.nx >= 2 * H) {
    static const int tiles[] = {512, 384, 256, 192, 128};
    static const int depths[] = {4, 3, 6, 8, 2};
    for (int X : tiles)
      for (int st : depths) {
        size_t smem = ops->tma_smem(X, st);
        // the AA odd step stages its destination rows as well
        if (smem > 0 && pl.p.layout == LBM_LAYOUT_AA) smem += aa_odd_smem(pl.Q, pl.esize, X);
        if (smem > 0 && smem <= 200 * 1024) {
          v.push_back(Variant{1, 0, 0, 0, X, st});
          v.push_back(Variant{1, 0, 2, 0, X, st});  // at most two resident blocks per SM
        }
        // A/B with 32- or 16-bit storage: the staged bulk stores (a store warp)
        const size_t bs = ops->tma_smem(X, st) + tma_bs_smem(pl.Q, pl.esize, X);
        if (pl.p.layout == LBM_LAYOUT_AB && pl.esize < 8 && ops->tma_smem(X, st) > 0 &&
            bs <= 200 * 1024)
          v.push_back(Variant{1, 0, 0, 1, X, st});
        // A/B with 16-bit storage: four nodes per consumer thread
        if (pl.p.layout == LBM_LAYOUT_AB && pl.esize == 2 && ops->tma_smem(X, st) > 0 &&
            ops->tma_smem(X, st) <= 200 * 1024)
          v.push_back(Variant{1, 4, 0, 0, X, st});
      }
  }
  for (int k = 0; k < ops->n_nv; ++k) {
    const int nv = ops->nvs[k];
    if (pl.p.nx % nv != 0) continue;
    if (pl.p.layout == LBM_LAYOUT_AA && nv != 1) continue;
    for (auto& s : shapes)
      if ((pl.p.ny + s[1] - 1) / s[1] <= 65535) v.push_back(Variant{0, nv, s[0], s[1], 0, 0});
  }
  return v;
}

int default_variant(const Plan& pl, const std::vector<Variant>& vs) {
  // the pipelined kernel when available, else the widest vector that keeps the
  // registers of one thread moderate, 256 threads
  for (size_t k = 0; k < vs.size(); ++k)
    if (vs[k].kind == 1) return (int)k;
  const int budget = pl.Q == 9 ? 16 : 8;  // bytes per plane per thread
  int best = 0, best_nv = 0;
  for (size_t k = 0; k < vs.size(); ++k) {
    const Variant& v = vs[k];
    if (v.kind != 0 || v.nv * pl.esize > budget || v.bx * v.by != 256) continue;
    if (v.nv > best_nv || (v.nv == best_nv && v.bx == 64)) {
      best = (int)k;
      best_nv = v.nv;
    }
  }
  return best;
}

}  // namespace lbm

struct lbm_ctx {
  Plan pl;
  const Ops* ops = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0;
  void* pop[2] = {nullptr, nullptr};
  const uint8_t* mask = nullptr;
  char* scratch = nullptr;
  unsigned int* flag = nullptr;  // divergence flag (own scratch, or the batch's per-lattice slot)
  bool bound = false;
  bool view = false;  // owned by a batch
  int cur = 0;        // A/B: index of the buffer holding the state
  long long t = 0;    // completed steps
  long long launches = 0;
  std::vector<Variant> vars;
  int var = 0;
  int var_odd = -1;   // AA: variant of the odd steps when tuned apart (-1: var)
  int sms = 0;
  OpenBC open{};  // open boundaries of the square-cylinder benchmark (off by default)
  bool fresh = true;  // the state was written directly (not yet streamed)
  int scheme = 1;     // forcing scheme: 1 Guo, 2 simplified projection + G_i
  long long wait_ns = 2000000000LL;
  int extra_tx = 0;
};

namespace lbm {

unsigned int* flag_ptr(lbm_ctx* c) { return c->flag; }

AuxLaunch aux_of(lbm_ctx* c) {
  AuxLaunch a{};
  a.g = c->pl.g;
  a.rho0 = c->pl.p.rho0;
  for (int k = 0; k < 3; ++k) a.F[k] = c->pl.p.force[k];
  a.pop = c->pop[c->pl.p.layout == LBM_LAYOUT_AA ? 0 : c->cur];
  a.mask = c->mask;
  a.layout = c->pl.p.layout;
  a.parity = (int)(c->t & 1);
  a.stream = c->stream;
  a.open = c->open;
  a.open.on = c->open.on && !c->fresh;
  return a;
}

StepLaunch step_of(lbm_ctx* c, const Variant& v) {
  StepLaunch s{};
  s.open = c->open;
  s.open.fix = c->open.on && !c->fresh;
  s.g = c->pl.g;
  s.collision = c->pl.kernel_collision;
  s.force = c->pl.force;
  s.c = c->pl.coef;
  s.err = reinterpret_cast<int*>(c->scratch + kErrOffset);
  s.wait_ns = c->wait_ns;
  s.extra_tx = c->extra_tx;
  s.sms = c->sms;
  s.mask = c->mask;
  s.flag = flag_ptr(c);
  s.step = (unsigned int)(c->t < 0xfffffffeLL ? c->t : 0xfffffffeLL);
  s.layout = c->pl.p.layout;
  s.parity = (int)(c->t & 1);
  s.v = v;
  s.stream = c->stream;
  s.scheme = c->scheme;
  s.phi = c->scratch + c->pl.field_off;
  if (s.layout == LBM_LAYOUT_AA) {
    s.src = c->pop[0];
    s.dst = c->pop[0];
  } else {
    s.src = c->pop[c->cur];
    s.dst = c->pop[1 - c->cur];
  }
  return s;
}

int ctx_new(const Plan& pl, cudaStream_t st, lbm_ctx** out) {
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return fail(LBM_ERR_ARG, "out of host memory");
  c->pl = pl;
  c->ops = pick_ops(pl.p.lattice, pl.p.storage);
  c->stream = st;
  cudaGetDevice(&c->device);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  c->vars = variants_for(pl, c->ops, false);
  c->var = default_variant(pl, c->vars);
  *out = c;
  return LBM_OK;
}

int ctx_bind(lbm_ctx* c, void* a, void* b, const uint8_t* mask, void* scratch) {
  c->pop[0] = a;
  c->pop[1] = b;
  c->mask = mask;
  c->scratch = static_cast<char*>(scratch);
  c->flag = reinterpret_cast<unsigned int*>(c->scratch + kFlagOffset);
  c->bound = true;
  c->cur = 0;
  c->t = 0;
  c->vars = variants_for(c->pl, c->ops, mask != nullptr);
  c->var = default_variant(c->pl, c->vars);
  c->var_odd = -1;
  return LBM_OK;
}

int reset_flag(lbm_ctx* c) {
  int rc = cuda_check(cudaMemsetAsync(c->scratch + kErrOffset, 0, sizeof(int), c->stream),
                      "reset error word");
  if (rc) return rc;
  return cuda_check(cudaMemsetAsync(flag_ptr(c), 0xff, sizeof(unsigned int), c->stream),
                    "reset divergence flag");
}

int ctx_step(lbm_ctx* c, int n) {
  for (int s = 0; s < n; ++s) {
    const bool odd_own = c->pl.p.layout == LBM_LAYOUT_AA && (c->t & 1) && c->var_odd >= 0 &&
                         c->var_odd < (int)c->vars.size();
    StepLaunch sl = step_of(c, c->vars[odd_own ? c->var_odd : c->var]);
    cudaError_t e = c->ops->step(sl);
    c->launches += c->scheme == 2 ? 2 : 1;
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "stream-collide launch", e);
    if (c->pl.p.layout == LBM_LAYOUT_AB) c->cur ^= 1;
    ++c->t;
    c->fresh = false;
  }
  return LBM_OK;
}

void ctx_set_state(lbm_ctx* c, int cur, long long t) {
  c->cur = cur;
  c->t = t;
}
void ctx_get_state(const lbm_ctx* c, int* cur, long long* t) {
  *cur = c->cur;
  *t = c->t;
}
void ctx_mark_view(lbm_ctx* c) { c->view = true; }
void ctx_set_flag(lbm_ctx* c, unsigned int* flag) { c->flag = flag; }
cudaStream_t ctx_stream(const lbm_ctx* c) { return c->stream; }
const Ops* ctx_ops(const lbm_ctx* c) { return c->ops; }
const std::vector<Variant>& ctx_variants(const lbm_ctx* c) { return c->vars; }
int ctx_variant(const lbm_ctx* c) { return c->var; }
StepLaunch ctx_step_launch(lbm_ctx* c, const Variant& v) { return step_of(c, v); }
void ctx_delete(lbm_ctx* c) { delete c; }
void ctx_add_launches(lbm_ctx* c, long long n) { c->launches += n; }
int ctx_fail(int code, const char* what) { return fail(code, what); }

}  // namespace lbm

#define CHECK_CTX(c)                                                  \
  do {                                                                \
    if (!(c)) return fail(LBM_ERR_ARG, "context is NULL");            \
    if (!(c)->bound) return fail(LBM_ERR_STATE, "buffers not bound"); \
  } while (0)

extern "C" {

int lbm_version(void) { return 100; }

const char* lbm_strerror(int code) {
  switch (code) {
    case LBM_OK:
      return "ok";
    case LBM_ERR_ARG:
      return "invalid argument";
    case LBM_ERR_CUDA:
      return "CUDA runtime error";
    case LBM_ERR_DIVERGED:
      return "simulation diverged (NaN/Inf, rho <= 0 or |u| > 1)";
    case LBM_ERR_TIMEOUT:
      return "bounded device wait timed out";
    case LBM_ERR_UNSUPPORTED:
      return "unsupported combination";
    case LBM_ERR_STATE:
      return "call out of order";
    case LBM_ERR_ALIGN:
      return "buffer not aligned as required (256 bytes; 8 for FP64 fields)";
  }
  return "unknown error";
}

const char* lbm_last_error(void) { return g_last_error.c_str(); }

int lbm_buffer_sizes(const lbm_params* p, size_t* pop_bytes, size_t* scratch_bytes) {
  Plan pl;
  int rc = plan(p, &pl);
  if (rc) return rc;
  if (pop_bytes) *pop_bytes = pl.pop_bytes;
  if (scratch_bytes) *scratch_bytes = pl.scratch_bytes;
  return LBM_OK;
}

int lbm_create(const lbm_params* p, void* cuda_stream, lbm_ctx** out) {
  if (!out) return fail(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  Plan pl;
  int rc = plan(p, &pl);
  if (rc) return rc;
  return ctx_new(pl, static_cast<cudaStream_t>(cuda_stream), out);
}

int lbm_bind_buffers(lbm_ctx* c, void* pop_a, void* pop_b, const uint8_t* solid_mask,
                     void* scratch) {
  if (!c) return fail(LBM_ERR_ARG, "context is NULL");
  if (c->view) return fail(LBM_ERR_STATE, "batch views are bound by their batch");
  if (!pop_a || !scratch) return fail(LBM_ERR_ARG, "pop_a and scratch are required");
  const bool aa = c->pl.p.layout == LBM_LAYOUT_AA;
  if (aa && pop_b) return fail(LBM_ERR_ARG, "AA layout takes one population buffer");
  if (!aa && !pop_b) return fail(LBM_ERR_ARG, "A/B layout needs pop_b");
  if (!aligned256(pop_a) || (pop_b && !aligned256(pop_b)) || !aligned256(scratch) ||
      (solid_mask && !aligned256(solid_mask)))
    return fail(LBM_ERR_ALIGN, "buffers must be 256-byte aligned");
  return ctx_bind(c, pop_a, pop_b, solid_mask, scratch);
}

// FP64 fields are read and written element by element by the kernels: a
// device pointer that is not 8-byte aligned is refused before any launch.
static bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

int lbm_init_equilibrium(lbm_ctx* c, const double* rho, const double* u) {
  CHECK_CTX(c);
  if (!rho || !u) return fail(LBM_ERR_ARG, "rho and u are required");
  if (!aligned8(rho) || !aligned8(u)) return fail(LBM_ERR_ALIGN, "rho and u must be 8-byte aligned");
  c->cur = 0;
  c->t = 0;
  c->fresh = true;
  int rc = reset_flag(c);
  if (rc) return rc;
  cudaError_t e = c->ops->init_eq(aux_of(c), rho, u);
  ++c->launches;
  return cuda_check(e, "init equilibrium");
}

// Device address of a host buffer the kernels can use in place: page-locked
// memory registered with CUDA and mapped into the device's address space
// (cudaHostAlloc / cudaHostRegister under unified addressing) and 8-byte
// aligned, else NULL (the caller then copies through the scratch buffer).
static const void* mapped_host(const void* p) {
  if (!aligned8(p)) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // an unregistered pointer is not an error here
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int lbm_init_equilibrium_host(lbm_ctx* c, const double* rho, const double* u) {
  CHECK_CTX(c);
  if (!rho || !u) return fail(LBM_ERR_ARG, "rho and u are required");
  const void* mr = mapped_host(rho);
  const void* mu = mapped_host(u);
  if (mr && mu) {
    // page-locked, mapped buffers: the init kernel reads them over the host link
    int rc = lbm_init_equilibrium(c, static_cast<const double*>(mr), static_cast<const double*>(mu));
    if (rc) return rc;
    return cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
  }
  double* fr = reinterpret_cast<double*>(c->scratch + c->pl.field_off);
  double* fu = fr + c->pl.N;
  const size_t nb = (size_t)c->pl.N * sizeof(double);
  int rc = cuda_check(cudaMemcpyAsync(fr, rho, nb, cudaMemcpyHostToDevice, c->stream), "copy rho");
  if (rc) return rc;
  rc = cuda_check(cudaMemcpyAsync(fu, u, nb * c->pl.D, cudaMemcpyHostToDevice, c->stream), "copy u");
  if (rc) return rc;
  rc = lbm_init_equilibrium(c, fr, fu);
  if (rc) return rc;
  return cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
}

int lbm_step(lbm_ctx* c, int n) {
  CHECK_CTX(c);
  if (n < 0) return fail(LBM_ERR_ARG, "n must be >= 0");
  if (c->view) return fail(LBM_ERR_STATE, "batch views are stepped by lbm_batch_step");
  return ctx_step(c, n);
}

int lbm_macros(lbm_ctx* c, double* rho, double* u) {
  CHECK_CTX(c);
  if (!rho || !u) return fail(LBM_ERR_ARG, "rho and u are required");
  if (!aligned8(rho) || !aligned8(u)) return fail(LBM_ERR_ALIGN, "rho and u must be 8-byte aligned");
  cudaError_t e = c->ops->macros(aux_of(c), rho, u);
  ++c->launches;
  return cuda_check(e, "macros");
}

int lbm_macros_host(lbm_ctx* c, double* rho, double* u) {
  CHECK_CTX(c);
  if (!rho || !u) return fail(LBM_ERR_ARG, "rho and u are required");
  const void* mr = mapped_host(rho);
  const void* mu = mapped_host(u);
  if (mr && mu) {
    // page-locked, mapped buffers: the macros kernel writes them over the host link
    int rc = lbm_macros(c, static_cast<double*>(const_cast<void*>(mr)),
                        static_cast<double*>(const_cast<void*>(mu)));
    if (rc) return rc;
    return cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
  }
  double* fr = reinterpret_cast<double*>(c->scratch + c->pl.field_off);
  double* fu = fr + c->pl.N;
  int rc = lbm_macros(c, fr, fu);
  if (rc) return rc;
  const size_t nb = (size_t)c->pl.N * sizeof(double);
  rc = cuda_check(cudaMemcpyAsync(rho, fr, nb, cudaMemcpyDeviceToHost, c->stream), "copy rho");
  if (rc) return rc;
  rc = cuda_check(cudaMemcpyAsync(u, fu, nb * c->pl.D, cudaMemcpyDeviceToHost, c->stream), "copy u");
  if (rc) return rc;
  return cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
}

int lbm_get_populations(lbm_ctx* c, double* f) {
  CHECK_CTX(c);
  if (!f) return fail(LBM_ERR_ARG, "f is NULL");
  if (!aligned8(f)) return fail(LBM_ERR_ALIGN, "f must be 8-byte aligned");
  cudaError_t e = c->ops->get_pop(aux_of(c), f);
  ++c->launches;
  return cuda_check(e, "get populations");
}

int lbm_set_populations(lbm_ctx* c, const double* f) {
  CHECK_CTX(c);
  if (!f) return fail(LBM_ERR_ARG, "f is NULL");
  if (!aligned8(f)) return fail(LBM_ERR_ALIGN, "f must be 8-byte aligned");
  int rc = reset_flag(c);
  if (rc) return rc;
  c->fresh = true;
  cudaError_t e = c->ops->set_pop(aux_of(c), f);
  ++c->launches;
  return cuda_check(e, "set populations");
}

static int run_diag(lbm_ctx* c, const double* uref, double* out8) {
  if (!uref) {
    // mass, momentum, kinetic energy, enstrophy, flag: two passes over the state
    double* partials = reinterpret_cast<double*>(c->scratch + kPartialOffset);
    double* out = reinterpret_cast<double*>(c->scratch + kResultOffset);
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device);
    long long blocks = (long long)c->pl.p.ny * c->pl.p.nz;
    const long long cap = dev_sms > 0 ? 8LL * dev_sms : 1024;
    if (blocks > cap) blocks = cap;
    if (blocks > kMaxPartials) blocks = kMaxPartials;
    cudaError_t e = c->ops->diag(aux_of(c), c->scratch + c->pl.field_off, partials, (int)blocks, out);
    c->launches += 3;
    int rc = cuda_check(e, "diagnostics");
    if (rc) return rc;
    rc = cuda_check(cudaMemcpyAsync(out8, out, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                    "copy diagnostics");
    if (rc) return rc;
    return cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
  }
  double* fr = reinterpret_cast<double*>(c->scratch + c->pl.field_off);
  double* fu = fr + c->pl.N;
  int rc = lbm_macros(c, fr, fu);
  if (rc) return rc;
  DiagLaunch d{};
  d.g = c->pl.g;
  d.D = c->pl.D;
  d.rho = fr;
  d.u = fu;
  d.uref = uref;
  d.mask = c->mask;
  d.partials = reinterpret_cast<double*>(c->scratch + kPartialOffset);
  d.out = reinterpret_cast<double*>(c->scratch + kResultOffset);
  int dev_sms = 0;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device);
  long long want = (c->pl.N + 255) / 256;
  long long cap = (long long)dev_sms * 4;
  if (cap > kMaxPartials) cap = kMaxPartials;
  d.blocks = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
  d.stream = c->stream;
  cudaError_t e = diag_l2(d);
  c->launches += 2;
  rc = cuda_check(e, "diagnostics");
  if (rc) return rc;
  rc = cuda_check(cudaMemcpyAsync(out8, d.out, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                  "copy diagnostics");
  if (rc) return rc;
  return cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
}

int lbm_diagnostics(lbm_ctx* c, double out[8]) {
  CHECK_CTX(c);
  if (!out) return fail(LBM_ERR_ARG, "out is NULL");
  double r[8];
  int rc = run_diag(c, nullptr, r);
  if (rc) return rc;
  for (int k = 0; k < 6; ++k) out[k] = r[k];
  out[6] = r[6] > 0.0 ? 1.0 : 0.0;
  out[7] = (double)c->t;
  return LBM_OK;
}

int lbm_velocity_l2(lbm_ctx* c, const double* u_ref, double* out) {
  CHECK_CTX(c);
  if (!u_ref || !out) return fail(LBM_ERR_ARG, "u_ref and out are required");
  if (!aligned8(u_ref)) return fail(LBM_ERR_ALIGN, "u_ref must be 8-byte aligned");
  double r[8];
  int rc = run_diag(c, u_ref, r);
  if (rc) return rc;
  *out = r[1] > 0.0 ? sqrt(r[0] / r[1]) : (r[0] > 0.0 ? INFINITY : 0.0);
  return LBM_OK;
}

int lbm_set_open_boundaries(lbm_ctx* c, double u_in, double rho_out) {
  CHECK_CTX(c);
  if (c->view) return fail(LBM_ERR_STATE, "batch views take no open boundaries");
  if (!(rho_out > 0.0)) {  // off
    c->open = OpenBC{};
    return LBM_OK;
  }
  if (c->pl.p.lattice != LBM_D2Q9 || c->pl.p.layout != LBM_LAYOUT_AB)
    return fail(LBM_ERR_UNSUPPORTED, "open boundaries: D2Q9 with the A/B layout");
  if (c->pl.g.per[0] || c->pl.p.nx < 2)
    return fail(LBM_ERR_ARG, "open boundaries need a non-periodic x axis with nx >= 2");
  if (c->scheme == 2) return fail(LBM_ERR_UNSUPPORTED, "open boundaries with forcing scheme 2");
  if (!(fabs(u_in) < 1.0)) return fail(LBM_ERR_ARG, "|u_in| must be < 1");
  c->open.on = 1;
  c->open.u_in = u_in;
  c->open.rho_out = rho_out;
  return LBM_OK;
}

int lbm_set_forcing_scheme(lbm_ctx* c, int scheme) {
  CHECK_CTX(c);
  if (scheme != 1 && scheme != 2) return fail(LBM_ERR_ARG, "forcing scheme must be 1 or 2");
  if (scheme == 1) {
    c->scheme = 1;
    return LBM_OK;
  }
  if (c->view) return fail(LBM_ERR_STATE, "batch views take forcing scheme 1 only");
  if (c->open.on) return fail(LBM_ERR_UNSUPPORTED, "forcing scheme 2 with open boundaries");
  c->scheme = 2;
  return LBM_OK;
}

int lbm_momentum_exchange(lbm_ctx* c, double out[3]) {
  CHECK_CTX(c);
  if (!out) return fail(LBM_ERR_ARG, "out is NULL");
  if (c->scheme == 2) return fail(LBM_ERR_UNSUPPORTED, "momentum exchange with forcing scheme 2");
  double* partials = reinterpret_cast<double*>(c->scratch + kPartialOffset);
  double* res = reinterpret_cast<double*>(c->scratch + kResultOffset);
  int dev_sms = 0;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device);
  long long blocks = (long long)c->pl.p.ny * c->pl.p.nz;
  const long long cap = dev_sms > 0 ? 8LL * dev_sms : 1024;
  if (blocks > cap) blocks = cap;
  if (blocks > kMaxPartials) blocks = kMaxPartials;
  cudaError_t e = c->ops->momentum(aux_of(c), c->pl.kernel_collision, c->pl.coef, partials,
                                   (int)blocks, res);
  c->launches += 2;
  int rc = cuda_check(e, "momentum exchange");
  if (rc) return rc;
  double r[8];
  rc = cuda_check(cudaMemcpyAsync(r, res, sizeof(r), cudaMemcpyDeviceToHost, c->stream),
                  "copy force");
  if (rc) return rc;
  rc = cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
  if (rc) return rc;
  for (int k = 0; k < 3; ++k) out[k] = r[k];
  return LBM_OK;
}

int lbm_status(lbm_ctx* c, long long* first_step) {
  CHECK_CTX(c);
  unsigned int v = 0;
  int err = 0;
  int rc = cuda_check(cudaMemcpyAsync(&v, flag_ptr(c), sizeof(v), cudaMemcpyDeviceToHost, c->stream),
                      "read divergence flag");
  if (rc) return rc;
  rc = cuda_check(cudaMemcpyAsync(&err, c->scratch + kErrOffset, sizeof(err), cudaMemcpyDeviceToHost,
                                  c->stream),
                  "read error word");
  if (rc) return rc;
  rc = cuda_check(cudaStreamSynchronize(c->stream), "synchronise");
  if (rc) return rc;
  if (first_step) *first_step = v == 0xffffffffu ? -1 : (long long)v;
  if (err) return fail(LBM_ERR_TIMEOUT, "a bounded device wait ran out");
  return v == 0xffffffffu ? LBM_OK : LBM_ERR_DIVERGED;
}

int lbm_step_count(const lbm_ctx* c, long long* t) {
  if (!c || !t) return fail(LBM_ERR_ARG, "NULL argument");
  *t = c->t;
  return LBM_OK;
}

int lbm_checkpoint(lbm_ctx* c, void* dst, size_t bytes, long long* t) {
  CHECK_CTX(c);
  if (!dst || bytes != c->pl.pop_bytes) return fail(LBM_ERR_ARG, "dst must hold pop_bytes");
  const void* src = c->pop[c->pl.p.layout == LBM_LAYOUT_AA ? 0 : c->cur];
  if (t) *t = c->t;
  return cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream), "checkpoint");
}

int lbm_restore(lbm_ctx* c, const void* src, size_t bytes, long long t) {
  CHECK_CTX(c);
  if (!src || bytes != c->pl.pop_bytes || t < 0) return fail(LBM_ERR_ARG, "bad snapshot");
  c->cur = 0;
  c->t = t;
  c->fresh = t == 0;
  int rc = reset_flag(c);
  if (rc) return rc;
  return cuda_check(cudaMemcpyAsync(c->pop[0], src, bytes, cudaMemcpyDeviceToDevice, c->stream),
                    "restore");
}

int lbm_set_wait_limit(lbm_ctx* c, double seconds, int test_extra_bytes) {
  if (!c || !(seconds > 0.0) || seconds > 60.0 || test_extra_bytes < 0 || test_extra_bytes > (1 << 16))
    return fail(LBM_ERR_ARG, "limit in (0, 60] s, extra bytes in [0, 65536]");
  c->wait_ns = (long long)(seconds * 1e9);
  c->extra_tx = test_extra_bytes;
  return LBM_OK;
}

int lbm_launch_count(const lbm_ctx* c, long long* launches) {
  if (!c || !launches) return fail(LBM_ERR_ARG, "NULL argument");
  *launches = c->launches;
  return LBM_OK;
}

int lbm_variant_count(const lbm_ctx* c, int* n) {
  if (!c || !n) return fail(LBM_ERR_ARG, "NULL argument");
  *n = (int)c->vars.size();
  return LBM_OK;
}

int lbm_variant_name(const lbm_ctx* c, int v, char* buf, size_t len) {
  if (!c || !buf || v < 0 || v >= (int)c->vars.size()) return fail(LBM_ERR_ARG, "bad variant");
  const Variant& x = c->vars[v];
  if (x.kind == 1 && x.by == 1)
    snprintf(buf, len, "tma_X%d_s%d_bs", x.X, x.stages);
  else if (x.kind == 1 && x.nv == 4)
    snprintf(buf, len, "tma_X%d_s%d_q", x.X, x.stages);
  else if (x.kind == 1 && x.bx > 0)
    snprintf(buf, len, "tma_X%d_s%d_b%d", x.X, x.stages, x.bx);
  else if (x.kind == 1)
    snprintf(buf, len, "tma_X%d_s%d", x.X, x.stages);
  else
    snprintf(buf, len, "nv%d_b%dx%d", x.nv, x.bx, x.by);
  return LBM_OK;
}

int lbm_get_variant(const lbm_ctx* c, int* v) {
  if (!c || !v) return fail(LBM_ERR_ARG, "NULL argument");
  *v = c->var;
  return LBM_OK;
}

int lbm_set_variant(lbm_ctx* c, int v) {
  if (!c || v < 0 || v >= (int)c->vars.size()) return fail(LBM_ERR_ARG, "bad variant");
  c->var = v;
  c->var_odd = -1;
  return LBM_OK;
}

int lbm_autotune(lbm_ctx* c, int reps, int* chosen, float* times_ms) {
  CHECK_CTX(c);
  if (reps < 1) reps = 1;
  const bool aa = c->pl.p.layout == LBM_LAYOUT_AA;
  using Key = std::tuple<int, int, int, int, int, int, int, int, int, int, int, int>;
  static std::mutex mu;
  static std::map<Key, std::pair<int, int>> cache;  // (variant, AA odd-step variant or -1)
  const Key key{c->pl.p.lattice, c->pl.p.storage, c->pl.kernel_collision, c->mask != nullptr,
                c->pl.p.nx,      c->pl.p.ny,      c->pl.p.nz,            c->pl.g.per[0],
                c->pl.g.per[1],  c->pl.g.per[2],  c->pl.p.layout,        c->scheme};
  if (!times_ms) {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end() && it->second.first < (int)c->vars.size() &&
        it->second.second < (int)c->vars.size()) {
      c->var = it->second.first;
      c->var_odd = it->second.second;
      if (chosen) *chosen = c->var;
      return LBM_OK;
    }
  }
  cudaEvent_t e0, e1;
  int rc = cuda_check(cudaEventCreate(&e0), "event");
  if (rc) return rc;
  rc = cuda_check(cudaEventCreate(&e1), "event");
  if (rc) {
    cudaEventDestroy(e0);
    return rc;
  }
  int best = c->var;
  float best_ms = 1e30f;
  const int keep = c->var, keep_odd = c->var_odd;
  // AA: the even and odd steps are different kernels; each gets its fastest
  // variant (timed on steps that really advance the lattice)
  int best_even = c->var, best_odd = c->var;
  float best_even_ms = 1e30f, best_odd_ms = 1e30f;
  cudaEvent_t e2 = nullptr;
  if (aa) rc = cuda_check(cudaEventCreate(&e2), "event");
  c->var_odd = -1;
  for (int v = 0; v < (int)c->vars.size() && rc == LBM_OK; ++v) {
    cudaError_t e = cudaSuccess;
    if (aa) {
      c->var = v;
      rc = ctx_step(c, (c->t & 1) ? 3 : 2);  // warm up, end on an even step count
      if (rc) break;
      float even_ms = 0.f, odd_ms = 0.f;
      for (int r = 0; r < reps && e == cudaSuccess && rc == LBM_OK; ++r) {
        e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) rc = ctx_step(c, 1);
        if (e == cudaSuccess && rc == LBM_OK) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess && rc == LBM_OK) rc = ctx_step(c, 1);
        if (e == cudaSuccess && rc == LBM_OK) e = cudaEventRecord(e2, c->stream);
        if (e == cudaSuccess && rc == LBM_OK) e = cudaEventSynchronize(e2);
        float a = 0.f, b = 0.f;
        if (e == cudaSuccess && rc == LBM_OK) e = cudaEventElapsedTime(&a, e0, e1);
        if (e == cudaSuccess && rc == LBM_OK) e = cudaEventElapsedTime(&b, e1, e2);
        even_ms += a;
        odd_ms += b;
      }
      if (rc) break;
      if (e != cudaSuccess) {
        rc = fail(LBM_ERR_CUDA, "autotune", e);
        break;
      }
      even_ms /= reps;
      odd_ms /= reps;
      if (times_ms) times_ms[v] = 0.5f * (even_ms + odd_ms);
      if (even_ms < best_even_ms) {
        best_even_ms = even_ms;
        best_even = v;
      }
      if (odd_ms < best_odd_ms) {
        best_odd_ms = odd_ms;
        best_odd = v;
      }
      continue;
    }
    {
      StepLaunch sl = step_of(c, c->vars[v]);  // reads the state, writes the other buffer
      e = c->ops->step(sl);
      c->launches += (1 + reps) * (c->scheme == 2 ? 2 : 1);
      if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
      for (int r = 0; r < reps && e == cudaSuccess; ++r) e = c->ops->step(sl);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = fail(LBM_ERR_CUDA, "autotune", e);
      break;
    }
    ms /= reps;
    if (times_ms) times_ms[v] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e2) cudaEventDestroy(e2);
  if (rc) {
    c->var = keep;
    c->var_odd = keep_odd;
    return rc;
  }
  if (aa) {
    best = best_even;
    c->var_odd = best_odd;
  }
  c->var = best;
  {
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = {best, c->var_odd};
  }
  if (chosen) *chosen = best;
  return LBM_OK;
}

int lbm_destroy(lbm_ctx* c) {
  if (!c) return LBM_OK;
  if (c->view) return fail(LBM_ERR_STATE, "batch views are destroyed with their batch");
  delete c;
  return LBM_OK;
}


int lbm_copy_ceiling(const void* src, void* dst, size_t bytes, void* cuda_stream) {
  if (!src || !dst || (bytes % 16) != 0 || (reinterpret_cast<uintptr_t>(src) & 15) ||
      (reinterpret_cast<uintptr_t>(dst) & 15))
    return fail(LBM_ERR_ARG, "copy needs 16-byte aligned pointers and sizes");
  return cuda_check(copy_ceiling(src, dst, bytes, static_cast<cudaStream_t>(cuda_stream)), "copy");
}

}  // extern "C"
