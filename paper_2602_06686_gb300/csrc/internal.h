// internal.h -- host-side plan of a lattice and helpers shared by capi.cu and
// batch.cu.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/lbm.h"
#include "dispatch.h"

namespace lbm {

// Scratch buffer layout (bytes).
constexpr size_t kFlagOffset = 0;        // unsigned int: earliest diverged step (0xffffffff: none)
constexpr size_t kErrOffset = 64;        // int: 1 when a bounded device wait ran out
constexpr size_t kBarrierOffset = 256;   // batch grid-barrier words and error status
constexpr size_t kPartialOffset = 4096;  // double [kMaxPartials][8] block partials
constexpr int kMaxPartials = 4096;
constexpr size_t kResultOffset = kPartialOffset + (size_t)kMaxPartials * 8 * sizeof(double);
constexpr size_t kFieldOffset = kResultOffset + 4096;  // FP64 rho [N], u [D][N] staging

struct Plan {
  lbm_params p;
  int Q, D, esize;
  GeoH g;
  long long N;
  size_t pop_bytes, scratch_bytes, field_off;
  double omega_plus, omega_minus;
  int kernel_collision;  // collision the kernels run (BGK -> TRT, RLB -> P-TRT)
  double cp, cm, hg;     // 1 - w+, 1 - w- (as run), 1 - w+/2
  bool force;            // any force component non-zero
  CoefV<double> coef;    // per-direction collision constants (FP64)
};

int plan(const lbm_params* p, Plan* out);
std::vector<Variant> variants_for(const Plan& pl, const Ops* ops, bool masked);
int default_variant(const Plan& pl, const std::vector<Variant>& vs);

int ctx_new(const Plan& pl, cudaStream_t st, lbm_ctx** out);
int ctx_bind(lbm_ctx* c, void* a, void* b, const uint8_t* mask, void* scratch);
void ctx_set_state(lbm_ctx* c, int cur, long long t);
void ctx_get_state(const lbm_ctx* c, int* cur, long long* t);
void ctx_mark_view(lbm_ctx* c);
void ctx_set_flag(lbm_ctx* c, unsigned int* flag);
cudaStream_t ctx_stream(const lbm_ctx* c);
const Ops* ctx_ops(const lbm_ctx* c);
const std::vector<Variant>& ctx_variants(const lbm_ctx* c);
int ctx_variant(const lbm_ctx* c);
StepLaunch ctx_step_launch(lbm_ctx* c, const Variant& v);
void ctx_delete(lbm_ctx* c);
void ctx_add_launches(lbm_ctx* c, long long n);
int ctx_fail(int code, const char* what);
int reset_flag(lbm_ctx* c);

}  // namespace lbm
