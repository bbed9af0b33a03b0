// batch.cu -- many independent lattices advanced together (the batched driver):
// arena plan, per-lattice views, tile lists, the persistent cooperative kernel
// captured in a CUDA graph, the sequential one-launch-per-lattice baseline and
// the tile-shape autotuner.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "internal.h"

using namespace lbm;

namespace {

// Batch scratch layout: [control 4096 B][per-lattice flags][descriptors][tiles][view region].
constexpr size_t kBatchBarrier = 256;
constexpr size_t kBatchFlags = 4096;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct BatchPlan {
  int n = 0;
  std::vector<Plan> pl;
  std::vector<size_t> off;  // byte offset of each lattice in an arena
  size_t arena = 0;
  size_t desc_off = 0, tiles_off = 0, view_off = 0, scratch = 0;
  size_t max_tiles = 0;
};

// Register-kernel tile shapes (threads x rows); the pipelined variants follow.
const int kShapes[][2] = {{32, 8}, {64, 4}, {128, 2}, {256, 1}, {32, 4}, {64, 2}, {128, 1}};
constexpr int kNumShapes = 7;
const int kTmaWidths[] = {128, 256};
const int kTmaDepths[] = {2, 3, 4};

struct BVariant {
  int kind;  // 0: register tiles (k_batch), 1: bulk-copy pipeline (k_batch_tma)
  int bx, by;
  int X, stages;
};

std::vector<BVariant> batch_variants(const Ops* ops) {
  std::vector<BVariant> v;
  if (ops->batch_tma)
    for (int X : kTmaWidths) {
      if (ops->Q == 27 && X != 256) continue;  // D3Q27 keeps one tile width
      for (int d : kTmaDepths) v.push_back(BVariant{1, 0, 0, X, d});
    }
  for (int k = 0; k < kNumShapes; ++k) v.push_back(BVariant{0, kShapes[k][0], kShapes[k][1], 0, 0});
  return v;
}

size_t tiles_for(const Plan& p, int bx, int by) {
  return (size_t)((p.p.nx + bx - 1) / bx) * ((p.p.ny + by - 1) / by) * p.p.nz;
}

int plan_batch(int n, const lbm_params* p, BatchPlan* out) {
  if (n < 1 || !p) return ctx_fail(LBM_ERR_ARG, "batch needs n >= 1 parameter sets");
  BatchPlan b;
  b.n = n;
  b.pl.resize(n);
  b.off.resize(n);
  long long maxN = 0;
  for (int i = 0; i < n; ++i) {
    int rc = plan(&p[i], &b.pl[i]);
    if (rc) return rc;
    const lbm_params& q = b.pl[i].p;
    if (q.lattice != p[0].lattice || q.storage != p[0].storage || q.collision != p[0].collision)
      return ctx_fail(LBM_ERR_ARG, "batch lattices share lattice, storage and collision");
    if (q.layout != LBM_LAYOUT_AB) return ctx_fail(LBM_ERR_UNSUPPORTED, "batches use the A/B layout");
    b.off[i] = b.arena;
    b.arena += round_up(b.pl[i].pop_bytes, 256);
    if (b.pl[i].N > maxN) maxN = b.pl[i].N;
  }
  for (int s = 0; s < kNumShapes; ++s) {
    size_t t = 0;
    for (int i = 0; i < n; ++i) t += tiles_for(b.pl[i], kShapes[s][0], kShapes[s][1]);
    if (t > b.max_tiles) b.max_tiles = t;
  }
  b.desc_off = round_up(kBatchFlags + (size_t)n * sizeof(unsigned int), 256);
  b.tiles_off = round_up(b.desc_off + (size_t)n * sizeof(BatchDesc), 256);
  b.view_off = round_up(b.tiles_off + b.max_tiles * sizeof(BatchTile), 4096);
  const int D = b.pl[0].D;
  b.scratch = round_up(b.view_off + kFieldOffset + (size_t)(1 + D) * (size_t)maxN * sizeof(double), 256);
  *out = b;
  return LBM_OK;
}

}  // namespace

struct lbm_batch {
  BatchPlan bp;
  cudaStream_t stream = nullptr;   // caller's stream
  cudaStream_t cap = nullptr;      // private stream used for graph capture
  const Ops* ops = nullptr;
  std::vector<lbm_ctx*> views;
  char* A = nullptr;
  char* B = nullptr;
  char* scratch = nullptr;
  bool bound = false;
  int cur = 0;          // 0: state in A, 1: state in B
  long long t = 0;      // completed steps
  int shape = 0;        // variant index into vars
  std::vector<BVariant> vars;
  std::vector<BatchDesc> desc;  // host copy of the descriptors
  bool any_force = false;
  int ntiles = 0;
  bool tiles_ready = false;
  double timeout_s = 2.0;
  int extra = 0;
  long long last_launches = 0;
  int sms = 0;
  std::map<std::tuple<int, int, int, int, int>, cudaGraphExec_t> graphs;  // n, parity, shape, extra, timeout_ms

  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
  }
};

namespace {

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LBM_OK;
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  return ctx_fail(LBM_ERR_CUDA, buf);
}

int upload_tiles(lbm_batch* b) {
  const BVariant& var = b->vars[b->shape];
  if (var.kind == 1) {
    // pipelined kernel: tiles are enumerated from the descriptors
    long long t = 0;
    for (int i = 0; i < b->bp.n; ++i) {
      const Plan& p = b->bp.pl[i];
      BatchDesc& d = b->desc[i];
      d.ntx = (p.p.nx + var.X - 1) / var.X;
      d.tile0 = (int)t;
      t += (long long)d.ntx * p.p.ny * p.p.nz;
      if (t >= (1LL << 31)) return ctx_fail(LBM_ERR_UNSUPPORTED, "batch has too many tiles");
    }
    b->ntiles = (int)t;
    int rc = cuda_fail(cudaMemcpyAsync(b->scratch + b->bp.desc_off, b->desc.data(),
                                       b->desc.size() * sizeof(BatchDesc), cudaMemcpyHostToDevice,
                                       b->stream),
                       "upload descriptors");
    if (rc) return rc;
    rc = cuda_fail(cudaStreamSynchronize(b->stream), "synchronise");
    if (rc) return rc;
    b->tiles_ready = true;
    b->drop_graphs();
    return LBM_OK;
  }
  const int bx = var.bx, by = var.by;
  std::vector<BatchTile> tiles;
  tiles.reserve(b->bp.max_tiles);
  for (int i = 0; i < b->bp.n; ++i) {
    const Plan& p = b->bp.pl[i];
    for (int z = 0; z < p.p.nz; ++z)
      for (int y0 = 0; y0 < p.p.ny; y0 += by)
        for (int x0 = 0; x0 < p.p.nx; x0 += bx) tiles.push_back(BatchTile{i, x0, y0, z});
  }
  b->ntiles = (int)tiles.size();
  int rc = cuda_fail(cudaMemcpyAsync(b->scratch + b->bp.tiles_off, tiles.data(),
                                     tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice,
                                     b->stream),
                     "upload tiles");
  if (rc) return rc;
  rc = cuda_fail(cudaStreamSynchronize(b->stream), "synchronise");
  if (rc) return rc;
  b->tiles_ready = true;
  b->drop_graphs();
  return LBM_OK;
}

BatchLaunch launch_of(lbm_batch* b, int n) {
  BatchLaunch L{};
  L.desc = reinterpret_cast<const BatchDesc*>(b->scratch + b->bp.desc_off);
  L.tiles = reinterpret_cast<const BatchTile*>(b->scratch + b->bp.tiles_off);
  L.ntiles = b->ntiles;
  L.A = b->A;
  L.B = b->B;
  L.nsteps = n;
  L.parity0 = b->cur;
  L.step0 = (unsigned int)(b->t < 0xfffffffeLL ? b->t : 0xfffffffeLL);
  L.flags = reinterpret_cast<unsigned int*>(b->scratch + kBatchFlags);
  L.bar = b->scratch + kBatchBarrier;
  L.timeout_ns = (long long)(b->timeout_s * 1e9);
  L.collision = b->bp.pl[0].kernel_collision;
  const BVariant& var = b->vars[b->shape];
  L.kind = var.kind;
  L.X = var.X;
  L.stages = var.stages;
  L.nlat = b->bp.n;
  L.force = b->any_force;
  L.bx = var.kind == 0 ? var.bx : 0;
  L.by = var.kind == 0 ? var.by : 0;
  const int per_sm = var.kind == 0
                         ? b->ops->batch_blocks_per_sm(L.collision, L.bx * L.by)
                         : b->ops->batch_tma_blocks_per_sm(L.collision, L.force, L.X, L.stages);
  int blocks = per_sm * b->sms;
  if (blocks > b->ntiles) blocks = b->ntiles;
  if (blocks < 1) blocks = 1;
  L.blocks = blocks;
  L.expected = (unsigned int)(blocks + b->extra);
  L.stream = b->stream;
  return L;
}

void sync_views(lbm_batch* b) {
  for (lbm_ctx* v : b->views) ctx_set_state(v, b->cur, b->t);
}

int run_persistent(lbm_batch* b, int n) {
  const int tmo = (int)(b->timeout_s * 1000.0);
  const auto key = std::make_tuple(n, b->cur, b->shape, b->extra, tmo);
  cudaGraphExec_t exec = nullptr;
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) {
    exec = it->second;
  } else {
    BatchLaunch L = launch_of(b, n);
    L.stream = b->cap;
    cudaGraph_t g = nullptr;
    int rc = cuda_fail(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (rc) return rc;
    cudaError_t e1 = cudaMemsetAsync(b->scratch + kBatchBarrier, 0, sizeof(int) * 4, b->cap);
    if (L.blocks < 1 || (L.kind == 1 ? b->ops->batch_tma_blocks_per_sm(L.collision, L.force, L.X,
                                                                          L.stages)
                                        : b->ops->batch_blocks_per_sm(L.collision, L.bx * L.by)) < 1) {
      cudaStreamEndCapture(b->cap, &g);
      if (g) cudaGraphDestroy(g);
      return ctx_fail(LBM_ERR_UNSUPPORTED, "batch variant does not fit on a multiprocessor");
    }
    cudaError_t e2 = e1 == cudaSuccess ? (L.kind == 1 ? b->ops->batch_tma(L) : b->ops->batch(L)) : e1;
    cudaError_t e3 = cudaStreamEndCapture(b->cap, &g);
    if (e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e2, "capture persistent batch kernel");
    }
    rc = cuda_fail(e3, "end capture");
    if (rc) return rc;
    cudaError_t e4 = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    rc = cuda_fail(e4, "instantiate graph");
    if (rc) return rc;
    b->graphs[key] = exec;
  }
  int rc = cuda_fail(cudaGraphLaunch(exec, b->stream), "graph launch");
  if (rc) return rc;
  b->last_launches = 1;
  int err = 0;
  rc = cuda_fail(cudaMemcpyAsync(&err, b->scratch + kBatchBarrier + 2 * sizeof(unsigned int), sizeof(int),
                                 cudaMemcpyDeviceToHost, b->stream),
                 "read barrier status");
  if (rc) return rc;
  rc = cuda_fail(cudaStreamSynchronize(b->stream), "synchronise");
  if (rc) return rc;
  b->cur ^= (n & 1);
  b->t += n;
  sync_views(b);
  if (err) return ctx_fail(LBM_ERR_TIMEOUT, "grid barrier wait ran out");
  return LBM_OK;
}

int run_sequential(lbm_batch* b, int n) {
  long long launches = 0;
  for (int s = 0; s < n; ++s) {
    for (int i = 0; i < b->bp.n; ++i) {
      lbm_ctx* v = b->views[i];
      ctx_set_state(v, b->cur, b->t);
      const std::vector<Variant>& vs = ctx_variants(v);
      StepLaunch sl = ctx_step_launch(v, vs[ctx_variant(v)]);
      sl.flag = reinterpret_cast<unsigned int*>(b->scratch + kBatchFlags) + i;
      cudaError_t e = b->ops->step(sl);
      ++launches;
      if (e != cudaSuccess) return cuda_fail(e, "sequential step launch");
    }
    b->cur ^= 1;
    ++b->t;
  }
  b->last_launches = launches;
  sync_views(b);
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_buffer_sizes(int n, const lbm_params* p, size_t* pop_bytes, size_t* scratch_bytes) {
  BatchPlan bp;
  int rc = plan_batch(n, p, &bp);
  if (rc) return rc;
  if (pop_bytes) *pop_bytes = bp.arena;
  if (scratch_bytes) *scratch_bytes = bp.scratch;
  return LBM_OK;
}

int lbm_batch_create(int n, const lbm_params* p, void* cuda_stream, lbm_batch** out) {
  if (!out) return ctx_fail(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return ctx_fail(LBM_ERR_ARG, "out of host memory");
  int rc = plan_batch(n, p, &b->bp);
  if (rc) {
    delete b;
    return rc;
  }
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  rc = cuda_fail(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "create capture stream");
  if (rc) {
    delete b;
    return rc;
  }
  for (int i = 0; i < n; ++i) {
    lbm_ctx* v = nullptr;
    rc = ctx_new(b->bp.pl[i], b->stream, &v);
    if (rc) {
      for (lbm_ctx* w : b->views) ctx_delete(w);
      cudaStreamDestroy(b->cap);
      delete b;
      return rc;
    }
    ctx_mark_view(v);
    b->views.push_back(v);
  }
  b->ops = ctx_ops(b->views[0]);
  b->vars = batch_variants(b->ops);
  b->shape = 0;  // the first pipelined variant where the storage has one
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) b->any_force |= b->bp.pl[i].p.force[a] != 0.0;
  *out = b;
  return LBM_OK;
}

int lbm_batch_bind(lbm_batch* b, void* pop_a, void* pop_b, void* scratch) {
  if (!b || !pop_a || !pop_b || !scratch) return ctx_fail(LBM_ERR_ARG, "NULL argument");
  if ((reinterpret_cast<uintptr_t>(pop_a) | reinterpret_cast<uintptr_t>(pop_b) |
       reinterpret_cast<uintptr_t>(scratch)) & 255u)
    return ctx_fail(LBM_ERR_ALIGN, "buffers must be 256-byte aligned");
  b->A = static_cast<char*>(pop_a);
  b->B = static_cast<char*>(pop_b);
  b->scratch = static_cast<char*>(scratch);
  b->cur = 0;
  b->t = 0;
  std::vector<BatchDesc>& desc = b->desc;
  desc.assign(b->bp.n, BatchDesc{});
  for (int i = 0; i < b->bp.n; ++i) {
    const Plan& p = b->bp.pl[i];
    desc[i].g = p.g;
    desc[i].cd = p.coef;
    desc[i].cf = coef_cast<float>(p.coef);
    desc[i].off = (long long)b->bp.off[i];
    ctx_bind(b->views[i], b->A + b->bp.off[i], b->B + b->bp.off[i], nullptr, b->scratch + b->bp.view_off);
    ctx_set_flag(b->views[i], reinterpret_cast<unsigned int*>(b->scratch + kBatchFlags) + i);
  }
  int rc = cuda_fail(cudaMemsetAsync(b->scratch + kBatchFlags, 0xff, sizeof(unsigned int) * b->bp.n, b->stream),
                     "reset flags");
  if (rc) return rc;
  rc = cuda_fail(cudaMemcpyAsync(b->scratch + b->bp.desc_off, desc.data(), desc.size() * sizeof(BatchDesc),
                                 cudaMemcpyHostToDevice, b->stream),
                 "upload descriptors");
  if (rc) return rc;
  b->bound = true;
  return upload_tiles(b);
}

int lbm_batch_lattice(lbm_batch* b, int i, lbm_ctx** view) {
  if (!b || !view || i < 0 || i >= b->bp.n) return ctx_fail(LBM_ERR_ARG, "bad lattice index");
  *view = b->views[i];
  return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int n, int mode) {
  if (!b || n < 0 || (mode != 0 && mode != 1)) return ctx_fail(LBM_ERR_ARG, "bad argument");
  if (!b->bound || !b->tiles_ready) return ctx_fail(LBM_ERR_STATE, "batch buffers not bound");
  if (n == 0) return LBM_OK;
  // Views may have been re-initialised (init_equilibrium puts the state in A).
  for (lbm_ctx* v : b->views) {
    int cur;
    long long t;
    ctx_get_state(v, &cur, &t);
    if (cur != b->cur || t != b->t) {
      if (t == 0 && cur == 0) {
        continue;  // freshly initialised view; reconciled below
      }
      return ctx_fail(LBM_ERR_STATE, "batch views were stepped or restored individually");
    }
  }
  bool fresh = false;
  for (lbm_ctx* v : b->views) {
    int cur;
    long long t;
    ctx_get_state(v, &cur, &t);
    fresh |= (t == 0 && cur == 0 && (b->t != 0 || b->cur != 0));
  }
  if (fresh) {
    for (lbm_ctx* v : b->views) {
      int cur;
      long long t;
      ctx_get_state(v, &cur, &t);
      if (!(t == 0 && cur == 0)) return ctx_fail(LBM_ERR_STATE, "re-initialise every lattice of the batch");
    }
    b->cur = 0;
    b->t = 0;
  }
  return mode == 0 ? run_persistent(b, n) : run_sequential(b, n);
}

int lbm_batch_variant_count(const lbm_batch* b, int* n) {
  if (!b || !n) return ctx_fail(LBM_ERR_ARG, "NULL argument");
  *n = (int)b->vars.size();
  return LBM_OK;
}

int lbm_batch_variant_name(const lbm_batch* b, int v, char* buf, size_t len) {
  if (!b || !buf || v < 0 || v >= (int)b->vars.size()) return ctx_fail(LBM_ERR_ARG, "bad variant");
  const BVariant& var = b->vars[v];
  if (var.kind == 1) snprintf(buf, len, "tma_X%d_s%d", var.X, var.stages);
  else snprintf(buf, len, "tile_b%dx%d", var.bx, var.by);
  return LBM_OK;
}

int lbm_batch_set_variant(lbm_batch* b, int v) {
  if (!b || v < 0 || v >= (int)b->vars.size()) return ctx_fail(LBM_ERR_ARG, "bad variant");
  if (b->shape == v && b->tiles_ready) return LBM_OK;
  b->shape = v;
  if (!b->bound) return LBM_OK;
  return upload_tiles(b);
}

int lbm_batch_autotune(lbm_batch* b, int steps, int* chosen, float* times_ms) {
  if (!b) return ctx_fail(LBM_ERR_ARG, "NULL argument");
  if (!b->bound) return ctx_fail(LBM_ERR_STATE, "batch buffers not bound");
  if (steps < 2) steps = 2;
  steps += steps & 1;  // even: the state returns to the same arena
  cudaEvent_t e0, e1;
  int rc = cuda_fail(cudaEventCreate(&e0), "event");
  if (rc) return rc;
  rc = cuda_fail(cudaEventCreate(&e1), "event");
  if (rc) {
    cudaEventDestroy(e0);
    return rc;
  }
  int best = b->shape;
  float best_ms = 1e30f;
  for (int v = 0; v < (int)b->vars.size() && rc == LBM_OK; ++v) {
    rc = lbm_batch_set_variant(b, v);
    if (rc) break;
    rc = run_persistent(b, steps);  // capture + warm-up
    if (rc) break;
    cudaEventRecord(e0, b->stream);
    rc = run_persistent(b, steps);
    if (rc) break;
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= steps;
    if (times_ms) times_ms[v] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (chosen) *chosen = best;
  return lbm_batch_set_variant(b, best);
}

int lbm_batch_set_barrier(lbm_batch* b, double timeout_s, int extra) {
  if (!b || !(timeout_s > 0.0) || timeout_s > 60.0 || extra < 0)
    return ctx_fail(LBM_ERR_ARG, "timeout in (0, 60] s and extra >= 0");
  b->timeout_s = timeout_s;
  b->extra = extra;
  return LBM_OK;
}

int lbm_batch_launches(const lbm_batch* b, long long* launches) {
  if (!b || !launches) return ctx_fail(LBM_ERR_ARG, "NULL argument");
  *launches = b->last_launches;
  return LBM_OK;
}

int lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  b->drop_graphs();
  for (lbm_ctx* v : b->views) ctx_delete(v);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return LBM_OK;
}

}  // extern "C"
