/*
 * lbm.h -- C ABI of the GB300 (sm_103a) library for the Purified
 * Two-Relaxation-Time (P-TRT) lattice Boltzmann update of Yu et al.,
 * arXiv 2602.06686, with the standard TRT and TRT-RLB comparators.
 *
 * What the library computes, per node and time step (a fused pull-stream +
 * collide update):
 *   f_i(x, t+1) = f*_i(x - e_i, t), or f*_ibar(x, t) when x - e_i is solid or
 *   outside a non-periodic axis (halfway bounce-back, Sec. 3.3 and Sec. 3.4),
 *   f* = f_eq + (1 - w+) R2 + (1 - w-) R3 + F_i/2 + (1 - w+/2) S+     (Eq. PTRT)
 * with rho and the half-force velocity u of Eq. macro, the third-order
 * equilibrium of Eq. feq, F_i = w_i e_i.F / cs^2, the symmetric Guo source
 * S+ = w_i [(e_i.u)(e_i.F)/cs^4 - u.F/cs^2] (Eq. source_guo) and
 *   P-TRT    R2 = fneq+ - P_G fneq (ghost subtraction, Thm 2nd), R3 = fneq- + F_i/2 (Eq. R3_force)
 *   TRT      R2 = fneq+,                                         R3 = fneq- + F_i/2
 *   TRT-RLB  R2, R3 = orthogonal projections of fneq onto span{H2}, span{H3} (Eq. R2R3_hermite)
 *   BGK      TRT with w- = w+;  RLB: P-TRT with w- = 1 (second-order regularised, single rate).
 * The force term "F_i/2 + (1-w-) (fneq- + F_i/2)" is the reading under which the
 * update conserves mass exactly and adds the impulse F (Eq. macro): Eq. PTRT as
 * printed omits the first-order term (1 - w+) R1 and Scheme I attaches -u.F/cs^2
 * to tau_s2.  On D3Q19 the ghost subspace is the orthogonal complement of
 * span{1, H2} in the symmetric subspace (the printed App. A.2 products are not
 * orthogonal).
 *
 * Rates: tau+ = 1/2 + nu/cs^2 (Eq. viscosity), tau- = 1/2 + Lambda/(tau+ - 1/2)
 * (Sec. 3.2, magic parameter Lambda_s).  cs^2 = 1/3.
 *
 * Lattices and population order:
 *   D2Q9  (Eq. D2Q9): 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1), 5 (1,1),
 *         6 (-1,1), 7 (-1,-1), 8 (1,-1); w = 4/9, 1/9, 1/36.
 *   D3Q19 (App. A.2, order not printed): 0 rest; 1..6 = +x,-x,+y,-y,+z,-z;
 *         7..10 = (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0); 11..14 = (1,0,1),(-1,0,-1),
 *         (1,0,-1),(-1,0,1); 15..18 = (0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1);
 *         w = 1/3, 1/18, 1/36.
 *   D3Q27 (App. D3Q27, order and weights not printed): 0..18 as D3Q19; 19..26 =
 *         (1,1,1),(-1,-1,-1),(1,1,-1),(-1,-1,1),(1,-1,1),(-1,1,-1),(-1,1,1),(1,-1,-1);
 *         w = 8/27, 2/27, 1/54, 1/216 (products of the D1Q3 weights).
 *         P-TRT on D3Q27 is the hybrid of Eq. PTRT_D3Q27: R2 the tensor (Hermite)
 *         projection, R3 = fneq- + F_i/2 (the fifth-order residual kept); TRT-RLB
 *         is the exact operator of the appendix (the residual removed).
 *
 * Conventions common to every call:
 *   - Device buffers are allocated by the caller and borrowed by the library
 *     (bound with lbm_bind_buffers); the library never allocates device memory.
 *     It allocates only its host-side context.
 *   - "device" pointers must be addresses in the current CUDA device's memory
 *     (or managed memory); "host" pointers are ordinary host memory.  Device
 *     FP64 fields must be 8-byte aligned (else LBM_ERR_ALIGN, before any
 *     launch); host fields of any alignment are accepted.
 *   - Field layout: scalar fields are [nz][ny][nx] (x fastest, no padding),
 *     vector fields are D consecutive scalar fields (component planes), and
 *     decoded populations are Q consecutive scalar fields, all FP64.
 *   - All work is enqueued on the stream given to lbm_create, asynchronously,
 *     unless a call says it synchronises.
 *   - Return value: LBM_OK (0) or a negative LBM_ERR_* code; nothing is thrown
 *     across the ABI and nothing exits the process.  lbm_strerror names a code.
 *     A NULL context, batch, parameter block or required output pointer is
 *     LBM_ERR_ARG, found before any CUDA call.
 *   - The time level: after lbm_init_equilibrium / lbm_set_populations and any
 *     number of lbm_step calls, lbm_macros and lbm_get_populations describe the
 *     pre-collision state f(x, t).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_ERR_ARG (-1)         /* invalid argument, size or pointer */
#define LBM_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define LBM_ERR_DIVERGED (-3)    /* NaN/Inf, rho <= 0 or |u| > 1 seen in an update */
#define LBM_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up */
#define LBM_ERR_UNSUPPORTED (-5) /* valid but not implemented combination */
#define LBM_ERR_STATE (-6)       /* call out of order (e.g. buffers not bound) */
#define LBM_ERR_ALIGN (-7)       /* a buffer is not aligned as required: 256 bytes for
                                    population, mask and scratch buffers, 8 bytes for
                                    FP64 device fields */

typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D3Q27 = 2 } lbm_lattice;
typedef enum {
  LBM_TRT = 0,
  LBM_TRT_RLB = 1,
  LBM_P_TRT = 2,
  LBM_BGK = 3,
  LBM_RLB = 4
} lbm_collision;
/* Storage of populations.  Every format stores the shifted value
 * df_i = f_i - w_i rho0 (round to nearest even); FP16/BF16 keep gradual
 * underflow.  Arithmetic is FP64 for LBM_F64 and FP32 otherwise. */
typedef enum {
  LBM_F64 = 0,
  LBM_F32 = 1,
  LBM_F16_SHIFTED = 2,
  LBM_BF16_SHIFTED = 3
} lbm_storage;
/* A/B: two buffers, read one, write the other.  AA: one buffer updated in place,
 * even steps local, odd steps neighbour-wise (halves the memory). */
typedef enum { LBM_LAYOUT_AB = 0, LBM_LAYOUT_AA = 1 } lbm_layout;

typedef struct {
  int lattice;           /* lbm_lattice */
  int nx, ny, nz;        /* lattice extent; nz = 1 for D2Q9 */
  double nu;             /* kinematic viscosity; or 0 and tau_plus > 0 */
  double tau_plus;       /* tau_s1; or 0 and nu > 0 */
  double Lambda;         /* magic parameter Lambda_s; or 0 and tau_minus > 0 */
  double tau_minus;      /* tau_s2; or 0 and Lambda > 0 */
  int collision;         /* lbm_collision */
  double force[3];       /* uniform body force (lattice units) */
  double rho0;           /* reference density of the shifted storage (e.g. 1) */
  int periodic[3];       /* 1 = periodic axis; 0 = halfway bounce-back walls just
                            outside the first and last node of that axis */
  int storage;           /* lbm_storage */
  int layout;            /* lbm_layout */
} lbm_params;

typedef struct lbm_ctx lbm_ctx;

/* Library version, e.g. 100 for 1.0.0. */
int lbm_version(void);

/* Static description of an error code (never NULL). */
const char* lbm_strerror(int code);

/* Byte sizes of the buffers a lattice needs: *pop_bytes for ONE population
 * buffer (A/B layout needs two, AA one) and *scratch_bytes for the scratch
 * buffer (diagnostics, host staging, status words).  Either output may be NULL.
 * Returns LBM_ERR_ARG for invalid parameters. */
int lbm_buffer_sizes(const lbm_params* p, size_t* pop_bytes, size_t* scratch_bytes);

/* Validates parameters, derives the rates and creates a context that enqueues
 * on `cuda_stream` (a cudaStream_t; NULL = legacy default stream) on the
 * current device.  The context is not usable for compute until buffers are
 * bound.  *out receives the context (owned by the caller; lbm_destroy frees). */
int lbm_create(const lbm_params* p, void* cuda_stream, lbm_ctx** out);

/* Binds caller-owned device buffers, all 256-byte aligned:
 *   pop_a, pop_b  population buffers of lbm_buffer_sizes' pop_bytes each
 *                 (pop_b must be NULL for the AA layout);
 *   solid_mask    uint8 [nz][ny][nx], nonzero = solid node, or NULL for none;
 *                 it is read at every step and must stay valid while bound;
 *   scratch       scratch_bytes of device memory.
 * The buffers must not overlap.  No data is read or written by this call. */
int lbm_bind_buffers(lbm_ctx* ctx, void* pop_a, void* pop_b, const uint8_t* solid_mask,
                     void* scratch);

/* Sets the state to the equilibrium f = f_eq(rho, u) (Eq. feq) and the step
 * counter to 0.  rho: device FP64 [N]; u: device FP64 [D][N]. */
int lbm_init_equilibrium(lbm_ctx* ctx, const double* rho, const double* u);

/* As lbm_init_equilibrium with HOST inputs; synchronises the stream before
 * returning.  Page-locked buffers mapped into the device's address space
 * (cudaHostAlloc, cudaHostRegister, torch pin_memory) are read in place by the
 * init kernel over the host link; other host memory is copied through the
 * scratch buffer first. */
int lbm_init_equilibrium_host(lbm_ctx* ctx, const double* rho, const double* u);

/* Advances n >= 0 time steps (the hot path).  Asynchronous; returns launch
 * status only.  Divergence is recorded on the device and reported by
 * lbm_status / lbm_diagnostics. */
int lbm_step(lbm_ctx* ctx, int n);

/* Density and half-force velocity (Eq. macro) of the current pre-collision
 * state into device FP64 buffers rho [N] and u [D][N].  Solid nodes get rho0, 0. */
int lbm_macros(lbm_ctx* ctx, double* rho, double* u);

/* As lbm_macros into HOST buffers; synchronises the stream.  Page-locked,
 * mapped buffers are written in place by the macros kernel; other host memory
 * receives a copy from the scratch buffer. */
int lbm_macros_host(lbm_ctx* ctx, double* rho, double* u);

/* Decoded FP64 pre-collision populations f [Q][N] (device).  Solid nodes: w_i rho0. */
int lbm_get_populations(lbm_ctx* ctx, double* f);

/* Replaces the state by the FP64 pre-collision populations f [Q][N] (device),
 * encoded to the storage format.  Values at solid nodes are ignored. */
int lbm_set_populations(lbm_ctx* ctx, const double* f);

/* FP64 diagnostics of the current state over fluid nodes, synchronising:
 *   out[0] mass sum rho, out[1..3] momentum sum rho u, out[4] kinetic energy
 *   1/2 sum rho |u|^2, out[5] enstrophy 1/2 sum |curl u|^2 with second-order
 *   central differences (a neighbour across a periodic axis wraps; across a
 *   non-periodic edge or on a solid node it counts as u = 0), out[6] 1 if any
 *   rho or u is not finite or rho <= 0, out[7] the step counter.
 * Per node, rho and u are formed in the update's arithmetic precision (FP32
 * for FP32/FP16/BF16 storage, FP64 for FP64 storage); the sums over nodes are
 * exact-rounded per thread (TwoSum) and carried in FP64 across threads and
 * blocks in a fixed order, so repeated calls on a state are bit-identical. */
int lbm_diagnostics(lbm_ctx* ctx, double out[8]);

/* Relative L2 error (Sec. 3) of the current velocity against u_ref (device
 * FP64 [D][N]) over fluid nodes: sqrt(sum |u - u_ref|^2 / sum |u_ref|^2).
 * Synchronises. */
int lbm_velocity_l2(lbm_ctx* ctx, const double* u_ref, double* out);

/* Open boundaries of the square-cylinder benchmark (Sec. 3.4), D2Q9 with the A/B
 * layout and a non-periodic x axis: the left boundary imposes the uniform
 * velocity (u_in, 0) by halfway bounce-back from a wall moving with it (the wall
 * half a spacing left of x = 0, density rho0), the right boundary is a
 * constant-pressure outlet by the Zou-He scheme (density rho_out and zero
 * transverse velocity at the nodes x = nx - 1).  The other axes keep their
 * periodic / wall settings.  rho_out <= 0 turns them off.  While on, lbm_step
 * runs a one-node-per-thread kernel that applies them (the variant is ignored)
 * and lbm_macros, lbm_get_populations and lbm_diagnostics report the state with
 * them applied.  A state written directly (lbm_init_equilibrium,
 * lbm_set_populations, lbm_restore at t = 0) is taken as given: the rules act
 * from the first streaming on.  LBM_ERR_UNSUPPORTED for D3Q19, D3Q27 or AA,
 * LBM_ERR_ARG for a periodic x axis, nx < 2 or |u_in| >= 1. */
int lbm_set_open_boundaries(lbm_ctx* ctx, double u_in, double rho_out);

/* Body-force scheme of the update (Sec. 2.1): 1 (default) the Guo source of
 * Eq. source_guo, taken with the single factor (1 - w+/2) so that mass is
 * conserved for every tau_s2; 2 the simplified projection of Eq. source_simple,
 * (1 - w+/2) w_i e_i.F / cs^2 plus the cubic-velocity correction G_i of Eq. Gi,
 * -(1 - w+/2) w_i H2_i,ab d_g Phi_abg / (6 cs^6) with Phi_aaa = rho u_a^3 (the
 * only non-zero entries; on D3Q19 also Phi_zzz).  G_i is applied with or
 * without a force.  Its derivative is taken at time t from the pre-collision
 * rho and half-force u: second-order central differences along each axis, the
 * one-sided difference where one neighbour is a solid node or beyond a
 * non-periodic edge, 0 where both are.  Scheme 2 runs two launches per step: a
 * pass that stores rho u_a^3 of every node in the scratch buffer's field area,
 * then the update.  On the A/B layout without a solid mask and with rows of
 * whole 16-byte units both run on the pipelined kernel (the update copies the
 * rho u^3 rows a tile needs through its ring) with the tile width and ring
 * depth of the selected pipelined variant, or the widest tile under a
 * register variant; otherwise
 * (a solid mask, the AA layout -- updated in place -- or D3Q27) on
 * one-node-per-thread kernels.  It changes neither the state's layout nor
 * lbm_macros / lbm_diagnostics.
 * LBM_ERR_ARG for another value; LBM_ERR_UNSUPPORTED for scheme 2 with open
 * boundaries on (lbm_set_open_boundaries and lbm_momentum_exchange also
 * refuse scheme 2); LBM_ERR_STATE on a batch view. */
int lbm_set_forcing_scheme(lbm_ctx* ctx, int scheme);

/* Force on the solid nodes by momentum exchange (Sec. 3.4), FP64, into out[3]:
 * with halfway bounce-back from resting solids every link from a fluid node to
 * a solid neighbour transfers 2 e_i f*_i, f* the collision of the current state
 * (the force of the next streaming step).  Neighbours beyond a non-periodic
 * edge are walls and not counted.  The drag coefficient of Sec. 3.4 is
 * C_d = 2 out[0] / (rho0 u_c^2 D).  Synchronises.  LBM_ERR_UNSUPPORTED under
 * forcing scheme 2. */
int lbm_momentum_exchange(lbm_ctx* ctx, double out[3]);

/* Synchronises the stream and reports LBM_ERR_DIVERGED if any update since the
 * last lbm_init_equilibrium / lbm_set_populations met NaN/Inf, rho <= 0 or
 * |u| > 1; *first_step (may be NULL) receives the earliest such step or -1. */
int lbm_status(lbm_ctx* ctx, long long* first_step);

/* Diagnostics without a scratch buffer (the paper has no counterpart; this is
 * a library facility).  For callers that cannot allocate device memory for
 * lbm_bind_buffers' scratch: for example a program whose device memory belongs
 * to another framework's pool, or a tool attached to a running simulation that
 * must not grow its footprint.  It computes the eight values of
 * lbm_diagnostics for the state held in `pop_state` and writes them to `out`
 * (device, 8 FP64) asynchronously on `cuda_stream`:
 *   p           the lattice's parameters (as given to lbm_create);
 *   pop_state   device buffer holding the current state (256-byte aligned, as
 *               for lbm_bind_buffers, and so is solid_mask; out 8-byte aligned;
 *               else LBM_ERR_ALIGN before any CUDA call): for the A/B layout
 *               the buffer the next step reads (pop_a after an even number of
 *               steps since initialisation, pop_b after an odd one), for AA the
 *               single buffer;
 *   solid_mask  device uint8 [nz][ny][nx] or NULL, as bound to the context;
 *   open_bc     host {u_in, rho_out} of lbm_set_open_boundaries, or NULL.  Pass
 *               it for a state that the update with open boundaries streamed
 *               (lbm_diagnostics then applies the inlet and outlet rules to the
 *               gathered populations); pass NULL for a lattice without open
 *               boundaries and for a state written directly and not stepped
 *               since (lbm_init_equilibrium, lbm_set_populations).  The same
 *               conditions as lbm_set_open_boundaries apply (D2Q9, A/B,
 *               x non-periodic, |u_in| < 1, rho_out > 0), else LBM_ERR_ARG or
 *               LBM_ERR_UNSUPPORTED;
 *   steps_done  steps completed since initialisation (selects the AA slot
 *               rule and is stored in out[7]).
 * For the same state it returns the same bits as lbm_diagnostics (the same
 * kernels and reduction order).  It allocates nothing: its working memory is
 * one fixed array of about 8.7 MB inside the library, which every GPU that
 * loads the library holds until the process exits.  Lattices of more than
 * 262144 nodes (e.g. 512 x 512, 64^3) are rejected with LBM_ERR_ARG.  The first
 * call in a CUDA context looks the array up (cudaGetSymbolAddress) with that
 * context current; make that first call before any stream capture.  All calls
 * on a device share the array, so calls whose work overlaps on the GPU race;
 * the array keeps the last call's contents. */
int lbm_diagnostics_noalloc(const lbm_params* p, const void* pop_state, const uint8_t* solid_mask,
                            const double* open_bc, long long steps_done, double* out,
                            void* cuda_stream);

/* Number of completed time steps since initialisation. */
int lbm_step_count(const lbm_ctx* ctx, long long* t);

/* Raw checkpoint of the state: copies the buffer that holds the current state
 * (pop_bytes, storage format, layout-dependent) to `dst` (device) and returns the
 * step counter in *t.  lbm_restore copies such a snapshot back and sets the step
 * counter, so that a resumed run is bit-identical to an uninterrupted one.
 * Both are asynchronous on the context's stream. */
int lbm_checkpoint(lbm_ctx* ctx, void* dst, size_t bytes, long long* t);
int lbm_restore(lbm_ctx* ctx, const void* src, size_t bytes, long long t);

/* Number of kernels this context has enqueued since creation (all entry points). */
int lbm_launch_count(const lbm_ctx* ctx, long long* launches);

/* Limit, in seconds (0 < limit <= 60, default 2), of every bounded wait of the
 * pipelined kernel variant (its shared-memory stage barriers).  For tests:
 * test_extra_bytes > 0 makes every stage wait for that many bytes that never
 * arrive, so each wait runs out, the kernel returns, and lbm_status reports
 * LBM_ERR_TIMEOUT; pass 0 to run normally. */
int lbm_set_wait_limit(lbm_ctx* ctx, double seconds, int test_extra_bytes);

/* Text of the most recent error raised in the calling thread (CUDA error name
 * and the call that failed), or "" if none. */
const char* lbm_last_error(void);

/* Kernel variants (nodes per thread, block shape) available for this context,
 * their names, the selected one, and selection by index.  lbm_set_variant runs
 * every step with the chosen variant; on the AA layout lbm_autotune may choose
 * another for the odd steps (lbm_get_variant reports the even steps' one). */
int lbm_variant_count(const lbm_ctx* ctx, int* n);
int lbm_variant_name(const lbm_ctx* ctx, int v, char* buf, size_t len);
int lbm_get_variant(const lbm_ctx* ctx, int* v);
int lbm_set_variant(lbm_ctx* ctx, int v);

/* Times every variant (reps steps each, CUDA events, after one warm-up) and
 * selects the fastest; *chosen (may be NULL) receives it, times_ms (may be
 * NULL, length lbm_variant_count) the per-step times.  A/B layout: the state
 * is not changed (trial steps read the current buffer and write the other one,
 * which the next step overwrites).  AA layout: there is no spare buffer, so the
 * trials are real steps in pairs (even, odd): the lattice advances by
 * 2 (reps + 1) or 2 reps + 3 steps per variant and the step counter with it;
 * the even and odd steps are different kernels and each gets its own fastest
 * variant (times_ms then holds the mean of the two per variant).  Results are
 * cached per (lattice, storage, collision, mask, extent, layout, forcing
 * scheme) for the process; a cached answer (times_ms NULL) runs nothing.
 * Under forcing scheme 2 the trials are scheme-2 steps.  Synchronises. */
int lbm_autotune(lbm_ctx* ctx, int reps, int* chosen, float* times_ms);

/* Frees the context (not the bound buffers); NULL is a no-op (LBM_OK).  A
 * lattice view of a batch is LBM_ERR_STATE: lbm_batch_destroy frees it. */
int lbm_destroy(lbm_ctx* ctx);

/* Streaming copy kernel (128-bit loads/stores, grid-stride) of `bytes` from
 * src to dst (device, 16-byte aligned, bytes a multiple of 16) on a stream: the
 * measured copy ceiling for the bandwidth roofline. */
int lbm_copy_ceiling(const void* src, void* dst, size_t bytes, void* cuda_stream);

/* ---------------------------------------------------------------- batches
 * Many independent lattices stepped together by ONE persistent kernel (one
 * cooperative launch for all steps, a bounded grid barrier between steps),
 * replayed from a CUDA graph.  All lattices share lattice, collision,
 * storage and layout (A/B); extents, rates and forces are per lattice.
 */
typedef struct lbm_batch lbm_batch;

/* Per-lattice population offsets are packed in lattice order; *pop_bytes is the
 * size of ONE arena (two are needed), *scratch_bytes of the scratch buffer. */
int lbm_batch_buffer_sizes(int n, const lbm_params* p, size_t* pop_bytes, size_t* scratch_bytes);

int lbm_batch_create(int n, const lbm_params* p, void* cuda_stream, lbm_batch** out);

/* Binds the two population arenas and the scratch buffer (device, 256-byte aligned). */
int lbm_batch_bind(lbm_batch* b, void* pop_a, void* pop_b, void* scratch);

/* A context that views lattice i of the batch (its slice of the arenas and the
 * shared scratch): lbm_init_equilibrium, lbm_macros, lbm_get_populations,
 * lbm_diagnostics ... work on it.  Owned by the batch; do not destroy it and
 * do not lbm_step it (lbm_batch_step advances every view). */
int lbm_batch_lattice(lbm_batch* b, int i, lbm_ctx** view);

/* Advances every lattice by n steps.  mode 0: the persistent cooperative kernel
 * captured once per n in a CUDA graph and replayed; mode 1: one ordinary launch
 * per lattice per step (the sequential baseline).  Returns LBM_ERR_TIMEOUT if a
 * grid barrier gave up (the state is then undefined), after synchronising. */
int lbm_batch_step(lbm_batch* b, int n, int mode);

/* Variants of the persistent kernel and the autotuner, as for single lattices
 * (mode-0 timing).  "tma_X<w>_s<d>" (FP32/FP16/BF16 storage; the default): the
 * bulk-copy pipeline over row segments of w nodes with a d-stage shared-memory
 * ring; "tile_b<x>x<y>": register tiles of x nodes by y rows. */
int lbm_batch_variant_count(const lbm_batch* b, int* n);
int lbm_batch_variant_name(const lbm_batch* b, int v, char* buf, size_t len);
int lbm_batch_set_variant(lbm_batch* b, int v);
int lbm_batch_autotune(lbm_batch* b, int steps, int* chosen, float* times_ms);

/* Grid-barrier wait limit in seconds (default 2.0).  For tests: `extra` > 0
 * makes each barrier wait for `extra` arrivals that never come, so the wait
 * must run out and lbm_batch_step must return LBM_ERR_TIMEOUT. */
int lbm_batch_set_barrier(lbm_batch* b, double timeout_s, int extra);

/* Number of kernel launches the last lbm_batch_step enqueued. */
int lbm_batch_launches(const lbm_batch* b, long long* launches);

/* Frees the batch and its lattice views; NULL is a no-op (LBM_OK). */
int lbm_batch_destroy(lbm_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
