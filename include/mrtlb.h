/*
 * mrtlb.h - C ABI of the GB300 implementation of the MRT finite-difference
 * lattice Boltzmann (FD-LB) model for compressible flow of Chen, Xu, Zhang &
 * Li, "Prandtl number effects in MRT lattice Boltzmann models for shocked and
 * unshocked compressible fluids" (arXiv:1106.0785).
 *
 * The model (Sec. II): sixteen discrete velocities v_i (Fig. 1), moments
 * f^ = M f with the SO(2) matrix M, collision -M^-1 S^ (f^ - f^eq) with the
 * equilibria of Eqs. 14a-14i, and the modified energy-flux relaxation for
 * moments 7 and 8 (the two rules following Eq. 16c).  The space-time scheme
 * is the one whose amplification matrix G is given in Sec. III: forward Euler
 * in time and a Lax-Wendroff difference along each axis.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns an mrtlb_status (0 = MRTLB_OK).  mrtlb_last_error()
 *   gives a human-readable message for the last failure on a context.
 * - Arrays on the host are borrowed for the duration of the call only.
 * - Device state buffers are owned by the caller (e.g. PyTorch tensors) and
 *   must outlive the context; the context owns only its own small scratch
 *   (staging for host copies, reduction accumulators, the error word), which
 *   mrtlb_destroy frees.
 * - Work is enqueued on the context's CUDA stream (params.stream, NULL = the
 *   legacy default stream).  mrtlb_step is asynchronous; a non-physical state
 *   (rho <= 0, T <= 0 or a non-finite value) met by a kernel is latched in a
 *   device error word and reported as MRTLB_ERR_NONPHYSICAL by the next
 *   synchronising call (mrtlb_macros, mrtlb_get_f, mrtlb_reduce,
 *   mrtlb_sync), as is an expired bounded wait (MRTLB_ERR_TIMEOUT).  The
 *   word stays set until a new state is set (mrtlb_init_equilibrium,
 *   mrtlb_set_f).
 * - Dense field layouts: a scalar field is [ny][nx] (x fastest); the
 *   distributions are [16][ny][nx], plane q = the paper's velocity i = q+1.
 * - Threads: calls on one context (or one batch, with its instances) must not
 *   overlap; different contexts may be driven from different host threads at
 *   the same time.  mrtlb_last_error(NULL) reports the calling thread's
 *   last failed mrtlb_create.
 */
#ifndef MRTLB_H
#define MRTLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MRTLB_NQ 16

typedef struct mrtlb_ctx mrtlb_ctx;

typedef enum {
  MRTLB_OK = 0,
  MRTLB_ERR_ARG = -1,          /* invalid argument, size or stability limit */
  MRTLB_ERR_UNSUPPORTED = -2,  /* velocity set or M other than the paper's */
  MRTLB_ERR_SINGULAR = -3,     /* M not invertible */
  MRTLB_ERR_CUDA = -4,         /* a CUDA runtime call failed */
  MRTLB_ERR_NONPHYSICAL = -5,  /* rho <= 0, T <= 0 or non-finite state met */
  MRTLB_ERR_TIMEOUT = -6,      /* a bounded device-side wait gave up */
  MRTLB_ERR_STATE = -7         /* call out of order (e.g. step before bind) */
} mrtlb_status;

typedef enum {
  MRTLB_BC_PERIODIC = 0,  /* ghost = opposite edge (Sec. IV A, IV B) */
  MRTLB_BC_OUTFLOW = 1,   /* zero-gradient extrapolation (Sec. IV B) */
  MRTLB_BC_WALL_NEE = 2,  /* non-equilibrium extrapolation wall (Sec. IV A) */
  MRTLB_BC_INFLOW = 3,    /* fixed state: ghost = f^eq(rho, u, T) of the side
                             (the shock-bubble's post-shock side, Sec. IV B) */
  MRTLB_BC_REFLECT = 4,   /* specular reflection: ghost = the edge node with
                             the velocity set mirrored across the side (Sec.
                             IV B, "reflection conditions") */
  MRTLB_BC_DIFFUSE = 5    /* diffuse reflection (Sec. IV A): velocities entering
                             the fluid leave the wall with rho_w f^eq(1, u_w,
                             T_w), the others copy the edge node; rho_w makes
                             the Lax-Wendroff update move no mass across the
                             side.  Refilled before every step. */
} mrtlb_bc_kind;

typedef enum { MRTLB_FP32 = 0, MRTLB_FP64 = 1 } mrtlb_precision;

typedef struct {
  int kind;        /* mrtlb_bc_kind */
  double ux, uy;   /* wall or inflow velocity (MRTLB_BC_WALL_NEE, _INFLOW, _DIFFUSE) */
  double T;        /* wall or inflow temperature (> 0 there) */
  double rho;      /* inflow density (MRTLB_BC_INFLOW only; > 0) */
} mrtlb_bc;

typedef struct {
  int nvel;          /* number of discrete velocities; must be 16 */
  const double* v;   /* nvel x 2 row-major (v_x, v_y): must be the D2V16 set of
                        Fig. 1 in the order fixed by rows m2, m3 of M */
  const double* M;   /* nvel x nvel row-major: must equal the paper's M */
  const double* s;   /* nvel relaxation rates s_1..s_16 (Sec. II), or NULL to
                        derive them: s5 = s6 = s_visc, s7 = s8 = Pr * s_visc,
                        all others s_other (Pr = s7/s5 = s8/s6 follows from
                        mu = rho T / s5, lambda = 2 rho T / s7, c_p = 2) */
  double Pr, s_visc, s_other;
  int eq_version;    /* equilibria of moments 12, 15, 16: 1, 2 or 3 (Sec. II) */
  int modified;      /* 1 = the paper's modified energy-flux collision */
  int nx, ny;        /* grid nodes along x and y */
  double dx, dy, dt; /* node spacings and time step */
  mrtlb_bc bc[4];    /* sides -x, +x, -y, +y; periodic sides come in pairs and
                        walls may sit on one axis only */
  int precision;     /* MRTLB_FP32: f stored and advanced in FP32, the
                        temperature numerator compensated to about twice FP32
                        precision; MRTLB_FP64: everything in FP64 */
  void* stream;      /* cudaStream_t to enqueue on; NULL = legacy default */
} mrtlb_params;

/* Validate params and build a context (host only, no device work).
 * Rejects a velocity set or M other than the paper's with
 * MRTLB_ERR_UNSUPPORTED; a Lax-Wendroff CFL number max|v_a| dt/d_a above 1
 * or a relaxation s_k dt above 2 (forward-Euler limit) with MRTLB_ERR_ARG.
 * On success *out owns the context; on failure *out is NULL. */
int mrtlb_create(const mrtlb_params* params, mrtlb_ctx** out);

/* Bytes one state buffer needs (padded device layout of 16 planes with a
 * one-node ghost layer; its inner layout is private to the library). */
int mrtlb_state_bytes(const mrtlb_ctx* ctx, size_t* bytes);

/* Bind two caller-owned device buffers of at least mrtlb_state_bytes bytes,
 * 256-byte aligned, used as the ping-pong pair f^n / f^{n+1}.  Allocates the
 * context's own scratch on first use.  Ghost layers are zeroed. */
int mrtlb_bind(mrtlb_ctx* ctx, void* f_a, void* f_b, size_t bytes);

/* Set the state to the discrete equilibrium f = M^-1 f^eq(rho, u, T)
 * (Eqs. 14a-14i and the chosen version) from FP64 fields [ny][nx] (host
 * pointers if on_device == 0, device pointers otherwise), then make wall
 * nodes consistent with their neighbours. */
int mrtlb_init_equilibrium(mrtlb_ctx* ctx, const double* rho, const double* ux,
                           const double* uy, const double* T, int on_device);

/* Advance nsteps >= 0 time steps.  Each step refills the wall nodes from
 * f^n (when there are walls), then advances every non-wall node
 * (Sec. II-III); the step kernel also writes the new values of edge nodes
 * into the ghost layer of f^{n+1} that mirrors them (periodic or outflow),
 * so a step costs one kernel launch, two with walls.  Asynchronous on the
 * context stream. */
int mrtlb_step(mrtlb_ctx* ctx, long nsteps);

/* Macroscopic fields of the current state as FP64 [ny][nx]: rho = f^_1,
 * u = (f^_2, f^_3)/rho, T = f^_4/rho - u^2/2 (Sec. II, R = 1).  Any pointer
 * may be NULL to skip that field.  Synchronises the stream and reports any
 * latched device error. */
int mrtlb_macros(mrtlb_ctx* ctx, double* rho, double* ux, double* uy,
                 double* T, int on_device);

/* Global sums in FP64 over all nodes: out[0] = sum rho, out[1] = sum j_x,
 * out[2] = sum j_y, out[3] = sum e, out[4] = max |T - T_prev| over the nodes
 * since the previous mrtlb_reduce call (0 on the first call).
 * Synchronises and reports any latched device error. */
int mrtlb_reduce(mrtlb_ctx* ctx, double out[5]);

/* Copy the state out / in as dense [16][ny][nx] in the context precision
 * (float for MRTLB_FP32, double for MRTLB_FP64).  Both synchronise when the
 * buffer is on the host.
 *
 * Host buffers (on_device = 0) of mrtlb_macros, mrtlb_get_f and mrtlb_set_f
 * are borrowed for the duration of the call.  Page-locked host memory that
 * is mapped into the device's address space (e.g. cudaHostAlloc, or a
 * PyTorch pinned tensor) is read or written by the kernels directly over the
 * host link; any other host memory goes through a library-owned device
 * staging buffer and one copy. */
int mrtlb_get_f(mrtlb_ctx* ctx, void* f, int on_device);
int mrtlb_set_f(mrtlb_ctx* ctx, const void* f, int on_device);

/* Self-test of the device-side wait bound (the paper has no counterpart):
 * one kernel waits on a barrier that nothing completes, gives up after the
 * bound every kernel wait of the library uses (about 2 s) and flags it, so
 * the call returns MRTLB_ERR_TIMEOUT; the error word is then cleared and the
 * context stays usable.  Returns an earlier latched error instead, if any. */
int mrtlb_selftest_wait(mrtlb_ctx* ctx);

/* Wait for the context's stream; report any latched device error. */
int mrtlb_sync(mrtlb_ctx* ctx);

/* Step kernel selection.  MRTLB_KERNEL_TILED is the TMA-fed row-marching
 * kernel (one CTA per column strip and row segment, rows streamed through a
 * shared-memory ring); MRTLB_KERNEL_PLAIN is one thread per node reading its
 * neighbours from global memory.  Both compute the same step; AUTO (the
 * default) takes the tiled kernel when its tensor maps could be built at
 * bind time.  Selecting TILED when it is unavailable gives
 * MRTLB_ERR_UNSUPPORTED. */
#define MRTLB_KERNEL_AUTO 0
#define MRTLB_KERNEL_PLAIN 1
#define MRTLB_KERNEL_TILED 2
int mrtlb_set_kernel(mrtlb_ctx* ctx, int which);

/* Per-launch timing of the step kernel.  Between mrtlb_timing_begin and
 * mrtlb_timing_end, every step-kernel launch (at most max_launches of them;
 * later ones are not timed) is bracketed by CUDA events recorded on the
 * context stream.  mrtlb_timing_end synchronises and returns the summed
 * device time in milliseconds and the number of timed launches. */
int mrtlb_timing_begin(mrtlb_ctx* ctx, int max_launches);
int mrtlb_timing_end(mrtlb_ctx* ctx, double* kernel_ms, long* launches);

/* Measured arithmetic ceiling of the current device, for the roofline of
 * the step beside the HBM bound (the paper has no counterpart).  One kernel
 * runs independent fused multiply-add chains on every SM at full occupancy,
 * with no memory traffic; the best of three timed launches (after one warm-up,
 * on a private stream, CUDA events) is returned in TFLOP/s, a fused
 * multiply-add counting two.  kind: MRTLB_PEAK_FP32 (scalar FP32),
 * MRTLB_PEAK_FP32_PAIR (packed FP32 pairs, the form the FP32 step uses),
 * MRTLB_PEAK_FP64.  Synchronous; about 0.1 s.  MRTLB_ERR_ARG for another kind
 * or a NULL output, MRTLB_ERR_CUDA if a launch fails. */
#define MRTLB_PEAK_FP32 0
#define MRTLB_PEAK_FP32_PAIR 1
#define MRTLB_PEAK_FP64 2
int mrtlb_measure_peak(int kind, double* tflops);

/* Kernel launches one time step enqueues (boundary fills and the step). */
int mrtlb_launches_per_step(const mrtlb_ctx* ctx);

/* Allocation-free conservation sums.  The paper has no counterpart: this is
 * a library convenience for callers that cannot call cudaMalloc, e.g. code
 * whose device memory belongs to another allocator with a fixed budget, or a
 * loop that must not pay cudaMalloc's implicit device-wide synchronisation.
 *
 * f: device pointer to a dense state [16][ny][nx] (float for MRTLB_FP32,
 * double for MRTLB_FP64), e.g. filled by mrtlb_get_f(ctx, f, 1).  Computes
 * the same out[0..4] as mrtlb_reduce: FP64 sums of rho, j_x, j_y, e and
 * max |T - T_prev|, where T_prev are the temperatures this function stored
 * on the same device at its previous call if that call had the same nx and
 * ny (out[4] = 0 otherwise).  stream: cudaStream_t (NULL = legacy default);
 * the call synchronises it.
 *
 * Scratch lives in one file-scope static device array of
 * MRTLB_NOALLOC_MAX_NODES + 8 doubles (8 MiB), which every GPU that loads
 * this library holds until the process exits.  nx * ny above
 * MRTLB_NOALLOC_MAX_NODES is rejected with MRTLB_ERR_ARG before any device
 * work.  The first call on each device, and the first in each new CUDA
 * context of that device (e.g. after cudaDeviceReset), resolves the array's
 * device address (cudaGetSymbolAddress) and the SM count with that device
 * current; make that first call before any stream capture.  The call
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * A call that fails leaves no T_prev to compare with (the next call reports
 * out[4] = 0).  All calls on a
 * device share the array (accumulators are cleared at each call, T_prev is
 * kept): calls that overlap on the GPU race.  CUDA failures give
 * MRTLB_ERR_CUDA. */
#define MRTLB_NOALLOC_MAX_NODES (1 << 20)
int mrtlb_reduce_noalloc(const void* f, int nx, int ny, int precision, void* stream,
                         double out[5]);

/* ------------------------------------------------------------------------
 * Batched stepping: many independent grids (e.g. Riemann, Couette and
 * Richtmyer-Meshkov instances of uneven sizes, rates, time steps and Mach
 * numbers) advanced together.  The instances are contexts created and bound
 * as usual (initialise them with mrtlb_init_equilibrium / mrtlb_set_f before
 * mrtlb_batch_create); they must share one precision and one stream and be
 * at the same buffer parity (no steps taken since their last init/set, or
 * the same number).  Per time step the batch makes one launch of a
 * persistent kernel over a tile list (instance, column strip, row segment)
 * of all instances, plus one launch for the NEE walls of all instances that
 * have walls; runs of graph_steps steps (default 64) replay as CUDA graphs.
 * The instances' own calls (macros, get_f, reduce, ...) keep working on the
 * advanced states; stepping an instance alone while it is in a batch, or
 * binding it to other buffers, makes the next mrtlb_batch_step return
 * MRTLB_ERR_STATE.  Rates set on an instance with mrtlb_set_rates take
 * effect at the next mrtlb_batch_step (or mrtlb_batch_tune), which copies
 * the instances' coefficient blocks into the batch's tables again (after
 * the steps already queued).  The batch owns its
 * tables and graphs, not the contexts.
 * ---------------------------------------------------------------------- */
typedef struct mrtlb_batch mrtlb_batch;

int mrtlb_batch_create(mrtlb_ctx* const* ctxs, int n, mrtlb_batch** out);
/* Advance every instance by nsteps time steps (asynchronous). */
int mrtlb_batch_step(mrtlb_batch* b, long nsteps);
/* Wait for the stream; report a latched device error of batched steps
 * (MRTLB_ERR_NONPHYSICAL: some instance met rho <= 0, T <= 0 or a non-finite
 * value; MRTLB_ERR_TIMEOUT: a bounded wait expired).  The batch has its own
 * error word, which the instances' calls do not read, and it stays set for
 * the life of the batch: after re-initialising its instances, make a new
 * batch. */
int mrtlb_batch_sync(mrtlb_batch* b);
/* Tile shape: strip width bx (FP32: 64 or 128; FP64: 64) and rows per
 * segment (>= 1).  The default is the single-grid shape with 32 rows. */
int mrtlb_batch_set_tiles(mrtlb_batch* b, int bx, int seglen);
int mrtlb_batch_get_tiles(const mrtlb_batch* b, int* bx, int* seglen, int* ntiles, int* grid);
/* Steps per captured CUDA graph (0 = plain launches). */
int mrtlb_batch_set_graph_steps(mrtlb_batch* b, int steps);
/* Autotuner: time trial_steps steps for each candidate tile shape and keep
 * the fastest; the instances' states are saved before and restored after
 * the trials.  With cache_path, a text file of "signature bx seglen us"
 * lines is read first (a hit skips the trials) and the result appended;
 * the signature hashes the precision, every instance's grid and boundary
 * kinds, and the device name. */
int mrtlb_batch_tune(mrtlb_batch* b, const char* cache_path, int trial_steps, int* bx_out,
                     int* seglen_out);
/* Total nodes over all instances. */
long long mrtlb_batch_nodes(const mrtlb_batch* b);
const char* mrtlb_batch_last_error(const mrtlb_batch* b);
void mrtlb_batch_destroy(mrtlb_batch* b);

/* Replace / read the relaxation rates s_1..s_16 (same limits as create).
 * Batches made earlier keep the rates they copied. */
int mrtlb_set_rates(mrtlb_ctx* ctx, const double* s);
int mrtlb_get_rates(const mrtlb_ctx* ctx, double* s);

/* ------------------------------------------------------------------------
 * Adjoint (reverse mode) of K time steps.  The paper has no adjoint; this is
 * the exact transpose of the discrete step above (Sec. II-III as
 * implemented: Lax-Wendroff advection, collision with the modified
 * energy-flux terms, NEE walls, periodic and outflow ghosts), for
 * gradients of a loss on the final state with respect to the initial state
 * and the relaxation rates.  Equilibrium versions 1, 2 and 3.
 *
 * mrtlb_adjoint_forward(ctx, K): advances the context K steps from its
 *   current state f^0 (like mrtlb_step) and keeps what the backward pass
 *   needs in segments of S steps: the S states of the last segment, plus a
 *   checkpoint at the start of every segment when there is more than one.
 *   S is the value set by mrtlb_adjoint_set_interval, else K (no
 *   recomputation) when K + 2 states fit in half the free device memory,
 *   else ceil(sqrt(K)).  Library-owned device memory: S + 2 state buffers,
 *   plus ceil(K/S) checkpoints when K > S; freed by mrtlb_adjoint_release or
 *   destroy.
 * mrtlb_adjoint_set_interval(ctx, S): the segment length of later
 *   mrtlb_adjoint_forward calls; S = 0 restores the automatic choice,
 *   S < 0 is MRTLB_ERR_ARG.  Memory against recomputation: each segment but
 *   the last is recomputed once per backward pass.
 * mrtlb_adjoint_backward(ctx, dL_dmacros, dL_dfK, dL_ds, dL_df0): seeds
 *   with dL/d(rho, u_x, u_y, T) of the final state as mrtlb_macros returns it
 *   (device FP64 [4][ny][nx], or NULL) and/or dL/df^K of the state as
 *   mrtlb_get_f returns it (device FP64 [16][ny][nx], or NULL); recomputes
 *   each segment whose states are not held from its checkpoint (the context
 *   keeps f^K) and runs the adjoint steps back to f^0.  It may be called
 *   again with another seed after the same forward pass.  dL_ds may be
 *   NULL: the adjoint steps then skip the rate gradients' work (the
 *   moments and equilibria only they need), and dL/df^0 is the same.  It returns
 *   MRTLB_ERR_STATE, computing nothing, when the context changed after the
 *   forward pass (mrtlb_step, mrtlb_set_f, mrtlb_init_equilibrium,
 *   mrtlb_bind, mrtlb_load, mrtlb_set_rates or a batched step), since its
 *   gradients would then mix two runs.  Outputs: dL_ds[16] (host;
 *   entries 5..16 of the paper's s, 0-based 4..15, accumulated in FP64;
 *   0..3 are zero since those rates have no effect) and dL/df^0 (device FP64
 *   [16][ny][nx], or NULL).  Synchronises.  A non-physical state met by a
 *   step of the forward pass (or of its recomputation) makes it return
 *   MRTLB_ERR_NONPHYSICAL, an expired bounded wait MRTLB_ERR_TIMEOUT; the
 *   outputs are then meaningless.
 * mrtlb_adjoint_pass(ctx): the id (1, 2, ... per context) of the forward
 *   pass that a backward pass would differentiate now, or 0 when there is
 *   none (no forward pass yet, one that failed, or a context changed since);
 *   a caller that holds several forward passes (e.g. an autograd graph)
 *   compares it with the id it recorded after its own forward pass.
 * mrtlb_equilibrium_adjoint: for a state initialised by
 *   mrtlb_init_equilibrium from (rho, u_x, u_y, T) (device FP64 [ny][nx]),
 *   maps dL/df (device FP64 [16][ny][nx]) to dL/d(rho, u_x, u_y, T)
 *   (device FP64 [ny][nx] each).  Synchronises. */
int mrtlb_adjoint_forward(mrtlb_ctx* ctx, long K);
int mrtlb_adjoint_set_interval(mrtlb_ctx* ctx, long S);
int mrtlb_adjoint_backward(mrtlb_ctx* ctx, const double* dL_dmacros, const double* dL_dfK,
                           double dL_ds[16], double* dL_df0);
long long mrtlb_adjoint_pass(const mrtlb_ctx* ctx);
int mrtlb_adjoint_release(mrtlb_ctx* ctx);
int mrtlb_equilibrium_adjoint(mrtlb_ctx* ctx, const double* dL_df, const double* rho,
                              const double* ux, const double* uy, const double* T,
                              double* dL_drho, double* dL_dux, double* dL_duy, double* dL_dT);

/* Checkpoint and resume.  mrtlb_save writes the current state to a file
 * (a header with the grid, precision, step count and a hash of every
 * parameter the step depends on, the dense state [16][ny][nx] in the
 * state's precision, and a checksum), through a sibling file that replaces
 * path only once it is complete; it synchronises.  mrtlb_load reads such a
 * file into a bound context with the same parameters (grid, spacings, time
 * step, current rates, equilibrium version, modification, precision and
 * sides) and restores the step count; a run resumed from the checkpoint of
 * step n continues bitwise as the original run.  Returns MRTLB_ERR_ARG for
 * an unreadable, truncated or corrupted file (checksum), another grid,
 * precision or parameter set, or an I/O failure, leaving the context as it
 * was. */
int mrtlb_save(mrtlb_ctx* ctx, const char* path);
int mrtlb_load(mrtlb_ctx* ctx, const char* path);

/* Number of time steps taken since the last init/set. */
long mrtlb_step_count(const mrtlb_ctx* ctx);

/* Message of the last error on ctx (never NULL; "" if none).  With
 * ctx == NULL it returns the message of the calling thread's last failed
 * mrtlb_create. */
const char* mrtlb_last_error(const mrtlb_ctx* ctx);

/* Release the context and the scratch it owns (not the bound buffers). */
void mrtlb_destroy(mrtlb_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MRTLB_H */
