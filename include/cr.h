/*
 * cr.h -- C ABI of the GB300 (sm_103a) cRKFR library.
 *
 * The library advances the semi-discrete system
 *     u_t + f(u)_x + B(u) g(u)_x = 0            (paper: eq. flux.and.non.cons, Sec. 2)
 * by the compact Runge-Kutta flux reconstruction method with flux-differencing
 * volume terms (Sec. 3): per step, element-local cRK stages (eq. crkfr.inner)
 * with the two-point volume flux (eq. entropy.cons.flux.dev) and the
 * non-symmetric non-conservative product (eq. entropy.cons.noncons.dev), the
 * time-averaged flux and solution (eq. disc.avg.flux), one Rusanov flux per
 * face node (eq. numflux.cons) with the reduced-communication
 * non-conservative flux B(u^{n,+-}) g^avg(U) (Sec. 2.3), and the final update
 * (eq. crkfr.non.cons.final) followed by the CFL time step reduction.
 *
 * Meshes are uniform periodic Cartesian grids of tensor-product elements with
 * GLL solution points on the reference element [0,1] (Sec. 2).
 *
 * State layout (all entry points): FP64 conserved variables, structure of
 * arrays [var][elem][node]; node index (i, j, k) flattened with i fastest,
 * element index (ex, ey, ez) flattened with ex fastest.  Variables:
 *   Euler (dim d):  rho, rho v_1..rho v_d, E         (M = d + 2)
 *   ideal GLM-MHD:  rho, rho v_1..3, E, B_1..3, psi  (M = 9, dim 2 only)
 *   E = p/(gamma-1) + rho|v|^2/2 [+ |B|^2/2 + psi^2/2].
 *
 * Every function returns an int status (CR_OK = 0, negative on error) and
 * never aborts or traps.  Errors leave the context usable unless stated.
 */
#ifndef CR_H
#define CR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CR_OK            0
#define CR_EINVAL       (-1)   /* invalid argument or descriptor                       */
#define CR_ENOMEM       (-2)   /* device allocation failed                             */
#define CR_ECUDA        (-3)   /* a CUDA runtime call failed                           */
#define CR_ENONPHYSICAL (-4)   /* a step produced rho <= 0, p <= 0 or a non-finite value */
#define CR_ETIMEOUT     (-5)   /* a bounded device wait (batched grid barrier) expired  */
#define CR_ENODEV       (-6)   /* no usable CUDA device / wrong architecture           */
#define CR_ETOOLARGE    (-7)   /* mesh needs more scratch than cr_step_noalloc holds    */

/* system (eq. flux.and.non.cons) */
#define CR_EULER   0           /* compressible Euler, dim 1..3                         */
#define CR_GLM_MHD 1           /* ideal GLM-MHD with Powell/GLM non-conservative terms, dim 2 */

/* two-point volume flux f_S (Sec. 3) */
#define CR_VOL_EC      0       /* Euler: Ranocha (EC + KEP); GLM-MHD: entropy conservative */
#define CR_VOL_KEP     1       /* Euler: Kennedy-Gruber (KEP, arithmetic means)         */
#define CR_VOL_CENTRAL 2       /* (f(u_p)+f(u_q))/2: reduces to collocation D f         */

/* surface flux (eq. numflux.cons) */
#define CR_SURF_RUSANOV 0

/* time stepping scheme */
#define CR_SCHEME_CRKFR 0      /* compact RKFR (eqs. crkfr.inner, crkfr.non.cons.final): element-local
                                  stages, one face exchange per step -- the paper's method      */
#define CR_SCHEME_RKFR  1      /* multi-stage RKFR (eq. rkfr.non.cons), the scheme cRKFR is derived
                                  from: the same RK tableau on the semi-discrete FR system, a
                                  face exchange (Rusanov flux of the stage traces) at every
                                  stage; for measuring the single-stage advantage                */

/* non-conservative numerical flux of the cRKFR step (GLM-MHD) */
#define CR_NCFLUX_REDUCED 0    /* B(u^{n,+-}) g^avg(U) from the time-averaged records: no data beyond
                                  the conservative flux's (Sec. 2.3; all of the paper's results)  */
#define CR_NCFLUX_STAGES  1    /* sum_j b_j B(u^{(j),+-}) g^avg(u^(j)) (eq. bad.numflux.non.cons):
                                  the face traces of every stage are exchanged (seven values per
                                  stage and face node); GLM-MHD with CR_SCHEME_CRKFR only        */

/* subcell blending limiter (the paper's Sec. 4 runs: the cRKFR update blended
 * per element with a first-order subcell finite-volume update, coefficient
 * from a modal smoothness indicator capped by alpha_max; compressible Euler
 * with CR_SCHEME_CRKFR and the single-solve form only) */
#define CR_LIMITER_NONE     0
#define CR_LIMITER_BLENDING 1

/* arithmetic of the element-local work */
#define CR_FP64          0     /* every step of the path in FP64                        */
#define CR_FP32_PAIRFLUX 1     /* stages, pair fluxes, time averages and face fluxes in
                                  FP32; the state update u^{n+1} = u^n - dt(...), the dt
                                  reduction and the diagnostic totals stay FP64          */

typedef struct {
  int eq;            /* CR_EULER | CR_GLM_MHD                                           */
  int dim;           /* 1, 2, 3 (GLM-MHD: 2)                                            */
  int degree_N;      /* polynomial degree N = 1..5 (N+1 GLL points per direction)        */
  int cells[3];      /* elements per direction; entries beyond dim are ignored           */
  double lo[3], hi[3];  /* periodic box                                                 */
  double gamma;      /* ratio of specific heats                                         */
  double cfl;        /* dt = cfl / max_nodes sum_d lambda_d / dx_d                       */
  double c_h;        /* GLM cleaning speed (GLM-MHD only), fixed for the run             */
  double dt_fixed;   /* > 0: use this dt every step instead of the CFL rule              */
  int vol;           /* CR_VOL_*                                                        */
  int surf;          /* CR_SURF_RUSANOV                                                 */
  int prec;          /* CR_FP64 | CR_FP32_PAIRFLUX                                      */
  int scheme;        /* CR_SCHEME_CRKFR (0) | CR_SCHEME_RKFR; the batched form and
                        cr_step_noalloc take CR_SCHEME_CRKFR only                        */
  int ncflux;        /* CR_NCFLUX_REDUCED (0) | CR_NCFLUX_STAGES; the batched form and
                        cr_step_noalloc take CR_NCFLUX_REDUCED only                      */
  int limiter;       /* CR_LIMITER_NONE (0) | CR_LIMITER_BLENDING: per element
                        u^{n+1} = (1 - a) u^H + a u^L, u^H the cRKFR update, u^L first-
                        order finite volumes on the subcells of the GLL points (widths
                        w_p dx), both with one blended, admissibility-corrected flux per
                        element-face node; a from the highest-mode energy of rho p;
                        CR_EULER, CR_SCHEME_CRKFR, single solve only                      */
  double alpha_max;  /* cap of the blending coefficient, 0..1 (limiter only)             */
} cr_mesh_desc;

typedef struct cr_ctx cr_ctx;   /* opaque; owned by the library */

/* Create a context on the current CUDA device.
 *   out        : receives the context (NULL on failure).
 *   desc       : n_solves descriptors (copied).
 *   n_solves   : 1 = one mesh advanced by two kernels per step (volume,
 *                face + update; with CRKFR_STEP_KERNELS=fused in the
 *                environment, variants whose lane layouts allow it run both
 *                parts in one cooperative persistent launch instead, which
 *                measured slower), replayed as a CUDA graph; CR_SCHEME_RKFR: the two
 *                kernels once per RK stage, the volume kernel on the stage
 *                state with a single stage); > 1 = batched form: the
 *                solves (meshes and degrees may differ) advance together, per
 *                step one persistent volume kernel and one persistent face /
 *                update kernel per degree present, all replayed from one CUDA
 *                graph; grid sizes are autotuned before the first step.  The
 *                batched form requires eq = CR_EULER, dim = 2 and the same
 *                prec and vol for all solves (and the same gamma per degree).
 *   cuda_stream: cudaStream_t on which all work is enqueued (NULL = legacy default).
 * The library allocates and owns all device buffers (state, stage/trace
 * scratch, step records; CR_SCHEME_RKFR adds a stage state and s - 1 stage
 * increments, CR_NCFLUX_STAGES the stage traces after the face records,
 * CR_LIMITER_BLENDING a second state buffer -- the limited step reads u^n
 * from one and writes u^{n+1} to the other --, one coefficient and flag per
 * element and the list of the elements the limiter touches).  Returns CR_EINVAL, CR_ENOMEM, CR_ECUDA, CR_ENODEV. */
int cr_init_mesh(cr_ctx **out, const cr_mesh_desc *desc, int n_solves, void *cuda_stream);

/* Caller-provided device memory.  cr_workspace_bytes stores in *bytes the
 * device memory a single-solve context with this descriptor needs for its
 * buffers (state, residual sums, face records, step record, totals, and what
 * the scheme, limiter or the single-launch option adds), each 256-byte
 * aligned; CR_EINVAL for an invalid descriptor.  No CUDA call.
 * cr_init_mesh_ws is cr_init_mesh with n_solves = 1 whose device buffers are
 * all carved out of `workspace` (a device pointer on the current device,
 * 256-byte aligned, at least `bytes` >= cr_workspace_bytes long) instead of
 * being allocated -- for callers whose own allocator (a framework's caching
 * pool) already holds the device.  The caller keeps ownership and must keep
 * the workspace alive and untouched until cr_destroy; CUDA graphs, streams and
 * events of the context are still created by the library.  CR_EINVAL for a
 * NULL, misaligned, too small, host or other-device workspace. */
int cr_workspace_bytes(const cr_mesh_desc *desc, size_t *bytes);
int cr_init_mesh_ws(cr_ctx **out, const cr_mesh_desc *desc, void *workspace, size_t bytes, void *cuda_stream);

/* Number of conserved variables and of nodes (elements x (N+1)^dim) of a solve. */
int cr_state_size(const cr_ctx *ctx, int solve, int *n_vars, long long *n_nodes);

/* Copy a state in (layout above; n_vars x n_nodes doubles).  u is a host
 * pointer (u_on_device = 0; pageable or pinned) or a device pointer on the
 * context's device (u_on_device = 1).  The caller keeps ownership.  Resets
 * t = 0 and the step counter, checks physicality (CR_ENONPHYSICAL) and
 * computes the first time step.  Synchronises the stream. */
int cr_set_state(cr_ctx *ctx, int solve, const double *u, int u_on_device);

/* Enqueue nsteps time steps on the stream (asynchronous; no host sync).
 * A non-physical result is reported by the next cr_sync / cr_get_state /
 * cr_get_info.  Returns CR_EINVAL for nsteps < 0 or a context without state. */
int cr_step(cr_ctx *ctx, int nsteps);

/* Wait for the stream and return the accumulated device status
 * (CR_OK, CR_ENONPHYSICAL, CR_ETIMEOUT) or CR_ECUDA. */
int cr_sync(cr_ctx *ctx);

/* Copy the state of a solve out (same layout and pointer rules as
 * cr_set_state).  Synchronises the stream; returns the device status. */
int cr_get_state(cr_ctx *ctx, int solve, double *u, int u_on_device);

/* Asynchronous state transfer, for host I/O that overlaps other work
 * (pipelined serving of many problems over several contexts).  Enqueue the
 * copy in (cr_set_state_async, which also resets t, the step counter and the
 * status and starts the first CFL reduction, like cr_set_state) or out
 * (cr_get_state_async) on the context's stream and return without waiting.
 * u must stay valid and unchanged until the stream has passed the copy
 * (cr_sync); only pinned host memory lets the copy overlap other work.  The
 * physicality of a state copied in is reported by the next cr_sync /
 * cr_get_state / cr_get_info, not here.  Same layout and pointer rules as
 * cr_set_state / cr_get_state; CR_EINVAL for a bad argument. */
int cr_set_state_async(cr_ctx *ctx, int solve, const double *u, int u_on_device);
int cr_get_state_async(cr_ctx *ctx, int solve, double *u, int u_on_device);

/* Time, last time step, steps taken and (if totals != NULL) FP64
 * quadrature-weighted domain totals: totals[0..M-1] conserved variables,
 * totals[M] kinetic energy, totals[M+1] entropy -rho s/(gamma-1),
 * s = ln p - gamma ln rho.  Synchronises the stream. */
int cr_get_info(cr_ctx *ctx, int solve, double *t, double *dt, long long *steps, double *totals);

/* Measurement: advance nsteps more steps with each kernel launched directly
 * (not from the graph) between CUDA events recorded on the context's stream;
 * before every step, if flush_buf != NULL, flush_bytes of that device buffer
 * are overwritten (cudaMemsetAsync) to evict the L2.  ms[0] receives the mean
 * duration of one volume-kernel launch, ms[1] of one face/update launch (the
 * batched form: ms[0] = the volume launches of all degrees of one step, ms[1]
 * = their face/update launches; CR_SCHEME_RKFR: ms[0] = the s volume
 * launches of one step, ms[1] = its s face/update launches; a single solve
 * whose step runs as one cooperative launch -- cr_tuning_info reports
 * "step": "fused" -- ms[0] = that launch, ms[1] = 0).  The state advances
 * exactly as with cr_step.  Synchronises the stream. */
int cr_time_kernels(cr_ctx *ctx, int nsteps, void *flush_buf, size_t flush_bytes, double *ms);

/* Measurement: throughput of one unit on the current device, measured with
 * CUDA events (best of 3 after a warm-up): kind 0 FP32 FMA, 1 FP64 FMA,
 * 2 MUFU reciprocal (FP32), 3 double->float conversion, 4 integer ALU
 * (lane-operations/s; an FMA counts once), 5 device copy (bytes/s read+write,
 * 2 GiB allocated for the call), 6 host->device and 7 device->host copy
 * engine with pinned host memory, 8 both directions at once (bytes/s per
 * direction; 64 MiB pinned buffers allocated for the call).  Synchronises
 * the device. */
int cr_probe_peak(int kind, double *result);

/* Self-check of the FP32 form's float <-> double conversions, which use
 * integer instructions instead of the hardware conversion (on this GPU the
 * hardware conversion runs on the narrow FP64 pipe).  The paper has no
 * counterpart.  Converts n seeded bit patterns (half of the doubles with
 * exponents confined to the FP32 range and its edges, plus infinities and
 * NaNs) both ways on the current device and stores in *mismatches how many
 * results differ from the hardware conversion (round to nearest both ways,
 * and the round-toward-zero conversion of the FP32 physicality check, which
 * gives NaN from 2^128 on); inputs below the normal FP32 range are expected
 * to give signed zero.  Returns CR_EINVAL for n < 0 or a
 * NULL pointer, CR_ENOMEM/CR_ECUDA on a device error.  Synchronises. */
int cr_check_conversions(long long n, unsigned long long seed, long long *mismatches);

/* One time step without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory while they advance a solve -- an application whose memory
 * pool already holds the device, or a host loop that must not stall other
 * streams (cudaMalloc/cudaFree can synchronise the device).
 *   desc       : one mesh descriptor (as for cr_init_mesh).
 *   u_in       : device pointer, state u^n (layout above), not modified
 *                unless u_in == u_out.
 *   u_out      : device pointer, receives u^{n+1}; may equal u_in.
 *   dt_out     : device pointer receiving the dt used (FP64), or NULL.
 *   cuda_stream: stream for all work (asynchronous; nothing is synchronised).
 * dt follows the descriptor (CFL rule on u^n, or dt_fixed); desc->scheme must
 * be CR_SCHEME_CRKFR, desc->ncflux CR_NCFLUX_REDUCED and desc->limiter
 * CR_LIMITER_NONE (CR_EINVAL otherwise).  The scratch
 * (residual sums, face traces, reductions, step record) lives in one static
 * device array of CR_NOALLOC_SCRATCH_BYTES per device, held until the
 * process exits; a mesh needing more returns CR_ETOOLARGE (roughly 80k nodes
 * of 2D Euler in FP64).  The first call on a device looks up that array's
 * device address and keeps it for the life of the process, so make it before
 * any stream capture, and do not call this entry point on a device after
 * cudaDeviceReset (the address belonged to the destroyed context).  Every
 * call shares the array: calls that overlap on the GPU race.  Physicality is
 * not reported; use the regular entry points for status.  Device pointers of
 * the wrong size are not detected (the sizes follow from desc). */
#define CR_NOALLOC_SCRATCH_BYTES (8u << 20)
int cr_step_noalloc(const cr_mesh_desc *desc, const double *u_in, double *u_out, double *dt_out,
                    void *cuda_stream);

/* Subcell blending limiter: copy the smoothed blending coefficient of every
 * element (E doubles, element order as in the state layout) that the last
 * step used -- computed from the state it started from; zeros before the
 * first step -- to a host (on_device = 0) or device pointer.  CR_EINVAL for a
 * context without the limiter.  Synchronises the stream. */
int cr_get_blend_alpha(cr_ctx *ctx, double *alpha, int on_device);

/* JSON description of the kernel configuration chosen for the context (the
 * autotuned persistent grids of the batched form), copied into buf (len
 * bytes, NUL-terminated).  CR_EINVAL if it does not fit. */
int cr_tuning_info(cr_ctx *ctx, char *buf, size_t len);

/* Release every device buffer and graph of the context. */
int cr_destroy(cr_ctx *ctx);

/* Static description of a status code. */
const char *cr_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* CR_H */
