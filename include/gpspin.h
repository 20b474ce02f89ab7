/*
 * gpspin.h -- C ABI of the GB300 split-step Crank-Nicolson solver for the 2D
 * rotating spin-1 Gross-Pitaevskii equation with Rashba or Dresselhaus
 * spin-orbit (SO) coupling and Rabi coupling (arXiv 2105.10517, Supplementary
 * Material, Eqs. S.1-S.6; solution method: split-step Crank-Nicolson in
 * imaginary or real time, program summary "Solution method").
 *
 * Conventions shared by every call
 *  - Plain C types only.  Host pointers are owned by the caller; device memory
 *    is owned by the handle and released by gp_destroy.
 *  - Wave functions are laid out psi[c][j][i] as interleaved (re, im) pairs,
 *    c = 0, 1, 2 for the components m_F = +1, 0, -1, j the y index (ny rows),
 *    i the x index (fastest).  Host buffers are always complex128
 *    (2 * 3 * nx * ny doubles), whatever the storage precision on the device.
 *  - Grid: cell centred, x_i = -xlen/2 + (i + 1/2) dx with dx = xlen / nx (same
 *    for y); psi vanishes outside the box (zero Dirichlet data).
 *  - Every call returns a gp_status (GP_OK = 0); a failing call leaves the
 *    handle usable unless it returns GP_ERR_CUDA.  Calls are synchronous with
 *    respect to the handle's stream: they return after the device work they
 *    enqueued has finished.  A handle must not be used from two threads at once.
 */
#ifndef GPSPIN_H
#define GPSPIN_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GP_OK = 0,
    GP_ERR_ARG = 1,       /* invalid argument or parameter set (nothing was changed)      */
    GP_ERR_OOM = 2,       /* device allocation failed                                     */
    GP_ERR_CUDA = 3,      /* a CUDA runtime call failed; the handle should be destroyed   */
    GP_ERR_NONFINITE = 4, /* a reduction met NaN/Inf in psi; the state is kept as is      */
    GP_ERR_UNSUPPORTED = 5,/* parameters outside what the tabulated solver supports       */
    GP_ERR_TOO_LARGE = 6, /* grid larger than the fixed scratch of gp_propagate_noalloc    */
    GP_ERR_TIMEOUT = 7,   /* a bounded device-side wait gave up; the state is unreliable   */
    GP_ERR_QUEUE_FULL = 8 /* gp_batch_submit: the batch's queue limit is reached            */
} gp_status;

typedef enum { GP_IMAG = 0, GP_REAL = 1 } gp_mode;
typedef enum { GP_SO_NONE = 0, GP_SO_RASHBA = 1, GP_SO_DRESSELHAUS = 2 } gp_so_type;
/* GP_FP64: complex128 storage and arithmetic throughout.
 * GP_FP32_MIXED: psi is stored and propagated as complex64 (FP32 sweeps and
 * pointwise substep); the Thomas coefficient tables are computed in FP64, the
 * norm and observable reductions run in FP64, and gp_refine_fp64 continues the
 * propagation in FP64 (the precision form of the method's hot path). */
typedef enum { GP_FP64 = 0, GP_FP32_MIXED = 1 } gp_precision;

/* Problem statement (Eqs. S.1-S.4 and the input parameters of the program
 * summary): grid nx x ny on [-xlen/2, xlen/2) x [-ylen/2, ylen/2), time step dt,
 * trap V = (wx^2 x^2 + wy^2 y^2)/2, nonlinearities c0 and c2, angular velocity
 * omeg (OMEG, the Omega of Eq. S.3), SO type (eta = +1 Rashba, -1 Dresselhaus)
 * and strength gamma, Rabi strength rabi (the R of Eqs. S.1-S.2). */
typedef struct {
    int nx, ny;
    double xlen, ylen;
    double dt;
    double wx, wy;
    double c0, c2, omeg;
    int so_type;     /* gp_so_type */
    double gamma, rabi;
    int precision;   /* gp_precision */
} gp_params;

/* Observables of the current state (normalisation/magnetisation conditions and
 * energy functional, Eq. S.6):
 *   norm[c]      = dx dy sum |psi_c|^2 for c = +1, 0, -1
 *   norm_total   = sum of the three
 *   magnetization= norm[0] - norm[2]
 *   energy       = E of Eq. (S.6), discretised consistently with the sweeps
 *   mu           = <H_GP> / N (the chemical potential of a stationary state)
 *   steps        = time steps taken by the handle so far                      */
typedef struct {
    double norm[3];
    double norm_total;
    double magnetization;
    double energy;
    double mu;
    long long steps;
} gp_obs;

typedef struct gp_handle gp_handle;

/* Validates params, allocates the device state on the current CUDA device and
 * returns a handle in *out.  cuda_stream is a cudaStream_t (NULL: the handle
 * creates its own non-blocking stream).  Fails with GP_ERR_ARG before any
 * allocation for nx or ny < 4, non-positive or non-finite lengths or dt,
 * non-finite physical parameters, or an unknown so_type / precision. */
int gp_create(const gp_params* params, void* cuda_stream, gp_handle** out);

/* Releases every device allocation of h.  NULL is ignored. */
void gp_destroy(gp_handle* h);

/* Replaces the physical parameters (dt, trap, c0, c2, omeg, SO, rabi) of h,
 * e.g. for an Omega quench.  The grid (nx, ny, xlen, ylen) and precision must
 * be unchanged.  The Thomas coefficient tables are rebuilt on the next
 * propagate call. */
int gp_set_params(gp_handle* h, const gp_params* params);

/* Copies a host wave function psi[3][ny][nx] (complex128) into h.  If
 * normalize != 0 it is rescaled on the device so that the total norm is 1. */
int gp_set_state(gp_handle* h, const double* psi_host, int normalize);

/* Writes the current wave function (complex128, psi[3][ny][nx]) into the
 * caller's host buffer psi_out.  Any pending imaginary-time normalisation is
 * applied to the copy. */
int gp_get_state(gp_handle* h, double* psi_out);

/* From host state to host state in one call: the same result as
 * gp_set_state(h, psi_in, 0), gp_propagate(h, nsteps, mode) and
 * gp_get_state(h, psi_out), and the handle holds the new state afterwards.
 * psi_in and psi_out are complex128 psi[3][ny][nx] host buffers owned by the
 * caller (they may be the same buffer); the call returns once psi_out is
 * written.  On a GP_FP64 handle with the first-order splitting (the default),
 * when the device can address the buffers
 * (pinned memory, or pageable memory on systems where the GPU reads host page
 * tables, such as NVLink-C2C hosts) and they are 16-byte aligned, the first
 * x-pass reads psi_in directly, so the host-to-device transfer overlaps the
 * pass's work, and the normalised result is written straight into psi_out;
 * otherwise the three calls above are made.  Errors as for those calls. */
int gp_propagate_host(gp_handle* h, const double* psi_in, long long nsteps, int mode, double* psi_out);

/* Device initial state: psi_c = sqrt(frac[c]) pi^{-1/2} exp(-(x^2+y^2)/2)
 * exp(i phi_c(x,y)), phi = phase_noise (2u - 1), u = top 53 bits of
 * splitmix64(seed ^ ((c ny + j) nx + i)) times 2^-53; then normalised to 1. */
int gp_init_gaussian(gp_handle* h, const double frac[3], unsigned long long seed, double phase_noise);

/* The same initial state with centre vortices built in (the SO-coupled states
 * described after Fig. S1: (-+1, 0, +-1) antiferromagnetic, (0, +-1, +-2)
 * ferromagnetic): component c is multiplied by (x + i sgn(l_c) y)^|l_c| before
 * normalisation, winding[c] = l_c in [-8, 8]. */
int gp_init_winding(gp_handle* h, const double frac[3], const int winding[3], unsigned long long seed,
                    double phase_noise);

/* Advances h by nsteps split-step Crank-Nicolson steps: P(dt) -> X(dt) -> Y(dt),
 * and in imaginary time (mode GP_IMAG) renormalisation to a total norm of 1
 * after every step.  mode GP_REAL propagates i d_t psi = H psi.  nsteps = 0 is
 * a no-op. */
int gp_propagate(gp_handle* h, long long nsteps, int mode);

/* Precision form: widens a GP_FP32_MIXED handle's complex64 state to complex128
 * (exactly) and advances it by nsteps FP64 steps in the given mode; the handle
 * propagates in FP64 from then on.  On a GP_FP64 handle it equals gp_propagate. */
int gp_refine_fp64(gp_handle* h, long long nsteps, int mode);

/* Splitting of the time step.  GP_SPLIT_LIE (the default) is the first-order
 * step P(dt) -> X(dt) -> Y(dt) of this library's reading of the paper's
 * split-step scheme.  GP_SPLIT_STRANG is an extension with no counterpart in the
 * paper: the second-order symmetric step P(dt/2) -> X(dt/2) -> Y(dt) -> X(dt/2)
 * -> P(dt/2), followed in imaginary time by the same renormalisation.  Strang
 * steps run on GP_FP64 handles without the magnetisation constraint
 * (GP_ERR_UNSUPPORTED otherwise); gp_propagate, gp_refine_fp64 and
 * gp_propagate_host follow the setting. */
enum { GP_SPLIT_LIE = 0, GP_SPLIT_STRANG = 1 };
int gp_set_splitting(gp_handle* h, int split);

/* Magnetisation-constrained imaginary time (both conditions printed below Eq.
 * S.5): with enable != 0, every imaginary-time step ends with psi_c <- sigma_c psi_c
 * such that N = 1 and N_{+1} - N_{-1} = m, with sigma_{+1} sigma_{-1} = sigma_0^2
 * (the normalised gradient flow for spin-1 condensates).  Only for gamma = R = 0,
 * where m is conserved by the equations (GP_ERR_ARG otherwise); |m| < 1. */
int gp_set_magnetization(gp_handle* h, int enable, double m);

/* Computes the observables of the current state on the device (FP64, fixed
 * reduction order, so repeated calls give bitwise identical results).
 * Returns GP_ERR_NONFINITE (and still fills *out) if psi holds NaN or Inf. */
int gp_observables(gp_handle* h, gp_obs* out);

/* Test hook: applies one substep to the state, which = 0 (pointwise P),
 * 1 (X sweep) or 2 (Y sweep), with the time step and mode given, without the
 * imaginary-time renormalisation and without counting a step. */
int gp_apply_substep(gp_handle* h, int which, int mode);

/* Timing hook: advances h by ONE step exactly as gp_propagate(h, 1, mode)
 * does (with the handle's splitting and magnetisation settings), recording
 * CUDA events on the handle's stream between its kernels, and writes the device
 * durations in milliseconds to ms_out[0] (x-pass: pending normalisation,
 * pointwise substep, X sweep; with GP_SPLIT_STRANG both x-passes of the step),
 * ms_out[1] (y-pass: Y sweep and partial norms), ms_out[2] (normalisation, 0 in
 * real time) and ms_out[3] (the whole step, first event to last).  ms_out must
 * hold 4 floats. */
int gp_profile_step(gp_handle* h, int mode, float* ms_out);

/* Test hook for failure detection: runs the bounded device-side wait that the
 * line passes use for their bulk copies, on the handle's stream, against an
 * mbarrier that no copy targets and no thread arrives on, so it gives up after
 * `polls` polls (1 .. 65536) with nothing in flight.  Returns GP_ERR_TIMEOUT,
 * exactly as gp_propagate does when a copy wait of a pass gives up; the state and
 * the handle are untouched and stay usable. */
int gp_check_wait_timeout(gp_handle* h, int polls);

/* No-allocation variant of gp_propagate (the paper has no counterpart: it
 * exists for callers that must not allocate device memory -- e.g. a plugin
 * whose host application owns the GPU memory pool, or a real-time loop under a
 * no-allocation rule -- and therefore cannot create a gp_handle).
 *   params  problem statement as for gp_create; nx and ny must be <= 256
 *           (otherwise GP_ERR_TOO_LARGE, before any device work).
 *   psi_dev DEVICE pointer owned by the caller, 16-byte aligned (otherwise
 *           GP_ERR_ARG, before any device work): psi[3][ny][nx] complex128,
 *           advanced in place by nsteps steps in mode GP_IMAG or GP_REAL;
 *           in imaginary time it is returned normalised to 1.
 *   cuda_stream  a cudaStream_t (NULL: the legacy default stream).
 * Returns GP_ERR_UNSUPPORTED for parameters outside the tabulated solver's
 * range, GP_ERR_TIMEOUT if a bounded device-side wait gave up (psi is then
 * unreliable) and GP_ERR_NONFINITE if a norm became NaN or Inf.
 * The call allocates nothing: its intermediate, coefficient tables, partial
 * sums and scalars live in fixed device arrays of the library (about 8.6 MB,
 * held on every device that loads the library until the process exits).  The
 * first call on a device looks up their addresses (cudaGetSymbolAddress), so
 * make that first call before any stream capture; a lookup that failed is
 * tried again by the next call.  All calls share these arrays: two calls whose
 * device work overlaps (other streams, other host threads) race and corrupt
 * each other's results.  Synchronous with respect to cuda_stream. */
int gp_propagate_noalloc(const gp_params* params, double* psi_dev, long long nsteps, int mode, void* cuda_stream);

/* ---- Served, batched solves --------------------------------------------------
 * Many imaginary-time solves of different grids and parameters advance together
 * (the batched and served forms of the hot path; the paper runs one solve per
 * program invocation).  A batch admits requests in arrival order while their
 * device-memory footprint fits in max_device_bytes, keeps each admitted solve's
 * psi and coefficient tables resident, advances all running solves of one
 * storage precision with one launch per substep (check_every steps per
 * gp_batch_step), checks convergence between ticks and retires finished solves,
 * freeing their memory for the next admission.  A solve's result is the same
 * alone and in any mix (bitwise: each CTA runs the single-instance arithmetic). */
typedef struct gp_batch gp_batch;
typedef enum {
    GP_REQ_QUEUED = 0,
    GP_REQ_RUNNING = 1,
    GP_REQ_DONE = 2,
    GP_REQ_FAILED = 3,   /* gp_batch_error gives the status that failed it */
    GP_REQ_UNKNOWN = 4,
    GP_REQ_CANCELLED = 5
} gp_req_state;
typedef enum { GP_POLICY_FP64 = 0, GP_POLICY_FP32_REFINE = 1 } gp_policy;

typedef struct {
    double frac[3];           /* initial state as gp_init_gaussian                          */
    unsigned long long seed;
    double phase_noise;
    double tol;               /* done when |E_k - E_(k-1)| < tol between checks (FP64 phase) */
    double tol32;             /* GP_POLICY_FP32_REFINE: leave FP32 when |dE| <= tol32 |E|     */
    long long cap;            /* step cap (a capped solve is reported as done)               */
    int policy;               /* gp_policy: FP64 throughout, or FP32 then FP64 refinement    */
    long long refine_steps;   /* GP_POLICY_FP32_REFINE: FP64 from cap - refine_steps at the latest */
} gp_request;

/* Device bytes one solve with these parameters and policy occupies. */
size_t gp_request_bytes(const gp_params* params, int policy);
int gp_batch_create(size_t max_device_bytes, int check_every, void* cuda_stream, gp_batch** out);
void gp_batch_destroy(gp_batch* b);
/* Queues a solve (params.precision is set from the policy); *id_out identifies it.
 * GP_ERR_QUEUE_FULL if the queue limit (gp_batch_set_queue_limit) is reached. */
int gp_batch_submit(gp_batch* b, const gp_params* params, const gp_request* req, long long* id_out);
/* Ticks are captured as CUDA graphs and replayed while the set of running
 * solves is unchanged (the default, enable != 0); enable = 0 launches every
 * kernel of every tick directly.  Results are bitwise the same either way. */
int gp_batch_use_graphs(gp_batch* b, int enable);
/* Launch form of the batched passes; each substep (and solve kind) is one
 * launch over the (instance, line group) work items of every running solve,
 * largest grids first.  max_ctas < 0 (the default): one CTA per work item;
 * max_ctas = 0: persistent, one CTA per resident slot, the CTAs taking the work
 * items from a device counter; max_ctas > 0: persistent with at most max_ctas
 * CTAs.  Results are bitwise the same in every form. */
int gp_batch_set_persistent(gp_batch* b, int max_ctas);
/* Limits the work in flight: a queued request is admitted only while the grid
 * points (nx * ny) of all running solves plus its own stay within max_sites,
 * except that one solve always runs; 0: no limit (admission by memory only).
 * With a limit that still fills the GPU, earlier requests take a larger share
 * of it and finish sooner, at the same solves/s. */
int gp_batch_set_running_limit(gp_batch* b, long long max_sites);
/* Limits the number of queued (not yet admitted) requests; 0: no limit. */
int gp_batch_set_queue_limit(gp_batch* b, int max_queued);
/* Cancels a queued or running solve between ticks: a queued one leaves the
 * queue, a running one releases its device memory at once (the next tick can
 * admit into it).  Its state becomes GP_REQ_CANCELLED; finished solves are left
 * as they are.  GP_ERR_ARG for an unknown id. */
int gp_batch_cancel(gp_batch* b, long long id);
/* The status that failed a GP_REQ_FAILED solve (GP_ERR_OOM when its memory could
 * not be had with no solve running to free any, GP_ERR_NONFINITE, ...), GP_OK
 * otherwise; GP_ERR_ARG for an unknown id. */
int gp_batch_error(gp_batch* b, long long id);
/* One tick: admit, advance every running solve by check_every steps, check, retire, admit. */
int gp_batch_step(gp_batch* b, int* n_running, int* n_queued);
/* State (gp_req_state), steps taken and last observables of a solve; psi_out
 * (complex128, may be NULL) receives the result once it is done; release != 0
 * forgets a finished solve. */
int gp_batch_poll(gp_batch* b, long long id, int* state, long long* steps, gp_obs* obs, double* psi_out, int release);

/* Autotuner: for the handle's current precision and the given mode, times the
 * x-pass and the y-pass for each candidate tiling -- lines per CTA (1, 2, 4, 8),
 * one CTA or a cluster of 2, 4 or 8 CTAs per line group, chunk lengths of the
 * parallel Thomas solve, and for complex128 the shared-memory and the
 * register-resident solve -- on the handle's stream, and keeps the fastest for
 * later propagation.  Each candidate is timed as the median of five launches
 * (after one warm-up), each started from a cold L2 (a scratch buffer of 1.5 x the L2 size is
 * written first; from a warm L2 if that buffer cannot be allocated).  The
 * state is saved and restored, so tuning does not change the solve; results
 * stay within the parity tolerances (only the summation order of partial
 * norms and the chunking change).  *ms_out (may be NULL) receives the tuned
 * x-pass + y-pass time.  Allocates one temporary copy of psi and the scratch
 * buffer, both freed before it returns. */
int gp_autotune(gp_handle* h, int mode, double* ms_out);

/* Sets the tiling of one pass (dir 0: x-pass, 1: y-pass) for the handle's current
 * precision and the given mode: cluster = CTAs per line group (1, 2, 4 or 8),
 * lines_per_cta, chunk = minimum chunk length of the parallel Thomas solve
 * (raised to what the precision needs), register_solve = the solve kind:
 * 1 register-resident chunks (complex64 chunk length 16, 24 or 32; complex128
 * chunk length 32, at most 384 threads per CTA), 0 shared-memory line arrays,
 * -1 the precision's default (complex64 register-resident up to chunk length
 * 32, complex128 shared memory).  GP_ERR_ARG or GP_ERR_UNSUPPORTED if the
 * tiling does not fit (threads, shared memory, chunks per CTA, chunk length).
 * Results stay within the parity tolerances for every valid tiling. */
int gp_set_tiling(gp_handle* h, int mode, int dir, int cluster, int lines_per_cta, int chunk, int register_solve);

/* Debug checks of a handle (0 turns them off).  GP_DEBUG_POISON: before each
 * pass of the first-order steps that gp_propagate, gp_refine_fp64 and
 * gp_propagate_host run (not the batched, second-order, single-substep or
 * no-allocation paths), every byte the pass must write (the
 * intermediate before the x-pass; the state between the passes, after the
 * x-pass has read it) is set to 0xFF, a NaN in both precisions, so an element
 * that a pass leaves unwritten reaches the state as a NaN: the norm and
 * observable reductions then report GP_ERR_NONFINITE, and results differ from
 * a run without the check.  Costs two memsets of the state's size per step.
 * GP_ERR_ARG for unknown flags. */
#define GP_DEBUG_POISON 1
int gp_set_debug(gp_handle* h, int flags);

/* The tiling the handle uses for a pass (dir 0: x-pass, 1: y-pass) in the given
 * mode and its current precision: out[0] CTAs per line group (cluster size),
 * out[1] lines per CTA, out[2] chunk length, out[3] chunks per line, out[4]
 * threads per CTA, out[5] dynamic shared memory bytes, out[6] CTAs per launch,
 * out[7] solve kind: 0 shared-memory line arrays, 1 register-resident chunks
 * (complex64 chunk length 16, 24 or 32; complex128 chunk length 32).  out must
 * hold 8 ints. */
int gp_tiling_info(gp_handle* h, int mode, int dir, int* out);

/* The default tiling of a pass (dir 0: x-pass, 1: y-pass) for these parameters
 * and mode, the one a handle starts with, computed on the host without a
 * device: out[0..7] as gp_tiling_info, then out[8] the fixup length F (rows
 * a chunk carry reaches above the precision's rounding), out[9] the chunk
 * stride and out[10] the line-channel stride in shared memory (elements), and
 * out[11] the extra shared-memory wavefronts that bank conflicts add to one
 * round of the solve's chunk-parallel accesses (0: none).  out must hold 12 ints.
 * GP_ERR_ARG or GP_ERR_UNSUPPORTED as gp_create would return them. */
int gp_plan_tiling(const gp_params* p, int mode, int dir, int* out);

/* Failure injection for tests of out-of-memory handling: the after-th device
 * allocation of the library from now on (0: the next one) fails as if the
 * device were full, once; after < 0 disarms.  Process-wide. */
void gp_inject_alloc_failure(long long after);

/* Checkpoints (the paper resumes runs from converged wave functions; this is
 * the exact form of that).  A checkpoint holds the handle's parameters, step
 * count, storage precision, pending imaginary-time scale and stored state, in
 * host byte order; restoring it into a handle of the same grid and precision
 * and propagating gives bitwise the results of the uninterrupted run (same
 * library build and tilings).  gp_checkpoint_bytes is the buffer size that
 * gp_checkpoint_save needs (0 for NULL); the caller owns the buffer and may
 * write it to a file.  gp_checkpoint_load returns GP_ERR_ARG, changing nothing,
 * for a buffer that is not a checkpoint of this format or whose grid or
 * precision differ from the handle's; it adopts the checkpoint's physical
 * parameters and step count. */
size_t gp_checkpoint_bytes(gp_handle* h);
int gp_checkpoint_save(gp_handle* h, void* buf, size_t size);
int gp_checkpoint_load(gp_handle* h, const void* buf, size_t size);

/* Human-readable text for a gp_status. */
const char* gp_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* GPSPIN_H */
