/*
 * fpt.h -- C ABI of the GB300 first-passage-time (FPT) engine.
 *
 * The engine integrates many independent noisy Josephson-junction trajectories in the tilted
 * washboard potential until each crosses its threshold, and records the escape time or the
 * switching bias ("Stochastic first passage time accelerated with CUDA", Sec. II, III).
 * Model, in plasma-frequency units (Eq. JJn with V0 = 1):
 *     underdamped   phi'' + alpha phi' + A sin phi = gamma(t) + sqrt(2 alpha D) xi(t)
 *     overdamped    phi'                           = gamma(t) - A sin phi + sqrt(2 D) xi(t)
 *     gamma(t) = gamma0 + nu t            (constant bias: Alg. 1; ramped bias: Alg. 3)
 * integrated with the Euler-Maruyama step of Alg. 1 / Alg. 3; escape is the first step k with
 * phi_k >= threshold.  Normals come from Philox4x32-10 (key = the request's 64-bit seed,
 * counter = (step block lo, hi, trajectory id lo, hi)) through the Box-Muller transform of
 * Sec. III.B, so every trajectory is reproducible from (seed, trajectory id) alone.
 *
 * Conventions for every entry point:
 *   - Every call returns an fpt_status; no exception or signal crosses the ABI.
 *   - Pointers named d_* are DEVICE pointers (cudaMalloc'd or torch tensors' data_ptr() on
 *     the current device); pointers without the prefix are HOST pointers.  The caller owns
 *     every buffer it passes; the engine owns the memory it allocates itself.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *     Entry points that take a stream only enqueue work on it and return without waiting.
 *   - On FPT_ECUDA / FPT_EINVAL a description is available from fpt_last_error(engine) (or
 *     fpt_last_error(NULL) for entry points without an engine); the text is thread-local.
 */
#ifndef FPT_H_
#define FPT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FPT_OK = 0,
    FPT_PENDING = 1,      /* request accepted and not finished yet */
    FPT_EINVAL = -1,      /* bad argument (message in fpt_last_error) */
    FPT_ENOMEM = -2,      /* device memory budget or allocation exhausted */
    FPT_EBUSY = -3,       /* operation conflicts with the engine's service thread */
    FPT_ENOTFOUND = -4,   /* unknown or released request id */
    FPT_ETIMEDOUT = -5,   /* fpt_wait ran out of time */
    FPT_ECUDA = -6,       /* a CUDA runtime call failed */
    FPT_EFULL = -7        /* submission queue full */
} fpt_status;

enum { FPT_UNDERDAMPED = 0, FPT_OVERDAMPED = 1 };
enum { FPT_FP32 = 0, FPT_FP64 = 1 };
/* Integrators.  FPT_EULER_MARUYAMA is the Euler scheme of Alg. 1 / Alg. 3.  FPT_HEUN is the
 * stochastic Heun predictor-corrector (one normal per step, drift averaged over both ends of the
 * step, bias taken at t_{k-1} and t_k): weak order 2 for the additive noise of Eq. (JJn).  The
 * paper integrates with Euler only; Heun is an option of this library, on the same random
 * stream (step k still draws normal k-1). */
enum { FPT_EULER_MARUYAMA = 0, FPT_HEUN = 1 };
enum { FPT_OUT_TIME = 0, FPT_OUT_BIAS = 1 };
enum { FPT_TH_ABSOLUTE = 0, FPT_TH_FROM_START = 1 };

/* One FPT problem (a "request").  Alg. 1 arguments (V0, beta, gamma, D, h) map to
 * (A = 1, alpha, gamma0, D, dt); Alg. 3 adds the ramp nu = delta-gamma / dt. */
typedef struct {
    int32_t model;          /* FPT_UNDERDAMPED | FPT_OVERDAMPED */
    int32_t precision;      /* FPT_FP32 (engine, plain kernel) | FPT_FP64 (plain kernel only) */
    int32_t integrator;     /* FPT_EULER_MARUYAMA | FPT_HEUN */
    int32_t output;         /* FPT_OUT_TIME: x = k*dt; FPT_OUT_BIAS: x = gamma0 + nu*dt*k */
    int32_t threshold_mode; /* FPT_TH_ABSOLUTE: phi* = threshold; FPT_TH_FROM_START: phi0 + threshold */
    int32_t keep_per_traj;  /* engine: 1 keeps every escape step for fpt_per_traj */
    double alpha;           /* damping (underdamped only), >= 0 */
    double D;               /* noise intensity, >= 0 */
    double gamma0;          /* bias at t = 0 */
    double nu;              /* bias ramp per unit time (0 = constant bias) */
    double sin_amp;         /* A: amplitude of the sin term (1 = junction; 0 = free drift) */
    double dt;              /* integration step h > 0 */
    double phi0;            /* start phase; NaN = arcsin(gamma0) (Alg. 1, 3; needs abs(gamma0) <= 1) */
    double v0;              /* start velocity (underdamped) */
    double threshold;       /* see threshold_mode; must exceed the start phase */
    uint64_t max_steps;     /* klim: a trajectory not escaped after max_steps is censored; <= 2^48 */
    int32_t hist_bins;      /* histogram of x over [hist_lo, hist_hi): 1 .. 1<<20 bins */
    int32_t reserved0;
    double hist_lo, hist_hi;
    double stop_rse;        /* engine: stop at the first prefix of whole id blocks whose relative
                               standard error of the mean of x is <= stop_rse; 0 = run all */
    uint32_t stop_block;    /* engine: trajectories per id block (0 = 4096) */
    uint32_t reserved1;
    uint64_t traj_offset;   /* id of the request's first trajectory (for sharding across GPUs) */
} fpt_params;

/* Exact sums over a set of finished trajectories (integer arithmetic: order-independent). */
typedef struct {
    uint64_t n_done, n_escaped;
    uint64_t s1_lo, s1_hi;      /* sum of escape steps k, 128-bit */
    uint64_t s2_lo, s2_hi;      /* sum of k^2, 128-bit */
    uint64_t under, over;       /* histogram out-of-range counts */
} fpt_sums;

typedef struct {
    int32_t state;              /* FPT_OK when finished, FPT_PENDING otherwise */
    int32_t reserved;
    uint64_t n_used;            /* trajectories in the result (prefix kept by the stop rule) */
    uint64_t n_escaped, n_censored;
    double mean, var, sem;      /* of x over escaped trajectories (var unbiased; sem = sqrt(var/n)) */
    uint64_t steps_total;       /* sum over used trajectories of their steps (censored: max_steps) */
    double latency_s;           /* submit -> finished, seconds (engine requests) */
} fpt_result;

/* ------------------------------------------------------------------------------------------
 * Plain one-trajectory-per-thread path (the structure of Alg. 1 / Alg. 3: thread i integrates
 * realisation i to its escape).  FP64 reproduces the FP64 oracle's arithmetic order exactly
 * (no fused multiply-add, unwrapped phase); FP32 uses the engine's FP32 step.
 * ------------------------------------------------------------------------------------------ */

/* Integrate trajectories traj0 .. traj0+n-1 of (params, seed).  d_steps[i] (device, int64,
 * n entries) receives the escape step k >= 1, or -1 when censored at max_steps.  Enqueued on
 * `stream`.  The kernel runs each trajectory to completion: a launch lasts up to max_steps
 * steps of the slowest trajectory.  Returns FPT_EINVAL for invalid params or n > 2^32. */
fpt_status fpt_plain_launch(const fpt_params *params, uint64_t seed, uint64_t traj0, uint64_t n,
                            int64_t *d_steps, void *stream);

/* Reduce per-trajectory escape steps (d_steps, n entries, -1 = censored) into exact sums and a
 * histogram of x (Alg. 1: T_e; Alg. 3: Gamma_e).  d_sums (device, one fpt_sums) and d_hist
 * (device, params->hist_bins uint64 counters, may be NULL) are ACCUMULATED into: zero them
 * first.  Bin of x: floor((x - lo) * (bins / (hi - lo))) in IEEE double, x < lo -> under,
 * x >= hi -> over.  Enqueued on `stream`. */
fpt_status fpt_reduce_steps(const fpt_params *params, const int64_t *d_steps, uint64_t n,
                            fpt_sums *d_sums, uint64_t *d_hist, void *stream);

/* Host-only: mean, unbiased variance and standard error of x from exact sums. */
fpt_status fpt_sums_finish(const fpt_params *params, const fpt_sums *sums, fpt_result *out);

/* ------------------------------------------------------------------------------------------
 * Persistent batched engine: one resident kernel serves every admitted request; lanes whose
 * trajectory has escaped take the next trajectory id from a device work queue (a finished
 * processor receives its next realisation at once, Sec. I and III.B, Fig. 6), so uneven
 * trajectory lengths do not idle warps.  FP32 state, FP64 bias/time and exact integer sums.
 * ------------------------------------------------------------------------------------------ */
typedef struct fpt_engine fpt_engine;

typedef struct {
    int32_t device;             /* CUDA device ordinal */
    int32_t max_requests;       /* resident request slots (1 .. 1024; 0 = 256) */
    uint64_t mem_budget_bytes;  /* device memory the engine may allocate (0 = 25 % of free) */
    void *stream;               /* cudaStream_t to run on (NULL = engine-owned stream) */
    int32_t threads_per_block;  /* 0 = default: 640 with one trajectory per thread, 256 with two */
    int32_t blocks_per_sm;      /* 0 = as many as fit */
    int32_t traj_per_thread;    /* 1 or 2 (0 = default 1) */
    uint32_t chunk_steps;       /* steps per resident-kernel launch, multiple of 16 (0 = 16384) */
    int32_t service_thread;     /* 1: an engine thread drives the GPU; 0: caller calls fpt_step */
    int32_t use_graph;          /* 1: replay a CUDA graph per iteration (default 1) */
    uint32_t young_chunk_steps; /* steps per launch while a request of at most as many
                                   trajectories as lanes was admitted within the last 16
                                   launches: shorter quanta for new small requests, which wait
                                   fewer steps of the others for admission, lanes and their
                                   result (multiple of 16, <= chunk_steps; 0 = chunk_steps).
                                   Results do not depend on it. */
} fpt_engine_config;

typedef struct {
    uint64_t iterations;        /* resident-kernel launches so far */
    uint64_t useful_steps;      /* trajectory steps integrated (summed over lanes) */
    uint64_t lane_step_slots;   /* lanes x steps offered by all launches */
    uint64_t escapes, censored; /* trajectories finished */
    uint32_t lanes;             /* resident lanes (threads x trajectories per thread) */
    uint32_t grid, block, traj_per_thread, chunk_steps;
    uint32_t resident_requests, pending_requests;
    double kernel_ms;           /* summed device time of the resident-kernel launches (CUDA events) */
    uint64_t preempted;         /* lane suspensions ordered so starved requests get their share */
    uint64_t check_flags;       /* bounds-checked build (FPT_CHECK): one bit per kind of index
                                   found out of range (the access was skipped); 0 otherwise and
                                   always 0 in the regular build */
} fpt_engine_counters;

/* Create an engine on config->device (NULL config = defaults). */
fpt_status fpt_create(const fpt_engine_config *config, fpt_engine **out);

/* Queue a request of n_traj trajectories (ids traj_offset .. traj_offset+n_traj-1).  Host
 * params are copied; *req_id receives the id.  The request is admitted into the resident
 * kernel when a slot and device memory are free.  FP32 only; FPT_EINVAL otherwise. */
fpt_status fpt_submit(fpt_engine *e, const fpt_params *params, uint64_t n_traj, uint64_t seed,
                      uint64_t *req_id);

/* Caller-driven mode (service_thread = 0): run n_iterations engine iterations (admission,
 * one resident-kernel launch, completion scan, status read-back) and return after the last
 * one finished on the device.  FPT_EBUSY when a service thread owns the engine. */
fpt_status fpt_step(fpt_engine *e, int n_iterations);

/* Result so far: FPT_OK when finished, FPT_PENDING while running (out->state says the same). */
fpt_status fpt_poll(fpt_engine *e, uint64_t req_id, fpt_result *out);

/* Block until the request finishes or timeout_s elapses (drives the engine itself when there
 * is no service thread).  FPT_ETIMEDOUT on timeout. */
fpt_status fpt_wait(fpt_engine *e, uint64_t req_id, double timeout_s, fpt_result *out);

/* Histogram of x over the used prefix (host buffer of nbins uint64).  Requires a finished
 * request and nbins == params.hist_bins. */
fpt_status fpt_histogram(fpt_engine *e, uint64_t req_id, uint64_t *counts, int nbins,
                         uint64_t *under, uint64_t *over);

/* Exact sums (host fpt_sums) over the used prefix of a finished request, for merging results
 * of requests sharded across GPUs (integer addition of the fields is exact). */
fpt_status fpt_request_sums(fpt_engine *e, uint64_t req_id, fpt_sums *out);

/* Per-trajectory x (host, n doubles; -1 for censored when output = time, NaN for bias), for
 * requests submitted with keep_per_traj = 1.  Entries past n_used are not part of the result. */
fpt_status fpt_per_traj(fpt_engine *e, uint64_t req_id, double *out, uint64_t n);
/* Same as escape steps (host, n int64; -1 censored). */
fpt_status fpt_per_traj_steps(fpt_engine *e, uint64_t req_id, int64_t *out, uint64_t n);

/* Checkpoint a running (or queued) request: its lanes are suspended into its ring at the end of
 * the next launch, then its whole state -- parameters, queue head, exact sums, id-block
 * accumulators, histogram rows, per-trajectory steps and suspended trajectories -- is written
 * to the host buffer `buf`, and the request is released.  With buf == NULL only *size is set
 * (an upper bound); otherwise *size is the buffer's capacity on input and the bytes written on
 * output.  fpt_restore continues it exactly: every trajectory ends with the escape step it
 * would have had without the interruption (the paper's 2-day runs, Sec. IV.B, motivate it).
 * Drives the engine itself when there is no service thread. */
fpt_status fpt_checkpoint(fpt_engine *e, uint64_t req_id, void *buf, size_t *size);

/* Re-admit a request from a checkpoint (host buffer of `size` bytes); *req_id gets its new id. */
fpt_status fpt_restore(fpt_engine *e, const void *buf, size_t size, uint64_t *req_id);

/* Free a finished (or cancel a running) request and its device memory. */
fpt_status fpt_release(fpt_engine *e, uint64_t req_id);

fpt_status fpt_get_counters(fpt_engine *e, fpt_engine_counters *out);

/* Launch shapes of the resident kernel: *blocks_per_sm receives how many CTAs of
 * threads_per_block threads (each integrating traj_per_thread trajectories) fit on one SM of
 * the current device, 0 when the kernel cannot launch with that shape (threads_per_block not a
 * multiple of 32, or above 640 for one trajectory per thread / 256 for two).  For autotuners:
 * fpt_engine_config.blocks_per_sm may be 1 .. this value.  FPT_EINVAL for traj_per_thread
 * other than 1 or 2; FPT_ECUDA if the occupancy query fails (no device). */
fpt_status fpt_engine_occupancy(int32_t traj_per_thread, int32_t threads_per_block,
                                int32_t *blocks_per_sm);

/* CUDA stream the engine runs on (cudaStream_t as void*). */
void *fpt_engine_stream(fpt_engine *e);

fpt_status fpt_destroy(fpt_engine *e);

const char *fpt_last_error(fpt_engine *e);
const char *fpt_status_string(fpt_status s);

/* ------------------------------------------------------------------------------------------
 * Allocation-free run (the paper has no counterpart; this is a library convenience).
 *
 * For callers that cannot allocate device memory while they run: a host program that has
 * already reserved the device memory for its own pool, code in a latency-critical loop where
 * cudaMalloc's implicit synchronisation is not acceptable, or a plugin host whose contract
 * forbids allocation during execution.  It integrates one request (FP32, same arithmetic as
 * fpt_plain_launch with precision FPT_FP32) with lanes that take the next trajectory as soon as
 * theirs finishes, all in ONE launch that runs until every trajectory has finished, and calls
 * no cudaMalloc / cudaFree or allocating library routine.
 *
 * Scratch: a fixed 8 MiB __device__ array inside the library (every GPU that loads the library
 * holds it until the process exits): a queue head, a finished-CTA counter and one record of
 * partial sums and per-bin counts per CTA.  With many histogram bins the launch uses as many
 * CTAs as have room for their record (fewer CTAs, same result); hist_bins is limited to 10240
 * (the per-CTA histogram lives in shared memory) and n_traj to 2^32 - 1 (32-bit per-CTA bin
 * counts); larger requests are rejected with FPT_EINVAL and a message giving the limit.  The
 * first call on each device (and the first after that device's context changed, e.g. after
 * cudaDeviceReset) looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call shares the array: the
 * header is cleared on `stream` before each launch, and calls that overlap on the GPU (other
 * streams, other threads) race on it.
 *
 * Arguments: params as for the engine but stop_rse must be 0; trajectories params->traj_offset
 * .. +n_traj-1 of `seed`.  d_steps (device, n_traj int64, may be NULL) receives each escape step
 * or -1; d_sums (one fpt_sums) and d_hist (params->hist_bins uint64) are ACCUMULATED into:
 * zero them first.  Enqueued on `stream`; returns without waiting.
 * ------------------------------------------------------------------------------------------ */
fpt_status fpt_run_noalloc(const fpt_params *params, uint64_t n_traj, uint64_t seed,
                           int64_t *d_steps, fpt_sums *d_sums, uint64_t *d_hist, void *stream);

/* ------------------------------------------------------------------------------------------
 * Random-number hooks (device buffers), for checking the device generator against the oracle.
 * ------------------------------------------------------------------------------------------ */

/* Philox4x32-10 words of blocks block0 .. block0+nblocks-1 of trajectory `traj`: 4 uint32 per
 * block into d_out (device, 4*nblocks entries). */
fpt_status fpt_philox_fill(uint64_t seed, uint64_t traj, uint64_t block0, uint64_t nblocks,
                           uint32_t *d_out, void *stream);

/* Normals n0 .. n0+n-1 of trajectory `traj` as the integrator draws them, unit variance, into
 * d_out (device, n doubles).  Normal n comes from words (x0,x1) (n mod 4 = 0, 1) or (x2,x3)
 * (n mod 4 = 2, 3) of Philox block n / 4, cosine first.  FPT_FP64: u = (x + 1/2) 2^-32,
 * R = sqrt(-2 ln u1), theta = 2 pi u2, each operation rounded.  FPT_FP32: the single-precision
 * map of the FP32 kernels (u1 rounded to 23 bits, fast log2 / sqrt / sincos, the angle
 * 2 pi (u2 - 2^-24) - pi with the radius negated: the FP64 pair rotated by 3.7e-7 rad). */
fpt_status fpt_normals_fill(int precision, uint64_t seed, uint64_t traj, uint64_t n0, uint64_t n,
                            double *d_out, void *stream);

/* ------------------------------------------------------------------------------------------
 * Paper units (Sec. II.A, Eq. JJn).  The paper writes the junction as
 *     phi'' + beta phi' = V0 (-sin phi + gamma + gamma_N),  <gamma_N gamma_N> = 2 D delta,
 *     D = beta theta,
 * in time units hbar / E_C, integrated with step h and bias increment delta_gamma per step
 * (Alg. 1, Alg. 3).  Rescaling time by sqrt(V0) maps it onto the engine's plasma-frequency units:
 *     alpha = beta / sqrt(V0),  D' = theta / V0 (= k_B T / E_J),  dt = sqrt(V0) h,
 *     nu = delta_gamma / dt  (bias per unit engine time),
 * with the fluctuation-dissipation noise sqrt(2 alpha D' dt) of fpt_params.  Host-only
 * arithmetic in IEEE double; outputs are host pointers; FPT_EINVAL for non-positive V0, h, dt
 * or non-finite arguments.
 * ------------------------------------------------------------------------------------------ */
fpt_status fpt_from_paper_units(double V0, double beta, double theta, double h, double delta_gamma,
                                double *alpha, double *D, double *dt, double *nu);
/* The inverse, for a chosen V0. */
fpt_status fpt_to_paper_units(double alpha, double D, double dt, double nu, double V0,
                              double *beta, double *theta, double *h, double *delta_gamma);
/* A physical junction (R ohm, C farad, Ic ampere, T kelvin) in the paper's units (Sec. II.A
 * normalisation): V0 = E_J / E_C, beta = hbar / (R (2e)^2), theta = k_B T / E_C, and the paper's
 * time unit hbar / E_C in seconds, with E_J = hbar Ic / 2e and E_C = (2e)^2 / C. */
fpt_status fpt_junction_paper_units(double R, double C, double Ic, double T, double *V0,
                                    double *beta, double *theta, double *time_unit_s);
/* Bias increment per step of a triangular bias sweep at sweep_hz that covers `span` of the
 * critical current in half a period, with step h in units of time_unit_s (Sec. IV.B, Fig. 10b). */
fpt_status fpt_sweep_delta_gamma(double sweep_hz, double h, double time_unit_s, double span,
                                 double *delta_gamma);

/* Library version string. */
const char *fpt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FPT_H_ */
