/*
 * ssp.h -- C ABI of libssp, a GB300 (sm_103a) implementation of the Super
 * Smoother periodogram of Gowanlock, Butler, Trilling & McNeill, "GPU-Enabled
 * Searches for Periodic Signals of Unknown Shape" (arXiv 2111.07396).
 *
 * For every (object, trial frequency) pair the library folds the light curve
 * (phase = frac(tt * f), tt = t - min t; Alg. 1), sorts it by phase (stable,
 * ties by original index), smooths the folded curve with Friedman's Super
 * Smoother (Listing 1, "SS") or the single-pass generalized-validation
 * variant (Sec. 3, "SP"), and reduces the smooth to
 *     power = 1 - chi2 / chi0,  chi2 = sum w (y - smo)^2,
 *     chi0 = sum w (y - ybar_w)^2,  w = dy^-2                  (Alg. 1)
 * then reports the period 1/f of the first maximum (findPeriod, Alg. 1).
 *
 * Conventions for every entry point:
 *  - Objects are concatenated in CSR order: object o owns n_per_object[o]
 *    consecutive points of t, y and dy.  Times need not be sorted.  Frequency
 *    is ordinary (cycles per time unit), not angular (App. A).
 *  - freq_grid holds n_freq explicit trial frequencies shared by all objects
 *    (Sec. 4.3, catalogs share one grid); any positive values, any order.
 *  - out_power is row-major [n_objects][n_freq]; its element type is double
 *    for SSP_FP64 and float for SSP_FP32C.  out_best_period is double
 *    [n_objects].
 *  - The caller owns every buffer; the library keeps no pointer after the
 *    call returns (the device entry point keeps none after its work on the
 *    stream completes).
 *  - Return value: SSP_OK or a negative ssp_status.  On error the outputs
 *    are unspecified; ssp_last_error() gives a message (per thread).
 *  - Results are deterministic and independent of how many objects share a
 *    call.
 */
#ifndef SSP_H
#define SSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SSP_SS = 0, /* Super Smoother, cross-validated spans (Listing 1) */
    SSP_SP = 1, /* SuperSmootherSP, generalized validation, one pass (Sec. 3):
                   a span chosen per point */
    SSP_SPG = 2 /* the other reading of Sec. 3: one span per frequency, the one
                   whose summed squared generalized-validation residuals
                   sum w (|y - s|/(1 - nu/m))^2 are least; no bass */
} ssp_variant;

typedef enum {
    SSP_FP64 = 0,  /* every step in binary64; phase fold bit-identical to Alg. 1 */
    SSP_FP32C = 1  /* exact fixed-point fold, FP32 smoothing with local origins,
                      compensated chi2; power written as float */
} ssp_precision;

/*
 * SSP_FP32C re-takes in binary64 the decisions that FP32 rounding could flip.
 * Its margins have defaults chosen for the 2e-4 tolerance; each can be
 * overridden, for testing and tuning only, by an environment variable read at
 * every launch, and only while SSP_TESTING=1 is set too (a value of 1e6 or
 * more, or an empty one, keeps the default; a negative margin disables its
 * test):
 *   SSP_NEAR_SS     SS tweeter-vs-midrange margin for n <= 256 (default 1e-6,
 *                   relative; scaled down for larger n, off above 2,048
 *                   points).  Flags the frequency for the binary64 recompute.
 *   SSP_NEAR_SS_ABS the same margin's absolute part, in FP32 units of the
 *                   object's largest centred magnitude (default 8, scaled
 *                   down for larger n like the relative part; off above
 *                   2,048 points).
 *   SSP_NEAR_SP     SP near-tie margin in FP32 units of the magnitude scale
 *                   (default 32).
 *   SSP_SENS_TAU    SP: power budget per point; a near-tie whose other choice
 *                   could move the power by more is settled in binary64
 *                   (default 1e-6).
 *   SSP_SENS_ULPS   SP: rounding of a residual, in ulps of its scale, in that
 *                   bound (default 2).
 *   SSP_REFIT_FRAC  a window whose centred spread fell below this fraction of
 *                   the largest moment its sliding sums held is refitted in
 *                   binary64 (default 1/128).
 * Wider margins cost time and keep accuracy; narrower ones can break the
 * tolerance.
 */

typedef enum {
    SSP_OK = 0,
    SSP_ERR_ARG = -1,         /* invalid argument or input value */
    SSP_ERR_NOMEM = -2,       /* device memory budget exceeded */
    SSP_ERR_CUDA = -3,        /* a CUDA call failed */
    SSP_ERR_TIMEOUT = -4,     /* a bounded wait expired (serving: stall_ms) */
    SSP_ERR_UNSUPPORTED = -5, /* valid request this build cannot run */
    SSP_ERR_BUSY = -6,        /* serving: too many requests in flight */
    SSP_PENDING = 1           /* serving: the request has not finished yet */
} ssp_status;

typedef struct {
    double spans[3];     /* tweeter, midrange, woofer spans as fractions of n;
                            default {0.05, 0.2, 0.5} (Listing 1).  Must satisfy
                            0 < spans[0] < spans[1] < spans[2] <= 1. */
    double alpha;        /* bass enhancement in [0, 10]; default 9 (Sec. 5.1);
                            0 disables it (Sec. 5.4, transits). */
    int periodic;        /* 1 (default): windows wrap around the phase circle
                            (Listing 1 iper = 2).  0: each window is the
                            2 ibw + 1 consecutive points slid to lie inside
                            [0, n-1] (Listing 1 iper = 1). */
    ssp_precision precision; /* default SSP_FP32C */
    double hbm_fraction; /* beta of Eq. 1: fraction of free device memory the
                            host entry point may use; default 0.75 (Sec. 4.1) */
    double span;         /* 0 (default): variable span (SS or SP).  In (0, 1]:
                            Listing 1's fixed-span mode, one running-line smooth
                            of that span, no cross-validation; the same for
                            both variants. */
} ssp_params;

/* Fill *p with the defaults listed above. */
void ssp_default_params(ssp_params *p);

/*
 * Periodograms of a catalog from HOST memory (Alg. 1 end to end, batched).
 *   t, y, dy        host f64 [sum n]; t and y finite, dy finite and > 0.
 *   n_per_object    host i64 [n_objects]; every n >= 4 (Listing 1 reads
 *                   x[3(n/4)-1]) and n <= 65535.
 *   freq_grid       host f64 [n_freq]; finite and > 0; 1 <= n_freq <= 2^31 - 1.
 *   params          NULL selects ssp_default_params.
 *   out_power       host [n_objects][n_freq], double (FP64) or float (FP32C).
 *   out_best_period host f64 [n_objects].
 * Copies inputs to the device, runs the whole path there, copies the results
 * back and returns when they are in host memory.  Objects are processed in
 * batches sized to hbm_fraction of free device memory (Eq. 1's role).
 * Errors: SSP_ERR_ARG (any rule above, n_objects < 1, n_freq < 1, bad
 * params), SSP_ERR_NOMEM (one object's minimum batch does not fit),
 * SSP_ERR_UNSUPPORTED (FP32C with a weight outside the float range),
 * SSP_ERR_CUDA.
 */
int ssp_periodogram(const double *t, const double *y, const double *dy,
                    const int64_t *n_per_object, int64_t n_objects,
                    const double *freq_grid, int64_t n_freq, ssp_variant variant,
                    const ssp_params *params, void *out_power, double *out_best_period);

/*
 * Same computation on DEVICE memory, enqueued on `stream` (a cudaStream_t;
 * NULL = the legacy default stream).  t, y, dy, freq_grid, out_power and
 * out_best_period are device pointers; n_per_object is a HOST array (the
 * launch plan is built from it).  Returns after enqueueing (plus the host
 * work of planning); results are valid once the stream reaches that point.
 * Input values are checked on the device: an object with a non-finite t or y,
 * or a dy that is not finite and > 0, gets NaN powers and a NaN best period.
 * Temporary device memory is taken from the stream-ordered allocator.
 * Errors: as ssp_periodogram, except that value checks become NaN outputs.
 */
int ssp_periodogram_device(const double *t, const double *y, const double *dy,
                           const int64_t *n_per_object, int64_t n_objects,
                           const double *freq_grid, int64_t n_freq, ssp_variant variant,
                           const ssp_params *params, void *out_power,
                           double *out_best_period, void *stream);

/*
 * The phase fold of Alg. 1 (computePhasedTime) exactly as the SSP_FP32C
 * kernels compute it, evaluated on the host (no GPU needed):
 *     out[i] = floor(frac(fl(tt[i] * f)) * 2^64)
 * where fl() is the binary64 product rounded to nearest even.  The kernels
 * obtain it with integer arithmetic (no FP64 instructions); for phases >=
 * 2^-11 it carries the binary64 phase exactly.  tt[i] must be finite and
 * >= 0, f finite and > 0 (else SSP_ERR_ARG).  out is caller-owned, u64 [n].
 */
int ssp_fold_fixed(const double *tt, int64_t n, double f, uint64_t *out);

/*
 * ssp_periodogram_device without any device allocation.  (The paper has no
 * counterpart; this entry point exists for callers that cannot call
 * cudaMalloc: programs whose device memory is owned by another allocator or
 * capped by a memory pool, which would see the library's own allocations
 * fail or overrun their budget, and services that forbid allocation after
 * start-up because an allocation can block or fail at an arbitrary time.)
 * Arguments and results are those of ssp_periodogram_device; inputs and
 * outputs are still the caller's device buffers, and n_per_object is a host
 * array.  Temporary storage is a fixed 8 MiB array in device memory that
 * this library declares at file scope; every GPU that loads the library
 * holds it until the process exits.
 * Limits: the request's scratch must fit the 8 MiB, and every object's
 * frame must fit shared memory (about 2,500 points per object); larger
 * requests return SSP_ERR_UNSUPPORTED with the reason in ssp_last_error().
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress).
 * All calls share the one array and the library clears what must start at
 * zero on every call, so calls whose work overlaps on the GPU (different
 * streams, or several host threads) race with each other and must be
 * serialised by the caller.  No profiling events are recorded.
 */
int ssp_periodogram_device_noalloc(const double *t, const double *y, const double *dy,
                                   const int64_t *n_per_object, int64_t n_objects,
                                   const double *freq_grid, int64_t n_freq, ssp_variant variant,
                                   const ssp_params *params, void *out_power,
                                   double *out_best_period, void *stream);

/*
 * Launch plans: the device pipeline captured into a CUDA graph (the paper
 * has no counterpart; it launches each kernel from the host, Sec. 4).  For
 * callers that run one shape again and again -- the same objects' point
 * counts, frequency count, variant and params, new values --
 * ssp_plan_create does the host work of ssp_periodogram_device once: it
 * builds the launch plan, takes the workspace (cudaMalloc, held until
 * ssp_plan_destroy), uploads the plan's tables and captures the pipeline
 * (counters cleared, prep, the periodogram kernels and their FP64
 * recompute, argmax) into a CUDA graph on the current device.
 * ssp_plan_execute then runs that graph on the caller's DEVICE arrays
 * (t, y, dy, freq_grid, out_power, out_best_period as in
 * ssp_periodogram_device, n_freq values in freq_grid) enqueued on `stream`
 * with one graph launch; its results are bit for bit those of
 * ssp_periodogram_device with the same plan.  Executions of one plan share
 * its workspace, so they must not overlap on the GPU (one stream, or the
 * caller's ordering).  The plan follows the threads-per-CTA choices in force
 * when it was created (ssp_autotune).
 * Errors: ssp_plan_create as ssp_periodogram_device (shape and params),
 * SSP_ERR_NOMEM (workspace), SSP_ERR_CUDA (capture); ssp_plan_execute
 * SSP_ERR_ARG (NULL arrays), SSP_ERR_CUDA.
 */
typedef struct ssp_plan ssp_plan;
int ssp_plan_create(const int64_t *n_per_object, int64_t n_objects, int64_t n_freq,
                    ssp_variant variant, const ssp_params *params, ssp_plan **out);
int ssp_plan_execute(ssp_plan *plan, const double *t, const double *y, const double *dy,
                     const double *freq_grid, void *out_power, double *out_best_period,
                     void *stream);
int ssp_plan_destroy(ssp_plan *plan);

/*
 * Serving: one light curve per request, results collected asynchronously.
 * (The paper's batches are whole catalogs, Sec. 4.3; a survey alert stream
 * instead delivers objects one at a time.)  A server owns one frequency grid,
 * one parameter set and two workers on the current device, and batches
 * continuously under a device-memory budget:
 *  - admission: a submitted request waits on the host until its inputs fit
 *    the device arena (device_bytes, one ring per variant); it is then
 *    uploaded and stays resident on the device until its batch has finished;
 *  - batching: whenever one of `slots` batch slots is free, the oldest
 *    admitted requests of one variant (at most max_batch_ptf points x
 *    frequencies) run the pipeline of ssp_periodogram_device on the slot's
 *    stream, reading their inputs in place; batches overlap on the GPU;
 *  - completion: each batch's requests finish when it does, in completion
 *    order, not launch order.
 * A request's results are identical to ssp_periodogram on that object alone,
 * whatever else is in flight.
 */
typedef struct ssp_server ssp_server;
typedef struct {
    double max_batch_ptf;   /* cap on points x frequencies per batch; <= 0: 4e9 */
    double max_wait_ms;     /* how long the oldest queued request may wait for
                               more to arrive when a batch slot is free; <= 0:
                               launch at once */
    int64_t max_in_flight;  /* requests submitted and not yet collected by
                               ssp_server_poll; <= 0: 1 << 20 */
    double stall_ms;        /* bounded wait for a batch on the GPU: a batch not
                               finished this long after it was launched ends
                               its requests with SSP_ERR_TIMEOUT; <= 0: 60000 */
    int64_t slots;          /* batches on the GPU at once, at most 16; <= 0: 4 */
    double device_bytes;    /* device arena holding admitted requests' inputs
                               (t, y, dy), split evenly over the three
                               variants; <= 0: 768 MiB */
} ssp_server_config;

/*
 * Creates a server for freq_grid (host, n_freq values, copied) and params
 * (NULL = defaults; copied); config NULL = defaults.  *out receives the
 * handle.  Errors: SSP_ERR_ARG (grid, params, more than 16 slots),
 * SSP_ERR_UNSUPPORTED, SSP_ERR_NOMEM (the arena does not fit), SSP_ERR_CUDA
 * (no device).
 */
int ssp_server_create(const double *freq_grid, int64_t n_freq, const ssp_params *params,
                      const ssp_server_config *config, ssp_server **out);

/*
 * Queues one object: t, y, dy are host arrays of n points, copied before the
 * call returns.  *out_ticket receives the request's ticket (increasing from
 * 1).  Errors: SSP_ERR_ARG (the value rules of ssp_periodogram, n outside
 * 4..65535), SSP_ERR_UNSUPPORTED, SSP_ERR_BUSY (max_in_flight requests are
 * submitted and not yet collected; nothing is queued), SSP_ERR_NOMEM (the
 * object alone exceeds its variant's share of the device arena).
 */
int ssp_server_submit(ssp_server *s, const double *t, const double *y, const double *dy,
                      int64_t n, ssp_variant variant, int64_t *out_ticket);

/*
 * Waits up to wait_ms (0 = do not wait) for a request that has finished and
 * was not reported by this call before; SSP_OK with its ticket in
 * *out_ticket, or SSP_PENDING if none finished in time.
 */
int ssp_server_next(ssp_server *s, int wait_ms, int64_t *out_ticket);

/*
 * Waits up to wait_ms for request `ticket`.  SSP_OK: out_power (n_freq
 * values, double for SSP_FP64 and float for SSP_FP32C) and
 * *out_best_period hold the results, *out_latency_ms (if not NULL) the time
 * from submission to completion, and the ticket is retired.  SSP_PENDING: not
 * finished yet.  The request's own error status (e.g. SSP_ERR_NOMEM, or
 * SSP_ERR_TIMEOUT when its batch outlived stall_ms) if its batch failed; the
 * ticket is retired and the server keeps serving.  SSP_ERR_ARG: unknown or
 * retired ticket.
 */
int ssp_server_poll(ssp_server *s, int64_t ticket, int wait_ms, void *out_power,
                    double *out_best_period, double *out_latency_ms);

/*
 * Stops the workers after the batches already on the GPU complete; queued and
 * uncollected requests are dropped.  Frees everything the server holds.
 */
int ssp_server_destroy(ssp_server *s);

/*
 * Autotuning of the launch plan (the paper has no counterpart).  Objects
 * are planned in five length ranges (n <= 384, <= 768, <= 1536, <= 2048,
 * larger); each range runs one launch whose threads per CTA follow a fixed
 * rule by default.  ssp_autotune times
 * the rule's choice, half of it and double it (within 32..512, at least two
 * centres per thread) for every range that the given objects (host arrays,
 * as ssp_periodogram) occupy.  The timing runs the full device pipeline on
 * those objects and an evenly spaced sample of freq_grid, about budget_ptf
 * points x frequencies per range (<= 0: 2e9); each candidate is run three
 * times and the last two are timed.  The fastest choice is kept for later
 * calls with this precision and variant in this process.
 * out_group_sizes (may be NULL) receives the five ranges' threads per CTA
 * after tuning.  Results of later calls stay within the precision's
 * tolerance but are not bitwise those of the rule, because the chunking
 * changes rounding.  Call it before other work, not concurrently with it.
 * Errors: as ssp_periodogram.
 */
int ssp_autotune(const double *t, const double *y, const double *dy, const int64_t *n_per_object,
                 int64_t n_objects, const double *freq_grid, int64_t n_freq, ssp_variant variant,
                 const ssp_params *params, double budget_ptf, int32_t *out_group_sizes);
/* Forgets every tuned choice: the fixed rule applies again. */
void ssp_autotune_clear(void);

/*
 * Search-and-refine (the outlook of Sec. 6: a cheap coarse search, then the
 * costly smoother only near its peaks), on host arrays as ssp_periodogram.
 *  1. The periodogram of coarse_variant on coarse_grid (n_coarse >= 2
 *     frequencies, strictly increasing).
 *  2. Per object, the n_peaks (1..64) largest local maxima of that power.
 *     A local maximum is p[q] >= p[q-1] and p[q] > p[q+1], a missing
 *     neighbour counting as lower. Ties go to the lower index, a maximum
 *     next to one already taken is skipped, and fewer than n_peaks maxima
 *     repeat the first.
 *  3. Per peak q, n_fine frequencies evenly from f[q-1] to f[q+1] (one coarse
 *     step beyond q at either end of the grid; a start at or below 0 moves
 *     to f[q]/2).
 *  4. The periodogram of fine_variant on those n_peaks * n_fine frequencies.
 * out_best_period[o] and out_best_power[o] (double, n_objects each) are the
 * period 1/f and the power of the first largest fine power.  The coarse
 * grid must resolve the peaks (steps below about 1/(time span)); the step
 * only sharpens them.  params as ssp_periodogram, with span = 0.
 * Errors: as ssp_periodogram; SSP_ERR_ARG also for the rules above and
 * n_peaks * n_fine > 2^22.
 */
int ssp_search_refine(const double *t, const double *y, const double *dy,
                      const int64_t *n_per_object, int64_t n_objects, const double *coarse_grid,
                      int64_t n_coarse, ssp_variant coarse_variant, ssp_variant fine_variant,
                      int n_peaks, int n_fine, const ssp_params *params, double *out_best_period,
                      double *out_best_power);

/*
 * Testing only (the paper has no counterpart): host-side fault injection, so
 * that tests reach the failure paths without faulting a GPU.  Honoured only
 * while SSP_TESTING=1 is set in the environment (else SSP_ERR_UNSUPPORTED).
 *   SSP_FAULT_ALLOC  the library's next `count` device allocations fail as
 *                    if the device were out of memory: the entry point (or
 *                    the served request) returns SSP_ERR_NOMEM and nothing
 *                    is left allocated or enqueued;
 *   SSP_FAULT_STALL  the serving worker treats its next `count` batches as
 *                    not finished within stall_ms: their requests end with
 *                    SSP_ERR_TIMEOUT (the batches themselves complete);
 *   SSP_FAULT_UPLOAD the serving worker's next `count` uploads of a request
 *                    into the device arena fail as a CUDA error would: those
 *                    requests end with SSP_ERR_CUDA and are never batched.
 * count 0 clears the kind.  Errors: SSP_ERR_ARG (unknown kind, count < 0).
 */
enum { SSP_FAULT_ALLOC = 1, SSP_FAULT_STALL = 2, SSP_FAULT_UPLOAD = 3 };
int ssp_test_fault(int kind, int count);

/* Static text for a status code (library plumbing; no counterpart in the
 * paper).  Never NULL; the text is static. */
const char *ssp_status_string(int status);
/* Detail of the last error returned on the calling thread ("" if none).  The
 * text belongs to the library and stays valid until the thread's next call. */
const char *ssp_last_error(void);

/* Library version string, "ssp <major>.<minor> sm_103a" (static text). */
const char *ssp_version(void);

/*
 * Per-phase timers (the paper's Tables 3-4 break time down the same way).
 * When enabled, every launch of a phase is bracketed by two CUDA events
 * recorded on the launching stream.  ssp_profile_read waits for the recorded
 * events, fills out[k] for k = SSP_PHASE_PREP (Alg. 1 compute_chi0_tt_weights),
 * SSP_PHASE_PGRAM_SS / SSP_PHASE_PGRAM_SP (fold + sort + smoother + chi2 of
 * SS, or of SP and SPG, one launch per length range), SSP_PHASE_REDO (SSP_FP32C
 * only: the FP64 launch that recomputes the frequencies whose FP32 decisions
 * came within their margins) and SSP_PHASE_ARGMAX (findPeriod), and clears
 * them if reset != 0.  Off by default; enabling adds two event records per
 * launch.
 */
enum {
    SSP_PHASE_PREP = 0,
    SSP_PHASE_PGRAM_SS = 1,
    SSP_PHASE_PGRAM_SP = 2,
    SSP_PHASE_REDO = 3,
    SSP_PHASE_ARGMAX = 4,
    SSP_N_PHASES = 5
};
typedef struct {
    int64_t launches; /* launches recorded */
    double ms;        /* summed event-to-event time, milliseconds */
} ssp_phase_time;
void ssp_profile_enable(int on);
int ssp_profile_read(ssp_phase_time out[SSP_N_PHASES], int reset);

#ifdef __cplusplus
}
#endif
#endif /* SSP_H */
