/*
 * aerafold.h -- C ABI of the AERA antenna-response unfolding library (GB300, sm_103a).
 *
 * The library evaluates, for every (station, candidate arrival direction) pair of a radio
 * event, the reconstruction step of arXiv 1507.07733, Sec. 2: the two-channel voltage
 * traces are taken to the frequency domain, the antenna vector effective length (VEL) is
 * interpolated for the direction from a tabulated (zenith, azimuth, frequency) pattern
 * (Sec. 3), a 2x2 complex system is solved per frequency bin for the E-field components
 * (E_theta, E_phi), the field is transformed back with its Hilbert envelope (Sec. 4), the
 * envelope maximum gives the station timing, and per direction the timing is compared with
 * a plane wave (the quantity the paper's triangulation minimises, Sec. 2).
 *
 * Conventions (fixed by this library where the paper is silent):
 *  - Forward DFT  X[k] = sum_n x[n] exp(-2 pi i k n / N), unnormalised.
 *  - The band is 30 MHz <= k fs / N <= 80 MHz (Sec. 1), both edges inclusive; every other
 *    bin of the unfolded field is zero. fs must make the band at most N/4 bins wide and
 *    keep 80 MHz below fs/2 (fs = 200 MHz gives exactly N/4 bins).
 *  - VEL interpolation is trilinear in (zenith, azimuth, frequency), real and imaginary
 *    parts separately; zenith and frequency clamp to the table, azimuth is periodic.
 *  - Solve: det = H0t H1p - H0p H1t, E_t = (H1p V0 - H0p V1)/det, E_p = (H0t V1 - H1t V0)/det
 *    where H[c][p] is the VEL of channel c for polarisation p. A bin with
 *    |det| <= 1e-6 (|H0t||H1p| + |H0p||H1t|) is near-singular: E = 0 there and the pair's
 *    status gets AR_STATUS_SINGULAR.
 *  - Analytic signal z_p[n] = (1/N) sum_{k in band} 2 E_p[k] exp(+2 pi i k n / N);
 *    E-field e_p = Re z_p; envelope env = sqrt(|z_theta|^2 + |z_phi|^2) (Sec. 4, read as the
 *    modulus of the analytic signal of each component, summed in quadrature).
 *  - Peak = argmax_n env[n], lowest index on exact ties; peak time = t_start + peak*1e9/fs ns.
 *  - Direction (zenith, azimuth) in radians, azimuth counter-clockwise from east (+x);
 *    n = (sin zen cos az, sin zen sin az, cos zen) points to the source. Plane-wave delay
 *    tau_s = -n.x_s * n_refr / c; t0 = mean_s(t_s - tau_s); residual r_s = t_s - tau_s - t0;
 *    chi2 = sum_s r_s^2. Positions in metres, times in ns, c = 299792458 m/s.
 *
 * Arithmetic: transforms, interpolation and solve in FP32; direction -> grid coordinates and
 * all timing (peak time, residual, t0, chi2) in FP64.
 *
 * Threading: one ar_ctx may be used from one host thread at a time. Calls taking a stream
 * are asynchronous on it unless stated otherwise. No call throws; every call returns an
 * ar_status, and ar_last_error() gives the message of the last failure on that context.
 */
#ifndef AERAFOLD_H
#define AERAFOLD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ar_status {
  AR_OK = 0,
  AR_ERR_INVALID_ARG = 1,    /* a NULL pointer, a count out of range, a bad descriptor      */
  AR_ERR_UNSUPPORTED_N = 2,  /* samples per channel not 1024, 2048 or 4096                 */
  AR_ERR_NO_PATTERN = 3,     /* pattern id never returned by ar_load_pattern              */
  AR_ERR_OUT_OF_MEMORY = 4,  /* a device or pinned-host allocation failed                 */
  AR_ERR_BUDGET = 5,         /* serving: the event does not fit the state budget at all   */
  AR_ERR_CUDA = 6,           /* a CUDA runtime call failed (message names it)              */
  AR_ERR_TIMEOUT = 7,        /* serving: ar_wait timed out                                  */
  AR_ERR_NOT_READY = 8,      /* serving: ticket still in flight                             */
  AR_ERR_DEVICE = 9          /* a kernel reported an internal error (a bounded wait ran out) */
} ar_status;

/* per-pair status bits (ar_outputs.status) */
#define AR_STATUS_SINGULAR 1u    /* at least one in-band bin was near-singular (E set to 0) */
#define AR_STATUS_ZEN_CLAMP 2u   /* the zenith lay outside the table and was clamped        */
#define AR_STATUS_BAD_DIR 4u     /* the direction was not finite, or its azimuth 2^52 or more
                                    azimuth steps from the pattern's az0: every output of the
                                    pair is 0 */
#define AR_STATUS_BAD_PATTERN 8u /* station_pattern named no loaded pattern: every output is 0 */

typedef struct ar_ctx ar_ctx;

typedef struct ar_config {
  int32_t device;               /* CUDA device ordinal                                      */
  int32_t autotune;             /* 1: the batched path times its tile choices on first use  */
  uint64_t state_budget_bytes;  /* serving admission budget for event state; 0 = 4 GiB      */
} ar_config;

/* Axes of a VEL table. Node (i, j, l) sits at zenith zen0 + i dzen, azimuth az0 + j daz,
 * frequency f0 + l df. Azimuth is periodic: n_az * daz must equal 2 pi. */
typedef struct ar_pattern_desc {
  int32_t n_zen;  double zen0_rad;  double dzen_rad;
  int32_t n_az;   double az0_rad;   double daz_rad;
  int32_t n_freq; double f0_hz;     double df_hz;
} ar_pattern_desc;

/* One event. In ar_unfold every array is DEVICE memory owned by the caller; in
 * ar_unfold_host every array is HOST memory. */
typedef struct ar_event {
  int32_t n_stations;          /* S >= 1                                                   */
  int32_t n_samples;           /* N: 1024, 2048 or 4096                                    */
  int32_t n_dirs;              /* D >= 1                                                   */
  int32_t pattern_id;          /* from ar_load_pattern; every station uses this pattern
                                  unless station_pattern is given (it must be loaded still) */
  double fs_hz;                /* sample rate                                              */
  double refractive_index;     /* n_refr of the plane-wave model; 0 means 1.0              */
  const float* traces;         /* [S][2][N] float32 voltages; 16-byte aligned              */
  const double* pos_m;         /* [S][3] station positions, metres                         */
  const double* t_start_ns;    /* [S] time of sample 0 of each station's trace, ns         */
  const double* dirs_rad;      /* [D][2] (zenith, azimuth), radians                        */
  const int32_t* station_pattern; /* [S] pattern id of each station's antenna (Sec. 3: every
                                  AERA antenna type's pattern resident at once), or NULL.
                                  Patterns may differ in grid. An id that was never loaded
                                  gives AR_STATUS_BAD_PATTERN and zero outputs for that
                                  station's pairs. The unfold kernel walks each direction's
                                  stations grouped by pattern, whatever their order here.  */
} ar_event;

/* Outputs, owned by the caller (DEVICE memory for ar_unfold, HOST memory for
 * ar_unfold_host). efield and envelope are both given (16-byte aligned) or both NULL
 * ("peaks only"); the others are required. */
typedef struct ar_outputs {
  float* efield;               /* [D][S][2][N]  e_theta, e_phi                             */
  float* envelope;             /* [D][S][N]                                                */
  int32_t* peak_idx;           /* [D][S]                                                   */
  float* peak_amp;             /* [D][S] envelope at the peak                              */
  double* peak_time_ns;        /* [D][S]                                                   */
  double* residual_ns;         /* [D][S]                                                   */
  double* t0_ns;               /* [D]                                                      */
  double* chi2;                /* [D] ns^2                                                 */
  uint32_t* status;            /* [D][S] AR_STATUS_* bits                                  */
  double* peak_time_fine_ns;   /* [D][S] or NULL. A variant the paper does not define: the
                                  peak time refined below the sample by the vertex of the
                                  parabola through the envelope at the peak and its two
                                  neighbours, t_start + (peak + delta) 1e9/fs with |delta| <=
                                  1/2 (delta = 0 at the trace ends or without a strict
                                  maximum), in FP64 from the FP32 envelope. When given, the
                                  residual, t0 and chi2 use these times.                  */
  float* snr;                  /* [D][S] or NULL. A variant the paper does not define: the
                                  pulse's signal-to-noise ratio (peak_amp / noise)^2, noise^2
                                  being the mean of envelope^2 over the samples more than N/16
                                  from the peak (0 when there are none or that mean is 0), in
                                  FP32. When given, the direction fit weights station s by
                                  w_s = snr (timing variance taken inversely proportional to
                                  the SNR): t0 = sum w (t - tau) / sum w, residual = t - tau -
                                  t0, chi2 = sum w residual^2; unweighted if the weights sum
                                  to 0.                                                   */
} ar_outputs;

/* Create a context on cfg->device (cfg may be NULL: device 0, defaults). The context owns
 * the device copies of loaded patterns, per-length twiddle tables and a workspace arena.
 * Errors: AR_ERR_INVALID_ARG (ctx NULL), AR_ERR_CUDA (no such device), AR_ERR_OUT_OF_MEMORY. */
ar_status ar_create(ar_ctx** ctx, const ar_config* cfg);

/* Synchronise the device, free everything the context owns, and free ctx. NULL is a no-op. */
ar_status ar_destroy(ar_ctx* ctx);

/* Message of the last failing call on ctx ("" if none). Valid until the next call on ctx.
 * ctx NULL gives the message of the last failing ar_create or ar_unfold_noalloc made by the
 * calling thread (each thread keeps its own; valid until that thread's next failing call). */
const char* ar_last_error(const ar_ctx* ctx);

/* Name of a status code. */
const char* ar_status_string(ar_status s);

/* Copy a VEL table to the device (Sec. 3: the patterns are copied and converted once and
 * stay on the device; all antenna types fit at the same time). host_table is
 * [n_zen][n_az][n_freq][2 channels][2 polarisations] complex64 (interleaved re, im), in
 * host memory that the caller keeps. n_zen >= 2, n_az >= 2, 2 <= n_freq <= 256.
 * Synchronous. Errors: AR_ERR_INVALID_ARG, AR_ERR_OUT_OF_MEMORY, AR_ERR_CUDA. */
ar_status ar_load_pattern(ar_ctx* ctx, const ar_pattern_desc* desc, const float* host_table,
                          int32_t* pattern_id);

/* Prepare the per-length tables and the workspace for events of up to max_stations
 * stations with n_samples samples at fs_hz using pattern_id, so that later ar_unfold calls
 * of that shape allocate nothing (needed before capturing ar_unfold into a CUDA graph).
 * Synchronous. Errors as ar_unfold's validation. */
ar_status ar_prepare(ar_ctx* ctx, int32_t n_samples, double fs_hz, int32_t pattern_id,
                     int32_t max_stations);

/* Unfold every (station, direction) pair of ev into out, asynchronously on stream
 * (a cudaStream_t; NULL = the legacy default stream). All pointers are device pointers.
 * Two kernels run in order: the forward transform of each station's two channels, then the
 * fused per-pair interpolation + solve + inverse transform + envelope + peak, in which the
 * CTA that finishes a direction's last pair also computes its plane-wave residual. Validation errors are returned before any launch;
 * a device-side error is reported by the next ar_sync on this context.
 * If the shape was not prepared, the first call allocates (synchronously).
 * Errors: AR_ERR_INVALID_ARG, AR_ERR_UNSUPPORTED_N, AR_ERR_NO_PATTERN,
 * AR_ERR_OUT_OF_MEMORY, AR_ERR_CUDA. */
ar_status ar_unfold(ar_ctx* ctx, const ar_event* ev, const ar_outputs* out, void* stream);

/* ---- the iterative reconstruction (Sec. 2 of the paper) ----
 * Initial station times from the voltage maxima (argmax of v0^2 + v1^2); a least-squares
 * plane-wave fit gives a direction (the paper's triangulation); the E-field of every station
 * is unfolded for that direction (as ar_unfold with one direction); the envelope maxima give
 * new times; repeat until the angle between successive fitted directions is below tol_rad,
 * the station times repeat, or max_iter unfold iterations have run. The fit is unweighted,
 * linear in (t0, nx, ny) for a fixed nz = sqrt(1 - nx^2 - ny^2), solved in closed form and
 * repeated four times with nz from the previous solution; FP64 throughout. All pointers are
 * DEVICE memory; ev->dirs_rad and ev->n_dirs are ignored. The whole loop is queued on stream
 * with a fixed shape (kernels after convergence return at once), so it can be captured in a
 * CUDA graph once the shape is prepared. */
typedef struct ar_recon_out {
  double* direction;    /* [2] zenith, azimuth of the last fit (NaN if none)                 */
  double* t0_ns;        /* [1] t0 of the last fit                                           */
  double* chi2;         /* [1] sum of squared residuals of the last fit, ns^2               */
  int32_t* iterations;  /* [1] unfold iterations run; -1 if the voltage maxima fit nothing   */
  double* history;      /* [max_iter + 1][2] direction after each fit, NaN after the last; may be NULL */
  ar_outputs last;      /* the last unfold's outputs, D = 1 layouts ([1][S] ...)            */
} ar_recon_out;

/* Errors: as ar_unfold; AR_ERR_INVALID_ARG also for fewer than 3 stations, max_iter outside
 * [0, 64] or tol_rad < 0. */
ar_status ar_reconstruct(ar_ctx* ctx, const ar_event* ev, int32_t max_iter, double tol_rad,
                         const ar_recon_out* out, void* stream);

/* Synchronise stream and report device-side errors raised since the last ar_sync
 * (AR_ERR_DEVICE), then clear them. */
ar_status ar_sync(ar_ctx* ctx, void* stream);

/* ar_unfold on HOST buffers: copies the event's arrays to device memory owned by the
 * context, runs the path on stream, copies every output back and synchronises. Returns
 * when the outputs are in the caller's host arrays. Host arrays may be pageable; pinned
 * memory makes the copies faster. Errors: as ar_unfold, plus AR_ERR_DEVICE. */
ar_status ar_unfold_host(ar_ctx* ctx, const ar_event* ev, const ar_outputs* out, void* stream);

/* Test of the error path of the kernels' bounded waits (not in the paper; for tests only).
 * mode 1: until set back to 0, ar_unfold's unfold kernel gives its corner-slab waits a limit
 * of 1 ms and has each slab mbarrier expect 16 bytes more than its four bulk copies deliver
 * (the copies themselves are unchanged and in bounds), so wherever the kernel stages the
 * slabs in shared memory (patterns whose slabs fit beside the CTAs per SM; larger ones are
 * read from L2 without a wait) each wait runs out: the kernel sets the error
 * word and its CTAs return early, the outputs of that call are undefined, and ar_sync reports
 * AR_ERR_DEVICE (bit 0). The context stays usable; the next call with mode 0 is normal.
 * Errors: AR_ERR_INVALID_ARG (NULL ctx, mode not 0 or 1). */
ar_status ar_set_test_fault(ar_ctx* ctx, int32_t mode);

/* Per-kernel timing. While enabled, ar_unfold records CUDA events on its stream around each
 * of its kernels (which keeps the second kernel from starting before the first ends).
 * ar_kernel_times waits for the last ar_unfold's events and writes the durations in
 * milliseconds: ms[0] station transform, ms[1] fused unfold (including the per-direction
 * residual), ms[2] always 0 (kept for layout stability).
 * Errors: AR_ERR_INVALID_ARG (NULL, or no timed ar_unfold yet), AR_ERR_CUDA. */
ar_status ar_set_profiling(ar_ctx* ctx, int32_t enable);
ar_status ar_kernel_times(ar_ctx* ctx, float* ms);

/* Tensor-core DFT variant of ar_unfold: the same outputs, in the same layouts, with both
 * transforms (the forward transform of the voltages, Sec. 4, and the inverse transform of
 * the analytic signal, Sec. 2) computed as DFT-as-GEMM on tcgen05 tensor cores in BF16 with
 * FP32 accumulation, on 512-sample sub-blocks: N = A x 512, and only the N/4 bins of the
 * 30-80 MHz band enter the GEMMs (j = j1 + A j2, 128 bins per sub-block phase j1). FP32
 * operands are split into BF16 parts: split_terms = 3 keeps hi*hi + hi*lo + lo*hi of a two-way
 * split (about 16 significant bits per product), 6 adds the terms of a three-way split down
 * to 2^-24 (FP32-level). Interpolation, solve, twiddles and the sub-block-phase DFTs are FP32
 * as in ar_unfold; direction cells and timing FP64. The library keeps a workspace of about
 * 20 B per station sample and up to 2^25 x 10 B for the pairs (processed in chunks of
 * 2^25 / N pairs).
 * ev, out: as ar_unfold (device memory); S * N <= 2^24.
 * With ar_set_profiling on, ar_kernel_times gives ms[0] = forward transform and the first
 * chunk's solve, ms[1] = the first chunk's inverse GEMM, ms[2] = the rest (post-pass, later
 * chunks, residual).
 * Errors: as ar_unfold, and AR_ERR_INVALID_ARG for split_terms not 3 or 6 or S * N > 2^24. */
ar_status ar_unfold_tc(ar_ctx* ctx, const ar_event* ev, const ar_outputs* out, int32_t split_terms, void* stream);

/* ---- batched launches over uneven events ----
 *
 * A batch plan runs many events of different sizes (stations, trace lengths, direction
 * counts) in one CUDA-graph launch: per trace length, one station kernel over all stations
 * and one persistent unfold kernel over all (station, direction) pairs of those events, with
 * the same per-pair arithmetic as ar_unfold (results are identical bit for bit). */
typedef struct ar_batch ar_batch;

typedef struct ar_batch_limits {
  int32_t max_events;    /* events per ar_batch_run (<= 65536)                               */
  int32_t max_stations;  /* stations summed over the events of one run                       */
  int32_t max_dirs;      /* directions summed over the events of one run                     */
  int32_t max_n_freq;    /* largest frequency-node count of the patterns used (2..256)       */
} ar_batch_limits;

/* Create a plan on ctx: allocates its device workspace (station spectra for max_stations
 * traces of up to 4096 samples, direction counters, descriptor tables), two pinned staging
 * buffers, and captures two CUDA graph instances. Synchronous.
 * Errors: AR_ERR_INVALID_ARG, AR_ERR_OUT_OF_MEMORY, AR_ERR_CUDA. */
ar_status ar_batch_create(ar_ctx* ctx, const ar_batch_limits* limits, ar_batch** plan);

/* Run n_events events (arrays on the host; each event's and output's arrays are DEVICE
 * pointers as for ar_unfold) as one graph launch on stream. Asynchronous: returns once the
 * launch is queued. Two runs may be in flight; a third waits on the host for the first to
 * finish with its staging buffer. If the context was created with autotune = 1, the first
 * run tunes the plan on its events (running the batch several times; the results are the
 * same each time): first every length class at a common 1..6 CTAs per SM, then each class on
 * its own, longest traces first, over its CTAs per SM and the placement of its corner slabs
 * (staged in shared memory where they fit, or read from L2), keeping what is fastest (see
 * ar_batch_tuning_info). Device errors are reported by ar_sync on the plan's context.
 * Errors: AR_ERR_INVALID_ARG, AR_ERR_UNSUPPORTED_N, AR_ERR_NO_PATTERN, AR_ERR_BUDGET (the
 * events exceed the plan's limits), AR_ERR_CUDA. */
ar_status ar_batch_run(ar_batch* plan, const ar_event* events, const ar_outputs* outs, int32_t n_events,
                       void* stream);

/* Chosen unfold CTAs per SM for the 1024-, 2048- and 4096-sample classes (ctas_per_sm[3]),
 * and the autotuner's measured graph time in ms for 1..6 CTAs per SM (candidate_ms[6], 0 if
 * not tried, e.g. beyond what every class can hold; may be NULL). A candidate k runs each
 * class at min(k, the most CTAs per SM it can hold). */
ar_status ar_batch_tuning(const ar_batch* plan, int32_t* ctas_per_sm, float* candidate_ms);

/* The plan per trace-length class (index 0, 1, 2 = 1024, 2048, 4096 samples), as the
 * autotuner left it (or the defaults: the most CTAs per SM, slabs staged where that costs no
 * occupancy). */
typedef struct ar_batch_plan_info {
  int32_t ctas_per_sm[3];      /* unfold CTAs per SM */
  int32_t slabs_staged[3];     /* 1: corner slabs staged in shared memory; 0: read from L2 */
  int32_t max_ctas_per_sm[3];  /* the most the class's unfold kernel can hold */
  int32_t tuned;               /* 1 once the autotuner has run (autotune = 1 and a first run) */
  int32_t candidates;          /* plans it timed */
  float default_ms;            /* graph time of the untuned plan on the tuning run's events */
  float tuned_ms;              /* graph time of the chosen plan on the same events */
} ar_batch_plan_info;

/* Errors: AR_ERR_INVALID_ARG (NULL). */
ar_status ar_batch_tuning_info(const ar_batch* plan, ar_batch_plan_info* info);

/* Wait for the plan's runs in flight and free it. NULL is a no-op. */
ar_status ar_batch_destroy(ar_batch* plan);

/* ---- serving: continuous batching ----
 *
 * A server accepts events whose arrays (inputs and outputs) are in HOST memory and returns
 * a ticket. A server thread admits queued events in arrival order while their device state
 * (inputs and outputs on the device) fits the state budget, copies the inputs in, runs the
 * admitted events as one batch launch and copies the outputs back, on three streams. With two
 * launches in flight, events that arrive while the GPU is busy join the next launch as memory
 * frees up, and its copies overlap the running launch. Results do not depend on which other
 * events share a launch (identical bit for bit alone and in the mix). */
typedef struct ar_server ar_server;

typedef struct ar_server_config {
  uint64_t state_budget_bytes;     /* device memory for admitted events; 0 = the context's budget */
  int32_t max_batch_events;        /* events per launch; 1 with max_inflight 1 = plain serving    */
  int32_t max_inflight;            /* launches in flight: 1 or 2                                  */
  int32_t max_stations_per_event;  /* larger events are refused at submit (AR_ERR_BUDGET)         */
  int32_t max_n_freq;              /* largest frequency-node count of the patterns used           */
} ar_server_config;

/* Start a server on ctx (allocates the state budget on the device, a batch plan and a server
 * thread). Errors: AR_ERR_INVALID_ARG, AR_ERR_OUT_OF_MEMORY, AR_ERR_CUDA. */
ar_status ar_server_create(ar_ctx* ctx, const ar_server_config* cfg, ar_server** server);

/* Queue one event. ev's arrays and out's arrays are HOST memory that must stay valid and
 * untouched until the ticket completes (pinned memory makes the copies asynchronous).
 * Directions per event <= 256. Errors: validation as ar_unfold; AR_ERR_BUDGET when the event
 * can never fit the state budget or the per-event limits. */
ar_status ar_submit(ar_server* server, const ar_event* ev, const ar_outputs* out, uint64_t* ticket);

/* AR_OK once the ticket's outputs are in place, AR_ERR_NOT_READY before, or the error that
 * ended it. Unknown ticket: AR_ERR_INVALID_ARG. */
ar_status ar_poll(ar_server* server, uint64_t ticket);

/* Block until the ticket completes (returns as ar_poll) or timeout_ms passes
 * (AR_ERR_TIMEOUT; the request stays queued). */
ar_status ar_wait(ar_server* server, uint64_t ticket, int32_t timeout_ms);

/* Host steady-clock times (ns) of the ticket's submission and completion (0 if not done). */
ar_status ar_ticket_times(ar_server* server, uint64_t ticket, int64_t* submit_ns, int64_t* done_ns);

/* Forget a completed ticket (its record is kept until then). */
ar_status ar_ticket_release(ar_server* server, uint64_t ticket);

/* Finish every queued and running event, stop the thread, free the server. NULL is a no-op. */
ar_status ar_server_destroy(ar_server* server);

/* ar_unfold without any device allocation, for callers that cannot call cudaMalloc: a
 * real-time acquisition loop whose device memory map is fixed after start-up, or a plug-in
 * running inside another program's CUDA context and memory pool. The paper has no
 * counterpart; it is an integration aid of this library.
 *
 * Same computation, conventions and output layouts as ar_unfold, with no context: the
 * caller passes the pattern descriptor and a DEVICE pointer to its VEL table (layout of
 * ar_load_pattern, 16-byte aligned; ev->pattern_id is ignored), the event's device arrays
 * and the device outputs. Everything else the kernels need (station spectra, twiddle and
 * frequency-cell tables, per-direction counters, the error word) lives in one fixed 4 MiB
 * array inside the library,
 * present on every GPU that loads it until the process exits.
 *  - Limits: n_stations x n_samples <= 983,040 (240 stations of 4096 samples, 480 of 2048,
 *    960 of 1024) and n_dirs <= 4096; larger events return AR_ERR_INVALID_ARG and a
 *    message naming the limit. One pattern per call: ev->station_pattern must be NULL.
 *  - Set-up: the first call on a device (with that device current) looks up the array's
 *    device address and sets kernel attributes; make that first call before any stream
 *    capture.
 *  - The array is shared by every call and keeps the last call's contents; each call clears
 *    the error word and rewrites the tables before use. Calls whose work overlaps on the GPU
 *    (different streams, or different host threads, without ordering) race on the array.
 *  - Asynchronous on stream; there is no context to report device-side errors afterwards.
 *  - Errors: AR_ERR_INVALID_ARG, AR_ERR_UNSUPPORTED_N, AR_ERR_CUDA; the message is
 *    ar_last_error(NULL). */
ar_status ar_unfold_noalloc(const ar_pattern_desc* desc, const float* device_table, const ar_event* ev,
                            const ar_outputs* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* AERAFOLD_H */
