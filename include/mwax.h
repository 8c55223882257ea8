/*
 * mwax.h -- C ABI of a single-GPU (NVIDIA B300, sm_103a) MWAX FX correlator stage.
 *
 * The library turns a sub-observation of int8 complex coarse-channel voltages
 * (tiles x 2 polarisations) into averaged visibilities, as the GPU stage of the
 * MWAX FX-engine does (Morrison et al., "MWAX: A New Correlator for the Murchison
 * Widefield Array", Sec. 2.5-2.7):
 *   F-step  unpack int8, fine-channel FFT of N points, per-path delay/phase
 *           correction (Sec. 2.5.1, 4.3), written as X-engine operands;
 *   X-step  Hermitian cross-power of all signal-path pairs per fine channel,
 *           summed over the frames of each integration (Sec. 2.5.2);
 *   average centre-symmetric channel averaging by fscrunch F (Sec. 2.6), written in
 *           MWAX_ORDER with the visibility weights table after each set (Sec. 2.7).
 * Every step runs in the library's own CUDA kernels.  There is no CPU fallback: on a
 * machine without a usable B300 the calls fail with MWAX_ECUDA.
 *
 * Conventions (the paper leaves these open; the library fixes them as follows):
 *   - sample rate Fs = 1,280,000 complex samples/s (Sec. 2.5);
 *   - signal path p = 2 * tile + pol, pol x = 0, y = 1;
 *   - voltages: int8 [block][path][block_samples][2] (re, im), block_samples = 64,000
 *     by default (one 50 ms data block per path, Sec. 2.5);
 *   - frame m = samples [m N, (m+1) N) of the call; forward unnormalised FFT
 *     X[k] = sum_n x[n] e^{-2 pi i k n / N};
 *   - channel c = u + floor(N/2) for ultrafine offset u (centre-symmetric, DC at
 *     c = N/2, Sec. 2.6); f_u = u Fs / N;
 *   - delay correction Y = X exp(+2 pi i (nu + f_u) tau_p(t_m)), with
 *     tau_p(t) = c0 + c1 t + c2 t^2 seconds, t_m = (m + 1/2) N / Fs seconds from the
 *     call's first sample, nu = sky frequency of the coarse channel (Sec. 2.5.1);
 *   - cross-power V_pq = sum_m Y_p conj(Y_q) (time is a sum, frequency a weighted
 *     mean over the ultrafine bins of each output channel, Sec. 2.6);
 *   - MWAX_ORDER: [integration][baseline][channel][pol], baselines (i <= j) row-major
 *     over the upper triangle including autos, pols xx, xy, yx, yy (Sec. 2.7);
 *   - after each integration's visibilities: weights float32 [baseline][pol], all 1.0
 *     (the paper's current occupancy weights, Sec. 2.7).
 */
#ifndef MWAX_H
#define MWAX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mwax_plan mwax_plan;

typedef enum {
    MWAX_OK = 0,
    MWAX_EINVAL = 1,        /* invalid argument or plan parameters                  */
    MWAX_ENOMEM = 2,        /* device or host allocation failed                      */
    MWAX_ECUDA = 3,         /* CUDA runtime error (no device, launch failure, ...)   */
    MWAX_EUNSUPPORTED = 4,  /* valid per the paper but not built (e.g. an FFT length) */
    MWAX_ETIMEOUT = 5       /* a device-side bounded wait gave up (status word)      */
} mwax_status;

typedef enum {
    MWAX_FP32 = 0,  /* FP32 FFT and FP32 CUDA-core cross-multiply (the paper's form)     */
    MWAX_FP16 = 1,  /* FP32 FFT, FP16 operands on tcgen05 tensor cores, FP32 accumulate  */
    MWAX_FP8 = 2,   /* FP32 FFT, e4m3 operands with per-path-per-channel scales, tcgen05 */
    MWAX_INT8 = 3,  /* no FFT (N = 1, F = 1), exact integer sums, int64 output           */
    MWAX_FP16X3 = 4 /* FP32 FFT; each operand an FP16 hi/lo pair (22 significant bits),
                       three FP16 products per complex term on tcgen05 (the lo x lo term,
                       2^-22 of the product, dropped), partial sums of 128 frames added in
                       FP32: FP32-level error on the tensor cores; 128 x 128 tiles,
                       operands 8 B per sample and path like MWAX_FP32                  */
} mwax_precision;

/* Plan parameters.  Zero-initialise and set what you need; zero selects the default. */
typedef struct {
    int n_tiles;                 /* T >= 1; signal paths n = 2 T                          */
    int fft_len;                 /* N: fine-channel FFT length (1 = no FFT)               */
    int fine_avg;                /* F: fscrunch, N % F == 0; output channels M = N / F    */
    double int_time_s;           /* integration time; int_time * Fs must be a multiple of N */
    long long samples_per_call;  /* samples per path per call; 0 = one integration        */
    int block_samples;           /* samples per path per data block; 0 = 64,000           */
    int precision;               /* mwax_precision; 0 = MWAX_FP32                          */
    double sky_freq_hz;          /* nu, centre frequency of the coarse channel; 0 allowed  */
    int keep_dc;                 /* 0 (default) = exclude DC from the centre channel when
                                    F > 1 (Sec. 2.6); 1 = keep it                          */
    size_t workspace_limit;      /* bytes of device workspace; 0 = 16 GiB                 */
    double sample_rate_hz;       /* coarse-channel sample rate Fs; 0 = 1.28 MS/s.  Above
                                    the channel spacing for oversampled channels (Sec. 4.5) */
    int keep_bins;               /* ultrafine channels passed to the X step, centred on DC;
                                    0 = all N.  Oversampled channels discard the rest
                                    (Sec. 4.5); M = keep_bins / F                           */
} mwax_plan_desc;

/* Derived sizes of a plan (all counts per call). */
typedef struct {
    int n_paths;                 /* n = 2 T                                   */
    long long n_baselines;       /* B = T (T + 1) / 2                         */
    int n_chan_out;              /* M = keep_bins / F (N / F by default)      */
    long long frames_per_int;    /* K = int_time Fs / N                       */
    long long n_ints;            /* integrations per call                     */
    size_t input_bytes;          /* n_blocks * n * block_samples * 2          */
    size_t vis_set_bytes;        /* one integration's visibilities            */
    size_t weights_bytes;        /* one integration's weights table           */
    size_t output_bytes;         /* n_ints * (vis_set_bytes + weights_bytes)  */
    size_t workspace_bytes;      /* device memory the plan holds: operand planes and
                                    F-step scratch (which a tuning choice may grow) */
    int precision;
    double x_flop_alg;           /* X-step work per call: 8 flop per complex multiply-
                                    accumulate over the n (n + 1) / 2 unique path pairs,
                                    each frame and each ultrafine channel feeding an
                                    output channel (exactly once)                      */
    double x_flop_issued;        /* the same count over what the X kernels execute with
                                    the current tuning: whole tiles (including the pairs
                                    below the diagonal and past n that a tile covers),
                                    frames rounded up to the kernel's K block, boundary
                                    channels of two runs computed by both.  FP16X3
                                    issues three FP16 products per term on top of it  */
} mwax_plan_info;

/*
 * Create a plan: FP32 precision, sky frequency 0, DC excluded, one integration per
 * call, 64,000-sample blocks.  Allocates the plan's device workspace on the current
 * device.  Returns NULL on error (see mwax_last_error()).
 * Validation (MWAX_EINVAL): n_tiles >= 1; fine_avg >= 1 and fft_len % fine_avg == 0;
 * block_samples % fft_len == 0; int_time_s * Fs an integer multiple of fft_len;
 * samples_per_call a multiple of both the integration length and block_samples.
 * FFT lengths built (else MWAX_EUNSUPPORTED): 1, 16, 32, 64, 128, 256, 512, 640,
 * 1280, 3200, 6400.  MWAX_INT8 needs fft_len = fine_avg = 1.
 */
mwax_plan* mwax_plan_create(int n_tiles, int fft_len, double int_time_s, int fine_avg);

/* Create a plan from a descriptor (see mwax_plan_desc).  NULL on error. */
mwax_plan* mwax_plan_create_ex(const mwax_plan_desc* desc);

/* Sizes of a plan.  MWAX_EINVAL on NULL arguments. */
mwax_status mwax_plan_get_info(const mwax_plan* plan, mwax_plan_info* info);

/* Bytes of one call's output (visibility sets and weight tables of all integrations). */
size_t mwax_plan_output_bytes(const mwax_plan* plan);

/* Bytes of one call's input voltages. */
size_t mwax_plan_input_bytes(const mwax_plan* plan);

/* Enqueue all further work of this plan on `cuda_stream` (a cudaStream_t; NULL = the
 * legacy default stream).  The plan does not own the stream. */
mwax_status mwax_plan_set_stream(mwax_plan* plan, void* cuda_stream);

/*
 * Correlate one call's worth of voltages (samples_per_call samples per path).
 *   voltages   device pointer, int8 [n_blocks][n][block_samples][2], caller-owned,
 *              16-byte aligned;
 *   delay_poly NULL (no delay/phase correction) or n x 3 float64 (c0 [s], c1 [s/s],
 *              c2 [s/s^2]) per signal path, host or device memory; read before return
 *              (host) or in stream order (device).  Must be NULL for MWAX_INT8;
 *   vis_out    device pointer, mwax_plan_output_bytes() bytes, caller-owned, 16-byte
 *              aligned.  Per integration: visibilities [B][M][4] complex float32
 *              (MWAX_INT8: [B][1][4] pairs of int64 re, im), then weights float32 [B][4].
 * The work is enqueued on the plan's stream and the call returns without waiting.
 * Errors found by the kernels (bounded waits that gave up) are reported by the next
 * mwax_plan_sync().  Not thread-safe per plan; use one plan per stream.
 */
mwax_status mwax_correlate(mwax_plan* plan, const int8_t* voltages, const double* delay_poly, void* vis_out);

/*
 * The same from host memory: copies the voltages to the device block by block on a
 * copy stream, overlapped with the correlation, and copies the result back into
 * vis_out (host).  Pinned host buffers give full PCIe bandwidth; pageable ones work.
 * Synchronous: returns when vis_out holds the result.
 */
mwax_status mwax_correlate_host(mwax_plan* plan, const int8_t* voltages, const double* delay_poly, void* vis_out);

/*
 * Streaming form of mwax_correlate_host for consecutive sub-observations (the real-time
 * loop of Sec. 2.3: data keep arriving while earlier data are correlated).  Enqueues the
 * copies, the correlation and the copy back, and returns without waiting.  The plan keeps
 * two device staging sets (voltages + output, allocated on first use) and alternates
 * between them, so the voltages of call k + 1 stream in while call k is correlated; the
 * correlations themselves run in call order on the plan's stream.
 *   voltages, vis_out   host memory as for mwax_correlate_host; pinned (page-locked)
 *                       buffers are needed for the copies to overlap.  The caller keeps
 *                       voltages unchanged and does not read vis_out until
 *                       mwax_plan_sync() returns;
 *   delay_poly          as for mwax_correlate_host (copied when the call is enqueued).
 * Errors found by the kernels are reported by mwax_plan_sync().  Not thread-safe per plan.
 */
mwax_status mwax_correlate_host_async(mwax_plan* plan, const int8_t* voltages, const double* delay_poly,
                                      void* vis_out);

/*
 * Extended call (Sec. 2.4, 4.1, 4.3): tabulated fractional delays and zeroing flags.
 *   voltages, vis_out   as for mwax_correlate (device, 16-byte aligned);
 *   delay_poly          as for mwax_correlate, or NULL;
 *   delay_table         NULL or float64 [n][table_steps] fractional delays in seconds, host
 *                       or device memory: entry s holds for samples
 *                       [s table_step_samples, (s + 1) table_step_samples) of the call, and a
 *                       frame takes the entry holding its centre (entries past the end repeat
 *                       the last).  Exclusive with delay_poly; not for MWAX_INT8;
 *   table_steps         entries per path (>= 1 with a table);
 *   table_step_samples  samples per entry; 0 = 6,400 (5 ms at 1.28 MS/s, the paper's cadence);
 *   zero_flags          NULL or uint8 [n_blocks][n], host or device memory: nonzero marks a
 *                       data block of a path that was zeroed (lost or excised).  Its samples
 *                       are excluded (read as zero) and each integration's weights table
 *                       receives the occupancy of every baseline/pol: the fraction of the
 *                       integration's frames whose blocks are unflagged in both paths;
 *   normalise           nonzero: divide each visibility by its occupancy weight (zero weight
 *                       leaves zeros).  Float precisions only (MWAX_EINVAL for MWAX_INT8).
 * Host-memory tables and flags are copied before the call returns.  The plan keeps one
 * device copy of each (grown on demand: the first call with a larger table allocates).
 */
typedef struct {
    const int8_t* voltages;
    const double* delay_poly;
    const double* delay_table;
    long long table_steps;
    long long table_step_samples;
    const uint8_t* zero_flags;
    int normalise;
    void* vis_out;
} mwax_call;
mwax_status mwax_correlate_ex(mwax_plan* plan, const mwax_call* call);

/*
 * Passband de-ripple (Sec. 4.2): a real magnitude gain per ultrafine channel, multiplied
 * into every spectral value with the delay phasor (visibilities scale by its square).
 * gain: host float32 [fft_len] in channel order c = u + N/2 (u = ultrafine offset from DC),
 * each finite and > 0; NULL restores a flat passband.  Applies to calls enqueued after it
 * returns.  MWAX_EUNSUPPORTED for MWAX_INT8 (exact integer sums).
 */
mwax_status mwax_plan_set_passband(mwax_plan* plan, const float* gain);

/* Wait for the plan's stream; returns MWAX_ETIMEOUT / MWAX_ECUDA if a kernel reported
 * an error since the last sync, and clears the device status word. */
mwax_status mwax_plan_sync(mwax_plan* plan);

/*
 * Bound of every device-side wait of the plan's X-step kernels (an operational control,
 * no counterpart in the paper): a wait gives up after kilocycles x 1000 SM clock cycles,
 * raises the kernel's abort flag, lets its own TMA loads and MMAs in flight complete (a
 * fixed bound of ~2 s that does not follow this limit), frees its tensor memory and
 * returns; mwax_plan_sync() then reports MWAX_ETIMEOUT and the call's output is
 * incomplete.  0 restores the default (2,000,000, about 1 s).  Applies to calls enqueued
 * after it returns; in a batch a launch takes the largest limit of its plans.
 */
mwax_status mwax_plan_set_wait_limit(mwax_plan* plan, unsigned int kilocycles);

/*
 * Per-stage device time (the paper's Table 2 breaks the FX-engine time down by
 * sub-function).  While enabled, CUDA events bracket each of the plan's kernel launches
 * on its stream.  mwax_plan_stage_times() waits for the stream and returns, per stage,
 * the summed milliseconds and the number of launches since the last call (then resets):
 * stage 0 = output init (zero + weights), 1 = F-step, 2 = X-step.  Launch counts are
 * kept whether or not timing is enabled.
 */
mwax_status mwax_plan_enable_timing(mwax_plan* plan, int enable);
mwax_status mwax_plan_stage_times(mwax_plan* plan, double ms[3], long long launches[3]);

/* ------------------------------------------------------------------ autotuning */

/* Launch choices of a plan.  fstep_variant: 0 = two-pass radix-32 F-step kernel (built
 * for N = 32..512; the generic kernel elsewhere), 1 = generic shared-memory Stockham
 * kernel, 2 = tensor-core DFT products (N = 1280, 6400 with FP16 operands out, i.e. the
 * MWAX_FP16 and MWAX_FP8 forms: the four-step DFT N = 80 x 16, 80 x 80 with both stages on
 * tcgen05; N = 32, 64, 128 in every float form: the direct DFT as one product; variant 0
 * elsewhere), 3 = 128-row tensor-core F-step (N = 128 x 10, 128 x 50 with FP16 operands
 * out: stage A on tcgen05 with every accumulator lane a bin, stage B a radix-5/2 DFT in
 * registers; variant 2 elsewhere), 4 = direct DFT with the frames on the accumulator lanes
 * (N = 32, 64, 128 with FP16 operands out: one tcgen05 product per 128 frames, each warp
 * store writing 32 consecutive frames of an operand row; variant 0 elsewhere).  run_len: output channels per X-step work item (0 = the plan's own choice: the
 * run length whose longest-first schedule of the work items on the GPU's resident CTA
 * slots is shortest).  window: column width of a tensor-core X-step tile, 128 or 256
 * (MWAX_FP16X3 always runs 128).  ms: device time of one call measured by the autotuner. */
typedef struct {
    int fstep_variant;
    int run_len;
    int window;
    double ms;
} mwax_tuning;

/*
 * Autotuner: runs the plan on the caller's buffers (same arguments as mwax_correlate),
 * three calls per candidate, timed with CUDA events on the plan's stream (the fastest of
 * the three counts).  First the F-step variant (radix-32 or generic, for N = 32..512;
 * the tensor-core direct DFT for N = 32, 64, 128 in the float forms; generic and both
 * tensor-core F-steps for N = 1280 and 6400 in the FP16 and FP8 forms) with
 * the plan's current X-step choice; then, with the faster variant, the tile window (256 or
 * 128 for the FP16 / FP8 forms; 128 only for MWAX_FP16X3) x the run length (the plan's
 * modelled choice, 3, 5, 11 and all output channels; candidates that configure the same
 * launches are timed once).  Keeps the fastest.  Synchronous.  vis_out is overwritten with
 * a valid result.  best (may be NULL) receives the choice and its time.
 */
mwax_status mwax_plan_autotune(mwax_plan* plan, const int8_t* voltages, const double* delay_poly, void* vis_out,
                               mwax_tuning* best);
/* Set or read a plan's launch choices (waits for the plan's stream before changing).
 * Choosing F-step variant 3 or 4 allocates its device scratch once if the plan has none
 * (the frames' delay terms, written by a small kernel before each F-step launch; variant 3
 * also one slot of frame-major spectra); MWAX_ENOMEM if that fails. */
mwax_status mwax_plan_set_tuning(mwax_plan* plan, const mwax_tuning* tuning);
mwax_status mwax_plan_get_tuning(const mwax_plan* plan, mwax_tuning* tuning);

/* ------------------------------------------------------------------ batches */

/*
 * Batch of plans (e.g. many coarse channels of mixed tile counts, FFT lengths,
 * integration times and precisions) correlated together on one stream.  Each call runs
 * every plan once: per round, the plans' F-steps on auxiliary streams, then one
 * persistent tcgen05 X-step launch per tensor-core kernel mode (all FP16 / FP8 plans; all
 * FP16X3 plans; all integer-mode plans), each over the merged work of its plans (one job
 * per plan, work items claimed dynamically, most expensive first); FP32 plans run their
 * own CUDA-core X-steps.  The paper processes one coarse channel per server (Sec. 2.1); a
 * batch processes many on one GPU.  The batch references the plans (they must outlive it,
 * stay on one device and not be used on their own while the batch runs) and uses the
 * plans' workspaces.  The plans' launch choices (mwax_plan_set_tuning, mwax_plan_autotune,
 * which may also allocate or release F-step scratch) are read when the batch is created:
 * change them only before.  Returns NULL on error.
 */
typedef struct mwax_batch mwax_batch;
mwax_batch* mwax_batch_create(mwax_plan* const* plans, int n_plans);

/* Stream of the batch's work (a cudaStream_t; NULL = legacy default stream). */
mwax_status mwax_batch_set_stream(mwax_batch* batch, void* cuda_stream);

/* CUDA graphs (default on): the first call runs eagerly; later calls capture the whole
 * schedule once per set of buffer pointers and replay it with one graph launch. */
mwax_status mwax_batch_set_graphs(mwax_batch* batch, int enable);

/*
 * One call of every plan: voltages[i], delay_poly[i] (device pointer or NULL; NULL array
 * = no delays) and vis_out[i] are plan i's arguments as for mwax_correlate (device
 * memory).  Asynchronous on the batch's stream.
 */
mwax_status mwax_batch_correlate(mwax_batch* batch, const int8_t* const* voltages, const double* const* delay_poly,
                                 void* const* vis_out);

/* Wait for the batch's stream; MWAX_ETIMEOUT if a bounded device wait gave up. */
mwax_status mwax_batch_sync(mwax_batch* batch);

/* Free the batch (not its plans).  NULL is a no-op. */
void mwax_batch_destroy(mwax_batch* batch);

/* ------------------------------------------------------------------ serving */

/*
 * Real-time serving loop: sub-observations arrive from the host (as the paper's FX-engine
 * receives 8 s subfiles through its input ring buffer, Sec. 2.5) and are admitted onto
 * the GPU in arrival order as device lanes and HBM free up.  Each lane is a CUDA stream
 * with its own cached plans and reusable device buffers; a request runs H2D copy ->
 * correlation -> D2H copy on its lane, and requests on different lanes overlap on the
 * device.  A scheduler thread inside the server makes all of its CUDA calls.
 */
typedef struct mwax_server mwax_server;

typedef struct {
    size_t hbm_budget;       /* device bytes for request buffers and plan workspaces; 0 = 64 GiB */
    int n_lanes;             /* requests in flight on the device at once; 0 = 4                  */
    size_t workspace_limit;  /* per-plan workspace when a request's desc leaves it 0; 0 = 2 GiB  */
} mwax_server_desc;

typedef struct {
    long long submitted, completed, failed, queued, in_flight;
    double p50_ms, p99_ms, max_ms;   /* latency from submission to result in host memory   */
    long long deadline_misses;       /* completed requests later than their deadline        */
    size_t hbm_in_use;               /* device bytes held by lanes (buffers and plans)       */
    long long cold_starts;           /* admissions that created a plan (first request of a
                                        shape on a lane, or after an eviction); their latency
                                        includes plan creation                                */
    double p50_warm_ms, p99_warm_ms; /* latency of the requests that found their plan cached
                                        (steady state: no plan creation)                     */
} mwax_server_stats;

/* Start a server on the current device (NULL desc = defaults).  NULL on error. */
mwax_server* mwax_server_create(const mwax_server_desc* desc);

/*
 * Submit one request: plan parameters (any precision; the plan is created on first use
 * per lane and cached), host voltages (pinned memory lets the copy overlap), host delay
 * polynomial or NULL, host output buffer of the plan's output_bytes, and a deadline in
 * seconds after submission (0 = none; only counted in the statistics).  Returns the
 * request id (>= 0) or -1.  Non-blocking; the buffers must stay valid until completion.
 */
long long mwax_server_submit(mwax_server* server, const mwax_plan_desc* desc, const int8_t* voltages,
                             const double* delay_poly, void* vis_out, double deadline_s);

/* 1 = done, 0 = pending, negative = -(mwax_status) of a failed request. */
int mwax_server_poll(mwax_server* server, long long request_id);

/* Block until the request completes. */
mwax_status mwax_server_wait(mwax_server* server, long long request_id);

/* Block until every submitted request has completed. */
mwax_status mwax_server_drain(mwax_server* server);

/* Counters and latency percentiles so far. */
mwax_status mwax_server_get_stats(mwax_server* server, mwax_server_stats* stats);

/* Start the statistics afresh (latencies, counts, misses, cold starts; requests already
 * submitted still complete, and count if they complete after the reset), e.g. after
 * warm-up requests that created the plans. */
mwax_status mwax_server_reset_stats(mwax_server* server);

/* Finish the queued requests, free everything.  NULL is a no-op. */
void mwax_server_destroy(mwax_server* server);

/* ------------------------------------------------------------------ tied-array beamformer */

/*
 * Multibeam beamformer (Sec. 4.4) on the correlator's F-step: the voltages are channelised
 * (N-point FFT, centre-symmetric channel order, no delay correction) and each beam steers
 * every path with its own tabulated fractional delays, then sums the tiles of each
 * polarisation:
 *     B_b,a[m, c] = sum_t Y_{2t+a}[m, c] exp(+2 pi i (nu + f_u) tau_b,2t+a(step(m)))
 * (f_u = (c - N/2) Fs / N; a frame takes the table step that holds its centre sample).
 * Optional detected outputs per interval of int_frames frames: Stokes I of each beam,
 * sum over the interval of |B_x|^2 + |B_y|^2, and the incoherent beam, sum over the
 * interval and the tiles of |Y|^2 per polarisation.  FP32 spectra; the beam sums on the
 * tensor cores from FP16 hi/lo pairs (default) or in FP32 on the CUDA cores (engine 1).
 */
typedef struct mwax_beamformer mwax_beamformer;

typedef struct {
    int n_tiles;                  /* T >= 1                                                   */
    int fft_len;                  /* N: a built FFT length >= 16                              */
    int n_beams;                  /* >= 1                                                     */
    long long samples_per_call;   /* whole blocks                                             */
    int block_samples;            /* 0 = 64,000                                               */
    double sky_freq_hz;           /* nu                                                        */
    double sample_rate_hz;        /* 0 = 1.28 MS/s                                            */
    long long table_step_samples; /* samples per delay-table entry; 0 = 6,400 (5 ms)          */
    int int_frames;               /* frames per detected sample; 0 = no detected outputs      */
    size_t workspace_limit;       /* device bytes for one chunk's spectra; 0 = 4 GiB          */
    int engine;                   /* 0 = tcgen05 tensor cores: per (5 ms step, 4 channels, pol,
                                     16 beams) the beams x tiles by tiles x frames product from
                                     FP16 hi/lo operand pairs, three products per term (FP32-
                                     level error); 1 = FP32 CUDA cores                        */
} mwax_beam_desc;

/* NULL on error (mwax_last_error()); allocates the spectra workspace on the current device. */
mwax_beamformer* mwax_beam_create(const mwax_beam_desc* desc);
mwax_status mwax_beam_set_stream(mwax_beamformer* bf, void* cuda_stream);

/* Output sizes in bytes: which = 0 coherent beams complex64 [n_beams][2][frames][N],
 * 1 Stokes I float32 [n_beams][n_det][N], 2 incoherent float32 [n_det][2][N], with
 * frames = samples_per_call / N and n_det = frames / int_frames (0 without int_frames). */
size_t mwax_beam_output_bytes(const mwax_beamformer* bf, int which);

/*
 * Form the beams of one call.  voltages: device, as for mwax_correlate (16-byte aligned);
 * beam_delay: float64 [n_beams][n][table_steps] seconds, host or device (a pinned host
 * table is waited for; entries past the end of the table repeat the last); beams_out:
 * device, required; power_out, incoh_out: device or NULL (need int_frames >= 1).
 * Asynchronous on the beamformer's stream.
 */
mwax_status mwax_beam_form(mwax_beamformer* bf, const int8_t* voltages, const double* beam_delay,
                           long long table_steps, void* beams_out, float* power_out, float* incoh_out);
/* Waits for the beamformer's stream; MWAX_ETIMEOUT if a bounded device wait of the
 * tensor-core engine gave up (the call's beams are then incomplete). */
mwax_status mwax_beam_sync(mwax_beamformer* bf);

/* Waits for the beamformer's stream, frees everything.  NULL is a no-op. */
void mwax_beam_destroy(mwax_beamformer* bf);

/* ------------------------------------------------------------------ roofline probe */

/*
 * FP32 FMA throughput probe (no counterpart in the paper: it measures the denominator of
 * the CUDA-core X-step's ALU roofline).  Enqueues `blocks` blocks of 256 threads, each
 * thread running 16 independent FMA chains for iters x 8 steps, on cuda_stream; sink is a
 * device buffer of blocks x 256 floats (written only in a case that does not occur).
 * Returns the number of FMAs enqueued (2 flop each), or -1 on invalid arguments or a
 * launch error.  Time it with events on the same stream.
 */
long long mwax_probe_fma(int blocks, int iters, float* sink, void* cuda_stream);

/* ------------------------------------------------------------------ allocation-free call */

/*
 * FP32 correlation of one small job that allocates no memory at all.  The paper has no
 * counterpart.  It is for callers that cannot call cudaMalloc: processes whose device
 * memory belongs to another allocator (a framework's caching pool that has reserved the
 * GPU), plug-ins whose host application forbids them to allocate, and real-time services
 * that ban allocation after start-up because an allocation may block or fail at any time.
 * desc as for mwax_plan_create_ex with precision MWAX_FP32, 1..32 tiles, fft_len
 * 32/64/128/256/512, all bins kept; voltages and vis_out device pointers as for
 * mwax_correlate, 16-byte aligned (vis_out: n_ints x (B M 4 complex64 + B 4 float32)
 * bytes); delay_poly NULL, host or device (host memory is read before the call returns);
 * cuda_stream a cudaStream_t (NULL = legacy default stream).
 * All device working memory is a fixed set of arrays inside the library image (a 32 MiB
 * operand array plus about 40 KB of tables and a status word, held on every GPU that
 * loads the library until exit); jobs whose operands exceed 32 MiB (n_ints x fft_len x 2 x
 * 2T x K rounded up to 128 frames x 4 bytes) are rejected with MWAX_EINVAL, as are
 * misaligned pointers.  The first call on a device (and context) looks up the arrays'
 * device addresses there, under a lock.  Every call uses the same arrays and rewrites
 * what it needs (tables, status, zero padding): calls that overlap on the GPU, on any
 * stream, race and corrupt each other.  Asynchronous on cuda_stream: errors found on the
 * host are returned; if a bounded device wait gives up, every weight of the call's output
 * is set to 0 (no valid data) instead, since no plan holds a status to query.
 */
mwax_status mwax_correlate_noalloc(const mwax_plan_desc* desc, const int8_t* voltages, const double* delay_poly,
                                   void* vis_out, void* cuda_stream);

/* Free the plan and its device workspace (waits for its stream and for host-call copies
 * still in flight first).  NULL is a no-op. */
void mwax_plan_destroy(mwax_plan* plan);

/* Message of the last error on the calling thread ("" if none). */
const char* mwax_last_error(void);

/* Library version string. */
const char* mwax_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MWAX_H */
