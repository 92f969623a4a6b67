/*
 * bege.h -- C ABI of libbege, the GPU matched-filter search for broadband
 * extended gravitational-wave emission (van Putten, arXiv:1708.01609).
 *
 * The library computes, for one strain segment y of N samples and a bank of
 * real templates w_k of L <= N samples (zero-padded to N), the circular
 * correlation of Eq. A1 through the three FFT steps of Eq. 3S,
 *     rho_k[n] = sum_{m<L} w_k[m] y[(n+m) mod N],   n = 0..N-1,
 * predicts sigma_k = sqrt((1/N) sum_n rho_k[n]^2) from the spectra by
 * Parseval's theorem (Eq. PT, read with unnormalised Fourier coefficients),
 * and returns only the tails |rho_k[n]| > kappa sigma_k (Eq. tail, the
 * "all hits" output of Sec. 3.3) as (template, lag, value) records.
 *
 * Conventions shared by every call:
 *   - Every call returns a bege_status (0 = BEGE_OK, negative = error).  On
 *     error, bege_last_error() gives a message for the calling thread.
 *   - Handles (segments, banks, jobs) are int32 ids owned by the context.
 *     The library owns all device memory it allocates; the caller owns every
 *     host buffer it passes and may reuse it as soon as the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream only enqueue work on it; the calls
 *     that return results to host memory synchronise on the job themselves.
 *   - Lags are circular indices 0..N-1.  Template indices are bank rows.
 *   - Sizes: N is a power of two in [2^10, 2^17]; 1 <= L <= min(N, 2^16).
 *   - Device: one context drives one GPU (sm_103a).  No CPU fallback exists:
 *     if no usable GPU is present bege_create fails with BEGE_ECUDA.
 */
#ifndef BEGE_H
#define BEGE_H

#include <stdint.h>

/* The library is built with hidden symbol visibility; only the calls
 * declared here are exported. */
#if defined(__GNUC__)
#define BEGE_API __attribute__((visibility("default")))
#else
#define BEGE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bege_ctx bege_ctx; /* opaque, library-owned */

typedef enum {
  BEGE_OK = 0,
  BEGE_EINVAL = -1,      /* malformed argument or unknown handle            */
  BEGE_ENOMEM = -2,      /* device or host allocation failed                */
  BEGE_EBUDGET = -3,     /* request would exceed hbm_budget_bytes           */
  BEGE_EOVERFLOW = -4,   /* more tails than the buffers hold; count is true */
  BEGE_ENOTREADY = -5,   /* job not finished (non-blocking query)           */
  BEGE_ETIMEDOUT = -6,   /* a bounded device wait gave up                   */
  BEGE_ECUDA = -7        /* CUDA runtime error (message in last_error)      */
} bege_status;

typedef struct {
  double fs;                  /* sample rate in Hz (the paper: 4096, Sec. 3)     */
  uint64_t hbm_budget_bytes;  /* cap on library-owned device memory; 0 = none    */
  uint64_t tail_capacity;     /* device tail records per job; 0 = 1<<20          */
  int32_t precision;          /* 0 = FP32; 1 = BF16x3, 2 = FP16x3: the precision
                                 form, column FFTs on tensor cores with split
                                 (hi + lo) 16-bit operands, FP32 accumulation
                                 (needs N >= 2^14, templates <= 4096 samples) */
  int32_t reserved;           /* must be 0                                       */
} bege_config;

/* Linear chirp f(t) = f0 + fdot t (Sec. 3, Eq. s bank over (f, fdot)). */
typedef struct {
  double f0;    /* Hz   */
  double fdot;  /* Hz/s */
} bege_chirp;

/* One tail record (Eq. tail, all hits): template row, lag n, signed rho. */
typedef struct {
  uint32_t tmpl;
  uint32_t lag;
  float value;
} bege_tail;

/* Create a context on CUDA device `device`.  `cfg` may be NULL for defaults
 * (fs = 4096, no budget, 1<<20 tail records, FP32).  *out receives the
 * context; destroy it with bege_destroy.  Errors: EINVAL (bad cfg), ECUDA. */
BEGE_API int bege_create(bege_ctx** out, int device, const bege_config* cfg);

/* Free every device buffer and handle of the context. */
BEGE_API int bege_destroy(bege_ctx* ctx);

/* Segment spectrum (Eq. 3S first step; Sec. 3.2 step i).  Copies `n` FP32
 * strain samples from HOST memory `strain`, computes the unnormalised DFT
 * D_j = sum_n y[n] e^{-2 pi i j n / N}, j = 0..N/2, and keeps it resident on
 * the device (with the derived product coefficients used by bege_correlate).
 * `channel` is a caller label (e.g. 0 = H1, 1 = L1) stored with the segment.
 * *seg_id receives the handle.  Errors: EINVAL (n not a power of two in
 * range, NULL pointers), EBUDGET, ENOMEM, ECUDA. */
BEGE_API int bege_load_segment(bege_ctx* ctx, const float* strain, int64_t n, int32_t channel,
                               void* stream, int32_t* seg_id);

/* As bege_load_segment, but `strain_dev` is a DEVICE pointer to n FP32
 * samples on the context's GPU (read on `stream`; not retained). */
BEGE_API int bege_load_segment_device(bege_ctx* ctx, const float* strain_dev, int64_t n,
                                      int32_t channel, void* stream, int32_t* seg_id);

/* Template bank from chirp parameters (Sec. 3: one-second chirps over the
 * (f, fdot) plane).  Row k is
 *     w_k[m] = T(m) sin(2 pi (f0 t_m + fdot t_m^2 / 2)),  t_m = m / fs,
 * m < L = round(tau fs), T a cosine taper over the fraction `taper_frac`
 * (half at each end), scaled to unit L2 norm; synthesised on the device with
 * an exact fixed-point phase and FP64 sin/taper/norm, stored as FP32.
 * `params` is a HOST array of `count` chirps.  Errors: EINVAL, EBUDGET,
 * ENOMEM, ECUDA. */
BEGE_API int bege_define_bank(bege_ctx* ctx, const bege_chirp* params, int64_t count, double tau,
                              double taper_frac, void* stream, int32_t* bank_id);

/* As bege_define_bank, with the time-symmetric chirps of the paper's banks
 * (Fig. 2 caption: each chirp superposed with itself backward in time, for
 * ascending and descending signals alike):
 *     w_k[m] = T(m) (sin(2 pi phi(t_m)) + sin(2 pi phi(t_{L-1-m}))),
 * phi(t) = f0 t + fdot t^2 / 2, scaled to unit L2 norm (all zeros if the
 * two halves cancel).  Errors: as bege_define_bank. */
BEGE_API int bege_define_bank_symmetric(bege_ctx* ctx, const bege_chirp* params, int64_t count,
                                        double tau, double taper_frac, void* stream,
                                        int32_t* bank_id);

/* Template bank from explicit samples: `samples` is a HOST array of
 * count x length FP32 values, row-major, used as given (no normalisation). */
BEGE_API int bege_define_bank_samples(bege_ctx* ctx, const float* samples, int64_t count,
                                      int64_t length, void* stream, int32_t* bank_id);

/* Correlate segment `seg_id` with bank rows [k_begin, k_end) and keep the
 * tails |rho_k[n]| > kappa sigma_k (Eq. 3S, Eq. PT, Eq. tail).  Asynchronous:
 * enqueues the work on `stream` and returns a job handle at once.  The bank's
 * L must not exceed the segment's N.  kappa must be finite and >= 0.
 * Errors: EINVAL, EBUDGET, ENOMEM, ECUDA. */
BEGE_API int bege_correlate(bege_ctx* ctx, int32_t seg_id, int32_t bank_id, int64_t k_begin,
                            int64_t k_end, float kappa, void* stream, int32_t* job_id);

/* Wait for job `job_id` and copy its tail records to HOST `out` (capacity
 * records).  *n_total receives the true number of tails; *n_written the
 * number copied = min(n_total, capacity, device tail capacity).  Records are
 * in device completion order (bege_sort_tails orders them).  Returns BEGE_EOVERFLOW (with the
 * counts filled in) when n_total exceeds what was copied, BEGE_ETIMEDOUT if
 * a bounded wait inside the kernel gave up (the job's results are invalid). */
BEGE_API int bege_fetch_tails(bege_ctx* ctx, int32_t job_id, bege_tail* out, int64_t capacity,
                              int64_t* n_written, int64_t* n_total);

/* Several segments of one length against the same template range (Sec. 3.2:
 * a template's transform serves a block of segments, steps ii-iv): per
 * template the forward transform runs once, then each segment's product,
 * inverse transform, sigma and tails follow with the arithmetic of
 * bege_correlate, so every result is bitwise the single search's.  Writes
 * one job handle per segment to job_ids[n_seg] (fetch, sigma and release as
 * usual; the jobs finish together).  1 <= n_seg <= 8; FP32 contexts only;
 * N >= 2^14 and templates of at most 4096 samples.  Extra device memory
 * while the jobs live: 64 KB per resident CTA (about 20 MB).
 * Errors: EINVAL, EBUDGET, ENOMEM, ECUDA. */
BEGE_API int bege_correlate_multi(bege_ctx* ctx, const int32_t* seg_ids, int32_t n_seg,
                                  int32_t bank_id, int64_t k_begin, int64_t k_end, float kappa,
                                  void* stream, int32_t* job_ids);

/* As bege_correlate, and the job also projects its hits onto one array of
 * the segment's N lags, keeping per lag the largest normalised value over
 * the bank (Eq. Ak over the templates, gathered as in Eq. Aa / Eq. BA with
 * the maximal value kept per sample): among templates k with
 * rho_k[n] > kappa sigma_k (signed, as Eq. C; strict, as Eq. tail), the
 * largest rho_k[n] / sigma_k and its template.  Raised with a 64-bit atomic
 * maximum on (value bits, complemented template), so equal values keep the
 * smaller template and the result does not depend on timing (the paper's
 * post-callback race, Sec. 3.3, does not arise).  All-hit records are still
 * collected as for bege_correlate.  Extra device memory: 8 N bytes.
 * Errors: as bege_correlate. */
BEGE_API int bege_correlate_max(bege_ctx* ctx, int32_t seg_id, int32_t bank_id, int64_t k_begin,
                                int64_t k_end, float kappa, void* stream, int32_t* job_id);

/* As bege_correlate, with the tails restricted to a finite band (Sec. 5,
 * for deep searches with a low threshold): records (k, n, rho_k[n]) with
 * kappa_lo sigma_k < |rho_k[n]| < kappa_hi sigma_k.  Fetch them with
 * bege_fetch_tails.  Errors: as bege_correlate; EINVAL unless
 * 0 <= kappa_lo < kappa_hi, both finite. */
BEGE_API int bege_correlate_band(bege_ctx* ctx, int32_t seg_id, int32_t bank_id, int64_t k_begin,
                                 int64_t k_end, float kappa_lo, float kappa_hi, void* stream,
                                 int32_t* job_id);

/* Options of bege_correlate_ex; each field off (zero) gives bege_correlate. */
typedef struct {
  float kappa;     /* tails |rho_k[n]| > kappa sigma_k (Eq. tail), finite, >= 0 */
  float kappa_hi;  /* 0 = no upper end; else also |rho_k[n]| < kappa_hi sigma_k (Sec. 5),
                      finite and > kappa */
  int32_t linear;  /* 1 = overlap-save: tails only at lags n <= N - L, where the
                      length-L template window y[n .. n+L-1] does not wrap, so
                      the circular correlation equals the linear one (Eq. A1 over
                      the segment alone); sigma_k stays the Parseval value over
                      all N lags.  0 = all N circular lags. */
  int32_t project; /* 1 = also keep the per-lag maximum of bege_correlate_max, over
                      the tails the other options keep */
} bege_search_opts;

/* The search with the tail epilogue's options combined: a band, the
 * overlap-save lag mask and the per-lag maximum (host struct, read during
 * the call only).  Records via bege_fetch_tails; a projection via
 * bege_fetch_max.  Errors: as bege_correlate; EINVAL for an invalid field
 * (linear and project must be 0 or 1). */
BEGE_API int bege_correlate_ex(bege_ctx* ctx, int32_t seg_id, int32_t bank_id, int64_t k_begin,
                               int64_t k_end, const bege_search_opts* opts, void* stream,
                               int32_t* job_id);

/* Wait for a bege_correlate_max job and copy its projection to HOST arrays
 * of n = N entries: snr[n] = rho / sigma of the kept hit and tmpl[n] its
 * template index, or snr 0 and tmpl -1 where no template passes.
 * Errors: EINVAL (not such a job, n != N), ETIMEDOUT, ECUDA. */
BEGE_API int bege_fetch_max(bege_ctx* ctx, int32_t job_id, float* snr, int32_t* tmpl, int64_t n);

/* Sort n HOST tail records in place by (template, lag), the order in which
 * Sec. 3.3 gathers tails per template.  Host only (no context, no device);
 * (template, lag) pairs are unique within one job, so the order is total.
 * Errors: EINVAL (NULL records with n > 0, n < 0). */
BEGE_API int bege_sort_tails(bege_tail* recs, int64_t n);

/* Wait for job `job_id` and report the device time in milliseconds of its
 * correlate kernel alone (CUDA events recorded on the job's stream right
 * before and after the launch).  Used for roofline accounting. */
BEGE_API int bege_job_kernel_ms(bege_ctx* ctx, int32_t job_id, float* ms);

/* Non-blocking: BEGE_OK if the job has finished, BEGE_ENOTREADY if not. */
BEGE_API int bege_query(bege_ctx* ctx, int32_t job_id);

/* Wait for job `job_id` and copy sigma_k (Eq. PT) for its rows to HOST `out`;
 * `count` must equal k_end - k_begin of the job. */
BEGE_API int bege_get_sigma(bege_ctx* ctx, int32_t job_id, float* out, int64_t count);

/* Debug: the full correlation rho_k[0..N-1] for rows [k_begin, k_end) into
 * HOST `out` ((k_end - k_begin) x N floats, row-major).  Same kernel as
 * bege_correlate; synchronous on `stream`. */
BEGE_API int bege_dump_correlation(bege_ctx* ctx, int32_t seg_id, int32_t bank_id, int64_t k_begin,
                                   int64_t k_end, float* out, void* stream);

/* Debug: the segment spectrum D_j, j = 0..N/2, as interleaved (re, im) FP32
 * into HOST `out` (N + 2 floats). */
BEGE_API int bege_get_segment_spectrum(bege_ctx* ctx, int32_t seg_id, float* out);

/* Debug: bank rows [k_begin, k_end) as FP32 into HOST `out` ((k_end-k_begin) x L). */
BEGE_API int bege_get_bank_samples(bege_ctx* ctx, int32_t bank_id, int64_t k_begin, int64_t k_end,
                                   float* out);

/* Segment length N / bank template length L of a handle (0 if unknown). */
BEGE_API int64_t bege_segment_length(bege_ctx* ctx, int32_t seg_id);
BEGE_API int64_t bege_bank_length(bege_ctx* ctx, int32_t bank_id);

/* Device bytes currently owned by the context. */
BEGE_API uint64_t bege_device_bytes(const bege_ctx* ctx);

/* Launch shapes of the correlate kernel for segment length n.  A shape is
 * (columns per CTA, threads per CTA); the cluster holds (n / 8192) / columns
 * CTAs.  bege_list_configs writes up to `max` pairs into `out` as
 * {nc0, threads0, nc1, threads1, ...} and the number available into *count. */
BEGE_API int bege_list_configs(bege_ctx* ctx, int64_t n, int32_t* out, int32_t max, int32_t* count);

/* Select the launch shape used by later bege_correlate calls for length n.
 * EINVAL if the shape is not one of bege_list_configs. */
BEGE_API int bege_set_config(bege_ctx* ctx, int64_t n, int32_t nc, int32_t threads);

/* The launch shape currently used for length n (the default if none set). */
BEGE_API int bege_get_config(bege_ctx* ctx, int64_t n, int32_t* nc, int32_t* threads);

/* Autotuner (batching form): time every launch shape for the segment's n on
 * bank rows [k_begin, k_end) of `bank_id` (`reps` timed runs each after one
 * warm-up, median of the kernel time), select the fastest for that n and
 * report its median time in *best_ms.  Synchronous on `stream`; the results
 * of the timing runs are discarded. */
BEGE_API int bege_autotune(bege_ctx* ctx, int32_t seg_id, int32_t bank_id, int64_t k_begin,
                           int64_t k_end, int32_t reps, void* stream, float* best_ms);

/* ---- Batching form ------------------------------------------------------
 * Many segments of different lengths, each against its own bank range, in
 * one persistent kernel launch captured with the batched segment-spectrum
 * kernel in a CUDA graph (Sec. 3.2: batch mode over blocks of segments and
 * groups of templates).  n must be one of 2^14, 2^15, 2^16, 2^17 and the
 * bank's template length at most 4096 samples (tau <= 1 s at 4096 Hz).
 * Batches always run the FP32 path, whatever the context's precision. */
typedef struct {
  const float* strain;   /* HOST pointer to n FP32 samples (copied at creation) */
  int64_t n;
  int32_t bank_id;
  int32_t reserved;      /* must be 0 */
  int64_t k_begin;       /* bank rows [k_begin, k_end) */
  int64_t k_end;
  float kappa;
  float reserved2;       /* must be 0 */
} bege_batch_entry;

/* Create a batch: copies the strains to the device, allocates per-entry
 * sigma and tail buffers (`tail_capacity` records per entry, 0 = the
 * context default) and captures the graph.  *batch_id receives the handle
 * (released with bege_release).  Errors: EINVAL, EBUDGET, ENOMEM, ECUDA. */
BEGE_API int bege_batch_create(bege_ctx* ctx, const bege_batch_entry* entries, int32_t count,
                               uint64_t tail_capacity, void* stream, int32_t* batch_id);

/* Launch the batch's graph on `stream` (asynchronous): segment spectra of
 * every entry, then all correlations.  Each run overwrites the previous
 * run's results. */
BEGE_API int bege_batch_run(bege_ctx* ctx, int32_t batch_id, void* stream);

/* Wait for the last run and report its device time (CUDA events around the
 * graph launch) in milliseconds. */
BEGE_API int bege_batch_elapsed_ms(bege_ctx* ctx, int32_t batch_id, float* ms);

/* Wait for the last run and copy entry `entry`'s tails / sigma to HOST
 * memory; same conventions as bege_fetch_tails / bege_get_sigma. */
BEGE_API int bege_batch_fetch_tails(bege_ctx* ctx, int32_t batch_id, int32_t entry, bege_tail* out,
                                    int64_t capacity, int64_t* n_written, int64_t* n_total);
BEGE_API int bege_batch_get_sigma(bege_ctx* ctx, int32_t batch_id, int32_t entry, float* out,
                                  int64_t count);

/* Execution plan of a batch.  plan 0: the persistent kernel (clusters of 8
 * CTAs taking work items of `chunk` templates from a queue; `order` 0 =
 * longest segments first, 1 = entries interleaved); plan 1: one launch per
 * entry with the per-length launch shape of bege_set_config. */
BEGE_API int bege_batch_set_plan(bege_ctx* ctx, int32_t batch_id, int32_t plan, int64_t chunk,
                                 int32_t order);
BEGE_API int bege_batch_get_plan(bege_ctx* ctx, int32_t batch_id, int32_t* plan, int64_t* chunk,
                                 int32_t* order);

/* Autotuner of the batching form: times every plan (plan 0 over chunks of
 * 64..2048 templates and both orders, plan 1 with the current per-length
 * shapes) with `reps` runs each after one warm-up, keeps the fastest (the
 * per-segment plan only if more than 1% faster than the best persistent one)
 * and reports its median time in *best_ms.  Synchronous on `stream`. */
BEGE_API int bege_batch_autotune(bege_ctx* ctx, int32_t batch_id, int32_t reps, void* stream,
                                 float* best_ms);

/* ---- Serving form ----------------------------------------------------------
 * A request loop with continuous batching over one resident bank (the paper's
 * low-latency use, Sec. 1, Sec. 6).  Requests are strain segments submitted
 * from any number of detector channels as they arrive.  A server thread
 * admits them in arrival order while the device bytes its requests hold stay
 * within the budget, loads each admitted segment's spectrum, cuts its
 * correlation with the whole bank into slices of `slice_templates` rows and
 * keeps up to `streams` slices in flight on separate CUDA streams, taking
 * slices round-robin from every admitted request: a request that arrives
 * while others run starts within one slice and its work overlaps theirs on
 * the device.  Every template sees the same kernel arithmetic whatever else
 * runs, so results do not depend on the mix.  When a request's last slice
 * completes its tails and sigma are copied to host memory and its device
 * memory is released.  bege_destroy stops the context's servers first. */
typedef struct {
  int32_t bank_id;
  int32_t streams;            /* slices in flight at once; 0 = 3                  */
  int64_t slice_templates;    /* bank rows per slice; 0 = 65536                   */
  float kappa;                /* threshold for every request (finite, >= 0)       */
  float reserved;             /* must be 0                                        */
  uint64_t hbm_budget_bytes;  /* device bytes the admitted requests may hold
                                 (segment spectra and slice buffers); 0 = only the
                                 context's own budget applies                     */
} bege_serve_config;

typedef struct {
  int32_t state;      /* 0 queued, 1 admitted (running), 2 done, 3 failed       */
  int32_t channel;    /* as submitted                                           */
  int64_t n;          /* segment length                                         */
  int64_t n_tails;    /* tail count (valid when done)                           */
  double t_submit;    /* host monotonic clock, seconds: submitted               */
  double t_admit;     /*   admitted                                             */
  double t_done;      /*   results on the host                                  */
  double gpu_ms;      /* summed kernel time of the request's slices             */
} bege_serve_info;

/* Start a server thread on `cfg->bank_id`.  *server_id receives the handle. */
BEGE_API int bege_serve_create(bege_ctx* ctx, const bege_serve_config* cfg, int32_t* server_id);

/* Queue a request: `strain` is a HOST array of n FP32 samples (copied before
 * the call returns; n a power of two in [2^10, 2^17], at least the bank's
 * template length).  *request_id receives a per-server id. */
BEGE_API int bege_serve_submit(bege_ctx* ctx, int32_t server_id, const float* strain, int64_t n,
                               int32_t channel, int64_t* request_id);

/* Block until the request is done (BEGE_OK), failed (its error), or
 * `timeout_ms` passes (BEGE_ETIMEDOUT; < 0 waits without limit). */
BEGE_API int bege_serve_wait(bege_ctx* ctx, int32_t server_id, int64_t request_id,
                             int32_t timeout_ms);

/* State and timings of a request. */
BEGE_API int bege_serve_info_get(bege_ctx* ctx, int32_t server_id, int64_t request_id,
                                 bege_serve_info* info);

/* Results of a done request, from host memory: tails (same conventions as
 * bege_fetch_tails) and sigma of every bank row (`count` = bank size). */
BEGE_API int bege_serve_fetch_tails(bege_ctx* ctx, int32_t server_id, int64_t request_id,
                                    bege_tail* out, int64_t capacity, int64_t* n_written,
                                    int64_t* n_total);
BEGE_API int bege_serve_get_sigma(bege_ctx* ctx, int32_t server_id, int64_t request_id, float* out,
                                  int64_t count);

/* Drop a done request's host-side results. */
BEGE_API int bege_serve_forget(bege_ctx* ctx, int32_t server_id, int64_t request_id);

/* Stop the server after the work in flight completes; queued requests that
 * were not admitted are dropped. */
BEGE_API int bege_serve_destroy(bege_ctx* ctx, int32_t server_id);

/* ---- Search without device allocation -----------------------------------
 * The paper has no counterpart of this call.  It serves callers that may not
 * allocate device memory themselves or have a library do it for them: for
 * example a program whose device memory all belongs to one pool it manages
 * (a framework's caching allocator, or an arena reserved at start-up so that
 * a latency-critical loop never calls cudaMalloc/cudaFree).  It runs the
 * whole search of one segment -- spectrum, correlation with bank rows
 * [k_begin, k_end), sigma and tails -- using only the caller's buffers plus
 * one fixed scratch array inside the library (about 1.05 MiB of device
 * memory per GPU, held from library load until process exit).  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 *   strain_dev      DEVICE, n FP32 samples, 8-byte aligned
 *   n               power of two in [2^10, 2^16] (the scratch holds at most
 *                   2^16 samples; larger n is rejected with BEGE_EINVAL)
 *   bank_dev        DEVICE, rows of `ld` FP32 samples, 32-byte aligned; row k
 *                   holds template k, zero beyond its length
 *   ld              row stride in floats, a multiple of 8, at most n
 *   kappa           finite, >= 0
 *   sigma_dev       DEVICE, k_end - k_begin FP32: sigma of row k at k - k_begin,
 *                   4-byte aligned
 *   tails_dev       DEVICE, tail_capacity records (bege_tail), 4-byte aligned
 *   tail_count_dev  DEVICE, one unsigned 64-bit count, 8-byte aligned; set to
 *                   zero by the call, then to the true number of tails (only
 *                   the first tail_capacity records are stored)
 *   stream          cudaStream_t as void*; the call only enqueues work
 *
 * The first call on a device looks up the scratch array's device address
 * (with that device current), so the first call on each device should come
 * before any stream capture.  Every call recomputes the twiddle tables for
 * its n in the scratch array on `stream`, ahead of its other kernels.  The scratch array keeps the last
 * call's contents and is shared by all calls on a device: calls whose work
 * overlaps on the GPU race and must be serialised by the caller.  Errors:
 * EINVAL (sizes, alignment, NULL), ECUDA. */
BEGE_API int bege_search_noalloc(const float* strain_dev, int64_t n, const float* bank_dev,
                                 int64_t ld, int64_t k_begin, int64_t k_end, float kappa,
                                 float* sigma_dev, bege_tail* tails_dev,
                                 uint64_t tail_capacity, unsigned long long* tail_count_dev,
                                 void* stream);

/* Release a segment, bank, job or batch handle and its device memory (job
 * buffers return to the context's pool).  Errors: EINVAL for an unknown
 * handle. */
BEGE_API int bege_release(bege_ctx* ctx, int32_t handle);

/* Message of the last error on the calling thread ("" if none).  ctx may be
 * NULL. */
BEGE_API const char* bege_last_error(const bege_ctx* ctx);

/* Library version string. */
BEGE_API const char* bege_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BEGE_H */
