/*
 * fc.h -- C ABI of the GB300 Feldman-Cousins grid-fit library (libfc.so).
 *
 * The library computes, for true grid points p and universes u, the
 * Feldman-Cousins statistic of the paper's §2 procedure and Algorithm 1:
 *
 *   1. s = S(p), the true point's spectrum;
 *   2. fake data d = Poisson(max(0, s + L_p z)), L_p = chol(diag(s) F diag(s)),
 *      z ~ N(0, I) from Philox4x32-10, in the full-bin space, then collapsed;
 *   3. chi2_g = (s_g - d)^T A (s_g - d) for every grid point g (Eq. 1 with
 *      the inverse covariance A = M^-1; Algorithm 2's residual form);
 *   4. q_min = the first grid index attaining the minimum (strict "<");
 *   5. rebuild M = C [diag(s_qmin) F diag(s_qmin) + diag(s_qmin)] C^T at q_min,
 *      invert it and rescan, until q_min repeats or max_iter scans are done;
 *   6. dchi2 = chi2_p - chi2_min, both under the last scan's A.
 *
 * Conventions for every entry point:
 *   - Return value: FC_OK (0) or a negative fc_status; nothing aborts, throws
 *     across the ABI or traps on the device.  fc_last_error() gives a message
 *     for the calling thread's last non-OK status.
 *   - Matrices and spectra are row-major, float64 unless stated.
 *   - Pointer arguments may be host or device memory (detected per call);
 *     the library copies inputs it keeps and never frees caller memory.
 *   - Output arrays belong to the caller and are written only on success.
 *   - Work runs on the context's CUDA stream; synchronous entry points return
 *     after the stream has finished the work.
 *   - A context is not thread-safe, except fc_submit / fc_poll / fc_cancel,
 *     which may be called from any thread.
 */
#ifndef FC_H_
#define FC_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FC_API __attribute__((visibility("default")))
#else
#define FC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fc_ctx fc_ctx;

typedef enum {
    FC_OK = 0,
    FC_PENDING = 1,          /* fc_poll: job still queued or running           */
    FC_ERR_ARG = -1,         /* invalid argument (sizes, ids, pointers, NaN)   */
    FC_ERR_NOT_SPD = -2,     /* a covariance had a non-positive Cholesky pivot */
    FC_ERR_BUDGET = -3,      /* would exceed the context's device-memory budget*/
    FC_ERR_CUDA = -4,        /* a CUDA runtime call failed                     */
    FC_ERR_TIMEOUT = -5,     /* a bounded device-side wait ran out             */
    FC_ERR_CANCELLED = -6,   /* job cancelled before it finished               */
    FC_ERR_NOT_FOUND = -7,   /* unknown grid id or ticket                      */
    FC_ERR_STATE = -8        /* call not valid in the current state            */
} fc_status;

enum { FC_PREC_FP64 = 0,     /* plain path: every step in binary64 on CUDA cores        */
       FC_PREC_MIXED = 1 };  /* BF16 tensor-core screen (tcgen05) with a certified
                                bound; candidates rescored in residual form in
                                double-float (a value = two binary32, about 48
                                significant bits, on the FP32 pipe -- not binary64);
                                covariances, Cholesky and inverse in binary64 */
enum { FC_FLUCT_POISSON_SYS = 0,  /* d = Poisson(max(0, s + L z)), L = chol(diag(s)F diag(s)) */
       FC_FLUCT_GAUSS = 1 };      /* test mode: d = s + L z, L = chol(diag(s)F diag(s)+diag(s)) */
enum { FC_COV_ITERATE = 0,   /* §2 step 5: refit the covariance at q_min until stable   */
       FC_COV_FIXED = 1,     /* Algorithm 1 as printed: A = M(p)^-1, one scan           */
       FC_COV_IDENTITY = 2 };/* test mode: A = I, one scan (nearest neighbour)          */

typedef struct {
    int32_t max_iter;   /* scans per universe including the first, >= 1 (default 5)  */
    int32_t precision;  /* FC_PREC_*  (default FC_PREC_MIXED)                        */
    int32_t top_k;      /* candidates kept by the mixed screen, 1..16 (default 8)    */
    int32_t fluct;      /* FC_FLUCT_* (default FC_FLUCT_POISSON_SYS)                 */
    int32_t cov;        /* FC_COV_*   (default FC_COV_ITERATE)                       */
} fc_opts;

/* Kernel choices of one grid.  They change speed only: every choice gives
 * the same dchi2, best fits and scan counts (the screen's decisions are
 * certified and resolved in double-float residual form).  fc_autotune picks them by timing. */
enum { FC_QVEC_AUTO = 0,     /* tensor cores (the faster kernel at every N_fit)      */
       FC_QVEC_SIMT = 1,     /* q_g = s~^T A s~ in binary32, A in shared memory    */
       FC_QVEC_TC = 2 };     /* q_g = |W s~|^2 on tcgen05 (bf16 hi/lo), K <= 128  */

enum { FC_ROUND_AUTO = 0,    /* LIST (the faster policy on every grid measured)             */
       FC_ROUND_TOPK = 1,    /* rounds: top-k, top-16, list, exact-size lists               */
       FC_ROUND_LIST = 2 };  /* rounds: top-k, list, exact-size lists (no top-16 round)     */

typedef struct {
    int32_t qvec;           /* FC_QVEC_*                                            */
    int32_t screen_stages;  /* screen pipeline depth, 0 = built-in choice (2..8)    */
    int32_t screen_ybuf;    /* A-image buffers of the screen, 0 = built-in (1 or 2) */
    int32_t cache_slots;    /* covariance-cache slots at most, 0 = as memory allows;
                               one scan needs a slot per distinct covariance index */
    int32_t first_round;    /* FC_ROUND_*                                           */
    int32_t slot_rows;      /* rows of a screen tile given to one covariance slot:
                               32 (a TMEM lane quadrant; a tile serves up to four
                               covariances) or 128 (a whole tile); 0 = built-in 32 */
} fc_tuning;

/* Counters and stage timings of the last synchronous call on a context.
 * Stage times are CUDA-event intervals on the context stream around each
 * stage's kernels, summed over scans (milliseconds). */
typedef struct {
    int64_t universes;        /* universes fitted                                     */
    int64_t scans;            /* universe-scans performed (sum of nscans)             */
    int64_t chi2_evals;       /* universe-scans x G: chi2 values the scans decided on */
    int64_t distinct_cov;     /* covariances built and inverted                       */
    int64_t screened;         /* universe-scans decided by the tensor-core screen     */
    int64_t rescored;         /* universe-scans whose candidates needed double-float
                                 residual rescoring                                  */
    int64_t rescreened;       /* universe-scans whose first certificate failed -> second screen round */
    int64_t fallback;         /* universe-scans no certified round decided -> exact
                                 residual scan over every g (double-float)           */
    int64_t kernel_launches;  /* CUDA kernels launched by the call                    */
    int64_t screen_launches;  /* launches of the tensor-core screen kernel             */
    double  screen_flops;     /* algorithmic flops of those launches: 2 N_fit per eval */
    double  ms_fake, ms_cov, ms_prep, ms_screen, ms_rescore, ms_fallback, ms_scan64, ms_finish, ms_total;
    int64_t evicted;          /* covariance-cache slots handed to another grid index  */
    int64_t cache_slots;      /* covariance-cache slots allocated for the grid        */
    int64_t max_distinct_cov; /* most distinct covariance indices one scan needed     */
    int64_t scan_waves;       /* cache-sized groups run by scans that needed more     */
    int64_t big_listed;       /* universe-scans sent to the exact-size list round     */
    int64_t screen_tiles;     /* 128-row universe tiles screened (all launches)       */
    int64_t screen_rows;      /* universe rows in them (fill = rows / (128 tiles))    */
    int64_t deferred;         /* serving: admission turns a queued job waited for memory
                                 (the budget held by running jobs)                   */
    int64_t device_bytes;     /* device memory the context holds now (all grids,
                                 caches, lanes and scratch)                          */
    int64_t residuals;        /* mixed path: residual-form chi2 evaluated in
                                 double-float (rescoring, chi2_p, chi2_min)          */
} fc_stats;

/* Fill *o with the defaults listed above. */
FC_API void fc_default_opts(fc_opts* o);

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context may hold (0 = no cap).  cuda_stream is a cudaStream_t to
 * run on (NULL = the context creates its own non-blocking stream).
 * Errors: FC_ERR_ARG (out NULL), FC_ERR_CUDA (no such device / no memory). */
FC_API fc_status fc_create(fc_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream);

/* Destroy a context and free its device memory.  Waits for queued jobs. */
FC_API fc_status fc_destroy(fc_ctx* ctx);

/* Load the grid spectra (the paper's S(q) for every q in the linearised grid
 * of §2).  S: G x N_full float64 row-major, finite and >= 0 (host or device).
 * collapse: N_full int32 entries mapping full bin -> fit bin in [0, N_fit), or
 * NULL for the identity (then N_fit must equal N_full).  1 <= N_full, N_fit <= 200.
 * The spectra are kept resident (float64 plus the BF16 copy of the screen).
 * On success *grid_id receives the new grid's id.
 * Errors: FC_ERR_ARG, FC_ERR_BUDGET, FC_ERR_CUDA. */
FC_API fc_status fc_load_grid(fc_ctx* ctx, const double* S, int64_t G, int32_t N_full,
                       const int32_t* collapse, int32_t N_fit, int32_t* grid_id);

/* Grid spectra generated on the device from an oscillation shape model, so a
 * large grid never exists on the host (the paper recomputes S(q) from its
 * model, §3 and Table 2; here the model is evaluated once and the spectra stay
 * resident).  The grid has D axes; grid point p is the row-major index over
 * them (axis 0 slowest) and the model's spectrum is
 *     s_i(p) = b_i + sum_t amp_t(p) sin^2(1.27 dm2_t(p) L_i / E_i) f_ti,
 * the terms added to b_i in order t = 0, 1, ..., where term t reads its
 * amplitude from axis amp_axis[t] and its dm2 from axis dm2_axis[t] (e.g. a
 * two-flavour model: D = 2, axes dm2 and sin^2 2theta, one term).
 * Everything after the spectra is fc_load_grid's (collapse, N_fit, the
 * resident arrays).  All model arrays are host memory. */
typedef struct {
    int32_t D;                  /* axes, 1..8 */
    const int32_t* axis_len;    /* [D] points per axis; G = their product */
    const double* axis_values;  /* the axes' values, axis 0 first: sum(axis_len) entries */
    int32_t n_terms;            /* oscillation terms, 1..4 */
    const int32_t* amp_axis;    /* [n_terms] axis of each term's amplitude */
    const int32_t* dm2_axis;    /* [n_terms] axis of each term's dm2 (eV^2) */
    const double* b;            /* [N_full] background */
    const double* f;            /* [n_terms][N_full] each term's signal shape */
    const double* L;            /* [N_full] baseline of each bin (m) */
    const double* E;            /* [N_full] energy of each bin (GeV), > 0 */
} fc_osc_model;

/* Errors: FC_ERR_ARG (sizes, axes, E <= 0, a spectrum not finite or < 0, and
 * fc_load_grid's), FC_ERR_BUDGET, FC_ERR_CUDA. */
FC_API fc_status fc_load_grid_osc(fc_ctx* ctx, const fc_osc_model* model, int32_t N_full, const int32_t* collapse,
                                  int32_t N_fit, int32_t* grid_id);

/* fc_load_grid_osc with flags.  FC_GRID_RECOMPUTE: keep no spectra.  As in
 * the paper's own kernels (§3, Table 2: S(q) recomputed from the physics model
 * for every evaluation, no caching), every spectrum row a kernel needs (a
 * covariance M(q), a true point's fake data, a rescored candidate, a probe, a
 * plain-path scan tile) is evaluated from the model where it is read.  The
 * sine of each term depends only on the value of its dm2 axis and the bin, so
 * it is tabulated once ((sum of those axis lengths) x N_full values); an
 * element then costs three multiplies and an add per term.  What stays
 * resident is the model, the centre, and the screen's bf16 hi/lo image of
 * s - centre with its per-point norms (4 K + 16 bytes per grid point instead
 * of 8 N_full + 28 N_fit + 4 K + 16).  A grid gives bit-identical results
 * stored or recomputed (both are filled by the same evaluation).  Other
 * flags: FC_ERR_ARG. */
enum { FC_GRID_RECOMPUTE = 1 };
FC_API fc_status fc_load_grid_osc_ex(fc_ctx* ctx, const fc_osc_model* model, int32_t N_full,
                                     const int32_t* collapse, int32_t N_fit, uint32_t flags, int32_t* grid_id);

/* Set the fractional systematic covariance F (N_full x N_full float64,
 * symmetric) of a loaded grid.  The systematic covariance of spectrum s is
 * diag(s) F diag(s); the statistical part is diag(s).  Invalidates the grid's
 * covariance cache.  Errors: FC_ERR_ARG, FC_ERR_NOT_FOUND. */
FC_API fc_status fc_set_frac_cov(fc_ctx* ctx, int32_t grid_id, const double* F, int32_t N_full);

/* Remove a grid and its caches.  Errors: FC_ERR_NOT_FOUND, FC_ERR_STATE (a
 * queued job still uses it). */
FC_API fc_status fc_unload_grid(fc_ctx* ctx, int32_t grid_id);

/* Feldman-Cousins pass for P true points x U universes (Algorithm 1 plus the
 * covariance refit of §2).  ps: P int64 grid indices in [0, G).  Outputs, laid
 * out [P][U] row-major: dchi2 (float64, required), bestfit (int64 final
 * best-fit grid index, nullable), nscans (int8 scans performed, nullable).
 * opts NULL = defaults.  Results depend only on (grid, F, seed, p, u, opts):
 * not on P, on the order of ps, or on other jobs sharing the device.
 * Errors: FC_ERR_ARG, FC_ERR_NOT_FOUND, FC_ERR_STATE (F not set),
 * FC_ERR_NOT_SPD, FC_ERR_BUDGET, FC_ERR_CUDA, FC_ERR_TIMEOUT. */
FC_API fc_status fc_run_points(fc_ctx* ctx, int32_t grid_id, const int64_t* ps, int32_t P, uint64_t seed,
                        int32_t U, const fc_opts* opts, double* dchi2, int64_t* bestfit, int8_t* nscans);

/* fc_run_points for one true point p (Algorithm 1's buildDeltaChi2 signature:
 * point, covariance via the grid's F, spectra, N_univ). */
FC_API fc_status fc_run_point(fc_ctx* ctx, int32_t grid_id, int64_t p, uint64_t seed, int32_t U,
                       const fc_opts* opts, double* dchi2, int64_t* bestfit, int8_t* nscans);

/* Fake data only (§2 step 2): d [P][U][N_fit] float32 (integer counts in the
 * Poisson mode), drawn exactly as fc_run_points draws them.  fluct: FC_FLUCT_*.
 * Errors as fc_run_points. */
FC_API fc_status fc_fake_data(fc_ctx* ctx, int32_t grid_id, const int64_t* ps, int32_t P, uint64_t seed,
                       int32_t U, int32_t fluct, float* d);

/* Fit-space inverse covariance A(q) = M(q)^-1 (N_fit x N_fit float64) and the
 * Cholesky factor L_p of the systematic covariance diag(s_p) F diag(s_p)
 * (N_full x N_full float64, lower, upper part zero) as the library computes
 * them (§2 step 5; step 2).  Either output may be NULL.  Errors as above. */
FC_API fc_status fc_covariance(fc_ctx* ctx, int32_t grid_id, int64_t q, double* A, double* L_sys);

/* One scan (§2 steps 3-4) of caller data against the grid under A(q_cov[u]):
 * d [U][N_fit] float32, q_cov [U] int64.  Outputs [U]: best (int64 first
 * index of the minimum), chi2_min (float64, residual form).  precision selects
 * the plain binary64 scan or the tensor-core screen with certified double-float
 * rescoring.  Errors as above. */
FC_API fc_status fc_scan(fc_ctx* ctx, int32_t grid_id, const float* d, const int64_t* q_cov, int32_t U,
                  int32_t precision, int32_t top_k, int64_t* best, double* chi2_min);

/* Per-row quantiles (linear interpolation between order statistics, numpy's
 * default): x [rows][n] float64, probs [nq] in [0,1], out [rows][nq].  Used
 * for the critical values of Fig. 1.  Errors: FC_ERR_ARG, FC_ERR_CUDA. */
FC_API fc_status fc_quantiles(fc_ctx* ctx, const double* x, int32_t rows, int32_t n, const double* probs,
                       int32_t nq, double* out);

/* The observed data's dchi2 at grid points ps (the statistic the critical
 * values are for, §1 and Fig. 1): the per-universe procedure of §2 run on the
 * given fit-space data vector d [N_fit] (float32, host or device) in place of
 * fake data -- first covariance at ps[i], refit at the best fit until it
 * repeats, dchi2 = chi2_p - chi2_min under the last scan's A -- so that
 * dchi2[i] is comparable with the distribution of ps[i]'s universes.
 * Outputs [P]: dchi2 (required), bestfit, nscans (nullable).  opts.fluct is
 * not used.  Errors as fc_run_points. */
FC_API fc_status fc_data_dchi2(fc_ctx* ctx, int32_t grid_id, const float* d, const int64_t* ps, int32_t P,
                               const fc_opts* opts, double* dchi2, int64_t* bestfit, int8_t* nscans);

/* Feldman-Cousins acceptance (the use of the distributions, §1 / Fig. 1):
 * crit[i] = the cl-quantile (numpy "linear" rule) of dchi2_univ[i][0..U-1]
 * (point i's universes, float64 [P][U]) and accepted[i] = 1 when
 * dchi2_data[i] <= crit[i], else 0.  All arrays host or device; crit may be
 * NULL.  Errors: FC_ERR_ARG (cl outside [0, 1], U < 1, U > 16384), FC_ERR_CUDA. */
FC_API fc_status fc_fc_region(fc_ctx* ctx, const double* dchi2_univ, int32_t P, int32_t U, const double* dchi2_data,
                              double cl, double* crit, uint8_t* accepted);

/* Feldman-Cousins acceptance with an adaptive number of universes per point
 * (the future-work outlook of §5.1: spend universes where the decision is close).
 * For point ps[i] with data statistic dchi2_data[i] (e.g. from fc_data_dchi2):
 * F_i = #{universes u of ps[i] : dchi2_u < dchi2_data[i]} / U_i, the
 * empirical distribution of the point's dchi2 at the data's value, and
 * accepted[i] = 1 when F_i <= cl (dchi2_data[i] at or below the cl-quantile).
 * Round 0 runs U0 universes at every point (fc_run_points' procedure, key
 * seed); a point stays open while |F_i - cl| <= z sqrt(cl (1 - cl) / U_i) and
 * U_i < U_max, and round r runs as many new universes as an open point already
 * has (key seed + r, so the total doubles; the last round is capped at U_max).
 * Counting runs on the device; only P counts per round return to the host.
 * Inputs ps [P] int64, dchi2_data [P] float64 (host or device); outputs
 * accepted [P] uint8 (required), U_used [P] int32 and frac [P] float64 (F_i),
 * nullable, host or device.  Errors: FC_ERR_ARG (NULL, P < 0,
 * not 1 <= U0 <= U_max <= 2^20, cl outside [0, 1], z < 0, NaN data),
 * FC_ERR_NOT_FOUND, FC_ERR_STATE (F not set), and those of fc_run_points. */
FC_API fc_status fc_fc_region_adaptive(fc_ctx* ctx, int32_t grid_id, const int64_t* ps, int32_t P,
                                       const double* dchi2_data, double cl, int32_t U0, int32_t U_max, double z,
                                       uint64_t seed, const fc_opts* opts, uint8_t* accepted, int32_t* U_used,
                                       double* frac);

/* Asynchronous serving (continuous batching).  A job = fc_run_points'
 * arguments; output pointers must stay valid until fc_poll returns a final
 * status.  fc_submit admits the job when the context's memory budget allows
 * (FC_ERR_BUDGET if it can never fit) and returns a ticket; queued jobs run
 * interleaved with running ones on the device. */
typedef struct {
    int32_t grid_id;
    const int64_t* ps;
    int32_t P;
    uint64_t seed;
    int32_t U;
    fc_opts opts;
    double* dchi2;
    int64_t* bestfit;
    int8_t* nscans;
} fc_job;

FC_API fc_status fc_submit(fc_ctx* ctx, const fc_job* job, uint64_t* ticket);
/* FC_PENDING while the job runs; its final status once (then the ticket is
 * released: a second poll gives FC_ERR_NOT_FOUND).  *latency_ms (nullable)
 * receives submit-to-completion time for a finished job. */
FC_API fc_status fc_poll(fc_ctx* ctx, uint64_t ticket, double* latency_ms);
/* Cancel a queued or running job; it finishes with FC_ERR_CANCELLED. */
FC_API fc_status fc_cancel(fc_ctx* ctx, uint64_t ticket);

/* Fake data exactly as fc_fake_data produces it, for callers that cannot
 * allocate device memory when they need it: code running inside another
 * framework's allocator callback (which may not re-enter the allocator), or
 * services whose request paths must not allocate after start-up (an
 * allocation can stall on the device or fail under memory pressure).  The paper has no
 * counterpart; it is a deployment variant of §2 step 2.
 * All pointers are device memory: S [G][N_full] float64, collapse [N_full]
 * int32 (NULL = identity, then N_fit == N_full), F [N_full][N_full] float64,
 * ps [P] int64, output d [P][U][N_fit] float32.  Work runs on cuda_stream
 * (NULL = legacy default stream); the call returns after it finished.
 * No cudaMalloc / cudaFree: the only scratch is a 16 MiB file-scope device
 * array held by every device that loads the library until the process exits.
 * Limit: 256 + P * N_full^2 * 12 + P * N_full * 4 <= 16 MiB (e.g. P <= 172
 * points at N_full = 90); larger P gives FC_ERR_ARG -- split the points.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the array: calls whose work overlaps on the GPU
 * race.  The point indices and the collapse map (entries in [0, N_fit), no
 * fit bin left empty) are checked on the device before use.  Any P the
 * scratch limit admits is accepted (launches are split as needed).
 * Errors: FC_ERR_ARG (sizes, a point index or collapse entry out of range),
 * FC_ERR_NOT_SPD, FC_ERR_CUDA (a failed copy or launch) -- message in
 * fc_last_error(NULL). */
FC_API fc_status fc_fake_data_noalloc(const double* S, int64_t G, int32_t N_full, const int32_t* collapse,
                                      int32_t N_fit, const double* F, const int64_t* ps, int32_t P, uint64_t seed,
                                      int32_t U, int32_t fluct, float* d, void* cuda_stream);

/* Set / read the kernel choices of a loaded grid.  A choice the grid cannot
 * use (FC_QVEC_TC above K = 128, a screen depth that does not fit in shared
 * memory, slot_rows other than 0, 32, 128) gives FC_ERR_ARG.  Lowering cache_slots below the slots in use
 * clears the grid's covariance cache.  fc_autotune keeps cache_slots and first_round.
 * Errors: FC_ERR_ARG, FC_ERR_NOT_FOUND. */
FC_API fc_status fc_set_tuning(fc_ctx* ctx, int32_t grid_id, const fc_tuning* t);
FC_API fc_status fc_get_tuning(fc_ctx* ctx, int32_t grid_id, fc_tuning* t);

/* Time the candidate kernel choices of a grid on short synthetic runs (one
 * scan of fake universes at seeded grid points: 64 points x 256 universes for
 * the q-vector kernel and the screen pipeline, 1024 points x 8 universes --
 * sparse covariances, as after a refit -- for the tile shape slot_rows; the
 * grid's F must be set), keep the fastest, and return it in *out (nullable).  cache_path (nullable):
 * a text file of earlier results keyed by device, G, N_full, N_fit; a hit
 * skips the timing, a miss appends the new result.  The covariance cache is
 * cleared afterwards.  Errors: as fc_run_points. */
FC_API fc_status fc_autotune(fc_ctx* ctx, int32_t grid_id, const char* cache_path, fc_tuning* out);

/* Measured fma rates of the context's device (TFLOP/s, 2 flops per fma):
 * binary64 and binary32, each from a probe kernel of independent fma chains
 * with no memory traffic, best of three timed launches.  The denominators of
 * the plain path's roofline (binary64 pipe) and of the double-float
 * rescoring's (binary32 pipe).  Errors: FC_ERR_ARG, FC_ERR_CUDA. */
FC_API fc_status fc_measure_peaks(fc_ctx* ctx, double* fp64_tflops, double* fp32_tflops);

/* Test hook for failure detection without a GPU fault.  Every wait of the
 * tensor-core screen on a pipeline barrier is bounded; when one runs out the
 * kernel records a timeout, lets the copies it issued land, frees its tensor
 * memory and returns, and the call gives FC_ERR_TIMEOUT with the context still
 * usable.  wait_ns: limit of those waits on this context (0 = the built-in
 * 2 s; at most 2 s).  screen_stop_after: >= 0 makes the copy producer of every
 * screen CTA stop issuing after that many pipeline stages, so that the
 * consumers' waits run out; -1 (default) = off.  Errors: FC_ERR_ARG. */
FC_API fc_status fc_set_wait_test(fc_ctx* ctx, uint64_t wait_ns, int64_t screen_stop_after);

/* Which certified rounds decided the scans of each universe in the last
 * synchronous fit on this context (fc_run_points, fc_run_point, fc_scan,
 * fc_data_dchi2): out [n] uint8 (host or device), [P][U] order, n = that
 * call's universe count; each entry ORs the FC_DECIDED_* bit of every round
 * that decided one of the universe's scans.  A diagnostic for tests: which
 * round decides never changes a result bit, because every round evaluates the
 * residual form in the same order (§2 steps 3-4, Algorithm 2).
 * Errors: FC_ERR_ARG (n is not the last fit's count), FC_ERR_STATE (no fit). */
enum { FC_DECIDED_CERT = 1,        /* top-k screen bounds alone certified the minimum    */
       FC_DECIDED_RESCORED = 2,    /* top-k candidates rescored, then certified          */
       FC_DECIDED_TOP16 = 4,       /* top-16 round (FC_ROUND_TOPK policy)                */
       FC_DECIDED_LIST = 8,        /* list round: every g whose bound is below the best  */
       FC_DECIDED_EXACT_LIST = 16, /* the same with exact-size lists (long lists)        */
       FC_DECIDED_SCAN = 32,       /* residual form over every g (mixed path's last step)*/
       FC_DECIDED_PLAIN = 64 };    /* plain binary64 scan (FC_PREC_FP64)                 */
FC_API fc_status fc_get_decided_by(fc_ctx* ctx, uint8_t* out, int64_t n);

/* Counters of the last synchronous run on this context. */
FC_API fc_status fc_get_stats(fc_ctx* ctx, fc_stats* out);
/* Counters summed over everything the serving worker has run (fc_submit jobs).
 * Takes the context's device lock, so it returns between two scans. */
FC_API fc_status fc_get_serve_stats(fc_ctx* ctx, fc_stats* out);

/* Message for the calling thread's last non-OK status ("" if none). */
FC_API const char* fc_last_error(const fc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* FC_H_ */
