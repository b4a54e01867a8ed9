/*
 * linmin.h — C ABI of the GB300 (sm_103a) LinMin unmixing library.
 *
 * LinMin (Schmidt, Legendre & Le Mouelic, "Minerals detection for
 * hyperspectral images using adapted linear unmixing: LinMin") fits every
 * observed spectrum y (L bands) of a cube by a non-negative, sum-to-one
 * combination x (P abundances) of a shared reference library:
 *
 *   Sec. 2.1, eq. LinearMixing:        X = A.S + E, E Gaussian;
 *   Sec. 2.1, eq. UnconstrainedProblem: least squares criterion;
 *   Sec. 2.2, eqs. NonNegativity, SumToOne: x >= 0, sum_j x_j = 1 (FCLS);
 *   Sec. 2.3, eq. RenormalizedProblem: the criterion is whitened by the
 *     noise covariance; here the covariance is diagonal, given as per-band
 *     standard deviations sigma_l, i.e. W = diag(1 / sigma_l);
 *   Sec. 2.2: the problem is solved per pixel by a primal-dual interior
 *     point least-squares method (IPLS);
 *   Sec. 2.3 (last paragraph): the uncertainty of each abundance comes from
 *     the Hessian of the criterion.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Library: float32, P spectra of L bands, spectrum j contiguous
 *   (library[j * L + l]); this is the paper's S (P x N_lambda, row-major),
 *   i.e. an L x P column-major matrix.
 * - Cube: float32, N pixels of L bands, pixel-major (BIP):
 *   cube[n * L + l]; the paper's X (M x N_lambda).
 * - sigma: float32, L per-band noise standard deviations, each finite > 0.
 * - Outputs (caller-allocated, float32 unless stated):
 *     abundances    N x P, pixel-major, x >= 0 and sum_j x_j = 1;
 *     uncertainties N x P, the standard deviation of each abundance under
 *                   the Gaussian noise model: the square root of the
 *                   diagonal of the top-left block of
 *                   [[G_SS, 1],[1^T, 0]]^-1 on the support S of the
 *                   solution, 0 off the support, with G = S W^2 S^T
 *                   (Hessian of 1/2 |W(y - S^T x)|^2; the paper's
 *                   criterion has no 1/2, its Hessian is 2G);
 *     residual_rms  N, sqrt(mean_l (y_l - sum_j x_j S_jl)^2), unwhitened;
 *     iterations    int32 N, interior-point iterations used; negative when
 *                   the pixel needed the retry path and did not reach its
 *                   stopping test within max_iter (its last iterate is
 *                   returned).
 *   Any output pointer may be NULL; that output is then not written.
 * - Pointers may be host or device memory (detected per call).  With device
 *   pointers the call is stream-ordered on the handle's stream and does not
 *   synchronise; with any host pointer it copies through device buffers and
 *   synchronises before returning.
 * - The handle owns all device scratch; it is not thread-safe: use one
 *   handle per host thread / stream.  Calls on one handle are serialised by
 *   its stream.
 * - Errors: every entry point returns a linmin_status; linmin_last_error()
 *   gives a one-line message for the last failing call on that handle.
 *   Invalid arguments are detected on the host before any work is queued.
 */
#ifndef LINMIN_H
#define LINMIN_H

#if defined(__GNUC__)
#define LINMIN_API __attribute__((visibility("default")))
#else
#define LINMIN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct linmin_ctx *linmin_handle;

typedef enum {
    LINMIN_OK = 0,
    LINMIN_ERR_INVALID = 1,        /* bad size, NULL input, sigma <= 0 / NaN */
    LINMIN_ERR_OOM = 2,            /* device allocation failed */
    LINMIN_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    LINMIN_ERR_RANK = 4,           /* rank [S^T; 1^T] < P: minimiser not unique */
    LINMIN_ERR_TIMEOUT = 5,        /* a bounded device wait gave up */
    LINMIN_ERR_NOT_CONVERGED = 6,  /* some pixels hit max_iter; see iterations < 0 */
    LINMIN_ERR_UNSUPPORTED = 7     /* P or L outside the built kernel range */
} linmin_status;

/* Projection precision (c = S W^2 y).
 *   LINMIN_PROJ_DF    double-float (two float32 words) on the CUDA cores;
 *   LINMIN_PROJ_TC    (default) tensor cores (tcgen05), exact: 8-bit integer slices
 *                     of y and of W^2 S / s in bf16, float32 accumulation
 *                     that stays exact, levels combined in double-float
 *                     (the accuracy of LINMIN_PROJ_DF);
 *   LINMIN_PROJ_BF16  tensor cores, bf16 y and W^2 S / s, float32
 *                     accumulation (fast, but c carries bf16 rounding: on
 *                     ill-conditioned libraries x moves by up to ~1e-2).
 * The fully constrained solve needs ~1e-11 relative in c to reach 1e-4 in
 * x on ill-conditioned libraries, hence the exact modes. */
enum { LINMIN_PROJ_DF = 0, LINMIN_PROJ_TC = 1, LINMIN_PROJ_BF16 = 2 };

/* Constraint set (Sec. 2.2 and the variants of Sec. 4):
 *   LINMIN_STO  x >= 0, sum x = 1 (fully constrained, FCLS; default);
 *   LINMIN_SLO  x >= 0, sum x <= 1;
 *   LINMIN_POS  x >= 0.
 * SLO is solved as STO on the library with a zero spectrum appended (its
 * coefficient is the slack 1 - sum x >= 0 and adds nothing to the fit);
 * POS as SLO on LINMIN_POS_SCALE * library, exact while sum x is below
 * LINMIN_POS_SCALE (a pixel that reaches the bound gets a negative
 * iteration count and counts as not converged).  Both need rank S = P
 * (LINMIN_ERR_RANK otherwise) and P <= LINMIN_MAX_P - 1.  The
 * uncertainties are the support-restricted ones: bordered where the sum
 * constraint binds, free where it does not. */
enum { LINMIN_STO = 0, LINMIN_SLO = 1, LINMIN_POS = 2 };
#define LINMIN_POS_SCALE 64

#define LINMIN_MAX_P 64
#define LINMIN_MAX_L 4096

typedef struct {
    int precision;        /* LINMIN_PROJ_TC (default), _DF or _BF16 */
    int constraint;       /* LINMIN_STO (default), LINMIN_SLO or LINMIN_POS */
    int max_iter;         /* interior-point iteration cap per pixel (default 100) */
    float tol;            /* retry path: complementarity tolerance, each
                             coordinate ends with min(x_i, lambda_i / s) <= tol,
                             s = trace(G)/P (default 1e-9) */
    float refine_mu;      /* retry path: switch to the double-float KKT
                             residual once mu / s <= refine_mu (default 1e-9) */
    void *cuda_stream;    /* cudaStream_t the handle runs on; NULL = default */
    int profile;          /* non-zero: record CUDA events around each phase of
                             linmin_unmix (see linmin_phase_times); default 0 */
} linmin_options;

/* Phases of linmin_unmix timed when linmin_options.profile is set. */
enum {
    LINMIN_PHASE_PREP = 0,      /* whitening, fp64 Gram, splits (3 kernels) */
    LINMIN_PHASE_PROJECT = 1,   /* double-float projection c = S W^2 y */
    LINMIN_PHASE_IPM = 2,       /* interior point, float32 residual, all pixels */
    LINMIN_PHASE_CROSSOVER = 3, /* double-float active-set finish + uncertainties */
    LINMIN_PHASE_RETRY = 4,     /* pixels the crossover could not finish:
                                   interior point with the double-float
                                   residual, then the crossover again */
    LINMIN_PHASE_RMS = 5,       /* residual RMS */
    LINMIN_NUM_PHASES = 6
};

/* Fill *opt with the defaults listed above.  Never fails for a non-NULL opt. */
LINMIN_API linmin_status linmin_default_options(linmin_options *opt);

/*
 * Create a handle for one reference library (Sec. 2.4/2.5: the mineral
 * spectra plus any additional level/slope spectra, all as columns).
 *   library  P x L float32 (see conventions), host or device, read during
 *            the call only (the handle keeps a device copy);
 *   L, P     1 <= P <= LINMIN_MAX_P, P <= L <= LINMIN_MAX_L;
 *   opt      NULL for defaults;
 *   out      receives the handle (NULL on failure).
 * Returns LINMIN_ERR_RANK when rank [S^T; 1^T] < P (checked in fp64 on the
 * host): the fully constrained minimiser is then not unique (Sec. 5: the
 * constraints remove degeneracies only when this rank is full).
 */
LINMIN_API linmin_status linmin_create(const float *library, int L, int P,
                            const linmin_options *opt, linmin_handle *out);

/*
 * Unmix N pixels: whitening (Sec. 2.3), projection c = S W^2 y,
 * primal-dual interior-point FCLS per pixel (Sec. 2.2) until the support of
 * the solution is identified, a double-float active-set crossover to the exact
 * minimiser (the few pixels it cannot finish are re-solved with a
 * double-float KKT residual), abundance uncertainties (Sec. 2.3) and the RMS
 * of the fit.
 *   cube  N x L float32, host or device;  N >= 0 (N = 0 is a no-op);
 *   sigma L float32 > 0, host or device;
 *   outputs as in the conventions (NULL = skip).
 * Device pointers: returns after queueing (use linmin_wait to learn about
 * non-converged pixels).  Host pointers: synchronous; returns
 * LINMIN_ERR_NOT_CONVERGED when some pixel has iterations < 0.
 */
LINMIN_API linmin_status linmin_unmix(linmin_handle h, const float *cube, long long N,
                           const float *sigma, float *abundances,
                           float *uncertainties, float *residual_rms,
                           int *iterations);

/*
 * linmin_unmix under a full noise covariance C (Sec. 2.3, eq.
 * RenormalizedProblem: the data are whitened as X' = X L with C^-1 = L L^T;
 * off-diagonal terms model band-correlated noise).
 *   cov_inv  the L x L inverse covariance C^-1, symmetric positive definite,
 *            row-major float64, host or device.  It is copied to the host
 *            and checked (finite, symmetric to 1e-9 of its largest entry,
 *            positive definite by an fp64 Cholesky) whenever its contents
 *            differ from the last checked one (LINMIN_ERR_INVALID
 *            otherwise); its symmetric part is used.
 * G = S C^-1 S^T and B = C^-1 S^T are formed in fp64 on the device; the
 * projection, the solve, the uncertainties (from G) and the unwhitened RMS
 * are those of linmin_unmix.  Other arguments and the return value as
 * linmin_unmix.  The handle keeps C^-1 (L^2 doubles) on the device.
 */
LINMIN_API linmin_status linmin_unmix_cov(linmin_handle h, const float *cube, long long N,
                                          const double *cov_inv, float *abundances,
                                          float *uncertainties, float *residual_rms,
                                          int *iterations);

/*
 * linmin_unmix (Sec. 2.2-2.3: the same whitening, interior point,
 * crossover, uncertainties and RMS) of n cubes of uneven sizes in one
 * queue: every cube's library preparation and projection, then ONE
 * float32 interior-point launch per group of cubes with the same P and
 * kernel bucket (a persistent grid, one work counter over all pixels of
 * the group, each pixel group reading its own cube's G~ through L1), then
 * every cube's crossover, retry and RMS.
 *   handles  n handles (distinct; sum-to-one; same device and the same
 *            cuda_stream, on which everything is queued);
 *   cubes[i] N[i] x L_i float32, sigmas[i] L_i float32 > 0,
 *   abundances[i] N[i] x P_i (required); uncertainties, residual_rms,
 *   iterations: arrays of n pointers or NULL, entries may be NULL;
 *   every buffer in device memory (LINMIN_ERR_INVALID otherwise).
 * Results equal those of linmin_unmix on each cube.  Returns after
 * queueing; linmin_wait(handles[i]) reports cube i's non-converged pixels.
 * handles[0] keeps the group descriptors on the device.
 */
LINMIN_API linmin_status linmin_unmix_batch(int n, const linmin_handle *handles,
                                            const float *const *cubes, const long long *N,
                                            const float *const *sigmas,
                                            float *const *abundances,
                                            float *const *uncertainties,
                                            float *const *residual_rms,
                                            int *const *iterations);

/* Synchronise the handle's stream.  *n_not_converged (may be NULL) receives
 * the number of pixels of the last linmin_unmix that hit max_iter.  Returns
 * LINMIN_ERR_NOT_CONVERGED when that number is non-zero. */
LINMIN_API linmin_status linmin_wait(linmin_handle h, long long *n_not_converged);

/* Device time (ms) of each phase of the last linmin_unmix on h, measured
 * with CUDA events on the handle's stream; requires opt.profile.  ms_out
 * receives min(n, LINMIN_NUM_PHASES) values; waits for that call's last
 * event.  Returns LINMIN_ERR_INVALID when profiling is off or nothing ran
 * yet. */
LINMIN_API linmin_status linmin_phase_times(linmin_handle h, float *ms_out, int n);

/* Number of past calls whose phase events a handle keeps. */
#define LINMIN_PHASE_RING 32

/* As linmin_phase_times for the call `back` calls before the last one
 * (back = 0: the last call), 0 <= back < LINMIN_PHASE_RING: calls queued
 * back to back can be timed phase by phase after one synchronisation.
 * LINMIN_ERR_INVALID when that call is not (or no longer) recorded. */
LINMIN_API linmin_status linmin_phase_times_at(linmin_handle h, int back, float *ms_out,
                                               int n);

/* Free the handle and its device memory (synchronises its stream first).
 * NULL is accepted. */
LINMIN_API linmin_status linmin_destroy(linmin_handle h);

/* One-line description of the last error on h (or of the last failed
 * linmin_create when h is NULL).  The string lives until the next call. */
LINMIN_API const char *linmin_last_error(linmin_handle h);

/* Number of kernel launches the last linmin_unmix on h queued (0 before the
 * first call or for N = 0; -1 for a NULL handle).  A fixed pipeline: 3
 * preparation kernels, the projection, the interior-point kernel, the
 * crossover (support, counting sort, a pass over every pixel and the
 * lane groups that take the pixels it could not finish through further
 * support changes: one launch, or for P > 24 two, the first for supports
 * of at most 24 coordinates), the retry path (two interior-point kernels,
 * support, the same lane-group launches) and the RMS. */
LINMIN_API int linmin_last_launches(linmin_handle h);

/* Lanes per pixel (G) of the interior-point kernel the handle runs: a
 * pixel's H is spread over G lanes, NS = ceil(P / G) rows per lane
 * (-1 for a NULL handle).  The default per P is the fastest measured on
 * GB300 (4 lanes wherever the registers of H allow it). */
LINMIN_API int linmin_get_lanes(linmin_handle h);

/* Use G lanes per pixel from now on (a compiled bucket with P <= NS*G <
 * P + 16 must exist, else LINMIN_ERR_UNSUPPORTED; the handle keeps its
 * previous choice).  Results stay within the same tolerances. */
LINMIN_API linmin_status linmin_set_lanes(linmin_handle h, int lanes);

/* Autotuner: time the interior-point kernel of every compiled bucket that
 * fits P (P <= NS*G < P + 16) on the first min(N, 32768) pixels of cube
 * (host or device; sigma likewise), best of two runs each, and keep the
 * fastest for the handle.  *lanes_out (may be NULL) receives its G,
 * ms_out[i] (may be NULL; n_ms entries) the time of candidate i,
 * *n_candidates (may be NULL) the number of candidates.  Synchronous. */
LINMIN_API linmin_status linmin_autotune(linmin_handle h, const float *cube, long long N,
                                         const float *sigma, int *lanes_out, float *ms_out,
                                         int n_ms, int *n_candidates);

/* Library version string. */
LINMIN_API const char *linmin_version(void);

/* Device allocations the library's handles hold now, over all devices
 * (handles of servers included).  With the environment variable
 * LINMIN_FAIL_ALLOC = N (N >= 1), read when a handle is created, that
 * handle's N-th device allocation fails as if the device were out of
 * memory, without calling CUDA (linmin_autofit: its allocation, for
 * N = 1): the entry point returns LINMIN_ERR_OOM, and this count shows
 * that nothing was kept.  Unset or 0: no injection.  The paper has no
 * counterpart: a diagnostic for the error paths. */
LINMIN_API linmin_status linmin_live_allocations(long long *count);

/* Measured FP32 throughput of the current device, the roofline peak of the
 * interior-point solve (which is bound by FP32 FMAs): TFLOP/s (2 flops
 * per FMA) of independent FMA chains on every SM, as scalar FFMA
 * (*tflops_ffma) and packed two-wide FFMA2 (*tflops_ffma2), each timed with
 * CUDA events on cuda_stream (NULL: the default stream) around a second
 * launch of fixed work (~2 ms).  Synchronous; uses a small stream-ordered
 * allocation.  The paper has no counterpart: a measurement utility. */
LINMIN_API linmin_status linmin_fp32_peak(double *tflops_ffma, double *tflops_ffma2,
                                          void *cuda_stream);

/* ------------------------------------------------------------------ */
/*
 * Serving: continuous batching of unmixing requests.  The paper has no
 * counterpart (it unmixes one cube at a time); this is the runtime that
 * runs cubes of different sizes and libraries as they arrive.
 *
 * A request (one cube against one library) is cut into chunks of at most
 * chunk_pixels pixels; `slots` worker threads, each with its own CUDA
 * stream, run the chunks of all requests, oldest request first, so the
 * chunks of different requests overlap on the device and a request that
 * arrives while others run starts as soon as a slot and device memory are
 * free.  Each worker keeps a handle (library copy, per-sigma factors,
 * scratch reserved for one chunk) per library it served; the device bytes
 * of all handles stay within hbm_budget_bytes (idle handles are destroyed,
 * least recently used first, to make room; otherwise the chunk waits).
 * Results are bit-identical to a linmin_unmix call over the whole cube.
 */
typedef struct linmin_server_s *linmin_server;

typedef struct {
    unsigned long long hbm_budget_bytes; /* device bytes of the server's handles
                                            (default 1 GiB; allocation
                                            granularity not counted) */
    int slots;                /* worker streams = chunks in flight (1..64, default 4) */
    long long chunk_pixels;   /* pixels per chunk (default 65536) */
    int max_iter;             /* interior-point cap per pixel (default 100) */
    int autotune;             /* != 0 (default): the first handle made for a library
                                 shape (L, P) on a device runs linmin_autotune on its
                                 first chunk, and later handles of that shape (in any
                                 server of the process) take its choice */
} linmin_server_options;

/* One cube.  Pointers as in linmin_create / linmin_unmix (host or device;
 * NULL outputs are skipped); every buffer must stay valid until
 * linmin_server_wait returns for the request. */
typedef struct {
    const float *library;     /* P x L */
    int L, P;
    const float *cube;        /* N x L */
    long long N;
    const float *sigma;       /* L */
    float *abundances;        /* N x P */
    float *uncertainties;     /* N x P */
    float *residual_rms;      /* N */
    int *iterations;          /* N */
} linmin_request;

typedef struct {
    unsigned long long requests, requests_done, chunks;
    unsigned long long handles_created, evictions;
    unsigned long long bytes, peak_bytes;  /* device bytes of handles: now / at most */
    int running, max_running;              /* chunks on the device: now / at most */
    long long libraries;                   /* distinct libraries kept (at most 64 beyond
                                              those in use: the least recently used idle
                                              ones are dropped with their handles) */
    long long autotuned;                   /* autotuner runs by this server (one per
                                              shape and device in the process) */
} linmin_server_stats;

LINMIN_API linmin_status linmin_server_default_options(linmin_server_options *opt);

/* Start the worker threads on the current device.  LINMIN_ERR_INVALID for
 * out-of-range options, LINMIN_ERR_CUDA without a usable device. */
LINMIN_API linmin_status linmin_server_create(const linmin_server_options *opt,
                                              linmin_server *out);

/* Queue a request; *ticket identifies it.  Checked before queueing (the
 * same errors as linmin_create, LINMIN_ERR_OOM when one chunk's handle
 * cannot fit the budget); a library is checked (and its rank computed) on
 * every submit.  Thread-safe. */
LINMIN_API linmin_status linmin_server_submit(linmin_server s, const linmin_request *req,
                                              long long *ticket);

/* *done = 1 once every chunk of the request has finished.  Thread-safe. */
LINMIN_API linmin_status linmin_server_poll(linmin_server s, long long ticket, int *done);

/* Block until the request has finished; returns its status (the worst of
 * its chunks: LINMIN_ERR_NOT_CONVERGED when some pixel hit max_iter) and,
 * in *latency_ms (may be NULL), the time from submit to completion.  The
 * ticket is released: wait once per ticket.  Thread-safe. */
LINMIN_API linmin_status linmin_server_wait(linmin_server s, long long ticket,
                                            double *latency_ms);

LINMIN_API linmin_status linmin_server_get_stats(linmin_server s, linmin_server_stats *st);

/* Device bytes one server handle holds for a library of L bands and P
 * spectra with scratch for chunk_pixels pixels (host_io != 0: with the
 * staging buffers of host-pointer requests); 0 when P is unsupported. */
LINMIN_API unsigned long long linmin_server_handle_bytes(int L, int P, long long chunk_pixels,
                                                         int host_io);

/* Reason of the last failed submit/wait on s. */
LINMIN_API const char *linmin_server_last_error(linmin_server s);

/* Finish the queued requests, stop the workers, free every handle. */
LINMIN_API linmin_status linmin_server_destroy(linmin_server s);

/* Size in MiB of the static device scratch array of linmin_unmix_noalloc. */
#define LINMIN_NOALLOC_SCRATCH_MB 64

/*
 * linmin_unmix_noalloc — the same unmixing as linmin_unmix for callers that
 * cannot allocate device memory: code running where cudaMalloc is not
 * allowed or not wanted, such as inside a host callback, a plugin that
 * must not touch its host application's memory pool, or a process that
 * has already reserved all device memory for itself.  It allocates nothing
 * (no cudaMalloc/cudaFree, no allocating library routine, no handle): its
 * scratch lives in one file-scope __device__ array of
 * LINMIN_NOALLOC_SCRATCH_MB MiB, which every GPU that loads this library
 * holds until the process exits.  The paper has no counterpart: this is
 * an integration entry point, not part of the method.
 *
 *   library, cube, sigma, outputs: as in linmin_create/linmin_unmix, but
 *            every non-NULL pointer must be device memory of the current
 *            device, or managed memory (else LINMIN_ERR_INVALID);
 *   cuda_stream: the cudaStream_t to run on (NULL: default stream); the
 *            call queues its work and returns without synchronising.
 * Limit: the scratch needed is, with every piece rounded up to 256 bytes,
 *   2 P^2 doubles + 1 double + 2 PP^2 + PP + P + 2 L*PQ floats + 1 int
 *   + 20 + P uint64 + P + 1 uint32 + N (4 P + 11) 4-byte words
 *   <=  LINMIN_NOALLOC_SCRATCH_MB MiB
 *   (PP = P rounded up to the kernel bucket 8, 16, 32, 36, 40, 48 or 64;
 *   PQ = P rounded up to a multiple of 4); for L = 184, P = 36 that is
 *   about 107,000 pixels.  A larger N returns LINMIN_ERR_INVALID before any
 *   work (linmin_noalloc_scratch_bytes gives the figure for a size).
 * Unlike linmin_create it does not check rank [S^T; 1^T] = P: the caller
 *   guarantees a library whose constrained minimiser is unique.
 * Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and caches it; make
 *   that first call before any stream capture on that device.
 * Concurrency: every call on a device shares the one array, and a call
 *   leaves its contents behind (counters are cleared at the start of each
 *   call).  Calls whose work overlaps on the GPU (different streams, or
 *   different host threads) race on it: serialise them on one stream.
 * Non-converged pixels are reported by iterations < 0 only.
 * Invalid inputs found on the device: the call returns before its work
 *   has run, so a sigma with a value that is not finite or not > 0, or a
 *   library whose whitened Gram has a zero trace, cannot change the status
 *   it returns.  Instead every output of that call is marked: abundances,
 *   uncertainties and RMS are NaN and every iteration count is INT_MIN.
 */
LINMIN_API linmin_status linmin_unmix_noalloc(const float *library, int L, int P,
                                              const float *cube, long long N,
                                              const float *sigma, float *abundances,
                                              float *uncertainties, float *residual_rms,
                                              int *iterations, void *cuda_stream);

/* Device bytes linmin_unmix_noalloc needs for (L, P, N), in *bytes
 * (host pointer; set to 0 on failure).  Returns LINMIN_OK when they fit in
 * the LINMIN_NOALLOC_SCRATCH_MB array, LINMIN_ERR_INVALID when they do not
 * (or N < 0, L out of range) and LINMIN_ERR_UNSUPPORTED for P outside
 * 1..LINMIN_MAX_P.  Host arithmetic only: no device call.  The paper has no
 * counterpart. */
LINMIN_API linmin_status linmin_noalloc_scratch_bytes(int L, int P, long long N,
                                                      unsigned long long *bytes);

/* ------------------------------------------------------------------ */
/*
 * Detection products.  After unmixing, a mineral counts as detected in a
 * pixel under the conditions the paper lists for real images (Sec. 4,
 * introduction): its abundance is above a threshold chosen per mineral,
 * its uncertainty is below its abundance, and the pixel's RMS is below
 * the noise level.  The thresholds come from the synthetic surface
 * mixtures of Sec. 3.1 (eq. Threshold), where the truth is known.  The
 * paper has no C interface for these; the entry points below are
 * stream-ordered device computations (no synchronisation).
 */

/* The paper's additional spectra (Sec. 2.5; Appendix, names 33-44), one row
 * of L values each in out (host, n_extras x L), with u = (w_l - w_0) /
 * (w_{L-1} - w_0) over the wavelengths w (host, L values increasing; NULL:
 * evenly spaced, u_l = l / (L - 1)):
 *   n_extras = 4:  Flat 1, Flat 0.0001, slope increasing u, slope
 *                  decreasing 1 - u;
 *   n_extras = 12: those four, then cos, sin, -cos, -sin of pi u / 2 (the
 *                  "1/4" functions: a quarter period over the domain), then
 *                  of pi u (the "1/2" functions).
 * Computed in double, rounded to float.  Under x >= 0, sum x = 1 neither
 * set leaves the minimiser unique: rank [S^T; 1^T] is 3 for the four and 7
 * for the twelve, so linmin_create refuses a library that holds all of
 * them (LINMIN_ERR_RANK).  L >= 2, else LINMIN_ERR_INVALID. */
LINMIN_API linmin_status linmin_extra_spectra(int L, const float *wavelengths, int n_extras,
                                              float *out);

/* Per-mineral detection summary (device memory, written by linmin_detect).
 * Entries at index >= n_minerals are zero. */
typedef struct {
    long long count[LINMIN_MAX_P];      /* pixels where mineral i is detected */
    long long argmax[LINMIN_MAX_P];     /* smallest pixel index holding the
                                           largest detected x_i; -1 if none */
    long long n_true[LINMIN_MAX_P];     /* with truth: pixels where i is present */
    long long true_pos[LINMIN_MAX_P];   /* with truth: present and detected */
    long long false_pos[LINMIN_MAX_P];  /* with truth: absent and detected */
    double xsum[LINMIN_MAX_P];          /* sum of the detected x_i (atomic
                                           order: last-bit differences run to
                                           run) */
    float xmax[LINMIN_MAX_P];           /* largest detected x_i; 0 if none */
    unsigned long long key[LINMIN_MAX_P]; /* scratch of the arg-max */
} linmin_detection;

/* Detect minerals pixel by pixel.  All array pointers are device memory:
 *   x, sx      N x P abundances and uncertainties (linmin_unmix outputs);
 *              sx may be NULL (no uncertainty condition);
 *   rms        N residual RMS, may be NULL (no RMS condition);
 *   iterations N, may be NULL; a pixel with iterations < 0 detects nothing;
 *   truth      N bit masks, may be NULL: bit i set when mineral i is
 *              present in the pixel (synthetic cubes), for the rates;
 *   x_min      host, n_minerals thresholds C_i (finite, >= 0);
 *   mask       N bit masks out, may be NULL: bit i set when mineral i is
 *              detected;
 *   out        one linmin_detection, may be NULL.
 * Mineral i < n_minerals is detected in pixel n when
 *   x[n,i] > x_min[i]  and  sx[n,i] < x[n,i]  and  rms[n] < rms_max
 * (strict comparisons of the float32 values; absent arrays drop their
 * condition).  Columns >= n_minerals (the additional spectra) are never
 * detected.  1 <= P <= LINMIN_MAX_P, 0 <= n_minerals <= P,
 * 0 <= N < 2^32; stream: cudaStream_t or NULL. */
LINMIN_API linmin_status linmin_detect(const float *x, const float *sx, const float *rms,
                                       const int *iterations, const unsigned long long *truth,
                                       long long N, int P, int n_minerals, const float *x_min,
                                       float rms_max, unsigned long long *mask,
                                       linmin_detection *out, void *stream);

/* Sums over the pixels where mineral i is present (pos) and absent (neg)
 * in a synthetic cube, for eq. Threshold (device memory): counts, sums,
 * and sums of squared deviations from the mean (m2; two passes, so the
 * variance m2 / n has no cancellation). */
typedef struct {
    long long n_pos[LINMIN_MAX_P], n_neg[LINMIN_MAX_P];
    double sum_pos[LINMIN_MAX_P], m2_pos[LINMIN_MAX_P];
    double sum_neg[LINMIN_MAX_P], m2_neg[LINMIN_MAX_P];
} linmin_threshold_sums;

/* Accumulate linmin_threshold_sums of x (device, N x P) split by truth
 * (device, N bit masks), for minerals i < n_minerals; out is device
 * memory, overwritten.  Two stream-ordered launches (sums, then squared
 * deviations from their means).  Same limits as linmin_detect. */
LINMIN_API linmin_status linmin_threshold_stats(const float *x, const unsigned long long *truth,
                                                long long N, int P, int n_minerals,
                                                linmin_threshold_sums *out, void *stream);

/* eq. Threshold, per mineral i < n_minerals, from stats on the host:
 *   C_i = 1/2 (mean_pos - 2 std_pos + mean_neg + 6 std_neg)
 * with population standard deviations (divided by the count).  A mineral
 * with no present or no absent pixel gets C_i = NaN. */
LINMIN_API linmin_status linmin_thresholds(const linmin_threshold_sums *stats, int n_minerals,
                                           float *c_out);

/* Auto-fit of the library (Sec. 2.4, "Estimation of degeneracies"): each
 * spectrum S_n is fitted by the P - 1 others, S_n = A'.S' + E, without
 * constraints and with A' >= 0, to show which spectra the others can
 * mimic.  Unweighted, fp64 on the device, one block per n.
 *   library   device, P x L (as in linmin_create);
 *   resid_ls  P x L, row n: the unconstrained residue E (S_n minus its
 *             projection on the span of the others; unique); may be NULL;
 *   resid_nn  P x L, row n: the residue under A' >= 0 (unique); may be NULL;
 *   coef_nn   P x P, row n: the non-negative coefficients of the other
 *             spectra (0 at n; unique when the others are independent);
 *             may be NULL;
 *   rms_ls, rms_nn  P: sqrt(mean_l E^2) of each residue; may be NULL;
 *   status    int P: 0 converged, 1 active-set iteration cap; may be
 *             NULL.  A spectrum numerically dependent on the passive ones
 *             (Cholesky pivot below 1e-14 of its diagonal) is left out.
 * All output arrays are device memory.  2 <= P <= LINMIN_MAX_P,
 * P <= L <= LINMIN_MAX_L.  Allocates P * P * L doubles of stream-ordered
 * scratch; stream: cudaStream_t or NULL; no synchronisation. */
LINMIN_API linmin_status linmin_autofit(const float *library, int L, int P, float *resid_ls,
                                        float *resid_nn, float *coef_nn, float *rms_ls,
                                        float *rms_nn, int *status, void *stream);

/* Unmix each pixel with a subset of the library: pixel n uses the
 * columns j < n_minerals whose bit j is set in mask[n] and every column
 * j >= n_minerals (the additional spectra), as if it were unmixed with
 * that sub-library alone; the abundances and uncertainties of its
 * left-out columns are 0.  This is the second pass of Sec. 5 (mask: the
 * detections of linmin_detect).  Arguments as linmin_unmix; mask is
 * device memory (N bit masks, bits >= n_minerals ignored);
 * 0 <= n_minerals < P (for SLO / POS handles: the caller's P).
 * The left-out columns are removed by an exact linear penalty on their
 * projections: c~_j -= K_n with K_n = 2 (max_k |c~_k| + P + 1) + 1, above
 * any multiplier the sub-problem can give x_j = 0 (c~ and the bound live
 * in the scaled problem G~ = G / s + 1 1^T, c~ = c / s + 1,
 * s = trace(G) / P), so the penalised problem has exactly the
 * sub-problem's minimiser; one extra kernel over the N x P projections. */
LINMIN_API linmin_status linmin_unmix_masked(linmin_handle h, const float *cube, long long N,
                                             const float *sigma, const unsigned long long *mask,
                                             int n_minerals, float *abundances,
                                             float *uncertainties, float *residual_rms,
                                             int *iterations);

/* Second pass (Sec. 5) in one call: a handle for the full library
 * (host or device, P x L, minerals first: columns < n_minerals; rank
 * checked as in linmin_create, and then every subset of its columns gives
 * a unique minimiser too), linmin_unmix_masked with the detection masks,
 * linmin_wait, and the handle freed.
 *   opt   options (NULL: defaults); the stream is opt->cuda_stream;
 *   cube, sigma, mask and the outputs are device memory.
 * Synchronous.  Returns LINMIN_ERR_NOT_CONVERGED when some pixel has
 * iterations < 0. */
LINMIN_API linmin_status linmin_second_pass(const float *library, int L, int P, int n_minerals,
                                            const linmin_options *opt, const float *cube,
                                            long long N, const float *sigma,
                                            const unsigned long long *mask, float *abundances,
                                            float *uncertainties, float *residual_rms,
                                            int *iterations);

#ifdef __cplusplus
}
#endif
#endif /* LINMIN_H */
