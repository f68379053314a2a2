/*
 * smol.h - C interface of the GB300 (sm_103a) solver for the truncated
 * aggregation-shattering Smoluchowski system with a low-rank kernel.
 *
 * What is computed (Matveev, Zhilin, Smirnov, "Adaptive time-stepping for
 * aggregation-shattering kinetics", arXiv 2407.16559):
 *
 *   Eq. (4), sizes s = 1..M (stored 0-based, n[s-1] = n_s):
 *     dn_1/dt = - n_1 sum_{i=1}^{M} K_{1,i} n_i
 *               + (lambda/2) sum_{i>=2} sum_{j>=2} (i+j) K_{i,j} n_i n_j
 *               + lambda n_1 sum_{j>=2} j K_{1,j} n_j
 *     dn_s/dt = 1/2 sum_{i+j=s} K_{i,j} n_i n_j - (1+lambda) n_s sum_{i=1}^{M} K_{s,i} n_i,
 *               s = 2..M.
 *   The last monomer term is read with the factor n_1 (every collision term is
 *   quadratic in n, and only then does shattering conserve mass).
 *   Births above M are dropped; death sums run to M (Eq. (2)).
 *
 *   Low-rank kernel (Sec. 1): K_{i,j} = sum_{alpha=1}^{R} U_{i,alpha} V_{alpha,j}.
 *   The birth term is evaluated as 1/2 sum_alpha (U_alpha . n) * (V_alpha . n), a
 *   linear convolution computed with zero-padded FFTs, and the death and monomer
 *   terms from rank-R moment sums, O(M R log M) per evaluation (Sec. 1, Sec. 2).
 *
 *   Constant point sources (Eq. (3), Sec. 3.1): dn_s/dt = S_s(n) + P_s
 *   (smol_set_sources); with lambda = 0 that is aggregation with sources.
 *
 *   Operator form (Eq. (5)): dn/dt = S(n), n(0) = n_0, integrated with the explicit
 *   RK2, RK4 and Runge-Kutta-Fehlberg 4(5) schemes of Sec. 2 with adaptive steps:
 *   step doubling for RK2 / RK4 (error ||n_hat - n||_2, Eq. (6) or the halve/double
 *   rule) and Fehlberg's rule for RKF45 (tau <- 0.9 tau (tol/err)^(1/5)).
 *
 * Conventions for every call:
 *   - 0 (SMOL_OK) is success; errors are negative SMOL_E* codes; smol_strerror()
 *     names them. A call that fails leaves the caller's buffers unspecified but
 *     valid; the system object stays usable unless SMOL_ECUDA was returned.
 *   - Device pointers ("d_") point to memory of the current CUDA device, 16-byte
 *     aligned, owned by the caller. Host pointers ("h_") are plain host memory.
 *   - Work is enqueued on the stream given in smol_opts.stream (NULL = legacy
 *     default stream). smol_rhs returns without synchronising; smol_integrate
 *     synchronises that stream once before it returns.
 *   - The library never allocates device memory on the solver's path: every device
 *     buffer it uses lives in the caller's workspace (smol_workspace_bytes) or is a
 *     caller argument. It allocates a small pinned host block per system for status
 *     read-back. The set-up calls smol_tune and smol_batch_tune allocate and free
 *     their own scratch.
 */
#ifndef SMOL_H
#define SMOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SMOL_OK                0   /* success; integrate reached t1 */
#define SMOL_STEADY            1   /* integrate stopped: ||S(n)||_2 / ||n||_2 < steady_rtol */
#define SMOL_EINVAL           -1   /* bad argument (M < 1, R outside 1..SMOL_MAX_R, NULL, t1 < t0, tol <= 0, ...) */
#define SMOL_ECUDA            -2   /* a CUDA runtime call failed */
#define SMOL_ENONFINITE       -3   /* NaN or Inf in the error estimate or the candidate state */
#define SMOL_ESTEP_UNDERFLOW  -4   /* step fell below tau_min_rel * max(1, |t|) */
#define SMOL_EMAXATTEMPTS     -5   /* max_attempts step attempts used before t1 */
#define SMOL_ETIMEOUT         -6   /* a bounded device wait gave up */
#define SMOL_ENOSPACE         -7   /* workspace smaller than smol_workspace_bytes() */
#define SMOL_EUNSUPPORTED     -8   /* shape beyond what the kernels support (see smol_max_m) */

/* Largest rank R of the kernel factors. */
#define SMOL_MAX_R 16

/* Schemes of Sec. 2. */
#define SMOL_RK2    0
#define SMOL_RK4    1
#define SMOL_RKF45  2

/* Arithmetic of the right-hand side.
 *   SMOL_FP64:     everything in FP64 (the plain solver).
 *   SMOL_FP32CONV: FFTs, spectral products, the inverse and the element-wise terms in
 *                  FP32, each transform's input scaled by a power of two; the state,
 *                  RK combination, error, step control, mass and the monomer equation
 *                  stay FP64 (results within 1e-4 of FP64).
 *   SMOL_DF64:     as SMOL_FP32CONV with FP32 replaced by double-float (pairs of FP32
 *                  numbers, ~48 significant bits) on the FP32 pipes: FP64-level results
 *                  (the FP64 tolerance, 1e-10) at FP32-pipe throughput; GB300 runs FP64
 *                  at 1/64 of its FP32 rate. */
#define SMOL_FP64      0
#define SMOL_FP32CONV  1
#define SMOL_DF64      2

/* Step rule for RK2 / RK4 with step doubling (Sec. 2).
 *   SMOL_CTRL_DOUBLE_HALVE: err > tol -> reject, tau /= 2; else accept, tau *= 2.
 *   SMOL_CTRL_FORMULA:      Eq. (6) tau_new = s tau (tol/err)^(1/p), s = 1/4,
 *                           accept iff err <= tol, factor clamped to [fac_min, fac_max]. */
#define SMOL_CTRL_DOUBLE_HALVE 0
#define SMOL_CTRL_FORMULA      1

/* Error norm: absolute ||.||_2 over all M entries, or divided by ||n^k||_2. */
#define SMOL_NORM_ABS 0
#define SMOL_NORM_REL 1

/* Option flags (smol_opts.flags). */
#define SMOL_FLAG_NO_PDL 1  /* launch every kernel after its predecessor has ended (no
                               programmatic dependent launch) */
/* The same for one kernel class only (the SMOL_PROF_* kinds below, shifted): */
#define SMOL_FLAG_NO_PDL_FWD_COLS 2
#define SMOL_FLAG_NO_PDL_ROWS     4
#define SMOL_FLAG_NO_PDL_INV_COLS 8
#define SMOL_FLAG_NO_PDL_STEP     16
/* Launch every evaluation's inverse column pass as its own kernel (by default it runs
   in one kernel with the next evaluation's forward column pass, or with the attempt's
   final combination). */
#define SMOL_FLAG_NO_FUSE         32
/* Single-system RKF45 integrations: each chunk of attempts is one cooperative launch of
   a persistent kernel whose CTAs run the phases of the attempts back to back, separated
   by grid-wide barriers, instead of a graph of 13 launches per attempt. The results are
   those of the graph path. Needs every CTA of the grid resident at once; otherwise (and
   for other schemes, fixed steps or batches) the graph path runs. A barrier wait that
   gives up (about 2 s) ends the integration with SMOL_ETIMEOUT. */
#define SMOL_FLAG_PERSISTENT      64
/* Single FP64 or double-float systems: column kernels with one thread per element pair
   of their tile, up to 512 threads a CTA (default: up to 256, two or more pairs a
   thread). Their per-element phases (stage input, epilogue, final combination) are
   chains of dependent FP64 operations, which the added warps overlap; the FFT passes
   keep one thread per butterfly. No effect on batches or on the FP32 form (whose column
   kernels keep to 256 threads). */
#define SMOL_FLAG_WIDE_COLS       128

/* Size classes of the per-size FFT schedules of a batch (smol_opts.batch_lgn1 / batch_g):
   class k holds the systems with FFT size Mp = 2^k. */
#define SMOL_SIZE_CLASSES 24

typedef struct smol_system smol_system;   /* opaque, created by smol_init_system */

typedef struct smol_opts {
    int32_t precision;      /* SMOL_FP64 | SMOL_FP32CONV | SMOL_DF64 */
    int32_t ctrl;           /* SMOL_CTRL_* (RK2 / RK4 only) */
    int32_t norm;           /* SMOL_NORM_* */
    int32_t log_capacity;   /* attempts kept in the device step log (ring); 0 = no log */
    double  tau0;           /* first step; <= 0: Euler criterion of Sec. 1 with a = euler_a */
    double  euler_a;        /* a of tau <= a [max_i sum_j K_ij n_j]^{-1}; default 0.1 */
    double  tau_min_rel;    /* SMOL_ESTEP_UNDERFLOW below tau_min_rel * max(1,|t|); default 1e-12 */
    double  steady_rtol;    /* > 0: stop with SMOL_STEADY when ||S(n)||_2/||n||_2 < steady_rtol */
    double  fixed_tau;      /* > 0: constant steps of this size, no error control */
    double  fac_min;        /* bounds of the step factor; defaults 0.1 and 4 */
    double  fac_max;
    int64_t max_attempts;   /* default 2^62 */
    int32_t chunk;          /* step attempts per CUDA-graph launch; default 32 */
    int32_t flags;          /* SMOL_FLAG_* bits; 0 = defaults */
    void*   stream;         /* cudaStream_t; NULL = legacy default stream */
    /* FFT schedule of a single system: 0 = the rule. */
    int32_t fft_lgn1;       /* log2 N1 of Mp = N1 N2 (column length), 1 <= fft_lgn1 < log2 Mp */
    int32_t fft_g;          /* columns per CTA of the column kernels, a power of two <= 64 */
    /* FFT schedules of a batch's systems by size class: entry k serves the systems whose
       FFT size is Mp = 2^k (the same meanings as fft_lgn1 and fft_g; 0 = the rule;
       smol_batch_tune_schedules fills them). */
    int8_t  batch_lgn1[SMOL_SIZE_CLASSES];
    int8_t  batch_g[SMOL_SIZE_CLASSES];
} smol_opts;

typedef struct smol_stats {
    double  t;               /* time reached */
    double  tau_next;        /* proposed next step (resume with tau0 = tau_next) */
    double  err_last;        /* error estimate of the last attempt */
    double  mass;            /* sum_s s n_s of the final state (FP64) */
    int64_t rhs_evals;       /* S(n) evaluations actually made (a retry reuses S(n^k)) */
    int64_t rhs_evals_paper; /* stages x RK steps evaluated, the count of the paper's tables */
    int64_t accepted;
    int64_t rejected;
    int64_t attempts;
    int32_t status;          /* SMOL_OK, SMOL_STEADY or a negative code */
    int32_t reserved;
} smol_stats;

/* Fills *opts with the defaults listed above. Never fails for a non-NULL pointer. */
void smol_default_opts(smol_opts* opts);

/* Largest M the kernels accept for rank R and precision when no transforms are shared
 * (T = 2R distinct forward transforms), or 0 if R is unsupported. */
int64_t smol_max_m(int32_t R, int32_t precision);

/* Largest M for T distinct forward transforms (1 <= T <= 2 SMOL_MAX_R). Columns of U and
 * rows of V that are equal up to a factor share a transform (a symmetric kernel given as
 * V = diag(s) U^T, as smol_lowrank_kernel returns it, has T = R), so smol_init_system
 * accepts up to this M for the factors' actual T. Returns 0 for an unsupported T. */
int64_t smol_max_m_transforms(int32_t T, int32_t precision);

/* Bytes of device workspace a system of size M, rank R needs under opts (NULL =
 * defaults). The workspace must stay allocated, untouched by the caller and
 * unused by other systems until smol_destroy. Returns 0 for an unsupported shape. */
size_t smol_workspace_bytes(int64_t M, int32_t R, const smol_opts* opts);

/* Creates a system for Eq. (4) with kernel K = U V and shattering rate lambda.
 *   h_U: host, M x R row-major (U[(s-1)*R + alpha] = U_{s,alpha}); copied.
 *   h_V: host, R x M row-major (V[alpha*M + (s-1)] = V_{alpha,s});  copied.
 *   lambda >= 0. opts may be NULL (defaults); it is copied.
 *   d_workspace: device, >= smol_workspace_bytes(M, R, opts) bytes, 256-byte aligned.
 * Columns of U and rows of V that are equal up to a constant factor share one
 * forward transform. Synchronises the stream once (tables are uploaded).
 * Errors: SMOL_EINVAL, SMOL_ENOSPACE, SMOL_EUNSUPPORTED, SMOL_ECUDA. */
int smol_init_system(smol_system** sys, int64_t M, int32_t R, const double* h_U,
                     const double* h_V, double lambda, const smol_opts* opts,
                     void* d_workspace, size_t workspace_bytes);

/* Re-targets the stream of later calls. */
int smol_set_stream(smol_system* sys, void* stream);

/* out = S(n), Eq. (4)-(5), FP64 in and out (d_n and d_out: device, M doubles each;
 * they may not overlap). Stream-ordered; does not synchronise. */
int smol_rhs(smol_system* sys, const double* d_n, double* d_out);

/* The terms of S(n) separately (device, M doubles each; any may be NULL):
 *   d_birth[s-1] = 1/2 sum_{i+j=s} K_ij n_i n_j          (0 for s = 1)
 *   d_loss[s-1]  = (1 + lambda [s>=2]) n_s sum_i K_si n_i (aggregation + shattering loss)
 *   d_source[0]  = monomer source from shattering (a single double)
 * so that S = birth - loss, plus source at s = 1. */
int smol_rhs_terms(smol_system* sys, const double* d_n, double* d_birth, double* d_loss,
                   double* d_source);

/* Integrates Eq. (5) from t0 to t1 with the given scheme (SMOL_RK2 / SMOL_RK4 /
 * SMOL_RKF45) and tolerance tol (> 0), starting from d_n (device, M doubles), and
 * writes n(t_end) back to d_n. Step control runs on the device; the host launches
 * captured CUDA graphs of opts.chunk attempts and reads a status block between
 * launches. A rejected attempt is repeated from the same n^k (Sec. 2), so the retry
 * keeps the first stage S(n^k) of the rejected attempt (rescaled to the new step)
 * instead of evaluating it again; stats->rhs_evals counts the evaluations made.
 * Returns the final status (SMOL_OK or SMOL_STEADY on success) and fills *stats when
 * non-NULL. */
int smol_integrate(smol_system* sys, double* d_n, double t0, double t1, double tol,
                   int32_t scheme, smol_stats* stats);

/* The same integration split into asynchronous parts, for callers that interleave it
 * with their own work or time it with CUDA events:
 *   smol_integrate_start:   validates, uploads the control block, enqueues the first-
 *                           step computation and (once per scheme / chunk size) captures
 *                           the CUDA graph of min(opts.chunk, opts.max_attempts) attempts.
 *                           Synchronises the stream once; d_n must stay valid until
 *                           smol_integrate_finish.
 *   smol_integrate_advance: enqueues one graph launch (that many attempts) on the
 *                           stream and returns at once. Attempts after termination
 *                           (t1 reached or a status set) do no work.
 *   smol_integrate_finish:  writes the state back to d_n (on the device), synchronises
 *                           the stream once and fills *stats; returns the status like
 *                           smol_integrate. Further smol_integrate_advance calls then
 *                           continue the same run from d_n.
 * smol_integrate is start + advance until done + finish. */
int smol_integrate_start(smol_system* sys, double* d_n, double t0, double t1, double tol, int32_t scheme);
int smol_integrate_advance(smol_system* sys);
int smol_integrate_finish(smol_system* sys, smol_stats* stats);

/* Kernel classes reported by smol_profile_attempts. */
#define SMOL_PROF_FWD_COLS 0   /* stage input, moments, forward column FFTs */
#define SMOL_PROF_ROWS     1   /* row FFTs, spectral product sum, inverse row FFTs */
#define SMOL_PROF_INV_COLS 2   /* inverse column FFTs and the right-hand-side epilogue */
#define SMOL_PROF_STEP     3   /* RK combination, error norm and step control */
#define SMOL_PROF_INV_FWD  4   /* fused: inverse columns of one evaluation + forward columns of the next */
#define SMOL_PROF_INV_STEP 5   /* fused: inverse columns of the last evaluation + combination and control */
#define SMOL_PROF_KINDS    6

/* Measurement aid: runs `reps` further attempts of the current run (between
 * smol_integrate_start and smol_integrate_finish) launched one kernel at a time with
 * CUDA events around each kernel on the system's stream, and returns the average
 * duration in milliseconds of each kernel class in kernel_ms[SMOL_PROF_KINDS] and the
 * number of launches timed in kernel_launches (may be NULL). Synchronises per attempt. */
int smol_profile_attempts(smol_system* sys, int32_t reps, double* kernel_ms, int64_t* kernel_launches,
                          int32_t nkinds);

/* Measurement aid: the fused multiply-add rate of this GPU in FP64 (precision =
 * SMOL_FP64) or FP32 (SMOL_FP32CONV), the arithmetic ceiling that the right-hand side's
 * transforms are reported against (the paper gives no hardware figures; it only states
 * the O(M R log M) cost of the FFT route, Sec. 1). Runs 4 CTAs of 256 threads per SM,
 * each thread 8 independent chains of `iters` dependent fused multiply-adds, once to
 * warm up and once timed with CUDA events on `stream` (cudaStream_t or NULL); returns
 * *tflops = 2 x 8 x iters x threads / time (FMA = 2 flop) and, when non-NULL, *ms the
 * timed kernel's duration. Synchronises the stream. SMOL_EINVAL or SMOL_ECUDA on error. */
int smol_fma_rate(int32_t precision, int64_t iters, void* stream, double* tflops, double* ms);

/* Measurement aid: SM clock cycles per operation of a chain of dependent operations op
 * (0: FP64 fused multiply-add, 1: FP64 add, 2: FP32 fused multiply-add, 3: FP32 -> FP64
 * conversion plus an FP64 multiply), run by `warps` (1..32) warps of one CTA at once, as
 * warp 0 times it with clock64. With one warp this is the operation's latency; with
 * several, the FP64 pipe's throughput shows once they contend. Synchronises `stream`.
 * SMOL_EINVAL or SMOL_ECUDA on error. */
int smol_op_latency(int32_t op, int32_t warps, void* stream, double* cycles);

/* Constant point sources of Eq. (3): dn_s/dt = S_s(n) + P_s at up to SMOL_MAX_SOURCES
 * sizes (Sec. 3.1 injects P_1 = 1 and P_100 = p). With lambda = 0 the system is Eq. (3);
 * with lambda > 0 the sources are added to Eq. (4). sizes are 1-based (1..M), values
 * finite; count = 0 removes them. They enter S(n) (smol_rhs and the integrators; for
 * s = 1 through the FP64 monomer equation) but not the separate terms of
 * smol_rhs_terms. They apply from the next smol_integrate / smol_integrate_start; a run
 * started before cannot then be continued with smol_integrate_advance (which returns
 * SMOL_EINVAL until the next start). Returns SMOL_OK or SMOL_EINVAL. */
#define SMOL_MAX_SOURCES 8
int smol_set_sources(smol_system* sys, int32_t count, const int64_t* sizes, const double* values);

/* Schedule autotuner (the FFT schedule and the launch mode are implementation choices
 * that the paper leaves open: it only states the O(M R log M) cost of the FFT route,
 * Sec. 1). For one system of the given problem it times `attempts` step attempts of
 * `scheme` at tolerance tol, after one warm-up chunk, for each candidate schedule:
 *   - log2 N1 of the four-step split Mp = N1 N2: the rule's value, one above it and
 *     two below;
 *   - columns per CTA of the column kernels: the rule's value and 2, 4 and 8 times it
 *     (at most 64);
 *   - launch mode: programmatic dependent launch for every kernel, for none, or for
 *     all but the forward column kernel; fused column passes (default) or not; for
 *     RKF45 also the persistent attempt kernel (SMOL_FLAG_PERSISTENT).
 * Candidates whose shared memory does not fit are skipped. *opts is read as the base
 * options and receives the fastest schedule in fft_lgn1, fft_g and flags (its other
 * fields are unchanged); *us_per_attempt (may be NULL) that schedule's microseconds
 * per attempt. d_n0 (device, M doubles, 16-byte aligned) is the state the attempts
 * start from; it is not modified. Allocates and frees its own device memory and
 * synchronises: a set-up call, not for timed regions. Returns SMOL_OK, SMOL_EINVAL,
 * SMOL_EUNSUPPORTED, or SMOL_ECUDA when no candidate could be timed (e.g. the
 * integration stopped with an error status during every timing). */
int smol_tune(int64_t M, int32_t R, const double* h_U, const double* h_V, double lambda,
              const double* d_n0, double tol, int32_t scheme, int32_t attempts, smol_opts* opts,
              double* us_per_attempt);

/* Copies the step log of the last smol_integrate (the most recent min(count, cap)
 * attempts, oldest first) to host arrays of cap entries each (any may be NULL).
 * *count receives the number of attempts made. */
int smol_get_log(smol_system* sys, double* h_t, double* h_tau, double* h_err,
                 int32_t* h_accepted, int32_t cap, int64_t* count);

/* First step of the next integration (Sec. 2 leaves the initial step to the user; the
 * Euler criterion of Sec. 1 is the default): tau0 > 0 replaces opts.tau0 for later
 * smol_integrate / smol_integrate_start calls of this system, tau0 = 0 restores it.
 * A run resumed from a checkpoint with tau0 = the previous call's stats.tau_next
 * continues the step sequence it would have taken. Takes effect at the next
 * smol_integrate / smol_integrate_start (a run already started keeps its step).
 * Returns SMOL_OK or SMOL_EINVAL. */
int smol_set_tau0(smol_system* sys, double tau0);

/* Number of distinct forward transforms T used per evaluation (<= 2R). */
int smol_num_transforms(const smol_system* sys);

/* ---- Batches of independent systems -------------------------------------------
 * `count` independent systems of Eq. (4) with their own size M[q], kernel factors
 * h_U[q] (M[q] x R) and h_V[q] (R x M[q]) and shattering rate lambda[q], sharing R,
 * the options and the tolerance. Every kernel launch of an integration spans all
 * systems (ragged block maps); each system keeps its own t, tau, controller state and
 * status, and stops on its own. Arguments follow the single-system calls; d_n is a
 * host array of `count` device pointers; stats (when non-NULL) has `count` entries.
 * smol_batch_integrate returns the first error status of any system, else SMOL_STEADY
 * if some system stopped at a steady state, else SMOL_OK. */
typedef struct smol_batch smol_batch;
size_t smol_batch_workspace_bytes(int32_t count, const int64_t* M, int32_t R, const smol_opts* opts);
int smol_batch_init(smol_batch** batch, int32_t count, const int64_t* M, int32_t R,
                    const double* const* h_U, const double* const* h_V, const double* lambda,
                    const smol_opts* opts, void* d_workspace, size_t workspace_bytes);
int smol_batch_set_stream(smol_batch* batch, void* stream);
int smol_batch_integrate(smol_batch* batch, double* const* d_n, double t0, double t1, double tol,
                         int32_t scheme, smol_stats* stats);
int smol_batch_integrate_start(smol_batch* batch, double* const* d_n, double t0, double t1,
                               double tol, int32_t scheme);
int smol_batch_integrate_advance(smol_batch* batch);
int smol_batch_integrate_finish(smol_batch* batch, smol_stats* stats);
/* Launch-mode autotuner of a batch (its FFT schedules are those it was initialised with:
 * the rule, or the tables of smol_batch_tune_schedules): times
 * `attempts` attempts of every system from copies of the states d_n[q] (not modified)
 * for each launch mode that smol_tune tries, keeps the fastest for later integrations
 * of this batch and returns its flags in *flags and its microseconds per attempt of the
 * whole batch in *us_per_attempt (either may be NULL). A run started before cannot be
 * continued afterwards (start a new one). */
/* Per-system first steps of the next batch integration (as smol_set_tau0): h_tau0
 * (host, count entries) each > 0, or 0 for the batch's opts.tau0. */
int smol_batch_set_tau0(smol_batch* batch, const double* h_tau0);
/* The point sources of system `system` of a batch (as smol_set_sources). */
int smol_batch_set_sources(smol_batch* batch, int32_t system, int32_t count, const int64_t* sizes,
                           const double* values);

/* Partition of a batch across nranks GPUs (host code; no GPU needed). The systems are
 * independent (Sec. 3 integrates each on its own), so a batch shards with no exchange in
 * the integration: each rank advances its own systems and the states and stats are
 * gathered once at the end. System q costs weight[q] x Mp log2 Mp per attempt (Mp = the
 * FFT size; weight: expected attempts, NULL = 1). Longest-processing-time-first
 * assignment: systems by decreasing cost, each to the least-loaded rank, ties to the
 * lower index; the makespan is within 4/3 of the optimum. rank_of[count] receives the
 * rank of each system, load[nranks] (may be NULL) each rank's total cost. Deterministic:
 * every rank computes the same partition. Returns SMOL_OK or SMOL_EINVAL. */
int smol_partition(int32_t count, const int64_t* M, const double* weight, int32_t nranks,
                   int32_t* rank_of, double* load);

int smol_batch_tune(smol_batch* batch, double* const* d_n, double tol, int32_t scheme,
                    int32_t attempts, int32_t* flags, double* us_per_attempt);

/* FFT schedules per size class for a batch: smol_tune's search applied to the batched
 * form (Sec. 3 integrates each system on its own; each keeps the FFT route of Sec. 1,
 * only the split Mp = N1 N2 and the columns per CTA change). Coordinate descent over the size
 * classes present, the class holding the most sizes first: for each, the candidates
 * log2 N1 = rule - 2 ... rule + 1 with 1, 2, 4 and 8 times the rule's columns per CTA
 * are timed on the whole batch (`attempts` attempts from the states d_n0 on scratch
 * copies; nothing of the caller's changes), with the other classes at their best so
 * far. The arguments are those of smol_batch_workspace_bytes / smol_batch_init plus the
 * states; *opts gives the precision, launch flags and starting tables, and receives the
 * chosen batch_lgn1 / batch_g (its other fields unchanged). The caller then sizes and
 * initialises the batch with *opts. Allocates and frees its own scratch (workspaces and
 * state copies). *us_per_attempt (may be NULL): the time of an attempt of the whole
 * batch with the chosen tables. SMOL_EINVAL, SMOL_EUNSUPPORTED or SMOL_ECUDA. */
int smol_batch_tune_schedules(int32_t count, const int64_t* M, int32_t R, const double* const* h_U,
                              const double* const* h_V, const double* lambda, double* const* d_n0,
                              double tol, int32_t scheme, int32_t attempts, smol_opts* opts,
                              double* us_per_attempt);
int smol_batch_get_log(smol_batch* batch, int32_t system, double* h_t, double* h_tau,
                       double* h_err, int32_t* h_accepted, int32_t cap, int64_t* count);
void smol_batch_destroy(smol_batch* batch);

/* No-allocation evaluation of S(n), FP64. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory or hand over a
 * workspace (code running while a CUDA graph is captured, hosts without a device
 * allocator, plug-ins that do not own the process's memory). It needs no system object
 * and calls no cudaMalloc / cudaFree or allocating library routine.
 *   M <= SMOL_STATIC_MAX_M, 1 <= R <= SMOL_STATIC_MAX_R, lambda >= 0.
 *   d_U: device, M x R row-major; d_V: device, R x M row-major; d_n, d_out: device,
 *   M doubles each, 16-byte aligned, not overlapping. stream: cudaStream_t or NULL.
 * Its scratch memory is a fixed device array of 15,321,344 bytes inside the library,
 * which every GPU that loads the library holds until exit. The first call on a device
 * looks up that array's device address and sets kernel attributes (once per device);
 * make that first call before any stream capture. All calls on a device share the
 * array, which keeps the last call's contents: calls that overlap on the GPU race and
 * must be serialised by the caller. Every call transforms U and V afresh (no
 * sharing of proportional factors). Returns SMOL_EUNSUPPORTED beyond the limits,
 * SMOL_EINVAL for bad pointers; does not synchronise. */
#define SMOL_STATIC_MAX_M 65536
#define SMOL_STATIC_MAX_R 3
int smol_rhs_static(int64_t M, int32_t R, const double* d_U, const double* d_V, double lambda,
                    const double* d_n, double* d_out, void* stream);

/* Collision kernels of Sec. 3.1 for smol_lowrank_kernel (sizes i, j >= 1):
 *   SMOL_KERNEL_CONST:          K_ij = 1
 *   SMOL_KERNEL_BROWNIAN:       K_ij = (i/j)^a + (j/i)^a + c, params = {a, c}
 *   SMOL_KERNEL_FREE_MOLECULAR: K_ij = (i^{1/3} + j^{1/3})^2 sqrt(1/i + 1/j)
 * The first two have exact ranks 1 and <= 3; the free-molecular kernel has no exact low
 * rank and is approximated. */
#define SMOL_KERNEL_CONST          0
#define SMOL_KERNEL_BROWNIAN       1
#define SMOL_KERNEL_FREE_MOLECULAR 2

/* Low-rank factors K ~= U V of a symmetric kernel on sizes 1..M (host code, no GPU), so
 * that the O(M R log M) right-hand side of Sec. 1 applies to a kernel without an exact
 * low rank; the paper takes such factors from a cross approximation (Sec. 1 and its
 * reference on the fast evaluation). Symmetric adaptive cross approximation of
 * D^-1 K D^-1, D = diag(sqrt |K_ii|), with diagonal pivots (Bunch-Kaufman 2 x 2 pivots
 * where a diagonal pivot is too small), until the residual is below tol relative to the
 * scaled matrix or max_rank terms are taken.
 *   params: kernel parameters (SMOL_KERNEL_BROWNIAN: {a, c}; may be NULL otherwise).
 *   h_U: host, >= M * max_rank doubles: receives U as M x R row-major (R = *rank);
 *   h_V: host, >= max_rank * M doubles: receives V as R x M row-major, V = diag(s) U^T
 *        with signs s = +-1 (so the factors share their R transforms: T = R).
 *   *err_est (may be NULL): max |K^ - K| / |K| over the first and last 8 rows and every
 *        ceil(M/64)-th row, all columns (exact kernel entries).
 * Returns SMOL_OK or SMOL_EINVAL (bad kind, M < 1, tol <= 0, max_rank < 1, NULL). */
int smol_lowrank_kernel(int32_t kind, const double* params, int64_t M, double tol, int32_t max_rank,
                        double* h_U, double* h_V, int32_t* rank, double* err_est);

/* Releases the system (not the workspace). Safe on NULL. */
void smol_destroy(smol_system* sys);

/* Static description of a status code. */
const char* smol_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* SMOL_H */
