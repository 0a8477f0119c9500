/*
 * sqrtba.h - C ABI of the GB300 (sm_103a) square root bundle adjustment
 * library (Demmel, Sommer, Cremers, Usenko: "Square Root Bundle Adjustment
 * for Large-Scale Reconstruction", CVPR 2021).
 *
 * The problem (Sec. 4): minimise E = sum_ij ||r_ij||^2 (Eq. ba_energy) over
 * n_cam cameras with d_p = 9 parameters each and n_pt 3-D landmarks, by
 * Levenberg-Marquardt on the damped linearised problem of
 * Eq. linearized_residual.  Landmarks are eliminated by nullspace
 * marginalisation (Sec. 4.3): every landmark's dense block [J_p | J_l | r]
 * (Sec. 5.1, Fig. 2) is QR-factored in place by three Householder
 * reflections (Sec. 5.2), landmark damping is folded in by six stored Givens
 * rotations (Sec. 5.3, Fig. 3), and the reduced camera system is solved by
 * block-Jacobi preconditioned CG on the normal equations through the stored
 * Q2^T J_p blocks (Sec. 5.4, Eq. cg_mult); landmarks are then recovered by
 * back substitution (Eq. backsub_nm).  All marginalisation and PCG arithmetic
 * is FP32 (Sec. 6.1, "sqrt BA-32"); the global cost sum, the model cost and
 * the LM gain ratio are accumulated in FP64 (each observation's term is formed
 * in FP32 and added to the FP64 sum).
 *
 * Conventions for every call
 *   - Camera layout (BAL, Sec. 6.2): 9 doubles per camera, row-major:
 *     axis-angle w[3], translation t[3], focal length f, radial k1, k2.
 *     P = R(w) X + t; points in front have P_z < 0; p = -P_xy / P_z;
 *     pixel = f (1 + k1 |p|^2 + k2 |p|^4) p; residual = pixel - observation.
 *   - Landmarks: 3 doubles each.  Observations: obs_cam[o], obs_pt[o] index
 *     the camera and landmark of observation o, obs_xy[2 o + 0/1] its pixel.
 *   - Host pointers are read during the call only; the library copies what
 *     it needs.  The library owns all device memory of a problem.
 *   - Work is issued in stream order on the CUDA stream given to ba_create
 *     (NULL = the library creates its own); a call that returns a scalar
 *     synchronises that stream.
 *   - Every call returns a ba_status; nothing throws across the ABI.  After a
 *     failure, ba_last_error() describes it.  A handle is used by one host
 *     thread at a time.
 */
#ifndef SQRTBA_H
#define SQRTBA_H

#include <stdint.h>

#if defined(__GNUC__)
#define SQRTBA_API __attribute__((visibility("default")))
#else
#define SQRTBA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ba_problem ba_problem; /* opaque */

typedef enum {
    BA_OK = 0,
    BA_ERR_INVALID_ARG = 1, /* bad index, non-finite value, landmark with < 2 observations,
                               duplicate (camera, landmark) pair, null pointer */
    BA_ERR_OOM = 2,         /* device allocation failed */
    BA_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    BA_ERR_STATE = 4,       /* calls out of order (e.g. PCG before marginalisation) */
    BA_ERR_NUMERIC = 5,     /* reserved: no call returns it (a preconditioner block that is not
                               positive definite is replaced by its diagonal and counted in
                               ba_pcg_report.precond_fallbacks; a non-finite candidate cost
                               rejects the LM step) */
    BA_ERR_TIMEOUT = 6      /* a bounded device-side wait gave up (2 s): the kernel returned
                               early and the results of the call are invalid.  Kernels record
                               it in an error word that the library reads back at the call's
                               synchronisation (or at the next call that synchronises), then
                               clears, so that the handle stays usable */
} ba_status;

/* Solver settings (Sec. 6.1 gives lambda0, the iteration limits and the
 * function tolerance). */
typedef struct {
    double lambda0;       /* initial LM damping, default 1e-4 */
    int32_t max_lm_iters; /* default 50; every linear solve counts as one iteration */
    double func_tol;      /* relative cost-change stop on an accepted step, default 1e-6 */
    int32_t max_cg_iters; /* default 500 */
    double cg_eta;        /* Nash-Sofer forcing tolerance, default 0.1 */
    int32_t use_graph;    /* 1 (default): PCG iterations replayed from a CUDA graph */
    int32_t autotune;     /* 1: the first PCG solve first runs the matvec autotuner
                             (ba_autotune); default 0 */
    int32_t use_learned;  /* 1: PCG with the learned warm start and corrected block
                             preconditioner of the model attached by ba_set_learned */
    int32_t pipeline_stages; /* 0 (default): the K3 / K4 tile pipeline runs 6 stages, or the
                             depths the autotuner chose; 4, 5 or 6 forces that depth */
    double target_cost;   /* > 0: the LM also stops after an accepted step whose cost is
                             <= target_cost (e.g. the f_tau of a tolerance test); default 0 */
    int32_t precond_from_blocks; /* 0 (default): the block-Jacobi blocks and g come from the
                             Gram identity (J_s^T J_s - T_s^T T_s per observation, see
                             ba_pcg_solve), except for cameras where that difference would
                             cancel (then from A_j; counted in ba_pcg_report.precond_exact);
                             1: summed from the stored blocks A_j, as the matvec reads them */
    int32_t implicit_blocks; /* 0 (default): Q2^T J_p is stored per landmark (2k x 9k floats,
                             Sec. 5.1).  1: the factorisation is stored instead (per
                             observation J_s and its Householder rows, per landmark the
                             compact-WY factor, R1, Q1^T r, P = V[0:3, :] Tm^T and the
                             damping rotations' effect, O(k) memory, the variant of
                             Table tab:complexities' storage discussion); products with
                             A_j are formed on the fly in K4, the top rows in K3 and K6.
                             Same results up to rounding; ba_debug_export_landmark then
                             exports only the undamped top rows, rebuilt from the records */
    double huber_delta;   /* > 0: robust norm (Sec. 6.2: Huber, 1 px there) by iteratively
                             reweighted least squares: E = sum rho(||r_ij||^2) with
                             rho(s) = s (s <= delta^2), 2 delta sqrt(s) - delta^2 (above);
                             each observation's rows [J | r] are scaled by sqrt(w),
                             w = min(1, delta / ||r_ij||), and the model cost is
                             sum rho(s) - w s + w ||r + J dx||^2.  0 (default): squared norm */
    int32_t schur_explicit; /* 1: the comparison solver of Sec. 6.4 ("explicit-32"): the reduced
                             camera system H~ = H_pp - H_pl (H_ll + lambda D_l^2)^-1 H_lp is formed
                             explicitly in FP32 at every damping (Sec. 4.2, Eq. red_normal_eq) and
                             solved by the same block-Jacobi PCG; landmarks by Eq. backsub_sc.
                             Kept to test the paper's claim that this form loses positive
                             definiteness in FP32 where the square-root form does not.
                             Excludes implicit_blocks.  0 (default): square root BA */
    int32_t reserved;     /* zero */
} ba_options;

/* Fills *opt with the defaults above. */
SQRTBA_API void ba_default_options(ba_options* opt);

typedef struct {
    int32_t iterations;   /* CG iterations performed */
    int32_t stop_reason;  /* 0 forcing test, 1 residual, 2 iteration limit, 3 breakdown, 4 zero rhs */
    double residual_norm; /* ||g - H~ x|| by the CG recursion */
    double rhs_norm;      /* ||g|| */
    int32_t learned;      /* 1 if the learned warm start / preconditioner was used */
    int32_t warm_start;   /* 1 if the learned warm start was kept (see ba_set_learned) */
    int32_t precond_fallbacks; /* block-Jacobi blocks that were not numerically positive
                             definite in FP32 and were replaced by their diagonal */
    int32_t precond_exact; /* Gram form only: cameras whose block and g were summed from the
                             stored blocks A_j because the Gram identity would cancel
                             (sum_s ||J_s||_F^2 > 64 tr(M_i)) */
} ba_pcg_report;

typedef struct {
    int32_t iteration;    /* 0-based index of this LM iteration */
    int32_t accepted;     /* 1 if the candidate replaced the state */
    int32_t relinearized; /* 1 if this iteration linearised (K1) */
    int32_t cg_iters;
    int32_t stop;         /* 1: LM terminated on this iteration (tolerance, lambda overflow) */
    int32_t pcg_stop_reason;
    double cost;          /* E at the state the iteration started from */
    double new_cost;      /* E at the candidate x (+) dx */
    double model_cost;    /* ||r + J dx||^2, undamped Gauss-Newton model */
    double lambda;        /* damping used */
    double rho;           /* (cost - new_cost) / (cost - model_cost) */
    int32_t precond_fallbacks; /* as in ba_pcg_report, for this iteration's solve */
    int32_t precond_exact;     /* as in ba_pcg_report, for this iteration's solve */
} ba_lm_report;

/* Creates a problem from host FP64 arrays (layouts above).  Observations are
 * validated and grouped by landmark on the device (Sec. 5.1).
 * Errors: BA_ERR_INVALID_ARG for n_cam < 1, n_pt < 1, n_obs < 2, an index out
 * of range, a non-finite value, a landmark with fewer than two observations
 * or a duplicate (camera, landmark) pair; BA_ERR_OOM; BA_ERR_CUDA.
 * cuda_stream: a cudaStream_t (e.g. a PyTorch stream) or NULL.
 * On success *out owns the problem; release it with ba_destroy. */
SQRTBA_API ba_status ba_create(const double* cams, int32_t n_cam, const double* pts, int32_t n_pt,
                    const int32_t* obs_cam, const int32_t* obs_pt, const double* obs_xy,
                    int64_t n_obs, const ba_options* opt, void* cuda_stream,
                    ba_problem** out);

/* Releases all device and host memory of a problem.  NULL is a no-op. */
SQRTBA_API ba_status ba_destroy(ba_problem* h);

/* Linearises at the current state (Sec. 4.1) and marginalises every landmark
 * (Sec. 4.3, 5.2): residuals and analytic Jacobians, D^2 = clamp(diag(J^T J),
 * 1e-6, 1e32), three Householder reflections per landmark block applied to
 * [J_p | r]; stores R1, Q1^T J_p, Q1^T r, Q2^T J_p, Q2^T r.  Leaves the blocks
 * undamped.  Also evaluates the cost at the current state. */
SQRTBA_API ba_status ba_linearize(ba_problem* h);

/* ba_linearize followed by ba_marginalize_qr(lambda) in one call (the
 * damping kernel runs straight after the factorisation, no undo needed).
 * Errors: BA_ERR_INVALID_ARG if lambda <= 0 or not finite. */
SQRTBA_API ba_status ba_linearize_damped(ba_problem* h, double lambda);

/* Applies landmark damping sqrt(lambda) D_l with six Givens rotations per
 * landmark block (Sec. 5.3, Fig. 3 a-b), first undoing the previous damping
 * with the stored rotations if the blocks are damped (Fig. 3 c).
 * Errors: BA_ERR_STATE if not linearised; BA_ERR_INVALID_ARG if lambda <= 0
 * or not finite. */
SQRTBA_API ba_status ba_marginalize_qr(ba_problem* h, double lambda);

/* Solves the damped reduced camera system H~ dx_p = -b~ with block-Jacobi
 * PCG (Sec. 5.4, Eq. cg_mult; Sec. 6.1): builds the per-camera 9x9 blocks of
 * H~ and g = -b~, then iterates the matvec
 * (Q2^T J_p)^T (Q2^T J_p v) + lambda D_p^2 v.  Stops by the Nash-Sofer test
 * with cg_eta, ||r|| <= 1e-10 ||g||, or max_cg_iters.  report may be NULL.
 * The blocks are sum_j A_ji^T A_ji over the landmarks camera i observes, and
 * b~_i = sum_j A_ji^T c_j (Eq. red_H, red_b).  The QR and Givens transforms
 * keep the Gram matrix of a block's pose and residual columns, so each term
 * equals J_s^T J_s - T_s^T T_s (and J_s^T r_s - T_s^T t) with J_s, r_s the
 * observation's Jacobian rows and residuals and T_s, t its columns of the
 * damped top rows [Q1^T J_p | R1 | Q1^T r]; by default the blocks are formed
 * that way (30 floats read per observation; in the implicit storage T_s is
 * rebuilt from the observation's Householder rows and its landmark's record),
 * with precond_from_blocks = 1 from the stored A_j and c_j (18 k floats per
 * observation).
 * Errors: BA_ERR_STATE if not marginalised. */
SQRTBA_API ba_status ba_pcg_solve(ba_problem* h, ba_pcg_report* report);

/* Back substitution dx_l = -R1^-1 (Q1^T r + Q1^T J_p dx_p) per landmark
 * (Eq. backsub_nm, damped), then *model_cost = ||r + J dx||^2 (FP64 sum).
 * Errors: BA_ERR_STATE if no PCG solution is present. */
SQRTBA_API ba_status ba_backsubstitute(ba_problem* h, double* model_cost);

/* *cost = E (Eq. ba_energy, FP64 sum of the FP32 terms ||r||^2) at the current state
 * (candidate = 0) or at the candidate x (+) dx (candidate = 1; rotation
 * updated as Exp(dw) R, everything else additively).
 * Errors: BA_ERR_STATE for candidate = 1 without a back-substituted step. */
SQRTBA_API ba_status ba_eval_cost(ba_problem* h, int32_t candidate, double* cost);

/* One Levenberg-Marquardt iteration (Sec. 6.1): linearise if needed,
 * marginalise with the current lambda, PCG, back substitution, candidate
 * cost, FP64 gain ratio, accept or reject and update lambda (Nielsen).  A
 * rejected step keeps the linearisation, so the next call only re-damps.
 * report may be NULL.  Returns BA_ERR_STATE once the LM has stopped. */
SQRTBA_API ba_status ba_lm_step(ba_problem* h, ba_lm_report* report);

/* Runs ba_lm_step until stop or max_lm_iters.  reports (may be NULL) has
 * room for max_reports entries; *n_reports (may be NULL) gets the count. */
SQRTBA_API ba_status ba_solve(ba_problem* h, ba_lm_report* reports, int32_t max_reports,
                   int32_t* n_reports);

/* Copies the current state to host FP64 arrays (cams: 9 n_cam, pts: 3 n_pt);
 * either pointer may be NULL.  The FP32 state is copied through one
 * process-wide page-locked staging buffer (grown to the largest state read,
 * kept for the life of the process; concurrent calls take turns). */
SQRTBA_API ba_status ba_get_params(ba_problem* h, double* cams, double* pts);

/* Replaces the state (host FP64 arrays, same layout), resets lambda to
 * lambda0 and the LM iteration counter, and marks the linearisation stale. */
SQRTBA_API ba_status ba_set_params(ba_problem* h, const double* cams, const double* pts);

/* Replaces the solver settings of a problem (validated as by ba_create);
 * the next LM step and solve use them. */
SQRTBA_API ba_status ba_set_options(ba_problem* h, const ba_options* opt);

/* Checkpoint of the LM state besides the parameters. */
typedef struct {
    double lambda;
    double nu;
    int32_t iteration;
    int32_t stopped;
} ba_lm_state;
SQRTBA_API ba_status ba_get_state(ba_problem* h, ba_lm_state* state);
SQRTBA_API ba_status ba_set_state(ba_problem* h, const ba_lm_state* state);

/* Sizes: n_cam, n_pt, n_obs, the number of FP32 values in the stored
 * Q2^T J_p blocks (sum over landmarks of 2k x 9k, each block padded to a
 * multiple of 4) and the total device bytes the problem holds. */
typedef struct {
    int32_t n_cam;
    int32_t n_pt;
    int64_t n_obs;
    int64_t a_pool_floats;
    int64_t sum_k2;
    int32_t k_max;
    int32_t reserved;
    int64_t device_bytes;
} ba_info;
SQRTBA_API ba_status ba_get_info(ba_problem* h, ba_info* info);

/* Timing of the phases of the hot path with CUDA events on the problem's
 * stream, and transfer / launch counters.  Slots of ms[] and count[]:
 *   0 linearisation + Householder QR (K1, with the D_p^2 kernel)
 *   1 landmark damping (K2)   2 preconditioner + right-hand side (K3)
 *   3 PCG matvec, one entry per launch (K4)   4 unused
 *   5 back substitution + model cost (K6)   6 cost evaluations (K7)
 * ms[i] is the summed duration, count[i] the number of timed intervals.
 * kernel_launches counts every kernel the library launched (a replayed
 * graph counts its kernels); h2d_bytes / d2h_bytes count the bytes copied
 * between host and device.  All counters restart at ba_set_profiling. */
typedef struct {
    double ms[8];
    int64_t count[8];
    int64_t kernel_launches;
    int64_t h2d_bytes;
    int64_t d2h_bytes;
} ba_profile;

/* enable != 0 turns event timing on (adds event records around the phases,
 * including event nodes inside the PCG graph); resets all counters. */
SQRTBA_API ba_status ba_set_profiling(ba_problem* h, int32_t enable);
SQRTBA_API ba_status ba_get_profile(ba_problem* h, ba_profile* out);

/* Human-readable description of the last failure on this handle (never
 * NULL; "" when none).  With h = NULL: the last failure of ba_create. */
SQRTBA_API const char* ba_last_error(const ba_problem* h);

/* Energy E = sum ||r||^2 (FP64 sum of FP32 residuals) of device-resident
 * FP32 data, without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate -
 * latency-critical loops in which cudaMalloc / cudaFree would synchronise
 * the device, and programs whose device memory is entirely owned by another
 * allocator (a framework's caching allocator, a fixed arena sized at start).
 *   d_cams [9 n_cam], d_pts [3 n_pt], d_obs_cam / d_obs_pt [n_obs],
 *   d_obs_xy [2 n_obs]: device pointers, any observation order, caller-owned.
 *   d_cost: device pointer to one double that receives E.
 * Work is enqueued on cuda_stream (NULL = legacy default stream) and the call
 * returns without synchronising.  The per-block partial sums live in a fixed
 * 128 KiB device array inside the library (16384 doubles), held by every
 * device that loads the library until the process exits; hence n_obs is
 * limited to 16384 * 1024 = 16,777,216 (larger: BA_ERR_INVALID_ARG with a
 * message in ba_last_error(NULL)).  The first call on a device looks up that
 * array's device address (a one-time set-up per device, with the device
 * current), so make that first call before any stream capture; the address
 * is kept for the life of the process, so a device reset (cudaDeviceReset)
 * after the first call is not supported.  cuda_stream must belong to the
 * current device (else BA_ERR_INVALID_ARG).  All calls share the array:
 * calls that overlap on the GPU (other streams or threads) race and must be
 * serialised by the caller.  An observation index out of range makes the
 * result NaN; no out-of-range access is made. */
SQRTBA_API ba_status ba_eval_cost_noalloc(const float* d_cams, int32_t n_cam, const float* d_pts,
                                          int32_t n_pt, const int32_t* d_obs_cam,
                                          const int32_t* d_obs_pt, const float* d_obs_xy,
                                          int64_t n_obs, double* d_cost, void* cuda_stream);

/* ---------------------------------------------------------------------- */
/* Autotuner of the K4 matvec work plan.                                   */
/* ---------------------------------------------------------------------- */

/* The matvec (K4) and the preconditioner's record pass (K3) stream the
 * landmark blocks, stored by decreasing k, as tiles: blocks with k <= ksmall
 * are grouped into tiles of up to small_bytes (specialised code per k),
 * larger blocks are cut into row tiles.  The tuner times the matvec (and,
 * with precond_from_blocks = 1, the record pass) on the current damped blocks
 * for ksmall in {8, 13, 21} and small_bytes in {8192, 16384, 32768} (median
 * of five launches each, CUDA events on the problem's stream, a non-zero
 * input), keeps the fastest plan of each, then times that plan with 4, 5 and
 * 6 pipeline stages (the matvec also with y accumulated in global instead of
 * shared memory) and keeps the fastest depth, then (when some blocks are cut
 * into row tiles) the largest k whose row tiles take eight rows a warp.  It
 * reports the choices; the record pass's fields report its plan in use when
 * it is not tuned.  The paper parallelises over landmarks with a
 * parallel-for (Sec. 6.1) and has no tuner.
 * Errors: BA_ERR_STATE if the blocks are not marginalised. */
typedef struct {
    int32_t ksmall;       /* chosen bucket limit of the matvec */
    int32_t small_bytes;  /* chosen tile size of the matvec's small-block buckets */
    double matvec_ms;     /* its matvec time */
    double default_ms;    /* matvec time of the default plan (21, 32768, 6 stages) */
    double tune_ms;       /* wall time of the tuning */
    int32_t pc_ksmall;    /* chosen plan of the preconditioner record pass */
    int32_t pc_small_bytes;
    int32_t ns;           /* chosen pipeline depth of the matvec (4, 5 or 6 stages of 32 KB) */
    int32_t y_smem;       /* 1: the matvec accumulates y in shared memory (0: in global memory,
                             chosen, or y does not fit beside the stages) */
    int32_t pc_ns;        /* chosen pipeline depth of the record pass */
    int32_t big8_kmax;    /* matvec row tiles (blocks too large for one stage) with k up to
                             this take eight rows a warp, larger ones four */
} ba_tune_report;
SQRTBA_API ba_status ba_autotune(ba_problem* h, ba_tune_report* report);

/* ---------------------------------------------------------------------- */
/* Batches of independent problems.                                        */
/* ---------------------------------------------------------------------- */

/* Many small problems of uneven size are solved together: their cameras,
 * landmarks and observations are concatenated into one index space, so
 * each phase (K1 linearise + QR, K2 damping, K3 preconditioner, K4 matvec,
 * K6 back substitution, K7 cost) is one launch over the whole batch, and
 * the PCG iterations run from one CUDA graph.  Each problem keeps its own LM
 * damping, CG scalars and stop rules, FP64 cost sums and accept / reject
 * decision (the rules of ba_lm_step); the decision runs on the device.  The
 * paper solves one problem at a time; this interface has no counterpart
 * there.  Every problem is relinearised in every batch iteration (a
 * rejected problem recomputes the same blocks). */
typedef struct ba_batch ba_batch; /* opaque */

/* One problem: the arrays and layouts of ba_create, indices local to it. */
typedef struct {
    const double* cams;
    int32_t n_cam;
    const double* pts;
    int32_t n_pt;
    const int32_t* obs_cam;
    const int32_t* obs_pt;
    const double* obs_xy;
    int64_t n_obs;
} ba_problem_desc;

/* Per-problem outcome of ba_batch_solve. */
typedef struct {
    int32_t iterations;   /* LM iterations (linear solves) */
    int32_t accepted;     /* accepted steps */
    int32_t cg_iters;     /* PCG iterations summed over its LM iterations */
    int32_t stop;         /* 1 function tolerance, 2 iteration limit, 3 lambda limit */
    double initial_cost;  /* E at the initial state */
    double final_cost;    /* E at the final state */
    double lambda;        /* final damping */
    double solve_ms;      /* from the start of ba_batch_solve to the end of the batch
                             iteration in which this problem stopped (CUDA events) */
} ba_batch_report;

typedef struct {
    int32_t n_problems;
    int32_t lm_iterations;  /* batch iterations until every problem stopped */
    int32_t tuned_ksmall;   /* matvec plan in use (see ba_autotune) */
    int32_t tuned_small_bytes;
    double total_ms;        /* device time of the whole solve (CUDA events) */
    double tune_ms;         /* autotuner wall time (0 if it did not run) */
    int64_t kernel_launches;
} ba_batch_summary;

/* Creates a batch of n >= 1 problems (each validated as by ba_create; an
 * index out of its own problem's range is BA_ERR_INVALID_ARG).  opt applies
 * to every problem; opt->autotune = 1 runs the matvec autotuner in the first
 * ba_batch_solve.  On success *out owns the batch (ba_batch_destroy). */
SQRTBA_API ba_status ba_batch_create(const ba_problem_desc* descs, int32_t n, const ba_options* opt,
                                     void* cuda_stream, ba_batch** out);
SQRTBA_API ba_status ba_batch_destroy(ba_batch* b);

/* Solves every problem from its current state until its LM stops.
 * reports (may be NULL) has room for n entries; summary may be NULL. */
SQRTBA_API ba_status ba_batch_solve(ba_batch* b, ba_batch_report* reports, ba_batch_summary* summary);

/* Restores every problem's initial state (the parameters given to
 * ba_batch_create), for repeated solves. */
SQRTBA_API ba_status ba_batch_restart(ba_batch* b);

/* Copies problem i's current state to host FP64 arrays (either may be NULL). */
SQRTBA_API ba_status ba_batch_get_params(ba_batch* b, int32_t i, double* cams, double* pts);

/* Profiling, counters and sizes of the whole batch (as ba_set_profiling,
 * ba_get_profile and ba_get_info; sizes are totals over the problems). */
SQRTBA_API ba_status ba_batch_set_profiling(ba_batch* b, int32_t enable);
SQRTBA_API ba_status ba_batch_get_profile(ba_batch* b, ba_profile* out);
SQRTBA_API ba_status ba_batch_get_info(ba_batch* b, ba_info* info);

/* Per batch LM iteration of the last ba_batch_solve: the number of problems
 * still iterating when it started (active) and its duration in ms (CUDA events
 * on the batch's stream).  A stopped problem costs nothing in K2, K3, K6, the
 * cost passes and the implicit matvec, and a problem whose last step was
 * rejected is not re-linearised (K2 undoes and redoes its damping), so the
 * durations follow the active counts.  Writes min(cap, *n) entries; *n gets the
 * number of iterations.  Any array may be NULL. */
SQRTBA_API ba_status ba_batch_iterations(ba_batch* b, int32_t cap, int32_t* active, float* ms, int32_t* n);

/* Like ba_last_error for a batch (b = NULL: the last ba_batch_create failure). */
SQRTBA_API const char* ba_batch_last_error(const ba_batch* b);

/* ---------------------------------------------------------------------- */
/* Learned warm start and block-preconditioner correction.                 */
/* ---------------------------------------------------------------------- */

/* The paper has no learned part; this is an extension of its block-Jacobi
 * PCG (Sec. 5.4).  Per camera i, with M_i the damped 9x9 diagonal block of
 * the reduced camera system (the block-Jacobi block), M_i = L_i L_i^T, and
 * g_i the camera's right-hand side, a small MLP (19 -> 256 -> 256 -> 256 ->
 * 54, GELU, BF16 weights and activations on the tensor cores, FP32
 * accumulation) maps the features
 *   [log diag(M_i) (9), (L_i^-1 g_i) / |L_i^-1 g_i| (9), log(observations of i)]
 * to o_i (9) and the lower triangle of E_i (45, row by row), giving
 *   a warm start            x0_i = (M_i^-1 g_i) * (1 + tanh(o_i))  (elementwise)
 *   a corrected block       B_i = L_i^-T (I + E_i)(I + E_i)^T L_i^-1,
 *                           diag(I + E_i) = 1 + 0.9 tanh(e_ii) > 0.1 (SPD).
 * With use_learned the PCG starts from x0 (kept only if the quadratic model
 * Q(x0) = -1/2 x0^T (g + r0) is negative, i.e. better than the zero start,
 * judged on the true residual r0 = g - H~ x0) and applies B_i instead of
 * M_i^-1.  If that CG breaks down or ends without a decrease of the
 * quadratic model below Q(0) = 0, the plain block-Jacobi CG from zero is run
 * instead (counted by ba_learned_fallbacks).
 *
 * Parameters: BA_MLP_PARAMS floats, FP32, in this order: W0 (256 x 19,
 * row-major, out x in), b0 (256), W1 (256 x 256), b1, W2 (256 x 256), b2,
 * W3 (54 x 256), b3 (54). */
#define BA_MLP_PARAMS 150582
typedef struct ba_mlp ba_mlp; /* opaque */

/* Creates a model from host FP32 parameters (copied).  Errors:
 * BA_ERR_INVALID_ARG for a null pointer or a non-finite value. */
SQRTBA_API ba_status ba_mlp_create(const float* params, void* cuda_stream, ba_mlp** out);
SQRTBA_API ba_status ba_mlp_destroy(ba_mlp* m);
/* Copies the FP32 master parameters to host memory. */
SQRTBA_API ba_status ba_mlp_get_params(ba_mlp* m, float* params);
/* Forward pass: d_feats (device, n x 19 FP32, row-major) -> d_out (device,
 * n x 54 FP32).  Synchronises the model's stream. */
SQRTBA_API ba_status ba_mlp_forward(ba_mlp* m, const float* d_feats, int32_t n, float* d_out);
/* Training samples from solver data (device pointers): d_M (n x 81, the
 * damped blocks M_i), d_g (n x 9), d_xstar (n x 9, the camera blocks of a
 * tight solve; may be NULL), d_count (n, observations per camera) ->
 * d_feats (n x 19) and d_aux (n x 72: L_i lower triangle row by row, w_i =
 * L_i^-1 g_i, s_i = M_i^-1 g_i, z*_i = L_i^T x*_i).  A block that is not
 * positive definite gives zero features and head inputs (zero loss). */
SQRTBA_API ba_status ba_mlp_prepare(ba_mlp* m, const float* d_M, const float* d_g, const float* d_xstar,
                                    const int32_t* d_count, int32_t n, float* d_feats, float* d_aux);
/* Mean training loss over n samples,
 *   ( |L^T x0 - z*|^2 + |F F^T w - z*|^2 ) / |z*|^2,  F = I + E,
 * i.e. |x0 - x*|_M^2 + |B g - x*|_M^2 normalised per camera, and (grads,
 * host, BA_MLP_PARAMS floats, may be NULL) its gradient. */
SQRTBA_API ba_status ba_mlp_loss_grad(ba_mlp* m, const float* d_feats, const float* d_aux, int32_t n,
                                      double* loss, float* grads);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the loss of n samples;
 * *loss (may be NULL) gets the loss before the step. */
SQRTBA_API ba_status ba_mlp_train_step(ba_mlp* m, const float* d_feats, const float* d_aux, int32_t n,
                                       float lr, double* loss);
SQRTBA_API const char* ba_mlp_last_error(const ba_mlp* m);
/* Attaches a model to a problem (NULL detaches); the model must outlive its
 * use and is run on the problem's stream. */
SQRTBA_API ba_status ba_set_learned(ba_problem* h, ba_mlp* model);
/* Number of learned solves that were replaced by the plain CG. */
SQRTBA_API ba_status ba_learned_fallbacks(ba_problem* h, int64_t* count);

/* ---------------------------------------------------------------------- */
/* Inspection exports for tests (copy device state to host buffers).       */
/* ---------------------------------------------------------------------- */

/* Grouping by landmark (Sec. 5.1): perm[n_obs] = input observation index in
 * (landmark, camera) order; pt_off[n_pt + 1] = landmark j owns sorted
 * positions pt_off[j] .. pt_off[j+1]-1; cam_off[n_cam + 1], cam_list[n_obs] =
 * camera i's sorted positions in increasing order.  Any pointer may be NULL. */
SQRTBA_API ba_status ba_debug_export_order(ba_problem* h, int32_t* perm, int64_t* pt_off,
                                int64_t* cam_off, int32_t* cam_list);

/* Landmark block j in its current (damped or undamped) state.  With k its
 * observation count and cameras in increasing index order:
 *   top[3 * (9k + 4)]  rows of Q^T [J_p | J_l | r] belonging to R1:
 *                      [Q1^T J_p (9k) | R1 row (3) | Q1^T r (1)] per row
 *   a[2k * 9k]         Q2^T J_p row-major (last 3 rows: the damping rows)
 *   c[2k]              Q2^T r
 *   rot[12]            the six Givens (cos, sin) pairs of the current damping
 * *k_out receives k; buffers must hold k_cap-sized data. */
SQRTBA_API ba_status ba_debug_export_landmark(ba_problem* h, int32_t j, int32_t k_cap, float* top,
                                   float* a, float* c, float* rot, int32_t* k_out);

/* D_p^2 (9 n_cam) and D_l^2 (3 n_pt) of the current linearisation. */
SQRTBA_API ba_status ba_debug_export_damping(ba_problem* h, float* dp2, float* dl2);

/* Per sorted observation s: residual r (2), J_p (18, row-major 2x9) and J_l
 * (6, row-major 2x3) at the current state.  Any pointer may be NULL. */
SQRTBA_API ba_status ba_debug_export_jacobians(ba_problem* h, float* r, float* jp, float* jl);

/* The block-Jacobi blocks M_i = sum_j A_ji^T A_ji + lambda D_p,i^2
 * (n_cam x 81) and g = -b~ (9 n_cam) of the last PCG solve. */
SQRTBA_API ba_status ba_debug_export_rcs_diag(ba_problem* h, float* m, float* g);

/* y = H~ v for a host vector v (9 n_cam) with the current blocks and lambda. */
SQRTBA_API ba_status ba_debug_matvec(ba_problem* h, const float* v, float* y);

/* Failure test of the bounded waits (no counterpart in the paper; tests only).
 * tile >= 0: every later matvec launch of this problem (ba_debug_matvec, the
 * PCG) leaves tile `tile` of the first CTA's tile range and the rest of that
 * range unissued, and its consumer waits give up after wait_ms milliseconds
 * (0 < wait_ms <= 2000); the call that synchronises next returns
 * BA_ERR_TIMEOUT.  No wait is unbounded and no copy is left in flight: the
 * producer lets the copies it issued land before the CTA exits.  tile < 0
 * restores normal operation (wait_ms ignored).  A captured PCG graph is
 * rebuilt on the next solve.  Errors: BA_ERR_INVALID_ARG for wait_ms out of
 * range. */
SQRTBA_API ba_status ba_debug_fail_matvec(ba_problem* h, int32_t tile, double wait_ms);

/* The last step: dx_p (9 n_cam) and dx_l (3 n_pt). */
SQRTBA_API ba_status ba_debug_export_step(ba_problem* h, float* dp, float* dl);

#ifdef __cplusplus
}
#endif

#endif /* SQRTBA_H */
