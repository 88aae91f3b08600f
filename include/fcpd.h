/*
 * fcpd.h -- C ABI of the GB300 (sm_103a) Fast Coherent Point Drift EM loop.
 *
 * Method: X.-W. Feng, D.-Z. Feng, Y. Zhu, "Fast Coherent Point Drift",
 * arXiv 2006.06281.  Notation is the paper's:
 *   X  (M x D)  model points -- they move        (Sec. I, Sec. II)
 *   Y  (N x D)  scene points -- they stay fixed
 *   T  = X + Phi W, the transformed model points (Eq. 9-11)
 *   Phi (M x M) Gaussian Gram matrix of X, width beta (Eq. 11)
 *   w  outlier weight, 0 <= w < 1 (Eq. 2); lambda regulariser (Eq. 7);
 *   sigma2 the variance of the Gaussian mixture (Eq. 1, Eq. 18).
 *
 * One registration = setup (Gram matrix + its eigendecomposition, Eq. 16,
 * done once) followed by EM iterations.  Each iteration runs on the GPU only:
 *   E-step   Eq. 4 posterior with the uniform-outlier constant c, then the
 *            corresponding constraint Eq. 5 (each row of P rescaled to sum 1),
 *            reduced to Ytil = P^ Y without ever storing the M x N matrix P;
 *   M-step   Eq. 17 (full basis) or Eq. 20 (top-K basis):
 *            T = X + U diag(l_i / (l_i + lambda sigma2)) U^T (Ytil - X);
 *   variance Eq. 18 over the row-normalised posterior, with the new T.
 *
 * Conventions for every entry point
 *   - Point arrays are row-major, point-major (D contiguous values per
 *     point), element type double for CPD_FP64 and float for CPD_FP32 and
 *     CPD_MIXED.
 *   - A point-array pointer may be HOST memory (pageable or pinned) or DEVICE
 *     memory of the current CUDA device; the library tells them apart with
 *     cudaPointerGetAttributes and stages host data through its own device
 *     buffers.  The caller owns every array it passes; the library keeps no
 *     pointer to caller memory after a call returns.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All device
 *     work is enqueued on it.  A call that returns host values (sigma2_out,
 *     iters_done, a host output array) synchronises that stream first.
 *   - Errors: every call returns a cpd_status.  Arguments are validated
 *     before any device work; on CPD_EINVAL nothing is enqueued and outputs
 *     are untouched.  No C++ exception crosses this boundary.
 *     cpd_last_error() gives a one-line description of the last failure on
 *     the calling thread.
 *   - A numeric failure found on the device (a row of P whose mass underflows
 *     to 0 so Eq. 5 cannot normalise it, or a variance that is not positive
 *     and finite) sets a device status word; later kernels of the same
 *     context become no-ops and the next synchronising call returns
 *     CPD_ENUMERIC.
 *   - Only D = 3 is implemented (the paper's experiments are 3-D point sets).
 *   - Host-side fault injection for tests: environment variable CPD_FAULT =
 *     "alloc" (first device allocation of cpd_setup fails -> CPD_ENOMEM),
 *     "solver" (the eigensolver reports failure -> CPD_ESOLVER),
 *     "nan_sigma" (the initial variance is NaN -> CPD_ENUMERIC on the first
 *     iteration), or a device wait made to run out without faulting the
 *     GPU -> CPD_ETIMEOUT: "barrier" (the batched kernel's waits between
 *     the phases of a pair),
 *     "bulk_wait" (the M-step's bulk-copy ring), "umma_wait" (the
 *     shared-model tensor-core products), "gemm_wait" (the BF16 tensor-core
 *     GEMM of the warm-start network).  Nothing is faulted on the GPU.
 */
#ifndef FCPD_H
#define FCPD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FCPD_ABI_VERSION 1

typedef enum {
    CPD_OK = 0,
    CPD_EINVAL = 1,    /* invalid argument                               */
    CPD_ENOMEM = 2,    /* device allocation failed                       */
    CPD_ECUDA = 3,     /* a CUDA runtime call failed                     */
    CPD_ESOLVER = 4,   /* the eigensolver failed (Eq. 16)                */
    CPD_ENUMERIC = 5,  /* row mass 0 (Eq. 5) or sigma2 not positive/finite */
    CPD_ETIMEOUT = 6,  /* a bounded device wait gave up                  */
    CPD_ESTATE = 7     /* call not valid in the context's current state  */
} cpd_status;

typedef enum {
    CPD_FP64 = 0,      /* double everywhere                              */
    CPD_FP32 = 1,      /* float points/basis, FP64 scalar reductions     */
    CPD_MIXED = 2      /* as CPD_FP32, but the eigenbasis U, U^T is stored
                          in FP16 (products and sums in FP32): the M-step
                          streams half the bytes; and while sigma2 is large
                          (sigma2 >= 4.4e-4 R^2, R the largest point norm)
                          the E-step's Gaussian exponents come from FP16
                          tensor-core products (tcgen05.mma kind::f16,
                          M = 128 tiles accumulated in tensor memory,
                          operands split into two FP16 parts, K = 16,
                          FP32 accumulation), below it from the FP32
                          passes.  Not a precision the paper uses; its
                          error against the FP64 oracle is measured and
                          stated, not bounded by the FP32 tolerance.
                          Points, outputs: float.                        */
} cpd_precision;

/* Registration parameters (Sec. IV "Parameter settings": w, beta, lambda). */
typedef struct {
    int32_t D;            /* point dimension; must be 3                        */
    int32_t precision;    /* cpd_precision                                     */
    double  w;            /* outlier weight, 0 <= w < 1 (Eq. 2)                */
    double  beta;         /* Gaussian kernel width > 0 (Eq. 10-11)             */
    double  lambda;       /* regularisation weight > 0 (Eq. 7, Eq. 15)         */
    double  sigma2_init;  /* initial variance; <= 0 means "from the data":
                             sum_mn |y_n - x_m|^2 / (D M N)                    */
    int64_t K;            /* 0 or M: full eigenbasis (Eq. 17);
                             1..M-1: the K largest eigenpairs (Eq. 19-20);
                             K > M is rejected with CPD_EINVAL                 */
    int32_t max_iter;     /* iteration count used by cpd_register (> 0)        */
    int32_t flags;        /* cpd_flags bits (0 = default)                      */
    double  tol;          /* > 0: stop once RMS_m |T_k - T_(k-1)| <= tol;
                             0: run the requested number of iterations        */
} cpd_params;

/*
 * cpd_params.flags (0 = default: the points in the caller's order, the dense
 * E-step).  With CPD_FLAG_PRUNE an FP32 or mixed context keeps its model
 * points (and every scene) in spatial order -- a 12-bit Morton order, sorted
 * on the device, stable -- and, once sigma2 is small enough that far tile
 * pairs of points have FP32 Gaussians that are exactly 0 (ex2 results below
 * 2^-126 flush to 0), its E-step skips those tile pairs: the sums are
 * bit-identical to evaluating them.  All arrays a caller passes or receives
 * stay in the caller's order.  Point sets larger than 2^20 are not sorted
 * (no pruning).  Pruning pays once sigma2 has collapsed to the noise level;
 * while it has not, the idle pruned launches cost a few microseconds per
 * pass, so it is not the default.
 */
typedef enum {
    CPD_FLAG_PRUNE = 1,          /* spatial order + exact pruning of the FP32 E-step       */
    CPD_FLAG_PRUNE_ALWAYS = 2,   /* (implies PRUNE) pruned layout in every iteration       */
    CPD_FLAG_PRUNE_NOSKIP = 4,   /* (implies PRUNE) pruned layout, every tile pair
                                    evaluated: the same sums as skipping, bit for bit
                                    (verification)                                        */
    CPD_FLAG_SPECTRAL_TRIM = 8,  /* FP32 / mixed: M-step over the leading directions only
                                    while the dropped ones are below FP32 rounding        */
    CPD_FLAG_FULL_EIG = 16       /* top-K basis (0 < K < M) from the full eigensolver
                                    instead of subspace iteration (verification)          */
} cpd_flags;

/*
 * CPD_FLAG_SPECTRAL_TRIM (Eq. 17).  Direction k of the eigenbasis enters T
 * through s_k (U^T R)_k with s_k = l_k / (l_k + lambda sigma2); the Gaussian
 * Gram matrix's spectrum decays so fast that, for all but a few hundred
 * directions, s_k < 2^-24.  The dropped part of U diag(s) U^T R then has norm
 * <= 2^-24 |R| (U orthonormal): below one FP32 rounding of T.  At setup the
 * context keeps the leading k_cap directions (those that can reach 2^-24
 * while sigma2 >= 1e-4 x the model points' variance per axis, rounded up to
 * 16); each iteration the device tests the largest dropped eigenvalue
 * against the current sigma2 and runs the M-step over the k_cap columns
 * when the bound holds, the full M-step when it does not.  T and sigma2
 * agree with the full M-step within FP32 rounding.  cpd_get_W then returns
 * the component of W in the kept directions (Phi W = T - X is preserved to
 * the same bound; W itself is ill-posed in the dropped ones).  Not for
 * CPD_FP64 or batched registrations (CPD_EINVAL); K <= k_cap leaves the
 * context unchanged.
 */

typedef struct cpd_ctx cpd_ctx;   /* opaque; owned by the library */

/* ABI version of the loaded library (FCPD_ABI_VERSION). */
int32_t cpd_abi_version(void);

/* Human-readable name of a status code (static string). */
const char *cpd_status_string(cpd_status s);

/* One-line description of the last failure on the calling thread ("" if none). */
const char *cpd_last_error(void);

/* Fill *p with defaults: D=3, FP32, w=0.1, beta=2, lambda=2, sigma2 from data,
 * full basis, max_iter=50, tol=0. */
void cpd_params_default(cpd_params *p);

/*
 * Setup (done once per model point set; Eq. 11, Eq. 16, Eq. 19).
 *   X      M x D points (host or device), element type per p->precision.
 *   M      number of model points, 1 <= M <= 46340.
 *   stream cudaStream_t all work of this context is enqueued on.
 *   out    receives the new context (owned by the caller; free with
 *          cpd_destroy).
 * Builds Phi in FP64 on the device and eigendecomposes it in FP64, clamps
 * the eigenvalues at 0, keeps the K largest (or all) eigenpairs in
 * descending order, stores the basis in the working precision and frees Phi.
 * The full basis comes from the dense symmetric eigensolver (cuSOLVER).  A
 * top-K basis with K + max(16, K/4) <= M/2 comes from subspace iteration
 * with Rayleigh-Ritz steps on a random start block (FP64 cuBLAS products,
 * cuSOLVER QR and a small (K + p) x (K + p) eigenproblem), stopped when every
 * kept pair has |Phi u - theta u| <= 1e-13 theta_max -- the dense solver's
 * rounding level -- at O(M^2 K) instead of O(M^3) work; if that does not
 * converge in 100 steps (or with CPD_FLAG_FULL_EIG) the dense solver is used.
 * All of it is setup only.  Synchronises `stream`.
 * Errors: CPD_EINVAL (arguments), CPD_ENOMEM, CPD_ESOLVER, CPD_ECUDA; *out is
 * left untouched on error.
 */
cpd_status cpd_setup(const void *X, int64_t M, const cpd_params *p, void *stream, cpd_ctx **out);

/*
 * Run EM iterations (Eq. 4, 5, 17/20, 18) against scene Y.
 *   Y          N x D scene points (host or device), context precision.
 *   N          number of scene points, >= 1.
 *   n_iter     iterations to run (>= 0); with p->tol > 0 fewer may run.
 *   T_out      if non-NULL, receives the current T (M x D, host or device).
 *   sigma2_out if non-NULL, receives the current sigma2 (host double).
 *   iters_done if non-NULL, receives the total iteration count of the
 *              context (host int).
 * The context keeps T, sigma2 and the iteration count between calls, so a
 * registration can be run in pieces; the first call after cpd_setup or
 * cpd_reset starts from W = 0 (T = X) and the initial variance.  A call with
 * a different Y (or N) continues from the current state with the new scene.
 * Iterations are replayed from a captured CUDA graph on `stream`; the call
 * synchronises only if it returns host values.
 */
cpd_status cpd_iterate(cpd_ctx *ctx, const void *Y, int64_t N, int32_t n_iter,
                       void *T_out, double *sigma2_out, int32_t *iters_done);

/*
 * cpd_iterate with per-kernel timing, for benchmarking: runs n_iter
 * (1..4096) iterations from one captured CUDA graph in which every 10th
 * iteration (and the last) also records a timing event after each kernel,
 * synchronises `stream`, and writes 9 floats to phase_ms (host): the
 * milliseconds per launch, averaged over those sampled iterations, of
 * [0] E pass A, [1] its reduction (+ c, Eq. 4), [2] E pass B, [3] its
 * reduction (Eq. 5), [4] projection U^T (Ytil - X), [5] diagonal update,
 * [6] expansion U B, [7] its reduction with T = X + U B and Eq. 18;
 * [8] the whole span from the first iteration's start to the last
 * iteration's end.
 */
cpd_status cpd_iterate_profiled(cpd_ctx *ctx, const void *Y, int64_t N, int32_t n_iter,
                                float *phase_ms);

/* Restart the context's registration: T = X, iteration count 0, sigma2
 * re-initialised on the next cpd_iterate.  The eigenbasis is kept. */
cpd_status cpd_reset(cpd_ctx *ctx);

/*
 * Optional ground truth for Eq. 22: Yhat (M x D, host or device) is the true
 * position of each model point.  Each following iteration records
 * RMSE = sqrt(mean_m |t_m - yhat_m|^2); if rmse_tol > 0 the loop stops at the
 * first iteration whose RMSE <= rmse_tol.  Yhat = NULL clears it.
 */
cpd_status cpd_set_ground_truth(cpd_ctx *ctx, const void *Yhat, double rmse_tol);

/* Synchronise and read the context state: sigma2, iterations completed, and
 * the device status word (a cpd_status; CPD_OK if no device failure). */
cpd_status cpd_get_state(cpd_ctx *ctx, double *sigma2, int32_t *iters, int32_t *device_status);

/*
 * Per-iteration history of the current registration (synchronises).
 * Entry k (0 <= k < n) describes iteration k+1: sigma2 after it (Eq. 18),
 * the Eq. 3 log-likelihood evaluated in its E-step, and its Eq. 22 RMSE
 * (NaN without ground truth).  Any output may be NULL.  Only the first
 * 65536 iterations are recorded.  CPD_EINVAL if n exceeds the count run.
 */
cpd_status cpd_get_history(cpd_ctx *ctx, int32_t n, double *sigma2_hist, double *loglik_hist,
                           double *rmse_hist);

/* W of the last M-step (Eq. 17 / Eq. 20), M x D into W_out (host or device).
 * CPD_ESTATE before the first iteration. */
cpd_status cpd_get_W(cpd_ctx *ctx, void *W_out);

/* The kept eigenbasis (Eq. 16 / 19): U_out (M x K row-major, host or
 * device; may be NULL; double for CPD_FP64, float otherwise -- the FP16
 * basis of CPD_MIXED is converted) and lam_out (K doubles, host,
 * descending, clamped at 0; may be NULL).  K is cpd_basis_rank(ctx). */
cpd_status cpd_get_basis(cpd_ctx *ctx, void *U_out, double *lam_out);
int64_t cpd_basis_rank(const cpd_ctx *ctx);

/* How the context's basis was computed: *method = 0 (dense eigensolver) or 1
 * (top-K subspace iteration); *steps = its Rayleigh-Ritz steps (0 for the
 * dense solver unless subspace iteration ran first and did not converge).
 * Either pointer may be NULL.  CPD_EINVAL for a NULL context. */
cpd_status cpd_eig_info(const cpd_ctx *ctx, int32_t *method, int32_t *steps);

/*
 * One M-step on the context's basis (Eq. 17 / 20), without touching the
 * context's registration state: T_out = X + U diag(l/(l + lambda sigma2))
 * U^T (Ytil - X) and, if W_out is non-NULL, W_out = U diag(1/(l + lambda
 * sigma2)) U^T (Ytil - X).  Ytil, T_out, W_out: M x D (host or device).
 */
cpd_status cpd_mstep(cpd_ctx *ctx, const void *Ytil, double sigma2, void *T_out, void *W_out);

/*
 * One E-step, no context needed (Eq. 4 then Eq. 5):
 *   T (M x D), Y (N x D): host or device, element type per `precision`
 *            (CPD_MIXED: float arrays; the tensor-core passes run when
 *            sigma2 is above their floor, else the FP32 passes).
 *   Ytil_out (M x D, required): sum_n p^_mn y_n, the row-normalised estimate.
 *   P1_out   (M doubles, optional, host or device): row mass sum_n p_mn
 *            before Eq. 5.
 *   den_out  (N doubles, optional, host or device): column denominators
 *            sum_m e_mn + c of Eq. 4.
 *   sums_out (2 host doubles, optional): [0] = sum_m sum_n p^_mn |y_n - t_m|^2
 *            (the Eq. 18 numerator at T itself), [1] = Eq. 3 log-likelihood.
 * Scratch is allocated on `stream` for the call and freed before return.
 * Synchronises `stream`.  CPD_ENUMERIC if a row mass is 0 or not finite.
 */
cpd_status cpd_estep(const void *T, int64_t M, const void *Y, int64_t N, int32_t precision,
                     double sigma2, double w, void *Ytil_out, void *P1_out, void *den_out,
                     double *sums_out, void *stream);

/*
 * cpd_estep without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * when they need an E-step -- loops that must not stall on the device
 * synchronisation cudaMalloc/cudaFree may cause, programs that reserve all
 * device memory up front under a fixed budget, and runtimes that hand the
 * library only arrays they already own.  It computes what cpd_estep computes
 * for precision CPD_FP32, with the same kernels, but takes all scratch from
 * one 24 MiB array that the library holds (as a static device variable) for
 * its lifetime on every GPU that loads it.
 *   T (M x 3 floats), Y (N x 3 floats), Ytil_out (M x 3 floats), and the
 *   optional P1_out (M doubles) and den_out (N doubles) must be arrays in the
 *   memory of the CURRENT device; sums_out (2 host doubles) is optional, as
 *   in cpd_estep.
 *   Limits: 1 <= M, N <= 32768 (the partial sums are planned so that every
 *   such size fits the array); larger sizes, host arrays or arrays of
 *   another device return CPD_EINVAL with a message.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress).  The call reads its results back to the host and
 * synchronises `stream` before it returns, so it cannot be called while
 * `stream` is being captured into a CUDA graph.  Every call uses the same
 * array, so calls that may overlap on the GPU (from different threads, or
 * enqueued on different streams without the returning synchronisation in
 * between) race and must be serialised by the caller.  The array keeps the
 * last call's contents; the call re-initialises everything that must start
 * from zero.
 */
cpd_status cpd_estep_noalloc(const void *T, int64_t M, const void *Y, int64_t N, double sigma2, double w,
                             void *Ytil_out, void *P1_out, void *den_out, double *sums_out, void *stream);

/*
 * Whole registration: cpd_setup, p->max_iter iterations of cpd_iterate (fewer
 * with p->tol > 0), outputs, cpd_destroy.
 *   T_out (required) M x D; W_out (optional) M x D; sigma2_out, iters_done
 *   optional host outputs.
 */
cpd_status cpd_register(const void *X, int64_t M, const void *Y, int64_t N, const cpd_params *p,
                        void *stream, void *T_out, void *W_out, double *sigma2_out,
                        int32_t *iters_done);

/*
 * Work of the pruned E-step: eval_frac[k] (k < n, host) is the fraction of
 * the 2 M N Gaussian pairs of passes A and B that iteration k+1 evaluated
 * (1 for dense iterations).  Synchronises.  CPD_EINVAL if n exceeds the
 * iterations run.
 */
cpd_status cpd_get_work(cpd_ctx *ctx, int32_t n, double *eval_frac);

/* 1 if the context keeps its points in spatial order (pruning possible). */
int32_t cpd_spatial_order(const cpd_ctx *ctx);

/*
 * Several registrations against the context's model (Eq. 17 with one
 * eigenbasis for all scenes).  Scene i (Y[i]: N[i] x 3 FP32, row-major, host
 * or device) is registered from W = 0 (sigma2_0 from the data, or the
 * context's sigma2_init) for exactly n_iter iterations; T_out[i] (M x 3 FP32,
 * host or device, caller-owned) receives its T and sigma2_out[i] (host) its
 * final sigma2.  Up to 8 scenes at a time share each pass over U and U^T:
 * their projections U^T R_i and expansions U B_i are one streaming kernel
 * with 3 S right-hand sides, so the M-step's basis traffic is paid once per
 * group instead of once per scene.  The E-steps, diagonal updates and Eq. 18
 * epilogues stay per scene (the same kernels as cpd_iterate).  The context's
 * own registration state is not touched.  Requires a CPD_FP32 context
 * without flags (CPD_EINVAL otherwise).  Synchronises.  A device failure of
 * any scene is returned (CPD_ENUMERIC, CPD_ETIMEOUT).
 */
cpd_status cpd_iterate_shared(cpd_ctx *ctx, int32_t n_scenes, const void *const *Y, const int64_t *N,
                              int32_t n_iter, void *const *T_out, double *sigma2_out);

/*
 * Spectral trim of a context (CPD_FLAG_SPECTRAL_TRIM): *k_cap (host) = the
 * directions the trimmed M-step keeps (0: no trim -- flag unset or nothing
 * to drop); *trimmed_iters (host) = iterations of the current registration
 * that ran the trimmed M-step (0 before any).  Synchronises.  CPD_EINVAL
 * for a null argument.
 */
cpd_status cpd_get_trim(cpd_ctx *ctx, int64_t *k_cap, int32_t *trimmed_iters);

/*
 * Launch layout of the iterations (not in the paper; Eq. 4, 5 and 17 are
 * unchanged): *pieces (host) = the row pieces pass B of the E-step runs in.
 * With pieces > 1 each piece's model rows go through pass B, their row
 * reduction and log-domain fix-up, and the M-step's projection U^T R of
 * those rows (Eq. 17) starts on a side stream while the next piece's pass B
 * runs, so the HBM-bound projection overlaps the ALU-bound pass B; the
 * diagonal update then sums every piece's partials.  Chosen at cpd_setup:
 * CPD_FP32 contexts without flags whose basis has more than 256 columns and
 * M >= 8192 use 3 pieces; all others 1.  The environment variable
 * FCPD_SPLIT_B, read at cpd_setup, sets the count (1..4; 1: off).  Each
 * piece's scene-point partial sums are split for its own grid, so results
 * differ from one piece in FP32 rounding only.  No device work.  CPD_EINVAL
 * for a null argument.
 */
cpd_status cpd_pass_b_pieces(cpd_ctx *ctx, int32_t *pieces);

/* ------------------------------------------------------------------------
 * Warm start (not in the paper).  In the top-K basis the displacement of
 * every iteration lies in span(U) (Eq. 20), so T - X = U c with c = U^T
 * (T - X): K x 3 eigen-coefficients.  A learned predictor of c (and of
 * sigma2) for a new scene can start the EM loop near its end; W = 0 stays
 * the fallback.  CPD_FP32 and CPD_MIXED contexts (the FP16 basis of the
 * mixed mode is the rounding of the same FP64 eigenvectors, so coefficients
 * of one apply to the other).
 * ---------------------------------------------------------------------- */

/* coef_out (n_coef x 3 floats, host or device) = U[:, :n_coef]^T (T - X) of
 * the current T.  Synchronises.  CPD_ESTATE before a registration started. */
cpd_status cpd_coefficients(cpd_ctx *ctx, int32_t n_coef, void *coef_out);

/* coef_out (n_coef x 3 floats, host or device) = U[:, :n_coef]^T (T - X) of
 * a caller's T (M x 3 floats, host or device; for instance a T of
 * cpd_iterate_shared).  The context's own registration is not touched.
 * Synchronises. */
cpd_status cpd_coefficients_of(cpd_ctx *ctx, int32_t n_coef, const void *T, void *coef_out);

/* Start the next registration at T = X + U[:, :n_coef] coef (coef: n_coef x 3
 * floats, host or device; n_coef = 0 gives T = X) with variance sigma2_0,
 * iteration count 0: the following cpd_iterate continues from there
 * (instead of T = X and the data variance).  Synchronises. */
cpd_status cpd_warm_start(cpd_ctx *ctx, int32_t n_coef, const void *coef, double sigma2_0);

/*
 * The warm-start network: a point-set encoder -- a shared per-point MLP
 * 3 -> 128 -> 128 -> 256 (ReLU), the maximum over the points, a head
 * 256 -> 256 (ReLU) -> n_out -- trained on the GPU with the mean-squared
 * error and Adam (beta1 0.9, beta2 0.999, eps 1e-8), all in CUDA kernels
 * of this library.  Parameter layout: per layer the weights (fan_in x
 * fan_out, row-major) then the biases, layers in order.
 *   create:   n_out 1..4096; max_batch 1..1024 scenes of n_points points
 *             (max_batch * n_points <= 2^24); seed of the initial weights.
 *             FP32 arithmetic throughout.
 *   create_ex: as create, with precision CPD_NET_FP32 (= create) or
 *             CPD_NET_BF16: the per-point layers 128 -> 128 and 128 -> 256
 *             and their gradient products multiply BF16 operands on the
 *             tensor cores with FP32 accumulation (master weights, Adam,
 *             biases, the 3 -> 128 layer, the head and every reduction in
 *             FP32).  BF16 needs a compute capability 10.x device
 *             (CPD_EINVAL otherwise) and about 2.3 KB more device memory per
 *             point of max_batch * n_points.  A tensor-core wait that
 *             expires fails the call with CPD_ETIMEOUT.
 *   forward / gradients / train_step: Y = B x n_points x 3 floats in DEVICE
 *             memory (B <= max_batch); pred_out (B x n_out), target
 *             (B x n_out), grad_out (num_params) host or device.  Each
 *             synchronises the network's stream.
 */
typedef struct cpd_net cpd_net;
enum { CPD_NET_FP32 = 0, CPD_NET_BF16 = 1 };
cpd_status cpd_net_create(int32_t n_out, int32_t max_batch, int32_t n_points, uint64_t seed, void *stream,
                          cpd_net **out);
cpd_status cpd_net_create_ex(int32_t n_out, int32_t max_batch, int32_t n_points, uint64_t seed, int32_t precision,
                             void *stream, cpd_net **out);
/* CPD_NET_FP32 or CPD_NET_BF16 (-1 for NULL). */
int32_t cpd_net_precision(const cpd_net *net);
int64_t cpd_net_num_params(const cpd_net *net);
cpd_status cpd_net_get_params(cpd_net *net, float *out);
cpd_status cpd_net_set_params(cpd_net *net, const float *in);
cpd_status cpd_net_forward(cpd_net *net, const float *Y, int32_t B, float *pred_out);
cpd_status cpd_net_gradients(cpd_net *net, const float *Y, const float *target, int32_t B, float *grad_out,
                             float *loss_out);
cpd_status cpd_net_train_step(cpd_net *net, const float *Y, const float *target, int32_t B, float lr,
                              float *loss_out);
void cpd_net_destroy(cpd_net *net);

/* Free a context (NULL is ignored).  Synchronises its stream first. */
void cpd_destroy(cpd_ctx *ctx);

/* ------------------------------------------------------------------------
 * Batched registrations.  The paper registers one pair at a time; these
 * entry points run many independent registrations (X_i, Y_i), i < n_pairs,
 * of uneven sizes together: every call advances all of them by the same
 * number of EM iterations (Eq. 4, 5, 17/20, 18, exactly as cpd_iterate) in
 * ONE persistent cooperative kernel launch, replayed from a CUDA graph.  The
 * launch's blocks take the work items of all pairs (tiles of the E-step
 * passes, row chunks of the basis products, reduction blocks) from a shared
 * queue, phase by phase and largest pairs first; an item waits only for its
 * own pair's previous phase, so the phases of different pairs overlap.
 * ---------------------------------------------------------------------- */
typedef struct cpd_batch cpd_batch;   /* opaque; owned by the library */

/*
 * Create a batch: setup of every pair (Eq. 11, Eq. 16, Eq. 19, as cpd_setup,
 * several pairs at a time on internal streams), scene upload, and the start
 * of every registration (T_i = X_i, initial variance).
 *   n_pairs            1..65536.
 *   X[i], M[i]         model points of pair i: M[i] x 3 floats (host or
 *                      device), 1 <= M[i] <= 46340.
 *   Y[i], N[i]         scene points of pair i: N[i] x 3 floats (host or
 *                      device), N[i] >= 1.
 *   p                  shared parameters; precision CPD_FP32, or CPD_MIXED
 *                      (each pair's basis stored in FP16 and streamed by the
 *                      M-step phases; the E-step phases stay FP32).  The
 *                      basis of pair i keeps min(p->K, M[i]) eigenpairs (all
 *                      with p->K = 0).  p->tol > 0 stops each pair on its own.
 *   barrier_timeout_s  wall-time limit of one wait inside the kernel (for a
 *                      pair's previous phase), in (0, 60]; 0 selects 5 s.  A
 *                      wait that exceeds it ends the launch with
 *                      CPD_ETIMEOUT.
 *   stream             cudaStream_t all later work of the batch runs on.
 * The caller's arrays are only read during the call.  Synchronises.
 * Errors: CPD_EINVAL (arguments, with the pair index), CPD_ENOMEM,
 * CPD_ESOLVER, CPD_ECUDA (including a device without cooperative launch);
 * *out is left untouched on error.
 */
cpd_status cpd_batch_create(int32_t n_pairs, const void *const *X, const int64_t *M, const void *const *Y,
                            const int64_t *N, const cpd_params *p, double barrier_timeout_s, void *stream,
                            cpd_batch **out);

/*
 * Run n_iter (0..2^20) EM iterations of every pair that has not stopped (by
 * p->tol or a device failure) in one launch, then synchronise.  CPD_ETIMEOUT
 * if a wait inside the kernel ran out (the registrations' state is then
 * undefined until cpd_batch_reset); per-pair failures are reported by
 * cpd_batch_state, not here.
 */
cpd_status cpd_batch_iterate(cpd_batch *b, int32_t n_iter);

/* Per-pair state, n_pairs entries in each (host) array, any of which may be
 * NULL: sigma2 (Eq. 18), iterations completed, device status (a cpd_status).
 * Synchronises. */
cpd_status cpd_batch_state(cpd_batch *b, double *sigma2, int32_t *iters, int32_t *device_status);

/* Current T of pair i: M[i] x 3 floats into T_out (host or device).
 * Synchronises if T_out is host memory. */
cpd_status cpd_batch_get_T(cpd_batch *b, int32_t i, void *T_out);

/* Sizes of pair i: model points, scene points, kept eigenpairs. */
cpd_status cpd_batch_info(const cpd_batch *b, int32_t i, int64_t *M, int64_t *N, int64_t *K);

/* Launch shape of the persistent kernel: pairs, resident blocks (the grid),
 * and work items per iteration over all phases. */
cpd_status cpd_batch_launch_shape(const cpd_batch *b, int32_t *n_pairs, int32_t *grid, int32_t *n_items);

/*
 * Where the last cpd_batch_iterate call spent its time: 8 floats (host).
 * [0..3]: milliseconds per iteration of the whole GPU's time spent inside
 * each phase's work items (block-time summed over the blocks, divided by
 * their number), averaged over the call's iterations: [0] E pass A with the
 * column reduction (Eq. 4) and its fix-up, [1] E pass B with the row
 * reduction (Eq. 5) and its fix-up, [2] projection U^T (Ytil - X) with the
 * diagonal update, [3] expansion with T and Eq. 18.  Phases of different
 * pairs overlap, so these add up to the call's time less the waits.
 * [4..7]: for the same phases, the fraction of the blocks' time on that
 * phase's items spent working rather than waiting for the pair's previous
 * phase (1 = never waited).  CPD_ESTATE before the first completed call.
 */
cpd_status cpd_batch_phase_ms(const cpd_batch *b, float *phase_ms);

/* Restart every registration: T_i = X_i, iteration count 0, initial variance
 * re-computed from the stored scene.  Synchronises. */
cpd_status cpd_batch_reset(cpd_batch *b);

/*
 * Autotuner of the persistent kernel's work items: times n_iter (1..64)
 * iterations of the batch under each of eight work-item plans -- E-step items
 * per resident block in {2, 4, 8, 16} x projection items of {256, 512} KB of
 * the basis, in that order -- keeps the fastest, and restarts every
 * registration (as cpd_batch_reset).  Optional outputs (host): the chosen
 * e_items and proj_kb, and ms_out[8], the measured milliseconds of each
 * candidate.  Synchronises.  The results of the registrations do not depend
 * on the plan beyond summation order.
 */
cpd_status cpd_batch_autotune(cpd_batch *b, int32_t n_iter, int32_t *e_items_out, int32_t *proj_kb_out,
                              float *ms_out);

/* Free a batch and all its pairs (NULL is ignored).  Synchronises first. */
void cpd_batch_destroy(cpd_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* FCPD_H */
