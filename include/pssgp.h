/*
 * pssgp.h -- C ABI of libpssgp: the parallel (associative-scan) Kalman filter,
 * RTS smoother and log marginal likelihood of a stationary temporal Gaussian
 * process in state-space form, with missing measurements at the prediction
 * times, in FP64 on one NVIDIA B300 (sm_103a).
 *
 * Method: Corenflos, Zhao, Sarkka, "Temporal Gaussian Process Regression in
 * Logarithmic Time".  Section, equation and proposition references below are
 * to that paper and its supplement.
 *
 * Conventions (all entry points):
 *  - Every function returns an int status: 0 (PSSGP_OK) or a negative value
 *    for an argument error detected on the host before anything is launched.
 *    Errors detected on the device are OR-ed into a status word kept in the
 *    workspace (positive bits below), cleared at the start of every call and
 *    read back with pssgp_get_status.
 *  - Array pointers are DEVICE pointers owned by the caller unless stated
 *    otherwise; the library never allocates, frees or retains them.  All
 *    scratch memory is a caller-provided device workspace `ws` (256-byte
 *    aligned) of at least pssgp_workspace_size(d, n) bytes.
 *  - Every device entry point is asynchronous on the CUDA stream `stream`
 *    (a cudaStream_t passed as void*, NULL = legacy default stream).  Two
 *    calls that share a workspace must not overlap on the GPU.
 *  - Time steps are indexed k = 0..n-1 (the paper's k = 1..n).  Times must be
 *    non-decreasing; equal times are allowed (zero-length step).
 *  - Per-step state outputs use an entry-major ("struct of arrays") layout
 *    with leading dimension ld >= n: entry e of step k is at [e * ld + k].
 *    Symmetric d x d matrices are stored packed, upper triangle row by row:
 *    entry (i, j), i <= j, has index i*d - i*(i-1)/2 + (j - i).
 *  - State vectors and covariances are reported in the coordinates of the
 *    model's SDE (Sec. 4.2 balancing is internal).
 *  - State dimension 1 <= d <= PSSGP_DMAX.  Measurements are scalar,
 *    y_k = H x(t_k) + e_k, e_k ~ N(0, R_k) with R_k > 0 (Eq. (gp-def)).
 */
#ifndef PSSGP_H
#define PSSGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSSGP_DMAX 8
/* Largest step count any entry point accepts (PSSGP_EINVAL above it): keeps
 * every workspace size n x record x 8 bytes far from int64 overflow. */
#define PSSGP_NMAX ((int64_t)1 << 40)

/* ---- status codes ------------------------------------------------------ */
#define PSSGP_OK 0
#define PSSGP_EINVAL (-1)      /* null pointer, n < 1 or > PSSGP_NMAX, ld < n, bad flag */
#define PSSGP_EDIM (-2)        /* d outside 1..PSSGP_DMAX                      */
#define PSSGP_EKERNEL (-3)     /* unknown kernel kind or invalid hyperparameter */
#define PSSGP_EWORKSPACE (-4)  /* workspace too small or misaligned            */
#define PSSGP_ECUDA (-5)       /* a CUDA runtime call failed                   */
#define PSSGP_EMODEL (-6)      /* model formation failed (Lyapunov/roots)      */
#define PSSGP_ESCRATCH (-7)    /* problem too large for the built-in scratch of
                                  pssgp_loglik_noalloc                          */
/* device-detected errors, OR-ed into the workspace status word */
#define PSSGP_ENAN 1           /* non-finite time or observed y                 */
#define PSSGP_EUNSORTED 2      /* times decrease somewhere                      */
#define PSSGP_ENOTPD 4         /* innovation variance or a pivot <= 0 / singular */
#define PSSGP_EBATCH 8         /* batched: bad offsets or a non-positive parameter */

/* ---- model ------------------------------------------------------------- */
#define PSSGP_MATERN12 1
#define PSSGP_MATERN32 2
#define PSSGP_MATERN52 3
#define PSSGP_RBF 4            /* Taylor approximation of the spectral density */

typedef struct pssgp_kernel {
  int32_t kind;          /* PSSGP_MATERN12 / 32 / 52 / PSSGP_RBF             */
  int32_t order;         /* RBF Taylor order n (state dimension d = n), 1..8 */
  double lengthscale;    /* > 0                                              */
  double variance;       /* > 0 (sigma^2 of the covariance function)         */
  int32_t balance;       /* 1: Sec. 4.2 diagonal balancing, 0: none          */
  int32_t reserved;
} pssgp_kernel;

/* Number of Taylor coefficients kept per matrix entry for the on-device
 * discretisation (see pssgp_model.fc / qc). */
#define PSSGP_NTAYLOR 16

/* Host-side model: the continuous SDE of Eq. (ssmodel) in balanced
 * coordinates z = D^{-1} x (Sec. 4.2), with the stationary covariance of
 * Sec. 4.1 and the tables the device discretisation uses.  Filled by
 * pssgp_model_build or pssgp_model_from_sde; plain data, copyable. */
typedef struct pssgp_model {
  int32_t d;
  int32_t kind;                          /* as pssgp_kernel.kind, 0 for a user SDE */
  double G[PSSGP_DMAX * PSSGP_DMAX];     /* drift, balanced, row-major d x d    */
  double W[PSSGP_DMAX * PSSGP_DMAX];     /* L q L^T, balanced                  */
  double Pinf[PSSGP_DMAX * PSSGP_DMAX];  /* stationary covariance, balanced    */
  double D[PSSGP_DMAX];                  /* x = D z; then H = e_0^T            */
  double gnorm;                          /* ||G||_1, balanced (information)    */
  /* Taylor tables (row-major entry e = i*d+j):
   *   F_e(h) = sum_m fc[e*PSSGP_NTAYLOR + m] h^m            (G^m / m!)
   *   Q_e(h) = h * sum_m qc[e*PSSGP_NTAYLOR + m] h^m         (W_{m+1} / (m+1)!,
   *            W_1 = W, W_{m+1} = G W_m + W_m G^T)
   * hthr_f[K] / hthr_q[K]: largest step h for which K terms keep the
   * truncation below 2^-54 (relative), from the exact norms ||G^m||_1 and
   * ||W_m||_1; steps longer than hmax are halved and doubled back. */
  double fc[PSSGP_DMAX * PSSGP_DMAX * PSSGP_NTAYLOR];
  double qc[PSSGP_DMAX * PSSGP_DMAX * PSSGP_NTAYLOR];
  double hthr_f[PSSGP_NTAYLOR + 1];
  double hthr_q[PSSGP_NTAYLOR + 1];
  double hmax;
  /* companion structure (rows 0..d-2 of G have only the superdiagonal
   * entry): then row i+1 of exp(hG) = sum of row i times rsup / rlast,
   *   F[i+1][j] = F[i][j-1] rsup[i*d+j] + F[i][d-1] rlast[i*d+j],
   * and only row 0 needs the Taylor series. */
  int32_t companion;
  int32_t reserved2;
  double rsup[PSSGP_DMAX * PSSGP_DMAX];
  double rlast[PSSGP_DMAX * PSSGP_DMAX];
  double lengthscale, variance;          /* metadata                            */
  /* hthr_f32[K] / hthr_q32[K]: largest step h for which the terms from K on
   * stay below 2^-36 (relative, same exact norms); those terms may be summed
   * in FP32 (error below 2^-55).  All 0 when a coefficient is outside the
   * FP32-safe range [1e-30, 1e30]. */
  double hthr_f32[PSSGP_NTAYLOR + 1];
  double hthr_q32[PSSGP_NTAYLOR + 1];
} pssgp_model;

/* Kernel -> SDE (G, L, q, H) (Sec. 2: exact for Matern nu = 1/2, 3/2, 5/2;
 * order-n Taylor approximation of the RBF spectral density followed by
 * spectral factorisation), stationary covariance by the vectorised Lyapunov
 * solve (Sec. 4.1), optional balancing (Sec. 4.2), discretisation tables.
 * Host only.  Returns PSSGP_EKERNEL for bad hyperparameters, PSSGP_EDIM for
 * an RBF order outside 1..8, PSSGP_EMODEL if the factorisation or the
 * Lyapunov solve fails. */
int pssgp_model_build(const pssgp_kernel* kernel, pssgp_model* out);

/* Same from an explicit SDE dx = G x dt + L dw, E[w w^T] = q, y = H x + e
 * (Eq. (ssmodel)).  Host pointers, G row-major d x d, L and H length d.
 * H must be a multiple of the first unit vector (H = h0 e_0^T, h0 != 0). */
int pssgp_model_from_sde(int32_t d, const double* G, const double* L, double q,
                         const double* H, int32_t balance, pssgp_model* out);

/* ---- workspace --------------------------------------------------------- */
/* Bytes of device workspace for a call on n merged steps with state
 * dimension d (valid for every entry point below with the same n, d, and
 * for every scan tuning: sized for the largest lane count). */
size_t pssgp_workspace_size(int32_t d, int64_t n);

/* Copies the device status word of the last call that used `ws` to *status,
 * synchronising `stream`.  Returns PSSGP_ECUDA on a CUDA error. */
int pssgp_get_status(void* ws, void* stream, int32_t* status);

/* ---- merge (Sec. 4.3) -------------------------------------------------- */
/* Inserts the M sorted prediction times into the N sorted training times as
 * missing measurements (stable: a training time precedes an equal prediction
 * time).  Outputs (device, length N+M): t, y (0 at prediction steps), mask
 * (1 observed, 0 missing); test_pos[j] = merged index of prediction j.
 * Unsorted input sets PSSGP_EUNSORTED, non-finite times PSSGP_ENAN.  The
 * workspace only carries the status word (>= 256 bytes). */
int pssgp_merge(const double* t_train, const double* y_train, int64_t N,
                const double* t_test, int64_t M,
                double* t, double* y, uint8_t* mask, int64_t* test_pos,
                void* ws, size_t ws_bytes, void* stream);

/* ---- discretisation (supplement Eq. (ss-gp-formation)) ------------------ */
/* For each step k: F_k = exp(G (t_k - t_{k-1})), Q_k = int_0^h e^{(h-s)G} W
 * e^{(h-s)G}^T ds, k >= 1; F_0 = 0, Q_0 = P_inf (the prior at the first time).
 * F: d*d entries x ld (entry i*d+j), Q: packed d(d+1)/2 x ld, in SDE
 * coordinates.  The workspace only carries the status word (>= 256 bytes). */
int pssgp_discretize(const pssgp_model* model, const double* t, int64_t n,
                     double* F, double* Q, int64_t ld,
                     void* ws, size_t ws_bytes, void* stream);

/* ---- filter (Sec. 3, Prop. 1) ------------------------------------------ */
/* Parallel Kalman filter: elements (A, b, C, eta, J) with missing
 * measurements (Sec. 3), combined by the filtering operator in a two-level
 * parallel scan; x_k = b*_k, P_k = C*_k (Prop. 1).  mask[k] = 0 marks a
 * missing measurement; a non-finite y at an observed step is taken as missing
 * and sets PSSGP_ENAN.  R: device pointer to one noise variance (R_per_step
 * = 0) or n of them (R_per_step = 1).  Outputs (nullable): xf d x ld,
 * Pf packed x ld, loglik (one device double, the log marginal likelihood by
 * prediction-error decomposition over the observed steps). */
int pssgp_filter(const pssgp_model* model, const double* t, const double* y,
                 const uint8_t* mask, const double* R, int32_t R_per_step,
                 int64_t n, double* xf, double* Pf, int64_t ld, double* loglik,
                 void* ws, size_t ws_bytes, void* stream);

/* ---- smoother (supplement Prop. 2) ------------------------------------- */
/* Parallel RTS smoother from the filter outputs xf, Pf (as written by
 * pssgp_filter, same ld): elements (E, g, L), reverse two-level scan of the
 * smoothing operator; m^s_k = g*_k, P^s_k = L*_k.  Outputs (nullable):
 * f_mean[k] = H m^s_k, f_var[k] = H P^s_k H^T (length n), xs d x ld,
 * Ps packed x ld. */
int pssgp_smooth(const pssgp_model* model, const double* t,
                 const double* xf, const double* Pf, int64_t n, int64_t ld,
                 double* f_mean, double* f_var, double* xs, double* Ps,
                 void* ws, size_t ws_bytes, void* stream);

/* ---- log marginal likelihood (Sec. 2, parameter estimation) ------------- */
/* The filter's log-likelihood only (no per-step output). */
int pssgp_loglik(const pssgp_model* model, const double* t, const double* y,
                 const uint8_t* mask, const double* R, int32_t R_per_step,
                 int64_t n, double* loglik, void* ws, size_t ws_bytes, void* stream);

/* Log marginal likelihoods of a batch of B independent series in one pass
 * (the hyperparameter search of Sec. 2 and Sec. 5 evaluates many
 * (lengthscale, variance, noise) candidates or many series at once).
 *  - Series s occupies steps offsets[s] .. offsets[s+1]-1 of t, y, mask
 *    (device arrays of length n; t sorted within each series).  offsets:
 *    device int64[B + 1], offsets[0] = 0, non-decreasing, offsets[B] = n;
 *    empty series are allowed and get loglik 0.
 *  - params: device double[3 B], per series (lengthscale, variance, noise
 *    variance R), all > 0.
 *  - model: any pssgp_model_build result of the kernel family; its
 *    lengthscale and variance fields say where it was built.  Series s uses
 *    the same family at (lengthscale_s, variance_s): for a stationary kernel
 *    whose covariance is variance * k(tau / lengthscale) the state-space
 *    model rescales exactly (F(h) -> F(h l0 / l), Q -> Q v / v0 in the
 *    time-scaled state coordinates, which leave H x unchanged).  Returns
 *    PSSGP_EMODEL if those fields are not positive and finite (a model from
 *    pssgp_model_from_sde carries none).
 *  - Each series starts from the stationary prior (F = 0, Q = P_inf), so
 *    the concatenation filters every series independently.
 *  - loglik: device double[B].  ws: pssgp_workspace_size(d, n) bytes.
 *  - Device status (pssgp_get_status): PSSGP_EBATCH for bad offsets or a
 *    non-positive parameter, plus the bits of pssgp_filter.
 *  - Failed series: a series with a parameter that is not positive and
 *    finite (PSSGP_EBATCH), a time that is not finite (PSSGP_ENAN) or
 *    decreases (PSSGP_EUNSORTED), or a non-finite y at an observed step
 *    (PSSGP_ENAN) gets loglik NaN (and, in pssgp_loglik_grad_batched, a NaN
 *    gradient row) and leaves every other series' results intact: before the
 *    scan its parameters become unit scales, its bad times zero-length steps
 *    and its bad observations missing ones, so nothing non-finite enters the
 *    flat scan.  The status word carries the union of all series' bits. */
int pssgp_loglik_batched(const pssgp_model* model, const int64_t* offsets,
                         int32_t B, const double* params, const double* t,
                         const double* y, const uint8_t* mask, int64_t n,
                         double* loglik, void* ws, size_t ws_bytes,
                         void* stream);

/* Posterior predictions of a batch of B independent series in one pass
 * (Sec. 4.3 per series: each series' prediction times merged into its
 * training times as missing measurements, then filter, smoother and
 * log-likelihood over the concatenation, as pssgp_predict for one series).
 *  - Series s: training times/values t_train, y_train at
 *    train_offsets[s] .. train_offsets[s+1]-1 (device arrays of length N)
 *    and prediction times t_test at test_offsets[s] .. test_offsets[s+1]-1
 *    (length M); both sorted within each series.  Offsets: device
 *    int64[B + 1], starting at 0, non-decreasing, ending at N (M).  A series
 *    may have no training or no prediction times (no training times: the
 *    prior at its prediction times).
 *  - params, model: as pssgp_loglik_batched (per series lengthscale,
 *    variance, noise variance R; the model of the family carries where it
 *    was built).
 *  - Outputs (device): mean_test, var_test: double[M], the posterior mean
 *    and variance of f at each prediction time, in the order of t_test;
 *    loglik (nullable): double[B], each series' log marginal likelihood.
 *  - Ties: a training time equal to a prediction time goes first.
 *  - Failed series (as pssgp_loglik_batched, and decreasing or non-finite
 *    training or prediction times): NaN outputs and loglik; the other series
 *    are not affected.  Bad offsets: PSSGP_EBATCH in the status word.
 *  - ws: pssgp_predict_batched_workspace_size(d, N, M, B) bytes (0 for
 *    arguments out of range). */
size_t pssgp_predict_batched_workspace_size(int32_t d, int64_t N, int64_t M,
                                            int32_t B);
int pssgp_predict_batched(const pssgp_model* model,
                          const int64_t* train_offsets,
                          const int64_t* test_offsets, int32_t B,
                          const double* params, const double* t_train,
                          const double* y_train, int64_t N,
                          const double* t_test, int64_t M, double* mean_test,
                          double* var_test, double* loglik, void* ws,
                          size_t ws_bytes, void* stream);

/* ---- gradient of the log marginal likelihood ------------------------------ */
/* d loglik / d(log lengthscale, log variance, log noise variance) by adjoint
 * (reverse-mode) scans: the filter pass stores the predicted moments, then
 * two backward scans of the smoothing operator's form (supplement Prop. 2)
 * give the adjoints of the predicted mean and covariance at every step, from
 * which the three derivatives are summed (dF/dlog l = -tau G F,
 * dQ/dlog l = -tau (G Q + Q G^T + W), dQ/dlog s2 = Q).  The model must come
 * from pssgp_model_build (its lengthscale and variance are the point of
 * differentiation; a model from pssgp_model_from_sde has none: the result is
 * then the derivative for the rescaled family of that SDE).  d/dlog R scales
 * every R_k together.
 * Workspace: pssgp_workspace_size_grad(d, n) bytes (larger than
 * pssgp_workspace_size: it holds the forward moments of every step). */
size_t pssgp_workspace_size_grad(int32_t d, int64_t n);

/* One series.  loglik: one device double (nullable); grad: device double[3]. */
int pssgp_loglik_grad(const pssgp_model* model, const double* t,
                      const double* y, const uint8_t* mask, const double* R,
                      int32_t R_per_step, int64_t n, double* loglik,
                      double* grad, void* ws, size_t ws_bytes, void* stream);

/* B series as in pssgp_loglik_batched.  loglik: device double[B] (nullable);
 * grad: device double[B][3], per series d/d(log l, log s2, log R) at its own
 * parameters. */
int pssgp_loglik_grad_batched(const pssgp_model* model, const int64_t* offsets,
                              int32_t B, const double* params, const double* t,
                              const double* y, const uint8_t* mask, int64_t n,
                              double* loglik, double* grad, void* ws,
                              size_t ws_bytes, void* stream);

/* ---- one long series split over several GPUs (Sec. 3, Prop. 1; supplement
 * Prop. 2) --------------------------------------------------------------------
 * The scans over time are scans of associative operators, so a series cut
 * into G contiguous chunks (chunk r on GPU r: its steps, in time order, after
 * those of chunk r-1) needs one exchange per direction:
 *   1. every rank: pssgp_split_filter_reduce -> its chunk's filter aggregate;
 *   2. all-gather the G filter aggregates (rank order) into aggs_f[G][nf];
 *   3. every rank: pssgp_split_filter_finish -> its filter outputs, the
 *      log-likelihood of its observations given all earlier ones (the chunks
 *      before it enter its scan as one element: their aggregates folded) and,
 *      with smoother = 1, its smoother elements (fused, as in pssgp_predict);
 *   4. every rank: pssgp_split_smooth_reduce -> its chunk's smoother aggregate;
 *   5. all-gather the G smoother aggregates into aggs_s[G][ns]; all-reduce
 *      (sum) the log-likelihoods;
 *   6. every rank: pssgp_split_smooth_finish -> its smoother outputs (the
 *      chunks after it folded into the smoothed state of its last step).
 * Chunk r's smoother aggregate covers the elements of its steps -1 .. n-2
 * (step -1: the last step of chunk r-1, whose filter state chunk r starts
 * from; chunk 0 has none, the last chunk also covers its step n-1), so the
 * chunks after r fold into the smoothed state of r's last step.
 * The first and last time of every chunk must be known to its neighbours
 * (t_prev: the time of the last step of chunk r-1; t_next: the time of the
 * first step of chunk r+1; NaN at the ends of the series).  Every rank uses
 * the same model.  Aggregates are device arrays of pssgp_split_agg_doubles
 * doubles in the library's internal (balanced) coordinates: opaque, to be
 * passed between these calls unchanged.  The workspace (pssgp_workspace_size
 * (d, n) bytes, n = the chunk's steps) carries state from each call to the
 * next: use the same workspace, inputs and scan tuning for all four.  A
 * *_reduce call of the filter clears the status word; the other calls add
 * their bits to it.  With G = 1 and smoother = 1 the sequence computes what
 * pssgp_predict computes on merged inputs.
 *
 * The gradient of the log-likelihood (as pssgp_loglik_grad) over a split
 * series takes smoother = 2 in steps 1 and 3 (the filter pass then keeps the
 * predicted moments and forms the mean adjoint's lane aggregates) and a
 * workspace of pssgp_workspace_size_grad(d, n) bytes, then two backward
 * exchanges instead of steps 4-6:
 *   4'. every rank: pssgp_split_grad_mean_reduce -> its chunk's mean-adjoint
 *       aggregate (Pi, gamma: mb_first = Pi mb_after + gamma, mb the adjoint
 *       of a predicted mean);
 *   5'. all-gather them; every rank: pssgp_split_grad_mean_finish (the
 *       chunks after it folded into the mean adjoint after its last step)
 *       -> its covariance-adjoint aggregate (Pi, L: Mb_first =
 *       Pi Mb_after Pi^T + L);
 *   6'. all-gather those; every rank: pssgp_split_grad_finish -> its chunk's
 *       three derivative sums; all-reduce (sum) them and the
 *       log-likelihoods.
 * The transition from a chunk's first time back to t_prev belongs to that
 * chunk (its derivative terms are summed there), the one after its last
 * step to the next chunk; step 3 also discretises the latter (t_next) for
 * the adjoints.  Every aggregate of 4'-6' has pssgp_split_agg_doubles(d, 1)
 * doubles and the smoother's operator (E = Pi, g, L). */

/* Doubles in one chunk aggregate: filter (smoother = 0) 2 d^2 + 3 d
 * (A, b, C, eta, J), smoother or adjoint (smoother = 1) d^2 + d + d(d+1)/2
 * (E, g, L); 0 for d outside 1..PSSGP_DMAX. */
int32_t pssgp_split_agg_doubles(int32_t d, int32_t smoother);

/* Step 1: discretises the chunk (step 0 is the transition from t_prev, or
 * the series' first step if t_prev is NaN), folds its filtering elements
 * (Sec. 3) and writes the chunk's aggregate to agg (device,
 * pssgp_split_agg_doubles(d, 0) doubles).  smoother: 0 filter and
 * log-likelihood, 1 step 3 will prepare the smoother, 2 the gradient (the
 * gradient's workspace size); t_next: as above.  Other arguments as
 * pssgp_filter for the chunk's n steps.  PSSGP_EINVAL for another value of
 * smoother or a time argument that is infinite. */
int pssgp_split_filter_reduce(const pssgp_model* model, const double* t,
                              const double* y, const uint8_t* mask,
                              const double* R, int32_t R_per_step, int64_t n,
                              double t_prev, double t_next, int32_t smoother,
                              double* agg, void* ws, size_t ws_bytes,
                              void* stream);

/* Step 3: aggs: device array of the G chunks' filter aggregates in rank
 * order; the ones before `rank` are folded into the filter state before the
 * chunk.  Outputs as pssgp_filter (xf, Pf nullable; with both null and
 * smoother = 0 only the log-likelihood is formed); loglik (nullable, one
 * device double): the sum over the chunk's observations of
 * log p(y_k | all earlier y).  t_next and smoother as in step 1 (the same
 * values). */
int pssgp_split_filter_finish(const pssgp_model* model, const double* t,
                              const double* y, const uint8_t* mask,
                              const double* R, int32_t R_per_step, int64_t n,
                              double t_next, int32_t smoother,
                              const double* aggs, int32_t G, int32_t rank,
                              double* xf, double* Pf, int64_t ld,
                              double* loglik, void* ws, size_t ws_bytes,
                              void* stream);

/* Step 4 (after step 3 with smoother = 1): writes the chunk's smoother
 * aggregate (supplement Prop. 2) to agg (device,
 * pssgp_split_agg_doubles(d, 1) doubles). */
int pssgp_split_smooth_reduce(const pssgp_model* model, int64_t n, double* agg,
                              void* ws, size_t ws_bytes, void* stream);

/* Step 6: aggs: device array of the G chunks' smoother aggregates in rank
 * order; the ones after `rank` are folded into the smoothed state of the
 * chunk's last step.  Outputs as pssgp_smooth (all nullable). */
int pssgp_split_smooth_finish(const pssgp_model* model, int64_t n, int64_t ld,
                              const double* aggs, int32_t G, int32_t rank,
                              double* f_mean, double* f_var, double* xs,
                              double* Ps, void* ws, size_t ws_bytes,
                              void* stream);

/* Step 4' (after step 3 with smoother = 2): writes the chunk's mean-adjoint
 * aggregate to agg (device, pssgp_split_agg_doubles(d, 1) doubles). */
int pssgp_split_grad_mean_reduce(const pssgp_model* model, int64_t n,
                                 double* agg, void* ws, size_t ws_bytes,
                                 void* stream);

/* Step 5': aggs: device array of the G chunks' mean-adjoint aggregates in
 * rank order; the ones after `rank` are folded into the mean adjoint after
 * the chunk.  Writes the chunk's covariance-adjoint aggregate to agg_cov
 * (device, pssgp_split_agg_doubles(d, 1) doubles). */
int pssgp_split_grad_mean_finish(const pssgp_model* model, int64_t n,
                                 const double* aggs, int32_t G, int32_t rank,
                                 double* agg_cov, void* ws, size_t ws_bytes,
                                 void* stream);

/* Step 6': aggs_cov: device array of the G chunks' covariance-adjoint
 * aggregates in rank order.  grad: device double[3], the chunk's terms of
 * d loglik / d(log lengthscale, log variance, log noise variance); their sum
 * over the ranks is pssgp_loglik_grad's gradient of the whole series.  R and
 * R_per_step as in step 1. */
int pssgp_split_grad_finish(const pssgp_model* model, const double* R,
                            int32_t R_per_step, int64_t n,
                            const double* aggs_cov, int32_t G, int32_t rank,
                            double* grad, void* ws, size_t ws_bytes,
                            void* stream);

/* Allocation-free variant of pssgp_loglik for callers that cannot allocate
 * device memory themselves -- for instance a plugin inside a host program
 * that owns every device allocation and does not let third-party code call
 * cudaMalloc, or a latency-critical loop that must never enter the driver's
 * allocator -- and therefore cannot pass a workspace.  The paper has no
 * counterpart; this is a deployment convenience.
 *  - Scratch: a fixed 32 MiB array inside the library's device image, held on
 *    every GPU that loads the library until the process exits.  That bounds
 *    the problem size: the workspace of the current scan tuning must fit in
 *    32 MiB, which allows n (merged steps) up to 290,464 at d = 1, 137,780
 *    at d = 2, 78,582 at d = 3, 24,593 at d = 6 and 14,573 at d = 8 (the
 *    largest n with pssgp_workspace_size(d, n) <= 32 MiB; per-step records
 *    plus the per-chunk aggregates).  Larger problems are rejected with PSSGP_ESCRATCH
 *    before anything is launched.
 *  - Every call looks up the scratch's device address in the current device's
 *    context (cudaGetSymbolAddress, with that device current); the first call
 *    on a device also loads the library's device code there, so make that
 *    first call before any stream capture.
 *  - All calls share the one scratch array per device, so calls that overlap
 *    on the GPU (different streams or threads) race and give wrong results;
 *    serialise them.  Nothing from a previous call is reused: the status word
 *    is cleared at the start, everything else is written before it is read.
 *  - Arguments as pssgp_loglik; `status` (device pointer to one int32,
 *    nullable) receives the device status bits of this call.  The per-kernel
 *    timing diagnostic (pssgp_timing) creates CUDA events, so while it is on
 *    this call returns PSSGP_EINVAL without launching anything. */
int pssgp_loglik_noalloc(const pssgp_model* model, const double* t, const double* y,
                         const uint8_t* mask, const double* R, int32_t R_per_step,
                         int64_t n, double* loglik, int32_t* status, void* stream);

/* ---- fused prediction path (Sec. 4.4, stages 4-5) ---------------------- */
/* merge -> discretise -> parallel filter -> parallel smoother -> gather, with
 * the smoother elements produced inside the filter pass.  Inputs: N sorted
 * training times/observations, M sorted prediction times, scalar noise
 * variance R (host value, > 0).  Outputs (device, length M): posterior mean
 * and variance of f at the prediction times; loglik (nullable, one device
 * double) of the training data.  Workspace: pssgp_workspace_size(d, N+M). */
int pssgp_predict(const pssgp_model* model, const double* t_train,
                  const double* y_train, int64_t N, const double* t_test,
                  int64_t M, double R, double* mean_test, double* var_test,
                  double* loglik, void* ws, size_t ws_bytes, void* stream);

/* pssgp_predict from and to HOST memory: copies the inputs (host arrays
 * t_train, y_train [N], t_test [M]) into staging after the workspace, runs
 * pssgp_predict, and copies mean_test, var_test [M] and loglik (nullable,
 * one double) back to host memory, all enqueued on `stream` (asynchronous:
 * synchronise the stream before reading the outputs).  With page-locked host
 * buffers the copies are truly asynchronous, so calls on two streams with two
 * workspaces overlap one call's copies with another's kernels.  Workspace:
 * pssgp_predict_host_workspace_size(d, N, M) bytes. */
size_t pssgp_predict_host_workspace_size(int32_t d, int64_t N, int64_t M);
int pssgp_predict_host(const pssgp_model* model, const double* t_train,
                       const double* y_train, int64_t N, const double* t_test,
                       int64_t M, double R, double* mean_test, double* var_test,
                       double* loglik, void* ws, size_t ws_bytes, void* stream);

/* ---- diagnostics ------------------------------------------------------- */
/* Chunk aggregates of the filter's first scan level, for tests: runs the
 * filter on (t, y, mask, R) with `lanes` lanes (a multiple of 128, 0 =
 * automatic) and copies lane c's within-chunk aggregate (A, b, C, eta, J in SDE
 * coordinates, row-major d x d / d, 3 d^2 + 2 d doubles) to the HOST array
 * agg + c*(3d^2+2d), and chunk c's first step to first[c] (host), after
 * synchronising.  Needs pssgp_workspace_size(d, n) + lanes*(2d^2+3d)*8 bytes
 * of workspace.  The lane count used is returned in *lanes_out. */
int pssgp_debug_filter_aggregates(const pssgp_model* model, const double* t,
                                  const double* y, const uint8_t* mask,
                                  const double* R, int64_t n, int32_t lanes,
                                  double* agg, int64_t* first, int32_t* lanes_out,
                                  void* ws, size_t ws_bytes, void* stream);

/* Per-kernel timing for measurement (not for use inside stream capture):
 * mode 1 enables it and resets the totals, mode 0 disables it, mode 2 waits
 * for the recorded CUDA events and copies the summed milliseconds and launch
 * counts of up to nslots kernels (host arrays) to ms / counts.  While enabled
 * every launch is bracketed by two events on its own stream. */
int pssgp_timing(int32_t mode, double* ms, int64_t* counts, int32_t nslots);
/* Name of timing slot `slot` ("" if unused). */
const char* pssgp_timing_name(int32_t slot);

/* Scan tuning: the number of chunks ("lanes", one per thread) of the scans
 * is SMs x warps_per_sm x 32 (rounded up to whole blocks of 128), i.e.
 * n / (SMs x warps_per_sm x 32) steps per thread; warps_per_sm is 1 to 16
 * (default 8 for d <= 3, else 4).  More lanes give each SM more warps to
 * hide latency but shorter chunks and more scan overhead.  Below 4 one call
 * leaves SMs idle: meant for several independent calls in flight on
 * different streams, where fewer, longer chunks per call cut the scan
 * overhead per step while the calls together fill the GPU.  PSSGP_EINVAL
 * outside 1..16.  Affects calls planned afterwards.  pssgp_set_warps_per_sm sets every state
 * dimension; pssgp_tune_set one (PSSGP_EDIM for d outside 1..8);
 * pssgp_tune_get returns the current value for d. */
int pssgp_set_warps_per_sm(int32_t warps_per_sm);
int pssgp_tune_set(int32_t d, int32_t warps_per_sm);
int pssgp_tune_get(int32_t d);

/* Autotuner: runs pssgp_loglik_batched (same arguments) once per candidate
 * warps_per_sm (4, 8, 12, 16) to warm up and then `reps` times between two
 * CUDA events on `stream`; keeps the fastest for model->d (pssgp_tune_set)
 * and reports it in *best_warps and its mean milliseconds per call in
 * *best_ms (nullable).  Synchronises `stream`.  On an error the previous
 * tuning is restored and the error returned. */
int pssgp_autotune_loglik_batched(const pssgp_model* model,
                                  const int64_t* offsets, int32_t B,
                                  const double* params, const double* t,
                                  const double* y, const uint8_t* mask,
                                  int64_t n, double* loglik, void* ws,
                                  size_t ws_bytes, void* stream, int32_t reps,
                                  int32_t* best_warps, float* best_ms);

/* ---- batched fit (Sec. 2: hyperparameters by maximising the marginal
 * likelihood) -------------------------------------------------------------- */
#define PSSGP_FIT_ADAM 0
#define PSSGP_FIT_LBFGS 1
typedef struct pssgp_fit_options {
  int32_t max_iter;      /* evaluations at most (e.g. 2000)                     */
  int32_t patience;      /* converged after this many iterations in a row with  */
  double tol;            /*   |l_t - l_{t-1}| / n_s < tol (e.g. 10, 1e-7)        */
  double lr;             /* Adam step on the log hyperparameters (e.g. 0.05)     */
  double beta1, beta2, eps;  /* Adam constants (0.9, 0.999, 1e-8)               */
  int32_t check_every;   /* read the converged flags and drop converged series  */
                         /*   from the scans every this many iterations (1 is  */
                         /*   usually fastest: the read is B bytes, and frozen */
                         /*   series still cost a full evaluation each)        */
  int32_t method;        /* PSSGP_FIT_ADAM, or PSSGP_FIT_LBFGS: limited-memory
                          * BFGS (6 pairs) with Armijo backtracking, steps of
                          * at most 2 in every log parameter; the convergence
                          * test runs on accepted steps; lr and the Adam
                          * constants are unused */
} pssgp_fit_options;

/* Bytes of device workspace for pssgp_fit_batched. */
size_t pssgp_fit_workspace_size(int32_t d, int64_t n, int32_t B);

/* Fits (log lengthscale, log variance, log noise variance) of B series by
 * Adam ascent or L-BFGS on each series' exact log marginal likelihood, with
 * the gradient of pssgp_loglik_grad_batched; every loop iteration evaluates
 * all series still being fitted in one call.
 *  - offsets_host: HOST int64[B + 1] (as pssgp_loglik_batched's offsets);
 *    t, y, mask: device arrays of length n.
 *  - theta: device double[B][3], the starting point in, the fitted log
 *    hyperparameters out (a converged series keeps the theta at which its
 *    convergence test passed).
 *  - loglik: device double[B], the log-likelihood at the returned theta;
 *    iters: device int32[B], the evaluations each series used (0 for empty
 *    series).  *iterations_run (host, nullable): iterations of the loop.
 *  - A series whose log-likelihood or gradient becomes non-finite stops.
 *  - Synchronises `stream` every check_every iterations (the converged flags
 *    are read on the host to re-pack the remaining series) and at the end.
 * Not capturable in a CUDA graph (it synchronises). */
int pssgp_fit_batched(const pssgp_model* model, const int64_t* offsets_host,
                      int32_t B, const double* t, const double* y,
                      const uint8_t* mask, int64_t n, double* theta,
                      double* loglik, int32_t* iters,
                      const pssgp_fit_options* opt, void* ws, size_t ws_bytes,
                      void* stream, int32_t* iterations_run);

/* ---- learned initialisation of the fit --------------------------------------
 * A small network proposes initial log hyperparameters for the marginal-
 * likelihood fit from a log periodogram of each series; it is trained on
 * series simulated from the state-space prior itself. */

/* Simulates B series from the prior of the model's kernel family at
 * per-series (lengthscale, variance, noise variance) = params[3 s .. 3 s + 2]
 * (device double[3 B]); series s has offsets[s + 1] - offsets[s] steps
 * (device int64[B + 1]).  Times: t_0 = 0, t_k = t_{k-1} - spacing log u_k (a
 * Poisson process of mean spacing `spacing`); state: x_0 ~ N(0, P_inf),
 * x_k = F_k x_{k-1} + chol(Q_k) z_k; y_k = f(t_k) + sqrt(R) z'_k.  Random
 * numbers: Philox4x32-10 with key (seed mod 2^32, seed / 2^32); step k of
 * series s uses counter (k, s, 0, 0) for the time increment (first 53-bit
 * uniform (a 2^21 + b / 2^11 + 1/2) 2^-53 of words a, b) and counters
 * (k, s, j, 0), j >= 1, for Box-Muller pairs of normals: the d state
 * normals, then the measurement normal.  chol(.) is the lower Cholesky
 * factor with a zero column where a pivot is at most 1e-10 of its diagonal
 * entry.  Outputs t, y: device double[n].  status: device int32, set to
 * PSSGP_ENAN if a value is not finite.  The model must come from
 * pssgp_model_build (PSSGP_EMODEL otherwise). */
int pssgp_simulate_prior(const pssgp_model* model, const int64_t* offsets,
                         int32_t B, const double* params, uint64_t seed,
                         double spacing, double* t, double* y, int32_t* status,
                         void* stream);

/* 65 features per series (device float[B][65]): log(P_j + 1e-8), j < 64, and
 * log s2, where s2 is the series' variance, dbar its mean spacing
 * (t_{n-1} - t_0) / (n - 1), A(w) = |sum_k (y_k - ybar) exp(-i w k dbar)|^2
 * / (n s2) the periodogram on the regular grid k dbar, and P_j the mean of
 * A at w_lo r^(j + (q - 3/2) / 4), q < 4, r = (w_hi / w_lo)^(1/63),
 * w_lo = 2 pi / 40.96, w_hi = 0.9 pi / 0.01; zeros for a series with fewer
 * than 2 steps or s2 = 0.  Computed in FP32 (phase re-anchored from FP64
 * every 128 steps). */
int pssgp_features(const int64_t* offsets, int32_t B, const double* t,
                   const double* y, float* feat, void* stream);

/* The network 65 -> 256 -> 256 -> 3 (ReLU), standardised inputs and outputs,
 * BF16 GEMMs on the tensor cores with FP32 accumulation, FP32 parameters and
 * Adam state.  `state`: a device buffer of pssgp_mlp_state_bytes() bytes
 * (256-byte aligned).  Parameter layout (pssgp_mlp_param_count() floats):
 * W1[256][80] (columns >= 65 zero), b1[256], W2[256][256], b2[256],
 * W3[16][256] (rows >= 3 zero), b3[16].  Normalisation block (144 floats):
 * feature mean[65], sd[65], target mean[3], sd[3].  Targets are log
 * hyperparameters (log l, log s2, log R), device double[rows][3]. */
size_t pssgp_mlp_state_bytes(void);
int32_t pssgp_mlp_param_count(void);
/* Device workspace for a minibatch (or prediction batch) of `rows` rows. */
size_t pssgp_mlp_workspace_size(int32_t rows);
/* Normalisation statistics from nrows training rows, He-uniform weights from
 * Philox4x32-10 (seed), zero biases and Adam state. */
int pssgp_mlp_init(void* state, uint64_t seed, const float* feat,
                   int64_t nrows, const double* theta, void* stream);
/* Sets parameters and normalisation (device float arrays in the layouts
 * above) and clears the Adam state. */
int pssgp_mlp_set_params(void* state, const float* params, const float* norm,
                         void* stream);
/* Loss 1/(2 rows) sum over rows and the 3 outputs of (out - target)^2 in
 * standardised units, its gradient (device float[param_count], layout
 * above), the loss (device float, nullable) and the raw outputs (device
 * float[rows][16], nullable).  rows must be a multiple of 8. */
int pssgp_mlp_grad(void* state, const float* feat, const double* theta,
                   int32_t rows, float* grad, float* loss, float* out,
                   void* ws, size_t ws_bytes, void* stream);
/* One Adam step (0.9, 0.999, 1e-8; step counts from 1) on the parameters. */
int pssgp_mlp_adam(void* state, const float* grad, float lr, int32_t step,
                   void* stream);
/* The network's GEMMs run on the 5th-generation tensor cores (tcgen05.mma
 * with the accumulator in tensor memory, operands loaded by TMA) unless
 * path = 1 selects the legacy mma.sync kernel (kept as a checked baseline).
 * Affects calls made afterwards.  A GEMM whose waits time out sets a word in
 * the workspace instead of hanging; PSSGP_ECUDA if a TMA descriptor cannot be
 * made. */
int pssgp_mlp_set_gemm(int32_t path);

/* Diagnostic: C[M][N] = A[M][K] B[N][K]^T (device bf16 row-major inputs, K a
 * multiple of 8; C device float row-major) with the GEMM of `path` (0
 * tcgen05, 1 mma.sync); *err (device int32) is cleared, and set to 1 if the
 * tcgen05 kernel's waits timed out. */
int pssgp_debug_gemm_bf16(const void* A, const void* B, int32_t M, int32_t N,
                          int32_t K, float* C, int32_t path, int32_t* err,
                          void* stream);

/* Proposed log hyperparameters (device double[rows][3]); a row with a
 * non-finite feature, or whose standardised output is not finite or lies
 * more than 4 standard deviations
 * of the training targets from their mean gets the plain default 0
 * (l = s2 = R = 1) instead. */
int pssgp_mlp_predict(const void* state, const float* feat, int32_t rows,
                      double* theta, void* ws, size_t ws_bytes, void* stream);

/* ---- CUDA graphs --------------------------------------------------------- */
/* Record the launches of any sequence of library calls made on `stream`
 * between pssgp_graph_begin and pssgp_graph_end (thread-local stream
 * capture) into a graph, and replay the whole sequence with one
 * pssgp_graph_launch.  The graph keeps the pointers and sizes of the
 * recorded calls: device data they point to (inputs, per-series parameters)
 * may change between launches, shapes may not.  `stream` must not be the
 * legacy default stream (PSSGP_EINVAL).  While recording, calls only enqueue
 * work: do not call pssgp_get_status, pssgp_timing(2) or the autotuner.
 * pssgp_graph_end returns PSSGP_ECUDA if the capture was invalidated. */
typedef struct pssgp_graph_s pssgp_graph;
int pssgp_graph_begin(void* stream);
int pssgp_graph_end(void* stream, pssgp_graph** out);
int pssgp_graph_launch(pssgp_graph* graph, void* stream);
int pssgp_graph_destroy(pssgp_graph* graph);

/* sizeof(pssgp_model) as compiled into the library, for bindings that mirror
 * the struct (ABI check). */
size_t pssgp_model_bytes(void);

/* Measured FP64 fused-multiply-add rate of this device (lane FMAs per
 * second): the fastest of three timed launches (after a warm-up) of a kernel
 * with eight independent FMA chains per thread at each of 4, 8 and 16 warps
 * per SM, about 10 ms each.  The denominator of the FP64 roofline (the nominal
 * rate is SMs x 128 lanes / 64 cycles per warp instruction x the SM clock).
 * Synchronous on the legacy default stream; allocates a small probe buffer of
 * its own. */
int pssgp_fp64_fma_rate(double* fma_per_s);

#ifdef __cplusplus
}
#endif
#endif /* PSSGP_H */
