/*
 * svgp.h -- C-ABI of the GB300 inverse-free SVGP (R-SVGP) training-step library.
 *
 * The library evaluates, on one GPU, the preconditioned inverse-free SVGP
 * bound of Cortinovis et al. (arXiv 2604.00697), Eq. (7), its gradients with
 * the auxiliary matrix T held fixed, and the matmul-only natural-gradient
 * (NG) update of T = L L^T of Prop. 1 / Eq. (6).  The problem statement it
 * follows is Section 2 (Eq. (1): SVGP ELBO over a minibatch X, y with
 * inducing inputs Z, SE-ARD hyperparameters, likelihood parameters) and
 * Section 3 (preconditioned mean m~, diagonal S~ = diag(s~), T = L L^T).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Every tensor argument is a DEVICE pointer to float32 (or float64 / int32
 *    where stated) owned by the caller; the library never frees it.  Row-major
 *    layouts: Z is M x D, X is B x D, L is M x M (ld = M), lower-triangular;
 *    entries above the diagonal must be zero.
 *  * Scalars that change during training (sf2, noise, gamma, Adam's
 *    hyperparameters) are also device pointers, so a sequence of calls can be
 *    captured once in a CUDA graph and replayed.
 *  * Values are CONSTRAINED values (lengthscales, variances, s~ > 0);
 *    gradients are dF/d(constrained value) of the bound F to be MAXIMISED.
 *  * All calls are asynchronous on the handle's stream.  The returned status
 *    covers argument validation and launch errors only.  Errors found on the
 *    device (non-finite bound, a bounded wait that timed out) are recorded in
 *    a device error word, read and cleared by svgp_sync_status().
 *  * The handle owns its workspace (allocated once in svgp_create for M and
 *    B_max) and is not thread-safe; use one handle per host thread/stream.
 *  * The handle also owns a second CUDA stream: within a call, products that
 *    depend only on earlier results of the same call (Psi, and the W product
 *    of the gradient) are forked onto it from the handle's stream and joined
 *    back before the call's last launch, so every call is complete in the
 *    handle's stream order and a graph captured on that stream holds both.
 */
#ifndef SVGP_H_
#define SVGP_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct svgp_handle svgp_handle;

typedef enum {
  SVGP_OK = 0,
  SVGP_ERR_INVALID_ARG = 1,   /* bad size, null pointer, unsupported option     */
  SVGP_ERR_CUDA = 2,          /* a CUDA runtime/driver call failed              */
  SVGP_ERR_OOM = 3,           /* workspace allocation failed                    */
  SVGP_ERR_NONFINITE = 4,     /* device: bound or a reduction is NaN/Inf        */
  SVGP_ERR_NOT_CONVERGED = 5, /* reserved: the NG loop reports via iters/resid. */
  SVGP_ERR_TIMEOUT = 6,       /* device: a bounded pipeline wait gave up        */
  SVGP_ERR_UNSUPPORTED = 7    /* option not built for this device / precision   */
} svgp_status;

/* Likelihood of the data term.  SVGP_LIK_GAUSSIAN: p(y | f) = N(y; f, noise),
 * its expectation in closed form (Appendix S3).  SVGP_LIK_BERNOULLI_PROBIT:
 * binary labels y in {0, 1}, p(y | f) = Phi((2y - 1) f) (the classification
 * experiments of Section 4.1), its expectation under N(mu_n, sigma_n^2) by a
 * gh_points-node Gauss-Hermite rule (svgp_gauss_hermite). */
typedef enum { SVGP_LIK_GAUSSIAN = 0, SVGP_LIK_BERNOULLI_PROBIT = 1 } svgp_lik;

/* Arithmetic of the dense contractions.  SVGP_FP32: FP32 SIMT FMA kernels
 * (no TF32).  SVGP_BF16: tcgen05 tensor-core kernels, BF16 operands with FP32
 * accumulation in TMEM (one MMA per product; relative error of the M x M
 * products grows like 2^-9 * cond(K~)).  SVGP_BF16X3: the same tensor-core
 * kernels with every M x M operand held as an unevaluated sum hi + lo of two
 * BF16 matrices and each product formed as hi*hi + hi*lo + lo*hi (three BF16
 * MMAs, FP32 accumulation; error like 2^-17 * cond(K~)).  SVGP_BF16X3K:
 * SVGP_BF16X3 with Kuu held as three BF16 planes (hi + lo + lo2, about 2^-26)
 * where it is the operand of L^T K~ (the preconditioner's A1 = L^T K~ L of
 * Section 3.2 and the NG update's A of Eq. (6)), formed as
 * L_hi (K_hi + K_lo + K_lo2) + L_lo (K_hi + K_lo) (five MMAs).  A1 is close
 * to I near the fixed point and the rounding of Kuu there dominates the
 * gradient error once cond(K~) reaches a few thousand; the other products
 * stay hi/lo.  The handle holds one more M x M BF16 plane.  Scalar
 * reductions are FP64 in every mode. */
typedef enum { SVGP_FP32 = 0, SVGP_BF16 = 1, SVGP_BF16X3 = 2, SVGP_BF16X3K = 3 } svgp_prec;

typedef struct {
  int M;              /* number of inducing points, 1 <= M <= 8192              */
  int D;              /* input dimension, 1 <= D <= 32                          */
  int B_max;          /* largest minibatch / prediction block, >= 1             */
  int lik;            /* svgp_lik                                               */
  int prec;           /* svgp_prec                                              */
  void* cuda_stream;  /* cudaStream_t to run on; NULL = legacy default stream   */
  int gh_points;      /* probit: nodes of the Gauss-Hermite rule, 1..32; 0 = 20 */
  int unpreconditioned; /* 0: the preconditioned bound of Eq. (7), m = Kuu P m~
                           (Section 3.2); 1: R-SVGP without the preconditioner,
                           m = Kuu m~ (Section 2): mu_n = k_nu m~ and the KL
                           term m~^T Kuu m~, everything else unchanged       */
} svgp_config;

/* Model state.  ell: D lengthscales; sf2: signal variance (1 float); noise:
 * Gaussian observation variance (1 float; read only by the Gaussian
 * likelihood, may be NULL for probit); m: preconditioned variational
 * mean m~ (M); s: diagonal of S~ (M, all > 0); L: factor of T (M x M). */
typedef struct {
  const float* Z;
  const float* ell;
  const float* sf2;
  const float* noise;
  const float* m;
  const float* s;
  const float* L;
} svgp_params;

/* Minibatch: X (B x D), y (B; labels 0 or 1 for probit: y > 0.5 is class 1).
 * N is the dataset size; the data term is scaled by N / B (stochastic SVGP).
 * 1 <= B <= B_max. */
typedef struct {
  const float* X;
  const float* y;
  int B;
  double N;
} svgp_batch;

/* Gradient outputs (device, float32, same shapes as svgp_params fields). */
typedef struct {
  float* dZ;
  float* dell;
  float* dsf2;
  float* dnoise;
  float* dm;
  float* ds;
} svgp_grads;

/* Layout of the float64 term vector written by svgp_bound / svgp_backward. */
enum {
  SVGP_T_F = 0,        /* the bound F = E - KL                                 */
  SVGP_T_E = 1,        /* (N/B) * sum_n E_q[log p(y_n | f_n)]                  */
  SVGP_T_KL = 2,       /* KL upper bound of Eq. (7)                            */
  SVGP_T_TRKT = 3,     /* tr(K~ T) = tr(L^T K~ L)                              */
  SVGP_T_TRPKUU = 4,   /* tr(P Kuu)                                            */
  SVGP_T_QUAD = 5,     /* m~^T P Kuu P m~                                      */
  SVGP_T_LOGDETT = 6,  /* log|T| = 2 sum_i log|L_ii|                           */
  SVGP_T_SQERR = 7,    /* sum_n (y_n - mu_n)^2 (Gaussian; 0 for probit)        */
  SVGP_T_SUMVAR = 8,   /* sum_n sigma_n^2 (probit: after clamping at 0)        */
  SVGP_T_LOGDETS = 9,  /* sum_i log s~_i                                       */
  SVGP_T_NCLAMP = 10,  /* probit: points whose sigma_n^2 rounded below 0 and
                          was clamped to 0 (0 for Gaussian)                    */
  SVGP_NTERMS = 11
};

/* Create a handle and its workspace.  On success *out owns device memory of
 * about 10 M^2 floats + O(B_max M / 64) and a second CUDA stream with two
 * events; destroy with svgp_destroy.  SVGP_ERR_CUDA if the stream or events
 * cannot be created. */
svgp_status svgp_create(const svgp_config* cfg, svgp_handle** out);
void svgp_destroy(svgp_handle* h);

/* Change the stream later calls are issued on (e.g. a graph-capture stream). */
svgp_status svgp_set_stream(svgp_handle* h, void* cuda_stream);

/* Bound, Eq. (7) (preconditioned R-SVGP), with the handle's likelihood.
 *   mu_n = k_nu P m~, sigma_n^2 = k_nn - k_nu P k_un, P = 2T - T K~ T,
 *   KL <= 1/2(-tr(P Kuu) + tr(K~T) - M + m~^T P Kuu P m~ - log|T| - log|S~|),
 *   F = (N/B) sum_n E_n - KL.
 * Gaussian: E_n in closed form, sum_n sigma_n^2 = B sf2 - <P, Kuf Kuf^T>.
 * Probit: sigma_n^2 per point (clamped at 0), s_n = 2 y_n - 1 and
 *   E_n = sum_k w_k / sqrt(pi) log Phi(s_n (mu_n + sqrt(2) sigma_n t_k))
 * over the nodes t_k and weights w_k of the rule for exp(-t^2).
 * terms_dev: device float64[SVGP_NTERMS] (layout above). */
svgp_status svgp_bound(svgp_handle* h, const svgp_params* p, const svgp_batch* b,
                       double* terms_dev);

/* svgp_bound with the two cubic traces of the KL bound replaced by
 * Hutchinson estimates over K probe vectors (Section 3.4):
 *   tr(K~ T)  ~ (1/K) sum_k z_k^T L^T K~ L z_k,
 *   tr(P Kuu) ~ (1/K) sum_k z_k^T P Kuu z_k;
 * every other term exact.  probes: device float[M x K] row-major (column k
 * is z_k; entries +-1 for Rademacher probes -- the caller draws them, so the
 * estimate is reproducible), 1 <= K <= SVGP_HUTCH_KMAX.  Nothing of order
 * M^3 is computed and P is never formed: the estimates take products of the
 * M x M matrices with the M x K probe block (about 14 M^2 K flops), the data
 * term takes k_n^T P k_n = 2 |L^T k_n|^2 - (T k_n)^T K~ (T k_n) per point from
 * products of L and K~ with the columns of Kuf (about 6 M^2 B flops), and
 * v = P m~ comes from FP32 matrix-vector products -- O((B + K) M^2) in all,
 * less than svgp_bound's O(M^3) chain once B + K is well below M.  The
 * products run on the tensor cores in the handle's operand precision (BF16
 * or hi/lo BF16 handles; FP32 SIMT for SVGP_FP32 handles, and when K exceeds
 * M rounded up to 128).  The first call, and a call whose B or K changes the
 * number of 128-column blocks, synchronises the handle's streams to rebuild
 * the products' schedules: make it outside stream capture.  The terms layout
 * is that of svgp_bound (SVGP_T_TRKT and SVGP_T_TRPKUU hold the estimates). */
#define SVGP_HUTCH_KMAX 256
svgp_status svgp_bound_hutchinson(svgp_handle* h, const svgp_params* p, const svgp_batch* b,
                                  const float* probes, int K, double* terms_dev);

/* Bound (as svgp_bound) plus its gradient w.r.t. Z, ell, sf2, noise, m~, s~
 * with T held fixed (Section 3.1: T is optimised separately by NG; Prop. 2
 * concerns exactly this gradient).  terms_dev may be NULL.  Probit: the
 * per-point derivatives g_n = dE_n/dmu_n and h_n = dE_n/dsigma_n^2 are those
 * of the quadrature rule itself (h_n from the rule's derivative in sigma_n;
 * below sigma_n = 1e-6 from 1/2 sum_k w_k / sqrt(pi) d^2/df^2 log Phi, its
 * limit); dnoise is 0 (the bound does not depend on noise). */
svgp_status svgp_backward(svgp_handle* h, const svgp_params* p, const svgp_batch* b,
                          double* terms_dev, const svgp_grads* g);

/* Natural-gradient update of L, Prop. 1 / Eq. (6), with K~ = Kuu(Z, ell, sf2)
 * + diag(s~) taken from p (p->L is ignored; L_inout is read and updated in
 * place).  For t = 0 .. max_iters-1:
 *   A = L^T K~ L;  r_t = ||A - I||_F / sqrt(M)                 (Eq. (8))
 *   if eps > 0 and r_t < eps: stop without updating            (Section 3.3)
 *   L <- L - gamma_dev[t] * L [tril(A) - 1/2 (I + diag A)]     (Prop. 1)
 * gamma_dev: device float[max_iters].  iters_dev (device int, may be NULL)
 * receives the number of updates applied; residual_dev (device double, may be
 * NULL) the last residual computed (that of L before the last update when no
 * early stop happened).  Non-convergence is not an error: it shows as
 * iters == max_iters with residual >= eps.  A residual that is not finite (a
 * diverging step size, or non-finite L, Z or s~) stops the loop before the
 * update and records SVGP_ERR_NONFINITE in the device error word. */
svgp_status svgp_ng_update_T(svgp_handle* h, const svgp_params* p, float* L_inout,
                             const float* gamma_dev, int max_iters, double eps,
                             int* iters_dev, double* residual_dev);

/* Gap of Prop. 3 (Section 3.3, Gaussian likelihood) for the batch b at
 * T = p->L p->L^T: with K~ = K~_- + sigma2 I (K~_- = Kuu + S~', S~' diagonal
 * and PD) the R-SVGP variance U_n and the lower bound L_n of the L-SVGP
 * variance differ by G_n = ||(I - K~ T) k_un||^2 / sigma2; writes
 * G = sum_n G_n to gap_dev (device double).  sigma2 <= 0 selects
 * sigma2 = min_i s~_i.  Computed as <N N^T, Kuf Kuf^T> / sigma2 with
 * N = I - T K~ by FP32 SIMT products (about 5 M^3 flops; Psi = Kuf Kuf^T in
 * the handle's precision). */
svgp_status svgp_variance_gap(svgp_handle* h, const svgp_params* p, const svgp_batch* b, double sigma2,
                              double* gap_dev);

/* svgp_ng_update_T with the gap stopping rule of Section 3.3 instead of the
 * Frobenius residual: for t = 0 .. max_iters-1, G_t = G(L_t) as in
 * svgp_variance_gap; if eps > 0 and G_t <= 2 noise eps: stop without
 * updating; else L <- NG step with gamma_dev[t] (Prop. 1).  iters_dev
 * (device int, may be NULL) receives the number of updates; gap_dev (device
 * double, may be NULL) the gap of the returned L.  Gaussian likelihood only
 * (SVGP_ERR_UNSUPPORTED otherwise). */
svgp_status svgp_ng_update_T_gap(svgp_handle* h, const svgp_params* p, const svgp_batch* b, float* L_inout,
                                 const float* gamma_dev, int max_iters, double eps, double sigma2,
                                 int* iters_dev, double* gap_dev);

/* One training step's device work in a single call: svgp_ng_update_T on
 * L_inout (same arguments and semantics), then svgp_backward with L = the
 * updated L_inout (p->L is ignored).  The scaled coordinates, Kuu and the Kuf
 * generator operands are prepared once for both parts; results equal those of
 * the two separate calls.  Not in the paper as an operation of its own: it is
 * the composition Section 3.3 runs every iteration (NG steps on T, then a
 * gradient step on the other parameters). */
svgp_status svgp_train_step(svgp_handle* h, const svgp_params* p, const svgp_batch* b,
                            float* L_inout, const float* gamma_dev, int max_iters, double eps,
                            int* iters_dev, double* residual_dev, double* terms_dev,
                            const svgp_grads* g);

/* Predictive moments at Ns test inputs Xs (Ns x D), same form as Eq. (7):
 * mean = K*u P m~, var = sf2 - diag(K*u P Ku*) (+ noise if include_noise).
 * 1 <= Ns <= B_max. mean, var: device float[Ns]. */
svgp_status svgp_predict(svgp_handle* h, const svgp_params* p, const float* Xs, int Ns,
                         float* mean, float* var, int include_noise);

/* One Adam ascent step on the flat unconstrained parameter vector
 * raw = [Z (M*D) | ell (D) | sf2 | noise | m~ (M) | s~ (M)].  Positive blocks
 * (ell, sf2, noise, s~) are softplus-transformed; grad is the flat gradient
 * w.r.t. constrained values in the same layout (svgp_grads may point into
 * it).  Writes the updated raw vector and its constrained image (which
 * svgp_params may point into).  hyper_dev: device float[10] =
 * {lr, beta1, beta2, eps, lr multiplier for Z, ell, sf2, noise, m~, s~};
 * beta1 applies to all blocks except Z, which uses hyper_dev[1] unless
 * zbeta1_dev (device float, may be NULL) is given.  step_dev: device int
 * incremented by the call (bias-correction counter).  m1, m2: moment vectors
 * (device, same length, zero-initialised by the caller). */
svgp_status svgp_adam_step(svgp_handle* h, float* raw, float* constrained, const float* grad,
                           float* m1, float* m2, int* step_dev, const float* hyper_dev,
                           const float* zbeta1_dev);

/* Gauss-Hermite rule for the weight exp(-t^2) with n nodes, 1 <= n <= 64:
 * integral of exp(-t^2) f(t) dt ~= sum_k weights[k] f(nodes[k]).  Host
 * function (host arrays of n doubles; no GPU needed), ascending nodes.
 * Computed by Newton's method on the orthonormal Hermite recurrence after
 * bracketing every sign change; weights 1 / (n q_{n-1}(t_k)^2) with q_j the
 * orthonormal polynomials.  Returns SVGP_OK or SVGP_ERR_INVALID_ARG. */
svgp_status svgp_gauss_hermite(int n, double* nodes, double* weights);

/* Number of floats in the flat parameter vector for this handle. */
int svgp_param_count(const svgp_handle* h);

/* Synchronise the handle's stream, read and clear the device error word.
 * Returns SVGP_OK, SVGP_ERR_NONFINITE, SVGP_ERR_TIMEOUT or SVGP_ERR_CUDA. */
svgp_status svgp_sync_status(svgp_handle* h);

/* Check of the failure path of the bounded device waits (not an operation
 * of the paper).  Every pipeline wait of the tensor-core kernels is bounded:
 * when it gives up, the kernel stops issuing work, waits (bounded) for its
 * own copies in flight, frees its TMEM, records SVGP_ERR_TIMEOUT in the
 * device error word and returns.  This call launches, on the handle's stream,
 * a one-block kernel whose bounded wait -- the same helper -- waits on an
 * mbarrier that nothing ever arrives on, with a limit of 2^26 SM cycles
 * (about 32 ms), so the wait runs out and the error word records the
 * timeout; the next svgp_sync_status returns SVGP_ERR_TIMEOUT and clears it.
 * No copy, MMA or memory access other than the error word is involved.
 * SVGP_ERR_UNSUPPORTED without a tensor-core (sm_103a) device. */
svgp_status svgp_check_wait_timeout(svgp_handle* h);

/* Human-readable text of the last host-side error on this handle. */
const char* svgp_last_error(const svgp_handle* h);
const char* svgp_status_string(int status);

/* 1 if the library's tensor-core (tcgen05) kernels can run on the current device. */
int svgp_has_tensor_cores(void);

/* Instrumentation.  Kinds of dense-contraction launches that can be timed. */
enum {
  SVGP_PROF_VT = 0,     /* L^T S        (S = K~ or G_P), full output           */
  SVGP_PROF_SYM = 1,    /* (L^T S) L    symmetric output                       */
  SVGP_PROF_LUPD = 2,   /* L Phi        NG update of L                          */
  SVGP_PROF_LS = 3,     /* L S          full output                             */
  SVGP_PROF_OUT = 4,    /* (L S) L^T    symmetric output (P, G_K~)              */
  SVGP_PROF_PSI = 5,    /* Kuf Kuf^T    Kuf generated on chip                   */
  SVGP_PROF_W = 6,      /* P Kuf        Kuf generated on chip, fused backward   */
  SVGP_PROF_NKINDS = 7
};

/* enable != 0: from now on every launch of the kinds above is bracketed by
 * two CUDA events recorded on the handle's stream (inside a stream capture
 * they become event nodes of the graph).  Clears the list of records.
 * enable == 0 stops recording.  Up to 512 launches are recorded. */
svgp_status svgp_profile_enable(svgp_handle* h, int enable);

/* After the recorded work has completed (synchronise first): total device
 * milliseconds and launch count per kind over the current record list (for a
 * replayed graph: of its latest replay).  ms, counts: host arrays of
 * SVGP_PROF_NKINDS entries. */
svgp_status svgp_profile_read(svgp_handle* h, float* ms, int* counts);

/* Split-K schedule of the persistent tensor-core GEMM (tuning; not an
 * operation of the paper).  The triangular products (kinds SVGP_PROF_SYM,
 * SVGP_PROF_LUPD and SVGP_PROF_OUT) have output tiles whose K ranges differ
 * by up to the whole matrix; a tile of at least kmin 64-deep k-blocks is
 * computed as two K chunks on two CTAs, the first writing FP32 partial sums
 * that the second adds before its epilogue.  svgp_create picks kmin from a
 * cost model; svgp_set_split sets it per kind: kmin > 0 one of the values
 * svgp_split_candidates lists, 0 no split, < 0 the cost model's choice.  The
 * full products (SVGP_PROF_VT, SVGP_PROF_LS) accept only 0.  It synchronises
 * the handle's streams and rewrites the schedule on the device: call it
 * outside stream capture, and capture again every CUDA graph captured on
 * this handle before the call (a graph keeps the grid size of the old
 * schedule; replaying it afterwards gives wrong results).  Results under
 * different thresholds agree up to the order of the FP32 sums.
 * SVGP_ERR_UNSUPPORTED for SVGP_FP32
 * handles.  svgp_get_split returns the kmin in force (-1: not applicable);
 * svgp_split_candidates writes up to n candidates (0 first) to out and
 * returns their count. */
svgp_status svgp_set_split(svgp_handle* h, int kind, int kmin);
int svgp_get_split(const svgp_handle* h, int kind);
int svgp_split_candidates(const svgp_handle* h, int kind, int* out, int n);

/* Number of kernel launches the library has issued in this process (all
 * handles; launches captured into a graph are counted once, at capture). */
long long svgp_launch_count(const svgp_handle* h);

/* Prediction without any device allocation.  (The paper has no counterpart:
 * this entry point exists for callers, not for the method.)
 *
 * Some callers cannot call cudaMalloc: code that runs while a framework
 * captures a CUDA graph, plug-ins and embedded runtimes that own a fixed
 * memory budget, or services that must not touch the allocator on a latency
 * path.  A handle allocates its workspace in svgp_create, so those callers
 * cannot use svgp_predict.  This function computes the same mean and
 * variance as svgp_predict on an SVGP_FP32 handle, with the same FP32
 * kernels, but takes no handle and allocates nothing: its scratch is one
 * array in the library's device memory of about 2.7 MB, which every GPU
 * that loads the library holds until the process exits.
 *
 * Limits: 1 <= M <= 256, 1 <= D <= 32, 1 <= Ns <= 4096; larger sizes return
 * SVGP_ERR_INVALID_ARG.  Arguments are as for svgp_predict (device pointers;
 * p->L is the M x M factor of T); cuda_stream is the stream to run on (NULL:
 * legacy default stream).  The first call on a device performs a one-time
 * set-up on the host (it looks up the array's device address and copies the
 * tile tables into the array), so make that first call before any stream
 * capture.  Every call uses the same array and
 * clears what must start at zero; calls that overlap on the GPU (on different
 * streams, or from different host threads) race and must be serialised by
 * the caller.  Returns SVGP_ERR_CUDA when a launch fails. */
svgp_status svgp_predict_noalloc(const svgp_params* p, int M, int D, const float* Xs, int Ns, float* mean,
                                 float* var, int include_noise, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SVGP_H_ */
