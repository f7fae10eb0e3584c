/*
 * ptflash.h -- C ABI of the GB300 batched isothermal two-phase flash.
 *
 * Method: arXiv 2205.03090 ("PTFlash: a deep learning framework for
 * isothermal two-phase equilibrium calculations").  SRK equation of state
 * (Appendix A), Michelsen stability analysis with Wilson-initialised
 * vapour-like and liquid-like trials (Sec. 2.2.1, Alg. 2), phase split by
 * successive substitution on K with a Rachford-Rice solve (Sec. 2.2.2,
 * Appendix C) and a trust-region Newton step on the Gibbs energy
 * (Appendix B), run in the order of the flowchart of Sec. 2.2.3; the
 * learned form adds the classifier / initializer networks of Sec. 4.
 *
 * Conventions shared by every call
 *  - Arrays are structure-of-arrays with the mixture index fastest: the
 *    composition of mixture m is z[i * n + m], i = 0 .. nc-1 (component-major).
 *  - Pressures P and critical pressures Pc must use the same unit (the gas
 *    constant cancels from the reduced EOS parameters); temperatures in K.
 *  - Device entry points take DEVICE pointers owned by the caller and a CUDA
 *    stream (cudaStream_t passed as void*, NULL = legacy default stream).
 *    They enqueue work and return without synchronising; results are valid
 *    once the stream has completed.  The context owns all scratch memory,
 *    so calls that share one context must be ordered on one stream.  A flash
 *    without stage events (ptflash_set_profiling) forks onto two streams the
 *    context owns (high and low priority) after the work already on `stream`
 *    and joins them back into `stream`: ordering on `stream` is unchanged,
 *    and the fork/join can be captured in a CUDA graph.
 *  - Precision: every decision and every returned number is computed in
 *    FP64.  FP32 runs the same iterations ahead of some FP64 ones (Rachford-
 *    Rice and cubic seeds, the first precheck evaluations, the early SS
 *    iterations); it only moves the point where the FP64 iteration starts.
 *  - Return value: 0 on success, a negative PTF_ERR_* code otherwise (no
 *    call aborts the process).  ptflash_strerror() names a code.
 *  - Per-mixture results carry a status bit set (PTF_ST_*).
 *  - Single-phase output: nphase = 1, beta = 0, x = y = z, K = 1.
 *    Two-phase output: nphase = 2, beta = vapour mole fraction theta_V in
 *    (0,1), K_i = y_i / x_i, and y is always the lower-density phase
 *    (larger compressibility factor).
 */
#ifndef PTFLASH_H
#define PTFLASH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define PTF_OK 0
#define PTF_ERR_INVALID_ARG (-1)   /* null pointer, bad size, bad component data */
#define PTF_ERR_CUDA (-2)          /* a CUDA call failed (see ptflash_last_cuda_error) */
#define PTF_ERR_NOT_READY (-3)     /* components (or network weights) not set */
#define PTF_ERR_NO_MEMORY (-4)     /* device allocation failed */
#define PTF_ERR_UNSUPPORTED (-5)   /* nc outside [2, 16] or beyond the context's nc_max */

/* per-mixture status bits */
#define PTF_ST_PRECHECK_UNSTABLE 1 /* the 3-iteration precheck proved instability (Sec. 2.2.3) */
#define PTF_ST_STAB_RUN 2          /* stability analysis ran */
#define PTF_ST_STAB_TR 4           /* a stability trial needed the trust region */
#define PTF_ST_SPLIT_TR 8          /* the split needed the trust region */
#define PTF_ST_MAXITER 16          /* an iteration cap was hit; result not converged */
#define PTF_ST_COLLAPSE 32         /* split collapsed (trivial K / negative flash): single phase */
#define PTF_ST_NONFINITE 64        /* non-finite input or state: single phase, values unusable */
#define PTF_ST_NN_STABLE 128       /* learned form: classifier said stable (p >= p_r) */
#define PTF_ST_NN_UNSTABLE 256     /* learned form: classifier said unstable (p <= p_l) */
#define PTF_ST_NN_INIT 512         /* learned form: K initialised by the initializer network */
#define PTF_ST_NN_REJECTED 1024    /* learned form: the plain method rejected the network route and redid the flash */

typedef struct ptflash_ctx ptflash_ctx;

/*
 * Options of one flash call (NULL = defaults; ptflash_default_options fills
 * the struct).  A zero cap or tolerance selects its default.  Caps must lie
 * in [1, 200] and tolerances be positive and finite, else the call returns
 * PTF_ERR_INVALID_ARG.  A run that reaches a cap without converging gets the
 * PTF_ST_MAXITER status bit (its outputs are the point where it stopped).
 */
typedef struct {
    int32_t use_nn;       /* 0 plain method (default); 1 classifier + initializer (Sec. 4.3) */
    double p_l, p_r;      /* classifier thresholds (defaults 0.02, 0.98; Sec. 5.2) */
    int32_t max_ss_stab;  /* SS evaluations per stability trial (default 9: K_ss of Alg. 2) */
    int32_t max_tr_stab;  /* trust-region iterations per stability trial (default 20: K_tr of Alg. 2) */
    int32_t max_ss_split; /* SS evaluations of the phase split (default 9: Sec. 2.2.2) */
    int32_t max_tr_split; /* split trust-region iterations (default 60; the paper gives none) */
    int32_t max_polish;   /* Newton steps after a split trust-region run (default 10) */
    double tol_stab;      /* stability stop: max |d tm / d W_i| (default 1e-6: Sec. 2.2.1, Appendix B.1) */
    double tol_split_tr;  /* split trust region hands on to the Newton polish below this fugacity
                             residual (default 1e-8: Appendix B.2) */
    double tol_fug;       /* split convergence: max_i |ln y_i + ln phi_i^V - ln x_i - ln phi_i^L|
                             (default 0.98e-10: 2 % below the 1e-10 target, so that the target
                             holds when another FP64 implementation re-evaluates the point) */
    double nn_lnk_dev;    /* learned form: a split started from the initializer's K is kept only if every
                             converged ln K_i lies within this distance of the network's (default 0.3);
                             otherwise the plain method redoes the mixture */
    int32_t tr_lanes;     /* lanes per trust-region run: 0 (default) one lane per run while a trust-region
                             queue lasts, then, once a warp's queue has drained, several lanes per run
                             (one per component) for the runs it has left; 1 one lane throughout; 2 several
                             lanes throughout.  The results are the same bit for bit in every mode (an
                             implementation choice, no counterpart in the paper); other values are
                             PTF_ERR_INVALID_ARG */
    int32_t reserved;
} ptflash_options;

/* Fill *opt with the defaults (plain method).  PTF_ERR_INVALID_ARG if NULL. */
int ptflash_default_options(ptflash_options* opt);

/*
 * Create a context on the current CUDA device with device scratch for up to
 * n_max mixtures of up to nc_max components per launch (larger batches are
 * processed in chunks of n_max).  Allocates device memory (cudaMalloc).
 * *out receives the context; release it with ptflash_destroy.
 */
int ptflash_create(ptflash_ctx** out, int nc_max, int64_t n_max);

/* Free the context and its device memory (synchronises the device). */
int ptflash_destroy(ptflash_ctx* ctx);

/*
 * Set the component system (Appendix A, Eq. mixing_rule and Table 1 data
 * layout): HOST arrays Tc[nc] (K), Pc[nc] (pressure unit of P), omega[nc]
 * (acentric factor), kij[nc*nc] (row-major binary interaction parameters,
 * symmetric with zero diagonal).  2 <= nc <= nc_max <= 16.  Copies the data.
 * PTF_ERR_INVALID_ARG for non-positive Tc/Pc, non-finite values, or an
 * asymmetric / nonzero-diagonal kij.
 */
int ptflash_set_components(ptflash_ctx* ctx, int nc, const double* Tc, const double* Pc, const double* omega,
                           const double* kij);

/*
 * Isothermal two-phase flash of n mixtures (Sec. 2.2.3; the learned form of
 * Sec. 4.3 when opt->use_nn = 1).
 * Learned form: the classifier's probability p of stability routes each
 * mixture.  p >= p_r: single phase (NN_STABLE) unless tpd is negative at one
 * of the trial phases z K, z / K of the initializer's K and of Wilson K, which
 * proves instability and sends the mixture down the plain route.  p <= p_l
 * (initializer K bracketing 1, NN_UNSTABLE): the plain precheck runs; if it
 * proves instability the split starts from the initializer's K, else the
 * mixture continues down the plain route.  A split from the initializer's K
 * is kept only if it converges (within the paper's 20 trust-region
 * iterations) to two phases with Delta G < 0 and its ln K within
 * opt->nn_lnk_dev of the network's; otherwise the plain method redoes the
 * mixture (NN_REJECTED).  Every other mixture takes the plain route:
 * precheck, stability analysis from Wilson K, split.
 * DEVICE arrays: P[n], T[n], z[nc*n]
 * inputs; nphase[n], beta[n], x[nc*n], y[nc*n], K[nc*n], status[n] outputs;
 * iters[n] optional (NULL to skip): packed iteration counts
 * split SS | split TR << 8 | stability SS << 16 | stability TR << 24
 * (each field saturates at 255; the stability fields sum both trials).
 * n == 0 is a no-op.  Outputs must not alias inputs.
 */
int ptflash_flash(ptflash_ctx* ctx, int64_t n, const double* P, const double* T, const double* z, int32_t* nphase,
                  double* beta, double* x, double* y, double* K, int32_t* status, int32_t* iters,
                  const ptflash_options* opt, void* stream);

/*
 * Same as ptflash_flash but every array is a HOST array (pinned memory gives
 * the best copy rate).  Copies inputs to context-owned device buffers, runs
 * the flash and copies the results back on `stream`, then synchronises the
 * stream before returning.  The first host call allocates the context's
 * staging buffers (n_max mixtures).
 */
int ptflash_flash_host(ptflash_ctx* ctx, int64_t n, const double* P, const double* T, const double* z,
                       int32_t* nphase, double* beta, double* x, double* y, double* K, int32_t* status,
                       int32_t* iters, const ptflash_options* opt, void* stream);

/*
 * Stability analysis alone (Sec. 2.2.1, Alg. 2: two Wilson trials, SS then
 * trust region, stop at a stationary point or a negative tm).  DEVICE arrays:
 * inputs P[n], T[n], z[nc*n]; outputs stable[n] (1 stable, 0 unstable:
 * min tm < -1e-10), tm_min[n] (modified tangent-plane distance
 * tm = 1 + sum W_i (ln W_i + ln phi_i(W) - ln z_i - ln phi_i(z) - 1) of the
 * trial with the lower tm, at the point where it stopped), K[nc*n] (the K
 * re-estimate z/W^L or W^V/z of Sec. 2.2.1), status[n].
 */
int ptflash_stability(ptflash_ctx* ctx, int64_t n, const double* P, const double* T, const double* z,
                      int32_t* stable, double* tm_min, double* K, int32_t* status, void* stream);

/*
 * Queue sizes of the most recent ptflash_flash / ptflash_stability call on
 * this context (synchronises the device): counts[0] mixtures sent to
 * stability analysis, [1] mixtures sent to phase split, [2] stability trials
 * that needed the trust region, [3] splits that needed the trust region,
 * summed over chunks.  counts must hold 4 entries.
 */
int ptflash_last_counts(ptflash_ctx* ctx, int64_t* counts);

/*
 * Per-stage timing (the GPU counterpart of the paper's per-subroutine
 * profiler, Table 4).  When enabled, each flash / stability call records a
 * CUDA event before every stage kernel and waits for each chunk to finish
 * (so profiled calls synchronise).  ptflash_last_stage_ms fills ms[0 .. count)
 * with the milliseconds of the last call's stages, summed over chunks:
 * [0] prep + precheck, [1] stability SS, [2] stability trust region,
 * [3] stability decision, [4] split SS, [5] split trust region.
 */
int ptflash_set_profiling(ptflash_ctx* ctx, int enable);
int ptflash_last_stage_ms(ptflash_ctx* ctx, double* ms, int count);

/*
 * ptflash_flash without any device allocation.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory once
 * running -- a simulator time-step loop that budgeted all GPU memory at
 * start-up, a host application whose own allocator owns the device heap, or
 * code that cannot afford the device-wide synchronisation cudaMalloc /
 * cudaFree may imply.  It takes the component data as HOST arrays (as
 * ptflash_set_components) and every batch array as a DEVICE array (as
 * ptflash_flash); no context is needed.  Its scratch is one file-scope
 * device array of 64 MiB that every GPU which loads this library holds until
 * the process exits; it calls no cudaMalloc, cudaFree or allocating library
 * routine.  n may not exceed ptflash_noalloc_max_mixtures(nc) (e.g. 118,000
 * mixtures at nc = 8): larger n returns PTF_ERR_INVALID_ARG.
 * The first call on a device (with that device current) looks up the
 * scratch's device address; make that first call before any stream capture.
 * Every call shares the one scratch array, which keeps the previous call's
 * contents (the call clears what must start at zero): calls that overlap on
 * the GPU -- from different streams or threads -- race and must not be made.
 */
int64_t ptflash_noalloc_max_mixtures(int nc);
int ptflash_flash_noalloc(int nc, const double* Tc, const double* Pc, const double* omega, const double* kij,
                          int64_t n, const double* P, const double* T, const double* z, int32_t* nphase,
                          double* beta, double* x, double* y, double* K, int32_t* status, int32_t* iters,
                          void* stream);

/*
 * Reverse-mode sensitivities of the flash result (beta, x, y) with respect to
 * (P, T, z): the implicit-function-theorem step the paper applies to the
 * Rachford-Rice root (Sec. 4.2.2) applied to the equilibrium of Eq. eq_cond
 * at the converged split.  The feed is read as mole numbers (the flash
 * depends on z / sum z).  For the functional l = gbeta.beta + gx.x + gy.y
 * summed per mixture, writes dl/dP to gP[n], dl/dT to gT[n] and dl/dz to
 * gz[nc * n] (component-major).  Two-phase mixtures: one solve with the Hessian
 * of G in n^V (Eq. split_hess) at the given x, y; single-phase mixtures
 * (x = y = z / sum z, beta = 0): gz_j = (g_j - sum_i g_i z_i / S) / S with
 * g = gx + gy, S = sum z, and gP = gT = 0.
 * Inputs: DEVICE P, T, z and the results nphase, beta, x, y of ptflash_flash
 * on them (converged results; the sensitivities of a MAXITER result are
 * those of the point it stopped at).  gbeta[n], gx[nc * n], gy[nc * n] may
 * each be NULL (zero).  astatus[n] (optional): 0 two-phase, 1 single phase,
 * 2 split Hessian not positive definite (that mixture's outputs are NaN).
 * Same context, stream and ownership rules as ptflash_flash.
 */
int ptflash_flash_adjoint(ptflash_ctx* c, int64_t n, const double* P, const double* T, const double* z,
                          const int32_t* nphase, const double* beta, const double* x, const double* y,
                          const double* gbeta, const double* gx, const double* gy, double* gP, double* gT,
                          double* gz, int32_t* astatus, void* stream);

/*
 * Uneven batches: many fluid systems, each with its own number of components
 * (2..16), component data and mixtures, flashed by one CUDA graph launch.  The
 * paper flashes batches of one fluid system (Sec. 3); a batch of systems is
 * the same plain method (Sec. 2.2.3) per mixture, with each mixture's own
 * component data.  Results equal ptflash_flash's for each system.
 *
 * ptflash_batch_create: HOST arrays.  nsys systems; system s has nc[s]
 *   components and n[s] >= 0 mixtures.  Tc, Pc, omega are packed by system
 *   (system s's components start at sum_{r<s} nc[r]); kij is packed by system
 *   (system s's nc[s] x nc[s] row-major, symmetric, zero-diagonal block starts
 *   at sum_{r<s} nc[r]^2).  Validates the data like ptflash_set_components,
 *   allocates every device buffer of the batch (component tables; per nc a
 *   workspace, staging of (4 nc + 3) doubles + 10 ints per mixture, a stream)
 *   and synchronises.  Returns PTF_ERR_UNSUPPORTED for nc outside [2, 16],
 *   PTF_ERR_NO_MEMORY if an allocation fails.
 * ptflash_batch_flash: DEVICE arrays packed like the systems: P, T, nphase,
 *   beta, status, iters (optional, may be NULL) hold N = sum n[s] entries,
 *   system s's mixtures from off[s] = sum_{r<s} n[r]; z, x, y, K hold system s's
 *   component-major [nc[s]][n[s]] block from zoff[s] = sum_{r<s} nc[r] n[r].
 *   One graph launch on `stream`: the systems are grouped by nc, and each
 *   group (its own stream branch of the graph) gathers its mixtures into a
 *   contiguous slice, runs the flash pipeline with per-mixture component
 *   tables and scatters the results.  The graph is captured on the first call
 *   and again whenever a pointer argument differs from the previous call's;
 *   calls on one batch must be ordered on one stream.
 * ptflash_batch_tune: times each nc group alone (synchronously, twice per
 *   candidate) with its persistent kernels at the device-filling default or
 *   at 1, 2, 3 or 4 resident 128-thread blocks per SM, keeps the fastest and
 *   drops the captured graph.  HOST blocks_per_sm[17] (optional) gets the
 *   choice per nc (0 = default, also for absent nc), HOST group_ms[17]
 *   (optional) its time.  Same array arguments as ptflash_batch_flash, whose
 *   outputs it overwrites.
 * ptflash_batch_info: number of nc groups, nodes of the captured graph (0
 *   before the first flash), total mixtures; any pointer may be NULL.
 */
typedef struct ptflash_batch ptflash_batch;
int ptflash_batch_create(ptflash_batch** out, int nsys, const int32_t* nc, const int64_t* n, const double* Tc,
                         const double* Pc, const double* omega, const double* kij);
int ptflash_batch_destroy(ptflash_batch* b);
int ptflash_batch_flash(ptflash_batch* b, const double* P, const double* T, const double* z, int32_t* nphase,
                        double* beta, double* x, double* y, double* K, int32_t* status, int32_t* iters,
                        void* stream);
int ptflash_batch_tune(ptflash_batch* b, const double* P, const double* T, const double* z, int32_t* nphase,
                       double* beta, double* x, double* y, double* K, int32_t* status, int32_t* iters,
                       int32_t* blocks_per_sm, float* group_ms);
int ptflash_batch_info(const ptflash_batch* b, int32_t* ngroups, int64_t* graph_nodes, int64_t* mixtures);

/*
 * Learned form (Sec. 4 of the paper).  which = 0: stability classifier (one
 * logit; p = sigmoid(logit) is the probability that the mixture is stable);
 * which = 1: ln K initializer (nc outputs).  Inputs are the nc + 2 features
 * (z_1..z_nc, P, T), standardised as (v - mean) / std (the paper's scaling
 * layer) and rounded to bfloat16; weights and hidden activations are
 * bfloat16, sums FP32, SiLU hidden units.  Two architectures:
 *   arch 0: 3 hidden layers of `hidden` units (32, 64 or 128; the paper's
 *     classifier is 3 x 32, Sec. 4.1.1);
 *   arch 1: the paper's initializer (Sec. 4.2.1): a hidden layer, 3 residual
 *     blocks of 2 hidden layers (h <- h + block(h)), all `hidden` units (32
 *     or 64), and a linear output on the concatenation [inputs; h].
 * Parameters: one FP32 vector W_0, b_0, W_1, b_1, ... with each W row-major
 * [out][in] (count: ptflash_nn_param_count_arch(arch, nc + 2, hidden, dout)).
 *
 * ptflash_nn_set_arch: HOST theta, mean[nc+2], std[nc+2]; copies them, makes
 *   the bfloat16 compute copy and resets the Adam state.  Components must be
 *   set.  ptflash_nn_set is arch 0.
 * ptflash_nn_set_theta_loss (initializer only): weight w >= 0 of the second
 *   training stage's |theta - theta_hat| term (Sec. 4.2.2; 0 turns it off).
 *   theta_hat is the Rachford-Rice root for the predicted K, solved in FP64,
 *   and its gradient comes from the implicit-function theorem.  With w > 0
 *   the initializer's targets Y carry 2 nc + 1 rows: ln K, theta, raw z.
 * ptflash_nn_get: copies the FP32 parameters to HOST theta (synchronises).
 * ptflash_nn_features: DEVICE X[(nc+2) * n] (row stride n), the standardised
 *   bfloat16 features of DEVICE P, T, z.
 * ptflash_nn_infer: DEVICE out[dout * n] network outputs for DEVICE P, T, z.
 * ptflash_nn_train_steps: `steps` Adam steps (Kingma & Ba; beta1, beta2, eps)
 *   of `batch` samples each (a multiple of 128).  DEVICE X[(nc+2) * n]
 *   features, Y targets (classifier: [n], 1 stable / 0 unstable, binary
 *   cross-entropy on the logit; initializer: [nc * n] ln K, absolute error
 *   summed over components, plus the theta term when set; all averaged over
 *   the batch), perm[steps * batch] sample indices, HOST lr[steps] learning
 *   rates, optional DEVICE loss[steps] (each entry incremented by that step's
 *   batch loss; zero it first).  The first call allocates training scratch.
 * ptflash_nn_eval: mean loss over DEVICE X[(nc+2) * n], Y (same layouts), and
 *   in *accuracy the classifier's accuracy at p = 1/2, or for the
 *   initializer with the theta term the mean |theta - theta_hat| (else 0);
 *   synchronises.
 */
int64_t ptflash_nn_param_count_arch(int arch, int din, int hidden, int dout);
int ptflash_nn_set_arch(ptflash_ctx* ctx, int which, int arch, int hidden, const float* theta, const float* mean,
                        const float* std);
int ptflash_nn_set_theta_loss(ptflash_ctx* ctx, int which, float weight);
int64_t ptflash_nn_param_count(int din, int hidden, int dout);
int ptflash_nn_set(ptflash_ctx* ctx, int which, int hidden, const float* theta, const float* mean, const float* std);
int ptflash_nn_get(ptflash_ctx* ctx, int which, float* theta);
int ptflash_nn_features(ptflash_ctx* ctx, int which, int64_t n, const double* P, const double* T, const double* z,
                        float* X, void* stream);
int ptflash_nn_infer(ptflash_ctx* ctx, int which, int64_t n, const double* P, const double* T, const double* z,
                     float* out, void* stream);
int ptflash_nn_train_steps(ptflash_ctx* ctx, int which, int64_t n, const float* X, const float* Y,
                           const int32_t* perm, int64_t steps, int batch, const float* lr, float beta1, float beta2,
                           float eps, float* loss, void* stream);
int ptflash_nn_eval(ptflash_ctx* ctx, int which, int64_t n, const float* X, const float* Y, double* loss,
                    double* accuracy, void* stream);

/*
 * Self-check of the library's own table-driven logarithm and exponential
 * (used on every hot path) against the CUDA math library, on the current
 * device.  log: 2n inputs (log-uniform over [1e-300, 1e300] and uniform over
 * [0.5, 2]); exp: 2n inputs (uniform over [-700, 700] and over [-40, 10]).
 * *max_ulp_log and *max_ulp_exp receive the largest errors in units of the
 * last place of the library's result.  Allocates a few bytes of device
 * memory and synchronises the device.
 */
int ptflash_check_math(int64_t n, double* max_ulp_log, double* max_ulp_exp);

/*
 * Phase EOS at given compositions, the primitive every stage evaluates
 * (Appendix A: Eqs. a_i, b_i and mixing_rule for A and B, the cubic of Eq.
 * cubic_Z, the admissible root Z > B with the lower residual Gibbs energy
 * gbar(Z) = Z - 1 - ln(Z - B) - (A/B) ln(1 + B/Z), and ln phi_i of Eq. lnphi).
 * DEVICE arrays: P[n], T[n], composition c[nc * n] (component-major, mole
 * fractions; not renormalised); outputs Z[n] and lnphi[nc * n].  Same
 * context, stream and ownership rules as ptflash_flash.  Non-positive or
 * non-finite inputs give non-finite outputs.
 */
int ptflash_phase_eos(ptflash_ctx* ctx, int64_t n, const double* P, const double* T, const double* c, double* Z,
                      double* lnphi, void* stream);

/*
 * FP64 throughput probe of the current device (the peak against which the
 * flash kernels' FP64 rate is read): one launch of 4 blocks of 256 threads per
 * SM, each thread running 8 independent chains of `iters` x 4 fused
 * multiply-adds, timed with CUDA events after a warm-up launch.  *tflops gets
 * the rate (2 flops per FMA), *ms the launch time.  Synchronises the device.
 * PTF_ERR_INVALID_ARG for iters outside [1, 2^32] or NULL outputs.  The paper
 * has no counterpart: this measures the hardware the flash runs on.
 */
int ptflash_fp64_fma_rate(int64_t iters, double* tflops, double* ms);

/* Human-readable name of an error code. */
const char* ptflash_strerror(int code);

/* The last CUDA error string seen by this library (thread-local), or "". */
const char* ptflash_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PTFLASH_H */
