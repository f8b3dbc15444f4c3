/*
 * hmc.h -- C ABI of libhmc: Hamiltonian Monte Carlo for Bayesian multinomial
 * (softmax) regression on one GB300 GPU (sm_103a).
 *
 * Method: Beam, Ghosh & Doyle, "Fast Hamiltonian Monte Carlo Using GPU
 * Computing" (arXiv 1402.4089).  The library keeps X, the labels, the
 * coefficients, momenta and gradients as persistent device state (Sec. 2.1,
 * last paragraph) and evaluates, for every leapfrog step, the log-posterior
 * kernel (Eq. logkernel / logkernelGPU) and its gradient (Eq. gradient /
 * fullgrad) in one fused pass over X.
 *
 * Conventions shared by every call
 *  - Every call returns hmc_status and never aborts the process.  A message
 *    for the last failure of the calling thread is in hmc_last_error().
 *  - Argument errors are detected before any device work: HMC_EINVAL.
 *  - The caller keeps ownership of every pointer it passes; the library
 *    copies what it keeps.  The handle owns all device memory it allocates.
 *  - "host or device" pointers are classified with cudaPointerGetAttributes;
 *    host buffers are copied through the handle's stream and the call
 *    synchronises that stream before it returns.  Calls given only device
 *    buffers are asynchronous on the handle's stream (opts.stream) unless
 *    stated otherwise; results are valid after that stream is synchronised.
 *  - A handle is not thread safe: one thread at a time per handle.
 *  - Coefficient layout ("beta layout"): for `chains` chains of a problem
 *    with p features and K classes, a dense array [chains][R][p] of the
 *    handle's state type (double for HMC_F64, float for HMC_F32), where R is
 *    the number of coefficient rows per chain of opts.layout (hmc_layout):
 *    R = K-1 for HMC_LAYOUT_FREE (row k of chain c is beta_{k+1}; beta_K = 0
 *    is implied by the identifiability constraint of Sec. 2.1 and never
 *    stored), R = K for HMC_LAYOUT_MASKED and HMC_LAYOUT_UNCONSTRAINED.  For a
 *    batch handle the problems' blocks follow one another in problem order.
 *  - Every device-side wait is bounded (opts.spin_limit); when a bound runs
 *    out the kernel stops, the call returns HMC_ETIMEOUT and the handle stays
 *    usable.
 */
#ifndef HMC_H
#define HMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hmc_ctx* hmc_handle;

typedef enum {
  HMC_OK = 0,
  HMC_EINVAL = 1,        /* bad argument (detected before any launch)          */
  HMC_ENOMEM = 2,        /* device or pinned-host allocation failed            */
  HMC_ECUDA = 3,         /* a CUDA runtime call failed; see hmc_last_error()   */
  HMC_ETIMEOUT = 4,      /* a bounded device wait ran out                      */
  HMC_ENONFINITE = 5,    /* non-finite value in X or a label outside [0, K)    */
  HMC_EUNSUPPORTED = 6   /* valid request the library or device cannot run    */
} hmc_status;

/* Prior on each free coefficient.  Sec. 2.1 uses the standard Cauchy
 * (scale 1): log kernel -log(1 + b^2/s^2).  The Gaussian N(0, s^2) has log
 * kernel -b^2/(2 s^2).  No normalising constants (Sec. 1.1). */
typedef enum { HMC_PRIOR_GAUSSIAN = 0, HMC_PRIOR_CAUCHY = 1 } hmc_prior_kind;

/* Coefficient layout and identifiability (Sec. 2.1; Appendix, the mask M
 * after Eq. fullgrad).
 *  HMC_LAYOUT_FREE          K-1 free coefficient rows per chain, beta_K = 0
 *                           implied (the default).
 *  HMC_LAYOUT_MASKED        K rows per chain in the p x K form of Eq. fullgrad;
 *                           row K is held at zero: the gradient and momentum of
 *                           beta_K are masked to zero, as the elementwise mask M
 *                           of the Appendix does, so values, gradients and
 *                           chains equal those of HMC_LAYOUT_FREE with a zero
 *                           row appended.  Row K of any input is ignored (read
 *                           as zero); row K of every output is zero.
 *  HMC_LAYOUT_UNCONSTRAINED K free rows per chain: identifiability is not
 *                           enforced (the prediction-only variant whose timings
 *                           are Figs 3-4); the softmax runs over K free logits
 *                           and the prior covers all p K coefficients. */
typedef enum { HMC_LAYOUT_FREE = 0, HMC_LAYOUT_MASKED = 1, HMC_LAYOUT_UNCONSTRAINED = 2 } hmc_layout;

/* Element types.  X may be stored as HMC_F64, HMC_F32, HMC_BF16 (round to
 * nearest even) or HMC_FP8E4M3 (per-column scale s_j = max_i|x_ij|/448,
 * x_ij/s_j rounded to nearest even, saturating).  The chain state (beta,
 * eta, grad) is HMC_F64 or HMC_F32. */
typedef enum { HMC_F64 = 0, HMC_F32 = 1, HMC_BF16 = 2, HMC_FP8E4M3 = 3 } hmc_dtype;

typedef struct {
  hmc_dtype x_storage;    /* storage type of X on the device (default HMC_F32)   */
  hmc_dtype state;        /* HMC_F64 or HMC_F32 (default HMC_F32)                */
  int32_t max_chains;     /* largest `chains` any later call may pass (default 1) */
  int32_t engine;         /* 0 auto, 1 CUDA-core fused kernel, 2 tensor-core fused kernel (BF16 or
                             FP8 storage; MMA operands BF16, FP32 accumulation), 3 tensor-core
                             two-pass kernels (BF16 or FP8 storage, FP8 codes widened to BF16 in
                             shared memory: logits, softmax and residual of every row tile in a
                             first pass, X^T R in a second; no TMEM limit on the chains of one
                             launch; X crosses HBM twice when larger than L2), 4
                             CUDA-core two-pass kernels (FP32 / FP64 storage: row logits, softmax
                             and residual in a first pass, X^T R in a second; up to 64 coefficient
                             columns per launch, no tile options).  Auto: FP32 / FP64 storage on
                             engine 1, or on engine 4 where no engine-1 tile fits (wide problems with
                             many classes: FP32 X with K - 1 > 12 and p > 10240), K - 1 exceeds
                             its class bound, or a single problem of n p >= 4e6 has chains (K - 1)
                             >= 19 columns (>= 14 at p >= 2048); BF16 and FP8 on engine 3 for a
                             single problem; in a batch, FP8 on engine 2 when the chains' columns
                             fit TMEM, else CUDA cores, and BF16 on engine 2 when every chain fits
                             one fused launch, else engine 3 */
  int64_t spin_limit;     /* iterations of every bounded device wait (0: default)  */
  void* stream;           /* cudaStream_t for all work of the handle (NULL: default stream) */
  int32_t tile[4];        /* {cluster size 1..16, exchange depth, sweep lookahead, ring slots}; 0 =
                             chosen.  Depth (partial-logit slots and R buffers, 1..4) and lookahead
                             (tiles between the two sweeps, 1..4) apply to the tensor-core engine and
                             must be 0 on the CUDA-core engine.  The chosen CUDA-core tile keeps the
                             most SMs streaming X with clusters of at most ceil(p / 256) CTAs, and
                             launches no more than one cluster per S SMs unless each still gets
                             about four 16-row tiles; the chosen tensor-core tile takes the most
                             chains TMEM holds, spread evenly over the launches a call needs.  On
                             the two-pass engine only tile[0] applies: the 128-row tiles of one
                             first-pass unit (1..4; 0 = chosen by the bytes the busiest SM streams) */
  int32_t layout;         /* hmc_layout of every coefficient buffer (default HMC_LAYOUT_FREE); the
                             kernels see K-1 free rows (K for HMC_LAYOUT_UNCONSTRAINED), which must
                             fit their class bounds */
} hmc_opts;

/* Per-chain counters of hmc_sample (host memory, one entry per chain). */
typedef struct {
  int64_t iterations;     /* proposals made                                   */
  int64_t accepted;       /* proposals accepted (Eq. accept)                  */
  int64_t diverged;       /* proposals with non-finite H (rejected)           */
  double sum_abs_dH;      /* sum over proposals of |H1 - H0|                  */
  double logpost;         /* log K of the chain's current state               */
} hmc_chain_stats;

/* Fill *opts with the defaults listed above. */
void hmc_default_opts(hmc_opts* opts);

/* Library version string (static storage). */
const char* hmc_version(void);

/* Message of the last failing call made by this thread ("" if none). */
const char* hmc_last_error(void);

/*
 * hmc_create -- upload one regression problem (Sec. 2.1): X (n x p), labels
 * y (n; y_i in [0, K) stands for the one-hot row of Y), K classes, prior.
 *   X        host or device, row-major n x p of x_dtype (HMC_F64 or HMC_F32);
 *            converted on the device to opts->x_storage and padded.
 *   y        host or device int32[n].
 *   n >= 0 (n = 0: prior only), p >= 1, 2 <= K <= 1024.
 *   prior_scale > 0.
 * Errors: HMC_EINVAL (shapes, dtypes, null pointers, scale), HMC_ENONFINITE
 * (label out of range or non-finite X, checked on the device), HMC_ENOMEM.
 * Synchronous.
 */
hmc_status hmc_create(const void* X, hmc_dtype x_dtype, const int32_t* y, int64_t n, int64_t p,
                      int32_t K, hmc_prior_kind prior, double prior_scale, const hmc_opts* opts,
                      hmc_handle* out);

/*
 * hmc_create_batch -- several independent regression problems in one handle
 * (each with its own n_b, p_b, K_b; same prior and options).  The fused pass
 * runs over all problems in one launch; the beta layout concatenates the
 * problems.  Arguments are arrays of length nprob with the meaning of
 * hmc_create's.  Synchronous.
 */
hmc_status hmc_create_batch(int32_t nprob, const void* const* X, hmc_dtype x_dtype,
                            const int32_t* const* y, const int64_t* n, const int64_t* p,
                            const int32_t* K, hmc_prior_kind prior, double prior_scale,
                            const hmc_opts* opts, hmc_handle* out);

/* Release every resource of the handle (NULL is accepted).  Synchronous. */
hmc_status hmc_destroy(hmc_handle h);

/* Coefficients of one chain in the beta layout (sum over problems of R_b p_b,
 * R_b the rows per chain of opts.layout). */
int64_t hmc_chain_size(hmc_handle h);

/*
 * hmc_logpost_grad -- log K (Eq. logkernel) and its gradient (Eq. gradient,
 * prior term with the sign of the derivative of the prior's log kernel) at
 * `chains` coefficient states.
 *   beta     host or device, beta layout (state type).
 *   logpost  host or device double[nprob * chains] (index b * chains + c
 *            for problem b, chain c), or NULL.
 *   grad     host or device, beta layout, or NULL.
 * 1 <= chains <= opts.max_chains.
 */
hmc_status hmc_logpost_grad(hmc_handle h, const void* beta, int32_t chains, double* logpost,
                            void* grad);

/*
 * hmc_leapfrog -- L leapfrog updates (Eqs. hmc1-hmc3) in place, no accept
 * test.  beta, eta: host or device, beta layout.  grad: in, the gradient at
 * beta, or NULL (then computed first); out, the gradient at the new beta.
 * logpost: out, log K at the new beta (as in hmc_logpost_grad), or NULL.
 * eps is the step size, L >= 0.
 */
hmc_status hmc_leapfrog(hmc_handle h, void* beta, void* eta, void* grad, double* logpost,
                        int32_t chains, int32_t L, double eps);

/*
 * hmc_sample -- `iters` HMC iterations of `chains` independent chains
 * (Sec. 1.1): draw eta ~ N(0, I) (Philox4x64-10, key (seed, 0), counter
 * (block, iteration, chain, 0)), L leapfrog updates, accept iff
 * log u < (H0 - H1) / T with H = -log K + eta.eta / 2 and T = 1 (Eq. accept;
 * u from counter (0, iteration, chain, 1)), else keep the old state.  A
 * non-finite H1 is rejected and counted as divergent.
 *   beta0    host or device beta layout: (re)start every chain there and
 *            reset the iteration counter to 0; NULL: continue from the
 *            handle's chain state (zeros on first use), counter continuing.
 *   samples  host or device [iters/thin][chains][...beta layout...] of the
 *            state type (the state after iterations thin-1, 2 thin-1, ...),
 *            or NULL.
 *   thin >= 1.  stats: host [nprob * chains] (index b * chains + c, filled
 *            on return) or NULL.
 * The chain state is the handle's; it persists across calls.  Synchronous.
 */
hmc_status hmc_sample(hmc_handle h, int32_t chains, int32_t L, double eps, int64_t iters,
                      uint64_t seed, const void* beta0, void* samples, int32_t thin,
                      hmc_chain_stats* stats);

/*
 * hmc_sample_tempered -- hmc_sample with a per-iteration acceptance
 * temperature (annealed burn-in of Sec. 3.2: accept with probability
 * alpha^(1/T_t)).  temps: host double[iters], every T_t >= 1; NULL means all 1.
 */
hmc_status hmc_sample_tempered(hmc_handle h, int32_t chains, int32_t L, double eps, int64_t iters,
                               uint64_t seed, const void* beta0, void* samples, int32_t thin,
                               hmc_chain_stats* stats, const double* temps);

/*
 * hmc_predict -- posterior predictive class probabilities and classes
 * (Sec. 3.2: predict the class with the highest average softmax value over the
 * posterior samples).  For every row x_i of Xnew: prob[i][k] = the mean over
 * the draws d of psi_k(x_i B_d) (Eq. softmax, all K classes, the implied zero
 * logit of class K included in the identifiable layouts), summed in draw order
 * in FP64; cls[i] = argmax_k prob[i][k], the lowest class on a tie.  Logits and
 * softmax are formed in the handle's state type from Xnew as given.
 *   b        problem index (0 for a single-problem handle).
 *   draws    host or device [ndraws][R][p_b] of the state type: coefficient
 *            states of problem b in the beta layout of one chain, e.g. the
 *            samples of hmc_sample on a single-problem handle read as
 *            (iters / thin) * chains draws.  ndraws >= 1.
 *   Xnew     host or device, row-major n_new x p_b of x_dtype (HMC_F64 or
 *            HMC_F32).  n_new >= 0.
 *   prob     host or device double[n_new][K], or NULL.
 *   cls      host or device int32[n_new], or NULL.
 * At most 32 classes (HMC_EUNSUPPORTED above).  Synchronous.
 */
hmc_status hmc_predict(hmc_handle h, int32_t b, const void* draws, int64_t ndraws, const void* Xnew,
                       hmc_dtype x_dtype, int64_t n_new, double* prob, int32_t* cls);

/*
 * hmc_annealing_schedule -- the acceptance temperatures of the annealed
 * burn-in of Sec. 3.2 for `iters` iterations: T_t = max(1, r T_{t-1}) with
 * T_0 = t0, iteration t = 1..iters accepting at T_t (once T reaches 1 it stays
 * there).  temps: host double[iters] (output), to be passed to
 * hmc_sample_tempered.  Requires t0 >= 1, 0 < r <= 1, iters >= 0 (else
 * HMC_EINVAL).  Host computation only; no handle, no device work.
 */
hmc_status hmc_annealing_schedule(double t0, double r, int64_t iters, double* temps);

/*
 * hmc_get_state -- copy the handle's chain state: beta and grad (beta layout,
 * host or device, or NULL), logpost (double[nprob * chains], host or device,
 * or NULL) and the next iteration index (host, or NULL).  Synchronous.
 */
hmc_status hmc_get_state(hmc_handle h, int32_t chains, void* beta, void* grad, double* logpost,
                         int64_t* next_iteration);

/*
 * hmc_state_save / hmc_state_load -- checkpoint and resume of the chain state
 * that hmc_sample continues from: beta, grad and log K of the handle's chains
 * (every problem) and the next global iteration index, which numbers the
 * counter-based momentum and accept draws (Sec. 1.1 proposals).  The file at
 * `path` (host path, overwritten by save) records the state type, the storage
 * type of X, the prior (kind and scale), the coefficient layout and every
 * problem's (n, p, K).  Load requires a handle that matches all of them and has
 * max_chains >= the saved chain count, and it evaluates log K and the gradient
 * at the saved coefficients: if they differ from the saved ones by more than
 * rounding (relative 1e-4; 1e-9 for HMC_F64), the checkpoint belongs to another
 * posterior (other X or labels) and is rejected.  On success the handle's chain
 * state is replaced, so hmc_sample with beta0 = NULL, the saved chain count and
 * the same seed continues the saved chains; the continuation is bitwise
 * identical to an uninterrupted run when the device and the tile configuration
 * are the same (pass opts.tile explicitly: a measured tile choice may differ
 * between runs), otherwise equal to rounding.  Another chain count starts over
 * from zero.  Save needs a chain state (HMC_EINVAL before the first
 * hmc_sample); a missing, truncated or mismatched file is HMC_EINVAL.
 * Synchronous.
 */
hmc_status hmc_state_save(hmc_handle h, const char* path);
hmc_status hmc_state_load(hmc_handle h, const char* path);

/*
 * hmc_get_x -- copy the device-resident X of problem b as stored (after
 * conversion): row-major n x p elements of opts.x_storage (8, 4, 2 or 1
 * bytes each), unpadded, into host or device memory `dst`; for HMC_FP8E4M3
 * also the p float column scales into `scales` (host or device, or NULL).
 * Synchronous.
 */
hmc_status hmc_get_x(hmc_handle h, int32_t b, void* dst, float* scales);

/*
 * hmc_describe -- JSON text (static per handle) describing the chosen
 * engine, tile configuration, padded sizes and device buffers.
 */
const char* hmc_describe(hmc_handle h);

/*
 * hmc_set_timing / hmc_fused_kernel_time -- device time of the fused kernel,
 * measured with CUDA events on the handle's stream around every fused launch
 * once enabled with hmc_set_timing(h, 1), or around every k-th one with
 * hmc_set_timing(h, k) for k > 1 (fewer events in a captured iteration);
 * enabling resets the totals: total milliseconds and timed launches since then.  hmc_sample replays a captured
 * graph per iteration without synchronising between replays; its events are
 * read after the last iteration, so a sampling call contributes the launches
 * of its last iteration.
 */
hmc_status hmc_set_timing(hmc_handle h, int32_t enable);
hmc_status hmc_fused_kernel_time(hmc_handle h, double* total_ms, int64_t* launches);

/*
 * hmc_first_pass_time -- for the two-pass tensor-core engine (opts.engine 3):
 * the part of hmc_fused_kernel_time's total spent in the first pass (logits,
 * softmax and residual), measured by an event between the two passes of every
 * timed gradient; 0 for the single-pass engines.  Reset by hmc_set_timing.
 */
hmc_status hmc_first_pass_time(hmc_handle h, double* first_ms);

/*
 * hmc_logpost_grad_noalloc -- log K and its gradient (the quantities of
 * hmc_logpost_grad) for `chains` coefficient states of one FP32 problem,
 * computed without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc at call time -- programs that give (nearly) all device memory
 * to their own pool allocator at start-up, and latency-critical loops that
 * must not pay cudaMalloc's implicit device synchronisation.  No handle is
 * used; the caller owns every buffer below (all device memory):
 *   X        FP32, row-major n x ldx; columns [p, ldx) must be zero.
 *            ldx >= p and a multiple of 16; a multiple of 256 finds a tile up
 *            to 10240 for any C = chains (K-1) <= 20, up to 16384 for C <= 12
 *            and up to 20480 for C <= 6 (the coefficient slice and the ring of
 *            one cluster CTA share its shared memory).
 *   y        int32[n], labels in [0, K); the fused pass flags any other
 *            value and the call then returns HMC_ENONFINITE (outputs invalid).
 *   beta     FP32 [chains][K-1][p]; chains * (K-1) <= 20.
 *   logpost  double[chains]; grad FP32 [chains][K-1][p].
 *   stream   cudaStream_t (NULL: legacy default stream).
 * The library's intermediates live in a 16 MiB static device array that
 * every GPU loading the library holds until the process exits.  Problems
 * whose intermediates do not fit are rejected with HMC_EINVAL and a message;
 * the array also bounds the clusters of the fused pass (one partial gradient
 * slice each), so the widest problems run on fewer SMs than through a handle.
 * The first call on a device takes that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture.  All calls share the array: calls whose GPU
 * work overlaps (other streams or threads) race on it.  The call does not
 * allocate (no cudaMalloc, cudaFree or allocating library routine) and is
 * synchronous: it waits for its stream and returns HMC_ETIMEOUT if a
 * bounded device wait ran out.
 */
hmc_status hmc_logpost_grad_noalloc(const float* X, int64_t ldx, const int32_t* y, int64_t n, int64_t p,
                                    int32_t K, hmc_prior_kind prior, double prior_scale,
                                    const float* beta, int32_t chains, double* logpost, float* grad,
                                    void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HMC_H */
