/*
 * ptahmc.h -- C ABI of the B300 engine for the standardized Fourier-coefficient
 * pulsar-timing-array posterior (Gundersen, van Haasteren, Cornish, Vallisneri,
 * Meyers, "A new framework for lightning-fast gravitational wave analysis of
 * pulsar timing data").
 *
 * The library evaluates, for a batch of B HMC chains, the log posterior of
 * Eq. (raw_det_posterior) with the timing model marginalised by Eq.
 * (Gmatrix_proj), sampled in prior-whitened coordinates a = L z
 * (Eqs. standardizing_transform, standardized_density with mu = 0 and
 * Sigma = phi of Eq. prior_cov), and its gradient; and it runs fixed-length HMC
 * trajectories (App. "Hamiltonian Monte Carlo").
 *
 * Conventions shared by every call:
 *  - Return value: PTA_OK (0) or a negative PTA_E* code; pta_last_error() then
 *    holds a one-line message.  No call aborts the process.
 *  - Host arrays passed to pta_add_pulsar are copied; the caller keeps them.
 *  - Pointers named *_dev are device pointers owned by the caller (for example
 *    torch tensors).  The library never frees or reallocates them and never
 *    synchronises the stream it is given, except in pta_finalize.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy stream.
 *  - The context owns every device buffer it allocates; pta_destroy frees them.
 *  - Units inside: residuals and covariances in ns / ns^2 (Sec. "Single
 *    precision"), time in s.  Inputs are in seconds and MHz.
 */
#ifndef PTAHMC_H
#define PTAHMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PTA_OK 0
#define PTA_EINVAL (-1)   /* bad argument (NULL, size, NaN, sigma <= 0, m >= n, ...) */
#define PTA_ESTATE (-2)   /* call out of order (add after finalize, eval before) */
#define PTA_ECUDA (-3)    /* a CUDA runtime call failed */
#define PTA_ENOMEM (-4)   /* device or host allocation failed */
#define PTA_ETIMEOUT (-5) /* a bounded device wait gave up */
#define PTA_ECHECK (-6)   /* check build (libptahmc_check.so) only: an index check failed; the
                            site, value and limit are in pta_last_error */

/* Precision of the TOA-length contractions F a, F^T w, M^T w (Sec. "Single
 * precision").  The log-det, the timing-model solve and the final sums are FP64 in
 * every mode; the per-frequency Cholesky of the dense bins (with its inverse and
 * adjoint) and the CURN transform's factorisation are FP64 in PTA_PREC_FP64, and
 * double-word (a pair of floats, ~48-bit significand, relative error ~1e-14) on the FP32
 * pipes otherwise (pta_set_cholesky restores FP64). */
#define PTA_PREC_FP64 0   /* plain path: stored FP64 basis, SIMT FP64 */
#define PTA_PREC_FP32 1   /* basis generated on the fly, SIMT FP32 */
#define PTA_PREC_TF32X3 2 /* tcgen05 tensor cores, 3-term split TF32 */
#define PTA_PREC_TF32 3   /* tcgen05, single TF32 product (reported only) */
#define PTA_PREC_BF16X3 4 /* tcgen05, 3-term split BF16 (reported only) */
/* Gram form of the same posterior (Eq. posterior_implemented): per pulsar
 * F^T N~^-1 F, F^T N^-1 dt'' and dt''^T N^-1 dt'' stored at finalize (FP64, the
 * matrix kept as FP32 hi/lo), each evaluation a P x P product per (pulsar, chain)
 * in compensated FP32 (error-free products and sums) with FP64 dot products.  No
 * continuous-wave signal (PTA_EINVAL). */
#define PTA_PREC_GRAM 5
/* tcgen05 tensor cores at better than FP32 accuracy (the exact-split path): the
 * residual is formed with the projected basis F~ = F - M (M^T N^-1 M)^-1 M^T N^-1 F,
 * stored once per model (built in FP64 on the first call in this mode; 8 bytes per
 * TOA and column, 0.7 GB for 67 pulsars, 3e5 TOAs and P = 260) as four fp16 pieces
 * on fixed power-of-two grids, and the FP64 coefficients are cut the same way, so the
 * leading products sum exactly in the FP32 accumulator (ten MMAs per K step for F a,
 * six for F^T w~); w~ is staged in device memory between the two contractions.
 * PTA_EINVAL when P (+ max m_I with the continuous-wave signal) > 512 or m_I > 128. */
#define PTA_PREC_F16SPLIT 6

typedef struct pta_ctx pta_ctx;

/* Model sizes.  n_gwb / n_rn / n_dm are the numbers of Fourier frequencies
 * k/T (k = 1..n) of the GWB, intrinsic red noise and DM processes (Eq.
 * Fourier_series; the DM basis is F (nu_ref/nu)^2, text after Eq. RN=Fa).
 * Achromatic processes share one basis of max(n_gwb, n_rn) bins. */
typedef struct {
  int n_gwb;
  int n_rn;
  int n_dm;
  int cw;             /* 1: add the circular-binary deterministic signal */
  int precision;      /* PTA_PREC_* */
  double nu_ref_mhz;  /* DM reference frequency; 0 selects 1400 MHz */
  int spectrum;       /* spectral models (Sec. Priors): 0 power laws; bit 0 (PTA_FREE_GWB) a free
                         spectrum for the GWB, bit 1 (PTA_FREE_RN) for every pulsar's red noise */
} pta_model_desc;
#define PTA_FREE_GWB 1
#define PTA_FREE_RN 2

/* One pulsar.  All arrays have n entries except efac/equad (n_backend) and M
 * (n x m, row-major).  White noise N_ii = efac[b_i]^2 sigma_i^2 + equad[b_i]^2
 * (Eq. WN_cov); M is the timing design matrix of Eq. (TM=Me). */
typedef struct {
  int n, m, n_backend;
  const double* toas_s;
  const double* freqs_mhz;
  const double* resid_s;
  const double* sigma_s;
  const int32_t* backend;
  const double* efac;
  const double* equad_s;
  const double* M;
  double pos[3];      /* unit vector to the pulsar */
  double dist_kpc;    /* distance prior mean (CW pulsar term) */
} pta_pulsar_desc;

/* Offsets into the parameter vector x[D] of one chain:
 *   z_ach[k][c][I]  k < max(n_gwb, n_rn), c = 0 sin / 1 cos, I < npsr
 *   z_dm [I][k][c]  k < n_dm
 *   th_rn[I][2]     (log10 A, gamma) intrinsic red noise, Eq. (power_law); with
 *                   PTA_FREE_RN th_rn[I][n_rn]: log10 kappa_Ik (variance per bin, s^2)
 *   th_dm[I][2]     (log10 A, gamma) DM            (absent if n_dm == 0)
 *   th_gwb[2]       (log10 A, gamma) GWB; with PTA_FREE_GWB th_gwb[n_gwb]: log10 rho_k (s^2)
 *                   (free-spectrum prior: log10 ~ U(-20, -5) per bin)
 *   th_cw[8]        log10 Mc[Msun], log10 f_gw[Hz], log10 h, cos iota, psi,
 *                   cos theta, phi, Phi0; then per pulsar (L_I[kpc], Phi_I)
 *                   (absent unless cw) */
typedef struct {
  int npsr, n_ach, n_dm, P;   /* P = 2 n_ach + 2 n_dm coefficients per pulsar */
  int d_z, d;                 /* standardized block size, total size */
  int z_ach, z_dm, th_rn, th_dm, th_gwb, th_cw;
  long long ntoa;             /* total TOAs */
  double tspan_s, t0_s;       /* basis span T and origin t0 */
  int n_th_rn, n_th_gwb;      /* red-noise parameters per pulsar, GWB parameters (2 or bins) */
} pta_layout_t;

int pta_create(pta_ctx** out, const pta_model_desc* desc);
/* Copies the pulsar's arrays.  PTA_EINVAL for inconsistent sizes, after
 * finalize, or beyond 166 pulsars (the per-frequency N_p x N_p Cholesky and its
 * adjoint are held in shared memory, 8 bytes per element). */
int pta_add_pulsar(pta_ctx* ctx, const pta_pulsar_desc* psr);
/* Precompute (noise weights, normalised timing model, its FP64 Cholesky, the
 * Hellings-Downs matrix of Eq. HD, tile table) and upload.  Synchronises. */
int pta_finalize(pta_ctx* ctx, void* stream);
int pta_layout(const pta_ctx* ctx, pta_layout_t* out);
/* Select the contraction precision (PTA_PREC_*) for later calls.  PTA_EINVAL for
 * an unknown mode, for the TF32 modes beyond 896 coefficients per pulsar, and for
 * PTA_PREC_BF16X3 when P > 416 or P + max m_I + n_low > 384, n_low = 16 projected
 * low-frequency columns (the 4 lowest achromatic and 4 lowest DM bins), and for
 * PTA_PREC_F16SPLIT when P (+ max m_I with the continuous-wave signal) > 512.  The
 * continuous-wave model runs with PTA_PREC_FP32 and PTA_PREC_F16SPLIT. */
int pta_set_precision(pta_ctx* ctx, int precision);
/* Autotuner of the FP32 TOA kernel's tile shape (no counterpart in the paper).
 * Times every table entry that can run this model (chains per CTA, TOAs per tile,
 * ghat rows per thread, instruction order) on B chains, three launches each after
 * one warm-up, on `stream` with CUDA events, and keeps the fastest for later calls.
 * Needs PTA_PREC_FP32 (PTA_EINVAL otherwise).  Overwrites the context's scratch
 * coefficients (it is not an evaluation) and synchronises `stream`.  `ms`, if not
 * NULL, receives the mean time per launch of entry i (-1 for entries that cannot
 * run) for i < n_ms; `chosen` the selected entry.  Recaptures HMC graphs lazily. */
int pta_autotune(pta_ctx* ctx, int B, void* stream, int* chosen, double* ms, int n_ms);
/* Tempered likelihood (App. "The standardizing transform for tempered likelihoods",
 * Eq. tempered_post): later evaluations (pta_logp_and_grad, the no-allocation call
 * and HMC trajectories) return log p_beta = -beta/2 sum_I chi2_I - |z|^2/2 + log p(eta)
 * and its gradient for chain b with beta = beta[b], under the untempered
 * prior-whitened transform (valid, as the paper notes).  The data constant of
 * pta_logp_constant is the beta = 1 one; the tempered likelihood's constant is beta
 * times its likelihood part.  beta: n doubles in device or host memory, copied on
 * `stream` (the caller's array may be reused once the stream passes the call); the
 * context keeps its own copy.  Evaluations of more than n chains then return
 * PTA_EINVAL.  n = 0 or beta = NULL turns tempering off.  Expected 0 <= beta. */
int pta_set_beta(pta_ctx* ctx, int n, const double* beta, void* stream);
/* Standardizing transform of the Fourier coefficients for later evaluations and HMC
 * trajectories (PTA_TRANSFORM_*).
 *   PTA_TRANSFORM_PRIOR (default): a_{.,k,c} = L_k z_{.,k,c} with Phi_k = L_k L_k^T per
 *     frequency bin (Eq. standardizing_transform with mu = 0, Sigma = phi);
 *     logp = -beta/2 sum_I chi2_I - |z|^2/2 + log p(eta).
 *   PTA_TRANSFORM_CURN: per pulsar a_I = ahat_I + L_I z_I (Eq. PTA_standard_transform_curn)
 *     with Sigma_I = (beta F_I^T N~_I^-1 F_I + phi_CURN,I^-1)^-1 = L_I L_I^T (lower
 *     Cholesky factor) and ahat_I = beta Sigma_I F_I^T N~_I^-1 dt_I; phi_CURN is the prior
 *     covariance without inter-pulsar correlations (rho_k + kappa_Ik, kappa^DM_Ik on the
 *     diagonal).  With tempering this is the tempered transform T_beta of App. "The
 *     standardizing transform for tempered likelihoods".  logp = -beta/2 sum_I chi2_I
 *     - 1/2 a^T phi^-1 a - 1/2 log det phi + sum_I log det L_I + log p(eta) with the
 *     Hellings-Downs-correlated phi (Eq. standardized_stochastic_posterior, the
 *     (2 pi)^(-D_z/2) and the data constant dropped as in the default transform).  z
 *     keeps the layout of pta_layout: the entry of coefficient (I, p) sits where the
 *     prior-whitened transform keeps it.  Each evaluation factorises one P x P matrix
 *     per (pulsar, chain), about P^3/3 multiply-adds (double-word outside PTA_PREC_FP64 and
 *     PTA_CHOL_FP64, in one CTA or, for P >= 234, over a cluster of 2 to 8 CTAs; FP64 for
 *     P >= 584), and keeps B N_p P (P + 1) / 2 doubles of inverse factors between the value
 *     and the gradient (PTA_ENOMEM from the evaluation if they do not fit).
 * With the continuous-wave signal h(theta) the mean is abar_I = beta Sigma_I F_I^T N~_I^-1
 * (dt_I - h_I) (Eq. decenter_det_PTA) and the CW gradient includes its dependence on theta;
 * this costs one extra TOA pass per evaluation and one more when the gradient is asked for.
 * PTA_EINVAL for an unknown value.  pta_logp_and_grad_noalloc rejects the CURN transform.
 * Recaptures HMC graphs. */
#define PTA_TRANSFORM_PRIOR 0
#define PTA_TRANSFORM_CURN 1
int pta_set_transform(pta_ctx* ctx, int transform);
/* Arithmetic of the per-frequency N_p x N_p Cholesky of the dense bins (Eq. prior_cov:
 * Phi_k = rho_k Gamma + diag(kappa_.k)), its inverse and the adjoint of a = L z.
 * PTA_CHOL_DW (the default): double-word arithmetic on the FP32 pipes (pairs of floats,
 * ~48-bit significand; factor, inverse and transform agree with FP64 to ~1e-14
 * relative), several times faster on B300, whose FP64 rate is 1/64 of its FP32 rate.
 * PTA_CHOL_FP64: the FP64 sweep, and the FP64 factorisation of the CURN transform.
 * PTA_PREC_FP64 always uses the FP64 sweeps.  The log-det and the final sums stay FP64
 * either way.  PTA_EINVAL for an unknown value; recaptures HMC graphs. */
#define PTA_CHOL_DW 0
#define PTA_CHOL_FP64 1
int pta_set_cholesky(pta_ctx* ctx, int mode);
/* Test hook for the bounded device waits (no counterpart in the paper).  code 1:
 * in PTA_PREC_BF16X3 evaluations the tensor-core kernel withholds the completion
 * signal of its first tile's F a product, so its epilogue's bounded mbarrier wait
 * runs out (a bounded poll, seconds at most); every CTA then drains its own copies and MMAs, frees
 * tensor memory and marks its chains with status bit 4 (PTA_OK is returned: the
 * context stays usable).  code 0 restores normal operation.  PTA_EINVAL otherwise. */
int pta_debug_inject(pta_ctx* ctx, int code);
/* Force TOA kernel table entry `cfg` (-1: the untuned default).  PTA_EINVAL if the
 * entry cannot run this model. */
int pta_set_toa_config(pta_ctx* ctx, int cfg);
/* Shape of table entry cfg: chains per CTA, TOAs per tile, ghat rows per thread,
 * and `order` = instruction order (bit 0: TOA-outermost F^T w) + 2 x next-tile
 * prefetch (bit 1) + 4 x persistent launch (bit 2: resident CTAs take work units,
 * longest first, from an atomic counter).  PTA_EINVAL past the end of the table. */
int pta_toa_config_info(int cfg, int* bc, int* tt, int* qpt, int* order);
/* Hyper-prior box for (log10 A, gamma) of the GWB, red noise and DM (Sec.
 * "Priors": log10 A ~ U(-20,-10), gamma ~ U(0,7) by default). */
int pta_set_hyperprior(pta_ctx* ctx, double log10a_lo, double log10a_hi,
                       double gamma_lo, double gamma_hi);
/* Prior support of every coordinate of x, into host arrays lo[D], hi[D]: the
 * (log10 A, gamma) boxes of pta_set_hyperprior, the free-spectrum box (-20, -5), the CW
 * box and the pulsar phases (0, 2 pi) are finite; z and the pulsar distances get
 * (-inf, inf).  PTA_ESTATE before pta_finalize. */
int pta_param_bounds(const pta_ctx* ctx, double* lo, double* hi);

/* Log posterior and gradient for B chains (the hot path).
 *   x_dev      [B x D] float32, row per chain (layout above)
 *   logp_dev   [B] float64: -1/2 sum_I r_I^T N~_I^-1 r_I - 1/2 |z|^2 + log p(theta),
 *              data-only constants dropped (see pta_logp_constant)
 *   grad_dev   [B x D] float32 d logp / d x, or NULL
 *   status_dev [B] int32, or NULL: 0 ok; 1 theta outside the prior box;
 *              2 per-frequency covariance not positive definite; 3 non-finite;
 *              4 a bounded device wait in the tensor-core kernel gave up.
 *              Any nonzero status sets logp = -inf and grad = 0 for that chain.
 * Asynchronous on `stream`. */
int pta_logp_and_grad(pta_ctx* ctx, int B, const float* x_dev, double* logp_dev,
                      float* grad_dev, int32_t* status_dev, void* stream);

/* One HMC transition per chain (Eqs. Hamiltonian, Hamilton's_eq,
 * Gaussian_momentum, HMC_acceptance): momentum p ~ N(0, M) from Philox4x32-10
 * (counter (j, chain, iteration), key seed), n_leapfrog leapfrog steps of size
 * step_dev[b] with inverse mass inv_mass_dev[D] (NULL = identity), Metropolis
 * accept.  x/logp/grad are read as the current state and overwritten with the
 * next state; logp/grad must hold the values at x on entry.
 * accepted_dev[B] receives 1/0.  The leapfrog loop runs as a CUDA graph that is
 * captured on first use for each (B, n_leapfrog) and replayed after.
 * Coordinates with a finite prior box [lo, hi] (pta_param_bounds) move during the
 * trajectory in u = logit((x - lo) / (hi - lo)), x = lo + (hi - lo) sigmoid(u), with the
 * log-Jacobian sum of log((hi - lo) s (1 - s)) added to the target (the unconstrained
 * reparameterisation of a box-bounded parameter; the paper's hyper-priors are uniform
 * boxes): trajectories never leave the prior support, and inv_mass_dev and the momentum
 * refer to u for those coordinates.  x, logp and grad on entry and exit are in x. */
int pta_hmc_trajectory(pta_ctx* ctx, int B, float* x_dev, double* logp_dev, float* grad_dev,
                       const float* step_dev, const float* inv_mass_dev, int n_leapfrog,
                       uint64_t seed, uint64_t iteration, int32_t* accepted_dev, void* stream);

/* Same result as pta_logp_and_grad, but the call allocates nothing: its per-call
 * workspace is a fixed 32 MiB array compiled into the library (held on every GPU
 * that loads the library until exit) instead of context-owned device memory.  The
 * paper has no counterpart; it exists for callers that cannot call cudaMalloc when
 * they evaluate: a host framework that owns every device allocation and forbids
 * allocations outside its own allocator, or a sampler loop that must not pay for or
 * risk an allocation failure in the middle of a run.  The context still holds the
 * data uploaded by pta_finalize.
 *   - B chains must fit in the array: otherwise PTA_EINVAL with the needed size in
 *     pta_last_error (for 67 pulsars and 3e5 TOAs: 1.24 MB per chain, 27 chains; the
 *     FP64 path also keeps FP64 partial sums, 1.62 MB per chain, 20 chains).
 *   - The first call on a device looks up the array's device address (with that
 *     device current) and caches it; make that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents: calls that
 *     overlap on the GPU race.  What must start at zero (the per-chain status flags
 *     and the work counter of persistent launches) is cleared on `stream` per call.
 *   - PTA_PREC_FP64 needs the stored FP64 basis, which pta_logp_and_grad builds on
 *     its first FP64 call; without it the call returns PTA_ESTATE.
 *   - PTA_PREC_BF16X3 and PTA_PREC_F16SPLIT (their packed coefficients and, for the
 *     latter, the staged w~ need their own buffers) and the
 *     continuous-wave model return PTA_EINVAL. */
int pta_logp_and_grad_noalloc(pta_ctx* ctx, int B, const float* x_dev, double* logp_dev,
                              float* grad_dev, int32_t* status_dev, void* stream);

/* The data-only constant dropped from logp:
 * -1/2 sum_I [log det(2 pi N_I) + log det(M_I^T N_I^-1 M_I) - m_I log 2 pi]
 * in ns units, minus (D_z/2) log 2 pi (host value, available after finalize). */
int pta_logp_constant(const pta_ctx* ctx, double* c);

/* Stage timing for measurement.  While enabled, pta_logp_and_grad records CUDA
 * events on the caller's stream around each of its stages and counts the kernels
 * it launches per stage.  pta_profile_read waits for the recorded events, writes
 * the accumulated milliseconds and launch counts per stage (arrays of
 * PTA_NSTAGES entries, either may be NULL) and, if reset != 0, clears them.
 * Stages: 0 prior forward (spectra, Cholesky, transform), 1 TOA contractions,
 * 2 FP64 epilogue (timing-model solve), 3 adjoint, 4 final sum; their sum is the
 * evaluation.  Entries 5-7 time single kernels inside those stages (no launches
 * counted): 5 the dense-bin Cholesky k_chol_forward, 6 the exact-split residual
 * kernel k_f16_res, 7 its F^T w~ kernel k_f16_ftw. */
#define PTA_NSTAGES 8
int pta_profile_enable(pta_ctx* ctx, int enable);
int pta_profile_read(pta_ctx* ctx, double* ms, long long* launches, int reset);

const char* pta_last_error(const pta_ctx* ctx);
void pta_destroy(pta_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
