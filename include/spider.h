/*
 * spider.h -- C ABI of the GB300-native SPIDER sampling step.
 *
 * SPIDER (Ross, Wilding, Azizzadenesheli, Kato; arXiv 2508.12117) samples the
 * joint posterior of M hypocentres theta_m = (x_m, y_m, z_m, t0_m) (Sec. 2.1:
 * theta = {(x_m, t_m^s)}) from N double-difference (dd) times with Stochastic
 * Gradient Langevin Dynamics (Sec. 3.2).  One step of this library:
 *
 *   1. draws a minibatch of whole observation blocks (Eq. sgd: n of N),
 *   2. evaluates travel times T(x_event; s_station) and dT/dx for every
 *      (event, station) pair the minibatch touches (Sec. 2.1, Eq. forwardmodel),
 *   3. forms residuals r_n = tau_obs_n - [(T_ik + t0_i) - (T_jk + t0_j)] (Eq. 1),
 *   4. whitens them with the marginal covariance of each station group,
 *      Sigma_g = sigma^2 I + kappa^2 W^1/2 A A^T W^1/2 (Eq. marginal_sigma),
 *   5. scatter-reduces dlogp/dT onto pairs and chains it to the events,
 *   6. adds the event and centroid priors (Sec. 3.1) and applies
 *      theta += eps * grad + sqrt(2 eps) * eta (Sec. 3.2).
 *
 * Conventions (every entry point):
 *   - returns SPIDER_OK (0) or a negative SPIDER_E_* code; the message of the
 *     last failure on a context is spider_last_error(ctx) (a static string for
 *     ctx == NULL failures);
 *   - the caller owns every pointer it passes; the library reads host inputs
 *     only during the call and copies what it keeps;
 *   - the context owns all device memory it allocates; spider_destroy frees it;
 *   - event order in every result is the caller's order (the library's own
 *     spatial renumbering is undone);
 *   - a context is not thread safe; distinct contexts are independent;
 *   - device work runs on the context's CUDA stream (the `stream` argument of
 *     spider_create, a cudaStream_t, or a private stream when NULL); calls that
 *     return host data synchronise that stream.
 */
#ifndef SPIDER_H
#define SPIDER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SPIDER_OK = 0,
  SPIDER_E_INVAL = -1,       /* bad argument or inconsistent input               */
  SPIDER_E_OOM = -2,         /* device or host allocation failed                 */
  SPIDER_E_CUDA = -3,        /* a CUDA call failed (message holds its string)    */
  SPIDER_E_NONFINITE = -4,   /* a NaN/Inf appeared in the state or the gradient  */
  SPIDER_E_TIMEOUT = -5,     /* a bounded device-side wait gave up               */
  SPIDER_E_UNSUPPORTED = -6  /* valid request this build cannot serve            */
};

/* travel-time model T(x; s) */
enum {
  SPIDER_TT_HOMOGENEOUS = 0,     /* T = |x - s| / v0 (Sec. 2.1, homogeneous medium) */
  SPIDER_TT_LINEAR_GRADIENT = 1, /* v = v0 + g z: T = arccosh(1 + g^2 r^2 / (2 v_x v_s)) / g */
  SPIDER_TT_MLP = 2              /* T = |x - s| * tau(x, s), tau an MLP 6 -> 4 x H SiLU -> 1
                                    (the EikoNet stand-in of Sec. 3.2) */
};

/* arithmetic of the MLP hidden layers.  The output layer, T, residuals and
 * positions are FP32 in every mode.  Layer 1 is FP32 in SPIDER_FP32; in
 * SPIDER_BF16 and SPIDER_FP8 it is a tensor-core product of BF16 operand pairs
 * (v = v_hi + v_lo for the inputs and W1), FP32-accumulated, whose only dropped
 * term is W1_lo x_lo (at most 2^-16 of each product), followed by FP32 bias and
 * SiLU. */
enum { SPIDER_FP32 = 0, SPIDER_BF16 = 1, SPIDER_FP8 = 2 };

typedef struct {
  int64_t M;               /* events, 2 <= M < 2^31                              */
  int64_t N;               /* dd observations, 1 <= N < 2^30 (a double difference
                              needs two events and at least one observation)     */
  const double *xyzt0;     /* M x 4 row-major initial catalog theta_0: x, y, z (km,
                              z positive down), t0 (s).  Also the mean of the event
                              prior (Sec. 3.1) and the centre of the centroid prior. */
  const int32_t *i;        /* N: first event xi^1_n, in [0, M)                   */
  const int32_t *j;        /* N: second event xi^2_n, in [0, M), != i            */
  const int32_t *k;        /* N: station eta_n, in [0, S)                        */
  const double *dt;        /* N: observed dd time tau_obs_n = t_i - t_j at k (s) */
  const float *w;          /* N edge weights w_e of Eq. correlation_decay, already
                              normalised; NULL: computed from theta_0 as
                              (d_e / ell)^p + eps_w, mean 1 per station group     */
} spider_catalog;

typedef struct {
  int32_t S;               /* stations                                           */
  const double *xyz;       /* S x 3 row-major station positions (km)             */
} spider_stations;

typedef struct {
  int32_t kind;            /* SPIDER_TT_*                                        */
  double v0, g;            /* homogeneous speed / gradient medium (km/s, 1/s)    */
  int32_t H;               /* MLP hidden width: a multiple of 32, 32..256        */
  const float *W[5];       /* MLP weights, (out, in) row-major: H x 6, H x H (x3),
                              1 x H.  Inputs are [x_src; x_rcv] in km.          */
  const float *b[5];       /* MLP biases: H (x4), 1                              */
} spider_net;

typedef struct {
  double sigma;            /* sigma_phi (s), iid noise of Eq. marginal_sigma     */
  double kappa;            /* kappa_phi (s), shared-event term; 0 = iid likelihood */
  double p, ell, eps_w;    /* Eq. correlation_decay exponent, length (km), floor  */
  double sig_e[4];         /* event prior sigmas (km, km, km, s)                  */
  double sig_c[4];         /* centroid prior sigmas (km, km, km, s)               */
  int64_t batch_n;         /* observations per minibatch; 0 or >= N = full batch */
  int64_t block_obs;       /* observations per minibatch block, 1..4096          */
  int32_t precision;       /* SPIDER_FP32 / SPIDER_BF16 / SPIDER_FP8             */
  int32_t thin;            /* keep every thin-th state as a sample (>= 1)        */
  int32_t reorder;         /* 1: renumber events along a Morton curve (locality) */
  int32_t chain;           /* Philox counter word 1 (chain id)                   */
  int32_t catalog;         /* Philox counter word 2 (catalog id)                 */
  float noise_scale;       /* multiplies sqrt(2 eps) eta (stage-3 ramp, Sec. 3.2) */
  int32_t pcg_max_it;      /* whitening solve: cap on inner CG iterations         */
  float pcg_tol;           /* whitening solve: target |u - A z| / |u|, with the
                              residual evaluated in double-float (refinement)     */
  int64_t sample_cap;      /* samples kept on the device (ring buffer)           */
  /* update rule of spider_sgld_step (Sec. 3.2):
   *   SPIDER_UPDATE_SGLD   theta += eps g + noise_scale sqrt(2 eps) eta
   *   SPIDER_UPDATE_PSGLD  Eq. pSGLD: v = beta2 v + (1 - beta2) g*g,
   *                        V = 1 / (sqrt(v) + upd_eps),
   *                        theta += eps V g + noise_scale sqrt(2 eps V) eta
   *   SPIDER_UPDATE_ADAM   stage 1 (Sec. 3.2): Adam on the log posterior (ascent),
   *                        no noise: m = beta1 m + (1 - beta1) g, v as above,
   *                        theta += eps (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + upd_eps),
   *                        t = step counter + 1                                  */
  int32_t update;
  float beta1, beta2;      /* moment decay rates, in [0, 1)                       */
  float upd_eps;           /* damping of the preconditioner (Sec. 4: 1e-5)        */
  /* data term of the log posterior:
   *   SPIDER_LOSS_WHITENED  Eq. marginal_sigma (Gaussian, whitened per station)
   *   SPIDER_LOSS_L1        stage 1 (Sec. 3.2): -(N/n) sum_n |r_n|, no whitening */
  int32_t loss;
} spider_config;

enum { SPIDER_UPDATE_SGLD = 0, SPIDER_UPDATE_PSGLD = 1, SPIDER_UPDATE_ADAM = 2 };
enum { SPIDER_LOSS_WHITENED = 0, SPIDER_LOSS_L1 = 1 };

typedef struct spider_ctx spider_ctx;

/* Fills *cfg with the defaults: Table 1 / Sec. 4 values (kappa 0.03 s, p 0.25,
 * ell 40 km, centroid sigma 0.01), event prior 0.5 km / 0.1 s (Sec. 4.1),
 * full batch, blocks of 4096, FP32, thin 1, reorder 1, noise 1, whitening 1000 / 1e-7,
 * SGLD update (beta1 0.9, beta2 0.99, upd_eps 1e-5: Sec. 4), whitened loss. */
void spider_config_default(spider_config *cfg);

/* Validates and copies the catalog, stations and network; builds the canonical
 * observation order, the (event, station) pair table, the minibatch blocks and
 * the edge weights; uploads everything; state theta := theta_0, step := 0.
 * stream: a cudaStream_t or NULL.  *out receives the context on success.
 * SPIDER_E_INVAL (with a message) for sizes out of range, indices out of range,
 * i == j, non-finite coordinates or times, or an invalid configuration. */
int spider_create(const spider_catalog *cat, const spider_stations *sta,
                  const spider_net *net, const spider_config *cfg, void *stream,
                  spider_ctx **out);

/* Many independent samplers in one context: n_catalogs catalogs (each with its
 * own stations) times `chains` chains each (Sec. 3.5 runs one chain per GPU;
 * here every chain of every catalog advances in the same kernel launches, and
 * spider_sgld_step relaunches one captured CUDA graph per step).  Sub-problem
 * s = catalog c * chains + h keeps its own events, minibatch, N/n scale,
 * centroid prior and Langevin noise: its blocks are drawn with the key
 * batch_seed XOR (s * 0x9E3779B97F4A7C15) and its noise uses counter
 * (event index in catalog c, h, c, 'NOIS') with key batch_seed (cfg->chain and
 * cfg->catalog are ignored).  States, gradients and samples are laid out
 * sub-problem by sub-problem: [c][h][event][4].  Inputs are copied. */
int spider_create_batch(int32_t n_catalogs, const spider_catalog *cats,
                        const spider_stations *stas, const spider_net *net,
                        const spider_config *cfg, int32_t chains, void *stream,
                        spider_ctx **out);

/* Gradient of the log posterior at the current state (Eq. sgd without the
 * step): minibatch keyed by batch_seed (0 = full batch), likelihood scaled by
 * N/n.  grad_out: host M x 4 FP32 (caller order) or NULL.  logpost_out: host
 * FP64 log posterior estimate (constants dropped) or NULL.  Synchronous. */
int spider_grad_logpost(spider_ctx *ctx, uint64_t batch_seed, float *grad_out,
                        double *logpost_out);

/* One SGLD step (Sec. 3.2): minibatch and Langevin noise both keyed by
 * batch_seed; theta += eps * grad + noise_scale * sqrt(2 eps) * eta.  Asynchronous
 * on the context stream; errors found on the device surface at the next
 * synchronous call.  While timing is off the step's kernels run as one CUDA
 * graph, captured on the first call (make it outside any other capture). */
int spider_sgld_step(spider_ctx *ctx, float eps, uint64_t batch_seed);

/* Copies up to `cap` stored samples (oldest first) as M x 4 FP64 each, caller
 * order, into out; *n_written = count.  Synchronous. */
int spider_samples(spider_ctx *ctx, double *out, int64_t cap, int64_t *n_written);

/* Current state (M x 4 FP64, caller order) and step counter.  Synchronous.
 * theta_0 + dtheta is formed on the device (theta_0 kept in FP64) and copied in
 * one transfer; a page-locked theta_out is written by DMA. */
int spider_get_state(spider_ctx *ctx, double *theta_out, int64_t *step_out);

/* Replaces the state and step counter (exact resume: with the same per-step
 * seeds the continued chain is bit-identical).  Synchronous. */
int spider_set_state(spider_ctx *ctx, const double *theta, int64_t step);

/* Moment state of the pSGLD / Adam updates: m (first moment, Adam) and v
 * (second moment), M x 4 FP64 each in caller order; either pointer may be NULL.
 * Both start at zero; spider_set_state leaves them alone, so an exact resume of
 * a pSGLD or Adam run restores both.  SPIDER_E_INVAL for the SGLD update (no
 * moments are kept).  Synchronous. */
int spider_get_moments(spider_ctx *ctx, double *m_out, double *v_out);

/* Sets the multiplier of the injected noise for the following steps (Sec. 3.2:
 * stage 2 runs with the noise off, stage 3 ramps it linearly to full
 * amplitude).  noise_scale >= 0.  Takes effect at the next spider_sgld_step. */
int spider_set_noise_scale(spider_ctx *ctx, float noise_scale);
int spider_set_moments(spider_ctx *ctx, const double *m, const double *v);

/* Stage-1 outlier rejection (Sec. 3.2: observations whose residual lies more
 * than k_mad median absolute deviations from the median are discarded; the
 * paper uses k_mad = 4).  Evaluates the residuals of every observation at the
 * current state, then per catalog (sub-problem) the median of r and
 * MAD = median |r - median| (an even count takes the mean of the two middle
 * values; FP32 values, exact selection), and keep_n = |r_n - median| <= k_mad MAD.
 * keep_out: host uint8[N] in the caller's observation order (1 = keep) or NULL;
 * n_kept_out: count kept or NULL; med_out, mad_out: host double[n_sub] or NULL
 * (n_sub = 1 for spider_create, catalogs x chains for spider_create_batch).
 * Build the next stage's catalog from the kept observations.  Synchronous. */
int spider_outlier_mask(spider_ctx *ctx, double k_mad, uint8_t *keep_out, int64_t *n_kept_out,
                        double *med_out, double *mad_out);

/* Linearisation-regime filter (Proposition 1, Eq. dd_linearization; Sec. 4
 * keeps observations whose linearisation error is at most 5 %).  At the current
 * state, observation (i, j, k) has dT = T(x_j, s_k) - T(x_i, s_k) and the
 * linearised dT_lin = grad_x T(x_i, s_k) . (x_j - x_i); it is kept when
 * |dT - dT_lin| <= max_rel |dT| (max_rel = 0.05 in the paper).  keep_out: host
 * uint8[N] in the caller's observation order (1 = keep) or NULL; n_kept_out:
 * count kept or NULL.  Build the next stage's catalog from the kept
 * observations.  Synchronous. */
int spider_linearisation_mask(spider_ctx *ctx, double max_rel, uint8_t *keep_out, int64_t *n_kept_out);

/* Posterior summaries from the n stored samples (the ring of spider_samples,
 * oldest first), per event and coordinate (x, y, z, t0):
 *   median_out, halfwidth_out: the median and half the length of the interval
 *     between the lo_pct and hi_pct percentiles (Sec. 3.5: e.g. [0.5, 99.5] for
 *     a 99 % credible interval; linear interpolation between order statistics
 *     at rank (n - 1) p / 100);
 *   calib_out: the fraction of samples below the true value `truth` (Sec. 4.1
 *     calibration; truth: host M x 4 FP64 caller order, or NULL);
 *   ess_out: effective sample size (Sec. 5) n / tau, tau = 1 + 2 sum_{t >= 1}
 *     rho_t over the lags while the autocorrelation rho_t stays positive.
 * Outputs are host M x 4 FP64 in caller order, or NULL.  SPIDER_E_INVAL with
 * fewer than 2 or more than 4096 stored samples.  Synchronous. */
int spider_uq(spider_ctx *ctx, const double *truth, double lo_pct, double hi_pct, double *median_out,
              double *halfwidth_out, double *calib_out, double *ess_out);

/* Waits for queued device work; returns the first device-side error, if any. */
int spider_sync(spider_ctx *ctx);

/* Limit of every bounded device-side wait of the step (the grid-wide barriers
 * of the component labelling and of the large-component CG), in ns; the
 * default is 2 s, at most 600 s.  0 makes a CTA give up as soon as it finds a
 * barrier incomplete.  A wait that gives up records SPIDER_E_TIMEOUT; every
 * later kernel of that step, and of the steps queued after it, then returns
 * without work (theta is left unchanged; the step counter still counts the
 * steps), until a synchronous call (spider_sync, spider_get_state, ...) reports
 * the error and clears it.  The tensor-core MLP kernel keeps its own 2 s limit
 * on its pipeline waits.  Takes effect at the next step. */
int spider_set_wait_limit_ns(spider_ctx *ctx, uint64_t limit_ns);

/* Per-stage device time of the most recent step or gradient, in ms, from CUDA
 * events on the context stream (enable with spider_set_timing(ctx, 1)):
 * out[0] selection+pair table, [1] travel times (the MLP), [2] residuals and
 * whitening, [3] scatter and event reduce + update, [4] whole call.  Also the
 * pairs evaluated (P_u), observations used and whitening CG iterations (the
 * largest count of any connected component of the minibatch graph). */
int spider_set_timing(spider_ctx *ctx, int enable);
int spider_last_timing(spider_ctx *ctx, float out_ms[5], int64_t *pairs,
                       int64_t *n_obs, int32_t *pcg_iters);

/* Device time of each part of the most recent timed step or gradient, in ms
 * (CUDA events on the context stream; zeros while timing is off):
 * out[0] selection + pair table, [1] travel times, [2] residuals and u = B^T r
 * (k_resid), [3] merge of u over blocks sharing a pair (k_merge_rhs),
 * [4] whitening solve (matrix, components, solvers), [5] q = Sigma^-1 r and
 * per-node sums (k_final), [6] scaled dlogp/dT onto pairs (k_merge_s),
 * [7] centroid, [8] priors + update per event (k_event), [9] log posterior.
 * *touched_events: events with at least one pair in the minibatch. */
int spider_last_kernel_timing(spider_ctx *ctx, float out_ms[10], int64_t *touched_events);

/* Phases of the whitening solve of the last timed evaluation, when it took
 * the piece-inverse path (all zero otherwise; synchronous): [0] labelling the
 * selected pieces and grouping them into units, [1] the units' set-up (their
 * shared nodes, the pieces' (A_p[G,G])^-1 and S^-1), [2] the units' Schur
 * rounds and convergence check, [3] the CTA passes for units beyond the
 * data-parallel limits, [4] waiting for the clean-piece solver on its side
 * stream, [5] the general component solver (a no-op unless a unit exceeded
 * every limit).  Device ms from CUDA events. */
int spider_last_whiten_timing(spider_ctx *ctx, float out_ms[6]);

/* Debug views of the last evaluation (synchronous):
 * spider_debug_blocks: selected block ids in selection order (int64, cap);
 * spider_debug_obs: for every observation of the last minibatch, its caller
 * index, residual r_n and whitened q_n = (Sigma^-1 r)_n (unscaled). */
int spider_debug_blocks(spider_ctx *ctx, int64_t *out, int64_t cap, int64_t *n);
int spider_debug_obs(spider_ctx *ctx, int64_t *idx_out, float *r_out, float *q_out,
                     int64_t cap, int64_t *n);

/* Launch-shape knobs that change speed but not results (every pair and every
 * connected component is computed independently of how work is spread):
 * knobs[0] CTAs per SM-slot of the per-component warp solver (1..8),
 * knobs[1] of the per-component CTA solver (1..4), knobs[2] CTAs per SM of
 * the FP32 MLP kernel (1..2), knobs[3] 1 (default): minibatch steps whiten
 * through the precomputed inverses of the block-local components when they
 * were built, 0: always through the general component solver; knobs[4]
 * (0..4, default 2) the share, in quarters, of the persistent grid the
 * clean-piece solver takes on its side stream while the units are solved
 * (0: it runs after them on the context's stream); knobs[5] (1, 2 (default)
 * or 4) threads per CTA of the per-block kernels (pair table, residuals,
 * whitened residuals), in units of 256 (the observations and nodes each thread
 * handles; changes only the rounding order of the FP64 log-likelihood sum);
 * knobs[6] 1 (default): the size classes of the units' small inverses
 * (piece blocks, then Schur complements) run side by side on four branch
 * streams, 0: one after the other on the context's stream.  The first
 * min(n, 7) knobs are set, the others kept.  Invalidates the captured step graph. */
int spider_set_tuning(spider_ctx *ctx, const int32_t *knobs, int32_t n);

/* Facts about a context (synchronous), out[0..n): [0] sub-problems,
 * [1] 1 if the SGLD step runs as a captured CUDA graph, [2] blocks per
 * minibatch step, [3] blocks in total, [4] pairs in total, [5] events,
 * [6] observations, [7] connected components of the last minibatch graph,
 * [8] block-local nodes (occurrences of pairs in blocks) in total,
 * [9] 1 if the inverses of the block-local components were precomputed,
 * [10] 1 if minibatch steps whiten through them, [11] units of pieces that
 * shared nodes in the last such step, [12] 1 if that step fell back to the
 * general component solver (a unit beyond the limits of the direct path),
 * [13] units of that step solved by the last unit pass, [14], [15] SM cycles /
 * 1024 spent on the units of the CTA pass and of the last pass, [16..30]
 * five counters per unit pass ([16..20] stay zero; [21..25] the CTA pass,
 * [26..30] the last pass): SM cycles / 1024 in set-up, the pieces' small
 * inverses, the inverse of S, the refinement rounds, and the units solved; [31..37] units the data-parallel unit solver handed to
 * the CTA passes since the context was created, by reason: too many pieces,
 * shared occurrences, shared nodes, shared nodes of one piece, a failed small
 * inverse, a failed inverse of S, a full pool; [38] kernel launches in the
 * captured step graph (0 until a graph step ran). */
int spider_info(spider_ctx *ctx, int64_t *out, int32_t n);

/* Sampler diagnostics of Sec. 3.6 at the current state, accumulated in FP64 on
 * the device: the minibatch gradient g (batch_seed) and the full-batch
 * gradient G are evaluated; grad_norms_out (host, M, caller order, or NULL)
 * receives |g_m|; *ratio_out receives the variance of the stochastic gradient
 * relative to the injected Langevin noise, eps^2 mean((g - G)^2) / (2 eps),
 * the quantity the paper tunes eps against (0.1-1). */
int spider_diagnostics(spider_ctx *ctx, uint64_t batch_seed, float eps, double *grad_norms_out,
                       double *ratio_out);

const char *spider_last_error(const spider_ctx *ctx);
void spider_destroy(spider_ctx *ctx);

/* ---- context-free pieces (device pointers, caller-owned) ----------------- */

typedef struct spider_netdev spider_netdev;

/* Uploads a travel-time network (any kind) for spider_tt_pairs. */
int spider_net_upload(const spider_net *net, int32_t precision, spider_netdev **out);
void spider_net_free(spider_netdev *nd);

/* Travel times and source Jacobians for P (source, receiver) pairs, the kernel
 * a step uses (Sec. 2.1; reverse-mode chain of Sec. 3.2 for the MLP).
 * src, rcv: device P x 4 FP32 (x, y, z, unused).  T_hi, T_lo: device P FP32
 * each, T = T_hi + T_lo to about 1e-12 relative (T_lo may be NULL).
 * J: device P x 4 FP32 (dT/dx, dT/dy, dT/dz, 0) or NULL.  stream: cudaStream_t
 * or NULL (legacy default).  Asynchronous. */
int spider_tt_pairs(const spider_netdev *nd, int64_t P, const float *src, const float *rcv,
                    float *T_hi, float *T_lo, float *J, void *stream);

/* Allocation-free variant of spider_tt_pairs for the MLP model in FP32.  The
 * paper has no counterpart: it exists for callers that may not allocate device
 * memory -- code running inside a runtime that owns all device memory up
 * front (a fixed arena or memory pool), latency-critical paths that cannot
 * afford cudaMalloc's implicit device synchronisation, or callers linked
 * into a process whose allocator must not be touched.  It calls no cudaMalloc,
 * cudaFree or other allocating routine; the caller still passes every input
 * and output (src, rcv, T_hi, T_lo, J as in spider_tt_pairs, all device
 * pointers) and the network as host arrays (net->W, net->b, checked for
 * finite values during the call and copied to the device by copies queued on
 * `stream`: pageable host arrays may be reused once the call returns,
 * page-locked ones must stay unchanged until the stream has passed the call).
 * What the kernel needs besides them -- the weights in the layouts it
 * reads, per-CTA slots for silu'(z) between the forward and the reverse sweep,
 * and the (hi, lo) staging of T -- lives in one fixed-size array of static
 * device memory (about 40 MB), which every GPU that loads this library holds
 * until the process exits.  Limits: net->kind == SPIDER_TT_MLP,
 * H in {32, 64, 128, 256}, 0 <= P <= 2^20; anything else returns
 * SPIDER_E_UNSUPPORTED or SPIDER_E_INVAL and spider_last_error(NULL) names the
 * limit.  The first call on a device looks up the array's device address
 * (once per device, with that device current) and keeps it; make that first
 * call before any stream capture, and do not call cudaDeviceReset while the
 * library is loaded.  All calls share the array and it keeps the last call's
 * contents; the kernel writes every word it reads within the same call, so
 * nothing needs clearing, but calls that overlap on the GPU (other streams,
 * other host threads) race on it and must be serialised by the caller.
 * Asynchronous on `stream` (a cudaStream_t or NULL). */
int spider_tt_pairs_noalloc(const spider_net *net, int64_t P, const float *src, const float *rcv,
                            float *T_hi, float *T_lo, float *J, void *stream);

/* Philox4x32-10 words computed on the device (host output, synchronous):
 * out[4 m + a] = word a of Philox(counter (c0 + m, c1, c2, c3), key = seed),
 * m in [0, n).  Exposed so the noise stream can be checked word for word. */
int spider_philox_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                        int64_t n, uint32_t *out);

#ifdef __cplusplus
}
#endif
#endif /* SPIDER_H */
