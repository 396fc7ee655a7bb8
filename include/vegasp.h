/*
 * vegasp.h -- C-ABI of libvegasp: the data-parallel hot path of vegas+
 * (G. P. Lepage, "Adaptive Multidimensional Integration: vegas Enhanced",
 * arXiv:2009.05112) on one NVIDIA GB300 (sm_103a).
 *
 * One adaptive iteration of vegas+ is
 *   vp_iterate: draw n_h samples in every stratification hypercube h (§3),
 *               map them through the per-axis vegas map x(y) and its Jacobian
 *               J(y) (§2.2 Eqs. y, jac; §2.4 Eq. y-Dspace), evaluate the
 *               integrand, accumulate the per-hypercube sums of J f and (J f)^2
 *               (§3 step 2), the per-axis increment histograms behind d_i
 *               (§2.3, §2.4) and the iteration's estimate I_j, sigma_j^2
 *               (§3 Eq. sumI);
 *   vp_adapt:   reallocate samples n_h = max(2, N_ev d_h / sum d), d_h =
 *               sigma_h^beta (§3 steps 2-4, Eqs. dh, nh) and refine every
 *               axis's grid (§2.3: smoothing, compression with alpha, the
 *               equal-share re-gridding), both from the same iteration's data
 *               (§3, last paragraph of the algorithm).
 *   vp_result:  combine iterations: weighted mean, its error, chi^2 (§2.5).
 *
 * The integral is I = int_a^b d^D x f(x) over a box (§2.1 Eq. Iy, §2.4).
 *
 * Conventions for every entry point:
 *  - Host pointers are read during the call only; the library copies what it
 *    keeps.  Device memory owned by a context is allocated when the context is
 *    created (through the allocator installed with vp_set_allocator, else
 *    cudaMallocAsync on the given stream) and released by the destroy call.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued asynchronously on it; calls that return data to the host
 *    synchronise that stream first.
 *  - Every call returns a vp_status.  On an error the context is unchanged
 *    (except after VP_ECUDA, which leaves the CUDA context as the runtime left
 *    it) and vp_last_error() describes it.  No exception crosses the ABI.
 *  - Contexts are not thread-safe: one host thread at a time per context.
 *  - The library runs on the current CUDA device; a context must be used on
 *    the device it was created on.
 */
#ifndef VEGASP_H
#define VEGASP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VP_OK = 0,
    VP_EINVAL = 1,      /* bad argument or size beyond a stated limit */
    VP_ENOMEM = 2,      /* device or host allocation failed */
    VP_ECUDA = 3,       /* a CUDA runtime call failed */
    VP_ETIMEOUT = 4,    /* a bounded host wait gave up */
    VP_ENONFINITE = 5,  /* the integrand produced NaN/Inf (flag read by vp_result) */
    VP_EBUSY = 6        /* no free slot / resource (server admission) */
} vp_status;

typedef enum { VP_FP64 = 0, VP_FP32 = 1 } vp_precision;

/* Integrand families (the paper's example shapes).  Parameter blobs are
 * arrays of doubles:
 *  VP_GAUSS     [K, {a_k, w_k, c_k[D]} x K]  f = sum_k a_k exp(-|x-c_k|^2/w_k^2)
 *               (§2.4 Eq. easy; w = 0.1 is the paper's coefficient 100)
 *  VP_BALL      [K, {a_k, r_k, c_k[D]} x K]  f = sum_k a_k Theta(|x-c_k| < r_k)
 *               (§2.4 Eq. balls; §1 footnote: the 20-D ball)
 *  VP_EXPNORM   [K, {a_k, s_k, c_k[D]} x K]  f = sum_k a_k exp(-s_k |x-c_k|)
 *               (§3.1 Eq. exponentials)
 *  VP_POSTERIOR [n, P, G, sigma_y, pw, log_ref, y[n], A[n][P]], D = P + G,
 *               x = (c_0..c_{P-1}, w_0..w_{G-1}), r_i = y_i - sum_m A[i][m] c_m,
 *               point i weighted by w = w_{i mod G},
 *               f = exp(sum_i log[(1-w) N(r_i; sigma_y) + w N(r_i; 10 sigma_y)]
 *                       - sum_m c_m^2/(2 pw^2) - log_ref)
 *               (App. B Eqs. posterior, prior with Gaussian priors; G = 1 is
 *               its 3-parameter fit, one weight per point its 21-parameter one).
 * Limits: K <= 64; POSTERIOR n <= 256. */
enum { VP_GAUSS = 0, VP_BALL = 1, VP_EXPNORM = 2, VP_POSTERIOR = 3 };

typedef struct {
    int kind;            /* VP_GAUSS ... VP_POSTERIOR */
    int n_param;         /* number of doubles in param */
    const double *param; /* blob as above; copied */
} vp_integrand;

typedef struct {
    int dim;            /* D, 1..24 */
    const double *lo;   /* [D] lower box edges a (§2.2: x_0 = a); copied */
    const double *hi;   /* [D] upper box edges b (x_{N_g} = b), hi > lo; copied */
    int n_g;            /* N_g increments per axis (§2.2), 1..4096 */
    int64_t n_ev;       /* N_ev samples per iteration (§3), >= 2 */
    double alpha;       /* grid compression exponent (§2.3), >= 0; 0 freezes the grid */
    double beta;        /* allocation damping exponent (§3 Eq. dh), >= 0 */
    uint64_t seed;      /* Philox key */
    uint32_t integral_id; /* Philox counter word 3: distinguishes integrals sharing a seed */
    int precision;      /* VP_FP64: map, integrand and moments in FP64.
                           VP_FP32: map and integrand in FP32, per-hypercube moments
                           Kahan-compensated FP32, flushed to FP64; d_h = sigma_h^beta
                           from the FP64 variance through FP32 log2/exp2 (relative
                           error ~1e-6); the estimate, the sums over hypercubes,
                           the reallocation quotient and the refinement stay FP64. */
    int plus2;          /* 0: n_h = max(2, N_ev d_h/sum d); 1: N_ev d_h/sum d + 2 (§3 Eq. nh) */
    int n_st;           /* 0: N_st = floor((N_ev/4)^(1/D)) (§3 Eq. Nst_vegasp),
                           computed exactly; > 0: use this many strata per axis */
    int max_it;         /* capacity of the iteration history (0 = 1024) */
    /* Strata per axis (§3.2, "Limitations and a Variation").  Hypercube h is
       the mixed-radix number whose digit on axis mu (axis 0 least significant)
       is its stratum there.  Accepted everywhere (contexts, batches, served
       requests); a single FP32 integral with more than 8 peaks whose D is 4,
       8, 12, 16, 20 or 24 and whose strata differ is refused (VP_EINVAL). */
    const int32_t *n_st_axis; /* NULL, or [D] strata per axis, each >= 1 (copied);
                                 overrides n_st and mixed */
    int mixed;          /* with n_st == 0 and n_st_axis == NULL: 1 = §3.2's mixed
                           rule, N_st + 1 strata on the first d axes and N_st on
                           the rest, N_st from Eq. Nst_vegasp and d the largest
                           with 4 (N_st + 1)^d N_st^(D - d) <= N_ev; 0 = uniform */
    /* Several integrals from the same samples (App. B): besides f itself (output
       0, which alone drives the adaptation), n_extra outputs f(x) x^a x^b,
       (a, b) = out_mono[2k], out_mono[2k + 1] for k < n_extra, each in
       -1..D-1 (-1: that factor is 1): the means and second moments of the
       paper's Bayesian example.  Every iteration then also records the
       estimates of all M = n_extra + 1 outputs and their covariance, summed
       over hypercubes (§2.1 Eq. sigest in several variables).  FP64 only, at
       most 2^22 hypercubes, n_extra <= 7; contexts and batches (in a batch
       such an integral is sampled by a launch of its own), not served
       requests. */
    int n_extra;
    const int32_t *out_mono; /* [2 n_extra] (copied) */
    int d_weighted;     /* the grid's d_i^mu (§2.3, §2.4): 0 = the mean of (J f)^2 over
                           the samples in the increment (the paper's form); 1 = the sum
                           of (J f)^2 / n_h, each sample weighted by its hypercube's
                           y-volume per sample (Omega_h / n_h, the common Omega dropped
                           since d is normalised), an estimate of the slab integral of
                           J^2 f^2 whatever the allocation (§3: the optimal map does not
                           depend on it) */
    int nst_div;        /* the divisor of the strata rule when n_st == 0: 0 or 4 =
                           vegas+'s §3 Eq. Nst_vegasp, floor((N_ev/4)^(1/D)) (and the
                           mixed rule's 4 samples per hypercube); 2 = classic vegas's
                           §3 Eq. Nst, floor((N_ev/2)^(1/D)), which with beta = 0 is
                           classic vegas's stratified sampling (§3: n_ev =
                           floor(N_ev/N_st^D) >= 2 samples per hypercube) */
} vp_params;

typedef struct {
    double mean;    /* weighted mean over iterations j >= discard (§2.5) */
    double sdev;    /* its standard error (§2.5) */
    double chi2;    /* sum_j (I_j - mean)^2 / sigma_j^2 (§2.5) */
    int dof;        /* n_it - 1 */
    int n_it;       /* iterations included */
    int64_t n_eval; /* integrand evaluations in all iterations so far */
    double last_i;  /* I_j of the latest iteration */
    double last_sdev; /* sigma_j of the latest iteration */
} vp_result_t;

typedef struct vp_ctx vp_ctx;

/* ---- allocator -------------------------------------------------------- */
/* Device memory for contexts comes from alloc/free when installed (e.g. a
 * framework's caching allocator), else from cudaMallocAsync/cudaFreeAsync.
 * alloc returns NULL on failure.  Pass NULLs to restore the default.  Applies
 * to contexts created afterwards; each context frees with the allocator it
 * was created with. */
typedef void *(*vp_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*vp_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
vp_status vp_set_allocator(vp_alloc_fn alloc, vp_free_fn free_fn, void *user);

/* ---- the four calls of the method --------------------------------------- */

/* Creates a context for one integral: validates the parameters (VP_EINVAL on
 * D outside 1..24, N_g outside 1..4096, N_ev < 2, lo >= hi, alpha/beta < 0 or
 * not finite, a malformed blob, N_st^D > 2^31, or (N_ev + 2 N_h) ceil(D/4) >=
 * 2^32 (the Philox counter word 0)), computes N_st, allocates every device
 * buffer, starts from a uniform grid (§2.3) and the equal split n_h =
 * max(2, floor(N_ev / N_h)).  *out receives the context. */
vp_status vp_map_create(const vp_params *params, const vp_integrand *f, void *stream,
                        vp_ctx **out);

/* One iteration's sampling, moments, histograms and estimate (steps a1-a6),
 * enqueued on stream.  Iteration t uses Philox counters (j ceil(D/4) + q, h, t,
 * integral_id) with key (seed_lo, seed_hi). */
vp_status vp_iterate(vp_ctx *ctx, void *stream);

/* Reallocation (a7) then grid refinement (a8, skipped when alpha == 0), from
 * the data of the latest vp_iterate. */
vp_status vp_adapt(vp_ctx *ctx, void *stream);

/* vp_iterate + vp_adapt replayed from a CUDA graph captured on first use. */
vp_status vp_step(vp_ctx *ctx, void *stream);
/* A step (as vp_step) that also reads the estimates back without waiting for
 * them: enqueues the step on `stream`, then an asynchronous copy of its I_j
 * and sigma_j^2 into pinned host memory the context owns, then waits for the
 * copy made by the previous vp_step_read call (its step finished while this
 * one was being enqueued) and returns those values in *i_j, *var_j with
 * *have = 1; *have = 0 on the first call (or the first after
 * vp_step_read_flush).  vp_step_read_flush waits for the last call's copy
 * and returns it the same way (*have = 0 if none is pending).  The
 * estimates are those vp_get_history records (§2.5's I_j, sigma_j^2). */
vp_status vp_step_read(vp_ctx *ctx, void *stream, int *have, double *i_j, double *var_j);
vp_status vp_step_read_flush(vp_ctx *ctx, int *have, double *i_j, double *var_j);

/* ---- one integral over several devices ---------------------------------- */
/* vegas+ shards by samples (§1: the method parallelises easily; §3 Eq. sumI
 * and the d_i of §2.3/§2.4 are sums over all samples).  Every rank creates a
 * context with the same parameters; per iteration each rank
 *   vp_iterate_part(ctx, rank, n_ranks, stream)   steps a1-a5 over samples
 *        [T rank / n_ranks, T (rank + 1) / n_ranks) of the T samples the
 *        current allocation draws (contiguous in the offsets, equal in
 *        samples), adding to the iteration's partial sums;
 *   vp_partials_export(ctx, buf, stream)   packs those sums into buf, a DEVICE
 *        vector of vp_partials_size doubles: [S1_h, S2_h (N_h each) | hsum,
 *        hcnt (D N_g each, counts as doubles)];
 *   (the caller sums buf over the ranks, e.g. an NCCL all-reduce in place)
 *   vp_partials_import(ctx, buf, stream)   replaces the sums by the total;
 *   vp_estimate(ctx, stream)   step a6 (and sigma_h, d_h) from them, recorded
 *        as the iteration (what vp_iterate does after its sampling);
 *   vp_adapt(ctx, stream)      as usual.
 * Identical sums give identical estimates, allocations and grids on every
 * rank.  FP32 peak families with more than 8 peaks, and contexts with extra
 * outputs, are refused (VP_EINVAL).  vp_iterate_part may be called for
 * several parts on one context (they add up).  Buffers are the caller's;
 * nothing is allocated. */
vp_status vp_iterate_part(vp_ctx *ctx, int part, int n_parts, void *stream);
vp_status vp_partials_size(vp_ctx *ctx, int64_t *n);
vp_status vp_partials_export(vp_ctx *ctx, double *buf, void *stream);
vp_status vp_partials_import(vp_ctx *ctx, const double *buf, void *stream);
vp_status vp_estimate(vp_ctx *ctx, void *stream);

/* Synchronises the context's stream, reads the iteration history and
 * combines iterations j >= discard (§2.5).  VP_ENONFINITE if any iteration saw
 * a non-finite integrand value (out still filled). */
vp_status vp_result(vp_ctx *ctx, int discard, vp_result_t *out);
/* §2.5, last paragraph: the unweighted combination for iterations run with a
 * frozen map (alpha = 0, see vp_set_damping) after the first `discard`:
 * mean = average of the I_j, sdev = average of the sigma_j / sqrt(N_it) (an
 * unbiased estimate, free of the weighted average's 1/N_ev bias); chi2 about
 * that mean (0 if some sigma_j is 0), dof = N_it - 1.  Same errors as
 * vp_result. */
vp_status vp_result_unweighted(vp_ctx *ctx, int discard, vp_result_t *out);
/* Changes the damping exponents for the following iterations: alpha (§2.3;
 * 0 freezes the grid, "preventing the algorithm from adapting", §2.5) and
 * beta (§3 Eq. dh; 0 gives the equal split), both finite and >= 0, else
 * VP_EINVAL with the context unchanged.  Synchronises the context's last
 * stream; the step graph is captured again when the refinement's presence
 * changes. */
vp_status vp_set_damping(vp_ctx *ctx, double alpha, double beta);

vp_status vp_map_destroy(vp_ctx *ctx);

/* Message of the latest failing call on this thread (never NULL). */
const char *vp_last_error(void);

/* ---- inspection and test hooks (host buffers; each synchronises) ------- */
/* n_st: the smallest strata count over the axes (N_st when uniform) */
vp_status vp_get_info(vp_ctx *ctx, int64_t *n_st, int64_t *n_hc, int *n_it);
/* strata[D]: the strata on every axis (§3.2) */
vp_status vp_get_strata(vp_ctx *ctx, int32_t *strata);
/* Several integrals (App. B), M = n_extra + 1 outputs.  vp_get_history_multi:
 * i_j[n][M] and cov_j[n][M][M] of the first n iterations.  vp_result_multi:
 * their combination over iterations j >= discard, the several-variable form
 * of §2.5's weighted average -- with W_j the pseudo-inverse of cov_j
 * (eigenvalues below 1e-12 of the largest dropped), mean = (sum W_j)^+
 * sum W_j I_j, cov = (sum W_j)^+, chi2 = sum_j (I_j - mean)^T W_j (I_j -
 * mean), dof = M (n_it - 1); if every W_j vanishes, the plain mean with cov 0.
 * mean[M], cov[M][M]; n_it may be NULL.  VP_EINVAL on a context without extra
 * outputs; VP_ENONFINITE as vp_result.  vp_get_moments_multi: the latest
 * iteration's per-hypercube sums x1[N_h][M] = sum J f g_k and x2[N_h][M (M +
 * 1)/2] = sum J^2 f^2 g_k g_l (k <= l, rows of the upper triangle). */
vp_status vp_get_history_multi(vp_ctx *ctx, int n, double *i_j, double *cov_j);
vp_status vp_result_multi(vp_ctx *ctx, int discard, double *mean, double *cov, double *chi2,
                          int *dof, int *n_it);
vp_status vp_get_moments_multi(vp_ctx *ctx, double *x1, double *x2);

/* §4.2 (preconditioned integrators): trains the vegas map on sample data
 * {x, f(x)} given before integrating.  n_iter times: every axis's histogram
 * over the data of J^2(y(x)) f^2(x) per increment, y(x) the inverse of the
 * current map (§4.2's d_i^mu, the sum over the data and n_i^mu the data points
 * in the increment), then the refinement of §2.3 with the context's alpha
 * (alpha = 0 changes nothing); the same data every time.  x[n][D] (host,
 * copied; every point inside the box, else VP_EINVAL), f[n] (host, copied;
 * finite) or NULL: the context's integrand evaluated at x in FP64.  The
 * allocation, the iteration history and the Philox counters are untouched;
 * setting alpha to 0 with vp_set_damping afterwards keeps the trained map
 * (§4.2).  Synchronises `stream`. */
vp_status vp_precondition(vp_ctx *ctx, int64_t n, const double *x, const double *f, int n_iter,
                          void *stream);

/* Checkpoint / resume.  The state of a context between iterations -- the FP64
 * grid, the allocation n_h and its offsets, the iteration count t (Philox
 * counter word 2), the scale of the FP32 path, the running totals and the
 * iteration history (and that of the extra outputs) -- as a byte blob, host
 * memory.  vp_export_state: *size receives the blob's size; with buf non-NULL
 * and cap >= *size the blob is written (else VP_EINVAL); synchronises the
 * context's last stream.  vp_import_state: into a context created with the
 * same parameters (dimension, N_g, N_ev, strata, seed, integral_id, integrand
 * kind, precision, outputs, history capacity; else VP_EINVAL, the context
 * unchanged), which then continues as the exporting one would: the samples
 * are counter-based, so the following iterations draw the same points and
 * agree with the uninterrupted run to FP rounding of the reductions. */
vp_status vp_export_state(vp_ctx *ctx, void *buf, size_t cap, size_t *size);
vp_status vp_import_state(vp_ctx *ctx, const void *buf, size_t size);
/* edges[D][N_g + 1] (FP64 master grid) */
vp_status vp_get_edges(vp_ctx *ctx, double *edges);
/* replaces the grid (edges[D][N_g+1], strictly increasing, ends = box) */
vp_status vp_set_edges(vp_ctx *ctx, const double *edges);
/* n_h[N_h] and offsets[N_h + 1] of the current allocation */
vp_status vp_get_alloc(vp_ctx *ctx, uint32_t *n_h, uint64_t *offsets);
/* per-hypercube sums S1_h = sum J f, S2_h = sum (J f)^2 of the latest iteration */
vp_status vp_get_moments(vp_ctx *ctx, double *s1, double *s2);
/* histograms hsum[D][N_g] = sum (J f)^2 and hcnt[D][N_g] = sample counts */
vp_status vp_get_hist(vp_ctx *ctx, double *hsum, double *hcnt);
/* I_j and sigma_j^2 of the first n iterations */
vp_status vp_get_history(vp_ctx *ctx, int n, double *i_j, double *var_j);
/* d_h[N_h] = sigma_h^beta (§3 Eq. dh) as the latest estimate (vp_iterate) or
 * vp_alloc_from_sigma / vp_alloc_from_dh left it, and *sum_d = their sum in
 * the library's fixed order (either pointer may be NULL).  On the FP64 path
 * and from a given sigma_h, beta = 1/2 and 3/4 are correctly rounded square
 * roots (sqrt(sigma), sqrt(sigma sqrt(sigma))), other beta pow; the FP32
 * path's estimate forms d_h from the variance with the FP32 log2 / exp2
 * units (relative error below 1e-6). */
vp_status vp_get_dh(vp_ctx *ctx, double *d_h, double *sum_d);
/* Reallocation (a7) from given d_h[N_h] (skips sigma_h and the damping) or
 * from given sigma_h[N_h] (applies d_h = sigma_h^beta); sets n_h and offsets. */
vp_status vp_alloc_from_dh(vp_ctx *ctx, const double *d_h, void *stream);
vp_status vp_alloc_from_sigma(vp_ctx *ctx, const double *sigma_h, void *stream);
/* Grid refinement (a8) from given histograms hsum/hcnt[D][N_g]. */
vp_status vp_refine_from_hist(vp_ctx *ctx, const double *hsum, const double *hcnt,
                              void *stream);
/* Evaluates n samples (h[k], j[k]) of iteration t with the sampling kernel's
 * own device code: x[n][D], idx[n][D] (increment indices), jac[n], f[n]. */
vp_status vp_eval_samples(vp_ctx *ctx, int64_t n, const uint64_t *h, const uint32_t *j,
                          uint32_t t, double *x, int32_t *idx, double *jac, double *f);
/* Device-side timing of the latest sampling launch made by vp_iterate, in ms
 * (CUDA events on the launching stream; the step graph of vp_step carries no
 * events); -1 if none recorded. */
vp_status vp_last_sample_ms(vp_ctx *ctx, float *ms);
/* Launch shape of the sampling kernel chosen by the autotuner (which runs at
 * the first vp_iterate/vp_step): scheme 0 = the one-integral kernel, its
 * samples split evenly over its warps, with clusters of `cluster` CTAs;
 * 1 = dynamic tasks with `run` samples per thread per chunk; 2 = the
 * one-integral kernel with half of its samples split evenly over its warps
 * and the other half pulled by the warps as they finish, in chunks of 32 x
 * `run` samples (sample costs differ with the allocation and the integrand);
 * `blocks` CTAs of `threads` threads. */
vp_status vp_get_tuning(vp_ctx *ctx, int *scheme, int *blocks, int *threads, int *cluster,
                        int *run);
/* Fixes the sampling kernel's launch shape instead of letting the autotuner
 * choose it (reproducible timing and profiling; no counterpart in the paper,
 * the shape does not change any result beyond FP summation order).
 * Arguments as in vp_get_tuning: schemes 0 and 2 require all `blocks` CTAs of
 * `threads` (256, 512, 768 or 1024, within the kernel's limit) resident at once, in
 * clusters of `cluster` (1, 2, 4, 8; > 1 only with shared-memory histograms);
 * scheme 1 takes threads = 256 and cluster = 1; run in 1..64.  Synchronises
 * the context's last stream; a step graph captured before is rebuilt at the
 * next vp_step.  VP_EINVAL (context unchanged) for shapes that cannot run. */
vp_status vp_set_tuning(vp_ctx *ctx, int scheme, int blocks, int threads, int cluster, int run);

/* ---- batches: many independent integrals per launch ----------------------- */
/* A batch iterates n independent integrals together (each with its own box,
 * integrand, N_ev, N_g, alpha, beta, seed and integral_id; validated as in
 * vp_map_create).  Every iteration of the batch runs one persistent sampling
 * launch per (integrand kind, precision) over a queue of (integral, sample
 * range) tasks, largest integrals first, then the per-hypercube and per-axis
 * kernels over all integrals at once; vp_batch_step replays the iteration and
 * adaptation of every integral from one CUDA graph.  Results are per integral,
 * identical in meaning to vp_result.  n: 1..1048576. */
typedef struct vp_batch vp_batch;
vp_status vp_batch_create(int n, const vp_params *params, const vp_integrand *f, void *stream,
                          vp_batch **out);
vp_status vp_batch_iterate(vp_batch *b, void *stream);
vp_status vp_batch_adapt(vp_batch *b, void *stream);
vp_status vp_batch_step(vp_batch *b, void *stream);
/* integral i (0-based) */
vp_status vp_batch_result(vp_batch *b, int i, int discard, vp_result_t *out);
/* all n results into out[n] (one synchronisation); the first non-OK status */
vp_status vp_batch_results(vp_batch *b, int discard, vp_result_t *out);
vp_status vp_batch_size(vp_batch *b, int *n);
/* I_j and sigma_j^2 of the first n iterations of integral i */
vp_status vp_batch_history(vp_batch *b, int i, int n, double *i_j, double *var_j);
/* Integral i's several outputs (App. B), as vp_result_multi and
 * vp_get_history_multi; VP_EINVAL for an integral without extra outputs or
 * an index out of range. */
vp_status vp_batch_result_multi(vp_batch *b, int i, int discard, double *mean, double *cov,
                                double *chi2, int *dof, int *n_it);
vp_status vp_batch_history_multi(vp_batch *b, int i, int n, double *i_j, double *cov_j);
vp_status vp_batch_destroy(vp_batch *b);

/* ---- serving: a stream of integration requests ------------------------------ */
/* A server iterates requests that arrive over time.  Each request is one
 * integral with a target relative error; the server runs the adaptive
 * iterations of §2 and §3 for every admitted request together -- one iteration
 * of all of them per server step, through the batched kernels above -- and
 * retires each one when the combination (§2.5) of its iterations j >= discard
 * has sdev <= rtol |mean| (after at least min_meas of them), or when it has
 * run p.max_it iterations.  A request's grid, allocation and accumulators stay
 * on the device from admission to retirement; a request's samples do not
 * depend on which other requests share its steps (its Philox counters carry
 * its own seed, integral_id and iteration count).
 * Admission is by device memory: the server reserves mem_budget bytes at
 * creation and admits queued requests, first come first served, while their
 * state fits in what is left (and fewer than max_active are running).
 * The paper serves one integral at a time; the server, its admission and the
 * stop rule's form are this library's. */
typedef struct {
    int64_t mem_budget; /* device bytes for request state; 0 = 256 MiB */
    int max_active;     /* requests iterated together, 1..65536; 0 = 4096 */
} vp_server_config;

typedef struct {
    vp_params p;        /* as for vp_map_create; p.max_it (> discard) caps the
                           iterations (0 = 1024) */
    vp_integrand f;     /* copied at submission */
    double rtol;        /* target relative error, > 0 */
    int discard;        /* warm-up iterations left out of the result, >= 0 */
    int min_meas;       /* least iterations in the result before the test, >= 1 */
    uint64_t tag;       /* caller's label, returned with the result */
} vp_request;

typedef struct {
    uint64_t id;        /* from vp_server_submit */
    uint64_t tag;
    vp_status status;   /* VP_OK, or VP_ENONFINITE (non-finite integrand value) */
    int converged;      /* 1: sdev <= rtol |mean|; 0: stopped at p.max_it */
    int n_iter;         /* iterations run */
    vp_result_t r;      /* combination of iterations j >= discard (§2.5) */
    double t_submit, t_admit, t_done; /* seconds on the steady clock (vp_server_clock) */
} vp_served;

typedef struct {
    int64_t submitted, finished, queued, active;
    int64_t steps;           /* server steps run */
    int64_t bytes_in_use, bytes_peak, mem_budget;
    int64_t n_eval;          /* integrand evaluations of all finished requests */
    double busy_s;           /* wall time spent in steps */
} vp_server_stats;

typedef struct vp_server vp_server;

/* Creates a server on the current device; its work runs on stream (NULL = a
 * stream of its own).  VP_ENOMEM if the budget cannot be reserved. */
vp_status vp_server_create(const vp_server_config *cfg, void *stream, vp_server **out);
/* Queues a request (thread-safe; copies everything).  VP_EINVAL as for
 * vp_map_create or for rtol/discard/min_meas/max_it out of range; VP_ENOMEM if
 * the request's state alone exceeds the budget.  *id (may be NULL) receives
 * its number, 0, 1, 2, ... in submission order. */
vp_status vp_server_submit(vp_server *s, const vp_request *req, uint64_t *id);
/* One server step on the calling thread: retire nothing new, admit what fits,
 * run one iteration + adaptation of every admitted request, then retire the
 * finished ones.  *n_active (may be NULL) receives the requests still running.
 * VP_EINVAL while the server's own worker thread runs. */
vp_status vp_server_step(vp_server *s, int *n_active);
/* Starts / stops a worker thread that runs steps while requests are queued or
 * running and sleeps otherwise.  Stopping waits for the current step. */
vp_status vp_server_start(vp_server *s);
vp_status vp_server_stop(vp_server *s);
/* Moves up to max finished requests, in the order they finished, into out;
 * *n receives how many.  If the worker failed, its error is returned. */
vp_status vp_server_poll(vp_server *s, int max, vp_served *out, int *n);
/* Blocks until `finished` requests have finished in all or timeout_s passes
 * (VP_ETIMEOUT then). */
vp_status vp_server_wait(vp_server *s, int64_t finished, double timeout_s);
vp_status vp_server_get_stats(vp_server *s, vp_server_stats *out);
/* The server's clock: seconds on the steady clock. */
double vp_server_clock(void);
/* Stops the worker and frees everything; unfinished requests are dropped. */
vp_status vp_server_destroy(vp_server *s);

/* ---- reallocation without device allocation --------------------------- */
/* vp_alloc_static: the reallocation step of vp_adapt (the fixed-order sum of
 * d_h, n_h = max(2, floor(N_ev d_h / sum d)) -- or floor(.) + 2 when plus2 is
 * set -- and the exclusive offsets) on buffers the caller provides, allocating
 * nothing.  The paper has no counterpart: this entry point is for callers that
 * cannot allocate device memory while they work, such as a serving process that
 * reserved all device memory up front for a pool it manages itself, or code
 * that must not call cudaMalloc mid-step because cudaMalloc can synchronise the
 * device.
 *   d_h      [n_hc] DEVICE doubles, finite and >= 0 (read)
 *   n_h      [n_hc] DEVICE uint32 (written)
 *   offsets  [n_hc + 1] DEVICE uint64 (written; offsets[n_hc] = sum of n_h)
 *   n_hc     1 .. 4,194,304 (VP_EINVAL beyond: the scratch holds 4096 blocks of
 *            1024 hypercubes); n_ev 2 .. 4,294,967,293 (every n_h, at most
 *            n_ev + 2, is a 32-bit integer)
 * Work is enqueued on stream; nothing is allocated and nothing is freed.  Its
 * scratch is one static device array of about 64 KB, which every GPU that loads
 * the library holds until the process exits.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call on a
 * device shares the array and leaves the last call's contents in it: calls
 * whose work overlaps on the GPU (other streams, other host threads) race, so
 * the caller must order them.  If the sum of d_h is not finite, n_h and offsets
 * are left unchanged.  VP_EINVAL: NULL buffer or size out of range; VP_ECUDA: a
 * launch failed. */
vp_status vp_alloc_static(const double *d_h, int64_t n_hc, int64_t n_ev, int plus2,
                          uint32_t *n_h, uint64_t *offsets, void *stream);

/* Measures the device's throughput of shared-memory atomic adds in the access
 * pattern of the sampling kernel's histograms (§2.3 d_i: one count per axis per
 * sample, and one FP32 sum per axis per sample where J f is nonzero): every
 * thread of one 768-thread CTA per SM adds to one random increment on each of
 * 20 axes of 1000 increments, 256 times.  f32 = 0: 32-bit integer adds (the
 * counts); f32 = 1: FP32 adds (the sums).  *per_s = adds per second, the best
 * of three timed launches after one warm-up (CUDA events on the legacy default
 * stream, which the call synchronises).  A measurement aid, not a step of the
 * method: the bench reports the sampling kernel against this bound.  Uses the
 * current device; allocates 4 bytes of device memory for the duration of the
 * call.  VP_EINVAL: NULL out; VP_ECUDA: a launch failed. */
vp_status vp_shared_atomic_rate(int f32, double *per_s);

#ifdef __cplusplus
}
#endif
#endif /* VEGASP_H */
