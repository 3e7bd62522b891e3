/*
 * fermi.h -- C ABI of the GB300 dense Chebyshev Fermi-operator solver.
 *
 * Computes the density matrix P = f(H) = [I + exp((H - mu I)/kT)]^{-1} of a dense real
 * symmetric Hamiltonian as a Chebyshev expansion sum_n c_n T_n(X) evaluated with Liang's
 * baby-step / giant-step scheme (arXiv 2306.12616, Sec. "Chebyshev expansions with
 * O(sqrt L) number of matrix multiplications", Eq. (fermi), Eq. (ansatz)), so that the
 * number of matrix products grows with the square root of the number of terms. The
 * chemical potential mu is either given or fixed by tr(P) = N_e.
 *
 * Conventions shared by every call:
 *  - Matrices are dense, row-major, float64, with a leading dimension ld >= n (elements).
 *    H must be symmetric; only then is P = f(H) well defined. Pointers prefixed "d" are
 *    device pointers on the context's device, prefixed "h" host pointers.
 *  - The caller owns H, P and every output buffer. The context owns its workspace
 *    (device scratch grown on demand and reused), which is freed by fo_destroy.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream). All
 *    device work is enqueued on it; a call only blocks when it must return host values
 *    (documented per call).
 *  - No call throws. Every call returns an fo_status; CUDA failures map to FO_ERR_CUDA
 *    and the message is kept in the context (fo_last_error).
 *  - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef FERMI_GB300_H
#define FERMI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fo_ctx fo_ctx;

typedef enum {
    FO_OK = 0,
    FO_ERR_ARG = 1,              /* invalid argument (size, pointer, parameter) */
    FO_ERR_CUDA = 2,             /* a CUDA runtime/driver call failed */
    FO_ERR_NOMEM = 3,            /* device workspace allocation failed */
    FO_ERR_NONFINITE = 4,        /* H holds NaN or Inf (found by the bounds pass) */
    FO_ERR_NO_BRACKET = 5,       /* mu bisection could not bracket tr(P) = N_e */
    FO_ERR_NOT_CONVERGED = 6,    /* mu bisection hit its iteration cap */
    FO_ERR_DEVICE_TIMEOUT = 7,   /* a bounded device-side wait gave up */
    FO_ERR_UNSUPPORTED = 8       /* feature not available for these arguments */
} fo_status;

/* Arithmetic of the matrix products. FP64 runs everything in float64. The split forms
 * keep float32 master copies of every matrix and run each product on the tensor cores
 * as a sum of products of 16-bit planes with float32 accumulation:
 *   BF16X3: A = a0 + a1 + a2 (bf16 planes), AB ~ sum_{i+j<=2} a_i b_j  (6 products)
 *   FP16X2: A = a0 + a1 (fp16 planes),      AB ~ a0 b0 + a0 b1 + a1 b0 (3 products)
 *   BF16X1: A = a0,                          AB ~ a0 b0                 (1 product)
 * Bounds, coefficients, traces, moments and the mu search stay float64 in all modes. */
typedef enum {
    FO_PREC_FP64 = 0,
    FO_PREC_BF16X3 = 1,
    FO_PREC_FP16X2 = 2,
    FO_PREC_BF16X1 = 3
} fo_precision;

typedef enum {
    FO_MU_FIXED = 0,    /* use params.mu */
    FO_MU_BISECT = 1,   /* bisection on sum_n c_n(mu) tau_n = N_e with exact moments */
    FO_MU_LEARNED = 2,  /* MLP proposal, verified on the trace; bisection as fallback */
    FO_MU_ORDER = 3     /* MLP proposal of each instance's expansion order: the expansion is cut
                           at the proposed order (x 1.25, rounded up to whole giant steps, at
                           most n_terms), products it makes zero or unused are skipped, and mu
                           is the bisection's on the exact moments of that expansion (started
                           at the MLP's mu). fo_result.order = the coefficients used, m = the
                           giant steps used, n_gemm = the instance's products */
} fo_mu_mode;

/* Flags (fo_params.flags). */
#define FO_FLAG_TRACE_ONLY_DIAG  0x1u  /* reserved */
#define FO_FLAG_NO_RESULT_SYNC   0x2u  /* density-matrix calls: never block, leave fo_result untouched */
#define FO_FLAG_GRAPH            0x4u  /* capture the call's kernels into a CUDA graph kept with its
                                          plan and replay it on later calls with the same plan */
#define FO_FLAG_POWER_BASIS      0x10u /* evaluate the paper's literal form: power-basis
                                          coefficients d_{i,j} (Eq. (formula for d0), (formula
                                          for d)) and the nested Horner scheme Y = S_j + T_k Y of
                                          Eq. (ansatz), instead of the Chebyshev-basis
                                          coefficients and the Clenshaw recurrence. The d_{i,j}
                                          grow like 2^j, so the result loses accuracy with m;
                                          FP16X2 is rejected (overflow) */
#define FO_FLAG_NO_TRACE_FIX     0x20u /* split forms with mu searched: return P as the expansion
                                          produced it, without the trace correction (see
                                          fo_density_matrix); for measuring what it changes */
#define FO_FLAG_ALLOW_LOOSE      0x40u /* split precisions: run the combinations whose error is
                                          measured above the 1e-6 bar of the split forms
                                          (FO_FLAG_STAGED, FO_FLAG_POWER_BASIS, and a forced k
                                          with m > k: the longer Clenshaw chain, ~1.4e-6 at
                                          m = 50); without this flag they fail with
                                          FO_ERR_UNSUPPORTED */
#define FO_FLAG_STAGED           0x8u  /* baby and giant steps in the staged form of Algorithm 1
                                          (Sec. "Speed up with multiple GPU streams"): the
                                          independent products of a stage in one launch, about
                                          log2 k launches instead of k - 1. Each doubling stage
                                          can amplify the error of its inputs by up to 4, so in
                                          the split forms the result is ~30x less accurate than
                                          with the default three-term recurrence (FP64 is
                                          unaffected at its 1e-10 bar) */

typedef struct {
    int32_t n_terms;          /* number of coefficients c_0..c_{n_terms-1}, >= 1 */
    int32_t k;                /* baby steps; 0 = ceil(sqrt(n_terms)); m = ceil(n_terms/k) */
    double  kT;               /* electronic temperature, same energy unit as H, > 0 */
    double  mu;               /* chemical potential for FO_MU_FIXED */
    int32_t precision;        /* fo_precision */
    int32_t mu_mode;          /* fo_mu_mode */
    int32_t use_given_bounds; /* 1: use emin/emax below instead of Gershgorin bounds */
    int32_t n_quad;           /* Chebyshev-Gauss nodes; 0 = max(2048, 4 n_terms) */
    double  emin, emax;       /* spectral bounds when use_given_bounds (emax > emin) */
    int32_t max_bisect;       /* bisection cap; 0 = 200 */
    uint32_t flags;           /* FO_FLAG_* */
    double  tr_tol;           /* FO_MU_LEARNED: accept the P evaluated at a proposed mu when its
                                 trace before the trace correction meets |tr P - N_e| <= tr_tol;
                                 0 = default: 1e-8 max(1, N_e) for FP64, 1e-7 n for the split
                                 forms (the band their float32 rounding of tr P lies in) */
    int32_t max_newton;       /* FO_MU_LEARNED: trace-corrected re-evaluations of P before the
                                 bisection fallback; 0 = 2, < 0 = none */
    int32_t tile_n;           /* tensor-core tile width: 0 = autotune per plan, or 128 / 256 */
    int32_t tile_ctas;        /* CTAs per SM of the product kernel: 0 = autotune, 1, or 2
                                 (2 only with 128-wide tiles); set together with tile_n;
                                 other values fail with FO_ERR_ARG */
    int32_t lanczos_steps;    /* 0: Gershgorin bounds. 1..64: tighter bounds from that many
                                 float64 Lanczos steps on H (start vector: splitmix64 draws),
                                 the extreme Ritz values widened by their residuals
                                 beta_{K+1} |y_K| and by 1% of the width, clamped to the
                                 Gershgorin interval. Not a guaranteed enclosure; ignored with
                                 use_given_bounds */
    int32_t tile_drain;       /* warps draining the tensor-memory accumulators: 0 = autotune,
                                 8, or 16 (with tile_n = 256); set together with tile_n;
                                 other values fail with FO_ERR_ARG */
    int32_t tile_store;       /* storage of the 16-bit operand planes of the split forms' matrix
                                 slots: 0 = chosen with the tile (autotuned with tile_n = 0,
                                 else 1); 1 = the full square (the symmetric products mirror
                                 each output tile); 2 = the 128 x 128 blocks on and above the
                                 diagonal only, a block below read by the tensor cores as the
                                 transpose of its counterpart above (MN-major operand tiles).
                                 Results are bit-identical; other values fail with FO_ERR_ARG */
    int32_t chain;            /* split forms: 0 = default (1), 1 = one launch per matrix product,
                                 2 = each chain of dependent products (the baby steps, the giant
                                 steps, the Clenshaw recurrence) as one launch whose tiles wait,
                                 per instance, for the previous step's tiles (bounded waits; a
                                 timeout fails the call with FO_ERR_DEVICE_TIMEOUT). Same bits */
    int32_t tile_persist;     /* split forms: 0 or 1 = one CTA per tile (default), 2 = the
                                 persistent product kernel (128-wide tiles, one CTA per SM walking
                                 the tiles; separate epilogue warps finish a tile while the next
                                 one's products run; with tile_n = 0 its two plane storages are
                                 autotuned). Same bits; measured slower than the default */
    int32_t chain_window;     /* chain launches: tiles run window by window, a window being
                                 consecutive instances (largest first) with at least this many
                                 tiles per step; 0 = one window (step by step over the batch) */
} fo_params;

typedef struct {
    double  mu;               /* chemical potential used for P */
    double  trace;            /* tr(P) of the returned P, float64 sum of its diagonal */
    double  trace_poly;       /* sum_n c_n(mu) tau_n from the moments (FO_MU_BISECT), else 0 */
    double  frob2;            /* ||P||_F^2 */
    double  emin, emax;       /* spectral bounds used */
    int32_t k, m;             /* baby / giant steps */
    int32_t n_gemm;           /* matrix products issued */
    int32_t bisect_iters;     /* bisection halvings (0 if not bisected) */
    int32_t learned_accepted; /* 1 if the learned mu was kept */
    int32_t status;           /* fo_status of the device-side stages */
    int32_t n_launches;       /* kernels of this library launched by the call (whole batch) */
    int32_t tile_n;           /* tensor-core tile width used (0 for FP64) */
    int32_t tile_ctas;        /* CTAs per SM of the product kernel used (0 for FP64) */
    int32_t evals;            /* evaluations of P (1 unless FO_MU_LEARNED corrected mu) */
    int32_t order;            /* expansion order proposed by the learned model (FO_MU_LEARNED) or
                                 the coefficients used (FO_MU_ORDER); 0 otherwise */
    int32_t tile_drain;       /* accumulator drain warps of the product kernel (0 for FP64) */
    int32_t tile_store;       /* operand plane storage used (1 or 2 as in fo_params; 0 for FP64) */
    double  trace_raw;        /* tr(P) as the expansion produced it, before the trace correction
                                 (equal to trace when none was applied) */
    double  trace_gamma;      /* gamma of the trace correction P + gamma (P - P^2) (0: none) */
    double  trace_proj;       /* float64 residual removed per diagonal entry by the trace
                                 projection after the correction (0: none) */
    int32_t tile_persist;     /* product kernel used: 2 persistent, 1 one CTA per tile, 0 FP64 */
} fo_result;

/* Stages of a density-matrix call, as recorded by the profiler. */
enum {
    FO_STAGE_BOUNDS = 0,      /* spectral bounds, scaling and plane split of X */
    FO_STAGE_PRODUCTS = 1,    /* matrix products (baby, giant and Clenshaw steps) */
    FO_STAGE_MOMENTS = 2,     /* traces and Frobenius products -> tau_n */
    FO_STAGE_MU = 3,          /* DOS weights and bisection */
    FO_STAGE_COEFFS = 4,      /* Chebyshev coefficients and giant-step coefficients */
    FO_STAGE_CONTRACT = 5,    /* R_l = sum_i g_{i,l} T_i */
    FO_STAGE_TRACE = 6,       /* tr P, ||P||_F^2 */
    FO_STAGE_CALL = 7,        /* the whole call */
    FO_PROFILE_STAGES = 8
};

/* Device-time profile accumulated over calls while profiling is enabled. Times come from
 * CUDA events recorded on the caller's stream around each stage (products: around each
 * launch). flops[FO_STAGE_PRODUCTS] is the algorithmic work of the products: a symmetric
 * product of n x n matrices needs n^2 (n+1) flops per split product (only the upper
 * triangle of the result is formed), times 6 / 3 / 1 split products for BF16X3 / FP16X2 /
 * BF16X1 and 1 for FP64. */
typedef struct {
    double  ms[FO_PROFILE_STAGES];
    double  flops[FO_PROFILE_STAGES];
    int64_t launches[FO_PROFILE_STAGES];
    int64_t calls;
} fo_profile;

/* Create a context on CUDA device `device`. *out is set on success. */
fo_status fo_create(fo_ctx **out, int device);
/* Free the context and its workspace (synchronises the device). NULL is accepted. */
fo_status fo_destroy(fo_ctx *ctx);
/* Message of the last failure in this context ("" if none). Owned by the context. */
const char *fo_last_error(const fo_ctx *ctx);
/* Static name of a status code. */
const char *fo_status_string(fo_status s);
/* Library version string, e.g. "fermi-gb300 0.1". */
const char *fo_version(void);

/*
 * Spectral bounds (Sec. "Chebyshev expansions": e_a, e_b enclose the spectrum).
 * Gershgorin discs: emin = min_i (h_ii - sum_{j!=i} |h_ij|), emax = max_i (h_ii + sum ...);
 * each row sum is formed exactly (128-bit integer fixed point) and rounded to float64 once,
 * so the bounds do not depend on the order of the terms. A degenerate interval
 * (width <= 1e-12 max(1,|e|)) becomes centre -+ 1. Writes d_bounds[0] = emin,
 * d_bounds[1] = emax (device, 2 doubles) and d_bounds[2] = 0.0 if H is finite, 1.0
 * otherwise (3 doubles). Asynchronous; n >= 1, ld >= n.
 */
fo_status fo_spectral_bounds(fo_ctx *ctx, const double *dH, int64_t n, int64_t ld,
                             double *d_bounds, void *stream);

/*
 * Spectral bounds for callers that cannot allocate device memory when they need them (for
 * example code running inside a memory pool it does not own, or an embedding that forbids
 * cudaMalloc after start-up). The paper has no counterpart: this is a service entry point.
 * It computes the same bounds as fo_spectral_bounds, bit for bit (both sum each row exactly
 * and round the sum once), with the same outputs in d_bounds[0..2], but needs no
 * context and allocates nothing: its per-block partial results live in a fixed
 * 128 KiB array in device memory that is part of the library image, resident on every GPU
 * that loads the library until the process exits.
 *  - n must not exceed FO_NOALLOC_MAX_N (the capacity of that array); larger n, NULL
 *    pointers or ld < n return FO_ERR_ARG, with nothing launched.
 *  - Every call looks up the array's device address on the current device
 *    (cudaGetSymbolAddress, which allocates nothing), so a device reset does not leave a
 *    stale address behind; the first call on a device also loads the library's device
 *    code there, so make it before any stream capture.
 *  - The call uses the current CUDA device; H and d_bounds must live on it.
 *  - Every call on a device shares the array, which keeps the last call's contents; each
 *    call overwrites what it reads, so no clearing is needed, but calls whose kernels
 *    overlap on the GPU (different streams or host threads) race and must be serialised.
 * Asynchronous on `stream`.
 */
#define FO_NOALLOC_MAX_N 32768
fo_status fo_spectral_bounds_noalloc(const double *dH, int64_t n, int64_t ld, double *d_bounds,
                                     void *stream);

/*
 * Chebyshev coefficients of the Fermi-Dirac function on [emin, emax] (Sec. "Chebyshev
 * expansions", Eq. (fermifunc)): Chebyshev-Gauss interpolation on n_quad nodes
 * (0 = max(2048, 4 n_terms)), c_0 = (1/M) sum_j f_j, c_n = (2/M) sum_j f_j cos(n theta_j),
 * theta_j = pi (j + 1/2) / M. Computed in float64 on the device into d_c[0..n_terms-1].
 * Asynchronous.
 */
fo_status fo_chebyshev_coeffs(fo_ctx *ctx, double kT, double mu, double emin, double emax,
                              int32_t n_terms, int32_t n_quad, double *d_c, void *stream);

/*
 * Density matrix (Eq. (fermi) with Eq. (ansatz)): dP[n x n, ldp] = sum_n c_n(mu) T_n(X),
 * X = (2H - (emin+emax) I)/(emax - emin). Baby steps T_1..T_k by the three-term
 * recurrence with the update 2 A B - C fused into the product epilogue; the expansion
 * is regrouped as sum_l T_l(T_k) R_l, R_l = sum_i g_{i,l} T_i (the bracket d_i^T a_l of
 * Eq. (formula for d)), and the giant steps run as a Clenshaw recurrence in T_k whose
 * product epilogue accumulates R_l. mu per params.mu_mode; n_e is the electron count
 * (tr P = n_e, spinless occupations in [0,1]).
 * Trace correction (split precisions with mu searched, m > 1, unless FO_FLAG_NO_TRACE_FIX):
 * the float32 masters of the split forms leave tr P off n_e by their rounding (~1e-8 n). With
 * gamma = (n_e - tr P)/(tr P - ||P||_F^2) the call applies P <- P + gamma (P - P^2), the
 * first-order shift of mu by gamma kT for the Fermi function (df/dmu = f(1-f)/kT), as one
 * more symmetric product P P with a float64 epilogue (for FO_PREC_BF16X3 in BF16x1: its
 * ~4e-3 relative error reaches P only through gamma, ~1e-6, so P moves by ~1e-8 at most;
 * FP16X2 keeps FP16x2), and then adds r/n to the diagonal,
 * r = n_e - tr P the float64 residual that this product's own rounding leaves (the
 * Frobenius-nearest matrix with trace n_e; skipped when |r| > 1e-4 max(1, n_e)). It is a
 * correction of rounding, not a search for mu: it is applied only when it moves P by at most
 * 1e-6 in ||.||_F/sqrt(n) (bound |n_e - tr P| / (2 sqrt(n tr(P - P^2)))) and |gamma| <= 1/4,
 * which holds for the rounding of every split form measured with mu by bisection; otherwise
 * (e.g. a learned mu accepted at a loose tr_tol) P keeps its trace and trace_gamma is 0. The
 * reported mu is that of the expansion; res->trace_raw keeps the trace before the
 * correction. If res != NULL
 * the call synchronises the
 * stream and fills *res; with res == NULL (or FO_FLAG_NO_RESULT_SYNC) it never blocks.
 * Returns the host-side status; device-side failures (non-finite H, no bracket) are
 * reported through res->status and the return value when res != NULL.
 */
fo_status fo_density_matrix(fo_ctx *ctx, const double *dH, int64_t n, int64_t ld,
                            double n_e, const fo_params *params, double *dP, int64_t ldp,
                            fo_result *res, void *stream);

/*
 * Density matrices of a batch of independent Hamiltonians of different sizes (e.g. the
 * replicas of a molecular-dynamics run) in one call: every stage of the method is one launch
 * over the whole batch (the products as one grouped tensor-core launch per step whose tiles
 * span all instances, largest first), so small instances fill the GPU together.
 *  - dH[b], dP[b]: device pointers of instance b (host array of batch pointers), n[b] its
 *    size, ld[b] / ldp[b] its leading dimensions (NULL: n[b]), n_e[b] its electron count,
 *    kT[b] its temperature (NULL: params->kT). All other parameters are shared.
 *  - The plan of a batch (sizes, layout, tensor maps, tile width) is cached in the context
 *    and reused while the sizes and parameters repeat; with FO_FLAG_GRAPH the whole call is
 *    replayed as one CUDA graph.
 *  - res: host array of batch results (in the caller's order), or NULL. With res != NULL
 *    (and no FO_FLAG_NO_RESULT_SYNC) the call synchronises and returns the first failing
 *    instance's status; otherwise it never blocks.
 */
fo_status fo_density_matrix_batched(fo_ctx *ctx, int32_t batch, const double *const *dH,
                                    const int64_t *n, const int64_t *ld, const double *n_e,
                                    const double *kT, const fo_params *params, double *const *dP,
                                    const int64_t *ldp, fo_result *res, void *stream);

/*
 * Same as fo_density_matrix with host buffers: copies hH to the device, runs, and
 * copies P back to hP (hP[n x n, ldp]). Pinned host memory makes the copies
 * asynchronous; the call always synchronises the stream before returning.
 */
fo_status fo_density_matrix_host(fo_ctx *ctx, const double *hH, int64_t n, int64_t ld,
                                 double n_e, const fo_params *params, double *hP,
                                 int64_t ldp, fo_result *res, void *stream);

/*
 * fo_density_matrix_batched with host buffers: copies every hH[b] to the device, runs the
 * batch, copies every P back to hP[b] (hP[b][n[b] x n[b], ldp[b]]), then synchronises.
 * Rows of one instance that are contiguous (ld[b] == n[b]) move as one linear copy; pinned
 * host memory makes the copies asynchronous. Arguments as in fo_density_matrix_batched.
 *
 * The copies run on two streams of the context (host to device, device to host) into one of
 * two device staging slots used in turn; the solve runs on `stream` after its inputs have
 * arrived, and the copy back waits for the solve. With FO_FLAG_NO_RESULT_SYNC the call
 * returns once everything is enqueued (res is left untouched): consecutive calls then
 * overlap the input copy of one call and the output copy of the previous one with a solve.
 * The caller keeps hH[b] unchanged and reads hP[b] only after fo_host_wait; a call reuses
 * a staging slot after the copies of the call two before it have finished.
 */
fo_status fo_density_matrix_batched_host(fo_ctx *ctx, int32_t batch, const double *const *hH,
                                         const int64_t *n, const int64_t *ld, const double *n_e,
                                         const double *kT, const fo_params *params,
                                         double *const *hP, const int64_t *ldp, fo_result *res,
                                         void *stream);

/*
 * Waits until every host-buffer call of the context has finished, its results copied to the
 * host buffers. Returns FO_OK, FO_ERR_DEVICE_TIMEOUT when a kernel of the last call gave up
 * a bounded wait (each call clears the device flag when it starts), or FO_ERR_CUDA.
 */
fo_status fo_host_wait(fo_ctx *ctx);

/*
 * Chebyshev moments tau_j = tr T_j(X), j < n_moments, of the scaled Hamiltonian on the
 * given bounds (d_bounds as written by fo_spectral_bounds), float64 into d_tau. Used as
 * features of the learned mu and exposed for spectral analysis. Moments up to 2k come
 * from baby-step traces and Frobenius products (tau_{a+b} = 2<T_a,T_b> - tau_{|a-b|},
 * Eq. (identity)); precision selects the arithmetic of the products. Asynchronous.
 */
fo_status fo_moments(fo_ctx *ctx, const double *dH, int64_t n, int64_t ld,
                     const double *d_bounds, int32_t n_moments, int32_t precision,
                     double *d_tau, void *stream);

/*
 * Learned chemical potential (FO_MU_LEARNED). A small fully connected network, float32,
 * 68 inputs -> 256 -> 256 -> 2 outputs with SiLU activations, held by the context:
 *   inputs  tau_1 .. tau_64 / N (Chebyshev moments tau_j = tr T_j(X) of the scaled
 *           Hamiltonian; only tau_j with j <= 2k are available from the k baby steps, the
 *           others are 0), N_e / N, kT_x = 2 kT / (emax - emin), emin / 100, emax / 100;
 *   outputs mu_x = (2 mu - (emin + emax)) / (emax - emin) and log2(L*) / log2(n_terms),
 *           L* the smallest number of terms whose coefficient tail sum_{j>=L*} |c_j| is at
 *           most 2.5e-7 (the proposed expansion order: the expansion cut there is within
 *           2.5e-7 of the full one in the 2-norm, since |T_j| <= 1 on the scaled spectrum;
 *           reported in fo_result.order, used to cut the expansion by FO_MU_ORDER).
 * Inputs and outputs are standardised with the training set's mean and standard deviation
 * (the normalisation vector: feature mean[68], feature std[68], target mean[2], target
 * std[2]). Parameters are stored W1 (256 x 68), b1 (256), W2 (256 x 256), b2 (256),
 * W3 (2 x 256), b3 (2): FO_MLP_PARAMS floats. The loss of training is the mean over the
 * batch of (mu_x error)^2 + 0.1 (order error)^2 in standardised units, minimised by Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8); all of forward, backward and update run in this
 * library's kernels. In a FO_MU_LEARNED call the proposed mu is kept when the float64
 * trace of P meets params.tr_tol; otherwise mu is corrected from tr P and ||P||_F^2
 * (Newton, then secant) and P re-evaluated up to params.max_newton times, and instances
 * still outside the tolerance fall back to exact moments and bisection (started at the
 * proposal). The call fails with FO_ERR_UNSUPPORTED while the context holds no model.
 */
#define FO_MLP_INPUTS  68
#define FO_MLP_OUTPUTS 2
#define FO_MLP_PARAMS  83970
#define FO_MLP_NORM    140

/*
 * Training pairs generated by the method itself: for every instance of the batch the exact
 * path (baby and giant steps, exact moments, bisection) finds mu, and the call writes the
 * network inputs into d_feat[batch x 68] and, if d_target != NULL, the targets
 * (mu_x, order) into d_target[batch x 2] (device float32, rows in the caller's order).
 * P is not formed. Arguments as in fo_density_matrix_batched (params->mu_mode is ignored).
 * res (optional, host array of batch) receives mu, bounds and status; the call then
 * synchronises.
 */
fo_status fo_learned_features(fo_ctx *ctx, int32_t batch, const double *const *dH,
                              const int64_t *n, const int64_t *ld, const double *n_e,
                              const double *kT, const fo_params *params, float *d_feat,
                              float *d_target, fo_result *res, void *stream);
/* Fresh parameters: Uniform(-a, a) weights, a = sqrt(6 / (fan_in + fan_out)), drawn with
 * splitmix64 from `seed`; zero biases; identity normalisation. Synchronous. */
fo_status fo_mlp_init(fo_ctx *ctx, uint64_t seed);
/* Copy parameters (FO_MLP_PARAMS floats) and normalisation (FO_MLP_NORM floats, NULL =
 * identity) from host memory into the context's model; resets the Adam state. */
fo_status fo_mlp_set_params(fo_ctx *ctx, const float *h_params, const float *h_norm);
/* Copy the model's parameters and normalisation to host memory (either may be NULL). */
fo_status fo_mlp_get_params(fo_ctx *ctx, float *h_params, float *h_norm);
/* Network outputs d_y[n x 2] for standardised inputs d_x[n x 68] (device). Asynchronous. */
fo_status fo_mlp_forward(fo_ctx *ctx, const float *d_x, int32_t n, float *d_y, void *stream);
/* Loss and gradient for standardised inputs d_x[n x 68] and targets d_t[n x 2]: every
 * parameter's gradient into d_grad[FO_MLP_PARAMS] (device, parameter layout), the loss into
 * *h_loss (host; the call then synchronises) unless h_loss == NULL. */
fo_status fo_mlp_gradients(fo_ctx *ctx, const float *d_x, const float *d_t, int32_t n,
                           float *d_grad, float *h_loss, void *stream);
/* Train on raw features d_feat[n x 68] and targets d_target[n x 2] (device): standardise
 * with their column statistics, then `epochs` passes of Adam steps over mini-batches of
 * `batch` rows in a splitmix64-shuffled order (seeded by `seed`); starts from the current
 * model, or a fresh one drawn from `seed` if the context has none. h_loss (host, epochs
 * floats, may be NULL) receives the mean mini-batch loss of every epoch. Synchronous. */
fo_status fo_mlp_train(fo_ctx *ctx, const float *d_feat, const float *d_target, int32_t n,
                       int32_t epochs, int32_t batch, float lr, uint64_t seed, float *h_loss,
                       void *stream);
/* Save / load the model (layout header, normalisation, parameters) to / from a file. */
fo_status fo_mlp_save(fo_ctx *ctx, const char *path);
fo_status fo_mlp_load(fo_ctx *ctx, const char *path);

/*
 * Enable (1) or disable (0) the stage profiler of this context; enabling clears it. While
 * enabled every density-matrix call records CUDA events around its stages.
 */
fo_status fo_profile_enable(fo_ctx *ctx, int32_t enable);
/*
 * Copy the accumulated profile to *out (synchronises on the recorded events); reset != 0
 * clears it afterwards.
 */
fo_status fo_profile_read(fo_ctx *ctx, fo_profile *out, int32_t reset);

/*
 * One recurrence product on float32 matrices (the kernel behind every step of the
 * expansion): dOut = alpha * A B^T + beta * C + D + shift * I_n, with A, B, C, D, dOut
 * n x n row-major float32 with leading dimension ld (C, D may be NULL), run on the tensor
 * cores in the split form `precision` (FO_PREC_BF16X3, FP16X2 or BF16X1; FP64 is
 * rejected). With symmetric != 0 only the entries on or above the diagonal are computed
 * and mirrored (the form the solver uses: the result is exactly symmetric, valid when the
 * true result is symmetric, e.g. A and B commuting symmetric matrices; then A B^T = A B);
 * with symmetric == 0 the full A B^T is computed. FP16X2 needs |entries| <= 1 in A and B.
 * Asynchronous.
 */
fo_status fo_recurrence_product(fo_ctx *ctx, int32_t precision, int32_t symmetric, int64_t n,
                                int64_t ld, const float *dA, const float *dB, const float *dC,
                                const float *dD, float alpha, float beta, float shift,
                                float *dOut, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FERMI_GB300_H */
