/*
 * csgs.h -- C ABI of the B300 (sm_103a) sensitivity-scoring library for provable
 * 3D Gaussian Splatting coreset pruning (arXiv 2607.02721).
 *
 * The paper's method (Sec. 3, Algorithm 1) for a pretrained scene G and a finite
 * query set Q (the pixel-rays of a fixed set of views):
 *   imp(g_i, q) = a(G, g_i, q) / A(G, q)            (Algorithm 1, step 2)
 *   s(g_i)      = max_q imp(g_i, q), S = sum_i s(g_i), p_i = s_i / S   (Eq. sen)
 *   draw m Gaussians i.i.d. from p, w_i = n_i / (m p_i)   (Algorithm 1, steps 4-5)
 * where a = c rho T is a Gaussian's front-to-back contribution to a pixel and A the
 * rendered value (Sec. 3 "Scalar rendering function").
 *
 * Conventions shared by every entry point
 *   - All calls are asynchronous on the context's CUDA stream unless they return a
 *     host value that needs the GPU result (documented per call); such calls
 *     synchronise that stream before returning.
 *   - "device" pointers are CUDA device memory on the context's device and are
 *     owned by the caller; the library never frees them.  "host" pointers are
 *     ordinary host memory.
 *   - Return value: CSGS_OK (0) or a negative csgs_status; csgs_last_error() gives a
 *     message.  Errors of asynchronous work surface at the next synchronising call.
 *   - Floating point: projection, compositing and transmittance are FP32; the
 *     total sensitivity S, the probabilities p and the weights w are FP64 (w is
 *     returned as FP32).
 *   - No entry point allocates memory it does not own: work buffers belong to the
 *     context (grown on demand, freed by csgs_destroy).
 */
#ifndef CSGS_H
#define CSGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t csgs_status;

#define CSGS_OK 0
#define CSGS_E_INVAL (-1)        /* bad argument: null pointer, size <= 0, bad camera, non-finite input */
#define CSGS_E_NOMEM (-2)        /* device allocation failed */
#define CSGS_E_CUDA (-3)         /* CUDA runtime error (message has the CUDA error string) */
#define CSGS_E_EMPTY (-4)        /* every query had A(G,q) = 0, so S = 0 (Sec. 3: such queries are discarded) */
#define CSGS_E_TIMEOUT (-5)      /* a bounded device wait ran out */
#define CSGS_E_DEVICE_CHECK (-6) /* a device-side check failed (e.g. instance capacity) */

typedef struct csgs_ctx csgs_ctx;

/* Scene G = {g_i = (mu_i, Sigma_i, alpha_i, c_i)} (Sec. 3 "3DGS scene") in structure-
 * of-arrays float32 layout.  Sigma_i = Rq diag(exp(log_scale))^2 Rq^T with Rq the
 * rotation of the (normalised) quaternion; alpha_i = sigmoid(opacity_logit);
 * c_i = max(0, SH(dir) + 0.5) with real SH of degree sh_degree evaluated along the
 * direction from the camera centre to mu_i. */
typedef struct {
    int64_t n;                   /* number of Gaussians N, 1 <= N < 2^31 */
    int32_t sh_degree;           /* 0..3 */
    int32_t is_device;           /* 1: pointers are device memory, 0: host memory */
    const float* means;          /* [3][N]: x[N], y[N], z[N] */
    const float* log_scales;     /* [3][N] */
    const float* quats;          /* [4][N]: w, x, y, z */
    const float* opacity_logits; /* [N] */
    const float* sh;             /* [(d+1)^2][3][N]: coefficient-major, then R, G, B */
} csgs_scene_desc;

/* A pinhole camera (query pose C = (R, t), Sec. 3 "Rendering query"): p_cam = R p + t
 * with x right, y down, z forward; pixel (u, v) has its centre at integer
 * coordinates, u = fx x/z + cx. */
typedef struct {
    float R[9];     /* row-major world-to-camera rotation */
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height; /* 1..16384 */
    float near_z;   /* Gaussians with camera depth <= near_z are culled (> 0).  Depths are sorted as
                       27-bit keys relative to near_z while every visible depth stays below about
                       2^16 near_z; a larger one makes the call repeat with 32-bit keys (same order) */
    float pad;
} csgs_camera;

/* Query resolutions (Sec. 3.5 "Sensitivity at Multiple Resolutions"): what one
 * query's objective aggregates before imp = a / A and s = max over queries. */
#define CSGS_RES_PIXEL 0   /* query = pixel, objective = obj_w . RGB ("Per-pixel construction") */
#define CSGS_RES_SCENE 1   /* one query over all views and pixels ("Per-tile and Per-scene") */
#define CSGS_RES_CHANNEL 2 /* query = (pixel, channel): the per-channel objective of Sec. 3 */
#define CSGS_RES_TILE 3    /* query = one 16x16 screen tile of one view */
#define CSGS_RES_IMAGE 4   /* query = one whole view */

/* Score variants (Sec. 3.5 "Additional variants"); A is the sum of the same terms. */
#define CSGS_VAR_L1 0      /* a = c rho T (the core score) */
#define CSGS_VAR_L2 1      /* a = (c rho T)^2 */
#define CSGS_VAR_NC 2      /* a = rho T (no colour) */

/* Screen-tile shapes of the binning and compositing (one CTA per tile, one thread per
 * pixel, warps of 8x4 pixels).  The footprint test is per pixel, so the shape decides
 * only how the work is split; the exponent is rounded in tile-centred coordinates, so
 * results of two shapes agree to FP32 rounding, not bit for bit.  The per-tile
 * resolution always uses 16x16 tiles (its query), and so does csgs_render_backward. */
#define CSGS_TILE_AUTO 0   /* the scene's shape chosen by csgs_autotune, else 16x16 */
#define CSGS_TILE_16X16 1
#define CSGS_TILE_32X8 2
#define CSGS_TILE_16X8 3
#define CSGS_TILE_8X8 4

/* Scoring / rendering conventions.  The paper fixes only the definitions; the
 * thresholds are those of the standard 3DGS rasteriser it relies on. */
typedef struct {
    int32_t resolution;    /* CSGS_RES_* */
    int32_t variant;       /* CSGS_VAR_* */
    float obj_w[3];        /* per-pixel objective weights (1,1,1) = total colour */
    float alpha_min;       /* pairs with rho < alpha_min are skipped (1/255) */
    float rho_max;         /* rho = min(rho_max, alpha k) (0.99) */
    float t_min;           /* traversal stops before T would drop below t_min (1e-4) */
    float cut2;            /* footprint: k = 0 where d^T Sigma'^-1 d > cut2 (9 = 3 sigma) */
    float dilation;        /* added to the diagonal of the 2-D covariance (0.3) */
    float clamp_fov;       /* J uses x/z, y/z clamped to clamp_fov * half-FOV tangent (1.3) */
    int32_t view_batch;    /* views projected per launch (0 = automatic) */
    int32_t collect_stats; /* bit 0: count evaluated and contributing pairs (slower kernels);
                              bit 1: time the phases with CUDA events on the stream */
    int32_t tile_shape;    /* CSGS_TILE_* (CSGS_TILE_AUTO) */
    int32_t persist_ctas;  /* per-pixel score: compositing as one persistent launch per view of
                              persist_ctas CTAs, each taking the next tile (longest lists first)
                              from a queue until none is left; 0 = the scene's choice by
                              csgs_autotune (else one CTA per tile), -1 = one CTA per tile.
                              Scores do not depend on it */
    int32_t accumulate;    /* 1: s_dev already holds the scores of other query views of the same
                              scene at the same resolution, and the call leaves in it the maximum
                              over both query sets (s is a maximum over queries, Eq. sen, so this
                              equals scoring the union; S is returned for the union).  Pixel,
                              channel, tile and image resolutions; CSGS_E_INVAL for the per-scene
                              one, whose s is a ratio of sums.  0: s_dev is overwritten */
} csgs_score_opts;

/* What csgs_autotune chose for a scene. */
typedef struct {
    int32_t view_batch;    /* views projected per launch */
    int32_t sort_blocks;   /* radix-sort grid (CTAs) */
    int32_t tile_shape;    /* CSGS_TILE_16X16, CSGS_TILE_32X8, CSGS_TILE_16X8 or CSGS_TILE_8X8 */
    int32_t persist_ctas;  /* persistent compositing CTAs, 0 = one CTA per tile */
    float probe_ms;        /* the chosen configuration's time for the probe views */
} csgs_tuning;

/* Counters of the last csgs_score / csgs_render call. */
typedef struct {
    int64_t views;
    int64_t rays;             /* pixel-rays processed */
    int64_t instances;        /* (Gaussian, tile) pairs summed over views */
    int64_t pairs_evaluated;  /* compositing pass 1: (ray, Gaussian) pairs tested before the stop (bit 0) */
    int64_t pairs_hit;        /* pass 1: pairs inside the footprint with rho >= alpha_min (bit 0) */
    int64_t pairs_evaluated2; /* scoring pass 2: pairs tested (bit 0) */
    int64_t pairs_hit2;       /* scoring pass 2: contributing pairs (bit 0) */
    int64_t violations;       /* csgs_render: pairs met before the stop with w alpha k >= 1 (bit 0) */
    int64_t capacity_retries; /* re-runs after growing the instance buffers, or after a visible depth beyond
                                 about 2^16 near_z switched the context to 32-bit depth keys */
    int64_t kernel_launches;  /* kernels this library launched in the call */
    int64_t composite_launches;
    int64_t queries;          /* pixel queries with A > 0 (|Q'| of Thm. 2; pixel and channel resolutions) */
    double score_ms;          /* the whole call on the stream (CUDA events) */
    double project_ms;        /* phase totals (bit 1) */
    double sort_ms;
    double composite_ms;
    int64_t entries_staged;   /* tile-list entries staged by compositing pass 1 (bit 0) */
    int64_t entries_staged2;  /* tile-list entries staged by pass 2 (bit 0) */
    double composite_busy_ms; /* time some compositing launch was running: the union of their spans, which
                                 overlap on the two compositing streams (bit 1) */
    int64_t view_batches;     /* csgs_score: view batches (one projection launch and one binning chain each) */
    int64_t warp_entries;     /* compositing pass 1: (warp, tile-list entry) iterations; 32 x this over
                                 pairs_evaluated is the lanes' idle share (bit 0, pixel and channel scores) */
    int64_t warp_entries2;    /* ... of scoring pass 2 (bit 0) */
    double objective_sum;     /* per-scene resolution: sum over the call's queries of the objective A(q), the
                                 denominator of its scores (lets view shards combine their scores) */
} csgs_stats;

/* Fill *o with the default conventions above. */
void csgs_default_opts(csgs_score_opts* o);

/* Create a context on CUDA device `device`.  cuda_stream: an existing cudaStream_t
 * to run on (not owned), or NULL to create one (owned).  *out receives the context. */
csgs_status csgs_create(csgs_ctx** out, int32_t device, void* cuda_stream);

/* Destroy a context: synchronises its stream, frees every scene and work buffer. */
void csgs_destroy(csgs_ctx* ctx);

/* Message of the last error on this context (owned by the context; valid until the
 * next call). */
const char* csgs_last_error(const csgs_ctx* ctx);

/* Copy a scene into the context (host or device source per desc->is_device).
 * Checks sizes and that every attribute is finite (non-finite -> CSGS_E_INVAL,
 * synchronising).  *scene_id receives the handle.  Attribute buffers of earlier freed
 * scenes of the same size are reused before new device memory is allocated. */
csgs_status csgs_load_scene(csgs_ctx* ctx, const csgs_scene_desc* desc, int32_t* scene_id);

/* csgs_load_scene without waiting: allocates (or reuses) the buffers, enqueues the
 * copies and the finiteness check on the context's own upload stream and returns.  The
 * first call that uses the scene (any call taking its id, csgs_free_scene excepted)
 * waits for the upload to finish; if an attribute is non-finite, that call fails with
 * CSGS_E_INVAL and the scene is released (the id becomes invalid).  The source must stay
 * unchanged until then; from pinned host memory the copies run on the copy engine
 * beside the context's kernels, so loading the next scene overlaps scoring the current
 * one.  At most 16 such loads may be pending (not yet used) at once (else CSGS_E_INVAL).
 * The paper has no counterpart: this is a deployment variant of the load. */
csgs_status csgs_load_scene_async(csgs_ctx* ctx, const csgs_scene_desc* desc, int32_t* scene_id);

/* Release a scene (after the context's stream has finished with it).  Its attribute
 * buffers stay with the context for later loads of the same size (up to 32 buffers;
 * the oldest beyond that, and all of them at csgs_destroy, return to the device). */
csgs_status csgs_free_scene(csgs_ctx* ctx, int32_t scene_id);

/* Set the query views of a scene (Algorithm 1, step 1): every pixel of each camera
 * is one query.  cams: host array of n_views cameras (copied). */
csgs_status csgs_set_queries(csgs_ctx* ctx, int32_t scene_id, const csgs_camera* cams, int32_t n_views);

/* Sensitivity scores (Algorithm 1, steps 2-3; Eq. sen) over all query views.
 * s_dev: device float[N], written with s_i (with opts->accumulate: the maximum of its
 * previous contents and this query set's s_i).  S_out: host double, total
 * sensitivity S of what s_dev holds on return (may be NULL).  Synchronises.  Returns
 * CSGS_E_EMPTY when S = 0. */
csgs_status csgs_score(csgs_ctx* ctx, int32_t scene_id, const csgs_score_opts* opts, float* s_dev, double* S_out);

/* Sensitivity scores of several scenes in one submission (Algorithm 1, steps 2-3, per
 * scene; each scene keeps its own query views).  scene_ids: host int32[n_scenes]
 * (1 <= n_scenes <= 64); s_devs: host array of n_scenes device float pointers, scene
 * k's scores (float[N_k]); S_out: host double[n_scenes], S per scene (required).
 * use_graph != 0: the first call runs every launch eagerly (this settles the
 * instance capacity), then captures the whole batch - every projection, sort,
 * composite and reduction launch of every scene - into one CUDA graph, which later
 * calls with the same scenes, views, options and output pointers replay with a
 * single launch.  A graph holds the context's work buffers, so the context must
 * not be used from another thread during the call.  Only statistics views, rays,
 * instances, queries, score_ms and kernel_launches are filled.  Synchronises.
 * Does not return CSGS_E_EMPTY: check S_out. */
csgs_status csgs_score_batch(csgs_ctx* ctx, int32_t n_scenes, const int32_t* scene_ids, const csgs_score_opts* opts,
                             float* const* s_devs, double* S_out, int32_t use_graph);

/* Choose, for one scene, the view batch (views projected per launch), the radix-sort
 * grid, the tile shape and the persistent compositing grid by timing csgs_score's work
 * on the first probe_views query views (0: min(16, views)), one dimension after the
 * other: view batches {1,2,4,8,16} x sort grids {74,148,296,592,1184,1776} blocks at the
 * requested shape (16x16 for CSGS_TILE_AUTO); then, for CSGS_TILE_AUTO (and not the
 * per-tile resolution), the shapes 32x8, 16x8 and 8x8 at the best pair; then, for the
 * per-pixel score with opts->persist_ctas 0, persistent launches of r, r - 1 and r - 2
 * CTAs per SM (r: the kernel's resident limit) against one CTA per tile.  The choices
 * are kept with the scene and apply to later csgs_score / csgs_score_batch calls on it
 * (the view batch where opts->view_batch is 0, the shape where opts->tile_shape is
 * CSGS_TILE_AUTO, the persistent grid where opts->persist_ctas is 0); the sort grid also
 * becomes the context's grid for scenes that were not tuned themselves.  The view batch,
 * the grid and the persistent launch do not change the scores; the shape changes them
 * only by FP32 rounding (see CSGS_TILE_*).  out (may be NULL) receives the choices.
 * Synchronises. */
csgs_status csgs_autotune(csgs_ctx* ctx, int32_t scene_id, const csgs_score_opts* opts, int32_t probe_views,
                          csgs_tuning* out);

/* Sensitivity sampling (Algorithm 1, steps 3-5): S = sum s (FP64), p = s / S,
 * m i.i.d. inverse-CDF draws with Philox4x32-10 uniforms (key = seed, counter =
 * draw index), counts n_i and weights w_i = n_i / (m p_i).
 * s_dev: device float[n] (non-negative).  idx_dev: device int32[m] receives the
 * distinct sampled indices in ascending order; w_dev: device float[m] their
 * weights; *n_distinct (host) their count.  Synchronises.
 * CSGS_E_EMPTY if S = 0; CSGS_E_INVAL if m <= 0 or n <= 0. */
csgs_status csgs_sample_coreset(csgs_ctx* ctx, const float* s_dev, int64_t n, int64_t m, uint64_t seed,
                                int32_t* idx_dev, float* w_dev, int64_t* n_distinct);

/* As csgs_sample_coreset, with the probabilities given: p_dev device double[n]
 * (sum 1).  draws_dev: optional device int32[m] receiving every draw J_t in draw
 * order (NULL to skip).  Used to check the sampler bit for bit. */
csgs_status csgs_sample_coreset_p(csgs_ctx* ctx, const double* p_dev, int64_t n, int64_t m, uint64_t seed,
                                  int32_t* idx_dev, float* w_dev, int64_t* n_distinct, int32_t* draws_dev);

/* Render one query view of a scene, optionally as the weighted pruned scene A_w of
 * Sec. 3 ("A pruned 3DGS scene"): Gaussian i gets rho' = min(rho_max, w_i alpha_i k)
 * and Gaussians not listed are removed.  idx_dev / w_dev: device int32[n_sel] /
 * float[n_sel] (both NULL: the full scene).  rgb_dev: device float[H][W][3].
 * T_dev: optional device float[H][W] final transmittance.  Asynchronous; the
 * validity-violation count appears in csgs_get_stats after csgs_sync. */
csgs_status csgs_render(csgs_ctx* ctx, int32_t scene_id, int32_t view, const int32_t* idx_dev, const float* w_dev,
                        int64_t n_sel, const csgs_score_opts* opts, float* rgb_dev, float* T_dev);

/* Per-pixel quantities of the transfer to true rendering (Sec. 3.3, Lemma "transfer",
 * Thm. 3) for one view and a weighted pruned scene w (idx_dev / w_dev as in
 * csgs_render): along the full-scene order, A = sum c rho T, the relaxed objective
 * A_th = sum w c rho T (full-scene transmittance), the true reduced render
 * A_w = sum w c rho T_w with T_w = prod (1 - w rho), gamma_q = max over retained
 * Gaussians of |log T - log T_w|, and min over pairs of (1 - w rho) (validity needs
 * it > 0).  Use the pure definitions (alpha_min = 0, rho_max = 1, t_min = 0) in opts.
 * out_dev: device float[H][W][11] = A[3], A_th[3], A_w[3], gamma_q, min factor.
 * Asynchronous. */
csgs_status csgs_transfer(csgs_ctx* ctx, int32_t scene_id, int32_t view, const int32_t* idx_dev, const float* w_dev,
                          int64_t n_sel, const csgs_score_opts* opts, float* out_dev);

/* Thm. 2 sample size: ceil(3 S / eps^2 * log(2 n_queries / delta)); 0 on bad input. */
double csgs_theorem2_sample_size(double S, double eps_c, double delta, int64_t n_queries);

/* Thm. 3 rendered error: max(1 - e^-gamma (1 - eps_c), e^gamma (1 + eps_c) - 1). */
double csgs_theorem3_eps(double gamma, double eps_c);

/* ------------------------------------------------------------------ surrogate model
 * Not in the paper: a learned stand-in for exact scoring over most query views.  A
 * BF16 MLP x (64 features) -> 256 (GELU) -> 256 (GELU) -> 1 predicts log-sensitivity;
 * it is trained on exact scores of a few views and applied with view statistics over
 * all views.  Both layers run on the tensor cores (tcgen05.mma, BF16 operands, FP32
 * accumulation in tensor memory); biases, GELU and the last layer are FP32.
 * Parameter block (FP32, CSGS_MLP_PARAMS floats): W1[256][64], b1[256], W2[256][256],
 * b2[256], w3[256], b3.  The context owns one model and its Adam state. */
#define CSGS_MLP_PARAMS 82689

/* Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, Adam state cleared. */
csgs_status csgs_mlp_init(csgs_ctx* ctx, uint64_t seed);
/* Copy a parameter block in (device float[CSGS_MLP_PARAMS]); clears the Adam state. */
csgs_status csgs_mlp_set_params(csgs_ctx* ctx, const float* P_dev);
/* Copy the parameter block out (device float[CSGS_MLP_PARAMS]); asynchronous. */
csgs_status csgs_mlp_get_params(csgs_ctx* ctx, float* P_dev);
/* y[B] = model(X); X_dev: device BF16 [B][64] row-major; y_dev: device float[B].
 * Synchronises; CSGS_E_TIMEOUT if a tensor-core completion is not observed. */
csgs_status csgs_mlp_forward(csgs_ctx* ctx, const void* X_dev, int64_t B, float* y_dev);
/* Gradient block of loss = mean_r (y_r - t_r)^2 over B rows (device float[CSGS_MLP_PARAMS]);
 * *loss_out (host, nullable) receives the loss.  Synchronises. */
csgs_status csgs_mlp_gradient(csgs_ctx* ctx, const void* X_dev, const float* t_dev, int64_t B, float* G_dev,
                              float* loss_out);
/* `steps` Adam steps (beta 0.9, 0.999, eps 1e-8, learning rate lr) on minibatches of
 * `batch` rows drawn with replacement from the n_rows rows of X / t (Philox, key = seed).
 * *final_loss (host, nullable): the last minibatch loss.  Synchronises. */
csgs_status csgs_mlp_train(csgs_ctx* ctx, const void* X_dev, const float* t_dev, int64_t n_rows, int32_t batch,
                           int32_t steps, float lr, uint64_t seed, float* final_loss);
/* Per-Gaussian statistics over the scene's query views (device float[N][3]): number of
 * views the footprint reaches, mean and max area (px^2) of the projected 3-sigma ellipse. */
csgs_status csgs_view_stats(csgs_ctx* ctx, int32_t scene_id, const csgs_score_opts* opts, float* stats_dev);
/* Model inputs (device BF16 [N][64]): mean/4, log-scale+4, unit quaternion, opacity logit,
 * 5 x SH coefficients (48 slots), log(1+views), log(1+mean area)/4, log(1+max area)/4,
 * extra/8, 0.  extra_dev (device float[N], nullable: 0): one more per-Gaussian input (the
 * surrogate passes the log of its cheap reduced-resolution score). */
csgs_status csgs_features(csgs_ctx* ctx, int32_t scene_id, const float* stats_dev, const float* extra_dev,
                          void* X_dev);
/* t = log(s + eps) (device float[n]). */
csgs_status csgs_log_target(csgs_ctx* ctx, const float* s_dev, int64_t n, float eps, float* t_dev);
/* The surrogate sensitivity from the prediction y and the exact scores of the scored
 * views (s_exact, nullable): fill_only = 0: s_out = max(exp(y) - eps, 0, s_exact) (never
 * below the exact score); fill_only = 1: s_exact where it is > 0, else max(exp(y) - eps, 0). */
csgs_status csgs_surrogate_combine(csgs_ctx* ctx, const float* y_dev, const float* s_exact_dev, int64_t n, float eps,
                                   int32_t fill_only, float* s_out);
/* Residual form of the surrogate (not in the paper): the network predicts the correction of
 * log s over a prior score p (the cheap reduced-resolution score) scaled by exp(mu), mu the
 * mean log-ratio of the exact to the prior score on the scored views.
 * csgs_log_ratio_mean: mean over the i with a_i > 0 and b_i > 0 of log a_i - log b_i (FP64,
 * fixed summation order) and how many i qualify (count_out nullable); 0 and 0 when none
 * does.  a_dev, b_dev: device float[n]; mean_out, count_out: host.  Synchronises. */
csgs_status csgs_log_ratio_mean(csgs_ctx* ctx, const float* a_dev, const float* b_dev, int64_t n, double* mean_out,
                                int64_t* count_out);
/* t = log(s + eps) - log(p + eps) - mu (device float[n]); mu finite. */
csgs_status csgs_log_residual_target(csgs_ctx* ctx, const float* s_dev, const float* p_dev, int64_t n, float eps,
                                     double mu, float* t_dev);
/* csgs_surrogate_combine with the prediction y taken as that correction: the predicted score
 * is max(exp(y + log(p + eps) + mu) - eps, 0). */
csgs_status csgs_surrogate_combine_prior(csgs_ctx* ctx, const float* y_dev, const float* p_dev,
                                         const float* s_exact_dev, int64_t n, float eps, double mu, int32_t fill_only,
                                         float* s_out);

/* ------------------------------------------------------------------ short recovery
 * The paper's short post-pruning finetune (Sec. 4, "short recovery"): gradients of a
 * loss on the weighted pruned render with respect to the means, SH coefficients and
 * opacity logits (scales and rotations fixed). */

/* Overwrite a scene's attributes in place (same N and SH degree; host or device
 * source as desc->is_device).  Asynchronous; no finiteness check. */
csgs_status csgs_update_scene(csgs_ctx* ctx, int32_t scene_id, const csgs_scene_desc* desc);

/* Backward of csgs_render (same view, weights and options): given grad_rgb_dev =
 * dL/dC (device float[H][W][3]), ADDS dL/d means to g_means_dev [3][N], dL/d SH to
 * g_sh_dev [(d+1)^2][3][N] and dL/d opacity logits to g_logit_dev [N] (all device
 * float).  Back to front through the compositing (dC/drho_i = c_i T_i - S_i / (1 -
 * rho_i), S_i the colour behind i), no gradient through the rho_max clamp or the
 * footprint and threshold decisions, then through the EWA projection and the SH colour
 * (including its view direction).  The transmittance in front of each contributor is
 * recovered from the back, T_i = T_(i+1) / (1 - rho_i), so opts->rho_max must stay below
 * 1 (a factor 1 - rho_i of 0 gives non-finite gradients).  Asynchronous. */
csgs_status csgs_render_backward(csgs_ctx* ctx, int32_t scene_id, int32_t view, const int32_t* idx_dev,
                                 const float* w_dev, int64_t n_sel, const csgs_score_opts* opts, const float* grad_rgb_dev,
                                 float* g_means_dev, float* g_sh_dev, float* g_logit_dev);

/* One Adam step (Kingma & Ba) on n device floats p with gradient g and moments m, v. */
csgs_status csgs_adam_update(csgs_ctx* ctx, float* p_dev, const float* g_dev, float* m_dev, float* v_dev, int64_t n,
                             float lr, float beta1, float beta2, float eps, int32_t step);

/* Wait for the context's stream and report errors of asynchronous work. */
csgs_status csgs_sync(csgs_ctx* ctx);

/* s_dev[i] = s_dev[i] * factor (FP64 product rounded to FP32), device float[n], on the
 * context's stream (asynchronous).  factor finite and >= 0 (else CSGS_E_INVAL).  The
 * per-scene resolution of Sec. 3.5 is a ratio of sums over queries: view shards combine
 * their scores s_r into the whole query set's by s = sum_r s_r A_r / sum_r A_r, with A_r
 * the shard's objective total (csgs_stats.objective_sum); this scales one shard. */
csgs_status csgs_scale_scores(csgs_ctx* ctx, float* s_dev, int64_t n, double factor);

/* S = sum_i s_i (Alg. 1 step 3) in FP64, in the fixed order csgs_score uses; s_dev:
 * device float[n].  Synchronises. */
csgs_status csgs_total_sensitivity(csgs_ctx* ctx, const float* s_dev, int64_t n, double* S_out);

/* Counters of the last score / render (synchronises). */
csgs_status csgs_get_stats(csgs_ctx* ctx, csgs_stats* out);

/* Largest n accepted by csgs_sample_coreset_noalloc. */
#define CSGS_NOALLOC_MAX_N 262144

/* csgs_sample_coreset_p without any memory allocation, for callers that cannot
 * allocate device memory: code inside a host framework that owns all GPU memory
 * through its own pool, real-time runtimes that forbid allocation after start-up,
 * and callers without a csgs_ctx (creating one allocates work buffers).  The paper
 * has no counterpart; this is a deployment variant of the same sampler.
 *   The sampler's scratch (integer CDF, draw counts, scan partials; about 3 MB) is a
 *   fixed file-scope device array that every GPU loading this library holds until
 *   the process exits; n must not exceed CSGS_NOALLOC_MAX_N (else CSGS_E_INVAL).
 *   It runs on the calling thread's current CUDA device, on cuda_stream (a
 *   cudaStream_t, NULL = the legacy default stream).  The first call on a device
 *   looks the array's device address up (cudaGetSymbolAddress).  Every call ends by
 *   synchronising cuda_stream (it reads the distinct count back to the host), so no
 *   call can be made while cuda_stream is being captured.  If a CUDA error from earlier
 *   work is already pending on the calling thread, the call returns CSGS_E_CUDA
 *   without launching anything and leaves that error pending; otherwise
 *   CSGS_E_CUDA reports this call's own launch or copy failure.  Every call shares
 *   the one array, which keeps the last call's contents (the counts are cleared by
 *   each call): calls that overlap on the GPU - other streams, other host threads -
 *   race and must be serialised by the caller.  No cudaMalloc, cudaFree or allocating library call
 *   is made.  Arguments and outputs as csgs_sample_coreset_p (without the draw
 *   list); *n_distinct is written on the host after the stream is synchronised. */
csgs_status csgs_sample_coreset_noalloc(const double* p_dev, int64_t n, int64_t m, uint64_t seed, int32_t* idx_dev,
                                        float* w_dev, int64_t* n_distinct, void* cuda_stream);

/* Diagnostic of the tensor-core path: C[128][N] = A[128][K] * B[N][K]^T with BF16 A, B
 * (device, row-major) and FP32 C (device), computed by one tcgen05.mma chain with the
 * accumulator in tensor memory.  K % 16 == 0, 16 <= K <= 128; N % 16 == 0, 16 <= N <= 256.
 * Synchronises; CSGS_E_TIMEOUT if the MMA completion was not observed in time. */
csgs_status csgs_debug_tc_gemm(csgs_ctx* ctx, const void* A_dev, const void* B_dev, float* C_dev, int32_t K,
                               int32_t N);

/* Diagnostic of the MN-major operand layout (used by the network's weight gradients):
 * C[128][N] = A^T B with A given as [K][128] and B as [K][N] (BF16, device, row-major),
 * both staged in the no-swizzle MN-major layout, FP32 C (device).  Shapes and errors as
 * csgs_debug_tc_gemm. */
csgs_status csgs_debug_tc_gemm_mn(csgs_ctx* ctx, const void* A_dev, const void* B_dev, float* C_dev, int32_t K,
                                  int32_t N);

/* Diagnostic of the bounded device waits: csgs_debug_tc_gemm with the threads' wait for
 * the MMA chain's completion limited to first_wait_cycles SM clock cycles (0: a single
 * non-blocking test of the completion barrier, which an MMA chain issued a moment
 * earlier has not reached).  A warp whose wait runs out records the error and then
 * waits, with the kernels' full budget (about one second), for the chain to drain, so
 * that no MMA is in flight when the kernel frees its tensor memory and returns; the
 * context stays usable.  Returns CSGS_E_TIMEOUT when the first wait ran out (C_dev is
 * then partly unwritten), CSGS_E_INVAL for a negative budget.  Synchronises.  The paper
 * has no counterpart: this exercises the failure path of the library's own waits. */
csgs_status csgs_debug_tc_gemm_wait(csgs_ctx* ctx, const void* A_dev, const void* B_dev, float* C_dev, int32_t K,
                                    int32_t N, int64_t first_wait_cycles);

/* Diagnostic: the surrogate network's activation as its kernels evaluate it:
 * out_dev[2i] = GELU(z_i) = z_i Phi(z_i), out_dev[2i+1] = GELU'(z_i) (erf by Abramowitz &
 * Stegun 7.1.26, |error| <= 1.5e-7, with the hardware reciprocal and exponential).
 * The epilogues evaluate GELU on pairs with packed FP32 instructions; out_dev[2i] is that
 * packed result, checked bit for bit against the one-value evaluation (NaN if the two
 * differ, for z_i or -z_i).  z_dev: device float[n]; out_dev: device float[2n].
 * Asynchronous. */
csgs_status csgs_debug_gelu(csgs_ctx* ctx, const float* z_dev, int64_t n, float* out_dev);

/* Total number of kernels this library has launched in the process (all contexts);
 * the difference across a region counts that region's launches. */
int64_t csgs_kernel_launch_count(void);

/* Diagnostic: the FP32 projection of every Gaussian into one query view (the EWA
 * step of the path, Sec. 3 "Scalar rendering function").  out_dev: device
 * float[N][16] = valid, mean x, mean y (each as the rounded sum of a two-float
 * value), conic a, b, c, covariance xx, xy, yy, depth, alpha, r, g, b, tile count,
 * mean x low word. */
csgs_status csgs_debug_project(csgs_ctx* ctx, int32_t scene_id, int32_t view, const csgs_score_opts* opts,
                               float* out_dev);

#ifdef __cplusplus
}
#endif

#endif /* CSGS_H */
