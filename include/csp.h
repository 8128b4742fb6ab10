/*
 * csp.h -- C ABI of the GB300 cross-scale predictive OMP library.
 *
 * Batched Orthogonal Matching Pursuit over the independent patches of a
 * linear inverse problem y = Phi D s + e (arXiv 1511.05174, Sec. III-C), in
 * two forms:
 *   - plain OMP against the fine dictionary (Sec. II-B, Algorithm 1);
 *   - cross-scale ("zero-tree") OMP (Sec. III-C, Algorithm 2, problems
 *     (P_low) and (P_high)): OMP on the coarsest scale, then at each finer
 *     scale an OMP restricted to the children f(Omega) of the atoms chosen
 *     one scale up (cross-scale map, Sec. III-B; multi-scale tree, Fig. 3).
 *
 * Conventions (all entry points):
 *   - Every call returns a csp_status; CSP_OK (0) on success, a negative code
 *     otherwise, with a message from csp_last_error().  No C++ exception
 *     crosses this boundary.
 *   - The caller owns every buffer it passes.  The library copies what it
 *     keeps (dictionaries, links, codes) into device memory it owns, and frees
 *     it in csp_destroy().
 *   - "device" pointers are CUDA global-memory pointers on the context's
 *     device; "host" pointers are ordinary (preferably pinned) host memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued asynchronously on it; outputs are valid once the stream has
 *     reached the point of the call.
 *   - Dictionaries are atom-major float32: atom i of level l occupies
 *     D[i * N_l .. i * N_l + N_l - 1].  Level 0 is the finest scale.
 *   - Patch vector layout at any level: index ((ly * Lx + lx) * Py + py) * Px + px
 *     for plane-grid position (ly, lx) (colour channel, frame or view) and
 *     pixel (py, px) of the patch.
 *   - Patch origins along an axis of extent E: min(i * stride, E - P) for
 *     i = 0 .. n-1, n = floor((E - P) / stride) + 1 (+1 when the stride misses
 *     E - P).  Patch b = iy * nx + ix (raster order).
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef CSP_H
#define CSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int csp_status;

#define CSP_OK               0
#define CSP_ERR_INVALID     -1   /* bad argument, size or state */
#define CSP_ERR_OOM         -2   /* device allocation failed or memory budget exceeded */
#define CSP_ERR_NOT_READY   -3   /* a required load/set call has not been made */
#define CSP_ERR_CUDA        -4   /* a CUDA runtime call failed */
#define CSP_ERR_TIMEOUT     -5   /* a bounded wait expired */
#define CSP_ERR_UNSUPPORTED -6   /* valid request the library does not implement   */

#define CSP_MAX_LEVELS 4
#define CSP_MAX_K      32        /* largest sparsity per level */

/* Sensing operators Phi (Sec. III-C "y = Phi x + e"; Sec. IV experiments). */
#define CSP_SENSE_IDENTITY       0  /* denoising: Phi = I, M = planes * P * P                 */
#define CSP_SENSE_BAYER_RGGB     1  /* demosaicing: one colour per pixel, RGGB, M = P * P     */
#define CSP_SENSE_CODED_EXPOSURE 2  /* video CS: per-pixel binary code per frame, M = P * P   */
#define CSP_SENSE_CODED_APERTURE 3  /* light-field CS: per-shot binary code per view,
                                       M = shots * P * P                                     */
#define CSP_SENSE_DENSE          4  /* patch CS: one dense Phi (M x N) for every patch,
                                       M = shots; measurements are per patch (pass Y to
                                       csp_solve directly: no extraction)                   */

#define CSP_MODE_PLAIN        0     /* Algorithm 1 on the fine dictionary                    */
#define CSP_MODE_CROSS_SCALE  1     /* Algorithm 2 over all loaded levels                    */

#define CSP_PREC_FP32 0             /* proxy inner products in FP32 on CUDA cores            */
#define CSP_PREC_BF16 1             /* proxy on tcgen05 tensor cores in BF16 (FP32 accumulate),
                                       top candidates re-scored in FP32                      */

typedef struct csp_ctx csp_ctx;

/* Signal and patch geometry (patches: Sec. IV; scales W/U: Sec. III-A/III-C). */
typedef struct csp_geometry {
    int H, W;                  /* pixels per plane                                       */
    int plane_rows;            /* Ly: plane grid rows (views) -- 1 for images and videos */
    int plane_cols;            /* Lx: colour channels, frames or view columns            */
    int P;                     /* patch side in pixels                                   */
    int stride;                /* patch origin step                                      */
    int n_levels;              /* number of scales, 1 .. CSP_MAX_LEVELS                  */
    int factors[CSP_MAX_LEVELS][4]; /* per level (fy, fx, sy, sx): downsampling of the plane
                                  grid rows/cols and pixel rows/cols relative to level 0;
                                  level 0 must be (1,1,1,1); each level must divide the
                                  next.  W = box average, U = nearest replicate, W U = I. */
} csp_geometry;

/* Sensing operator.  `codes` and `phi` are HOST pointers, copied by the library:
 *   CODED_EXPOSURE: codes uint8 [planes][H][W] (frame-major), values 0/1;
 *   CODED_APERTURE: codes uint8 [shots][planes], values 0/1;
 *   DENSE: phi float32 [shots][planes * P * P] row-major (shots = M, a multiple
 *          of 4, at most 256), the same Phi for every patch;
 *   otherwise ignored (may be NULL). */
typedef struct csp_sensing {
    int kind;
    int shots;
    const uint8_t *codes;
    const float *phi;
} csp_sensing;

/* Solve parameters.
 *   K[l]       -- sparsity budget at level l (1 .. CSP_MAX_K) used when K_patch[l] is NULL;
 *   K_patch[l] -- optional DEVICE int8 [B] per-patch budgets for level l (values 0 .. CSP_MAX_K);
 *   Kmax       -- row length of the support/coef outputs (>= every level-0 budget).
 * In CSP_MODE_PLAIN only level 0 is read. */
typedef struct csp_solve_params {
    int mode;
    int precision;
    int K[CSP_MAX_LEVELS];
    const int8_t *K_patch[CSP_MAX_LEVELS];
    int Kmax;
} csp_solve_params;

/* Solve statistics of the last csp_solve on a context (host copy, filled
 * when the solve's stream work is complete and csp_solve_stats is called). */
typedef struct csp_solve_stats {
    int64_t patches;
    int64_t fp64_fallbacks;    /* projections redone in FP64 (pivot ratio below threshold) */
    int64_t early_stops;       /* patches that ended with k_eff < budget                    */
    int64_t overflow;          /* patches whose candidate set exceeded the kernel capacity  */
    int64_t restricted_scores; /* candidate inner products <a_i, r> computed by the restricted
                                  (finer-scale) steps, summed over patches and iterations   */
    int64_t timeouts;          /* 1 when a bounded device wait expired (results invalid;
                                  csp_solve_stats_get then returns CSP_ERR_TIMEOUT)         */
    int64_t synthesized;       /* 1 when the last call was csp_reconstruct and its finest
                                  restricted level wrote x_hat_p itself (no synthesis pass) */
} csp_solve_stats;

/* Create a context on CUDA `device`.  mem_budget_bytes caps the device memory
 * the context may hold (0 = no cap); exceeding it yields CSP_ERR_OOM. */
csp_status csp_create(csp_ctx **out, int device, size_t mem_budget_bytes);

/* Free every device allocation of the context and the context itself.
 * Waits for the context's outstanding work. NULL is ignored. */
void csp_destroy(csp_ctx *ctx);

/* Message of the last failed call on this context ("" if none).  Valid until
 * the next call on the context.  ctx may be NULL (creation errors). */
const char *csp_last_error(const csp_ctx *ctx);

/* Set geometry (Sec. IV patches; Fig. 3 scales).  Invalidates loaded
 * dictionaries' derived data.  Errors: CSP_ERR_INVALID on inconsistent sizes. */
csp_status csp_set_geometry(csp_ctx *ctx, const csp_geometry *geom);

/* Set the sensing operator Phi of y = Phi x + e (Sec. III-C).  Requires
 * geometry.  Errors: CSP_ERR_INVALID (plane count incompatible with kind),
 * CSP_ERR_NOT_READY (no geometry). */
csp_status csp_set_sensing(csp_ctx *ctx, const csp_sensing *sensing);

/* Load the dictionary D^(level) (N_l x T_l, atom-major float32, Sec. III-A).
 * N_l must equal the level's patch dimension.  The library copies it.
 * is_device_ptr: 0 = D is a host pointer, 1 = device pointer. */
csp_status csp_load_dictionary(csp_ctx *ctx, int level, const float *D, int N_l, int T_l,
                               int is_device_ptr);

/* Load the cross-scale map f between `level` and `level + 1` (Sec. III-B).
 * parent: HOST int32 [T_l], parent[i] in [0, T_{l+1}) is the coarse atom that
 * atom i of `level` is a child of.  parent == NULL with Q > 0 selects the
 * paper's block rule parent[i] = floor(i / Q) (requires T_l = Q * T_{l+1}).
 * Requires both dictionaries loaded.  Errors: CSP_ERR_INVALID (range, size). */
csp_status csp_load_scale_links(csp_ctx *ctx, int level, const int32_t *parent, int T_l, int Q);

/* Patch count B and measurement dimension M of the current geometry and
 * sensing. */
csp_status csp_problem_size(const csp_ctx *ctx, int64_t *B_out, int *M_out);

/* Patch extraction (Sec. III-C measurements, Sec. IV overlapping patches):
 * meas (DEVICE float32) is the measurement image -- IDENTITY [planes][H][W],
 * BAYER / CODED_EXPOSURE [H][W], CODED_APERTURE [shots][H][W]; Y_out (DEVICE
 * float32 [B][M]) receives one measurement vector per patch. */
csp_status csp_extract_patches(csp_ctx *ctx, const float *meas, float *Y_out, int64_t *B_out,
                               void *stream);

/* Solve every patch (Algorithm 1 or Algorithm 2).  Y: DEVICE float32 [B][M].
 * Outputs (DEVICE, [B][Kmax]): support_out = fine-dictionary atom indices in
 * selection order (-1 padded), coef_out = least-squares coefficients
 * (0 padded), k_eff_out (DEVICE int8 [B]) = atoms chosen (< budget when the
 * residual vanished, a chosen atom was linearly dependent, or the candidate set
 * ran out).  Workspace is owned by the context and reused across calls. */
csp_status csp_solve(csp_ctx *ctx, const csp_solve_params *params, const float *Y, int64_t B,
                     int32_t *support_out, float *coef_out, int8_t *k_eff_out, void *stream);

/* Statistics of the most recent csp_solve (synchronises its stream). */
csp_status csp_solve_stats_get(csp_ctx *ctx, csp_solve_stats *out);

/* Synthesis and overlap-add (Sec. IV: overlapping patches; uniform average
 * over the covering patches): x_hat_p = D^(0)_|Omega alpha for every patch,
 * image_out (DEVICE float32 [planes][H][W]) = per-pixel mean of the covering
 * patches' values.  Deterministic (fixed summation order). */
csp_status csp_aggregate(csp_ctx *ctx, const int32_t *support, const float *coef,
                         const int8_t *k_eff, int64_t B, int Kmax, float *image_out,
                         void *stream);

/* Allocation-free variant of csp_aggregate.  The paper has no counterpart:
 * this exists for callers that cannot allocate device memory when they
 * aggregate (code recorded while a stream is captured into a CUDA graph,
 * processes whose memory pool owns the device and forbids later allocations,
 * latency-bound loops that must not enter the driver's allocator).  Same
 * arguments, result and launch order as csp_aggregate; the per-patch
 * synthesis scratch is a fixed 16 MiB array (4,194,304 floats) in the
 * library's device image, held by every GPU that loads the library until the
 * process exits.  Requires B * N0 <= 4,194,304 (N0 = fine patch dimension),
 * else CSP_ERR_INVALID with a message.  Calls no cudaMalloc/cudaFree.
 * csp_create looks up the array's device address (once per device, with that
 * device current), which is when the driver reserves its memory; should that
 * lookup have failed, the first call on the device repeats it, and that first
 * call should then come before any stream capture.  All calls share the array:
 * calls whose work overlaps on the GPU race on it. */
csp_status csp_aggregate_noalloc(csp_ctx *ctx, const int32_t *support, const float *coef,
                                 const int8_t *k_eff, int64_t B, int Kmax, float *image_out,
                                 void *stream);

/* The whole path on DEVICE buffers (Sec. IV; Algorithms 1 and 2): the patch
 * vectors of the geometry's patch grid from the measurement image `meas`
 * (layout as in csp_extract_patches), the solve with `params` (as csp_solve;
 * per-patch budgets are not accepted, K_patch must be NULL), and the synthesis
 * x_hat_p = D0 alpha_p with the overlap-add into image_out (float32
 * [planes][H][W], as csp_aggregate).  The patch vectors, supports and
 * coefficients live in buffers of the context.  Same image as the three calls;
 * with the Gram-Schmidt restricted solver (variants 5-7, Kb <= 8) the finest
 * level writes x_hat_p itself, which saves the synthesis pass.  In graph mode
 * (csp_set_graph_mode) identical calls are replayed from one CUDA graph.
 * Errors: those of the three calls; CSP_ERR_UNSUPPORTED for dense sensing (no
 * measurement image).  Stream-ordered; returns before the work completes. */
csp_status csp_reconstruct(csp_ctx *ctx, const csp_solve_params *params, const float *meas, float *image_out,
                           void *stream);

/* End-to-end reconstruction from HOST buffers: copies the measurement image
 * (layout as in csp_extract_patches) to the device, runs csp_reconstruct and
 * copies the image (float32 [planes][H][W]) back into image_host.  Per-patch
 * budgets are not accepted here (K_patch must be NULL).  A page-locked
 * image_host is written directly by the overlap-add through its device mapping
 * (over the host link, no staging copy); a page-locked, 16-byte aligned
 * meas_host is read by a copy kernel through its mapping; in graph mode, with a
 * page-locked meas_host, the whole call is recorded in one graph.  Returns when
 * the image is in host memory. */
csp_status csp_reconstruct_host(csp_ctx *ctx, const csp_solve_params *params,
                                const float *meas_host, float *image_host, void *stream);

/* ---- Dictionary learning: modified K-SVD -----------------------------------
 * Sec. II ("Dictionary learning"): K-SVD alternates sparse coding of the
 * training signals with an atom-by-atom dictionary update.  Sec. III
 * ("Learning cross-scale sparse models"): Step 1 runs K-SVD on the
 * downsampled signals W x_i (csp_downsample) with plain OMP; Step 2 runs
 * K-SVD on the x_i with the coding restricted to the children of each
 * signal's coarse support (csp_solve, CSP_MODE_CROSS_SCALE).  Sec. III
 * ("Initialization of dictionary"): heuristics 1-2 (csp_ksvd_init_atoms) and
 * 3-4 (replace_unused of csp_ksvd_update).  These calls need no sensing
 * operator and, except csp_downsample, no geometry; they use the context's
 * device, workspace and memory budget. */

/* W of Sec. III-A for training signals: X_low[i] = W_level x_i (box average
 * over the level's factor blocks).  X: DEVICE float32 [N][N_0] level-0 patch
 * vectors of the geometry's layout; X_low: DEVICE float32 [N][N_level].
 * Requires geometry.  Stream-ordered. */
csp_status csp_downsample(csp_ctx *ctx, int level, const float *X, int64_t N, float *X_low, void *stream);

/* One dictionary-update sweep of K-SVD.  Atoms k = 0 .. T-1 are visited in
 * order; visiting k: E_k = the residuals r_i = x_i - D s_i of the signals
 * whose support holds k, each with alpha_ik d_k added back; d_k becomes the
 * leading left singular vector of E_k (the dominant eigenvector of E_k E_k^T,
 * found in FP32 by the power method from the old d_k until a step moves the
 * vector by at most 4e-6, at most 1000 steps), signed
 * so that <d_new, d_old> >= 0; alpha_ik becomes <e_i, d_k>; the residuals
 * follow.  An atom with E_k = 0 keeps its value.
 * approximate = 1 replaces the singular vector by one alternating step from
 *   the current coefficients (Rubinstein, Zibulevsky and Elad 2008, "Efficient
 *   implementation of the K-SVD algorithm using Batch OMP"): d_k = E_k^T
 *   alpha_k / ||E_k^T alpha_k|| (kept when zero), then alpha_ik = <e_i, d_k>;
 *   the error never grows.  0 = the exact update.
 * D: DEVICE float32 [T][M] (atom-major), updated in place.
 * X: DEVICE float32 [N][M] training signals.
 * support / coef: DEVICE [N][Kmax] as csp_solve writes them (atom ids into D,
 *   -1 padded; coef updated in place); k_eff: DEVICE int8 [N].  A support
 *   must not repeat an atom.
 * replace_unused = 1: an atom with no users becomes the normalised signal of
 *   largest residual norm among the eligible ones (ties: lowest index), and
 *   that signal is not picked again in this sweep (heuristics 3-4).  Eligible:
 *   every signal of nonzero norm, or, with repl_parent (DEVICE int32 [T], the
 *   coarse parent of each atom) and repl_support (DEVICE int32 [N][Kc], coarse
 *   supports, -1 padded), the signals whose coarse support holds the atom's
 *   parent.  replace_unused = 0: unused atoms keep their value.
 * err_out: DEVICE float32 [1] or NULL; receives ||X - D S||_F^2 after the sweep.
 * Limits: 1 <= M <= 192 and T <= 4096 (else CSP_ERR_UNSUPPORTED),
 *   N * Kmax < 2^31.  Errors found on the device (k_eff outside [0, Kmax],
 *   atom id outside [0, T), a repeated atom) return CSP_ERR_INVALID before D
 *   or coef change.  Deterministic.  Synchronous: returns when the sweep is
 *   complete (work is ordered after earlier work on `stream`). */
csp_status csp_ksvd_update(csp_ctx *ctx, float *D, int M, int T, const float *X, int64_t N,
                           const int32_t *support, float *coef, const int8_t *k_eff, int Kmax,
                           int replace_unused, int approximate, const int32_t *repl_parent,
                           const int32_t *repl_support, int Kc, float *err_out, void *stream);

/* Counters of the last csp_ksvd_update on this context: power_steps = the
 * power-method steps summed over the visited atoms (a step is one product
 * with E_k E_k^T; at most 1000 per atom; the approximate update counts one
 * product E_k^T alpha_k per atom), replaced = atoms replaced by
 * heuristics 3-4, ranks = thread blocks of the sweep's cluster (16 where the
 * device holds such a cluster, else 8).  Any pointer may be NULL. */
csp_status csp_ksvd_stats_get(csp_ctx *ctx, int64_t *power_steps, int64_t *replaced, int64_t *ranks);

/* Initialisation picks of the modified K-SVD.  Atom t = x_i / ||x_i|| with
 * i = item floor(u_t n) of a pool of n signals in ascending order: all N
 * signals when parent is NULL (heuristic 1, the coarse dictionary from W X);
 * else the signals whose coarse support (support_low DEVICE int32 [N][Kc],
 * keff_low DEVICE int8 [N]) holds parent[t] (heuristic 2: the children of
 * coarse atom k from X restricted to Omega_k), all N when that pool is empty.
 * D: DEVICE float32 [T][M] (written; an atom whose pick is a zero signal keeps
 * its value).  X: DEVICE float32 [N][M].  parent: DEVICE int32 [T] in
 * [0, T_low).  u: DEVICE float64 [T], uniform in [0, 1).  Synchronous. */
csp_status csp_ksvd_init_atoms(csp_ctx *ctx, float *D, int M, int T, const float *X, int64_t N,
                               const int32_t *parent, const int32_t *support_low, const int8_t *keff_low,
                               int Kc, int T_low, const double *u, void *stream);

/* ---- Serving: continuous batching of reconstruction jobs -----------------
 * Not part of the paper's method: a request loop around csp_solve.  A server
 * owns one CUDA device, a device-memory budget for in-flight jobs and a
 * scheduler thread.  Models (dictionaries, links, patch geometry without the
 * image extent, sensing kind and solve parameters) stay resident.  Jobs
 * (an image of a model: extent, measurements, per-job codes) are queued by
 * csp_submit and admitted in arrival order while their device memory fits the
 * budget and a batch slot is free; admitted jobs of the same model are
 * coalesced into one batched solve (one set of launches over all their
 * patches, up to max_batch_patches), and batches run concurrently on
 * n_streams CUDA streams, so jobs that arrive while others are on the GPU
 * start as soon as memory and a slot free up.  Every patch is solved
 * independently, so a job's result does not depend on the jobs it shares a
 * batch with.  Supported sensing kinds: IDENTITY, BAYER_RGGB, CODED_EXPOSURE.
 * Admission counts each job's batch memory and its share of the solver
 * workspace; each stream keeps its workspace at the largest batch it ran. */
typedef struct csp_server csp_server;

typedef struct csp_server_config {
    int device;                 /* CUDA device                                             */
    size_t mem_budget_bytes;    /* device memory for in-flight jobs (0: 16 GiB)             */
    int64_t max_batch_patches;  /* patches coalesced into one solve at most (0: 262144)    */
    int n_streams;              /* batches in flight at once, 1..8 (0: 2)                  */
} csp_server_config;

typedef struct csp_model_desc {
    csp_geometry geom;          /* H and W are ignored (they are per job)                  */
    int sense_kind;             /* CSP_SENSE_IDENTITY, _BAYER_RGGB or _CODED_EXPOSURE      */
    const float *D[CSP_MAX_LEVELS];        /* HOST, atom-major [T_l][N_l] (copied)        */
    int T[CSP_MAX_LEVELS];
    const int32_t *parent[CSP_MAX_LEVELS]; /* HOST links of levels 0 .. n_levels-2        */
    csp_solve_params params;    /* mode, precision, K, Kmax (K_patch must be NULL)         */
} csp_model_desc;

typedef struct csp_job_desc {
    int model_id;
    int H, W;                   /* image extent                                           */
    const float *meas_host;     /* measurement image (layout as csp_extract_patches); read
                                   when the job starts, keep it alive until the job is done */
    const uint8_t *codes_host;  /* CODED_EXPOSURE: [planes][H][W] 0/1 codes (copied at submit) */
    float *image_host;          /* output image [planes][H][W], written before "done"      */
} csp_job_desc;

typedef struct csp_job_info {
    int64_t patches;
    double t_submit, t_admit, t_done;  /* seconds on the server's steady clock             */
    int batch_jobs;             /* jobs coalesced into this job's batch                    */
    int64_t batch_patches;
    csp_status status;          /* CSP_OK, CSP_ERR_NOT_READY while queued/running, or error */
    /* Stage times of the job's batch (milliseconds; shared by the jobs of one batch):
     * enqueue_ms   host time the scheduler spent staging inputs and enqueueing the batch;
     * copy_in_ms   device: host-to-device copies (the measurements straight from the
     *              caller's buffer), patch extraction and code blocks;
     * solve_ms     device: the solve (with per-patch operator builds for per-pixel Phi);
     * build_ms     device: of solve_ms, the builds of the per-patch operators of the
     *              full-dictionary level (coded exposure; 0 otherwise);
     * aggregate_ms device: synthesis and overlap-add of the batch's images;
     * copy_out_ms  device: device-to-host copies of the images;
     * t_gpu_done   seconds on the server's clock when the scheduler saw the batch complete;
     * host_out_ms  host copy of this job's image into the caller's buffer (0 when the
     *              device wrote it there directly). */
    double enqueue_ms, copy_in_ms, solve_ms, aggregate_ms, copy_out_ms, t_gpu_done, host_out_ms, build_ms;
} csp_job_info;

csp_status csp_server_create(csp_server **out, const csp_server_config *cfg);
/* Waits for every job, stops the scheduler, frees everything. NULL is ignored. */
void csp_server_destroy(csp_server *srv);
const char *csp_server_last_error(const csp_server *srv);
/* Register a model; prepares its effective dictionaries.  model_id out. */
csp_status csp_server_add_model(csp_server *srv, const csp_model_desc *desc, int *model_id);
/* paused != 0: admit no further job until resumed (batches already in flight
 * complete; queued jobs stay queued).  Used to drain the server or to queue a
 * burst of jobs that should start together. */
csp_status csp_server_pause(csp_server *srv, int paused);
/* Queue a job.  CSP_ERR_OOM if its device memory exceeds the whole budget
 * (it could never be admitted), CSP_ERR_INVALID on bad arguments. */
csp_status csp_submit(csp_server *srv, const csp_job_desc *job, uint64_t *job_id);
/* Non-blocking: *done = 1 once the image is in image_host (or the job failed). */
csp_status csp_poll(csp_server *srv, uint64_t job_id, int *done);
/* Blocks until done or timeout_us (< 0: no limit); CSP_ERR_TIMEOUT if not done. */
csp_status csp_wait(csp_server *srv, uint64_t job_id, int64_t timeout_us);
csp_status csp_job_info_get(csp_server *srv, uint64_t job_id, csp_job_info *out);
/* Forget a finished job (its info is no longer available).  CSP_ERR_NOT_READY
 * while it is queued or running. */
csp_status csp_job_release(csp_server *srv, uint64_t job_id);

/* ---- Autotuning (not part of the paper's method) --------------------------
 * Kernel variants that compute the same result with different work
 * decompositions (here: the restricted finer-scale solver, either re-reading
 * candidate rows from L2 with cooperative lane groups, staging them in
 * shared memory, or scoring candidates through the level's precomputed Gram
 * matrix -- the "Batch-OMP" form of the same iteration, scoring p0 - G alpha,
 * or its Gram-Schmidt form, which updates the correlations per appended atom
 * and solves for alpha once -- each with 4, 8 or 16 lanes per patch for
 * M <= 64, twice that for larger M; the Gram-Schmidt form also with each
 * lane's candidates held in registers, 8, 16 or 4 lanes per patch).  csp_autotune
 * runs csp_solve once per variant on the given batch (same arguments as
 * csp_solve, outputs overwritten), then times three more runs with CUDA events
 * and takes the fastest, keeps the fastest variant for this context and reports
 * the times; then, with that variant, times the forms of the full-dictionary
 * level (csp_set_top_level_form) that apply and keeps the fastest.  A
 * cross-scale batch of the context's own patch grid (B = the grid's patch
 * count) is timed with the synthesis x_hat_p = D0 alpha_p of every patch into
 * workspace scratch, as csp_reconstruct runs it (inside the finest restricted
 * kernel for the variants that write it, else by the synthesis kernel), since
 * the variants differ there too.  Synchronises `stream`. */
#define CSP_TUNE_VARIANTS 14 /* 0: L2-cooperative, 1: shared-memory staged, 2-4: Gram-matrix proxy, 5-7: Gram-Schmidt
                                form, each narrow to wide; 8-10: Gram-Schmidt form with the candidates' state in
                                registers, 8, 16 and 4 lanes per patch (budgets <= 8, at most 8 candidates a
                                lane; else as 6); 11-13: as 8-10 with each patch's Gram block G[C][C] staged in
                                shared memory (at most 32 candidates, 16 with 16 lanes; else as 6) */
typedef struct csp_tune_result {
    int restricted_variant;            /* chosen variant index                      */
    double ms[CSP_TUNE_VARIANTS];      /* solve time per variant (ms)               */
    int top_level_form;                /* chosen full-dictionary form (1, 2 or 3), see
                                          csp_set_top_level_form                     */
    double ms_top[3];                  /* solve time with forms 1, 2 and 3 (0 when a
                                          form does not apply)                       */
} csp_tune_result;

csp_status csp_autotune(csp_ctx *ctx, const csp_solve_params *params, const float *Y, int64_t B,
                        int32_t *support_out, float *coef_out, int8_t *k_eff_out, void *stream,
                        csp_tune_result *out);

/* Pin the restricted-solver variant (0 .. CSP_TUNE_VARIANTS - 1), e.g. from a
 * stored csp_tune_result (a new context starts with variant 8).  Variants 8-10
 * run as variant 6 where M is above 8 x lanes (16 x lanes with 4 lanes), Kb > 8
 * or more than 8 candidates per lane.  Variants 2-10 fall back to 0 on levels
 * whose Gram matrix was not kept (T^2 floats above 256 MiB or beyond the memory
 * budget) and on per-pixel operators.
 * Errors: CSP_ERR_INVALID for an unknown variant. */
csp_status csp_set_kernel_variant(csp_ctx *ctx, int restricted_variant);

/* Aggregation path of csp_aggregate (same arithmetic in the same order, so the
 * same image): 0 automatic (two-pass unless its scratch of B * N0 floats
 * exceeds 1 GiB), 1 two-pass (synthesis into device scratch, then the
 * per-pixel average), 2 fused shared-memory tiles (no scratch; falls back to
 * two-pass when a patch footprint does not fit a tile).  CSP_ERR_INVALID for
 * another value. */
csp_status csp_set_aggregate_path(csp_ctx *ctx, int path);

/* Form of the full-dictionary OMP (plain OMP; the coarsest level of
 * cross-scale OMP): 0 automatic (the default: form 2 wherever it applies, else
 * form 1; csp_autotune replaces it by the fastest form it measured),
 * 1 one launch per iteration for the proxy and one for the update, 2 fused:
 * all iterations of 128 patches in one CTA with residuals and factors on
 * chip (shared effective dictionary with T <= 256, a multiple of 64, M <= 64,
 * K <= 8, BF16 precision; other shapes use form 1), 3 the Gram form (the
 * "Batch-OMP" form of Sec. III-C's cost terms, no residual): the correlations
 * P0 = Y A^T once by an FP32 GEMM, then every iteration from the level's Gram
 * matrix G = A A^T with all atoms as candidates -- the proxy c = P0 - Q_C z,
 * Q_C = A^T U updated by one Gram row per appended atom -- in FP32 at every
 * precision (shared dictionary kept with its Gram matrix, T <= 256, K <= 8,
 * M <= 256; other shapes use forms 2 or 1).  Forms 1 and 2 select the same
 * atoms (same tensor-core proxy, FP32 re-score of its best four); form 3 scores
 * every atom in FP32.  CSP_ERR_INVALID for another value. */
csp_status csp_set_top_level_form(csp_ctx *ctx, int form);

/* Work order of solves with per-patch budgets (K_patch of level 0 given) on
 * one operator group (not Bayer phases): 0 (default) every level runs a static
 * grid over the patches in their order; 1 the patches are first sorted by
 * their level-0 budget, largest first (a counting sort on the device), every
 * level takes them in that order, and the restricted Gram and Gram-Schmidt
 * kernels (variants 2-7) run persistent warps that take the next group of
 * patches from a work queue with one atomic add -- long problems start first
 * and warps that finish early take more (uneven K across patches, Sec. IV
 * light fields; scheduling only: every patch's result is the same).  Nothing
 * in the queue waits.  CSP_ERR_INVALID for another value. */
csp_status csp_set_work_order(csp_ctx *ctx, int order);

/* Test hook for failure detection (not part of the method).  on != 0: the
 * tensor-core proxy's TMA producer issues no atom-tile loads, so the MMA
 * thread's bounded mbarrier wait expires (after about 2 s), the kernel records
 * an error code, every CTA leaves its pipeline and frees its tensor memory,
 * and csp_solve_stats_get returns CSP_ERR_TIMEOUT.  Nothing faults; with the
 * hook off again the context solves normally.  Applies to BF16 solves that use
 * the per-iteration form. */
csp_status csp_set_wait_test(csp_ctx *ctx, int on);

/* Graph mode (not part of the method).  on != 0: csp_solve records the launches
 * of a call in a CUDA graph (after running the call once normally) and replays
 * the graph for the following calls with the same parameters, buffers and
 * batch size, as long as the context's set-up, kernel variant and form are
 * unchanged; any other call is run normally and recorded in place of the old
 * graph.  Results are identical.  Profiling (csp_profile_enable) turns replay
 * off.  The caller must keep the buffers of a recorded call alive while graph
 * mode is on (or turn it off, which frees the graph). */
csp_status csp_set_graph_mode(csp_ctx *ctx, int on);

/* Pipelined cross-scale solve (not part of the method).  on != 0 (the
 * default): when the full-dictionary level runs in the fused form, all
 * patches fall in one mosaic phase group (always so without a mosaic) and
 * there are more of them than one wave of that kernel holds, that wave's patches go down the finer levels on a second
 * stream of the context while the fused kernel runs the rest, and the call's
 * stream waits for both.  Results are identical either way; off: everything
 * on the call's stream.  Errors: CSP_ERR_INVALID for a NULL ctx. */
csp_status csp_set_pipeline(csp_ctx *ctx, int on);

/* ---- Instrumentation (not part of the paper's method) ----------------------
 * Every kernel launch of a context is counted per kernel kind.  While
 * profiling is enabled, each launch is also bracketed by CUDA events on its
 * stream, so that csp_profile_read reports the device time per kind. */
typedef struct csp_kernel_time {
    char name[32];             /* kernel kind, e.g. "proxy_fp32", "restricted"            */
    int64_t launches;          /* launches since the last reset                          */
    double total_ms;           /* summed event time (0 when profiling was off)           */
} csp_kernel_time;

/* on != 0 enables event timing of every launch from now on. */
csp_status csp_profile_enable(csp_ctx *ctx, int on);

/* Synchronises the context's recorded events, fills up to `cap` entries
 * (kinds with at least one launch) and their count in *n_out; reset != 0
 * clears the counters afterwards. */
csp_status csp_profile_read(csp_ctx *ctx, csp_kernel_time *out, int cap, int *n_out, int reset);

#ifdef __cplusplus
}
#endif

#endif /* CSP_H */
