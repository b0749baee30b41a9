/*
 * nbvgs.h — C ABI of the GB300 object-aware Gaussian-splat next-best-view
 * scorer (arXiv 2602.08266, "Informative Object-centric Next Best View for
 * Object-aware 3D Gaussian Splatting in Cluttered Scenes").
 *
 * What the library computes, per NBV step (Sec. III):
 *   - renders every camera with an object-aware 3D Gaussian Splatting
 *     rasterizer: colour, depth, accumulated opacity and the K+1 object
 *     channels O' = sum_i softmax(o_i) alpha_i T_i, with the background
 *     residual O = O' + e0 (1 - 1^T O')                         (Eqs. 1-2);
 *   - from the same compositing pass, the per-Gaussian Gauss-Newton blocks
 *     of the rendering Jacobian, J^T C J with the per-Gaussian confidence
 *     c_g = max_k(p_gk)^-alpha_obj sigma_g^-alpha_opa              (Eqs. 6-9),
 *     or its object-centric form (Eq. 12) when a target object is given;
 *   - the block-diagonal log-det information gain of each candidate over
 *     the training views, IG_f(T,c) = f(T u c) - f(T) for f in {rgb,d,o},
 *     normalised by the mean gain of the training views and weighted,
 *     IG = IG_rgb + beta_d IG_d + beta_o IG_o                   (Eqs. 5, 10, 11);
 *   - the argmax candidate: the next best view                  (Eq. 5).
 *
 * Readings of points the paper leaves open (the same ones the test oracle
 * takes): H_g = lambda I + c_g sum_v A_vg with lambda = lambda_damp; the
 * parameters are the raw ones (mean, log-scale, unnormalised quaternion,
 * opacity logit, SH coefficients, object logits); depth D = sum_i w_i z_i;
 * pixel centres at (x+0.5, y+0.5); depth-sort ties broken by Gaussian index.
 *
 * Conventions.
 *  - Every call is asynchronous on the context's CUDA stream unless it says
 *    otherwise. Inputs are copied into context-owned device memory; outputs
 *    go to caller-owned buffers. A context is not thread-safe.
 *  - Every call returns NBV_OK (0) or a negative NBV_ERR_* code; no C++
 *    exception crosses the ABI. nbv_last_error() gives a message. After an
 *    error the context keeps its last good state; NBV_ERR_CUDA errors are
 *    sticky (the context must be destroyed).
 *  - Cameras are world->camera rigid transforms in OpenCV axes (x right,
 *    y down, z forward): x_cam = R x_world + t, R row-major.
 */
#ifndef NBVGS_H_
#define NBVGS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nbv_ctx nbv_ctx;

enum {
  NBV_OK = 0,
  NBV_ERR_ARG = -1,            /* invalid argument (sizes, NaN, zero quaternion, target > K) */
  NBV_ERR_CUDA = -2,           /* a CUDA call failed; the context is unusable */
  NBV_ERR_OOM = -3,            /* device allocation failed */
  NBV_ERR_STATE = -4,          /* calls out of order (e.g. score before prepare) */
  NBV_ERR_TIMEOUT = -5,        /* a bounded device wait gave up */
  NBV_ERR_EMPTY = -6,          /* a normaliser of Eq. 10 is zero (e.g. target carried by no Gaussian) */
  NBV_ERR_UNIMPLEMENTED = -7
};

/* Hyper-parameters and rasterizer conventions. nbv_config_default() fills
 * the paper's values (Sec. IV-A.2: alpha_obj = alpha_opa = 0.3, beta_d = 10,
 * beta_o = 1) and the standard splatting constants. */
typedef struct {
  int K;                 /* number of objects; K+1 object channels, channel 0 = background */
  int sh_degree;         /* 0..3 */
  float alpha_obj;       /* Eq. 7 exponent on max_k p_gk */
  float alpha_opa;       /* Eq. 7 exponent on the opacity */
  float beta_d;          /* Eq. 11 depth weight */
  float beta_o;          /* Eq. 11 object weight */
  float lambda_damp;     /* damping added to every per-Gaussian block (a reading; default 0.1) */
  float near_z;          /* cull Gaussians with camera z <= near_z (0.2) */
  float alpha_min;       /* skip a splat below this opacity (1/255) */
  float alpha_max;       /* clamp a splat's opacity here (0.99) */
  float t_min;           /* stop a ray before transmittance falls below this (1e-4) */
  float dilation;        /* added to the 2D covariance diagonal, px^2 (0.3) */
  float guard;           /* guard band of the projection Jacobian, x tan(fov/2) (1.3) */
  int tile_w, tile_h;    /* screen tile: 16 x 16 (default) or 32 x 8; 0 x 0 = 16 x 16 until nbv_autotune */
  int batched;           /* 0: one launch sequence per candidate view; 1: all candidates in one
                            multi-view launch sequence (one sort, a persistent (view, tile)
                            compositing launch, one gains launch) replayed as a CUDA graph */
  int stage;             /* Gaussians the compositing kernel stages in shared memory per round:
                            32 (default) or 16; only speed depends on it */
  int max_batch_views;   /* batched path: candidates per multi-view pass (0 = as many as keep the
                            per-(view, Gaussian) state under 45% of the free device memory);
                            larger sets run in chunks, eagerly, and only a single-chunk set is
                            replayed as a CUDA graph */
  int criterion;         /* per-Gaussian information criterion of Eq. 6's block-diagonal form:
                            0 (default) log det(H_T + c A_v) - log det H_T, the paper's;
                            1 tr(H_T^-1 c A_v), its first-order term (an expected-information
                              criterion in the manner of FisherRF);
                            2 tr(c A_v), T-optimality (no training prior).
                            Normalisation (Eq. 10) and weighting (Eq. 11) are unchanged */
  int tf32_contraction;  /* arithmetic of the tensor-core sum over pixels of the per-pixel
                            Gauss-Newton terms (Eqs. 6, 9), FP32 accumulation in every case:
                            1 single TF32 products (10-bit operands, about 2^-11 relative per
                            term); 2 error-compensated, each product as three TF32 products of
                            the operands' high and low parts (about 21 significant bits);
                            0 (default) automatic: 1 for the log-det criterion, whose logarithm
                            compresses the rounding, 2 for the linear trace criteria.
                            This applies to the candidates' blocks; the training views' blocks
                            (summed into the factorised training Hessians) always use 2 */
} nbv_config;

typedef struct {
  float R[9];            /* world->camera rotation, row-major */
  float t[3];            /* world->camera translation */
  float fx, fy, cx, cy;  /* pinhole intrinsics, pixels */
  int width, height;     /* image size, pixels */
} nbv_camera;

/* Fill *cfg with the defaults for K objects and SH degree sh_degree. */
void nbv_config_default(nbv_config* cfg, int K, int sh_degree);

/* Create a context bound to the CUDA device current on the calling thread
 * and to `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * On success *out owns every device buffer the context allocates later.
 * Errors: NBV_ERR_ARG (bad config: K < 1 or > 98 (the per-Gaussian object
 * gain's u x u workspace, u = 6 + K, must fit one block's shared memory),
 * sh_degree outside 0..3,
 * tile not 16x16, 32x8 or 0x0, non-finite or out-of-range constants),
 * NBV_ERR_CUDA. */
int nbv_create(const nbv_config* cfg, void* cuda_stream, nbv_ctx** out);

/* Free every device buffer of the context (synchronises its stream). NULL is ignored. */
void nbv_destroy(nbv_ctx* ctx);

/* Load (copy) n Gaussians, the paper's parameterisation (Sec. III-A.1):
 *   means [n][3], log_scales [n][3], quats [n][4] (w,x,y,z, any non-zero
 *   norm), opacity [n] (logit rho, sigma = sigmoid(rho)),
 *   sh [n][(d+1)^2][3], obj_logits [n][K+1].
 * All float32, C-contiguous. ptrs_on_device = 1: device pointers (copied
 * device-to-device on the stream); 0: host pointers (copied host-to-device;
 * the call returns after the copy was queued from a staging buffer, so the
 * caller may reuse its memory). Resets any prepared state.
 * Errors: NBV_ERR_ARG (n < 1, NULL, a zero quaternion, a non-finite value),
 * NBV_ERR_OOM, NBV_ERR_CUDA. Validation runs on the device after the copy
 * (one synchronisation of the stream); after a load that fails it, the
 * context holds no usable scene (prepare and render return NBV_ERR_STATE)
 * until a load succeeds. */
int nbv_load_gaussians(nbv_ctx* ctx, int64_t n, const float* means, const float* log_scales,
                       const float* quats, const float* opacity, const float* sh,
                       const float* obj_logits, int ptrs_on_device);

/* Set the training views T (Eqs. 5, 10) or the candidate views C (host
 * array of n cameras, copied). New training views reset the prepared state;
 * passing the cameras the context already holds, byte for byte, changes
 * nothing (the prepared state and a captured multi-view graph are kept).
 * Errors: NBV_ERR_ARG (n < 0, n > 65535, non-finite pose, width/height not
 * in 1..16384, fx or fy <= 0). */
int nbv_set_train_views(nbv_ctx* ctx, int n, const nbv_camera* cams);
int nbv_set_candidates(nbv_ctx* ctx, int n, const nbv_camera* cams);

/* Build the training-view state of one NBV step: per Gaussian and output the
 * damped, confidence-weighted training Hessian block
 *   H_T,g = lambda I + c_g sum_{t in T} J_t,g^T J_t,g      (Eqs. 6-9 / 12)
 * factorised once, and the training gains IG_f(T,t) that normalise Eq. 10.
 * target_obj = -1 scores the whole scene (Eq. 7); 0..K restricts the
 * confidence to that object (Eq. 12).
 * Errors: NBV_ERR_STATE (no Gaussians or no training views), NBV_ERR_ARG
 * (target_obj outside -1..K), NBV_ERR_OOM, NBV_ERR_CUDA. */
int nbv_prepare(nbv_ctx* ctx, int target_obj);

/* Render candidate `cand` (Eqs. 1-2) into caller-owned DEVICE buffers, any
 * of which may be NULL: rgb [H][W][3], depth [H][W], alpha [H][W],
 * obj [H][W][K+1]. Does not need nbv_prepare.
 * Errors: NBV_ERR_STATE (no Gaussians), NBV_ERR_ARG (cand out of range). */
int nbv_render(nbv_ctx* ctx, int cand, float* rgb, float* depth, float* alpha, float* obj);

/* Score every candidate: ig_out [n_cand][4] = {IG_rgb, IG_d, IG_o} raw
 * (Eq. 5 per output) and the normalised weighted total (Eqs. 10-11).
 * out_on_device = 1: ig_out is a device pointer (asynchronous); 0: a host
 * pointer (the call synchronises). Needs nbv_prepare.
 * Errors: NBV_ERR_STATE, NBV_ERR_EMPTY (a training normaliser is zero;
 * totals are then NaN), NBV_ERR_OOM, NBV_ERR_CUDA. */
int nbv_score(nbv_ctx* ctx, float* ig_out, int out_on_device);

/* The next best view of the last nbv_score: argmax of the total, lowest
 * index on ties (Eq. 5). Synchronises. Errors: NBV_ERR_STATE, NBV_ERR_EMPTY. */
int nbv_argmax(nbv_ctx* ctx, int* best_view, float* best_score);

/* The training gains of the last nbv_prepare, host array [n_train][3]
 * (IG_rgb, IG_d, IG_o). Synchronises. Errors: NBV_ERR_STATE. */
int nbv_train_gains(nbv_ctx* ctx, float* out);

/* Per-Gaussian log-det gains of candidate `cand`, DEVICE array [n][3]: the
 * terms log det(H_T,g + c_g A_c,g) - log det H_T,g whose sum over g is
 * IG_f(T,c) (Sec. III-B.1, block-diagonal determinant); 0 for Gaussians with
 * c_g = 0. The information contraction of this call is error-compensated
 * whatever tf32_contraction says (single terms are inspected here; the
 * logarithm of a view sum does not average their rounding). Needs
 * nbv_prepare. Errors: NBV_ERR_STATE, NBV_ERR_ARG. */
int nbv_gaussian_gains(nbv_ctx* ctx, int cand, float* delta);

/* Inspection of one view's projection and tile lists (for verification).
 * view_set 0 = candidates, 1 = training views. Device arrays of length n:
 * rect [n][4] = {x0,x1,y0,y1} tile range (-1 when culled), radius [n],
 * zbits [n] (float bits of camera z), mean2d [n][2], conic [n][3].
 * Any pointer may be NULL. */
int nbv_debug_project(nbv_ctx* ctx, int view_set, int view, int32_t* rect, float* radius,
                      uint32_t* zbits, float* mean2d, float* conic);

/* Sorted tile lists of one view: *count receives the number of (tile,
 * Gaussian) entries; if count <= cap, offsets [ntiles+1] and ids [count]
 * (device arrays) receive the per-tile ranges and Gaussian ids in blend
 * order. A tile lists the Gaussians whose 3-sigma rectangle covers it and
 * that can pass the alpha cut-off at one of its pixel centres (the bound
 * of the tile culling, which drops only tiles without such a pixel, so no
 * rendered value depends on it). view_set 0 / 1 bins the candidate / training view on its own;
 * view_set 2 returns candidate `view` as the last multi-view score binned it
 * (NBV_ERR_STATE when no multi-view score ran since the inputs changed);
 * with a target object (Eq. 12) that pass lists splats only in the tiles
 * where a splat of the target can pass its alpha cut-off, the only tiles
 * whose lists the information gain reads.
 * Synchronises. */
int nbv_debug_tile_lists(nbv_ctx* ctx, int view_set, int view, int64_t* offsets, int32_t* ids,
                         int64_t cap, int64_t* count);

/* Phases timed by the profiler. */
enum {
  NBV_PHASE_PREP = 0,      /* scene preparation: sigmoid, softmax, confidences (Eqs. 7, 12) */
  NBV_PHASE_PROJECT = 1,   /* projection, EWA covariance, SH colour */
  NBV_PHASE_SORT = 2,      /* scan, tile duplication, radix sort, tile ranges */
  NBV_PHASE_COMPOSITE = 3, /* fused compositing + information blocks (Eqs. 1-2, 6-9) */
  NBV_PHASE_FACTORS = 4,   /* training Hessians and their factorisation */
  NBV_PHASE_GAINS = 5,     /* per-Gaussian log-det gains and their sums (Eqs. 5-6) */
  NBV_PHASE_SCORE = 6,     /* normalisation, weighting, argmax (Eqs. 10-11) */
  NBV_PHASE_TRAIN_COMPOSITE = 7, /* compositing + information blocks of the training views (prepare);
                                    NBV_PHASE_COMPOSITE holds the candidates' information pass */
  NBV_PHASE_FORWARD = 8,   /* the candidates' forward pass (transmittance and list ends per pixel) */
  NBV_NUM_PHASES = 9
};

/* Switch per-phase timing on (1) or off (0); either call clears the
 * accumulated times and work counters. While on, every phase of every call
 * is bracketed by CUDA events recorded on the context stream, and the
 * batched path enqueues its kernels directly instead of replaying its CUDA
 * graph (same kernels, same order). Synchronises. */
int nbv_set_profiling(nbv_ctx* ctx, int on);

/* Accumulated device time (ms) and kernel launches per phase since
 * profiling was switched on; arrays of NBV_NUM_PHASES. Synchronises. */
int nbv_phase_times(nbv_ctx* ctx, double* ms, int64_t* launches);

/* Work counters of the compositing kernel since profiling was switched on,
 * for the candidates' launches (which = 0) or the training views' launches
 * of prepare (which = 1): [0] (pixel, splat) pairs evaluated in the forward
 * pass, [1] pairs blended, [2] (tile, Gaussian) block flushes, [3] (pixel,
 * splat) pairs of the information pass (blended pixels of splats with
 * c_g > 0), [4] compositing launches, [5] (view, tile, Gaussian) entries
 * of their binning passes. Synchronises. Errors: NBV_ERR_ARG. */
int nbv_work_stats(nbv_ctx* ctx, int which, int64_t* out6);

/* Throughput of fused multiply-adds on the FP32 pipes of the current device:
 * a register-resident loop of independent fma.rn.f32 (packed = 0) or
 * packed fma.rn.f32x2 (packed = 1) chains over (SMs x 8) blocks of 256
 * threads, timed with CUDA events on cuda_stream after one untimed launch.
 * *tflops = 2 flops per lane FMA / seconds / 1e12. Synchronises. A
 * measurement of the roofline's FP32 peak; it computes nothing of the method.
 * Errors: NBV_ERR_ARG (NULL tflops), NBV_ERR_CUDA. */
int nbv_measure_fp32_fma(int packed, void* cuda_stream, double* tflops);

/* Pick the screen tile (16 x 16 or 32 x 8) and the number of Gaussians the
 * compositing kernel stages in shared memory per round (16 or 32) that
 * score the current candidate set fastest on the batched path: every
 * combination prepares and scores once untimed, then once timed with CUDA
 * events. The choice is kept for this context and remembered for later
 * contexts with the same K, SH degree and candidate resolutions. A tile
 * shape decides which Gaussians each tile lists (a Gaussian is listed in
 * the tiles of its 3-sigma rectangle where it can pass the alpha cut-off),
 * so it changes rendered values
 * slightly; the stage depth changes nothing but speed. Ends with the
 * context prepared (same target as before, or -1). Synchronises.
 * Errors: NBV_ERR_STATE (no Gaussians, training or candidate views), those of
 * nbv_prepare and nbv_score. */
int nbv_autotune(nbv_ctx* ctx, int* tile_w, int* tile_h, int* stage);

/* The context's tile shape and stage depth. */
int nbv_get_tiling(const nbv_ctx* ctx, int* tile_w, int* tile_h, int* stage);

/* Largest input of nbv_sort_tile_keys_noalloc (2^20 pairs). */
#define NBV_NOALLOC_MAX_PAIRS (1 << 20)

/* Tile-key sort that allocates no device memory. The paper has no
 * counterpart; it is the binning stage's stable LSD radix sort offered to
 * callers that may not allocate while they run: applications that reserve
 * the whole GPU up front under their own allocator, or latency-critical
 * code where a cudaMalloc (which can synchronise the device) is not allowed.
 *
 * Sorts n (key, value) pairs by the low key_bits bits of the keys, stably
 * (equal keys keep their input order), from keys_in/vals_in (device, only
 * read) into keys_out/vals_out (device, caller-owned, must not alias the
 * inputs), asynchronously on cuda_stream. The working memory (a copy of the
 * pairs and the radix histograms, about 13 MB) is a fixed array in the
 * library image: every GPU that loads the library holds it until the process
 * exits, and it keeps the last call's contents. No part of it needs to start
 * at zero. Calls that overlap on the GPU (on different streams or threads)
 * share that array and race; serialise them.
 * The first call on each device looks up the array's device address (set-up,
 * cached per device); make that first call before any stream capture.
 * A launch error that earlier work left pending on the calling thread is
 * cleared on entry (cudaGetLastError), so that NBV_ERR_CUDA reports this
 * call's own launches.
 * Errors: NBV_ERR_ARG (n < 0, n > NBV_NOALLOC_MAX_PAIRS, key_bits outside
 * 1..64, a NULL buffer, or an output whose bytes overlap an input or the
 * other output), NBV_ERR_CUDA. */
int nbv_sort_tile_keys_noalloc(const uint64_t* keys_in, const uint32_t* vals_in, int64_t n,
                               int key_bits, uint64_t* keys_out, uint32_t* vals_out,
                               void* cuda_stream);

/* Largest number of (view, tile, Gaussian) entries one binning pass may
 * hold (their offsets and tile ranges are 32-bit). 0 restores the default,
 * 2^32 - 4097. The entries of every pass are counted in 64 bits on the
 * device before anything is duplicated: the batched path splits a candidate
 * set whose pass would exceed the limit into smaller multi-view passes (run
 * eagerly, one after the other); a single view above it fails with
 * NBV_ERR_ARG and nothing is written. Drops a captured multi-view graph.
 * Errors: NBV_ERR_ARG (max_entries < 0 or above the default). */
int nbv_set_entry_limit(nbv_ctx* ctx, int64_t max_entries);

/* Message of the last error on this context (never NULL). */
const char* nbv_last_error(const nbv_ctx* ctx);

/* Number of kernel launches the context issued so far. */
int64_t nbv_launch_count(const nbv_ctx* ctx);

/* ------------------------------------------------------------------------
 * Differentiable rendering for the map refinement of the NBV loop (a pattern
 * layered on the method: the paper refines the map with its reconstruction
 * losses, Eqs. 3-4).
 * ---------------------------------------------------------------------- */

/* Render any camera (host struct) into DEVICE buffers like nbv_render. */
int nbv_render_view(nbv_ctx* ctx, const nbv_camera* cam, float* rgb, float* depth, float* alpha, float* obj);

/* Backward pass of the rasterizer (Eqs. 1-2) for one camera: given DEVICE
 * gradients of a loss with respect to the rendered colour [H][W][3], depth
 * [H][W], opacity [H][W] and object channels [H][W][K+1] (any may be NULL:
 * zero), ADD the gradients with respect to the loaded Gaussians' raw
 * parameters to the DEVICE arrays g_means [n][3], g_log_scales [n][3],
 * g_quats [n][4] (unnormalised), g_opacity [n] (logit), g_sh [n][(d+1)^2][3]
 * and g_obj_logits [n][K+1]. The forward pass is recomputed per tile (no
 * per-pixel lists are kept); a splat clamped at alpha_max passes no gradient
 * to its geometry or opacity; decisions (culling, tiles, the 1/255 and 1e-4
 * cut-offs) are held fixed. Asynchronous on the context stream. */
int nbv_render_backward(nbv_ctx* ctx, const nbv_camera* cam, const float* g_rgb, const float* g_depth,
                        const float* g_alpha, const float* g_obj, float* g_means, float* g_log_scales,
                        float* g_quats, float* g_opacity, float* g_sh, float* g_obj_logits);

/* ------------------------------------------------------------------------
 * Learned candidate pre-scoring (a pattern layered on the method; the paper
 * scores every candidate exactly). A per-view descriptor of the projected
 * Gaussians feeds a 3-layer MLP (BF16 weights and activations, FP32
 * accumulation on the tensor cores) trained on the exact normalised scores
 * (Eq. 11) that nbv_score produces; nbv_score_pruned keeps the candidates
 * it ranks highest and scores only those exactly.
 * ---------------------------------------------------------------------- */

/* Descriptor length: 6 x 64 image-grid cells + 56 object bins + 8 totals. */
#define NBV_DESC_DIM 448

/* Descriptors of every candidate into `out` (DEVICE float [n_cand][448]):
 * for each Gaussian whose centre projects in front of the near plane and
 * inside the image, with opacity sigma, confidence c_g (Eq. 7 / 12, as the
 * last nbv_prepare set it), camera depth z, training observation
 * o_g = sum over the training views and their pixels of w^2 (w = alpha T)
 * and angular novelty nu = 1 - max over the training cameras of the cosine
 * between the directions from the camera centres to the Gaussian:
 *   [0, 64)    sum sigma over an 8 x 8 grid of image cells,
 *   [64, 128)  sum c_g sigma per cell,
 *   [128, 192) sum c_g sigma / z per cell,
 *   [192, 256) sum c_g sigma / (1 + o_g) per cell,
 *   [256, 320) sum c_g sigma nu per cell,
 *   [320, 384) sum c_g sigma nu^2 per cell,
 *   [384, 440) sum c_g sigma per most-probable object id (ids >= 55 share bin 55),
 *   [440, 448) view totals of c_g sigma nu, c_g sigma [nu > 0.1],
 *              c_g sigma [nu > 0.3], c_g sigma sqrt(nu), sigma, c_g sigma,
 *              c_g sigma / (1 + o_g), c_g sigma / z,
 * each feature then mapped to log(1 + s x) with s = 64 / n (cells), (K + 1) / n
 * (object bins) or 1 / n (totals), n = number of Gaussians. Cells:
 * floor(8 mx / W), floor(8 my / H) of the projected centre, computed in
 * single precision. Errors: NBV_ERR_STATE (no prepare), NBV_ERR_ARG. */
int nbv_descriptors(nbv_ctx* ctx, float* out);

typedef struct nbv_mlp nbv_mlp;

/* An MLP d_in -> width -> width -> 1 with ReLU (width a multiple of 16,
 * <= 256; d_in <= 4096), He-uniform initial weights drawn from `seed`
 * (splitmix64), zero biases. Parameters (FP32, flattened in this order):
 * W1 [width][d_in], b1 [width], W2 [width][width], b2 [width], w3 [width],
 * b3. Runs on `cuda_stream`. */
int nbv_mlp_create(int d_in, int width, uint64_t seed, void* cuda_stream, nbv_mlp** out);
void nbv_mlp_destroy(nbv_mlp* mlp);
int64_t nbv_mlp_num_params(const nbv_mlp* mlp);
/* Copy the FP32 parameters to / from a DEVICE array of nbv_mlp_num_params. */
int nbv_mlp_get_params(nbv_mlp* mlp, float* out);
int nbv_mlp_set_params(nbv_mlp* mlp, const float* in);
/* y [rows] = MLP(x [rows][d_in]), DEVICE arrays. The input, the weights and
 * the hidden activations are rounded to BF16; products accumulate in FP32.
 * Synchronises. Errors: NBV_ERR_TIMEOUT if a tensor-core wait gave up. */
int nbv_mlp_forward(nbv_mlp* mlp, const float* x, int rows, float* y);
/* Gradient of the mean squared error mean_m (y_m - t_m)^2 over the
 * parameters (DEVICE float [num_params], same order), by the hand-written
 * backward: the two hidden layers' input and weight gradients are tensor-core
 * products of the BF16 activations; biases and the head reduce in double.
 * *loss (host) receives the loss before the step. Synchronises. */
int nbv_mlp_gradients(nbv_mlp* mlp, const float* x, const float* t, int rows, float* grads, double* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) of
 * learning rate lr on the mean squared error of this batch; loss may be
 * NULL (then the call does not synchronise). */
int nbv_mlp_train_step(nbv_mlp* mlp, const float* x, const float* t, int rows, float lr, double* loss);

/* D [M][N] (row stride ldd, FP32) = sum_k A(m, k) B(n, k) with BF16
 * A(m, k) = A[m a_sm + k a_sk], B(n, k) = B[n b_sn + k b_sk] (DEVICE
 * arrays; the strides express any transposition), on tcgen05 tensor cores
 * with tensor-memory accumulators. *d_err (DEVICE int, may be NULL) is set
 * if a bounded wait for the tensor cores gave up. Asynchronous. */
int nbv_gemm_bf16(const uint16_t* A, int64_t a_sm, int64_t a_sk, const uint16_t* B, int64_t b_sn, int64_t b_sk,
                  float* D, int64_t ldd, int M, int N, int K, int* d_err, void* cuda_stream);

/* Polls the first wait of every nbv_gemm_bf16 launch for the tensor cores'
 * commit makes before it gives up (polls = 0: at once; polls < 0 restores
 * the default 2^20). After giving up a launch records *d_err = 1 (NBV_ERR_TIMEOUT
 * for the MLP calls), waits once more with the full bound for the work it
 * has in flight, frees its tensor memory and returns, so the device stays
 * usable. For tests of that path; process-wide, not thread-safe.
 * Errors: NBV_ERR_ARG (polls above 2^32 - 1). */
int nbv_set_gemm_wait_polls(int64_t polls);

/* Pre-score every candidate with the MLP over its descriptor, keep the
 * `keep` highest predictions (ties to the lower index) and score only those
 * exactly (nbv_score's path); pred (DEVICE [n_cand], may be NULL) receives
 * the predictions, kept (HOST int [keep]) the kept candidate indices in
 * descending prediction order, exact (HOST float [keep][4], may be NULL)
 * their exact rows as nbv_score gives them, *best / *best_score the
 * argmax among the kept ones (an index into the full candidate list). The
 * context's candidate set is unchanged on return. Synchronises.
 * Errors: NBV_ERR_ARG (keep < 1, MLP input size not NBV_DESC_DIM), NBV_ERR_STATE
 * (no prepare), those of nbv_score. */
int nbv_score_pruned(nbv_ctx* ctx, nbv_mlp* mlp, int keep, float* pred, int* kept, float* exact, int* best,
                     float* best_score);

#ifdef __cplusplus
}
#endif

#endif /* NBVGS_H_ */
